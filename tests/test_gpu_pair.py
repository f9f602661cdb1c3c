"""The two-cells-per-thread form of the fused step (lbm_set_tile_cells with 2 cells per
thread; FP32, FP16 and BF16 storage with FP32 arithmetic): each thread owns the cells
(x, y) and (x, y + 1) and runs their common arithmetic on packed FP32 pairs.

* Against the CPU oracle after 200 steps, with the per-format bounds of the one-cell
  form (test_gpu_precision), on the N = 3 compound drop (walls, ragged tiles), both tile
  shapes, every policy.
* Against the one-cell form: the same step to FP32 rounding (1e-5 on phi after 100 steps
  in FP32), on every boundary kind and N = 2, 3, 4, including a lattice with an odd
  number of rows (the last pair of a column has one cell).
* The 512 x 512 sessile drop: the freezing front after 2000 steps within 0.05 lattice
  units of the one-cell form, and the conserved volumes to 1e-6 relative."""
import numpy as np
import pytest

import oracle
from paper_2603_22902_gb300 import workloads as W
from paper_2603_22902_gb300.metrics import front_height
from tests._cases import small_cases
from tests.test_gpu_precision import BOUNDS

pytestmark = pytest.mark.gpu

FIELDS = ("phi", "T", "fl", "ux", "uy", "p")


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for the gpu tests")
    from paper_2603_22902_gb300 import build as B
    B.build()
    from paper_2603_22902_gb300 import lbm as L
    return L


def run(L, case, prec, tile, steps):
    s = L.Solver(case, precision=prec, tile=tile).set_fields()
    s.step(steps)
    F = s.fields_numpy()
    d = s.diagnostics()
    s.close()
    assert d["nonfinite"] == 0
    return F, d


@pytest.mark.parametrize("prec", ["fp32", "fp16s", "bf16s"])
@pytest.mark.parametrize("tile", [(32, 8, 2), (32, 16, 2)])
def test_pair_form_against_oracle(lbm, prec, tile):
    case = W.compound_drop(n=44, R_core=8.0, R_shell=15.0, ny=36, noise=1e-3, mobility=0.02)
    G, _ = run(lbm, case, prec, tile, 200)
    O = oracle.Oracle(case).step(200).fields()
    errs = {k: float(np.abs(G[k] - O[k]).max()) for k in BOUNDS[prec]}
    print(prec, tile, errs)
    for k, b in BOUNDS[prec].items():
        assert errs[k] <= b, (k, errs[k], b)


def odd_rows():
    c = W.sessile_drop(n=50, R=14.0, theta=70.0, ny=37)
    return c


@pytest.mark.parametrize("name", list(small_cases().keys()) + ["odd_rows_50x37"])
def test_pair_form_equals_one_cell_form_fp32(lbm, name):
    case = odd_rows() if name == "odd_rows_50x37" else small_cases()[name]
    A, da = run(lbm, case, "fp32", (32, 8), 100)
    for tile in [(32, 8, 2), (32, 16, 2)]:
        B, db = run(lbm, case, "fp32", tile, 100)
        errs = {k: float(np.abs(A[k] - B[k]).max()) for k in FIELDS}
        print(name, tile, errs)
        assert errs["phi"] <= 1e-5 and errs["fl"] <= 1e-4 and errs["ux"] <= 1e-6 and errs["uy"] <= 1e-6, errs
        assert errs["T"] <= 1e-4 * max(1.0, float(np.abs(A["T"]).max())), errs
        for p in range(case.N):
            assert abs(da["mass"][p] - db["mass"][p]) <= 1e-6 * max(1.0, abs(da["mass"][p]))


@pytest.mark.parametrize("prec", ["fp16s", "fp32"])
def test_pair_form_sessile_drop_512(lbm, prec):
    case = W.sessile_drop()
    A, da = run(lbm, case, prec, (32, 8), 2000)
    B, db = run(lbm, case, prec, (32, 16, 2), 2000)
    fa, fb = front_height(A, case.nx), front_height(B, case.nx)
    print(prec, "front one-cell", fa, "pair", fb)
    assert abs(fa - fb) <= 0.05
    for p in range(case.N):
        assert abs(da["mass"][p] - db["mass"][p]) <= 1e-6 * da["mass"][p]


def test_pair_form_refused_for_fp64(lbm):
    case = W.sessile_drop(n=40, R=10.0, ny=30)
    with pytest.raises(lbm.LBMError) as e:
        lbm.Solver(case, precision="fp64", tile=(32, 8, 2))
    assert e.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LBMError) as e:
        lbm.Solver(case, precision="fp16s", tile=(64, 4, 2))
    assert e.value.code == lbm.LBM_EINVAL
