"""The TMA-staged forms of the step (lbm_set_staging; FP16 and BF16 storage, N = 2): each
interior tile's inputs are copied into shared memory by tensor copies, either by a
persistent grid that copies the next tile while it computes the current one (mode 1) or by
one block per tile (mode 2).  It runs the arithmetic of the one-launch form cell by
cell, so the two forms must agree to the rounding of contractions, and the staged form
must hold the one-launch form's bounds against the CPU oracle."""
import numpy as np
import pytest

import oracle
from paper_2603_22902_gb300 import workloads as W
from paper_2603_22902_gb300.metrics import front_height
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


def run(L, case, prec, staged, steps):
    s = L.Solver(case, precision=prec, staged=staged).set_fields()
    s.step(steps)
    F = s.fields_numpy()
    d = s.diagnostics()
    s.close()
    assert d["nonfinite"] == 0
    return F, d


CASES = {
    "sessile_96x80": lambda: W.sessile_drop(n=96, R=28.0, ny=80, theta=70.0),
    "periodic_drop_128x72": lambda: W.perturbed(W.periodic_drop(n=128, R=20.0, ny=72, rho_gas=0.2, sigma=2e-3),
                                                seed=1),
    "sessile_cap_160x64_walls": lambda: W.sessile_cap(160, 64, 18.0, theta=110.0, ste=0.3, T_wall=-1.5),
    "film_16x256": lambda: W.film(nx=16, ny=256),
}


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("prec", ["fp16s", "bf16s"])
@pytest.mark.parametrize("name", list(CASES))
def test_staged_equals_one_launch_form(lbm, prec, name, mode):
    case = CASES[name]()
    if name == "sessile_cap_160x64_walls":
        case.bc = (W.WALL, W.WALL, W.WALL, W.WALL)
    A, da = run(lbm, case, prec, 0, 300)
    B, db = run(lbm, case, prec, mode, 300)
    errs = {k: float(np.abs(A[k] - B[k]).max()) for k in FIELDS}
    print(name, prec, errs)
    assert errs["phi"] <= 1e-6 and errs["fl"] <= 1e-6 and errs["ux"] <= 1e-8 and errs["uy"] <= 1e-8, errs
    assert errs["T"] <= 1e-6 * max(1.0, float(np.abs(A["T"]).max())) and errs["p"] <= 1e-8, errs
    for p in range(case.N):
        assert abs(da["mass"][p] - db["mass"][p]) <= 1e-9 * max(1.0, da["mass"][p])


@pytest.mark.parametrize("mode", [1, 2])
@pytest.mark.parametrize("prec", ["fp16s", "bf16s"])
def test_staged_against_oracle(lbm, prec, mode):
    case = W.sessile_cap(96, 48, 14.0, theta=70.0, ste=0.2, T_wall=-1.5)
    G, _ = run(lbm, case, prec, mode, 200)
    O = oracle.Oracle(case).step(200).fields()
    errs = {k: float(np.abs(G[k] - O[k]).max()) for k in BOUNDS[prec]}
    print(prec, errs)
    for k, b in BOUNDS[prec].items():
        assert errs[k] <= b, (k, errs[k], b)


@pytest.mark.parametrize("mode", [1, 2])
def test_staged_sessile_drop_512(lbm, mode):
    case = W.sessile_drop()
    A, da = run(lbm, case, "fp16s", 0, 2000)
    B, db = run(lbm, case, "fp16s", mode, 2000)
    fa, fb = front_height(A, case.nx), front_height(B, case.nx)
    print("front one-launch", fa, "staged", fb, "max |dphi|", float(np.abs(A["phi"] - B["phi"]).max()))
    assert abs(fa - fb) <= 1e-3
    for p in range(case.N):
        assert abs(da["mass"][p] - db["mass"][p]) <= 1e-8 * da["mass"][p]


def test_staging_refused_where_not_compiled(lbm):
    for prec, case in (("fp64", W.sessile_drop(n=96, R=20.0, ny=64)),
                       ("fp16s", W.compound_drop(n=96, R_core=10.0, R_shell=20.0, ny=64)),
                       ("fp16s", W.sessile_drop(n=90, R=20.0, ny=64))):
        with pytest.raises(lbm.LBMError) as e:
            lbm.Solver(case, precision=prec, staged=2)
        assert e.value.code == lbm.LBM_EINVAL
