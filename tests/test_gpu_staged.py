"""Staged loads of the 16-bit storage policies (lbm_set_staging): on lattices with nx a
multiple of 8, each block copies its tile's rows of every plane to shared memory with
asynchronous 16-byte copies and runs the step from that copy.  The step's arithmetic is
the same as with direct loads from global memory, so the two forms must agree: to the
bit where the compiler fuses the same multiply-adds in both kernels, and always within
the rounding of the 16-bit format (one unit of an FP16 or BF16 stored population can flip
where an FP32 intermediate lies on a rounding boundary).  Cases cover a periodic axis
narrower than a tile (film, nx = 16), walls on every side, N = 2, 3, 4, and every tile
shape; each runs 200 steps and is also held to the oracle with the bounds of the direct
form (test_gpu_precision)."""
import numpy as np
import pytest

import oracle
from paper_2603_22902_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# stored 16-bit populations: an FP16 unit is 2^-11 of a value of O(1), BF16 2^-8
AGREE = {"fp16s": {"phi": 2e-3, "T": 2e-2, "ux": 1e-4, "p": 5e-5},
         "bf16s": {"phi": 2e-2, "T": 1e-1, "ux": 5e-4, "p": 5e-4}}
ORACLE = {"fp16s": {"phi": 5e-3, "T": 6e-2, "ux": 2e-4, "p": 1e-4},
          "bf16s": {"phi": 5e-2, "T": 2e-1, "ux": 1e-3, "p": 1e-3}}


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for the gpu tests")
    from paper_2603_22902_gb300 import build as B
    B.build()
    from paper_2603_22902_gb300 import lbm as L
    return L


def cases():
    quad = W.periodic_drop(n=32, R=7.0, N=4, rho_gas=0.5, sigma=1e-3)
    quad.phi[2] = 0.3 * quad.phi[1]
    quad.phi[3] = 0.2 * quad.phi[1]
    quad.phi[1] = 0.5 * quad.phi[1]
    quad.phases[2]["latent"] = 4.0
    quad.bc = (W.WALL, W.WALL, W.WALL, W.WALL)
    quad.tbc = (W.ADIABATIC, W.ADIABATIC, W.DIRICHLET, W.ADIABATIC)
    quad.T_wall = (0.0, 0.0, -0.5, 0.0)
    quad.T = np.full((quad.ny, quad.nx), 0.2)
    return {"film_16x256": W.film(nx=16, ny=256),
            "sessile_48x40": W.sessile_drop(n=48, R=14.0, theta=60.0, ny=40),
            "compound_N3_48x40": W.compound_drop(n=48, R_core=8.0, R_shell=15.0, ny=40, noise=1e-3),
            "pool_N3_walls_32": W.lateral_pool(n=32),
            "N4_walls_32": quad}


def run(L, case, prec, staged, steps=200, tile=None):
    s = L.Solver(case, precision=prec, tile=tile)
    L.lbm_set_staging(s.h, staged)
    s.set_fields()
    s.step(steps)
    F = s.fields_numpy()
    d = s.diagnostics()
    s.close()
    return F, d


@pytest.mark.parametrize("prec", ["fp16s", "bf16s"])
@pytest.mark.parametrize("name", list(cases().keys()))
def test_staged_agrees_with_direct_loads(lbm, prec, name):
    case = cases()[name]
    assert case.nx % 8 == 0
    Fs, ds = run(lbm, case, prec, True)
    Fd, dd = run(lbm, case, prec, False)
    assert ds["nonfinite"] == 0 and dd["nonfinite"] == 0
    diff = {k: float(np.abs(Fs[k] - Fd[k]).max()) for k in AGREE[prec]}
    O = oracle.Oracle(case).step(200).fields()
    err = {k: float(np.abs(Fs[k] - O[k]).max()) for k in ORACLE[prec]}
    print(prec, name, "staged - direct", diff, "staged - oracle", err)
    for k, b in AGREE[prec].items():
        assert diff[k] <= b, (k, diff[k], b)
    for k, b in ORACLE[prec].items():
        assert err[k] <= b, (k, err[k], b)


@pytest.mark.parametrize("tile", [(32, 4), (64, 4), (16, 16)])
def test_staged_tile_shapes(lbm, tile):
    case = W.sessile_drop(n=64, R=16.0, theta=80.0, ny=48)
    Fs, _ = run(lbm, case, "fp16s", True, tile=tile)
    Fd, _ = run(lbm, case, "fp16s", False, tile=tile)
    diff = {k: float(np.abs(Fs[k] - Fd[k]).max()) for k in AGREE["fp16s"]}
    print(tile, diff)
    for k, b in AGREE["fp16s"].items():
        assert diff[k] <= b, (tile, k, diff[k], b)
