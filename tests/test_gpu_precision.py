"""Reduced-precision storage (FP32, FP16 / BF16 moving populations with FP32 rest
populations) against FP64: short-run agreement with the CPU oracle within the format's
resolution, and the freezing-front position of the sessile-drop problem (512 x 512)
within 0.5 lattice units of the FP64 GPU path after 20000 steps, the step count of the
single-droplet problem, at both ends of its Stefan range; and the compound drop
(1024 x 1024, N = 3) for its 50000 steps in FP32 and double words against FP64.

Front position: height of the solid at the drop's centre line, sum_y f_s phi_1 over
the four central columns (the solid grows from the cold wall at y = 0)."""
import numpy as np
import pytest

import oracle
from paper_2603_22902_gb300 import workloads as W
from paper_2603_22902_gb300.metrics import front_height

pytestmark = pytest.mark.gpu

# max |reduced - oracle| after 200 steps: a few units of the format's resolution of
# phi (FP32 ~1e-7, FP16 ~5e-4, BF16 ~4e-3) and of T (plus the gas-side amplification).
# u = sum_i c_i f_i / rho: a stored f_i / (w_i F_SCALE) of O(1) rounds by ~5e-4 of
# itself in FP16, i.e. ~5e-7 in f_i where |f_i| ~ 1e-3, and the gas (rho = 0.01)
# multiplies that by 100, so a few units are ~2e-4 in u.
BOUNDS = {"fp32": {"phi": 2e-4, "T": 1e-3, "ux": 1e-5, "p": 1e-5},
          "fp16s": {"phi": 5e-3, "T": 6e-2, "ux": 2e-4, "p": 1e-4},
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


@pytest.mark.parametrize("prec", ["fp32", "fp16s", "bf16s"])
def test_short_run_against_oracle(lbm, prec):
    case = W.compound_drop(n=44, R_core=8.0, R_shell=15.0, ny=36, noise=1e-3, mobility=0.02)
    s = lbm.Solver(case, precision=prec).set_fields()
    s.step(200)
    G = s.fields_numpy()
    d = s.diagnostics()
    s.close()
    O = oracle.Oracle(case).step(200).fields()
    errs = {k: float(np.abs(G[k] - O[k]).max()) for k in BOUNDS[prec]}
    print(prec, errs)
    assert d["nonfinite"] == 0
    for k, b in BOUNDS[prec].items():
        assert errs[k] <= b, (k, errs[k], b)


@pytest.mark.parametrize("ste", [0.1, 0.5])
def test_reduced_precision_front_position(lbm, ste):
    # both ends of the single-droplet problem's Stefan range
    case = W.sessile_drop(ste=ste)
    steps = 20000
    res = {}
    for prec in ("fp64", "df64", "fp32", "fp16s", "bf16s"):
        s = lbm.Solver(case, precision=prec).set_fields()
        s.step(steps)
        F = s.fields_numpy()
        d = s.diagnostics()
        s.close()
        assert d["nonfinite"] == 0, prec
        res[prec] = (F, front_height(F, case.nx), d)
    F64, s64, _ = res["fp64"]
    assert s64 > 5.0                         # the front has moved
    report = {}
    for prec in ("df64", "fp32", "fp16s", "bf16s"):
        F, sf, d = res[prec]
        report[prec] = {"front": sf, "front_err": abs(sf - s64),
                        "phi_max": float(np.abs(F["phi"] - F64["phi"]).max()),
                        "T_max": float(np.abs(F["T"] - F64["T"]).max()),
                        "solid_rel": abs(d["solid"][0] / res["fp64"][2]["solid"][0] - 1.0)}
    print("ste", ste, "front fp64", s64, report)
    for prec in ("df64", "fp32", "fp16s"):
        assert report[prec]["front_err"] <= 0.5, (prec, report[prec])
    assert report["df64"]["front_err"] <= 1e-6, report["df64"]


def test_compound_drop_full_run(lbm):
    """The encapsulated compound drop (1024 x 1024, N = 3) for its 50 000 steps in FP64, FP32
    and double words: every run stays finite, and the solid heights of the core and of the
    shell at the centre line (sum_y f_s phi_p over the four central columns) agree with
    FP64 within 0.5 lattice units (FP32) and 1e-6 (double words)."""
    case = W.compound_drop()
    cols = slice(case.nx // 2 - 2, case.nx // 2 + 2)
    res = {}
    for prec in ("fp64", "fp32", "df64"):
        s = lbm.Solver(case, precision=prec).set_fields()
        s.step(50000)
        F = s.fields_numpy()
        d = s.diagnostics()
        s.close()
        assert d["nonfinite"] == 0, prec
        fs = 1.0 - F["fl"]
        res[prec] = ([float((fs * F["phi"][p])[:, cols].sum(axis=0).mean()) for p in range(2)], d["solid"])
    fronts64, solid64 = res["fp64"]
    assert fronts64[0] > 10.0                # the core has frozen from the wall
    report = {prec: {"fronts": res[prec][0], "front_err": [abs(a - b) for a, b in zip(res[prec][0], fronts64)],
                     "solid_rel": [abs(a / b - 1.0) for a, b in zip(res[prec][1][:2], solid64[:2])]}
              for prec in ("fp32", "df64")}
    print("compound fronts fp64", fronts64, report)
    assert max(report["fp32"]["front_err"]) <= 0.5, report["fp32"]
    assert max(report["df64"]["front_err"]) <= 1e-6, report["df64"]
    assert max(report["fp32"]["solid_rel"]) <= 1e-2, report["fp32"]
    assert max(report["df64"]["solid_rel"]) <= 1e-6, report["df64"]
