"""Conservation on the GPU paths (FP64 and double words), the GPU counterparts of the
oracle's invariant pins: without phase change, total enthalpy sum_x rho H is conserved
with periodic sides and adiabatic walls, and total momentum sum_x rho u in a periodic box
without surface tension or gravity, to round-off of the arithmetic over 2000 steps.
rho is rebuilt on the host from phi_p by the mixture rule (f_l = 1 without phase change)."""
import numpy as np
import pytest

from paper_2603_22902_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for the gpu tests")
    from paper_2603_22902_gb300 import build as B
    B.build()
    from paper_2603_22902_gb300 import lbm as L
    return L


def density(case, F):
    return sum(F["phi"][p] * case.phases[p]["rho_l"] for p in range(case.N))


def enthalpy_case():
    c = W.periodic_drop(n=64, R=18.0, rho_gas=0.1, cy=28.0)
    c.bc = (W.PERIODIC, W.PERIODIC, W.WALL, W.WALL)
    c.tbc = (W.ADIABATIC, W.ADIABATIC, W.ADIABATIC, W.ADIABATIC)
    c.phases[1]["lam_l"] = c.phases[1]["lam_s"] = 0.03
    c.phases[1]["cp_l"] = c.phases[1]["cp_s"] = 10.0
    return W.perturbed(c, seed=7, amp_u=1e-3, amp_T=0.4)


# relative bounds: FP64 rounding accumulated over 2000 steps, double words 2^5 times coarser
BOUND = {"fp64": 1e-12, "df64": 1e-11}


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_total_enthalpy_conserved(lbm, prec):
    c = enthalpy_case()
    s = lbm.Solver(c, precision=prec).set_fields()
    F0 = s.fields_numpy()
    rH0 = F0["H"] * density(c, F0)
    s.step(2000)
    F1 = s.fields_numpy()
    s.close()
    assert np.all(F1["fl"] == 1.0)
    rH1 = F1["H"] * density(c, F1)
    rel = abs(rH1.sum() - rH0.sum()) / np.abs(rH0).sum()
    print(prec, "enthalpy drift", rel)
    assert np.abs(F1["T"] - F0["T"]).max() > 1e-3
    assert rel <= BOUND[prec]


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_total_momentum_conserved(lbm, prec):
    c = W.perturbed(W.periodic_drop(n=64, R=18.0, rho_gas=0.3, sigma=0.0), seed=9, amp_u=2e-3)
    s = lbm.Solver(c, precision=prec).set_fields()
    F0 = s.fields_numpy()
    r0 = density(c, F0)
    P0 = np.array([(r0 * F0["ux"]).sum(), (r0 * F0["uy"]).sum()])
    scale = np.abs(r0 * F0["ux"]).sum() + np.abs(r0 * F0["uy"]).sum()
    s.step(2000)
    F1 = s.fields_numpy()
    s.close()
    r1 = density(c, F1)
    P1 = np.array([(r1 * F1["ux"]).sum(), (r1 * F1["uy"]).sum()])
    rel = np.abs(P1 - P0).max() / scale
    print(prec, "momentum drift", rel)
    assert np.abs(F1["ux"] - F0["ux"]).max() > 1e-5
    assert rel <= BOUND[prec]
