"""Invariants of the coupled scheme that pin the oracle (Sections 2-3):

* the t = 0 populations carry the moments of the equilibria defined in Section 3;
* per-phase volume sum_x phi_p is conserved when nothing freezes (mdot = 0);
* total momentum sum_x rho u is conserved in a periodic box without surface tension,
  gravity or phase change, also with a density contrast (the source terms S and Lambda
  add no first moment);
* total enthalpy sum_x rho H is conserved when nothing changes phase, with periodic sides
  and adiabatic (bounce-back) walls (the enthalpy LBE's equilibria carry rho H exactly and
  its source vanishes with mdot);
* sum_p phi_p = 1 is kept exactly when there is no flow;
* reduction consistency: an absent phase stays absent and N = 3 with phi_3 = 0
  reproduces the N = 2 run bit for bit (Section 2);
* N = 2 reproduces the textbook two-phase conservative Allen-Cahn model with the
  standard free energy (R = 4 phi (1 - phi) n / eps, mu = beta g' - kappa lap phi);
* mirror and 90-degree rotation symmetry of the discrete operators.
"""
import numpy as np
import pytest

import oracle
from paper_2603_22902_gb300 import workloads as W

CX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
CY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])


def test_initial_populations_carry_equilibrium_moments():
    c = W.perturbed(W.sessile_drop(n=24, R=8.0, T0=0.5), seed=11, amp_u=2e-3, amp_T=0.3)
    o = oracle.Oracle(c)
    f, g, h = o.populations()
    F = o.fields()
    rhoH0 = np.array([[oracle.inverse_map(c, c.phi[:, j, i], c.T[j, i]) for i in range(c.nx)]
                      for j in range(c.ny)])
    # zeroth moments: sum f = 0 (p = 0), sum g_p = phi_p, sum h = rho H
    assert np.abs(f.sum(0)).max() < 1e-15
    assert np.abs(g.sum(1) - c.phi).max() < 1e-15
    assert np.abs(h.sum(0) - rhoH0).max() < 1e-14
    # first moments: rho u, phi_p u, rho c_p T u
    rho = F["rho"]
    jx, jy = np.tensordot(CX, f, 1), np.tensordot(CY, f, 1)
    assert np.abs(jx - rho * c.ux).max() < 1e-16 and np.abs(jy - rho * c.uy).max() < 1e-16
    gxm = np.einsum("i,pijk->pjk", CX, g)
    assert np.abs(gxm - c.phi * c.ux).max() < 1e-16
    hx = np.tensordot(CX, h, 1)
    cp = np.ones_like(rho) * np.where(c.phi[0] > -1, 1.0, 1.0)
    cp = (1 - F["fl"]) * (c.phi[0] * 1.0 + c.phi[1] * c.phases[1]["cp_s"]) + F["fl"] * (
        c.phi[0] * 1.0 + c.phi[1] * c.phases[1]["cp_l"])
    assert np.abs(hx - rho * cp * F["T"] * c.ux).max() < 1e-13
    # second moment of f: p/c_s^2 * c_s^2 I + rho u u at p = 0
    pxx = np.tensordot(CX * CX, f, 1)
    assert np.abs(pxx - rho * c.ux * c.ux).max() < 1e-16


def test_phase_volume_conserved_without_freezing():
    c = W.periodic_drop(n=32, R=9.0, rho_gas=0.1, cy=12.0)
    c.bc = (W.PERIODIC, W.PERIODIC, W.WALL, W.WALL)
    c = W.perturbed(c, seed=5, amp_u=1e-3)
    o = oracle.Oracle(c)
    m0 = o.fields()["phi"].sum(axis=(1, 2))
    o.step(400)
    m1 = o.fields()["phi"].sum(axis=(1, 2))
    assert np.abs(m1 / m0 - 1.0).max() < 1e-12


@pytest.mark.parametrize("rho_gas", [1.0, 0.3])
def test_total_momentum_conserved_without_forces(rho_gas):
    c = W.periodic_drop(n=32, R=9.0, rho_gas=rho_gas, sigma=0.0, cy=14.0)
    c = W.perturbed(c, seed=9, amp_u=2e-3)
    o = oracle.Oracle(c)
    F0 = o.fields()
    P0 = np.array([(F0["rho"] * F0["ux"]).sum(), (F0["rho"] * F0["uy"]).sum()])
    scale = float(np.abs(F0["rho"] * F0["ux"]).sum() + np.abs(F0["rho"] * F0["uy"]).sum())
    o.step(300)
    F1 = o.fields()
    P1 = np.array([(F1["rho"] * F1["ux"]).sum(), (F1["rho"] * F1["uy"]).sum()])
    assert np.abs(F1["ux"] - F0["ux"]).max() > 1e-5        # the flow has evolved
    assert np.abs(P1 - P0).max() <= 1e-12 * scale, (P0, P1)


@pytest.mark.parametrize("rho_gas", [1.0, 0.1])
def test_total_enthalpy_conserved_without_phase_change(rho_gas):
    c = W.periodic_drop(n=32, R=9.0, rho_gas=rho_gas, cy=14.0)
    c.bc = (W.PERIODIC, W.PERIODIC, W.WALL, W.WALL)
    c.tbc = (W.ADIABATIC, W.ADIABATIC, W.ADIABATIC, W.ADIABATIC)
    c.phases[1]["lam_l"] = c.phases[1]["lam_s"] = 0.03     # conductivity contrast
    # rho c_p of the light phase kept at the reference value (a smaller one makes the
    # total-enthalpy LBE unstable with these temperature jumps; see the droplet workloads)
    c.phases[1]["cp_l"] = c.phases[1]["cp_s"] = 1.0 / rho_gas
    c = W.perturbed(c, seed=7, amp_u=1e-3, amp_T=0.4)
    o = oracle.Oracle(c)
    F0 = o.fields()
    E0 = float((F0["H"] * F0["rho"]).sum())
    o.step(300)
    F1 = o.fields()
    E1 = float((F1["H"] * F1["rho"]).sum())
    assert np.abs(F1["T"] - F0["T"]).max() > 1e-3        # heat has moved
    assert abs(E1 - E0) <= 1e-12 * float(np.abs(F0["H"] * F0["rho"]).sum()), (E0, E1)


@pytest.mark.parametrize("N", [3, 4])
def test_sum_of_order_parameters_exact_without_flow(N):
    c = W.periodic_drop(n=24, R=6.0, N=N, sigma=0.0)
    share = c.phi[1] / (N - 1)
    for p in range(1, N):
        c.phi[p] = share
    c.bc = (W.WALL, W.WALL, W.WALL, W.WALL)
    o = oracle.Oracle(c).step(300)
    F = o.fields()
    assert np.abs(F["phi"].sum(0) - 1.0).max() < 1e-13
    assert np.abs(F["ux"]).max() == 0.0


def test_absent_phase_reduction_is_exact():
    c2 = W.sessile_drop(n=24, R=7.0, T_wall=-1.0, theta=70.0)
    c3 = c2.copy()
    c3.N = 3
    c3.phi = np.concatenate([c2.phi, np.zeros((1, c2.ny, c2.nx))])
    c3.phases = c2.phases + [W.phase(rho_l=0.5, rho_s=0.4, latent=3.0)]
    s = np.zeros((3, 3))
    s[:2, :2] = c2.sigma
    s[0, 2] = s[2, 0] = 2e-3
    s[1, 2] = s[2, 1] = 1e-3
    c3.sigma = s
    wc = np.zeros((4, 3, 3))
    wc[:, :2, :2] = c2.wet_cos
    # the absent phase wets the wall at its own angles: its ghost terms carry phi_3 = 0
    # as a factor, so the pairwise wetting ghost reduces to the N = 2 law exactly
    for p, ang in ((0, 50.0), (1, 110.0)):
        wc[W.YMIN, p, 2] = np.cos(np.radians(ang))
        wc[W.YMIN, 2, p] = -wc[W.YMIN, p, 2]
    c3.wet_cos = wc
    o2, o3 = oracle.Oracle(c2).step(150), oracle.Oracle(c3).step(150)
    F2, F3 = o2.fields(), o3.fields()
    assert np.all(F3["phi"][2] == 0.0)
    for k in ("T", "H", "fl", "ux", "uy", "p", "rho"):
        assert np.array_equal(F2[k], F3[k]), k
    assert np.array_equal(F2["phi"], F3["phi"][:2])
    g3 = o3.populations()[1][2]
    assert np.all(g3 == 0.0)


def test_absent_fourth_phase_reduction_is_exact():
    # the same with N = 3 -> 4: the three-phase pool freezing under gas, plus an absent
    # fourth phase with its own tensions and latent heat
    c3 = W.lateral_pool(n=24, rho_ratio1=1.05, rho_ratio2=0.95)
    c4 = c3.copy()
    c4.N = 4
    c4.phi = np.concatenate([c3.phi, np.zeros((1, c3.ny, c3.nx))])
    c4.phases = c3.phases + [W.phase(rho_l=0.7, rho_s=0.6, latent=2.0)]
    s = np.full((4, 4), 1.5e-3)
    np.fill_diagonal(s, 0.0)
    s[:3, :3] = c3.sigma
    c4.sigma = s
    wc = np.zeros((4, 4, 4))
    wc[:, :3, :3] = c3.wet_cos
    c4.wet_cos = wc
    o3, o4 = oracle.Oracle(c3).step(150), oracle.Oracle(c4).step(150)
    F3, F4 = o3.fields(), o4.fields()
    assert np.all(F4["phi"][3] == 0.0)
    for k in ("T", "H", "fl", "ux", "uy", "p", "rho"):
        assert np.array_equal(F3[k], F4[k]), k
    assert np.array_equal(F3["phi"], F4["phi"][:3])
    assert np.all(o4.populations()[1][3] == 0.0)


def test_two_phase_reduces_to_textbook_model():
    # The pairwise terms equal the textbook ones while phi_1 + phi_2 = 1 holds exactly:
    # at t = 0 (u and p carry F_s / 2 and the F_0 term) and for phi after one step
    # (phi(x) gathers the neighbours' post-collision g, which carry R_p).  Later the
    # weakly compressible flow makes sum_p phi_p drift from 1 and the two models part.
    c = W.periodic_drop(n=32, R=9.0, rho_gas=0.2, sigma=2e-3, cx=15.3, cy=17.1)
    a, b = oracle.Oracle(c), oracle.Oracle(c, two_phase_textbook=True)
    A, B = a.fields(), b.fields()
    for k in ("ux", "uy", "p"):
        assert np.abs(A[k]).max() > 1e-6, k
        assert np.abs(A[k] - B[k]).max() < 1e-13 * np.abs(A[k]).max(), k
    A, B = a.step(1).fields(), b.step(1).fields()
    assert np.abs(A["phi"] - B["phi"]).max() < 1e-15


def test_mirror_symmetry():
    c = W.sessile_drop(n=32, R=9.0, theta=60.0)  # symmetric about x = nx/2
    F = oracle.Oracle(c).step(120).fields()
    assert np.abs(F["phi"] - F["phi"][:, :, ::-1]).max() < 1e-13
    assert np.abs(F["T"] - F["T"][:, ::-1]).max() < 1e-13
    assert np.abs(F["ux"] + F["ux"][:, ::-1]).max() < 1e-15
    assert np.abs(F["uy"] - F["uy"][:, ::-1]).max() < 1e-15


def test_rotation_symmetry():
    c = W.perturbed(W.periodic_drop(n=20, R=5.0, rho_gas=0.3, cx=8.0, cy=11.0), seed=9, amp_u=1e-3)
    r = c.copy()
    r.phi = np.rot90(c.phi, 1, axes=(1, 2)).copy()
    # np.rot90 over (y, x) with y pointing up turns the plane clockwise by 90 degrees:
    # (x, y) -> (y, -x), so (ux, uy) -> (uy, -ux)
    r.ux = np.rot90(c.uy).copy()
    r.uy = np.rot90(-c.ux).copy()
    Fa = oracle.Oracle(c).step(100).fields()
    Fb = oracle.Oracle(r).step(100).fields()
    assert np.abs(np.rot90(Fa["phi"], 1, axes=(1, 2)) - Fb["phi"]).max() < 1e-13
    assert np.abs(np.rot90(Fa["p"]) - Fb["p"]).max() < 1e-15
    assert np.abs(np.rot90(Fa["uy"]) - Fb["ux"]).max() < 1e-15
    assert np.abs(np.rot90(-Fa["ux"]) - Fb["uy"]).max() < 1e-15


def _periodic_centroid(phi):
    """Centroid of phi on a periodic lattice, from the first Fourier mode of each axis."""
    ny, nx = phi.shape
    out = []
    for prof, n in ((phi.sum(0), nx), (phi.sum(1), ny)):
        th = 2.0 * np.pi * (np.arange(n) + 0.5) / n
        out.append(np.angle((prof * np.exp(1j * th)).sum()) % (2.0 * np.pi) * n / (2.0 * np.pi))
    return out


def test_uniform_translation_with_equal_densities():
    # Galilean invariance: a drop of the gas's density carried by a uniform velocity
    # u0 moves by u0 t and keeps that velocity (advection in the phase-field equilibria
    # and the flow equilibria).  A dropped c_i . u term in g_eq leaves the drop behind.
    n, u0, steps = 48, (0.02, 0.01), 1000
    c = W.periodic_drop(n=n, R=10.0, sigma=1e-3, rho_gas=1.0, mu=0.1)
    c.ux = np.full((n, n), u0[0])
    c.uy = np.full((n, n), u0[1])
    o = oracle.Oracle(c)
    x0 = _periodic_centroid(o.fields()["phi"][0])
    F = o.step(steps).fields()
    x1 = _periodic_centroid(F["phi"][0])
    for a, b, u in zip(x0, x1, u0):
        d = (b - a + n / 2) % n - n / 2
        assert abs(d / (u * steps) - 1.0) < 1e-3, (d, u * steps)
    assert abs(F["ux"].mean() / u0[0] - 1.0) < 1e-3 and abs(F["uy"].mean() / u0[1] - 1.0) < 1e-3


def test_openmp_build_is_bitwise_the_serial_oracle():
    # The benchmark times the oracle also as a -fopenmp build; its per-cell loops write
    # only their own cells, so the threaded run must give bitwise the same fields.
    case = W.compound_drop(n=44, R_core=8.0, R_shell=15.0, ny=36, noise=1e-3, mobility=0.02)
    A = oracle.Oracle(case).step(60).fields()
    B = oracle.Oracle(case, omp=True).step(60).fields()
    for k in A:
        assert np.array_equal(A[k], B[k]), k
