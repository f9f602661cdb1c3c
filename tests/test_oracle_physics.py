"""Physical pins of the oracle: results the paper or classical analysis fixes.

* flat interface: the tanh profile of Section 4 is an equilibrium of the
  conservative Allen-Cahn equation (|grad phi| = 4 phi (1 - phi) / eps);
* Laplace law dp = sigma / R for a 2-D drop (surface force of Section 2);
* Dirichlet wall + enthalpy LBE without phase change: T = T_w erfc(y / 2 sqrt(alpha t));
* film freezing (Section 4.1): Neumann front s = 2 kappa sqrt(alpha_s t), the interface
  rise h - h_0 = s (1 - rho_s / rho_l) and the final height of Table 1;
* Janus drop (Section 4.3): the wetting lengths of Table 2 (the pairwise wetting ghost
  of the order parameters for N = 3);
* frozen layer under a driven channel: the penalty force of the flow LBE weighted by the
  solid volume fraction, against the steady Brinkman profile.
"""
import math
import os

import numpy as np
import pytest

import oracle
from paper_2603_22902_gb300 import workloads as W
from tests._analytic import (brinkman_profile, cap_angle, fit_circle, janus_contact_lengths,
                             janus_wetting_lengths, level_crossings, neumann_front, neumann_kappa,
                             neumann_kappa_superheated, neumann_triangle)

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_neumann_kappa_small_stefan_series():
    # expanding exp(k^2) erf(k) for small k gives Ste = 2 k^2 (1 + 2 k^2 / 3) + O(k^6)
    for ste in (1e-4, 1e-3, 1e-2):
        k = neumann_kappa(ste)
        assert abs(2 * k * k * (1 + 2 * k * k / 3) - ste) < 2 * ste ** 3


def test_neumann_kappa_superheated_limits():
    # no superheat: the one-phase root; superheat slows the front
    for ste in (0.05, 0.1, 0.5):
        assert abs(neumann_kappa_superheated(ste, 0.0) - neumann_kappa(ste)) < 1e-14
        ks = [neumann_kappa_superheated(ste, sh) for sh in (0.0, 0.5, 1.0, 2.0)]
        assert all(a > b for a, b in zip(ks, ks[1:]))
    # small k: erfc(k) -> 1, exp(k^2) erf(k) -> 2 k / sqrt(pi), so the balance reads
    # Ste sqrt(pi) / (2 k) - superheat Ste = k sqrt(pi) + O(k Ste): k -> sqrt(Ste / 2)
    for ste in (1e-6, 1e-8):
        assert abs(neumann_kappa_superheated(ste, 1.0) / math.sqrt(ste / 2.0) - 1.0) < 10 * math.sqrt(ste)


def test_flat_interface_is_stationary():
    # The tanh profile of the initial state (Section 4.1) is an equilibrium of the
    # conservative Allen-Cahn equation: the lattice profile settles within 1e-2 of it
    # and then stays put for 10 000 steps, interfaces at their initial heights.
    c = W.flat_interface(nx=4, ny=64)
    o = oracle.Oracle(c)
    F0 = o.fields()
    o.step(2000)
    F1 = o.fields()
    o.step(8000)
    F2 = o.fields()
    assert np.abs(F1["phi"][0] - F0["phi"][0]).max() < 1e-2
    assert np.abs(F2["phi"][0] - F1["phi"][0]).max() < 1e-5
    assert abs(F2["phi"][0].sum() / F0["phi"][0].sum() - 1.0) < 1e-11
    col = [[v] for v in F2["phi"][0][:, 0]]
    heights = sorted(p[1] for p in level_crossings(col))
    assert len(heights) == 2
    assert abs(heights[0] - 16.0) < 1e-6 and abs(heights[1] - 48.0) < 1e-6


def _laplace_ratio(eps, n=64, R=16.0, sigma=1e-3):
    """Delta p R / sigma of a drop in a periodic box: the mean pressure inside r < R/2
    minus the mean outside r > R + 2 eps, averaged over 20 samples 100 steps apart after
    2000 steps.  Gas density 0.1 and viscosity 0.3 damp the drop's start-up oscillation
    (the pressure starts at 0), so that the average is steady to ~1e-3."""
    c = W.periodic_drop(n=n, R=R, sigma=sigma, rho_gas=0.1, mu=0.3, eps=eps)
    o = oracle.Oracle(c)
    o.step(2000)
    X, Y = W.grid(n, n)
    r = np.hypot(X - n / 2.0, Y - n / 2.0)
    vals = []
    for _ in range(20):
        p = o.step(100).fields()["p"]
        vals.append((p[r < R / 2].mean() - p[r > R + 2 * eps].mean()) * R / sigma)
    return float(np.mean(vals))


@pytest.mark.slow
def test_laplace_law():
    # Delta p = sigma / R in 2D.  The chemical potential and surface force reach it as
    # the interface is resolved: at eps = 8 lattice units within 3 %; at eps = 4 (the
    # paper's width) the pressure jump is ~7 % low, and that error is at least 3 times
    # the eps = 8 one (it falls as (dx / eps)^2).
    r8, r4 = _laplace_ratio(8.0), _laplace_ratio(4.0)
    print("Laplace dp R / sigma: eps 8", r8, "eps 4", r4)
    assert abs(r8 - 1.0) < 0.03
    assert abs(r4 - 1.0) >= 3.0 * abs(r8 - 1.0)
    assert abs(r4 - 1.0) < 0.10


def test_dirichlet_wall_conduction_erfc():
    from math import erfc
    c = W.film(nx=4, ny=128, T_wall=1.0, T0=0.0)
    c.phases[0]["latent"] = 0.0
    c.phi[0][:] = 1.0
    c.phi[1][:] = 0.0
    F = oracle.Oracle(c).step(2000).fields()
    y = np.arange(128) + 0.5   # half-way wall at y = 0
    alpha = 0.1 / (1.0 * 1.0)
    Tex = np.array([erfc(v / (2 * math.sqrt(alpha * 2000))) for v in y])
    assert np.abs(F["T"][:, 0] - Tex).max() < 1e-3


def _front(F, below):
    """Solid thickness from the wall: sum of f_s phi_1 over the rows below `below`."""
    return float(((1 - F["fl"]) * F["phi"][0])[:below].sum(axis=0).mean())


@pytest.mark.slow
def test_neumann_front_without_density_change():
    c = W.film(nx=4, ny=256, rho_ratio=1.0, ste=0.1)
    F = oracle.Oracle(c).step(5000).fields()
    s = _front(F, 128)
    s_ex = neumann_front(0.1, 0.1 / 1.0, 5000)
    assert abs(s / s_ex - 1.0) < 0.03


@pytest.mark.slow
def test_neumann_front_superheated_liquid():
    # The liquid starts at T_0 = 1 above T_m = 0 (the paper's film setting, Section 4.1):
    # the two-phase Neumann solution with equal solid and liquid properties, kappa =
    # 0.1891 against 0.2200 without superheat.  The gas above the film has the liquid's
    # rho c_p and lambda, so the medium is thermally uniform.  Within 3 % at 5000 steps.
    c = W.film(nx=4, ny=256, rho_ratio=1.0, ste=0.1, T0=1.0)
    F = oracle.Oracle(c).step(5000).fields()
    s = _front(F, 128)
    s_ex = 2.0 * neumann_kappa_superheated(0.1, 1.0) * math.sqrt(0.1 * 5000)
    assert abs(s / s_ex - 1.0) < 0.03


@pytest.mark.slow
def test_film_volume_change():
    rr = 0.9
    c = W.film(nx=4, ny=256, rho_ratio=rr, ste=0.1)
    o = oracle.Oracle(c)
    h0 = o.fields()["phi"][0].sum(axis=0).mean()
    F = o.step(5000).fields()
    s = _front(F, 64)
    h = F["phi"][0].sum(axis=0).mean()
    # mass conservation of the freezing liquid: h - h_0 = s (1 - rho_s / rho_l)
    assert abs((h - h0) - s * (1 - rr)) < 0.2
    # front within the paper's 5 % of the Neumann solution
    assert abs(s / neumann_front(0.1, 0.1 / rr, 5000) - 1.0) < 0.05


def _table1():
    rows = []
    with open(os.path.join(GOLDEN, "table1_film_height.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                rows.append([float(v) for v in line.split()])
    return np.array(rows)


@pytest.mark.slow
@pytest.mark.parametrize("rr", [0.9, 0.95])
def test_table1_final_height(rr):
    tab = _table1()
    row = tab[np.argmin(np.abs(tab[:, 0] - rr))]
    analytic, paper_numeric = row[1], row[2]
    assert abs(analytic - 1.0 / rr) < 1e-4              # the printed analytic column is rho_l / rho_s
    c = W.film(nx=4, ny=48, h0=16.0, ste=0.1, rho_ratio=rr)
    o = oracle.Oracle(c)
    h0 = o.fields()["phi"][0].sum(axis=0).mean()
    F = o.step(12000).fields()
    assert F["fl"][:14].max() < 1e-12                    # the bulk of the film has frozen
    hf = F["phi"][0].sum(axis=0).mean()
    assert abs(hf / h0 / analytic - 1.0) < 0.015
    assert abs(hf / h0 / paper_numeric - 1.0) < 0.05     # the paper's own 5 % level


@pytest.mark.slow
@pytest.mark.parametrize("rr", [0.7, 0.75, 0.8, 0.85])
def test_table1_large_expansion_rows(rr):
    # The rows with the largest volume change.  At mobility 0.02 the films with
    # rho_s / rho_l <= 0.8 diverge within the first 1000 steps (the start-up freezing at
    # the wall drives the volume source faster than the phase field relaxes); Section 4.1
    # gives no mobility, and at 0.05 every row runs.  The whole film freezes by step
    # 16 000.  The paper's own level is 5 % on h_f / h_0 (Table 1).  The expansion h_f - h_0
    # comes out ~1 / h_0 short of the mass-conserving h_0 (rho_l / rho_s - 1) at every row
    # (6.4 % at h_0 = 16, 3.2 % at h_0 = 32): the volume source phi_p mdot of the phase
    # equations gives the gas its share of the expansion in the cells of the diffuse top
    # interface.  Bounded here by 10 %.
    tab = _table1()
    row = tab[np.argmin(np.abs(tab[:, 0] - rr))]
    analytic, paper_numeric = row[1], row[2]
    assert abs(analytic - 1.0 / rr) < 1e-4
    c = W.film(nx=4, ny=48, h0=16.0, ste=0.1, rho_ratio=rr, mobility=0.05)
    o = oracle.Oracle(c)
    h0 = o.fields()["phi"][0].sum(axis=0).mean()
    F = o.step(16000).fields()
    assert np.isfinite(F["phi"]).all()
    assert (F["fl"] * F["phi"][0]).sum(axis=0).mean() < 1e-6       # no liquid left
    hf = F["phi"][0].sum(axis=0).mean()
    assert abs(hf / h0 / paper_numeric - 1.0) < 0.05
    assert abs((hf / h0 - 1.0) / (analytic - 1.0) - 1.0) < 0.10


def _lens_angles(F, case):
    """Angles of the lens's upper and lower arcs with the flat 1-3 interface: circles
    fitted to the phi_2 = 1/2 crossings more than 3 lu above / below that interface,
    whose height is the phi_1 = 1/2 crossing in the outermost column."""
    col = [[v] for v in F["phi"][0][:, 0]]
    y0 = [p[1] for p in level_crossings(col) if abs(p[1] - case.meta["y_top"]) < 8.0][0]
    pts = level_crossings(F["phi"][1])
    xu, yu, Ru = fit_circle([p for p in pts if p[1] > y0 + 3.0])
    xd, yd, Rd = fit_circle([p for p in pts if p[1] < y0 - 3.0])
    return cap_angle(yu, Ru, y0, up=True), cap_angle(yd, Rd, y0, up=False)


@pytest.mark.slow
@pytest.mark.parametrize("s12,s23,s13", [(1e-2, 1e-2, 1e-2), (1e-2, 0.7e-2, 1.2e-2)])
def test_lens_junction_angles(s12, s23, s13):
    # A lens of phase 2 on a flat 1-3 interface, started as a disc (both arcs at 90
    # degrees): after 6000 steps the arcs meet the interface at the angles of the
    # tension balance (Section 2; 60 + 60 degrees, i.e. 120-degree interfacial angles,
    # for equal tensions, as Section 4.2 states for its three-phase pool), within 3 degrees.
    # Unequal tensions make the two arcs differ, so a swapped pair of sigma_pq fails.
    case = W.liquid_lens(s12=s12, s23=s23, s13=s13)
    F = oracle.Oracle(case).step(6000).fields()
    up, dn = _lens_angles(F, case)
    eu, ed = neumann_triangle(s12, s23, s13)
    print("lens arcs", up, dn, "balance", eu, ed)
    assert abs(up - eu) < 3.0 and abs(dn - ed) < 3.0


@pytest.mark.slow
@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_wetting_angle(theta):
    # A drop started as a half disc (90 degrees) on a wall that wets at theta relaxes
    # to a circular cap meeting the wall at theta (the wetting ghost of the order
    # parameter), within 3 degrees after 6000 steps.  No phase change (T > T_m), equal
    # densities and viscosities.  A sign error in the wetting term gives 180 - theta.
    case = W.sessile_cap(72, 36, 12.0, theta=90.0, T_wall=1.0, T0=1.0, rho_gas=1.0, mu_l=0.1,
                         mu_gas=0.1, cp_gas=1.0, lam_gas=0.1, sigma=1e-2)
    case.wet_cos = W.wetting(2, {W.YMIN: {(0, 1): theta}})
    F = oracle.Oracle(case).step(6000).fields()
    xc, yc, R = fit_circle([p for p in level_crossings(F["phi"][0]) if p[1] > 3.0])
    got = cap_angle(yc, R, 0.0, up=True)
    print("wetting", theta, got)
    assert abs(got - theta) < 3.0


@pytest.mark.slow
@pytest.mark.parametrize("r1,r2", [(1.05, 0.95), (1.1, 1.0)])
def test_pool_volume_change_per_phase(r1, r2):
    # Two liquids side by side under gas (Section 4.2, Fig. 4), frozen through from the
    # bottom wall (32 x 32, 9000 steps).  Each liquid's volume changes by
    # rho_l / rho_s - 1: contraction for rho_s > rho_l, expansion for rho_s < rho_l, none
    # for rho_s = rho_l.  The phase-field source phi_p mdot shares a liquid's change with
    # the other phases present in its interface cells, so at this size 83-88 % of the
    # change reaches the liquid itself (the shortfall falls as 1 / size) and a liquid with
    # rho_s = rho_l changes by ~0.5 %.
    c = W.lateral_pool(n=32, rho_ratio1=r1, rho_ratio2=r2)
    o = oracle.Oracle(c)
    V0 = [o.fields()["phi"][p].sum() for p in range(2)]
    F = o.step(9000).fields()
    assert (F["fl"] * (F["phi"][0] + F["phi"][1])).sum() < 1e-4        # frozen through
    for p, r in enumerate((r1, r2)):
        dV = F["phi"][p].sum() / V0[p] - 1.0
        if r == 1.0:
            assert abs(dV) < 0.1 * abs(1.0 / r1 - 1.0), (p, dV)
        else:
            assert 0.75 < dV / (1.0 / r - 1.0) <= 1.0, (p, dV)


@pytest.mark.slow
def test_poiseuille_and_frozen_channel():
    # Liquid: the steady profile is u(y) = g y (H - y) / (2 nu) (the flow LBE's viscosity
    # tau_f = mu / (rho c_s^2) + 1/2 and its body force, Section 3), within 2e-3 of its
    # peak (the wall slip of half-way bounce-back at tau_f = 0.8 is second order).
    # Frozen: the penalty force f_s (u_s - u*) holds the solid at u_s = 0 (Section 3, flow LBE):
    # below 1e-3 of the liquid's peak velocity, and it stays frozen.
    H, g, mu = 32, 1e-6, 0.1
    y = np.arange(H) + 0.5
    exact = g / (2.0 * mu) * y * (H - y)
    F = oracle.Oracle(W.channel(1.0, H, g, mu)).step(40000).fields()
    assert np.abs(F["ux"] - exact[:, None]).max() < 2e-3 * exact.max()
    assert np.abs(F["uy"]).max() < 1e-12
    F = oracle.Oracle(W.channel(-1.0, H, g, mu)).step(40000).fields()
    assert F["fl"].max() == 0.0
    assert np.abs(F["ux"]).max() < 1e-3 * exact.max()


def _table2():
    rows = np.loadtxt(os.path.join(GOLDEN, "table2_janus_lengths.txt"))
    return {int(r[0]): (r[1], r[2], r[3], r[4]) for r in rows}


def test_janus_geometry_reproduces_table2_analytic():
    # The equilibrium of a 2D Janus drop (circular arcs, Young's law at the three wall
    # contact lines with the 1-2 angle from the same wall energies, tension balance at
    # the triple junction, equal areas pi R^2 / 4) gives the analytic column of Table 2
    # (Section 4.3) to the printed four digits.
    for th23, (l1, l2, _, _) in _table2().items():
        L1, L2 = janus_wetting_lengths(75.0, th23)
        print("Janus analytic", th23, L1, L2, "Table 2", l1, l2)
        assert abs(L1 - l1) < 1.5e-4 and abs(L2 - l2) < 1.5e-4


@pytest.mark.slow
def test_janus_wetting_lengths():
    # Janus drop of Section 4.3 (theta_13 = 75 degrees, equal tensions) at R = 24, eps = 4
    # (eps / R = 1/6, the paper's 1/12 at R = 60 is a GPU test), three angles theta_23 in
    # parallel threads, 12 000 steps: the wetting lengths L1 / R and L2 / R within 5 % of
    # Table 2's analytic values (the paper's own results are within 3.05 %).  This pins the
    # pairwise wetting ghost phi_p + (4 / eps) sum_q cos(theta_pq) phi_p phi_q for N = 3
    # with every pair wetting at its own angle.  Measured: 60: -1.7 / -1.5 %, 90: -0.2 /
    # -0.5 %, 120: +0.6 / -2.2 %.  A sign error in the ghost, or the 1-2 pair left neutral,
    # moves the lengths by far more.
    import threading
    ref = _table2()
    R = 24.0
    got = {}

    def run(th23):
        c = W.janus_drop(nx=120, ny=60, R=R, theta23=float(th23), eps=4.0, mobility=0.1, mu=0.1)
        F = oracle.Oracle(c).step(12000).fields()
        got[th23] = janus_contact_lengths(F["phi"])

    ths = [60, 90, 120]
    T = [threading.Thread(target=run, args=(t,)) for t in ths]
    for t in T:
        t.start()
    for t in T:
        t.join()
    for th in ths:
        L1, L2 = got[th][0] / R, got[th][1] / R
        a1, a2 = ref[th][0], ref[th][1]
        print("Janus", th, L1, L2, "analytic", a1, a2, "rel", L1 / a1 - 1, L2 / a2 - 1)
        assert abs(L1 / a1 - 1.0) < 0.05 and abs(L2 / a2 - 1.0) < 0.05


@pytest.mark.slow
def test_penalty_weight_in_mixed_cells():
    # A frozen layer of phase-changing material (y < 12) under a channel of ambient fluid,
    # driven by a body force, everything below T_m.  In the steady unidirectional flow the
    # flow LBE reduces to nu u'' + g + f = 0 with the penalty force f = chi (0 - u*) and
    # u = u* + f / 2 (Section 3), i.e. nu u'' - chi / (1 - chi / 2) u + g = 0: a Brinkman
    # equation whose damping is the penalty weight chi.  With chi the solid volume fraction
    # f_s * sum of the phase-changing phi_p (the reading of the penalty in cells that also
    # hold ambient fluid), the lattice profile must be the solution of that equation with
    # the lattice's own chi within 1 % of the peak (measured 0.49 %), and with the tanh chi
    # of the initial layer within 2 % (1.3 %); the solid stays still.  The literal weight
    # f_s freezes the whole channel, since every cell of the ambient fluid holds a tail of
    # phase-changing material below T_m (f_s = 1): that profile misses by more than 50 %.
    c = W.frozen_layer_channel()
    H, g, nu, h = c.ny, c.meta["g"], c.meta["mu"], c.meta["h"]
    y = np.arange(H) + 0.5
    F = oracle.Oracle(c).step(25000).fields()
    chi = ((1.0 - F["fl"]) * F["phi"][0]).mean(axis=1)
    u = F["ux"].mean(axis=1)
    yb, ub = brinkman_profile(H, y, chi, g, nu)
    exact = np.interp(y, yb, ub)
    err = np.abs(u - exact).max() / exact.max()
    yt, ut = brinkman_profile(H, y, 0.5 - 0.5 * np.tanh(2.0 * (y - h) / c.eps), g, nu)
    err_tanh = np.abs(u - np.interp(y, yt, ut)).max() / exact.max()
    solid = F["phi"][0].mean(axis=1) > 0.99
    print("penalty: Brinkman error", err, "with tanh chi", err_tanh, "solid |u|", np.abs(u[solid]).max())
    assert err < 1e-2 and err_tanh < 2e-2
    assert np.abs(u[solid]).max() < 1e-3 * exact.max()
    assert np.abs(F["uy"]).max() < 1e-6 * exact.max() and F["fl"][F["phi"][0] > 0.5].max() == 0.0
    L = oracle.Oracle(c, penalty_literal=True).step(25000).fields()
    err_lit = np.abs(L["ux"].mean(axis=1) - exact).max() / exact.max()
    print("literal penalty weight: error", err_lit)
    assert err_lit > 0.5
