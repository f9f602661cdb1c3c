"""Pins of the oracle's mixture rule (eq. 2) and enthalpy map (eq. H), Section 2.

Each check is fixed by the paper or by mathematics, not by re-typing the oracle:
the reduction to the classical constant-density map (the paper states it),
continuity at both break points, the inverse round trip, monotonicity, the
linear mixture of eq. 2 in pure solid / pure liquid, and f_s = 0 in the ambient
fluid (Fig. 1 caption).
"""
import numpy as np
import pytest

import oracle
from paper_2603_22902_gb300 import workloads as W


def _case(rho_s=0.9, cp_s=0.8, cp_l=1.3, latent=5.0, T_sol=-0.1, T_liq=0.2, N=2):
    phases = [W.phase(rho_l=1.0, rho_s=rho_s, cp_l=cp_l, cp_s=cp_s, mu_l=0.1, mu_s=0.3,
                      lam_l=0.1, lam_s=0.2, latent=latent),
              W.phase(rho_l=0.05, cp_l=2.0, mu_l=0.01, lam_l=0.03)]
    phases += [W.phase(rho_l=0.5, rho_s=0.5, cp_l=1.0) for _ in range(N - 2)]
    c = W.Case(name="map", nx=4, ny=4, N=N, phases=phases, sigma=np.zeros((N, N)),
               T_sol=T_sol, T_liq=T_liq)
    return c


def classic_map(H, cs, cl, L, Ts, Tl):
    """Classical enthalpy method, constant density: H = c_p T + L f_l per unit mass."""
    Hs, Hl = cs * Ts, cl * Tl + L
    if H < Hs:
        return 0.0, H / cs
    if H > Hl:
        return 1.0, Tl + (H - Hl) / cl
    fl = (H - Hs) / (Hl - Hs)
    return fl, Ts + fl * (Tl - Ts)


@pytest.mark.parametrize("rho", [1.0, 0.37])
def test_constant_density_reduces_to_classic_map(rho):
    # Section 2: the density-weighted map "reduces to the conventional forms when rho_s = rho_l"
    c = _case(rho_s=rho, cp_s=0.8, cp_l=1.3, latent=5.0)
    c.phases[0]["rho_l"] = rho
    phi = np.array([1.0, 0.0])
    for H in np.linspace(-2.0, 9.0, 157):
        fl, T, rho_out, psi, chi = oracle.enthalpy_map(c, phi, rho * H)
        fl_ref, T_ref = classic_map(H, 0.8, 1.3, 5.0, -0.1, 0.2)
        assert abs(fl - fl_ref) <= 1e-14
        assert abs(T - T_ref) <= 1e-13 * max(1.0, abs(T_ref))
        assert abs(rho_out - rho) <= 1e-15


def test_map_continuous_at_break_points():
    c = _case()
    for phi in (np.array([1.0, 0.0]), np.array([0.6, 0.4]), np.array([0.05, 0.95])):
        As = oracle.inverse_map(c, phi, c.T_sol)   # start of the mushy range
        Al = oracle.inverse_map(c, phi, c.T_liq)   # end of the mushy range
        for Hb in (As, Al):
            d = 1e-9 * max(1.0, abs(Hb))
            lo = oracle.enthalpy_map(c, phi, Hb - d)
            hi = oracle.enthalpy_map(c, phi, Hb + d)
            # f_l jumps by at most d / (Al - As); T by at most d / min(rho c_p)
            assert abs(hi[0] - lo[0]) <= 4 * d / (Al - As) + 1e-15
            assert abs(hi[1] - lo[1]) <= 4 * d / 0.04 + 1e-15


def test_inverse_round_trip_and_monotone():
    for Ts, Tl in ((-0.1, 0.2), (0.0, 0.0)):
        c = _case(T_sol=Ts, T_liq=Tl)
        for phi in (np.array([1.0, 0.0]), np.array([0.7, 0.3]), np.array([0.2, 0.8])):
            Ts_grid = np.concatenate([np.linspace(-2, 2, 41), [Ts, Tl]])
            for T in Ts_grid:
                rhoH = oracle.inverse_map(c, phi, T)
                fl, T_back, *_ = oracle.enthalpy_map(c, phi, rhoH)
                if Ts < Tl or T != Ts:
                    assert abs(T_back - T) <= 1e-13, (phi, T, T_back)
                if T >= Tl:
                    assert fl == 1.0
            Hs = np.linspace(oracle.inverse_map(c, phi, -2.0), oracle.inverse_map(c, phi, 2.0), 301)
            out = np.array([oracle.enthalpy_map(c, phi, H)[:2] for H in Hs])
            assert np.all(np.diff(out[:, 0]) >= 0.0)
            assert np.all(np.diff(out[:, 1]) >= -1e-15)


def test_mixture_rule_pure_solid_and_liquid():
    # eq. 2: xi = sum_p [f_s phi_p xi_p^s + (1 - f_s) phi_p xi_p^l]
    c = _case()
    phi = np.array([0.3, 0.7])
    fl, T, rho, psi, chi = oracle.enthalpy_map(c, phi, 1e3)      # far above liquidus
    assert fl == 1.0 and abs(rho - (0.3 * 1.0 + 0.7 * 0.05)) < 1e-15 and psi == 0.0 and chi == 0.0
    fl, T, rho, psi, chi = oracle.enthalpy_map(c, phi, -1e3)     # far below solidus
    assert fl == 0.0 and abs(rho - (0.3 * 0.9 + 0.7 * 0.05)) < 1e-15
    # psi is the phase-change part of rho: rho - sum_p phi_p rho_p^l
    assert abs(psi - (rho - (0.3 * 1.0 + 0.7 * 0.05))) < 1e-15
    assert abs(chi - 0.3) < 1e-15                                 # solid volume fraction


def test_ambient_fluid_is_never_solid():
    # Fig. 1 caption: the ambient fluid has f_s = 0 whatever its temperature
    c = _case()
    phi = np.array([0.0, 1.0])
    for T in (-5.0, -0.5, 0.0, 3.0):
        rhoH = oracle.inverse_map(c, phi, T)
        fl, T_back, rho, psi, chi = oracle.enthalpy_map(c, phi, rhoH)
        assert fl == 1.0 and psi == 0.0 and chi == 0.0
        assert abs(rhoH - 0.05 * 2.0 * T) < 1e-15           # rho c_p T of the ambient phase
        assert abs(T_back - T) < 1e-14
