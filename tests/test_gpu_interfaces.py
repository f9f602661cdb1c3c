"""Interface equilibria on the GPU, held to the oracle pins' bounds: a lens of phase 2
on a flat 1-3 interface relaxes to the angles of the tension balance (Section 2), and a
drop on a wetting wall relaxes to its contact angle (the wetting ghost of the order
parameter), each within 3 degrees after 6000 steps, on the FP64, double-word and FP32
policies; the Laplace pressure jump of large drops; the per-phase volume change of a
frozen two-liquid pool converging with the lattice size; the Janus drop's wetting lengths
of Table 2 at the paper's size; and the penalty-weighted channel over a frozen layer
against the Brinkman profile."""
import numpy as np
import pytest

from paper_2603_22902_gb300 import workloads as W
from tests._analytic import (brinkman_profile, cap_angle, fit_circle, janus_contact_lengths, janus_wetting_lengths,
                             level_crossings, neumann_triangle)

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


def run(L, case, prec, steps=6000):
    s = L.Solver(case, precision=prec).set_fields()
    s.step(steps)
    F = s.fields_numpy()
    d = s.diagnostics()
    s.close()
    assert d["nonfinite"] == 0
    return F


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
@pytest.mark.parametrize("s12,s23,s13", [(1e-2, 1e-2, 1e-2), (1e-2, 0.7e-2, 1.2e-2)])
def test_lens_junction_angles(lbm, prec, s12, s23, s13):
    case = W.liquid_lens(s12=s12, s23=s23, s13=s13)
    F = run(lbm, case, prec)
    col = [[v] for v in F["phi"][0][:, 0]]
    y0 = [p[1] for p in level_crossings(col) if abs(p[1] - case.meta["y_top"]) < 8.0][0]
    pts = level_crossings(F["phi"][1])
    _, yu, Ru = fit_circle([p for p in pts if p[1] > y0 + 3.0])
    _, yd, Rd = fit_circle([p for p in pts if p[1] < y0 - 3.0])
    up, dn = cap_angle(yu, Ru, y0, up=True), cap_angle(yd, Rd, y0, up=False)
    eu, ed = neumann_triangle(s12, s23, s13)
    print(prec, "lens arcs", up, dn, "balance", eu, ed)
    assert abs(up - eu) < 3.0 and abs(dn - ed) < 3.0


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
@pytest.mark.parametrize("theta", [60.0, 120.0])
def test_wetting_angle(lbm, prec, theta):
    case = W.sessile_cap(72, 36, 12.0, theta=90.0, T_wall=1.0, T0=1.0, rho_gas=1.0, mu_l=0.1,
                         mu_gas=0.1, cp_gas=1.0, lam_gas=0.1, sigma=1e-2)
    case.wet_cos = W.wetting(2, {W.YMIN: {(0, 1): theta}})
    F = run(lbm, case, prec)
    _, yc, R = fit_circle([p for p in level_crossings(F["phi"][0]) if p[1] > 3.0])
    got = cap_angle(yc, R, 0.0, up=True)
    print(prec, "wetting", theta, got)
    assert abs(got - theta) < 3.0


@pytest.mark.parametrize("R", [20.0, 30.0, 40.0])
def test_laplace_law_large_drops(lbm, R):
    # Delta p = sigma / R at the radii the oracle pin cannot afford on the CPU (box 160^2,
    # gas density 0.1, viscosity 0.3, pressure jump averaged over 50 samples 100 steps
    # apart after 6000 steps): within 3 % at eps = 8; at eps = 4 the jump is ~7 % low
    # at every radius (the second-order error of the interface's resolution)
    import numpy as np
    sigma, n = 1e-3, 160
    X, Y = W.grid(n, n)
    r = np.hypot(X - n / 2.0, Y - n / 2.0)
    out = {}
    for eps in (8.0, 4.0):
        case = W.periodic_drop(n=n, R=R, sigma=sigma, rho_gas=0.1, mu=0.3, eps=eps)
        s = lbm.Solver(case).set_fields()
        s.step(6000)
        vals = []
        for _ in range(50):
            s.step(100)
            p = s.fields_numpy()["p"]
            vals.append((p[r < R / 2].mean() - p[r > R + 2 * eps].mean()) * R / sigma)
        s.close()
        out[eps] = float(np.mean(vals))
    print("laplace R", R, out)
    assert abs(out[8.0] - 1.0) < 0.03
    assert abs(out[4.0] - 1.0) >= 3.0 * abs(out[8.0] - 1.0)
    assert abs(out[4.0] - 1.0) < 0.10


def test_pool_volume_change_converges(lbm):
    # The two-liquid pool (Section 4.2, Fig. 4) frozen through at sides 32, 64 and 128:
    # the part of each liquid's volume change rho_l / rho_s - 1 that its phase field does
    # not take (the share given to the other phases of its interface cells) halves with
    # each doubling of the size, and is below 5 % at 128; a liquid with rho_s = rho_l
    # changes by a vanishing amount likewise.
    short, leak = [], []
    for n, steps in ((32, 9000), (64, 36000), (128, 144000)):
        res = {}
        for r1, r2 in ((1.05, 0.95), (1.1, 1.0)):
            case = W.lateral_pool(n=n, rho_ratio1=r1, rho_ratio2=r2)
            s = lbm.Solver(case).set_fields()
            F0 = s.fields_numpy()
            V0 = [F0["phi"][p].sum() for p in range(2)]
            s.step(steps)
            F = s.fields_numpy()
            s.close()
            assert (F["fl"] * (F["phi"][0] + F["phi"][1])).sum() < 1e-3
            res[(r1, r2)] = [F["phi"][p].sum() / V0[p] - 1.0 for p in range(2)]
        a = res[(1.05, 0.95)]
        short.append(max(1.0 - a[0] / (1 / 1.05 - 1), 1.0 - a[1] / (1 / 0.95 - 1)))
        leak.append(abs(res[(1.1, 1.0)][1]))
    print("pool shortfall", short, "leak", leak)
    for k in range(2):
        assert 1.7 < short[k] / short[k + 1] < 2.3
        assert 1.7 < leak[k] / leak[k + 1] < 2.3
    assert 0.0 < short[2] < 0.05


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_poiseuille_and_frozen_channel(lbm, prec):
    # The oracle pin's channel on the GPU: the liquid's steady profile within 2e-3 of
    # Poiseuille's peak, and the same channel frozen held below 1e-3 of it by the penalty
    import numpy as np
    H, g, mu = 32, 1e-6, 0.1
    y = np.arange(H) + 0.5
    exact = g / (2.0 * mu) * y * (H - y)
    F = run(lbm, W.channel(1.0, H, g, mu), prec, steps=40000)
    print(prec, "poiseuille rel err", float(np.abs(F["ux"] - exact[:, None]).max() / exact.max()))
    assert np.abs(F["ux"] - exact[:, None]).max() < 2e-3 * exact.max()
    F = run(lbm, W.channel(-1.0, H, g, mu), prec, steps=40000)
    print(prec, "frozen channel umax", float(np.abs(F["ux"]).max()))
    assert F["fl"].max() == 0.0
    assert np.abs(F["ux"]).max() < 1e-3 * exact.max()


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_uniform_translation_with_equal_densities(lbm, prec):
    # the oracle pin's translating drop: displacement u0 t within 1e-3, velocity kept
    import numpy as np
    from tests.test_oracle_invariants import _periodic_centroid
    n, u0, steps = 48, (0.02, 0.01), 1000
    case = W.periodic_drop(n=n, R=10.0, sigma=1e-3, rho_gas=1.0, mu=0.1)
    case.ux = np.full((n, n), u0[0])
    case.uy = np.full((n, n), u0[1])
    x0 = _periodic_centroid(case.phi[0])
    F = run(lbm, case, prec, steps=steps)
    x1 = _periodic_centroid(F["phi"][0])
    for a, b, u in zip(x0, x1, u0):
        d = (b - a + n / 2) % n - n / 2
        print(prec, "translation", d, u * steps)
        assert abs(d / (u * steps) - 1.0) < 1e-3
    assert abs(F["ux"].mean() / u0[0] - 1.0) < 1e-3 and abs(F["uy"].mean() / u0[1] - 1.0) < 1e-3


@pytest.mark.parametrize("th23", [30.0, 60.0, 90.0, 120.0])
def test_janus_wetting_lengths_table2(lbm, th23):
    # Section 4.3 at the paper's size: domain 300 x 150, R = 60, eps = 5, theta_13 = 75
    # degrees, equal tensions 0.01.  Stepped in chunks of 20 000 until the lengths change by
    # less than 0.1 % of R per chunk (at most 400 000 steps); then within 5 % of Table 2's
    # analytic values (the paper's own errors reach 3.05 %), and the double-word run of the
    # same length gives the same lengths to 1e-6 of R.
    R = 60.0
    case = W.janus_drop(theta23=th23, mobility=0.1)
    ana = janus_wetting_lengths(75.0, th23)
    out = {}
    for prec in ("fp64", "df64"):
        s = lbm.Solver(case, precision=prec).set_fields()
        prev, steps = None, 0
        while True:
            s.step(20000)
            steps += 20000
            L = np.array(janus_contact_lengths(s.fields_numpy()["phi"])) / R
            if prec == "df64":
                if steps >= out["fp64"][1]:
                    break
            elif (prev is not None and np.abs(L - prev).max() < 1e-3) or steps >= 400000:
                break
            prev = L
        d = s.diagnostics()
        s.close()
        assert d["nonfinite"] == 0
        out[prec] = (L, steps)
    L1, L2 = out["fp64"][0]
    print("Janus", th23, "steps", out["fp64"][1], "L/R", L1, L2, "analytic", ana,
          "rel", L1 / ana[0] - 1, L2 / ana[1] - 1, "df64 diff", np.abs(out["df64"][0] - out["fp64"][0]).max())
    assert abs(L1 / ana[0] - 1.0) < 0.05 and abs(L2 / ana[1] - 1.0) < 0.05
    assert np.abs(out["df64"][0] - out["fp64"][0]).max() < 1e-6


@pytest.mark.parametrize("prec", ["fp64", "df64", "fp32"])
def test_penalty_weight_in_mixed_cells(lbm, prec):
    # The oracle pin of the penalty weight (test_oracle_physics): a frozen layer under a
    # driven channel of ambient fluid; the steady profile solves nu u'' - k(y) u + g = 0,
    # k = chi / (1 - chi / 2), with chi the solid volume fraction, within 1 % of the peak.
    c = W.frozen_layer_channel()
    H, g, nu = c.ny, c.meta["g"], c.meta["mu"]
    y = np.arange(H) + 0.5
    F = run(lbm, c, prec, steps=25000)
    chi = ((1.0 - F["fl"]) * F["phi"][0]).mean(axis=1)
    u = F["ux"].mean(axis=1)
    yb, ub = brinkman_profile(H, y, chi, g, nu)
    exact = np.interp(y, yb, ub)
    err = np.abs(u - exact).max() / exact.max()
    solid = F["phi"][0].mean(axis=1) > 0.99
    print(prec, "penalty: Brinkman error", err, "solid |u|", np.abs(u[solid]).max())
    assert err < 1e-2
    assert np.abs(u[solid]).max() < 1e-3 * exact.max()
