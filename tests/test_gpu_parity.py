"""GPU parity: the FP64 CUDA path (through the C ABI) against the CPU oracle on the
same seeded inputs.

Bar: max |GPU - oracle| <= 1e-10 on every exported field (phi_p, T, f_l, u, p, and the
specific enthalpy H scaled by max(1, |H|max), since H = rho H / rho reaches ~100 in
a gas of density 0.01) after 1000 steps on small cases that span several tiles and
ragged tails, and after a few steps at the full sizes of the paper's problems in the
launch configuration the benchmark times.  The oracle is compiled with
-ffp-contract=off, the kernels with FMA contraction; the bound absorbs that.

Exception, measured on the oracle itself: with a gas of density 0.01 the scheme
amplifies round-off (a 1e-15 relative change of one temperature grows to ~1e-6 by step
400-1000; the pairwise normal n_pq is taken of near-zero gradients of phi tails of
~1e-7 in the gas).  No implementation that is not bitwise identical to the oracle can
hold 1e-10 there at 1000 steps.  For those droplet cases the bar is 1e-10 up to step
150, and at 1000 steps the GPU must stay within 10x the oracle's own divergence under
a 1e-15 perturbation, with the conserved sums matching to 1e-10.
"""
import numpy as np
import pytest

import oracle
from paper_2603_22902_gb300 import workloads as W
from tests._cases import sensitive_cases, small_cases

pytestmark = pytest.mark.gpu

TOL = 1e-10
FIELDS = ("phi", "T", "H", "fl", "ux", "uy", "p")


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for the gpu tests")
    from paper_2603_22902_gb300 import build as B
    B.build()
    from paper_2603_22902_gb300 import lbm as L
    return L


def compare(G, O, tol=TOL):
    errs = {}
    for k in FIELDS:
        scale = max(1.0, float(np.abs(O[k]).max())) if k == "H" else 1.0
        errs[k] = float(np.abs(G[k] - O[k]).max()) / scale
    bad = {k: v for k, v in errs.items() if not (v <= tol)}
    assert not bad, f"parity failed: {errs}"
    return errs


def run_pair(L, case, steps, tile=None):
    s = L.Solver(case, tile=tile).set_fields()
    s.step(steps)
    G = s.fields_numpy()
    s.close()
    O = oracle.Oracle(case).step(steps).fields()
    return G, O


@pytest.mark.parametrize("name", list(small_cases().keys()))
def test_parity_1000_steps(lbm, name):
    case = small_cases()[name]
    G, O = run_pair(lbm, case, 1000)
    errs = compare(G, O)
    print(name, errs)


@pytest.mark.parametrize("name", list(sensitive_cases().keys()))
def test_parity_round_off_sensitive_droplets(lbm, name):
    case = sensitive_cases()[name]
    G, O = run_pair(lbm, case, 150)
    print(name, "150 steps", compare(G, O))
    s = lbm.Solver(case).set_fields()
    s.step(1000)
    G = s.fields_numpy()
    d = s.diagnostics()
    s.close()
    pert = case.copy()
    pert.T = pert.T.copy()
    pert.T[case.ny // 2, case.nx // 2] *= 1.0 + 1e-15
    oa, ob = oracle.Oracle(case).step(1000), oracle.Oracle(pert).step(1000)
    O, Op = oa.fields(), ob.fields()
    for k in FIELDS:
        floor = float(np.abs(O[k] - Op[k]).max())
        err = float(np.abs(G[k] - O[k]).max())
        assert err <= max(TOL, 10.0 * floor), (k, err, floor)
    fs = 1.0 - O["fl"]
    for p in range(case.N):
        assert abs(d["mass"][p] - O["phi"][p].sum()) <= 1e-10 * O["phi"][p].sum()
        assert abs(d["solid"][p] - (fs * O["phi"][p]).sum()) <= 1e-8


def test_tile_shapes_agree(lbm):
    # Every tile shape runs the same per-cell arithmetic; each shape is a separate
    # instantiation, and the compiler may fuse a different multiply-add into an FMA in
    # each, so the shapes agree to rounding (the same CPU emulation of the source is
    # bitwise identical across shapes), not bit for bit.
    case = W.sessile_drop(n=45, R=12.0, theta=70.0, ny=38)
    ref = None
    for tile in [(32, 8), (32, 4), (64, 4), (16, 16)]:
        s = lbm.Solver(case, tile=tile).set_fields()
        s.step(60)
        F = s.fields_numpy()
        s.close()
        if ref is None:
            ref = F
        else:
            for k in FIELDS:
                d = float(np.abs(F[k] - ref[k]).max())
                assert d <= 1e-12, (tile, k, d)


def test_host_and_device_io_agree(lbm):
    import torch
    L = lbm
    case = W.film(nx=16, ny=64, h0=32.0)
    s = L.Solver(case).set_fields()
    s.step(25)
    Fd = s.fields_numpy()
    out = {k: np.empty((case.ny, case.nx)) for k in ("T", "H", "fl", "ux", "uy", "p")}
    out["phi"] = np.empty((case.N, case.ny, case.nx))
    L.lbm_get_fields(s.h, out["phi"], out["T"], out["H"], out["fl"], out["ux"], out["uy"], out["p"], L.LBM_HOST)
    for k in FIELDS:
        assert np.array_equal(out[k], Fd[k]), k
    # host-buffer initialisation equals device initialisation
    s2 = L.Solver(case)
    L.lbm_set_fields(s2.h, np.ascontiguousarray(case.phi), np.ascontiguousarray(case.T),
                     np.ascontiguousarray(case.ux), np.ascontiguousarray(case.uy), L.LBM_HOST)
    s2.step(25)
    F2 = s2.fields_numpy()
    for k in FIELDS:
        assert np.array_equal(F2[k], Fd[k]), k
    s.close()
    s2.close()


def test_save_load_continues_bitwise(lbm):
    case = W.compound_drop(n=40, R_core=7.0, R_shell=13.0, noise=0.0)
    a = lbm.Solver(case).set_fields().step(30)
    blob = a.save_state()
    a.step(20)
    Fa = a.fields_numpy()
    b = lbm.Solver(case).load_state(blob)
    assert b.steps == 30
    b.step(20)
    Fb = b.fields_numpy()
    for k in FIELDS:
        assert np.array_equal(Fa[k], Fb[k]), k
    a.close()
    b.close()


def test_diagnostics_match_oracle(lbm):
    case = W.sessile_drop(n=40, R=12.0, theta=90.0, ny=32)
    s = lbm.Solver(case).set_fields().step(300)
    d = s.diagnostics()
    O = oracle.Oracle(case).step(300).fields()
    fs = 1.0 - O["fl"]
    for p in range(case.N):
        assert abs(d["mass"][p] - O["phi"][p].sum()) < 1e-9
        assert abs(d["solid"][p] - (fs * O["phi"][p]).sum()) < 1e-9
    assert abs(d["max_sum_dev"] - np.abs(O["phi"].sum(0) - 1).max()) < 1e-12
    assert d["nonfinite"] == 0 and d["steps"] == 300
    s.close()


def test_state_errors(lbm):
    case = W.film(nx=8, ny=16)
    s = lbm.Solver(case)
    with pytest.raises(lbm.LBMError) as e:
        s.step(1)
    assert e.value.code == lbm.LBM_ESTATE
    s.close()


@pytest.mark.parametrize("name,maker,steps", [
    ("film_16x256_full", lambda: W.film(), 3),
    ("sessile_drop_512", lambda: W.sessile_drop(), 2),
])
def test_parity_full_size_few_steps(lbm, name, maker, steps):
    case = maker()
    G, O = run_pair(lbm, case, steps)
    print(name, compare(G, O))


def test_full_size_compound_sampled(lbm):
    """1024^2, N = 3: a few steps, compared on a sampled band of rows (the oracle runs the
    whole grid; the comparison keeps the test's memory small)."""
    case = W.compound_drop()
    G, O = run_pair(lbm, case, 2)
    rows = np.r_[0:8, 150:170, 500:520, 1016:1024]
    sub = lambda F: {k: (F[k][:, rows] if k == "phi" else F[k][rows]) for k in FIELDS}
    print("compound_1024", compare(sub(G), sub(O)))


def test_mass_conserved_without_freezing_long_run(lbm):
    case = W.sessile_drop(n=256, R=60.0, T_wall=2.0, theta=75.0)
    s = lbm.Solver(case).set_fields()
    m0 = s.diagnostics()["mass"]
    s.step(3000)
    d = s.diagnostics()
    assert d["nonfinite"] == 0
    for p in range(case.N):
        assert abs(d["mass"][p] / m0[p] - 1.0) < 1e-11
    s.close()
