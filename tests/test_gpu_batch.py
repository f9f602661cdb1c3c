"""Batches of independent cases (lbm_batch_*): the batch launches run the per-cell step
of lbm_step, so every case of a batch must match the same case stepped alone (FP64: to
rounding, since the batch kernels are other instantiations of the same source), and
one case through the batch must match the CPU oracle to the 1e-10 parity bar.  Both
launch forms, all three tile shapes, odd step counts in both forms (each call is replayed
as a captured graph; the persistent launch flips its own parity, the per-step form ends an
odd call with a parity-flip kernel), members stepped alone between batch steps, and the
autotuner's restoration of the state are covered, for FP64 and for double words (32x8 tiles).  The staged form (16-bit storage, N = 2,
32x8 tiles) runs the staged step's arithmetic: its cases must match the per-step form's
and the single runs' to one unit of the 16-bit format, like the per-step form."""
import numpy as np
import pytest

import oracle
from paper_2603_22902_gb300 import workloads as W

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


def singles(lbm, cases, steps, precision="fp64"):
    out = []
    for c in cases:
        s = lbm.Solver(c, precision=precision).set_fields()
        s.step(steps)
        out.append(s.fields_numpy())
        s.close()
    return out


def max_err(A, B):
    return max(float(np.abs(A[k] - B[k]).max()) for k in FIELDS)


@pytest.mark.parametrize("mode", ["persistent", "per_step"])
@pytest.mark.parametrize("tile", [(32, 8), (64, 4), (16, 16)])
def test_batch_matches_single_runs(lbm, mode, tile):
    cases = W.small_batch()
    steps = 60
    ref = singles(lbm, cases, steps)
    solvers = [lbm.Solver(c).set_fields() for c in cases]
    b = lbm.Batch(solvers).set_plan(mode=mode, tiles=[tile] * lbm.BATCH_CLASSES)
    b.step(steps).sync()
    for s, c, R in zip(solvers, cases, ref):
        assert s.steps == steps
        e = max_err(s.fields_numpy(), R)
        assert e <= 1e-12, (c.name, mode, tile, e)
    plan = b.plan.as_dict()
    print(mode, tile, plan)
    b.close()
    for s in solvers:
        s.close()


def test_batch_case_against_oracle(lbm):
    cases = W.small_batch()
    steps = 200
    solvers = [lbm.Solver(c).set_fields() for c in cases]
    b = lbm.Batch(solvers)
    b.step(steps).sync()
    for k in (0, 1):   # a sessile cap (wetting, Dirichlet wall) and the film (outflow)
        G = solvers[k].fields_numpy()
        O = oracle.Oracle(cases[k]).step(steps).fields()
        e = max_err(G, O)
        assert e <= 1e-10, (cases[k].name, e)
    b.close()
    for s in solvers:
        s.close()


@pytest.mark.parametrize("mode", ["persistent", "per_step", "staged"])
def test_batch_odd_calls_graph_replay_and_member_steps(lbm, mode):
    # (FP64 cases: the staged mode runs its groups in the per-step form)
    cases = W.small_batch()
    ref = singles(lbm, cases, 9)
    solvers = [lbm.Solver(c).set_fields() for c in cases]
    b = lbm.Batch(solvers).set_plan(mode=mode, tiles=[(32, 8)] * lbm.BATCH_CLASSES)
    b.step(3).step(3)            # second call replays the captured graph; parity flips twice
    solvers[2].step(1)           # a member stepped on its own between batch calls
    b.step(1)
    b.sync()
    for s in solvers[:2] + solvers[3:]:
        assert s.steps == 7
    assert solvers[2].steps == 8
    solvers_rest = [s for i, s in enumerate(solvers) if i != 2]
    for s in solvers_rest:
        s.step(2)
    solvers[2].step(1)
    import torch
    torch.cuda.synchronize()
    for s, c, R in zip(solvers, cases, ref):
        e = max_err(s.fields_numpy(), R)
        assert e <= 1e-12, (c.name, e)
    plan = b.plan.as_dict()
    print(mode, plan)
    if mode != "persistent":
        assert plan["graph"]       # the per-step calls replay a captured graph
    b.close()
    for s in solvers:
        s.close()


def test_batch_autotune_restores_state(lbm):
    cases = W.small_batch()
    solvers = [lbm.Solver(c).set_fields() for c in cases]
    b = lbm.Batch(solvers)
    b.step(5).sync()
    before = [s.fields_numpy() for s in solvers]
    plan = b.autotune(trial_steps=4)
    print("autotuned plan", plan)
    assert plan["mode"] in ("persistent", "per_step")
    after = [s.fields_numpy() for s in solvers]
    for s, A, B_ in zip(solvers, before, after):
        assert s.steps == 5
        for k in FIELDS:
            assert np.array_equal(A[k], B_[k]), k
    b.step(3).sync()
    ref = singles(lbm, cases, 8)
    for s, R in zip(solvers, ref):
        assert max_err(s.fields_numpy(), R) <= 1e-12
    b.close()
    for s in solvers:
        s.close()


@pytest.mark.parametrize("prec", ["fp32", "fp16s"])
def test_reduced_precision_batch_matches_single_runs(lbm, prec):
    # FP32 arithmetic of another instantiation may round differently; with 16-bit
    # storage such a difference can move a stored value by one unit of the format.
    cases = W.small_batch()
    steps = 60
    ref = singles(lbm, cases, steps, prec)
    solvers = [lbm.Solver(c, precision=prec).set_fields() for c in cases]
    b = lbm.Batch(solvers)
    b.step(steps).sync()
    bound = {"fp32": 1e-5, "fp16s": 2e-2}[prec]
    for s, c, R in zip(solvers, cases, ref):
        e = max_err(s.fields_numpy(), R)
        assert e <= bound, (c.name, prec, e)
    b.close()
    for s in solvers:
        s.close()


@pytest.mark.parametrize("mode", ["persistent", "per_step"])
def test_double_word_batch(lbm, mode):
    # the double-word policy in both batch forms (32x8 tiles): every case as its single run
    # to rounding, one case against the oracle at the parity bar; other tile shapes refused
    cases = W.small_batch()
    steps = 60
    ref = singles(lbm, cases, steps, "df64")
    solvers = [lbm.Solver(c, precision="df64").set_fields() for c in cases]
    b = lbm.Batch(solvers).set_plan(mode=mode, tiles=[(32, 8)] * lbm.BATCH_CLASSES)
    b.step(steps).sync()
    for s, c, R in zip(solvers, cases, ref):
        e = max_err(s.fields_numpy(), R)
        assert e <= 1e-12, (c.name, mode, e)
    b.step(140).sync()
    O = oracle.Oracle(cases[0]).step(200).fields()
    e = max_err(solvers[0].fields_numpy(), O)
    assert e <= 1e-10, (cases[0].name, e)
    p = b.plan
    p.tile[0][0], p.tile[0][1] = 64, 4
    with pytest.raises(lbm.LBMError) as err:
        lbm.lbm_batch_set_plan(b.b, p)
    assert err.value.code == lbm.LBM_EINVAL
    plan = b.autotune(trial_steps=4)
    assert all(tuple(t) == (32, 8) for t in plan["tile"]), plan
    b.close()
    for s in solvers:
        s.close()


def stageable_batch():
    """FP16-storage cases whose nx are multiples of 8 (every size class of a 32x8 group
    can be staged), with walls, outflow, periodic sides and ragged tiles."""
    return [W.sessile_cap(48, 40, 14.0, theta=70.0, ste=0.2, T_wall=-1.5),
            W.film(nx=16, ny=64, h0=32.0),
            W.periodic_drop(n=40, R=9.0, ny=29),
            W.sessile_cap(72, 44, 16.0, theta=120.0, ste=0.08, T_wall=-0.7),
            W.sessile_cap(136, 33, 12.0, theta=95.0, ste=0.4, T_wall=-2.0)]


@pytest.mark.parametrize("prec", ["fp16s", "bf16s"])
def test_staged_batch_equals_per_step_and_single_runs(lbm, prec):
    cases = stageable_batch()
    ref = singles(lbm, cases, 31, prec)      # single handles: the staged step by default
    out = {}
    for mode in ("per_step", "staged"):
        solvers = [lbm.Solver(c, precision=prec).set_fields() for c in cases]
        b = lbm.Batch(solvers).set_plan(mode=mode, tiles=[(32, 8)] * lbm.BATCH_CLASSES)
        b.step(10).step(10)                  # the second call replays the captured graph
        solvers[1].step(1)                   # a member stepped on its own between calls
        b.step(11).sync()
        plan = b.plan.as_dict()
        assert plan["mode"] == mode and plan["graph"], plan
        out[mode] = [s.fields_numpy() for s in solvers]
        steps = [s.steps for s in solvers]
        assert steps == [31, 32, 31, 31, 31], steps
        b.close()
        for s in solvers:
            s.close()
    # another instantiation may fuse a different FP32 multiply-add, and a 16-bit store
    # then moves by one unit of the format (the bound of the per-step form's test)
    for k, (A, B_) in enumerate(zip(out["per_step"], out["staged"])):
        e = max_err(A, B_)
        print(cases[k].name, "staged vs per-step", e)
        assert e <= 2e-2, (cases[k].name, e)
    for k in (0, 2, 3, 4):                   # the members stepped by the batch only
        e = max_err(out["staged"][k], ref[k])
        print(cases[k].name, "staged batch vs single", e)
        assert e <= 2e-2, (cases[k].name, e)


def test_staged_batch_n3(lbm):
    # N = 3 cases in the staged form (three blocks per SM): against the per-step form and
    # the single runs, within one unit of the 16-bit format like the N = 2 batch
    cases = [W.liquid_lens(nx=64, ny=48, R=10.0), W.compound_drop(n=128, R_core=12.0, R_shell=24.0),
             W.compound_drop(n=96, R_core=10.0, R_shell=20.0, ny=72)]
    ref = singles(lbm, cases, 30, "fp16s")
    out = {}
    for mode in ("per_step", "staged"):
        solvers = [lbm.Solver(c, precision="fp16s").set_fields() for c in cases]
        b = lbm.Batch(solvers).set_plan(mode=mode, tiles=[(32, 8)] * lbm.BATCH_CLASSES)
        b.step(15).step(15).sync()
        assert b.plan.as_dict()["mode"] == mode
        out[mode] = [s.fields_numpy() for s in solvers]
        b.close()
        for s in solvers:
            s.close()
    for k, c in enumerate(cases):
        e1 = max_err(out["per_step"][k], out["staged"][k])
        e2 = max_err(out["staged"][k], ref[k])
        print(c.name, "staged vs per-step", e1, "vs single", e2)
        assert e1 <= 2e-2 and e2 <= 2e-2, (c.name, e1, e2)


def test_staged_batch_autotune_and_fallback(lbm):
    # the autotuner considers the staged form where a group allows it; a 32x8 group with
    # a case whose nx is not a multiple of 8 runs the per-step form in the staged mode
    cases = stageable_batch()
    solvers = [lbm.Solver(c, precision="fp16s").set_fields() for c in cases]
    b = lbm.Batch(solvers)
    plan = b.autotune(trial_steps=4)
    print("autotuned plan", plan)
    assert plan["mode"] in ("persistent", "per_step", "staged")
    b.close()
    for s in solvers:
        s.close()
    mixed = cases[:2] + [W.periodic_drop(n=37, R=9.0, ny=29)]
    ref = singles(lbm, mixed, 12, "fp16s")
    solvers = [lbm.Solver(c, precision="fp16s").set_fields() for c in mixed]
    b = lbm.Batch(solvers).set_plan(mode="staged", tiles=[(32, 8)] * lbm.BATCH_CLASSES)
    b.step(12).sync()
    for s, c, R in zip(solvers, mixed, ref):
        e = max_err(s.fields_numpy(), R)
        assert e <= 2e-2, (c.name, e)
    b.close()
    for s in solvers:
        s.close()


def test_batch_rejects_mixed_members(lbm):
    a = lbm.Solver(W.small_batch()[0]).set_fields()
    c = lbm.Solver(W.small_batch()[1], precision="fp32").set_fields()
    d = lbm.Solver(W.periodic_drop(n=20, R=5.0, N=3))
    with pytest.raises(lbm.LBMError) as e:
        lbm.Batch([a, c])
    assert e.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LBMError) as e:
        lbm.Batch([a, a])
    assert e.value.code == lbm.LBM_EINVAL
    with pytest.raises(lbm.LBMError) as e:
        lbm.Batch([d])
    assert e.value.code == lbm.LBM_ESTATE
    b = lbm.Batch([a])
    p = b.plan
    p.tile[0][0], p.tile[0][1] = 8, 8
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_batch_set_plan(b.b, p)
    assert e.value.code == lbm.LBM_EINVAL
    b.close()
    for s in (a, c, d):
        s.close()


def test_batch_sweep_full_run(lbm):
    # the 256-drop sweep (sides 128-512, seed 4) for its 10 000 steps in FP16 storage,
    # one autotuned batch: every case stays finite with a bounded velocity
    cases = W.batch_sweep()
    solvers = [lbm.Solver(c, precision="fp16s").set_fields() for c in cases]
    b = lbm.Batch(solvers)
    b.autotune(trial_steps=10)
    b.step(10000 - solvers[0].steps)
    b.sync()
    umax = []
    for s in solvers:
        assert s.steps == 10000
        assert s.diagnostics()["nonfinite"] == 0, s.case.name
        F = s.fields_numpy()
        umax.append(float(np.hypot(F["ux"], F["uy"]).max()))
    b.close()
    for s in solvers:
        s.close()
    print("sweep 10000 steps: peak |u| median", float(np.median(umax)), "max", max(umax))
    assert max(umax) < 0.05
