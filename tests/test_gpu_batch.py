"""Batches of independent cases (lbm_batch_*): the batch launches run the per-cell step
of lbm_step, so every case of a batch must match the same case stepped alone (FP64: to
rounding, since the batch kernels are other instantiations of the same source), and
one case through the batch must match the CPU oracle to the 1e-10 parity bar.  Both
launch forms, all three tile shapes, odd step counts in both forms (each call is replayed
as a captured graph; the persistent launch flips its own parity, the per-step form ends an
odd call with a parity-flip kernel), members stepped alone between batch steps, and the
autotuner's restoration of the state are covered."""
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


@pytest.mark.parametrize("mode", ["persistent", "per_step"])
def test_batch_odd_calls_graph_replay_and_member_steps(lbm, mode):
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
    if mode == "per_step":
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
