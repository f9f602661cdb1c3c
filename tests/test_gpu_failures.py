"""Failure detection on the GPU, in host-safe forms: no device fault, trap or unbounded
wait is ever provoked.

* A non-finite population written on the host into a saved state (lbm_save_state /
  lbm_load_state) must make lbm_step with diag_every = 1 return LBM_EUNSTABLE, and the
  handle must stay usable: new fields, and the next steps are finite again.
* The persistent batch's grid-barrier wait, bounded to a single poll
  (lbm_batch_set_wait_limit), must give up, and lbm_batch_sync must report LBM_ETIMEOUT.
  Every wait of the launch is bounded, so the kernel ends in any case.  After the default
  bound is restored and the cases get new fields, a normal call must again equal the same
  cases stepped alone.
"""
import struct

import numpy as np
import pytest

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


@pytest.mark.parametrize("precision,fmt", [("fp64", "<d"), ("fp32", "<f"), ("fp16s", "<f")])
def test_nonfinite_state_is_reported_unstable(lbm, precision, fmt):
    case = W.sessile_drop(n=64, R=16.0, theta=70.0, ny=48)
    s = lbm.Solver(case, precision=precision, diag_every=1).set_fields()
    s.step(3)  # a healthy state passes the check every step
    assert s.diagnostics()["nonfinite"] == 0
    blob = bytearray(s.save_state())
    # layout: step counter (8 bytes), then the rest block of the populations, whose
    # first plane is f_0 ([ny][nx], FP64 for fp64, FP32 for the other two policies)
    cell = 20 * case.nx + 31
    size = struct.calcsize(fmt)
    off = 8 + size * cell
    blob[off:off + size] = struct.pack(fmt, float("nan"))
    s.load_state(bytes(blob))
    with pytest.raises(lbm.LBMError) as e:
        s.step(1)
    assert e.value.code == lbm.LBM_EUNSTABLE
    assert "non-finite" in str(e.value)
    assert s.diagnostics()["nonfinite"] >= 1
    # the handle stays usable
    s.set_fields()
    s.step(5)
    d = s.diagnostics()
    assert d["nonfinite"] == 0 and d["steps"] == 5
    s.close()


def test_persistent_barrier_timeout_is_reported(lbm):
    cases = W.small_batch()
    solvers = [lbm.Solver(c).set_fields() for c in cases]
    b = lbm.Batch(solvers).set_plan(mode="persistent")
    b.set_wait_limit(1)
    b.step(200)
    with pytest.raises(lbm.LBMError) as e:
        b.sync()
    assert e.value.code == lbm.LBM_ETIMEOUT
    # the barrier is reset by the failing sync; the default bound and fresh fields give
    # a normal call again, equal to the cases stepped alone
    b.set_wait_limit(0)
    for s in solvers:
        s.set_fields()
    steps = 30
    b.step(steps).sync()
    for s, c in zip(solvers, cases):
        r = lbm.Solver(c).set_fields()
        r.step(steps)
        R = r.fields_numpy()
        r.close()
        G = s.fields_numpy()
        err = max(float(np.abs(G[k] - R[k]).max()) for k in FIELDS)
        assert err <= 1e-12, (c.name, err)
    b.close()
    for s in solvers:
        s.close()


def test_wait_limit_rejects_negative(lbm):
    cases = W.small_batch()[:1]
    s = lbm.Solver(cases[0]).set_fields()
    b = lbm.Batch([s])
    with pytest.raises(lbm.LBMError) as e:
        b.set_wait_limit(-1)
    assert e.value.code == lbm.LBM_EINVAL
    b.close()
    s.close()
