"""Gradients through the hand-written adjoint of the FP64 step (lbm_adjoint_fl_loss),
for the loss L = sum_x (phi_pcm f_l - f_target)^2 of the freezing pool with impurities
(N = 4), where phi_pcm f_l is the liquid fraction of the phase-changing material.
The parameters are the bottom wall temperature, the Stefan number and lambda_s / lambda_l
of the freezing liquid.  The gradient is checked three ways:
- against central finite differences of the GPU forward runs (1e-4 relative);
- against central differences of the CPU oracle's loss (the oracle-driven reference
  gradient);
- for independence of the checkpoint interval.
The torch.autograd.Function passes it through."""
import numpy as np
import pytest

import oracle
from paper_2603_22902_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# Generic parameter values: with round ones (T_0 = 0.5, T_wall = -1, T_m = 0) cells of
# the wall rows land exactly on a kink of eq. H at some step, where the loss has only
# one-sided derivatives (the adjoint then mixes them, and central differences straddle
# the kink).  Away from kinks the loss is smooth and the adjoint is its derivative.
THETA = {"T_wall": -1.0137, "ste": 0.2071, "lam_ratio": 1.043}
# Central differences at three step sizes, of which the median is taken: a step that
# straddles one of the loss's kinks (a cell crossing a branch of eq. H in between) is an
# outlier, and the three rarely all straddle one.
STEPS = {"T_wall": (1e-4, 3e-5, 1e-5), "ste": (2e-5, 6e-6, 2e-6), "lam_ratio": (1e-4, 3e-5, 1e-5)}


@pytest.fixture(scope="module")
def lbm():
    import torch
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for the gpu tests")
    from paper_2603_22902_gb300 import build as B
    B.build()
    from paper_2603_22902_gb300 import lbm as L
    return L


def small(**kw):
    args = dict(n=64, n_disks=4, r_range=(5, 7))
    args.update(kw)
    return W.impurity_freeze(**args)


def gpu_loss(case, target, nsteps, lbm):
    from paper_2603_22902_gb300.grad import final_liquid_fraction
    q = final_liquid_fraction(case, nsteps)
    return float(((q - target) ** 2).sum())


def fd_gradient(loss_of, theta):
    g = []
    for k in ("T_wall", "ste", "lam_ratio"):
        est = []
        for h in STEPS[k]:
            tp = dict(theta, **{k: theta[k] + h})
            tm = dict(theta, **{k: theta[k] - h})
            est.append((loss_of(tp) - loss_of(tm)) / (2 * h))
        g.append(float(np.median(est)))
    return np.array(g)


def test_adjoint_against_gpu_finite_differences(lbm):
    from paper_2603_22902_gb300.grad import final_liquid_fraction, run_adjoint, theta_gradient
    nsteps = 300
    target = final_liquid_fraction(small(**dict(THETA, T_wall=-1.3)), nsteps)
    case = small(**THETA)
    g = run_adjoint(case, target, nsteps, checkpoint_every=64)
    ad = theta_gradient(case, g)
    fd = fd_gradient(lambda t: gpu_loss(small(**t), target, nsteps, lbm), THETA)
    print("loss", g.loss, "adjoint", ad, "fd", fd)
    assert abs(g.loss - gpu_loss(case, target, nsteps, lbm)) <= 1e-12 * max(1.0, g.loss)
    # a 64^2 pool: few cells, so the kinks of the loss (one per cell crossing a branch
    # of eq. H at some step) are dense in theta, and central differences carry ~1e-4
    for a, f in zip(ad, fd):
        assert abs(a - f) <= 1e-3 * abs(f) + 1e-10, (ad, fd)


def test_impurity_pool_gradient_full_size(lbm):
    # the pool with 24 impurity disks, 512^2, 4000 steps, checkpoint every 200
    from paper_2603_22902_gb300.grad import final_liquid_fraction, run_adjoint, theta_gradient
    nsteps = 4000
    target = final_liquid_fraction(W.impurity_freeze(**dict(THETA, T_wall=-1.3)), nsteps)
    case = W.impurity_freeze(**THETA)
    g = run_adjoint(case, target, nsteps, checkpoint_every=200)
    ad = theta_gradient(case, g)
    fd = fd_gradient(lambda t: gpu_loss(W.impurity_freeze(**t), target, nsteps, lbm), THETA)
    print("512^2 loss", g.loss, "adjoint", ad, "fd", fd, "rel", np.abs(ad - fd) / np.abs(fd))
    for a, f in zip(ad, fd):
        assert abs(a - f) <= 1e-4 * abs(f), (ad, fd)


def test_adjoint_against_oracle_gradient(lbm):
    from paper_2603_22902_gb300.grad import run_adjoint, theta_gradient
    build = lambda **t: W.impurity_freeze(n=32, n_disks=2, r_range=(4, 5), **t)
    nsteps = 60
    from paper_2603_22902_gb300.grad import pcm_liquid_fraction
    tcase = build(**dict(THETA, T_wall=-1.3))
    target = pcm_liquid_fraction(tcase, oracle.Oracle(tcase).step(nsteps).fields())
    case = build(**THETA)
    g = run_adjoint(case, target, nsteps, checkpoint_every=16)
    ad = theta_gradient(case, g)

    def oracle_loss(t):
        c = build(**t)
        q = pcm_liquid_fraction(c, oracle.Oracle(c).step(nsteps).fields())
        return float(((q - target) ** 2).sum())

    ref = fd_gradient(oracle_loss, THETA)
    print("adjoint", ad, "oracle fd", ref)
    assert abs(g.loss - oracle_loss(THETA)) <= 1e-10 * max(1.0, g.loss)
    for a, f in zip(ad, ref):
        assert abs(a - f) <= 1e-4 * abs(f) + 1e-10, (ad, ref)


def test_checkpoint_interval_does_not_change_the_gradient(lbm):
    from paper_2603_22902_gb300.grad import final_liquid_fraction, run_adjoint
    nsteps = 37
    case = small(n=40, n_disks=2, r_range=(4, 5), **THETA)
    target = final_liquid_fraction(small(n=40, n_disks=2, r_range=(4, 5), **dict(THETA, T_wall=-1.3)), nsteps)
    ref = None
    for K in (1, 6, 37, 100):
        g = run_adjoint(case, target, nsteps, checkpoint_every=K)
        v = [g.loss] + list(g.T_wall) + list(g.rhoL) + list(g.lambda_s) + list(g.lambda_l)
        if ref is None:
            ref = v
        assert v == ref, K


def test_autograd_function(lbm):
    import torch
    from paper_2603_22902_gb300.grad import FreezeLoss, final_liquid_fraction, run_adjoint, theta_gradient
    nsteps = 80
    build = lambda **t: small(n=48, n_disks=3, r_range=(4, 6), **t)
    target = final_liquid_fraction(build(**dict(THETA, T_wall=-1.3)), nsteps)
    theta = torch.tensor([THETA["T_wall"], THETA["ste"], THETA["lam_ratio"]], dtype=torch.float64,
                         requires_grad=True)
    loss = FreezeLoss().apply(theta, build, target, nsteps, 20)
    (2.0 * loss).backward()
    case = build(**THETA)
    g = run_adjoint(case, target, nsteps, 20)
    assert float(loss.detach()) == g.loss
    assert np.allclose(theta.grad.numpy(), 2.0 * theta_gradient(case, g), rtol=0, atol=0)


def test_adjoint_rejects_other_precisions(lbm):
    case = small(n=24, n_disks=1, r_range=(3, 4), **THETA)
    s = lbm.Solver(case, precision="fp32")
    z = np.zeros((case.ny, case.nx))
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_adjoint_fl_loss(s.h, np.ascontiguousarray(case.phi), z, None, None, z, None, lbm.LBM_HOST, 5, 2)
    assert e.value.code == lbm.LBM_EINVAL
    s.close()
