"""The y-slab decomposition on one GPU: a lattice cut into bands of rows (one slab
handle per band, lbm_slab_*), exchanging the halo messages device to device after every
step, must step exactly like the single handle on the whole lattice.  Every cell is
computed by the same kernel from the same inputs, so the bands' own rows must equal the
single run to 1e-12 (bit for bit in practice), on walls, outflow and periodic y sides,
N = 2, 3, 4, FP64, double words and FP16 storage; the bands' diagnostics sums, combined,
must equal the single handle's diagnostics; one run is checked against the CPU oracle
to the parity bar; and two processes, one band each on the same GPU, exchanging their
messages through torch.distributed (gloo, host buffers) as ranks of a multi-GPU run do
(NCCL, device buffers), step exactly like the single handle too.  The overlapped
schedule (each step split into inner and edge tile rows, the exchange on a second stream
between them) must equal the plain one bit for bit."""
import os
import socket

import numpy as np
import pytest

import oracle
from paper_2603_22902_gb300 import workloads as W
from paper_2603_22902_gb300.slab import LocalExchange, split_rows

pytestmark = pytest.mark.gpu

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


def quad_case():
    q = W.periodic_drop(n=40, R=9.0, N=4, rho_gas=0.5, sigma=1e-3, ny=36)
    q.phi[2] = 0.3 * q.phi[1]
    q.phi[3] = 0.2 * q.phi[1]
    q.phi[1] = 0.5 * q.phi[1]
    q.phases[2]["latent"] = 4.0
    q.phases[2]["rho_s"] = 0.9
    q.bc = (W.PERIODIC, W.PERIODIC, W.WALL, W.WALL)
    q.tbc = (W.ADIABATIC, W.ADIABATIC, W.DIRICHLET, W.ADIABATIC)
    q.T_wall = (0.0, 0.0, -0.5, 0.0)
    q.T = np.full((q.ny, q.nx), 0.2)
    return W.perturbed(q, seed=4, amp_u=5e-4)


CASES = {
    "sessile_walls_2": (lambda: W.sessile_drop(n=96, R=28.0, ny=80, theta=70.0), [(0, 37), (37, 80)]),
    "periodic_drop_3": (lambda: W.perturbed(W.periodic_drop(n=64, R=14.0, ny=52, rho_gas=0.2, sigma=2e-3), seed=1),
                        None),
    "compound_walls_3": (lambda: W.compound_drop(n=64, R_core=10.0, R_shell=20.0, ny=60, noise=1e-3), None),
    "film_outflow_2": (lambda: W.film(nx=16, ny=128, h0=64.0), None),
    "N4_walls_4": (quad_case, [(0, 5), (5, 17), (17, 30), (30, 36)]),
}


def run_bands(L, case, bands, steps, precision="fp64", overlap=False):
    import torch
    solvers = [L.SlabSolver(case, y0, y1, precision=precision).set_fields() for y0, y1 in bands]
    ex = LocalExchange(solvers, case.bc[2] == W.PERIODIC,
                       alloc=lambda n: torch.empty(n, dtype=torch.uint8, device="cuda"))
    if overlap:
        # the exchange on a second stream, between the inner and the edge part of each step
        ex.step(steps, overlap=True, streams=(torch.cuda.current_stream(), torch.cuda.Stream()))
    else:
        ex.step(steps)
    parts = [s.own(s.fields_numpy()) for s in solvers]
    F = {k: np.concatenate([P[k] for P in parts], axis=-2) for k in FIELDS}
    sums = ex.sums(case.N)
    for s in solvers:
        s.close()
    return F, sums


@pytest.mark.parametrize("name", list(CASES))
@pytest.mark.parametrize("precision", ["fp64", "df64", "fp16s"])
def test_bands_equal_the_single_lattice(lbm, name, precision):
    maker, bands = CASES[name]
    case = maker()
    bands = bands or split_rows(case.ny, int(name[-1]))
    steps = 200
    s = lbm.Solver(case, precision=precision).set_fields()
    s.step(steps)
    R = s.fields_numpy()
    d = s.diagnostics()
    s.close()
    F, sums = run_bands(lbm, case, bands, steps, precision)
    errs = {k: float(np.abs(F[k] - R[k]).max()) for k in FIELDS}
    print(name, precision, bands, errs)
    assert all(v <= 1e-12 for v in errs.values()), errs
    for p in range(case.N):
        assert abs(sums["mass"][p] - d["mass"][p]) <= 1e-12 * max(1.0, abs(d["mass"][p]))
        assert abs(sums["solid"][p] - d["solid"][p]) <= 1e-12 * max(1.0, abs(d["solid"][p]))
    assert abs(sums["max_sum_dev"] - d["max_sum_dev"]) <= 1e-13
    assert sums["nonfinite"] == 0 == d["nonfinite"]


def test_bands_match_the_oracle(lbm):
    case = W.compound_drop(n=44, R_core=8.0, R_shell=15.0, ny=36, noise=1e-3, mobility=0.02)
    F, _ = run_bands(lbm, case, [(0, 12), (12, 36)], 500)
    O = oracle.Oracle(case).step(500).fields()
    for k in FIELDS:
        scale = max(1.0, float(np.abs(O[k]).max())) if k == "H" else 1.0
        assert float(np.abs(F[k] - O[k]).max()) / scale <= 1e-10, k


def test_slab_arguments(lbm):
    import torch
    L = lbm
    case = W.sessile_drop(n=32, R=8.0, ny=24)
    grid, phases, th, bc, num = L.make_structs(case)
    with pytest.raises(L.LBMError) as e:
        L.lbm_slab_create(grid, 0, 24, case.N, phases, th, bc, num)   # no cut: use lbm_create
    assert e.value.code == L.LBM_EINVAL
    with pytest.raises(L.LBMError):
        L.lbm_slab_create(grid, 10, 30, case.N, phases, th, bc, num)  # beyond ny
    s = L.SlabSolver(case, 0, 12).set_fields()
    assert (s.ny_local, s.ghost_below, s.ghost_above) == (13, 0, 1)
    msg = torch.empty(s.msg_bytes[2], dtype=torch.uint8, device="cuda")
    with pytest.raises(L.LBMError) as e:
        s.pack(2, 1, msg)                       # y-min is the global wall, not a cut
    assert e.value.code == L.LBM_EINVAL
    with pytest.raises(L.LBMError) as e:
        s.pack(3, 3, msg)                       # phases are 1 and 2
    assert e.value.code == L.LBM_EINVAL
    s.close()


def _rank_worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch
    import torch.distributed as dist
    from paper_2603_22902_gb300 import lbm as L
    from paper_2603_22902_gb300.slab import DistExchange
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    case = W.compound_drop(n=48, R_core=8.0, R_shell=15.0, ny=40, noise=1e-3, mobility=0.02)
    y0, y1 = split_rows(case.ny, world)[rank]
    band = L.SlabSolver(case, y0, y1).set_fields()
    ex = DistExchange(band, case.bc[2] == W.PERIODIC,
                      alloc=lambda n: torch.empty(n, dtype=torch.uint8, device="cuda"),
                      host_alloc=lambda n: torch.empty(n, dtype=torch.uint8))
    ex.step(150)
    F = band.own(band.fields_numpy())
    sums = ex.sums(case.N)
    band.close()
    dist.destroy_process_group()
    q.put((rank, F, sums))


def test_bands_on_two_ranks_equal_the_single_lattice(lbm):
    import torch.multiprocessing as mp
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        r, F, sums = q.get(timeout=300)
        out[r] = (F, sums)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    case = W.compound_drop(n=48, R_core=8.0, R_shell=15.0, ny=40, noise=1e-3, mobility=0.02)
    s = lbm.Solver(case).set_fields()
    s.step(150)
    R = s.fields_numpy()
    d = s.diagnostics()
    s.close()
    F = {k: np.concatenate([out[0][0][k], out[1][0][k]], axis=-2) for k in FIELDS}
    errs = {k: float(np.abs(F[k] - R[k]).max()) for k in FIELDS}
    print("two ranks", errs)
    assert all(v <= 1e-12 for v in errs.values()), errs
    for r in (0, 1):
        sums = out[r][1]
        for p in range(case.N):
            assert abs(sums["mass"][p] - d["mass"][p]) <= 1e-12 * max(1.0, d["mass"][p])
        assert sums["nonfinite"] == 0


@pytest.mark.parametrize("name", ["sessile_walls_2", "periodic_drop_3", "compound_walls_3", "N4_walls_4"])
@pytest.mark.parametrize("precision", ["fp64", "fp16s"])
def test_overlapped_schedule_equals_plain(lbm, name, precision):
    # every step split into its inner tile rows and its edge rows (lbm_slab_step_part),
    # with the previous step's exchange on a second stream between the two: each
    # destination slot is written by one cell either way, so the bands' rows must equal the
    # plain schedule's bit for bit
    maker, bands = CASES[name]
    case = maker()
    bands = bands or split_rows(case.ny, int(name[-1]))
    A, sa = run_bands(lbm, case, bands, 60, precision)
    B, sb = run_bands(lbm, case, bands, 60, precision, overlap=True)
    for k in FIELDS:
        assert np.array_equal(A[k], B[k]), (name, precision, k, float(np.abs(A[k] - B[k]).max()))
    assert sa == sb


def test_step_part_order_is_checked(lbm):
    case = W.sessile_drop(n=96, R=28.0, ny=80, theta=70.0)
    s = lbm.SlabSolver(case, 0, 40).set_fields()
    with pytest.raises(lbm.LBMError) as e:
        s.step_part(lbm.LBM_SLAB_EDGE)          # edge rows before the inner rows
    assert e.value.code == lbm.LBM_ESTATE
    s.step_part(lbm.LBM_SLAB_INNER)
    with pytest.raises(lbm.LBMError) as e:
        s.step_part(lbm.LBM_SLAB_INNER)         # the inner rows twice
    assert e.value.code == lbm.LBM_ESTATE
    with pytest.raises(lbm.LBMError) as e:
        s.step(1)                               # a whole step in between
    assert e.value.code == lbm.LBM_ESTATE
    s.step_part(lbm.LBM_SLAB_EDGE)
    assert s.steps == 1
    with pytest.raises(lbm.LBMError) as e:
        s.step_part(3)
    assert e.value.code == lbm.LBM_EINVAL
    s.close()
    whole = lbm.Solver(case).set_fields()
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_slab_step_part(whole.h, lbm.LBM_SLAB_INNER)   # not a slab handle
    assert e.value.code == lbm.LBM_EINVAL
    whole.close()
