"""Thin ctypes binding of the C ABI in ``include/lbm.h`` (argument marshalling only).

Every step of the solver runs in ``liblbm_gb300.so`` (sm_103a CUDA kernels).  There
is no Python or CPU fallback: if the library is missing or no CUDA device is present
the calls raise.  PyTorch is used only for device buffers and the current stream.

The module exposes the C functions under their C names (``lbm_create``,
``lbm_set_fields``, ``lbm_step``, ``lbm_get_fields`` ...) plus ``Solver``, a small
owner object that builds the parameter structures from a ``workloads.Case``.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "liblbm_gb300.so")
# LBM_CHECK_BOUNDS=1 selects the bounds-checked debug build (liblbm_gb300_check.so)
if os.environ.get("LBM_CHECK_BOUNDS") == "1":
    LIB_PATH = os.path.join(HERE, "liblbm_gb300_check.so")

MAXN = 4
LBM_OK, LBM_EINVAL, LBM_ENOMEM, LBM_ECUDA, LBM_EUNSTABLE, LBM_ETIMEOUT, LBM_ESTATE = 0, -1, -2, -3, -4, -5, -6
LBM_BC_PERIODIC, LBM_BC_WALL, LBM_BC_OUTFLOW = 0, 1, 2
LBM_T_ADIABATIC, LBM_T_DIRICHLET = 0, 1
LBM_FP64, LBM_FP32, LBM_FP16S, LBM_BF16S, LBM_DF64 = 0, 1, 2, 3, 4
LBM_HOST, LBM_DEVICE = 0, 1
PRECISIONS = {"fp64": LBM_FP64, "fp32": LBM_FP32, "fp16s": LBM_FP16S, "bf16s": LBM_BF16S, "df64": LBM_DF64}

_D = ctypes.c_double


class lbm_grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int)]


class lbm_phase(ctypes.Structure):
    _fields_ = [(n, _D) for n in ("rho_l", "rho_s", "mu_l", "mu_s", "lambda_l", "lambda_s", "cp_l", "cp_s", "latent")]


class lbm_thermal(ctypes.Structure):
    _fields_ = [("T_sol", _D), ("T_liq", _D), ("rho_ref", _D), ("cp_ref", _D),
                ("u_solid", _D * 2), ("accel", _D * 2)]


class lbm_bc(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int * 4), ("tkind", ctypes.c_int * 4), ("T_wall", _D * 4),
                ("wet_cos", (_D * (MAXN * MAXN)) * 4)]


class lbm_numerics(ctypes.Structure):
    _fields_ = [("eps", _D), ("mobility", _D), ("sigma", _D * (MAXN * MAXN)),
                ("precision", ctypes.c_int), ("diag_every", ctypes.c_int)]


class lbm_diag(ctypes.Structure):
    _fields_ = [("mass", _D * MAXN), ("solid", _D * MAXN), ("max_sum_dev", _D),
                ("nonfinite", ctypes.c_longlong), ("steps", ctypes.c_longlong)]


LBM_BATCH_PERSISTENT, LBM_BATCH_PER_STEP, LBM_BATCH_STAGED = 0, 1, 2
_BATCH_MODES = {"persistent": LBM_BATCH_PERSISTENT, "per_step": LBM_BATCH_PER_STEP, "staged": LBM_BATCH_STAGED}
BATCH_CLASSES = 4


class lbm_batch_plan(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int), ("blocks_per_sm", ctypes.c_int),
                ("tile", (ctypes.c_int * 2) * BATCH_CLASSES), ("graph", ctypes.c_int)]

    def as_dict(self):
        return {"mode": {v: k for k, v in _BATCH_MODES.items()}.get(self.mode, self.mode),
                "blocks_per_sm": self.blocks_per_sm, "tile": [tuple(t) for t in self.tile],
                "graph": bool(self.graph)}


class lbm_fl_grad(ctypes.Structure):
    _fields_ = [("loss", _D), ("T_wall", _D * 4), ("rhoL", _D * MAXN), ("lambda_s", _D * MAXN),
                ("lambda_l", _D * MAXN)]


_lib = None
_lock = threading.Lock()
_VP = ctypes.c_void_p


def library():
    """Load liblbm_gb300.so; raises if it has not been built."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(LIB_PATH):
                raise RuntimeError(
                    f"{LIB_PATH} is missing: build it with paper_2603_22902_gb300.build.build() "
                    "(nvcc, sm_103a); there is no CPU fallback")
            lib = ctypes.CDLL(LIB_PATH)
            P = ctypes.POINTER
            lib.lbm_create.argtypes = [P(lbm_grid), ctypes.c_int, P(lbm_phase), P(lbm_thermal), P(lbm_bc),
                                       P(lbm_numerics), P(_VP)]
            lib.lbm_set_stream.argtypes = [_VP, _VP]
            lib.lbm_set_fields.argtypes = [_VP, _VP, _VP, _VP, _VP, ctypes.c_int]
            lib.lbm_step.argtypes = [_VP, ctypes.c_long]
            lib.lbm_get_fields.argtypes = [_VP] + [_VP] * 7 + [ctypes.c_int]
            lib.lbm_get_diagnostics.argtypes = [_VP, P(lbm_diag)]
            lib.lbm_save_state.argtypes = [_VP, _VP, P(ctypes.c_size_t)]
            lib.lbm_load_state.argtypes = [_VP, _VP, ctypes.c_size_t]
            lib.lbm_get_steps.argtypes = [_VP]
            lib.lbm_get_steps.restype = ctypes.c_longlong
            lib.lbm_set_tile.argtypes = [_VP, ctypes.c_int, ctypes.c_int]
            lib.lbm_set_staging.argtypes = [_VP, ctypes.c_int]
            lib.lbm_debug_bounds.argtypes = [_VP, ctypes.POINTER(ctypes.c_longlong)]
            lib.lbm_debug_bounds.restype = ctypes.c_int
            lib.lbm_last_error.argtypes = [_VP]
            lib.lbm_last_error.restype = ctypes.c_char_p
            lib.lbm_destroy.argtypes = [_VP]
            lib.lbm_adjoint_fl_loss.argtypes = [_VP] + [_VP] * 6 + [ctypes.c_int, ctypes.c_long, ctypes.c_int,
                                                                     P(lbm_fl_grad)]
            lib.lbm_slab_create.argtypes = [P(lbm_grid), ctypes.c_int, ctypes.c_int, ctypes.c_int, P(lbm_phase),
                                            P(lbm_thermal), P(lbm_bc), P(lbm_numerics), P(_VP)]
            lib.lbm_slab_geometry.argtypes = [_VP, P(ctypes.c_int)]
            lib.lbm_slab_message_bytes.argtypes = [_VP, ctypes.c_int]
            lib.lbm_slab_message_bytes.restype = ctypes.c_longlong
            lib.lbm_slab_pack.argtypes = [_VP, ctypes.c_int, ctypes.c_int, _VP]
            lib.lbm_slab_unpack.argtypes = [_VP, ctypes.c_int, ctypes.c_int, _VP]
            lib.lbm_slab_sums.argtypes = [_VP, P(_D)]
            lib.lbm_slab_step_part.argtypes = [_VP, ctypes.c_int]
            lib.lbm_measure_fp64_rate.argtypes = [P(_D), P(_D)]
            lib.lbm_batch_create.argtypes = [ctypes.c_int, P(_VP), P(_VP)]
            lib.lbm_batch_set_stream.argtypes = [_VP, _VP]
            lib.lbm_batch_set_plan.argtypes = [_VP, P(lbm_batch_plan)]
            lib.lbm_batch_get_plan.argtypes = [_VP, P(lbm_batch_plan)]
            lib.lbm_batch_step.argtypes = [_VP, ctypes.c_long]
            lib.lbm_batch_sync.argtypes = [_VP]
            lib.lbm_batch_set_wait_limit.argtypes = [_VP, ctypes.c_longlong]
            lib.lbm_batch_autotune.argtypes = [_VP, ctypes.c_int, P(lbm_batch_plan)]
            lib.lbm_batch_last_error.argtypes = [_VP]
            lib.lbm_batch_last_error.restype = ctypes.c_char_p
            lib.lbm_batch_destroy.argtypes = [_VP]
            for name in ("lbm_create", "lbm_set_stream", "lbm_set_fields", "lbm_step", "lbm_get_fields",
                         "lbm_get_diagnostics", "lbm_save_state", "lbm_load_state", "lbm_set_tile", "lbm_set_staging",
                         "lbm_measure_fp64_rate", "lbm_slab_create", "lbm_slab_geometry", "lbm_slab_pack", "lbm_slab_unpack", "lbm_slab_sums", "lbm_slab_step_part",
                         "lbm_batch_create", "lbm_batch_set_stream", "lbm_batch_set_plan", "lbm_batch_get_plan",
                         "lbm_batch_step", "lbm_batch_sync", "lbm_batch_autotune", "lbm_batch_set_wait_limit", "lbm_adjoint_fl_loss"):
                getattr(lib, name).restype = ctypes.c_int
            _lib = lib
    return _lib


class LBMError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (status {code})")
        self.code = code


def _check(rc, h=None):
    if rc != LBM_OK:
        msg = library().lbm_last_error(h).decode(errors="replace")
        raise LBMError(rc, msg)
    return rc


def _ptr(a):
    """Device pointer of a torch tensor, host pointer of a numpy array, or None."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.dtype == np.float64 and a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


# ---- C functions under their C names --------------------------------------

def lbm_create(grid, N, phases, thermal, bc, numerics):
    h = _VP()
    arr = (lbm_phase * N)(*phases)
    _check(library().lbm_create(ctypes.byref(grid), N, arr, ctypes.byref(thermal), ctypes.byref(bc),
                                ctypes.byref(numerics), ctypes.byref(h)))
    return h


def lbm_slab_create(grid, y0, y1, N, phases, thermal, bc, numerics):
    h = _VP()
    arr = (lbm_phase * N)(*phases)
    _check(library().lbm_slab_create(ctypes.byref(grid), int(y0), int(y1), N, arr, ctypes.byref(thermal),
                                     ctypes.byref(bc), ctypes.byref(numerics), ctypes.byref(h)))
    return h


def lbm_slab_geometry(h):
    out = (ctypes.c_int * 4)()
    _check(library().lbm_slab_geometry(h, out), h)
    return tuple(out)


def lbm_slab_message_bytes(h, phase):
    return int(library().lbm_slab_message_bytes(h, int(phase)))


def lbm_slab_pack(h, side, phase, msg):
    return _check(library().lbm_slab_pack(h, int(side), int(phase), _ptr(msg)), h)


def lbm_slab_unpack(h, side, phase, msg):
    return _check(library().lbm_slab_unpack(h, int(side), int(phase), _ptr(msg)), h)


LBM_SLAB_INNER, LBM_SLAB_EDGE = 1, 2


def lbm_slab_step_part(h, part):
    return _check(library().lbm_slab_step_part(h, int(part)), h)


def lbm_slab_sums(h, N):
    out = (_D * (2 * N + 2))()
    _check(library().lbm_slab_sums(h, out), h)
    v = list(out)
    return dict(mass=v[:N], solid=v[N:2 * N], max_sum_dev=v[2 * N], nonfinite=int(v[2 * N + 1]))


def lbm_measure_fp64_rate():
    """(G FP64 thread-instructions per second, best launch ms) of the current device."""
    r, ms = _D(), _D()
    _check(library().lbm_measure_fp64_rate(ctypes.byref(r), ctypes.byref(ms)))
    return r.value, ms.value


def lbm_set_stream(h, stream_ptr):
    return _check(library().lbm_set_stream(h, stream_ptr), h)


def lbm_set_fields(h, phi, T, ux, uy, where):
    return _check(library().lbm_set_fields(h, _ptr(phi), _ptr(T), _ptr(ux), _ptr(uy), where), h)


def lbm_step(h, nsteps):
    return _check(library().lbm_step(h, int(nsteps)), h)


def lbm_get_fields(h, phi, T, H, fl, ux, uy, p, where):
    return _check(library().lbm_get_fields(h, *[_ptr(a) for a in (phi, T, H, fl, ux, uy, p)], where), h)


def lbm_get_diagnostics(h, N):
    d = lbm_diag()
    _check(library().lbm_get_diagnostics(h, ctypes.byref(d)), h)
    return dict(mass=list(d.mass[:N]), solid=list(d.solid[:N]), max_sum_dev=d.max_sum_dev,
                nonfinite=int(d.nonfinite), steps=int(d.steps))


def lbm_save_state(h) -> bytes:
    n = ctypes.c_size_t(0)
    _check(library().lbm_save_state(h, None, ctypes.byref(n)), h)
    buf = ctypes.create_string_buffer(n.value)
    _check(library().lbm_save_state(h, buf, ctypes.byref(n)), h)
    return buf.raw


def lbm_load_state(h, data: bytes):
    buf = ctypes.create_string_buffer(data, len(data))
    return _check(library().lbm_load_state(h, buf, len(data)), h)


def lbm_get_steps(h) -> int:
    return int(library().lbm_get_steps(h))


def lbm_set_tile(h, bx, by):
    return _check(library().lbm_set_tile(h, bx, by), h)


def lbm_set_staging(h, mode):
    return _check(library().lbm_set_staging(h, int(mode)), h)


def lbm_debug_bounds(h):
    out = (ctypes.c_longlong * 3)()
    _check(library().lbm_debug_bounds(h, out), h)
    return list(out)


def lbm_destroy(h):
    library().lbm_destroy(h)


def lbm_adjoint_fl_loss(h, phi0, T0, ux0, uy0, fl_target, weight, where, nsteps, checkpoint_every):
    g = lbm_fl_grad()
    _check(library().lbm_adjoint_fl_loss(h, *[_ptr(a) for a in (phi0, T0, ux0, uy0, fl_target, weight)], where,
                                         int(nsteps), int(checkpoint_every), ctypes.byref(g)), h)
    return g


def _bcheck(rc, b=None):
    if rc != LBM_OK:
        msg = library().lbm_batch_last_error(b).decode(errors="replace")
        raise LBMError(rc, msg)
    return rc


def lbm_batch_create(handles):
    b = _VP()
    arr = (_VP * len(handles))(*[h.value if isinstance(h, _VP) else h for h in handles])
    _bcheck(library().lbm_batch_create(len(handles), arr, ctypes.byref(b)))
    return b


def lbm_batch_set_stream(b, stream_ptr):
    return _bcheck(library().lbm_batch_set_stream(b, stream_ptr), b)


def lbm_batch_set_plan(b, plan):
    return _bcheck(library().lbm_batch_set_plan(b, ctypes.byref(plan)), b)


def lbm_batch_get_plan(b):
    plan = lbm_batch_plan()
    _bcheck(library().lbm_batch_get_plan(b, ctypes.byref(plan)), b)
    return plan


def lbm_batch_step(b, nsteps):
    return _bcheck(library().lbm_batch_step(b, int(nsteps)), b)


def lbm_batch_sync(b):
    return _bcheck(library().lbm_batch_sync(b), b)


def lbm_batch_set_wait_limit(b, polls):
    return _bcheck(library().lbm_batch_set_wait_limit(b, int(polls)), b)


def lbm_batch_autotune(b, trial_steps):
    plan = lbm_batch_plan()
    _bcheck(library().lbm_batch_autotune(b, int(trial_steps), ctypes.byref(plan)), b)
    return plan


def lbm_batch_destroy(b):
    library().lbm_batch_destroy(b)


# ---- parameter structures from a case ---------------------------------------

def make_structs(case, precision="fp64", diag_every=0):
    grid = lbm_grid(case.nx, case.ny)
    phases = [lbm_phase(ph["rho_l"], ph["rho_s"], ph["mu_l"], ph["mu_s"], ph["lam_l"], ph["lam_s"],
                        ph["cp_l"], ph["cp_s"], ph["latent"]) for ph in case.phases]
    th = lbm_thermal()
    th.T_sol, th.T_liq, th.rho_ref, th.cp_ref = case.T_sol, case.T_liq, case.rho_ref, case.cp_ref
    th.u_solid[0], th.u_solid[1] = case.u_solid
    th.accel[0], th.accel[1] = case.accel
    bc = lbm_bc()
    wc = np.asarray(case.wet_cos, dtype=np.float64).reshape(4, case.N, case.N)
    for s in range(4):
        bc.kind[s], bc.tkind[s], bc.T_wall[s] = case.bc[s], case.tbc[s], case.T_wall[s]
        for p in range(case.N):
            for q in range(case.N):
                bc.wet_cos[s][p * MAXN + q] = wc[s, p, q]
    num = lbm_numerics()
    num.eps, num.mobility = case.eps, case.mobility
    sig = np.asarray(case.sigma, dtype=np.float64)
    for p in range(case.N):
        for q in range(case.N):
            num.sigma[p * MAXN + q] = sig[p, q]
    num.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    num.diag_every = diag_every
    return grid, phases, th, bc, num


class Solver:
    """One solver handle on the current CUDA device, fed from a ``workloads.Case``."""

    def __init__(self, case, precision="fp64", diag_every=0, tile=None, stream=None, staged=None):
        import torch
        self.torch = torch
        self.case = case
        self.N, self.nx, self.ny = case.N, case.nx, case.ny
        grid, phases, th, bc, num = make_structs(case, precision, diag_every)
        self.h = lbm_create(grid, case.N, phases, th, bc, num)
        if stream is None:
            stream = torch.cuda.current_stream()
        lbm_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream))
        if tile is not None:
            lbm_set_tile(self.h, *tile)
        if staged is not None:   # None: the library's default (staged where it applies)
            lbm_set_staging(self.h, 1 if staged else 0)

    def set_fields(self, phi=None, T=None, ux=None, uy=None):
        """Initial state from device tensors (default: the case's own fields)."""
        t = self.torch
        dev = t.device("cuda")
        c = self.case
        conv = lambda a: a.to(dev, t.float64).contiguous() if isinstance(a, t.Tensor) else \
            t.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device=dev)
        self._init = [conv(c.phi if phi is None else phi), conv(c.T if T is None else T),
                      conv(c.ux if ux is None else ux), conv(c.uy if uy is None else uy)]
        lbm_set_fields(self.h, *self._init, LBM_DEVICE)
        return self

    def step(self, n=1):
        lbm_step(self.h, n)
        return self

    @property
    def steps(self):
        return lbm_get_steps(self.h)

    def fields(self):
        """phi[N,ny,nx], T, H, fl, ux, uy, p as float64 device tensors (stream-ordered)."""
        t = self.torch
        ny, nx = self.ny, self.nx
        out = {k: t.empty((ny, nx), dtype=t.float64, device="cuda") for k in ("T", "H", "fl", "ux", "uy", "p")}
        out["phi"] = t.empty((self.N, ny, nx), dtype=t.float64, device="cuda")
        lbm_get_fields(self.h, out["phi"], out["T"], out["H"], out["fl"], out["ux"], out["uy"], out["p"], LBM_DEVICE)
        return out

    def fields_numpy(self):
        F = self.fields()
        self.torch.cuda.current_stream().synchronize()
        return {k: v.cpu().numpy() for k, v in F.items()}

    def diagnostics(self):
        return lbm_get_diagnostics(self.h, self.N)

    def save_state(self) -> bytes:
        return lbm_save_state(self.h)

    def load_state(self, data: bytes):
        lbm_load_state(self.h, data)
        return self

    def close(self):
        if getattr(self, "h", None):
            lbm_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SlabSolver(Solver):
    """Rows [y0, y1) of a case's lattice as a slab handle (lbm_slab_create): the band plus
    a ghost row beyond each cut side.  set_fields() takes the case's global fields and
    hands the band's rows (ghost rows included, wrapped on a periodic axis) to the
    library."""

    def __init__(self, case, y0, y1, precision="fp64", tile=None, stream=None):
        import torch
        self.torch = torch
        self.case = case
        self.y0, self.y1 = int(y0), int(y1)
        grid, phases, th, bc, num = make_structs(case, precision, 0)
        self.h = lbm_slab_create(grid, self.y0, self.y1, case.N, phases, th, bc, num)
        self.ny_local, self.ghost_below, self.ghost_above, _ = lbm_slab_geometry(self.h)
        self.N, self.nx, self.ny = case.N, case.nx, self.ny_local
        if stream is None:
            stream = torch.cuda.current_stream()
        lbm_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream))
        if tile is not None:
            lbm_set_tile(self.h, *tile)
        self.rows = np.arange(self.y0 - self.ghost_below, self.y1 + self.ghost_above) % case.ny
        self.msg_bytes = {ph: lbm_slab_message_bytes(self.h, ph) for ph in (1, 2)}

    def set_fields(self, phi=None, T=None, ux=None, uy=None):
        c = self.case
        r = self.rows
        pick = lambda a, g: np.ascontiguousarray((g if a is None else a)[..., r, :])
        return Solver.set_fields(self, pick(phi, c.phi), pick(T, c.T), pick(ux, c.ux), pick(uy, c.uy))

    def own(self, F):
        """The band's own rows of a field dict from fields() / fields_numpy()."""
        lo, hi = self.ghost_below, self.ny_local - self.ghost_above
        return {k: v[..., lo:hi, :] for k, v in F.items()}

    def step_part(self, part):
        """Half of one step: LBM_SLAB_INNER, then LBM_SLAB_EDGE (which completes it)."""
        lbm_slab_step_part(self.h, part)
        return self

    def set_stream(self, stream):
        """Queue the handle's later work on `stream` (a torch.cuda.Stream)."""
        lbm_set_stream(self.h, ctypes.c_void_p(stream.cuda_stream))

    def pack(self, side, phase, msg):
        lbm_slab_pack(self.h, side, phase, msg)

    def unpack(self, side, phase, msg):
        lbm_slab_unpack(self.h, side, phase, msg)

    def sums(self):
        return lbm_slab_sums(self.h, self.N)


class Batch:
    """Independent Solvers advanced together (lbm_batch_*); the Solvers stay usable
    for fields, diagnostics and state I/O and must outlive the batch."""

    def __init__(self, solvers, stream=None):
        import torch
        self.torch = torch
        self.solvers = list(solvers)
        self.b = lbm_batch_create([s.h for s in self.solvers])
        if stream is None:
            stream = torch.cuda.current_stream()
        lbm_batch_set_stream(self.b, ctypes.c_void_p(stream.cuda_stream))

    @property
    def plan(self):
        return lbm_batch_get_plan(self.b)

    def set_plan(self, mode=None, blocks_per_sm=None, tiles=None):
        p = lbm_batch_get_plan(self.b)
        if mode is not None:
            p.mode = _BATCH_MODES.get(mode, mode)
        if blocks_per_sm is not None:
            p.blocks_per_sm = blocks_per_sm
        if tiles is not None:
            for k, (bx, by) in enumerate(tiles):
                p.tile[k][0], p.tile[k][1] = bx, by
        lbm_batch_set_plan(self.b, p)
        return self

    def step(self, n=1):
        lbm_batch_step(self.b, n)
        return self

    def sync(self):
        lbm_batch_sync(self.b)
        return self

    def set_wait_limit(self, polls):
        lbm_batch_set_wait_limit(self.b, polls)
        return self

    def autotune(self, trial_steps=20):
        return lbm_batch_autotune(self.b, trial_steps).as_dict()

    def close(self):
        if getattr(self, "b", None):
            lbm_batch_destroy(self.b)
            self.b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
