"""C-ABI checks that need no GPU: the library builds for sm_103a, loads, exports every
function declared in include/lbm.h, and rejects invalid parameter sets (validation
runs before any CUDA call)."""
import os
import re

import numpy as np
import pytest

from paper_2603_22902_gb300 import build as B
from paper_2603_22902_gb300 import lbm
from paper_2603_22902_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return lbm.library()


def declared_functions():
    names = []
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            with open(os.path.join(ROOT, "include", fn)) as fh:
                text = fh.read()
            names += re.findall(r"^\s*(?:[A-Za-z_][\w\s\*]*?)\b(lbm_\w+)\s*\(", text, re.M)
    return sorted(set(names))


def test_every_declared_function_is_exported(lib):
    names = declared_functions()
    assert "lbm_create" in names and "lbm_step" in names and len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n


def _create(case, **mods):
    grid, phases, th, bc, num = lbm.make_structs(case)
    for k, v in mods.items():
        obj, field = k.split("__")
        target = {"grid": grid, "th": th, "bc": bc, "num": num, "phase0": phases[0]}[obj]
        if isinstance(v, tuple):
            arr = getattr(target, field)
            arr[v[0]] = v[1]
        else:
            setattr(target, field, v)
    return lbm.lbm_create(grid, case.N, phases, th, bc, num)


@pytest.mark.parametrize("mods", [
    dict(grid__nx=2),
    dict(grid__ny=2),
    dict(grid__nx=65536, grid__ny=40000),   # more than 2^31 cells
    dict(num__eps=0.0),
    dict(num__mobility=-1.0),
    dict(num__precision=7),
    dict(phase0__mu_l=0.0),
    dict(phase0__lambda_s=0.0),
    dict(phase0__rho_l=-1.0),
    dict(th__T_sol=1.0, th__T_liq=0.0),
    dict(bc__kind=(0, 1)),           # x-min wall, x-max periodic: unpaired
    dict(bc__kind=(0, 2)),           # outflow on an x side
    dict(bc__tkind=(3, 1)),          # Dirichlet on an outflow side (film top)
])
def test_invalid_parameters_rejected(lib, mods):
    case = W.film(nx=8, ny=16)
    with pytest.raises(lbm.LBMError) as e:
        _create(case, **mods)
    assert e.value.code == lbm.LBM_EINVAL


@pytest.mark.parametrize("N", [1, 5])
def test_phase_count_out_of_range_rejected(lib, N):
    case = W.film(nx=8, ny=16)
    grid, phases, th, bc, num = lbm.make_structs(case)
    phases = (list(phases) * N)[:N]
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_create(grid, N, phases, th, bc, num)
    assert e.value.code == lbm.LBM_EINVAL


def test_asymmetric_sigma_rejected(lib):
    case = W.periodic_drop(n=8, R=2.0, N=3)
    grid, phases, th, bc, num = lbm.make_structs(case)
    num.sigma[0 * lbm.MAXN + 1] = 2e-3
    with pytest.raises(lbm.LBMError) as e:
        lbm.lbm_create(grid, 3, phases, th, bc, num)
    assert e.value.code == lbm.LBM_EINVAL
    assert b"sigma" in lib.lbm_last_error(None)


def test_batch_arguments_rejected_before_any_cuda_call(lib):
    import ctypes
    out = ctypes.c_void_p()
    assert lib.lbm_batch_create(0, None, ctypes.byref(out)) == lbm.LBM_EINVAL
    assert out.value is None
    arr = (ctypes.c_void_p * 2)(None, None)
    assert lib.lbm_batch_create(2, arr, ctypes.byref(out)) == lbm.LBM_EINVAL
    assert b"NULL handle" in lib.lbm_batch_last_error(None)
    assert lib.lbm_batch_step(None, 1) == lbm.LBM_EINVAL
    assert lib.lbm_batch_autotune(None, 1, None) == lbm.LBM_EINVAL


def test_adjoint_arguments_rejected_before_any_cuda_call(lib):
    assert lib.lbm_adjoint_fl_loss(None, None, None, None, None, None, None, 0, 1, 1, None) == lbm.LBM_EINVAL


def test_no_device_fails_loudly(lib):
    # without a CUDA device a valid parameter set is refused with LBM_ECUDA: there is no
    # CPU path behind the C ABI
    import torch
    if torch.cuda.is_available():
        pytest.skip("a CUDA device is present")
    case = W.film(nx=8, ny=16)
    with pytest.raises(lbm.LBMError) as e:
        _create(case)
    assert e.value.code == lbm.LBM_ECUDA


def test_missing_library_fails_loudly(monkeypatch):
    # the binding never falls back to anything when the built library is absent
    monkeypatch.setattr(lbm, "_lib", None)
    monkeypatch.setattr(lbm, "LIB_PATH", os.path.join(ROOT, "no-such-dir", "liblbm_gb300.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        lbm.library()
