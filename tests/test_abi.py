"""The C-ABI library builds for sm_103a, loads, exports every symbol that
include/lbm.h declares, and validates parameters before touching a GPU."""
import ctypes as C
import os
import re

import pytest

from paper_2203_01316_gb300 import build, lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    build.build()
    return lbm.lib()


def _declared():
    txt = open(os.path.join(ROOT, "include", "lbm.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_c_abi_only():
    txt = open(os.path.join(ROOT, "include", "lbm.h")).read()
    assert 'extern "C"' in txt
    for bad in ("torch", "at::", "c10", "std::"):
        assert bad not in re.sub(r"/\*.*?\*/", "", txt, flags=re.S)


def test_every_declared_symbol_is_exported(L):
    declared = _declared()
    assert len(declared) >= 20
    assert sorted(lbm.SYMBOLS) == declared
    for name in declared:
        assert hasattr(L, name), name


def _params(**kw):
    p = lbm.Params()
    p.nx, p.ny, p.nz, p.lat_h, p.hkind, p.storage, p.periodic_x = 8, 8, 8, 27, 0, 0, 1
    p.nu, p.k, p.Pr, p.omega_bulk, p.rho0, p.T_ref = 0.02, 2e-4, 0.0, 1.0, 1.0, 0.0
    for k, v in kw.items():
        setattr(p, k, v)
    return p


@pytest.mark.parametrize("bad", [dict(nx=0), dict(lat_h=19), dict(hkind=7), dict(storage=9), dict(nu=-1.0),
                                 dict(k=0.0, Pr=0.0), dict(k=2e-4, Pr=50.0), dict(omega_bulk=2.5),
                                 dict(nx=2048, ny=2048, nz=32), dict(periodic_x=0, nx=3), dict(wall_bc=3),
                                 dict(inlet_bc=2), dict(step_kernel=5), dict(hkind=4)])
def test_invalid_parameters_rejected_without_gpu(L, bad):
    h = C.c_void_p()
    st = L.lbm_create(C.byref(_params(**bad)), C.byref(h))
    assert st == lbm.LBM_ERR_INVALID
    assert h.value is None
    assert len(L.lbm_last_error(None)) > 0


def test_null_handles_are_rejected(L):
    assert L.lbm_step(None, 1) == lbm.LBM_ERR_INVALID
    assert L.lbm_destroy(None) == lbm.LBM_OK


def test_every_entry_point_rejects_a_null_context_without_gpu(L):
    # every call that takes a context returns LBM_ERR_INVALID for a null one
    # (null pointers and zeros for the other arguments) before any CUDA call
    scalars = (C.c_int, C.c_int64, C.c_double, C.c_size_t)
    checked = 0
    for name in lbm.SYMBOLS:
        if name in ("lbm_create", "lbm_destroy", "lbm_last_error"):
            continue
        fn = getattr(L, name)
        args = [0 if t in scalars else None for t in fn.argtypes]
        assert fn(*args) == lbm.LBM_ERR_INVALID, name
        checked += 1
    assert checked == len(lbm.SYMBOLS) - 3
