"""lbm_balances_noalloc, the entry point for callers that cannot allocate
device memory (a host framework that owns every buffer and passes them in,
or an application with a device budget fixed at start-up), must give the
same totals as the context's lbm_balances on the same populations.

The test calls it through the C ABI twice in a row (two different states),
on caller-owned device buffers; this file is collected last so that a run
stopping at the first failure has already run every other test."""
import ctypes as C
import struct

import numpy as np
import pytest

from paper_2203_01316_gb300 import inputs as I
from paper_2203_01316_gb300 import lbm

pytestmark = pytest.mark.gpu

REL_TOL = 1e-9  # the tolerance of the balance checks in the parity tests


def _state_arrays(s):
    """The context's stored FP32 populations (deviation form) as host arrays."""
    blob = s.save_state()
    magic, version, nx, ny, nz, qh, storage, fbytes, hbytes, step = struct.unpack_from("<8sI5iQQQ", blob, 0)
    assert magic == b"LBMSTATE" and storage == 0
    off = struct.calcsize("<8sI5iQQQ")
    f = np.frombuffer(blob, dtype=np.float32, count=fbytes // 4, offset=off)
    h = np.frombuffer(blob, dtype=np.float32, count=hbytes // 4, offset=off + fbytes)
    return f, h, qh


def test_noalloc_totals_match_lbm_balances_twice():
    import torch
    from paper_2203_01316_gb300 import Solver

    w = I.heated_sphere(41, 19, 13, D=7.0, cx=14.0, seed=9, u_in=0.03, T_in=0.1)
    nx, ny, nz = w["dims"]
    N = nx * ny * nz
    rho0, T_ref = 1.0, 0.5
    s = Solver(nx, ny, nz, nu=0.03, k=2e-3, storage="f32", periodic_x=False, rho0=rho0, T_ref=T_ref)
    s.set_geometry(w["flags"], w["links"], n_walls=1)
    s.set_bc(0, 1.0)
    s.set_inlet(w["u_in"], w["T_in"])
    s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])

    L = lbm.lib()
    dev = torch.device("cuda", 0)
    flags = torch.from_numpy(np.asarray(w["flags"], np.uint8)).to(dev)
    totals = torch.zeros(3, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    for steps in (4, 9):  # two calls in a row, on two different states
        s.step(steps)
        mass, energy = s.balances()
        fh, hh, qh = _state_arrays(s)
        f = torch.from_numpy(fh.copy()).to(dev)
        h = torch.from_numpy(hh.copy()).to(dev)
        torch.cuda.synchronize()
        st = L.lbm_balances_noalloc(C.c_void_p(f.data_ptr()), C.c_void_p(h.data_ptr()), qh, N,
                                    C.c_void_p(flags.data_ptr()), rho0, T_ref,
                                    C.c_void_p(totals.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert st == lbm.LBM_OK, L.lbm_last_error(None)
        torch.cuda.synchronize()
        got = totals.cpu().numpy()
        assert abs(got[0] - mass) <= REL_TOL * abs(mass)
        assert abs(got[1] - energy) <= REL_TOL * abs(energy)
        assert got[2] == 0.0
    s.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    L = lbm.lib()
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    st = L.lbm_balances_noalloc(p, p, 27, 33554432 + 1, None, 0.0, 0.0, p, None)
    assert st == lbm.LBM_ERR_INVALID
    assert b"static scratch capacity" in L.lbm_last_error(None)
