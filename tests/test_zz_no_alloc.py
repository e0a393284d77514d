"""lbm_balances_noalloc serves callers that cannot allocate device memory: a
host framework that owns every device buffer and hands them in (a plugin or
custom-call interface with no allocator), or an application whose device
budget is fixed at start-up.  It must give the same totals as the context's
lbm_balances on the same post-collision state.

Each case calls it through the C ABI twice in a row (two different states)
on caller-owned device buffers built from the context's populations.  The
cases cover both h lattices, flags given and flags NULL, symmetry rows (flag
4, which lbm_balances skips), a heat source (the App. D half-step correction)
and a grid of several 16,384-node blocks, so the final pass reduces more than
one partial slot.  This file is collected last so that a run stopping at the
first failure has already run every other test."""
import ctypes as C

import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01316_gb300 import inputs as I
from paper_2203_01316_gb300 import lbm

pytestmark = pytest.mark.gpu

REL_TOL = 1e-9  # the tolerance of the balance checks in the parity tests
NODES_PER_BLOCK = 256 * 64  # nodes one partial slot of the static scratch covers


def _caller_arrays(s, rho0, T_ref, qh, dev):
    """The context's post-collision state as caller-owned FP32 deviation
    arrays [Q][N] on the device (the library's populations are FP64 and
    unshifted; removing the weights' shift recovers the stored values)."""
    import torch
    f, h = s.populations()
    _, w27, _, _ = O.lattice(27)
    _, wh, _, _ = O.lattice(qh)
    fd = (f - w27[:, None] * rho0).astype(np.float32)
    hd = (h - wh[:, None] * T_ref).astype(np.float32)
    return torch.from_numpy(fd).to(dev), torch.from_numpy(hd).to(dev)


def _case(name):
    if name == "sphere_q27":
        w = I.heated_sphere(41, 19, 13, D=7.0, cx=14.0, seed=9, u_in=0.03, T_in=0.1)
        return w, dict(qh=27), None
    if name == "sphere_q7_multiblock":
        w = I.heated_sphere(64, 32, 24, D=9.0, cx=20.0, seed=5, u_in=0.03, T_in=0.1)
        assert np.prod(w["dims"]) > 2 * NODES_PER_BLOCK
        return w, dict(qh=7), None
    if name == "periodic_no_flags":
        w = I.periodic_tgv(32)
        w["nwalls"] = 1
        return w, dict(qh=27), None
    if name == "symmetry_rows":
        w = I.confined_cylinder(0.2, seed=4)
        assert np.any(w["flags"] == I.MIRROR)
        return w, dict(qh=27), None
    if name == "heat_source_multiblock":
        w = I.plate_channel(48, 24, 20, q_bottom=0.3, q_top=0.7, seed=11)
        theta = I.uniform(21, int(np.prod(w["dims"])), 0.0, 1e-3).astype(np.float32)
        theta[w["flags"] == I.SOLID] = 0.0
        return w, dict(qh=27), theta
    raise KeyError(name)


@pytest.mark.parametrize("name", ["sphere_q27", "sphere_q7_multiblock", "periodic_no_flags", "symmetry_rows",
                                  "heat_source_multiblock"])
def test_noalloc_totals_match_lbm_balances_twice(name):
    import torch
    from paper_2203_01316_gb300 import Solver

    w, opt, theta = _case(name)
    nx, ny, nz = w["dims"]
    N = nx * ny * nz
    qh = opt["qh"]
    rho0, T_ref = 1.0, w.get("T_in", 0.5)
    s = Solver(nx, ny, nz, nu=0.03, k=2e-3, lat_h=qh, storage="f32", periodic_x=w["periodic_x"], rho0=rho0,
               T_ref=T_ref)
    s.set_geometry(w["flags"], w["links"], n_walls=w["nwalls"])
    for i in range(w["nwalls"]):
        s.set_bc(i, T_ref + 1.0)
    if not w["periodic_x"]:
        s.set_inlet(w["u_in"], w["T_in"])
    if theta is not None:
        s.set_source(theta)
    s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])

    L = lbm.lib()
    dev = torch.device("cuda", 0)
    flags = None
    if name != "periodic_no_flags":
        flags = torch.from_numpy(np.asarray(w["flags"], np.uint8)).to(dev)
    th = torch.from_numpy(theta).to(dev) if theta is not None else None
    totals = torch.zeros(3, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    for steps in (4, 9):  # two calls in a row, on two different states
        s.step(steps)
        mass, energy = s.balances()
        f, h = _caller_arrays(s, rho0, T_ref, qh, dev)
        totals.fill_(-1.0)
        torch.cuda.synchronize()
        st = L.lbm_balances_noalloc(C.c_void_p(f.data_ptr()), C.c_void_p(h.data_ptr()), qh, N,
                                    C.c_void_p(flags.data_ptr()) if flags is not None else None,
                                    C.c_void_p(th.data_ptr()) if th is not None else None, rho0, T_ref,
                                    C.c_void_p(totals.data_ptr()), C.c_void_p(stream.cuda_stream))
        assert st == lbm.LBM_OK, L.lbm_last_error(None)
        torch.cuda.synchronize()
        got = totals.cpu().numpy()
        assert abs(got[0] - mass) <= REL_TOL * abs(mass), (name, steps, got[0], mass)
        assert abs(got[1] - energy) <= REL_TOL * abs(energy), (name, steps, got[1], energy)
        assert got[2] == 0.0
    s.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    L = lbm.lib()
    dummy = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    st = L.lbm_balances_noalloc(p, p, 27, 33554432 + 1, None, None, 0.0, 0.0, p, None)
    assert st == lbm.LBM_ERR_INVALID
    assert b"static scratch capacity" in L.lbm_last_error(None)
