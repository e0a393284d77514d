"""The GPU adjoint (lbm_step_record + lbm_adjoint_step behind the
torch.autograd.Function of paper_2203_01316_gb300.autograd) against the
oracle's adjoint on the same inputs, and against central finite
differences of the FP64 GPU path on the plate-channel workload of the
differentiation form (128 x 64 x 64, 500 steps, Nusselt number of the top
wall over the last 100, checkpoints every 50).

Tolerances: FP64 storage agrees with the oracle to 1e-9 of the largest
gradient entry; FP32 storage to 1e-4 relative (the stated gradient target);
the objective value to 1e-10 (FP64) and 1e-6 (FP32) relative over 11
steps, and FP32 against FP64 to 1e-4 over the 500-step workload."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01316_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _torch():
    import torch
    return torch


def _solver(w, storage, qh, kind, nu, k, F, Tw, theta, T_ref=0.5, wall_bc="iabb"):
    from paper_2203_01316_gb300 import Solver
    nx, ny, nz = w["dims"]
    s = Solver(nx, ny, nz, nu=nu, k=k, lat_h=qh, hkind=kind, storage=storage, periodic_x=w["periodic_x"],
               T_ref=T_ref, wall_bc=wall_bc)
    s.set_geometry(w["flags"], w["links"], n_walls=w["nwalls"])
    for i, T in enumerate(Tw):
        s.set_bc(i, T)
    if not w["periodic_x"]:
        s.set_inlet(w["u_in"], w["T_in"])
    s.set_force(F)
    s.set_source(theta.astype(np.float32))
    s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    return s


def _gpu_gradients(s, theta, Tw, nsteps, window, obj_spec, every):
    torch = _torch()
    from paper_2203_01316_gb300.autograd import thermal_objective
    kind, idx, weight = obj_spec
    obj = s.objective(kind, idx, weight)
    state0 = s.save_state(torch.empty(s.state_size(), dtype=torch.uint8, device="cuda"))
    th = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
    tw = torch.tensor(Tw, dtype=torch.float64, requires_grad=True)
    J = thermal_objective(th, tw, s, state0, nsteps, window, obj, every=every)
    J.backward()
    return float(J.item()), th.grad.cpu().numpy(), tw.grad.numpy(), state0


def _plate():
    w = I.plate_channel(nx=12, ny=10, nz=6, q_bottom=0.3, q_top=0.7, theta_max=1e-3, seed=21)
    N = len(w["rho"])
    w["u"] = I.uniform(22, 3 * N, -0.03, 0.03).reshape(3, N)
    w["T"] = I.uniform(23, N, 0.2, 1.0)
    return w


def _channel():
    w = I.heated_sphere(20, 11, 9, D=5.0, cx=8.0, seed=24, u_in=0.04, T_in=0.2)
    w["theta"] = I.uniform(25, len(w["rho"]), 0.0, 1e-3)
    return w


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("case,qh,kind,obj,wall_bc", [
    ("plate", 27, "trt", ("surface", 1, 0.9), "iabb"),
    ("plate", 27, "srt", ("section", 4, 1.0), "iabb"),
    ("plate", 27, "1st", ("surface", 0, 1.0), "iabb"),
    ("plate", 7, "trt", ("surface", 1, 1.0), "iabb"),
    ("plate", 27, "trt", ("surface", 1, 1.0), "eq"),
    ("plate", 27, "trt", ("surface", 0, 1.0), "abb"),
    ("channel", 27, "trt", ("surface", 0, 1.0), "iabb"),
    ("channel", 7, "srt", ("section", 17, 1.0), "iabb"),
    ("plate", 27, "cum1st", ("surface", 1, 0.9), "iabb"),
    ("plate", 7, "cum1st", ("section", 4, 1.0), "iabb"),
    ("channel", 27, "cum1st", ("surface", 0, 1.0), "iabb"),
    ("plate", 27, "cum1st", ("surface", 0, 1.0), "abb"),
])
def test_adjoint_matches_oracle(storage, case, qh, kind, obj, wall_bc):
    w = _plate() if case == "plate" else _channel()
    Tw = [1.0, 0.1][: w["nwalls"]]
    nu, k, F = 0.05, 0.01, ((2e-4, 0.0, 1e-4) if case == "plate" else (0.0, 0.0, 0.0))
    theta = w["theta"].astype(np.float32).astype(np.float64)
    s = _solver(w, storage, qh, kind, nu, k, F, Tw, theta, wall_bc=wall_bc)
    f0, h0 = s.populations()
    nsteps, window, every = 11, (4, 11), 4
    Jg, dth_g, dTw_g, _ = _gpu_gradients(s, theta, Tw, nsteps, window, obj, every)
    nx, ny, nz = w["dims"]
    p = O.make_params(nx=nx, ny=ny, nz=nz, qh=qh, hkind=kind, periodic_x=w["periodic_x"], nu=nu, k=k, F=F,
                      u_in=w.get("u_in", (0, 0, 0)), T_in=w.get("T_in", 0.0), wall_bc=wall_bc)
    o = O.Oracle(p)
    o.set_geometry(w["flags"], w["links"], nwalls=w["nwalls"])
    for i, T in enumerate(Tw):
        o.set_wall_temperature(i, float(np.float32(T)))
    o.set_theta(theta)
    Jo, dth_o, dTw_o = o.adjoint(f0, h0, nsteps, window, obj, nwalls=w["nwalls"])
    tol = 1e-9 if storage == "f64" else 1e-4
    scale = np.abs(dth_o).max()
    assert abs(Jg - Jo) <= (1e-10 if storage == "f64" else 1e-6) * max(abs(Jo), 1e-3)
    assert np.abs(dth_g - dth_o).max() <= tol * scale
    assert np.abs(dTw_g - dTw_o).max() <= tol * max(np.abs(dTw_o).max(), 1e-12)


def test_cumulant_adjoint_needs_h_records():
    # the Cumulants-1st collision is not linear in h: the record-free entry
    # point refuses it, the one with the level's h record accepts it
    torch = _torch()
    from paper_2203_01316_gb300 import LBMError
    w = _plate()
    theta = w["theta"].astype(np.float32).astype(np.float64)
    s = _solver(w, "f32", 27, "cum1st", 0.05, 0.01, (0.0, 0.0, 0.0), [1.0, 0.1], theta)
    N = s.N
    u = torch.empty(3 * N, dtype=torch.float32, device="cuda")
    h = torch.empty(27 * N, dtype=torch.float32, device="cuda")
    s.step_record(1, u, h_rec=h)
    mu = torch.zeros(27 * N, dtype=torch.float32, device="cuda")
    out = torch.empty_like(mu)
    st = s.L.lbm_adjoint_step(s._h, u.data_ptr(), mu.data_ptr(), out.data_ptr(), None, None)
    assert st == 1  # LBM_ERR_INVALID
    with pytest.raises(LBMError):
        s._check(s.L.lbm_adjoint_step_h(s._h, u.data_ptr(), None, mu.data_ptr(), out.data_ptr(), None, None))
    s.adjoint_step(u, mu, out, h_level=h)
    s.sync()
    assert torch.count_nonzero(out).item() == 0
    # the h record holds the post-collision deviations of the state reached
    _, hp = s.populations()
    rec = h.view(27, N).cpu().numpy().astype(np.float64) + 0.5 * O.lattice(27)[1][:, None]
    fl = w["flags"] != I.SOLID
    assert np.abs(rec[:, fl] - hp[:, fl]).max() < 1e-6


def _config4():
    w = I.plate_channel(nx=128, ny=64, nz=64, q_bottom=0.5, q_top=0.5, seed=1234, theta_max=1e-5, T0=0.5)
    ny = 64
    Hc = w["H_c"]
    nu, Pr, umax = 0.02, 100.0, 0.03
    Fx = 8.0 * nu * umax / Hc ** 2
    N = len(w["rho"])
    y = (np.arange(N) // 128) % ny
    yb, yt = 0.5, ny - 1.5
    u = np.zeros((3, N))
    u[0] = np.clip(4.0 * umax * (y - yb) * (yt - y) / Hc ** 2, 0.0, None)
    w["u"] = u
    return w, nu, nu / Pr, (Fx, 0.0, 0.0), Hc


def test_config4_adjoint_vs_fp64_finite_differences():
    # J = mean Nusselt number of the top wall over the last 100 of 500 steps;
    # dJ/dtheta at 20 seeded nodes and dJ/dT_w of both walls from the adjoint
    # (checkpoints every 50) against FP64 central differences.  J is affine
    # in theta and T_w (CM kinds), so the difference quotient has no
    # truncation error; the step is 1e-2 (theta) and 1e-3 (T_w): the
    # prescribed 1e-3 |theta| puts delta J of nodes far from the wall at the
    # FP64 rounding floor of J.
    # FP32 storage: normwise, max |g - fd| <= 1e-4 max |g| (entries 1e6-1e8
    # below the maximum are beyond FP32 resolution), per entry 1e-3 for
    # entries above 1e-3 max |g|.  FP64 storage: per entry 1e-4.
    torch = _torch()
    from paper_2203_01316_gb300.autograd import thermal_objective
    w, nu, k, F, Hc = _config4()
    nx, ny, nz = w["dims"]
    theta = w["theta"].astype(np.float32).astype(np.float64)
    Tw = [1.0, 0.0]
    A = nx * nz
    weight = Hc / (k * A * 1.0) / 100.0
    nsteps, window, every = 500, (401, 500), 50
    grads = {}
    for st in ("f32", "f64"):
        sv = _solver(w, st, 27, "trt", nu, k, F, Tw, theta)
        grads[st] = _gpu_gradients(sv, theta, Tw, nsteps, window, ("surface", 1, weight), every)
        sv.close()
    s64 = _solver(w, "f64", 27, "trt", nu, k, F, Tw, theta)
    obj = s64.objective("surface", 1, weight)
    state0 = s64.save_state(torch.empty(s64.state_size(), dtype=torch.uint8, device="cuda"))

    def J64(th, tw):
        with torch.no_grad():
            return float(thermal_objective(torch.tensor(th, device="cuda"), torch.tensor(tw), s64, state0,
                                           nsteps, window, obj, every=nsteps).item())

    J0 = J64(theta, Tw)
    # the FP32 forward's mean Nusselt number (a wall flux) after 500 steps
    # agrees with FP64 to 1.8e-5 relative; bound it by the gradient target
    assert abs(grads["f32"][0] - J0) <= 1e-4 * abs(J0)
    assert abs(grads["f64"][0] - J0) <= 1e-10 * abs(J0)
    gmax = np.abs(grads["f64"][1]).max()
    fluid = np.nonzero(np.asarray(w["flags"]) == I.FLUID)[0]
    nodes = fluid[(I.splitmix64(77, 20) % np.uint64(len(fluid))).astype(np.int64)]
    for n in nodes:
        h = 1e-2
        tp = theta.copy(); tp[n] += h
        tm = theta.copy(); tm[n] -= h
        fd = (J64(tp, Tw) - J64(tm, Tw)) / (2 * h)
        g32, g64 = grads["f32"][1][n], grads["f64"][1][n]
        assert abs(g64 - fd) <= 1e-4 * abs(fd) + 1e-10 * gmax, (n, g64, fd)
        assert abs(g32 - fd) <= 1e-4 * gmax, (n, g32, fd)
        if abs(fd) >= 1e-3 * gmax:
            assert abs(g32 - fd) <= 1e-3 * abs(fd), (n, g32, fd)
    for wall in (0, 1):
        h = 1e-3
        Tp = list(Tw); Tp[wall] += h
        Tm = list(Tw); Tm[wall] -= h
        fd = (J64(theta, Tp) - J64(theta, Tm)) / (2 * h)
        for st in ("f32", "f64"):
            assert abs(grads[st][2][wall] - fd) <= 1e-4 * abs(fd), (st, wall, grads[st][2][wall], fd)
    assert math.isfinite(J0)


@pytest.mark.parametrize("kind", ["trt", "cum1st"])
def test_two_level_checkpoints_give_the_same_gradients(kind):
    """every2 < every re-runs each segment keeping second-level states; the
    recomputed states and records are the same bits, so J and both gradients
    are identical to the one-level run."""
    torch = _torch()
    from paper_2203_01316_gb300.autograd import thermal_objective
    w = _plate()
    N = len(w["rho"])
    theta = I.uniform(23, N, 0.0, 1e-3)
    theta[np.asarray(w["flags"]) == I.SOLID] = 0.0
    s = _solver(w, "f32", 27, kind, 0.05, 0.01, (1e-5, 0.0, 0.0), [1.0, 0.1], theta)
    obj = s.objective("surface", 1, 1.0)
    state0 = s.save_state(torch.empty(s.state_size(), dtype=torch.uint8, device="cuda"))
    out = []
    for every, every2 in ((12, None), (12, 5), (12, 1)):
        th = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
        tw = torch.tensor([1.0, 0.1], dtype=torch.float64, requires_grad=True)
        J = thermal_objective(th, tw, s, state0, 31, (20, 31), obj, every=every, every2=every2)
        J.backward()
        out.append((float(J.item()), th.grad.cpu().numpy(), tw.grad.numpy()))
    for J, g, gw in out[1:]:
        assert J == out[0][0]
        assert np.array_equal(g, out[0][1]) and np.array_equal(gw, out[0][2])
    assert np.abs(out[0][1]).max() > 0
    s.close()
