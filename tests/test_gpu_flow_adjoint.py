"""The adjoint of the coupled f + h evolution on the GPU (lbm_step_record_pre
+ lbm_adjoint_flow_step behind paper_2203_01316_gb300.autograd.FlowObjective)
against the oracle's coupled adjoint (oracle.adjoint_flow, itself pinned by
finite differences of the nonlinear J): gradients of the heat-flux
objectives with respect to the body force F, the inlet velocity u_in, the
source theta and the wall temperatures, and of the momentum-exchange force
on a wall (drag, lift, wall shear: f alone) with respect to F and u_in.

Tolerances: FP64 storage agrees with the oracle to 1e-8 of the largest
entry of each gradient (the oracle's Jacobians are 4-point differences,
accurate to about 1e-11); FP32 to 1e-4 of it (the FP32 h-only adjoint's
bound).  J: 1e-10 (FP64) and 1e-6 (FP32) relative; for a force objective
relative to weight x levels (its link sums have O(1) terms at every level
and cancel to a far smaller J)."""
import numpy as np
import pytest

from oracle import oracle as O

from test_gpu_adjoint import _channel, _plate, _solver

pytestmark = pytest.mark.gpu


def _gpu(s, theta, Tw, F, uin, nsteps, window, obj_spec, every, every2=None):
    import torch
    from paper_2203_01316_gb300.autograd import flow_objective
    kind, idx, weight = obj_spec[:3]
    obj = s.objective(kind, idx, weight, obj_spec[3] if len(obj_spec) > 3 else 0)
    state0 = s.save_state(torch.empty(s.state_size(), dtype=torch.uint8, device="cuda"))
    th = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
    tw = torch.tensor(Tw, dtype=torch.float64, requires_grad=True)
    tF = torch.tensor(F, dtype=torch.float64, requires_grad=True)
    tu = torch.tensor(uin, dtype=torch.float64, requires_grad=True)
    J = flow_objective(th, tw, tF, tu, s, state0, nsteps, window, obj, every=every, every2=every2)
    J.backward()
    return (float(J.item()), th.grad.cpu().numpy(), tw.grad.numpy(), tF.grad.numpy(), tu.grad.numpy())


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("case,qh,kind,obj", [
    ("plate", 27, "trt", ("surface", 1, 0.9)),
    ("plate", 27, "cum1st", ("surface", 0, 1.0)),
    ("channel", 27, "trt", ("surface", 0, 1.0)),
    ("channel", 7, "srt", ("section", 17, 1.0)),
    ("plate", 27, "trt", ("force", 0, 1.0, 0)),
    ("channel", 27, "trt", ("force", 0, 1.0, 0)),
    ("channel", 7, "cum1st", ("force", 0, 0.5, 1)),
])
def test_flow_adjoint_matches_oracle(storage, case, qh, kind, obj):
    w = _plate() if case == "plate" else _channel()
    Tw = [1.0, 0.1][: w["nwalls"]]
    nu, k = 0.05, 0.01
    F = (2e-4, 0.0, 1e-4) if case == "plate" else (1e-5, 0.0, 0.0)
    uin = tuple(w.get("u_in", (0.0, 0.0, 0.0)))
    theta = w["theta"].astype(np.float32).astype(np.float64)
    s = _solver(w, storage, qh, kind, nu, k, F, Tw, theta)
    f0, h0 = s.populations()
    nsteps, window, every = 11, (4, 11), 4
    Jg, dth_g, dTw_g, dF_g, du_g = _gpu(s, theta, Tw, F, uin, nsteps, window, obj, every)
    nx, ny, nz = w["dims"]
    p = O.make_params(nx=nx, ny=ny, nz=nz, qh=qh, hkind=kind, periodic_x=w["periodic_x"], nu=nu, k=k, F=F,
                      u_in=uin, T_in=w.get("T_in", 0.0))
    o = O.Oracle(p)
    o.set_geometry(w["flags"], w["links"], nwalls=w["nwalls"])
    for i, T in enumerate(Tw):
        o.set_wall_temperature(i, float(np.float32(T)))
    o.set_theta(theta)
    Jo, dth_o, dTw_o, dF_o, du_o = o.adjoint_flow(f0, h0, nsteps, window, obj, nwalls=w["nwalls"])
    tol = 1e-8 if storage == "f64" else 1e-4
    # a force is a difference of link sums whose terms are O(w rho0) at every
    # level, so its J is compared on that scale rather than on its own size
    jscale = abs(Jo) if obj[0] != "force" else max(abs(Jo), obj[2] * (window[1] - window[0] + 1))
    assert abs(Jg - Jo) <= (1e-10 if storage == "f64" else 1e-6) * max(jscale, 1e-3)
    if obj[0] == "force":  # f alone enters J: h's adjoint stays exactly zero
        assert np.all(dth_o == 0.0) and np.all(dTw_o == 0.0)
        assert np.all(dth_g == 0.0) and np.all(dTw_g == 0.0)
    else:
        assert np.abs(dth_g - dth_o).max() <= tol * np.abs(dth_o).max()
        assert np.abs(dTw_g - dTw_o).max() <= tol * max(np.abs(dTw_o).max(), 1e-12)
    flow_scale = max(np.abs(dF_o).max(), np.abs(du_o).max())
    assert flow_scale > 0
    assert np.abs(dF_g - dF_o).max() <= tol * flow_scale, (dF_g, dF_o)
    assert np.abs(du_g - du_o).max() <= tol * flow_scale, (du_g, du_o)
    if case == "channel" and (obj[0] == "surface" or obj[:2] == ("force", 0) and obj[3] == 0):
        assert abs(du_o[0]) > 1e-3 * flow_scale  # the inlet velocity matters here (heat flux, drag)


def test_flow_adjoint_refuses_16_bit_storage():
    import torch
    from paper_2203_01316_gb300 import LBMError
    w = _plate()
    theta = w["theta"].astype(np.float32).astype(np.float64)
    s = _solver(w, "f16", 27, "trt", 0.05, 0.01, (0.0, 0.0, 0.0), [1.0, 0.1], theta)
    N = s.N
    f = torch.empty(27 * N, dtype=torch.float32, device="cuda")
    h = torch.empty(27 * N, dtype=torch.float32, device="cuda")
    with pytest.raises(LBMError):
        s.step_record_pre(1, f, h)


def test_flow_adjoint_two_level_checkpoints_give_the_same_gradients():
    """every2 < every: the same recomputed bits, so the same J and gradients
    (theta, T_w, F, u_in) as one checkpoint level, from the same saved state."""
    import torch
    from paper_2203_01316_gb300.autograd import flow_objective
    w = _channel()
    Tw = [1.0]
    F = (1e-5, 0.0, 0.0)
    uin = tuple(w["u_in"])
    theta = w["theta"].astype(np.float32).astype(np.float64)
    s = _solver(w, "f32", 27, "trt", 0.05, 0.01, F, Tw, theta)
    obj = s.objective("surface", 0, 1.0)
    state0 = s.save_state(torch.empty(s.state_size(), dtype=torch.uint8, device="cuda"))
    out = []
    for every2 in (None, 4, 1):
        th = torch.tensor(theta, dtype=torch.float64, device="cuda", requires_grad=True)
        tw = torch.tensor(Tw, dtype=torch.float64, requires_grad=True)
        tF = torch.tensor(F, dtype=torch.float64, requires_grad=True)
        tu = torch.tensor(uin, dtype=torch.float64, requires_grad=True)
        J = flow_objective(th, tw, tF, tu, s, state0, 13, (5, 13), obj, every=6, every2=every2)
        J.backward()
        out.append([float(J.item()), th.grad.cpu().numpy(), tw.grad.numpy(), tF.grad.numpy(), tu.grad.numpy()])
    for r in out[1:]:
        assert r[0] == out[0][0]
        for a, b in zip(r[1:], out[0][1:]):
            assert np.array_equal(a, b)
    assert np.abs(out[0][3]).max() > 0
    s.close()
