"""The GPU adjoints with the boundary rules of the Sec. 4.4 confined cylinder
(symmetry rows, reading R15; the Zou-He inlet, reading R20) against the
oracle's adjoints on the same inputs (which are themselves pinned against
differences of J in test_oracle_adjoint_bc):

* the h adjoint (lbm_adjoint_step / lbm_adjoint_step_h) with symmetry rows,
  with the Zou-He inlet and with both, for the central-moment kinds on both
  lattices and for Cumulants-1st;
* the coupled f + h adjoint (lbm_adjoint_flow_step) with the same three
  boundary sets: gradients with respect to theta, T_w, F and (with the
  Zou-He inlet) u_in.

Tolerances as in test_gpu_adjoint and test_gpu_flow_adjoint: FP64 storage
to 1e-9 (h adjoint) or 1e-8 (coupled) of the largest entry, FP32 to 1e-4;
J to 1e-10 (FP64) and 1e-6 (FP32) relative."""
import numpy as np
import pytest

from oracle import oracle as O

from test_gpu_flow_adjoint import _gpu as _gpu_flow
from test_oracle_adjoint_bc import _case

pytestmark = pytest.mark.gpu

NSTEPS, WINDOW, EVERY = 9, (3, 9), 4


def _solver(w, p, storage, Tw):
    from paper_2203_01316_gb300 import Solver
    nx, ny, nz = w["dims"]
    s = Solver(nx, ny, nz, nu=p["nu"], k=p["k"], lat_h=p["qh"], hkind=p["hkind"], storage=storage,
               periodic_x=p["periodic_x"], T_ref=0.5, inlet_bc=p["inlet_bc"])
    s.set_geometry(w["flags"], w["links"], n_walls=1)
    s.set_bc(0, Tw)
    if not p["periodic_x"]:
        s.set_inlet(p["u_in"], p["T_in"])
    s.set_force(p["F"])
    s.set_source(w["theta"].astype(np.float32))
    s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    s.step(3)
    return s


def _oracle(w, p, Tw):
    o = O.Oracle(O.make_params(**p))
    o.set_geometry(w["flags"], w["links"], nwalls=1)
    o.set_wall_temperature(0, float(np.float32(Tw)))
    o.set_theta(w["theta"].astype(np.float32).astype(np.float64))
    return o


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("bc", ["mirror", "zou_he", "both"])
@pytest.mark.parametrize("qh,kind,obj", [(27, "trt", ("surface", 0, 1.0)), (7, "srt", ("section", 9, 1.0)),
                                         (27, "cum1st", ("surface", 0, 0.7))])
def test_h_adjoint_with_boundary_rules_matches_oracle(storage, bc, qh, kind, obj):
    import torch
    from paper_2203_01316_gb300.autograd import thermal_objective
    w, p = _case(bc, qh, kind, ny=10)
    Tw = 0.9
    s = _solver(w, p, storage, Tw)
    f0, h0 = s.populations()
    o_obj = s.objective(*obj)
    state0 = s.save_state(torch.empty(s.state_size(), dtype=torch.uint8, device="cuda"))
    th = torch.tensor(w["theta"].astype(np.float32).astype(np.float64), device="cuda", requires_grad=True)
    tw = torch.tensor([Tw], dtype=torch.float64, requires_grad=True)
    J = thermal_objective(th, tw, s, state0, NSTEPS, WINDOW, o_obj, every=EVERY)
    J.backward()
    Jg, dth_g, dTw_g = float(J.item()), th.grad.cpu().numpy(), tw.grad.numpy()
    Jo, dth_o, dTw_o = _oracle(w, p, Tw).adjoint(f0, h0, NSTEPS, WINDOW, obj)
    tol = 1e-9 if storage == "f64" else 1e-4
    assert abs(Jg - Jo) <= (1e-10 if storage == "f64" else 1e-6) * max(abs(Jo), 1e-3)
    scale = np.abs(dth_o).max()
    assert scale > 0
    assert np.abs(dth_g - dth_o).max() <= tol * scale
    assert np.abs(dTw_g - dTw_o).max() <= tol * max(np.abs(dTw_o).max(), 1e-12)
    s.close()


@pytest.mark.parametrize("storage", ["f64", "f32"])
@pytest.mark.parametrize("bc", ["mirror", "zou_he", "both"])
@pytest.mark.parametrize("qh,kind,obj", [(27, "trt", ("surface", 0, 1.0)), (27, "trt", ("force", 0, 1.0, 0)),
                                         (7, "cum1st", ("force", 0, 1.0, 1))])
def test_coupled_adjoint_with_boundary_rules_matches_oracle(storage, bc, qh, kind, obj):
    w, p = _case(bc, qh, kind, ny=10)
    Tw = 0.9
    s = _solver(w, p, storage, Tw)
    f0, h0 = s.populations()
    theta = w["theta"].astype(np.float32).astype(np.float64)
    Jg, dth_g, dTw_g, dF_g, du_g = _gpu_flow(s, theta, [Tw], p["F"], p["u_in"], NSTEPS, WINDOW, obj, EVERY)
    Jo, dth_o, dTw_o, dF_o, du_o = _oracle(w, p, Tw).adjoint_flow(f0, h0, NSTEPS, WINDOW, obj)
    tol = 1e-8 if storage == "f64" else 1e-4
    if obj[0] == "force":
        assert abs(Jg - Jo) <= (1e-10 if storage == "f64" else 1e-6) * abs(obj[2]) * (WINDOW[1] - WINDOW[0])
    else:
        assert abs(Jg - Jo) <= (1e-10 if storage == "f64" else 1e-6) * max(abs(Jo), 1e-3)
    scale = max(np.abs(dF_o).max(), np.abs(du_o).max())
    assert np.abs(dF_g - dF_o).max() <= tol * scale
    if bc == "mirror":
        assert np.all(du_g == 0.0) and np.all(du_o == 0.0)
    else:
        assert np.abs(du_g - du_o).max() <= tol * scale, (du_g, du_o)
        assert np.abs(du_o).max() > 1e-3 * scale  # the inlet velocity matters
    if obj[0] == "surface":
        assert np.abs(dth_g - dth_o).max() <= tol * np.abs(dth_o).max()
        assert np.abs(dTw_g - dTw_o).max() <= tol * max(np.abs(dTw_o).max(), 1e-12)
    s.close()
