"""Pins of the oracle's adjoint of the h evolution against finite differences.

For the CM kinds the h step is affine in h, theta and the wall temperatures
(Eq. H_cm_collision, Eq. IABB, App. D), and the objectives are linear
fluxes, so J(theta, T_w) is affine: central differences in FP64 are exact up
to rounding, and any mistake in a transpose shows up as an O(1) relative
error."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01316_gb300 import inputs as I


def _plate_case(qh=27, kind="trt", qb=0.3, qt=0.7, seed=5, wall_bc="iabb"):
    w = I.plate_channel(nx=6, ny=9, nz=4, q_bottom=qb, q_top=qt, theta_max=1e-3, seed=seed)
    N = len(w["rho"])
    w["u"] = I.uniform(seed + 1, 3 * N, -0.03, 0.03).reshape(3, N)
    w["T"] = I.uniform(seed + 2, N, 0.2, 1.0)
    p = O.make_params(nx=6, ny=9, nz=4, qh=qh, hkind=kind, nu=0.05, k=0.01, F=(2e-4, 0.0, 1e-4), wall_bc=wall_bc)
    return w, p


def _channel_case(qh=27, kind="trt", seed=6):
    w = I.heated_sphere(14, 9, 8, D=4.0, cx=6.0, seed=seed, u_in=0.04, T_in=0.2)
    nx, ny, nz = w["dims"]
    p = O.make_params(nx=nx, ny=ny, nz=nz, qh=qh, hkind=kind, periodic_x=False, nu=0.05, k=0.01,
                      u_in=w["u_in"], T_in=w["T_in"])
    N = nx * ny * nz
    w["theta"] = I.uniform(seed + 3, N, 0.0, 1e-3)
    return w, p


def _setup(w, p, Tw):
    o = O.Oracle(p)
    o.set_geometry(w["flags"], w["links"], nwalls=w["nwalls"])
    for i, T in enumerate(Tw):
        o.set_wall_temperature(i, T)
    o.set_theta(w["theta"])
    o.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    fpost, hpost = o.post()
    return o, fpost, hpost


def _J(w, p, Tw, theta, fpost, hpost, nsteps, window, obj):
    o = O.Oracle(p)
    o.set_geometry(w["flags"], w["links"], nwalls=w["nwalls"])
    for i, T in enumerate(Tw):
        o.set_wall_temperature(i, T)
    o.set_theta(theta)
    J, _, _ = o.adjoint(fpost, hpost, nsteps, window, obj, nwalls=w["nwalls"], gradients=False)
    return J


@pytest.mark.parametrize("qh,kind,wall_bc", [(27, "trt", "iabb"), (27, "srt", "iabb"), (27, "1st", "iabb"),
                                             (7, "trt", "iabb"), (27, "trt", "eq"), (27, "trt", "abb")])
@pytest.mark.parametrize("obj", [("surface", 1, 0.7), ("section", 3, 1.3)])
def test_plate_adjoint_matches_finite_differences(qh, kind, wall_bc, obj):
    w, p = _plate_case(qh, kind, wall_bc=wall_bc)
    Tw = [1.0, 0.1]
    o, fpost, hpost = _setup(w, p, Tw)
    nsteps, window = 10, (4, 10)
    J, dth, dTw = o.adjoint(fpost, hpost, nsteps, window, obj, nwalls=2)
    theta = w["theta"].copy()
    rng = np.random.default_rng(7)
    fluid = np.nonzero(w["flags"] == I.FLUID)[0]
    for n in rng.choice(fluid, 6, replace=False):
        eps = 1e-3
        tp = theta.copy(); tp[n] += eps
        tm = theta.copy(); tm[n] -= eps
        fd = (_J(w, p, Tw, tp, fpost, hpost, nsteps, window, obj) -
              _J(w, p, Tw, tm, fpost, hpost, nsteps, window, obj)) / (2 * eps)
        assert abs(dth[n] - fd) <= 1e-8 * max(abs(fd), 1e-3), (n, dth[n], fd)
    for wall in range(2):
        eps = 1e-3
        Tp = list(Tw); Tp[wall] += eps
        Tm = list(Tw); Tm[wall] -= eps
        fd = (_J(w, p, Tp, theta, fpost, hpost, nsteps, window, obj) -
              _J(w, p, Tm, theta, fpost, hpost, nsteps, window, obj)) / (2 * eps)
        assert abs(dTw[wall] - fd) <= 1e-8 * max(abs(fd), 1e-3), (wall, dTw[wall], fd)
    # solid nodes carry no sensitivity
    assert np.all(dth[w["flags"] == I.SOLID] == 0.0)


@pytest.mark.parametrize("qh", [27, 7])
def test_channel_adjoint_directional_derivative(qh):
    # inlet/outlet planes and a sphere with thin gaps: the gradient's
    # projection on a random direction equals the exact directional change
    w, p = _channel_case(qh)
    Tw = [1.0]
    o, fpost, hpost = _setup(w, p, Tw)
    nx = w["dims"][0]
    for obj in (("surface", 0, 1.0), ("section", nx - 2, 1.0)):
        nsteps, window = 9, (3, 9)
        J, dth, dTw = o.adjoint(fpost, hpost, nsteps, window, obj, nwalls=1)
        v = np.random.default_rng(9).uniform(-1, 1, len(dth))
        eps = 1e-4
        theta = w["theta"]
        fd = (_J(w, p, Tw, theta + eps * v, fpost, hpost, nsteps, window, obj) -
              _J(w, p, Tw, theta - eps * v, fpost, hpost, nsteps, window, obj)) / (2 * eps)
        assert abs(dth @ v - fd) <= 1e-8 * max(abs(fd), 1e-6)
        assert np.all(dth[w["flags"] == I.INLET] == 0.0)


def _richardson(Jof, x0, eps):
    """Central difference with one Richardson step: the O(eps^2) truncation
    of the nonlinear J cancels, leaving O(eps^4)."""
    d1 = (Jof(x0 + eps) - Jof(x0 - eps)) / (2 * eps)
    d2 = (Jof(x0 + eps / 2) - Jof(x0 - eps / 2)) / eps
    return (4 * d2 - d1) / 3


@pytest.mark.parametrize("qh", [27, 7])
@pytest.mark.parametrize("obj", [("surface", 1, 0.7), ("section", 3, 1.3)])
def test_cumulant_adjoint_matches_finite_differences(qh, obj):
    # Cumulants-1st (Eq. H_cu_collision): h* = (H + Q) M(v) with v depending on
    # h / H, so J is not affine; the reverse sweep uses the collision's
    # Jacobian at the recorded pre-collision states
    w, p = _plate_case(qh, "cum1st")
    Tw = [1.0, 0.1]
    o, fpost, hpost = _setup(w, p, Tw)
    nsteps, window = 10, (4, 10)
    J, dth, dTw = o.adjoint(fpost, hpost, nsteps, window, obj, nwalls=2)
    theta = w["theta"].copy()
    fluid = np.nonzero(w["flags"] == I.FLUID)[0]
    for n in np.random.default_rng(8).choice(fluid, 5, replace=False):
        def Jt(x, n=n):
            t = theta.copy()
            t[n] = x
            return _J(w, p, Tw, t, fpost, hpost, nsteps, window, obj)
        fd = _richardson(Jt, theta[n], 1e-3)
        assert abs(dth[n] - fd) <= 1e-8 * max(abs(fd), 1e-3), (n, dth[n], fd)
    for wall in range(2):
        def JT(x, wall=wall):
            T = list(Tw)
            T[wall] = x
            return _J(w, p, T, theta, fpost, hpost, nsteps, window, obj)
        fd = _richardson(JT, Tw[wall], 1e-3)
        assert abs(dTw[wall] - fd) <= 1e-8 * max(abs(fd), 1e-3), (wall, dTw[wall], fd)
    assert np.all(dth[w["flags"] == I.SOLID] == 0.0)


def test_cumulant_adjoint_at_unit_rate_equals_cm_kinds():
    # at s^H = 1 (k = 1/6) the mean is fully relaxed to u: every kind
    # collapses to h* = (H + Q) M(u), the same affine map, so the
    # Cumulants-1st gradient equals the CM-TRT one
    w, p = _plate_case(27, "cum1st")
    p.k = 1.0 / 6.0
    Tw = [1.0, 0.1]
    o, fpost, hpost = _setup(w, p, Tw)
    Jc, dc, dTc = o.adjoint(fpost, hpost, 6, (2, 6), ("surface", 0, 1.0), nwalls=2)
    p.hkind = O.KINDS["trt"]
    o2, _, _ = _setup(w, p, Tw)
    Jt, dt, dTt = o2.adjoint(fpost, hpost, 6, (2, 6), ("surface", 0, 1.0), nwalls=2)
    assert abs(Jc - Jt) < 1e-13 * abs(Jt)
    assert np.abs(dc - dt).max() < 1e-12 * np.abs(dt).max()
    assert np.abs(dTc - dTt).max() < 1e-12 * np.abs(dTt).max()


def test_objective_value_matches_surface_flux():
    # J over a one-level window at level 0 is the surface flux of Sec. 4.4
    w, p = _plate_case()
    o, fpost, hpost = _setup(w, p, [1.0, 0.1])
    J, _, _ = o.adjoint(fpost, hpost, 0, (0, 0), ("surface", 0, 1.0), nwalls=2, gradients=False)
    o2 = O.Oracle(p)
    o2.set_geometry(w["flags"], w["links"], nwalls=2)
    o2.set_wall_temperature(0, 1.0); o2.set_wall_temperature(1, 0.1)
    o2.set_theta(w["theta"])
    o2.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    assert abs(J - o2.surface_flux(0)) < 1e-14


# ---- the coupled f + h adjoint: gradients with respect to the flow --------
def _J_flow(w, p, Tw, fpost, hpost, nsteps, window, obj, F=None, u_in=None):
    q = O.make_params(nx=p.nx, ny=p.ny, nz=p.nz, qh=p.qh, hkind=p.hkind, periodic_x=bool(p.periodic_x), nu=p.nu,
                      k=p.k, F=tuple(p.F) if F is None else F, u_in=tuple(p.u_in) if u_in is None else u_in,
                      T_in=p.T_in, wall_bc=p.wall_bc)
    return _J(w, q, Tw, w["theta"], fpost, hpost, nsteps, window, obj)


def _replace(vec, d, x):
    v = list(vec)
    v[d] = x
    return tuple(v)


@pytest.mark.parametrize("case,kind,qh", [("plate", "trt", 27), ("plate", "cum1st", 27), ("channel", "trt", 27),
                                          ("channel", "srt", 7)])
def test_flow_adjoint_matches_finite_differences(case, kind, qh):
    # Eq. hydro_cu_collision + Eq. H_cm_collision (or H_cu_collision) coupled
    # through u: dJ/dF and dJ/du_in against Richardson-extrapolated central
    # differences of the nonlinear J; the theta and T_w gradients equal the
    # h-only adjoint's
    if case == "plate":
        w, p = _plate_case(qh, kind)
        Tw, obj, (nsteps, window) = [1.0, 0.1], ("surface", 1, 0.7), (8, (3, 8))
    else:
        w, p = _channel_case(qh, kind)
        Tw, obj, (nsteps, window) = [1.0], ("surface", 0, 1.0), (9, (3, 9))
    o, fpost, hpost = _setup(w, p, Tw)
    J, dth, dTw, dF, duin = o.adjoint_flow(fpost, hpost, nsteps, window, obj, nwalls=len(Tw))
    J0, dth0, dTw0 = o.adjoint(fpost, hpost, nsteps, window, obj, nwalls=len(Tw))
    assert abs(J - J0) <= 1e-14 * abs(J0)
    assert np.abs(dth - dth0).max() <= 1e-9 * np.abs(dth0).max()
    assert np.abs(dTw - dTw0).max() <= 1e-9 * np.abs(dTw0).max()
    scale = max(np.abs(dF).max(), np.abs(duin).max())
    for d in range(3):
        fd = _richardson(lambda x: _J_flow(w, p, Tw, fpost, hpost, nsteps, window, obj,
                                           F=_replace(p.F, d, x)), p.F[d], 2e-4)
        assert abs(dF[d] - fd) <= 1e-7 * max(abs(fd), 1e-3 * scale), (d, dF[d], fd)
    if case == "channel":
        for d in range(3):
            fd = _richardson(lambda x: _J_flow(w, p, Tw, fpost, hpost, nsteps, window, obj,
                                               u_in=_replace(p.u_in, d, x)), p.u_in[d], 2e-4)
            assert abs(duin[d] - fd) <= 1e-7 * max(abs(fd), 1e-3 * scale), (d, duin[d], fd)
    else:
        assert np.all(duin == 0.0)
