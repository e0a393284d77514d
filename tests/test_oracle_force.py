"""Pins of the oracle's momentum-exchange wall force (reading R21: not in the
paper; Ladd 1994, Mei et al. 2002) and of the coupled adjoint of an objective
built on it.

* Momentum balance, exact at every step in a periodic box: the collision adds
  F to the momentum of every fluid node (Eq. hydro_cu_collision with the body
  force) and the wall links are the only other place momentum leaves, so
  sum over walls of the force = N_fluid F - (P^{k+1} - P^k), P the momentum
  of the pre-collision state.  This holds whatever Eq. IBB returns, so it
  checks the force's own sum (a dropped link, a wrong sign, a wrong IBB
  branch) against the step, not against itself.
* A closed body in fluid at rest: the force vanishes.
* Gradients of a force objective (adjoint_flow) against Richardson
  differences of the nonlinear J, and the J value against wall_force."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01316_gb300 import inputs as I


def _box_case(seed=11, wall_bc="iabb", nx=12, ny=10, nz=8):
    """Periodic box with plates (walls 1, 2; q 0.3 / 0.7) and a sphere (wall 0)."""
    flags = I.channel_flags(nx, ny, nz, periodic_x=True)
    plates = I.plate_walls(flags, 0.3, 0.7, wall_bottom=1, wall_top=2)
    sphere = I.add_spheres(flags, [(5.3, 4.8, 3.6)], [2.1], wall_ids=[0])
    links = I.merge_links(plates, sphere)
    flags = flags.reshape(-1)
    # links of fluid nodes only (the sphere may have covered plate-link nodes)
    keep = flags[links["node"]] == I.FLUID
    links = {k: v[keep] for k, v in links.items()}
    N = flags.size
    u = I.uniform(seed, 3 * N, -0.04, 0.04).reshape(3, N)
    u[:, flags == I.SOLID] = 0.0
    w = {"dims": (nx, ny, nz), "flags": flags, "links": links, "nwalls": 3, "periodic_x": True,
         "rho": 1.0 + I.uniform(seed + 1, N, -0.02, 0.02), "u": u,
         "T": I.uniform(seed + 2, N, 0.2, 1.0), "theta": np.zeros(N)}
    p = O.make_params(nx=nx, ny=ny, nz=nz, qh=27, hkind="trt", nu=0.05, k=0.01, F=(3e-4, -1e-4, 2e-4),
                      wall_bc=wall_bc)
    return w, p


def _oracle(w, p):
    o = O.Oracle(p)
    o.set_geometry(w["flags"], w["links"], nwalls=w["nwalls"])
    o.set_theta(w["theta"])
    o.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    return o


def _momentum(o):
    f, _ = o.state()
    e = O.lattice(27)[0]
    return e.T.astype(np.float64) @ f.sum(axis=1)


@pytest.mark.parametrize("wall_bc", ["iabb", "abb"])
def test_wall_force_balances_momentum(wall_bc):
    w, p = _box_case(wall_bc=wall_bc)
    o = _oracle(w, p)
    n_fluid = int(np.count_nonzero(w["flags"] == I.FLUID))
    F = np.array(p.F[:3])
    for _ in range(4):
        P0 = _momentum(o)
        Fw = sum(o.wall_force(i) for i in range(3))
        o.step(1)
        P1 = _momentum(o)
        expect = n_fluid * F - (P1 - P0)
        assert np.abs(Fw - expect).max() <= 1e-12 * max(np.abs(expect).max(), 1.0), (Fw, expect)
        assert np.abs(Fw).max() > 1e-3  # the walls do take momentum


def test_wall_force_of_closed_body_at_rest_vanishes():
    w, p = _box_case()
    N = w["flags"].size
    w["rho"], w["u"] = np.ones(N), np.zeros((3, N))
    p = O.make_params(nx=p.nx, ny=p.ny, nz=p.nz, qh=27, hkind="trt", nu=0.05, k=0.01)
    o = _oracle(w, p)
    F = o.wall_force(0)
    assert np.abs(F).max() <= 1e-14
    # the plates alone (not closed: their links only point outward) take the
    # reference pressure 2 sum w_a e_a rho0 each, equal and opposite
    Fb, Ft = o.wall_force(1), o.wall_force(2)
    assert abs(Fb[1]) > 1e-2 and np.abs(Fb + Ft).max() <= 1e-12


def _J_force(w, p, fpost, hpost, nsteps, window, obj, F=None):
    q = O.make_params(nx=p.nx, ny=p.ny, nz=p.nz, qh=p.qh, hkind=p.hkind, periodic_x=bool(p.periodic_x), nu=p.nu,
                      k=p.k, F=tuple(p.F) if F is None else F, wall_bc=p.wall_bc)
    o = _oracle(w, q)
    J, _, _ = o.adjoint(fpost, hpost, nsteps, window, obj, nwalls=w["nwalls"], gradients=False)
    return J


def _richardson(Jof, x0, eps):
    d1 = (Jof(x0 + eps) - Jof(x0 - eps)) / (2 * eps)
    d2 = (Jof(x0 + eps / 2) - Jof(x0 - eps / 2)) / eps
    return (4 * d2 - d1) / 3


def test_force_objective_value_matches_wall_force():
    w, p = _box_case()
    o = _oracle(w, p)
    fpost, hpost = o.post()
    Fw = o.wall_force(0)
    for c in range(3):
        J, _, _ = o.adjoint(fpost, hpost, 0, (0, 0), ("force", 0, 2.0, c), nwalls=3, gradients=False)
        assert J == pytest.approx(2.0 * Fw[c], rel=1e-14, abs=1e-16)


def test_force_objective_needs_the_coupled_adjoint():
    w, p = _box_case()
    o = _oracle(w, p)
    fpost, hpost = o.post()
    with pytest.raises(O.OracleError, match="adjoint_flow"):
        o.adjoint(fpost, hpost, 2, (0, 2), ("force", 0, 1.0, 0), nwalls=3)


@pytest.mark.parametrize("wall,comp,wall_bc", [(0, 0, "iabb"), (0, 1, "iabb"), (2, 1, "iabb"), (0, 2, "abb")])
def test_force_objective_gradient_matches_finite_differences(wall, comp, wall_bc):
    # the drag-type objective sum_k F_comp(s^k): only f enters it, so dJ/dtheta
    # and dJ/dT_w vanish and dJ/dF runs through the f adjoint alone
    w, p = _box_case(wall_bc=wall_bc)
    o = _oracle(w, p)
    fpost, hpost = o.post()
    nsteps, window, obj = 7, (2, 7), ("force", wall, 0.8, comp)
    J, dth, dTw, dF, duin = o.adjoint_flow(fpost, hpost, nsteps, window, obj, nwalls=3)
    assert np.all(dth == 0.0) and np.all(dTw == 0.0) and np.all(duin == 0.0)
    J0 = _J_force(w, p, fpost, hpost, nsteps, window, obj)
    assert abs(J - J0) <= 1e-14 * abs(J0)
    scale = np.abs(dF).max()
    assert scale > 1.0
    for d in range(3):
        fd = _richardson(lambda x: _J_force(w, p, fpost, hpost, nsteps, window, obj,
                                            F=tuple(x if i == d else p.F[i] for i in range(3))), p.F[d], 2e-4)
        assert abs(dF[d] - fd) <= 1e-7 * max(abs(fd), 1e-3 * scale), (d, dF[d], fd)
