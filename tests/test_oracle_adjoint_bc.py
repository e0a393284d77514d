"""The oracle's adjoints with the boundary rules of the Sec. 4.4 confined
cylinder: symmetry rows (reading R15) and the Zou-He inlet (reading R20).

A symmetry node pushes its mirrored node's post-collision populations with
e_y reversed, so its transpose adds what the symmetry node's pushes receive
to the mirrored node's reversed populations.  The Zou-He rule is affine in a
node's arrivals for fixed u_in; its transpose is A^T with A read off the
rule's own images of unit arrivals, and the inlet nodes then collide like
fluid nodes.  Each is checked against differences of the nonlinear J:
central differences in theta and T_w (J is affine in them for the
central-moment kinds, so the difference has no truncation error) and
Richardson-extrapolated ones in F and u_in (1e-7 of the largest entry, as
for the other coupled-adjoint pins)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01316_gb300 import inputs as I


def _case(bc, qh=27, kind="trt", seed=21, nx=14, ny=9, nz=8):
    """A cylinder (wall 0) in a channel with symmetry rows ("mirror"), a
    Zou-He inlet and outlet ("zou_he") or both ("both")."""
    mirror = bc in ("mirror", "both")
    zou_he = bc in ("zou_he", "both")
    flags = I.channel_flags(nx, ny, nz, periodic_x=not zou_he)
    links = I.add_spheres(flags, [(5.6, 4.3, 3.5)], [1.7], wall_ids=[0])
    if mirror:
        flags[:, 0, :] = I.MIRROR
        flags[:, ny - 1, :] = I.MIRROR
    flags = flags.reshape(-1)
    N = flags.size
    u = I.uniform(seed, 3 * N, -0.02, 0.02).reshape(3, N)
    u[0] += 0.03
    w = {"dims": (nx, ny, nz), "flags": flags, "links": links, "nwalls": 1, "periodic_x": not zou_he,
         "rho": 1.0 + I.uniform(seed + 1, N, -0.01, 0.01), "u": u, "T": I.uniform(seed + 2, N, 0.2, 1.0),
         "theta": I.uniform(seed + 3, N, 0.0, 1e-3)}
    w["theta"][flags == I.SOLID] = 0.0
    w["theta"][flags == I.MIRROR] = 0.0
    p = dict(nx=nx, ny=ny, nz=nz, qh=qh, hkind=kind, periodic_x=not zou_he, nu=0.05, k=0.01,
             F=(2e-5, 1e-5, 0.0), u_in=(0.04, 0.003, -0.002) if zou_he else (0.0, 0.0, 0.0), T_in=0.3,
             inlet_bc="zou_he" if zou_he else "equilibrium")
    return w, p


def _oracle(w, p, Tw, theta=None, **over):
    q = dict(p)
    q.update(over)
    o = O.Oracle(O.make_params(**q))
    o.set_geometry(w["flags"], w["links"], nwalls=1)
    o.set_wall_temperature(0, Tw)
    o.set_theta(w["theta"] if theta is None else theta)
    return o


def _start(w, p, Tw):
    o = _oracle(w, p, Tw)
    o.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    o.step(3)
    return o.post()


def _richardson(Jof, x0, eps):
    d1 = (Jof(x0 + eps) - Jof(x0 - eps)) / (2 * eps)
    d2 = (Jof(x0 + eps / 2) - Jof(x0 - eps / 2)) / eps
    return (4 * d2 - d1) / 3


def _probe_nodes(w):
    """Fluid nodes next to the symmetry rows, at and next to the inlet, next
    to the cylinder, at the outlet corners (whose copy rule reads the
    symmetry rows), and one in the bulk."""
    nx, ny, nz = w["dims"]
    fl = w["flags"].reshape(nz, ny, nx)
    cand = [(1, 1, 1), (0, 1, 4), (0, 0, 3), (1, 0, 7), (0, 1, 1), (0, 7, 9), (1, 4, 11), (0, 3, 3),
            (0, 1, nx - 1), (2, ny - 2, nx - 1), (1, 1, nx - 2)]
    return [I.node_index(x, y, z, nx, ny) for z, y, x in cand if fl[z, y, x] in (I.FLUID, I.INLET)]


@pytest.mark.parametrize("bc", ["mirror", "zou_he", "both"])
@pytest.mark.parametrize("qh,kind,obj", [(27, "trt", ("surface", 0, 1.0)), (7, "srt", ("section", 9, 1.0)),
                                         (27, "cum1st", ("surface", 0, 0.7))])
def test_h_adjoint_with_boundary_rules(bc, qh, kind, obj):
    w, p = _case(bc, qh, kind)
    Tw = 0.9
    fpost, hpost = _start(w, p, Tw)
    nsteps, window = 9, (3, 9)
    o = _oracle(w, p, Tw)
    J, dth, dTw = o.adjoint(fpost, hpost, nsteps, window, obj)

    def J_of(theta=None, T=Tw):
        return _oracle(w, p, T, theta).adjoint(fpost, hpost, nsteps, window, obj, gradients=False)[0]

    assert J == pytest.approx(J_of(), rel=1e-14)
    scale = np.abs(dth).max()
    assert scale > 0
    diff = _richardson if kind == "cum1st" else lambda f, x, e: (f(x + e) - f(x - e)) / (2 * e)
    for n in _probe_nodes(w):
        def Jt(x, n=n):
            th = w["theta"].copy()
            th[n] = x
            return J_of(theta=th)
        fd = diff(Jt, w["theta"][n], 1e-2 if kind != "cum1st" else 1e-3)
        assert abs(dth[n] - fd) <= 1e-8 * max(abs(fd), 1e-3 * scale), (n, dth[n], fd)
    fd = diff(lambda T: J_of(T=T), Tw, 1e-2 if kind != "cum1st" else 1e-3)
    assert abs(dTw[0] - fd) <= 1e-8 * max(abs(fd), 1e-6), (dTw[0], fd)


@pytest.mark.parametrize("bc", ["mirror", "zou_he", "both"])
@pytest.mark.parametrize("qh,kind,obj", [(27, "trt", ("surface", 0, 1.0)), (27, "trt", ("force", 0, 1.0, 0)),
                                         (7, "cum1st", ("force", 0, 1.0, 1))])
def test_coupled_adjoint_with_boundary_rules(bc, qh, kind, obj):
    w, p = _case(bc, qh, kind)
    Tw = 0.9
    fpost, hpost = _start(w, p, Tw)
    nsteps, window = 8, (3, 8)
    o = _oracle(w, p, Tw)
    J, dth, dTw, dF, duin = o.adjoint_flow(fpost, hpost, nsteps, window, obj)
    if obj[0] == "surface":  # theta and T_w as in the h-only adjoint
        J0, dth0, dTw0 = _oracle(w, p, Tw).adjoint(fpost, hpost, nsteps, window, obj)
        assert abs(J - J0) <= 1e-14 * abs(J0)
        assert np.abs(dth - dth0).max() <= 1e-9 * np.abs(dth0).max()
        assert abs(dTw[0] - dTw0[0]) <= 1e-9 * abs(dTw0[0])

    def J_of(**over):
        return _oracle(w, p, Tw, **over).adjoint(fpost, hpost, nsteps, window, obj, gradients=False)[0]

    scale = max(np.abs(dF).max(), np.abs(duin).max())
    assert scale > 0
    for d in range(3):
        fd = _richardson(lambda x: J_of(F=tuple(x if i == d else p["F"][i] for i in range(3))), p["F"][d], 2e-4)
        assert abs(dF[d] - fd) <= 1e-7 * max(abs(fd), 1e-3 * scale), ("F", d, dF[d], fd)
    if bc == "mirror":
        assert np.all(duin == 0.0)
        return
    for d in range(3):
        fd = _richardson(lambda x: J_of(u_in=tuple(x if i == d else p["u_in"][i] for i in range(3))),
                         p["u_in"][d], 2e-4)
        assert abs(duin[d] - fd) <= 1e-7 * max(abs(fd), 1e-3 * scale), ("u_in", d, duin[d], fd)
    assert abs(duin[0]) > 1e-3 * scale  # the inlet velocity matters
