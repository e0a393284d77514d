"""lbm_step_record_pre records what the coupled adjoint reads of a level's
pre-collision arrivals: the ten raw moments of f (the cumulant collision of
Eq. hydro_cu_collision reads f only through its density, momentum and second
moments), the h arrivals, and with the Zou-He inlet the inlet nodes' full f
arrivals after the rule (Sec. 4.4).  Checked, in FP64 storage, against the
oracle's own streaming (Eq. IBB, Eq. IABB, the planes, symmetry rows, the
Zou-He rule) of the same post-collision state, at every node that collides."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01316_gb300 import inputs as I

from _cases import make_pair, small_channel

pytestmark = pytest.mark.gpu


def _moments(g):
    """The ten raw moments of populations g[27, N], in the record's order."""
    e = O.lattice(27)[0].astype(np.float64)
    ex, ey, ez = e[:, 0:1], e[:, 1:2], e[:, 2:3]
    return np.stack([g.sum(0), (ex * g).sum(0), (ey * g).sum(0), (ez * g).sum(0), (ex * ex * g).sum(0),
                     (ey * ey * g).sum(0), (ez * ez * g).sum(0), (ex * ey * g).sum(0), (ex * ez * g).sum(0),
                     (ey * ez * g).sum(0)])


def _check(s, o, flags, rho0, T_ref, qh, zou_he):
    import torch
    N = s.N
    nx, ny, nz = s.nx, s.ny, s.nz
    F, H = s.flow_record_size()
    assert F == 10 * N + (27 * ny * nz if zou_he else 0) and H == qh * N
    f, h = s.populations()
    frec = torch.full((F,), float("nan"), dtype=torch.float64, device="cuda")
    hrec = torch.full((H,), float("nan"), dtype=torch.float64, device="cuda")
    s.step_record_pre(1, frec, hrec)
    o.set_post(f, h)
    o.stream()
    g, gh = o.state()
    w27 = O.lattice(27)[1]
    wh = O.lattice(qh)[1]
    gd = g - w27[:, None] * rho0
    ghd = gh - wh[:, None] * T_ref
    flags = np.asarray(flags)
    collide = (flags == I.FLUID) | (flags == I.OUTLET) | ((flags == I.INLET) if zou_he else False)
    rec = frec.cpu().numpy()
    m_gpu = rec[:10 * N].reshape(10, N)[:, collide]
    m_ref = _moments(gd)[:, collide]
    scale = np.abs(m_ref).max()
    assert np.abs(m_gpu - m_ref).max() <= 1e-12 * scale
    h_gpu = hrec.cpu().numpy().reshape(qh, N)[:, collide]
    assert np.abs(h_gpu - ghd[:, collide]).max() <= 1e-12 * np.abs(ghd[:, collide]).max()
    if zou_he:
        inl = rec[10 * N:].reshape(27, ny * nz)
        rows = np.arange(ny * nz)
        nodes = nx * rows  # x = 0, row y + ny z
        at_inlet = flags[nodes] == I.INLET
        ref = gd[:, nodes[at_inlet]]
        assert at_inlet.sum() > 0
        assert np.abs(inl[:, at_inlet] - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("qh", [27, 7])
def test_records_match_the_oracle_arrivals_channel(qh):
    w = small_channel()
    s, o = make_pair(w, nu=0.03, k=2e-3, qh=qh, storage="f64", T_ref=0.2)
    s.step(3)
    _check(s, o, w["flags"], 1.0, 0.2, qh, zou_he=False)
    s.close()


def test_records_match_the_oracle_arrivals_zou_he_and_symmetry_rows():
    from paper_2203_01316_gb300 import Solver
    w = I.confined_cylinder(0.2, seed=4)
    nx, ny, nz = w["dims"]
    nu, k = 0.03, 0.003
    s = Solver(nx, ny, nz, nu=nu, k=k, storage="f64", periodic_x=False, T_ref=w["T_in"], inlet_bc="zou_he")
    s.set_geometry(w["flags"], w["links"], n_walls=1)
    s.set_bc(0, w["T_cyl"])
    s.set_inlet(w["u_in"], w["T_in"])
    s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    o = O.Oracle(O.make_params(nx=nx, ny=ny, nz=nz, periodic_x=False, nu=nu, k=k, u_in=w["u_in"],
                               T_in=w["T_in"], inlet_bc="zou_he"))
    o.set_geometry(w["flags"], w["links"], nwalls=1)
    o.set_wall_temperature(0, w["T_cyl"])
    s.step(5)
    _check(s, o, w["flags"], 1.0, w["T_in"], 27, zou_he=True)
    s.close()
