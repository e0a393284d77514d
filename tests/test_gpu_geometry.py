"""lbm_build_spheres builds the flags and wall links of spheres in a channel on
the device.  They must equal, bit for bit (flags, node, direction, wall and
the float bits of q), the oracle's own node-by-node construction
(orc_build_spheres, pinned in test_oracle_geometry) on seeded sphere sets
that cross the periodic y and z faces, and the numpy construction of the
512x256x256 porous bed (33.5M nodes, 200 spheres) at full size; a geometry
built on the device then steps like the same geometry handed in."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01316_gb300 import inputs as I

from test_oracle_geometry import _spheres

pytestmark = pytest.mark.gpu


def _same_links(a, b):
    for key in ("node", "dir", "wall"):
        assert np.array_equal(np.asarray(a[key], np.int32), np.asarray(b[key], np.int32)), key
    assert np.array_equal(np.asarray(a["q"], np.float32).view(np.uint32),
                          np.asarray(b["q"], np.float32).view(np.uint32))


@pytest.mark.parametrize("seed,dims", [(1, (30, 20, 18)), (4, (40, 24, 22)), (7, (37, 19, 23))])
def test_device_geometry_equals_the_oracle(seed, dims):
    from paper_2203_01316_gb300 import Solver
    nx, ny, nz = dims
    c, r = _spheres(seed, 4, nx, ny, nz, 2.0, 4.5)
    walls = np.arange(4) % 2
    s = Solver(nx, ny, nz, nu=0.03, k=2e-3, storage="f32", periodic_x=False)
    flags = s.build_spheres(c, r, wall_ids=walls, n_walls=2)
    fo, Lo = O.build_spheres(nx, ny, nz, c, r, wall_ids=walls)
    assert np.array_equal(flags, fo)
    _same_links(s.links(), Lo)
    s.close()


def test_device_geometry_steps_like_the_given_geometry():
    from paper_2203_01316_gb300 import Solver
    w = I.heated_sphere(48, 24, 24, D=9.0, cx=14.0, seed=3, u_in=0.03, T_in=0.0)
    nx, ny, nz = w["dims"]
    a = Solver(nx, ny, nz, nu=0.03, k=2e-3, storage="f32", periodic_x=False)
    b = Solver(nx, ny, nz, nu=0.03, k=2e-3, storage="f32", periodic_x=False)
    a.set_geometry(w["flags"], w["links"], n_walls=1)
    b.build_spheres([w["centre"]], [w["D"] / 2.0])
    for s in (a, b):
        s.set_bc(0, 1.0)
        s.set_inlet(w["u_in"], w["T_in"])
        s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
        s.step(20)
    fa, ha = a.populations()
    fb, hb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ha, hb)
    a.close()
    b.close()


def test_porous_bed_full_size_equals_numpy():
    from paper_2203_01316_gb300 import Solver
    w = I.porous_bed(seed=1234)
    nx, ny, nz = w["dims"]
    s = Solver(nx, ny, nz, nu=0.01, Pr=1000.0, lat_h=7, storage="f32", periodic_x=False)
    flags = s.build_spheres(w["centres"], w["radii"])
    assert np.array_equal(flags, np.asarray(w["flags"], np.uint8))
    _same_links(s.links(), w["links"])
    s.close()
