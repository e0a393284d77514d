"""The seeded input generators that feed both the oracle and the GPU path
(no method arithmetic in them): the counter generator against splitmix64's
published outputs, and the geometry builders against their definitions --
every wall link crosses the body at its q, every fluid-to-solid neighbour has
exactly one link, spheres of the porous bed keep their gap."""
import numpy as np

from oracle import oracle as O
from paper_2203_01316_gb300 import inputs as I

E27 = O.lattice(27)[0]


def test_splitmix64_published_outputs():
    # the first outputs of splitmix64 from state 0 (Steele, Lea and Flood,
    # OOPSLA 2014; Vigna's reference implementation)
    out = I.splitmix64(0, 3)
    assert [int(v) for v in out] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    # offsets continue the same sequence
    assert int(I.splitmix64(0, 1, offset=2)[0]) == 0x06C45D188009454F
    u = I.uniform(1234, 10000)
    assert 0.0 <= u.min() and u.max() < 1.0 and abs(u.mean() - 0.5) < 0.01


def _check_links(flags3, links, bodies):
    """Every link: fluid node, solid target, |x_b + q e_a - c| = R for its
    body, q in (0, 1]; every fluid->solid neighbour pair has exactly one
    link; links sorted by (node, dir)."""
    nz, ny, nx = flags3.shape
    node, dr, q, wall = links["node"], links["dir"], links["q"], links["wall"]
    assert np.all(np.diff(node.astype(np.int64) * 27 + dr) > 0)
    assert np.all((q > 0) & (q <= 1))
    x = node % nx
    y = (node // nx) % ny
    z = node // (nx * ny)
    flat = flags3.reshape(-1)
    assert np.all(flat[node] == I.FLUID)
    e = E27[dr]
    tx, ty, tz = x + e[:, 0], (y + e[:, 1]) % ny, (z + e[:, 2]) % nz
    assert np.all((tx >= 0) & (tx < nx))
    assert np.all(flat[tx + nx * (ty + ny * tz)] == I.SOLID)
    for w, (c, R) in enumerate(bodies):
        sel = wall == w
        p = np.stack([x[sel], y[sel], z[sel]], 1) + q[sel, None].astype(np.float64) * e[sel]
        d = p - c
        d[:, 1] -= ny * np.round(d[:, 1] / ny)
        d[:, 2] -= nz * np.round(d[:, 2] / nz)
        r = np.sqrt((d ** 2).sum(1))
        assert np.abs(r - R).max() < 1e-5 * max(R, 1.0), w
    # completeness
    have = set(zip(node.tolist(), dr.tolist()))
    want = set()
    fl = np.nonzero(flat == I.FLUID)[0]
    fx, fy, fz = fl % nx, (fl // nx) % ny, fl // (nx * ny)
    for a in range(1, 27):
        ex, ey, ez = E27[a]
        gx = fx + ex
        ok = (gx >= 0) & (gx < nx)
        t = gx[ok] + nx * ((fy[ok] + ey) % ny + ny * ((fz[ok] + ez) % nz))
        hit = flat[t] == I.SOLID
        want |= set(zip(fl[ok][hit].tolist(), [a] * int(hit.sum())))
    assert have == want


def test_heated_sphere_links():
    w = I.heated_sphere(40, 20, 18, D=8.0, cx=14.0, seed=3)
    nx, ny, nz = w["dims"]
    _check_links(w["flags"].reshape(nz, ny, nx), w["links"], [(w["centre"], w["D"] / 2)])
    assert np.all(w["flags"].reshape(nz, ny, nx)[:, :, 0] == I.INLET)
    assert np.all(w["flags"].reshape(nz, ny, nx)[:, :, nx - 1] == I.OUTLET)


def test_porous_bed_spheres_keep_their_gap():
    w = I.porous_bed(nx=96, ny=48, nz=40, n_spheres=12, dmin=6.0, dmax=10.0, gap=2.0, seed=5)
    nx, ny, nz = w["dims"]
    c, R = w["centres"], w["radii"]
    assert len(R) == 12 and np.all((R >= 3.0) & (R <= 5.0))
    for i in range(len(R)):
        assert R[i] + 2.0 + 1.0 <= c[i, 0] <= nx - 1 - (R[i] + 2.0 + 1.0) + 1e-9
        for j in range(i):
            d = c[i] - c[j]
            d[1] -= ny * round(d[1] / ny)
            d[2] -= nz * round(d[2] / nz)
            assert np.sqrt(d @ d) >= R[i] + R[j] + 2.0
    # links of touching-free spheres: each link's body is the nearest centre
    flags3 = w["flags"].reshape(nz, ny, nx)
    links = w["links"]
    node = links["node"]
    x, y, z = node % nx, (node // nx) % ny, node // (nx * ny)
    e = E27[links["dir"]]
    p = np.stack([x, y, z], 1) + links["q"][:, None].astype(np.float64) * e
    best = np.full(len(node), np.inf)
    for ci, Ri in zip(c, R):
        d = p - ci
        d[:, 1] -= ny * np.round(d[:, 1] / ny)
        d[:, 2] -= nz * np.round(d[:, 2] / nz)
        best = np.minimum(best, np.abs(np.sqrt((d ** 2).sum(1)) - Ri))
    assert best.max() < 1e-4
    assert np.count_nonzero(flags3 == I.SOLID) > 0


def test_plate_walls_and_confined_cylinder():
    w = I.plate_channel(nx=8, ny=9, nz=5, q_bottom=0.3, q_top=0.7)
    nx, ny, nz = w["dims"]
    flags3 = w["flags"].reshape(nz, ny, nx)
    L = w["links"]
    y = (L["node"] // nx) % ny
    assert np.all(np.where(y == 1, L["wall"] == 0, L["wall"] == 1))
    assert np.allclose(L["q"], np.where(y == 1, 0.3, 0.7))
    assert np.all(flags3[:, 0, :] == I.SOLID) and np.all(flags3[:, ny - 1, :] == I.SOLID)
    cc = I.confined_cylinder(0.1)
    nx, ny, nz = cc["dims"]
    f3 = cc["flags"].reshape(nz, ny, nx)
    assert nz == 1 and np.all(f3[0, 0, :] == I.MIRROR) and np.all(f3[0, ny - 1, :] == I.MIRROR)
    assert np.all(f3[0, 1:ny - 1, 0] == I.INLET) and np.all(f3[0, 1:ny - 1, nx - 1] == I.OUTLET)
