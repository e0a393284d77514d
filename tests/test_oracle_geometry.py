"""The oracle's sphere geometry builder (orc_build_spheres: flags and wall
links with Sec. 3's q, the fraction of the link at which the wall lies),
pinned on the CPU against what the geometry fixes:

* every link's wall point x_b + q e_a lies on the sphere (|.| = R to float
  rounding of q), q in (0, 1], the node fluid and the target solid;
* completeness: every fluid node's neighbour inside a ball (x inside the box)
  is a link, and nothing else is;
* a sphere centred on a node gives links symmetric under the 48 symmetries
  of the cube;
* it equals the workload generator's independent numpy construction
  (inputs.add_spheres) bit for bit, periodic images in y and z included."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01316_gb300 import inputs as I

E = O.lattice(27)[0]


def _spheres(seed, n, nx, ny, nz, rmin, rmax):
    """Seeded non-touching spheres that may cross the y and z faces."""
    rng = np.random.default_rng(seed)
    cs, rs = [], []
    while len(rs) < n:
        R = rng.uniform(rmin, rmax)
        c = np.array([rng.uniform(R + 2, nx - R - 3), rng.uniform(0, ny), rng.uniform(0, nz)])
        ok = True
        for c2, R2 in zip(cs, rs):
            d = c - c2
            d[1] -= ny * np.round(d[1] / ny)
            d[2] -= nz * np.round(d[2] / nz)
            if np.linalg.norm(d) < R + R2 + 2:
                ok = False
        if ok:
            cs.append(c)
            rs.append(R)
    return np.array(cs), np.array(rs)


def _xyz(n, nx, ny):
    return n % nx, (n // nx) % ny, n // (nx * ny)


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_links_lie_on_the_spheres_and_are_complete(seed):
    nx, ny, nz = 30, 20, 18
    c, r = _spheres(seed, 4, nx, ny, nz, 2.5, 4.5)
    flags, L = O.build_spheres(nx, ny, nz, c, r, wall_ids=np.arange(4) % 2)
    assert len(L["node"]) > 0
    assert np.all(np.diff(L["node"].astype(np.int64) * 32 + L["dir"]) > 0)  # sorted, unique
    q = L["q"].astype(np.float64)
    assert np.all((q > 0) & (q <= 1))
    x, y, z = _xyz(L["node"], nx, ny)
    assert np.all(flags[L["node"]] == I.FLUID)
    seen = set()
    for k in range(len(q)):
        e = E[L["dir"][k]]
        p = np.array([x[k], y[k], z[k]], float) + q[k] * e
        # the wall point is on one ball (some image in y and z)
        best = np.inf
        for i in range(len(r)):
            for ky in (-1, 0, 1):
                for kz in (-1, 0, 1):
                    d = p - (c[i] + [0, ky * ny, kz * nz])
                    err = abs(np.linalg.norm(d) - r[i])
                    if err < best:
                        best, wi = err, i
        assert best <= 1e-5 * max(r), (k, best)
        assert L["wall"][k] == wi % 2
        seen.add((int(L["node"][k]), int(L["dir"][k])))
    # completeness by brute force over every fluid node and direction
    for n in np.flatnonzero(flags == I.FLUID):
        xn, yn, zn = _xyz(n, nx, ny)
        for a in range(1, 27):
            xt = xn + E[a][0]
            if xt < 0 or xt >= nx:
                continue
            t = xt + nx * (((yn + E[a][1]) % ny) + ny * ((zn + E[a][2]) % nz))
            assert (flags[t] == I.SOLID) == ((int(n), a) in seen)


def test_node_centred_sphere_is_cube_symmetric():
    n = 21
    c = np.array([[10.0, 10.0, 10.0]])
    flags, L = O.build_spheres(n, n, n, c, [5.3], periodic_x=True)
    x, y, z = _xyz(L["node"], n, n)
    table = {}
    for k in range(len(L["q"])):
        d = (x[k] - 10, y[k] - 10, z[k] - 10)
        table[(d, tuple(E[L["dir"][k]]))] = L["q"][k]
    import itertools
    for perm in itertools.permutations(range(3)):
        for sign in itertools.product((-1, 1), repeat=3):
            for (d, e), q in table.items():
                d2 = tuple(sign[i] * d[perm[i]] for i in range(3))
                e2 = tuple(sign[i] * e[perm[i]] for i in range(3))
                assert table[(d2, e2)] == q


@pytest.mark.parametrize("seed", [4, 5])
def test_equals_the_numpy_construction(seed):
    nx, ny, nz = 40, 24, 22
    c, r = _spheres(seed, 5, nx, ny, nz, 2.0, 5.0)
    walls = np.arange(5) % 3
    fo, Lo = O.build_spheres(nx, ny, nz, c, r, wall_ids=walls)
    fl = I.channel_flags(nx, ny, nz)
    Ln = I.add_spheres(fl, c, r, wall_ids=walls)
    assert np.array_equal(fo, fl.reshape(-1))
    for key in ("node", "dir", "wall"):
        assert np.array_equal(Lo[key], np.asarray(Ln[key], np.int32)), key
    assert np.array_equal(Lo["q"].view(np.uint32), np.asarray(Ln["q"], np.float32).view(np.uint32))
