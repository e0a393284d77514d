"""Pins of the oracle's symmetry rows (the top and bottom symmetry planes of
the confined-cylinder case, Sec. 4.4; reading R15: specular reflection at
the plane halfway between a symmetry row and its neighbour row).

* One streaming step against the specular-reflection rule written out
  directly: an arrival whose source lies in a symmetry row comes from the
  node beside it in x and z with e_y reversed.
* Mirror symmetry: a periodic domain of height 2H started from a state that
  is symmetric about y = H - 1/2 stays symmetric, and its lower half is the
  H-row domain between two symmetry planes; the two runs agree to rounding.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01316_gb300 import inputs as I


def _flip_y(e):
    out = np.empty(len(e), int)
    for a, v in enumerate(e):
        out[a] = [b for b, w in enumerate(e) if w[0] == v[0] and w[1] == -v[1] and w[2] == v[2]][0]
    return out


@pytest.mark.parametrize("qh", [27, 7])
def test_stream_with_symmetry_rows_is_specular_reflection(qh):
    nx, ny, nz = 5, 7, 4
    N = nx * ny * nz
    flags = np.zeros((nz, ny, nx), np.uint8)
    flags[:, 0, :] = I.MIRROR
    flags[:, ny - 1, :] = I.MIRROR
    o = O.Oracle(O.make_params(nx=nx, ny=ny, nz=nz, qh=qh))
    o.set_geometry(flags.reshape(-1), None)
    rng = np.random.default_rng(3)
    fs = rng.uniform(0.0, 1.0, (27, N))
    hs = rng.uniform(0.0, 1.0, (qh, N))
    fs[:, flags.reshape(-1) == I.MIRROR] = 0.0
    hs[:, flags.reshape(-1) == I.MIRROR] = 0.0
    o.set_post(fs, hs)
    assert o.stream() == 0
    f, h = o.state()
    for pops, post, Q in ((f, fs, 27), (h, hs, qh)):
        e = O.lattice(Q)[0]
        fl = _flip_y(e)
        for z in range(nz):
            for y in range(1, ny - 1):
                for x in range(nx):
                    n = x + nx * (y + ny * z)
                    for a in range(Q):
                        sx, sy, sz = (x - e[a][0]) % nx, y - e[a][1], (z - e[a][2]) % nz
                        if sy in (0, ny - 1):
                            ref = post[fl[a], sx + nx * (y + ny * sz)]
                        else:
                            ref = post[a, sx + nx * (sy + ny * sz)]
                        assert pops[a, n] == ref, (Q, a, x, y, z)
        assert np.all(pops[:, flags.reshape(-1) == I.MIRROR] == 0.0)


def test_symmetry_rows_equal_half_of_a_mirror_symmetric_periodic_domain():
    nx, H, nz = 8, 6, 3
    ny_full = 2 * H
    rng = np.random.default_rng(5)
    # smooth random fields on the full grid, made symmetric about y = H - 1/2
    # (T, u_x, u_z even, u_y odd under y -> 2H - 1 - y)
    x = np.arange(nx)[None, None, :]
    y = np.arange(ny_full)[None, :, None]
    z = np.arange(nz)[:, None, None]
    def smooth(seed):
        r = np.random.default_rng(seed)
        a, b, c = r.uniform(-1, 1, 3)
        return (a * np.sin(2 * np.pi * x / nx + b) * np.cos(np.pi * (y + 0.5) / H)
                + c * np.cos(2 * np.pi * z / nz) * np.cos(2 * np.pi * (y + 0.5) / H))
    T = 0.8 + 0.1 * smooth(1)
    ux = 0.03 + 0.02 * smooth(2)
    uz = 0.01 * smooth(3)
    uy = 0.02 * np.sin(np.pi * (y + 0.5) / H) * np.cos(2 * np.pi * x / nx) * np.ones_like(T)
    mirror = ny_full - 1 - np.arange(ny_full)
    assert np.allclose(T, T[:, mirror, :]) and np.allclose(uy, -uy[:, mirror, :])
    rho = np.ones_like(T) + 0.01 * smooth(4)
    full = O.Oracle(O.make_params(nx=nx, ny=ny_full, nz=nz, nu=0.04, k=0.01, F=(1e-4, 0.0, 0.0)))
    Nf = nx * ny_full * nz
    full.set_geometry(np.zeros(Nf, np.uint8), None)
    full.init_fields(rho.reshape(-1), np.stack([ux, uy, uz]).reshape(-1), T.reshape(-1))
    # half domain: fluid rows 1..H hold full rows 0..H-1, symmetry rows 0 and H+1
    ny = H + 2
    flags = np.zeros((nz, ny, nx), np.uint8)
    flags[:, 0, :] = I.MIRROR
    flags[:, ny - 1, :] = I.MIRROR
    def half(a):
        out = np.ones((nz, ny, nx))
        out[:, 1:H + 1, :] = a[:, :H, :]
        return out
    half_o = O.Oracle(O.make_params(nx=nx, ny=ny, nz=nz, nu=0.04, k=0.01, F=(1e-4, 0.0, 0.0)))
    half_o.set_geometry(flags.reshape(-1), None)
    half_o.init_fields(half(rho).reshape(-1), np.stack([half(ux), half(uy), half(uz)]).reshape(-1),
                       half(T).reshape(-1))
    full.step(25)
    half_o.step(25)
    rf, uf, Tf = full.macros()
    rh, uh, Th = half_o.macros()
    sel = lambda a: a.reshape(-1, nz, ny, nx)[..., 1:H + 1, :] if a.ndim == 2 else a.reshape(nz, ny, nx)[:, 1:H + 1, :]
    low = lambda a: a.reshape(-1, nz, ny_full, nx)[..., :H, :] if a.ndim == 2 else a.reshape(nz, ny_full, nx)[:, :H, :]
    assert np.abs(sel(Th) - low(Tf)).max() < 1e-13
    assert np.abs(sel(uh) - low(uf)).max() < 1e-13
    assert np.abs(sel(rh) - low(rf)).max() < 1e-13
    # and the full run stayed symmetric
    Tf3 = Tf.reshape(nz, ny_full, nx)
    assert np.abs(Tf3 - Tf3[:, mirror, :]).max() < 1e-13


def test_symmetry_row_rules():
    nx, ny, nz = 6, 5, 2
    o = O.Oracle(O.make_params(nx=nx, ny=ny, nz=nz))
    flags = np.zeros((nz, ny, nx), np.uint8)
    flags[:, 0, :3] = I.MIRROR  # a partial row
    with pytest.raises(O.OracleError):
        o.set_geometry(flags.reshape(-1), None)
    flags[:, 0, :] = I.MIRROR
    flags[:, 2, :] = I.MIRROR  # not a boundary row
    with pytest.raises(O.OracleError):
        o.set_geometry(flags.reshape(-1), None)
    flags[:, 2, :] = I.FLUID
    flags[0, 1, 2] = I.SOLID  # the mirrored node is solid
    with pytest.raises(O.OracleError):
        o.set_geometry(flags.reshape(-1), None)
    flags[0, 1, 2] = I.FLUID
    o.set_geometry(flags.reshape(-1), None)
