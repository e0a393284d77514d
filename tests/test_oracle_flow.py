"""Pins of the oracle's streaming, boundary conditions and time evolution:
brute-force index checks, the special cases the paper names (IBB at q=1/2
is bounce-back, IABB at q=1/2 is anti-bounce-back), invariant states, and
closed-form solutions (shear-wave and temperature-mode decay, the Gaussian
hill of Sec. 4.1, steady conduction and Poiseuille flow between walls)."""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01316_gb300 import inputs as I

CS2 = 1.0 / 3.0


def _sim(nx, ny, nz, flags=None, links=None, nwalls=1, **kw):
    p = O.make_params(nx=nx, ny=ny, nz=nz, **kw)
    o = O.Oracle(p)
    if flags is None:
        flags = np.zeros(nx * ny * nz, np.uint8)
    o.set_geometry(np.asarray(flags).reshape(-1), links, nwalls=nwalls)
    return o


def test_streaming_brute_force_periodic():
    nx, ny, nz = 4, 3, 5
    N = nx * ny * nz
    o = _sim(nx, ny, nz)
    fs = np.arange(27 * N, dtype=float).reshape(27, N)
    hs = -np.arange(27 * N, dtype=float).reshape(27, N)
    o.set_post(fs, hs)
    assert o.stream() == 0
    f, h = o.state()
    e = I.E27
    for a in range(27):
        for n in range(N):
            x, y, z = n % nx, (n // nx) % ny, n // (nx * ny)
            t = ((x + e[a, 0]) % nx) + nx * (((y + e[a, 1]) % ny) + ny * ((z + e[a, 2]) % nz))
            assert f[a, t] == fs[a, n] and h[a, t] == hs[a, n]


def test_planes_inlet_and_outlet():
    nx, ny, nz = 6, 3, 2
    N = nx * ny * nz
    flags = I.channel_flags(nx, ny, nz, periodic_x=False).reshape(-1)
    o = _sim(nx, ny, nz, flags, periodic_x=False, u_in=(0.02, 0.0, 0.0), T_in=0.3)
    fs = np.arange(27 * N, dtype=float).reshape(27, N) + 1.0
    o.set_post(fs, fs.copy())
    assert o.stream() == 0
    f, h = o.state()
    e = I.E27
    feq = O.equilibrium(1.0, [0.02, 0, 0])
    heq = O.equilibrium(0.3, [0.02, 0, 0])
    for n in range(N):
        x, y, z = n % nx, (n // nx) % ny, n // (nx * ny)
        if x == 0:
            assert np.array_equal(f[:, n], feq) and np.array_equal(h[:, n], heq)
        if x == nx - 1:
            for a in range(27):
                if e[a, 0] < 0:
                    src = (nx - 1) + nx * (((y - e[a, 1]) % ny) + ny * ((z - e[a, 2]) % nz))
                    assert f[a, n] == fs[a, src]


def _plate(ny, qb, qt, nx=1, nz=1):
    flags = I.channel_flags(nx, ny, nz, periodic_x=True)
    links = I.plate_walls(flags, qb, qt)
    return flags.reshape(-1), links


@pytest.mark.parametrize("qb,qt", [(0.5, 0.5), (0.3, 0.8)])
def test_wall_link_formulas(qb, qt):
    # Eq. (IBB) and Eq. (IABB) applied link by link; at q = 1/2 they are BB/ABB
    ny = 6
    flags, links = _plate(ny, qb, qt)
    o = _sim(1, ny, 1, flags, links, nwalls=2)
    Tw = (0.9, 0.2)
    for w in (0, 1):
        o.set_wall_temperature(w, Tw[w])
    rng = np.random.default_rng(20)
    fs = rng.uniform(0.1, 1.0, (27, ny))
    hs = rng.uniform(0.1, 1.0, (27, ny))
    o.set_post(fs, hs)
    assert o.stream() == 0
    f, h = o.state()
    e, w, opp, _ = O.lattice(27)
    for n, a, q, wall in zip(links["node"], links["dir"], links["q"], links["wall"]):
        q = float(q)
        ab = opp[a]
        xf = n - e[a, 1]  # 1-wide in x and z: node index is y
        if q <= 0.5:
            fe = 2 * q * fs[a, n] + (1 - 2 * q) * fs[a, xf]
            he = -(2 * q * hs[a, n] + (1 - 2 * q) * hs[a, xf]) + 2 * w[a] * Tw[wall]
        else:
            fe = (fs[a, n] + (2 * q - 1) * fs[ab, n]) / (2 * q)
            he = (-hs[a, n] + (2 * q - 1) * hs[ab, n] + 2 * w[a] * Tw[wall]) / (2 * q)
        assert abs(f[ab, n] - fe) < 1e-15 and abs(h[ab, n] - he) < 1e-15
        if q == 0.5:
            assert f[ab, n] == fs[a, n]                                     # BB
            assert abs(h[ab, n] - (-hs[a, n] + 2 * w[a] * Tw[wall])) < 1e-15  # ABB


@pytest.mark.parametrize("Q", [27, 7])
def test_uniform_state_with_walls_is_invariant(Q):
    ny = 7
    flags, links = _plate(ny, 0.3, 0.8, nx=2, nz=2)
    o = _sim(2, ny, 2, flags, links, nwalls=2, qh=Q, k=1e-3)
    for w in (0, 1):
        o.set_wall_temperature(w, 0.7)
    N = 4 * ny
    o.init_fields(np.ones(N), np.zeros((3, N)), np.full(N, 0.7))
    f0, h0 = o.state()
    o.step(20)
    f1, h1 = o.state()
    fl = flags != I.SOLID
    assert np.allclose(f1[:, fl], f0[:, fl], atol=1e-15)
    assert np.allclose(h1[:, fl], h0[:, fl], atol=1e-15)


def test_periodic_totals_conserved():
    w = I.periodic_tgv(8)
    o = _sim(8, 8, 8, hkind="trt")
    o.init_fields(w["rho"], w["u"], w["T"])
    m0, e0 = o.balances()
    o.step(5)
    m1, e1 = o.balances()
    assert abs(m1 - m0) < 1e-11 and abs(e1 - e0) < 1e-11


def test_shear_wave_decay_rate():
    # u_y = A sin(2 pi x / L) decays as exp(-nu k^2 t) (Navier-Stokes)
    L, A, nu = 32, 1e-4, 0.02
    kx = 2 * math.pi / L
    x = np.arange(L)
    u = np.zeros((3, L))
    u[1] = A * np.sin(kx * x)
    o = _sim(L, 1, 1, nu=nu)
    o.init_fields(np.ones(L), u, np.ones(L))
    amps = []
    for t in (50, 350):
        o.step(t - (50 if amps else 0))
        _, uu, _ = o.macros()
        amps.append(2.0 / L * np.sum(uu[1] * np.sin(kx * x)))
    rate = math.log(amps[0] / amps[1]) / 300.0
    assert abs(rate / (nu * kx * kx) - 1.0) < 0.01


@pytest.mark.parametrize("kind", ["trt", "srt", "cum1st"])
def test_temperature_mode_advection_diffusion(kind):
    # T = 1 + a sin(k (x - U t)) exp(-kappa k^2 t) for uniform u = (U, 0, 0)
    L, a, U, kappa = 32, 0.01, 0.05, 0.02
    kx = 2 * math.pi / L
    x = np.arange(L)
    u = np.zeros((3, L))
    u[0] = U
    o = _sim(L, 1, 1, k=kappa, hkind=kind)
    o.init_fields(np.ones(L), u, 1.0 + a * np.sin(kx * x))
    samples = []
    for t in (40, 240):  # U * 200 = 10 lattice units: phase stays below pi
        o.step(t - (40 if samples else 0))
        _, _, T = o.macros()
        c = np.sum((T - 1) * np.exp(-1j * kx * x)) * 2.0 / L
        samples.append(c)
    rate = math.log(abs(samples[0]) / abs(samples[1])) / 200.0
    dphase = np.angle(samples[1] / samples[0])
    assert abs(rate / (kappa * kx * kx) - 1.0) < 0.015
    assert abs(-dphase / (kx * U * 200.0) - 1.0) < 0.01


def test_gaussian_hill_closed_form():
    # Sec. 4.1, Eq. (GaussianHill_anal_solution) in N = 2 dimensions
    L, s0, kappa, ux, t = 48, 16.0, 0.05, 0.05, 200
    y, x = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    x0 = y0 = L / 2.0

    def hill(tt):
        s2 = s0 + 2 * kappa * tt
        c = np.zeros_like(x, dtype=float)
        for ix in (-1, 0, 1):
            for iy in (-1, 0, 1):
                r2 = (x - x0 - ux * tt + ix * L) ** 2 + (y - y0 + iy * L) ** 2
                c += (s0 / s2) * np.exp(-r2 / (2 * s2))
        return c

    N = L * L
    u = np.zeros((3, N))
    u[0] = ux
    o = _sim(L, L, 1, k=kappa, hkind="trt")
    o.init_fields(np.ones(N), u, hill(0.0).reshape(-1))
    o.step(t)
    _, _, T = o.macros()
    Ta = hill(float(t)).reshape(-1)
    l2 = math.sqrt(np.sum((Ta - T) ** 2) / np.sum(Ta ** 2))
    # measured 4.4e-3 here and 6.4e-4 at twice the resolution (96^2,
    # sigma0^2 = 64): discretisation error; a wrong diffusivity gives > 0.1
    assert l2 < 6e-3


@pytest.mark.parametrize("Q", [27, 7])
@pytest.mark.parametrize("qb,qt", [(0.5, 0.5), (0.3, 0.8), (0.7, 0.2)])
def test_steady_conduction_slab(Q, qb, qt):
    # steady conduction between walls at y = 1 - qb (T=1) and y = ny-2+qt
    # (T=0): linear profile, Nusselt number 1 (Sec. 4.4 definition with the
    # wall distance as length scale)
    ny, kappa = 12, 0.1
    flags, links = _plate(ny, qb, qt)
    o = _sim(1, ny, 1, flags, links, nwalls=2, qh=Q, k=kappa)
    o.set_wall_temperature(0, 1.0)
    o.set_wall_temperature(1, 0.0)
    o.init_fields(np.ones(ny), np.zeros((3, ny)), np.full(ny, 0.5))
    o.step(4000)
    _, _, T = o.macros()
    Hc = (ny - 3) + qb + qt
    y = np.arange(ny, dtype=float)
    Texp = 1.0 - (y - (1.0 - qb)) / Hc
    fl = flags == I.FLUID
    assert np.abs(T[fl] - Texp[fl]).max() < 1e-6
    qdot = o.surface_flux(0)
    Nu = qdot * Hc / (kappa * 1.0 * 1.0)
    assert abs(Nu - 1.0) < 1e-5


@pytest.mark.parametrize("qb,qt", [(0.5, 0.5), (0.25, 0.75), (0.8, 0.6)])
def test_poiseuille_between_interpolated_walls(qb, qt):
    # body-force driven channel: u = F/(2 rho nu) (y - y_b)(y_t - y)
    ny, nu, Fx = 14, 1.0 / 6.0, 1e-5
    flags, links = _plate(ny, qb, qt)
    o = _sim(1, ny, 1, flags, links, nwalls=2, nu=nu, F=(Fx, 0.0, 0.0))
    o.init_fields(np.ones(ny), np.zeros((3, ny)), np.ones(ny))
    o.step(5000)
    _, u, _ = o.macros()
    yb, yt = 1.0 - qb, ny - 2 + qt
    y = np.arange(ny, dtype=float)
    uexp = Fx / (2 * nu) * (y - yb) * (yt - y)
    fl = flags == I.FLUID
    umax = uexp.max()
    assert np.abs(u[0, fl] - uexp[fl]).max() < 0.02 * umax


def test_geometry_validation():
    ny = 6
    flags, links = _plate(ny, 0.5, 0.5)
    p = O.make_params(nx=1, ny=ny, nz=1)
    o = O.Oracle(p)
    bad = dict(links)
    bad["q"] = links["q"].copy()
    bad["q"][0] = 0.0
    with pytest.raises(O.OracleError):
        o.set_geometry(flags, bad, nwalls=2)
    short = {k: v[1:] for k, v in links.items()}
    with pytest.raises(O.OracleError):
        o.set_geometry(flags, short, nwalls=2)
    with pytest.raises(O.OracleError):
        o.set_geometry(flags, links, nwalls=1)  # wall id 1 out of range
    o.set_geometry(flags, links, nwalls=2)


# ---- first-order wall variants (Sec. 3): BB + EQ, BB + ABB ---------------
@pytest.mark.parametrize("mode", ["eq", "abb"])
def test_first_order_wall_formulas(mode):
    ny = 6
    flags, links = _plate(ny, 0.3, 0.8)
    o = _sim(1, ny, 1, flags, links, nwalls=2, wall_bc=mode)
    Tw = (0.9, 0.2)
    for w in (0, 1):
        o.set_wall_temperature(w, Tw[w])
    rng = np.random.default_rng(40)
    fs = rng.uniform(0.1, 1.0, (27, ny))
    hs = rng.uniform(0.1, 1.0, (27, ny))
    o.set_post(fs, hs)
    assert o.stream() == 0
    f, h = o.state()
    e, w, opp, _ = O.lattice(27)
    for n, a, wall in zip(links["node"], links["dir"], links["wall"]):
        ab = opp[a]
        assert f[ab, n] == fs[a, n]                                      # BB
        if mode == "eq":
            assert abs(h[ab, n] - w[a] * Tw[wall]) < 1e-16                # EQ: wall equilibrium
        else:
            assert abs(h[ab, n] - (-hs[a, n] + 2 * w[a] * Tw[wall])) < 1e-15  # ABB


@pytest.mark.parametrize("mode", ["eq", "abb"])
def test_first_order_walls_keep_uniform_state(mode):
    ny = 7
    flags, links = _plate(ny, 0.3, 0.8, nx=2, nz=2)
    o = _sim(2, ny, 2, flags, links, nwalls=2, k=1e-3, wall_bc=mode)
    for w in (0, 1):
        o.set_wall_temperature(w, 0.7)
    N = 4 * ny
    o.init_fields(np.ones(N), np.zeros((3, N)), np.full(N, 0.7))
    f0, h0 = o.state()
    o.step(20)
    f1, h1 = o.state()
    fl = flags != I.SOLID
    assert np.allclose(f1[:, fl], f0[:, fl], atol=1e-15) and np.allclose(h1[:, fl], h0[:, fl], atol=1e-15)


def test_abb_slab_puts_the_walls_half_way():
    # ABB ignores q: the steady conduction profile is linear between the
    # half-way points y = 0.5 and y = ny - 1.5 whatever q says (first order)
    ny, kappa = 12, 0.1
    flags, links = _plate(ny, 0.3, 0.8)
    o = _sim(1, ny, 1, flags, links, nwalls=2, k=kappa, wall_bc="abb")
    o.set_wall_temperature(0, 1.0)
    o.set_wall_temperature(1, 0.0)
    o.init_fields(np.ones(ny), np.zeros((3, ny)), np.full(ny, 0.5))
    o.step(4000)
    _, _, T = o.macros()
    y = np.arange(ny, dtype=float)
    Texp = 1.0 - (y - 0.5) / (ny - 2)
    fl = flags == I.FLUID
    assert np.abs(T[fl] - Texp[fl]).max() < 1e-6
    assert abs(o.surface_flux(0) * (ny - 2) / kappa - 1.0) < 1e-5


def test_eq_slab_is_linear_and_conserves_the_flux():
    ny, kappa = 12, 0.1
    flags, links = _plate(ny, 0.3, 0.8)
    o = _sim(1, ny, 1, flags, links, nwalls=2, k=kappa, wall_bc="eq")
    o.set_wall_temperature(0, 1.0)
    o.set_wall_temperature(1, 0.0)
    o.init_fields(np.ones(ny), np.zeros((3, ny)), np.full(ny, 0.5))
    o.step(6000)
    _, _, T = o.macros()
    Ti = T[2:ny - 2]
    assert np.abs(np.diff(Ti, 2)).max() < 1e-9
    assert abs(o.surface_flux(0) + o.surface_flux(1)) < 1e-9


@pytest.mark.parametrize("qh", [27, 7])
def test_zou_he_inlet_sets_the_prescribed_moments(qh):
    # Sec. 4.4 inlet, reading R20: after streaming, every inlet node carries
    # the prescribed velocity (x-momentum rho u_in, no transverse momentum)
    # and the zeroth moment of h is rho T_in, whatever the state behind it
    nx, ny, nz = 9, 6, 5
    flags = np.asarray(I.channel_flags(nx, ny, nz)).reshape(-1)
    N = nx * ny * nz
    uin, Tin = (0.05, 0.0, 0.0), 0.7
    o = O.Oracle(O.make_params(nx=nx, ny=ny, nz=nz, qh=qh, periodic_x=False, nu=0.05, k=0.01, u_in=uin, T_in=Tin,
                               inlet_bc="zou_he"))
    o.set_geometry(flags, None)
    rng = np.random.default_rng(40)
    u = np.stack([0.05 + 0.02 * rng.uniform(-1, 1, N), 0.02 * rng.uniform(-1, 1, N), 0.02 * rng.uniform(-1, 1, N)])
    o.init_fields(1.0 + 0.01 * rng.uniform(-1, 1, N), u.reshape(-1), 0.7 + 0.2 * rng.uniform(-1, 1, N))
    o.step(3)
    f, h = o.state()
    e = O.lattice(27)[0].astype(float)
    inlet = np.nonzero(flags == I.INLET)[0]
    rho = f[:, inlet].sum(axis=0)
    mom = e.T @ f[:, inlet]
    assert np.abs(mom[0] - rho * uin[0]).max() < 1e-14
    assert np.abs(mom[1:]).max() < 1e-14
    assert np.abs(h[:, inlet].sum(axis=0) - rho * Tin).max() < 1e-14
    # the rest of the state is far from the inlet state
    assert np.abs(f[:, inlet + 1].sum(axis=0) - 1.0).max() > 1e-4


def test_zou_he_uniform_channel_is_steady():
    nx, ny, nz = 12, 5, 4
    flags = np.asarray(I.channel_flags(nx, ny, nz)).reshape(-1)
    N = nx * ny * nz
    o = O.Oracle(O.make_params(nx=nx, ny=ny, nz=nz, periodic_x=False, nu=0.05, k=0.01, u_in=(0.04, 0.0, 0.0),
                               T_in=0.7, inlet_bc="zou_he"))
    o.set_geometry(flags, None)
    u = np.zeros((3, N))
    u[0] = 0.04
    o.init_fields(np.ones(N), u.reshape(-1), np.full(N, 0.7))
    o.step(30)
    r, uu, T = o.macros()
    assert np.abs(r - 1).max() < 1e-14 and np.abs(uu[0] - 0.04).max() < 1e-14
    assert np.abs(uu[1:]).max() < 1e-14 and np.abs(T - 0.7).max() < 1e-14
