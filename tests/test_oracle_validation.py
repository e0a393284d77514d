"""Pins of the oracle against the closed forms of the paper's validation
cases (arXiv 2203.01316):

* Sec. 4.3, steady conduction between concentric cylinders: the radial
  profile T(r) = T_in + (T_out - T_in) ln(r/r_in) / ln(r_out/r_in); with
  interpolated anti-bounce-back walls (Eq. IABB) the error falls at second
  order, with the first-order rules (BB + ABB, BB + EQ) at about first order;
* Sec. 4.1, Gaussian hill: at s^H = 1 (k = 1/6) every h kind relaxes fully
  to the equilibrium, so one step is T(x) <- sum_a h^eq_a(T(x - e_a), u), a
  lattice convolution computed here by FFT from the closed form of the
  discrete equilibrium; at smaller k the error against the continuous
  solution falls at second order under grid refinement.
"""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01316_gb300 import inputs as I


# ---- concentric cylinders -------------------------------------------------
def test_annulus_links_cross_their_circle():
    w = I.concentric_cylinders(20, seed=3)
    c = w["centre"]
    e = O.lattice(27)[0]
    lk = w["links"]
    n = w["dims"][0]
    x = lk["node"] % n
    y = lk["node"] // n
    d = e[lk["dir"]]
    q = lk["q"].astype(np.float64)
    px = x + q * d[:, 0] - c[0]
    py = y + q * d[:, 1] - c[1]
    R = np.where(lk["wall"] == 0, w["R_inner"], w["R_outer"])
    # q is stored in FP32: the crossing point is on the circle to FP32 accuracy
    assert np.abs(np.hypot(px, py) - R).max() < 1e-5 * R.max()
    assert np.all((q > 0) & (q <= 1))
    fl = w["flags"].reshape(n, n)
    assert np.all(fl[y, x] == I.FLUID)
    assert np.all(fl[(y + d[:, 1]) % n, (x + d[:, 0]) % n] == I.SOLID)
    assert np.all(d[:, 2] * 0 == 0) and np.all((d[:, 0] != 0) | (d[:, 1] != 0))
    # both walls are present and every fluid node next to solid is linked
    assert set(np.unique(lk["wall"]).tolist()) == {0, 1}


def _annulus_error(D, wall_bc):
    w = I.concentric_cylinders(D)
    n = w["dims"][0]
    k = 0.1
    p = O.make_params(nx=n, ny=n, nz=1, qh=27, hkind="trt", periodic_x=True, nu=1.0 / 6.0, k=k, wall_bc=wall_bc)
    o = O.Oracle(p)
    o.set_geometry(w["flags"], w["links"], nwalls=2)
    o.set_wall_temperature(0, 1.0)
    o.set_wall_temperature(1, 0.0)
    o.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    # about twelve diffusion times across the gap: steady to rounding
    o.step(int(12 * (D / 4.0) ** 2 / k) + 200)
    T1 = o.macros()[2].copy()
    o.step(20)
    T = o.macros()[2]
    fl = w["flags"] == I.FLUID
    assert np.abs(T - T1)[fl].max() < 1e-12
    r = w["r"][fl]
    Ta = 1.0 - np.log(r / w["R_inner"]) / np.log(w["R_outer"] / w["R_inner"])
    return float(np.sqrt(np.sum((Ta - T[fl]) ** 2) / np.sum(Ta ** 2)))


def test_annulus_conduction_orders():
    errs = {bc: [_annulus_error(D, bc) for D in (8, 16)] for bc in ("iabb", "abb", "eq")}
    order = {bc: np.log2(e[0] / e[1]) for bc, e in errs.items()}
    assert order["iabb"] >= 2.0, errs
    assert errs["iabb"][1] < 1e-2
    for bc in ("abb", "eq"):
        assert order[bc] < 1.5, (bc, errs)
        assert errs[bc][1] > 5 * errs["iabb"][1], (bc, errs)


# ---- Gaussian hill ---------------------------------------------------------
def _transfer(L, u, Q):
    """Fourier symbol of one s^H = 1 step on a periodic L x L plane (nz = 1):
    the D3Q27 equilibrium is the product of 1-D weights
    (1 - a, (a +- u)/2) with a = c_s^2 + u^2; the D3Q7 one keeps the same arms
    and puts the remainder 1 - sum_i a_i at rest."""
    th = np.fft.fftfreq(L) * 2.0 * np.pi
    cs2 = 1.0 / 3.0
    ax, ay = cs2 + u[0] ** 2, cs2 + u[1] ** 2
    arm_x = 0.5 * (ax + u[0]) * np.exp(-1j * th) + 0.5 * (ax - u[0]) * np.exp(1j * th)
    arm_y = 0.5 * (ay + u[1]) * np.exp(-1j * th) + 0.5 * (ay - u[1]) * np.exp(1j * th)
    if Q == 27:
        return np.outer((1.0 - ay) + arm_y, (1.0 - ax) + arm_x)
    return (1.0 - ax - ay) + arm_y[:, None] + arm_x[None, :]


def _oracle_hill(L, s0, k, n, u, kind, Q=27):
    w = I.gaussian_hill(L, s0)
    w["u"][0], w["u"][1] = u
    p = O.make_params(nx=L, ny=L, nz=1, qh=Q, hkind=kind, periodic_x=True, nu=1.0 / 6.0, k=k)
    o = O.Oracle(p)
    o.set_geometry(w["flags"], w["links"], nwalls=1)
    o.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    o.step(n)
    return w["T"].reshape(L, L) - 1.0, o.macros()[2].reshape(L, L) - 1.0


@pytest.mark.parametrize("Q,kind", [(27, "trt"), (27, "srt"), (27, "1st"), (27, "cum1st"), (7, "trt"),
                                    (7, "cum1st")])
def test_hill_at_unit_rate_is_the_lattice_convolution(Q, kind):
    L, n, u = 24, 30, (0.06, -0.035)
    C0, C = _oracle_hill(L, 9.0, 1.0 / 6.0, n, u, kind, Q)
    ref = np.real(np.fft.ifft2(np.fft.fft2(C0) * _transfer(L, u, Q) ** n))
    assert np.abs(C - ref).max() < 1e-13


def _closed_form(L, s0, k, n, ux):
    yy, xx = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    s2 = s0 + 2.0 * k * n
    cx = (L / 2.0 + ux * n) % L
    return sum((s0 / s2) * np.exp(-((xx - cx + i * L) ** 2 + (yy - L / 2.0 + j * L) ** 2) / (2.0 * s2))
               for i in (-1, 0, 1) for j in (-1, 0, 1))


def test_hill_second_order_under_refinement():
    # the same physical case (sigma0 = L/8, t such that sigma^2 doubles,
    # k = 0.05, u_x L = 1.6) on L = 32 and L = 64: the error falls about 4x
    errs = []
    for L in (32, 64):
        s0 = (L / 8.0) ** 2
        k = 0.05
        n = int(round(s0 / (2 * k)))
        ux = 1.6 / L
        _, C = _oracle_hill(L, s0, k, n, (ux, 0.0), "trt")
        Ca = _closed_form(L, s0, k, n, ux)
        errs.append(float(np.sqrt(np.sum((Ca - C) ** 2) / np.sum(Ca ** 2))))
    assert 3.3 < errs[0] / errs[1] < 4.8, errs


# ---- z-invariant plane at rest: the D3Q27 h step is a D2Q9 scheme ---------
_E9 = np.array([(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)])
_W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
_OPP9 = [0, 3, 4, 1, 2, 7, 8, 5, 6]


def _d2q9_step(h, s, kind):
    """One collide + stream of a D2Q9 model at u = 0, written from the
    definitions of Sec. 2.1.1 in population space: SRT relaxes every
    population to w H; TRT (s_odd = s, s_even = 1) relaxes the part odd
    under e -> -e with s and sets the even part to equilibrium; CM-1st
    keeps (1 - s) of the two first moments and puts everything else at
    equilibrium (the 1-D dual of the moment c on {-1, 0, 1} is c/2)."""
    H = h.sum(0)
    eq = _W9[:, None, None] * H[None]
    if kind == "srt":
        hs = h - s * (h - eq)
    elif kind == "trt":
        hs = eq + (1.0 - s) * 0.5 * (h - h[_OPP9])
    else:
        mx = np.tensordot(_E9[:, 0].astype(float), h, 1)
        my = np.tensordot(_E9[:, 1].astype(float), h, 1)
        hs = eq.copy()
        for a, (ex, ey) in enumerate(_E9):
            if ey == 0 and ex != 0:
                hs[a] += (1.0 - s) * 0.5 * ex * mx
            if ex == 0 and ey != 0:
                hs[a] += (1.0 - s) * 0.5 * ey * my
    return np.stack([np.roll(np.roll(hs[a], _E9[a][0], 1), _E9[a][1], 0) for a in range(9)])


@pytest.mark.parametrize("kind", ["trt", "srt", "1st"])
def test_plane_at_rest_reduces_to_d2q9(kind):
    # summing the D3Q27 populations over e_z commutes with the product-basis
    # collision and with streaming on a one-node-thick periodic plane, so at
    # u = 0 (central = raw moments) the oracle's temperature must follow the
    # D2Q9 scheme above, at k = 1e-3 (s^H close to 2)
    L, n, k = 12, 25, 1e-3
    s = 1.0 / (3.0 * k + 0.5)
    w = I.gaussian_hill(L, 4.0)
    w["T"] = w["T"] + I.uniform(21, L * L, -0.05, 0.05)
    o = O.Oracle(O.make_params(nx=L, ny=L, nz=1, hkind=kind, periodic_x=True, nu=1.0 / 6.0, k=k))
    o.set_geometry(w["flags"], w["links"], nwalls=1)
    o.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    h = _W9[:, None, None] * w["T"].reshape(L, L)[None]
    for step in range(n):
        o.step(1)
        h = _d2q9_step(h, s, kind)
        assert np.abs(o.macros()[2].reshape(L, L) - h.sum(0)).max() < 1e-13, step
