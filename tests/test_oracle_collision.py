"""Pins of the oracle's collision operators: invariants, fixed points and the
identities the paper states (arXiv 2203.01316, Sec. 2.1.1)."""
import numpy as np
import pytest

from oracle import oracle as O

CS2 = 1.0 / 3.0


def _perturbed(Q, psi, u, rng, scale=0.2):
    g = O.equilibrium(psi, u, Q=Q)
    w = O.lattice(Q)[1]
    return g + scale * psi * w * rng.uniform(-1, 1, Q)


@pytest.mark.parametrize("F", [(0.0, 0.0, 0.0), (1e-3, -2e-3, 5e-4)])
def test_f_collision_conserves_mass_and_momentum(F):
    rng = np.random.default_rng(10)
    e = O.lattice(27)[0].astype(float)
    p = O.make_params(nu=0.03, F=F, omega_bulk=0.8)
    for _ in range(4):
        f = _perturbed(27, 1.0 + 0.05 * rng.uniform(-1, 1), rng.uniform(-0.1, 0.1, 3), rng)
        fs, u = O.collide_f(p, f)
        assert abs(fs.sum() - f.sum()) < 1e-14
        assert np.allclose(e.T @ fs, e.T @ f + np.array(F), atol=1e-15)
        assert np.allclose(u, (e.T @ f + 0.5 * np.array(F)) / f.sum(), atol=1e-15)


@pytest.mark.parametrize("Q,kind", [(27, "trt"), (27, "srt"), (27, "1st"), (7, "trt"), (7, "srt")])
@pytest.mark.parametrize("src", [0.0, 3e-4])
def test_h_collision_conserves_energy_plus_source(Q, kind, src):
    rng = np.random.default_rng(11)
    p = O.make_params(qh=Q, hkind=kind, k=1e-3)
    for _ in range(4):
        u = rng.uniform(-0.1, 0.1, 3)
        h = _perturbed(Q, 1.2, u, rng)
        hs = O.collide_h(p, h, u, Q=src)
        # App. D: the stored variable is h - q/2, collision adds the full Q
        assert abs(hs.sum() - (h.sum() + src)) < 1e-14


@pytest.mark.parametrize("Q,kind", [(27, "trt"), (27, "srt"), (27, "1st"), (7, "trt"), (7, "srt"), (7, "1st")])
def test_equilibrium_is_fixed_point(Q, kind):
    rng = np.random.default_rng(12)
    for _ in range(3):
        u = rng.uniform(-0.12, 0.12, 3)
        p = O.make_params(qh=Q, hkind=kind, nu=0.011, k=3e-5)
        feq = O.equilibrium(1.02, u)
        fs, uu = O.collide_f(p, feq)
        assert np.allclose(fs, feq, atol=1e-15)
        assert np.allclose(uu, u, atol=1e-15)
        heq = O.equilibrium(0.7, u, Q=Q)
        assert np.allclose(O.collide_h(p, heq, u), heq, atol=1e-15)


def test_full_relaxation_gives_product_equilibrium():
    # with every rate 1 (nu = 1/6 gives omega1 = 1) all cumulants reach their
    # equilibria: the result is the product-form Maxwellian discretisation
    rng = np.random.default_rng(13)
    p = O.make_params(nu=1.0 / 6.0)
    f = _perturbed(27, 1.1, [0.05, -0.02, 0.03], rng, scale=0.3)
    fs, u = O.collide_f(p, f)
    assert np.allclose(fs, O.equilibrium(f.sum(), u), atol=1e-15)


def test_cm_srt_equals_bgk():
    # Sec. 2.1.1, CM-SRT: h* = (1 - s) h + s h^eq
    rng = np.random.default_rng(14)
    for Q in (27, 7):
        k = 2e-3
        s = 1.0 / (3.0 * k + 0.5)
        p = O.make_params(qh=Q, hkind="srt", k=k)
        u = rng.uniform(-0.1, 0.1, 3)
        h = _perturbed(Q, 0.9, u, rng)
        heq = O.equilibrium(h.sum(), u, Q=Q)
        assert np.allclose(O.collide_h(p, h, u), (1 - s) * h + s * heq, atol=1e-15)


def test_d3q7_first_order_equals_trt():
    # Sec. 4.2: on D3Q7 CM-1st and CM-TRT cannot be distinguished
    rng = np.random.default_rng(15)
    u = rng.uniform(-0.1, 0.1, 3)
    h = _perturbed(7, 1.0, u, rng)
    a = O.collide_h(O.make_params(qh=7, hkind="1st", k=1e-4), h, u, Q=1e-5)
    b = O.collide_h(O.make_params(qh=7, hkind="trt", k=1e-4), h, u, Q=1e-5)
    assert np.array_equal(a, b)


def test_d3q27_kinds_differ():
    rng = np.random.default_rng(16)
    u = rng.uniform(-0.1, 0.1, 3)
    h = _perturbed(27, 1.0, u, rng)
    outs = [O.collide_h(O.make_params(hkind=k, k=1e-4), h, u) for k in ("trt", "srt", "1st")]
    for i in range(3):
        for j in range(i + 1, 3):
            assert np.abs(outs[i] - outs[j]).max() > 1e-6


def test_cm_post_collision_central_moments():
    # the post-collision central moments are (1-s) Y + s Y_eq with s per kind
    rng = np.random.default_rng(17)
    k = 1e-3
    sH = 1.0 / (3.0 * k + 0.5)
    mom = O.lattice(27)[3]
    order = mom.sum(axis=1)
    u = rng.uniform(-0.1, 0.1, 3)
    h = _perturbed(27, 1.0, u, rng)
    T = O.matrix_T(u)
    Y = T @ h
    E = np.array([0.0 if 1 in m else CS2 ** (list(m).count(2)) for m in mom])
    for kind, rate in (("trt", np.where(order % 2 == 1, sH, 1.0)),
                       ("1st", np.where(order == 1, sH, 1.0))):
        Ys = T @ O.collide_h(O.make_params(hkind=kind, k=k), h, u)
        assert np.allclose(Ys, Y + rate * (h.sum() * E - Y), atol=1e-14)


def test_f_second_order_cumulant_relaxation():
    # R1: off-diagonal and deviatoric second cumulants relax with omega1,
    # the trace with omega_bulk; higher orders to zero at rate 1
    rng = np.random.default_rng(18)
    nu, wb = 0.02, 0.7
    w1 = 1.0 / (3 * nu + 0.5)
    f = _perturbed(27, 1.0, [0.04, 0.01, -0.03], rng)
    C = O.cumulants(f)
    fs, _ = O.collide_f(O.make_params(nu=nu, omega_bulk=wb), f)
    Cs = O.cumulants(fs)
    assert np.allclose(Cs[4:7], (1 - w1) * C[4:7], atol=1e-15)
    assert abs((Cs[7] - Cs[8]) - (1 - w1) * (C[7] - C[8])) < 1e-15
    assert abs((Cs[7] - Cs[9]) - (1 - w1) * (C[7] - C[9])) < 1e-15
    assert abs(Cs[7:10].sum() - (C[7:10].sum() + wb * (1.0 - C[7:10].sum()))) < 1e-15
    assert np.allclose(Cs[10:], 0.0, atol=1e-15)
    # partial relaxation of higher orders
    fs2, _ = O.collide_f(O.make_params(nu=nu, omega3=0.5, omega4=0.25, omega5=0.0, omega6=0.9), f)
    Cs2 = O.cumulants(fs2)
    mom = O.lattice(27)[3]
    order = mom.sum(axis=1)
    wn = {3: 0.5, 4: 0.25, 5: 0.0, 6: 0.9}
    for r in range(10, 27):
        assert abs(Cs2[r] - (1 - wn[order[r]]) * C[r]) < 1e-14


# ---- Cumulants-1st (Eq. H_cu_collision) ------------------------------------
def _w1(c, u):
    return 1.0 - u * u - CS2 if c == 0 else 0.5 * (u * u + c * u + CS2)


@pytest.mark.parametrize("Q", [0.0, 2e-3])
def test_cumulant_h_collision_is_maxwellian_at_relaxed_mean(Q):
    # with every order >= 2 at equilibrium the post-collision cumulants are
    # (H + Q/2, v, cs^2 I, 0, ...), v = (1 - s) mean + s u: the product-form
    # discrete Maxwellian at velocity v (closed form)
    rng = np.random.default_rng(30)
    e = O.lattice(27)[0]
    k = 2e-3
    s = 1.0 / (3 * k + 0.5)
    p = O.make_params(hkind="cum1st", k=k)
    for _ in range(3):
        u = rng.uniform(-0.1, 0.1, 3)
        h = _perturbed(27, 1.3, rng.uniform(-0.1, 0.1, 3), rng, scale=0.3)
        mean = (e.T @ h) / h.sum()
        v = (1 - s) * mean + s * u
        Hs = h.sum() + Q
        closed = np.array([Hs * _w1(a, v[0]) * _w1(b, v[1]) * _w1(c, v[2]) for a, b, c in e])
        assert np.allclose(O.collide_h(p, h, u, Q=Q), closed, atol=1e-14)


def test_cumulant_h_collision_d3q7_and_equilibrium_fixed_point():
    rng = np.random.default_rng(31)
    p = O.make_params(qh=7, hkind="cum1st", k=1e-3)
    u = rng.uniform(-0.1, 0.1, 3)
    heq = O.equilibrium(0.8, u, Q=7)
    assert np.allclose(O.collide_h(p, heq, u), heq, atol=1e-15)
    h = _perturbed(7, 0.8, u, rng)
    hs = O.collide_h(p, h, u, Q=1e-3)
    assert abs(hs.sum() - (h.sum() + 1e-3)) < 1e-14
    heq27 = O.equilibrium(0.8, u)
    assert np.allclose(O.collide_h(O.make_params(hkind="cum1st", k=1e-3), heq27, u), heq27, atol=1e-15)
