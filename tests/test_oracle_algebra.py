"""Pins of the oracle's lattice, transforms, equilibria and cumulants against
what the paper prints and what the mathematics fixes (arXiv 2203.01316)."""
import itertools
import math
import os

import numpy as np
import pytest

from oracle import oracle as O

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
CS2 = 1.0 / 3.0


def _golden_velocities():
    rows = {}
    for line in open(os.path.join(GOLDEN, "d3q27_velocities.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, *vals = line.split()
        rows[name] = [int(v) for v in vals]
    return np.array([rows["e_x"], rows["e_y"], rows["e_z"]]).T


def _golden_moments():
    for line in open(os.path.join(GOLDEN, "moment_order.txt")):
        if line.startswith("#") or not line.strip():
            continue
        return np.array([[int(c) for c in tok] for tok in line.split()])


def test_velocities_and_moment_order_match_paper():
    e, w, opp, mom = O.lattice(27)
    assert np.array_equal(e, _golden_velocities())
    assert np.array_equal(mom, _golden_moments())
    assert len({tuple(v) for v in e}) == 27


def test_opposite_directions():
    e, w, opp, mom = O.lattice(27)
    assert np.array_equal(e[opp], -e)
    e7, w7, opp7, _ = O.lattice(7)
    assert np.array_equal(e7[opp7], -e7)


def test_weights_closed_form_and_d2q9_reduction():
    # u = 0 equilibrium is the product of 1-D weights (2/3, 1/6, 1/6)
    e, w, _, _ = O.lattice(27)
    w1 = {0: 2.0 / 3.0, 1: 1.0 / 6.0, -1: 1.0 / 6.0}
    expect = np.array([w1[a] * w1[b] * w1[c] for a, b, c in e])
    assert np.allclose(w, expect, atol=1e-15, rtol=0)
    assert set(np.round(w * 216).astype(int)) == {64, 16, 4, 1}  # 8/27, 2/27, 1/54, 1/216
    # Sec. 3: summing the D3Q27 weights over z gives the D2Q9 weights
    d2q9 = {}
    for (a, b, _), wi in zip(e, w):
        d2q9[(a, b)] = d2q9.get((a, b), 0.0) + wi
    assert math.isclose(d2q9[(0, 0)], 4.0 / 9.0, abs_tol=1e-15)
    for k in [(1, 0), (-1, 0), (0, 1), (0, -1)]:
        assert math.isclose(d2q9[k], 1.0 / 9.0, abs_tol=1e-15)
    for k in [(1, 1), (1, -1), (-1, 1), (-1, -1)]:
        assert math.isclose(d2q9[k], 1.0 / 36.0, abs_tol=1e-15)


def test_d3q7_reading():
    # reading: D3Q7 = {0, +-x, +-y, +-z} with cs^2 = 1/3 -> rest weight 0, moving 1/6
    e7, w7, _, mom7 = O.lattice(7)
    e27, _, _, _ = O.lattice(27)
    assert np.array_equal(e7, e27[[0, 1, 2, 3, 7, 8, 9]])
    assert abs(w7[0]) < 1e-15 and np.allclose(w7[1:], 1.0 / 6.0, atol=1e-15)
    assert [tuple(m) for m in mom7] == [(0, 0, 0), (1, 0, 0), (0, 1, 0), (0, 0, 1),
                                       (2, 0, 0), (0, 2, 0), (0, 0, 2)]


def _binomial_shift(u, mom):
    """Central moments from raw moments per axis: k_m = sum_j C(m,j)(-u)^(m-j) m_j.
    Built from the binomial theorem, independently of the oracle's T(u)."""
    Q = len(mom)
    N = np.zeros((Q, Q))
    index = {tuple(m): i for i, m in enumerate(mom)}
    for r, (m, n, o) in enumerate(mom):
        for j1 in range(m + 1):
            for j2 in range(n + 1):
                for j3 in range(o + 1):
                    c = (math.comb(m, j1) * (-u[0]) ** (m - j1) * math.comb(n, j2) *
                         (-u[1]) ** (n - j2) * math.comb(o, j3) * (-u[2]) ** (o - j3))
                    N[r, index[(j1, j2, j3)]] += c
    return N


@pytest.mark.parametrize("Q", [27, 7])
def test_T_equals_N_M_and_shift_inverse(Q):
    # Appendix C: T = N M, so N = T M^-1; the shift by u is undone by -u
    rng = np.random.default_rng(1)
    e, _, _, mom = O.lattice(Q)
    M = O.matrix_M(Q)
    assert np.linalg.matrix_rank(M) == Q
    brute = np.array([[float(np.prod([ev ** m for ev, m in zip(e[a], mom[r])])) for a in range(Q)]
                      for r in range(Q)])
    assert np.array_equal(M, brute)
    for _ in range(3):
        u = rng.uniform(-0.2, 0.2, 3)
        T = O.matrix_T(u, Q)
        N = _binomial_shift(u, mom)
        assert np.allclose(T, N @ M, atol=1e-14, rtol=0)
        assert np.allclose(_binomial_shift(-u, mom) @ N, np.eye(Q), atol=1e-14)
        assert np.allclose(np.linalg.solve(T, T @ np.arange(Q)), np.arange(Q), atol=1e-12)


def test_equilibrium_product_form():
    # App. A route T(u)^-1 Y_eq against the closed form H prod_d w1(e_d, u_d)
    rng = np.random.default_rng(2)
    e, _, _, _ = O.lattice(27)

    def w1(c, u):
        return 1.0 - u * u - CS2 if c == 0 else 0.5 * (u * u + c * u + CS2)

    for _ in range(5):
        u = rng.uniform(-0.15, 0.15, 3)
        H = rng.uniform(0.5, 2.0)
        g = O.equilibrium(H, u)
        closed = np.array([H * w1(a, u[0]) * w1(b, u[1]) * w1(c, u[2]) for a, b, c in e])
        assert np.allclose(g, closed, atol=1e-15, rtol=1e-13)


def test_equilibrium_d3q7_closed_form():
    rng = np.random.default_rng(3)
    u = rng.uniform(-0.1, 0.1, 3)
    H = 1.3
    g = O.equilibrium(H, u, Q=7)
    exp = np.zeros(7)
    exp[0] = H * (1.0 - 3 * CS2 - u @ u)
    for d in range(3):
        exp[1 + d] = 0.5 * H * (CS2 + u[d] ** 2 + u[d])
        exp[4 + d] = 0.5 * H * (CS2 + u[d] ** 2 - u[d])
    assert np.allclose(g, exp, atol=1e-15)


def _moment(e, g, m, n, o, u=(0.0, 0.0, 0.0)):
    return float(np.sum((e[:, 0] - u[0]) ** m * (e[:, 1] - u[1]) ** n * (e[:, 2] - u[2]) ** o * g))


def test_equilibrium_raw_moments_appendix_A():
    # Appendix A prints the D2Q9 raw moments of h^eq in the order
    # 00,10,01,20,02,11,21,12,22; the D3Q27 equilibrium's moments with o = 0
    # must equal them (z factor sums to one).
    e, _, _, _ = O.lattice(27)
    ux, uy, H = 0.07, -0.04, 1.7
    g = O.equilibrium(H, [ux, uy, 0.02])
    idx = [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2), (1, 1), (2, 1), (1, 2), (2, 2)]
    printed = H * np.array([1.0, ux, uy, ux ** 2 + CS2, uy ** 2 + CS2, ux * uy,
                            uy * (ux ** 2 + CS2), ux * (uy ** 2 + CS2),
                            ux ** 2 * uy ** 2 + CS2 * ux ** 2 + CS2 * uy ** 2 + CS2 ** 2])
    got = np.array([_moment(e, g, m, n, 0) for m, n in idx])
    assert np.allclose(got, printed, atol=1e-15, rtol=1e-13)


def test_symmetric_antisymmetric_central_moments_appendix_B():
    # Appendix B prints the central moments of h^seq and h^aeq (D2Q9 order);
    # checked through the oracle's T(u) and opposite table.
    e, _, opp, mom = O.lattice(27)
    ux, uy, H = 0.06, 0.035, 1.0
    u = np.array([ux, uy, 0.0])
    g = O.equilibrium(H, u)
    seq = 0.5 * (g + g[opp])
    aeq = 0.5 * (g - g[opp])
    T = O.matrix_T(u)
    cs, ca = T @ seq, T @ aeq
    index = {tuple(m): i for i, m in enumerate(mom)}
    idx = [(0, 0), (1, 0), (0, 1), (2, 0), (0, 2), (1, 1), (2, 1), (1, 2), (2, 2)]
    p_seq = np.array([1.0, -ux, -uy, 2 * ux ** 2 + CS2, 2 * uy ** 2 + CS2, 2 * ux * uy,
                      -uy * (4 * ux ** 2 + CS2), -ux * (4 * uy ** 2 + CS2),
                      8 * ux ** 2 * uy ** 2 + 2 * CS2 * (ux ** 2 + uy ** 2) + CS2 ** 2])
    p_aeq = np.array([0.0, ux, uy, -2 * ux ** 2, -2 * uy ** 2, -2 * ux * uy,
                      uy * (4 * ux ** 2 + CS2), ux * (4 * uy ** 2 + CS2),
                      -(8 * ux ** 2 * uy ** 2 + 2 * CS2 * (ux ** 2 + uy ** 2))])
    got_s = np.array([cs[index[(m, n, 0)]] for m, n in idx])
    got_a = np.array([ca[index[(m, n, 0)]] for m, n in idx])
    assert np.allclose(got_s, H * p_seq, atol=1e-15)
    assert np.allclose(got_a, H * p_aeq, atol=1e-15)


def _random_distribution(rng, scale=0.3):
    g = O.equilibrium(1.0, rng.uniform(-0.1, 0.1, 3))
    return g * (1.0 + scale * rng.uniform(-1, 1, 27))


def _partition_cumulant(e, g, mno):
    """Joint cumulant by the set-partition formula
    k(X1..Xn) = sum_pi (|pi|-1)! (-1)^(|pi|-1) prod_B E[prod_{i in B} X_i]
    for the normalised distribution g/rho, variables x (m times), y, z."""
    p = g / g.sum()
    var = [0] * mno[0] + [1] * mno[1] + [2] * mno[2]
    n = len(var)

    def partitions(items):
        if not items:
            yield []
            return
        first, rest = items[0], items[1:]
        for part in partitions(rest):
            for i in range(len(part)):
                yield part[:i] + [[first] + part[i]] + part[i + 1:]
            yield [[first]] + part

    total = 0.0
    for part in partitions(list(range(n))):
        k = len(part)
        prod = 1.0
        for block in part:
            prod *= float(np.sum(p * np.prod([e[:, var[i]] for i in block], axis=0)))
        total += math.factorial(k - 1) * (-1) ** (k - 1) * prod
    return total


def test_cumulants_match_partition_formula():
    rng = np.random.default_rng(4)
    e, _, _, mom = O.lattice(27)
    for _ in range(2):
        g = _random_distribution(rng)
        Cv = O.cumulants(g)
        assert math.isclose(Cv[0], g.sum(), rel_tol=1e-15)
        for r in range(1, 27):
            ref = _partition_cumulant(e.astype(float), g, tuple(mom[r]))
            assert abs(Cv[r] - ref) < 1e-13, (tuple(mom[r]), Cv[r], ref)


def test_cumulant_roundtrip_and_low_orders():
    rng = np.random.default_rng(5)
    e, _, _, mom = O.lattice(27)
    for _ in range(5):
        g = _random_distribution(rng)
        Cv = O.cumulants(g)
        assert np.allclose(O.cumulants_inverse(Cv), g, atol=1e-14, rtol=0)
        rho = g.sum()
        mean = (e.T @ g) / rho
        # orders 2 and 3: cumulant = central moment / rho
        for r in range(4, 17):
            m = tuple(mom[r])
            assert abs(Cv[r] - _moment(e, g, *m, u=mean) / rho) < 1e-15


def test_independent_axes_have_zero_mixed_cumulants():
    e, _, _, mom = O.lattice(27)
    px = {-1: 0.2, 0: 0.5, 1: 0.3}
    py = {-1: 0.1, 0: 0.6, 1: 0.3}
    pz = {-1: 0.25, 0: 0.45, 1: 0.3}
    g = 1.4 * np.array([px[a] * py[b] * pz[c] for a, b, c in e])
    Cv = O.cumulants(g)
    for r in range(4, 27):
        m = mom[r]
        if np.count_nonzero(m) > 1:
            assert abs(Cv[r]) < 1e-15, tuple(m)
    var_x = sum(px[a] * a * a for a in px) - sum(px[a] * a for a in px) ** 2
    assert abs(Cv[7] - var_x) < 1e-15
