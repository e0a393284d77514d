"""The identity behind the reverse-mode velocity derivative of the coupled
adjoint (k_adjoint_flow, h_velocity_adjoint), checked on the oracle's own
central-moment collision C_h(g; u) (Eq. H_cm_collision with the App. D
source): with Y = T(u) g the central moments of the arrivals and the
relaxation rates S per order,

    dC_h/du_d = T(u)^-1 (S_d T(u) C_h(g; u) - (1 - S) S_d T(u) g),

where (S_d Y)_mno = m_d Y_(m - e_d)no lowers the d-th order by one (dT/du_d
= -S_d T on the three-point stencil).  Both lattices, the three
central-moment kinds, with a source; against central differences of the
oracle's collision in u (the collision is polynomial in u, so the step-1e-4
difference is accurate to about 1e-8 relative)."""
import numpy as np
import pytest

from oracle import oracle as O


def _rates(kind, k):
    sH = 1.0 / (3.0 * k + 0.5)
    if kind == "srt":
        return lambda order: sH
    if kind == "1st":
        return lambda order: sH if order == 1 else 1.0
    return lambda order: sH if order % 2 == 1 else 1.0


@pytest.mark.parametrize("qh", [27, 7])
@pytest.mark.parametrize("kind", ["trt", "srt", "1st"])
def test_velocity_derivative_of_the_h_collision(qh, kind):
    rng = np.random.default_rng(3 + qh)
    k = 3e-3
    p = O.make_params(qh=qh, hkind=kind, k=k)
    e, w, _, mom = O.lattice(qh)
    u = np.array([0.04, -0.03, 0.02])
    g = O.equilibrium(0.8, u + 0.01, qh) + 0.01 * rng.standard_normal(qh)
    Q = 2e-3
    lam = rng.standard_normal(qh)
    order = mom.sum(axis=1)
    s = np.array([_rates(kind, k)(o) for o in order])
    T = O.matrix_T(u, qh)
    Ti = np.linalg.inv(T)
    Y = T @ g
    Ys = T @ O.collide_h(p, g, u, Q)
    index = {tuple(m): i for i, m in enumerate(mom)}
    z = Ti.T @ lam
    for d in range(3):
        def shift(V):
            out = np.zeros(qh)
            for i, m in enumerate(mom):
                if m[d] >= 1:
                    lo = list(m)
                    lo[d] -= 1
                    out[i] = m[d] * V[index[tuple(lo)]]
            return out
        w_rev = z @ (shift(Ys) - (1.0 - s) * shift(Y))
        eps = 1e-4
        up, um = u.copy(), u.copy()
        up[d] += eps
        um[d] -= eps
        w_fd = lam @ (O.collide_h(p, g, up, Q) - O.collide_h(p, g, um, Q)) / (2 * eps)
        assert abs(w_rev - w_fd) <= 1e-8 * max(1.0, abs(w_fd)), (d, w_rev, w_fd)
