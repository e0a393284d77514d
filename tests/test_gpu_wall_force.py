"""The momentum-exchange wall force on the GPU (lbm_wall_force) against the
oracle's (the force objective of oracle.adjoint with no steps, which reads
the given post-collision state), and the exact momentum balance of a
periodic box on the GPU path itself.

Tolerances: both sides read the same stored populations; the GPU evaluates
Eq. IBB in the storage's arithmetic type (FP64, or FP32 for the other
storages) and sums in FP64, so the difference is bounded by a few units of
that type's rounding per link times the largest stored deviation, plus the
FP64 rounding of the sums of full populations (O(1) per link):
4 x links x (eps_R max |f - w rho0| + eps_64)."""
import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01316_gb300 import inputs as I

from test_gpu_adjoint import _solver
from test_oracle_force import _box_case

pytestmark = pytest.mark.gpu


def _box_solver(storage, wall_bc="iabb"):
    w, p = _box_case(wall_bc=wall_bc)
    theta = np.zeros(w["flags"].size)
    s = _solver(w, storage, 27, "trt", p.nu, p.k, tuple(p.F[:3]), [1.0, 0.5, 0.2], theta, wall_bc=wall_bc)
    return w, p, s


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("wall_bc", ["iabb", "abb"])
def test_wall_force_matches_oracle(storage, wall_bc):
    w, p, s = _box_solver(storage, wall_bc)
    s.step(5)
    f0, h0 = s.populations()
    o = O.Oracle(p)
    o.set_geometry(w["flags"], w["links"], nwalls=3)
    Wf = O.lattice(27)[1]
    dev = np.abs(f0 - Wf[:, None] * (w["flags"] != I.SOLID)[None, :]).max()
    eps = np.finfo(np.float64 if storage == "f64" else np.float32).eps
    for wall in range(3):
        Fg = s.wall_force(wall)
        Fo = np.array([o.adjoint(f0, h0, 0, (0, 0), ("force", wall, 1.0, c), nwalls=3, gradients=False)[0]
                       for c in range(3)])
        nl = int(np.count_nonzero(w["links"]["wall"] == wall))
        tol = 4 * nl * (eps * max(dev, 1e-3) + np.finfo(np.float64).eps)
        assert np.abs(Fg - Fo).max() <= tol, (wall, Fg, Fo)


def test_wall_force_balances_momentum_fp64():
    # periodic box: the walls take N_fluid F minus the fluid's momentum change
    w, p, s = _box_solver("f64")
    e = O.lattice(27)[0].astype(np.float64)
    n_fluid = int(np.count_nonzero(w["flags"] == I.FLUID))
    F = np.array(p.F[:3])
    f0, _ = s.populations()
    for _ in range(3):
        Fw = sum(s.wall_force(i) for i in range(3))
        s.step(1)
        f1, _ = s.populations()
        expect = n_fluid * F - e.T @ (f1.sum(axis=1) - f0.sum(axis=1))
        assert np.abs(Fw - expect).max() <= 1e-11, (Fw, expect)
        assert np.abs(Fw).max() > 1e-3
        f0 = f1


def test_force_objective_refused_by_the_h_adjoint():
    import torch
    from paper_2203_01316_gb300 import LBMError
    w, p, s = _box_solver("f32")
    N = s.N
    u = torch.zeros(3 * N, dtype=torch.float32, device="cuda")
    mu = torch.zeros(27 * N, dtype=torch.float32, device="cuda")
    out = torch.empty_like(mu)
    with pytest.raises(LBMError, match="coupled adjoint"):
        s.adjoint_step(u, mu, out, obj=s.objective("force", 0, 1.0, 0))
    with pytest.raises(LBMError, match="component"):
        s.objective_accumulate(s.objective("force", 0, 1.0, 3), torch.zeros(1, dtype=torch.float64, device="cuda"))
