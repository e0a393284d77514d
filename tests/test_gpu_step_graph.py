"""lbm_step with LBM_STEP_AUTO replays CUDA graphs of two steps; it must give
the same bits as LBM_STEP_CLASSIC, which launches every step: over an odd
number of steps (graph replays plus a plain step), across parameter changes
between calls (the graph is captured again), with the three launches of a
step with symmetry rows and the Zou-He inlet, in FP32, FP64 and with
stochastically rounded FP16 and BF16 storage (whose graphs advance a device
copy of the time level that seeds the rounding)."""
import numpy as np
import pytest

from paper_2203_01316_gb300 import inputs as I

from _cases import make_pair

pytestmark = pytest.mark.gpu


def _both(make):
    a, b = make("auto"), make("classic")
    return a, b


def _same(a, b):
    fa, ha = a.populations()
    fb, hb = b.populations()
    assert np.array_equal(fa, fb) and np.array_equal(ha, hb)


@pytest.mark.parametrize("storage", ["f32", "f64", "f16", "bf16"])
def test_graph_steps_equal_plain_steps(storage):
    w = I.heated_sphere(38, 19, 11, D=7.0, cx=12.0, seed=7, u_in=0.03, T_in=0.2)
    a, b = _both(lambda k: make_pair(w, nu=0.03, k=2e-3, storage=storage, wall_T=(0.8,), T_ref=0.2,
                                     oracle=False, step_kernel=k)[0])
    for s in (a, b):
        s.step(37)
    _same(a, b)
    for s in (a, b):  # parameters change between calls: the graph is captured again
        s.set_inlet((0.02, 0.001, 0.0), 0.3)
        s.set_bc(0, 0.9)
        s.step(12)
    _same(a, b)
    a.close()
    b.close()


def test_graph_steps_with_symmetry_rows_and_zou_he():
    from paper_2203_01316_gb300 import Solver
    w = I.confined_cylinder(0.2, seed=4)
    nx, ny, nz = w["dims"]

    def make(kernel):
        s = Solver(nx, ny, nz, nu=0.03, k=3e-3, storage="f32", periodic_x=False, T_ref=w["T_in"],
                   inlet_bc="zou_he", step_kernel=kernel)
        s.set_geometry(w["flags"], w["links"], n_walls=1)
        s.set_bc(0, w["T_cyl"])
        s.set_inlet(w["u_in"], w["T_in"])
        s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
        return s

    a, b = _both(make)
    for s in (a, b):
        s.step(101)
    _same(a, b)
    a.close()
    b.close()
