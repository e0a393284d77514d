"""The staged step kernel (rows of the pull copied into shared memory by
asynchronous bulk copies) against the classic kernel (direct loads): both
run the same arithmetic on the same values, so every stored population must
agree bit for bit after several steps, for every storage type the staged
kernel serves and both h lattices; and the staged kernel must pass the
oracle's one-step check itself."""
import numpy as np
import pytest

from paper_2203_01316_gb300 import inputs as I

from _cases import make_pair

pytestmark = pytest.mark.gpu


def _cases():
    ch = I.heated_sphere(64, 13, 9, D=5.0, cx=20.0, seed=31, u_in=0.03, T_in=0.2)
    per = I.periodic_tgv(32)
    pl = I.plate_channel(nx=96, ny=11, nz=5, q_bottom=0.3, q_top=0.7, theta_max=1e-3, seed=32)
    return {"channel": ch, "periodic": per, "plate": pl}


@pytest.mark.parametrize("case", ["channel", "periodic", "plate"])
@pytest.mark.parametrize("storage", ["f32", "f16", "bf16"])
@pytest.mark.parametrize("qh", [27, 7])
def test_staged_equals_classic_bitwise(case, storage, qh):
    from paper_2203_01316_gb300 import Solver
    w = _cases()[case]
    nx, ny, nz = w["dims"]
    out = []
    for kernel in ("classic", "staged"):
        s = Solver(nx, ny, nz, nu=0.03, k=2e-3, lat_h=qh, storage=storage, periodic_x=w["periodic_x"],
                   T_ref=0.4, step_kernel=kernel)
        s.set_geometry(w["flags"], w["links"], n_walls=w["nwalls"])
        for i in range(w["nwalls"]):
            s.set_bc(i, 1.0 - 0.7 * i)
        if not w["periodic_x"]:
            s.set_inlet(w["u_in"], w["T_in"])
        if case == "plate":
            s.set_force((2e-4, 0.0, 1e-4))
            s.set_source(w["theta"].astype(np.float32))
        s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
        s.step(9)
        s.sync()
        out.append(s.save_state())
        s.close()
    assert out[0] == out[1]


def test_staged_rejected_where_it_does_not_apply():
    from paper_2203_01316_gb300 import LBMError, Solver
    with pytest.raises(LBMError):
        Solver(37, 8, 8, nu=0.03, k=2e-3, storage="f32", step_kernel="staged")
    with pytest.raises(LBMError):
        Solver(64, 8, 8, nu=0.03, k=2e-3, storage="f64", step_kernel="staged")


def test_auto_selects_the_classic_kernel():
    # same bits either way; auto must equal classic exactly
    from paper_2203_01316_gb300 import Solver
    w = _cases()["channel"]
    nx, ny, nz = w["dims"]
    out = []
    for kernel in ("auto", "classic"):
        s = Solver(nx, ny, nz, nu=0.03, k=2e-3, storage="f32", periodic_x=False, step_kernel=kernel)
        s.set_geometry(w["flags"], w["links"], n_walls=1)
        s.set_inlet(w["u_in"], w["T_in"])
        s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
        s.step(3)
        out.append(s.save_state())
    assert out[0] == out[1]


@pytest.mark.parametrize("storage,tol", [("f32", 2e-6)])
def test_staged_one_step_against_oracle(storage, tol):
    from oracle import oracle as O
    w = _cases()["channel"]
    s, o = make_pair(w, nu=0.03, k=2e-3, storage=storage, wall_T=(0.8,), T_ref=0.1)
    s.step(6)
    f0, h0 = s.populations()
    o.set_post(f0, h0)
    assert o.stream() == 0
    fo, ho = o.post()
    s.step(1)
    f1, h1 = s.populations()
    assert np.abs(f1 - fo).max() < tol and np.abs(h1 - ho).max() < tol
