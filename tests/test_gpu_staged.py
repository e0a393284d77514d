"""The staged step kernel (rows of the pull copied into shared memory by
asynchronous bulk copies) against the classic kernel (direct loads): both
run the same arithmetic on the same values, so every stored population must
agree to rounding level after two steps, relative to the largest stored
magnitude: 1e-6 for FP32 (26e-6 for the rest population of h, which closes
the zeroth moment from the others), 4 units in the last place for FP16/BF16
(ptxas may contract multiply-adds differently in the two kernels),
for every storage type the staged kernel serves and both h lattices; a wrong
source row shows up as a gross difference.  The staged kernel must also pass
the oracle's one-step check itself."""
import struct

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
        s.step(2)
        s.sync()
        out.append(_stored(s.save_state(), storage))
        s.close()
    a, b = out
    # rounding-level differences only: FP32 1e-6 of the largest stored
    # magnitude (wall links and collisions carry contraction differences),
    # 16-bit 4 units in the last place of it; a wrong source row is ~1e-2.
    # In FP32 the rest population of h closes the zeroth moment from the
    # other Q_h - 1 outputs, so it carries the sum of their differences:
    # (Q_h - 1) times the bound.
    N = nx * ny * nz
    assert a.size == (27 + qh) * N
    scale = np.abs(a).max()
    if storage == "f32":
        d = np.abs(a - b)
        rest = slice(27 * N, 28 * N)
        assert d[rest].max() <= (qh - 1) * 1e-6 * scale
        d[rest] = 0.0
        assert d.max() <= 1e-6 * scale
    else:
        assert np.abs(a - b).max() <= 4.0 * _ulp(np.array([scale]), storage)[0]


def _stored(blob, storage):
    """Stored values of a state blob as float64 (header: 8s, I, 5i, 3Q)."""
    off = struct.calcsize("<8sI5iQQQ")
    raw = np.frombuffer(blob, dtype=np.uint8, offset=off)
    if storage == "f32":
        return raw.view(np.float32).astype(np.float64)
    if storage == "f16":
        return raw.view(np.float16).astype(np.float64)
    return (raw.view(np.uint16).astype(np.uint32) << 16).view(np.float32).astype(np.float64)


def _ulp(x, storage):
    mant = {"f32": 23, "f16": 10, "bf16": 7}[storage]
    emin = {"f32": -126, "f16": -14, "bf16": -126}[storage]
    e = np.floor(np.log2(np.maximum(np.abs(x), 1e-300)))
    return np.exp2(np.maximum(e, emin) - mant)


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
