"""The sub-box stepping that the full-size GPU parity test uses
(box_one_step): on a grid the oracle can step whole, the interior of a box
stepped alone equals the whole grid's step there, bit for bit."""
import numpy as np

from oracle import oracle as O
from paper_2203_01316_gb300 import inputs as I

from _cases import box_one_step


def test_box_step_equals_the_whole_grid_step():
    w = I.heated_sphere(48, 26, 22, D=8.0, cx=20.0, seed=9, u_in=0.03, T_in=0.2)
    nx, ny, nz = w["dims"]
    N = nx * ny * nz
    w["u"] = w["u"] + I.uniform(3, 3 * N, -0.01, 0.01).reshape(3, N)
    w["u"][:, w["flags"] == I.SOLID] = 0.0
    w["T"] = I.uniform(4, N, 0.1, 0.9)
    nu, k = 0.03, 2e-3
    p = O.make_params(nx=nx, ny=ny, nz=nz, qh=27, hkind="trt", periodic_x=False, nu=nu, k=k, u_in=w["u_in"],
                      T_in=w["T_in"])
    o = O.Oracle(p)
    o.set_geometry(w["flags"], w["links"], nwalls=1)
    o.set_wall_temperature(0, 1.0)
    o.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    o.step(4)
    f0, h0 = o.post()
    c = np.floor(w["centre"]).astype(int)
    box = (c[0] - 9, c[0] + 10, c[1] - 9, c[1] + 10, c[2] - 8, c[2] + 9)
    idx, fb, hb = box_one_step(f0, h0, w, box, nu=nu, k=k, wall_T=(1.0,))
    assert o.stream() == 0
    f1, h1 = o.post()
    assert np.array_equal(fb, f1[:, idx]) and np.array_equal(hb, h1[:, idx])
    assert np.any(w["flags"][idx] == I.SOLID)  # the sphere is in the box
