"""16-bit storage (FP16 / BF16 deviations, FP32 arithmetic) against the FP64
oracle.

* One step from identical populations: every stored value within one unit in
  the last place of its 16-bit format (stochastic rounding picks either
  neighbour of the FP32 result; nearest rounding the closer one) plus 1e-6
  for the FP32 arithmetic.
* The heated-sphere crop (96 x 32 x 32, D = 8, Pr = 1000) over 200 steps:
  the sphere's Nusselt number, averaged over the last 20 steps, within 0.5%
  of the oracle for FP16 storage (the stated target) and within 2% for BF16,
  both with stochastic rounding; FP32 within 1e-4.  The relative L2 errors
  of u and T over the fluid nodes are stated beside it (FP32 at the 1e-5
  target; the 16-bit bounds sit just above the measured values).
"""
import math

import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01316_gb300 import inputs as I

from _cases import make_pair, small_channel

pytestmark = pytest.mark.gpu

MANT = {"f16": 10, "bf16": 7}


def _ulp(x, storage):
    """One unit in the last place of |x| in the 16-bit format."""
    a = np.abs(x)
    e = np.floor(np.log2(np.maximum(a, 1e-300)))
    if storage == "f16":
        e = np.maximum(e, -14.0)  # subnormal spacing 2^-24
    return np.exp2(e - MANT[storage])


@pytest.mark.parametrize("storage", ["f16", "bf16"])
@pytest.mark.parametrize("round_nearest", [False, True])
@pytest.mark.parametrize("qh", [27, 7])
def test_one_step_16bit(storage, round_nearest, qh):
    from paper_2203_01316_gb300 import Solver
    w = small_channel()
    nx, ny, nz = w["dims"]
    s = Solver(nx, ny, nz, nu=0.03, k=2e-3, lat_h=qh, storage=storage, periodic_x=False, T_ref=0.1,
               round_nearest=round_nearest)
    s.set_geometry(w["flags"], w["links"], n_walls=1)
    s.set_bc(0, 0.8)
    s.set_inlet(w["u_in"], w["T_in"])
    s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    s.step(5)
    p = O.make_params(nx=nx, ny=ny, nz=nz, qh=qh, periodic_x=False, nu=0.03, k=2e-3, u_in=w["u_in"],
                      T_in=w["T_in"])
    o = O.Oracle(p)
    o.set_geometry(w["flags"], w["links"], nwalls=1)
    o.set_wall_temperature(0, 0.8)
    f0, h0 = s.populations()
    o.set_post(f0, h0)
    assert o.stream() == 0
    fo, ho = o.post()
    s.step(1)
    f1, h1 = s.populations()
    _, w27, _, _ = O.lattice(27)
    _, wh, _, _ = O.lattice(qh)
    fdev = fo - w27[:, None] * 1.0
    hdev = ho - wh[:, None] * 0.1
    solid = np.asarray(w["flags"]) == I.SOLID
    scale = 1.0 if not round_nearest else 0.5
    bf = scale * _ulp(fdev, storage) + 1e-6
    bh = scale * _ulp(hdev, storage) + 1e-6
    assert np.all((np.abs(f1 - fo) <= bf)[:, ~solid])
    assert np.all((np.abs(h1 - ho) <= bh)[:, ~solid])


# relative L2 errors of u and T over the fluid nodes after the crop's 200
# steps, against the FP64 oracle, with the populations stored relative to
# the inflow temperature (T_ref = T_in): FP32 at the stated 1e-5 target, the
# 16-bit formats at upper bounds a little above the measured values
# (measured: FP32 6.0e-7 / 1.4e-6, FP16 3.9e-4 / 3.3e-4, BF16 3.4e-3 / 2.8e-3)
CROP_UT_BOUND = {"f32": (1e-5, 1e-5), "f16": (1e-3, 1e-3), "bf16": (1e-2, 1e-2)}


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_stochastic_rounding_is_unbiased(storage):
    """One step of a 48^3 periodic Taylor-Green box: the stored 16-bit values
    minus the oracle's exact post-collision values, in units of the format's
    spacing, average to zero (stochastic rounding rounds up with probability
    equal to the discarded fraction, so its error has zero mean; truncation
    would average -1/2, a bias in the random bits a clear fraction of it).
    Bound: 5 standard deviations of the mean of M errors of variance <= 1/4."""
    from paper_2203_01316_gb300 import Solver
    w = I.periodic_tgv(48)
    n = w["dims"][0]
    s = Solver(n, n, n, nu=0.03, k=2e-3, storage=storage, periodic_x=True, T_ref=1.0)
    s.set_geometry(w["flags"], w["links"], n_walls=1)
    s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    s.step(2)
    o = O.Oracle(O.make_params(nx=n, ny=n, nz=n, periodic_x=True, nu=0.03, k=2e-3))
    o.set_geometry(w["flags"], w["links"], nwalls=1)
    f0, h0 = s.populations()
    o.set_post(f0, h0)
    assert o.stream() == 0
    fo, ho = o.post()
    s.step(1)
    f1, h1 = s.populations()
    _, w27, _, _ = O.lattice(27)
    err = []
    for got, ref, shift in ((f1, fo, w27[:, None] * 1.0), (h1, ho, w27[:, None] * 1.0)):
        dev = ref - shift
        # stored values of at least 2^-8: their spacing (>= 2^-18 in FP16)
        # dwarfs the FP32 arithmetic's error (about 1e-9 here), which would
        # otherwise blur the rounding error of the smallest values
        big = np.abs(dev) >= 2.0 ** -8
        err.append(((got - ref) / _ulp(dev, storage))[big])
    e = np.concatenate(err)
    assert e.size > 5 * 10 ** 5
    assert np.all(np.abs(e) <= 1.0 + 1e-3)
    M = e.size
    assert abs(e.mean()) <= 5.0 * 0.5 / math.sqrt(M), (e.mean(), M)
    assert np.mean(np.abs(e) > 1e-3) > 0.5  # most values were rounded, not exact


def test_crop_nusselt_and_field_errors_16bit():
    from paper_2203_01316_gb300 import Solver
    w = I.heated_sphere(96, 32, 32, D=8.0, cx=24.0, seed=1234, u_in=0.02, T_in=0.0)
    nx, ny, nz = w["dims"]
    nu, k = 0.008, 8e-6     # Re = 20, Pr = 1000
    steps, win = 200, 20
    D = 8.0
    scale = D / (k * math.pi * D * D * 1.0) / win
    fluid = np.asarray(w["flags"]) == I.FLUID
    p = O.make_params(nx=nx, ny=ny, nz=nz, periodic_x=False, nu=nu, k=k, u_in=w["u_in"], T_in=0.0)
    o = O.Oracle(p)
    o.set_geometry(w["flags"], w["links"], nwalls=1)
    o.set_wall_temperature(0, 1.0)
    o.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    o.step(steps - win)
    Nu_ref = 0.0
    for _ in range(win):
        Nu_ref += o.surface_flux(0) * scale
        o.step(1)
    _, uo, To = o.macros()
    for storage, tol in (("f32", 1e-4), ("f16", 5e-3), ("bf16", 2e-2)):
        s = Solver(nx, ny, nz, nu=nu, k=k, storage=storage, periodic_x=False, T_ref=w["T_in"])
        s.set_geometry(w["flags"], w["links"], n_walls=1)
        s.set_bc(0, 1.0)
        s.set_inlet(w["u_in"], 0.0)
        s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
        s.step(steps - win)
        Nu = 0.0
        for _ in range(win):
            Nu += s.surface_flux(0) * scale
            s.step(1)
        _, ug, Tg = s.macros()
        eu = float(np.sqrt(np.sum((ug[:, fluid] - uo[:, fluid]) ** 2) / np.sum(uo[:, fluid] ** 2)))
        eT = float(np.sqrt(np.sum((Tg[fluid] - To[fluid]) ** 2) / np.sum(To[fluid] ** 2)))
        eNu = abs(Nu - Nu_ref) / abs(Nu_ref)
        print(f"crop 96x32x32 {storage}: rel L2 u {eu:.3e}, T {eT:.3e}, Nu {eNu:.3e}")
        assert eNu <= tol, (storage, Nu, Nu_ref)
        bu, bT = CROP_UT_BOUND[storage]
        assert eu <= bu and eT <= bT, (storage, eu, eT)
        s.close()
