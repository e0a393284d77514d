"""Symmetry rows and the Zou-He inlet (the boundary rules of the Sec. 4.4
confined cylinder) and the confined-cylinder case on the GPU path, through
the C ABI:

* one step of a small confined cylinder (inlet, outlet, two symmetry rows,
  a cylinder with wall links) against the oracle, every population, FP32
  and FP64, central-moment and cumulant h kinds, both wall-rule orders, both
  inlet rules (tolerances as in test_gpu_parity: 2e-6 FP32, 1e-13 FP64; the
  T ~ 10 temperature level is stored as deviations from T_ref = 10);
* the Zou-He inlet's prescribed moments on the GPU state;
* the half domain between two symmetry planes against the lower half of a
  mirror-symmetric periodic domain twice as tall (FP64, 1e-12);
* the geometry rules (the adjoints through these rules: test_gpu_adjoint_bc);
* the coarse mesh at Pr = 10 with CM-TRT and second-order walls against the
  Nusselt number the paper prints for it and its FEM reference."""
import os

import numpy as np
import pytest

from oracle import oracle as O
from paper_2203_01316_gb300 import inputs as I

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))


def _pair(w, storage, kind, wall_bc, nu=0.03, k=3e-3, inlet_bc="equilibrium"):
    from paper_2203_01316_gb300 import Solver
    nx, ny, nz = w["dims"]
    s = Solver(nx, ny, nz, nu=nu, k=k, hkind=kind, storage=storage, periodic_x=False, T_ref=w["T_in"],
               wall_bc=wall_bc, inlet_bc=inlet_bc)
    s.set_geometry(w["flags"], w["links"], n_walls=1)
    s.set_bc(0, w["T_cyl"])
    s.set_inlet(w["u_in"], w["T_in"])
    s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    o = O.Oracle(O.make_params(nx=nx, ny=ny, nz=nz, hkind=kind, periodic_x=False, nu=nu, k=k, u_in=w["u_in"],
                               T_in=w["T_in"], wall_bc=wall_bc, inlet_bc=inlet_bc))
    o.set_geometry(w["flags"], w["links"], nwalls=1)
    o.set_wall_temperature(0, w["T_cyl"])
    o.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    return s, o


@pytest.mark.parametrize("storage,tol", [("f32", 2e-6), ("f64", 1e-13)])
@pytest.mark.parametrize("kind,wall_bc,inlet_bc", [("trt", "iabb", "equilibrium"), ("1st", "eq", "equilibrium"),
                                                   ("cum1st", "iabb", "zou_he"), ("srt", "eq", "zou_he"),
                                                   ("trt", "iabb", "zou_he")])
def test_confined_one_step_matches_oracle(storage, tol, kind, wall_bc, inlet_bc):
    w = I.confined_cylinder(0.2, seed=4)
    s, o = _pair(w, storage, kind, wall_bc, inlet_bc=inlet_bc)
    s.step(6)
    f0, h0 = s.populations()
    o.set_post(f0, h0)
    assert o.stream() == 0
    fo, ho = o.post()
    s.step(1)
    f1, h1 = s.populations()
    assert np.abs(f1 - fo).max() < tol
    assert np.abs(h1 - ho).max() < tol
    assert np.all(f1[:, w["flags"] == I.MIRROR] == 0.0)


@pytest.mark.parametrize("inlet_bc", ["equilibrium", "zou_he"])
def test_confined_multi_step_fp64_matches_oracle(inlet_bc):
    w = I.confined_cylinder(0.2, seed=5)
    s, o = _pair(w, "f64", "trt", "iabb", inlet_bc=inlet_bc)
    s.step(40)
    o.step(40)
    fg, hg = s.populations()
    fo, ho = o.post()
    assert np.abs(fg - fo).max() < 1e-12 and np.abs(hg - ho).max() < 1e-11
    nx, ny, _ = w["dims"]
    ex = O.lattice(27)[0][:, 0]
    live = (w["flags"] != I.SOLID) & (w["flags"] != I.MIRROR)
    for xs in w["sections"]:
        plane = live & (np.arange(nx * ny) % nx == xs)
        ref = float((ex[:, None] * ho[:, plane]).sum())
        assert abs(s.section_flux(xs) - ref) < 1e-10 * max(1.0, abs(ref))
    assert abs(s.surface_flux(0) - o.surface_flux(0)) < 1e-10 * max(1.0, abs(o.surface_flux(0)))


def test_zou_he_inlet_moments_on_gpu():
    # the inlet nodes' pre-collision moments: rho u_in in x, none across,
    # rho T_in for h (the oracle streams the GPU's post-collision state)
    w = I.confined_cylinder(0.2, seed=6)
    s, o = _pair(w, "f64", "trt", "iabb", inlet_bc="zou_he")
    s.step(5)
    f0, h0 = s.populations()
    o.set_post(f0, h0)
    assert o.stream() == 0
    f, h = o.state()
    inlet = np.nonzero(w["flags"] == I.INLET)[0]
    e = O.lattice(27)[0].astype(float)
    rho = f[:, inlet].sum(axis=0)
    mom = e.T @ f[:, inlet]
    assert np.abs(mom[0] - rho * w["u_in"][0]).max() < 1e-13
    assert np.abs(mom[1:]).max() < 1e-13
    assert np.abs(h[:, inlet].sum(axis=0) - rho * w["T_in"]).max() < 1e-12


def test_half_domain_equals_mirror_symmetric_periodic_domain():
    from paper_2203_01316_gb300 import Solver
    nx, H, nz = 16, 10, 2
    nyf = 2 * H
    x = np.arange(nx)[None, None, :]
    y = np.arange(nyf)[None, :, None]
    z = np.arange(nz)[:, None, None]
    T = 0.8 + 0.1 * np.sin(2 * np.pi * x / nx) * np.cos(np.pi * (y + 0.5) / H) + 0 * z
    ux = 0.03 + 0.02 * np.cos(2 * np.pi * (y + 0.5) / H) * np.cos(2 * np.pi * z / nz)
    uy = 0.02 * np.sin(np.pi * (y + 0.5) / H) * np.cos(2 * np.pi * x / nx) + 0 * z
    uz = np.zeros_like(T)
    rho = 1.0 + 0.01 * np.cos(2 * np.pi * x / nx) * np.cos(np.pi * (y + 0.5) / H) + 0 * z
    T, ux, uy, uz, rho = (np.broadcast_to(a, (nz, nyf, nx)).copy() for a in (T, ux, uy, uz, rho))
    full = Solver(nx, nyf, nz, nu=0.04, k=0.01, storage="f64", T_ref=0.8)
    full.set_geometry(np.zeros(nx * nyf * nz, np.uint8), None)
    full.set_force((1e-4, 0.0, 0.0))
    full.init_fields(rho.reshape(-1), np.stack([ux, uy, uz]).reshape(-1), T.reshape(-1))
    ny = H + 2
    flags = np.zeros((nz, ny, nx), np.uint8)
    flags[:, 0, :] = I.MIRROR
    flags[:, ny - 1, :] = I.MIRROR

    def half(a):
        out = np.ones((nz, ny, nx))
        out[:, 1:H + 1, :] = a[:, :H, :]
        return out
    hs = Solver(nx, ny, nz, nu=0.04, k=0.01, storage="f64", T_ref=0.8)
    hs.set_geometry(flags.reshape(-1), None)
    hs.set_force((1e-4, 0.0, 0.0))
    hs.init_fields(half(rho).reshape(-1), np.stack([half(ux), half(uy), half(uz)]).reshape(-1),
                   half(T).reshape(-1))
    full.step(60)
    hs.step(60)
    _, uf, Tf = full.macros()
    _, uh, Th = hs.macros()
    Tf = Tf.reshape(nz, nyf, nx)[:, :H]
    Th = Th.reshape(nz, ny, nx)[:, 1:H + 1]
    uf = uf.reshape(3, nz, nyf, nx)[:, :, :H]
    uh = uh.reshape(3, nz, ny, nx)[:, :, 1:H + 1]
    assert np.abs(Th - Tf).max() < 1e-12
    assert np.abs(uh - uf).max() < 1e-12


def test_symmetry_and_inlet_geometry_rules():
    from paper_2203_01316_gb300 import LBMError, Solver
    w = I.confined_cylinder(0.2)
    nx, ny, nz = w["dims"]
    s = Solver(nx, ny, nz, nu=0.03, k=3e-3, periodic_x=False, T_ref=10.0)
    bad = w["flags"].copy().reshape(ny, nx)
    bad[0, 5] = I.FLUID  # a partial symmetry row
    with pytest.raises(LBMError):
        s.set_geometry(bad.reshape(-1), w["links"], n_walls=1)
    bad = w["flags"].copy().reshape(ny, nx)
    bad[3, :] = np.where(bad[3, :] == I.FLUID, I.MIRROR, bad[3, :])  # not a boundary row
    with pytest.raises(LBMError):
        s.set_geometry(bad.reshape(-1), w["links"], n_walls=1)
    s.set_geometry(w["flags"], w["links"], n_walls=1)
    z = Solver(nx, ny, nz, nu=0.03, k=3e-3, periodic_x=False, T_ref=10.0, inlet_bc="zou_he")
    bad = w["flags"].copy().reshape(ny, nx)
    bad[5, 1] = I.SOLID  # a solid node next to the Zou-He inlet
    with pytest.raises(LBMError):
        z.set_geometry(bad.reshape(-1), w["links"], n_walls=1)


def _paper_table():
    rows = {}
    with open(os.path.join(HERE, "golden", "confined_cylinder_nu.txt")) as fh:
        for line in fh:
            if line.startswith("#") or not line.strip():
                continue
            t = line.split()
            rows[(t[0], float(t[1]))] = [float(v) for v in t[2:]]
    return rows


def test_confined_coarse_pr10_trt_second_order_nusselt():
    import bench
    r = bench.confined_nu(1, "trt", "iabb", 10.0)
    paper = _paper_table()[("coarse", 10.0)]
    paper_trt_2nd, fem = paper[5], paper[8]
    assert r["converged"], r
    # measured 4.94: 2.5% above the FEM reference 4.82 and the paper's 4.81
    # (cylinder position and symmetry-plane placement are readings here)
    assert abs(r["Nu"] - fem) < 0.04 * fem, (r, fem, paper_trt_2nd)
    assert abs(r["Nu"] - paper_trt_2nd) < 0.04 * paper_trt_2nd
