"""Builds the GPU solver and the FP64 oracle from one seeded workload, so the
parity tests feed both sides the same inputs."""
import numpy as np

from oracle import oracle as O
from paper_2203_01316_gb300 import inputs as I


def make_pair(w, nu, k, qh=27, hkind="trt", storage="f32", F=(0.0, 0.0, 0.0), wall_T=(1.0,),
              rho0=1.0, T_ref=0.0, theta=None, omega_bulk=1.0, oracle=True, wall_bc="iabb"):
    from paper_2203_01316_gb300 import Solver
    nx, ny, nz = w["dims"]
    u_in = w.get("u_in", (0.0, 0.0, 0.0))
    T_in = w.get("T_in", 0.0)
    s = Solver(nx, ny, nz, nu=nu, k=k, lat_h=qh, hkind=hkind, storage=storage, periodic_x=w["periodic_x"],
               omega_bulk=omega_bulk, rho0=rho0, T_ref=T_ref, wall_bc=wall_bc)
    s.set_geometry(w["flags"], w["links"], n_walls=w["nwalls"])
    for i, T in enumerate(wall_T[: w["nwalls"]]):
        s.set_bc(i, T)
    if not w["periodic_x"]:
        s.set_inlet(u_in, T_in)
    s.set_force(F)
    if theta is not None:
        s.set_source(theta.astype(np.float32))
    s.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    o = None
    if oracle:
        p = O.make_params(nx=nx, ny=ny, nz=nz, qh=qh, hkind=hkind, periodic_x=w["periodic_x"], nu=nu, k=k,
                          F=F, u_in=u_in, T_in=T_in, omega_bulk=omega_bulk, wall_bc=wall_bc)
        o = O.Oracle(p)
        o.set_geometry(w["flags"], w["links"], nwalls=w["nwalls"])
        for i, T in enumerate(wall_T[: w["nwalls"]]):
            o.set_wall_temperature(i, float(np.float32(T)))
        if theta is not None:
            o.set_theta(theta.astype(np.float32).astype(np.float64))
        o.init_fields(w["rho"], w["u"].reshape(-1), w["T"])
    return s, o


def rel_l2(a, b, mask=None):
    a = np.asarray(a); b = np.asarray(b)
    if mask is not None:
        a = a[..., mask]; b = b[..., mask]
    return float(np.sqrt(np.sum((a - b) ** 2) / np.sum(b ** 2)))


def small_channel(nx=37, ny=19, nz=11, D=7.0, seed=7, u_in=0.03, T_in=0.2):
    """Multi-tile, ragged (no dimension a multiple of 32) channel with one sphere."""
    w = I.heated_sphere(nx, ny, nz, D=D, cx=nx / 3.0, seed=seed, u_in=u_in, T_in=T_in)
    return w
