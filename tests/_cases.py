"""Builds the GPU solver and the FP64 oracle from one seeded workload, so the
parity tests feed both sides the same inputs."""
import numpy as np

from oracle import oracle as O
from paper_2203_01316_gb300 import inputs as I


def make_pair(w, nu, k, qh=27, hkind="trt", storage="f32", F=(0.0, 0.0, 0.0), wall_T=(1.0,),
              rho0=1.0, T_ref=0.0, theta=None, omega_bulk=1.0, oracle=True, wall_bc="iabb", step_kernel="auto",
              round_nearest=False):
    from paper_2203_01316_gb300 import Solver
    nx, ny, nz = w["dims"]
    u_in = w.get("u_in", (0.0, 0.0, 0.0))
    T_in = w.get("T_in", 0.0)
    s = Solver(nx, ny, nz, nu=nu, k=k, lat_h=qh, hkind=hkind, storage=storage, periodic_x=w["periodic_x"],
               omega_bulk=omega_bulk, rho0=rho0, T_ref=T_ref, wall_bc=wall_bc, step_kernel=step_kernel,
               round_nearest=round_nearest)
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


def box_one_step(f_post, h_post, w, box, qh=27, hkind="trt", nu=0.03, k=2e-3, wall_T=(1.0,), F=(0.0, 0.0, 0.0)):
    """The oracle's next post-collision state on the interior of a sub-box of
    a large grid, for parity where the oracle cannot step the whole grid.

    box = (x0, x1, y0, y1, z0, z1), half-open, away from the inlet and outlet
    planes, with every solid node of the grid near it strictly inside it: the
    sub-box is stepped as a periodic grid, so its outermost layer pulls wrong
    values, and only the nodes one layer in are returned.  A node's step reads
    only its neighbours' post-collision values, its own links and q, so those
    interior nodes are computed from exactly their inputs in the full grid.
    Returns (global node indices, f[27, n], h[qh, n])."""
    nx, ny, nz = w["dims"]
    x0, x1, y0, y1, z0, z1 = box
    assert 1 <= x0 < x1 <= nx - 1 and 0 <= y0 < y1 <= ny and 0 <= z0 < z1 <= nz
    flags = np.asarray(w["flags"]).reshape(nz, ny, nx)
    sub = flags[z0:z1, y0:y1, x0:x1]
    bx, by, bz = x1 - x0, y1 - y0, z1 - z0
    # solids only two layers in from the box faces, and none in a two-node
    # halo outside it (so no link crosses the faces)
    halo = np.zeros_like(flags, dtype=bool)
    halo[max(z0 - 2, 0):z1 + 2, max(y0 - 2, 0):y1 + 2, max(x0 - 2, 0):x1 + 2] = True
    core = np.zeros_like(flags, dtype=bool)
    core[z0 + 2:z1 - 2, y0 + 2:y1 - 2, x0 + 2:x1 - 2] = True
    assert not np.any((flags == I.SOLID) & halo & ~core), "solid nodes near the box faces"
    assert np.all((sub == I.FLUID) | (sub == I.SOLID))
    zz, yy, xx = np.meshgrid(np.arange(z0, z1), np.arange(y0, y1), np.arange(x0, x1), indexing="ij")
    gidx = (xx + nx * (yy + ny * zz)).reshape(-1)
    local = -np.ones(nx * ny * nz, np.int64)
    local[gidx] = np.arange(gidx.size)
    links = w["links"]
    keep = local[links["node"]] >= 0
    sl = {"node": local[links["node"][keep]].astype(np.int32), "dir": links["dir"][keep],
          "q": links["q"][keep], "wall": links["wall"][keep]}
    p = O.make_params(nx=bx, ny=by, nz=bz, qh=qh, hkind=hkind, periodic_x=True, nu=nu, k=k, F=F)
    o = O.Oracle(p)
    o.set_geometry(sub.reshape(-1), sl, nwalls=w["nwalls"])
    for i, T in enumerate(wall_T[: w["nwalls"]]):
        o.set_wall_temperature(i, float(np.float32(T)))
    o.set_post(np.ascontiguousarray(f_post[:, gidx]), np.ascontiguousarray(h_post[:, gidx]))
    assert o.stream() == 0
    fo, ho = o.post()
    inner = np.zeros((bz, by, bx), bool)
    inner[1:-1, 1:-1, 1:-1] = True
    inner = inner.reshape(-1)
    return gidx[inner], fo[:, inner], ho[:, inner]
