"""Seeded synthetic inputs: geometries (node flags + wall links with their
wall-distance fractions q) and initial macroscopic fields.

This module holds no lattice Boltzmann arithmetic; it only builds what the
method consumes.  Both the GPU library and the CPU oracle are fed from it.

Random numbers come from splitmix64 (Steele, Lea & Flood 2014): output i of
seed s is mix(s + i * 0x9E3779B97F4A7C15), with the published mixing
constants; a double in [0,1) is the top 53 bits times 2^-53.

Conventions shared with the library:
  node index n = x + nx*(y + ny*z); flags 0 fluid, 1 solid, 2 inlet, 3 outlet;
  a wall link (n, a) means node n is fluid and n + e_a is solid, with q the
  fraction of the link at which the wall is crossed (Sec. 3 of the paper:
  "distance along the link between boundary node and wall").
"""
from __future__ import annotations

import math

import numpy as np

# D3Q27 velocity list in the paper's order (Sec. 2.1); geometry needs it to
# know which neighbour each link points at.
E27 = np.array([
    [0, 1, 0, 0, 1, 1, 0, -1, 0, 0, 1, 1, -1, -1, 0, 0, 1, -1, -1, 0, -1, 1, 1, 1, -1, -1, -1],
    [0, 0, 1, 0, 1, 0, 1, 0, -1, 0, -1, 0, 1, 0, 1, -1, 1, -1, 0, -1, 1, -1, 1, -1, 1, -1, -1],
    [0, 0, 0, 1, 0, 1, 1, 0, 0, -1, 0, -1, 0, 1, -1, 1, 1, 0, -1, -1, 1, 1, -1, -1, -1, 1, -1],
], dtype=np.int64).T

FLUID, SOLID, INLET, OUTLET, MIRROR = 0, 1, 2, 3, 4

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def splitmix64(seed: int, n: int, offset: int = 0) -> np.ndarray:
    """Outputs offset+1 .. offset+n of splitmix64 seeded with `seed` (uint64)."""
    i = np.arange(offset + 1, offset + n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed) + i * _GAMMA
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        z = z ^ (z >> np.uint64(31))
    return z


def uniform(seed: int, n: int, lo=0.0, hi=1.0, offset: int = 0) -> np.ndarray:
    u = (splitmix64(seed, n, offset) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return lo + (hi - lo) * u


def node_index(x, y, z, nx, ny):
    return x + nx * (y + ny * z)


def _empty_links():
    return {"node": np.zeros(0, np.int32), "dir": np.zeros(0, np.int32),
            "q": np.zeros(0, np.float32), "wall": np.zeros(0, np.int32)}


def _sort_links(node, dr, q, wall):
    node = np.asarray(node, np.int64)
    dr = np.asarray(dr, np.int64)
    order = np.lexsort((dr, node))
    return {"node": node[order].astype(np.int32), "dir": dr[order].astype(np.int32),
            "q": np.asarray(q, np.float32)[order], "wall": np.asarray(wall, np.int32)[order]}


def channel_flags(nx, ny, nz, periodic_x=False):
    """All-fluid box; with periodic_x False the x=0 plane is the inlet and
    x=nx-1 the outlet."""
    flags = np.zeros((nz, ny, nx), np.uint8)
    if not periodic_x:
        flags[:, :, 0] = INLET
        flags[:, :, nx - 1] = OUTLET
    return flags


def add_spheres(flags, centres, radii, wall_ids=None):
    """Mark closed balls |x-c|^2 <= R^2 solid (periodic images in y and z)
    and return the wall links of every fluid node next to them.  q is the
    smallest t in (0,1] with |x_b + t e_a - c| = R, computed in float64 and
    stored as float32.  Spheres must not touch one another."""
    nz, ny, nx = flags.shape
    centres = np.asarray(centres, np.float64).reshape(-1, 3)
    radii = np.asarray(radii, np.float64).reshape(-1)
    if wall_ids is None:
        wall_ids = np.zeros(len(radii), np.int32)
    boxes = []
    for c, R in zip(centres, radii):
        x0 = max(int(math.floor(c[0] - R)) - 1, 0)
        x1 = min(int(math.ceil(c[0] + R)) + 1, nx - 1)
        xs = np.arange(x0, x1 + 1)
        ys = np.arange(int(math.floor(c[1] - R)) - 1, int(math.ceil(c[1] + R)) + 2)
        zs = np.arange(int(math.floor(c[2] - R)) - 1, int(math.ceil(c[2] + R)) + 2)
        Z, Y, X = np.meshgrid(zs, ys, xs, indexing="ij")
        d2 = (X - c[0]) ** 2 + (Y - c[1]) ** 2 + (Z - c[2]) ** 2
        inside = d2 <= R * R
        flags[Z[inside] % nz, Y[inside] % ny, X[inside]] = SOLID
        boxes.append((X, Y, Z))
    nodes, dirs, qs, walls = [], [], [], []
    for (X, Y, Z), c, R, wid in zip(boxes, centres, radii, wall_ids):
        fluid = flags[Z % nz, Y % ny, X] == FLUID
        Xb, Yb, Zb = X[fluid], Y[fluid], Z[fluid]
        for a in range(1, 27):
            ex, ey, ez = E27[a]
            Xt = Xb + ex
            ok = (Xt >= 0) & (Xt < nx)
            Yt, Zt = Yb + ey, Zb + ez
            tgt_in = ((Xt - c[0]) ** 2 + (Yt - c[1]) ** 2 + (Zt - c[2]) ** 2) <= R * R
            hit = ok & tgt_in
            if not hit.any():
                continue
            dx, dy, dz = Xb[hit] - c[0], Yb[hit] - c[1], Zb[hit] - c[2]
            ee = float(ex * ex + ey * ey + ez * ez)
            de = dx * ex + dy * ey + dz * ez
            dd = dx * dx + dy * dy + dz * dz
            disc = np.maximum(de * de - ee * (dd - R * R), 0.0)
            t = (-de - np.sqrt(disc)) / ee
            t = np.clip(t, np.nextafter(0.0, 1.0), 1.0)
            q32 = t.astype(np.float32)
            q32 = np.where(q32 <= 0.0, np.float32(np.finfo(np.float32).tiny), q32)
            nodes.append(node_index(Xb[hit], Yb[hit] % ny, Zb[hit] % nz, nx, ny))
            dirs.append(np.full(hit.sum(), a))
            qs.append(q32)
            walls.append(np.full(hit.sum(), wid))
    if not nodes:
        return _empty_links()
    return _sort_links(np.concatenate(nodes), np.concatenate(dirs), np.concatenate(qs),
                       np.concatenate(walls))


def merge_links(*lists):
    return _sort_links(np.concatenate([l["node"] for l in lists]),
                       np.concatenate([l["dir"] for l in lists]),
                       np.concatenate([l["q"] for l in lists]),
                       np.concatenate([l["wall"] for l in lists]))


def plate_walls(flags, q_bottom=0.5, q_top=0.5, wall_bottom=0, wall_top=1):
    """Solid layers y=0 and y=ny-1; links of the fluid layers y=1 and y=ny-2
    crossing them, with the walls at y = 1 - q_bottom and y = ny-2 + q_top."""
    nz, ny, nx = flags.shape
    flags[:, 0, :] = SOLID
    flags[:, ny - 1, :] = SOLID
    nodes, dirs, qs, walls = [], [], [], []
    zz, xx = np.meshgrid(np.arange(nz), np.arange(nx), indexing="ij")
    for a in range(1, 27):
        ex, ey, ez = E27[a]
        if ey == 0:
            continue
        yb = 1 if ey < 0 else ny - 2
        sel = flags[zz, yb, xx] == FLUID
        if not sel.any():
            continue
        # a link whose target x leaves a non-periodic box hits the plane, not the wall
        n = node_index(xx[sel], yb, zz[sel], nx, ny)
        nodes.append(n)
        dirs.append(np.full(n.size, a))
        qs.append(np.full(n.size, q_bottom if ey < 0 else q_top, np.float32))
        walls.append(np.full(n.size, wall_bottom if ey < 0 else wall_top))
    return _sort_links(np.concatenate(nodes), np.concatenate(dirs), np.concatenate(qs),
                       np.concatenate(walls))


# ---- workloads -------------------------------------------------------------
def periodic_tgv(n=32, u0=(0.05, 0.03, 0.01), A=0.01, dT=0.1):
    """Fully periodic n^3 box: uniform velocity u0 plus a Taylor-Green vortex
    of amplitude A and wavenumber 2 pi/n, T = 1 + dT sin sin sin."""
    k = 2.0 * math.pi / n
    z, y, x = np.meshgrid(np.arange(n), np.arange(n), np.arange(n), indexing="ij")
    ux = u0[0] + A * np.sin(k * x) * np.cos(k * y) * np.cos(k * z)
    uy = u0[1] - A * np.cos(k * x) * np.sin(k * y) * np.cos(k * z)
    uz = np.full_like(ux, u0[2], dtype=np.float64)
    T = 1.0 + dT * np.sin(k * x) * np.sin(k * y) * np.sin(k * z)
    rho = np.ones_like(T)
    return {"dims": (n, n, n), "flags": np.zeros((n, n, n), np.uint8), "links": _empty_links(),
            "rho": rho.reshape(-1), "u": np.stack([ux, uy, uz]).reshape(3, -1),
            "T": T.reshape(-1), "periodic_x": True, "nwalls": 1}


def heated_sphere(nx=192, ny=64, nz=64, D=16.0, cx=48.0, seed=1234, u_in=0.02, T_in=0.0):
    """Channel with a sphere of diameter D centred at (cx, ny/2, nz/2) plus a
    seeded offset drawn uniformly in [0,1)^3; inlet at x=0, outlet at
    x=nx-1, periodic y and z; fluid starts at (rho=1, u_in, T_in)."""
    off = uniform(seed, 3)
    c = np.array([cx, ny / 2.0, nz / 2.0]) + off
    flags = channel_flags(nx, ny, nz, periodic_x=False)
    links = add_spheres(flags, [c], [D / 2.0])
    N = nx * ny * nz
    u = np.zeros((3, N))
    u[0] = u_in
    return {"dims": (nx, ny, nz), "flags": flags.reshape(-1), "links": links,
            "rho": np.ones(N), "u": u, "T": np.full(N, T_in), "periodic_x": False,
            "nwalls": 1, "centre": c, "D": D, "u_in": (u_in, 0.0, 0.0), "T_in": T_in}


def plate_channel(nx=128, ny=64, nz=64, q_bottom=0.5, q_top=0.5, seed=1234, theta_max=1e-5,
                  T0=0.5):
    """Periodic-x channel between a bottom wall (wall 0) and a top wall
    (wall 1); per-node heat source theta drawn uniformly in [0, theta_max]."""
    flags = channel_flags(nx, ny, nz, periodic_x=True)
    links = plate_walls(flags, q_bottom, q_top)
    N = nx * ny * nz
    theta = uniform(seed, N, 0.0, theta_max)
    theta[flags.reshape(-1) == SOLID] = 0.0
    return {"dims": (nx, ny, nz), "flags": flags.reshape(-1), "links": links,
            "rho": np.ones(N), "u": np.zeros((3, N)), "T": np.full(N, T0), "periodic_x": True,
            "nwalls": 2, "theta": theta, "H_c": (ny - 3) + q_bottom + q_top}


def porous_bed(nx=512, ny=256, nz=256, n_spheres=200, dmin=12.0, dmax=24.0, gap=2.0,
               seed=1234, u_in=0.01, T_in=0.0, max_tries=200000):
    """Channel with n_spheres non-overlapping spheres (diameters uniform in
    [dmin, dmax], surface gap >= gap with periodic minimum image in y and z,
    at least R + gap from the inlet and outlet planes), placed by rejection
    sampling from splitmix64."""
    centres, radii = [], []
    ctr = 0
    tries = 0
    while len(radii) < n_spheres and tries < max_tries:
        r = uniform(seed, 4, offset=ctr)
        ctr += 4
        tries += 1
        R = 0.5 * (dmin + (dmax - dmin) * r[0])
        c = np.array([R + gap + 1.0 + r[1] * (nx - 2 * (R + gap + 1.0) - 1.0), r[2] * ny, r[3] * nz])
        ok = True
        for c2, R2 in zip(centres, radii):
            d = c - c2
            d[1] -= ny * round(d[1] / ny)
            d[2] -= nz * round(d[2] / nz)
            if math.sqrt(float(d @ d)) < R + R2 + gap:
                ok = False
                break
        if ok:
            centres.append(c)
            radii.append(R)
    flags = channel_flags(nx, ny, nz, periodic_x=False)
    links = add_spheres(flags, centres, radii)
    N = nx * ny * nz
    u = np.zeros((3, N))
    u[0] = u_in
    return {"dims": (nx, ny, nz), "flags": flags.reshape(-1), "links": links,
            "rho": np.ones(N), "u": u, "T": np.full(N, T_in), "periodic_x": False,
            "nwalls": 1, "centres": np.array(centres), "radii": np.array(radii),
            "u_in": (u_in, 0.0, 0.0), "T_in": T_in}


def concentric_cylinders(D, seed=1234, margin=2):
    """Two coaxial cylinders along z (2-D: nz = 1): the inner one of
    diameter D/2 (wall 0) and the outer one of diameter D (wall 1), centre
    offset by a seeded sub-lattice shift; fluid between them.  Solid is
    r <= D/4 or r >= D/2 (distance in the x-y plane); q is the fraction of
    each link at which its projection crosses the circle."""
    n = int(math.ceil(D)) + 2 * margin
    off = uniform(seed, 2)
    c = np.array([n / 2.0 + off[0] - 0.5, n / 2.0 + off[1] - 0.5])
    R1, R2 = D / 4.0, D / 2.0
    y, x = np.meshgrid(np.arange(n), np.arange(n), indexing="ij")
    r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2
    flags = np.where((r2 <= R1 * R1) | (r2 >= R2 * R2), SOLID, FLUID).astype(np.uint8)
    nodes, dirs, qs, walls = [], [], [], []
    fl = flags == FLUID
    Xb, Yb = x[fl], y[fl]
    for a in range(1, 27):
        ex, ey, _ = E27[a]
        if ex == 0 and ey == 0:
            continue
        Xt, Yt = (Xb + ex) % n, (Yb + ey) % n
        tgt_solid = flags[Yt, Xt] == SOLID
        if not tgt_solid.any():
            continue
        dx, dy = Xb[tgt_solid] - c[0], Yb[tgt_solid] - c[1]
        tr2 = (Xb[tgt_solid] + ex - c[0]) ** 2 + (Yb[tgt_solid] + ey - c[1]) ** 2
        inner = tr2 <= R1 * R1
        ee = float(ex * ex + ey * ey)
        de = dx * ex + dy * ey
        dd = dx * dx + dy * dy
        R = np.where(inner, R1, R2)
        disc = np.maximum(de * de - ee * (dd - R * R), 0.0)
        # entering the inner circle: the smaller root; leaving the outer one: the larger
        t = np.where(inner, (-de - np.sqrt(disc)) / ee, (-de + np.sqrt(disc)) / ee)
        t = np.clip(t, np.nextafter(0.0, 1.0), 1.0)
        nodes.append(node_index(Xb[tgt_solid], Yb[tgt_solid], 0, n, n))
        dirs.append(np.full(int(tgt_solid.sum()), a))
        qs.append(t.astype(np.float32))
        walls.append(np.where(inner, 0, 1))
    links = _sort_links(np.concatenate(nodes), np.concatenate(dirs), np.concatenate(qs), np.concatenate(walls))
    N = n * n
    return {"dims": (n, n, 1), "flags": flags.reshape(-1), "links": links, "rho": np.ones(N),
            "u": np.zeros((3, N)), "T": np.full(N, 0.5), "periodic_x": True, "nwalls": 2,
            "centre": c, "R_inner": R1, "R_outer": R2,
            "r": np.sqrt(r2).reshape(-1)}


def gaussian_hill(L=256, sigma0_sq=100.0, C0=1.0, T0=1.0):
    """Periodic L x L x 1 box with T = T0 + C0 exp(-|x - x0|^2 / (2 sigma0^2))
    at rest (Sec. 4.1 initial condition; T0 keeps the zeroth moment of h
    positive for every collision kind)."""
    y, x = np.meshgrid(np.arange(L), np.arange(L), indexing="ij")
    x0 = L / 2.0
    C = C0 * np.exp(-((x - x0) ** 2 + (y - x0) ** 2) / (2.0 * sigma0_sq))
    N = L * L
    return {"dims": (L, L, 1), "flags": np.zeros(N, np.uint8), "links": _empty_links(), "rho": np.ones(N),
            "u": np.zeros((3, N)), "T": (T0 + C).reshape(-1), "periodic_x": True, "nwalls": 1}


def confined_cylinder(S=1, xc=None, seed=None, U=None, T_in=10.0, T_cyl=11.0):
    """Sec. 4.4 confined cylinder: a channel of L = 1000 S by H = 150 S nodes
    between two symmetry planes (rows y = 0 and y = ny - 1 are symmetry rows,
    so ny = H + 2 and the planes lie H apart), nz = 1; cylinder of diameter
    D = 30 S centred on the channel axis at x = xc (default L/5, a reading);
    inlet plane x = 0 at u = (U, 0, 0) with U = 0.01/S and T_in = 10, outlet
    x = L - 1; cylinder wall 0 at T_cyl = 11.  q from the exact crossing of
    the circle (2-D); a seeded sub-node offset of the centre when seed is
    given."""
    L, H, D = int(round(1000 * S)), int(round(150 * S)), 30.0 * S
    nx, ny = L, H + 2
    if xc is None:
        xc = L / 5.0
    c = np.array([float(xc), (ny - 1) / 2.0])
    if seed is not None:
        c += uniform(seed, 2, -0.5, 0.5)
    R = D / 2.0
    y, x = np.meshgrid(np.arange(ny), np.arange(nx), indexing="ij")
    r2 = (x - c[0]) ** 2 + (y - c[1]) ** 2
    flags = np.where(r2 <= R * R, SOLID, FLUID).astype(np.uint8)
    flags[:, 0] = INLET
    flags[:, nx - 1] = OUTLET
    flags[0, :] = MIRROR
    flags[ny - 1, :] = MIRROR
    fl = flags == FLUID
    Xb, Yb = x[fl], y[fl]
    nodes, dirs, qs = [], [], []
    for a in range(1, 27):
        ex, ey, _ = E27[a]
        if ex == 0 and ey == 0:
            continue
        Xt, Yt = Xb + ex, Yb + ey
        ok = (Xt >= 0) & (Xt < nx) & (Yt >= 0) & (Yt < ny)
        hit = np.zeros(len(Xb), bool)
        hit[ok] = flags[Yt[ok], Xt[ok]] == SOLID
        if not hit.any():
            continue
        dx, dy = Xb[hit] - c[0], Yb[hit] - c[1]
        ee = float(ex * ex + ey * ey)
        de = dx * ex + dy * ey
        dd = dx * dx + dy * dy
        disc = np.maximum(de * de - ee * (dd - R * R), 0.0)
        t = np.clip((-de - np.sqrt(disc)) / ee, np.nextafter(0.0, 1.0), 1.0)
        nodes.append(node_index(Xb[hit], Yb[hit], 0, nx, ny))
        dirs.append(np.full(int(hit.sum()), a))
        qs.append(t.astype(np.float32))
    links = _sort_links(np.concatenate(nodes), np.concatenate(dirs), np.concatenate(qs),
                        np.zeros(sum(len(v) for v in nodes), np.int64))
    N = nx * ny
    if U is None:
        U = 0.01 / S
    u = np.zeros((3, N))
    u[0] = np.where(flags.reshape(-1) == SOLID, 0.0, U)
    return {"dims": (nx, ny, 1), "flags": flags.reshape(-1), "links": links, "rho": np.ones(N), "u": u,
            "T": np.full(N, T_in), "periodic_x": False, "nwalls": 1, "u_in": (U, 0.0, 0.0), "T_in": T_in,
            "T_cyl": T_cyl, "D": D, "H": H, "centre": c, "S": S,
            "sections": (int(round(50 * S)), nx - 1 - int(round(100 * S)))}
