"""ctypes binding of the FP64 CPU oracle (lbm_oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the test suite, by the package smoke
check and by the CPU-baseline leg of the benchmark.  The GPU library never
imports, links or calls it.

`build()` compiles the C file with gcc (no fast-math, no FMA contraction, so
x86 and Arm give the same bits); `Oracle` wraps one simulation.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbm_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lib = None

KINDS = {"trt": 0, "srt": 1, "1st": 2, "cum1st": 3}


def build(force: bool = False) -> str:
    """Compile liboracle.so in-tree; returns its path."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math",
           "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int),
                ("qh", C.c_int), ("hkind", C.c_int), ("periodic_x", C.c_int),
                ("nu", C.c_double), ("k", C.c_double),
                ("omega_bulk", C.c_double), ("omega3", C.c_double), ("omega4", C.c_double),
                ("omega5", C.c_double), ("omega6", C.c_double),
                ("F", C.c_double * 3), ("u_in", C.c_double * 3), ("T_in", C.c_double), ("wall_bc", C.c_int),
                ("inlet_bc", C.c_int)]

WALL_BC = {"iabb": 0, "eq": 1, "abb": 2}
INLET_BC = {"equilibrium": 0, "zou_he": 1}


def make_params(nx=1, ny=1, nz=1, qh=27, hkind="trt", periodic_x=True, nu=0.02, k=2e-4,
                omega_bulk=1.0, omega3=1.0, omega4=1.0, omega5=1.0, omega6=1.0,
                F=(0.0, 0.0, 0.0), u_in=(0.0, 0.0, 0.0), T_in=0.0, wall_bc="iabb", inlet_bc="equilibrium") -> Params:
    p = Params()
    p.nx, p.ny, p.nz, p.qh = nx, ny, nz, qh
    p.hkind = KINDS[hkind] if isinstance(hkind, str) else int(hkind)
    p.periodic_x = 1 if periodic_x else 0
    p.nu, p.k = nu, k
    p.omega_bulk, p.omega3, p.omega4, p.omega5, p.omega6 = omega_bulk, omega3, omega4, omega5, omega6
    for d in range(3):
        p.F[d] = F[d]
        p.u_in[d] = u_in[d]
    p.T_in = T_in
    p.wall_bc = WALL_BC[wall_bc] if isinstance(wall_bc, str) else int(wall_bc)
    p.inlet_bc = INLET_BC[inlet_bc] if isinstance(inlet_bc, str) else int(inlet_bc)
    return p


def _d(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def lib():
    global _lib
    if _lib is None:
        _lib = C.CDLL(build())
        L = _lib
        L.orc_create.restype = C.c_void_p
        L.orc_create.argtypes = [C.POINTER(Params)]
        L.orc_destroy.argtypes = [C.c_void_p]
        L.orc_set_geometry.restype = C.c_int
        L.orc_set_geometry.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_int]
        L.orc_set_wall_temperature.argtypes = [C.c_void_p, C.c_int, C.c_double]
        L.orc_set_theta.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_init_fields.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        for name in ("orc_set_state", "orc_get_state", "orc_set_post", "orc_get_post"):
            getattr(L, name).argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_collide.argtypes = [C.c_void_p]
        L.orc_stream.restype = C.c_int
        L.orc_stream.argtypes = [C.c_void_p]
        L.orc_step.restype = C.c_int
        L.orc_step.argtypes = [C.c_void_p, C.c_int]
        L.orc_macros.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_balances.argtypes = [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.orc_surface_flux.restype = C.c_double
        L.orc_surface_flux.argtypes = [C.c_void_p, C.c_int]
        L.orc_lattice.argtypes = [C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_matrix_M.argtypes = [C.c_int, C.c_void_p]
        L.orc_matrix_T.argtypes = [C.c_int, C.c_void_p, C.c_void_p]
        L.orc_equilibrium.argtypes = [C.c_int, C.c_double, C.c_void_p, C.c_void_p]
        L.orc_cumulants.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_cumulants_inverse.argtypes = [C.c_void_p, C.c_void_p]
        L.orc_collide_f.argtypes = [C.POINTER(Params), C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_collide_h.argtypes = [C.POINTER(Params), C.c_void_p, C.c_void_p, C.c_double, C.c_void_p]
        L.orc_num_threads.restype = C.c_int
        L.orc_set_num_threads.argtypes = [C.c_int]
        L.orc_set_num_threads.restype = None
        L.orc_adjoint.restype = C.c_int
        L.orc_adjoint.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                  C.c_int, C.c_int, C.c_int, C.c_double, C.POINTER(C.c_double), C.c_void_p,
                                  C.c_void_p]
        L.orc_adjoint_flow.restype = C.c_int
        L.orc_adjoint_flow.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int,
                                       C.c_int, C.c_int, C.c_int, C.c_double, C.POINTER(C.c_double), C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p]
        L.orc_wall_force.argtypes = [C.c_void_p, C.c_int, C.c_void_p]
        L.orc_build_spheres.restype = C.c_int64
        L.orc_build_spheres.argtypes = [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                        C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p, C.c_void_p,
                                        C.c_void_p]
    return _lib


# ---- geometry --------------------------------------------------------------
def build_spheres(nx, ny, nz, centres, radii, wall_ids=None, periodic_x=False):
    """Flags and wall links of closed balls in an nx x ny x nz channel
    (orc_build_spheres: Sec. 3's q along each link, FP64, node by node).
    Returns (flags uint8[N], links dict of node, dir, q, wall)."""
    c = np.ascontiguousarray(np.asarray(centres, np.float64).reshape(-1, 3))
    r = np.ascontiguousarray(np.asarray(radii, np.float64).reshape(-1))
    w = None if wall_ids is None else np.ascontiguousarray(np.asarray(wall_ids, np.int32).reshape(-1))
    N = nx * ny * nz
    flags = np.empty(N, np.uint8)
    args = (nx, ny, nz, 1 if periodic_x else 0, int(r.size), c.ctypes.data, r.ctypes.data,
            w.ctypes.data if w is not None else None, flags.ctypes.data)
    n = lib().orc_build_spheres(*args, 0, None, None, None, None)
    node = np.empty(n, np.int32); dr = np.empty(n, np.int32)
    q = np.empty(n, np.float32); wall = np.empty(n, np.int32)
    m = lib().orc_build_spheres(*args, n, node.ctypes.data, dr.ctypes.data, q.ctypes.data, wall.ctypes.data)
    assert m == n
    return flags, {"node": node, "dir": dr, "q": q, "wall": wall}


# ---- single-node helpers -------------------------------------------------
def lattice(Q=27):
    e = np.zeros((Q, 3), np.int32)
    mom = np.zeros((Q, 3), np.int32)
    w = np.zeros(Q)
    opp = np.zeros(Q, np.int32)
    lib().orc_lattice(Q, e.ctypes.data, w.ctypes.data, opp.ctypes.data, mom.ctypes.data)
    return e, w, opp, mom


def matrix_M(Q=27):
    M = np.zeros((Q, Q))
    lib().orc_matrix_M(Q, M.ctypes.data)
    return M


def matrix_T(u, Q=27):
    T = np.zeros((Q, Q))
    uu = np.ascontiguousarray(u, dtype=np.float64)
    lib().orc_matrix_T(Q, uu.ctypes.data, T.ctypes.data)
    return T


def equilibrium(psi, u, Q=27):
    g = np.zeros(Q)
    uu = np.ascontiguousarray(u, dtype=np.float64)
    lib().orc_equilibrium(Q, float(psi), uu.ctypes.data, g.ctypes.data)
    return g


def cumulants(g):
    g = np.ascontiguousarray(g, dtype=np.float64)
    Cv = np.zeros(27)
    lib().orc_cumulants(g.ctypes.data, Cv.ctypes.data)
    return Cv


def cumulants_inverse(Cv):
    Cv = np.ascontiguousarray(Cv, dtype=np.float64)
    g = np.zeros(27)
    lib().orc_cumulants_inverse(Cv.ctypes.data, g.ctypes.data)
    return g


def collide_f(params: Params, f):
    f = np.ascontiguousarray(f, dtype=np.float64)
    fs = np.zeros(27)
    u = np.zeros(3)
    lib().orc_collide_f(C.byref(params), f.ctypes.data, fs.ctypes.data, u.ctypes.data)
    return fs, u


def collide_h(params: Params, h, u, Q=0.0):
    h = np.ascontiguousarray(h, dtype=np.float64)
    uu = np.ascontiguousarray(u, dtype=np.float64)
    hs = np.zeros(len(h))
    lib().orc_collide_h(C.byref(params), h.ctypes.data, uu.ctypes.data, float(Q), hs.ctypes.data)
    return hs


def num_threads() -> int:
    return int(lib().orc_num_threads())


def set_num_threads(n: int) -> None:
    """Threads used by the oracle's OpenMP loops from now on."""
    lib().orc_set_num_threads(int(n))


# ---- simulation ----------------------------------------------------------
def _objective_args(objective):
    """(kind, wall, plane, component) of an objective tuple: ("surface", wall,
    weight), ("section", plane_x, weight) or ("force", wall, weight, component)."""
    name = objective[0]
    if name == "surface":
        return 0, int(objective[1]), 0, 0
    if name == "section":
        return 1, 0, int(objective[1]), 0
    if name == "force":
        return 2, int(objective[1]), 0, int(objective[3])
    raise ValueError(f"unknown objective {name!r}")


class OracleError(RuntimeError):
    pass


class Oracle:
    """One FP64 oracle simulation.  Arrays are numpy, populations [Q][N] with
    node index n = x + nx*(y + ny*z)."""

    def __init__(self, params: Params):
        self.p = params
        self.N = params.nx * params.ny * params.nz
        self.qh = params.qh
        self._h = lib().orc_create(C.byref(params))

    def close(self):
        if self._h:
            lib().orc_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_geometry(self, flags, links=None, nwalls=1):
        flags = np.ascontiguousarray(flags, dtype=np.uint8).reshape(-1)
        if links is None:
            node = np.zeros(0, np.int32); dr = node; q = np.zeros(0, np.float32); wall = node
        else:
            node = np.ascontiguousarray(links["node"], dtype=np.int32)
            dr = np.ascontiguousarray(links["dir"], dtype=np.int32)
            q = np.ascontiguousarray(links["q"], dtype=np.float32)
            wall = np.ascontiguousarray(links["wall"], dtype=np.int32)
        rc = lib().orc_set_geometry(self._h, flags.ctypes.data, len(node), node.ctypes.data,
                                    dr.ctypes.data, q.ctypes.data, wall.ctypes.data, int(nwalls))
        if rc != 0:
            raise OracleError(f"orc_set_geometry rejected the geometry (code {rc})")

    def set_wall_temperature(self, wall, T):
        lib().orc_set_wall_temperature(self._h, int(wall), float(T))

    def set_theta(self, theta):
        th = np.ascontiguousarray(theta, dtype=np.float64).reshape(-1)
        lib().orc_set_theta(self._h, th.ctypes.data)

    def init_fields(self, rho, u, T):
        rho = np.ascontiguousarray(rho, dtype=np.float64).reshape(-1)
        u = np.ascontiguousarray(u, dtype=np.float64).reshape(-1)
        T = np.ascontiguousarray(T, dtype=np.float64).reshape(-1)
        lib().orc_init_fields(self._h, rho.ctypes.data, u.ctypes.data, T.ctypes.data)

    def step(self, n=1):
        rc = lib().orc_step(self._h, int(n))
        if rc != 0:
            raise OracleError(f"{rc} populations were left unset by streaming")

    def collide(self):
        lib().orc_collide(self._h)

    def stream(self):
        return lib().orc_stream(self._h)

    def state(self):
        f = np.zeros((27, self.N)); h = np.zeros((self.qh, self.N))
        lib().orc_get_state(self._h, f.ctypes.data, h.ctypes.data)
        return f, h

    def set_state(self, f, h):
        f = np.ascontiguousarray(f, dtype=np.float64); h = np.ascontiguousarray(h, dtype=np.float64)
        lib().orc_set_state(self._h, f.ctypes.data, h.ctypes.data)

    def post(self):
        """Post-collision populations of the current state (state unchanged)."""
        lib().orc_collide(self._h)
        f = np.zeros((27, self.N)); h = np.zeros((self.qh, self.N))
        lib().orc_get_post(self._h, f.ctypes.data, h.ctypes.data)
        return f, h

    def set_post(self, fs, hs):
        fs = np.ascontiguousarray(fs, dtype=np.float64); hs = np.ascontiguousarray(hs, dtype=np.float64)
        lib().orc_set_post(self._h, fs.ctypes.data, hs.ctypes.data)

    def macros(self):
        rho = np.zeros(self.N); u = np.zeros(3 * self.N); T = np.zeros(self.N)
        lib().orc_macros(self._h, rho.ctypes.data, u.ctypes.data, T.ctypes.data)
        return rho, u.reshape(3, self.N), T

    def balances(self):
        m = C.c_double(); e = C.c_double()
        lib().orc_balances(self._h, C.byref(m), C.byref(e))
        return m.value, e.value

    def surface_flux(self, wall):
        return float(lib().orc_surface_flux(self._h, int(wall)))

    def wall_force(self, wall):
        """Momentum-exchange force on a wall for the next transition (collides
        the current state first, like surface_flux)."""
        F = np.zeros(3)
        lib().orc_wall_force(self._h, int(wall), F.ctypes.data)
        return F

    def adjoint(self, f_post, h_post, nsteps, window, objective, nwalls=1, gradients=True):
        """J = weight * sum over levels k in window of the flux F(s^k), from the
        post-collision state (f_post, h_post) = s^0 over nsteps steps.
        objective: ("surface", wall, weight), ("section", plane_x, weight) or
        ("force", wall, weight, component) (the last for J only here; its
        gradients need adjoint_flow).
        Returns (J, dJ/dtheta[N], dJ/dT_w[nwalls]) (gradients None if not asked)."""
        kind, wall, plane, comp = _objective_args(objective)
        f_post = np.ascontiguousarray(f_post, dtype=np.float64)
        h_post = np.ascontiguousarray(h_post, dtype=np.float64)
        J = C.c_double()
        dth = np.zeros(self.N) if gradients else None
        dTw = np.zeros(nwalls) if gradients else None
        rc = lib().orc_adjoint(self._h, f_post.ctypes.data, h_post.ctypes.data, int(nsteps), int(window[0]),
                               int(window[1]), kind, wall, plane, comp, float(objective[2]), C.byref(J),
                               dth.ctypes.data if gradients else None, dTw.ctypes.data if gradients else None)
        if rc != 0:
            raise OracleError("orc_adjoint: " + {-4: "force objectives need adjoint_flow"}.get(rc, "streaming error"))
        return J.value, dth, dTw

    def adjoint_flow(self, f_post, h_post, nsteps, window, objective, nwalls=1):
        """Adjoint of the coupled f + h evolution: (J, dJ/dtheta[N],
        dJ/dT_w[nwalls], dJ/dF[3], dJ/du_in[3]) for the objective of
        adjoint() (F: body force; u_in: inlet velocity of the equilibrium
        inlet plane)."""
        kind, wall, plane, comp = _objective_args(objective)
        f_post = np.ascontiguousarray(f_post, dtype=np.float64)
        h_post = np.ascontiguousarray(h_post, dtype=np.float64)
        J = C.c_double()
        dth = np.zeros(self.N)
        dTw = np.zeros(nwalls)
        dF = np.zeros(3)
        duin = np.zeros(3)
        rc = lib().orc_adjoint_flow(self._h, f_post.ctypes.data, h_post.ctypes.data, int(nsteps), int(window[0]),
                                    int(window[1]), kind, wall, plane, comp, float(objective[2]), C.byref(J),
                                    dth.ctypes.data, dTw.ctypes.data, dF.ctypes.data, duin.ctypes.data)
        if rc != 0:
            raise OracleError("orc_adjoint_flow: streaming error")
        return J.value, dth, dTw, dF, duin
