"""Python binding of liblbm.so (include/lbm.h): argument marshalling only.

Every computation runs in the CUDA library; this module converts numpy
arrays / torch tensors to pointers and lbm_status codes to exceptions.  There
is no fallback: if the library is missing the import of `lib()` fails.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "liblbm.so")

LBM_OK, LBM_ERR_INVALID, LBM_ERR_NOMEM, LBM_ERR_CUDA, LBM_ERR_DIVERGED, LBM_ERR_STATE = range(6)
STATUS = {1: "LBM_ERR_INVALID", 2: "LBM_ERR_NOMEM", 3: "LBM_ERR_CUDA", 4: "LBM_ERR_DIVERGED", 5: "LBM_ERR_STATE"}
HKIND = {"trt": 0, "srt": 1, "1st": 2, "cum1st": 3}
INLET_BC = {"equilibrium": 0, "zou_he": 1}
STORAGE = {"f32": 0, "f64": 1, "f16": 2, "bf16": 3}

# every symbol declared in include/lbm.h
SYMBOLS = ["lbm_create", "lbm_destroy", "lbm_set_geometry", "lbm_set_bc", "lbm_set_inlet", "lbm_set_force",
           "lbm_set_source", "lbm_init_fields", "lbm_step", "lbm_macros", "lbm_get_populations", "lbm_balances",
           "lbm_surface_flux", "lbm_nusselt", "lbm_state_size", "lbm_save_state", "lbm_load_state",
           "lbm_stream_map", "lbm_get_links", "lbm_sync", "lbm_last_error", "lbm_balances_noalloc",
           "lbm_section_flux", "lbm_objective_accumulate", "lbm_step_record", "lbm_adjoint_step",
           "lbm_adjoint_wall_gradient", "lbm_step_record_h", "lbm_adjoint_step_h", "lbm_step_record_pre",
           "lbm_flow_record_size", "lbm_build_spheres", "lbm_adjoint_flow_step", "lbm_adjoint_flow_gradient", "lbm_wall_force"]
OBJ_SURFACE, OBJ_SECTION, OBJ_FORCE = 0, 1, 2


class Objective(C.Structure):
    """lbm_objective: J += weight * F(level), F the surface flux of a wall,
    the section flux of a plane or one component of a wall's force."""
    _fields_ = [("kind", C.c_int), ("wall_id", C.c_int), ("plane_x", C.c_int), ("component", C.c_int),
                ("weight", C.c_double)]


class LBMError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class Params(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("lat_h", C.c_int), ("hkind", C.c_int),
                ("storage", C.c_int), ("periodic_x", C.c_int), ("nu", C.c_double), ("k", C.c_double),
                ("Pr", C.c_double), ("omega_bulk", C.c_double), ("rho0", C.c_double), ("T_ref", C.c_double),
                ("cuda_stream", C.c_void_p), ("round_nearest", C.c_int), ("step_kernel", C.c_int),
                ("wall_bc", C.c_int), ("inlet_bc", C.c_int)]
WALL_BC = {"iabb": 0, "eq": 1, "abb": 2}
STEP_KERNEL = {"auto": 0, "classic": 1}


_lib = None


def lib():
    """Load liblbm.so (built by paper_2203_01316_gb300.build); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"liblbm.so is not built ({LIB_PATH}); run python -m paper_2203_01316_gb300.build")
    try:  # let the CUDA runtime come from the one PyTorch loaded
        import torch  # noqa: F401
    except Exception:
        pass
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, dbl = C.c_void_p, C.c_int, C.c_int64, C.c_double
    sig = {
        "lbm_create": [C.POINTER(Params), C.POINTER(vp)],
        "lbm_destroy": [vp],
        "lbm_set_geometry": [vp, vp, i64, vp, vp, vp, vp, i32, i32],
        "lbm_set_bc": [vp, i32, dbl],
        "lbm_set_inlet": [vp, dbl, dbl, dbl, dbl],
        "lbm_set_force": [vp, dbl, dbl, dbl],
        "lbm_set_source": [vp, vp, i32],
        "lbm_init_fields": [vp, vp, vp, vp, i32],
        "lbm_step": [vp, i32],
        "lbm_macros": [vp, vp, vp, vp, i32],
        "lbm_get_populations": [vp, vp, vp, i32],
        "lbm_balances": [vp, C.POINTER(dbl), C.POINTER(dbl)],
        "lbm_surface_flux": [vp, i32, C.POINTER(dbl)],
        "lbm_nusselt": [vp, i32, dbl, dbl, dbl, C.POINTER(dbl)],
        "lbm_state_size": [vp, C.POINTER(C.c_size_t)],
        "lbm_save_state": [vp, vp, C.POINTER(C.c_size_t), i32],
        "lbm_load_state": [vp, vp, C.c_size_t, i32],
        "lbm_section_flux": [vp, i32, C.POINTER(dbl)],
        "lbm_wall_force": [vp, i32, vp],
        "lbm_objective_accumulate": [vp, C.POINTER(Objective), vp],
        "lbm_step_record": [vp, i32, vp, i32],
        "lbm_adjoint_step": [vp, vp, vp, vp, C.POINTER(Objective), vp],
        "lbm_step_record_h": [vp, i32, vp, vp],
        "lbm_step_record_pre": [vp, i32, vp, vp],
        "lbm_flow_record_size": [vp, C.POINTER(C.c_int64), C.POINTER(C.c_int64)],
        "lbm_build_spheres": [vp, i32, vp, vp, vp, i32, vp],
        "lbm_adjoint_flow_step": [vp, vp, vp, vp, vp, vp, vp, C.POINTER(Objective), vp],
        "lbm_adjoint_flow_gradient": [vp, C.POINTER(dbl), C.POINTER(dbl), i32],
        "lbm_adjoint_step_h": [vp, vp, vp, vp, vp, C.POINTER(Objective), vp],
        "lbm_adjoint_wall_gradient": [vp, C.POINTER(dbl), i32],
        "lbm_stream_map": [vp, vp, i32],
        "lbm_get_links": [vp, C.POINTER(i64), vp, vp, vp, vp],
        "lbm_sync": [vp],
        "lbm_last_error": [vp],
        "lbm_balances_noalloc": [vp, vp, i32, i64, vp, vp, dbl, dbl, vp, vp],
    }
    for name, args in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = C.c_int
    L.lbm_last_error.restype = C.c_char_p
    _lib = L
    return L


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _ptr(x, dtype):
    """(pointer, is_device, keepalive) of a numpy array or torch tensor."""
    if x is None:
        return None, 0, None
    if _is_torch(x):
        import torch
        tdt = {np.float64: torch.float64, np.float32: torch.float32, np.int32: torch.int32,
               np.uint8: torch.uint8}[dtype]
        t = x.contiguous()
        if t.dtype != tdt:
            t = t.to(tdt)
        return t.data_ptr(), 1 if t.is_cuda else 0, t
    a = np.ascontiguousarray(x, dtype=dtype)
    return a.ctypes.data, 0, a


class Solver:
    """One lattice Boltzmann context (see include/lbm.h for the semantics).

    nx, ny, nz: grid; nu: viscosity; k or Pr: thermal diffusivity or Prandtl
    number; lat_h: 27 or 7; hkind: 'trt' | 'srt' | '1st' | 'cum1st'; storage:
    'f32' | 'f64' | 'f16' | 'bf16'; periodic_x: True, or False for an
    inlet/outlet channel; stream: a torch.cuda.Stream or raw handle, or None
    for a library-owned stream; round_nearest: 16-bit storage rounds to
    nearest instead of stochastically; step_kernel: 'auto' | 'classic'
    (implementation of the step); wall_bc: 'iabb'
    (Eq. IBB/IABB with q) | 'eq' (BB + EQ) | 'abb' (BB + ABB); inlet_bc:
    'equilibrium' (fixed inlet equilibria) | 'zou_he'."""

    def __init__(self, nx, ny, nz, nu, k=0.0, Pr=0.0, lat_h=27, hkind="trt", storage="f32", periodic_x=True,
                 omega_bulk=1.0, rho0=1.0, T_ref=0.0, stream=None, round_nearest=False, step_kernel="auto",
                 wall_bc="iabb", inlet_bc="equilibrium"):
        self.L = lib()
        p = Params()
        p.nx, p.ny, p.nz = int(nx), int(ny), int(nz)
        p.lat_h = int(lat_h)
        p.hkind = HKIND[hkind] if isinstance(hkind, str) else int(hkind)
        p.storage = STORAGE[storage] if isinstance(storage, str) else int(storage)
        p.periodic_x = 1 if periodic_x else 0
        p.nu, p.k, p.Pr = float(nu), float(k), float(Pr)
        p.omega_bulk, p.rho0, p.T_ref = float(omega_bulk), float(rho0), float(T_ref)
        if stream is not None and hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        p.cuda_stream = stream
        p.round_nearest = 1 if round_nearest else 0
        p.step_kernel = STEP_KERNEL[step_kernel] if isinstance(step_kernel, str) else int(step_kernel)
        p.wall_bc = WALL_BC[wall_bc] if isinstance(wall_bc, str) else int(wall_bc)
        p.inlet_bc = INLET_BC[inlet_bc] if isinstance(inlet_bc, str) else int(inlet_bc)
        self.params = p
        self.nx, self.ny, self.nz = p.nx, p.ny, p.nz
        self.N = p.nx * p.ny * p.nz
        self.qh = p.lat_h
        self.cumulant_h = p.hkind == HKIND["cum1st"]
        h = C.c_void_p()
        st = self.L.lbm_create(C.byref(p), C.byref(h))
        if st != LBM_OK:
            raise LBMError(st, self.L.lbm_last_error(None).decode())
        self._h = h

    # -- plumbing --
    def _check(self, st):
        if st != LBM_OK:
            raise LBMError(st, self.L.lbm_last_error(self._h).decode())

    def close(self):
        if getattr(self, "_h", None):
            self.L.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- set-up --
    def set_geometry(self, flags, links=None, n_walls=1):
        fp, fdev, k0 = _ptr(flags, np.uint8)
        if links is None or len(links["node"]) == 0:
            self._check(self.L.lbm_set_geometry(self._h, fp, 0, None, None, None, None, int(n_walls), fdev))
            return
        n_p, n_dev, k1 = _ptr(links["node"], np.int32)
        d_p, d_dev, k2 = _ptr(links["dir"], np.int32)
        q_p, q_dev, k3 = _ptr(links["q"], np.float32)
        w_p, w_dev, k4 = _ptr(links["wall"], np.int32)
        if len({fdev, n_dev, d_dev, q_dev, w_dev}) != 1:
            raise ValueError("flags and links must all be host arrays or all device tensors")
        self._check(self.L.lbm_set_geometry(self._h, fp, len(links["node"]), n_p, d_p, q_p, w_p, int(n_walls), fdev))

    def build_spheres(self, centres, radii, wall_ids=None, n_walls=1):
        """Geometry of closed balls (centres [n, 3], radii [n]) built on the
        device and installed; returns the flags (uint8[N])."""
        c = np.ascontiguousarray(np.asarray(centres, np.float64).reshape(-1, 3))
        r = np.ascontiguousarray(np.asarray(radii, np.float64).reshape(-1))
        w = None if wall_ids is None else np.ascontiguousarray(np.asarray(wall_ids, np.int32).reshape(-1))
        flags = np.empty(self.N, np.uint8)
        self._check(self.L.lbm_build_spheres(self._h, int(r.size), c.ctypes.data if r.size else None,
                                             r.ctypes.data if r.size else None,
                                             w.ctypes.data if w is not None else None, int(n_walls),
                                             flags.ctypes.data))
        return flags

    def set_bc(self, wall, T):
        self._check(self.L.lbm_set_bc(self._h, int(wall), float(T)))

    def set_inlet(self, u, T):
        self._check(self.L.lbm_set_inlet(self._h, float(u[0]), float(u[1]), float(u[2]), float(T)))
        self.inlet = (tuple(float(v) for v in u), float(T))

    def set_force(self, F):
        self._check(self.L.lbm_set_force(self._h, float(F[0]), float(F[1]), float(F[2])))

    def set_source(self, theta):
        p, dev, keep = _ptr(theta, np.float32)
        self._check(self.L.lbm_set_source(self._h, p, dev))

    def init_fields(self, rho, u, T):
        rp, rd, k0 = _ptr(rho, np.float64)
        up, ud, k1 = _ptr(u, np.float64)
        tp, td, k2 = _ptr(T, np.float64)
        if len({rd, ud, td}) != 1:
            raise ValueError("rho, u, T must all be host arrays or all device tensors")
        self._check(self.L.lbm_init_fields(self._h, rp, up, tp, rd))

    # -- time stepping --
    def step(self, n=1):
        self._check(self.L.lbm_step(self._h, int(n)))

    def sync(self):
        self._check(self.L.lbm_sync(self._h))

    # -- outputs --
    def macros(self, device=None):
        """(rho[N], u[3, N], T[N]) as numpy (device None) or torch tensors on `device`."""
        if device is None:
            rho = np.empty(self.N); u = np.empty(3 * self.N); T = np.empty(self.N)
            self._check(self.L.lbm_macros(self._h, rho.ctypes.data, u.ctypes.data, T.ctypes.data, 0))
            return rho, u.reshape(3, self.N), T
        import torch
        rho = torch.empty(self.N, dtype=torch.float64, device=device)
        u = torch.empty(3 * self.N, dtype=torch.float64, device=device)
        T = torch.empty(self.N, dtype=torch.float64, device=device)
        self._check(self.L.lbm_macros(self._h, rho.data_ptr(), u.data_ptr(), T.data_ptr(), 1))
        return rho, u.view(3, self.N), T

    def populations(self):
        f = np.empty((27, self.N)); h = np.empty((self.qh, self.N))
        self._check(self.L.lbm_get_populations(self._h, f.ctypes.data, h.ctypes.data, 0))
        return f, h

    def balances(self):
        m = C.c_double(); e = C.c_double()
        self._check(self.L.lbm_balances(self._h, C.byref(m), C.byref(e)))
        return m.value, e.value

    def surface_flux(self, wall):
        q = C.c_double()
        self._check(self.L.lbm_surface_flux(self._h, int(wall), C.byref(q)))
        return q.value

    def nusselt(self, wall, length, area, dT):
        v = C.c_double()
        self._check(self.L.lbm_nusselt(self._h, int(wall), float(length), float(area), float(dT), C.byref(v)))
        return v.value

    def state_size(self) -> int:
        n = C.c_size_t()
        self._check(self.L.lbm_state_size(self._h, C.byref(n)))
        return n.value

    def save_state(self, out=None):
        """bytes (host) or, with `out` a CUDA uint8 tensor of state_size()
        bytes, a device copy written into `out`."""
        n = C.c_size_t(self.state_size())
        if out is not None:
            self._check(self.L.lbm_save_state(self._h, out.data_ptr(), C.byref(n), 1))
            return out
        buf = C.create_string_buffer(n.value)
        self._check(self.L.lbm_save_state(self._h, buf, C.byref(n), 0))
        return buf.raw[: n.value]

    def load_state(self, data):
        if _is_torch(data):
            self._check(self.L.lbm_load_state(self._h, data.data_ptr(), data.numel(), 1 if data.is_cuda else 0))
        else:
            self._check(self.L.lbm_load_state(self._h, data, len(data), 0))

    def section_flux(self, plane_x):
        q = C.c_double()
        self._check(self.L.lbm_section_flux(self._h, int(plane_x), C.byref(q)))
        return q.value

    def wall_force(self, wall):
        """Momentum-exchange force on a wall (numpy float64[3])."""
        F = np.zeros(3)
        self._check(self.L.lbm_wall_force(self._h, int(wall), F.ctypes.data))
        return F

    # -- adjoint (device tensors; see include/lbm.h) --
    @staticmethod
    def objective(kind, index, weight=1.0, component=0):
        """kind "surface" (index: wall), "section" (index: plane x) or
        "force" (index: wall; component 0, 1, 2)."""
        o = Objective()
        o.kind = {"surface": OBJ_SURFACE, "section": OBJ_SECTION, "force": OBJ_FORCE}[kind]
        o.wall_id = int(index) if o.kind != OBJ_SECTION else 0
        o.plane_x = int(index) if o.kind == OBJ_SECTION else 0
        o.component = int(component)
        o.weight = float(weight)
        return o

    def objective_accumulate(self, obj, J_device):
        self._check(self.L.lbm_objective_accumulate(self._h, C.byref(obj), J_device.data_ptr()))

    def step_record(self, n, u_rec, advance_h=True, h_rec=None):
        """n steps recording u per step into u_rec ([n, 3, N] device tensor);
        with h_rec ([n, Q_h, N]) also the post-collision h deviations, which
        the Cumulants-1st adjoint needs (advances h)."""
        if h_rec is not None:
            self._check(self.L.lbm_step_record_h(self._h, int(n), u_rec.data_ptr() if n > 0 else None,
                                                 h_rec.data_ptr() if n > 0 else None))
            return
        self._check(self.L.lbm_step_record(self._h, int(n), u_rec.data_ptr() if n > 0 else None,
                                           1 if advance_h else 0))

    def adjoint_step(self, u_level, mu_next, out, obj=None, dtheta=None, h_level=None):
        """One reverse level; h_level (the level's h record) is required for
        the Cumulants-1st kind and ignored by the central-moment kinds."""
        args = (u_level.data_ptr() if u_level is not None else None, mu_next.data_ptr(), out.data_ptr(),
                C.byref(obj) if obj is not None else None, dtheta.data_ptr() if dtheta is not None else None)
        if h_level is not None or self.cumulant_h:
            self._check(self.L.lbm_adjoint_step_h(self._h, args[0],
                                                  h_level.data_ptr() if h_level is not None else None, *args[1:]))
        else:
            self._check(self.L.lbm_adjoint_step(self._h, *args))

    def flow_record_size(self):
        """Elements (F, H) of one level's f and h records of step_record_pre."""
        f = C.c_int64()
        h = C.c_int64()
        self._check(self.L.lbm_flow_record_size(self._h, C.byref(f), C.byref(h)))
        return int(f.value), int(h.value)

    def step_record_pre(self, n, f_rec, h_rec):
        """n steps recording what the coupled adjoint needs of each level's
        pre-collision arrivals into device tensors f_rec (n x F elements: the
        ten f moments, plus the Zou-He inlet nodes' arrivals) and h_rec
        (n x Q_h N: the h arrivals), FP32/FP64; (F, Q_h N) = flow_record_size()."""
        self._check(self.L.lbm_step_record_pre(self._h, int(n), f_rec.data_ptr() if n > 0 else None,
                                               h_rec.data_ptr() if n > 0 else None))

    def adjoint_flow_step(self, f_level, h_level, muf_next, muh_next, muf_out, muh_out, obj=None, dtheta=None):
        """One level of the coupled f + h adjoint (f_level, h_level None at
        the initial level)."""
        self._check(self.L.lbm_adjoint_flow_step(
            self._h, f_level.data_ptr() if f_level is not None else None,
            h_level.data_ptr() if h_level is not None else None, muf_next.data_ptr(), muh_next.data_ptr(),
            muf_out.data_ptr(), muh_out.data_ptr(), C.byref(obj) if obj is not None else None,
            dtheta.data_ptr() if dtheta is not None else None))

    def adjoint_flow_gradient(self, reset=True):
        """(dJ/dF[3], dJ/du_in[3]) accumulated by adjoint_flow_step."""
        dF = (C.c_double * 3)()
        du = (C.c_double * 3)()
        self._check(self.L.lbm_adjoint_flow_gradient(self._h, dF, du, 1 if reset else 0))
        return np.array(dF[:]), np.array(du[:])

    def adjoint_wall_gradient(self, n_walls, reset=True):
        g = (C.c_double * n_walls)()
        self._check(self.L.lbm_adjoint_wall_gradient(self._h, g, 1 if reset else 0))
        return np.array(g[:], dtype=np.float64)

    def stream_map(self):
        src = np.empty((27, self.N), np.int32)
        self._check(self.L.lbm_stream_map(self._h, src.ctypes.data, 0))
        return src

    def links(self):
        n = C.c_int64(0)
        self._check(self.L.lbm_get_links(self._h, C.byref(n), None, None, None, None))
        node = np.empty(n.value, np.int32); dr = np.empty(n.value, np.int32)
        q = np.empty(n.value, np.float32); wall = np.empty(n.value, np.int32)
        cap = C.c_int64(n.value)
        self._check(self.L.lbm_get_links(self._h, C.byref(cap), node.ctypes.data, dr.ctypes.data,
                                         q.ctypes.data, wall.ctypes.data))
        return {"node": node, "dir": dr, "q": q, "wall": wall}
