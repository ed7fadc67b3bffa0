"""ctypes wrapper of the FP64 C oracle (test infrastructure only).

Parameters are passed as a plain dict whose keys are the fields of
``orc_params`` in ``lbm_oracle.h``; missing keys take the defaults below.
"""
import ctypes as C

import numpy as np

from . import build as _build

REC_FIELDS = ("t", "mass_n", "mass_phi", "mom_y", "neck", "breakup", "volume",
              "centroid_y", "velocity", "satellites", "runs", "head_y", "tail_y")


class _Params(C.Structure):
    _fields_ = [
        ("nx", C.c_int), ("ny", C.c_int),
        ("geometry", C.c_int),
        ("nozzle_width", C.c_int), ("nozzle_length", C.c_int), ("wall_thickness", C.c_int),
        ("rho_ink", C.c_double), ("rho_air", C.c_double),
        ("nu_ink", C.c_double), ("nu_air", C.c_double),
        ("sigma", C.c_double), ("width_W", C.c_double),
        ("tau_phi", C.c_double), ("gamma", C.c_double),
        ("theta_deg", C.c_double),
        ("F0", C.c_double), ("F_neg", C.c_double),
        ("T1", C.c_longlong), ("T2", C.c_longlong), ("T_idle", C.c_longlong),
        ("axial_bc", C.c_int),
        ("init_kind", C.c_int),
        ("init_x", C.c_double), ("init_y", C.c_double), ("init_r", C.c_double),
        ("jitter", C.c_double),
        ("seed", C.c_ulonglong),
        ("diag_every", C.c_int),
        ("nz", C.c_int),
        ("init_z", C.c_double),
    ]


DEFAULTS = dict(nx=8, ny=8, geometry=0, nozzle_width=0, nozzle_length=0, wall_thickness=0,
                rho_ink=10.0, rho_air=1.0, nu_ink=0.1, nu_air=0.05, sigma=0.01, width_W=3.0,
                tau_phi=0.8, gamma=0.0, theta_deg=90.0, F0=0.0, F_neg=0.0, T1=0, T2=0,
                T_idle=0, axial_bc=0, init_kind=0, init_x=0.0, init_y=0.0, init_r=0.0,
                jitter=1e-6, seed=0, diag_every=0, nz=1, init_z=0.0)

_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(_build.build())
        dp = C.POINTER(C.c_double)
        lib.orc_create.restype = C.c_void_p
        lib.orc_create.argtypes = [C.POINTER(_Params)]
        lib.orc_destroy.argtypes = [C.c_void_p]
        lib.orc_step.argtypes = [C.c_void_p, C.c_longlong]
        lib.orc_time.restype = C.c_longlong
        lib.orc_time.argtypes = [C.c_void_p]
        lib.orc_get_state.argtypes = [C.c_void_p, dp, dp]
        lib.orc_set_state.argtypes = [C.c_void_p, dp, dp, C.c_longlong]
        lib.orc_derived.argtypes = [C.c_void_p, dp]
        lib.orc_fields.argtypes = [C.c_void_p, dp, dp, dp, dp, dp]
        lib.orc_history.restype = C.c_int
        lib.orc_history.argtypes = [C.c_void_p, dp, C.c_int]
        lib.orc_kinds.argtypes = [C.c_void_p, C.POINTER(C.c_ubyte)]
        lib.orc_stream_only.argtypes = [C.c_void_p, dp, dp, dp, dp]
        lib.orc_feq.argtypes = [C.c_double] * 5 + [dp]
        lib.orc_geq.argtypes = [C.c_double] * 6 + [dp]
        lib.orc_force_term.argtypes = [C.c_double] * 5 + [dp]
        lib.orc_omega_of_theta.restype = C.c_double
        lib.orc_omega_of_theta.argtypes = [C.c_double]
        lib.orc_uniform.restype = C.c_double
        lib.orc_uniform.argtypes = [C.c_ulonglong, C.c_int, C.c_int]
        lib.orc_threads.restype = C.c_int
        lib.orc_threads.argtypes = []
        lib.orc_set_threads.argtypes = [C.c_int]
        _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def make_params(d):
    full = dict(DEFAULTS)
    unknown = set(d) - set(full)
    if unknown:
        raise KeyError("unknown oracle parameters: %s" % sorted(unknown))
    full.update(d)
    return _Params(**full)


class OracleSim:
    """One FP64 lattice; arrays are returned as numpy (9|5, ny, nx) float64."""

    def __init__(self, params: dict):
        self.lib = _load()
        self.params = dict(DEFAULTS, **params)
        self._p = make_params(params)
        self.nx, self.ny = self._p.nx, self._p.ny
        self.h = self.lib.orc_create(C.byref(self._p))
        if not self.h:
            raise ValueError("oracle rejected parameters")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.orc_destroy(h)
            self.h = None

    def step(self, n=1):
        self.lib.orc_step(self.h, int(n))

    @property
    def t(self):
        return self.lib.orc_time(self.h)

    def state(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((5, self.ny, self.nx))
        self.lib.orc_get_state(self.h, _dp(f), _dp(g))
        return f, g

    def set_state(self, f, g, t=0):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        self.lib.orc_set_state(self.h, _dp(f), _dp(g), int(t))

    def derived(self):
        out = np.empty(8)
        self.lib.orc_derived(self.h, _dp(out))
        keys = ("phis", "n0", "A", "kappa", "q", "h", "gamma", "Omega")
        return dict(zip(keys, out.tolist()))

    def fields(self):
        arrs = [np.empty((self.ny, self.nx)) for _ in range(5)]
        self.lib.orc_fields(self.h, *[_dp(a) for a in arrs])
        return dict(zip(("n", "phi", "mu", "ux", "uy"), arrs))

    def history(self):
        n = self.lib.orc_history(self.h, None, 0)
        out = np.empty((max(n, 1), len(REC_FIELDS)))
        self.lib.orc_history(self.h, _dp(out), n)
        return out[:n]

    def kinds(self):
        out = np.empty((self.ny, self.nx), dtype=np.uint8)
        self.lib.orc_kinds(self.h, out.ctypes.data_as(C.POINTER(C.c_ubyte)))
        return out

    def stream_only(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        fo = np.empty_like(f)
        go = np.empty_like(g)
        self.lib.orc_stream_only(self.h, _dp(f), _dp(g), _dp(fo), _dp(go))
        return fo, go


def feq(n, phi, mu, ux, uy):
    out = np.empty(9)
    _load().orc_feq(n, phi, mu, ux, uy, _dp(out))
    return out


def geq(phi, mu, ux, uy, gamma, q):
    out = np.empty(5)
    _load().orc_geq(phi, mu, ux, uy, gamma, q, _dp(out))
    return out


def force_term(tau, ux, uy, Fx, Fy):
    out = np.empty(9)
    _load().orc_force_term(tau, ux, uy, Fx, Fy, _dp(out))
    return out


def omega_of_theta(theta_deg):
    return _load().orc_omega_of_theta(theta_deg)


def uniform(seed, x, y):
    return _load().orc_uniform(seed, x, y)


def threads():
    """Threads the oracle's per-cell passes run on (1 without OpenMP)."""
    return _load().orc_threads()


def set_threads(n):
    """Run the per-cell passes on n threads (results are bit-identical)."""
    _load().orc_set_threads(int(n))


def _load3():
    lib = _load()
    if not getattr(lib, "_orc3_ready", False):
        dp = C.POINTER(C.c_double)
        lib.orc3_create.restype = C.c_void_p
        lib.orc3_create.argtypes = [C.POINTER(_Params)]
        lib.orc3_destroy.argtypes = [C.c_void_p]
        lib.orc3_step.argtypes = [C.c_void_p, C.c_longlong]
        lib.orc3_time.restype = C.c_longlong
        lib.orc3_time.argtypes = [C.c_void_p]
        lib.orc3_get_state.argtypes = [C.c_void_p, dp, dp]
        lib.orc3_set_state.argtypes = [C.c_void_p, dp, dp, C.c_longlong]
        lib.orc3_kinds.argtypes = [C.c_void_p, C.POINTER(C.c_ubyte)]
        lib.orc3_history.restype = C.c_int
        lib.orc3_history.argtypes = [C.c_void_p, dp, C.c_int]
        lib.orc3_stream_only.argtypes = [C.c_void_p, dp, dp, dp, dp]
        lib.orc3_feq.argtypes = [C.c_double] * 3 + [dp, dp]
        lib.orc3_geq.argtypes = [C.c_double, C.c_double, dp, C.c_double, C.c_double, dp]
        lib.orc3_force_term.argtypes = [C.c_double, dp, dp, dp]
        lib.orc3_lattice.argtypes = [C.POINTER(C.c_int)] * 3 + [dp]
        lib.orc3_uniform.restype = C.c_double
        lib.orc3_uniform.argtypes = [C.c_ulonglong, C.c_int, C.c_int, C.c_int]
        lib._orc3_ready = True
    return lib


class OracleSim3:
    """One FP64 3-D lattice (D3Q19/D3Q7); arrays are (19|7, nz, ny, nx)."""

    def __init__(self, params: dict):
        self.lib = _load3()
        self.params = dict(DEFAULTS, **params)
        self._p = make_params(params)
        self.nx, self.ny, self.nz = self._p.nx, self._p.ny, self._p.nz
        self.h = self.lib.orc3_create(C.byref(self._p))
        if not self.h:
            raise ValueError("oracle rejected parameters")

    def __del__(self):
        h = getattr(self, "h", None)
        if h:
            self.lib.orc3_destroy(h)
            self.h = None

    def step(self, n=1):
        self.lib.orc3_step(self.h, int(n))

    @property
    def t(self):
        return self.lib.orc3_time(self.h)

    def state(self):
        f = np.empty((19, self.nz, self.ny, self.nx))
        g = np.empty((7, self.nz, self.ny, self.nx))
        self.lib.orc3_get_state(self.h, _dp(f), _dp(g))
        return f, g

    def set_state(self, f, g, t=0):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        self.lib.orc3_set_state(self.h, _dp(f), _dp(g), int(t))

    def kinds(self):
        out = np.empty((self.nz, self.ny, self.nx), dtype=np.uint8)
        self.lib.orc3_kinds(self.h, out.ctypes.data_as(C.POINTER(C.c_ubyte)))
        return out

    def history(self):
        n = self.lib.orc3_history(self.h, None, 0)
        out = np.empty((max(n, 1), len(REC_FIELDS)))
        self.lib.orc3_history(self.h, _dp(out), n)
        return out[:n]

    def stream_only(self, f, g):
        f = np.ascontiguousarray(f, dtype=np.float64)
        g = np.ascontiguousarray(g, dtype=np.float64)
        fo, go = np.empty_like(f), np.empty_like(g)
        self.lib.orc3_stream_only(self.h, _dp(f), _dp(g), _dp(fo), _dp(go))
        return fo, go


def lattice3():
    lib = _load3()
    ex, ey, ez = (C.c_int * 19)(), (C.c_int * 19)(), (C.c_int * 19)()
    w = np.empty(19)
    lib.orc3_lattice(ex, ey, ez, _dp(w))
    return np.array(ex[:]), np.array(ey[:]), np.array(ez[:]), w


def feq3(n, phi, mu, u):
    out = np.empty(19)
    _load3().orc3_feq(n, phi, mu, _dp(np.ascontiguousarray(u, dtype=np.float64)), _dp(out))
    return out


def geq3(phi, mu, u, gamma, q):
    out = np.empty(7)
    _load3().orc3_geq(phi, mu, _dp(np.ascontiguousarray(u, dtype=np.float64)), gamma, q, _dp(out))
    return out


def force_term3(tau, u, F):
    out = np.empty(19)
    _load3().orc3_force_term(tau, _dp(np.ascontiguousarray(u, dtype=np.float64)),
                             _dp(np.ascontiguousarray(F, dtype=np.float64)), _dp(out))
    return out
