"""Thin ctypes binding of libinkjet.so (include/inkjet.h).

Argument marshalling only: every step of the lattice update runs in the
library's CUDA kernels.  Functions carry the C names.  Parameters are plain
dicts keyed by the fields of ``ij_params``; missing keys take DEFAULTS.
Device memory comes from PyTorch's caching allocator and work is enqueued on
PyTorch's current CUDA stream unless told otherwise.

Importing this module loads the library and raises if it is missing; there
is no fallback of any kind.
"""
import ctypes as C
import os
import re

import numpy as np

from . import build as _build

IJ_OK, IJ_ERR_PARAM, IJ_ERR_CUDA, IJ_ERR_NUMERIC, IJ_ERR_TIMEOUT, IJ_ERR_STATE, IJ_ERR_OOM = range(7)
REC_FIELDS = ("step", "mass_n", "mass_phi", "mom_y", "neck", "breakup_step", "droplet_volume",
              "droplet_centroid_y", "droplet_velocity", "satellites", "runs", "head_y", "tail_y")
HEADER = os.path.join(_build.ROOT, "include", "inkjet.h")


class InkjetError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("inkjet status %d: %s" % (status, msg))
        self.status = status


class ij_params(C.Structure):
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
        ("precision", C.c_int),
        ("dim", C.c_int),
        ("nz", C.c_int),
        ("init_z", C.c_double),
    ]


class ij_obs(C.Structure):
    _fields_ = [(name, C.c_double) for name in REC_FIELDS]


DEFAULTS = dict(nx=8, ny=8, geometry=0, nozzle_width=0, nozzle_length=0, wall_thickness=0,
                rho_ink=10.0, rho_air=1.0, nu_ink=0.1, nu_air=0.05, sigma=0.01, width_W=3.0,
                tau_phi=0.8, gamma=0.0, theta_deg=90.0, F0=0.0, F_neg=0.0, T1=0, T2=0,
                T_idle=0, axial_bc=0, init_kind=0, init_x=0.0, init_y=0.0, init_r=0.0,
                jitter=1e-6, seed=0, diag_every=0, precision=0, dim=2, nz=1, init_z=0.0)

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

_lib = C.CDLL(_build.build())
_vp, _ll, _i, _dp, _fp = C.c_void_p, C.c_longlong, C.c_int, C.POINTER(C.c_double), C.c_void_p
_sig = {
    "ij_create": [C.POINTER(ij_params), _i, ALLOC_FN, FREE_FN, _vp, _vp, C.POINTER(_vp)],
    "ij_step": [_vp, _ll],
    "ij_observe": [_vp, _i, C.POINTER(ij_obs), _fp, _i],
    "ij_history": [_vp, _i, _dp, _i, C.POINTER(_i)],
    "ij_get_state": [_vp, _i, _fp, _fp, _i],
    "ij_set_state": [_vp, _i, _fp, _fp, _ll, _i],
    "ij_time": [_vp, C.POINTER(_ll)],
    "ij_launch_count": [_vp, C.POINTER(_ll)],
    "ij_kernel_timing": [_vp, _i, _dp, C.POINTER(_ll)],
    "ij_step_noalloc": [C.POINTER(ij_params), _ll, _fp, _fp, _fp, _fp, _fp, _fp, _vp],
    "ij_tune": [_vp, _i, _i, _i],
    "ij_autotune": [_vp, _i],
    "ij_use_graph": [_vp, _i],
    "ij_get_tuning": [_vp, _i, C.POINTER(_i), C.POINTER(_i), C.POINTER(_i), C.POINTER(_i)],
    "ij_destroy": [_vp],
}
for _name, _args in _sig.items():
    getattr(_lib, _name).argtypes = _args
    getattr(_lib, _name).restype = C.c_int
_lib.ij_last_error.restype = C.c_char_p
_lib.ij_last_error.argtypes = []


def library_path():
    return _lib._name


def declared_symbols():
    """Names of the entry points include/inkjet.h declares."""
    with open(HEADER) as fh:
        text = fh.read()
    return sorted(set(re.findall(r"\b(ij_[a-z_]+)\s*\(", text)) - {"ij_alloc_fn", "ij_free_fn"})


def _lattice(h, index):
    """Parameters of lattice ``index``; an out-of-range index is passed to
    the library (with no buffers) so that it reports the error itself."""
    if 0 <= index < len(h.lattices):
        return h.lattices[index]
    _check(_lib.ij_get_state(h.ptr, int(index), None, None, 0))
    raise InkjetError(IJ_ERR_PARAM, "index out of range")


def _grid(p):
    """Cell-array shape of a lattice: (ny, nx), or (nz, ny, nx) in 3-D."""
    if p.get("dim", 2) == 3:
        return (p["nz"], p["ny"], p["nx"])
    return (p["ny"], p["nx"])


def _nq(p):
    """Number of f and g directions: D2Q9/D2Q5 or D3Q19/D3Q7."""
    return (19, 7) if p.get("dim", 2) == 3 else (9, 5)


def _check(status):
    if status != IJ_OK:
        raise InkjetError(status, _lib.ij_last_error().decode())
    return status


def make_params(d):
    full = dict(DEFAULTS)
    unknown = set(d) - set(full)
    if unknown:
        raise KeyError("unknown parameters: %s" % sorted(unknown))
    full.update(d)
    return ij_params(**full)


class Handle:
    """Owns an ij_handle plus the allocator callbacks it was created with."""

    def __init__(self, ptr, lattices, callbacks):
        self.ptr = C.c_void_p(ptr)
        self.lattices = lattices
        self._callbacks = callbacks

    def __del__(self):
        if getattr(self, "ptr", None) and self.ptr.value:
            _lib.ij_destroy(self.ptr)
            self.ptr = C.c_void_p(None)


def _torch_allocator(device, stream):
    import torch

    def alloc(size, ctx):
        return torch.cuda.caching_allocator_alloc(size, device, stream)

    def free(ptr, ctx):
        torch.cuda.caching_allocator_delete(ptr)

    return ALLOC_FN(alloc), FREE_FN(free)


def ij_create(params, stream=None, allocator="torch"):
    """Create a batch of lattices; ``params`` is a dict or a list of dicts.
    ``stream``: a torch.cuda.Stream, a raw cudaStream_t int, or None for
    torch's current stream.  ``allocator``: "torch" or "cuda"."""
    plist = [params] if isinstance(params, dict) else list(params)
    arr = (ij_params * len(plist))(*[make_params(p) for p in plist])
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    raw_stream = stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)
    if allocator == "torch":
        cbs = _torch_allocator(torch.cuda.current_device(), raw_stream)
    else:
        cbs = (ALLOC_FN(), FREE_FN())
    out = C.c_void_p()
    _check(_lib.ij_create(arr, len(plist), cbs[0], cbs[1], None, C.c_void_p(raw_stream),
                          C.byref(out)))
    return Handle(out.value, [dict(DEFAULTS, **p) for p in plist], cbs)


def ij_step(h, nsteps):
    _check(_lib.ij_step(h.ptr, int(nsteps)))


def ij_observe(h, index=0, phi=True):
    """Latest diagnostics record (dict) and phi as a numpy (ny, nx) array
    ((nz, ny, nx) in 3-D)."""
    obs = ij_obs()
    p = _lattice(h, index)
    arr = np.empty(_grid(p), dtype=np.float32) if phi else None
    _check(_lib.ij_observe(h.ptr, index, C.byref(obs),
                           arr.ctypes.data_as(C.c_void_p) if phi else None, 0))
    return {k: getattr(obs, k) for k in REC_FIELDS}, arr


def ij_observe_device(h, index, phi_tensor):
    """Write phi of lattice ``index`` into a float32 CUDA tensor (ny, nx)
    ((nz, ny, nx) in 3-D)."""
    p = _lattice(h, index)
    if (tuple(phi_tensor.shape) != _grid(p) or not phi_tensor.is_contiguous()
            or str(phi_tensor.dtype) != "torch.float32" or not phi_tensor.is_cuda):
        raise ValueError("phi must be a contiguous float32 CUDA tensor of shape %s" % (_grid(p),))
    obs = ij_obs()
    _check(_lib.ij_observe(h.ptr, index, C.byref(obs), C.c_void_p(phi_tensor.data_ptr()), 1))
    return {k: getattr(obs, k) for k in REC_FIELDS}


def ij_history(h, index=0):
    n = C.c_int()
    _check(_lib.ij_history(h.ptr, index, None, 0, C.byref(n)))
    out = np.zeros((max(n.value, 1), len(REC_FIELDS)))
    _check(_lib.ij_history(h.ptr, index, out.ctypes.data_as(_dp), n.value, C.byref(n)))
    return out[:n.value]


def ij_get_state(h, index=0):
    p = _lattice(h, index)
    qf, qg = _nq(p)
    f = np.empty((qf,) + _grid(p), dtype=np.float32)
    g = np.empty((qg,) + _grid(p), dtype=np.float32)
    _check(_lib.ij_get_state(h.ptr, index, f.ctypes.data_as(C.c_void_p),
                             g.ctypes.data_as(C.c_void_p), 0))
    return f, g


def ij_set_state(h, index, f, g, t):
    p = _lattice(h, index)
    qf, qg = _nq(p)
    f = np.ascontiguousarray(f, dtype=np.float32)
    g = np.ascontiguousarray(g, dtype=np.float32)
    if f.shape != (qf,) + _grid(p) or g.shape != (qg,) + _grid(p):
        raise ValueError("state shapes must be %s and %s" % ((qf,) + _grid(p), (qg,) + _grid(p)))
    _check(_lib.ij_set_state(h.ptr, index, f.ctypes.data_as(C.c_void_p),
                             g.ctypes.data_as(C.c_void_p), int(t), 0))


def ij_time(h):
    t = C.c_longlong()
    _check(_lib.ij_time(h.ptr, C.byref(t)))
    return t.value


def ij_launch_count(h):
    n = C.c_longlong()
    _check(_lib.ij_launch_count(h.ptr, C.byref(n)))
    return n.value


def ij_kernel_timing(h, enable=-1):
    """(total ms, launches) of the step-kernel launches timed since the last
    reset; enable=1/0 then switches timing on/off and resets."""
    ms, n = C.c_double(), C.c_longlong()
    _check(_lib.ij_kernel_timing(h.ptr, int(enable), C.byref(ms), C.byref(n)))
    return ms.value, n.value


def ij_tune(h, block_size=0, chunk=32, prefetch=2):
    _check(_lib.ij_tune(h.ptr, int(block_size), int(chunk), int(prefetch)))


def ij_use_graph(h, enable=True):
    _check(_lib.ij_use_graph(h.ptr, int(bool(enable))))


def ij_autotune(h, reps=3):
    _check(_lib.ij_autotune(h.ptr, int(reps)))
    return ij_get_tuning(h)


def ij_get_tuning(h):
    """List of dicts (block_size, chunk, prefetch, items), one per bucket."""
    out, k = [], 0
    vals = [C.c_int() for _ in range(4)]
    while _lib.ij_get_tuning(h.ptr, k, *[C.byref(v) for v in vals]) == IJ_OK:
        out.append(dict(zip(("block_size", "chunk", "prefetch", "items"), [v.value for v in vals])))
        k += 1
    return out


def ij_destroy(h):
    if h.ptr.value:
        _check(_lib.ij_destroy(h.ptr))
        h.ptr = C.c_void_p(None)


def ij_last_error():
    return _lib.ij_last_error().decode()
