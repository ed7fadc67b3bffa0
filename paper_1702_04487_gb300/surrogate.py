"""Surrogate of the inkjet lattice Boltzmann model (include/surrogate.h).

Thin ctypes binding of the sg_* entry points of libinkjet.so, plus the host
logic of the service around them:

- ``sample_inputs``: seeded rows of the seven surrogate inputs (contact
  angle, surface tension, F0, T1, T2, idle time, nozzle width) of the
  lattices the uneven-sweep sampler draws (``sample_raw``: w ~ U{16..48},
  angle ~ U[20, 160] degrees, surface tension log-uniform over a factor 4,
  F0 ~ U[1e-4, 4e-4], T1, T2 ~ U{500..3000}, no idle time), with the drive
  mapped onto each nozzle's capillary scales (``scaled_drive``) so that the
  draws eject a droplet: the row holds the lattice's own force density and
  pulse lengths;
- ``lattice_params``: the lattice of one input row (nozzle w wide, domain
  4w x 30w, nozzle length 4w, walls 4 -- the uneven-sweep geometry);
- ``lbm_outcomes``: runs input rows on the batched lattice Boltzmann path
  (one handle, every row a lattice) and reads breakup time, droplet
  velocity, droplet volume and satellites from the FP64 diagnostics;
- ``SurrogateService``: answers queries with the ensemble where the gate
  accepts them and re-runs the rest on the lattice Boltzmann model.

Every contraction and element-wise step of training and inference runs in
the library's kernels; this module only marshals arguments and orchestrates
the two paths.
"""
import ctypes as C
import hashlib

import numpy as np

from . import inkjet as ij
from . import workloads as W

N_IN, N_OUT = 7, 4
INPUT_NAMES = ("theta_deg", "sigma", "F0", "T1", "T2", "T_idle", "width")
OUTPUT_NAMES = ("breakup_step", "droplet_velocity", "droplet_volume", "satellites")


class sg_config(C.Structure):
    _fields_ = [("members", C.c_int), ("hidden", C.c_int), ("batch", C.c_int),
                ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("seed", C.c_ulonglong), ("log_inputs", C.c_int), ("log_outputs", C.c_int),
                ("out_weight", C.c_float * 4), ("lr_cosine", C.c_int)]


_lib = ij._lib
_vp, _i, _fp = C.c_void_p, C.c_int, C.c_void_p
_sig = {
    "sg_create": [C.POINTER(sg_config), ij.ALLOC_FN, ij.FREE_FN, _vp, _vp, C.POINTER(_vp)],
    "sg_set_data": [_vp, _fp, _fp, _i],
    "sg_train": [_vp, _i, C.POINTER(C.c_double)],
    "sg_predict": [_vp, _fp, _i, _fp, _fp, _fp, _i],
    "sg_set_gate": [_vp, C.c_float, C.c_float, C.c_float],
    "sg_param_count": [_vp, C.POINTER(C.c_longlong)],
    "sg_get_params": [_vp, _i, _fp],
    "sg_set_params": [_vp, _i, _fp],
    "sg_get_transform": [_vp, _fp, _fp, _fp, _fp],
    "sg_gradients": [_vp, _fp, _fp, _i, _fp, _fp],
    "sg_destroy": [_vp],
    "sg_gemm_bf16": [_fp, _i, _fp, _i, _i, _i, _i, _fp, _i, _vp],
}
for _name, _args in _sig.items():
    getattr(_lib, _name).argtypes = _args
    getattr(_lib, _name).restype = C.c_int
_lib.sg_last_error.restype = C.c_char_p
_lib.sg_last_error.argtypes = []


def _check(status):
    if status != ij.IJ_OK:
        raise ij.InkjetError(status, _lib.sg_last_error().decode())


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p)


def gemm_bf16(A, B, M, N, K, C_out, lda, ldb, ldc, stream=None):
    """C_out = A B^T on device tensors (A, B bfloat16, C_out float32)."""
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    _check(_lib.sg_gemm_bf16(C.c_void_p(A.data_ptr()), lda, C.c_void_p(B.data_ptr()), ldb, M, N, K,
                             C.c_void_p(C_out.data_ptr()), ldc, C.c_void_p(s.cuda_stream)))


DEFAULT_CONFIG = dict(members=5, hidden=256, batch=256, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8,
                      seed=1, log_inputs=0b0011110, log_outputs=0b0101,
                      out_weight=(1.0, 1.0, 1.0, 0.25), lr_cosine=1)


class Surrogate:
    """One ensemble (sg_handle)."""

    def __init__(self, stream=None, **cfg):
        import torch
        c = dict(DEFAULT_CONFIG, **cfg)
        conf = sg_config(c["members"], c["hidden"], c["batch"], c["lr"], c["beta1"], c["beta2"],
                         c["eps"], c["seed"], c["log_inputs"], c["log_outputs"],
                         (C.c_float * 4)(*c["out_weight"]), int(c["lr_cosine"]))
        self.config = c
        s = torch.cuda.current_stream() if stream is None else stream
        raw = s.cuda_stream
        dev = torch.cuda.current_device()

        def alloc(size, ctx):
            return torch.cuda.caching_allocator_alloc(size, dev, raw)

        def free(ptr, ctx):
            torch.cuda.caching_allocator_delete(ptr)

        self._cbs = (ij.ALLOC_FN(alloc), ij.FREE_FN(free))
        out = C.c_void_p()
        _check(_lib.sg_create(C.byref(conf), self._cbs[0], self._cbs[1], None, C.c_void_p(raw),
                              C.byref(out)))
        self.ptr = out

    def __del__(self):
        if getattr(self, "ptr", None) is not None and self.ptr.value:
            _lib.sg_destroy(self.ptr)
            self.ptr = C.c_void_p(None)

    @property
    def members(self):
        return self.config["members"]

    def set_data(self, x, y):
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        assert x.shape[1] == N_IN and y.shape == (x.shape[0], N_OUT)
        _check(_lib.sg_set_data(self.ptr, _ptr(x), _ptr(y), x.shape[0]))

    def train(self, steps):
        loss = C.c_double()
        _check(_lib.sg_train(self.ptr, int(steps), C.byref(loss)))
        return loss.value

    def predict(self, x, gate=True):
        """Ensemble mean [n][4], spread [n][4] and (gate) accept [n] of raw inputs."""
        x = np.ascontiguousarray(x, dtype=np.float32)
        n = x.shape[0]
        mean = np.empty((n, N_OUT), np.float32)
        sd = np.empty((n, N_OUT), np.float32)
        acc = np.empty(n, np.int32) if gate else None
        _check(_lib.sg_predict(self.ptr, _ptr(x), n, _ptr(mean), _ptr(sd),
                               _ptr(acc) if gate else None, 0))
        return mean, sd, acc

    def set_gate(self, tau, tau_v=None, nn_cut=0.0):
        """Relative ensemble spread allowed on breakup time (tau) and droplet
        velocity (tau_v, default tau); nn_cut <= 0 keeps the data's cut."""
        tv = tau if tau_v is None else tau_v
        _check(_lib.sg_set_gate(self.ptr, float(tau), float(tv), float(nn_cut)))

    def param_count(self):
        n = C.c_longlong()
        _check(_lib.sg_param_count(self.ptr, C.byref(n)))
        return n.value

    def get_params(self, member):
        out = np.empty(self.param_count(), np.float32)
        _check(_lib.sg_get_params(self.ptr, member, _ptr(out)))
        return out

    def set_params(self, member, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        assert p.size == self.param_count()
        _check(_lib.sg_set_params(self.ptr, member, _ptr(p)))

    def transform(self):
        a, b = np.empty(N_IN, np.float32), np.empty(N_IN, np.float32)
        c, d = np.empty(N_OUT, np.float32), np.empty(N_OUT, np.float32)
        _check(_lib.sg_get_transform(self.ptr, _ptr(a), _ptr(b), _ptr(c), _ptr(d)))
        return a, b, c, d

    def gradients(self, x, y):
        x = np.ascontiguousarray(x, dtype=np.float32)
        y = np.ascontiguousarray(y, dtype=np.float32)
        g = np.empty((self.members, self.param_count()), np.float32)
        loss = np.empty(self.members, np.float64)
        _check(_lib.sg_gradients(self.ptr, _ptr(x), _ptr(y), x.shape[0], _ptr(g), _ptr(loss)))
        return g, loss


def unpack(p, hidden):
    """Member parameter vector -> lists Wt [out][in] and b [out] per layer."""
    nin = (16, hidden, hidden, hidden, hidden)
    nout = (hidden, hidden, hidden, hidden, 16)
    Wt, b, off = [], [], 0
    for i, o in zip(nin, nout):
        Wt.append(p[off:off + i * o].reshape(o, i))
        off += i * o
        b.append(p[off:off + o])
        off += o
    return Wt, b


# ---------------------------------------------------------------------------
# Inputs, lattices and outcomes.

# The sampler box: the uneven-sweep sampler (nozzle widths, angles, the
# factor 4 of surface tension, the sweep's drive draws, no idle time) about a
# surface-tension base of SIGMA_SG.
SIGMA_SG = 0.0025
SAMPLER_BOX = dict(theta_deg=(20.0, 160.0), sigma=(SIGMA_SG / 2, 2 * SIGMA_SG), F0=(1e-4, 4e-4),
                   T1=(500, 3000), T2=(500, 3000), T_idle=(0, 0), width=(16, 48))

# Drive scaling.  The sweep's raw draws (F0 about 2.5e-4, pulses of 500-3000
# steps) only bulge the meniscus of these nozzles; a draw is mapped onto the
# nozzle's capillary scales instead: pulse lengths in units of the capillary
# time t_c = sqrt(rho_ink w^3 / sigma) (T -> T / 1750 * T_STAR * t_c) and the
# force density in units of sigma / w^2 (F -> F0 / 2.5e-4 * F_STAR * sigma /
# w^2), capped where the channel's mean velocity at the end of the push
# (start-up of plane Poiseuille flow, viscous time w^2 / (pi^2 nu)) would
# pass U_CAP, below which the lattice stays stable.  Scanned on 256 draws:
# 96 % pinch off a droplet within 28000 steps, none goes unstable.
RHO_INK, NU_INK = 10.0, 0.1
F_STAR, T_STAR, U_CAP = 800.0, 0.25, 0.06
LBM_STEPS = 30000  # longest run of a query (the latest breakups come near 28000)


def scaled_drive(theta, sigma, F0, T1, T2, w):
    """Force density and pulse lengths of the lattice of one sampler draw."""
    tc = np.sqrt(RHO_INK * w ** 3 / sigma)
    t1 = max(50, int(round(T1 / 1750.0 * T_STAR * tc)))
    t2 = max(50, int(round(T2 / 1750.0 * T_STAR * tc)))
    F = F0 / 2.5e-4 * F_STAR * sigma / w ** 2
    tau_v = w * w / (np.pi ** 2 * NU_INK)
    u_per_force = w * w / (12.0 * RHO_INK * NU_INK) * (1.0 - np.exp(-t1 / tau_v))
    return min(F, U_CAP / u_per_force), t1, t2


def sample_raw(n, seed):
    """n draws of the uneven-sweep sampler: angle uniform, surface tension
    log-uniform, F0 uniform, durations and width uniform integers."""
    rng = np.random.default_rng(seed)
    b = SAMPLER_BOX
    x = np.empty((n, N_IN))
    x[:, 0] = rng.uniform(*b["theta_deg"], n)
    x[:, 1] = np.exp(rng.uniform(np.log(b["sigma"][0]), np.log(b["sigma"][1]), n))
    x[:, 2] = rng.uniform(*b["F0"], n)
    x[:, 3] = rng.integers(b["T1"][0], b["T1"][1] + 1, n)
    x[:, 4] = rng.integers(b["T2"][0], b["T2"][1] + 1, n)
    x[:, 5] = rng.integers(b["T_idle"][0], b["T_idle"][1] + 1, n)
    x[:, 6] = rng.integers(b["width"][0], b["width"][1] + 1, n)
    return x


def sample_inputs(n, seed):
    """n input rows: the lattices of n sampler draws (their own force
    density F0 and pulse lengths T1, T2 after ``scaled_drive``)."""
    x = sample_raw(n, seed)
    for r in x:
        r[2], r[3], r[4] = scaled_drive(*r[:5], int(r[6]))
    return x


def row_seed(row):
    """Jitter seed of an input row: a hash of its values, so that a query
    gets the same lattice (and the same outcome) wherever it is run."""
    digest = hashlib.blake2b(np.asarray(row, dtype=np.float64).tobytes(), digest_size=8).digest()
    return int.from_bytes(digest, "little")


def lattice_params(row, seed=None):
    theta, sigma, F0, T1, T2, T_idle, w = [float(v) for v in row]
    seed = row_seed(row) if seed is None else seed
    w = int(round(w))
    return dict(nx=4 * w, ny=30 * w, geometry=W.GEOM_NOZZLE, nozzle_width=w, nozzle_length=4 * w,
                wall_thickness=4, rho_ink=RHO_INK, rho_air=1.0, nu_ink=NU_INK, nu_air=0.05,
                sigma=sigma, width_W=3.0, tau_phi=0.8, gamma=0.0, theta_deg=theta, F0=F0,
                F_neg=F0 / 2, T1=int(round(T1)), T2=int(round(T2)), T_idle=int(round(T_idle)),
                axial_bc=W.BC_ZERO_GRADIENT, init_kind=W.INIT_MENISCUS, jitter=1e-6, seed=seed,
                diag_every=10)


def outcomes_from_history(hist, after=(0, 100)):
    """Breakup time, and droplet velocity, volume and satellites averaged
    over the records from breakup + after[0] to breakup + after[1] (the
    droplet just after pinch-off, before the weak drive lets it slow down).
    NaN row when no breakup happened early enough to fill the window."""
    tb = hist[-1, 5]
    if tb <= 0 or hist[-1, 0] < tb + after[1]:
        return np.full(N_OUT, np.nan)
    sel = (hist[:, 0] >= tb + after[0]) & (hist[:, 0] <= tb + after[1])
    return np.array([tb, hist[sel, 8].mean(), hist[sel, 6].mean(), hist[sel, 9].mean()])


def lbm_outcomes(rows, steps=LBM_STEPS, stream=None, chunk=4096, precision=0, segment=2000):
    """Run every input row as a lattice of the batched LBM path (one handle,
    up to `chunk` rows) for at most `steps` steps, in segments of `segment`
    steps, stopping once every lattice has its outcomes (or is frozen by a
    numeric failure); returns outcomes [n][4] (NaN rows: no breakup in time).
    precision 1 stores the populations in FP16 (offsets)."""
    out = np.full((len(rows), N_OUT), np.nan)
    for a in range(0, len(rows), chunk):
        part = rows[a:a + chunk]
        h = ij.ij_create([dict(lattice_params(r), precision=precision) for r in part],
                         stream=stream)
        todo = list(range(len(part)))
        t = 0
        while todo and t < steps:
            n = min(segment, steps - t)
            try:
                ij.ij_step(h, n)
            except ij.InkjetError as e:
                if e.status != ij.IJ_ERR_NUMERIC:
                    raise
                break  # every lattice is frozen
            t += n
            left = []
            for k in todo:
                try:
                    ij.ij_observe(h, k, phi=False)
                except ij.InkjetError as e:
                    if e.status != ij.IJ_ERR_NUMERIC:
                        raise
                    continue  # frozen by a numeric failure: no outcome
                o = outcomes_from_history(ij.ij_history(h, k))
                if np.isfinite(o).all():
                    out[a + k] = o
                else:
                    left.append(k)
            todo = left
        ij.ij_destroy(h)
    return out


class SurrogateService:
    """Answers queries with the ensemble where the gate accepts them and
    with the lattice Boltzmann model elsewhere."""

    def __init__(self, surrogate, lbm_steps=LBM_STEPS):
        self.sg = surrogate
        self.lbm_steps = lbm_steps

    def query(self, x):
        mean, sd, acc = self.sg.predict(x, gate=True)
        out = mean.astype(np.float64)
        rej = np.nonzero(acc == 0)[0]
        if len(rej):
            out[rej] = lbm_outcomes(x[rej], steps=self.lbm_steps)
        return out, acc.astype(bool)


def relative_error(pred, ref):
    return np.abs(pred - ref) / np.maximum(np.abs(ref), 1e-30)


def finite_rows(y):
    return np.all(np.isfinite(y), axis=1)


def describe_inputs():
    """The sampler box and the drive mapping of the input rows."""
    return dict({k: SAMPLER_BOX[k] for k in INPUT_NAMES},
                drive="F0, T1, T2 on the nozzle's capillary scales: F_STAR %g, T_STAR %g, U_CAP %g"
                      % (F_STAR, T_STAR, U_CAP))


__all__ = ["Surrogate", "SurrogateService", "sample_inputs", "lattice_params", "lbm_outcomes",
           "outcomes_from_history", "gemm_bf16", "unpack", "relative_error", "finite_rows",
           "describe_inputs", "scaled_drive", "sample_raw", "SAMPLER_BOX", "LBM_STEPS"]
