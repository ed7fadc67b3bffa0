"""Parity of the 3-D CUDA path with the FP64 oracle at the size of the 3-D
round-nozzle workload (128 x 128 x 640, radius 24, length 160, contact
angles 60 and 120 degrees), both lattices in one handle as the benchmark
runs them, with the autotuned z chunk; and on a 128 x 128 x 160 slab of the
same cross-section with the default chunk.

Both sides start from the same state (the oracle's initial state, rounded to
what the storage holds) and are compared population by population after a
few steps:
 - FP32 storage: within 1e-5 of max |f| (f) and of phi* (g), as the small
   3-D cases;
 - FP16 offset storage: every stored value is rounded to 11 significant bits
   each step, so after s steps a population may differ from the exact one by
   about s rounding errors of the largest deviation f_i - w_i n0 it carries;
   the bound is (s + 1) 2^-11 max |f_i - w_i n0| plus the FP32 bound.
"""
import numpy as np
import pytest

from oracle import OracleSim3, lattice3
from paper_1702_04487_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PHIS = 4.5  # (rho_ink - rho_air) / 2 of these lattices
N0 = 5.5    # rest density (rho_ink + rho_air) / 2


@pytest.fixture(scope="module")
def ij():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1702_04487_gb300 import inkjet
    return inkjet


def _orc(p):
    return OracleSim3({k: v for k, v in p.items() if k not in ("dim", "precision")})


def _run(ij, ps, steps, autotune):
    h = ij.ij_create(ps)
    if autotune:
        ij.ij_autotune(h, 1)
    orcs = []
    for k, p in enumerate(ps):
        o = _orc(p)
        f, g = o.state()
        ij.ij_set_state(h, k, f.astype(np.float32), g.astype(np.float32), 0)
        # the state as stored (FP16 storage rounds it), decoded exactly
        fs, gs = ij.ij_get_state(h, k)
        o.set_state(fs.astype(np.float64), gs.astype(np.float64), 0)
        orcs.append(o)
        del f, g, fs, gs
    ij.ij_step(h, steps)
    _, _, _, w = lattice3()
    out = []
    for k, o in enumerate(orcs):
        o.step(steps)
        fo, go = o.state()
        fg, gg = ij.ij_get_state(h, k)
        ef = float(np.abs(fg - fo).max())
        eg = float(np.abs(gg - go).max())
        dev = float(np.abs(fo - w[:, None, None, None] * N0 * (fo != 0)).max())
        out.append((ef, eg, float(np.abs(fo).max()), dev))
        del fo, go, fg, gg
    return out


def _check(res, precision, steps):
    for ef, eg, fmax, dev in res:
        tf, tg = 1e-5 * fmax, 1e-5 * PHIS
        if precision == 1:
            tf += (steps + 1) * 2.0 ** -11 * dev
            tg += (steps + 1) * 2.0 ** -11 * PHIS
        print("3-D %s: max |f - f_oracle| %.2e (bound %.2e), max |g - g_oracle| %.2e (bound %.2e)"
              % ("FP16" if precision else "FP32", ef, tf, eg, tg))
        assert ef < tf and eg < tg, (ef, tf, eg, tg)


@pytest.mark.parametrize("precision", [0, 1])
def test_round_nozzle_full_size_batch(ij, precision):
    """Both lattices of the 128 x 128 x 640 workload, in one handle, autotuned."""
    ps = [W.cfg4(60.0, precision, seed=4), W.cfg4(120.0, precision, seed=5)]
    _check(_run(ij, ps, steps=2, autotune=True), precision, 2)


@pytest.mark.parametrize("precision", [0, 1])
def test_round_nozzle_slab(ij, precision):
    """A 128 x 128 x 160 slab of the same nozzle, default launch shape."""
    ps = [W.cfg4(60.0, precision, seed=4, nz=160)]
    _check(_run(ij, ps, steps=3, autotune=False), precision, 3)
