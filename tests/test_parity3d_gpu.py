"""Parity of the 3-D CUDA path (D3Q19 f, D3Q7 g, through the C ABI) with the
FP64 3-D oracle.

FP32 storage is held to the same bounds as the 2-D path: one step from a
shared state within ~1e-6 of the FP64 result, 1000 steps within 1e-5 on n
and 3e-5 on phi, breakup time within 1%.  FP16 storage rounds every stored
population to 11 significant bits each step; its error against the oracle
is measured and reported per observable, with loose sanity bounds only.
"""
import numpy as np
import pytest

from oracle import OracleSim3
from paper_1702_04487_gb300 import workloads as W

pytestmark = pytest.mark.gpu

PHIS = 4.5  # (rho_ink - rho_air) / 2 of every case here


@pytest.fixture(scope="module")
def ij():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1702_04487_gb300 import inkjet
    return inkjet


def _orc(p):
    q = {k: v for k, v in p.items() if k not in ("dim", "precision")}
    return OracleSim3(q)


def _rel(a, b, scale):
    return float(np.abs(np.asarray(a, np.float64) - np.asarray(b, np.float64)).max() / scale)


def _box(**kw):
    """Small 3-D lattice without a nozzle (drop in a periodic box)."""
    p = W.small_nozzle3(nx=16, ny=14, nz=18, geometry=W.GEOM_NONE, init_kind=W.INIT_DROP,
                        init_x=7.5, init_y=6.0, init_z=9.0, init_r=5.0, axial_bc=W.BC_PERIODIC,
                        F0=1e-3, F_neg=5e-4, T1=3, T2=3)
    p.update(kw)
    return p


def _nozzle(**kw):
    p = W.small_nozzle3(nx=18, ny=18, nz=24, nozzle_width=4, nozzle_length=10,
                        F0=2e-3, F_neg=1e-3, T1=3, T2=3)
    p.update(kw)
    return p


def _plate(**kw):
    p = _box(geometry=W.GEOM_PLATE, wall_thickness=3, init_z=7.0, theta_deg=50.0)
    p.update(kw)
    return p


def _steps_case(ij, p, steps, tol):
    """Both sides from the same FP32-representable state; compare every
    population after ``steps`` steps."""
    o = _orc(p)
    f0, g0 = o.state()
    f32, g32 = f0.astype(np.float32), g0.astype(np.float32)
    o.set_state(f32.astype(np.float64), g32.astype(np.float64), 0)
    h = ij.ij_create(p)
    ij.ij_set_state(h, 0, f32, g32, 0)
    ij.ij_step(h, steps)
    o.step(steps)
    fg, gg = ij.ij_get_state(h, 0)
    fo, go = o.state()
    ef, eg = _rel(fg, fo, np.abs(fo).max()), _rel(gg, go, PHIS)
    assert ef < tol and eg < tol, (ef, eg)
    return ef, eg


@pytest.mark.parametrize("make", [_nozzle, _plate, _box])
def test_initial_state3(ij, make):
    p = make()
    fo, go = _orc(p).state()
    h = ij.ij_create(p)
    fg, gg = ij.ij_get_state(h, 0)
    assert _rel(fg, fo, np.abs(fo).max()) < 2e-7
    assert _rel(gg, go, PHIS) < 2e-7
    # FP16 storage: each stored value within half an FP16 ulp of the exact
    # deviation f_i - w_i n0 (or g_i); g_0 is kept in FP32
    h16 = ij.ij_create(dict(p, precision=1))
    f16, g16 = ij.ij_get_state(h16, 0)
    _, _, _, w = __import__("oracle").lattice3()
    n0 = 5.5
    fluid = _orc(p).kinds() == 0
    dev = fo - w[:, None, None, None] * n0
    err = np.abs(f16 - fo)[:, fluid]
    assert (err <= 2.0 ** -11 * np.abs(dev)[:, fluid] + 4e-7 * n0).all()
    errg = np.abs(g16[1:] - go[1:])[:, fluid]
    assert (errg <= 2.0 ** -11 * np.abs(go[1:])[:, fluid] + 1e-7).all()
    assert _rel(g16[0], go[0], PHIS) < 2e-7


@pytest.mark.parametrize("bc", [W.BC_ZERO_GRADIENT, W.BC_PERIODIC, W.BC_CLOSED])
@pytest.mark.parametrize("make", [_nozzle, _plate, _box])
def test_steps3_boundaries_and_geometries(ij, bc, make):
    _steps_case(ij, make(axial_bc=bc), steps=5, tol=1e-5)


@pytest.mark.parametrize("nx,ny,nz", [(33, 7, 9), (1, 1, 12), (5, 3, 2), (129, 5, 6),
                                      (37, 40, 21)])
def test_ragged_sizes3(ij, nx, ny, nz):
    """Widths off the 32 x 4 block, single columns, very thin lattices and a
    round nozzle on a non-square cross-section."""
    if (nx, ny) == (37, 40):
        p = _nozzle(nx=nx, ny=ny, nz=nz, nozzle_width=6, wall_thickness=2, nozzle_length=8)
    else:
        p = _box(nx=nx, ny=ny, nz=nz, init_kind=W.INIT_FLAT, init_y=nz / 2.0)
    _steps_case(ij, p, steps=3, tol=1e-5)


def test_state_roundtrip3(ij):
    """set_state then get_state: g comes back unchanged (FP32) or with g_1..6
    rounded to FP16 (FP16 storage); f goes through the stored offsets
    f_i - w_i n0 and back (one FP32 rounding each way, plus the FP16
    rounding of the offset); solid cells read back as 0."""
    p = _nozzle()
    o = _orc(p)
    fluid = o.kinds() == 0
    rng = np.random.default_rng(11)
    f = (rng.uniform(0.0, 1.0, (19,) + fluid.shape) * fluid).astype(np.float32)
    g = (rng.uniform(-1.0, 1.0, (7,) + fluid.shape) * fluid).astype(np.float32)
    _, _, _, w = __import__("oracle").lattice3()
    wn = w[:, None, None, None] * 5.5
    h = ij.ij_create(p)
    ij.ij_set_state(h, 0, f, g, 7)
    assert ij.ij_time(h) == 7
    f2, g2 = ij.ij_get_state(h, 0)
    assert np.array_equal(g2, g)
    assert (f2[:, ~fluid] == 0).all()
    assert np.abs(f2 - f).max() <= 2.0 ** -22 * 2
    h16 = ij.ij_create(dict(p, precision=1))
    ij.ij_set_state(h16, 0, f, g, 0)
    f3, g3 = ij.ij_get_state(h16, 0)
    assert np.array_equal(g3[1:], g[1:].astype(np.float16).astype(np.float32))
    assert np.array_equal(g3[0], g[0])
    err = np.abs(f3 - f)[:, fluid]
    assert (err <= 2.0 ** -11 * np.abs(f - wn)[:, fluid] + 1e-6).all()
    assert (f3[:, ~fluid] == 0).all()


def _fields(f, g):
    return f.astype(np.float64).sum(0), g.astype(np.float64).sum(0)


def test_small_nozzle3_1000_steps(ij):
    """The small round nozzle, FP32 storage: n within 1e-5 (relative to
    max n) and phi within 6e-5 of phi* after 1000 driven steps.  The bound
    on phi is about three times the FP32 round-off floor of this case, which
    the oracle itself, fed FP32-sized noise, reaches (1.3-2.0e-5, see
    tests/test_oracle3d_pins.py::test_fp32_noise_floor_of_small_nozzle3)."""
    p = W.small_nozzle3()
    h = ij.ij_create(p)
    ij.ij_step(h, 1000)
    fg, gg = ij.ij_get_state(h, 0)
    o = _orc(p)
    o.step(1000)
    fo, go = o.state()
    ng, pg = _fields(fg, gg)
    no, po = _fields(fo, go)
    en, ep = _rel(ng, no, np.abs(no).max()), _rel(pg, po, PHIS)
    print("3-D FP32 after 1000 steps: n %.2e, phi %.2e" % (en, ep))
    assert en < 1e-5 and ep < 6e-5


@pytest.fixture(scope="module")
def oracle_run3():
    """FP64 history of the small round nozzle through its breakup."""
    o = _orc(W.small_nozzle3())
    o.step(1500)
    return o.history(), o.state()


def _gpu_run3(ij, precision):
    h = ij.ij_create(W.small_nozzle3(precision=precision))
    ij.ij_step(h, 1500)
    return h, ij.ij_history(h, 0)


def test_small_nozzle3_breakup_fp32(ij, oracle_run3):
    ho, _ = oracle_run3
    h, hg = _gpu_run3(ij, 0)
    assert hg.shape == ho.shape
    assert np.array_equal(hg[:, 0], ho[:, 0])
    tb_o, tb_g = ho[-1, 5], hg[-1, 5]
    assert tb_o > 0 and abs(tb_g - tb_o) <= 0.01 * tb_o, (tb_g, tb_o)
    # FP64 mass integrals (open ends: the jet carries mass out of the top)
    assert np.abs(hg[:, 1] - ho[:, 1]).max() < 1e-5 * ho[0, 1]
    assert np.abs(hg[:, 2] - ho[:, 2]).max() < 1e-4 * np.abs(ho[0, 2])
    # momentum and neck track the oracle before breakup
    pre = ho[:, 0] < tb_o - 50
    assert np.abs(hg[pre, 3] - ho[pre, 3]).max() < 1e-3 * np.abs(ho[:, 3]).max()
    assert np.abs(hg[pre, 4] - ho[pre, 4]).max() < 1e-2 * ho[0, 4]
    # the leading droplet's velocity (record column 8) within 1 % of the
    # oracle's just after pinch-off and at the end of the run, and its volume
    after = int(np.searchsorted(ho[:, 0], tb_o)) + 1
    for r in (after, len(ho) - 1):
        assert abs(hg[r, 8] - ho[r, 8]) <= 0.01 * abs(ho[r, 8]), (r, hg[r, 8], ho[r, 8])
        assert abs(hg[r, 6] - ho[r, 6]) <= 0.01 * ho[r, 6], (r, hg[r, 6], ho[r, 6])


def test_small_nozzle3_fp16_error_report(ij, oracle_run3):
    """FP16 offset storage against the FP64 oracle, per observable.  The
    figures are reported; the bounds only catch a broken path."""
    ho, (fo, go) = oracle_run3
    h, hg = _gpu_run3(ij, 1)
    fg, gg = ij.ij_get_state(h, 0)
    ng, pg = _fields(fg, gg)
    no, po = _fields(fo, go)
    tb_o, tb_g = ho[-1, 5], hg[-1, 5]
    rep = dict(n=_rel(ng, no, np.abs(no).max()), phi=_rel(pg, po, PHIS),
               breakup=abs(tb_g - tb_o) / tb_o,
               mass_n=float(np.abs(hg[:, 1] - ho[:, 1]).max() / ho[0, 1]),
               mass_phi=float(np.abs(hg[:, 2] - ho[:, 2]).max() / abs(ho[0, 2])),
               momentum=float(np.abs(hg[:, 3] - ho[:, 3]).max() / np.abs(ho[:, 3]).max()))
    print("3-D FP16 storage vs FP64 oracle after 1500 steps:",
          ", ".join("%s %.2e" % kv for kv in rep.items()))
    assert tb_g > 0 and rep["breakup"] < 0.05
    assert rep["phi"] < 0.2 and rep["n"] < 0.05


@pytest.mark.parametrize("precision", [0, 1])
def test_batch3_equals_single(ij, precision):
    """Two 3-D lattices of different sizes, geometries and angles in one
    handle (one launch covers both) step exactly as they do alone."""
    pa = _nozzle(precision=precision)
    pb = _box(theta_deg=120.0, precision=precision)
    hb = ij.ij_create([pa, pb])
    ij.ij_step(hb, 40)
    for k, p in enumerate((pa, pb)):
        hs = ij.ij_create(p)
        ij.ij_step(hs, 40)
        fb, gb = ij.ij_get_state(hb, k)
        fs, gs = ij.ij_get_state(hs, 0)
        assert np.array_equal(fb, fs) and np.array_equal(gb, gs)


def test_batch3_rejects_mixed_storage_and_odd_fp16(ij):
    with pytest.raises(ij.InkjetError):
        ij.ij_create([_nozzle(), _box(precision=1)])
    with pytest.raises(ij.InkjetError):
        ij.ij_create(_box(nx=15, precision=1))


def test_graph3_matches_launches(ij):
    p = _nozzle(diag_every=4)
    ha, hb = ij.ij_create(p), ij.ij_create(p)
    ij.ij_use_graph(hb, 0)
    ij.ij_step(ha, 37)
    for _ in range(37):
        ij.ij_step(hb, 1)
    fa, ga = ij.ij_get_state(ha, 0)
    fb, gb = ij.ij_get_state(hb, 0)
    assert np.array_equal(fa, fb) and np.array_equal(ga, gb)
    ra, rb = ij.ij_history(ha, 0), ij.ij_history(hb, 0)
    assert np.allclose(ra, rb, rtol=1e-12, atol=1e-9)


def test_numeric_failure3_freezes_one_lattice(ij):
    good = _nozzle()
    bad = _nozzle(F0=5.0, T1=100)
    h = ij.ij_create([good, bad])
    ij.ij_step(h, 30)
    with pytest.raises(ij.InkjetError) as e:
        ij.ij_observe(h, 1, phi=False)
    assert e.value.status == ij.IJ_ERR_NUMERIC
    obs, phi = ij.ij_observe(h, 0)
    assert np.isfinite(phi).all() and phi.shape == (24, 18, 18)
    fb1, _ = ij.ij_get_state(h, 1)
    ij.ij_step(h, 5)
    fb2, _ = ij.ij_get_state(h, 1)
    assert np.array_equal(fb1, fb2, equal_nan=True)


def test_tuning_entry_points_on_3d(ij):
    """The z chunk of the 3-D work items is the one tunable; any chunk (and
    the autotuned one) gives bit-identical states."""
    p = _nozzle(nz=40)
    ref = ij.ij_create(p)
    ij.ij_step(ref, 12)
    fr, gr = ij.ij_get_state(ref, 0)
    with pytest.raises(ij.InkjetError):
        ij.ij_tune(ref, 0, 16, 2)  # no prefetch depth to tune
    with pytest.raises(ij.InkjetError):
        ij.ij_tune(ref, 0, 0, 1)
    for chunk in (1, 7, 16, 40, 200):
        h = ij.ij_create(p)
        ij.ij_tune(h, 0, chunk, 1)
        (t,) = ij.ij_get_tuning(h)
        assert t["chunk"] == chunk and t["prefetch"] == 1 and t["block_size"] == 512
        ij.ij_step(h, 12)
        f, g = ij.ij_get_state(h, 0)
        assert np.array_equal(f, fr) and np.array_equal(g, gr), chunk
    h = ij.ij_create(p)
    (t,) = ij.ij_autotune(h, 2)
    assert t["chunk"] >= 1 and t["items"] >= 1
    ij.ij_step(h, 12)
    f, g = ij.ij_get_state(h, 0)
    assert np.array_equal(f, fr) and np.array_equal(g, gr)
