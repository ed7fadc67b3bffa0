"""2-D FP16 storage (f as offsets f_i - w_i n0, g_1..4 as is, g_0 in FP32;
every update in FP32, round to nearest on store) against the FP64 oracle.

One step from a state the FP16 path holds exactly: every stored value is the
rounding of an FP32 result, so each population is within half an FP16 ulp of
the oracle's value (at most 2^-11 of the stored offset, plus the FP32
round-off the FP32 tests allow).  Over long runs the FP16 rounding is not
bounded by the method, so the error of each observable is reported; the
bounds there only catch a broken path.
"""
import numpy as np
import pytest

from oracle import OracleSim
from paper_1702_04487_gb300 import workloads as W

pytestmark = pytest.mark.gpu

W9 = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
HALF = 2.0 ** -11  # half an ulp of FP16, relative


def _oracle(p):
    """The FP64 oracle of a lattice (it has one precision: no storage key)."""
    return OracleSim({k: v for k, v in p.items() if k != "precision"})


@pytest.fixture(scope="module")
def ij():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1702_04487_gb300 import inkjet
    return inkjet


def _fp16_step_case(ij, p, steps=1, noise=3e-6):
    """Start the oracle from the decoded FP16 state, step both, and bound
    every population."""
    p = dict(p, precision=1)
    h = ij.ij_create(p)
    fa, ga = ij.ij_get_state(h, 0)
    o = _oracle(p)
    o.set_state(fa.astype(np.float64), ga.astype(np.float64), 0)
    ij.ij_step(h, steps)
    o.step(steps)
    fg, gg = ij.ij_get_state(h, 0)
    fo, go = o.state()
    fluid = o.kinds() == 0
    n0 = 0.5 * (p["rho_ink"] + p["rho_air"])
    phis = 0.5 * (p["rho_ink"] - p["rho_air"])
    sf = np.abs(fo).max()
    dev = (fo - W9[:, None, None] * n0) * fluid
    ef = np.abs(fg.astype(np.float64) - fo)
    bf = steps * (HALF * np.abs(dev) + noise * sf)
    assert np.all(ef <= bf), float((ef - bf).max())
    eg = np.abs(gg.astype(np.float64) - go)
    bg = steps * (HALF * np.abs(go) + noise * phis)
    bg[0] = steps * noise * phis  # g_0 stays FP32
    assert np.all(eg <= bg), float((eg - bg).max())
    return fa, fg, sf


def test_initial_state_is_the_rounded_fp64_state(ij):
    p = dict(W.cfg1(), precision=1)
    h = ij.ij_create(p)
    fg, gg = ij.ij_get_state(h, 0)
    o = _oracle(p)
    fo, go = o.state()
    n0 = 0.5 * (p["rho_ink"] + p["rho_air"])
    dev = (fo - W9[:, None, None] * n0) * (o.kinds() == 0)
    assert np.all(np.abs(fg - fo) <= HALF * np.abs(dev) + 2e-7 * np.abs(fo).max())
    assert np.all(np.abs(gg[0] - go[0]) <= 2e-7 * 4.5)
    # FP64 -> FP32 -> FP16: half an FP16 ulp plus one FP32 rounding, and
    # half the FP16 subnormal spacing near zero
    assert np.all(np.abs(gg[1:] - go[1:]) <= (HALF + 2.0 ** -23) * np.abs(go[1:]) + 2.0 ** -25)


def test_one_step_cfg1_fp16(ij):
    fa, fg, sf = _fp16_step_case(ij, W.cfg1())
    assert np.abs(fg - fa).max() > 1e-4 * sf  # the state moved


@pytest.mark.parametrize("bc", [W.BC_ZERO_GRADIENT, W.BC_PERIODIC, W.BC_CLOSED])
@pytest.mark.parametrize("geom", ["nozzle", "plate", "none"])
def test_boundaries_and_geometries_fp16(ij, bc, geom):
    kw = dict(axial_bc=bc)
    if geom == "plate":
        kw.update(geometry=W.GEOM_PLATE, wall_thickness=3, init_kind=W.INIT_DROP, init_x=20,
                  init_y=9, init_r=9, theta_deg=50.0)
    elif geom == "none":
        kw.update(geometry=W.GEOM_NONE, init_kind=W.INIT_DROP, init_x=10, init_y=40, init_r=8)
    _fp16_step_case(ij, W.small_nozzle(**kw))


@pytest.mark.parametrize("nx,ny", [(38, 53), (2, 7), (4, 2), (6, 1), (300, 41), (514, 19),
                                   (256, 30), (258, 30), (30, 9)])
def test_ragged_and_degenerate_sizes_fp16(ij, nx, ny):
    """Even widths only (pairs of FP16 columns): below one strip, one
    column pair, several strips with a ragged last strip, a strip edge on
    the nozzle wall."""
    if nx >= 20:
        p = W.small_nozzle(nx=nx, ny=ny, nozzle_width=max(4, nx // 4),
                           nozzle_length=max(1, ny // 3), wall_thickness=2)
    else:
        p = W.small_nozzle(nx=nx, ny=ny, geometry=W.GEOM_NONE, init_kind=W.INIT_FLAT,
                           init_y=ny / 2.0, axial_bc=W.BC_PERIODIC)
    _fp16_step_case(ij, p)


@pytest.mark.parametrize("cx", [58, 59, 60, 61, 62, 63])
def test_wall_on_strip_edges_fp16(ij, cx):
    """Nozzle walls across the edges of the 60-column strips (nx = 180: the
    walls cross columns 60 and 120); at cx = 62 lanes 0 / 31 stage the g of
    the column outside the strip."""
    nx = 180
    width = nx - 2 * cx
    p = W.small_nozzle(nx=nx, ny=40, nozzle_width=width, nozzle_length=20, wall_thickness=4)
    _fp16_step_case(ij, p)


def test_batch_graph_and_tuning_fp16_bitwise(ij):
    """FP16 lattices of different sizes in one handle step exactly as alone;
    graph replay and other launch shapes change nothing."""
    ps = [dict(q, ny=min(q["ny"], 200), precision=1) for q in W.cfg3_sample(count=4, seed=31)]
    hb = ij.ij_create(ps)
    ij.ij_use_graph(hb, False)
    ij.ij_step(hb, 23)
    hg = ij.ij_create(ps)
    ij.ij_step(hg, 10)
    ij.ij_tune(hg, 0, 8, 4)
    ij.ij_step(hg, 13)
    for k, q in enumerate(ps):
        h1 = ij.ij_create(q)
        ij.ij_tune(h1, 0, 48, 1)
        ij.ij_step(h1, 23)
        fb, gb = ij.ij_get_state(hb, k)
        f1, g1 = ij.ij_get_state(h1, 0)
        fgr, ggr = ij.ij_get_state(hg, k)
        assert np.array_equal(fb, f1) and np.array_equal(gb, g1)
        assert np.array_equal(fb, fgr) and np.array_equal(gb, ggr)
        # the record's lattice sums add per-item FP64 partial sums, whose
        # grouping follows the launch shape: equal to FP64 rounding
        ob, _ = ij.ij_observe(hb, k, phi=False)
        og, _ = ij.ij_observe(hg, k, phi=False)
        assert ob.keys() == og.keys()
        assert all(abs(ob[key] - og[key]) <= 1e-12 * max(1.0, abs(ob[key])) for key in ob)


def test_mixed_precision_batch_is_rejected(ij):
    """One launch covers every lattice of a handle, so they share the
    storage format."""
    with pytest.raises(ij.InkjetError) as e:
        ij.ij_create([dict(W.small_nozzle(), precision=1), W.small_nozzle()])
    assert e.value.status == ij.IJ_ERR_PARAM


def test_set_get_state_round_trip(ij):
    """get_state returns absolute FP32 populations and set_state rounds them
    to FP16 offsets again: g comes back exactly (g_0 is FP32, g_1..4 decode
    and re-encode exactly); f within one FP32 rounding of the absolute value
    (the sum with w_i n0 is rounded on the way out)."""
    p = dict(W.small_nozzle(), precision=1)
    h = ij.ij_create(p)
    ij.ij_step(h, 7)
    f1, g1 = ij.ij_get_state(h, 0)
    h2 = ij.ij_create(p)
    ij.ij_set_state(h2, 0, f1, g1, 7)
    assert ij.ij_time(h2) == 7
    f2, g2 = ij.ij_get_state(h2, 0)
    assert np.array_equal(g1, g2)
    assert np.all(np.abs(f2 - f1) <= 2.0 ** -22 * np.abs(f1).max())


def test_observe_phi_fp16(ij):
    p = dict(W.cfg1(), precision=1)
    h = ij.ij_create(p)
    ij.ij_step(h, 30)
    obs, phi = ij.ij_observe(h, 0)
    f, g = ij.ij_get_state(h, 0)
    assert np.allclose(phi, g.sum(0), atol=2e-6 * 4.5, rtol=0)


@pytest.fixture(scope="module")
def cfg1_runs(ij):
    p = W.cfg1()
    o = _oracle(p)
    o.step(1000)
    f1000, g1000 = o.state()
    o.step(3000)
    return p, (f1000, g1000), o.history()


def test_cfg1_fp16_error_report(ij, cfg1_runs):
    """cfg 1 in FP16 storage against the FP64 oracle: n and phi after 1000
    steps, breakup time, droplet velocity and volume after 4000 steps, and the
    drift of the two masses.  Printed; the bounds only catch a broken path."""
    p, (fo, go), ho = cfg1_runs
    h = ij.ij_create(dict(p, precision=1))
    ij.ij_step(h, 1000)
    fg, gg = ij.ij_get_state(h, 0)
    ng, pg = fg.astype(np.float64).sum(0), gg.astype(np.float64).sum(0)
    no, po = fo.sum(0), go.sum(0)
    ij.ij_step(h, 3000)
    obs, _ = ij.ij_observe(h, 0, phi=False)
    hg = ij.ij_history(h, 0)
    tb = ho[-1, 5]
    rep = dict(n=float(np.abs(ng - no).max() / np.abs(no).max()),
               phi=float(np.abs(pg - po).max() / 4.5),
               breakup=abs(obs["breakup_step"] - tb) / tb,
               velocity=abs(obs["droplet_velocity"] - ho[-1, 8]) / abs(ho[-1, 8]),
               volume=abs(obs["droplet_volume"] - ho[-1, 6]) / ho[-1, 6],
               mass_n=float(np.abs(hg[:, 1] - ho[:, 1]).max() / ho[0, 1]),
               mass_phi=float(np.abs(hg[:, 2] - ho[:, 2]).max() / abs(ho[0, 2])))
    print("2-D FP16 storage vs FP64 oracle (cfg 1):",
          ", ".join("%s %.2e" % kv for kv in rep.items()))
    assert obs["breakup_step"] > 0 and rep["breakup"] < 0.05
    assert rep["velocity"] < 0.1 and rep["volume"] < 0.1
    assert rep["n"] < 0.02 and rep["phi"] < 0.2
