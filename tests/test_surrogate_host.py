"""Host logic of the surrogate service (no GPU): the input sampler, the
lattice of an input row and the outcome read-out from a diagnostics
history."""
import numpy as np

from paper_1702_04487_gb300 import surrogate as S


def test_sampler_is_seeded_and_inside_the_box():
    a, b = S.sample_raw(500, 3), S.sample_raw(500, 3)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, S.sample_raw(500, 4))
    for k, name in enumerate(S.INPUT_NAMES):
        lo, hi = S.SAMPLER_BOX[name]
        assert a[:, k].min() >= lo and a[:, k].max() <= hi
    for k in (3, 4, 5, 6):
        assert np.array_equal(a[:, k], np.round(a[:, k]))
    # the uneven-sweep ranges: widths 16..48, angles 20..160 degrees, a
    # factor 4 of surface tension
    assert S.SAMPLER_BOX["width"] == (16, 48) and S.SAMPLER_BOX["theta_deg"] == (20.0, 160.0)
    lo, hi = S.SAMPLER_BOX["sigma"]
    assert np.isclose(hi / lo, 4.0)
    # input rows: the same draws with the lattice's own drive
    x = S.sample_inputs(500, 3)
    assert np.array_equal(x[:, [0, 1, 5, 6]], a[:, [0, 1, 5, 6]])
    for r, q in zip(x[:20], a[:20]):
        assert tuple(r[2:5]) == S.scaled_drive(*q[:5], int(q[6]))


def test_lattice_of_an_input_row():
    """The uneven-sweep geometry (4w x 30w, nozzle 4w long, walls 4) with the
    row's own drive; the drive of a sampler draw on the nozzle's capillary
    scales."""
    row = [60.0, 0.0025, 3e-4, 2000, 1000, 0, 32]
    p = S.lattice_params(row, seed=5)
    assert (p["nx"], p["ny"], p["nozzle_width"], p["nozzle_length"]) == (128, 960, 32, 128)
    assert (p["F0"], p["F_neg"], p["T1"], p["T2"], p["T_idle"]) == (3e-4, 1.5e-4, 2000, 1000, 0)
    assert p["seed"] == 5 and p["nozzle_width"] + 2 * p["wall_thickness"] <= p["nx"]
    F, t1, t2 = S.scaled_drive(60.0, 0.0025, 2.5e-4, 1750, 875, 32)
    tc = np.sqrt(10.0 * 32 ** 3 / 0.0025)  # capillary time of the nozzle
    assert t1 == round(S.T_STAR * tc) and t2 == round(0.5 * S.T_STAR * tc)
    # the reference draw F0 = 2.5e-4 is F_STAR sigma / w^2, unless the channel
    # would pass U_CAP by the end of the push
    tau = 32 ** 2 / (np.pi ** 2 * 0.1)
    u = S.F_STAR * 0.0025 / 32 ** 2 * 32 ** 2 / 12.0 * (1 - np.exp(-t1 / tau))
    assert np.isclose(F, S.F_STAR * 0.0025 / 32 ** 2 * min(1.0, S.U_CAP / u))


def test_drive_scaling_is_monotone_and_capped():
    """A stronger draw never gives a weaker force, and the estimated channel
    velocity at the end of the push never passes U_CAP."""
    rng = np.random.default_rng(2)
    for _ in range(200):
        th, sg, F0, T1, T2, w = (rng.uniform(20, 160), rng.uniform(1.25e-3, 5e-3),
                                 rng.uniform(1e-4, 4e-4), rng.integers(500, 3001),
                                 rng.integers(500, 3001), int(rng.integers(16, 49)))
        Fa, t1, _ = S.scaled_drive(th, sg, F0, T1, T2, w)
        Fb, _, _ = S.scaled_drive(th, sg, 1.5 * F0, T1, T2, w)
        assert Fb >= Fa > 0
        tau = w * w / (np.pi ** 2 * 0.1)
        assert Fa * w * w / 12.0 * (1 - np.exp(-t1 / tau)) <= S.U_CAP * (1 + 1e-12)


def _history(tb, t_end=2000, every=10):
    t = np.arange(0, t_end + 1, every, dtype=float)
    h = np.zeros((len(t), 13))
    h[:, 0] = t
    h[:, 5] = np.where(t >= tb, tb, -1.0) if tb > 0 else -1.0
    h[:, 6] = 1000.0 + t          # volume
    h[:, 8] = 0.01 + 1e-6 * t     # velocity
    h[:, 9] = (t > tb + 150) * 1.0
    return h


def test_outcomes_are_averaged_over_the_window_after_breakup():
    out = S.outcomes_from_history(_history(1003.5), after=(100, 300))
    sel = np.arange(1110, 1301, 10, dtype=float)
    assert out[0] == 1003.5
    assert np.isclose(out[1], (0.01 + 1e-6 * sel).mean())
    assert np.isclose(out[2], (1000.0 + sel).mean())
    assert np.isclose(out[3], (sel > 1153.5).mean())


def test_no_breakup_or_too_late_gives_nan():
    assert np.isnan(S.outcomes_from_history(_history(-1))).all()
    assert np.isnan(S.outcomes_from_history(_history(1950.0))).all()


def test_row_seed_is_a_function_of_the_row():
    a = S.sample_inputs(4, 9)
    assert S.row_seed(a[0]) == S.row_seed(a[0].copy())
    assert len({S.row_seed(r) for r in a}) == 4
    assert S.lattice_params(a[1])["seed"] == S.row_seed(a[1])
