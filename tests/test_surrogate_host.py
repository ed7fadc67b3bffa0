"""Host logic of the surrogate service (no GPU): the input sampler, the
lattice of an input row and the outcome read-out from a diagnostics
history."""
import numpy as np

from paper_1702_04487_gb300 import surrogate as S


def test_sampler_is_seeded_and_inside_the_box():
    a, b = S.sample_inputs(500, 3), S.sample_inputs(500, 3)
    assert np.array_equal(a, b)
    assert not np.array_equal(a, S.sample_inputs(500, 4))
    for k, name in enumerate(S.INPUT_NAMES):
        lo, hi = S.INPUT_BOX[name]
        assert a[:, k].min() >= lo and a[:, k].max() <= hi
    for k in (3, 4, 5, 6):
        assert np.array_equal(a[:, k], np.round(a[:, k]))


def test_lattice_of_an_input_row():
    row = [60.0, 0.0015, 2e-3, 1000, 1000, 3000, 18]
    p = S.lattice_params(row, seed=5)
    assert (p["nx"], p["ny"], p["nozzle_width"], p["nozzle_length"]) == (72, 432, 18, 54)
    assert p["F_neg"] == p["F0"] / 2 and p["T_idle"] == 3000 and p["seed"] == 5
    assert p["nozzle_width"] + 2 * p["wall_thickness"] <= p["nx"]


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
