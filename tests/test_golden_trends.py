"""The paper's printed trend data (tests/golden/paper_trends.json).

The printed numbers are in microseconds with an unprinted lattice mapping, so
they pin only directions: breakup later with a more hydrophobic inner wall
(Fig. 4) and earlier with a higher surface tension (Fig. 6).  The GPU sweep
tests check the same directions on the model.
"""
import json
import os

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_trends.json")


def load():
    with open(GOLDEN) as fh:
        return json.load(fh)


def test_printed_breakup_trends_are_monotone():
    d = load()
    ang = d["fig4_breakup_us_vs_contact_angle_deg"]
    vals = [ang[k] for k in sorted(ang, key=float)]
    assert all(a < b for a, b in zip(vals, vals[1:]))
    sig = d["fig6_breakup_us_vs_surface_tension_mN_per_m"]
    vals = [sig[k] for k in sorted(sig, key=float)]
    assert all(a >= b for a, b in zip(vals, vals[1:]))
