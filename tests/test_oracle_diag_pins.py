"""Closed-form pins of the oracle's diagnostics record (2-D and 3-D).

The record is what the GPU path is compared against for the observables the
paper reports (breakup time, droplet velocity and volume; "Reproducing the
experiment" and the wettability and surface-tension sweeps), so each of its
columns is tied here to a value computed by hand from a state set by the
test.  The rules pinned are the readings of the repository:

  - ink weight e = clamp(phi / phi*, 0, 1); row (plane) integrals
    w = sum e, m = sum e n, p = sum e n u_y over fluid cells;
  - runs: maximal row ranges with w > 1/2; the leading droplet is the
    highest run; volume = sum w over it, centroid = sum y w / sum w,
    velocity = sum p / sum m over it (e n-weighted mean of u_y);
  - satellites = (runs that start at or above the nozzle exit) - 1;
  - neck = least w over rows at or above L - L/2 with more than the nozzle
    width (3-D: pi R^2) of run ink above them; breakup = first record with
    neck < 0.01, its time interpolated linearly in the neck between that
    record and the previous one;
  - mass of n and phi, and total momentum sum n u_y.

The states are set directly (g_0 = phi, the moving g zero; f with a chosen
density and axial momentum), with a surface tension of 1e-12 so that the
interfacial force mu grad(phi) is negligible and u_y is the set momentum
over the set density.
"""
import numpy as np
import pytest

from oracle import OracleSim, OracleSim3, lattice3
from paper_1702_04487_gb300 import workloads as W

PHIS = 4.5
N0 = 5.5


def _params2(**kw):
    p = dict(nx=6, ny=40, geometry=W.GEOM_NONE, nozzle_width=0, nozzle_length=0,
             wall_thickness=0, rho_ink=10.0, rho_air=1.0, nu_ink=0.1, nu_air=0.05,
             sigma=1e-12, width_W=3.0, tau_phi=0.8, theta_deg=90.0, F0=0.0, F_neg=0.0,
             T1=0, T2=0, axial_bc=W.BC_PERIODIC, init_kind=W.INIT_UNIFORM, init_r=-PHIS,
             jitter=0.0, diag_every=1)
    p.update(kw)
    return p


def _state2(s, e_rows, n_rows=None, u_rows=None):
    """f, g of a 2-D state whose every column has phi = e phi*, density n
    and axial velocity u (rest weights plus an up/down pair); solid cells 0."""
    ny, nx = s.ny, s.nx
    e = np.asarray(e_rows, float)
    n = np.full(ny, N0) if n_rows is None else np.asarray(n_rows, float)
    u = np.zeros(ny) if u_rows is None else np.asarray(u_rows, float)
    f = np.zeros((9, ny, nx))
    # f_0 + f_2 + f_4 = n and f_2 - f_4 = n u (directions 2 = +y, 4 = -y)
    f[2] = (0.1 * n + 0.5 * n * u)[:, None]
    f[4] = (0.1 * n - 0.5 * n * u)[:, None]
    f[0] = (0.8 * n)[:, None]
    g = np.zeros((5, ny, nx))
    g[0] = (e * PHIS)[:, None]
    fluid = s.kinds() == 0
    return f * fluid, g * fluid


def _record(p, e_rows, n_rows=None, u_rows=None, t=0, sim=None):
    s = sim or OracleSim(p)
    f, g = _state2(s, e_rows, n_rows, u_rows)
    s.set_state(f, g, t)
    s.step(1)
    return s.history()[-1], s


def test_volume_and_centroid_of_the_leading_run():
    """Two runs of rows; the leading (higher) one has ink weights e(y) that
    vary row by row: volume = nx sum e over its rows, centroid the
    w-weighted mean row, mass of n and phi the plain sums."""
    ny, nx = 40, 6
    e = np.zeros(ny)
    e[3:7] = 1.0                       # lower run
    e[20:26] = [0.3, 0.9, 1.0, 1.0, 0.6, 0.2]   # upper run: rows 20..24 (w = 1.2 at row 25)
    e[26] = 0.05                       # w = 0.3: outside the run
    r, _ = _record(_params2(), e)
    w = nx * e
    run = np.arange(20, 26)
    assert r[10] == 2
    assert abs(r[6] - w[run].sum()) < 1e-12
    assert abs(r[7] - (run * w[run]).sum() / w[run].sum()) < 1e-12
    assert abs(r[1] - N0 * nx * ny) < 1e-9
    assert abs(r[2] - PHIS * nx * e.sum()) < 1e-9


def test_velocity_is_the_ink_and_density_weighted_mean_of_the_leading_run():
    """u_y, n and e vary over the leading run: the record's velocity is
    sum e n u / sum e n over its rows, not the mean of u or of any other run;
    the momentum column is sum n u over every cell."""
    ny, nx = 40, 6
    rng = np.random.default_rng(7)
    e = np.zeros(ny)
    e[4:9] = 1.0
    e[22:30] = rng.uniform(0.2, 1.0, 8)
    n = rng.uniform(2.0, 9.0, ny)
    u = rng.uniform(-0.05, 0.05, ny)
    u[4:9] = 0.09                      # the lower run moves differently
    r, _ = _record(_params2(), e, n, u)
    run = np.arange(22, 30)
    run = run[nx * e[run] > 0.5]
    assert run[0] == 22 and run[-1] == 29  # one run of 8 rows
    expect = (e[run] * n[run] * u[run]).sum() / (e[run] * n[run]).sum()
    assert abs(r[8] - expect) < 1e-10 * abs(expect)
    assert abs(r[3] - nx * (n * u).sum()) < 1e-10
    assert abs(r[1] - nx * n.sum()) < 1e-9


def _nozzle2(**kw):
    return _params2(nx=12, ny=48, geometry=W.GEOM_NOZZLE, nozzle_width=4, nozzle_length=10,
                    wall_thickness=2, **kw)


def test_satellites_count_runs_starting_at_or_above_the_exit():
    """Ink in the nozzle channel (rows 0..L-1) plus three separated slabs
    above the exit: four runs, three of them above, two satellites.  A slab
    that starts exactly at the exit row counts as above; a run that starts
    inside the nozzle and reaches past the exit does not."""
    p = _nozzle2()
    L = p["nozzle_length"]
    e = np.zeros(48)
    e[:L] = 1.0
    e[14:17] = 1.0
    e[22:25] = 1.0
    e[32:36] = 1.0
    r, _ = _record(p, e)
    assert r[10] == 4 and r[9] == 2
    # the channel run extended to row L + 2: it starts below the exit
    e2 = e.copy()
    e2[:L + 3] = 1.0
    r, _ = _record(p, e2)
    assert r[10] == 4 and r[9] == 2
    # the lowest slab moved down to start at the exit row, the channel air
    e3 = e.copy()
    e3[:L] = 0.0
    e3[14:17] = 0.0
    e3[L:L + 3] = 1.0
    r, _ = _record(p, e3)
    assert r[10] == 3 and r[9] == 2
    # one slab only above the exit: no satellite
    e4 = np.zeros(48)
    e4[:L] = 1.0
    e4[20:30] = 1.0
    r, _ = _record(p, e4)
    assert r[10] == 2 and r[9] == 0


def test_neck_and_interpolated_breakup_time():
    """The neck is the least row weight at or above L - L/2 with more than
    the nozzle width of run ink above it; breakup is interpolated linearly
    in the neck between the two records that bracket 0.01."""
    p = _nozzle2()
    L, nx = p["nozzle_length"], 12
    e = np.zeros(48)
    e[:L] = 1.0                 # nozzle rows: w = 8 (channel and the air beside the walls)
    e[L:30] = 1.0               # column above the exit, full width: w = 12
    e[20] = 0.1                 # thin row: w = 1.2
    e[29] = 1.0 / 24            # top row: w = 0.5, not run ink
    r0, s = _record(p, e, t=0)
    assert abs(r0[4] - 1.2) < 1e-12 and r0[5] == -1
    # rows L - L/2 .. L-1 have w = 8; rows below L - L/2 are not scanned
    e_b = e.copy()
    e_b[20] = 0.004 / nx * 10   # w = 0.04: still above 0.01
    r1, s = _record(p, e_b, t=10, sim=s)
    assert abs(r1[4] - 0.04) < 1e-12 and r1[5] == -1
    e_c = e.copy()
    e_c[20] = 0.0005            # w = 0.006 < 0.01: breakup between t = 10 and 20
    r2, s = _record(p, e_c, t=20, sim=s)
    tb = 10 + 10 * (0.04 - 0.01) / (0.04 - 0.006)
    assert abs(r2[4] - 0.006) < 1e-12 and abs(r2[5] - tb) < 1e-9
    # later records keep the first breakup time
    r3, s = _record(p, e, t=30, sim=s)
    assert abs(r3[5] - tb) < 1e-9
    # without a previous record, breakup is the record's own time
    r4, _ = _record(p, e_c, t=40)
    assert r4[5] == 40
    # rows below L - L/2 are not scanned; rows at or above it are
    e_f = e.copy()
    e_f[L // 2 - 1] = 0.01      # w = 0.08, one row below L - L/2
    r_f, _ = _record(p, e_f, t=0)
    assert abs(r_f[4] - 1.2) < 1e-12
    e_f[L // 2 - 1] = 1.0
    e_f[L // 2] = 0.01          # the first scanned row
    r_f, _ = _record(p, e_f, t=0)
    assert abs(r_f[4] - 0.08) < 1e-12
    # the neck ignores rows with too little run ink above (the top rows)
    e_d = e.copy()
    e_d[27] = 0.0               # rows 28 (w 12) above: 12 > 4, so row 27 counts
    r5, _ = _record(p, e_d, t=0)
    assert r5[4] == 0.0
    e_e = e.copy()
    e_e[28] = 0.0               # above row 28: only row 29 (w 0.5, not run ink)
    r6, _ = _record(p, e_e, t=0)
    assert abs(r6[4] - 1.2) < 1e-12


# ------------------------------------------------------------------ 3-D
def _params3(**kw):
    p = _params2(nx=3, ny=4, nz=40)
    p.update(kw)
    return p


def _record3(p, e_planes, n_planes=None, u_planes=None, t=0):
    s = OracleSim3(p)
    ex, ey, ez, _ = lattice3()
    up, down = int(np.flatnonzero((ez == 1) & (ex == 0) & (ey == 0))[0]), \
        int(np.flatnonzero((ez == -1) & (ex == 0) & (ey == 0))[0])
    nz, ny, nx = s.nz, s.ny, s.nx
    e = np.asarray(e_planes, float)
    n = np.full(nz, N0) if n_planes is None else np.asarray(n_planes, float)
    u = np.zeros(nz) if u_planes is None else np.asarray(u_planes, float)
    f = np.zeros((19, nz, ny, nx))
    f[up] = (0.1 * n + 0.5 * n * u)[:, None, None]
    f[down] = (0.1 * n - 0.5 * n * u)[:, None, None]
    f[0] = (0.8 * n)[:, None, None]
    g = np.zeros((7, nz, ny, nx))
    g[0] = (e * PHIS)[:, None, None]
    fluid = s.kinds() == 0
    s.set_state(f * fluid, g * fluid, t)
    s.step(1)
    return s.history()[-1], s


def test_volume_centroid_velocity_along_z():
    nx, ny, nz = 3, 4, 40
    rng = np.random.default_rng(9)
    e = np.zeros(nz)
    e[2:6] = 1.0
    e[18:27] = rng.uniform(0.2, 1.0, 9)
    n = rng.uniform(2.0, 9.0, nz)
    u = rng.uniform(-0.05, 0.05, nz)
    r, _ = _record3(_params3(), e, n, u)
    run = np.arange(18, 27)
    w = nx * ny * e
    assert r[10] == 2
    assert abs(r[6] - w[run].sum()) < 1e-12
    assert abs(r[7] - (run * w[run]).sum() / w[run].sum()) < 1e-12
    expect = (e[run] * n[run] * u[run]).sum() / (e[run] * n[run]).sum()
    assert abs(r[8] - expect) < 1e-10 * abs(expect)
    assert abs(r[1] - nx * ny * n.sum()) < 1e-9
    assert abs(r[3] - nx * ny * (n * u).sum()) < 1e-10


def test_satellites_and_neck_along_z_in_the_round_nozzle():
    """Round nozzle of radius 2 (z < 8): channel ink plus three slabs above
    the exit -> two satellites; a thin plane above the exit is the neck
    (more than pi R^2 of run ink above it)."""
    p = _params3(nx=10, ny=10, nz=40, geometry=W.GEOM_NOZZLE, nozzle_width=2, nozzle_length=8,
                 wall_thickness=2)
    L = 8
    e = np.zeros(40)
    e[:L] = 1.0
    e[12:15] = 1.0
    e[20:23] = 1.0
    e[30:34] = 1.0
    r, s = _record3(p, e)
    assert r[10] == 4 and r[9] == 2
    e2 = np.zeros(40)
    e2[:30] = 1.0
    e2[20] = 0.01            # plane weight 1.0 (100 fluid cells per open plane)
    r2, _ = _record3(p, e2)
    assert r2[10] == 1 and abs(r2[4] - 1.0) < 1e-12
    assert abs(r[6] - 100 * 4) < 1e-12  # the leading slab: 4 open planes of 100 cells
