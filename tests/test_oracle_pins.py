"""Pins of the FP64 oracle against what the paper and the mathematics fix.

Each test ties one part of the oracle to something other than itself: a
closed-form moment identity, an exact invariant, a textbook special case, an
analytic equilibrium or a brute-force check.  A plausible slip in the oracle
(a dropped term, a wrong sign, weight or index) fails at least one of them.
"""
import numpy as np
import pytest

from oracle import OracleSim, feq, force_term, geq, omega_of_theta, uniform
from paper_1702_04487_gb300 import workloads as W

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
OPP = np.array([0, 3, 4, 1, 2, 7, 8, 5, 6])

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _rng_cases(n=20, seed=11):
    rng = np.random.default_rng(seed)
    for _ in range(n):
        yield (rng.uniform(1, 10), rng.uniform(-5, 5), rng.uniform(-1e-2, 1e-2),
               rng.uniform(-0.1, 0.1), rng.uniform(-0.1, 0.1))


# ---------------------------------------------------------------- Eq. 5-6
def test_feq_moments_closed_form():
    """Eq. 5-6: sum f0 = n, sum f0 c = n u, sum f0 cc = (n/3 + phi mu) I + n u u."""
    for n, phi, mu, ux, uy in _rng_cases():
        f = feq(n, phi, mu, ux, uy)
        p = n / 3 + phi * mu
        assert abs(f.sum() - n) < 1e-13 * n
        assert abs((f * EX).sum() - n * ux) < 1e-13 * n
        assert abs((f * EY).sum() - n * uy) < 1e-13 * n
        assert abs((f * EX * EX).sum() - (p + n * ux * ux)) < 1e-13 * n
        assert abs((f * EY * EY).sum() - (p + n * uy * uy)) < 1e-13 * n
        assert abs((f * EX * EY).sum() - n * ux * uy) < 1e-13 * n


# ---------------------------------------------------------------- Eq. 4
def test_force_term_moments_guo():
    """Eq. 4 forcing: zeroth moment 0, first (1-1/2tau) F, second
    (1-1/2tau)(uF + Fu) -- the Guo moments that fix u = (sum f c + F/2)/n."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        tau = rng.uniform(0.55, 2.0)
        ux, uy, Fx, Fy = rng.uniform(-0.1, 0.1, 4)
        F = force_term(tau, ux, uy, Fx, Fy)
        a = 1 - 1 / (2 * tau)
        assert abs(F.sum()) < 1e-15
        assert abs((F * EX).sum() - a * Fx) < 1e-15
        assert abs((F * EY).sum() - a * Fy) < 1e-15
        assert abs((F * EX * EX).sum() - a * 2 * ux * Fx) < 1e-15
        assert abs((F * EY * EY).sum() - a * 2 * uy * Fy) < 1e-15
        assert abs((F * EX * EY).sum() - a * (ux * Fy + uy * Fx)) < 1e-15


# ---------------------------------------------------------------- Eq. 9-10
def test_geq_moments_rest_direction_reading():
    """Eq. 9-10 with the special index read as the rest direction:
    sum g0 = phi, sum g0 c = phi u / q, sum g0 cc = Gamma mu I (isotropic)."""
    ex, ey = EX[:5], EY[:5]
    for n, phi, mu, ux, uy in _rng_cases(seed=5):
        gamma, q = 7.3, 1 / 1.3
        g = geq(phi, mu, ux, uy, gamma, q)
        assert abs(g.sum() - phi) < 1e-13
        assert abs((g * ex).sum() - phi * ux / q) < 1e-13
        assert abs((g * ey).sum() - phi * uy / q) < 1e-13
        assert abs((g * ex * ex).sum() - gamma * mu) < 1e-13
        assert abs((g * ey * ey).sum() - gamma * mu) < 1e-13
        assert abs((g * ex * ey).sum()) < 1e-13


# ---------------------------------------------------------------- wetting
def test_wetting_potential_inverts_cahn_relation():
    """Omega(theta) inverts cos(theta) = ((1+Omega)^1.5 - (1-Omega)^1.5)/2
    (forward relation evaluated independently here); neutral wall at 90 deg;
    Omega decreasing in theta."""
    prev = None
    for th in np.linspace(0.0, 180.0, 37):
        om = omega_of_theta(th)
        assert abs(0.5 * ((1 + om) ** 1.5 - (1 - om) ** 1.5) - np.cos(np.radians(th))) < 1e-12
        if prev is not None:
            assert om < prev
        prev = om
    assert omega_of_theta(90.0) == 0.0


def test_splitmix64_published_vector():
    """The jitter generator is SplitMix64 (Steele, Lea & Flood 2014); its
    first output from state 0 is 0xE220A8397B1DCDAF.  U(0, 0, 0) applies it
    twice: splitmix(0 ^ splitmix(0))."""
    def sm(z):
        m = (1 << 64) - 1
        z = (z + 0x9E3779B97F4A7C15) & m
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
        return z ^ (z >> 31)
    assert sm(0) == 0xE220A8397B1DCDAF
    for seed, x, y in [(0, 0, 0), (5, 3, 7), (123456789, 63, 255)]:
        ctr = (y << 32) | x
        expect = (sm(seed ^ sm(ctr)) >> 11) * 2.0 ** -53
        assert uniform(seed, x, y) == expect


# ---------------------------------------------------------------- streaming
@pytest.mark.parametrize("bc", [W.BC_PERIODIC, W.BC_CLOSED])
def test_streaming_is_an_exact_permutation(bc):
    """Eq. 3 streaming with halfway bounce-back (and the q = 1 g streaming)
    moves integer-tagged populations without loss or duplication, and is
    undone exactly by reversing every direction, streaming, and reversing
    back (time reversibility), including every bounce-back link."""
    p = W.small_nozzle(nx=30, ny=20, nozzle_width=10, nozzle_length=12, wall_thickness=3,
                       axial_bc=bc)
    s = OracleSim(p)
    fluid = s.kinds() == 0
    ny, nx = fluid.shape
    f = np.arange(9 * ny * nx, dtype=np.float64).reshape(9, ny, nx) + 1
    g = np.arange(5 * ny * nx, dtype=np.float64).reshape(5, ny, nx) + 1e6
    fo, go = s.stream_only(f, g)
    assert np.array_equal(np.sort(fo[:, fluid].ravel()), np.sort(f[:, fluid].ravel()))
    assert np.array_equal(np.sort(go[:, fluid].ravel()), np.sort(g[:, fluid].ravel()))
    fr, gr = s.stream_only(fo[OPP], go[OPP[:5]])
    assert np.array_equal(fr[OPP][:, fluid], f[:, fluid])
    assert np.array_equal(gr[OPP[:5]][:, fluid], g[:, fluid])


def test_q1_reduces_to_textbook_bgk_streaming():
    """With tau_phi = 1/2 (q = 1) the shift term of Eq. 8 vanishes and the g
    update is plain BGK: g_i(x + c_i) = g_i + (g0_i - g_i) / tau_phi, here
    rebuilt with numpy rolls on a periodic lattice."""
    p = W.small_nozzle(nx=24, ny=20, geometry=W.GEOM_NONE, axial_bc=W.BC_PERIODIC,
                       init_kind=W.INIT_DROP, init_x=12, init_y=9, init_r=5,
                       tau_phi=0.5, F0=1e-3)
    s = OracleSim(p)
    s.step(5)
    fl = s.fields()
    f0, g0 = s.state()
    q, gamma = s.derived()["q"], s.derived()["gamma"]
    assert q == 1.0
    post = np.empty_like(g0)
    for y in range(p["ny"]):
        for x in range(p["nx"]):
            ge = geq(fl["phi"][y, x], fl["mu"][y, x], fl["ux"][y, x], fl["uy"][y, x], gamma, q)
            post[:, y, x] = g0[:, y, x] + (ge - g0[:, y, x]) / 0.5
    expect = np.stack([np.roll(np.roll(post[i], EY[i], 0), EX[i], 1) for i in range(5)])
    s.step(1)
    _, g1 = s.state()
    assert np.abs(g1 - expect).max() < 1e-13 * np.abs(expect).max()


# ---------------------------------------------------------------- invariants
@pytest.mark.parametrize("bc", [W.BC_PERIODIC, W.BC_CLOSED])
def test_mass_of_both_components_conserved(bc):
    """Sum n and sum phi over fluid cells stay constant to 1e-12 relative
    with walls, wetting (60 deg), drive and two viscosities: halfway
    bounce-back of f and the mass-conserving split of Eq. 8 at walls."""
    p = W.small_nozzle(axial_bc=bc, diag_every=1, F0=2e-3, F_neg=1e-3, T1=300, T2=300)
    s = OracleSim(p)
    s.step(1500)
    h = s.history()
    n0, p0 = h[0, 1], h[0, 2]
    scale_phi = 4.5 * p["nx"] * p["ny"]
    assert np.abs(h[:, 1] - n0).max() < 1e-12 * n0
    assert np.abs(h[:, 2] - p0).max() < 1e-12 * scale_phi
    assert np.abs(h[:, 3]).max() > 1e-3  # the drive did move the fluid


def test_momentum_budget_of_uniform_driven_box():
    """Single phase (phi = phi*, so mu = 0 and C = 1), no walls, periodic:
    every step adds exactly F(t) N of momentum (Eq. 4 forcing), so the
    half-force momentum sum n u_y at step t is (sum_{s<t} F(s) + F(t)/2) N
    through the positive pulse, the negative pulse and the idle."""
    p = W.small_nozzle(nx=12, ny=10, geometry=W.GEOM_NONE, axial_bc=W.BC_PERIODIC,
                       init_kind=W.INIT_UNIFORM, init_r=4.5, F0=1e-4, F_neg=4e-5, T1=7, T2=5,
                       diag_every=1)
    s = OracleSim(p)
    s.step(20)
    h = s.history()
    F = np.array([1e-4] * 7 + [-4e-5] * 5 + [0.0] * 8)
    N = p["nx"] * p["ny"]
    expect = (np.concatenate([[0.0], np.cumsum(F)[:-1]]) + F / 2) * N
    assert np.allclose(h[:, 3], expect, rtol=1e-12, atol=1e-16)


def test_momentum_budget_of_repeated_waveform():
    """The same budget with T_idle > 0: the positive / negative / idle cycle
    repeats with period T1 + T2 + T_idle (Fig. 1 as a periodic waveform)."""
    p = W.small_nozzle(nx=12, ny=10, geometry=W.GEOM_NONE, axial_bc=W.BC_PERIODIC,
                       init_kind=W.INIT_UNIFORM, init_r=4.5, F0=1e-4, F_neg=4e-5, T1=7, T2=5,
                       T_idle=4, diag_every=1)
    s = OracleSim(p)
    s.step(40)
    h = s.history()
    cycle = [1e-4] * 7 + [-4e-5] * 5 + [0.0] * 4
    F = np.array((cycle * 3)[:40])
    N = p["nx"] * p["ny"]
    expect = (np.concatenate([[0.0], np.cumsum(F)[:-1]]) + F / 2) * N
    assert np.allclose(h[:, 3], expect, rtol=1e-12, atol=1e-16)


def test_uniform_state_is_stationary_under_zero_gradient_ends():
    """A uniform fluid at rest stays uniform to round-off with the
    'fully developed' (zero-gradient) axial ends."""
    p = W.small_nozzle(nx=10, ny=14, geometry=W.GEOM_NONE, axial_bc=W.BC_ZERO_GRADIENT,
                       init_kind=W.INIT_UNIFORM, init_r=-4.5)
    s = OracleSim(p)
    f0, g0 = s.state()
    s.step(100)
    f1, g1 = s.state()
    assert np.abs(f1 - f0).max() < 1e-14 and np.abs(g1 - g0).max() < 1e-13


# ---------------------------------------------------------------- physics
def test_poiseuille_in_bare_nozzle():
    """Single-phase flow driven through the nozzle channel with periodic
    ends relaxes to u(x) = F (a^2 - x^2) / (2 n nu), walls halfway between
    nodes; exact for halfway bounce-back at tau = 1/2 + sqrt(3/16) (neutral
    walls, so phi stays uniform and the C-weighted drive is F everywhere)."""
    w, t = 10, 2
    nu = np.sqrt(3.0 / 16.0) / 3.0
    p = W.small_nozzle(nx=w + 2 * t, ny=3, nozzle_width=w, nozzle_length=3, wall_thickness=t,
                       axial_bc=W.BC_PERIODIC, init_kind=W.INIT_UNIFORM, init_r=4.5,
                       nu_ink=nu, nu_air=nu, F0=1e-5, T1=10 ** 9, T2=0, theta_deg=90.0)
    s = OracleSim(p)
    s.step(6000)
    uy = s.fields()["uy"][1, t:t + w]
    xc = np.arange(w) - (w - 1) / 2.0
    a = w / 2.0
    expect = 1e-5 * (a * a - xc * xc) / (2 * 5.5 * nu)
    assert np.abs(uy - expect).max() < 1e-9 * expect.max()


def test_flat_interface_profile_and_surface_tension():
    """psi = A (phi^2 - phi*^2)^2 with A, kappa from (sigma, W): a flat
    interface relaxes to phi* tanh(z / W), and kappa * integral(phi')^2
    returns sigma."""
    p = W.small_nozzle(nx=4, ny=80, geometry=W.GEOM_NONE, axial_bc=W.BC_CLOSED,
                       init_kind=W.INIT_FLAT, init_y=40, jitter=0.0, nu_air=0.1, F0=0.0, F_neg=0.0)
    s = OracleSim(p)
    s.step(4000)
    phi = s.fields()["phi"][:, 0]
    d = s.derived()
    y = np.arange(80)
    assert np.abs(phi - d["phis"] * np.tanh((40 - y) / 3.0)).max() < 0.01 * d["phis"]
    sigma_num = d["kappa"] * np.sum(np.gradient(phi) ** 2)
    assert abs(sigma_num - p["sigma"]) < 0.03 * p["sigma"]


@pytest.mark.slow
def test_laplace_law_recovers_surface_tension():
    """Static drops: the bulk pressure jump n/3 + phi mu - psi (inside minus
    outside) equals sigma / R to 5% at R = 10, 14, 20, the error shrinking
    as the interface width W = 3 becomes small against R."""
    errs = []
    for R in (10, 14, 20):
        p = W.small_nozzle(nx=64, ny=64, geometry=W.GEOM_NONE, axial_bc=W.BC_PERIODIC,
                           init_kind=W.INIT_DROP, init_x=32, init_y=32, init_r=R, jitter=0.0,
                           nu_air=0.1, F0=0.0, F_neg=0.0)
        s = OracleSim(p)
        s.step(5000)
        fl = s.fields()
        d = s.derived()
        psi = d["A"] * (fl["phi"] ** 2 - d["phis"] ** 2) ** 2
        pres = fl["n"] / 3 + fl["phi"] * fl["mu"] - psi
        errs.append(abs((pres[32, 32] - pres[0, 0]) * R - p["sigma"]) / p["sigma"])
    assert max(errs) < 0.05
    assert errs[2] < errs[0] and errs[2] < 0.02


@pytest.mark.parametrize("theta,tol", [(60.0, 0.04), (120.0, 0.04), (30.0, 0.08)])
def test_wall_profile_matches_cahn_wetting(theta, tol):
    """Ink or air bulk against a wetting plate: the relaxed near-wall phi
    follows the continuum Cahn solution whose wall value solves
    phi_w^2 = phi*^2 (1 +- Omega) (coth profile above phi*, tanh below),
    to within the lattice's O(1/W^2) error."""
    kappa = 3 * W.SIGMA_BASE * 3 / (4 * 4.5 ** 2)
    for sign in (1.0, -1.0):
        p = W.small_nozzle(nx=4, ny=60, geometry=W.GEOM_PLATE, wall_thickness=2,
                           axial_bc=W.BC_ZERO_GRADIENT, init_kind=W.INIT_UNIFORM,
                           init_r=sign * 4.5, theta_deg=theta, gamma=0.07 / kappa, F0=0.0, F_neg=0.0,
                           nu_air=0.1)
        s = OracleSim(p)
        s.step(20000)
        d = s.derived()
        phi = s.fields()["phi"][2:, 0]
        z = np.arange(2, 60) - 1.5
        ps, om = d["phis"], d["Omega"]
        pw = sign * ps * np.sqrt(1 + sign * om)
        Wd = np.sqrt(d["kappa"] / (2 * d["A"])) / ps
        if abs(pw) > ps:
            prof = sign * ps / np.tanh((z + Wd * np.arctanh(ps / abs(pw))) / Wd)
        else:
            prof = sign * ps * np.tanh((z + Wd * np.arctanh(abs(pw) / ps)) / Wd)
        assert np.abs(phi - prof).max() < tol * ps


def _contour_points(phi, kinds):
    pts = []
    ny, nx = phi.shape
    for y in range(ny):
        for x in range(nx):
            if kinds[y, x]:
                continue
            for dx, dy in ((1, 0), (0, 1)):
                x2, y2 = (x + dx) % nx, y + dy
                if y2 >= ny or kinds[y2, x2]:
                    continue
                a, b = phi[y, x], phi[y2, x2]
                if a * b < 0:
                    t = a / (a - b)
                    pts.append((x + dx * t, y + dy * t))
    return np.array(pts)


def _cap_angle(phi, kinds, y_wall):
    pts = _contour_points(phi, kinds)
    pts = pts[pts[:, 1] >= y_wall + 2]
    x, y = pts[:, 0], pts[:, 1]
    sol = np.linalg.lstsq(np.c_[2 * x, 2 * y, np.ones_like(x)], x * x + y * y, rcond=None)[0]
    xc, yc, c = sol
    R = np.sqrt(c + xc * xc + yc * yc)
    return np.degrees(np.arccos((y_wall - yc) / R))


@pytest.mark.slow
def test_sessile_drop_contact_angle():
    """A drop on the wetting plate: started as the exact 120-degree cap it
    keeps its angle (within 3 deg), and a half-disc (90 deg) on a 60-degree
    wall spreads monotonically towards 60."""
    kappa = 3 * W.SIGMA_BASE * 3 / (4 * 4.5 ** 2)
    yw, R0 = 1.5, 12.0
    base = dict(nx=80, ny=40, geometry=W.GEOM_PLATE, wall_thickness=2, axial_bc=W.BC_CLOSED,
                init_kind=W.INIT_DROP, init_x=40, init_r=R0, jitter=0.0, gamma=0.07 / kappa,
                F0=0.0, F_neg=0.0, nu_air=0.1)
    s = OracleSim(W.small_nozzle(**dict(base, theta_deg=120.0,
                                        init_y=yw - R0 * np.cos(np.radians(120.0)))))
    s.step(6000)
    assert abs(_cap_angle(s.fields()["phi"], s.kinds(), yw) - 120.0) < 3.0
    s = OracleSim(W.small_nozzle(**dict(base, theta_deg=60.0, init_y=2.0)))
    angles = []
    for _ in range(3):
        s.step(3000)
        angles.append(_cap_angle(s.fields()["phi"], s.kinds(), yw))
    assert angles[0] < 88 and angles[0] > angles[1] > angles[2] > 60.0


def _components(mask):
    """4-connected components, x periodic (plain flood fill)."""
    ny, nx = mask.shape
    lab = np.zeros(mask.shape, dtype=int)
    n = 0
    for y0 in range(ny):
        for x0 in range(nx):
            if mask[y0, x0] and not lab[y0, x0]:
                n += 1
                stack = [(y0, x0)]
                lab[y0, x0] = n
                while stack:
                    y, x = stack.pop()
                    for dy, dx in ((1, 0), (-1, 0), (0, 1), (0, -1)):
                        yy, xx = y + dy, (x + dx) % nx
                        if 0 <= yy < ny and mask[yy, xx] and not lab[yy, xx]:
                            lab[yy, xx] = n
                            stack.append((yy, xx))
    return n


@pytest.mark.slow
def test_breakup_rule_agrees_with_connected_components():
    """The row-integral breakup rule (cfg 1, ejecting drive) flags pinch-off
    when brute-force 4-connected labelling of the ink cells (phi > 0) is
    about to split: one body of ink 100 steps before the flag, two or more
    within 40 steps after it."""
    p = W.cfg1()
    s = OracleSim(p)
    s.step(3400)
    while s.history()[-1, 5] < 0:
        s.step(10)
        assert s.t <= 4000
    tb = s.history()[-1, 5]
    assert 3400 < tb < 4000
    s2 = OracleSim(p)
    s2.step(int(tb) - 100)
    assert _components(s2.fields()["phi"] > 0) == 1
    s2.step(100 + 40)
    assert _components(s2.fields()["phi"] > 0) >= 2


@pytest.mark.slow
def test_fp32_noise_floor_of_cfg1():
    """The round-off floor that bounds any FP32 implementation of cfg 1: two
    oracle runs that each take a relative 2^-24 (FP32 rounding) perturbation
    of every population after every step end up, after 1000 steps, a few
    1e-6 to ~1.5e-5 of phi* from the exact run, concentrated at the driven
    meniscus.  The GPU parity bound on phi (1e-5) lies inside this floor."""
    p = W.cfg1("spec")
    ref = OracleSim(p)
    noisy = OracleSim(p)
    rng = np.random.default_rng(12)
    eps = 2.0 ** -24
    for t in range(1, 1001):
        ref.step(1)
        noisy.step(1)
        f, g = noisy.state()
        noisy.set_state(f * (1 + eps * rng.uniform(-1, 1, f.shape)),
                        g * (1 + eps * rng.uniform(-1, 1, g.shape)), t)
    d = np.abs(noisy.state()[1].sum(0) - ref.state()[1].sum(0)).max() / 4.5
    assert 2e-6 < d < 1.5e-5


# ------------------------------------------------------- head and tail
def _slab_record(rows_phi, nx=4):
    """Diagnostics record of a state at rest whose order parameter is
    phi(y) = rows_phi[y] in every column (no walls, periodic)."""
    ny = len(rows_phi)
    p = W.small_nozzle(nx=nx, ny=ny, geometry=W.GEOM_NONE, axial_bc=W.BC_PERIODIC,
                       init_kind=W.INIT_UNIFORM, init_r=-4.5, diag_every=1)
    n0 = 0.5 * (p["rho_ink"] + p["rho_air"])
    wts = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
    f = np.broadcast_to(wts[:, None, None] * n0, (9, ny, nx)).copy()
    g = np.zeros((5, ny, nx))
    g[0] = np.asarray(rows_phi, dtype=np.float64)[:, None]
    s = OracleSim(p)
    s.set_state(f, g, 0)
    s.step(1)
    return s.history()[0]


def test_head_and_tail_closed_form():
    """Head and tail of the leading run (rows with more than half a cell of
    ink) where the row ink weight crosses 1/2, interpolated between rows:
    on slabs of 4 columns they have closed forms."""
    ps = 4.5
    ink, air = ps, -ps
    # sharp slab over rows 6..11: w = 4 inside, 0 outside
    r = _slab_record([air] * 6 + [ink] * 6 + [air] * 8)
    assert r[10] == 1
    assert abs(r[11] - (11 + 3.5 / 4)) < 1e-12 and abs(r[12] - (6 - 3.5 / 4)) < 1e-12
    # partial rows outside: w = 0.4 above (e = 0.1), 0.2 below (e = 0.05)
    r = _slab_record([air] * 5 + [0.05 * ps] + [ink] * 6 + [0.1 * ps] + [air] * 7)
    assert abs(r[11] - (11 + 3.5 / 3.6)) < 1e-12 and abs(r[12] - (6 - 3.5 / 3.8)) < 1e-12
    # two runs: the leading droplet is the higher one (rows 10..13)
    r = _slab_record([air] * 2 + [ink] * 3 + [air] * 5 + [ink] * 4 + [air] * 6)
    assert r[10] == 2
    assert abs(r[11] - (13 + 3.5 / 4)) < 1e-12 and abs(r[12] - (10 - 3.5 / 4)) < 1e-12
    # a run reaching the top row ends there
    r = _slab_record([air] * 14 + [ink] * 6)
    assert r[11] == 19 and abs(r[12] - (14 - 3.5 / 4)) < 1e-12
    # no run
    r = _slab_record([air] * 12)
    assert r[10] == 0 and r[11] == -1 and r[12] == -1
