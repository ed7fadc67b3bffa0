"""Brute-force agreement of the FP64 C oracle with a second, naive transcription.

The C oracle (oracle/lbm_oracle.c) is checked here against an independent
restatement of one time step of the method, written in plain NumPy from the
paper's equations and the readings the repository takes where the paper is
silent:

  - moments n = sum f_i, phi = sum g_i (Eq. 3, 8);
  - wetting ghost values of phi on solid cells (Cahn surface energy,
    "Reproducing the experiment"), with the wetting potential found here by
    bisection of cos(theta) = ((1+Omega)^1.5 - (1-Omega)^1.5)/2 instead of
    the oracle's closed-form root;
  - isotropic D2Q9 stencils and mu = 4 A phi (phi^2 - phi*^2) - kappa lap phi;
  - drive F(t) C along +y on the nozzle channel (Fig. 1) and the half-force
    velocity u = (sum f c + F/2) / n (Eq. 4 is a Guo-type forcing term);
  - the f collision of Eq. 4-6 with tau_n = 1/2 + 3 nu(C);
  - the g update of Eq. 8-10 (rest direction special) split into a part
    (1 - q) g_i that stays and a part q g_i + Omega_i that moves;
  - pull streaming with np.roll, halfway bounce-back at solid sources, and
    the axial ends as an extended lattice (zero-gradient, periodic, closed).

Nothing is imported from the oracle but its public step and state calls:
the naive side derives A, kappa, q, Gamma, h and the initial state itself.
On 8 x 8 (and 12 x 10) lattices both agree to 1e-13 after 100 steps, so a
slip in either (a dropped term, a wrong sign, index or weight, a boundary
rule applied on the wrong row) shows here.
"""
import numpy as np
import pytest

from oracle import OracleSim
from paper_1702_04487_gb300 import workloads as W

EX = np.array([0, 1, 0, -1, 0, 1, -1, -1, 1])
EY = np.array([0, 0, 1, 0, -1, 1, 1, -1, -1])
WT = np.array([4 / 9] + [1 / 9] * 4 + [1 / 36] * 4)
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]
FACES = [(1, 0), (0, 1), (-1, 0), (0, -1)]
DIAGS = [(1, 1), (-1, 1), (-1, -1), (1, -1)]


def _splitmix64(z):
    m = (1 << 64) - 1
    z = (z + 0x9E3779B97F4A7C15) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def _uniform(seed, x, y):
    ctr = ((y & 0xFFFFFFFF) << 32) | (x & 0xFFFFFFFF)
    return (_splitmix64(seed ^ _splitmix64(ctr)) >> 11) / 2.0 ** 53


def _omega_by_bisection(theta_deg):
    """Root in [-1, 1] of ((1+O)^1.5 - (1-O)^1.5)/2 = cos(theta) (increasing in O)."""
    target = np.cos(np.radians(theta_deg))
    lo, hi = -1.0, 1.0
    for _ in range(200):
        mid = 0.5 * (lo + hi)
        if 0.5 * ((1 + mid) ** 1.5 - (1 - mid) ** 1.5) < target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


class Naive:
    """One lattice, FP64, written cell rule by cell rule."""

    def __init__(self, p):
        full = dict(p)
        self.p = full
        self.nx, self.ny = full["nx"], full["ny"]
        self.phis = 0.5 * (full["rho_ink"] - full["rho_air"])
        self.n0 = 0.5 * (full["rho_ink"] + full["rho_air"])
        sig, Wd = full["sigma"], full["width_W"]
        self.A = 3 * sig / (8 * Wd * self.phis ** 4)
        self.kappa = 3 * sig * Wd / (4 * self.phis ** 2)
        self.q = 1 / (full["tau_phi"] + 0.5)
        self.gamma = full["gamma"] if full["gamma"] > 0 else 0.04 / self.kappa
        om = _omega_by_bisection(full["theta_deg"])
        self.h = om * self.phis ** 2 * np.sqrt(2 * self.kappa * self.A)
        w = full.get("nozzle_width", 0)
        self.cx0 = (self.nx - w) // 2
        self.cx1 = self.cx0 + w
        self.L = full.get("nozzle_length", 0)
        self.kind = np.zeros((self.ny, self.nx), dtype=int)
        for y in range(self.ny):
            for x in range(self.nx):
                self.kind[y, x] = self._geom(x, y)
        self.t = 0
        self._init_state()

    # ---- geometry and the extended lattice
    def _geom(self, x, y):
        g, t = self.p["geometry"], self.p.get("wall_thickness", 0)
        if g == W.GEOM_NOZZLE:
            left = self.cx0 - t <= x < self.cx0
            right = self.cx1 <= x < self.cx1 + t
            if y < self.L and (left or right):
                return 2 if x in (self.cx0 - 1, self.cx1) else 1
            return 0
        if g == W.GEOM_PLATE:
            return (2 if y == t - 1 else 1) if y < t else 0
        return 0

    def _row(self, y):
        """Mapped row of an axial index, or None outside a closed domain."""
        if 0 <= y < self.ny:
            return y
        bc = self.p["axial_bc"]
        if bc == W.BC_PERIODIC:
            return y % self.ny
        if bc == W.BC_ZERO_GRADIENT:
            return 0 if y < 0 else self.ny - 1
        return None

    def kind_at(self, x, y):
        r = self._row(y)
        return 1 if r is None else self.kind[r, x % self.nx]

    def _phi_hat(self, phi, x, y):
        """phi on fluid points; wetting ghost value on solid points."""
        k = self.kind_at(x, y)
        if k == 0:
            return phi[self._row(y), x % self.nx]
        shift = self.h / self.kappa if k == 2 else 0.0
        vals = [phi[self._row(y + dy), (x + dx) % self.nx] + shift
                for dx, dy in FACES if self.kind_at(x + dx, y + dy) == 0]
        if not vals:
            vals = [phi[self._row(y + dy), (x + dx) % self.nx]
                    for dx, dy in DIAGS if self.kind_at(x + dx, y + dy) == 0]
        return sum(vals) / len(vals) if vals else 0.0

    # ---- the paper's local rules
    def _mu_grad(self, phi):
        """mu, dphi/dx, dphi/dy on the rows -1..ny (arrays [ny+2][nx])."""
        nx, ny = self.nx, self.ny
        ph = np.array([[self._phi_hat(phi, x, y) for x in range(nx)]
                       for y in range(-2, ny + 2)])
        ctr = ph[1:ny + 3]
        lap = np.zeros_like(ctr)
        gx = np.zeros_like(ctr)
        gy = np.zeros_like(ctr)
        for i in range(1, 9):
            nb = np.roll(ph, -EX[i], axis=1)[1 + EY[i]:ny + 3 + EY[i]]
            lap += 6 * WT[i] * (nb - ctr)
            gx += 3 * WT[i] * EX[i] * nb
            gy += 3 * WT[i] * EY[i] * nb
        mu = 4 * self.A * ctr * (ctr ** 2 - self.phis ** 2) - self.kappa * lap
        return mu, gx, gy

    def _drive(self, t):
        p = self.p
        tt = t % (p["T1"] + p["T2"] + p["T_idle"]) if p["T_idle"] > 0 else t
        if tt < p["T1"]:
            return p["F0"]
        if tt < p["T1"] + p["T2"]:
            return -p["F_neg"]
        return 0.0

    def _extended(self, a):
        """Field on rows 0..ny-1 -> rows -1..ny by the axial mapping (0 outside a closed domain)."""
        out = np.zeros((a.shape[0], self.ny + 2, self.nx))
        for ye in range(-1, self.ny + 1):
            r = self._row(ye)
            if r is not None:
                out[:, ye + 1] = a[:, r]
        return out

    def _init_state(self):
        p, nx, ny = self.p, self.nx, self.ny
        phi = np.zeros((ny, nx))
        for y in range(ny):
            for x in range(nx):
                if self.kind[y, x]:
                    continue
                kind = p["init_kind"]
                if kind == W.INIT_MENISCUS:
                    dx = max(self.cx0 - x, x - (self.cx1 - 1))
                    if dx <= 0:
                        v = self.phis * np.tanh((self.L - y) / p["width_W"])
                        if abs(y - self.L) < 2 * p["width_W"]:
                            v += p["jitter"] * (2 * _uniform(p["seed"], x, y) - 1)
                    elif y < self.L:
                        v = -self.phis
                    else:
                        v = self.phis * np.tanh(-np.hypot(dx, y - self.L) / p["width_W"])
                elif kind == W.INIT_DROP:
                    ddx = x - p["init_x"]
                    ddx -= nx * np.floor(ddx / nx + 0.5)
                    v = self.phis * np.tanh((p["init_r"] - np.hypot(ddx, y - p["init_y"]))
                                            / p["width_W"])
                elif kind == W.INIT_FLAT:
                    v = self.phis * np.tanh((p["init_y"] - y) / p["width_W"])
                else:
                    v = p["init_r"]
                phi[y, x] = v
        mu = self._mu_grad(phi)[0][1:ny + 1]
        n = self.n0
        pr = phi * mu + n / 3
        self.f = np.zeros((9, ny, nx))
        self.g = np.zeros((5, ny, nx))
        fluid = self.kind == 0
        for i in range(9):
            Ai = 9 * n / 4 - 15 * pr / 4 if i == 0 else 3 * pr
            self.f[i] = np.where(fluid, WT[i] * Ai, 0.0)
        self.g[0] = np.where(fluid, phi - 2 * self.gamma * mu, 0.0)
        for i in range(1, 5):
            self.g[i] = np.where(fluid, 0.5 * self.gamma * mu, 0.0)

    def step(self):
        p, nx, ny = self.p, self.nx, self.ny
        f, g = self.f, self.g
        n = f.sum(0)
        phi = g.sum(0)
        mx = np.tensordot(EX, f, axes=1)
        my = np.tensordot(EY, f, axes=1)
        mu, gx, gy = self._mu_grad(phi)
        # every cell field on the extended rows -1..ny
        nE =self._extended(n[None])[0]
        phiE = self._extended(phi[None])[0]
        mxE = self._extended(mx[None])[0]
        myE = self._extended(my[None])[0]
        fE = self._extended(f)
        gE = self._extended(g)
        kindE = np.ones((ny + 2, nx), dtype=int)
        drive = np.zeros((ny + 2, nx), dtype=bool)
        for ye in range(-1, ny + 1):
            r = self._row(ye)
            if r is None:
                continue
            kindE[ye + 1] = self.kind[r]
            for x in range(nx):
                if p["geometry"] == W.GEOM_NOZZLE:
                    drive[ye + 1, x] = self.cx0 <= x < self.cx1 and r < self.L
                else:
                    drive[ye + 1, x] = True
        fluidE = kindE == 0
        safe_n = np.where(fluidE, nE, 1.0)
        C = np.clip(0.5 * (phiE / self.phis + 1), 0.0, 1.0)
        Fx = mu * gx
        Fy = mu * gy + np.where(drive, self._drive(self.t) * C, 0.0)
        ux = (mxE + 0.5 * Fx) / safe_n
        uy = (myE + 0.5 * Fy) / safe_n
        tau = 0.5 + 3 * (p["nu_air"] + C * (p["nu_ink"] - p["nu_air"]))
        pr = phiE * mu + nE / 3
        u2 = ux ** 2 + uy ** 2
        fs = np.zeros_like(fE)
        for i in range(9):
            cu = EX[i] * ux + EY[i] * uy
            Ai = 9 * nE / 4 - 15 * pr / 4 if i == 0 else 3 * pr
            feq = WT[i] * Ai + WT[i] * nE * (3 * cu - 1.5 * u2 + 4.5 * cu ** 2)
            Fi = (1 - 1 / (2 * tau)) * 3 * WT[i] * (
                ((EX[i] - ux) + 3 * cu * EX[i]) * Fx + ((EY[i] - uy) + 3 * cu * EY[i]) * Fy)
            fs[i] = np.where(fluidE, fE[i] + (feq - fE[i]) / tau + Fi, 0.0)
        q, tphi = self.q, p["tau_phi"]
        moving = np.zeros_like(gE)
        staying = np.zeros_like(gE)
        for i in range(5):
            cu = EX[i] * ux + EY[i] * uy
            geq = (-2 * self.gamma * mu + phiE) if i == 0 else \
                (0.5 * self.gamma * mu + phiE * cu / (2 * q))
            om = (geq - gE[i]) / tphi
            if i == 0:
                staying[0] = gE[0] + om
            else:
                moving[i] = q * gE[i] + om
                staying[i] = (1 - q) * gE[i]
        # pull streaming: value from (x - c_i, y - c_i), or the own opposite
        # population when that source is solid (halfway bounce-back)
        fluid = self.kind == 0
        fn = f.copy()
        gn = g.copy()
        for i in range(9):
            src = np.roll(fs[i], EX[i], axis=1)[1 - EY[i]:ny + 1 - EY[i]]
            solid_src = np.roll(~fluidE, EX[i], axis=1)[1 - EY[i]:ny + 1 - EY[i]]
            val = np.where(solid_src, fs[OPP[i]][1:ny + 1], src)
            fn[i] = np.where(fluid, val, f[i])
        gn[0] = np.where(fluid, staying[0][1:ny + 1], g[0])
        for i in range(1, 5):
            src = np.roll(moving[i], EX[i], axis=1)[1 - EY[i]:ny + 1 - EY[i]]
            solid_src = np.roll(~fluidE, EX[i], axis=1)[1 - EY[i]:ny + 1 - EY[i]]
            val = staying[i][1:ny + 1] + np.where(solid_src, moving[OPP[i]][1:ny + 1], src)
            gn[i] = np.where(fluid, val, g[i])
        self.f, self.g = fn, gn
        self.t += 1


def _base(**kw):
    p = dict(nx=8, ny=8, geometry=W.GEOM_NOZZLE, nozzle_width=2, nozzle_length=3,
             wall_thickness=2, rho_ink=10.0, rho_air=1.0, nu_ink=0.1, nu_air=0.05,
             sigma=0.01, width_W=3.0, tau_phi=0.8, gamma=0.0, theta_deg=60.0,
             F0=1e-3, F_neg=5e-4, T1=40, T2=30, T_idle=0, axial_bc=W.BC_ZERO_GRADIENT,
             init_kind=W.INIT_MENISCUS, init_x=0.0, init_y=0.0, init_r=0.0, jitter=1e-6,
             seed=5, diag_every=0)
    p.update(kw)
    return p


CASES = {
    "nozzle_zero_gradient": _base(),
    "nozzle_periodic": _base(axial_bc=W.BC_PERIODIC),
    "nozzle_closed": _base(axial_bc=W.BC_CLOSED),
    "nozzle_repeated_waveform_120deg": _base(theta_deg=120.0, T1=15, T2=10, T_idle=12),
    "nozzle_12x10_thin_walls": _base(nx=12, ny=10, nozzle_width=4, wall_thickness=1,
                                     nozzle_length=4, theta_deg=45.0),
    "plate_drop_closed": _base(geometry=W.GEOM_PLATE, wall_thickness=2, axial_bc=W.BC_CLOSED,
                               init_kind=W.INIT_DROP, init_x=4.0, init_y=3.0, init_r=2.5,
                               theta_deg=60.0),
    "open_drop_periodic": _base(geometry=W.GEOM_NONE, axial_bc=W.BC_PERIODIC,
                                init_kind=W.INIT_DROP, init_x=3.5, init_y=4.0, init_r=2.5),
}


@pytest.mark.parametrize("name", sorted(CASES))
def test_oracle_agrees_with_naive_transcription(name):
    """Initial state and 100 steps: every population within 1e-13 (relative
    to max|f| and phi*) of the naive NumPy transcription."""
    p = CASES[name]
    o = OracleSim(p)
    nv = Naive(p)
    phis = nv.phis
    fo, go = o.state()
    assert np.abs(fo - nv.f).max() < 1e-14 * np.abs(fo).max()
    assert np.abs(go - nv.g).max() < 1e-14 * phis
    for _ in range(100):
        nv.step()
    o.step(100)
    fo, go = o.state()
    ef = np.abs(fo - nv.f).max() / np.abs(fo).max()
    eg = np.abs(go - nv.g).max() / phis
    assert ef < 1e-13 and eg < 1e-13, (ef, eg)
    # the run did something: the state moved away from the initial one
    assert np.abs(nv.g.sum(0) - Naive(p).g.sum(0)).max() > 1e-6 * phis


def test_naive_transcription_detects_a_planted_slip():
    """The comparison has teeth: the naive side with one sign of the forcing
    term flipped (a plausible slip) departs from the oracle by far more than
    the 1e-13 bound within 100 steps."""
    p = CASES["nozzle_zero_gradient"]

    class Slipped(Naive):
        def _drive(self, t):
            return -Naive._drive(self, t)

    o = OracleSim(p)
    nv = Slipped(p)
    for _ in range(100):
        nv.step()
    o.step(100)
    fo, _ = o.state()
    assert np.abs(fo - nv.f).max() / np.abs(fo).max() > 1e-9
