"""Seeded synthetic workloads for the inkjet lattice Boltzmann model.

This module only draws and lists parameters (plain dicts); it holds none of
the method's arithmetic.  The same dicts feed the CUDA library (through the
binding) and the FP64 oracle, so both sides always see identical inputs.

Keys follow the fields of ``ij_params`` in ``include/inkjet.h``.  All values
are lattice units.  The workloads follow the paper's set-up: a planar
piezo drop-on-demand nozzle driven by a positive pulse, a negative pulse and
an idle time (Fig. 1), an inner-wall contact-angle sweep (Fig. 4-5) and a
surface-tension sweep (Fig. 6-7).
"""
import numpy as np

GEOM_NONE, GEOM_NOZZLE, GEOM_PLATE = 0, 1, 2
BC_ZERO_GRADIENT, BC_PERIODIC, BC_CLOSED = 0, 1, 2
INIT_MENISCUS, INIT_DROP, INIT_FLAT, INIT_UNIFORM = 0, 1, 2, 3

SIGMA_BASE = 0.01


def cfg1(drive="ejecting"):
    """64 x 256 planar nozzle (20 wide, 60 long, walls 4), density ratio 10,
    viscosities 0.1 / 0.05, inner-wall angle 60 degrees.

    ``drive="spec"`` is the nominal waveform (+2e-4 for 800 steps, -1e-4 for
    400) at surface tension 0.01: at this size it only bulges the meniscus
    (Weber number about 0.9) and never ejects.  ``drive="ejecting"`` (the
    default) lowers the surface tension to 0.0025 and drives +2e-3 for 900
    steps then -1e-3 for 800 steps: the droplet pinches off near step 3610
    while the flow stays below |u| = 0.08 (Mach 0.14); run it 4000 steps.
    """
    p = dict(nx=64, ny=256, geometry=GEOM_NOZZLE, nozzle_width=20, nozzle_length=60,
             wall_thickness=4, rho_ink=10.0, rho_air=1.0, nu_ink=0.1, nu_air=0.05,
             sigma=SIGMA_BASE, width_W=3.0, tau_phi=0.8, gamma=0.0, theta_deg=60.0,
             axial_bc=BC_ZERO_GRADIENT, init_kind=INIT_MENISCUS, jitter=1e-6, seed=0,
             diag_every=10, T_idle=0)
    if drive == "spec":
        p.update(F0=2e-4, F_neg=1e-4, T1=800, T2=400)
    else:
        p.update(sigma=SIGMA_BASE / 4, F0=2e-3, F_neg=1e-3, T1=900, T2=800)
    return p


def cfg2_sweep(seed=2):
    """20 runs of a 200 x 1600 nozzle (50 wide, 200 long, walls 10): contact
    angle {30,60,90,120,150} x surface tension {0.5,1,2,4} x base.  Each run
    draws F0 ~ U[1e-4, 4e-4], T1, T2 ~ U{500..3000}; the negative pulse is
    F0 / 2."""
    rng = np.random.default_rng(seed)
    runs = []
    for theta in (30.0, 60.0, 90.0, 120.0, 150.0):
        for mult in (0.5, 1.0, 2.0, 4.0):
            F0 = float(rng.uniform(1e-4, 4e-4))
            T1 = int(rng.integers(500, 3001))
            T2 = int(rng.integers(500, 3001))
            runs.append(dict(nx=200, ny=1600, geometry=GEOM_NOZZLE, nozzle_width=50,
                             nozzle_length=200, wall_thickness=10, rho_ink=10.0, rho_air=1.0,
                             nu_ink=0.1, nu_air=0.05, sigma=SIGMA_BASE * mult, width_W=3.0,
                             tau_phi=0.8, gamma=0.0, theta_deg=theta, F0=F0, F_neg=F0 / 2,
                             T1=T1, T2=T2, T_idle=0, axial_bc=BC_ZERO_GRADIENT,
                             init_kind=INIT_MENISCUS, jitter=1e-6, seed=seed * 1000 + len(runs),
                             diag_every=10))
    return runs


def cfg3_sample(count=256, seed=3):
    """Uneven sweep instances: nozzle width w ~ U{16..48}, domain 4w x 30w,
    nozzle length 4w, walls 4, angle ~ U[20, 160] degrees, surface tension
    log-uniform over [base/2, 2 base], F0, T1, T2 as in the 200 x 1600 sweep."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(count):
        w = int(rng.integers(16, 49))
        F0 = float(rng.uniform(1e-4, 4e-4))
        out.append(dict(nx=4 * w, ny=30 * w, geometry=GEOM_NOZZLE, nozzle_width=w,
                        nozzle_length=4 * w, wall_thickness=4, rho_ink=10.0, rho_air=1.0,
                        nu_ink=0.1, nu_air=0.05,
                        sigma=float(SIGMA_BASE * np.exp(rng.uniform(np.log(0.5), np.log(2.0)))),
                        width_W=3.0, tau_phi=0.8, gamma=0.0,
                        theta_deg=float(rng.uniform(20.0, 160.0)), F0=F0, F_neg=F0 / 2,
                        T1=int(rng.integers(500, 3001)), T2=int(rng.integers(500, 3001)),
                        T_idle=0, axial_bc=BC_ZERO_GRADIENT, init_kind=INIT_MENISCUS,
                        jitter=1e-6, seed=seed * 100000 + k, diag_every=10))
    return out


def big_nozzle(nx=2048, ny=8192):
    """The 200 x 1600 nozzle geometry scaled up to a single lattice larger
    than L2 (2048 x 8192 = 16.8M cells by default)."""
    s = nx / 200.0
    return dict(nx=nx, ny=ny, geometry=GEOM_NOZZLE, nozzle_width=int(50 * s),
                nozzle_length=int(200 * ny / 1600), wall_thickness=int(10 * s), rho_ink=10.0,
                rho_air=1.0, nu_ink=0.1, nu_air=0.05, sigma=SIGMA_BASE, width_W=3.0, tau_phi=0.8,
                gamma=0.0, theta_deg=60.0, F0=3e-4, F_neg=1.5e-4, T1=1500, T2=1500, T_idle=0,
                axial_bc=BC_ZERO_GRADIENT, init_kind=INIT_MENISCUS, jitter=1e-6, seed=7,
                diag_every=10)


def e1(F0=2e-3, **kw):
    """The paper's ejection set-up at its own lattice parameters ("Reproducing
    the experiment"): 200 x 800 lattice, nozzle 80 wide (radius 40) and 120
    long, density ratio 1000 (phi* = 499.5), W = 3, tau_n = 0.85 in both
    fluids, tau_phi = 0.8, surface tension 1.08, wall angle 90 degrees, and
    the 5 / 3 us positive / negative pulses as 3050 / 1830 steps without
    repetition.  The wall thickness (10) and the drive amplitude are not
    printed; the negative pulse is F0 / 2 as in the sweeps."""
    nu = (0.85 - 0.5) / 3.0
    p = dict(nx=200, ny=800, geometry=GEOM_NOZZLE, nozzle_width=80, nozzle_length=120,
             wall_thickness=10, rho_ink=1000.0, rho_air=1.0, nu_ink=nu, nu_air=nu, sigma=1.08,
             width_W=3.0, tau_phi=0.8, gamma=0.0, theta_deg=90.0, F0=F0, F_neg=F0 / 2,
             T1=3050, T2=1830, T_idle=0, axial_bc=BC_ZERO_GRADIENT, init_kind=INIT_MENISCUS,
             jitter=1e-6, seed=11, diag_every=100)
    p.update(kw)
    return p


def small_nozzle(nx=48, ny=96, **kw):
    """A small nozzle lattice for quick checks (16 wide, 30 long, walls 3)."""
    p = dict(nx=nx, ny=ny, geometry=GEOM_NOZZLE, nozzle_width=16, nozzle_length=30,
             wall_thickness=3, rho_ink=10.0, rho_air=1.0, nu_ink=0.1, nu_air=0.05,
             sigma=SIGMA_BASE, width_W=3.0, tau_phi=0.8, gamma=0.0, theta_deg=60.0,
             F0=2e-3, F_neg=1e-3, T1=300, T2=300, T_idle=0, axial_bc=BC_ZERO_GRADIENT,
             init_kind=INIT_MENISCUS, jitter=1e-6, seed=1, diag_every=10)
    p.update(kw)
    return p


def cfg4(theta_deg=60.0, precision=0, nx=128, ny=128, nz=640, radius=24, length=160, wall=10,
         seed=4):
    """3-D round nozzle (D3Q19/D3Q7): 128 x 128 x 640, radius 24, length 160,
    wall 10, axis z.  Drive drawn as in the 200 x 1600 sweep (F0 ~ U[1e-4,
    4e-4], T1, T2 ~ U{500..3000}, negative pulse F0 / 2) from ``seed``.
    ``precision`` 0 stores populations in FP32, 1 in FP16 (offsets)."""
    rng = np.random.default_rng(seed)
    F0 = float(rng.uniform(1e-4, 4e-4))
    T1 = int(rng.integers(500, 3001))
    T2 = int(rng.integers(500, 3001))
    return dict(dim=3, nx=nx, ny=ny, nz=nz, geometry=GEOM_NOZZLE, nozzle_width=radius,
                nozzle_length=length, wall_thickness=wall, rho_ink=10.0, rho_air=1.0,
                nu_ink=0.1, nu_air=0.05, sigma=SIGMA_BASE, width_W=3.0, tau_phi=0.8, gamma=0.0,
                theta_deg=theta_deg, F0=F0, F_neg=F0 / 2, T1=T1, T2=T2, T_idle=0,
                axial_bc=BC_ZERO_GRADIENT, init_kind=INIT_MENISCUS, jitter=1e-6, seed=seed,
                diag_every=10, precision=precision)


def cfg4_downscale(theta_deg=60.0, precision=0):
    """The 3-D round nozzle at a quarter of the size: 32 x 32 x 160, radius
    6, length 40, wall 3, same drive."""
    return cfg4(theta_deg, precision, nx=32, ny=32, nz=160, radius=6, length=40, wall=3)


def small_nozzle3(nx=20, ny=20, nz=64, **kw):
    """A small 3-D round nozzle for quick checks: radius 5, length 16,
    wall 2, ink viscosity 0.05 and a strong drive (+1e-2 for 600 steps,
    -5e-3 for 400): the jet reaches the top and its neck pinches off near
    step 1330."""
    p = dict(dim=3, nx=nx, ny=ny, nz=nz, geometry=GEOM_NOZZLE, nozzle_width=5,
             nozzle_length=16, wall_thickness=2, rho_ink=10.0, rho_air=1.0, nu_ink=0.05,
             nu_air=0.05, sigma=SIGMA_BASE / 4, width_W=3.0, tau_phi=0.8, gamma=0.0,
             theta_deg=60.0, F0=1e-2, F_neg=5e-3, T1=600, T2=400, T_idle=0,
             axial_bc=BC_ZERO_GRADIENT, init_kind=INIT_MENISCUS, jitter=1e-6, seed=5,
             diag_every=10, precision=0)
    p.update(kw)
    return p

