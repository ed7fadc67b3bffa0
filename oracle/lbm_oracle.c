/*
 * FP64 CPU oracle: the binary-fluid lattice Boltzmann inkjet model
 * (He et al., arXiv:1702.04487, "Methods", Eq. 1-10), written as plain
 * whole-field loops in the order the paper states the method.
 *
 * TEST INFRASTRUCTURE ONLY: see lbm_oracle.h.  Nothing here is tiled, fused
 * or reordered; each pass below is one step of the method.  Passes whose
 * cells are independent (each iteration writes only its own cell) may run
 * their rows on several OpenMP threads; the arithmetic of every cell is the
 * same on any number of threads, so results are bit-identical.
 *
 * Readings of what the paper leaves open (each is listed, with its reason,
 * in the design notes of the repository):
 *  - velocity with forcing: n u = sum_i f_i c_i + F/2 (Eq. 4 is a Guo-type
 *    forcing term, whose (1 - 1/2 tau) prefactor implies this half-force
 *    velocity);
 *  - Eq. 10 names index "1" as special; with i = 0..4 that index is taken to
 *    be the rest direction (otherwise the second moment of g^(0) is
 *    anisotropic and its first moment is not phi u / q);
 *  - free energy psi = A (phi^2 - phi*^2)^2, mu = 4 A phi (phi^2 - phi*^2)
 *    - kappa lap(phi), with A = 3 sigma / (8 W phi*^4) and
 *    kappa = 3 sigma W / (4 phi*^2) from the flat tanh profile;
 *  - wetting (Sect. "Reproducing the experiment", ref. 29): Cahn surface
 *    energy -h phi_s imposed through ghost values of phi on solid cells,
 *    cos(theta) = ((1+Omega)^1.5 - (1-Omega)^1.5)/2,
 *    Omega = h / (phi*^2 sqrt(2 kappa A));
 *  - Eq. 8 split into a part (1-q) g_i that stays and a part q g_i + Omega_i
 *    that moves; at a solid target the moving part returns into the
 *    opposite direction of the same cell (mass conserving);
 *  - f bounce-back halfway between cells; two viscosities through
 *    tau_n = 1/2 + 3 nu(C), nu linear in the ink fraction C;
 *  - drive (Fig. 1): force density F(t) C along +y on the nozzle channel.
 */
#include "lbm_oracle.h"

#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* D2Q9 velocity set: rest, 4 axis directions, 4 diagonals (Eq. 5-6). */
static const int EX[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1};
static const int EY[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
static const int OPP[9] = {0, 3, 4, 1, 2, 7, 8, 5, 6};
static const double WT[9] = {4.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0, 1.0 / 9.0,
                             1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0, 1.0 / 36.0};

struct orc_sim {
  orc_params p;
  int nx, ny;
  /* derived constants */
  double phis, n0, A, kappa, q, h, gamma, Omega;
  int cx0, cx1, L; /* nozzle channel columns [cx0, cx1), nozzle rows [0, L) */
  long long t;
  /* state */
  double *f, *g, *fn, *gn;
  /* per-step work fields.  Moments n, phi, mx, my: [ny][nx].  The fields
   * of the collision (mu, gradient, u, C, F_y) live on the extended rows
   * -1..ny ([ny+2][nx]); phih on rows -2..ny+1 ([ny+4][nx]). */
  double *n, *phi, *mx, *my, *mu, *dpx, *dpy, *ux, *uy, *C, *Fy;
  double *phih;          /* phi with ghost values on solid points */
  double *fs;            /* [9][ny+2][nx]: post-collision f, rows -1..ny */
  double *P;             /* [5][ny+2][nx]: moving part of g, rows -1..ny */
  double *S;             /* [5][ny][nx]: staying part; S[0] = g0 + Omega_0 */
  unsigned char* kind;   /* [ny][nx]: 0 fluid, 1 solid, 2 solid wetting face */
  double *wrow, *mrow, *prow;
  /* diagnostics */
  double* hist;
  int nhist, caphist;
  int have_prev;
  double m_prev, t_prev, breakup;
};

/* ---------------------------------------------------------------------- */
/* Counter-based uniform numbers: SplitMix64 (Steele, Lea & Flood, 2014).  */
static uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

double orc_uniform(unsigned long long seed, int x, int y) {
  uint64_t ctr = ((uint64_t)(uint32_t)y << 32) | (uint64_t)(uint32_t)x;
  uint64_t r = splitmix64((uint64_t)seed ^ splitmix64(ctr));
  return (double)(r >> 11) * (1.0 / 9007199254740992.0);
}

/* ---------------------------------------------------------------------- */
/* Eq. 5-6: D2Q9 equilibrium with A_0 = 9n/4 - 15 p / 4, A_i = 3 p,
 * p = phi mu + n / 3. */
void orc_feq(double n, double phi, double mu, double ux, double uy, double* feq) {
  double p = phi * mu + n / 3.0;
  double u2 = ux * ux + uy * uy;
  for (int i = 0; i < 9; i++) {
    double Ai = (i == 0) ? (9.0 / 4.0) * n - 15.0 * p / 4.0 : 3.0 * p;
    double cu = EX[i] * ux + EY[i] * uy;
    feq[i] = WT[i] * Ai + WT[i] * n * (3.0 * cu - 1.5 * u2 + 4.5 * cu * cu);
  }
}

/* Eq. 9-10 (rest direction special): g0_0 = -2 Gamma mu + phi,
 * g0_i = Gamma mu / 2 + phi (c_i . u) / (2 q). */
void orc_geq(double phi, double mu, double ux, double uy, double gamma, double q, double* geq) {
  for (int i = 0; i < 5; i++) {
    double Ai = (i == 0) ? -2.0 * gamma * mu : 0.5 * gamma * mu;
    double Bi = (i == 0) ? 1.0 : 0.0;
    double Ci = 1.0 / (2.0 * q);
    double cu = EX[i] * ux + EY[i] * uy;
    geq[i] = Ai + Bi * phi + Ci * phi * cu;
  }
}

/* Eq. 4, second term: (1 - 1/(2 tau)) (w_i / cs^2)
 * [(c_i - u) + (c_i . u) c_i / cs^2] . F, with cs^2 = 1/3 and delta t = 1. */
void orc_force_term(double tau, double ux, double uy, double Fx, double Fy, double* Fi) {
  const double cs2 = 1.0 / 3.0;
  for (int i = 0; i < 9; i++) {
    double cu = EX[i] * ux + EY[i] * uy;
    double vx = (EX[i] - ux) + cu * EX[i] / cs2;
    double vy = (EY[i] - uy) + cu * EY[i] / cs2;
    Fi[i] = (1.0 - 1.0 / (2.0 * tau)) * (WT[i] / cs2) * (vx * Fx + vy * Fy);
  }
}

/* Inverse of Cahn's wetting relation cos(theta) = ((1+O)^1.5 - (1-O)^1.5)/2
 * in closed form (root of a depressed cubic in trigonometric form). */
double orc_omega_of_theta(double theta_deg) {
  double th = theta_deg * M_PI / 180.0;
  double s = sin(th);
  double alpha = acos(s * s);
  double c = cos(alpha / 3.0);
  double sg = (th < M_PI / 2.0) ? 1.0 : ((th > M_PI / 2.0) ? -1.0 : 0.0);
  return 2.0 * sg * sqrt(c * (1.0 - c));
}

/* ---------------------------------------------------------------------- */
/* Geometry.  Nozzle reading: a channel of width w centred in x, walls of
 * thickness t on both sides for 0 <= y < L; the channel-facing wall faces
 * are the nozzle inner wall and carry the contact angle.  Plate: rows
 * 0 <= y < t are solid, the top face carries the contact angle. */
static int geom_kind(const orc_sim* s, int x, int y) {
  const orc_params* p = &s->p;
  if (p->geometry == ORC_GEOM_NOZZLE) {
    int t = p->wall_thickness;
    if (y < s->L && ((x >= s->cx0 - t && x < s->cx0) || (x >= s->cx1 && x < s->cx1 + t)))
      return (x == s->cx0 - 1 || x == s->cx1) ? 2 : 1;
    return 0;
  }
  if (p->geometry == ORC_GEOM_PLATE) {
    if (y < p->wall_thickness) return (y == p->wall_thickness - 1) ? 2 : 1;
    return 0;
  }
  return 0;
}

static int wrap(int v, int m) {
  int r = v % m;
  return r < 0 ? r + m : r;
}

/* Map an axial index to the domain.  Returns 0 when the cell lies outside a
 * closed domain (a non-wetting solid), 1 otherwise with *ym set. */
static int map_y(const orc_sim* s, int y, int* ym) {
  if (y >= 0 && y < s->ny) {
    *ym = y;
    return 1;
  }
  if (s->p.axial_bc == ORC_BC_PERIODIC) {
    *ym = wrap(y, s->ny);
    return 1;
  }
  if (s->p.axial_bc == ORC_BC_ZERO_GRADIENT) {
    *ym = y < 0 ? 0 : s->ny - 1;
    return 1;
  }
  return 0;
}

/* Kind of any lattice point after the boundary mapping. */
static int kind_at(const orc_sim* s, int x, int y) {
  int ym;
  if (!map_y(s, y, &ym)) return 1;
  return s->kind[(size_t)ym * s->nx + wrap(x, s->nx)];
}

static double phi_fluid_at(const orc_sim* s, const double* phi, int x, int y) {
  int ym;
  map_y(s, y, &ym);
  return phi[(size_t)ym * s->nx + wrap(x, s->nx)];
}

static int in_drive_region(const orc_sim* s, int x, int y) {
  if (s->p.geometry == ORC_GEOM_NOZZLE) return x >= s->cx0 && x < s->cx1 && y < s->L;
  return 1;
}

/* Fig. 1: positive pulse, negative pulse, idle; repeats with period
 * T1 + T2 + T_idle when T_idle > 0, otherwise idles for ever. */
static double drive_at(const orc_params* p, long long t) {
  long long tt = t;
  if (p->T_idle > 0) tt = t % (p->T1 + p->T2 + p->T_idle);
  if (tt < p->T1) return p->F0;
  if (tt < p->T1 + p->T2) return -p->F_neg;
  return 0.0;
}

/* ---------------------------------------------------------------------- */
/* Wetting ghost value of a solid point (x, y): the mean, over its fluid face
 * neighbours, of phi_f + h_s / kappa, where h_s = h on a wetting face and 0
 * elsewhere (kappa dphi/dn = -h at the wall); solid points touching fluid
 * only diagonally take the plain mean of those diagonal neighbours. */
static double ghost_value(const orc_sim* s, const double* phi, int x, int y) {
  int k = kind_at(s, x, y);
  double hk = (k == 2) ? s->h / s->kappa : 0.0;
  double sum = 0.0;
  int cnt = 0;
  for (int d = 1; d <= 4; d++) {
    int xn = x + EX[d], yn = y + EY[d];
    if (kind_at(s, xn, yn) == 0) {
      sum += phi_fluid_at(s, phi, xn, yn) + hk;
      cnt++;
    }
  }
  if (cnt) return sum / cnt;
  for (int d = 5; d <= 8; d++) {
    int xn = x + EX[d], yn = y + EY[d];
    if (kind_at(s, xn, yn) == 0) {
      sum += phi_fluid_at(s, phi, xn, yn);
      cnt++;
    }
  }
  return cnt ? sum / cnt : 0.0;
}

/* The axial ends extend the lattice: outside rows take the mapped row's
 * phi and geometry (replicated edge rows for the zero-gradient ends, wrapped
 * rows for periodic ends) and every rule is then applied on the extended
 * lattice; outside a closed domain lie non-wetting solid rows.
 * fill_phih: phi on fluid points and ghost values on solid points, for the
 * extended rows -2..ny+1. */
static void fill_phih(orc_sim* s, const double* phi) {
  int nx = s->nx, ny = s->ny;
#pragma omp parallel for schedule(static)
  for (int y = -2; y < ny + 2; y++)
    for (int x = 0; x < nx; x++)
      s->phih[(size_t)(y + 2) * nx + x] =
          kind_at(s, x, y) == 0 ? phi_fluid_at(s, phi, x, y) : ghost_value(s, phi, x, y);
}

static double phih_at(const orc_sim* s, int x, int y) {
  return s->phih[(size_t)(y + 2) * s->nx + wrap(x, s->nx)];
}

/* Chemical potential and gradient on fluid points from the isotropic D2Q9
 * stencils: lap = 6 sum_i w_i (phi(x+c_i) - phi(x)), grad = 3 sum_i w_i c_i
 * phi(x+c_i); mu = 4 A phi (phi^2 - phi*^2) - kappa lap. */
static void chem_potential(orc_sim* s) {
  int nx = s->nx, ny = s->ny;
#pragma omp parallel for schedule(static)
  for (int y = -1; y <= ny; y++)
    for (int x = 0; x < nx; x++) {
      size_t c = (size_t)(y + 1) * nx + x;
      if (kind_at(s, x, y) != 0) continue;
      double p0 = phih_at(s, x, y);
      double lap = 0.0, gx = 0.0, gy = 0.0;
      for (int i = 1; i < 9; i++) {
        double pn = phih_at(s, x + EX[i], y + EY[i]);
        lap += 6.0 * WT[i] * (pn - p0);
        gx += 3.0 * WT[i] * EX[i] * pn;
        gy += 3.0 * WT[i] * EY[i] * pn;
      }
      s->mu[c] = 4.0 * s->A * p0 * (p0 * p0 - s->phis * s->phis) - s->kappa * lap;
      s->dpx[c] = gx;
      s->dpy[c] = gy;
    }
}

static double ink_fraction(const orc_sim* s, double phi) {
  double c = 0.5 * (phi / s->phis + 1.0);
  return c < 0.0 ? 0.0 : (c > 1.0 ? 1.0 : c);
}

/* ---------------------------------------------------------------------- */
orc_sim* orc_create(const orc_params* p) {
  if (p->nx < 1 || p->ny < 1) return NULL;
  orc_sim* s = (orc_sim*)calloc(1, sizeof(orc_sim));
  s->p = *p;
  s->nx = p->nx;
  s->ny = p->ny;
  int nx = s->nx, ny = s->ny;
  size_t N = (size_t)nx * ny, NM = (size_t)nx * (ny + 2), NH = (size_t)nx * (ny + 4);
  /* derived constants (free energy, relaxation, wetting) */
  s->phis = 0.5 * (p->rho_ink - p->rho_air);
  s->n0 = 0.5 * (p->rho_ink + p->rho_air);
  s->A = 3.0 * p->sigma / (8.0 * p->width_W * pow(s->phis, 4));
  s->kappa = 3.0 * p->sigma * p->width_W / (4.0 * s->phis * s->phis);
  s->q = 1.0 / (p->tau_phi + 0.5);
  /* default mobility: Gamma kappa = 0.04, half the largest value found stable
   * on the planar nozzle at contact angles 20-160 degrees */
  s->gamma = p->gamma > 0 ? p->gamma : 0.04 / s->kappa;
  s->Omega = orc_omega_of_theta(p->theta_deg);
  s->h = s->Omega * s->phis * s->phis * sqrt(2.0 * s->kappa * s->A);
  s->cx0 = (nx - p->nozzle_width) / 2;
  s->cx1 = s->cx0 + p->nozzle_width;
  s->L = p->nozzle_length;

  s->f = calloc(9 * N, sizeof(double));
  s->g = calloc(5 * N, sizeof(double));
  s->fn = calloc(9 * N, sizeof(double));
  s->gn = calloc(5 * N, sizeof(double));
  double** w[] = {&s->n, &s->phi, &s->mx, &s->my};
  for (size_t k = 0; k < sizeof(w) / sizeof(w[0]); k++) *w[k] = calloc(N, sizeof(double));
  double** we[] = {&s->mu, &s->dpx, &s->dpy, &s->ux, &s->uy, &s->C, &s->Fy};
  for (size_t k = 0; k < sizeof(we) / sizeof(we[0]); k++) *we[k] = calloc(NM, sizeof(double));
  s->phih = calloc(NH, sizeof(double));
  s->fs = calloc(9 * NM, sizeof(double));
  s->P = calloc(5 * NM, sizeof(double));
  s->S = calloc(5 * N, sizeof(double));
  s->kind = calloc(N, 1);
  s->wrow = calloc(ny, sizeof(double));
  s->mrow = calloc(ny, sizeof(double));
  s->prow = calloc(ny, sizeof(double));
  s->caphist = 64;
  s->hist = calloc((size_t)s->caphist * ORC_REC, sizeof(double));
  s->breakup = -1.0;

  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) s->kind[(size_t)y * nx + x] = (unsigned char)geom_kind(s, x, y);

  /* initial order parameter */
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      size_t c = (size_t)y * nx + x;
      double v = 0.0;
      if (s->kind[c] == 0) {
        if (p->init_kind == ORC_INIT_MENISCUS) {
          /* signed distance d to the ink held in the channel below y = L:
           * d = L - y above/below the meniscus inside the channel columns,
           * minus the distance to the channel's top corners beside it */
          int dx = s->cx0 - x > x - (s->cx1 - 1) ? s->cx0 - x : x - (s->cx1 - 1);
          int inch = dx <= 0;
          if (inch)
            v = s->phis * tanh((s->L - y) / p->width_W);
          else if (y < s->L)
            v = -s->phis;
          else
            v = s->phis * tanh(-sqrt((double)dx * dx + (double)(y - s->L) * (y - s->L)) / p->width_W);
          if (inch && fabs((double)(y - s->L)) < 2.0 * p->width_W)
            v += p->jitter * (2.0 * orc_uniform(p->seed, x, y) - 1.0);
        } else if (p->init_kind == ORC_INIT_DROP) {
          double dx = x - p->init_x;
          dx -= nx * floor(dx / nx + 0.5); /* periodic minimal image */
          double dy = y - p->init_y;
          v = s->phis * tanh((p->init_r - sqrt(dx * dx + dy * dy)) / p->width_W);
        } else if (p->init_kind == ORC_INIT_FLAT) {
          v = s->phis * tanh((p->init_y - y) / p->width_W);
        } else {
          v = p->init_r;
        }
      }
      s->phi[c] = v;
    }
  /* initial mu from the initial phi (with wetting ghosts); n = n0, u = 0 */
  fill_phih(s, s->phi);
  chem_potential(s);
  for (size_t c = 0; c < N; c++) {
    double fe[9], ge[5];
    if (s->kind[c] != 0) continue;
    double mu = s->mu[c + (size_t)nx];
    orc_feq(s->n0, s->phi[c], mu, 0.0, 0.0, fe);
    orc_geq(s->phi[c], mu, 0.0, 0.0, s->gamma, s->q, ge);
    for (int i = 0; i < 9; i++) s->f[i * N + c] = fe[i];
    for (int i = 0; i < 5; i++) s->g[i * N + c] = ge[i];
  }
  return s;
}

void orc_destroy(orc_sim* s) {
  if (!s) return;
  double* a[] = {s->f, s->g, s->fn, s->gn, s->n, s->phi, s->mx, s->my, s->mu, s->dpx, s->dpy, s->ux,
                 s->uy, s->C, s->Fy, s->phih, s->fs, s->P, s->S, s->wrow, s->mrow, s->prow, s->hist};
  for (size_t k = 0; k < sizeof(a) / sizeof(a[0]); k++) free(a[k]);
  free(s->kind);
  free(s);
}

long long orc_time(const orc_sim* s) { return s->t; }

void orc_derived(const orc_sim* s, double* out) {
  out[0] = s->phis;
  out[1] = s->n0;
  out[2] = s->A;
  out[3] = s->kappa;
  out[4] = s->q;
  out[5] = s->h;
  out[6] = s->gamma;
  out[7] = s->Omega;
}

void orc_kinds(const orc_sim* s, unsigned char* out) { memcpy(out, s->kind, (size_t)s->nx * s->ny); }

void orc_get_state(const orc_sim* s, double* f, double* g) {
  size_t N = (size_t)s->nx * s->ny;
  memcpy(f, s->f, 9 * N * sizeof(double));
  memcpy(g, s->g, 5 * N * sizeof(double));
}

void orc_set_state(orc_sim* s, const double* f, const double* g, long long t) {
  size_t N = (size_t)s->nx * s->ny;
  memcpy(s->f, f, 9 * N * sizeof(double));
  memcpy(s->g, g, 5 * N * sizeof(double));
  s->t = t;
}

/* ---------------------------------------------------------------------- */
/* Pass 1 (Eq. 3, 8 definitions): n = sum f_i, phi = sum g_i, momentum. */
static void moments(orc_sim* s) {
  size_t N = (size_t)s->nx * s->ny;
#pragma omp parallel for schedule(static)
  for (size_t c = 0; c < N; c++) {
    if (s->kind[c] != 0) continue;
    double n = 0, mx = 0, my = 0, phi = 0;
    for (int i = 0; i < 9; i++) {
      double fi = s->f[i * N + c];
      n += fi;
      mx += fi * EX[i];
      my += fi * EY[i];
    }
    for (int i = 0; i < 5; i++) phi += s->g[i * N + c];
    s->n[c] = n;
    s->mx[c] = mx;
    s->my[c] = my;
    s->phi[c] = phi;
  }
}

/* Pass 4 (Eq. 2, 4): total force mu grad(phi) + F_b and the half-force
 * velocity, on the extended rows. */
static void velocity(orc_sim* s, long long t) {
  int nx = s->nx, ny = s->ny;
  double Fd = drive_at(&s->p, t);
#pragma omp parallel for schedule(static)
  for (int y = -1; y <= ny; y++) {
    int ym;
    if (!map_y(s, y, &ym)) continue;
    for (int x = 0; x < nx; x++) {
      size_t c = (size_t)ym * nx + x, e = (size_t)(y + 1) * nx + x;
      if (s->kind[c] != 0) continue;
      double C = ink_fraction(s, s->phi[c]);
      double Fb = in_drive_region(s, x, ym) ? Fd * C : 0.0;
      double Fx = s->mu[e] * s->dpx[e];
      double Fy = s->mu[e] * s->dpy[e] + Fb;
      s->C[e] = C;
      s->Fy[e] = Fy;
      s->ux[e] = (s->mx[c] + 0.5 * Fx) / s->n[c];
      s->uy[e] = (s->my[c] + 0.5 * Fy) / s->n[c];
    }
  }
}

/* Pass 5: collision of f (Eq. 4-6) and of g (Eq. 8-10), on the extended
 * rows (an outside row collides the populations of its mapped row). */
static void collide(orc_sim* s) {
  int nx = s->nx, ny = s->ny;
  size_t N = (size_t)nx * ny, NM = (size_t)nx * (ny + 2);
  const orc_params* p = &s->p;
#pragma omp parallel for schedule(static)
  for (int y = -1; y <= ny; y++) {
    int ym;
    if (!map_y(s, y, &ym)) continue;
    for (int x = 0; x < nx; x++) {
      size_t c = (size_t)ym * nx + x, e = (size_t)(y + 1) * nx + x;
      if (s->kind[c] != 0) continue;
      double C = s->C[e];
      double nu = p->nu_air + C * (p->nu_ink - p->nu_air);
      double tau = 0.5 + 3.0 * nu;
      double Fx = s->mu[e] * s->dpx[e];
      double Fy = s->Fy[e];
      double fe[9], Fi[9], ge[5];
      orc_feq(s->n[c], s->phi[c], s->mu[e], s->ux[e], s->uy[e], fe);
      orc_force_term(tau, s->ux[e], s->uy[e], Fx, Fy, Fi);
      for (int i = 0; i < 9; i++) {
        double fi = s->f[i * N + c];
        s->fs[i * NM + e] = fi + (fe[i] - fi) / tau + Fi[i];
      }
      orc_geq(s->phi[c], s->mu[e], s->ux[e], s->uy[e], s->gamma, s->q, ge);
      int inside = y >= 0 && y < ny;
      for (int i = 0; i < 5; i++) {
        double gi = s->g[i * N + c];
        double om = (ge[i] - gi) / p->tau_phi;
        if (i == 0) {
          if (inside) s->S[c] = gi + om;
        } else {
          s->P[i * NM + e] = s->q * gi + om;
          if (inside) s->S[i * N + c] = (1.0 - s->q) * gi;
        }
      }
    }
  }
}

/* Pass 6: streaming (Eq. 3) with halfway bounce-back, and the g update of
 * Eq. 8 as G_i(y) = (1-q) g_i(y) + [q g_i + Omega_i](y - c_i); a moving part
 * whose source is solid is the cell's own part of the opposite direction. */
static void stream(orc_sim* s) {
  int nx = s->nx, ny = s->ny;
  size_t N = (size_t)nx * ny, NM = (size_t)nx * (ny + 2);
#pragma omp parallel for schedule(static)
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      size_t c = (size_t)y * nx + x, cm = (size_t)(y + 1) * nx + x;
      if (s->kind[c] != 0) continue;
      s->fn[c] = s->fs[cm];
      for (int i = 1; i < 9; i++) {
        int xs = x - EX[i], ys = y - EY[i];
        if (kind_at(s, xs, ys) != 0)
          s->fn[i * N + c] = s->fs[OPP[i] * NM + cm];
        else
          s->fn[i * N + c] = s->fs[i * NM + (size_t)(ys + 1) * nx + wrap(xs, nx)];
      }
      s->gn[c] = s->S[c];
      for (int i = 1; i < 5; i++) {
        int xs = x - EX[i], ys = y - EY[i];
        double moving;
        if (kind_at(s, xs, ys) != 0)
          moving = s->P[OPP[i] * NM + cm];
        else
          moving = s->P[i * NM + (size_t)(ys + 1) * nx + wrap(xs, nx)];
        s->gn[i * N + c] = s->S[i * N + c] + moving;
      }
    }
  /* solid cells keep their (unused) values */
  for (size_t c = 0; c < N; c++)
    if (s->kind[c] != 0) {
      for (int i = 0; i < 9; i++) s->fn[i * N + c] = s->f[i * N + c];
      for (int i = 0; i < 5; i++) s->gn[i * N + c] = s->g[i * N + c];
    }
  double* tf = s->f;
  s->f = s->fn;
  s->fn = tf;
  double* tg = s->g;
  s->g = s->gn;
  s->gn = tg;
}

void orc_stream_only(orc_sim* s, const double* fin, const double* gin, double* fout, double* gout) {
  int nx = s->nx, ny = s->ny;
  size_t N = (size_t)nx * ny, NM = (size_t)nx * (ny + 2);
  double q_saved = s->q;
  s->q = 1.0;
  for (int y = 0; y < ny; y++)
    for (int x = 0; x < nx; x++) {
      size_t c = (size_t)y * nx + x, cm = (size_t)(y + 1) * nx + x;
      for (int i = 0; i < 9; i++) s->fs[i * NM + cm] = fin[i * N + c];
      s->S[c] = gin[c];
      for (int i = 1; i < 5; i++) {
        s->P[i * NM + cm] = gin[i * N + c];
        s->S[i * N + c] = 0.0;
      }
    }
  for (int e = 0; e < 2; e++) {
    int y = e == 0 ? -1 : ny, ym;
    if (!map_y(s, y, &ym)) continue;
    for (int x = 0; x < nx; x++) {
      size_t dst = (size_t)(y + 1) * nx + x, src = (size_t)ym * nx + x;
      for (int i = 0; i < 9; i++) s->fs[i * NM + dst] = fin[i * N + src];
      for (int i = 1; i < 5; i++) s->P[i * NM + dst] = gin[i * N + src];
    }
  }
  double *f0 = s->f, *g0 = s->g;
  s->f = (double*)fin; /* solid cells copy their input values */
  s->g = (double*)gin;
  double *fn0 = s->fn, *gn0 = s->gn;
  s->fn = fout;
  s->gn = gout;
  stream(s); /* swaps f<->fn: undo below */
  s->f = f0;
  s->g = g0;
  s->fn = fn0;
  s->gn = gn0;
  s->q = q_saved;
}

/* ---------------------------------------------------------------------- */
/* Diagnostics of the state at time t (before its update), in FP64.
 * Ink weight e = clamp(phi / phi*, 0, 1): 1 in bulk ink, 0 for C <= 1/2, so
 * the small ink fraction of bulk air never counts.  Rows: w(y) = sum_x e,
 * m(y) = sum_x e n, p(y) = sum_x e n u_y over fluid cells.  Runs: maximal row ranges with w > 1/2.  Neck: the least w(y) over
 * rows y >= y_scan that have more than V_min of run ink (the w of run rows)
 * above them; breakup is the first record whose neck falls below
 * NECK_BREAK (1/100 of a cell of ink: the last thread of ink across the
 * neck row is vanishing), its time interpolated linearly in the neck width
 * between this record and the previous one.  The leading droplet is the highest run (volume, centroid,
 * e n-weighted velocity); satellites = (runs that start at or above the
 * nozzle exit) - 1.  Its head and tail are where w(y) crosses 1/2 at the
 * run's upper and lower ends, by linear interpolation between the last row
 * inside and the first row outside (the end row itself at the lattice's
 * edge; -1 without a run); their velocities are differences between
 * records. */
#define NECK_BREAK 0.01

static void diagnose(orc_sim* s, long long t) {
  int nx = s->nx, ny = s->ny;
  double mass_n = 0, mass_phi = 0, mom_y = 0;
  for (int y = 0; y < ny; y++) {
    double w = 0, m = 0, pr = 0;
    for (int x = 0; x < nx; x++) {
      size_t c = (size_t)y * nx + x;
      if (s->kind[c] != 0) continue;
      double e = s->phi[c] / s->phis, n = s->n[c], uy = s->uy[c + (size_t)nx];
      e = e < 0.0 ? 0.0 : (e > 1.0 ? 1.0 : e);
      w += e;
      m += e * n;
      pr += e * n * uy;
      mass_n += n;
      mass_phi += s->phi[c];
      mom_y += n * uy;
    }
    s->wrow[y] = w;
    s->mrow[y] = m;
    s->prow[y] = pr;
  }
  int nozzle = s->p.geometry == ORC_GEOM_NOZZLE;
  int y_exit = nozzle ? s->L : 0;
  int y_scan = nozzle ? s->L - s->L / 2 : 0;
  double vmin = nozzle ? (double)s->p.nozzle_width : 1.0;
  double neck = 1e30, above = 0.0;
  for (int y = ny - 1; y >= 0; y--) {
    if (y >= y_scan && above > vmin && s->wrow[y] < neck) neck = s->wrow[y];
    if (s->wrow[y] > 0.5) above += s->wrow[y];
  }
  if (s->breakup < 0 && neck < NECK_BREAK) {
    if (s->have_prev && s->m_prev >= NECK_BREAK && s->m_prev < 1e29)
      s->breakup = s->t_prev + (t - s->t_prev) * (s->m_prev - NECK_BREAK) / (s->m_prev - neck);
    else
      s->breakup = (double)t;
  }
  s->have_prev = 1;
  s->m_prev = neck;
  s->t_prev = (double)t;
  /* runs of rows with w > 1/2 */
  int nruns = 0, nabove = 0, lead0 = -1, lead1 = -1;
  for (int y = 0; y < ny;) {
    if (s->wrow[y] > 0.5) {
      int y0 = y;
      while (y < ny && s->wrow[y] > 0.5) y++;
      nruns++;
      if (y0 >= y_exit) nabove++;
      lead0 = y0;
      lead1 = y;
    } else {
      y++;
    }
  }
  double vol = 0, ycm = 0, mm = 0, pp = 0;
  for (int y = lead0; lead0 >= 0 && y < lead1; y++) {
    vol += s->wrow[y];
    ycm += y * s->wrow[y];
    mm += s->mrow[y];
    pp += s->prow[y];
  }
  double rec[ORC_REC] = {0};
  rec[0] = (double)t;
  rec[1] = mass_n;
  rec[2] = mass_phi;
  rec[3] = mom_y;
  rec[4] = neck;
  rec[5] = s->breakup;
  rec[6] = vol;
  rec[7] = vol > 0 ? ycm / vol : 0.0;
  rec[8] = mm > 0 ? pp / mm : 0.0;
  rec[9] = nabove > 1 ? nabove - 1 : 0;
  rec[10] = nruns;
  rec[11] = rec[12] = -1.0;
  if (lead0 >= 0) {
    int top = lead1 - 1;
    rec[11] = lead1 < ny ? top + (s->wrow[top] - 0.5) / (s->wrow[top] - s->wrow[lead1]) : top;
    rec[12] = lead0 > 0 ? lead0 - (s->wrow[lead0] - 0.5) / (s->wrow[lead0] - s->wrow[lead0 - 1])
                        : lead0;
  }
  if (s->nhist == s->caphist) {
    s->caphist *= 2;
    s->hist = realloc(s->hist, (size_t)s->caphist * ORC_REC * sizeof(double));
  }
  memcpy(s->hist + (size_t)s->nhist * ORC_REC, rec, sizeof(rec));
  s->nhist++;
}

int orc_history(const orc_sim* s, double* out, int max_records) {
  int n = s->nhist < max_records ? s->nhist : max_records;
  if (out && n > 0) memcpy(out, s->hist, (size_t)n * ORC_REC * sizeof(double));
  return s->nhist;
}

/* One time step in the paper's order: moments, wetting ghosts and chemical
 * potential, forces and velocity, collision, streaming. */
static void step_once(orc_sim* s) {
  moments(s);
  fill_phih(s, s->phi);
  chem_potential(s);
  velocity(s, s->t);
  if (s->p.diag_every > 0 && s->t % s->p.diag_every == 0) diagnose(s, s->t);
  collide(s);
  stream(s);
  s->t++;
}

void orc_step(orc_sim* s, long long nsteps) {
  for (long long k = 0; k < nsteps; k++) step_once(s);
}

void orc_fields(orc_sim* s, double* n, double* phi, double* mu, double* ux, double* uy) {
  size_t N = (size_t)s->nx * s->ny;
  moments(s);
  fill_phih(s, s->phi);
  chem_potential(s);
  velocity(s, s->t);
  for (size_t c = 0; c < N; c++) {
    int fl = s->kind[c] == 0;
    size_t e = c + (size_t)s->nx;
    if (n) n[c] = fl ? s->n[c] : 0.0;
    if (phi) phi[c] = fl ? s->phi[c] : 0.0;
    if (mu) mu[c] = fl ? s->mu[e] : 0.0;
    if (ux) ux[c] = fl ? s->ux[e] : 0.0;
    if (uy) uy[c] = fl ? s->uy[e] : 0.0;
  }
}

/* Threads of the per-cell passes (1 without OpenMP). */
int orc_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}
