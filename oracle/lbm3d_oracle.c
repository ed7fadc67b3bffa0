/*
 * FP64 CPU oracle of the 3-D lift of the binary-fluid LBM inkjet model
 * (He et al., arXiv:1702.04487, "Methods", Eq. 3-10, lifted from D2Q9/D2Q5
 * to D3Q19/D3Q7) with a round nozzle.
 *
 * TEST INFRASTRUCTURE ONLY (see lbm_oracle.h): plain whole-field loops in the
 * order of the method, no tiling or fusion, shared with nothing else.  Passes
 * whose cells are independent may run their planes on several OpenMP
 * threads, with bit-identical results on any number of threads.
 *
 * The paper is 2-D.  The 3-D lattice keeps the same readings as the 2-D
 * oracle (Guo half-force velocity, rest direction special in the g
 * equilibrium, Cahn wetting through ghost phi, mass-conserving Eq. 8 at
 * walls, extended-lattice axial ends) and matches moments for the new
 * lattices:
 *  - D3Q19 f^(0)_i = w_i A_i + w_i n (3 c.u - 1.5 u^2 + 4.5 (c.u)^2) with
 *    w = 1/3, 1/18 (6 axis), 1/36 (12 edge), A_i = 3 p for i >= 1 and
 *    A_0 = 3 n - 6 p (p = phi mu + n/3), so that sum f0 = n and
 *    sum f0 c c = p I + n u u (the analogue of Eq. 5-6);
 *  - D3Q7 g^(0)_0 = phi - 3 Gamma mu, g^(0)_i = Gamma mu / 2 +
 *    phi (c_i.u) / (2 q), so that sum g0 = phi, sum g0 c = phi u / q,
 *    sum g0 c c = Gamma mu I (the analogue of Eq. 9-10);
 *  - stencils lap = 6 sum_i w_i (phi_i - phi), grad = 3 sum_i w_i c_i phi_i
 *    over D3Q19.
 * Geometry: z is the nozzle axis.  Round nozzle: channel r < R for z < L and
 * a wall of thickness t (R <= r < R + t, r measured from the lattice centre
 * ((nx-1)/2, (ny-1)/2)); wall cells with a lateral face neighbour in the
 * channel form the wetting inner wall.  Plate: solid layers z < t, the top
 * layer wetting.  x and y are periodic.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "lbm_oracle.h"

static const int EX[19] = {0, 1, -1, 0, 0, 0, 0, 1, -1, 1, -1, 1, -1, 1, -1, 0, 0, 0, 0};
static const int EY[19] = {0, 0, 0, 1, -1, 0, 0, 1, 1, -1, -1, 0, 0, 0, 0, 1, -1, 1, -1};
static const int EZ[19] = {0, 0, 0, 0, 0, 1, -1, 0, 0, 0, 0, 1, 1, -1, -1, 1, 1, -1, -1};
static int OPP[19];
static double WT[19];

typedef struct {
  orc_params p;
  int nz;
  int nx, ny;
  double phis, n0, A, kappa, q, h, gamma, Omega;
  double cx, cy, R;
  long long t;
  double *f, *g, *fn, *gn;
  double *n, *phi, *mx, *my, *mz;       /* [nz][ny][nx] */
  double *phih;                          /* [nz+4][ny][nx]: planes -2..nz+1 */
  double *mu, *dpx, *dpy, *dpz, *ux, *uy, *uz, *C, *Fz; /* [nz+2][ny][nx] */
  double *fs, *P, *S;
  unsigned char* kind;
  double *wrow, *mrow, *prow;
  double* hist;
  int nhist, caphist, have_prev;
  double m_prev, t_prev, breakup;
} orc3;

/* Weights and opposite directions of the table above, filled on first use
 * (always from one thread: orc3_create, or a direct call of the per-cell
 * functions) and read only afterwards. */
static int tables_ready = 0;

static void init_tables(void) {
  if (tables_ready) return;
  for (int i = 0; i < 19; i++) {
    int a = EX[i] * EX[i] + EY[i] * EY[i] + EZ[i] * EZ[i];
    WT[i] = a == 0 ? 1.0 / 3.0 : (a == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
    for (int j = 0; j < 19; j++)
      if (EX[j] == -EX[i] && EY[j] == -EY[i] && EZ[j] == -EZ[i]) OPP[i] = j;
  }
  tables_ready = 1;
}

static int wrap(int v, int m) {
  int r = v % m;
  return r < 0 ? r + m : r;
}

/* ---------------------------------------------------------------------- */
/* D3Q19 equilibrium (moment-matched Eq. 5-6). */
void orc3_feq(double n, double phi, double mu, const double* u, double* feq) {
  init_tables();
  double p = phi * mu + n / 3.0;
  double u2 = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  for (int i = 0; i < 19; i++) {
    double Ai = i == 0 ? 3.0 * n - 6.0 * p : 3.0 * p;
    double cu = EX[i] * u[0] + EY[i] * u[1] + EZ[i] * u[2];
    feq[i] = WT[i] * Ai + WT[i] * n * (3.0 * cu - 1.5 * u2 + 4.5 * cu * cu);
  }
}

/* D3Q7 equilibrium (moment-matched Eq. 9-10), directions 0..6 of the table. */
void orc3_geq(double phi, double mu, const double* u, double gamma, double q, double* geq) {
  for (int i = 0; i < 7; i++) {
    double Ai = i == 0 ? -3.0 * gamma * mu : 0.5 * gamma * mu;
    double Bi = i == 0 ? 1.0 : 0.0;
    double cu = EX[i] * u[0] + EY[i] * u[1] + EZ[i] * u[2];
    geq[i] = Ai + Bi * phi + phi * cu / (2.0 * q);
  }
}

/* Eq. 4 forcing term on D3Q19. */
void orc3_force_term(double tau, const double* u, const double* F, double* Fi) {
  init_tables();
  for (int i = 0; i < 19; i++) {
    double cu = EX[i] * u[0] + EY[i] * u[1] + EZ[i] * u[2];
    double c[3] = {(double)EX[i], (double)EY[i], (double)EZ[i]};
    double v = 0.0;
    for (int a = 0; a < 3; a++) v += ((c[a] - u[a]) + 3.0 * cu * c[a]) * F[a];
    Fi[i] = (1.0 - 1.0 / (2.0 * tau)) * 3.0 * WT[i] * v;
  }
}

void orc3_lattice(int* ex, int* ey, int* ez, double* w) {
  init_tables();
  for (int i = 0; i < 19; i++) {
    ex[i] = EX[i];
    ey[i] = EY[i];
    ez[i] = EZ[i];
    w[i] = WT[i];
  }
}

/* ---------------------------------------------------------------------- */
static double radius2(const orc3* s, int x, int y) {
  double dx = x - s->cx, dy = y - s->cy;
  return dx * dx + dy * dy;
}

static int in_channel(const orc3* s, int x, int y) { return radius2(s, x, y) < s->R * s->R; }

static int geom_kind(const orc3* s, int x, int y, int z) {
  const orc_params* p = &s->p;
  if (p->geometry == ORC_GEOM_NOZZLE) {
    double r2 = radius2(s, x, y), Ro = s->R + p->wall_thickness;
    if (z < p->nozzle_length && r2 >= s->R * s->R && r2 < Ro * Ro) {
      const int fx[4] = {1, -1, 0, 0}, fy[4] = {0, 0, 1, -1};
      for (int d = 0; d < 4; d++)
        if (in_channel(s, wrap(x + fx[d], s->nx), wrap(y + fy[d], s->ny))) return 2;
      return 1;
    }
    return 0;
  }
  if (p->geometry == ORC_GEOM_PLATE) {
    if (z < p->wall_thickness) return z == p->wall_thickness - 1 ? 2 : 1;
    return 0;
  }
  return 0;
}

static int map_z(const orc3* s, int z, int* zm) {
  if (z >= 0 && z < s->nz) {
    *zm = z;
    return 1;
  }
  if (s->p.axial_bc == ORC_BC_PERIODIC) {
    *zm = wrap(z, s->nz);
    return 1;
  }
  if (s->p.axial_bc == ORC_BC_ZERO_GRADIENT) {
    *zm = z < 0 ? 0 : s->nz - 1;
    return 1;
  }
  return 0;
}

static size_t cidx(const orc3* s, int x, int y, int z) {
  return ((size_t)z * s->ny + y) * s->nx + x;
}

static int kind_at(const orc3* s, int x, int y, int z) {
  int zm;
  if (!map_z(s, z, &zm)) return 1;
  return s->kind[cidx(s, wrap(x, s->nx), wrap(y, s->ny), zm)];
}

static double phi_fluid_at(const orc3* s, int x, int y, int z) {
  int zm;
  map_z(s, z, &zm);
  return s->phi[cidx(s, wrap(x, s->nx), wrap(y, s->ny), zm)];
}

/* Ghost phi of a solid point: mean over fluid face neighbours of
 * phi + h_s / kappa, else the plain mean over fluid edge neighbours. */
static double ghost_value(const orc3* s, int x, int y, int z) {
  int k = kind_at(s, x, y, z);
  double hk = k == 2 ? s->h / s->kappa : 0.0, sum = 0.0;
  int cnt = 0;
  for (int i = 1; i <= 6; i++)
    if (kind_at(s, x + EX[i], y + EY[i], z + EZ[i]) == 0) {
      sum += phi_fluid_at(s, x + EX[i], y + EY[i], z + EZ[i]) + hk;
      cnt++;
    }
  if (cnt) return sum / cnt;
  for (int i = 7; i < 19; i++)
    if (kind_at(s, x + EX[i], y + EY[i], z + EZ[i]) == 0) {
      sum += phi_fluid_at(s, x + EX[i], y + EY[i], z + EZ[i]);
      cnt++;
    }
  return cnt ? sum / cnt : 0.0;
}

static double* phih_ptr(orc3* s, int x, int y, int z) {
  return s->phih + ((size_t)(z + 2) * s->ny + wrap(y, s->ny)) * s->nx + wrap(x, s->nx);
}

static void fill_phih(orc3* s) {
#pragma omp parallel for schedule(static)
  for (int z = -2; z < s->nz + 2; z++)
    for (int y = 0; y < s->ny; y++)
      for (int x = 0; x < s->nx; x++)
        *phih_ptr(s, x, y, z) = kind_at(s, x, y, z) == 0 ? phi_fluid_at(s, x, y, z) : ghost_value(s, x, y, z);
}

static int drive_region(const orc3* s, int x, int y, int z) {
  if (s->p.geometry == ORC_GEOM_NOZZLE) return z < s->p.nozzle_length && in_channel(s, x, y);
  return 1;
}

static double drive_at(const orc_params* p, long long t) {
  long long tt = t;
  if (p->T_idle > 0) tt = t % (p->T1 + p->T2 + p->T_idle);
  if (tt < p->T1) return p->F0;
  if (tt < p->T1 + p->T2) return -p->F_neg;
  return 0.0;
}

/* SplitMix64 (Steele, Lea & Flood 2014). */
static uint64_t splitmix64(uint64_t z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* Uniform [0, 1) of (seed, x, y, z): splitmix64(seed ^ splitmix64(counter)),
 * counter = z << 42 ^ y << 21 ^ x. */
static double uniform3(unsigned long long seed, int x, int y, int z) {
  uint64_t c = ((uint64_t)(uint32_t)z << 42) ^ ((uint64_t)(uint32_t)y << 21) ^ (uint64_t)(uint32_t)x;
  return (double)(splitmix64((uint64_t)seed ^ splitmix64(c)) >> 11) * (1.0 / 9007199254740992.0);
}

double orc3_uniform(unsigned long long seed, int x, int y, int z) { return uniform3(seed, x, y, z); }

/* ---------------------------------------------------------------------- */
static void chem_and_velocity(orc3* s, long long t) {
  int nx = s->nx, ny = s->ny, nz = s->nz;
  double Fd = drive_at(&s->p, t);
#pragma omp parallel for schedule(static)
  for (int z = -1; z <= nz; z++) {
    int zm;
    if (!map_z(s, z, &zm)) continue;
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        size_t c = cidx(s, x, y, zm), e = ((size_t)(z + 1) * ny + y) * nx + x;
        if (s->kind[c] != 0) continue;
        double p0 = s->phi[c], lap = 0.0, g[3] = {0, 0, 0};
        for (int i = 1; i < 19; i++) {
          double pn = *phih_ptr(s, x + EX[i], y + EY[i], z + EZ[i]);
          lap += 6.0 * WT[i] * (pn - p0);
          g[0] += 3.0 * WT[i] * EX[i] * pn;
          g[1] += 3.0 * WT[i] * EY[i] * pn;
          g[2] += 3.0 * WT[i] * EZ[i] * pn;
        }
        double mu = 4.0 * s->A * p0 * (p0 * p0 - s->phis * s->phis) - s->kappa * lap;
        double C = 0.5 * (p0 / s->phis + 1.0);
        C = C < 0 ? 0 : (C > 1 ? 1 : C);
        double Fb = drive_region(s, x, y, zm) ? Fd * C : 0.0;
        s->mu[e] = mu;
        s->dpx[e] = g[0];
        s->dpy[e] = g[1];
        s->dpz[e] = g[2];
        s->C[e] = C;
        s->Fz[e] = mu * g[2] + Fb;
        s->ux[e] = (s->mx[c] + 0.5 * mu * g[0]) / s->n[c];
        s->uy[e] = (s->my[c] + 0.5 * mu * g[1]) / s->n[c];
        s->uz[e] = (s->mz[c] + 0.5 * s->Fz[e]) / s->n[c];
      }
  }
}

#define NECK_BREAK3 0.01

static void diagnose(orc3* s, long long t) {
  int nx = s->nx, ny = s->ny, nz = s->nz;
  double mass_n = 0, mass_phi = 0, mom = 0;
  for (int z = 0; z < nz; z++) {
    double w = 0, m = 0, pr = 0;
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        size_t c = cidx(s, x, y, z), e = ((size_t)(z + 1) * ny + y) * nx + x;
        if (s->kind[c] != 0) continue;
        double ev = s->phi[c] / s->phis;
        ev = ev < 0 ? 0 : (ev > 1 ? 1 : ev);
        w += ev;
        m += ev * s->n[c];
        pr += ev * s->n[c] * s->uz[e];
        mass_n += s->n[c];
        mass_phi += s->phi[c];
        mom += s->n[c] * s->uz[e];
      }
    s->wrow[z] = w;
    s->mrow[z] = m;
    s->prow[z] = pr;
  }
  int nozzle = s->p.geometry == ORC_GEOM_NOZZLE;
  int L = s->p.nozzle_length;
  int z_exit = nozzle ? L : 0, z_scan = nozzle ? L - L / 2 : 0;
  double vmin = nozzle ? M_PI * s->R * s->R : 1.0;
  double neck = 1e30, above = 0.0;
  for (int z = nz - 1; z >= 0; z--) {
    if (z >= z_scan && above > vmin && s->wrow[z] < neck) neck = s->wrow[z];
    if (s->wrow[z] > 0.5) above += s->wrow[z];
  }
  if (s->breakup < 0 && neck < NECK_BREAK3) {
    if (s->have_prev && s->m_prev >= NECK_BREAK3 && s->m_prev < 1e29)
      s->breakup = s->t_prev + (t - s->t_prev) * (s->m_prev - NECK_BREAK3) / (s->m_prev - neck);
    else
      s->breakup = (double)t;
  }
  s->have_prev = 1;
  s->m_prev = neck;
  s->t_prev = (double)t;
  int nruns = 0, nabove = 0, lead0 = -1, lead1 = -1;
  for (int z = 0; z < nz;) {
    if (s->wrow[z] > 0.5) {
      int z0 = z;
      while (z < nz && s->wrow[z] > 0.5) z++;
      nruns++;
      if (z0 >= z_exit) nabove++;
      lead0 = z0;
      lead1 = z;
    } else {
      z++;
    }
  }
  double vol = 0, zc = 0, mm = 0, pp = 0;
  for (int z = lead0; lead0 >= 0 && z < lead1; z++) {
    vol += s->wrow[z];
    zc += z * s->wrow[z];
    mm += s->mrow[z];
    pp += s->prow[z];
  }
  double rec[ORC_REC] = {0};
  rec[0] = (double)t;
  rec[1] = mass_n;
  rec[2] = mass_phi;
  rec[3] = mom;
  rec[4] = neck;
  rec[5] = s->breakup;
  rec[6] = vol;
  rec[7] = vol > 0 ? zc / vol : 0.0;
  rec[8] = mm > 0 ? pp / mm : 0.0;
  rec[9] = nabove > 1 ? nabove - 1 : 0;
  rec[10] = nruns;
  /* head and tail of the leading droplet along z, as in the 2-D oracle */
  rec[11] = rec[12] = -1.0;
  if (lead0 >= 0) {
    int top = lead1 - 1;
    rec[11] = lead1 < nz ? top + (s->wrow[top] - 0.5) / (s->wrow[top] - s->wrow[lead1]) : top;
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

static void moments(orc3* s) {
  size_t N = (size_t)s->nx * s->ny * s->nz;
#pragma omp parallel for schedule(static)
  for (size_t c = 0; c < N; c++) {
    if (s->kind[c] != 0) continue;
    double n = 0, m[3] = {0, 0, 0}, phi = 0;
    for (int i = 0; i < 19; i++) {
      double fi = s->f[i * N + c];
      n += fi;
      m[0] += fi * EX[i];
      m[1] += fi * EY[i];
      m[2] += fi * EZ[i];
    }
    for (int i = 0; i < 7; i++) phi += s->g[i * N + c];
    s->n[c] = n;
    s->mx[c] = m[0];
    s->my[c] = m[1];
    s->mz[c] = m[2];
    s->phi[c] = phi;
  }
}

static void collide(orc3* s) {
  int nx = s->nx, ny = s->ny, nz = s->nz;
  size_t N = (size_t)nx * ny * nz, NM = (size_t)nx * ny * (nz + 2);
  const orc_params* p = &s->p;
#pragma omp parallel for schedule(static)
  for (int z = -1; z <= nz; z++) {
    int zm;
    if (!map_z(s, z, &zm)) continue;
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        size_t c = cidx(s, x, y, zm), e = ((size_t)(z + 1) * ny + y) * nx + x;
        if (s->kind[c] != 0) continue;
        double C = s->C[e], tau = 0.5 + 3.0 * (p->nu_air + C * (p->nu_ink - p->nu_air));
        double u[3] = {s->ux[e], s->uy[e], s->uz[e]};
        double F[3] = {s->mu[e] * s->dpx[e], s->mu[e] * s->dpy[e], s->Fz[e]};
        double fe[19], Fi[19], ge[7];
        orc3_feq(s->n[c], s->phi[c], s->mu[e], u, fe);
        orc3_force_term(tau, u, F, Fi);
        for (int i = 0; i < 19; i++) {
          double fi = s->f[i * N + c];
          s->fs[i * NM + e] = fi + (fe[i] - fi) / tau + Fi[i];
        }
        orc3_geq(s->phi[c], s->mu[e], u, s->gamma, s->q, ge);
        int inside = z >= 0 && z < nz;
        for (int i = 0; i < 7; i++) {
          double gi = s->g[i * N + c], om = (ge[i] - gi) / p->tau_phi;
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

static void stream(orc3* s) {
  int nx = s->nx, ny = s->ny, nz = s->nz;
  size_t N = (size_t)nx * ny * nz, NM = (size_t)nx * ny * (nz + 2);
#pragma omp parallel for schedule(static)
  for (int z = 0; z < nz; z++)
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        size_t c = cidx(s, x, y, z), e = ((size_t)(z + 1) * ny + y) * nx + x;
        if (s->kind[c] != 0) {
          for (int i = 0; i < 19; i++) s->fn[i * N + c] = s->f[i * N + c];
          for (int i = 0; i < 7; i++) s->gn[i * N + c] = s->g[i * N + c];
          continue;
        }
        s->fn[c] = s->fs[e];
        for (int i = 1; i < 19; i++) {
          int xs = x - EX[i], ys = y - EY[i], zs = z - EZ[i];
          if (kind_at(s, xs, ys, zs) != 0)
            s->fn[i * N + c] = s->fs[OPP[i] * NM + e];
          else
            s->fn[i * N + c] = s->fs[i * NM + ((size_t)(zs + 1) * ny + wrap(ys, ny)) * nx + wrap(xs, nx)];
        }
        s->gn[c] = s->S[c];
        for (int i = 1; i < 7; i++) {
          int xs = x - EX[i], ys = y - EY[i], zs = z - EZ[i];
          double moving = kind_at(s, xs, ys, zs) != 0
                              ? s->P[OPP[i] * NM + e]
                              : s->P[i * NM + ((size_t)(zs + 1) * ny + wrap(ys, ny)) * nx + wrap(xs, nx)];
          s->gn[i * N + c] = s->S[i * N + c] + moving;
        }
      }
  double *t1 = s->f, *t2 = s->g;
  s->f = s->fn;
  s->fn = t1;
  s->g = s->gn;
  s->gn = t2;
}

static void step_once(orc3* s) {
  moments(s);
  fill_phih(s);
  chem_and_velocity(s, s->t);
  if (s->p.diag_every > 0 && s->t % s->p.diag_every == 0) diagnose(s, s->t);
  collide(s);
  stream(s);
  s->t++;
}

/* ---------------------------------------------------------------------- */
void* orc3_create(const orc_params* p) {
  const int nz = p->nz;
  if (p->nx < 1 || p->ny < 1 || nz < 1) return NULL;
  init_tables();
  orc3* s = calloc(1, sizeof(orc3));
  s->p = *p;
  s->nx = p->nx;
  s->ny = p->ny;
  s->nz = nz;
  size_t N = (size_t)s->nx * s->ny * nz, NM = (size_t)s->nx * s->ny * (nz + 2),
         NH = (size_t)s->nx * s->ny * (nz + 4);
  s->phis = 0.5 * (p->rho_ink - p->rho_air);
  s->n0 = 0.5 * (p->rho_ink + p->rho_air);
  s->A = 3.0 * p->sigma / (8.0 * p->width_W * pow(s->phis, 4));
  s->kappa = 3.0 * p->sigma * p->width_W / (4.0 * s->phis * s->phis);
  s->q = 1.0 / (p->tau_phi + 0.5);
  s->gamma = p->gamma > 0 ? p->gamma : 0.04 / s->kappa;
  s->Omega = orc_omega_of_theta(p->theta_deg);
  s->h = s->Omega * s->phis * s->phis * sqrt(2.0 * s->kappa * s->A);
  s->cx = 0.5 * (s->nx - 1);
  s->cy = 0.5 * (s->ny - 1);
  s->R = p->nozzle_width;  /* in 3-D the nozzle_width field holds the radius */
  s->f = calloc(19 * N, sizeof(double));
  s->g = calloc(7 * N, sizeof(double));
  s->fn = calloc(19 * N, sizeof(double));
  s->gn = calloc(7 * N, sizeof(double));
  double** a[] = {&s->n, &s->phi, &s->mx, &s->my, &s->mz};
  for (int k = 0; k < 5; k++) *a[k] = calloc(N, sizeof(double));
  double** b[] = {&s->mu, &s->dpx, &s->dpy, &s->dpz, &s->ux, &s->uy, &s->uz, &s->C, &s->Fz};
  for (int k = 0; k < 9; k++) *b[k] = calloc(NM, sizeof(double));
  s->phih = calloc(NH, sizeof(double));
  s->fs = calloc(19 * NM, sizeof(double));
  s->P = calloc(7 * NM, sizeof(double));
  s->S = calloc(7 * N, sizeof(double));
  s->kind = calloc(N, 1);
  s->wrow = calloc(nz, sizeof(double));
  s->mrow = calloc(nz, sizeof(double));
  s->prow = calloc(nz, sizeof(double));
  s->caphist = 64;
  s->hist = calloc((size_t)s->caphist * ORC_REC, sizeof(double));
  s->breakup = -1.0;
  for (int z = 0; z < nz; z++)
    for (int y = 0; y < s->ny; y++)
      for (int x = 0; x < s->nx; x++) s->kind[cidx(s, x, y, z)] = (unsigned char)geom_kind(s, x, y, z);
  int L = p->nozzle_length;
  for (int z = 0; z < nz; z++)
    for (int y = 0; y < s->ny; y++)
      for (int x = 0; x < s->nx; x++) {
        size_t c = cidx(s, x, y, z);
        double v = 0.0;
        if (s->kind[c] == 0) {
          if (p->init_kind == ORC_INIT_MENISCUS) {
            double r = sqrt(radius2(s, x, y));
            if (r < s->R) {
              v = s->phis * tanh((L - z) / p->width_W);
              if (fabs((double)(z - L)) < 2.0 * p->width_W)
                v += p->jitter * (2.0 * uniform3(p->seed, x, y, z) - 1.0);
            } else if (z < L) {
              v = -s->phis;
            } else {
              double dr = r - s->R, dz = (double)(z - L);
              v = s->phis * tanh(-sqrt(dr * dr + dz * dz) / p->width_W);
            }
          } else if (p->init_kind == ORC_INIT_DROP) {
            double dx = x - p->init_x, dy = y - p->init_y, dz = z - p->init_z;
            dx -= s->nx * floor(dx / s->nx + 0.5);
            dy -= s->ny * floor(dy / s->ny + 0.5);
            v = s->phis * tanh((p->init_r - sqrt(dx * dx + dy * dy + dz * dz)) / p->width_W);
          } else if (p->init_kind == ORC_INIT_FLAT) {
            v = s->phis * tanh((p->init_y - z) / p->width_W);
          } else {
            v = p->init_r;
          }
        }
        s->phi[c] = v;
      }
  fill_phih(s);
  for (int z = 0; z < nz; z++)
    for (int y = 0; y < s->ny; y++)
      for (int x = 0; x < s->nx; x++) {
        size_t c = cidx(s, x, y, z);
        if (s->kind[c] != 0) continue;
        double p0 = s->phi[c], lap = 0.0;
        for (int i = 1; i < 19; i++) lap += 6.0 * WT[i] * (*phih_ptr(s, x + EX[i], y + EY[i], z + EZ[i]) - p0);
        double mu = 4.0 * s->A * p0 * (p0 * p0 - s->phis * s->phis) - s->kappa * lap;
        double u[3] = {0, 0, 0}, fe[19], ge[7];
        orc3_feq(s->n0, p0, mu, u, fe);
        orc3_geq(p0, mu, u, s->gamma, s->q, ge);
        for (int i = 0; i < 19; i++) s->f[i * N + c] = fe[i];
        for (int i = 0; i < 7; i++) s->g[i * N + c] = ge[i];
      }
  return s;
}

void orc3_destroy(void* h) {
  orc3* s = h;
  if (!s) return;
  double* a[] = {s->f, s->g, s->fn, s->gn, s->n, s->phi, s->mx, s->my, s->mz, s->phih, s->mu,
                 s->dpx, s->dpy, s->dpz, s->ux, s->uy, s->uz, s->C, s->Fz, s->fs, s->P, s->S,
                 s->wrow, s->mrow, s->prow, s->hist};
  for (size_t k = 0; k < sizeof(a) / sizeof(a[0]); k++) free(a[k]);
  free(s->kind);
  free(s);
}

void orc3_step(void* h, long long nsteps) {
  for (long long k = 0; k < nsteps; k++) step_once((orc3*)h);
}

long long orc3_time(const void* h) { return ((const orc3*)h)->t; }

void orc3_get_state(const void* h, double* f, double* g) {
  const orc3* s = h;
  size_t N = (size_t)s->nx * s->ny * s->nz;
  memcpy(f, s->f, 19 * N * sizeof(double));
  memcpy(g, s->g, 7 * N * sizeof(double));
}

void orc3_set_state(void* h, const double* f, const double* g, long long t) {
  orc3* s = h;
  size_t N = (size_t)s->nx * s->ny * s->nz;
  memcpy(s->f, f, 19 * N * sizeof(double));
  memcpy(s->g, g, 7 * N * sizeof(double));
  s->t = t;
}

void orc3_kinds(const void* h, unsigned char* out) {
  const orc3* s = h;
  memcpy(out, s->kind, (size_t)s->nx * s->ny * s->nz);
}

int orc3_history(const void* h, double* out, int max_records) {
  const orc3* s = h;
  int n = s->nhist < max_records ? s->nhist : max_records;
  if (out && n > 0) memcpy(out, s->hist, (size_t)n * ORC_REC * sizeof(double));
  return s->nhist;
}

/* Streaming with identity collision (q = 1), for the permutation test. */
void orc3_stream_only(void* h, const double* fin, const double* gin, double* fout, double* gout) {
  orc3* s = h;
  int nx = s->nx, ny = s->ny, nz = s->nz;
  size_t N = (size_t)nx * ny * nz, NM = (size_t)nx * ny * (nz + 2);
  for (int z = -1; z <= nz; z++) {
    int zm;
    if (!map_z(s, z, &zm)) continue;
    for (int y = 0; y < ny; y++)
      for (int x = 0; x < nx; x++) {
        size_t c = cidx(s, x, y, zm), e = ((size_t)(z + 1) * ny + y) * nx + x;
        for (int i = 0; i < 19; i++) s->fs[i * NM + e] = fin[i * N + c];
        for (int i = 1; i < 7; i++) s->P[i * NM + e] = gin[i * N + c];
        if (z >= 0 && z < nz) {
          s->S[c] = gin[c];
          for (int i = 1; i < 7; i++) s->S[i * N + c] = 0.0;
        }
      }
  }
  double *f0 = s->f, *g0 = s->g, *fn0 = s->fn, *gn0 = s->gn;
  s->f = (double*)fin;
  s->g = (double*)gin;
  s->fn = fout;
  s->gn = gout;
  stream(s);
  s->f = f0;
  s->g = g0;
  s->fn = fn0;
  s->gn = gn0;
}
