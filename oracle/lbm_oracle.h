/*
 * FP64 CPU oracle for the binary-fluid lattice Boltzmann inkjet model of
 * He, Yang, Qin, Wen & Zhang, "The roles of wettability and surface tension
 * in droplet formation during inkjet printing" (arXiv:1702.04487).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct
 * reference that the CUDA path is checked against.  Only the test suite,
 * the smoke check and the benchmark's CPU-baseline leg may load it; the
 * product path never does.  It shares no code, header, table or helper with
 * the CUDA library.
 *
 * Every quantity is in lattice units.  Lattice layout of every field is
 * structure-of-arrays: f[i][y][x] (i = 0..8, D2Q9) and g[i][y][x]
 * (i = 0..4, D2Q5), x fastest.  x is the lateral, periodic axis; y is the
 * nozzle axis (ejection towards +y).
 */
#ifndef LBM_ORACLE_H
#define LBM_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* geometry kinds */
#define ORC_GEOM_NONE 0   /* no solid cells */
#define ORC_GEOM_NOZZLE 1 /* planar nozzle: channel with two walls, 0 <= y < L */
#define ORC_GEOM_PLATE 2  /* flat wetting plate along the bottom, 0 <= y < t */

/* axial (y) boundary handling */
#define ORC_BC_ZERO_GRADIENT 0 /* "fully developed": outside rows replicate edge rows */
#define ORC_BC_PERIODIC 1
#define ORC_BC_CLOSED 2 /* rows -1 and ny are non-wetting solid walls */

/* initial order-parameter field */
#define ORC_INIT_MENISCUS 0 /* ink fills the nozzle channel, flat diffuse meniscus at y = L */
#define ORC_INIT_DROP 1     /* circular ink drop (init_x, init_y, radius init_r) in air */
#define ORC_INIT_FLAT 2     /* ink below y = init_y, air above, full width */
#define ORC_INIT_UNIFORM 3  /* phi = init_r everywhere (single phase when +-phi*) */

typedef struct {
  int nx, ny;
  int geometry;
  int nozzle_width, nozzle_length, wall_thickness;
  double rho_ink, rho_air; /* phi* = (rho_ink-rho_air)/2, n0 = (rho_ink+rho_air)/2 */
  double nu_ink, nu_air;   /* kinematic viscosities of the two fluids */
  double sigma, width_W;   /* surface tension and interface width */
  double tau_phi, gamma;   /* relaxation time of g and mobility coefficient Gamma */
  double theta_deg;        /* contact angle of the wetting wall faces */
  double F0, F_neg;        /* drive: +F0, then -F_neg, then idle */
  long long T1, T2, T_idle;
  int axial_bc;
  int init_kind;
  double init_x, init_y, init_r;
  double jitter;
  unsigned long long seed;
  int diag_every;
  int nz;        /* 3-D only: lattice depth along the nozzle axis z */
  double init_z; /* 3-D only: drop centre z */
} orc_params;

typedef struct orc_sim orc_sim;

/* number of doubles in one diagnostics record */
#define ORC_REC 13

orc_sim* orc_create(const orc_params* p);
void orc_destroy(orc_sim* s);
void orc_step(orc_sim* s, long long nsteps);
long long orc_time(const orc_sim* s);
void orc_get_state(const orc_sim* s, double* f, double* g);
void orc_set_state(orc_sim* s, const double* f, const double* g, long long t);
/* out: phi*, n0, A, kappa, q, h, Gamma, Omega */
void orc_derived(const orc_sim* s, double* out);
/* Macroscopic fields of the current state: n, phi, mu, ux, uy (each ny*nx). */
void orc_fields(orc_sim* s, double* n, double* phi, double* mu, double* ux, double* uy);
/* Diagnostics records produced so far (ORC_REC doubles each). */
int orc_history(const orc_sim* s, double* out, int max_records);
/* Cell kinds: 0 fluid, 1 solid, 2 solid on a wetting face. */
void orc_kinds(const orc_sim* s, unsigned char* out);
/* Streaming with boundary rules alone (identity collision, q = 1). */
void orc_stream_only(orc_sim* s, const double* fin, const double* gin, double* fout, double* gout);

/* 3-D lift (lbm3d_oracle.c): D3Q19 / D3Q7, z the nozzle axis; the nozzle
 * radius is nozzle_width.  Same conventions as the 2-D calls above. */
void* orc3_create(const orc_params* p);
void orc3_destroy(void* s);
void orc3_step(void* s, long long nsteps);
long long orc3_time(const void* s);
void orc3_get_state(const void* s, double* f, double* g);
void orc3_set_state(void* s, const double* f, const double* g, long long t);
void orc3_kinds(const void* s, unsigned char* out);
int orc3_history(const void* s, double* out, int max_records);
void orc3_stream_only(void* s, const double* fin, const double* gin, double* fout, double* gout);
void orc3_feq(double n, double phi, double mu, const double* u, double* feq19);
void orc3_geq(double phi, double mu, const double* u, double gamma, double q, double* geq7);
void orc3_force_term(double tau, const double* u, const double* F, double* F19);
void orc3_lattice(int* ex, int* ey, int* ez, double* w);
double orc3_uniform(unsigned long long seed, int x, int y, int z);

/* Per-cell building blocks, exposed for the closed-form tests. */
void orc_feq(double n, double phi, double mu, double ux, double uy, double* feq9);
void orc_geq(double phi, double mu, double ux, double uy, double gamma, double q, double* geq5);
void orc_force_term(double tau, double ux, double uy, double Fx, double Fy, double* F9);
double orc_omega_of_theta(double theta_deg);
double orc_uniform(unsigned long long seed, int x, int y);
/* Threads of the per-cell passes (OpenMP; 1 when built without it).  Every
 * result is bit-identical on any number of threads. */
int orc_threads(void);
void orc_set_threads(int n);

#ifdef __cplusplus
}
#endif
#endif
