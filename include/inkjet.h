/*
 * inkjet.h -- C ABI of libinkjet.so, a GB300 (sm_103a) implementation of the
 * binary-fluid lattice Boltzmann inkjet model of He, Yang, Qin, Wen & Zhang,
 * "The roles of wettability and surface tension in droplet formation during
 * inkjet printing" (arXiv:1702.04487).
 *
 * The library advances one or more 2-D lattices of the Zheng-Shu-Chew
 * binary-fluid model (Eq. 1-10, "Methods"): a D2Q9 population f for the mean
 * density n and momentum, a D2Q5 population g for the order parameter phi,
 * driven by the time-dependent positive/negative/idle body force of Fig. 1
 * inside a planar nozzle whose inner wall carries a contact angle ("wetting
 * boundary condition", Sect. "Reproducing the experiment").
 *
 * 3-D lattices (dim = 3) lift the same model to D3Q19 (f) and D3Q7 (g) by
 * matching the moments of Eq. 5-6 and 9-10; the nozzle is round and its axis
 * is z.  Their populations are f[i][z][y][x] (i = 0..18) and g[i][z][y][x]
 * (i = 0..6): rest, +x, -x, +y, -y, +z, -z, then the 12 edge directions
 * (+x+y, -x+y, +x-y, -x-y, +x+z, -x+z, +x-z, -x-z, +y+z, -y+z, +y-z, -y-z).
 * Each step is one fused launch over every lattice of the handle (a CTA per
 * 28 x 12 column tile and z chunk marches up z, streaming in push form),
 * then the wetting ghosts of the new phi; the state is double-buffered per
 * lattice, and a lattice frozen by a numeric failure keeps its last good
 * state.  All 3-D lattices of a handle share the storage format (FP16
 * storage needs an even nx).  The diagnostics below run over z planes
 * (w(z) = sum over x, y of e; mom_y is the sum of n u_z; the neck criterion
 * needs more than pi R^2 of run ink above).  All lattices of a handle have
 * the same dim.
 *
 * Conventions for every entry point:
 *  - All quantities are lattice units (delta x = delta t = 1).
 *  - Every call returns an ij_status and never aborts the process.
 *  - Population layout is structure-of-arrays, x fastest: f[i][y][x] with
 *    i = 0..8 (rest, +x, +y, -x, -y, +x+y, -x+y, -x-y, +x-y) and g[i][y][x]
 *    with i = 0..4 (the first five of those).  x is the lateral, periodic
 *    axis (width nx); y is the nozzle axis (height ny), ejection along +y.
 *  - Device state is owned by the handle; caller buffers are owned by the
 *    caller and only read or written during the call (or, for *_on_device
 *    buffers, by work the call enqueues on the handle's stream).
 *  - Work is enqueued on the CUDA stream given at creation; calls that
 *    return results to the host synchronise that stream.
 *  - Numeric failures are per lattice: a lattice whose step met NaN or
 *    |u| > 0.3 (Mach limit of the lattice) is frozen and reported by
 *    ij_observe; the other lattices of a batch keep stepping.  Once every
 *    lattice of a handle is frozen, ij_step returns IJ_ERR_NUMERIC.
 */
#ifndef INKJET_H
#define INKJET_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ij_handle_s* ij_handle;

typedef enum {
  IJ_OK = 0,
  IJ_ERR_PARAM = 1,   /* invalid argument; nothing was changed */
  IJ_ERR_CUDA = 2,    /* a CUDA call failed; see ij_last_error */
  IJ_ERR_NUMERIC = 3, /* NaN or |u| > 0.3 met in a step of a lattice */
  IJ_ERR_TIMEOUT = 4, /* a bounded wait inside a kernel ran out (the surrogate's
                         tensor-core pipeline); the LBM step kernels never wait */
  IJ_ERR_STATE = 5,   /* call not allowed in the handle's state */
  IJ_ERR_OOM = 6      /* the allocator returned NULL */
} ij_status;

/* geometry */
#define IJ_GEOM_NONE 0   /* no solid cells */
#define IJ_GEOM_NOZZLE 1 /* planar nozzle: channel [cx0, cx0+w), walls of thickness t
                            on both sides for 0 <= y < L, cx0 = (nx - w) / 2; the
                            channel-facing wall faces carry the contact angle */
#define IJ_GEOM_PLATE 2  /* solid rows 0 <= y < t; their top face carries the angle */

/* axial (y) ends */
#define IJ_BC_ZERO_GRADIENT 0 /* "fully developed": outside rows replicate the edge row */
#define IJ_BC_PERIODIC 1
#define IJ_BC_CLOSED 2        /* non-wetting solid rows at y = -1 and y = ny */

/* initial order parameter (n = n0, u = 0, f = f^(0), g = g^(0) everywhere) */
#define IJ_INIT_MENISCUS 0 /* ink fills the nozzle, flat diffuse meniscus at y = L */
#define IJ_INIT_DROP 1     /* ink drop of radius init_r at (init_x, init_y) */
#define IJ_INIT_FLAT 2     /* ink below y = init_y */
#define IJ_INIT_UNIFORM 3  /* phi = init_r everywhere */

/* population storage */
#define IJ_FP32 0        /* f as FP32 deviations f_i - w_i n0, g as FP32 */
#define IJ_FP16_STORE 1  /* f deviations and g_1.. in FP16, g_0 in FP32; every
                            update is computed in FP32.  2-D: nx must be even, and
                            all lattices of one handle share the precision */

typedef struct {
  int nx, ny;                 /* lattice size, nx, ny >= 1 */
  int geometry;               /* IJ_GEOM_* */
  int nozzle_width, nozzle_length, wall_thickness;
  double rho_ink, rho_air;    /* phi* = (rho_ink - rho_air)/2, n0 = (rho_ink + rho_air)/2 */
  double nu_ink, nu_air;      /* kinematic viscosities; tau_n = 1/2 + 3 nu(C) */
  double sigma, width_W;      /* surface tension and interface width (W = 3 in the paper) */
  double tau_phi, gamma;      /* relaxation time of g (0.8 in the paper) and mobility
                                 coefficient Gamma; gamma <= 0 selects 0.04 / kappa */
  double theta_deg;           /* contact angle of the wetting wall faces, degrees */
  double F0, F_neg;           /* drive: +F0 for T1 steps, -F_neg for T2 steps, then idle */
  long long T1, T2, T_idle;   /* T_idle > 0 repeats the waveform with period T1+T2+T_idle */
  int axial_bc;               /* IJ_BC_* */
  int init_kind;              /* IJ_INIT_* */
  double init_x, init_y, init_r;
  double jitter;              /* amplitude of the meniscus jitter (SplitMix64 of seed, x, y) */
  unsigned long long seed;
  int diag_every;             /* steps between diagnostics records (0: none) */
  int precision;              /* IJ_FP32 | IJ_FP16_STORE */
  int dim;                    /* 2 (D2Q9/D2Q5) or 3 (D3Q19/D3Q7); 0 means 2 */
  int nz;                     /* 3-D: lattice depth along the nozzle axis z (then the
                                 axis is z, x and y periodic, nozzle_width is the radius
                                 of a round nozzle centred at ((nx-1)/2, (ny-1)/2)) */
  double init_z;              /* 3-D: drop centre z for IJ_INIT_DROP */
} ij_params;

/* One diagnostics record, evaluated on the state at time `step` (before
 * that step's update), in FP64.  Ink weight e = clamp(phi / phi*, 0, 1); row
 * integrals w(y) = sum_x e; runs are row ranges with w > 1/2.  The neck is the
 * least w(y) over rows y >= L/2 with more than nozzle_width of run ink above;
 * breakup is the first record whose neck drops below 0.01, its time
 * interpolated linearly between records.  The leading droplet is the highest
 * run. */
typedef struct {
  double step;
  double mass_n, mass_phi;   /* sum of n and phi over fluid cells */
  double mom_y;              /* sum of n u_y over fluid cells */
  double neck;
  double breakup_step;       /* -1 until breakup */
  double droplet_volume;     /* sum of e over the leading run */
  double droplet_centroid_y;
  double droplet_velocity;   /* e n-weighted mean u_y over the leading run */
  double satellites;         /* runs starting at or above y = L, minus one */
  double runs;
  double head_y, tail_y;     /* where w crosses 1/2 at the upper / lower end of the
                                leading run, interpolated between rows (-1: no run);
                                head and tail velocities are their differences
                                between records */
} ij_obs;

/* Device-memory allocator callbacks; NULL selects cudaMalloc / cudaFree. */
typedef void* (*ij_alloc_fn)(size_t bytes, void* ctx);
typedef void (*ij_free_fn)(void* ptr, void* ctx);

/*
 * ij_create -- build `count` independent lattices (a batch) and initialise
 * them (n = n0, u = 0, phi from init_kind, mu from phi with the wetting
 * ghosts, f = f^(0) of Eq. 5-6, g = g^(0) of Eq. 9-10).
 *   params   : array of `count` parameter blocks (host memory, read only).
 *   count    : 1 .. 65536.  Lattices may differ in every parameter.
 *   alloc/free/ctx : device allocator (both NULL or both set).
 *   stream   : cudaStream_t to enqueue on (NULL: legacy default stream).
 *   out      : receives the handle.
 * Errors: IJ_ERR_PARAM (bad sizes or physics: nx, ny < 1, rho_ink <= rho_air,
 * sigma <= 0, W <= 0, tau_phi <= 0, nu <= 0, nozzle wider than the domain),
 * IJ_ERR_OOM, IJ_ERR_CUDA.  On error *out is NULL and nothing is leaked.
 */
ij_status ij_create(const ij_params* params, int count, ij_alloc_fn alloc, ij_free_fn free_fn,
                    void* ctx, void* stream, ij_handle* out);

/*
 * ij_step -- advance every lattice of the handle by nsteps time steps (Eq. 3
 * for f with the collision of Eq. 4-6, Eq. 8 for g with Eq. 9-10), each step
 * one fused kernel pass; a diagnostics record is taken at every step t with
 * t % diag_every == 0.  Asynchronous on the handle's stream.  nsteps >= 0.
 * Returns IJ_ERR_NUMERIC when every lattice of the handle is frozen (flags are
 * read without synchronising, so this shows up at most one call late).
 */
ij_status ij_step(ij_handle h, long long nsteps);

/*
 * ij_observe -- synchronise, then return the latest diagnostics record of
 * lattice `index` in *out (may be NULL) and its order parameter
 * phi = sum_i g_i (ny*nx floats, 3-D: nz*ny*nx; solid cells 0) into phi_out (may be NULL;
 * device pointer if phi_on_device, else host).  Returns IJ_ERR_NUMERIC (with
 * the outputs filled) if this lattice is frozen by a numeric failure.
 */
ij_status ij_observe(ij_handle h, int index, ij_obs* out, float* phi_out, int phi_on_device);

/* ij_history -- copy up to max_records diagnostics records of lattice
 * `index` (oldest first, 13 doubles each in ij_obs order) into host memory
 * `out` (may be NULL); *count receives the number of records held. */
ij_status ij_history(ij_handle h, int index, double* out, int max_records, int* count);

/* ij_get_state / ij_set_state -- copy the populations of lattice `index`
 * (f: 9*ny*nx floats, g: 5*ny*nx floats, layout above; 3-D: f 19*nz*ny*nx,
 * g 7*nz*ny*nx) out of / into the handle as absolute FP32 values (FP16
 * storage is widened on the way out and rounded on the way in); set_state
 * also sets the time of the handle to t.  Host or device buffers. */
ij_status ij_get_state(ij_handle h, int index, float* f, float* g, int on_device);
ij_status ij_set_state(ij_handle h, int index, const float* f, const float* g, long long t,
                       int on_device);

/* ij_time -- current time step of the handle (all lattices share it). */
ij_status ij_time(ij_handle h, long long* t);

/* ij_launch_count -- number of kernels this handle has launched. */
ij_status ij_launch_count(ij_handle h, long long* launches);

/* ij_kernel_timing -- measurement aid, no counterpart in the paper.  Reads
 * (synchronising) the summed duration in ms of the step-kernel launches timed
 * so far, and their number, into *total_ms / *launches (either may be NULL);
 * then, if enable >= 0, switches CUDA-event timing of every step-kernel launch
 * on (1) or off (0) and resets the sums.  Events are recorded on the handle's
 * stream immediately around each launch. */
ij_status ij_kernel_timing(ij_handle h, int enable, double* total_ms, long long* launches);

/*
 * Launch-shape tuning (no counterpart in the paper).  The step kernel runs
 * one warp per work item: a strip of 60 columns, two per lane (plus two halo
 * columns on each side), times a range of rows of one lattice, with the
 * populations staged `prefetch` rows (1..4) ahead of use; every block is
 * one warp (32 threads), so a finished item frees its slot at once.  Every
 * lattice of a handle is in the one bucket of 32-thread blocks.  The work
 * list comes in two forms, chosen by `chunk`:
 *   chunk >= 1 : rows cut into chunks of `chunk` rows; the list starts with
 *                the rows of nozzle-wall strips below the nozzle exit
 *                (costlier per row) and ends with the last eighth of each
 *                lattice's rows, both in chunks a quarter as long;
 *   chunk <= 0 : cost-balanced (the default, 0): with S the number of items
 *                the GPU runs at once, each strip's first rows -- 7/8 of its
 *                cost, wall rows counting 2.2 -- are cut into pieces of
 *                equal cost near one S-th of the total (one wave that ends
 *                together), the rest into short pieces listed last; -1: the
 *                whole strip in equal pieces, no tail; -2: 3/4 and a tail of
 *                shorter pieces; -3, -4, -5: the whole strip in pieces for 2,
 *                3, 4 full waves.
 *
 * ij_tune      -- set chunk (>= -5) and prefetch (block_size: 32, or <= 0
 *                 for every bucket).  Synchronises.
 * ij_autotune  -- time `reps` trial launches of every candidate (chunks
 *                 8..128 in steps of 8, 160, 192, 256 and 0 .. -5; prefetch
 *                 1..4) on the current state
 *                 and keep the fastest.  Trial launches leave the state and
 *                 the time unchanged.  Synchronises.
 * ij_get_tuning -- block size, chunk, prefetch and item count of bucket
 *                 `bucket` (0-based); IJ_ERR_PARAM past the last bucket.
 * 3-D handles have one bucket of 512-thread blocks (one CTA per 28 x 12
 * column tile and z chunk); its one tunable is the z chunk: ij_tune takes
 * chunk >= 1 and prefetch 1 (block_size 512 or <= 0), ij_autotune times
 * chunks of 8 .. 256 planes.  Results do not depend on the chunk.
 */
ij_status ij_tune(ij_handle h, int block_size, int chunk, int prefetch);
/* ij_use_graph -- run whole diagnostics periods (diag_every steps, or 16
 * when diagnostics are off) of ij_step as one replay of a captured CUDA
 * graph (enable = 1, the default) or as separate launches (0).  Both give
 * identical results; the graph removes per-launch overhead. */
ij_status ij_use_graph(ij_handle h, int enable);
ij_status ij_autotune(ij_handle h, int reps);
ij_status ij_get_tuning(ij_handle h, int bucket, int* block_size, int* chunk, int* prefetch,
                        int* items);

/*
 * ij_step_noalloc -- one time step of ONE lattice between device buffers the
 * caller owns, allocating no device memory.  The paper has no counterpart:
 * this is a service for callers that may not allocate where they step the
 * lattice -- a plugin inside another framework that owns all device memory
 * through its own pool, or a loop that must keep a fixed memory footprint
 * (allocator calls have a latency and a fragmentation it cannot bound).  It
 * computes exactly what ij_step computes for a one-lattice handle.
 *   params        : the lattice (host memory); nx, ny, geometry as in ij_create;
 *                   2-D FP32 storage only (dim 3 or IJ_FP16_STORE returns
 *                   IJ_ERR_PARAM).
 *   t             : time of the input state (selects the drive F(t)).
 *   f_in, g_in    : device, the state at t.  f holds the stored layout
 *                   f_i - w_i n0 on fluid cells (n0 = (rho_ink + rho_air)/2,
 *                   w = 4/9, 1/9, 1/36) and 0 on solid cells; g holds g_i.
 *                   Same [i][y][x] order as above.  Read only.
 *   f_out, g_out  : device, receive the state at t+1 in the same layout (solid
 *                   cells 0); must not alias the inputs.
 *   record_out    : device, 13 doubles (ij_obs order) receiving the
 *                   diagnostics record of the state at t, or NULL for none.
 *                   Each call starts a fresh breakup history, so breakup_step
 *                   is t when the neck is already closed, else -1.
 *   status_out    : device, one unsigned receiving the step's numeric flag, or
 *                   NULL.  Nonzero means the step met NaN or |u| > 0.3: the
 *                   kernel then stops writing, so f_out and g_out are only
 *                   partly written and must be discarded.
 *   stream        : cudaStream_t to enqueue on (NULL: the legacy default
 *                   stream); it must belong to the current device, else
 *                   IJ_ERR_PARAM.  The call is asynchronous.
 * Limits: ny <= 8192 and at most 16384 work items (strips of 60 columns times
 * chunks of 64 rows); larger lattices are rejected with IJ_ERR_PARAM.
 * Descriptors and scratch live in one fixed device array of about 0.7 MB per
 * GPU that loads the library, kept until the process exits.  The first call
 * on a device looks up that array's device address, so make it before any
 * stream capture.  Every call shares the array: calls whose GPU work
 * overlaps (for example on two streams) race, so order them on one stream.
 * The descriptor, the time and the work list are copied from static host
 * buffers with cudaMemcpyAsync under a mutex (no host heap either).
 * Errors: IJ_ERR_PARAM, IJ_ERR_CUDA.
 */
ij_status ij_step_noalloc(const ij_params* params, long long t, const float* f_in,
                          const float* g_in, float* f_out, float* g_out, double* record_out,
                          unsigned* status_out, void* stream);

/* ij_destroy -- synchronise and release everything (NULL is accepted). */
ij_status ij_destroy(ij_handle h);

/* ij_last_error -- message of the last failure on this thread (never NULL). */
const char* ij_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
