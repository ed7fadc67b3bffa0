// Internal device-side descriptors of the 2-D binary-fluid LBM step.
// Shared by the kernels (lbm2d_kernels.cu) and the host API (inkjet_api.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "inkjet.h"

namespace ij {

enum { GEOM_NONE = 0, GEOM_NOZZLE = 1, GEOM_PLATE = 2 };
enum { BC_ZG = 0, BC_PER = 1, BC_CLOSED = 2 };
enum { INIT_MENISCUS = 0, INIT_DROP = 1, INIT_FLAT = 2, INIT_UNIFORM = 3 };

constexpr int kRec = 13;        // doubles per diagnostics record
constexpr int kHistCap = 1024;  // records kept per lattice (ring)
constexpr unsigned kStatusNumeric = 1u;

// One lattice.  FP32 constants feed the step kernel; FP64 ones the
// initialisation and the diagnostics.
struct Inst {
  int nx, ny, geom, cx0, cx1, L, wt, bc;
  int y_exit, y_scan, init_kind;
  int fp16;  // FP16 storage (the same for every lattice of a handle)
  // step constants (FP32)
  float phis, inv_phis, A4, kappa, hk, q, omq, inv_tphi, gamma, inv2q, nu_air, dnu, F0, Fneg;
  float n0;  // rest density: f is stored as the deviation f_i - w_i n0
  long long T1, T2, Tidle;
  // initialisation and diagnostics constants (FP64)
  double d_phis, d_n0, d_A, d_kappa, d_h, d_gamma, d_q, d_W, init_x, init_y, init_r, jitter, vmin;
  unsigned long long seed;
  // populations, double-buffered by time parity: f[t & 1] holds the state at
  // t.  f holds deviations from the rest equilibrium, f_i - w_i n0, so that
  // FP32 rounds the small part that varies (about 50x smaller ulp); g is
  // stored as is.  FP16 storage: f as 9N halves; g as g_0 in FP32 [N]
  // followed by g_1..4 as halves [4][N] (nx even, so pairs of halves of
  // neighbouring columns are 4-byte aligned).
  float* f[2];
  float* g[2];
  // diagnostics scratch and results
  double* rows;    // [3][ny]: sum e, sum e n, sum e n u_y per row
  double* sums;    // [4]: sum n, sum phi, sum n u_y, unused
  double* hist;    // [kHistCap][kRec] ring of records
  double* dstate;  // [8]: have_prev, neck_prev, t_prev, breakup, record count
  unsigned* status;  // this lattice's numeric flag (NaN or |u| > 0.3 seen)
};

// A unit of work of the step kernel (one warp): `ch` rows starting at y0 of
// the strip of lattice `inst` that writes columns xs .. xs + nout - 1
// (nout <= 60); lane l holds columns xs - halo + 2 l and the next one
// (periodic wrap, halo = 2).  Half-warp items (half = 1, nout <= 28): lanes
// 0-15 take rows y0 .. y0+ch-1 and lanes 16-31 rows y1 .. y1+ch-1 of the
// same strip (y1 < 0: lanes 16-31 idle), lane l holding columns
// xs - halo + 2 (l mod 16) and the next one.
struct Item {
  int inst, xs, nout, halo, y0, ch, half, y1;
};

constexpr int kStepThreads = 32;  // one warp per block, one work item each
constexpr int kStepBlocksPerSM = 10;  // resident blocks per SM the registers are sized for
constexpr int kMaxPrefetch = 4;    // rows staged ahead of use: 1 .. 4

size_t step_smem_bytes(int nthreads, int prefetch, bool h16);
// bytes of one time buffer of f / of g
size_t state_bytes_f(const Inst& I);
size_t state_bytes_g(const Inst& I);
cudaError_t set_step_smem_limit();
// Work items of one lattice (row chunks of `chunk` rows x strips, a narrow
// last strip in half-warp items) into out (at most cap); returns the count,
// or -1 when cap is too small.
int make_items(const Inst& I, int k, int chunk, Item* out, int cap);
int items_per_lattice(const Inst& I, int chunk);
// The same for rows ya .. yb-1 only (allow_half: narrow strips in half-warp
// items; out may be null to count).
int make_items_range(const Inst& I, int k, int chunk, int ya, int yb, Item* out, int cap,
                     bool allow_half);
int items_per_range(const Inst& I, int chunk, int ya, int yb, bool allow_half);

// host helpers of inkjet_api.cu
ij_status validate_params(const ij_params& p, int k);
Inst derive_params(const ij_params& p);
ij_status report(ij_status st, const char* msg);

cudaError_t launch_init(const Inst* d_inst, const Inst& h_inst, int index, cudaStream_t s);
// odd: some lattice of the launch has an odd nx (FP32 storage only); its
// column pairs are then copied and stored one column at a time
cudaError_t launch_step(const Inst* d_inst, const Item* d_items, int n_items, int nthreads,
                        int grid, const long long* d_t, int t_off, bool diag, int prefetch,
                        bool h16, bool odd, cudaStream_t s);
// default number of rows staged ahead of use
int step_prefetch_for(int nthreads);
// work items the GPU runs at once: SMs x resident blocks of the step kernel
// (launch without diagnostics) at this prefetch and storage
int step_slots(int prefetch, bool h16, bool odd);
cudaError_t launch_finalize(const Inst* d_inst, int n_inst, const long long* d_t,
                            cudaStream_t s);
cudaError_t launch_advance(long long* d_t, int by, cudaStream_t s);
cudaError_t launch_phi(const Inst* d_inst, const Inst& h_inst, int index, const long long* d_t,
                       float* out, cudaStream_t s);
// absolute populations <-> stored deviations (solid cells: 0 <-> 0)
cudaError_t launch_f_export(const Inst* d_inst, const Inst& h_inst, int index, const float* src,
                            float* dst, cudaStream_t s);
cudaError_t launch_f_import(const Inst* d_inst, const Inst& h_inst, int index, const float* src,
                            float* dst, cudaStream_t s);
// FP16 storage of time parity `parity` <-> absolute FP32 f [9][N], g [5][N]
// (export when !to_device_state; f or g may be null on export)
cudaError_t launch_convert16(const Inst* d_inst, const Inst& h_inst, int index, int parity,
                             float* f, float* g, bool to_device_state, cudaStream_t s);

}  // namespace ij
