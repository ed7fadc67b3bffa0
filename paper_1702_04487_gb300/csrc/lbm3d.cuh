// Internal descriptors of the 3-D (D3Q19 / D3Q7) lift of the binary-fluid
// LBM step.  Shared by lbm3d_kernels.cu and the host API.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm2d.cuh"

namespace ij {

// One 3-D lattice.  Populations are stored as a state (the populations at t)
// and a post-collision copy, each as:
//   f  [19][N]  deviations f_i - w_i n0       (FP32, or FP16 in FP16 storage)
//   g  [6][N]   g_1..g_6                      (FP32, or FP16)
//   g0 [N]      g_0 (always FP32: its per-step increments are far below the
//               FP16 resolution of values of size phi*)
// plus phi [N] (FP32) of the state, read by the stencils of the next step.
struct Inst3 {
  int nx, ny, nz, geom, L, wt, bc, fp16;
  float cx, cy, R2, Ro2;  // channel r^2 < R2, nozzle wall R2 <= r^2 < Ro2
  float phis, inv_phis, A4, kappa, hk, q, omq, inv_tphi, gamma, inv2q, nu_air, dnu, F0, Fneg, n0;
  long long T1, T2, Tidle;
  double d_phis, d_n0, d_A, d_kappa, d_h, d_gamma, d_q, d_W, init_x, init_y, init_z, init_r,
      jitter;
  int init_kind, pad0;
  unsigned long long seed;
  void* f;
  void* g;
  float* g0;
  void* fp;
  void* gp;
  float* g0p;
  float* phi;
  double* rows;  // [3][nz]
  double* sums;  // [4]
  unsigned* status;
};

cudaError_t launch_init3(const Inst3* d_inst, const Inst3& h, int index, cudaStream_t s);
// collision (with diagnostics plane sums when diag) then streaming, for one
// lattice; t = *d_t + t_off
cudaError_t launch_collide3(const Inst3* d_inst, const Inst3& h, int index, const long long* d_t,
                            int t_off, bool diag, cudaStream_t s);
cudaError_t launch_stream3(const Inst3* d_inst, const Inst3& h, int index, cudaStream_t s);
// state <-> absolute FP32 populations f[19][N], g[7][N] (solid cells 0);
// import also refreshes phi
cudaError_t launch_export3(const Inst3* d_inst, const Inst3& h, int index, float* f, float* g,
                           cudaStream_t s);
cudaError_t launch_import3(const Inst3* d_inst, const Inst3& h, int index, const float* f,
                           const float* g, cudaStream_t s);
// phi of the state with solid cells zeroed
cudaError_t launch_phi3(const Inst3* d_inst, const Inst3& h, int index, float* out, cudaStream_t s);

}  // namespace ij
