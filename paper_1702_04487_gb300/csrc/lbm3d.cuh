// Internal descriptors of the 3-D (D3Q19 / D3Q7) lift of the binary-fluid
// LBM step.  Shared by lbm3d_kernels.cu and the host API.
#pragma once
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include "lbm2d.cuh"

namespace ij {

// One 3-D lattice.  The state is double-buffered: buffer b holds
//   f  [19][N]  deviations f_i - w_i n0       (FP32, or FP16 in FP16 storage)
//   g  [6][N]   g_1..g_6                      (FP32, or FP16)
//   g0 [N]      g_0 (always FP32: its per-step increments are far below the
//               FP16 resolution of values of size phi*)
//   phi [nz+4][ny][nx]  phi with wetting ghosts: phi = sum g on fluid cells,
//               the ghost value on solid cells within reach of a fluid
//               stencil, planes -2..nz+1 (the extended planes of the axial
//               ends, which collide too), read by the stencils of the next
//               step.
// The current buffer is *cur, flipped after each step of a lattice that is
// not frozen (a lattice frozen by a numeric failure keeps the state of the
// step before).
struct Inst3 {
  int nx, ny, nz, geom, L, wt, bc, fp16;
  float cx, cy, R2, Ro2;  // channel r^2 < R2, nozzle wall R2 <= r^2 < Ro2
  float phis, inv_phis, A4, kappa, hk, q, omq, inv_tphi, gamma, inv2q, nu_air, dnu, F0, Fneg, n0;
  long long T1, T2, Tidle;
  double d_phis, d_n0, d_A, d_kappa, d_h, d_gamma, d_q, d_W, init_x, init_y, init_z, init_r,
      jitter;
  int init_kind, n_ghost;
  unsigned long long seed;
  void* f[2];
  void* g[2];
  float* g0[2];
  float* phi[2];
  int* ghost;    // [n_ghost]: in-domain solid cells within reach of a fluid stencil
  int* cur;      // index of the buffer holding the current state
  double* rows;  // [3][nz]
  double* sums;  // [4]
  unsigned* status;
};

// A work item of the 3-D step kernel (one CTA of 16 warps): the tile of
// columns x in [xs, xs + 28), y in [ys, ys + 12) (clipped to the lattice) of
// lattice `inst`, planes z0 .. z0 + ch - 1.
struct Item3 {
  int inst, xs, ys, z0, ch;
};

constexpr int kTile3X = 28, kTile3Y = 12;  // written columns of a 3-D work item
constexpr int kStep3Threads = 512;          // threads of a step3 CTA (32 x 16 columns)

// Solid cells of lattice h within reach of a fluid D3Q19 stencil (cell
// indices z * ny * nx + y * nx + x), written to out when not null; returns
// their number.  Host code.
int ghost_cells3(const Inst3& h, int* out);
// Work items of every lattice into out (null: count only); returns the count.
int make_items3(const Inst3* h, int n_inst, int chunk, Item3* out);

cudaError_t launch_init3(const Inst3* d_inst, const Inst3& h, int index, cudaStream_t s);
// one time step of every lattice (items over all of them) at t = d_t[0] +
// t_off, from buffer *cur into the other one
cudaError_t launch_step3(const Inst3* d_inst, const Item3* d_items, int n_items, int n_inst,
                         const long long* d_t, int t_off, bool diag, bool h16, cudaStream_t s);
// wetting ghosts and extended planes of phi in buffer *cur (next: the other
// buffer, which the step just wrote)
cudaError_t launch_ghost3(const Inst3* d_inst, const Inst3* h, int n_inst, bool next, cudaStream_t s);
// *cur ^= 1 for every lattice that is not frozen
cudaError_t launch_flip3(const Inst3* d_inst, int n_inst, cudaStream_t s);
// state (current buffer) <-> absolute FP32 populations f[19][N], g[7][N]
// (solid cells 0); import also refreshes phi with its ghosts
cudaError_t launch_export3(const Inst3* d_inst, const Inst3& h, int index, float* f, float* g,
                           cudaStream_t s);
cudaError_t launch_import3(const Inst3* d_inst, const Inst3& h, int index, const float* f,
                           const float* g, cudaStream_t s);
// phi of the current state with solid cells zeroed
cudaError_t launch_phi3(const Inst3* d_inst, const Inst3& h, int index, float* out, cudaStream_t s);
size_t step3_smem_bytes(bool h16);
cudaError_t set_step3_smem_limit();

}  // namespace ij
