// Kernels of the 2-D binary-fluid lattice Boltzmann inkjet step
// (He et al., arXiv:1702.04487, "Methods", Eq. 3-10).
//
// Step kernel design (bandwidth-bound stencil, no tensor cores):
//  - one warp per work item: a strip of 28 written columns (plus two halo
//    columns each side) by a chunk of rows of one lattice; the warp marches
//    up the rows, so every cell's populations are read once and written
//    once per step (structure-of-arrays, coalesced);
//  - neighbours along x come from warp shuffles, along y from registers;
//    populations are staged P rows ahead with cp.async into a per-warp ring
//    in shared memory, and warps never wait on one another;
//  - per row iteration: phi of row R, wetting ghost values of row R-1, the
//    collision of f (Eq. 4-6) and g (Eq. 8-10) on row R-2, the streaming of
//    row R-3 with halfway bounce-back and the stay/move split of Eq. 8;
//  - geometry is analytic (no mask array);
//  - storage is FP32, or FP16 (f as offsets from w_i n0, g_1..4 as is, g_0
//    in FP32) with every update in FP32;
//  - diagnostics rows (ink weight, mass, momentum) are summed in FP32 per
//    strip row and in FP64 across rows and strips, on diagnostics steps.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "lbm2d.cuh"

namespace ij {
namespace {

// D2Q9 lattice (Eq. 5-6): rest, +x, +y, -x, -y, +x+y, -x+y, -x-y, +x-y.
// Compile-time values, so that products with 0 and +-1 fold away.
__device__ __forceinline__ constexpr int cEX(int i) {
  return i == 1 || i == 5 || i == 8 ? 1 : (i == 3 || i == 6 || i == 7 ? -1 : 0);
}
__device__ __forceinline__ constexpr int cEY(int i) {
  return i == 2 || i == 5 || i == 6 ? 1 : (i == 4 || i == 7 || i == 8 ? -1 : 0);
}
#define W1 (1.0f / 9.0f)
#define W2 (1.0f / 36.0f)

__device__ __forceinline__ int wrapi(int v, int m) {
  int r = v % m;
  return r < 0 ? r + m : r;
}

// Axial mapping of a pipeline row; false outside a closed domain.
__device__ __forceinline__ bool map_row(const Inst& I, int y, int& ym) {
  if ((unsigned)y < (unsigned)I.ny) {
    ym = y;
    return true;
  }
  if (I.bc == BC_PER) {
    ym = wrapi(y, I.ny);
    return true;
  }
  if (I.bc == BC_ZG) {
    ym = y < 0 ? 0 : I.ny - 1;
    return true;
  }
  return false;
}

// The same mapping and near-solid test from values held in registers.
__device__ __forceinline__ bool map_row_v(int y, int ny, int bc, int& ym) {
  if ((unsigned)y < (unsigned)ny) {
    ym = y;
    return true;
  }
  if (bc == BC_PER) {
    ym = wrapi(y, ny);
    return true;
  }
  if (bc == BC_ZG) {
    ym = y < 0 ? 0 : ny - 1;
    return true;
  }
  return false;
}
__device__ __forceinline__ bool near_solid_v(int geom, int bc, int ny, int L, int wt, bool colwall,
                                             int y) {
  if (bc == BC_CLOSED && (y == 0 || y == ny - 1)) return true;
  if (geom == GEOM_NOZZLE) {
    if (!colwall) return false;
    if (bc == BC_PER && (y == 0 || y == ny - 1)) return true;
    return y - 1 < L;
  }
  if (geom == GEOM_PLATE) {
    if (bc == BC_PER && (y == 0 || y == ny - 1)) return true;
    return y - 1 < wt;
  }
  return false;
}

// Kind of an in-domain cell: 0 fluid, 1 solid, 2 solid on a wetting face.
__device__ __forceinline__ int geom_kind(const Inst& I, int x, int y) {
  if (I.geom == GEOM_NOZZLE) {
    if (y < I.L && ((x >= I.cx0 - I.wt && x < I.cx0) || (x >= I.cx1 && x < I.cx1 + I.wt)))
      return (x == I.cx0 - 1 || x == I.cx1) ? 2 : 1;
    return 0;
  }
  if (I.geom == GEOM_PLATE) {
    if (y < I.wt) return (y == I.wt - 1) ? 2 : 1;
    return 0;
  }
  return 0;
}

__device__ __forceinline__ int kind_at(const Inst& I, int x, int y) {
  int ym;
  if (!map_row(I, y, ym)) return 1;
  return geom_kind(I, wrapi(x, I.nx), ym);
}

// Fig. 1 waveform: +F0, then -F_neg, then idle (periodic if T_idle > 0).
__device__ __forceinline__ float drive_at(const Inst& I, long long t) {
  long long tt = t;
  if (I.Tidle > 0) tt = t % (I.T1 + I.T2 + I.Tidle);
  if (tt < I.T1) return I.F0;
  if (tt < I.T1 + I.T2) return -I.Fneg;
  return 0.0f;
}

// Asynchronous 4-byte global -> shared copies (cp.async) of five / four
// populations p, p + N, ... into shared addresses sa, sa + 128, ... (one
// population row of a warp apart), issued only when pred is set: one
// predicate and predicated instructions, no branch.
__device__ __forceinline__ void cp5_if(unsigned sa, const float* p, int N, bool pred) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %6, 0;\n"
      " @p cp.async.ca.shared.global [%0], [%1], 4;\n"
      " @p cp.async.ca.shared.global [%0+128], [%2], 4;\n"
      " @p cp.async.ca.shared.global [%0+256], [%3], 4;\n"
      " @p cp.async.ca.shared.global [%0+384], [%4], 4;\n"
      " @p cp.async.ca.shared.global [%0+512], [%5], 4;\n}\n" ::"r"(sa),
      "l"(p), "l"(p + N), "l"(p + 2 * N), "l"(p + 3 * N), "l"(p + 4 * N), "r"((int)pred)
      : "memory");
}
__device__ __forceinline__ void cp4_if(unsigned sa, const float* p, int N, bool pred) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %5, 0;\n"
      " @p cp.async.ca.shared.global [%0], [%1], 4;\n"
      " @p cp.async.ca.shared.global [%0+128], [%2], 4;\n"
      " @p cp.async.ca.shared.global [%0+256], [%3], 4;\n"
      " @p cp.async.ca.shared.global [%0+384], [%4], 4;\n}\n" ::"r"(sa),
      "l"(p), "l"(p + N), "l"(p + 2 * N), "l"(p + 3 * N), "r"((int)pred)
      : "memory");
}
// FP16 storage: one 4-byte copy, and groups of 4 / 5 copies of the 4-byte
// half pairs at p, p + N, ... (halves) into sa, sa + DS, ...
__device__ __forceinline__ void cp1_if(unsigned sa, const void* p, bool pred) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %2, 0;\n"
      " @p cp.async.ca.shared.global [%0], [%1], 4;\n}\n" ::"r"(sa),
      "l"(p), "r"((int)pred)
      : "memory");
}
template <int DS>
__device__ __forceinline__ void cp4h_if(unsigned sa, const __half* p, int N, bool pred) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %5, 0;\n"
      " @p cp.async.ca.shared.global [%0], [%1], 4;\n"
      " @p cp.async.ca.shared.global [%0+%6], [%2], 4;\n"
      " @p cp.async.ca.shared.global [%0+%7], [%3], 4;\n"
      " @p cp.async.ca.shared.global [%0+%8], [%4], 4;\n}\n" ::"r"(sa),
      "l"(p), "l"(p + N), "l"(p + 2 * N), "l"(p + 3 * N), "r"((int)pred), "n"(DS), "n"(2 * DS),
      "n"(3 * DS)
      : "memory");
}
template <int DS>
__device__ __forceinline__ void cp5h_if(unsigned sa, const __half* p, int N, bool pred) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %6, 0;\n"
      " @p cp.async.ca.shared.global [%0], [%1], 4;\n"
      " @p cp.async.ca.shared.global [%0+%7], [%2], 4;\n"
      " @p cp.async.ca.shared.global [%0+%8], [%3], 4;\n"
      " @p cp.async.ca.shared.global [%0+%9], [%4], 4;\n"
      " @p cp.async.ca.shared.global [%0+%10], [%5], 4;\n}\n" ::"r"(sa),
      "l"(p), "l"(p + N), "l"(p + 2 * N), "l"(p + 3 * N), "l"(p + 4 * N), "r"((int)pred),
      "n"(DS), "n"(2 * DS), "n"(3 * DS), "n"(4 * DS)
      : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Bit i set when the source x - c_i, y - c_i of direction i is solid.
__device__ __noinline__ unsigned solid_sources(const Inst& I, int x, int y) {
  unsigned m = 0;
  for (int i = 1; i < 9; i++)
    if (kind_at(I, x - cEX(i), y - cEY(i)) != 0) m |= 1u << i;
  return m;
}

// Kind of the in-domain cell (column kind colk, row ym): 0 fluid, 1 solid,
// 2 solid on a wetting face.  colk is the kind a nozzle-wall column has below
// y = L (0 for channel and air columns).
__device__ __forceinline__ int row_kind(int geom, int colk, int L, int wt, int ym) {
  if (geom == GEOM_NOZZLE) return ym < L ? colk : 0;
  if (geom == GEOM_PLATE) return ym < wt ? (ym == wt - 1 ? 2 : 1) : 0;
  return 0;
}

__device__ __forceinline__ int column_kind(const Inst& I, int x) {
  if (I.geom != GEOM_NOZZLE) return 0;
  if ((x >= I.cx0 - I.wt && x < I.cx0) || (x >= I.cx1 && x < I.cx1 + I.wt))
    return (x == I.cx0 - 1 || x == I.cx1) ? 2 : 1;
  return 0;
}

// ---------------------------------------------------------------------------
// The fused step: one warp per work item (a strip of columns x a chunk of
// rows of one lattice); warps never wait on one another.
//
// Lane l of a strip holds column x = xs - 2 + l (periodic wrap).  The strip
// writes the nout <= 28 columns of lanes 2 .. nout+1; lanes 1 and nout+2
// collide too (the streaming pulls their post-collision populations), and
// lanes 0 and 31 only contribute phi to the stencil.  When lane 0 or 31
// sits on a wall, its ghost value needs phi beyond the strip: that lane
// stages the g of the column outside as well.  Neighbours along x are
// exchanged with warp shuffles; along y each lane keeps its own column's
// last rows in registers while the warp marches up the rows.
//
// Per row iteration (pipeline row R): phi of row R (sum of g); the wetting
// ghost values of row R-1 (only rows with a solid cell in the strip); the
// collision of row R-2 (Eq. 4-6 for f, Eq. 8-10 for g); the streaming of
// row R-3 with halfway bounce-back and the stay/move split of Eq. 8, stored
// to the other time buffer.  Every lane stages its own column's 14
// populations of row R+P into the warp's shared-memory ring with cp.async,
// P rows ahead of use, and reads back only what it staged itself.
//
// FP16 storage (H): a cp.async moves 4 bytes at least, so each even lane
// stages the half pair of its own column and the next (x even: strips start
// at even columns and nx is even, so a pair never straddles the wrap); every
// lane stages its FP32 g_0; the edge lanes stage the outer column's g into
// slots of their own.  One staged row holds (in 4-byte words) g_0[32],
// g_1..4 as [4][16] half pairs, f_0..8 as [9][16] half pairs, then the outer
// g_0 and g_1..4 pairs of lane 0 and of lane 31.
constexpr int kWarpsPerBlock = kStepThreads / 32;
constexpr int kRowFloats = 14 * 32;  // one staged row of a warp: g[5][32], then f[9][32]
constexpr int kRowWordsH = 256;      // the same in FP16 storage (250 used)
constexpr unsigned kFull = 0xffffffffu;

template <bool DIAG, int P, bool H>
__global__ void __launch_bounds__(kWarpsPerBlock * 32, kStepBlocksPerSM)
    step_kernel(const Inst* __restrict__ insts, const Item* __restrict__ items, int n_items,
                const long long* __restrict__ d_t, int t_off) {
  constexpr int D = P + 3;  // ring rows: R+P .. R-2 are live
  constexpr int kRowW = H ? kRowWordsH : kRowFloats;
  extern __shared__ float4 smem4[];
  // with one warp per block the warp index is the constant 0, so the compiler
  // sees the work item, its lattice and the row loop as warp-uniform
  const int lane = threadIdx.x & 31, warp = kWarpsPerBlock == 1 ? 0 : threadIdx.x >> 5;
  // FP32: each lane's column of the ring; FP16: the warp's ring
  float* ring = reinterpret_cast<float*>(smem4) + warp * D * kRowW + (H ? 0 : lane);
  const unsigned ring_sa = (unsigned)__cvta_generic_to_shared(ring);
  const long long t = *d_t + t_off;
  // staged g_i / f_i of this lane's column, and the sum of the outer g
  auto ring_g = [&](const float* row, int i) -> float {
    if (!H) return row[i * 32];
    if (i == 0) return row[lane];
    return __half2float(reinterpret_cast<const __half*>(row + 32 + (i - 1) * 16)[lane]);
  };
  auto ring_f = [&](const float* row, int i) -> float {
    if (!H) return row[(5 + i) * 32];
    return __half2float(reinterpret_cast<const __half*>(row + 96 + i * 16)[lane]);
  };
  auto ring_outer = [&](const float* row) -> float {
    if (!H) return row[160] + row[192] + row[224] + row[256] + row[288];
    // lane 0: outer column x - 1 is odd, the upper half; lane 31: x + 1 even
    const float* o = row + 240 + (lane == 0 ? 0 : 5);
    float sum = o[0];
#pragma unroll
    for (int i = 1; i < 5; i++) {
      const __half2 hp = reinterpret_cast<const __half2*>(o)[i];
      sum += lane == 0 ? __high2float(hp) : __low2float(hp);
    }
    return sum;
  };

  for (int item = blockIdx.x * kWarpsPerBlock + warp; item < n_items;
       item += gridDim.x * kWarpsPerBlock) {
    const Item it = items[item];
    const Inst& I = insts[it.inst];
    // a lattice whose numeric flag is set is frozen
    const unsigned st0 = lane == 0 ? *(volatile const unsigned*)I.status : 0u;
    if (__shfl_sync(kFull, st0, 0) & kStatusNumeric) continue;
    const int nx = I.nx, ny = I.ny, geom = I.geom, L = I.L, wt = I.wt, bc = I.bc;
    const int N = nx * ny;  // < 2^31 / 9 (checked on the host)
    const int y0 = it.y0, ch = it.ch;
    const int x = wrapi(it.xs - it.halo + lane, nx);
    const bool out_lane = lane >= it.halo && lane < it.halo + it.nout;
    const bool col_lane = lane >= it.halo - 1 && lane <= it.halo + it.nout;
    const int ck = column_kind(I, x);
    const int ckW = column_kind(I, wrapi(x - 1, nx)), ckE = column_kind(I, wrapi(x + 1, nx));
    const bool colwall = geom == GEOM_NOZZLE && (ck | ckW | ckE) != 0;
    // lanes 0 and 31 on a wall column: the column outside the strip (xo)
    const bool edge = (lane == 0 || lane == 31) && ck != 0;
    const int xo = wrapi(lane == 0 ? x - 1 : x + 1, nx);
    const int cko = lane == 0 ? ckW : ckE;
    const bool drive_col = geom != GEOM_NOZZLE || (x >= I.cx0 && x < I.cx1);
    const float phis = I.phis, inv_phis = I.inv_phis, A4 = I.A4, kappa = I.kappa, hk = I.hk;
    const float omq = I.omq, inv_tphi = I.inv_tphi, gamma = I.gamma, inv2q = I.inv2q;
    const float qmt = I.q - I.inv_tphi;
    const float nu_air = I.nu_air, dnu = I.dnu, n0 = I.n0;
    const float Fd = drive_at(I, t);
    const float* __restrict__ fin = I.f[t & 1];
    const float* __restrict__ gin = I.g[t & 1];
    float* __restrict__ fout = I.f[(t + 1) & 1];
    float* __restrict__ gout = I.g[(t + 1) & 1];
    // FP16 storage: f halves; g_0 FP32 [N], then g_1..4 halves [4][N]
    const __half* __restrict__ fhin = reinterpret_cast<const __half*>(fin);
    const __half* __restrict__ ghin = reinterpret_cast<const __half*>(gin + N);
    __half* __restrict__ fhout = reinterpret_cast<__half*>(fout);
    __half* __restrict__ ghout = reinterpret_cast<__half*>(gout + N);
    const bool any_edge = H && __any_sync(kFull, edge);

    // Stage pipeline row r into ring slot sp (the lane's own column, or in
    // FP16 storage the pair of columns of an even lane; f only for rows that
    // are collided), as one cp.async group.
    auto stage = [&](int r, int sp) {
      int ym;
      if (r <= y0 + ch + 2 && map_row_v(r, ny, bc, ym)) {  // uniform over the warp
        const unsigned d = ring_sa + sp * (kRowW * 4);
        const bool own = row_kind(geom, ck, L, wt, ym) == 0;
        const bool frow = r >= y0 - 1 && r <= y0 + ch;
        // a solid edge lane with a fluid cell beyond the strip stages that
        // cell's g (FP32: where its own f would be; FP16: slots of its own)
        const bool outer = edge && !own && row_kind(geom, cko, L, wt, ym) == 0;
        if (!H) {
          const bool fneed = own && col_lane && frow;
          const float* qg = gin + (ym * nx + x);
          const float* qf = outer ? gin + (ym * nx + xo) : fin + (ym * nx + x);
          cp5_if(d, qg, N, own);
          cp5_if(d + 5 * 128, qf, N, fneed || outer);
          cp4_if(d + 10 * 128, qf + 5 * N, N, fneed);
        } else {
          const int c = ym * nx + x;
          cp1_if(d + lane * 4, gin + c, own);
          // the even lane of a pair copies for both (x + 1 has kind ckE)
          const bool pair = (lane & 1) == 0 && (own || row_kind(geom, ckE, L, wt, ym) == 0);
          const bool fpair = pair && frow && lane <= it.halo + it.nout;
          const unsigned dp = d + (lane >> 1) * 4;
          cp4h_if<64>(dp + 128, ghin + c, N, pair);
          cp5h_if<64>(dp + 384, fhin + c, N, fpair);
          cp4h_if<64>(dp + 384 + 5 * 64, fhin + 5 * N + c, N, fpair);
          if (any_edge) {
            const int co = ym * nx + xo;
            const unsigned dq = d + 960 + (lane == 0 ? 0 : 20);
            cp1_if(dq, gin + co, outer);
            cp4h_if<4>(dq + 4, ghin + (co & ~1), N, outer);
          }
        }
      }
      cp_async_commit();
    };
#pragma unroll
    for (int j = 0; j < P; j++) stage(y0 - 3 + j, j);

    // per pipeline row of the own column: raw phi of rows R, R-1, R-2
    // (pr0..pr2), phi with ghosts of rows R-1, R-2, R-3 (pe0..pe2), kinds of
    // rows R .. R-3 (k0..k3), mapped rows R .. R-2 (m0..m2; -1 outside a
    // closed domain)
    float pr0 = 0.f, pr1 = 0.f, pr2 = 0.f, pe0 = 0.f, pe1 = 0.f, pe2 = 0.f;
    float px0 = 0.f, px1 = 0.f, px2 = 0.f;  // raw phi outside the strip (edge lanes)
    int k0 = 1, k1 = 1, k2 = 1, k3 = 1;
    int m0 = -1, m1 = -1, m2 = -1;
    // post-collision f_1..8 and moving g parts P_1..4 of row R-3 (cB); of
    // row R-4 only what the pull takes from it: f*_2, f*_5, f*_6, P_2 (cA);
    // rest f_0*, g_0* and stay parts (1-q) g_1..4 of row R-3 (oB)
    float cA[4], cB[12], oB[6];
#pragma unroll
    for (int i = 0; i < 4; i++) cA[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 12; i++) cB[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 6; i++) oB[i] = 0.f;
    // the new row's values: lanes that do not collide keep the last ones
    // (never read: their pulling neighbours bounce back)
    float cn[12], on[6];
#pragma unroll
    for (int i = 0; i < 12; i++) cn[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 6; i++) on[i] = 0.f;
    double acc_n = 0.0, acc_phi = 0.0, acc_mom = 0.0;
    int sl = 0;  // ring slot of row R

#pragma unroll 1
    for (int k = 0; k < ch + 6; k++) {
      const int R = y0 - 3 + k;
      {
        int sp = sl + P;
        if (sp >= D) sp -= D;  // the slot of row R+P is the slot of row R-3
        stage(R + P, sp);
      }
      cp_async_wait<P>();  // this lane's copies of row R have landed
      k3 = k2;
      k2 = k1;
      k1 = k0;
      m2 = m1;
      m1 = m0;
      pr2 = pr1;
      pr1 = pr0;
      px2 = px1;
      px1 = px0;
      pe2 = pe1;
      pe1 = pe0;
      {
        int ym;
        m0 = map_row_v(R, ny, bc, ym) ? ym : -1;
        k0 = m0 >= 0 ? row_kind(geom, ck, L, wt, m0) : 1;
        const float* sg = ring + sl * kRowW;
        pr0 = k0 == 0 ? ring_g(sg, 0) + ring_g(sg, 1) + ring_g(sg, 2) + ring_g(sg, 3) +
                            ring_g(sg, 4)
                      : 0.0f;
        px0 = edge && k0 != 0 && m0 >= 0 && row_kind(geom, cko, L, wt, m0) == 0
                  ? ring_outer(sg)
                  : 0.0f;
      }
      // ---- phi with wetting ghosts of row R-1
      pe0 = pr1;
      if (__any_sync(kFull, k1 != 0)) {
        float aW = __shfl_up_sync(kFull, pr0, 1), aE = __shfl_down_sync(kFull, pr0, 1);
        float bW = __shfl_up_sync(kFull, pr1, 1), bE = __shfl_down_sync(kFull, pr1, 1);
        float cW = __shfl_up_sync(kFull, pr2, 1), cE = __shfl_down_sync(kFull, pr2, 1);
        if (edge && lane == 0) {
          aW = px0;
          bW = px1;
          cW = px2;
        } else if (edge) {
          aE = px0;
          bE = px1;
          cE = px2;
        }
        if (k1 != 0) {
          // kinds of the neighbours in rows R (a), R-1 (b), R-2 (c)
          const int kaW = m0 >= 0 ? row_kind(geom, ckW, L, wt, m0) : 1;
          const int kaE = m0 >= 0 ? row_kind(geom, ckE, L, wt, m0) : 1;
          const int kbW = m1 >= 0 ? row_kind(geom, ckW, L, wt, m1) : 1;
          const int kbE = m1 >= 0 ? row_kind(geom, ckE, L, wt, m1) : 1;
          const int kcW = m2 >= 0 ? row_kind(geom, ckW, L, wt, m2) : 1;
          const int kcE = m2 >= 0 ? row_kind(geom, ckE, L, wt, m2) : 1;
          // mean over fluid face neighbours of phi + h_s / kappa, else the
          // plain mean over fluid diagonal neighbours
          const float h = k1 == 2 ? hk : 0.0f;
          float sum = 0.0f;
          int cnt = 0;
          if (kbE == 0) { sum += bE + h; cnt++; }
          if (k0 == 0) { sum += pr0 + h; cnt++; }
          if (kbW == 0) { sum += bW + h; cnt++; }
          if (k2 == 0) { sum += pr2 + h; cnt++; }
          if (cnt == 0) {
            if (kaE == 0) { sum += aE; cnt++; }
            if (kaW == 0) { sum += aW; cnt++; }
            if (kcW == 0) { sum += cW; cnt++; }
            if (kcE == 0) { sum += cE; cnt++; }
          }
          pe0 = cnt ? sum / (float)cnt : 0.0f;
        }
      }
      // ---- collision of row Rc = R-2 into cn / on
      const int Rc = R - 2;
      {
        const float nW = __shfl_up_sync(kFull, pe0, 1), nE = __shfl_down_sync(kFull, pe0, 1);
        const float cW = __shfl_up_sync(kFull, pe1, 1), cE = __shfl_down_sync(kFull, pe1, 1);
        const float sW = __shfl_up_sync(kFull, pe2, 1), sE = __shfl_down_sync(kFull, pe2, 1);
        // diagnostics of this cell: ink weight e, e n, e n u_y, n, phi, n u_y
        float dg[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        // Every lane runs the collision (no divergent branch, so the
        // collision and the streaming below form one block the compiler can
        // interleave); only lanes with a fluid cell that is pulled from
        // (cvalid) raise the flag or count in the diagnostics.  The results
        // of the other lanes are never read: a fluid cell pulling from a
        // solid one takes its own bounce-back value instead.
        const bool cvalid = col_lane && k2 == 0;
        if (k >= 4) {
          int s2 = sl - 2;
          if (s2 < 0) s2 += D;
          const float* sg = ring + s2 * kRowW;
          float g2[5], fr[9];
#pragma unroll
          for (int i = 0; i < 5; i++) g2[i] = ring_g(sg, i);
#pragma unroll
          for (int i = 0; i < 9; i++) fr[i] = ring_f(sg, i);
          const float pC = pe1;
          // lap = 6 sum_i w_i (phi_i - phi) from the differences, which are
          // exact where neighbours are close (no cancellation of O(10) terms)
          const float lap = (2.0f / 3.0f) * ((cE - pC) + (pe0 - pC) + (cW - pC) + (pe2 - pC)) +
                            (1.0f / 6.0f) * ((nE - pC) + (nW - pC) + (sW - pC) + (sE - pC));
          const float gx = (cE - cW) * (1.0f / 3.0f) + (nE - nW - sW + sE) * (1.0f / 12.0f);
          const float gy = (pe0 - pe2) * (1.0f / 3.0f) + (nE + nW - sW - sE) * (1.0f / 12.0f);
          const float phi = pr2;  // sum of g2 in the same order (raw phi of row R-2)
          const float mu = A4 * phi * ((phi - phis) * (phi + phis)) - kappa * lap;
          float C = 0.5f * (phi * inv_phis + 1.0f);
          C = fminf(fmaxf(C, 0.0f), 1.0f);
          const float Fb = (drive_col && m2 < L) || geom != GEOM_NOZZLE ? Fd * C : 0.0f;
          const float Fx = mu * gx, Fy = mu * gy + Fb;
          // fr holds deviations f_i - w_i n0: their sum is n - n0
          const float dn = fr[0] + fr[1] + fr[2] + fr[3] + fr[4] + fr[5] + fr[6] + fr[7] + fr[8];
          const float n = n0 + dn;
          const float mx = fr[1] - fr[3] + fr[5] - fr[6] - fr[7] + fr[8];
          const float my = fr[2] - fr[4] + fr[5] + fr[6] - fr[7] - fr[8];
          const float inv_n = __frcp_rn(n);  // 1 / n, correctly rounded
          const float ux = (mx + 0.5f * Fx) * inv_n, uy = (my + 0.5f * Fy) * inv_n;
          const float u2 = ux * ux + uy * uy;
          if (cvalid && !(u2 < 0.09f)) atomicOr(I.status, kStatusNumeric);
          const float om = __frcp_rn(0.5f + 3.0f * (nu_air + C * dnu));
          const float pref = 3.0f * (1.0f - 0.5f * om);
          // A_i - n0 = 3 (phi mu + n / 3) - n0 for i >= 1 (Eq. 6), on deviations
          const float p3 = dn + 3.0f * phi * mu;
          const float uF = ux * Fx + uy * Fy;
          const float base = -1.5f * u2;  // velocity-independent part of the bracket of Eq. 5
          // Moving directions first (deviations feq_i - w_i n0); the rest
          // direction then takes the balance, feq_0 - w_0 n0 = (n - n0) -
          // sum_{i>=1} (feq_i - w_i n0) and F_0 = -sum_{i>=1} F_i.  This equals
          // A_0 of Eq. 6 (the moments of Eq. 5-6 and of the forcing term are
          // exact) but conserves mass in FP32, whose rounded weights 4/9,
          // 1/9, 1/36 do not sum to one.  Opposite directions i, i' share the
          // even part of the equilibrium and of the forcing term and differ
          // in the sign of the odd part: feq = E +- O, F = FE +- FO with
          // E = w (p3 + n (base + 4.5 cu^2)), O = 3 w n cu,
          // FE = w pref (3 cu cF - uF), FO = w pref cF.  The collision
          // f* = (1 - om) f + om feq + F then reads f*_i = (1 - om) f_i + A +- B
          // with A = om E + FE and B = om O + FO.
          float fs[9];
          float sumA = 0.0f;
          const float omc = 1.0f - om, on3 = om * 3.0f * n;
#pragma unroll
          for (int i = 1; i < 9; i++) {
            if (i == 3 || i == 4 || i == 7 || i == 8) continue;  // handled with its pair
            const int ib = i == 1 ? 3 : (i == 2 ? 4 : (i == 5 ? 7 : 8));
            const float w = i < 5 ? W1 : W2;
            const float ex = (float)cEX(i), ey = (float)cEY(i);
            const float cu = ex * ux + ey * uy;
            const float cF = ex * Fx + ey * Fy;
            const float E = w * fmaf(n, fmaf(4.5f * cu, cu, base), p3);
            const float wp = w * pref;
            const float FE = wp * fmaf(3.0f * cu, cF, -uF);
            const float A = fmaf(om, E, FE);
            const float B = fmaf(w * on3, cu, wp * cF);
            sumA += A;
            fs[i] = fmaf(omc, fr[i], A + B);
            fs[ib] = fmaf(omc, fr[ib], A - B);
          }
          fs[0] = fmaf(omc, fr[0], fmaf(om, dn, -2.0f * sumA));
#pragma unroll
          for (int i = 1; i < 9; i++) cn[i - 1] = fs[i];
          // order parameter: Eq. 9-10 with the rest direction special; the
          // moving part q g_i + Omega_i streams, (1 - q) g_i stays
          const float gmu = gamma * mu;
          const float pq = phi * inv2q;
          float sum_ge = 0.0f;
#pragma unroll
          for (int i = 1; i < 5; i++) {
            const float cu = (float)cEX(i) * ux + (float)cEY(i) * uy;
            const float ge = 0.5f * gmu + pq * cu;
            sum_ge += ge;
            cn[7 + i] = fmaf(qmt, g2[i], ge * inv_tphi);  // q g + (ge - g) / tau_phi
            on[1 + i] = omq * g2[i];
          }
          // rest direction: g0_0 = phi - sum_{i>=1} g0_i (Eq. 10 as a
          // balance, so that sum g0 = phi exactly); with phi - g_0 =
          // sum_{i>=1} g_i the relaxation uses small terms only
          on[0] = fs[0];
          on[1] = g2[0] + ((g2[1] + g2[2] + g2[3] + g2[4]) - sum_ge) * inv_tphi;
          if (DIAG && cvalid && out_lane && Rc >= y0 && Rc < y0 + ch) {
            const float e = fminf(fmaxf(phi * inv_phis, 0.0f), 1.0f);
            dg[0] = e;
            dg[1] = e * n;
            dg[2] = dg[1] * uy;
            dg[3] = n;
            dg[4] = phi;
            dg[5] = n * uy;
          }
        }
        if (DIAG && k >= 4 && Rc >= y0 && Rc < y0 + ch) {
          // the strip's 28 cells of the row are summed in FP32, every
          // total across strips, rows and chunks in FP64
#pragma unroll
          for (int o = 16; o > 0; o >>= 1)
#pragma unroll
            for (int j = 0; j < 6; j++) dg[j] += __shfl_down_sync(kFull, dg[j], o);
          if (lane == 0) {
            atomicAdd(I.rows + Rc, (double)dg[0]);
            atomicAdd(I.rows + ny + Rc, (double)dg[1]);
            atomicAdd(I.rows + 2 * ny + Rc, (double)dg[2]);
            acc_n += (double)dg[3];
            acc_phi += (double)dg[4];
            acc_mom += (double)dg[5];
          }
        }
      }
      // ---- streaming of row Y = R-3: pull f_i(Y) = f*_i(Y - c_i) and
      // g_i(Y) = (1 - q) g_i(Y) + P_i(Y - c_i); rows Y-1 (cA), Y (cB), Y+1 (cn)
      {
        const float w1 = __shfl_up_sync(kFull, cB[0], 1), w5 = __shfl_up_sync(kFull, cA[1], 1);
        const float w8 = __shfl_up_sync(kFull, cn[7], 1), wP1 = __shfl_up_sync(kFull, cB[8], 1);
        const float e3 = __shfl_down_sync(kFull, cB[2], 1), e6 = __shfl_down_sync(kFull, cA[2], 1);
        const float e7 = __shfl_down_sync(kFull, cn[6], 1), eP3 = __shfl_down_sync(kFull, cB[10], 1);
        const bool svalid = out_lane && k3 == 0;
        if (k >= 6) {
          const int Y = R - 3;
          float fn[9];
          fn[0] = oB[0];
          fn[1] = w1;
          fn[2] = cA[0];
          fn[3] = e3;
          fn[4] = cn[3];
          fn[5] = w5;
          fn[6] = e6;
          fn[7] = e7;
          fn[8] = w8;
          float P1 = wP1, P2 = cA[3], P3 = eP3, P4 = cn[11];
          if (svalid && near_solid_v(geom, bc, ny, L, wt, colwall, Y)) {
            // halfway bounce-back: a population whose source is solid is the
            // cell's own post-collision population of the opposite direction
            const unsigned sm = solid_sources(I, x, Y);
            if (sm) {
              if (sm & (1u << 1)) { fn[1] = cB[2]; P1 = cB[10]; }
              if (sm & (1u << 2)) { fn[2] = cB[3]; P2 = cB[11]; }
              if (sm & (1u << 3)) { fn[3] = cB[0]; P3 = cB[8]; }
              if (sm & (1u << 4)) { fn[4] = cB[1]; P4 = cB[9]; }
              if (sm & (1u << 5)) fn[5] = cB[6];
              if (sm & (1u << 6)) fn[6] = cB[7];
              if (sm & (1u << 7)) fn[7] = cB[4];
              if (sm & (1u << 8)) fn[8] = cB[5];
            }
          }
          if (svalid && !H) {
            float* fo = fout + Y * nx + x;
            float* go = gout + Y * nx + x;
#pragma unroll
            for (int i = 0; i < 9; i++) fo[i * N] = fn[i];
            go[0] = oB[1];
            go[N] = oB[2] + P1;
            go[2 * N] = oB[3] + P2;
            go[3 * N] = oB[4] + P3;
            go[4 * N] = oB[5] + P4;
          } else if (svalid) {
            // round to nearest even on store
            __half* fo = fhout + Y * nx + x;
            __half* go = ghout + Y * nx + x;
#pragma unroll
            for (int i = 0; i < 9; i++) fo[i * N] = __float2half_rn(fn[i]);
            gout[Y * nx + x] = oB[1];
            go[0] = __float2half_rn(oB[2] + P1);
            go[N] = __float2half_rn(oB[3] + P2);
            go[2 * N] = __float2half_rn(oB[4] + P3);
            go[3 * N] = __float2half_rn(oB[5] + P4);
          }
        }
      }
      cA[0] = cB[1];  // f*_2
      cA[1] = cB[4];  // f*_5
      cA[2] = cB[5];  // f*_6
      cA[3] = cB[9];  // P_2
#pragma unroll
      for (int i = 0; i < 12; i++) cB[i] = cn[i];
#pragma unroll
      for (int i = 0; i < 6; i++) oB[i] = on[i];
      sl = sl + 1 == D ? 0 : sl + 1;
    }
    cp_async_wait<0>();  // no copy may land after the warp moves on
    if (DIAG && lane == 0) {
      atomicAdd(I.sums + 0, acc_n);
      atomicAdd(I.sums + 1, acc_phi);
      atomicAdd(I.sums + 2, acc_mom);
    }
  }
}

// ---------------------------------------------------------------------------
// Initialisation (FP64): phi_0 of the chosen profile into a temporary.
__device__ unsigned long long splitmix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__global__ void init_phi_kernel(const Inst* __restrict__ insts, int index, double* phi0) {
  const Inst& I = insts[index];
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= I.nx) return;
  double v = 0.0;
  if (geom_kind(I, x, y) == 0) {
    if (I.init_kind == INIT_MENISCUS) {
      int dx = max(I.cx0 - x, x - (I.cx1 - 1));
      if (dx <= 0) {
        v = I.d_phis * tanh((I.L - y) / I.d_W);
        if (fabs((double)(y - I.L)) < 2.0 * I.d_W) {
          unsigned long long ctr = ((unsigned long long)(unsigned)y << 32) | (unsigned)x;
          unsigned long long r = splitmix64(I.seed ^ splitmix64(ctr));
          double u = (double)(r >> 11) * (1.0 / 9007199254740992.0);
          v += I.jitter * (2.0 * u - 1.0);
        }
      } else if (y < I.L) {
        v = -I.d_phis;
      } else {
        double dy = (double)(y - I.L);
        v = I.d_phis * tanh(-sqrt((double)dx * dx + dy * dy) / I.d_W);
      }
    } else if (I.init_kind == INIT_DROP) {
      double ddx = x - I.init_x;
      ddx -= I.nx * floor(ddx / I.nx + 0.5);
      double ddy = y - I.init_y;
      v = I.d_phis * tanh((I.init_r - sqrt(ddx * ddx + ddy * ddy)) / I.d_W);
    } else if (I.init_kind == INIT_FLAT) {
      v = I.d_phis * tanh((I.init_y - y) / I.d_W);
    } else {
      v = I.init_r;
    }
  }
  phi0[(size_t)y * I.nx + x] = v;
}

__device__ double phi0_hat(const Inst& I, const double* phi0, int x, int y) {
  int k = kind_at(I, x, y);
  int ym = 0;
  if (k == 0) {
    map_row(I, y, ym);
    return phi0[(size_t)ym * I.nx + wrapi(x, I.nx)];
  }
  double hk = (k == 2) ? I.d_h / I.d_kappa : 0.0;
  const int fx[4] = {1, 0, -1, 0}, fy[4] = {0, 1, 0, -1};
  double sum = 0.0;
  int cnt = 0;
  for (int d = 0; d < 4; d++) {
    int xx = x + fx[d], yy = y + fy[d];
    if (kind_at(I, xx, yy) == 0) {
      map_row(I, yy, ym);
      sum += phi0[(size_t)ym * I.nx + wrapi(xx, I.nx)] + hk;
      cnt++;
    }
  }
  if (cnt) return sum / cnt;
  const int dx[4] = {1, -1, -1, 1}, dy[4] = {1, 1, -1, -1};
  for (int d = 0; d < 4; d++) {
    int xx = x + dx[d], yy = y + dy[d];
    if (kind_at(I, xx, yy) == 0) {
      map_row(I, yy, ym);
      sum += phi0[(size_t)ym * I.nx + wrapi(xx, I.nx)];
      cnt++;
    }
  }
  return cnt ? sum / cnt : 0.0;
}

// f = f^(0)(n0, u = 0), g = g^(0)(u = 0) with mu from phi_0 (FP64).
__global__ void init_pop_kernel(const Inst* __restrict__ insts, int index, const double* phi0) {
  const Inst& I = insts[index];
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= I.nx) return;
  const size_t N = (size_t)I.nx * I.ny, cc = (size_t)y * I.nx + x;
  float* f = I.f[0];  // deviations f_i - w_i n0
  float* g = I.g[0];
  // FP16 storage: f halves, g_0 FP32, g_1..4 halves after it
  __half* fh = reinterpret_cast<__half*>(f);
  __half* gh = reinterpret_cast<__half*>(g + N);
  auto put_f = [&](int i, float v) {
    if (I.fp16)
      fh[i * N + cc] = __float2half_rn(v);
    else
      f[i * N + cc] = v;
  };
  auto put_g = [&](int i, float v) {
    if (I.fp16 && i > 0)
      gh[(i - 1) * N + cc] = __float2half_rn(v);
    else
      g[i * N + cc] = v;
  };
  if (geom_kind(I, x, y) != 0) {
    for (int i = 0; i < 9; i++) put_f(i, 0.0f);
    for (int i = 0; i < 5; i++) put_g(i, 0.0f);
    return;
  }
  const double wt[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9,
                        1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
  const int ex[9] = {0, 1, 0, -1, 0, 1, -1, -1, 1}, ey[9] = {0, 0, 1, 0, -1, 1, 1, -1, -1};
  const double p0 = phi0[cc];
  double lap = 0.0;
  for (int i = 1; i < 9; i++) lap += 6.0 * wt[i] * (phi0_hat(I, phi0, x + ex[i], y + ey[i]) - p0);
  const double mu = 4.0 * I.d_A * p0 * (p0 * p0 - I.d_phis * I.d_phis) - I.d_kappa * lap;
  const double n = I.d_n0, p = p0 * mu + n / 3.0;
  for (int i = 0; i < 9; i++) {
    double Ai = i == 0 ? 2.25 * n - 3.75 * p : 3.0 * p;
    put_f(i, (float)(wt[i] * Ai - wt[i] * n));
  }
  put_g(0, (float)(p0 - 2.0 * I.d_gamma * mu));
  for (int i = 1; i < 5; i++) put_g(i, (float)(0.5 * I.d_gamma * mu));
}

__global__ void zero_kernel(float* a, size_t n) {
  size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  for (; i < n; i += (size_t)gridDim.x * blockDim.x) a[i] = 0.0f;
}

// ---------------------------------------------------------------------------
// Diagnostics record (FP64), one block of kFinThreads per lattice.  Each thread
// owns a contiguous range of rows; suffix sums, minima and run boundaries are
// combined across threads through shared memory.  The row accumulators are
// cleared for the next record.
constexpr int kFinThreads = 256;

__device__ double block_sum(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = kFinThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__device__ double block_min(double v, double* sh) {
  sh[threadIdx.x] = v;
  __syncthreads();
  for (int o = kFinThreads / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + o]);
    __syncthreads();
  }
  const double r = sh[0];
  __syncthreads();
  return r;
}

__global__ void __launch_bounds__(kFinThreads) finalize_kernel(const Inst* __restrict__ insts,
                                                              const long long* d_t) {
  __shared__ double sh[kFinThreads];
  __shared__ double suffix[kFinThreads + 1];
  const Inst& I = insts[blockIdx.x];
  const int ny = I.ny, tid = threadIdx.x;
  const double* w = I.rows;
  const double* m = I.rows + ny;
  const double* pr = I.rows + 2 * ny;
  const int per = (ny + kFinThreads - 1) / kFinThreads;
  const int ya = min(ny, tid * per), yb = min(ny, ya + per);
  // run ink of this thread's rows, then the run ink strictly above each thread
  double mine = 0.0;
  for (int y = ya; y < yb; y++)
    if (w[y] > 0.5) mine += w[y];
  sh[tid] = mine;
  __syncthreads();
  if (tid == 0) {
    suffix[kFinThreads] = 0.0;
    for (int k = kFinThreads - 1; k >= 0; k--) suffix[k] = suffix[k + 1] + sh[k];
  }
  __syncthreads();
  // neck: least w(y) over rows y >= y_scan with more than vmin of run ink above
  double above = suffix[tid + 1], neck = 1e30;
  for (int y = yb - 1; y >= ya; y--) {
    if (y >= I.y_scan && above > I.vmin && w[y] < neck) neck = w[y];
    if (w[y] > 0.5) above += w[y];
  }
  neck = block_min(neck, sh);
  // runs of rows with w > 1/2
  double starts = 0.0, starts_above = 0.0, last_start = -1.0;
  for (int y = ya; y < yb; y++)
    if (w[y] > 0.5 && (y == 0 || w[y - 1] <= 0.5)) {
      starts += 1.0;
      if (y >= I.y_exit) starts_above += 1.0;
      last_start = y;
    }
  const double nruns = block_sum(starts, sh);
  const double nabove = block_sum(starts_above, sh);
  const int lead0 = (int)(-block_min(-last_start, sh));
  double end = ny;
  if (lead0 >= 0)
    for (int y = max(ya, lead0 + 1); y < yb; y++)
      if (!(w[y] > 0.5)) {
        end = y;
        break;
      }
  const int lead1 = (int)block_min(end, sh);
  double vol = 0, ycm = 0, mm = 0, pp = 0;
  if (lead0 >= 0)
    for (int y = max(ya, lead0); y < min(yb, lead1); y++) {
      vol += w[y];
      ycm += y * w[y];
      mm += m[y];
      pp += pr[y];
    }
  vol = block_sum(vol, sh);
  ycm = block_sum(ycm, sh);
  mm = block_sum(mm, sh);
  pp = block_sum(pp, sh);
  if (tid == 0) {
    const double t = (double)*d_t;
    double* st = I.dstate;
    const double thr = 0.01;  // neck width at pinch-off, cells of ink
    if (st[3] < 0.0 && neck < thr) {
      if (st[0] > 0.0 && st[1] >= thr && st[1] < 1e29)
        st[3] = st[2] + (t - st[2]) * (st[1] - thr) / (st[1] - neck);
      else
        st[3] = t;
    }
    st[0] = 1.0;
    st[1] = neck;
    st[2] = t;
    const long long cnt = (long long)st[4];
    double* rec = I.hist + (cnt % kHistCap) * kRec;
    rec[0] = t;
    rec[1] = I.sums[0];
    rec[2] = I.sums[1];
    rec[3] = I.sums[2];
    rec[4] = neck;
    rec[5] = st[3];
    rec[6] = vol;
    rec[7] = vol > 0 ? ycm / vol : 0.0;
    rec[8] = mm > 0 ? pp / mm : 0.0;
    rec[9] = nabove > 1 ? nabove - 1 : 0;
    rec[10] = nruns;
    // head and tail of the leading run: where w crosses 1/2 at its ends,
    // interpolated between the last row inside and the first row outside
    rec[11] = rec[12] = -1.0;
    if (lead0 >= 0) {
      const int top = lead1 - 1;
      rec[11] = lead1 < ny ? top + (w[top] - 0.5) / (w[top] - w[lead1]) : (double)top;
      rec[12] = lead0 > 0 ? lead0 - (w[lead0] - 0.5) / (w[lead0] - w[lead0 - 1]) : (double)lead0;
    }
    st[4] = (double)(cnt + 1);
    I.sums[0] = I.sums[1] = I.sums[2] = I.sums[3] = 0.0;
  }
  __syncthreads();
  for (int y = tid; y < 3 * ny; y += kFinThreads) I.rows[y] = 0.0;
}

__global__ void advance_kernel(long long* d_t, int by) { *d_t += by; }

// phi = sum_i g_i of the current state (solid cells 0).
__global__ void phi_kernel(const Inst* __restrict__ insts, int index, const long long* d_t,
                           float* out) {
  const Inst& I = insts[index];
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= I.nx) return;
  const size_t N = (size_t)I.nx * I.ny, cc = (size_t)y * I.nx + x;
  const float* g = I.g[*d_t & 1];
  float p = 0.0f;
  if (geom_kind(I, x, y) == 0) {
    if (I.fp16) {
      const __half* gh = reinterpret_cast<const __half*>(g + N);
      p = g[cc];
      for (int i = 0; i < 4; i++) p += __half2float(gh[i * N + cc]);
    } else {
      for (int i = 0; i < 5; i++) p += g[i * N + cc];
    }
  }
  out[cc] = p;
}

// FP16 storage <-> absolute FP32 populations f [9][N], g [5][N] of the
// state at time parity `par` (solid cells 0); rounding to nearest on import.
template <bool EXPORT>
__global__ void convert16_kernel(const Inst* __restrict__ insts, int index, int par, float* f,
                                 float* g) {
  const Inst& I = insts[index];
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= I.nx) return;
  const size_t N = (size_t)I.nx * I.ny, cc = (size_t)y * I.nx + x;
  const bool fluid = geom_kind(I, x, y) == 0;
  __half* fh = reinterpret_cast<__half*>(I.f[par]);
  float* g0 = I.g[par];
  __half* gh = reinterpret_cast<__half*>(g0 + N);
  const float wt[9] = {4.0f / 9, 1.0f / 9, 1.0f / 9, 1.0f / 9, 1.0f / 9,
                       1.0f / 36, 1.0f / 36, 1.0f / 36, 1.0f / 36};
  if (EXPORT) {
    if (f)
      for (int i = 0; i < 9; i++)
        f[i * N + cc] = fluid ? __half2float(fh[i * N + cc]) + wt[i] * I.n0 : 0.0f;
    if (g) {
      g[cc] = fluid ? g0[cc] : 0.0f;
      for (int i = 1; i < 5; i++) g[i * N + cc] = fluid ? __half2float(gh[(i - 1) * N + cc]) : 0.0f;
    }
  } else {
    for (int i = 0; i < 9; i++)
      fh[i * N + cc] = __float2half_rn(fluid ? f[i * N + cc] - wt[i] * I.n0 : 0.0f);
    g0[cc] = fluid ? g[cc] : 0.0f;
    for (int i = 1; i < 5; i++) gh[(i - 1) * N + cc] = __float2half_rn(fluid ? g[i * N + cc] : 0.0f);
  }
}

// Stored deviations <-> absolute populations f_i = dev_i + w_i n0.
template <bool EXPORT>
__global__ void f_convert_kernel(const Inst* __restrict__ insts, int index, const float* src,
                                 float* dst) {
  const Inst& I = insts[index];
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y;
  if (x >= I.nx) return;
  const size_t N = (size_t)I.nx * I.ny, cc = (size_t)y * I.nx + x;
  const bool fluid = geom_kind(I, x, y) == 0;
  const float wt[9] = {4.0f / 9, 1.0f / 9, 1.0f / 9, 1.0f / 9, 1.0f / 9,
                       1.0f / 36, 1.0f / 36, 1.0f / 36, 1.0f / 36};
  for (int i = 0; i < 9; i++) {
    const float r = wt[i] * I.n0;
    dst[i * N + cc] = fluid ? (EXPORT ? src[i * N + cc] + r : src[i * N + cc] - r) : 0.0f;
  }
}

}  // namespace

// ---------------------------------------------------------------------------
size_t step_smem_bytes(int nthreads, int prefetch, bool h16) {
  return (size_t)(nthreads / 32) * (prefetch + 3) * (h16 ? kRowWordsH : kRowFloats) * sizeof(float);
}

size_t state_bytes_f(const Inst& I) { return (size_t)I.nx * I.ny * 9 * (I.fp16 ? 2 : 4); }
size_t state_bytes_g(const Inst& I) { return (size_t)I.nx * I.ny * (I.fp16 ? 12 : 20); }

cudaError_t launch_init(const Inst* d_inst, const Inst& h, int index, cudaStream_t s) {
  dim3 blk(128), grd((h.nx + 127) / 128, h.ny);
  double* phi0 = reinterpret_cast<double*>(h.f[1]);  // f[1] is free before the first step
  init_phi_kernel<<<grd, blk, 0, s>>>(d_inst, index, phi0);
  init_pop_kernel<<<grd, blk, 0, s>>>(d_inst, index, phi0);
  zero_kernel<<<256, 256, 0, s>>>(h.f[1], state_bytes_f(h) / 4);
  zero_kernel<<<256, 256, 0, s>>>(h.g[1], state_bytes_g(h) / 4);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const Inst* d_inst, int n_inst, const long long* d_t, cudaStream_t s) {
  finalize_kernel<<<n_inst, kFinThreads, 0, s>>>(d_inst, d_t);
  return cudaGetLastError();
}

cudaError_t launch_advance(long long* d_t, int by, cudaStream_t s) {
  advance_kernel<<<1, 1, 0, s>>>(d_t, by);
  return cudaGetLastError();
}

cudaError_t launch_phi(const Inst* d_inst, const Inst& h, int index, const long long* d_t,
                       float* out, cudaStream_t s) {
  dim3 blk(128), grd((h.nx + 127) / 128, h.ny);
  phi_kernel<<<grd, blk, 0, s>>>(d_inst, index, d_t, out);
  return cudaGetLastError();
}

cudaError_t launch_f_export(const Inst* d_inst, const Inst& h, int index, const float* src,
                            float* dst, cudaStream_t s) {
  dim3 blk(128), grd((h.nx + 127) / 128, h.ny);
  f_convert_kernel<true><<<grd, blk, 0, s>>>(d_inst, index, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_f_import(const Inst* d_inst, const Inst& h, int index, const float* src,
                            float* dst, cudaStream_t s) {
  dim3 blk(128), grd((h.nx + 127) / 128, h.ny);
  f_convert_kernel<false><<<grd, blk, 0, s>>>(d_inst, index, src, dst);
  return cudaGetLastError();
}

cudaError_t launch_convert16(const Inst* d_inst, const Inst& h, int index, int parity, float* f,
                             float* g, bool to_device_state, cudaStream_t s) {
  dim3 blk(128), grd((h.nx + 127) / 128, h.ny);
  if (to_device_state)
    convert16_kernel<false><<<grd, blk, 0, s>>>(d_inst, index, parity, f, g);
  else
    convert16_kernel<true><<<grd, blk, 0, s>>>(d_inst, index, parity, f, g);
  return cudaGetLastError();
}

template <bool DIAG, bool H>
cudaError_t launch_step_p(const Inst* d_inst, const Item* d_items, int n_items, int nthreads,
                          int grid, const long long* d_t, int t_off, int prefetch, size_t smem,
                          cudaStream_t s) {
  switch (prefetch) {
    case 1:
      step_kernel<DIAG, 1, H><<<grid, nthreads, smem, s>>>(d_inst, d_items, n_items, d_t, t_off);
      break;
    case 2:
      step_kernel<DIAG, 2, H><<<grid, nthreads, smem, s>>>(d_inst, d_items, n_items, d_t, t_off);
      break;
    case 3:
      step_kernel<DIAG, 3, H><<<grid, nthreads, smem, s>>>(d_inst, d_items, n_items, d_t, t_off);
      break;
    default:
      step_kernel<DIAG, 4, H><<<grid, nthreads, smem, s>>>(d_inst, d_items, n_items, d_t, t_off);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_step(const Inst* d_inst, const Item* d_items, int n_items, int nthreads,
                        int grid, const long long* d_t, int t_off, bool diag, int prefetch,
                        bool h16, cudaStream_t s) {
  if (nthreads != kStepThreads || prefetch < 1 || prefetch > kMaxPrefetch)
    return cudaErrorInvalidValue;
  if (n_items <= 0) return cudaSuccess;
  const size_t smem = step_smem_bytes(nthreads, prefetch, h16);
  if (h16)
    return diag ? launch_step_p<true, true>(d_inst, d_items, n_items, nthreads, grid, d_t, t_off,
                                            prefetch, smem, s)
                : launch_step_p<false, true>(d_inst, d_items, n_items, nthreads, grid, d_t, t_off,
                                             prefetch, smem, s);
  return diag ? launch_step_p<true, false>(d_inst, d_items, n_items, nthreads, grid, d_t, t_off,
                                           prefetch, smem, s)
              : launch_step_p<false, false>(d_inst, d_items, n_items, nthreads, grid, d_t, t_off,
                                            prefetch, smem, s);
}

int step_prefetch_for(int) { return 3; }

cudaError_t set_step_smem_limit() {
  const int lim = (int)step_smem_bytes(kStepThreads, kMaxPrefetch, false);
  cudaError_t e = cudaSuccess;
#define SET_LIM(DG, PF)                                                                         \
  if (e == cudaSuccess)                                                                         \
    e = cudaFuncSetAttribute(step_kernel<DG, PF, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             lim);                                                              \
  if (e == cudaSuccess)                                                                         \
    e = cudaFuncSetAttribute(step_kernel<DG, PF, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             lim);
  SET_LIM(true, 1) SET_LIM(false, 1) SET_LIM(true, 2) SET_LIM(false, 2)
  SET_LIM(true, 3) SET_LIM(false, 3) SET_LIM(true, 4) SET_LIM(false, 4)
#undef SET_LIM
  return e;
}

int make_items_range(const Inst& I, int k, int chunk, int ya, int yb, Item* out, int cap) {
  constexpr int halo = 2, W = 32 - 2 * halo;  // 28 written columns per strip
  const int nstrip = (I.nx + W - 1) / W;
  int n = 0;
  for (int y0 = ya; y0 < yb; y0 += chunk)
    for (int s = 0; s < nstrip; s++) {
      if (n >= cap) return -1;
      Item& it = out[n++];
      it.inst = k;
      it.xs = s * W;
      it.nout = I.nx - s * W < W ? I.nx - s * W : W;
      it.halo = halo;
      it.y0 = y0;
      it.ch = yb - y0 < chunk ? yb - y0 : chunk;
    }
  return n;
}

int make_items(const Inst& I, int k, int chunk, Item* out, int cap) {
  return make_items_range(I, k, chunk, 0, I.ny, out, cap);
}

int items_per_range(const Inst& I, int chunk, int ya, int yb) {
  return yb > ya ? ((I.nx + 27) / 28) * ((yb - ya + chunk - 1) / chunk) : 0;
}

int items_per_lattice(const Inst& I, int chunk) { return items_per_range(I, chunk, 0, I.ny); }

}  // namespace ij
