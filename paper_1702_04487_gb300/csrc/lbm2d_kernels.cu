// Kernels of the 2-D binary-fluid lattice Boltzmann inkjet step
// (He et al., arXiv:1702.04487, "Methods", Eq. 3-10).
//
// Step kernel design (bandwidth-bound stencil, no tensor cores):
//  - one thread per lattice column; a block owns a strip of columns and a
//    chunk of rows and marches up the rows, so every cell's populations are
//    read once and written once per step (structure-of-arrays, coalesced);
//  - per row iteration, four pipelined stages over shared-memory ring
//    buffers of three rows: (1) phi = sum g of row R, (2) wetting ghost
//    values of row R-1, (3) chemical potential, forces, velocity and the
//    collision of f (Eq. 4-6) and g (Eq. 8-10) on row R-2, (4) streaming of
//    row R-3 with halfway bounce-back and the stay/move split of Eq. 8;
//  - geometry is analytic (no mask array) and the x-halo of a strip is
//    recomputed by its two edge threads;
//  - diagnostics rows (ink weight, mass, momentum) are reduced in FP64 by
//    warp shuffles and atomics inside the same pass on diagnostics steps.
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

// Conservative test: may a fluid cell (x, y) have a solid neighbour?
__device__ __forceinline__ bool near_solid(const Inst& I, bool colwall, int y) {
  if (I.bc == BC_CLOSED && (y == 0 || y == I.ny - 1)) return true;
  if (I.geom == GEOM_NOZZLE) {
    if (!colwall) return false;
    if (I.bc == BC_PER && (y == 0 || y == I.ny - 1)) return true;
    return y - 1 < I.L;
  }
  if (I.geom == GEOM_PLATE) {
    if (I.bc == BC_PER && (y == 0 || y == I.ny - 1)) return true;
    return y - 1 < I.wt;
  }
  return false;
}

__device__ __forceinline__ bool in_drive(const Inst& I, int x, int ym) {
  if (I.geom == GEOM_NOZZLE) return x >= I.cx0 && x < I.cx1 && ym < I.L;
  return true;
}

// Fig. 1 waveform: +F0, then -F_neg, then idle (periodic if T_idle > 0).
__device__ __forceinline__ float drive_at(const Inst& I, long long t) {
  long long tt = t;
  if (I.Tidle > 0) tt = t % (I.T1 + I.T2 + I.Tidle);
  if (tt < I.T1) return I.F0;
  if (tt < I.T1 + I.T2) return -I.Fneg;
  return 0.0f;
}

// Wetting ghost value of a solid point from a 3x3 window of phi (centre
// w[4], rows w[0..2] below, w[6..8] above) and the kinds of its neighbours:
// the mean over fluid face neighbours of phi + h_s / kappa, else the mean
// over fluid diagonal neighbours.
__device__ __noinline__ float ghost_rule(const Inst& I, int kind, int x, int y, const float* w) {
  float hk = (kind == 2) ? I.hk : 0.0f;
  const int fx[4] = {1, 0, -1, 0}, fy[4] = {0, 1, 0, -1};
  float sum = 0.0f;
  int cnt = 0;
  for (int d = 0; d < 4; d++)
    if (kind_at(I, x + fx[d], y + fy[d]) == 0) {
      sum += w[(fy[d] + 1) * 3 + fx[d] + 1] + hk;
      cnt++;
    }
  if (cnt) return sum / (float)cnt;
  const int dx[4] = {1, -1, -1, 1}, dy[4] = {1, 1, -1, -1};
  for (int d = 0; d < 4; d++)
    if (kind_at(I, x + dx[d], y + dy[d]) == 0) {
      sum += w[(dy[d] + 1) * 3 + dx[d] + 1];
      cnt++;
    }
  return cnt ? sum / (float)cnt : 0.0f;
}

// Asynchronous 4-byte global -> shared copies (cp.async), grouped per row.
__device__ __forceinline__ void cp_async4(float* dst, const float* src) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(src) : "memory");
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

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
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
// The fused step.  Shared memory per block (NT = blockDim.x, D = P + 3):
//   ring[D] rows of populations staged by cp.async, P rows ahead of use:
//           g[5][NT+4] (slot j <-> column xs+j-2) and f[9][NT] (slot c <-> xs+c)
//   raw[4][NT+4]  phi of rows R..R-3 (ring), slot j <-> column xs+j-2
//   gh [3][NT+2]  phi with ghost values, slot j <-> column xs+j-1
//   col[3][12][NT] post-collision f_1..8 and moving g parts P_1..4
//   red[NT/32][3] diagnostics partial sums (FP64)
template <bool DIAG, int P>
__global__ void __launch_bounds__(256, 2) step_kernel(const Inst* __restrict__ insts,
                                                      const Item* __restrict__ items, int n_items,
                                                      const long long* __restrict__ d_t, int t_off) {
  constexpr int D = P + 3;
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  const int NT = blockDim.x;
  const int c = threadIdx.x;
  const int GW = NT + 4, RS = 5 * GW + 9 * NT;  // g row width, ring slot size (floats)
  float* ring = smem;
  float* raw = ring + D * RS;
  float* gh = raw + 4 * (NT + 4);
  float* col = gh + 3 * (NT + 2);
  double* red = reinterpret_cast<double*>(col + 36 * NT);
  const long long t = *d_t + t_off;

  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const Item it = items[item];
    const Inst& I = insts[it.inst];
    // a lattice whose numeric flag is set is frozen; thread 0 reads the flag
    // and the barrier-reduction makes the decision uniform across the block
    if (__syncthreads_or(c == 0 ? (int)*(volatile unsigned*)I.status : 0)) continue;
    // per-lattice constants in registers
    const int nx = I.nx, ny = I.ny, geom = I.geom, L = I.L, wt = I.wt, bc = I.bc;
    const int wc = it.wc, y0 = it.y0, ch = it.ch;
    const int N = nx * ny;  // < 2^31 / 9 (checked on the host)
#define phis2 (I.phis * I.phis)
#define inv_phis (I.inv_phis)
#define A4 (I.A4)
#define kappa (I.kappa)
#define qf (I.q)
#define omq (I.omq)
#define inv_tphi (I.inv_tphi)
#define gamma (I.gamma)
#define inv2q (I.inv2q)
#define nu_air (I.nu_air)
#define dnu (I.dnu)
#define n0 (I.n0)
    const float* __restrict__ fin = I.f[t & 1];
    const float* __restrict__ gin = I.g[t & 1];
    float* __restrict__ fout = I.f[(t + 1) & 1];
    float* __restrict__ gout = I.g[(t + 1) & 1];
    const float Fd = drive_at(I, t);
    const bool active = c < wc;
    const int x = wrapi(it.xs + c, nx);
    const bool owned = active && (it.single || (c >= 1 && c <= wc - 2 && it.xs + c < nx));
    const int xe = (c < 2) ? c : wc + c;  // extra raw slot of threads 0..3
    const int xex = wrapi(it.xs + xe - 2, nx);
    const int xg = (c == 0) ? 0 : wc + 1;  // extra ghost slot of threads 0..1
    const int xgx = wrapi(it.xs + xg - 1, nx);
    const int ck = column_kind(I, x), cke = column_kind(I, xex), ckg = column_kind(I, xgx);
    const bool drive_col = geom != GEOM_NOZZLE || (x >= I.cx0 && x < I.cx1);
    // does the strip (with its halo) contain a nozzle-wall column?  Rows with
    // no solid cell in the strip need no ghost values: their phi is used as is
    bool strip_wall = false;
    if (geom == GEOM_NOZZLE) {
      const int a0 = I.cx0 - I.wt, b1 = I.cx1 + I.wt;
      if (it.single) {
        strip_wall = true;
      } else {
        for (int j = -2; j < wc + 2 && !strip_wall; j++) {
          const int xx = wrapi(it.xs + j, nx);
          strip_wall = xx >= a0 && xx < b1 && column_kind(I, xx) != 0;
        }
      }
    }
    bool colwall = false;
    if (geom == GEOM_NOZZLE)
      colwall = ck != 0 || column_kind(I, wrapi(x - 1, nx)) != 0 ||
                column_kind(I, wrapi(x + 1, nx)) != 0;

    // rotating per-row state of the own column: kinds of rows R..R-3, mapped
    // rows of R..R-2
    int k0 = 1, k1 = 1, k2 = 1, k3 = 1;
    int m0 = 0, m1 = 0, m2 = 0;
    // block-uniform: does pipeline row R, R-1, R-2, R-3 hold a solid cell?
    bool h0 = true, h1 = true, h2 = true, h3 = true;
    int keR = 1;  // kind of the extra raw column (threads 0..3) in row R
    // Stage the populations of pipeline row r into ring slot `slot` (own
    // column; the g halo columns by threads 0..3; f only for rows that are
    // collided), as one cp.async group.
    auto stage_row = [&](int r, int slot) {
      int ym;
      const bool in = r <= y0 + ch + 2 && map_row(I, r, ym);
      if (in) {
        float* sg = ring + slot * RS;
        const int off = ym * nx;
        if (active && row_kind(geom, ck, L, wt, ym) == 0) {
          const float* q = gin + off + x;
#pragma unroll
          for (int i = 0; i < 5; i++) cp_async4(sg + i * GW + c + 2, q + i * N);
          if (r >= y0 - 1 && r <= y0 + ch) {
            const float* qf_ = fin + off + x;
            float* sf = sg + 5 * GW;
#pragma unroll
            for (int i = 0; i < 9; i++) cp_async4(sf + i * NT + c, qf_ + i * N);
          }
        }
        if (c < 4 && row_kind(geom, cke, L, wt, ym) == 0) {
          const float* q = gin + off + xex;
#pragma unroll
          for (int i = 0; i < 5; i++) cp_async4(sg + i * GW + xe, q + i * N);
        }
      }
      cp_async_commit();
    };
    int rs0 = 0;  // ring slot of row R
#pragma unroll
    for (int j = 0; j < P; j++) stage_row(y0 - 3 + j, j);
    // own post-collision values kept for the next iteration's pull
    float cf0 = 0.f, cG0 = 0.f, cS0 = 0.f, cS1 = 0.f, cS2 = 0.f, cS3 = 0.f;
    double acc_n = 0.0, acc_phi = 0.0, acc_mom = 0.0;
    // ring slots of pipeline rows R (s0), R-1 (s1), R-2 (s2) for gh and col;
    // raw keeps four rows: R (r0), R-1 (r1), R-2 (r2), R-3 (r3)
    int s0 = 0, s1 = 2, s2 = 1;
    int r0 = 0, r1 = 3, r2 = 2, r3 = 1;

    for (int k = 0; k < ch + 6; k++) {
      const int R = y0 - 3 + k;
      // ---------------- stage 1: phi of row R (staged P iterations ago)
      {
        int slot = rs0 + P;
        if (slot >= D) slot -= D;  // slot of row R+P, last used by row R-3
        stage_row(R + P, slot);
      }
      cp_async_wait<P>();  // this thread's copies of row R have landed
      k3 = k2;
      k2 = k1;
      k1 = k0;
      m2 = m1;
      m1 = m0;
      h3 = h2;
      h2 = h1;
      h1 = h0;
      {
        int ym;
        const bool in = map_row(I, R, ym);
        m0 = ym;
        h0 = !in || (geom == GEOM_NOZZLE && strip_wall && ym < L) || (geom == GEOM_PLATE && ym < wt);
        k0 = in ? row_kind(geom, ck, L, wt, ym) : 1;
        const float* sg = ring + rs0 * RS;
        if (active)
          raw[r0 * (NT + 4) + c + 2] =
              k0 == 0 ? sg[c + 2] + sg[GW + c + 2] + sg[2 * GW + c + 2] + sg[3 * GW + c + 2] +
                            sg[4 * GW + c + 2]
                      : 0.0f;
        if (c < 4) {
          keR = in ? row_kind(geom, cke, L, wt, ym) : 1;
          raw[r0 * (NT + 4) + xe] =
              keR == 0 ? sg[xe] + sg[GW + xe] + sg[2 * GW + xe] + sg[3 * GW + xe] + sg[4 * GW + xe]
                       : 0.0f;
        }
      }
      int rs2 = rs0 - 2;  // ring slot of row R-2
      if (rs2 < 0) rs2 += D;
      __syncthreads();
      // ---------------- stage 2: ghost values of row R-1 (rows with solids)
      if (k >= 2 && h1) {
        const float* ra = raw + r2 * (NT + 4);  // row R-2
        const float* rb = raw + r1 * (NT + 4);  // row R-1
        const float* rc = raw + r0 * (NT + 4);  // row R
        float* go = gh + s1 * (NT + 2);
        if (active) {
          const int j = c + 1;
          float v;
          if (k1 == 0) {
            v = rb[j + 1];
          } else {
            float w[9] = {ra[j], ra[j + 1], ra[j + 2], rb[j], rb[j + 1], rb[j + 2],
                          rc[j], rc[j + 1], rc[j + 2]};
            v = ghost_rule(I, k1, x, R - 1, w);
          }
          go[j] = v;
        }
        if (c < 2) {
          const int j = xg;
          int ym;
          const int kk = map_row(I, R - 1, ym) ? row_kind(geom, ckg, L, wt, ym) : 1;
          float v;
          if (kk == 0) {
            v = rb[j + 1];
          } else {
            float w[9] = {ra[j], ra[j + 1], ra[j + 2], rb[j], rb[j + 1], rb[j + 2],
                          rc[j], rc[j + 1], rc[j + 2]};
            v = ghost_rule(I, kk, xgx, R - 1, w);
          }
          go[j] = v;
        }
        __syncthreads();
      }
      // ---------------- stage 3: collision of row R-2
      const float pf0 = cf0, pG0 = cG0, pS0 = cS0, pS1 = cS1, pS2 = cS2, pS3 = cS3;
      double dw = 0.0, dm = 0.0, dp = 0.0;
      const int Rc = R - 2;
      if (k >= 4 && active && k2 == 0) {
        const float* sg2 = ring + rs2 * RS;  // g and f of row Rc, own column
        float g2[5], fr[9];
#pragma unroll
        for (int i = 0; i < 5; i++) g2[i] = sg2[i * GW + c + 2];
#pragma unroll
        for (int i = 0; i < 9; i++) fr[i] = sg2[5 * GW + i * NT + c];
        // phi with ghosts of rows Rc-1 (slot of R-3 = slot of R), Rc, Rc+1;
        // a row without solid cells is read from raw (one column shifted)
        const float* hb = h3 ? gh + s0 * (NT + 2) : raw + r3 * (NT + 4) + 1;
        const float* hc = h2 ? gh + s2 * (NT + 2) : raw + r2 * (NT + 4) + 1;
        const float* ht = h1 ? gh + s1 * (NT + 2) : raw + r1 * (NT + 4) + 1;
        const int j = c + 1;
        const float pC = hc[j];
        const float pE = hc[j + 1], pW = hc[j - 1], pN = ht[j], pS = hb[j];
        const float pNE = ht[j + 1], pNW = ht[j - 1], pSW = hb[j - 1], pSE = hb[j + 1];
        // lap = 6 sum_i w_i (phi_i - phi) from the differences, which are
        // exact where neighbours are close (no cancellation of O(10) terms)
        const float lap = (2.0f / 3.0f) * ((pE - pC) + (pN - pC) + (pW - pC) + (pS - pC)) +
                          (1.0f / 6.0f) * ((pNE - pC) + (pNW - pC) + (pSW - pC) + (pSE - pC));
        const float gx = (pE - pW) * (1.0f / 3.0f) + (pNE - pNW - pSW + pSE) * (1.0f / 12.0f);
        const float gy = (pN - pS) * (1.0f / 3.0f) + (pNE + pNW - pSW - pSE) * (1.0f / 12.0f);
        const float phi = g2[0] + g2[1] + g2[2] + g2[3] + g2[4];
        const float mu = A4 * phi * ((phi - I.phis) * (phi + I.phis)) - kappa * lap;
        float C = 0.5f * (phi * inv_phis + 1.0f);
        C = fminf(fmaxf(C, 0.0f), 1.0f);
        const float Fb = (drive_col && m2 < L) || geom != GEOM_NOZZLE ? Fd * C : 0.0f;
        const float Fx = mu * gx, Fy = mu * gy + Fb;
        // fr holds deviations f_i - w_i n0: their sum is n - n0
        const float dn = fr[0] + fr[1] + fr[2] + fr[3] + fr[4] + fr[5] + fr[6] + fr[7] + fr[8];
        const float n = n0 + dn;
        const float mx = fr[1] - fr[3] + fr[5] - fr[6] - fr[7] + fr[8];
        const float my = fr[2] - fr[4] + fr[5] + fr[6] - fr[7] - fr[8];
        const float inv_n = 1.0f / n;
        const float ux = (mx + 0.5f * Fx) * inv_n, uy = (my + 0.5f * Fy) * inv_n;
        const float u2 = ux * ux + uy * uy;
        if (!(u2 < 0.09f)) atomicOr(I.status, kStatusNumeric);
        const float om = 1.0f / (0.5f + 3.0f * (nu_air + C * dnu));
        const float pref = 3.0f * (1.0f - 0.5f * om);
        // A_i - n0 = 3 (phi mu + n / 3) - n0 for i >= 1 (Eq. 6), on deviations
        const float p3 = dn + 3.0f * phi * mu;
        const float uF = ux * Fx + uy * Fy;
        const float base = -1.5f * u2;  // velocity-independent part of the bracket of Eq. 5
        // Moving directions first (deviations feq_i - w_i n0); the rest
        // direction then takes the balance, feq_0 - w_0 n0 = (n - n0) -
        // sum_{i>=1} (feq_i - w_i n0) and F_0 = -sum_{i>=1} F_i.  This equals
        // A_0 = 9n/4 - 15 p / 4 of Eq. 6 (the moments of Eq. 5-6 and of the
        // forcing term are exact) but conserves mass in FP32, whose rounded
        // weights 4/9, 1/9, 1/36 do not sum to one.
        // Opposite directions i, i' share the even part of the equilibrium
        // and of the forcing term and differ in the sign of the odd part:
        // feq = E +- O, F = FE +- FO with E = w (p3 + n (base + 4.5 cu^2)),
        // O = 3 w n cu, FE = w pref (3 cu cF - uF), FO = w pref cF.
        float fs[9];
        float sum_eq = 0.0f, sum_F = 0.0f;
        const float n3 = 3.0f * n;
#pragma unroll
        for (int i = 1; i < 9; i++) {
          if (i == 3 || i == 4 || i == 7 || i == 8) continue;  // handled with its pair
          const int ib = i == 1 ? 3 : (i == 2 ? 4 : (i == 5 ? 7 : 8));
          const float w = i < 5 ? W1 : W2;
          const float ex = (float)cEX(i), ey = (float)cEY(i);
          const float cu = ex * ux + ey * uy;
          const float cF = ex * Fx + ey * Fy;
          const float E = w * (p3 + n * (base + 4.5f * cu * cu));
          const float O = (w * n3) * cu;
          const float wp = w * pref;
          const float FE = wp * (3.0f * cu * cF - uF);
          const float FO = wp * cF;
          sum_eq += 2.0f * E;
          sum_F += 2.0f * FE;
          fs[i] = fr[i] + om * ((E + O) - fr[i]) + (FE + FO);
          fs[ib] = fr[ib] + om * ((E - O) - fr[ib]) + (FE - FO);
        }
        fs[0] = fr[0] + om * ((dn - sum_eq) - fr[0]) - sum_F;
        // order parameter: Eq. 9-10 with the rest direction special
        const float gmu = gamma * mu;
        const float pq = phi * inv2q;
        float* cl = col + s2 * 12 * NT;
#pragma unroll
        for (int i = 1; i < 9; i++) cl[(i - 1) * NT + c] = fs[i];
        float sum_ge = 0.0f;
        float S[4];
#pragma unroll
        for (int i = 1; i < 5; i++) {
          const float cu = (float)cEX(i) * ux + (float)cEY(i) * uy;
          const float ge = 0.5f * gmu + pq * cu;
          sum_ge += ge;
          const float omi = (ge - g2[i]) * inv_tphi;
          cl[(7 + i) * NT + c] = qf * g2[i] + omi;
          S[i - 1] = omq * g2[i];
        }
        cS0 = S[0];
        cS1 = S[1];
        cS2 = S[2];
        cS3 = S[3];
        // rest direction: g0_0 = phi - 2 Gamma mu (Eq. 10), taken as the
        // balance phi - sum_{i>=1} g0_i so that sum g0 = phi exactly; with
        // phi - g_0 = sum_{i>=1} g_i the relaxation uses small terms only
        // (no difference of two rounded values of size phi*)
        const float om0 = ((g2[1] + g2[2] + g2[3] + g2[4]) - sum_ge) * inv_tphi;
        cf0 = fs[0];
        cG0 = g2[0] + om0;
        if (DIAG && owned && Rc >= y0 && Rc < y0 + ch) {
          const float e = fminf(fmaxf(phi * inv_phis, 0.0f), 1.0f);
          dw = (double)e;
          dm = (double)e * (double)n;
          dp = dm * (double)uy;
          acc_n += (double)n;
          acc_phi += (double)phi;
          acc_mom += (double)n * (double)uy;
        }
      }
      if (DIAG && k >= 4 && Rc >= y0 && Rc < y0 + ch) {
        dw = warp_sum(dw);
        dm = warp_sum(dm);
        dp = warp_sum(dp);
        if ((c & 31) == 0) {
          red[(c >> 5) * 3 + 0] = dw;
          red[(c >> 5) * 3 + 1] = dm;
          red[(c >> 5) * 3 + 2] = dp;
        }
      }
      __syncthreads();
      if (DIAG && c == 0 && k >= 4 && Rc >= y0 && Rc < y0 + ch) {
        double sw = 0, sm = 0, sp = 0;
        for (int wq = 0; wq < NT / 32; wq++) {
          sw += red[wq * 3 + 0];
          sm += red[wq * 3 + 1];
          sp += red[wq * 3 + 2];
        }
        atomicAdd(I.rows + Rc, sw);
        atomicAdd(I.rows + ny + Rc, sm);
        atomicAdd(I.rows + 2 * ny + Rc, sp);
      }
      // ---------------- stage 4: streaming of row R-3
      if (k >= 6 && owned && k3 == 0) {
        const int Y = R - 3;
        const float* cb = col + s1 * 12 * NT;  // row Y-1 (slot of R-4 = slot of R-1)
        const float* cm = col + s0 * 12 * NT;  // row Y   (slot of R-3 = slot of R)
        const float* ct = col + s2 * 12 * NT;  // row Y+1 (slot of R-2)
        const int cw = it.single ? (c == 0 ? wc - 1 : c - 1) : c - 1;
        const int ce = it.single ? (c == wc - 1 ? 0 : c + 1) : c + 1;
        float fn[9];
        fn[0] = pf0;
        // pull f_i(Y) = f*_i(Y - c_i); g_i(Y) = (1-q) g_i(Y) + P_i(Y - c_i)
        fn[1] = cm[0 * NT + cw];
        fn[2] = cb[1 * NT + c];
        fn[3] = cm[2 * NT + ce];
        fn[4] = ct[3 * NT + c];
        fn[5] = cb[4 * NT + cw];
        fn[6] = cb[5 * NT + ce];
        fn[7] = ct[6 * NT + ce];
        fn[8] = ct[7 * NT + cw];
        float P1 = cm[8 * NT + cw], P2 = cb[9 * NT + c], P3 = cm[10 * NT + ce], P4 = ct[11 * NT + c];
        if (near_solid(I, colwall, Y)) {
          // halfway bounce-back: a population whose source is solid is the
          // cell's own post-collision population of the opposite direction
          const unsigned sm = solid_sources(I, x, Y);
          if (sm) {
            if (sm & (1u << 1)) { fn[1] = cm[2 * NT + c]; P1 = cm[10 * NT + c]; }
            if (sm & (1u << 2)) { fn[2] = cm[3 * NT + c]; P2 = cm[11 * NT + c]; }
            if (sm & (1u << 3)) { fn[3] = cm[0 * NT + c]; P3 = cm[8 * NT + c]; }
            if (sm & (1u << 4)) { fn[4] = cm[1 * NT + c]; P4 = cm[9 * NT + c]; }
            if (sm & (1u << 5)) fn[5] = cm[6 * NT + c];
            if (sm & (1u << 6)) fn[6] = cm[7 * NT + c];
            if (sm & (1u << 7)) fn[7] = cm[4 * NT + c];
            if (sm & (1u << 8)) fn[8] = cm[5 * NT + c];
          }
        }
        float* fo = fout + Y * nx + x;
        float* go = gout + Y * nx + x;
#pragma unroll
        for (int i = 0; i < 9; i++) fo[i * N] = fn[i];
        go[0] = pG0;
        go[N] = pS0 + P1;
        go[2 * N] = pS1 + P2;
        go[3 * N] = pS2 + P3;
        go[4 * N] = pS3 + P4;
      }
      // rotate the ring slots: the slot of R-2 becomes the slot of R+1
      const int sn = s2;
      s2 = s1;
      s1 = s0;
      s0 = sn;
      rs0 = rs0 + 1 == D ? 0 : rs0 + 1;
      const int rn = r3;
      r3 = r2;
      r2 = r1;
      r1 = r0;
      r0 = rn;
    }
    cp_async_wait<0>();  // no copy may land after the block moves on
    if (DIAG) {
      // lattice sums of this item, one atomic per warp (every lane of the
      // block takes part; the block size is a multiple of 32)
      double a = warp_sum(acc_n), b = warp_sum(acc_phi), m = warp_sum(acc_mom);
      if ((c & 31) == 0) {
        atomicAdd(I.sums + 0, a);
        atomicAdd(I.sums + 1, b);
        atomicAdd(I.sums + 2, m);
      }
    }
    __syncthreads();
  }
}

#undef phis2
#undef inv_phis
#undef A4
#undef kappa
#undef qf
#undef omq
#undef inv_tphi
#undef gamma
#undef inv2q
#undef nu_air
#undef dnu
#undef n0

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
  if (geom_kind(I, x, y) != 0) {
    for (int i = 0; i < 9; i++) f[i * N + cc] = 0.0f;
    for (int i = 0; i < 5; i++) g[i * N + cc] = 0.0f;
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
    f[i * N + cc] = (float)(wt[i] * Ai - wt[i] * n);
  }
  g[cc] = (float)(p0 - 2.0 * I.d_gamma * mu);
  for (int i = 1; i < 5; i++) g[i * N + cc] = (float)(0.5 * I.d_gamma * mu);
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
    rec[11] = 0.0;
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
  if (geom_kind(I, x, y) == 0)
    for (int i = 0; i < 5; i++) p += g[i * N + cc];
  out[cc] = p;
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
size_t step_smem_bytes(int nt, int prefetch) {
  // nt is a multiple of 32, so the float part keeps the doubles 8-byte aligned
  size_t ring = (size_t)(prefetch + 3) * (5 * (size_t)(nt + 4) + 9 * (size_t)nt);
  size_t floats = ring + 4 * (size_t)(nt + 4) + 3 * (size_t)(nt + 2) + 36 * (size_t)nt;
  return floats * sizeof(float) + (size_t)(nt / 32) * 3 * sizeof(double);
}

cudaError_t launch_init(const Inst* d_inst, const Inst& h, int index, cudaStream_t s) {
  dim3 blk(128), grd((h.nx + 127) / 128, h.ny);
  double* phi0 = reinterpret_cast<double*>(h.f[1]);  // f[1] is free before the first step
  init_phi_kernel<<<grd, blk, 0, s>>>(d_inst, index, phi0);
  init_pop_kernel<<<grd, blk, 0, s>>>(d_inst, index, phi0);
  const size_t N = (size_t)h.nx * h.ny;
  zero_kernel<<<256, 256, 0, s>>>(h.f[1], 9 * N);
  zero_kernel<<<256, 256, 0, s>>>(h.g[1], 5 * N);
  return cudaGetLastError();
}

cudaError_t launch_step(const Inst* d_inst, const Item* d_items, int n_items, int nthreads,
                        int grid, const long long* d_t, int t_off, bool diag, int prefetch,
                        cudaStream_t s) {
  const size_t smem = step_smem_bytes(nthreads, prefetch);
  if (prefetch == 1) {
    if (diag)
      step_kernel<true, 1><<<grid, nthreads, smem, s>>>(d_inst, d_items, n_items, d_t, t_off);
    else
      step_kernel<false, 1><<<grid, nthreads, smem, s>>>(d_inst, d_items, n_items, d_t, t_off);
  } else {
    if (diag)
      step_kernel<true, 2><<<grid, nthreads, smem, s>>>(d_inst, d_items, n_items, d_t, t_off);
    else
      step_kernel<false, 2><<<grid, nthreads, smem, s>>>(d_inst, d_items, n_items, d_t, t_off);
  }
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

int step_prefetch_for(int nthreads) {
  return 2 * step_smem_bytes(nthreads, 2) <= 227 * 1024 ? 2 : 1;
}

cudaError_t set_step_smem_limit() {
  const int lim = (int)step_smem_bytes(256, 2);
  cudaError_t e = cudaFuncSetAttribute(step_kernel<true, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(step_kernel<false, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(step_kernel<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(step_kernel<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
  return e;
}

}  // namespace ij
