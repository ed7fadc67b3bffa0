// Kernels of the 2-D binary-fluid lattice Boltzmann inkjet step
// (He et al., arXiv:1702.04487, "Methods", Eq. 3-10).
//
// Step kernel design (bandwidth-bound stencil, no tensor cores):
//  - one warp per work item: a strip of up to 60 written columns (two
//    columns per lane, plus two halo columns each side) by a chunk of rows
//    of one lattice; the warp marches up the rows, so every cell's
//    populations are read once and written once per step
//    (structure-of-arrays, 8-byte column pairs, coalesced);
//  - neighbours along x come from the lane's other column or a warp
//    shuffle, along y from registers; populations are staged P rows ahead
//    with cp.async into a per-warp ring in shared memory, and warps never
//    wait on one another;
//  - per row iteration: phi of row R, wetting ghost values of row R-1, the
//    collision of f (Eq. 4-6) and g (Eq. 8-10) on row R-2, and the streaming
//    in push form (halfway bounce-back, the stay/move split of Eq. 8): row
//    R-3 is completed with the downward movers of row R-2 and stored;
//  - geometry is analytic (no mask array);
//  - storage is FP32, or FP16 (f as offsets from w_i n0, g_1..4 as is, g_0
//    in FP32) with every update in FP32;
//  - diagnostics rows (ink weight e, e n, e n u_y) are summed in FP32 per
//    strip row and in FP64 across strips; the lattice totals of n, phi and
//    n u_y in FP32 per lane over an item and in FP64 across lanes and items.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

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

// Asynchronous global -> shared copies (cp.async), `n` of them: source p +
// i * N elements, destination sa + i * SS bytes, i = 0 .. n-1.  B bytes per
// copy (4 or 8).  The caller issues them under a warp-uniform condition.
template <int B, int SS>
__device__ __forceinline__ void cp5(unsigned sa, const void* p, size_t strideB) {
  const char* q = static_cast<const char*>(p);
  asm volatile(
      "{\n"
      " cp.async.ca.shared.global [%0], [%1], %6;\n"
      " cp.async.ca.shared.global [%0+%7], [%2], %6;\n"
      " cp.async.ca.shared.global [%0+%8], [%3], %6;\n"
      " cp.async.ca.shared.global [%0+%9], [%4], %6;\n"
      " cp.async.ca.shared.global [%0+%10], [%5], %6;\n}\n" ::"r"(sa),
      "l"(q), "l"(q + strideB), "l"(q + 2 * strideB), "l"(q + 3 * strideB), "l"(q + 4 * strideB),
      "n"(B), "n"(SS), "n"(2 * SS), "n"(3 * SS), "n"(4 * SS)
      : "memory");
}
template <int B, int SS>
__device__ __forceinline__ void cp4(unsigned sa, const void* p, size_t strideB) {
  const char* q = static_cast<const char*>(p);
  asm volatile(
      "{\n"
      " cp.async.ca.shared.global [%0], [%1], %5;\n"
      " cp.async.ca.shared.global [%0+%6], [%2], %5;\n"
      " cp.async.ca.shared.global [%0+%7], [%3], %5;\n"
      " cp.async.ca.shared.global [%0+%8], [%4], %5;\n}\n" ::"r"(sa),
      "l"(q), "l"(q + strideB), "l"(q + 2 * strideB), "l"(q + 3 * strideB), "n"(B), "n"(SS),
      "n"(2 * SS), "n"(3 * SS)
      : "memory");
}
// The same, issued only when pred is set (one predicate for the group).
template <int B, int SS>
__device__ __forceinline__ void cp5_if(unsigned sa, const void* p, size_t strideB, bool pred) {
  const char* q = static_cast<const char*>(p);
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %6, 0;\n"
      " @p cp.async.ca.shared.global [%0], [%1], %7;\n"
      " @p cp.async.ca.shared.global [%0+%8], [%2], %7;\n"
      " @p cp.async.ca.shared.global [%0+%9], [%3], %7;\n"
      " @p cp.async.ca.shared.global [%0+%10], [%4], %7;\n"
      " @p cp.async.ca.shared.global [%0+%11], [%5], %7;\n}\n" ::"r"(sa),
      "l"(q), "l"(q + strideB), "l"(q + 2 * strideB), "l"(q + 3 * strideB), "l"(q + 4 * strideB),
      "r"((int)pred), "n"(B), "n"(SS), "n"(2 * SS), "n"(3 * SS), "n"(4 * SS)
      : "memory");
}
template <int B, int SS>
__device__ __forceinline__ void cp4_if(unsigned sa, const void* p, size_t strideB, bool pred) {
  const char* q = static_cast<const char*>(p);
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %5, 0;\n"
      " @p cp.async.ca.shared.global [%0], [%1], %6;\n"
      " @p cp.async.ca.shared.global [%0+%7], [%2], %6;\n"
      " @p cp.async.ca.shared.global [%0+%8], [%3], %6;\n"
      " @p cp.async.ca.shared.global [%0+%9], [%4], %6;\n}\n" ::"r"(sa),
      "l"(q), "l"(q + strideB), "l"(q + 2 * strideB), "l"(q + 3 * strideB), "r"((int)pred),
      "n"(B), "n"(SS), "n"(2 * SS), "n"(3 * SS)
      : "memory");
}
// One predicated copy of B bytes.
template <int B>
__device__ __forceinline__ void cp1_if(unsigned sa, const void* p, bool pred) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %2, 0;\n"
      " @p cp.async.ca.shared.global [%0], [%1], %3;\n}\n" ::"r"(sa),
      "l"(p), "r"((int)pred), "n"(B)
      : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
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

// Wetting ghost value of a solid cell of kind k (reading of the wetting
// boundary condition of "Reproducing the experiment"): the mean over its
// fluid face neighbours (E, N, W, S) of phi + h_s / kappa (h_s = h on a
// wetting face, else 0); a solid cell touching fluid only diagonally takes
// the plain mean of those diagonal neighbours (NE, NW, SW, SE).
__device__ __forceinline__ float ghost_phi(int k, float hk, float pE, int kE, float pN, int kN,
                                           float pW, int kW, float pS, int kS, float pNE, int kNE,
                                           float pNW, int kNW, float pSW, int kSW, float pSE,
                                           int kSE) {
  const float h = k == 2 ? hk : 0.0f;
  float sum = 0.0f;
  int cnt = 0;
  if (kE == 0) { sum += pE + h; cnt++; }
  if (kN == 0) { sum += pN + h; cnt++; }
  if (kW == 0) { sum += pW + h; cnt++; }
  if (kS == 0) { sum += pS + h; cnt++; }
  if (cnt == 0) {
    if (kNE == 0) { sum += pNE; cnt++; }
    if (kNW == 0) { sum += pNW; cnt++; }
    if (kSW == 0) { sum += pSW; cnt++; }
    if (kSE == 0) { sum += pSE; cnt++; }
  }
  // the mean: a product with 1 / cnt (within one rounding of sum / cnt)
  return cnt == 1 ? sum : (cnt == 2 ? 0.5f * sum : (cnt == 3 ? sum * (1.0f / 3.0f) : 0.25f * sum));
}

// 1 / x from the hardware's approximate reciprocal refined by one
// Newton-Raphson step for 1/x (r <- r (2 - x r), written r + r (1 - x r)):
// the relative error squares, from about 2^-22 to below the FP32 rounding
// of the result; no slow path for special values (x is a density or a
// relaxation time, positive and of order one).
__device__ __forceinline__ float recip(float x) {
  const float r = __fdividef(1.0f, x);
  return fmaf(r, fmaf(-x, r, 1.0f), r);
}

// Per-lattice constants of the collision, in registers.
struct CollK {
  float phis, inv_phis, A4, kappa, omq, inv_tphi, gamma, inv2q, qmt, nu_air, dnu, n0, Fd;
};

// Collision of one fluid cell (Eq. 4-6 for f, Eq. 8-10 for g).
//  fr: f_i - w_i n0 of the cell; g: g_i; phi = sum g (raw); pC .. pSE: phi
//  with wetting ghosts of the cell and its 8 neighbours.
//  Out: fs = post-collision f_i - w_i n0 (i = 0..8); gP[i-1] = q g_i +
//  Omega_i (the part that moves, i = 1..4); gS[i-1] = (1 - q) g_i (the part
//  that stays); g0n = g_0 + Omega_0; n, uy, u2 of the cell.
__device__ __forceinline__ void collide_cell(const float (&fr)[9], const float (&g)[5], float phi,
                                             float pC, float pE, float pN, float pW, float pS,
                                             float pNE, float pNW, float pSW, float pSE,
                                             bool driven, const CollK& K, float (&fs)[9],
                                             float (&gP)[4], float (&gS)[4], float& g0n, float& n,
                                             float& uy, float& u2) {
  // lap = 6 sum_i w_i (phi_i - phi) from the differences, which are exact
  // where neighbours are close (no cancellation of O(10) terms)
  const float lap = (2.0f / 3.0f) * ((pE - pC) + (pN - pC) + (pW - pC) + (pS - pC)) +
                    (1.0f / 6.0f) * ((pNE - pC) + (pNW - pC) + (pSW - pC) + (pSE - pC));
  // gradient: (nE - sW) and (nW - sE) shared by both components
  const float dA_ = pNE - pSW, dB_ = pNW - pSE;
  const float gx = (pE - pW) * (1.0f / 3.0f) + (dA_ - dB_) * (1.0f / 12.0f);
  const float gy = (pN - pS) * (1.0f / 3.0f) + (dA_ + dB_) * (1.0f / 12.0f);
  const float mu = K.A4 * phi * ((phi - K.phis) * (phi + K.phis)) - K.kappa * lap;
  float C = 0.5f * (phi * K.inv_phis + 1.0f);
  C = fminf(fmaxf(C, 0.0f), 1.0f);
  const float Fb = driven ? K.Fd * C : 0.0f;
  const float Fx = mu * gx, Fy = mu * gy + Fb;
  // fr holds deviations f_i - w_i n0: their sum is n - n0
  const float dn = fr[0] + fr[1] + fr[2] + fr[3] + fr[4] + fr[5] + fr[6] + fr[7] + fr[8];
  n = K.n0 + dn;
  // n - (n0 + dn) exactly (n0 > |dn|: the error of the rounded sum is
  // representable), carried into 1 / n to first order
  const float n_lo = dn - (n - K.n0);
  const float mx = fr[1] - fr[3] + fr[5] - fr[6] - fr[7] + fr[8];
  const float my = fr[2] - fr[4] + fr[5] + fr[6] - fr[7] - fr[8];
  const float inv_hi = recip(n);
  const float inv_n = fmaf(-n_lo * inv_hi, inv_hi, inv_hi);
  const float ux = (mx + 0.5f * Fx) * inv_n;
  uy = (my + 0.5f * Fy) * inv_n;
  u2 = ux * ux + uy * uy;
  const float om = recip(0.5f + 3.0f * (K.nu_air + C * K.dnu));
  const float pref = 3.0f - 1.5f * om;  // 3 (1 - 1 / (2 tau)): the forcing prefactor over c_s^2
  // A_i - n0 = 3 (phi mu + n / 3) - n0 for i >= 1 (Eq. 6), on deviations
  const float p3 = dn + 3.0f * phi * mu;
  const float uF = ux * Fx + uy * Fy;
  // Moving directions first (deviations feq_i - w_i n0); the rest direction
  // then takes the balance, feq_0 - w_0 n0 = (n - n0) - sum_{i>=1} (feq_i -
  // w_i n0) and F_0 = -sum_{i>=1} F_i.  This equals A_0 of Eq. 6 (the
  // moments of Eq. 5-6 and of the forcing term are exact) but conserves
  // mass in FP32, whose rounded weights 4/9, 1/9, 1/36 do not sum to one.
  // Opposite directions i, i' share the even part of the equilibrium and of
  // the forcing term and differ in the sign of the odd part: with cu = c_i.u
  // and cF = c_i.F, the collision f* = (1 - om) f + om feq + F reads
  //   f*_i = (1 - om) f_i + w (a +- b),
  //   a = om (p3 + n (4.5 cu^2 - 1.5 u^2)) + pref (3 cu cF - u.F)
  //     = a0 + cu (a1 cu + a2 cF),
  //   b = 3 om n cu + pref cF = b1 cu + pref cF,
  // with a0 = om (p3 - 1.5 n u^2) - pref u.F, a1 = 4.5 om n, a2 = 3 pref,
  // b1 = 3 om n (Eq. 5 for feq, Eq. 4's forcing term).
  const float omn = om * n;
  const float a0 = fmaf(om, fmaf(-1.5f * n, u2, p3), -pref * uF);
  const float a1 = 4.5f * omn, a2 = 3.0f * pref, b1 = 3.0f * omn;
  const float omc = 1.0f - om;
  float sum1 = 0.0f, sum2 = 0.0f;  // a of the axis / diagonal pairs
#pragma unroll
  for (int i = 1; i < 9; i++) {
    if (i == 3 || i == 4 || i == 7 || i == 8) continue;  // handled with its pair
    const int ib = i == 1 ? 3 : (i == 2 ? 4 : (i == 5 ? 7 : 8));
    const float w = i < 5 ? W1 : W2;
    const float ex = (float)cEX(i), ey = (float)cEY(i);
    const float cu = ex * ux + ey * uy;
    const float cF = ex * Fx + ey * Fy;
    const float a = fmaf(cu, fmaf(a1, cu, a2 * cF), a0);
    const float b = fmaf(b1, cu, pref * cF);
    if (i < 5) sum1 += a; else sum2 += a;
    fs[i] = fmaf(omc, fr[i], w * (a + b));
    fs[ib] = fmaf(omc, fr[ib], w * (a - b));
  }
  fs[0] = fmaf(omc, fr[0], fmaf(om, dn, -2.0f * fmaf(W1, sum1, W2 * sum2)));
  // order parameter: Eq. 9-10 with the rest direction special; the moving
  // part q g_i + Omega_i streams, (1 - q) g_i stays
  const float gmu = K.gamma * mu;
  const float pq = phi * K.inv2q;
  float sum_ge = 0.0f;
#pragma unroll
  for (int i = 1; i < 5; i++) {
    const float cu = (float)cEX(i) * ux + (float)cEY(i) * uy;
    const float ge = 0.5f * gmu + pq * cu;
    sum_ge += ge;
    gP[i - 1] = fmaf(K.qmt, g[i], ge * K.inv_tphi);  // q g + (ge - g) / tau_phi
    gS[i - 1] = K.omq * g[i];
  }
  // rest direction: g0_0 = phi - sum_{i>=1} g0_i (Eq. 10 as a balance, so
  // that sum g0 = phi exactly); with phi - g_0 = sum_{i>=1} g_i the
  // relaxation uses small terms only
  g0n = g[0] + ((g[1] + g[2] + g[3] + g[4]) - sum_ge) * K.inv_tphi;
}

// ---------------------------------------------------------------------------
// The fused step: one warp per work item (a strip of columns x a chunk of
// rows of one lattice); warps never wait on one another.
//
// Lane l holds two neighbouring columns, A = xs - 2 + 2 l and B = A + 1
// (periodic wrap).  The strip writes the nout <= 60 columns xs .. xs+nout-1
// (lanes 1..30 when nout = 60); columns xs - 1 and xs + nout collide too
// (their populations stream into the strip), and xs - 2, xs + nout + 1 only
// give phi to the stencil.  A solid edge column (lane 0's A, lane 31's B)
// needs phi beyond the strip for its ghost value: that lane also stages the
// g of the column outside.  Half-warp items (a strip of nout <= 28 columns):
// lanes 0-15 and 16-31 each hold the strip, on the row ranges y0 and y1 of
// the same length, with every shuffle confined to its 16 lanes -- a narrow
// last strip of a lattice then takes half a warp per row.  Neighbours along x: the other column of the lane,
// or the neighbouring lane's by warp shuffle; along y: registers, as the warp
// marches up the rows.
//
// Per row iteration (pipeline row R): raw phi of row R (sum of g); wetting
// ghosts of row R-1 (rows with a solid cell in the warp only); the collision
// of row R-2 (Eq. 4-6 and 8-10); then the streaming in push form: row R-3,
// whose in-row and upward pulls were gathered when row R-3 collided, takes
// the downward movers of row R-2 and is stored; row R-2's own pulls (rest,
// sideways movers, stay parts, the upward movers of row R-3) are gathered
// into the same registers.  A pull whose source is solid takes the cell's
// own post-collision population of the opposite direction (halfway
// bounce-back; the moving g part likewise returns, conserving mass).
//
// Staging: each lane copies its own column pair with cp.async into a
// per-warp ring in shared memory and reads back only what it copied: g of
// row R+P (ring of P+3 rows) and f of row R+P-2 (ring of P+1 rows, f is
// needed at the collision only), as one group per row.  FP32: 8-byte copies
// of (A, B), which are contiguous and 8-byte aligned when nx is even (ODD
// instantiation: two 4-byte copies).  FP16 storage: 4-byte half pairs of f
// and g_1..4, 8-byte FP32 pairs of g_0; every update in FP32.
constexpr int kStripCols = 60;  // written columns of one work item
constexpr unsigned kFull = 0xffffffffu;

template <int P, bool H>
struct StepRing {
  static constexpr int DG = P + 3;  // g rows R+P .. R-2
  static constexpr int DF = P + 1;  // f rows R+P-2 .. R-2
  // words (4 bytes) of one row: FP32 g [5][64], f [9][64]; FP16 g_0 [64]
  // FP32 then g_1..4 [4][32] half pairs, f [9][32] half pairs
  static constexpr int GW = H ? 192 : 320;
  static constexpr int FW = H ? 288 : 576;
  // outer column of the edge lanes: [4 edge lanes (0, 31, or 0, 15, 16, 31
  // in half-warp items)][5 values, 2 words each]
  static constexpr int OW = 40;
};

template <bool DIAG, int P, bool H, bool ODD>
__global__ void __launch_bounds__(32, kStepBlocksPerSM)
    step_kernel(const Inst* __restrict__ insts, const Item* __restrict__ items, int n_items,
                const long long* __restrict__ d_t, int t_off) {
  using RG = StepRing<P, H>;
  static_assert(!(H && ODD), "FP16 storage needs an even nx");
  extern __shared__ float4 smem4[];
  float* const sg = reinterpret_cast<float*>(smem4);  // g ring
  float* const so = sg + RG::DG * RG::GW;              // outer-column ring
  float* const sf = so + RG::DG * RG::OW;              // f ring
  const unsigned sg_a = (unsigned)__cvta_generic_to_shared(sg);
  const unsigned so_a = (unsigned)__cvta_generic_to_shared(so);
  const unsigned sf_a = (unsigned)__cvta_generic_to_shared(sf);
  const int lane = threadIdx.x;
  const long long t = *d_t + t_off;

  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const Item it = items[item];
    const Inst& I = insts[it.inst];
    // a lattice whose numeric flag is set is frozen
    const unsigned st0 = lane == 0 ? *(volatile const unsigned*)I.status : 0u;
    if (__shfl_sync(kFull, st0, 0) & kStatusNumeric) continue;
    const int nx = I.nx, ny = I.ny, geom = I.geom, L = I.L, wt = I.wt, bc = I.bc;
    const int N = nx * ny;  // < 2^31 / 9 (checked on the host)
    // half-warp items: width 16, half h on rows from y1; an empty second half
    // (y1 < 0) stages, collides and writes nothing
    const int wid = it.half ? 16 : 32, ll = lane & (wid - 1), hh = it.half ? lane >> 4 : 0;
    const bool act = hh == 0 || it.y1 >= 0;
    const int y0 = hh ? it.y1 : it.y0, ch = it.ch;
    const int uA = it.xs - 2 + 2 * ll, uB = uA + 1;  // unwrapped columns
    const int xA = wrapi(uA, nx), xB = wrapi(uB, nx);
    const int ckA = column_kind(I, xA), ckB = column_kind(I, xB);
    const int ckW = column_kind(I, wrapi(uA - 1, nx));  // west of A
    const int ckE = column_kind(I, wrapi(uB + 1, nx));  // east of B
    // Kinds of the lane's four columns W (west of A), A, B, E (east of B) in
    // one row, 2 bits each (W lowest); the last four rows R .. R-3 are kept
    // in one word, row R in the low byte.  A row's kinds follow from its
    // mapped row m alone: nozzle rows below L take the columns' kinds, plate
    // rows below wt are solid (the top one wetting), rows outside a closed
    // domain are non-wetting solids.
    const unsigned ckpack = (unsigned)ckW | ((unsigned)ckA << 2) | ((unsigned)ckB << 4) |
                            ((unsigned)ckE << 6);
    auto row_bits = [&](int m) -> unsigned {
      if (m < 0) return 0x55u;
      if (geom == GEOM_NOZZLE) return m < L ? ckpack : 0u;
      if (geom == GEOM_PLATE) return m < wt ? (m == wt - 1 ? 0xAAu : 0x55u) : 0u;
      return 0u;
    };
    // the first lane's A / the last lane's B (of the warp or half-warp) on a
    // wall column: the column outside (xo); eo: the lane's outer slot
    const bool lft = ll == 0, rgt = ll == wid - 1;
    const bool edge = (lft && ckA != 0) || (rgt && ckB != 0);
    const int xo = lft ? wrapi(uA - 1, nx) : wrapi(uB + 1, nx);
    const int cko = lft ? ckW : ckE, cke = lft ? ckA : ckB;
    const int eo = 2 * hh + (lft ? 0 : 1);
    const bool any_edge = __any_sync(kFull, edge);
    const bool dA = geom != GEOM_NOZZLE || (xA >= I.cx0 && xA < I.cx1);
    const bool dB = geom != GEOM_NOZZLE || (xB >= I.cx0 && xB < I.cx1);
    const int xe = it.xs + it.nout;
    const bool vA = act && uA >= it.xs - 1 && uA <= xe;  // collision results used
    const bool vB = act && uB >= it.xs - 1 && uB <= xe;
    const bool wA = act && uA >= it.xs && uA < xe, wB = act && uB >= it.xs && uB < xe;  // written
    CollK K;
    K.phis = I.phis;
    K.inv_phis = I.inv_phis;
    K.A4 = I.A4;
    K.kappa = I.kappa;
    K.omq = I.omq;
    K.inv_tphi = I.inv_tphi;
    K.gamma = I.gamma;
    K.inv2q = I.inv2q;
    K.qmt = I.q - I.inv_tphi;
    K.nu_air = I.nu_air;
    K.dnu = I.dnu;
    K.n0 = I.n0;
    K.Fd = drive_at(I, t);
    const float hk = I.hk;
    const float* __restrict__ fin = I.f[t & 1];
    const float* __restrict__ gin = I.g[t & 1];
    float* __restrict__ fout = I.f[(t + 1) & 1];
    float* __restrict__ gout = I.g[(t + 1) & 1];
    // FP16 storage: f halves [9][N]; g_0 FP32 [N], then g_1..4 halves [4][N]
    const __half* __restrict__ fhin = reinterpret_cast<const __half*>(fin);
    const __half* __restrict__ ghin = reinterpret_cast<const __half*>(gin + N);
    __half* __restrict__ fhout = reinterpret_cast<__half*>(fout);
    __half* __restrict__ ghout = reinterpret_cast<__half*>(gout + N);

    // Stage g of row rg into g slot sgs and f of row rf into f slot sfs (one
    // cp.async group).  Whether a row is needed depends on the iteration only
    // (both halves of a half-warp item have ch rows); a row outside a closed
    // domain is skipped lane by lane (the halves of a half-warp item sit on
    // different rows).  kg: stage g (iteration k + P <= ch + 5); kf: stage f
    // (4 <= k + P <= ch + 5).
    auto stage = [&](bool kg, int rg, int sgs, bool kf, int rf, int sfs) {
      int ym = 0;
      if (kg) {
        const bool ok = act && map_row_v(rg, ny, bc, ym);
        const unsigned d = sg_a + sgs * (RG::GW * 4);
        const int c = ym * nx + xA;
        if (ODD) {
          cp5_if<4, 256>(d + lane * 8, gin + c, (size_t)N * 4, ok);
          cp5_if<4, 256>(d + lane * 8 + 4, gin + ym * nx + xB, (size_t)N * 4, ok);
        } else if (!H) {
          cp5_if<8, 256>(d + lane * 8, gin + c, (size_t)N * 4, ok);
        } else {
          cp1_if<8>(d + lane * 8, gin + c, ok);
          cp4_if<4, 128>(d + 256 + lane * 4, ghin + c, (size_t)N * 2, ok);
        }
        if (any_edge) {
          // a solid edge column next to a fluid one outside the strip
          const bool need = ok && edge && row_kind(geom, cke, L, wt, ym) != 0 &&
                            row_kind(geom, cko, L, wt, ym) == 0;
          const unsigned o = so_a + sgs * (RG::OW * 4) + eo * 40;
          const int co = ym * nx + (ODD ? xo : (xo & ~1));
          if (!H) {
#pragma unroll
            for (int i = 0; i < 5; i++)
              cp1_if<ODD ? 4 : 8>(o + i * 8, gin + (size_t)i * N + co, need);
          } else {
            cp1_if<8>(o, gin + co, need);
#pragma unroll
            for (int i = 1; i < 5; i++)
              cp1_if<4>(o + i * 8, ghin + (size_t)(i - 1) * N + co, need);
          }
        }
      }
      if (kf) {
        const bool ok = act && map_row_v(rf, ny, bc, ym);
        const unsigned d = sf_a + sfs * (RG::FW * 4);
        const int c = ym * nx + xA;
        if (ODD) {
          cp5_if<4, 256>(d + lane * 8, fin + c, (size_t)N * 4, ok);
          cp4_if<4, 256>(d + 5 * 256 + lane * 8, fin + 5 * (size_t)N + c, (size_t)N * 4, ok);
          const int cb = ym * nx + xB;
          cp5_if<4, 256>(d + lane * 8 + 4, fin + cb, (size_t)N * 4, ok);
          cp4_if<4, 256>(d + 5 * 256 + lane * 8 + 4, fin + 5 * (size_t)N + cb, (size_t)N * 4, ok);
        } else if (!H) {
          cp5_if<8, 256>(d + lane * 8, fin + c, (size_t)N * 4, ok);
          cp4_if<8, 256>(d + 5 * 256 + lane * 8, fin + 5 * (size_t)N + c, (size_t)N * 4, ok);
        } else {
          cp5_if<4, 128>(d + lane * 4, fhin + c, (size_t)N * 2, ok);
          cp4_if<4, 128>(d + 5 * 128 + lane * 4, fhin + 5 * (size_t)N + c, (size_t)N * 2, ok);
        }
      }
      cp_async_commit();
    };
    // staged values of this lane: g_i / f_i of columns A and B of a slot
    auto load_g = [&](int slot, float (&a)[5], float (&b)[5]) {
      const float* r = sg + slot * RG::GW;
      if (!H) {
#pragma unroll
        for (int i = 0; i < 5; i++) {
          const float2 v = reinterpret_cast<const float2*>(r + i * 64)[lane];
          a[i] = v.x;
          b[i] = v.y;
        }
      } else {
        const float2 v = reinterpret_cast<const float2*>(r)[lane];
        a[0] = v.x;
        b[0] = v.y;
#pragma unroll
        for (int i = 1; i < 5; i++) {
          const float2 w = __half22float2(reinterpret_cast<const __half2*>(r + 64 + (i - 1) * 32)[lane]);
          a[i] = w.x;
          b[i] = w.y;
        }
      }
    };
    auto load_f = [&](int slot, float (&a)[9], float (&b)[9]) {
      const float* r = sf + slot * RG::FW;
#pragma unroll
      for (int i = 0; i < 9; i++) {
        float2 v;
        if (!H)
          v = reinterpret_cast<const float2*>(r + i * 64)[lane];
        else
          v = __half22float2(reinterpret_cast<const __half2*>(r + i * 32)[lane]);
        a[i] = v.x;
        b[i] = v.y;
      }
    };
    // raw phi of the outer column (edge lanes)
    auto load_outer = [&](int slot) -> float {
      const float* o = so + slot * RG::OW + eo * 10;
      const int wd = (ODD || !lft) ? 0 : 1;  // the first lane: the odd column of its pair
      if (!H) return o[wd] + ((o[2 + wd] + o[4 + wd]) + (o[6 + wd] + o[8 + wd]));
      float s = 0.0f;  // g_1..4 first, as for the lane's own columns
#pragma unroll
      for (int i = 1; i < 5; i++) {
        const __half2 hp = *reinterpret_cast<const __half2*>(o + 2 * i);
        s += wd ? __high2float(hp) : __low2float(hp);
      }
      return o[wd] + s;
    };

#pragma unroll
    for (int j = 0; j < P; j++)
      stage(j <= ch + 5, y0 - 3 + j, j, j >= 4 && j <= ch + 5, y0 - 5 + j, j);

    // raw phi of rows R, R-1, R-2 (pr*0..2) and of the outer column (px*);
    // phi with ghosts of rows R-1, R-2, R-3 (pe*0..2) and of the columns
    // west of A (peW*) and east of B (peE*); mapped rows R .. R-2 (m0..m2),
    // packed kinds of rows R .. R-3 (kp)
    float prA0 = 0.f, prA1 = 0.f, prA2 = 0.f, prB0 = 0.f, prB1 = 0.f, prB2 = 0.f;
    float px0 = 0.f, px1 = 0.f, px2 = 0.f;
    float peA0 = 0.f, peA1 = 0.f, peA2 = 0.f, peB0 = 0.f, peB1 = 0.f, peB2 = 0.f;
    float peW0 = 0.f, peW1 = 0.f, peW2 = 0.f, peE0 = 0.f, peE1 = 0.f, peE2 = 0.f;
    int m0 = -1, m1 = -1, m2 = -1;
    unsigned kp = 0x55555555u;
    // kind of column c (0 W, 1 A, 2 B, 3 E) in row R - j
#define KD(c, j) ((int)((kp >> (8 * (j) + 2 * (c))) & 3u))
    // gathered pulls of the row being streamed, per column: f_0..3, f_5,
    // f_6 and g_0..4 (g_4 without its moving part yet); the upward movers
    // for the next row (f_2 own, f_5 from the west, f_6 from the east, the
    // moving g_2 own); own f*_5, f*_6 (bounce-back of f_7, f_8)
    float aA[11], aB[11], upA[4], upB[4], bbA[2], bbB[2];
#pragma unroll
    for (int i = 0; i < 11; i++) aA[i] = aB[i] = 0.f;
#pragma unroll
    for (int i = 0; i < 4; i++) upA[i] = upB[i] = 0.f;
    bbA[0] = bbA[1] = bbB[0] = bbB[1] = 0.f;
    // lattice totals sum n, sum phi, sum n u_y of the lane's cells over the
    // item (diagnostics steps), in FP64: a sum of a few hundred FP32 values
    // is exact in FP64, so the totals do not depend on how rows are cut into
    // items (only on the FP64 order of the final additions)
    double sn = 0.0, sphi = 0.0, smom = 0.0;

#pragma unroll 1
    for (int k = 0; k < ch + 6; k++) {
      const int R = y0 - 3 + k;
      // ring slots (compile-time moduli): g of row R / R+P, f of row R-2 / R+P-2
      const unsigned ku = (unsigned)k;
      const int gr = ku % RG::DG, gw = (ku + P) % RG::DG;
      const int fr_ = ku % RG::DF, fw = (ku + P) % RG::DF;
      stage(k + P <= ch + 5, R + P, gw, k + P >= 4 && k + P <= ch + 5, R + P - 2, fw);
      cp_async_wait<P>();  // this lane's copies of g row R and f row R-2 have landed
      m2 = m1;
      m1 = m0;
      {
        int ym;
        m0 = map_row_v(R, ny, bc, ym) ? ym : -1;
      }
      kp = (kp << 8) | row_bits(m0);
      prA2 = prA1; prA1 = prA0; prB2 = prB1; prB1 = prB0;
      px2 = px1; px1 = px0;
      peA2 = peA1; peA1 = peA0; peB2 = peB1; peB1 = peB0;
      peW2 = peW1; peW1 = peW0; peE2 = peE1; peE1 = peE0;
      const int kA0 = KD(1, 0), kB0 = KD(2, 0), kA1 = KD(1, 1), kB1 = KD(2, 1);
      // ---- raw phi of row R
      {
        float ga[5], gb[5];
        load_g(gr, ga, gb);
        // phi = g_0 + the small g_1..4, added first: one rounding at the
        // scale of phi* instead of four
        prA0 = kA0 == 0 ? ga[0] + ((ga[1] + ga[2]) + (ga[3] + ga[4])) : 0.0f;
        prB0 = kB0 == 0 ? gb[0] + ((gb[1] + gb[2]) + (gb[3] + gb[4])) : 0.0f;
        px0 = 0.0f;
        if (any_edge && edge && m0 >= 0 && row_kind(geom, cke, L, wt, m0) != 0 &&
            row_kind(geom, cko, L, wt, m0) == 0)
          px0 = load_outer(gr);
      }
      // ---- phi with wetting ghosts of row R-1
      peA0 = prA1;
      peB0 = prB1;
      if (__any_sync(kFull, ((kp >> 8) & 0x3Cu) != 0u)) {
        float wN = __shfl_up_sync(kFull, prB0, 1, wid), wC = __shfl_up_sync(kFull, prB1, 1, wid);
        float wS = __shfl_up_sync(kFull, prB2, 1, wid);
        float eN = __shfl_down_sync(kFull, prA0, 1, wid), eC = __shfl_down_sync(kFull, prA1, 1, wid);
        float eS = __shfl_down_sync(kFull, prA2, 1, wid);
        if (edge && lft) {
          wN = px0; wC = px1; wS = px2;
        } else if (edge) {
          eN = px0; eC = px1; eS = px2;
        }
        const int kA2 = KD(1, 2), kB2 = KD(2, 2);
        const int kW0 = KD(0, 0), kW1 = KD(0, 1), kW2 = KD(0, 2);
        const int kE0 = KD(3, 0), kE1 = KD(3, 1), kE2 = KD(3, 2);
        if (kA1 != 0)
          peA0 = ghost_phi(kA1, hk, prB1, kB1, prA0, kA0, wC, kW1, prA2, kA2, prB0, kB0, wN, kW0,
                           wS, kW2, prB2, kB2);
        if (kB1 != 0)
          peB0 = ghost_phi(kB1, hk, eC, kE1, prB0, kB0, prA1, kA1, prB2, kB2, eN, kE0, prA0, kA0,
                           prA2, kA2, eS, kE2);
      }
      peW0 = __shfl_up_sync(kFull, peB0, 1, wid);
      peE0 = __shfl_down_sync(kFull, peA0, 1, wid);
      if (k < 4) continue;  // warp-uniform: rows below y0 - 1 do not collide
      // ---- collision of row Rc = R-2 (both columns)
      const int Rc = R - 2;
      const int kA2 = KD(1, 2), kB2 = KD(2, 2);
      float fsA[9], fsB[9], gPA[4], gPB[4], gSA[4], gSB[4], g0A, g0B;
      float dg[3] = {0.f, 0.f, 0.f};  // row sums of e, e n, e n u_y
      {
        float ga[5], gb[5], fa[9], fb[9];
        load_g((ku + RG::DG - 2) % RG::DG, ga, gb);
        load_f(fr_, fa, fb);
        const bool drv = geom != GEOM_NOZZLE || (m2 >= 0 && m2 < L);
        float nA, uyA, u2A, nB, uyB, u2B;
        collide_cell(fa, ga, prA2, peA1, peB1, peA0, peW1, peA2, peB0, peW0, peW2, peB2,
                     drv && dA, K, fsA, gPA, gSA, g0A, nA, uyA, u2A);
        collide_cell(fb, gb, prB2, peB1, peE1, peB0, peA1, peB2, peE0, peA0, peA2, peE2,
                     drv && dB, K, fsB, gPB, gSB, g0B, nB, uyB, u2B);
        // only fluid cells whose results are used raise the flag or count
        const bool cA = vA && kA2 == 0, cB = vB && kB2 == 0;
        if ((cA && !(u2A < 0.09f)) || (cB && !(u2B < 0.09f))) atomicOr(I.status, kStatusNumeric);
        if (DIAG && k >= 5 && k < ch + 5) {  // Rc in [y0, y0 + ch)
          const bool oA = cA && wA, oB = cB && wB;
          const float eA = fminf(fmaxf(prA2 * K.inv_phis, 0.0f), 1.0f);
          const float eB = fminf(fmaxf(prB2 * K.inv_phis, 0.0f), 1.0f);
          if (oA) {
            dg[0] += eA; dg[1] += eA * nA; dg[2] += eA * nA * uyA;
            sn += (double)nA; sphi += (double)prA2; smom += (double)(nA * uyA);
          }
          if (oB) {
            dg[0] += eB; dg[1] += eB * nB; dg[2] += eB * nB * uyB;
            sn += (double)nB; sphi += (double)prB2; smom += (double)(nB * uyB);
          }
        }
      }
      if (DIAG && k >= 5 && k < ch + 5) {
        // the strip's cells of the row are summed in FP32, every total
        // across strips, rows and chunks in FP64
        for (int o = wid >> 1; o > 0; o >>= 1)
#pragma unroll
          for (int j = 0; j < 3; j++) dg[j] += __shfl_down_sync(kFull, dg[j], o, wid);
        if (ll == 0 && act) {
          atomicAdd(I.rows + Rc, (double)dg[0]);
          atomicAdd(I.rows + ny + Rc, (double)dg[1]);
          atomicAdd(I.rows + 2 * ny + Rc, (double)dg[2]);
        }
      }
      // movers that cross to the neighbouring lane
      const float sh7 = __shfl_down_sync(kFull, fsA[7], 1, wid);  // f*_7 of B's east neighbour
      const float sh8 = __shfl_up_sync(kFull, fsB[8], 1, wid);    // f*_8 of A's west neighbour
      const float sh1 = __shfl_up_sync(kFull, fsB[1], 1, wid);
      const float shP1 = __shfl_up_sync(kFull, gPB[0], 1, wid);
      const float sh3 = __shfl_down_sync(kFull, fsA[3], 1, wid);
      const float shP3 = __shfl_down_sync(kFull, gPA[2], 1, wid);
      const float sh5 = __shfl_up_sync(kFull, fsB[5], 1, wid);
      const float sh6 = __shfl_down_sync(kFull, fsA[6], 1, wid);
      // does any lane have a solid source among rows Rc-1 .. Rc (warp-uniform)
      const bool solid_rows = __any_sync(kFull, (kp >> 16) != 0u);
      // ---- row Y = R-3: downward movers of row Rc, bounce-back, store
      if (k >= 6) {
        const int Y = R - 3;
        float f4A = fsA[4], f7A = fsB[7], f8A = sh8, p4A = gPA[3];
        float f4B = fsB[4], f7B = sh7, f8B = fsA[8], p4B = gPB[3];
        const int kA3 = KD(1, 3), kB3 = KD(2, 3);  // row Y
        if (solid_rows) {
          const int kW2 = KD(0, 2), kE2 = KD(3, 2);
          // sources (x, Y+1), (x+1, Y+1), (x-1, Y+1)
          if (kA2 != 0) { f4A = upA[0]; p4A = upA[3]; }
          if (kB2 != 0) { f7A = bbA[0]; }
          if (kW2 != 0) { f8A = bbA[1]; }
          if (kB2 != 0) { f4B = upB[0]; p4B = upB[3]; }
          if (kE2 != 0) { f7B = bbB[0]; }
          if (kA2 != 0) { f8B = bbB[1]; }
        }
        // Solid cells of the written columns are written too, with the 0
        // they hold (their populations are never read as such): every store
        // then covers whole column pairs and no DRAM sector is left partly
        // written (which costs a read-modify-write).
        float fA[9] = {aA[0], aA[1], aA[2], aA[3], f4A, aA[4], aA[5], f7A, f8A};
        float fB[9] = {aB[0], aB[1], aB[2], aB[3], f4B, aB[4], aB[5], f7B, f8B};
        float gA[5] = {aA[6], aA[7], aA[8], aA[9], aA[10] + p4A};
        float gB[5] = {aB[6], aB[7], aB[8], aB[9], aB[10] + p4B};
        if (solid_rows) {
#pragma unroll
          for (int i = 0; i < 9; i++) {
            fA[i] = kA3 == 0 ? fA[i] : 0.0f;
            fB[i] = kB3 == 0 ? fB[i] : 0.0f;
          }
#pragma unroll
          for (int i = 0; i < 5; i++) {
            gA[i] = kA3 == 0 ? gA[i] : 0.0f;
            gB[i] = kB3 == 0 ? gB[i] : 0.0f;
          }
        }
        const int cA = Y * nx + xA, cB = Y * nx + xB;
        if (!ODD && wA && wB) {
          if (!H) {
#pragma unroll
            for (int i = 0; i < 9; i++)
              *reinterpret_cast<float2*>(fout + (size_t)i * N + cA) = make_float2(fA[i], fB[i]);
#pragma unroll
            for (int i = 0; i < 5; i++)
              *reinterpret_cast<float2*>(gout + (size_t)i * N + cA) = make_float2(gA[i], gB[i]);
          } else {
            // round to nearest even on store
#pragma unroll
            for (int i = 0; i < 9; i++)
              *reinterpret_cast<__half2*>(fhout + (size_t)i * N + cA) = __floats2half2_rn(fA[i], fB[i]);
            *reinterpret_cast<float2*>(gout + cA) = make_float2(gA[0], gB[0]);
#pragma unroll
            for (int i = 1; i < 5; i++)
              *reinterpret_cast<__half2*>(ghout + (size_t)(i - 1) * N + cA) =
                  __floats2half2_rn(gA[i], gB[i]);
          }
        } else {
          if (!H) {
            if (wA) {
#pragma unroll
              for (int i = 0; i < 9; i++) fout[(size_t)i * N + cA] = fA[i];
#pragma unroll
              for (int i = 0; i < 5; i++) gout[(size_t)i * N + cA] = gA[i];
            }
            if (wB) {
#pragma unroll
              for (int i = 0; i < 9; i++) fout[(size_t)i * N + cB] = fB[i];
#pragma unroll
              for (int i = 0; i < 5; i++) gout[(size_t)i * N + cB] = gB[i];
            }
          } else {
            if (wA) {
#pragma unroll
              for (int i = 0; i < 9; i++) fhout[(size_t)i * N + cA] = __float2half_rn(fA[i]);
              gout[cA] = gA[0];
#pragma unroll
              for (int i = 1; i < 5; i++) ghout[(size_t)(i - 1) * N + cA] = __float2half_rn(gA[i]);
            }
            if (wB) {
#pragma unroll
              for (int i = 0; i < 9; i++) fhout[(size_t)i * N + cB] = __float2half_rn(fB[i]);
              gout[cB] = gB[0];
#pragma unroll
              for (int i = 1; i < 5; i++) ghout[(size_t)(i - 1) * N + cB] = __float2half_rn(gB[i]);
            }
          }
        }
      }
      // ---- gather the pulls of row Rc (rest, sideways, upward movers of
      // row Rc-1, stay parts) into aA / aB; keep the upward movers of row Rc
      {
        // f_0, f_1 (from x-1), f_2 (from x, Rc-1), f_3 (from x+1),
        // f_5 (from x-1, Rc-1), f_6 (from x+1, Rc-1); g_0 .. g_4
        float f1A = sh1, f3A = fsB[3], f2A = upA[0], f5A = upA[1], f6A = upA[2];
        float p1A = shP1, p3A = gPB[2], p2A = upA[3];
        float f1B = fsA[1], f3B = sh3, f2B = upB[0], f5B = upB[1], f6B = upB[2];
        float p1B = gPA[0], p3B = shP3, p2B = upB[3];
        if (solid_rows) {
          const int kW2 = KD(0, 2), kE2 = KD(3, 2);
          const int kA3 = KD(1, 3), kB3 = KD(2, 3), kW3 = KD(0, 3), kE3 = KD(3, 3);
          // A: sources (x-1, Rc) = W, (x+1, Rc) = B, (x, Rc-1) = A,
          // (x-1, Rc-1) = W, (x+1, Rc-1) = B
          if (kW2 != 0) { f1A = fsA[3]; p1A = gPA[2]; }
          if (kB2 != 0) { f3A = fsA[1]; p3A = gPA[0]; }
          if (kA3 != 0) { f2A = fsA[4]; p2A = gPA[3]; }
          if (kW3 != 0) f5A = fsA[7];
          if (kB3 != 0) f6A = fsA[8];
          // B: (x-1, Rc) = A, (x+1, Rc) = E, (x, Rc-1) = B, (x-1, Rc-1) = A,
          // (x+1, Rc-1) = E
          if (kA2 != 0) { f1B = fsB[3]; p1B = gPB[2]; }
          if (kE2 != 0) { f3B = fsB[1]; p3B = gPB[0]; }
          if (kB3 != 0) { f2B = fsB[4]; p2B = gPB[3]; }
          if (kA3 != 0) f5B = fsB[7];
          if (kE3 != 0) f6B = fsB[8];
        }
        aA[0] = fsA[0]; aA[1] = f1A; aA[2] = f2A; aA[3] = f3A; aA[4] = f5A; aA[5] = f6A;
        aA[6] = g0A; aA[7] = gSA[0] + p1A; aA[8] = gSA[1] + p2A; aA[9] = gSA[2] + p3A;
        aA[10] = gSA[3];
        aB[0] = fsB[0]; aB[1] = f1B; aB[2] = f2B; aB[3] = f3B; aB[4] = f5B; aB[5] = f6B;
        aB[6] = g0B; aB[7] = gSB[0] + p1B; aB[8] = gSB[1] + p2B; aB[9] = gSB[2] + p3B;
        aB[10] = gSB[3];
        upA[0] = fsA[2]; upA[1] = sh5; upA[2] = fsB[6]; upA[3] = gPA[1];
        upB[0] = fsB[2]; upB[1] = fsA[5]; upB[2] = sh6; upB[3] = gPB[1];
        bbA[0] = fsA[5]; bbA[1] = fsA[6];
        bbB[0] = fsB[5]; bbB[1] = fsB[6];
      }
    }
#undef KD
    cp_async_wait<0>();  // no copy may land after the warp moves on
    if (DIAG) {
      double tn = sn, tphi = sphi, tmom = smom;
      for (int o = wid >> 1; o > 0; o >>= 1) {
        tn += __shfl_down_sync(kFull, tn, o, wid);
        tphi += __shfl_down_sync(kFull, tphi, o, wid);
        tmom += __shfl_down_sync(kFull, tmom, o, wid);
      }
      if (ll == 0 && act) {
        atomicAdd(I.sums + 0, tn);
        atomicAdd(I.sums + 1, tphi);
        atomicAdd(I.sums + 2, tmom);
      }
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
  // per warp: g ring (P+3 rows) with the edge lanes' outer column, f ring (P+1 rows)
  const int gw = h16 ? 192 : 320, fw = h16 ? 288 : 576, ow = 40;
  return (size_t)(nthreads / 32) * ((prefetch + 3) * (gw + ow) + (prefetch + 1) * fw) * sizeof(float);
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

template <bool DIAG, bool H, bool ODD>
cudaError_t launch_step_p(const Inst* d_inst, const Item* d_items, int n_items, int grid,
                          const long long* d_t, int t_off, int prefetch, size_t smem,
                          cudaStream_t s) {
  switch (prefetch) {
    case 1:
      step_kernel<DIAG, 1, H, ODD><<<grid, 32, smem, s>>>(d_inst, d_items, n_items, d_t, t_off);
      break;
    case 2:
      step_kernel<DIAG, 2, H, ODD><<<grid, 32, smem, s>>>(d_inst, d_items, n_items, d_t, t_off);
      break;
    case 3:
      step_kernel<DIAG, 3, H, ODD><<<grid, 32, smem, s>>>(d_inst, d_items, n_items, d_t, t_off);
      break;
    default:
      step_kernel<DIAG, 4, H, ODD><<<grid, 32, smem, s>>>(d_inst, d_items, n_items, d_t, t_off);
      break;
  }
  return cudaGetLastError();
}

cudaError_t launch_step(const Inst* d_inst, const Item* d_items, int n_items, int nthreads,
                        int grid, const long long* d_t, int t_off, bool diag, int prefetch,
                        bool h16, bool odd, cudaStream_t s) {
  if (nthreads != kStepThreads || prefetch < 1 || prefetch > kMaxPrefetch || (h16 && odd))
    return cudaErrorInvalidValue;
  if (n_items <= 0) return cudaSuccess;
  const size_t smem = step_smem_bytes(nthreads, prefetch, h16);
#define LAUNCH_STEP(DG, HH, OD) \
  launch_step_p<DG, HH, OD>(d_inst, d_items, n_items, grid, d_t, t_off, prefetch, smem, s)
  if (h16) return diag ? LAUNCH_STEP(true, true, false) : LAUNCH_STEP(false, true, false);
  if (odd) return diag ? LAUNCH_STEP(true, false, true) : LAUNCH_STEP(false, false, true);
  return diag ? LAUNCH_STEP(true, false, false) : LAUNCH_STEP(false, false, false);
#undef LAUNCH_STEP
}

int step_prefetch_for(int) { return 1; }

int step_slots(int prefetch, bool h16, bool odd) {
  int dev = 0, sms = 0, nb = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return 1;
  const size_t smem = step_smem_bytes(kStepThreads, prefetch, h16);
  cudaError_t e;
#define SLOTS_P(PF)                                                                          \
  e = h16 ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, step_kernel<false, PF, true, false>, \
                                                          kStepThreads, smem)               \
          : odd ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(                            \
                      &nb, step_kernel<false, PF, false, true>, kStepThreads, smem)          \
                : cudaOccupancyMaxActiveBlocksPerMultiprocessor(                            \
                      &nb, step_kernel<false, PF, false, false>, kStepThreads, smem);
  switch (prefetch) {
    case 1: SLOTS_P(1) break;
    case 2: SLOTS_P(2) break;
    case 3: SLOTS_P(3) break;
    default: SLOTS_P(4) break;
  }
#undef SLOTS_P
  if (e != cudaSuccess || nb < 1) return sms > 0 ? sms : 1;
  return sms * nb;
}

cudaError_t set_step_smem_limit() {
  const int lim = (int)step_smem_bytes(kStepThreads, kMaxPrefetch, false);
  cudaError_t e = cudaSuccess;
#define SET_LIM(DG, PF, HH, OD)                                                               \
  if (e == cudaSuccess)                                                                       \
    e = cudaFuncSetAttribute(step_kernel<DG, PF, HH, OD>,                                     \
                             cudaFuncAttributeMaxDynamicSharedMemorySize, lim);
#define SET_LIM_P(PF) \
  SET_LIM(true, PF, false, false) SET_LIM(false, PF, false, false) \
  SET_LIM(true, PF, true, false) SET_LIM(false, PF, true, false)   \
  SET_LIM(true, PF, false, true) SET_LIM(false, PF, false, true)
  SET_LIM_P(1) SET_LIM_P(2) SET_LIM_P(3) SET_LIM_P(4)
#undef SET_LIM_P
#undef SET_LIM
  return e;
}

// Items of one strip over rows ya .. yb-1 in chunks of `chunk` rows.  A
// narrow strip (nout <= 28, allow_half) pairs consecutive full-length chunks
// into half-warp items; a chunk left over (odd count or the short last one)
// is a half-warp item of its own.  Writes up to cap items into out (out may
// be null to count); returns the count.
int strip_items(const Inst& I, int k, int xs, int nout, int chunk, int ya, int yb, bool allow_half,
                Item* out, int cap) {
  constexpr int halo = 2;
  int n = 0;
  auto put = [&](int y0, int ch, int half, int y1) {
    if (out && n < cap) out[n] = Item{k, xs, nout, halo, y0, ch, half, y1};
    n++;
  };
  if (!allow_half || nout > kStripCols / 2 - 2) {
    for (int y0 = ya; y0 < yb; y0 += chunk) put(y0, yb - y0 < chunk ? yb - y0 : chunk, 0, -1);
    return n;
  }
  int y0 = ya;
  for (; y0 + 2 * chunk <= yb; y0 += 2 * chunk) put(y0, chunk, 1, y0 + chunk);
  for (; y0 < yb; y0 += chunk) put(y0, yb - y0 < chunk ? yb - y0 : chunk, 1, -1);
  return n;
}

int make_items_range(const Inst& I, int k, int chunk, int ya, int yb, Item* out, int cap,
                     bool allow_half) {
  const int W = kStripCols;  // 60 written columns per full strip (2 per lane)
  const int nstrip = (I.nx + W - 1) / W;
  int n = 0;
  // row-major: the strips of one chunk of rows next to each other (items
  // that run together share halo sectors and DRAM pages)
  for (int y0 = ya; y0 < yb; y0 += chunk)
    for (int s = 0; s < nstrip; s++) {
      const int xs = s * W, nout = I.nx - xs < W ? I.nx - xs : W;
      const bool half = allow_half && nout <= W / 2 - 2;
      if (half && ((y0 - ya) / chunk) % 2 == 1) continue;  // taken with the chunk below
      const int y1 = half ? std::min(yb, y0 + 2 * chunk) : std::min(yb, y0 + chunk);
      const int m = strip_items(I, k, xs, nout, chunk, y0, y1, allow_half, out ? out + n : nullptr,
                                out ? cap - n : 0);
      if (out && n + m > cap) return -1;
      n += m;
    }
  return n;
}

int make_items(const Inst& I, int k, int chunk, Item* out, int cap) {
  return make_items_range(I, k, chunk, 0, I.ny, out, cap, true);
}

int items_per_range(const Inst& I, int chunk, int ya, int yb, bool allow_half) {
  return yb > ya ? make_items_range(I, 0, chunk, ya, yb, nullptr, 0, allow_half) : 0;
}

int items_per_lattice(const Inst& I, int chunk) { return items_per_range(I, chunk, 0, I.ny, true); }

}  // namespace ij
