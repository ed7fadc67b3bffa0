// Kernels of the 3-D lift (D3Q19 f, D3Q7 g) of the binary-fluid LBM inkjet
// step (He et al., arXiv:1702.04487, Eq. 3-10 lifted by moment matching).
//
// One time step is one fused launch over every lattice of a handle plus two
// small ones:
//  step3:  a CTA of 16 warps holds a 32 (x, lanes) x 16 (y, warps) tile of
//          columns and marches up z.  Per plane: the populations of the next
//          plane are staged with cp.async; phi with wetting ghosts comes from
//          a ring of planes in shared memory; each cell collides (moments,
//          D3Q19 stencils, chemical potential, drive, half-force velocity,
//          Eq. 4-6 and 8-10 lifted); the streaming is in push form: movers
//          along x cross lanes by shuffle, movers along y cross warps through
//          shared memory, movers along z stay in registers until the next
//          plane; a plane is stored as soon as the plane above it has
//          collided.  The inner 28 x 12 columns are written; the ring around
//          them collides (its movers enter the tile) or gives phi only.
//  ghost3: phi of the new state on the solid cells within reach of a fluid
//          stencil (the wetting ghost values) and on the extended planes of
//          the axial ends;
//  flip3:  the new state becomes current (lattices not frozen).
// Storage is FP32 or FP16 (f deviations and g_1..6; g_0 FP32); arithmetic
// is FP32.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>

#include <algorithm>

#include "lbm3d.cuh"

namespace ij {
namespace {

// D3Q19 directions in the public order: rest, +-x, +-y, +-z, then the edges
// (+x+y, -x+y, +x-y, -x-y, +x+z, -x+z, +x-z, -x-z, +y+z, -y+z, +y-z, -y-z);
// D3Q7 uses the first seven.
__host__ __device__ __forceinline__ constexpr int ex3(int i) {
  return i == 1 || i == 7 || i == 9 || i == 11 || i == 13 ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14 ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int ey3(int i) {
  return i == 3 || i == 7 || i == 8 || i == 15 || i == 17 ? 1
         : (i == 4 || i == 9 || i == 10 || i == 16 || i == 18 ? -1 : 0);
}
__host__ __device__ __forceinline__ constexpr int ez3(int i) {
  return i == 5 || i == 11 || i == 12 || i == 15 || i == 16 ? 1
         : (i == 6 || i == 13 || i == 14 || i == 17 || i == 18 ? -1 : 0);
}
__device__ __forceinline__ constexpr float w3(int i) {
  return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}

template <bool H>
__device__ __forceinline__ float ldS(const void* p, size_t i) {
  if (H) return __half2float(reinterpret_cast<const __half*>(p)[i]);
  return reinterpret_cast<const float*>(p)[i];
}
template <bool H>
__device__ __forceinline__ void stS(void* p, size_t i, float v) {
  if (H)
    reinterpret_cast<__half*>(p)[i] = __float2half_rn(v);
  else
    reinterpret_cast<float*>(p)[i] = v;
}
template <bool H>
__device__ __forceinline__ void stS(void* p, unsigned i, float v) {
  if (H)
    reinterpret_cast<__half*>(p)[i] = __float2half_rn(v);
  else
    reinterpret_cast<float*>(p)[i] = v;
}
// The same with the streaming (evict-first) cache hint: the new state is
// read again only in the next step, so its lines should not push the current
// state's planes, which neighbouring tiles still read, out of L2.
template <bool H>
__device__ __forceinline__ void stCS(void* p, unsigned i, float v) {
  if (H) {
    const __half h = __float2half_rn(v);
    asm volatile("st.global.cs.b16 [%0], %1;\n" ::"l"(reinterpret_cast<__half*>(p) + i),
                 "h"(__half_as_ushort(h))
                 : "memory");
  } else {
    asm volatile("st.global.cs.f32 [%0], %1;\n" ::"l"(reinterpret_cast<float*>(p) + i), "f"(v)
                 : "memory");
  }
}
// The value stS stores, as read back later.
template <bool H>
__device__ __forceinline__ float stored(float v) {
  return H ? __half2float(__float2half_rn(v)) : v;
}

// Periodic wrap of a coordinate at most two periods outside [0, m).
__host__ __device__ __forceinline__ int wrap3(int v, int m) {
  if (v < 0) v += m;
  if (v < 0) v += m;
  if (v >= m) v -= m;
  if (v >= m) v -= m;
  return v;
}
// Periodic wrap of any coordinate (tiles of lattices narrower than a tile).
__host__ __device__ __forceinline__ int wrap_any(int v, int m) {
  const int r = v % m;
  return r < 0 ? r + m : r;
}

__host__ __device__ __forceinline__ bool map_z(const Inst3& I, int z, int& zm) {
  if ((unsigned)z < (unsigned)I.nz) {
    zm = z;
    return true;
  }
  if (I.bc == BC_PER) {
    zm = wrap_any(z, I.nz);
    return true;
  }
  if (I.bc == BC_ZG) {
    zm = z < 0 ? 0 : I.nz - 1;
    return true;
  }
  return false;
}

__host__ __device__ __forceinline__ float rr2(const Inst3& I, int x, int y) {
  const float dx = x - I.cx, dy = y - I.cy;
  return dx * dx + dy * dy;
}
// Is column (x, y) in the nozzle wall ring R^2 <= r^2 < Ro^2?
__host__ __device__ __forceinline__ bool wall_column3(const Inst3& I, int x, int y) {
  const float r2 = rr2(I, x, y);
  return r2 >= I.R2 && r2 < I.Ro2;
}

// Kind of an in-domain cell: 0 fluid, 1 solid, 2 solid on a wetting face
// (a nozzle-wall cell with a lateral face neighbour in the channel, or the
// top layer of the plate).
__host__ __device__ int geom_kind3(const Inst3& I, int x, int y, int z) {
  if (I.geom == GEOM_NOZZLE) {
    if (z >= I.L || !wall_column3(I, x, y)) return 0;
    if (rr2(I, wrap3(x + 1, I.nx), y) < I.R2 || rr2(I, wrap3(x - 1, I.nx), y) < I.R2 ||
        rr2(I, x, wrap3(y + 1, I.ny)) < I.R2 || rr2(I, x, wrap3(y - 1, I.ny)) < I.R2)
      return 2;
    return 1;
  }
  if (I.geom == GEOM_PLATE) {
    if (z < I.wt) return z == I.wt - 1 ? 2 : 1;
    return 0;
  }
  return 0;
}

// Kind of any lattice point after the axial mapping (outside a closed
// domain: a non-wetting solid).
__host__ __device__ __forceinline__ int kind_at3(const Inst3& I, int x, int y, int z) {
  int zm;
  if (!map_z(I, z, zm)) return 1;
  return geom_kind3(I, wrap_any(x, I.nx), wrap_any(y, I.ny), zm);
}

__host__ __device__ __forceinline__ size_t cell3(const Inst3& I, int x, int y, int z) {
  return ((size_t)z * I.ny + y) * I.nx + x;
}
// index of (x, y, z), z in -2..nz+1, in a phi array of nz + 4 planes
__device__ __forceinline__ size_t ecell3(const Inst3& I, int x, int y, int z) {
  return ((size_t)(z + 2) * I.ny + y) * I.nx + x;
}

// phi with wetting ghosts at any lattice point (x, y, z), z in -2..nz+1, from
// phi of the fluid cells (an array of nz + 4 planes whose in-domain fluid
// entries hold sum g): fluid points take the value of their mapped cell;
// solid points the mean over fluid face neighbours of phi + h_s / kappa
// (h_s = h on a wetting face, else 0), or, touching fluid only along edges,
// the plain mean over those (reading of the wetting boundary condition of
// "Reproducing the experiment").
template <typename T>
__device__ T phi_hat3(const Inst3& I, const float* phi, int x, int y, int z, T hk_wet) {
  int zm;
  const int k = kind_at3(I, x, y, z);
  if (k == 0) {
    map_z(I, z, zm);
    return (T)phi[ecell3(I, wrap_any(x, I.nx), wrap_any(y, I.ny), zm)];
  }
  const T hk = k == 2 ? hk_wet : (T)0;
  T sum = 0;
  int cnt = 0;
  for (int i = 1; i <= 6; i++) {
    const int xx = x + ex3(i), yy = y + ey3(i), zz = z + ez3(i);
    if (kind_at3(I, xx, yy, zz) == 0) {
      map_z(I, zz, zm);
      sum += (T)phi[ecell3(I, wrap_any(xx, I.nx), wrap_any(yy, I.ny), zm)] + hk;
      cnt++;
    }
  }
  if (cnt) return sum / (T)cnt;
  for (int i = 7; i < 19; i++) {
    const int xx = x + ex3(i), yy = y + ey3(i), zz = z + ez3(i);
    if (kind_at3(I, xx, yy, zz) == 0) {
      map_z(I, zz, zm);
      sum += (T)phi[ecell3(I, wrap_any(xx, I.nx), wrap_any(yy, I.ny), zm)];
      cnt++;
    }
  }
  return cnt ? sum / (T)cnt : (T)0;
}

__device__ __forceinline__ float drive3(const Inst3& I, long long t) {
  long long tt = t;
  if (I.Tidle > 0) tt = t % (I.T1 + I.T2 + I.Tidle);
  if (tt < I.T1) return I.F0;
  if (tt < I.T1 + I.T2) return -I.Fneg;
  return 0.0f;
}

// 1 / x: hardware approximate reciprocal and one Newton-Raphson step for 1/x.
__device__ __forceinline__ float recip3(float x) {
  const float r = __fdividef(1.0f, x);
  return fmaf(r, fmaf(-x, r, 1.0f), r);
}

// Per-lattice constants of the collision, in registers.
struct CollK3 {
  float phis, inv_phis, A4, kappa, omq, inv_tphi, gamma, inv2q, qmt, nu_air, dnu, n0, Fd;
};

// Collision of one fluid cell (Eq. 4-6 and 8-10 lifted to D3Q19 / D3Q7).
//  fr: f_i - w_i n0; g: g_0..6; phi = sum g (raw); nb[i]: phi with wetting
//  ghosts at x + c_i (nb[0] at the cell).
//  Out: fs = post-collision f_i - w_i n0; gP[i-1] = q g_i + Omega_i (the part
//  that moves, i = 1..6); gS[i-1] = (1 - q) g_i (the part that stays); g0n =
//  g_0 + Omega_0; n, u_z, |u|^2.
__device__ __forceinline__ void collide3_cell(const float (&fr)[19], const float (&g)[7], float phi,
                                              const float (&nb)[19], bool driven, const CollK3& K,
                                              float (&fs)[19], float (&gP)[6], float (&gS)[6],
                                              float& g0n, float& n, float& uz, float& u2) {
  // isotropic D3Q19 stencils: lap = 6 sum_i w_i (phi_i - phi), from the
  // differences; grad = 3 sum_i w_i c_i phi_i
  const float pC = nb[0];
  float sf = 0.0f, se = 0.0f;
#pragma unroll
  for (int i = 1; i < 19; i++) {
    if (i <= 6)
      sf += nb[i] - pC;
    else
      se += nb[i] - pC;
  }
  const float lap = (1.0f / 3.0f) * sf + (1.0f / 6.0f) * se;
  float gxyz[3];
#pragma unroll
  for (int a = 0; a < 3; a++) {
    float fa = 0.0f, ea = 0.0f;
#pragma unroll
    for (int i = 1; i < 19; i++) {
      const int c = a == 0 ? ex3(i) : (a == 1 ? ey3(i) : ez3(i));
      if (c == 0) continue;
      const float v = c > 0 ? nb[i] : -nb[i];
      if (i <= 6)
        fa += v;
      else
        ea += v;
    }
    gxyz[a] = fa * (1.0f / 6.0f) + ea * (1.0f / 12.0f);
  }
  const float mu = K.A4 * phi * ((phi - K.phis) * (phi + K.phis)) - K.kappa * lap;
  float C = 0.5f * (phi * K.inv_phis + 1.0f);
  C = fminf(fmaxf(C, 0.0f), 1.0f);
  const float Fb = driven ? K.Fd * C : 0.0f;
  const float Fx = mu * gxyz[0], Fy = mu * gxyz[1], Fz = mu * gxyz[2] + Fb;
  // fr holds deviations f_i - w_i n0: their sum is n - n0
  float dn = 0.0f, mx = 0.0f, my = 0.0f, mz = 0.0f;
#pragma unroll
  for (int i = 0; i < 19; i++) {
    dn += fr[i];
    if (ex3(i)) mx += ex3(i) > 0 ? fr[i] : -fr[i];
    if (ey3(i)) my += ey3(i) > 0 ? fr[i] : -fr[i];
    if (ez3(i)) mz += ez3(i) > 0 ? fr[i] : -fr[i];
  }
  n = K.n0 + dn;
  const float n_lo = dn - (n - K.n0);  // n - (n0 + dn) exactly
  const float inv_hi = recip3(n);
  const float inv_n = fmaf(-n_lo * inv_hi, inv_hi, inv_hi);
  const float ux = (mx + 0.5f * Fx) * inv_n, uy = (my + 0.5f * Fy) * inv_n;
  uz = (mz + 0.5f * Fz) * inv_n;
  u2 = ux * ux + uy * uy + uz * uz;
  const float om = recip3(0.5f + 3.0f * (K.nu_air + C * K.dnu));
  const float pref = 3.0f - 1.5f * om;  // 3 (1 - 1 / (2 tau))
  // A_i - n0 = 3 (phi mu + n / 3) - n0 for i >= 1 (the lift of Eq. 6)
  const float p3 = dn + 3.0f * phi * mu;
  const float uF = ux * Fx + uy * Fy + uz * Fz;
  // opposite pairs: f*_i = (1 - om) f_i + w (a +- b) with
  // a = a0 + cu (a1 cu + a2 cF), b = b1 cu + pref cF (as in the 2-D step);
  // the rest direction takes the balance (mass conserved in FP32)
  const float omn = om * n;
  const float a0 = fmaf(om, fmaf(-1.5f * n, u2, p3), -pref * uF);
  const float a1 = 4.5f * omn, a2 = 3.0f * pref, b1 = 3.0f * omn;
  const float omc = 1.0f - om;
  float sum1 = 0.0f, sum2 = 0.0f;  // a of the face / edge pairs
#pragma unroll
  for (int i = 1; i < 19; i++) {
    // the first direction of each opposite pair: 1, 3, 5, 7, 8, 11, 12, 15, 16
    if (!(i == 1 || i == 3 || i == 5 || i == 7 || i == 8 || i == 11 || i == 12 || i == 15 ||
          i == 16))
      continue;
    const int ib = i <= 6 ? i + 1 : (i == 7 ? 10 : i == 8 ? 9 : i == 11 ? 14 : i == 12 ? 13 : i == 15 ? 18 : 17);
    const float w = i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f;
    const float cu = (float)ex3(i) * ux + (float)ey3(i) * uy + (float)ez3(i) * uz;
    const float cF = (float)ex3(i) * Fx + (float)ey3(i) * Fy + (float)ez3(i) * Fz;
    const float a = fmaf(cu, fmaf(a1, cu, a2 * cF), a0);
    const float b = fmaf(b1, cu, pref * cF);
    if (i <= 6) sum1 += a; else sum2 += a;
    fs[i] = fmaf(omc, fr[i], w * (a + b));
    fs[ib] = fmaf(omc, fr[ib], w * (a - b));
  }
  fs[0] = fmaf(omc, fr[0], fmaf(om, dn, -2.0f * fmaf(1.0f / 18.0f, sum1, (1.0f / 36.0f) * sum2)));
  // order parameter: D3Q7 with the rest direction special; the moving part
  // q g_i + Omega_i streams, (1 - q) g_i stays
  const float gmu = K.gamma * mu, pq = phi * K.inv2q;
  float sum_ge = 0.0f, sum_g = 0.0f;
#pragma unroll
  for (int i = 1; i < 7; i++) {
    const float cu = (float)ex3(i) * ux + (float)ey3(i) * uy + (float)ez3(i) * uz;
    const float ge = 0.5f * gmu + pq * cu;
    sum_ge += ge;
    sum_g += g[i];
    gP[i - 1] = fmaf(K.qmt, g[i], ge * K.inv_tphi);  // q g + (ge - g) / tau_phi
    gS[i - 1] = K.omq * g[i];
  }
  // rest: g0_0 = phi - sum_{i>=1} g0_i (the balance); phi - g_0 = sum g_i
  g0n = g[0] + (sum_g - sum_ge) * K.inv_tphi;
}

// ---------------------------------------------------------------------------
// The fused 3-D step.
constexpr int kW3 = 16;                   // warps of a CTA: rows y of the tile
constexpr int kThreads3 = 32 * kW3;
static_assert(kThreads3 == kStep3Threads, "step3 block size");
constexpr int kPopW32 = 26 * 32;          // words of one staged plane of a warp: f[19][32], g0[32], g1..6[6][32]
constexpr int kPopW16 = 19 * 16 + 32 + 6 * 16;  // FP16: f half pairs [19][16], g0 [32], g half pairs [6][16]
constexpr unsigned kFull = 0xffffffffu;
constexpr int kXch = 12;                  // values a cell sends to a neighbouring row
// bit of column (x + dx, y + dy) in a lane's 3 x 3 column mask
__host__ __device__ constexpr int cbit(int dx, int dy) { return (dy + 1) * 3 + (dx + 1); }

__device__ __forceinline__ void cp4_async(unsigned sa, const void* p) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(p) : "memory");
}
__device__ __forceinline__ void cp_commit3() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_wait3() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// Per-item constants and buffers, kept in shared memory rather than in
// registers (read where used).
struct Ctx3 {
  CollK3 K;
  const void* fin;
  const void* gin;
  const float* g0in;
  const float* phin;
  void* fout;
  void* gout;
  float* g0out;
  float* phout;
  // planes; axial boundary; solid planes from the bottom (nozzle length or
  // plate thickness), which are full planes (plate) or the wall ring; driven
  // planes below dzl (nozzle length, else all); cells of a plane
  int nz, bc, zsol, full, dzl, plane;
};
static_assert(sizeof(Ctx3) <= 40 * sizeof(float), "Ctx3 outgrew its shared-memory slot");

// Shared memory of one CTA, in words: the staged planes of every warp (two
// slots), the phi ring (four planes of the tile), the row exchange (two
// slots of kXch values per cell) and the diagnostics partials (two slots).
template <bool H>
struct Smem3 {
  static constexpr int PW = H ? kPopW16 : kPopW32;
  static constexpr int pops = kW3 * 2 * PW;
  static constexpr int ring = 4 * kW3 * 32;
  static constexpr int xch = 2 * kXch * kW3 * 32;
  static constexpr int diag = 2 * kW3 * 8;
  static constexpr int ctx = 40;  // the item's Ctx3
  static constexpr int words = pops + ring + xch + diag + ctx;
};

template <bool DIAG, bool H>
__global__ void __launch_bounds__(kThreads3, 1)
    step3_kernel(const Inst3* __restrict__ insts, const Item3* __restrict__ items, int n_items,
                 const long long* __restrict__ d_t, int t_off) {
  using S = Smem3<H>;
  extern __shared__ float4 smem4[];
  float* const sm = reinterpret_cast<float*>(smem4);
  float* const ring = sm + S::pops;      // [4][kW3][32]: phi of plane z in slot (z + 8) & 3
  float* const xch = ring + S::ring;     // [2][kXch][kW3][32]
  float* const dsm = xch + S::xch;       // [2][kW3][8]
  Ctx3* const ctx = reinterpret_cast<Ctx3*>(dsm + S::diag);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  float* const mypop = sm + w * 2 * S::PW;
  const unsigned mypop_a = (unsigned)__cvta_generic_to_shared(mypop);
  const long long t = d_t[0] + t_off;

  for (int item = blockIdx.x; item < n_items; item += gridDim.x) {
    const Item3 it = items[item];
    const Inst3& I = insts[it.inst];
    // a lattice whose numeric flag is set is frozen (uniform over the CTA)
    const bool lead = threadIdx.x == 0;
    if (__syncthreads_or(lead && (*(volatile const unsigned*)I.status & kStatusNumeric))) continue;
    const int nx = I.nx, ny = I.ny;
    const int z0 = it.z0, ch = it.ch;
    const int xu = it.xs - 2 + lane, yu = it.ys - 2 + w;  // unwrapped column of this thread
    const int x = wrap_any(xu, nx), y = wrap_any(yu, ny);
    const int cxy = y * nx + x;
    const int xe = min(it.xs + kTile3X, nx), ye = min(it.ys + kTile3Y, ny);
    const bool written = xu >= it.xs && xu < xe && yu >= it.ys && yu < ye;
    // collision results that flow into written cells (the ring of the tile)
    const bool used = xu >= it.xs - 1 && xu <= xe && yu >= it.ys - 1 && yu <= ye;
    // wall columns among (x + dx, y + dy): bit cbit(dx, dy)
    unsigned wallmask = 0u;
    if (I.geom == GEOM_NOZZLE) {
#pragma unroll
      for (int dy = -1; dy <= 1; dy++)
#pragma unroll
        for (int dx = -1; dx <= 1; dx++)
          if (wall_column3(I, wrap_any(x + dx, nx), wrap_any(y + dy, ny))) wallmask |= 1u << cbit(dx, dy);
    }
    const bool drive_col = I.geom != GEOM_NOZZLE || rr2(I, x, y) < I.R2;
    if (lead) {
      const int par = *I.cur;  // buffer of the state at t
      CollK3& K = ctx->K;
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
      K.Fd = drive3(I, t);
      ctx->fin = I.f[par];
      ctx->gin = I.g[par];
      ctx->g0in = I.g0[par];
      ctx->phin = I.phi[par];
      ctx->fout = I.f[par ^ 1];
      ctx->gout = I.g[par ^ 1];
      ctx->g0out = I.g0[par ^ 1];
      ctx->phout = I.phi[par ^ 1];
      ctx->nz = I.nz;
      ctx->bc = I.bc;
      ctx->zsol = I.geom == GEOM_NOZZLE ? I.L : (I.geom == GEOM_PLATE ? I.wt : 0);
      ctx->full = I.geom == GEOM_PLATE;
      ctx->dzl = I.geom == GEOM_NOZZLE ? I.L : 0x7fffffff;
      ctx->plane = nx * ny;
    }
    __syncthreads();
    const CollK3 K = ctx->K;  // in registers for the item
    // mapped plane of extended plane z (false: outside a closed domain)
    auto mapz = [&](int z, int& zm) -> bool {
      const int nzz = ctx->nz;
      if ((unsigned)z < (unsigned)nzz) {
        zm = z;
        return true;
      }
      const int bc = ctx->bc;
      if (bc == BC_PER) {
        zm = wrap_any(z, nzz);
        return true;
      }
      zm = z < 0 ? 0 : nzz - 1;
      return bc == BC_ZG;
    };
    // solid cells among the nine columns in mapped plane zm
    auto solid_of = [&](bool in, int zm) -> unsigned {
      if (!in) return 0x1FFu;
      return zm < ctx->zsol ? (ctx->full ? 0x1FFu : wallmask) : 0u;
    };
    // cell offsets fit in 32 bits: 19 nx ny nz < 2^31 (checked on the host)
    auto cell_of = [&](int zm) -> unsigned { return (unsigned)zm * (unsigned)ctx->plane + (unsigned)cxy; };

    // Stage the populations of plane zs (its mapped plane) into slot sl, as
    // one cp.async group (FP16: even lanes copy the half pair of their column
    // and the next; nx is even, so pairs never straddle the wrap).
    auto stage = [&](bool in, int zm, int sl, bool need) {
      if (need && in) {
        const unsigned N = (unsigned)ctx->plane * (unsigned)ctx->nz;
        const unsigned c = cell_of(zm);
        const unsigned d = mypop_a + sl * (S::PW * 4);
        if (!H) {
          const float* f = static_cast<const float*>(ctx->fin);
          const float* g = static_cast<const float*>(ctx->gin);
#pragma unroll
          for (int i = 0; i < 19; i++) cp4_async(d + (i * 32 + lane) * 4, f + (c + i * N));
          cp4_async(d + (19 * 32 + lane) * 4, ctx->g0in + c);
#pragma unroll
          for (int i = 0; i < 6; i++) cp4_async(d + ((20 + i) * 32 + lane) * 4, g + (c + i * N));
        } else {
          const __half* f = static_cast<const __half*>(ctx->fin);
          const __half* g = static_cast<const __half*>(ctx->gin);
          cp4_async(d + (304 + lane) * 4, ctx->g0in + c);
          if ((lane & 1) == 0) {
#pragma unroll
            for (int i = 0; i < 19; i++) cp4_async(d + (i * 16 + (lane >> 1)) * 4, f + (c + i * N));
#pragma unroll
            for (int i = 0; i < 6; i++) cp4_async(d + (336 + i * 16 + (lane >> 1)) * 4, g + (c + i * N));
          }
        }
      }
      cp_commit3();
    };
    auto load_cell = [&](int sl, float (&fr)[19], float (&gr)[7]) {
      const float* r = mypop + sl * S::PW;
      if (!H) {
#pragma unroll
        for (int i = 0; i < 19; i++) fr[i] = r[i * 32 + lane];
        gr[0] = r[19 * 32 + lane];
#pragma unroll
        for (int i = 1; i < 7; i++) gr[i] = r[(19 + i) * 32 + lane];
      } else {
        const __half* rh = reinterpret_cast<const __half*>(r);
#pragma unroll
        for (int i = 0; i < 19; i++) fr[i] = __half2float(rh[i * 32 + lane]);
        gr[0] = r[304 + lane];
#pragma unroll
        for (int i = 1; i < 7; i++) gr[i] = __half2float(rh[672 + (i - 1) * 32 + lane]);
      }
    };
    // phi with ghosts at (x + dx, y + dy, z) from the ring (lanes 0 and 31
    // read past their row, into the next row, ring plane or region of the
    // CTA's shared memory; their collisions are not used)
    auto ring_at = [&](int z, int dx, int dy) -> float {
      return ring[((((z + 8) & 3) * kW3) + w + dy) * 32 + lane + dx];
    };
    // phi with wetting ghosts at (x, y, z), z in -2 .. nz + 1
    auto phi_hat_at = [&](int z) -> float {
      return ctx->phin[(unsigned)(z + 2) * (unsigned)ctx->plane + (unsigned)cxy];
    };

    // prologue: populations of plane z0 - 1, phi of planes z0 - 2 .. z0.
    // The first and last rows of the CTA only give phi to the stencils of
    // their neighbour rows: they stage nothing and do not collide.
    const bool coll = w != 0 && w != kW3 - 1;
    int zmCur;
    bool inCur = mapz(z0 - 1, zmCur);
    stage(inCur, zmCur, 0, coll);
#pragma unroll
    for (int j = -2; j <= 0; j++) ring[((((z0 + j) + 8) & 3) * kW3 + w) * 32 + lane] = phi_hat_at(z0 + j);
    __syncthreads();
    // Carried from plane Zc - 1 to the next iteration: its upward movers
    // (f_5 own, f_11 from x - 1, f_12 from x + 1, f_15 from y - 1, f_16 from
    // y + 1, the moving g_5 own), its own f*_11, f*_12, f*_15, f*_16
    // (bounce-back of f_14, f_13, f_18, f_17), and, for its cells whose pulls
    // were stored at the gather, the parts of phi = g_0 + ((g_1 + g_2) +
    // (g_3 + g_4) + (g_5 + g_6)) known then and the stay part of g_6.
    float hu5 = 0.f, hu11 = 0.f, hu12 = 0.f, hu15 = 0.f, hu16 = 0.f, hug5 = 0.f;
    float bb11 = 0.f, bb12 = 0.f, bb15 = 0.f, bb16 = 0.f;
    float pg0 = 0.f, pg14 = 0.f, pg5 = 0.f, gs6 = 0.f;
    unsigned smPrev, smCur = solid_of(inCur, zmCur);
    {
      int zm;
      const bool in = mapz(z0 - 2, zm);
      smPrev = solid_of(in, zm);
    }
    bool drvCur = drive_col && zmCur < ctx->dzl;
    double sn = 0.0;  // diagnostics: lanes 3, 4, 5 of the first row total n, phi, n u_z
    // phi at the centre and the four faces (+x, -x, +y, -y) of planes Zc - 1
    // (pm) and Zc (pc), carried from the iterations that loaded them
    float pm[5], pc[5];
    {
      constexpr int fx[5] = {0, 1, -1, 0, 0}, fy[5] = {0, 0, 0, 1, -1};
#pragma unroll
      for (int j = 0; j < 5; j++) {
        pm[j] = ring_at(z0 - 2, fx[j], fy[j]);
        pc[j] = ring_at(z0 - 1, fx[j], fy[j]);
      }
    }
#pragma unroll 1
    for (int k = 0; k < ch + 2; k++) {
      const int Zc = z0 - 1 + k;
      // the next plane: its mapping, staging, solid cells and drive
      int zmN;
      const bool inN = mapz(Zc + 1, zmN);
      stage(inN, zmN, (k + 1) & 1, coll && k <= ch);
      const float phn = k <= ch ? phi_hat_at(Zc + 2) : 0.0f;  // into the ring before the barrier
      const unsigned smN = solid_of(inN, zmN);
      const bool drvN = drive_col && zmN < ctx->dzl;
      const bool fluidC = ((smCur >> cbit(0, 0)) & 1u) == 0u;
      float fs[19], gP[6], gS[6], g0n, n, uz, u2, phi;
      float s1, s2, s11, s12, s13, s14, sg1, sg2;
      float* X = xch + (k & 1) * (kXch * kW3 * 32);
      if (coll) {
        cp_wait3<1>();  // this lane's copies of plane Zc have landed
        if (H) __syncwarp();  // odd lanes read the half pairs their even neighbour copied
        // ---- collision of (x, y, Zc)
        {
          float fr[19], gr[7], nb[19];
          load_cell(k & 1, fr, gr);
          // D3Q19 neighbours: plane Zc (centre, faces, the four corners),
          // planes Zc +- 1 (centre and faces)
          float pn[5];
          {
            constexpr int fx[5] = {0, 1, -1, 0, 0}, fy[5] = {0, 0, 0, 1, -1};
#pragma unroll
            for (int j = 0; j < 5; j++) pn[j] = ring_at(Zc + 1, fx[j], fy[j]);
          }
          nb[0] = pc[0];
          nb[1] = pc[1];
          nb[2] = pc[2];
          nb[3] = pc[3];
          nb[4] = pc[4];
          nb[5] = pn[0];
          nb[6] = pm[0];
          nb[7] = ring_at(Zc, 1, 1);
          nb[8] = ring_at(Zc, -1, 1);
          nb[9] = ring_at(Zc, 1, -1);
          nb[10] = ring_at(Zc, -1, -1);
          nb[11] = pn[1];
          nb[12] = pn[2];
          nb[13] = pm[1];
          nb[14] = pm[2];
          nb[15] = pn[3];
          nb[16] = pn[4];
          nb[17] = pm[3];
          nb[18] = pm[4];
#pragma unroll
          for (int j = 0; j < 5; j++) {
            pm[j] = pc[j];
            pc[j] = pn[j];
          }
          phi = gr[0] + ((gr[1] + gr[2]) + (gr[3] + gr[4]) + (gr[5] + gr[6]));
          collide3_cell(fr, gr, phi, nb, drvCur, K, fs, gP, gS, g0n, n, uz, u2);
        }
        if (used && fluidC && !(u2 < 0.09f)) atomicOr(I.status, kStatusNumeric);
        // movers that cross lanes (along x)
        s1 = __shfl_up_sync(kFull, fs[1], 1);
        s2 = __shfl_down_sync(kFull, fs[2], 1);
        s11 = __shfl_up_sync(kFull, fs[11], 1);
        s12 = __shfl_down_sync(kFull, fs[12], 1);
        s13 = __shfl_up_sync(kFull, fs[13], 1);
        s14 = __shfl_down_sync(kFull, fs[14], 1);
        sg1 = __shfl_up_sync(kFull, gP[0], 1);
        sg2 = __shfl_down_sync(kFull, gP[1], 1);
        // movers that cross rows (along y), to the exchange: towards y + 1
        // f_3, f_7, f_8, f_15, f_17, g_3; towards y - 1 f_4, f_9, f_10,
        // f_16, f_18, g_4
        const float out[kXch] = {fs[3], fs[7], fs[8], fs[15], fs[17], gP[2],
                                 fs[4], fs[9], fs[10], fs[16], fs[18], gP[3]};
#pragma unroll
        for (int v = 0; v < kXch; v++) X[(v * kW3 + w) * 32 + lane] = out[v];
      }
      ring[((((Zc + 2) + 8) & 3) * kW3 + w) * 32 + lane] = phn;
      if (DIAG && coll) {
        // diagnostics of the state at t over the written fluid cells of
        // plane Zc: the row sums (FP32) of e, e n, e n u_z, n, phi, n u_z
        float dg[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        if (k >= 1 && k <= ch && written && fluidC) {
          const float e = fminf(fmaxf(phi * K.inv_phis, 0.0f), 1.0f);
          dg[0] = e;
          dg[1] = e * n;
          dg[2] = dg[1] * uz;
          dg[3] = n;
          dg[4] = phi;
          dg[5] = n * uz;
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1)
#pragma unroll
          for (int j = 0; j < 6; j++) dg[j] += __shfl_down_sync(kFull, dg[j], o);
        if (lane == 0) {
          float* D = dsm + ((k & 1) * kW3 + w) * 8;
#pragma unroll
          for (int j = 0; j < 6; j++) D[j] = dg[j];
        }
      }
      __syncthreads();
      if (DIAG && w == 0 && lane < 6 && k >= 1 && k <= ch) {
        // the first row (which does not collide): lane j sums value j of the
        // rows in FP64; plane sums of e, e n, e n u_z, item totals of n,
        // phi, n u_z
        double sr = 0.0;
        for (int ww = 1; ww < kW3 - 1; ww++) sr += (double)dsm[((k & 1) * kW3 + ww) * 8 + lane];
        if (lane < 3)
          atomicAdd(I.rows + lane * ctx->nz + Zc, sr);
        else
          sn += sr;
      }
      if (coll) {
        // incoming movers from the neighbouring rows: (x - c_x, y - c_y)
        // (lanes 0 and 31 read past their row, the second and second-last
        // rows read the first and last, which hold no movers: those values
        // flow only into cells that are not written; every address stays in
        // the CTA's shared memory)
        auto xget = [&](int v, int dx, int dy) -> float { return X[(v * kW3 + w + dy) * 32 + lane + dx]; };
        const float u3 = xget(0, 0, -1), u7 = xget(1, -1, -1), u8 = xget(2, 1, -1);
        const float u15 = xget(3, 0, -1), u17 = xget(4, 0, -1), ug3 = xget(5, 0, -1);
        const float d4 = xget(6, 0, 1), d9 = xget(7, -1, 1), d10 = xget(8, 1, 1);
        const float d16 = xget(9, 0, 1), d18 = xget(10, 0, 1), dg4 = xget(11, 0, 1);
        // does any cell of the warp have a solid source in planes Zc - 1, Zc
        const bool any_solid = __any_sync(kFull, (smPrev | smCur) != 0u);
        auto sol = [](unsigned m, int dx, int dy) { return ((m >> cbit(dx, dy)) & 1u) != 0u; };
        // ---- plane Zc - 1: the downward movers of plane Zc, then store
        if (k >= 2) {
          float f6 = fs[6], f13 = s13, f14 = s14, f17 = u17, f18 = d18, p6 = gP[5];
          if (any_solid) {
            const bool s00 = sol(smCur, 0, 0);
            f6 = s00 ? hu5 : f6;
            p6 = s00 ? hug5 : p6;
            f13 = sol(smCur, -1, 0) ? bb12 : f13;
            f14 = sol(smCur, 1, 0) ? bb11 : f14;
            f17 = sol(smCur, 0, -1) ? bb16 : f17;
            f18 = sol(smCur, 0, 1) ? bb15 : f18;
          }
          // solid cells are never stored: both buffers hold 0 there
          if (written && !sol(smPrev, 0, 0)) {
            const int zo = Zc - 1;
            const float g6 = gs6 + p6;
            const unsigned N = (unsigned)ctx->plane * (unsigned)ctx->nz, c = cell_of(zo);
            stCS<H>(ctx->fout, 6 * N + c, f6);
            stCS<H>(ctx->fout, 13 * N + c, f13);
            stCS<H>(ctx->fout, 14 * N + c, f14);
            stCS<H>(ctx->fout, 17 * N + c, f17);
            stCS<H>(ctx->fout, 18 * N + c, f18);
            stCS<H>(ctx->gout, 5 * N + c, g6);
            // phi of the new state as the next step sums it (stored values)
            stCS<false>(ctx->phout, c + 2u * (unsigned)ctx->plane, pg0 + (pg14 + (pg5 + stored<H>(g6))));
          }
        }
        // ---- gather the pulls of plane Zc (rest, in-plane movers, upward
        // movers of plane Zc - 1, stay parts)
        {
          float f1 = s1, f2 = s2, f3 = u3, f4 = d4, f7 = u7, f8 = u8, f9 = d9, f10 = d10;
          float f5 = hu5, f11 = hu11, f12 = hu12, f15 = hu15, f16 = hu16;
          float q1 = sg1, q2 = sg2, q3 = ug3, q4 = dg4, q5 = hug5;
          if (any_solid) {
            const bool cxm = sol(smCur, -1, 0), cxp = sol(smCur, 1, 0);
            const bool cym = sol(smCur, 0, -1), cyp = sol(smCur, 0, 1), p00 = sol(smPrev, 0, 0);
            f1 = cxm ? fs[2] : f1;
            q1 = cxm ? gP[1] : q1;
            f2 = cxp ? fs[1] : f2;
            q2 = cxp ? gP[0] : q2;
            f3 = cym ? fs[4] : f3;
            q3 = cym ? gP[3] : q3;
            f4 = cyp ? fs[3] : f4;
            q4 = cyp ? gP[2] : q4;
            f7 = sol(smCur, -1, -1) ? fs[10] : f7;
            f8 = sol(smCur, 1, -1) ? fs[9] : f8;
            f9 = sol(smCur, -1, 1) ? fs[8] : f9;
            f10 = sol(smCur, 1, 1) ? fs[7] : f10;
            f5 = p00 ? fs[6] : f5;
            q5 = p00 ? gP[5] : q5;
            f11 = sol(smPrev, -1, 0) ? fs[14] : f11;
            f12 = sol(smPrev, 1, 0) ? fs[13] : f12;
            f15 = sol(smPrev, 0, -1) ? fs[18] : f15;
            f16 = sol(smPrev, 0, 1) ? fs[17] : f16;
          }
          // every pull of plane Zc but f_6, f_13, f_14, f_17, f_18 and the
          // moving part of g_6 is complete: store it now
          if (written && k >= 1 && k <= ch && fluidC) {
            const unsigned N = (unsigned)ctx->plane * (unsigned)ctx->nz, c = cell_of(Zc);
            const float fo[14] = {fs[0], f1, f2, f3, f4, f5, f7, f8, f9, f10, f11, f12, f15, f16};
            constexpr int fi[14] = {0, 1, 2, 3, 4, 5, 7, 8, 9, 10, 11, 12, 15, 16};
#pragma unroll
            for (int j = 0; j < 14; j++) stCS<H>(ctx->fout, fi[j] * N + c, fo[j]);
            const float go[6] = {g0n, gS[0] + q1, gS[1] + q2, gS[2] + q3, gS[3] + q4, gS[4] + q5};
            stCS<false>(ctx->g0out, c, go[0]);
#pragma unroll
            for (int j = 1; j < 6; j++) stCS<H>(ctx->gout, (j - 1) * N + c, go[j]);
            pg0 = go[0];
            pg14 = (stored<H>(go[1]) + stored<H>(go[2])) + (stored<H>(go[3]) + stored<H>(go[4]));
            pg5 = stored<H>(go[5]);
            gs6 = gS[5];
          }
        }
        hu5 = fs[5]; hu11 = s11; hu12 = s12; hu15 = u15; hu16 = d16; hug5 = gP[4];
        bb11 = fs[11]; bb12 = fs[12]; bb15 = fs[15]; bb16 = fs[16];
      }
      smPrev = smCur;
      smCur = smN;
      drvCur = drvN;
    }
    cp_wait3<0>();  // no copy may land after the CTA moves on
    if (DIAG && w == 0 && lane >= 3 && lane < 6) atomicAdd(I.sums + (lane - 3), sn);
  }
}

// phi with wetting ghosts of the state in buffer *cur (next: the other) on
// the listed solid cells and on every point of the four extended planes; reads
// in-domain fluid entries only, so the writes never race with the reads.
// Grid: (blocks, lattices).
__global__ void __launch_bounds__(256) ghost3_kernel(const Inst3* __restrict__ insts, int next) {
  const Inst3& I = insts[blockIdx.y];
  if (*(volatile const unsigned*)I.status & kStatusNumeric) return;
  float* phi = I.phi[*I.cur ^ next];
  const long long plane = (long long)I.nx * I.ny;
  const long long total = I.n_ghost + 4 * plane;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    if (k < I.n_ghost) {
      const int c = I.ghost[k];
      x = c % I.nx;
      y = (c / I.nx) % I.ny;
      z = c / (I.nx * I.ny);
    } else {
      const long long e = k - I.n_ghost;
      const int p = (int)(e / plane), r = (int)(e % plane);
      x = r % I.nx;
      y = r / I.nx;
      z = p < 2 ? p - 2 : I.nz + (p - 2);
    }
    phi[ecell3(I, x, y, z)] = phi_hat3<float>(I, phi, x, y, z, I.hk);
  }
}

// ---------------------------------------------------------------------------
// Initialisation (FP64, then rounded to the storage), into buffer *cur; the
// other buffer's f is the FP64 scratch of phi0.
__device__ unsigned long long splitmix64_3(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__global__ void init_phi3_kernel(const Inst3* __restrict__ insts, int index) {
  const Inst3& I = insts[index];
  double* phi0 = static_cast<double*>(I.f[*I.cur ^ 1]);
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= I.nx || y >= I.ny) return;
  double v = 0.0;
  if (geom_kind3(I, x, y, z) == 0) {
    if (I.init_kind == INIT_MENISCUS) {
      const double dx = x - 0.5 * (I.nx - 1), dy = y - 0.5 * (I.ny - 1);
      const double r = sqrt(dx * dx + dy * dy), R = sqrt((double)I.R2);
      if (r * r < (double)I.R2) {
        v = I.d_phis * tanh((I.L - z) / I.d_W);
        if (fabs((double)(z - I.L)) < 2.0 * I.d_W) {
          unsigned long long ctr = ((unsigned long long)(unsigned)z << 42) ^
                                   ((unsigned long long)(unsigned)y << 21) ^ (unsigned)x;
          unsigned long long rr = splitmix64_3(I.seed ^ splitmix64_3(ctr));
          v += I.jitter * (2.0 * ((double)(rr >> 11) * (1.0 / 9007199254740992.0)) - 1.0);
        }
      } else if (z < I.L) {
        v = -I.d_phis;
      } else {
        const double dr = r - R, dz = (double)(z - I.L);
        v = I.d_phis * tanh(-sqrt(dr * dr + dz * dz) / I.d_W);
      }
    } else if (I.init_kind == INIT_DROP) {
      double dx = x - I.init_x, dy = y - I.init_y, dz = z - I.init_z;
      dx -= I.nx * floor(dx / I.nx + 0.5);
      dy -= I.ny * floor(dy / I.ny + 0.5);
      v = I.d_phis * tanh((I.init_r - sqrt(dx * dx + dy * dy + dz * dz)) / I.d_W);
    } else if (I.init_kind == INIT_FLAT) {
      v = I.d_phis * tanh((I.init_y - z) / I.d_W);
    } else {
      v = I.init_r;
    }
  }
  phi0[cell3(I, x, y, z)] = v;
}

// phi0 with wetting ghosts (FP64) at any lattice point
__device__ double phi0_hat3(const Inst3& I, const double* phi0, int x, int y, int z) {
  const int k = kind_at3(I, x, y, z);
  int zm = 0;
  if (k == 0) {
    map_z(I, z, zm);
    return phi0[cell3(I, wrap_any(x, I.nx), wrap_any(y, I.ny), zm)];
  }
  const double hk = k == 2 ? I.d_h / I.d_kappa : 0.0;
  double sum = 0.0;
  int cnt = 0;
  for (int i = 1; i <= 6; i++) {
    const int xx = x + ex3(i), yy = y + ey3(i), zz = z + ez3(i);
    if (kind_at3(I, xx, yy, zz) == 0) {
      map_z(I, zz, zm);
      sum += phi0[cell3(I, wrap_any(xx, I.nx), wrap_any(yy, I.ny), zm)] + hk;
      cnt++;
    }
  }
  if (cnt) return sum / cnt;
  for (int i = 7; i < 19; i++) {
    const int xx = x + ex3(i), yy = y + ey3(i), zz = z + ez3(i);
    if (kind_at3(I, xx, yy, zz) == 0) {
      map_z(I, zz, zm);
      sum += phi0[cell3(I, wrap_any(xx, I.nx), wrap_any(yy, I.ny), zm)];
      cnt++;
    }
  }
  return cnt ? sum / cnt : 0.0;
}

// equilibrium populations of phi0 at rest (solid cells 0); phi of the fluid
// cells as the step sums it
template <bool H>
__global__ void init_pop3_kernel(const Inst3* __restrict__ insts, int index) {
  const Inst3& I = insts[index];
  const int par = *I.cur;
  const double* phi0 = static_cast<const double*>(I.f[par ^ 1]);
  void* F = I.f[par];
  void* G = I.g[par];
  float* G0 = I.g0[par];
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= I.nx || y >= I.ny) return;
  const size_t N = (size_t)I.nx * I.ny * I.nz, c = cell3(I, x, y, z);
  if (geom_kind3(I, x, y, z) != 0) {
    for (int i = 0; i < 19; i++) stS<H>(F, i * N + c, 0.0f);
    for (int i = 0; i < 6; i++) stS<H>(G, i * N + c, 0.0f);
    G0[c] = 0.0f;
    return;
  }
  const double p0 = phi0[c];
  double lap = 0.0;
  for (int i = 1; i < 19; i++)
    lap += 6.0 * (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0) *
           (phi0_hat3(I, phi0, x + ex3(i), y + ey3(i), z + ez3(i)) - p0);
  const double mu = 4.0 * I.d_A * p0 * (p0 * p0 - I.d_phis * I.d_phis) - I.d_kappa * lap;
  const double n = I.d_n0, p = p0 * mu + n / 3.0;
  for (int i = 0; i < 19; i++) {
    const double w = i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    const double Ai = i == 0 ? 3.0 * n - 6.0 * p : 3.0 * p;
    stS<H>(F, i * N + c, (float)(w * Ai - w * n));
  }
  const float g0 = (float)(p0 - 3.0 * I.d_gamma * mu);
  G0[c] = g0;
  const float gi = (float)(0.5 * I.d_gamma * mu), gq = stored<H>(gi);
  for (int i = 0; i < 6; i++) stS<H>(G, i * N + c, gi);
  I.phi[par][ecell3(I, x, y, z)] = g0 + ((gq + gq) + (gq + gq) + (gq + gq));
}

// Export: absolute FP32 populations of the current state (solid cells 0).
// Import: encode them into the current buffer and sum phi of the fluid cells.
template <bool H, bool EXPORT>
__global__ void convert3_kernel(const Inst3* __restrict__ insts, int index, float* f, float* g) {
  const Inst3& I = insts[index];
  const int par = *I.cur;
  void* F = I.f[par];
  void* G = I.g[par];
  float* G0 = I.g0[par];
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= I.nx || y >= I.ny) return;
  const size_t N = (size_t)I.nx * I.ny * I.nz, c = cell3(I, x, y, z);
  const bool fluid = geom_kind3(I, x, y, z) == 0;
  if (EXPORT) {
    for (int i = 0; i < 19; i++) f[i * N + c] = fluid ? ldS<H>(F, i * N + c) + w3(i) * I.n0 : 0.0f;
    g[c] = fluid ? G0[c] : 0.0f;
    for (int i = 1; i < 7; i++) g[i * N + c] = fluid ? ldS<H>(G, (i - 1) * N + c) : 0.0f;
  } else {
    if (!fluid) {
      for (int i = 0; i < 19; i++) stS<H>(F, i * N + c, 0.0f);
      for (int i = 0; i < 6; i++) stS<H>(G, i * N + c, 0.0f);
      G0[c] = 0.0f;
      return;
    }
    float gq[7];
    for (int i = 0; i < 19; i++) stS<H>(F, i * N + c, f[i * N + c] - w3(i) * I.n0);
    G0[c] = g[c];
    gq[0] = g[c];
    for (int i = 1; i < 7; i++) {
      stS<H>(G, (i - 1) * N + c, g[i * N + c]);
      gq[i] = stored<H>(g[i * N + c]);
    }
    I.phi[par][ecell3(I, x, y, z)] = gq[0] + ((gq[1] + gq[2]) + (gq[3] + gq[4]) + (gq[5] + gq[6]));
  }
}

__global__ void phi3_kernel(const Inst3* __restrict__ insts, int index, float* out) {
  const Inst3& I = insts[index];
  const float* phi = I.phi[*I.cur];
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= I.nx || y >= I.ny) return;
  out[cell3(I, x, y, z)] = geom_kind3(I, x, y, z) == 0 ? phi[ecell3(I, x, y, z)] : 0.0f;
}

__global__ void flip3_kernel(const Inst3* __restrict__ insts, int n_inst) {
  for (int k = threadIdx.x; k < n_inst; k += blockDim.x) {
    const Inst3& I = insts[k];
    if (!(*(volatile const unsigned*)I.status & kStatusNumeric)) *I.cur ^= 1;
  }
}

dim3 grid3(const Inst3& h) { return dim3((h.nx + 31) / 32, (h.ny + 3) / 4, h.nz); }

}  // namespace

int ghost_cells3(const Inst3& h, int* out) {
  int zmax = 0;
  if (h.geom == GEOM_NOZZLE) zmax = std::min(h.L, h.nz);
  if (h.geom == GEOM_PLATE) zmax = std::min(h.wt, h.nz);
  int cnt = 0;
  for (int z = 0; z < zmax; z++)
    for (int y = 0; y < h.ny; y++)
      for (int x = 0; x < h.nx; x++) {
        if (geom_kind3(h, x, y, z) == 0) continue;
        bool reach = false;
        for (int i = 1; i < 19 && !reach; i++)
          reach = kind_at3(h, x + ex3(i), y + ey3(i), z + ez3(i)) == 0;
        if (!reach) continue;
        if (out) out[cnt] = (int)cell3(h, x, y, z);
        cnt++;
      }
  return cnt;
}

// Tiles of 28 x 12 columns, z chunks of `chunk` planes; a z chunk of every
// tile of every lattice before the next chunk, tiles row-major, so that
// CTAs running at the same time march over neighbouring tiles (their halo
// reads meet in L2).
int make_items3(const Inst3* h, int n_inst, int chunk, Item3* out) {
  int zc_max = 0;
  for (int k = 0; k < n_inst; k++) zc_max = std::max(zc_max, (h[k].nz + chunk - 1) / chunk);
  int cnt = 0;
  for (int zc = 0; zc < zc_max; zc++)
    for (int k = 0; k < n_inst; k++) {
      const Inst3& I = h[k];
      const int z0 = zc * chunk;
      if (z0 >= I.nz) continue;
      const int ch = std::min(chunk, I.nz - z0);
      for (int ys = 0; ys < I.ny; ys += kTile3Y)
        for (int xs = 0; xs < I.nx; xs += kTile3X) {
          if (out) out[cnt] = Item3{k, xs, ys, z0, ch};
          cnt++;
        }
    }
  return cnt;
}

size_t step3_smem_bytes(bool h16) {
  return (h16 ? Smem3<true>::words : Smem3<false>::words) * sizeof(float);
}

cudaError_t set_step3_smem_limit() {
  cudaError_t e;
  const int b32 = (int)step3_smem_bytes(false), b16 = (int)step3_smem_bytes(true);
  if ((e = cudaFuncSetAttribute(step3_kernel<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b32)))
    return e;
  if ((e = cudaFuncSetAttribute(step3_kernel<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, b32)))
    return e;
  if ((e = cudaFuncSetAttribute(step3_kernel<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b16)))
    return e;
  return cudaFuncSetAttribute(step3_kernel<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, b16);
}

cudaError_t launch_init3(const Inst3* d, const Inst3& h, int index, cudaStream_t s) {
  init_phi3_kernel<<<grid3(h), dim3(32, 4), 0, s>>>(d, index);
  if (h.fp16)
    init_pop3_kernel<true><<<grid3(h), dim3(32, 4), 0, s>>>(d, index);
  else
    init_pop3_kernel<false><<<grid3(h), dim3(32, 4), 0, s>>>(d, index);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  return launch_ghost3(d + index, &h, 1, false, s);
}

cudaError_t launch_step3(const Inst3* d, const Item3* items, int n_items, int n_inst,
                         const long long* d_t, int t_off, bool diag, bool h16, cudaStream_t s) {
  (void)n_inst;
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return e;
  const int grid = std::max(1, std::min(n_items, sms));
  const size_t sb = step3_smem_bytes(h16);
  if (h16) {
    if (diag)
      step3_kernel<true, true><<<grid, kThreads3, sb, s>>>(d, items, n_items, d_t, t_off);
    else
      step3_kernel<false, true><<<grid, kThreads3, sb, s>>>(d, items, n_items, d_t, t_off);
  } else {
    if (diag)
      step3_kernel<true, false><<<grid, kThreads3, sb, s>>>(d, items, n_items, d_t, t_off);
    else
      step3_kernel<false, false><<<grid, kThreads3, sb, s>>>(d, items, n_items, d_t, t_off);
  }
  return cudaGetLastError();
}

cudaError_t launch_ghost3(const Inst3* d, const Inst3* h, int n_inst, bool next, cudaStream_t s) {
  long long most = 0;
  for (int k = 0; k < n_inst; k++)
    most = std::max(most, (long long)h[k].n_ghost + 4LL * h[k].nx * h[k].ny);
  const int bx = (int)std::max(1LL, std::min(256LL, (most + 255) / 256));
  ghost3_kernel<<<dim3(bx, n_inst), 256, 0, s>>>(d, next ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_flip3(const Inst3* d, int n_inst, cudaStream_t s) {
  flip3_kernel<<<1, 256, 0, s>>>(d, n_inst);
  return cudaGetLastError();
}

cudaError_t launch_export3(const Inst3* d, const Inst3& h, int index, float* f, float* g,
                           cudaStream_t s) {
  if (h.fp16)
    convert3_kernel<true, true><<<grid3(h), dim3(32, 4), 0, s>>>(d, index, f, g);
  else
    convert3_kernel<false, true><<<grid3(h), dim3(32, 4), 0, s>>>(d, index, f, g);
  return cudaGetLastError();
}

cudaError_t launch_import3(const Inst3* d, const Inst3& h, int index, const float* f,
                           const float* g, cudaStream_t s) {
  float* fm = const_cast<float*>(f);
  float* gm = const_cast<float*>(g);
  if (h.fp16)
    convert3_kernel<true, false><<<grid3(h), dim3(32, 4), 0, s>>>(d, index, fm, gm);
  else
    convert3_kernel<false, false><<<grid3(h), dim3(32, 4), 0, s>>>(d, index, fm, gm);
  cudaError_t e = cudaGetLastError();
  if (e) return e;
  return launch_ghost3(d + index, &h, 1, false, s);
}

cudaError_t launch_phi3(const Inst3* d, const Inst3& h, int index, float* out, cudaStream_t s) {
  phi3_kernel<<<grid3(h), dim3(32, 4), 0, s>>>(d, index, out);
  return cudaGetLastError();
}

}  // namespace ij
