// Kernels of the 3-D lift (D3Q19 f, D3Q7 g) of the binary-fluid LBM inkjet
// step (He et al., arXiv:1702.04487, Eq. 3-10 lifted by moment matching).
//
// One time step is two launches over all cells of a lattice:
//  collide3: moments, ghost-aware D3Q19 stencils of phi, chemical potential,
//            drive, half-force velocity, collision of f (Eq. 4-6 lifted) and
//            of g (Eq. 8-10 lifted); writes the post-collision copy;
//  stream3:  pulls f*_i(x - c_i) with halfway bounce-back and
//            g_i = (1-q) g_i(x) + P_i(x - c_i) (Eq. 8), in place into the
//            state, and refreshes phi.
// Storage is FP32 or FP16 (f deviations and g_1..6); arithmetic is FP32.
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <math.h>

#include "lbm3d.cuh"

namespace ij {
namespace {

// D3Q19 directions in the public order: rest, +-x, +-y, +-z, then the edges.
__device__ __forceinline__ constexpr int ex3(int i) {
  return i == 1 || i == 7 || i == 9 || i == 11 || i == 13 ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14 ? -1 : 0);
}
__device__ __forceinline__ constexpr int ey3(int i) {
  return i == 3 || i == 7 || i == 8 || i == 15 || i == 17 ? 1
         : (i == 4 || i == 9 || i == 10 || i == 16 || i == 18 ? -1 : 0);
}
__device__ __forceinline__ constexpr int ez3(int i) {
  return i == 5 || i == 11 || i == 12 || i == 15 || i == 16 ? 1
         : (i == 6 || i == 13 || i == 14 || i == 17 || i == 18 ? -1 : 0);
}
__device__ __forceinline__ constexpr int opp3(int i) {
  return i == 0 ? 0 : (i <= 6 ? (i % 2 ? i + 1 : i - 1) : (i == 7 ? 10 : i == 8 ? 9 : i == 9 ? 8 : i == 10 ? 7 : i == 11 ? 14 : i == 12 ? 13 : i == 13 ? 12 : i == 14 ? 11 : i == 15 ? 18 : i == 16 ? 17 : i == 17 ? 16 : 15));
}
__device__ __forceinline__ constexpr float w3(int i) {
  return i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
}

template <bool H>
__device__ __forceinline__ float ldS(const void* p, size_t i) {
  if (H) return __half2float(reinterpret_cast<const __half*>(p)[i]);
  return __ldg(reinterpret_cast<const float*>(p) + i);
}
template <bool H>
__device__ __forceinline__ void stS(void* p, size_t i, float v) {
  if (H)
    reinterpret_cast<__half*>(p)[i] = __float2half_rn(v);
  else
    reinterpret_cast<float*>(p)[i] = v;
}
// The value stS stores, as read back later.  Kernels that need what they
// just stored use this instead of a load: ldS goes through the read-only
// path, which does not see the kernel's own stores.
template <bool H>
__device__ __forceinline__ float stored(float v) {
  return H ? __half2float(__float2half_rn(v)) : v;
}

// Periodic wrap of a coordinate at most two periods outside [0, m) (every
// caller offsets an in-range coordinate by one or two cells): compares and
// adds instead of an integer division.
__device__ __forceinline__ int wrap3(int v, int m) {
  if (v < 0) v += m;
  if (v < 0) v += m;
  if (v >= m) v -= m;
  if (v >= m) v -= m;
  return v;
}

// Periodic wrap of v >= -m into [0, m): a compare and add, and a remainder
// only on the rare path past one period (halo columns and rows of lattices
// narrower than a tile).
__device__ __forceinline__ int wrap_tile(int v, int m) {
  if (v < 0) v += m;
  if (v >= m) v %= m;
  return v;
}

__device__ __forceinline__ bool map_z(const Inst3& I, int z, int& zm) {
  if ((unsigned)z < (unsigned)I.nz) {
    zm = z;
    return true;
  }
  if (I.bc == BC_PER) {
    zm = wrap3(z, I.nz);
    return true;
  }
  if (I.bc == BC_ZG) {
    zm = z < 0 ? 0 : I.nz - 1;
    return true;
  }
  return false;
}

__device__ __forceinline__ float rr2(const Inst3& I, int x, int y) {
  const float dx = x - I.cx, dy = y - I.cy;
  return dx * dx + dy * dy;
}

// Kind of an in-domain cell: 0 fluid, 1 solid, 2 solid on a wetting face.
__device__ int geom_kind3(const Inst3& I, int x, int y, int z) {
  if (I.geom == GEOM_NOZZLE) {
    if (z >= I.L) return 0;
    const float r2 = rr2(I, x, y);
    if (r2 < I.R2 || r2 >= I.Ro2) return 0;
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

__device__ __forceinline__ int kind_at3(const Inst3& I, int x, int y, int z) {
  int zm;
  if (!map_z(I, z, zm)) return 1;
  return geom_kind3(I, wrap3(x, I.nx), wrap3(y, I.ny), zm);
}

__device__ __forceinline__ size_t cell3(const Inst3& I, int x, int y, int z) {
  return ((size_t)z * I.ny + y) * I.nx + x;
}

__device__ __forceinline__ float phi_at3(const Inst3& I, int x, int y, int z) {
  int zm;
  map_z(I, z, zm);
  return I.phi[cell3(I, wrap3(x, I.nx), wrap3(y, I.ny), zm)];
}

// Wetting ghost phi of a solid point: mean over fluid face neighbours of
// phi + h_s / kappa, else the plain mean over fluid edge neighbours.
__device__ __noinline__ float ghost3(const Inst3& I, int x, int y, int z) {
  const int k = kind_at3(I, x, y, z);
  const float hk = k == 2 ? I.hk : 0.0f;
  float sum = 0.0f;
  int cnt = 0;
#pragma unroll
  for (int i = 1; i <= 6; i++)
    if (kind_at3(I, x + ex3(i), y + ey3(i), z + ez3(i)) == 0) {
      sum += phi_at3(I, x + ex3(i), y + ey3(i), z + ez3(i)) + hk;
      cnt++;
    }
  if (cnt) return sum / (float)cnt;
#pragma unroll
  for (int i = 7; i < 19; i++)
    if (kind_at3(I, x + ex3(i), y + ey3(i), z + ez3(i)) == 0) {
      sum += phi_at3(I, x + ex3(i), y + ey3(i), z + ez3(i));
      cnt++;
    }
  return cnt ? sum / (float)cnt : 0.0f;
}

// May a fluid cell at (x, y, z) have a solid neighbour (conservative)?
__device__ __forceinline__ bool near_solid3(const Inst3& I, int x, int y, int z) {
  if (I.bc == BC_CLOSED && (z == 0 || z == I.nz - 1)) return true;
  const bool zedge = I.bc == BC_PER && (z == 0 || z == I.nz - 1);
  if (I.geom == GEOM_NOZZLE) {
    if (z - 1 >= I.L && !zedge) return false;
    if (x < 2 || x >= I.nx - 2 || y < 2 || y >= I.ny - 2) return true;
    const float r = sqrtf(rr2(I, x, y)), R = sqrtf(I.R2), Ro = sqrtf(I.Ro2);
    return r >= R - 2.0f && r < Ro + 2.0f;
  }
  if (I.geom == GEOM_PLATE) return zedge || z - 1 < I.wt;
  return false;
}

__device__ __forceinline__ float drive3(const Inst3& I, long long t) {
  long long tt = t;
  if (I.Tidle > 0) tt = t % (I.T1 + I.T2 + I.Tidle);
  if (tt < I.T1) return I.F0;
  if (tt < I.T1 + I.T2) return -I.Fneg;
  return 0.0f;
}

// ---------------------------------------------------------------------------
// Collision of the planes [zfirst, zlast) of a 32 x 4 column tile; the block
// marches up z and keeps phi of planes z-1, z, z+1 of the tile (with a
// one-cell halo) in shared memory, so that the D3Q19 stencil of a fluid cell
// away from walls reads shared memory only.  The ring has four slots (plane
// zz in slot zz & 3): the plane loaded at the start of an iteration goes to
// the slot of plane z-2, which no warp still reads once every warp has
// passed the previous iteration's barrier, so one barrier per plane
// suffices.
constexpr int kZChunk = 8;
constexpr int kTX = 32, kTY = 4;

template <bool H, bool DIAG>
__global__ void __launch_bounds__(kTX * kTY) collide3_kernel(const Inst3* __restrict__ insts, int index,
                                                       const long long* __restrict__ d_t,
                                                       int t_off) {
  __shared__ float tile[4][kTY + 2][kTX + 2];
  __shared__ float red[kTY][6];
  const Inst3& I = insts[index];
  // a lattice whose numeric flag is set is frozen; one read per block keeps
  // the decision uniform over the block's barriers below
  const bool lead = threadIdx.x == 0 && threadIdx.y == 0;
  if (__syncthreads_or(lead && (*(volatile const unsigned*)I.status & kStatusNumeric))) return;
  const int tid = threadIdx.y * kTX + threadIdx.x;
  const int x = blockIdx.x * kTX + threadIdx.x;
  const int y = blockIdx.y * kTY + threadIdx.y;
  // zero-gradient ends: the planes z = -1 and z = nz of the extended lattice
  // collide too (their populations are the edge plane's, their stencils
  // their own), so that the streaming can pull from them
  const int zoff = I.bc == BC_ZG ? 1 : 0;
  const int zfirst = (int)blockIdx.z * kZChunk - zoff;
  const int zlast = min(zfirst + kZChunk, I.nz + zoff);
  const size_t N = (size_t)I.nx * I.ny * I.nz, NP = (size_t)I.nx * I.ny * (I.nz + 2);
  const long long t = *d_t + t_off;
  const float drive = drive3(I, t);
  const bool inxy = x < I.nx && y < I.ny;
  // phi of plane zz (extended index) into its ring slot, with the tile's halo
  auto load_plane = [&](int zz) {
    const int slot = zz & 3;
    int zm = 0;
    const bool ok = map_z(I, zz, zm);
    for (int idx = tid; idx < (kTY + 2) * (kTX + 2); idx += kTX * kTY) {
      const int lx = idx % (kTX + 2), ly = idx / (kTX + 2);  // constant divisors
      const int gx = wrap_tile((int)blockIdx.x * kTX + lx - 1, I.nx);
      const int gy = wrap_tile((int)blockIdx.y * kTY + ly - 1, I.ny);
      tile[slot][ly][lx] = ok ? I.phi[cell3(I, gx, gy, zm)] : 0.0f;
    }
  };
  load_plane(zfirst - 1);
  load_plane(zfirst);
  for (int z = zfirst; z < zlast; z++) {
    load_plane(z + 1);
    __syncthreads();
    int zm = z;
    const bool inz = map_z(I, z, zm);
    const bool inr = inxy && inz;
    const size_t c = inr ? cell3(I, x, y, zm) : 0;
    const size_t cp = inr ? ((size_t)(z + 1) * I.ny + y) * I.nx + x : 0;  // post-collision plane
    const bool fluid = inr && geom_kind3(I, x, y, zm) == 0;
    const bool owned = z >= 0 && z < I.nz;  // diagnostics count in-domain cells only
    float dg[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (fluid) {
      float fr[19], gr[7];
#pragma unroll
      for (int i = 0; i < 19; i++) fr[i] = ldS<H>(I.f, i * N + c);
      gr[0] = I.g0[c];
#pragma unroll
      for (int i = 1; i < 7; i++) gr[i] = ldS<H>(I.g, (i - 1) * N + c);
      const float phi = gr[0] + gr[1] + gr[2] + gr[3] + gr[4] + gr[5] + gr[6];
      // D3Q19 stencils on phi with wetting ghosts
      const bool ns = near_solid3(I, x, y, zm) || !owned;
      float lap = 0.0f, gx = 0.0f, gy = 0.0f, gz = 0.0f;
#pragma unroll
      for (int i = 1; i < 19; i++) {
        const int xn = x + ex3(i), yn = y + ey3(i), zn = z + ez3(i);
        float pn;
        if (ns && kind_at3(I, xn, yn, zn) != 0)
          pn = ghost3(I, xn, yn, zn);
        else
          pn = tile[zn & 3][threadIdx.y + 1 + ey3(i)][threadIdx.x + 1 + ex3(i)];
        lap += 6.0f * w3(i) * (pn - phi);
        gx += 3.0f * w3(i) * (float)ex3(i) * pn;
        gy += 3.0f * w3(i) * (float)ey3(i) * pn;
        gz += 3.0f * w3(i) * (float)ez3(i) * pn;
      }
      const float mu = I.A4 * phi * ((phi - I.phis) * (phi + I.phis)) - I.kappa * lap;
      float C = fminf(fmaxf(0.5f * (phi * I.inv_phis + 1.0f), 0.0f), 1.0f);
      const bool dreg = I.geom != GEOM_NOZZLE || (zm < I.L && rr2(I, x, y) < I.R2);
      const float Fb = dreg ? drive * C : 0.0f;
      const float Fx = mu * gx, Fy = mu * gy, Fz = mu * gz + Fb;
      float dn = 0.0f, mx = 0.0f, my = 0.0f, mz = 0.0f;
#pragma unroll
      for (int i = 0; i < 19; i++) {
        dn += fr[i];
        mx += (float)ex3(i) * fr[i];
        my += (float)ey3(i) * fr[i];
        mz += (float)ez3(i) * fr[i];
      }
      const float n = I.n0 + dn, inv_n = __frcp_rn(n);
      const float ux = (mx + 0.5f * Fx) * inv_n, uy = (my + 0.5f * Fy) * inv_n,
                  uz = (mz + 0.5f * Fz) * inv_n;
      const float u2 = ux * ux + uy * uy + uz * uz;
      if (!(u2 < 0.09f)) atomicOr(I.status, kStatusNumeric);
      const float om = __frcp_rn(0.5f + 3.0f * (I.nu_air + C * I.dnu));
      const float pref = 3.0f * (1.0f - 0.5f * om);
      const float p3 = dn + 3.0f * phi * mu;  // A_i - n0 for i >= 1
      const float uF = ux * Fx + uy * Fy + uz * Fz, base = -1.5f * u2;
      const float n3 = 3.0f * n;
      float fs[19], sum_eq = 0.0f, sum_F = 0.0f;
      // opposite pairs share the even parts (see the 2-D kernel)
#pragma unroll
      for (int i = 1; i < 19; i++) {
        if (opp3(i) < i) continue;
        const int ib = opp3(i);
        const float w = w3(i);
        const float cu = (float)ex3(i) * ux + (float)ey3(i) * uy + (float)ez3(i) * uz;
        const float cF = (float)ex3(i) * Fx + (float)ey3(i) * Fy + (float)ez3(i) * Fz;
        const float E = w * (p3 + n * (base + 4.5f * cu * cu)), O = (w * n3) * cu;
        const float wp = w * pref, FE = wp * (3.0f * cu * cF - uF), FO = wp * cF;
        sum_eq += 2.0f * E;
        sum_F += 2.0f * FE;
        fs[i] = fr[i] + om * ((E + O) - fr[i]) + (FE + FO);
        fs[ib] = fr[ib] + om * ((E - O) - fr[ib]) + (FE - FO);
      }
      fs[0] = fr[0] + om * ((dn - sum_eq) - fr[0]) - sum_F;
#pragma unroll
      for (int i = 0; i < 19; i++) stS<H>(I.fp, i * NP + cp, fs[i]);
      // order parameter: D3Q7, rest direction special
      const float gmu = I.gamma * mu, pq = phi * I.inv2q;
      float sum_ge = 0.0f, sum_g = 0.0f;
#pragma unroll
      for (int i = 1; i < 7; i++) {
        const float cu = (float)ex3(i) * ux + (float)ey3(i) * uy + (float)ez3(i) * uz;
        const float ge = 0.5f * gmu + pq * cu;
        sum_ge += ge;
        sum_g += gr[i];
        stS<H>(I.gp, (i - 1) * NP + cp, I.q * gr[i] + (ge - gr[i]) * I.inv_tphi);
      }
      I.g0p[cp] = gr[0] + (sum_g - sum_ge) * I.inv_tphi;
      if (DIAG && owned) {
        const float e = fminf(fmaxf(phi * I.inv_phis, 0.0f), 1.0f);
        dg[0] = e;
        dg[1] = e * n;
        dg[2] = dg[1] * uz;
        dg[3] = n;
        dg[4] = phi;
        dg[5] = n * uz;
      }
    }
    if (DIAG && owned) {  // uniform over the block: one plane
      // a warp's 32 cells summed in FP32, the warps and every total in FP64
      const int lane = tid & 31, warp = tid >> 5;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int k = 0; k < 6; k++) dg[k] += __shfl_down_sync(0xffffffffu, dg[k], o);
      if (lane == 0)
#pragma unroll
        for (int k = 0; k < 6; k++) red[warp][k] = dg[k];
      __syncthreads();
      if (tid == 0) {
        double s[6] = {0, 0, 0, 0, 0, 0};
        for (int wq = 0; wq < kTY; wq++)
          for (int k = 0; k < 6; k++) s[k] += (double)red[wq][k];
        atomicAdd(I.rows + z, s[0]);
        atomicAdd(I.rows + I.nz + z, s[1]);
        atomicAdd(I.rows + 2 * I.nz + z, s[2]);
        atomicAdd(I.sums + 0, s[3]);
        atomicAdd(I.sums + 1, s[4]);
        atomicAdd(I.sums + 2, s[5]);
      }
    }
  }
}

template <bool H>
__global__ void __launch_bounds__(128) stream3_kernel(const Inst3* __restrict__ insts, int index) {
  const Inst3& I = insts[index];
  // the flag raised by this step's collision freezes the state at time t
  if (*(volatile const unsigned*)I.status & kStatusNumeric) return;
  const int x = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= I.nx || y >= I.ny || geom_kind3(I, x, y, z) != 0) return;
  const size_t N = (size_t)I.nx * I.ny * I.nz, NP = (size_t)I.nx * I.ny * (I.nz + 2);
  const size_t c = cell3(I, x, y, z), cp = ((size_t)(z + 1) * I.ny + y) * I.nx + x;
  const bool ns = near_solid3(I, x, y, z);
  // post-collision plane of a source plane zs: the extended planes -1 and nz
  // of zero-gradient ends are stored, periodic ones wrap
  auto post = [&](int xs, int ys, int zs) -> size_t {
    const int zq = I.bc == BC_PER ? wrap3(zs, I.nz) : zs;
    return ((size_t)(zq + 1) * I.ny + wrap3(ys, I.ny)) * I.nx + wrap3(xs, I.nx);
  };
  float fn[19];
  fn[0] = ldS<H>(I.fp, cp);
#pragma unroll
  for (int i = 1; i < 19; i++) {
    const int xs = x - ex3(i), ys = y - ey3(i), zs = z - ez3(i);
    if (ns && kind_at3(I, xs, ys, zs) != 0)
      fn[i] = ldS<H>(I.fp, opp3(i) * NP + cp);
    else
      fn[i] = ldS<H>(I.fp, i * NP + post(xs, ys, zs));
  }
  float g0 = I.g0p[cp], phi = g0;
  float gn[7];
#pragma unroll
  for (int i = 1; i < 7; i++) {
    const int xs = x - ex3(i), ys = y - ey3(i), zs = z - ez3(i);
    float moving;
    if (ns && kind_at3(I, xs, ys, zs) != 0)
      moving = ldS<H>(I.gp, (opp3(i) - 1) * NP + cp);
    else
      moving = ldS<H>(I.gp, (i - 1) * NP + post(xs, ys, zs));
    gn[i] = I.omq * ldS<H>(I.g, (i - 1) * N + c) + moving;
  }
#pragma unroll
  for (int i = 0; i < 19; i++) stS<H>(I.f, i * N + c, fn[i]);
  I.g0[c] = g0;
#pragma unroll
  for (int i = 1; i < 7; i++) {
    stS<H>(I.g, (i - 1) * N + c, gn[i]);
    phi += stored<H>(gn[i]);
  }
  I.phi[c] = phi;
}

// ---------------------------------------------------------------------------
// Initialisation (FP64), as in the 2-D path.
__device__ unsigned long long splitmix64_3(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__global__ void init_phi3_kernel(const Inst3* __restrict__ insts, int index, double* phi0) {
  const Inst3& I = insts[index];
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

__device__ double phi0_hat3(const Inst3& I, const double* phi0, int x, int y, int z) {
  const int k = kind_at3(I, x, y, z);
  int zm = 0;
  if (k == 0) {
    map_z(I, z, zm);
    return phi0[cell3(I, wrap3(x, I.nx), wrap3(y, I.ny), zm)];
  }
  const double hk = k == 2 ? I.d_h / I.d_kappa : 0.0;
  double sum = 0.0;
  int cnt = 0;
  for (int i = 1; i <= 6; i++) {
    const int xx = x + ex3(i), yy = y + ey3(i), zz = z + ez3(i);
    if (kind_at3(I, xx, yy, zz) == 0) {
      map_z(I, zz, zm);
      sum += phi0[cell3(I, wrap3(xx, I.nx), wrap3(yy, I.ny), zm)] + hk;
      cnt++;
    }
  }
  if (cnt) return sum / cnt;
  for (int i = 7; i < 19; i++) {
    const int xx = x + ex3(i), yy = y + ey3(i), zz = z + ez3(i);
    if (kind_at3(I, xx, yy, zz) == 0) {
      map_z(I, zz, zm);
      sum += phi0[cell3(I, wrap3(xx, I.nx), wrap3(yy, I.ny), zm)];
      cnt++;
    }
  }
  return cnt ? sum / cnt : 0.0;
}

template <bool H>
__global__ void init_pop3_kernel(const Inst3* __restrict__ insts, int index, const double* phi0) {
  const Inst3& I = insts[index];
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= I.nx || y >= I.ny) return;
  const size_t N = (size_t)I.nx * I.ny * I.nz, c = cell3(I, x, y, z);
  if (geom_kind3(I, x, y, z) != 0) {
    for (int i = 0; i < 19; i++) stS<H>(I.f, i * N + c, 0.0f);
    for (int i = 0; i < 6; i++) stS<H>(I.g, i * N + c, 0.0f);
    I.g0[c] = 0.0f;
    I.phi[c] = 0.0f;
    return;
  }
  const double p0 = phi0[c];
  double lap = 0.0;
  for (int i = 1; i < 19; i++)
    lap += 6.0 * (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0) * (phi0_hat3(I, phi0, x + ex3(i), y + ey3(i), z + ez3(i)) - p0);
  const double mu = 4.0 * I.d_A * p0 * (p0 * p0 - I.d_phis * I.d_phis) - I.d_kappa * lap;
  const double n = I.d_n0, p = p0 * mu + n / 3.0;
  for (int i = 0; i < 19; i++) {
    const double w = i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
    const double Ai = i == 0 ? 3.0 * n - 6.0 * p : 3.0 * p;
    stS<H>(I.f, i * N + c, (float)(w * Ai - w * n));
  }
  const float g0 = (float)(p0 - 3.0 * I.d_gamma * mu);
  I.g0[c] = g0;
  float phi = g0;
  const float gi = (float)(0.5 * I.d_gamma * mu);
  for (int i = 0; i < 6; i++) {
    stS<H>(I.g, i * N + c, gi);
    phi += stored<H>(gi);
  }
  I.phi[c] = phi;
}

template <bool H, bool EXPORT>
__global__ void convert3_kernel(const Inst3* __restrict__ insts, int index, float* f, float* g) {
  const Inst3& I = insts[index];
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= I.nx || y >= I.ny) return;
  const size_t N = (size_t)I.nx * I.ny * I.nz, c = cell3(I, x, y, z);
  const bool fluid = geom_kind3(I, x, y, z) == 0;
  if (EXPORT) {
    for (int i = 0; i < 19; i++) {
      const float w = i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
      f[i * N + c] = fluid ? ldS<H>(I.f, i * N + c) + w * I.n0 : 0.0f;
    }
    g[c] = fluid ? I.g0[c] : 0.0f;
    for (int i = 1; i < 7; i++) g[i * N + c] = fluid ? ldS<H>(I.g, (i - 1) * N + c) : 0.0f;
  } else {
    if (!fluid) return;
    for (int i = 0; i < 19; i++) {
      const float w = i == 0 ? 1.0f / 3.0f : (i <= 6 ? 1.0f / 18.0f : 1.0f / 36.0f);
      stS<H>(I.f, i * N + c, f[i * N + c] - w * I.n0);
    }
    I.g0[c] = g[c];
    float phi = g[c];
    for (int i = 1; i < 7; i++) {
      stS<H>(I.g, (i - 1) * N + c, g[i * N + c]);
      phi += stored<H>(g[i * N + c]);
    }
    I.phi[c] = phi;
  }
}

__global__ void phi3_kernel(const Inst3* __restrict__ insts, int index, float* out) {
  const Inst3& I = insts[index];
  const int x = blockIdx.x * blockDim.x + threadIdx.x, y = blockIdx.y * blockDim.y + threadIdx.y;
  const int z = blockIdx.z;
  if (x >= I.nx || y >= I.ny) return;
  const size_t c = cell3(I, x, y, z);
  out[c] = geom_kind3(I, x, y, z) == 0 ? I.phi[c] : 0.0f;
}

dim3 grid3(const Inst3& h) { return dim3((h.nx + 31) / 32, (h.ny + 3) / 4, h.nz); }
dim3 grid3c(const Inst3& h) {
  return dim3((h.nx + kTX - 1) / kTX, (h.ny + kTY - 1) / kTY,
              (h.nz + (h.bc == BC_ZG ? 2 : 0) + kZChunk - 1) / kZChunk);
}

}  // namespace

cudaError_t launch_init3(const Inst3* d, const Inst3& h, int index, cudaStream_t s) {
  double* phi0 = reinterpret_cast<double*>(h.fp);  // the post-collision copy is free before step 0
  init_phi3_kernel<<<grid3(h), dim3(32, 4), 0, s>>>(d, index, phi0);
  if (h.fp16)
    init_pop3_kernel<true><<<grid3(h), dim3(32, 4), 0, s>>>(d, index, phi0);
  else
    init_pop3_kernel<false><<<grid3(h), dim3(32, 4), 0, s>>>(d, index, phi0);
  return cudaGetLastError();
}

cudaError_t launch_collide3(const Inst3* d, const Inst3& h, int index, const long long* d_t,
                            int t_off, bool diag, cudaStream_t s) {
  const dim3 g = grid3c(h), b(kTX, kTY);
  if (h.fp16) {
    if (diag)
      collide3_kernel<true, true><<<g, b, 0, s>>>(d, index, d_t, t_off);
    else
      collide3_kernel<true, false><<<g, b, 0, s>>>(d, index, d_t, t_off);
  } else {
    if (diag)
      collide3_kernel<false, true><<<g, b, 0, s>>>(d, index, d_t, t_off);
    else
      collide3_kernel<false, false><<<g, b, 0, s>>>(d, index, d_t, t_off);
  }
  return cudaGetLastError();
}

cudaError_t launch_stream3(const Inst3* d, const Inst3& h, int index, cudaStream_t s) {
  if (h.fp16)
    stream3_kernel<true><<<grid3(h), dim3(32, 4), 0, s>>>(d, index);
  else
    stream3_kernel<false><<<grid3(h), dim3(32, 4), 0, s>>>(d, index);
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
  if (h.fp16)
    convert3_kernel<true, false><<<grid3(h), dim3(32, 4), 0, s>>>(d, index, const_cast<float*>(f),
                                                                 const_cast<float*>(g));
  else
    convert3_kernel<false, false><<<grid3(h), dim3(32, 4), 0, s>>>(d, index, const_cast<float*>(f),
                                                                  const_cast<float*>(g));
  return cudaGetLastError();
}

cudaError_t launch_phi3(const Inst3* d, const Inst3& h, int index, float* out, cudaStream_t s) {
  phi3_kernel<<<grid3(h), dim3(32, 4), 0, s>>>(d, index, out);
  return cudaGetLastError();
}

}  // namespace ij
