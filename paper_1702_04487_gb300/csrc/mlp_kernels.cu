// Kernels of the surrogate network: a BF16 tensor-core GEMM on the 5th
// generation tensor cores (tcgen05.mma, accumulator in tensor memory) with
// fused epilogues, and the small element-wise kernels around it (input
// transform and minibatch gather, loss, bias gradients, Adam, output
// transform, acceptance gate).
//
// GEMM shape: C[M x N] = A[M x K] B[N x K]^T with A and B row-major (K
// contiguous, "K-major").  A CTA of 128 threads owns a 128 x BN tile of C,
// BN in {16, 32, 64, 128, 256}.  K advances in slices of 64 (128 bytes of
// BF16, one row of a 128-byte swizzle atom) through a ring of kStages
// shared-memory buffers.  One thread drives the pipeline: it loads slices of
// A and of B with the tensor memory accelerator (cp.async.bulk.tensor,
// 128-byte swizzle written by the copy itself, completion counted in bytes
// on the buffer's load mbarrier) up to kStages ahead -- every slice of the
// surrogate's K <= 256 at once -- issues the four K=16 MMAs of a slice once
// it has landed and commits them to the buffer's MMA mbarrier, and refills
// the buffer of the previous slice once its MMAs are done.  If a bounded
// wait gives up, every copy and MMA still in flight is waited for (again
// bounded) before the tensor memory is released and the CTA exits; the
// output is then left unwritten and the timeout flag set.  The epilogue reads the accumulator with
// tcgen05.ld (warp w owns tensor-memory lanes 32w..32w+31, i.e. rows
// 32w..32w+31 of the tile).
#include <cuda.h>
#include <math.h>

#include "mlp.cuh"

namespace sg {
namespace {

constexpr int BM = 128;
constexpr int BK = 64;
constexpr int kStages = 4;  // shared-memory buffers of K slices
constexpr int kThreads = 128;
constexpr int kWaitLimit = 1 << 22;  // try_wait rounds before giving up

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint32_t bar, int count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
}
// Wait for the completion of the barrier phase of the given parity; false
// after kWaitLimit rounds.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity) {
  for (int i = 0; i < kWaitLimit; i++) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major tile in the 128-byte swizzle
// layout: rows of 128 bytes, 8-row atoms of 1024 bytes stacked along M/N
// (stride byte offset 1024); the leading byte offset is unused for this
// layout.  Bits: start address >> 4 [0,14), leading offset >> 4 [16,30),
// stride offset >> 4 [32,46), version 1 [46,48), swizzle mode 2 [61,64).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;
  d |= (uint64_t)(1024 >> 4) << 32;
  d |= (uint64_t)1 << 46;
  d |= (uint64_t)2 << 61;
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator [4,6) = 1, A and B
// BF16 [7,10) = [10,13) = 1, both K-major, N >> 3 at [17,23), M >> 4 at
// [24,29).
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                         uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
__device__ __forceinline__ void mma_commit(uint32_t bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
      : "memory");
}

// 16 consecutive FP32 accumulator columns of this thread's lane (row).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; j++) v[j] = __uint_as_float(r[j]);
}

__device__ __forceinline__ float gelu_f(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad_f(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
         x * 0.39894228040143268f * expf(-0.5f * x * x);
}

template <int BN>
__host__ __device__ constexpr int stage_bytes() {
  return BM * BK * 2 + BN * BK * 2;
}
template <int BN>
__host__ __device__ constexpr int tmem_cols() {
  return BN < 32 ? 32 : BN;
}

// Arm the load barrier for `bytes` of asynchronous copies (one arrival).
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes)
               : "memory");
}

// One box of a 3-D tensor map (x = K offset, y = row, z = member) into
// shared memory; completion is counted on `bar`.
__device__ __forceinline__ void tma_load3(uint32_t dst, const CUtensorMap* map, int x, int y, int z,
                                          uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(bar)
      : "memory");
}

template <int BN>
__global__ void __launch_bounds__(kThreads, 1)
    gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                const GemmArgs a) {
  extern __shared__ uint8_t smem_raw[];
  uint8_t* smem = reinterpret_cast<uint8_t*>(
      (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  constexpr int kA = BM * BK * 2;
  constexpr int kStage = stage_bytes<BN>();
  constexpr uint32_t kCols = tmem_cols<BN>();
  constexpr uint32_t kIdesc = idesc_bf16(BM, BN);
  // bars[b]: the load of buffer b landed; bars[kStages + b]: its MMAs done
  uint64_t* bars = reinterpret_cast<uint64_t*>(smem + kStages * kStage);
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * kStages);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int z = blockIdx.z;
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int za = a.sA ? z : 0, zb = a.sB ? z : 0;  // a zero stride shares one operand

  if (tid == 0) {
#pragma unroll
    for (int i = 0; i < 2 * kStages; i++) mbar_init(smem_u32(&bars[i]), 1);
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(
                     smem_u32(tmem_slot)),
                 "r"(kCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int nk = (a.K + BK - 1) / BK;
  bool ok = true;
  if (tid == 0) {
    // slice kt lives in buffer kt % kStages; its load completes phase
    // (kt / kStages) & 1 of bars[buffer], its MMAs the same phase of
    // bars[kStages + buffer]
    auto load = [&](int kt) {
      const int b = kt % kStages;
      const uint32_t ta = smem_u32(smem + b * kStage), tb = ta + kA;
      mbar_expect_tx(smem_u32(&bars[b]), (uint32_t)kStage);
      tma_load3(ta, &tmA, kt * BK, m0, za, smem_u32(&bars[b]));
      tma_load3(tb, &tmB, kt * BK, n0, zb, smem_u32(&bars[b]));
    };
    auto phase = [](int kt) { return (uint32_t)((kt / kStages) & 1); };
    int loaded = 0;     // slices whose loads were issued
    int landed = 0;     // slices whose loads were seen complete
    int committed = 0;  // slices whose MMAs were committed
    int freed = 0;      // slices whose MMAs were seen complete
    for (; loaded < nk && loaded < kStages; loaded++) load(loaded);
    for (int kt = 0; kt < nk; kt++) {
      const int b = kt % kStages;
      if (!mbar_wait(smem_u32(&bars[b]), phase(kt))) {
        ok = false;
        break;
      }
      landed = kt + 1;
      tc_fence_after();
      const uint32_t ta = smem_u32(smem + b * kStage), tb = ta + kA;
#pragma unroll
      for (int k = 0; k < BK / 16; k++)
        mma_bf16(tmem, sw128_desc(ta + 32 * k), sw128_desc(tb + 32 * k), kIdesc,
                 (kt > 0 || k > 0) ? 1u : 0u);
      mma_commit(smem_u32(&bars[kStages + b]));
      committed = kt + 1;
      // refill the buffer of the previous slice once its MMAs are done
      if (kt >= 1 && loaded < nk) {
        if (!mbar_wait(smem_u32(&bars[kStages + (kt - 1) % kStages]), phase(kt - 1))) {
          ok = false;
          break;
        }
        freed = kt;
        load(loaded++);
      }
    }
    // Before the accumulator is read, the tensor memory released or the CTA
    // exits, every copy issued must have landed and every MMA committed must
    // be done -- also after a timeout above (these waits are bounded too).
    for (int kt = landed; kt < loaded; kt++)
      ok = mbar_wait(smem_u32(&bars[kt % kStages]), phase(kt)) && ok;
    for (int kt = freed > committed - kStages ? freed : committed - kStages; kt < committed; kt++)
      ok = mbar_wait(smem_u32(&bars[kStages + kt % kStages]), phase(kt)) && ok;
  }
  ok = __syncthreads_and(ok);
  tc_fence_after();

  if (ok) {
    // Epilogue through shared memory (the operand buffers are free once every
    // MMA is done): each warp takes its 32 rows x 16 columns from tensor
    // memory (lane = row), then works row by row -- half-warps on two rows,
    // lanes along n -- so that bias, aux and every row-major output are read
    // and written in contiguous runs; the transposed BF16 copy is written
    // from the lane = row layout, contiguous along m.
    float* T = reinterpret_cast<float*>(smem) + warp * (32 * 17);
    const int m = m0 + warp * 32 + lane;
    const bool mrow = m < a.M;
    const float* bias = a.bias ? a.bias + z * a.sBias : nullptr;
    const int jj = lane & 15, rh = lane >> 4;
#pragma unroll 1
    for (int c0 = 0; c0 < BN; c0 += 16) {
      float v[16];
      tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, v);
      const int nb = n0 + c0;
      if (nb >= a.N) continue;  // uniform over the CTA
#pragma unroll
      for (int j = 0; j < 16; j++) T[lane * 17 + j] = v[j];
      __syncwarp();
      const int n = nb + jj;
#pragma unroll 4
      for (int i = 0; i < 16; i++) {
        const int r = 2 * i + rh, mm = m0 + warp * 32 + r;
        if (mm >= a.M || n >= a.N) continue;
        float x = T[r * 17 + jj];
        if (a.epi == EPI_F32) {
          a.Cf[z * a.sCf + (size_t)mm * a.ldcf + n] = x;
          continue;
        }
        if (a.epi == EPI_BIAS_F32) {
          a.Cf[z * a.sCf + (size_t)mm * a.ldcf + n] = x + bias[n];
          continue;
        }
        if (a.epi == EPI_BIAS_GELU) {
          x += bias[n];
          if (a.Zout) a.Zout[z * a.sZ + (size_t)mm * a.ldz + n] = x;
          x = gelu_f(x);
        } else {  // EPI_GELU_BWD
          x *= gelu_grad_f(a.aux[z * a.sAux + (size_t)mm * a.ldaux + n]);
        }
        const bf16 hb = __float2bfloat16_rn(x);
        if (a.Cb) a.Cb[z * a.sCb + (size_t)mm * a.ldcb + n] = hb;
        T[r * 17 + jj] = __bfloat162float(hb);  // for the transposed copy
      }
      __syncwarp();
      if (a.Ct && mrow && (a.epi == EPI_BIAS_GELU || a.epi == EPI_GELU_BWD)) {
#pragma unroll
        for (int j = 0; j < 16; j++)
          if (nb + j < a.N)
            a.Ct[z * a.sCt + (size_t)(nb + j) * a.ldct + m] = __float2bfloat16_rn(T[lane * 17 + j]);
      }
      __syncwarp();  // the next chunk overwrites T
    }
  } else if (tid == 0) {
    atomicOr(a.status, kStatusTimeout);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kCols)
                 : "memory");
  }
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// The driver's tensor-map encoder, looked up once through the runtime (no
// link against the driver library).
EncodeTiledFn encode_tiled() {
  static EncodeTiledFn fn = nullptr;
  static bool looked = false;
  if (!looked) {
    looked = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                         &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  }
  return fn;
}

// 3-D tensor map of a BF16 operand: K (contiguous) x rows (leading dimension
// ld) x layers (stride layer, or one layer), boxes of 64 x box_rows x 1 in
// the 128-byte swizzle; out-of-range elements read as zero.
cudaError_t make_map(CUtensorMap* m, const bf16* base, int K, int rows, int ld,
                     long long layer, int layers, int box_rows) {
  EncodeTiledFn enc = encode_tiled();
  if (!enc) return cudaErrorNotSupported;
  const cuuint64_t dims[3] = {(cuuint64_t)K, (cuuint64_t)rows, (cuuint64_t)layers};
  const cuuint64_t strides[2] = {(cuuint64_t)ld * 2,
                                 (cuuint64_t)(layers > 1 ? layer : (long long)ld * rows) * 2};
  const cuuint32_t box[3] = {(cuuint32_t)BK, (cuuint32_t)box_rows, 1};
  const cuuint32_t es[3] = {1, 1, 1};
  const CUresult r = enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<bf16*>(base), dims,
                         strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                         CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

template <int BN>
cudaError_t launch_bn(const GemmArgs& a, int members, cudaStream_t s) {
  const size_t smem = gemm_smem_bytes(BN);
  CUtensorMap ma, mb;
  cudaError_t e0 = make_map(&ma, a.A, a.K, a.M, a.lda, a.sA, a.sA ? members : 1, BM);
  if (e0 == cudaSuccess) e0 = make_map(&mb, a.B, a.K, a.N, a.ldb, a.sB, a.sB ? members : 1, BN);
  if (e0 != cudaSuccess) return e0;
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(gemm_kernel<BN>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  dim3 grid((a.M + BM - 1) / BM, (a.N + BN - 1) / BN, members);
  gemm_kernel<BN><<<grid, kThreads, smem, s>>>(ma, mb, a);
  return cudaGetLastError();
}

}  // namespace

size_t gemm_smem_bytes(int bn) {
  return 1024 + kStages * (size_t)(BM * BK * 2 + bn * BK * 2) + 16 * kStages + 16;
}

cudaError_t launch_gemm(const GemmArgs& a, int members, cudaStream_t s) {
  // the narrowest tile that covers N, halved (down to 32 columns) while the
  // grid has fewer than ~2 tiles per SM of a 152-SM part
  int bn = a.N <= 16 ? 16 : a.N <= 32 ? 32 : a.N <= 64 ? 64 : a.N <= 128 ? 128 : 256;
  const long long mt = (a.M + BM - 1) / BM;
  while (bn > 32 && mt * ((a.N + bn - 1) / bn) * members < 304) bn /= 2;
  switch (bn) {
    case 16: return launch_bn<16>(a, members, s);
    case 32: return launch_bn<32>(a, members, s);
    case 64: return launch_bn<64>(a, members, s);
    case 128: return launch_bn<128>(a, members, s);
    default: return launch_bn<256>(a, members, s);
  }
}

}  // namespace sg

// ---------------------------------------------------------------------------
// Element-wise kernels around the GEMMs.
namespace sg {
namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {
  // SplitMix64 finaliser (Steele, Lea & Flood 2014)
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

__device__ __forceinline__ float xform(float v, int d, const Xform& xf) {
  if ((xf.log_mask >> d) & 1) v = logf(v);
  return (v - xf.mean[d]) / xf.scale[d];
}

__global__ void prep_inputs_kernel(const float* __restrict__ x, int n, const Xform xf,
                                   bf16* __restrict__ X, float* __restrict__ Xf) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
#pragma unroll
  for (int d = 0; d < kInPad; d++) {
    const float v = d < kIn ? xform(x[(size_t)r * kIn + d], d, xf) : 0.0f;
    if (X) X[(size_t)r * kInPad + d] = __float2bfloat16_rn(v);
    if (Xf && d < kIn) Xf[(size_t)r * kIn + d] = v;
  }
}

__global__ void prep_targets_kernel(const float* __restrict__ y, int n, const Xform yf,
                                    float* __restrict__ T) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n) return;
#pragma unroll
  for (int d = 0; d < kOut; d++) T[(size_t)r * kOut + d] = xform(y[(size_t)r * kOut + d], d, yf);
}

__global__ void gather_kernel(const bf16* __restrict__ X, const float* __restrict__ T, int n,
                              int bm, unsigned long long seed, const long long* __restrict__ d_step,
                              bf16* __restrict__ Xb, bf16* __restrict__ Xbt,
                              float* __restrict__ Tb) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x, mem = blockIdx.y;
  if (r >= bm) return;
  const unsigned long long ctr =
      ((unsigned long long)mem << 56) ^ ((unsigned long long)*d_step << 24) ^ (unsigned)r;
  const int src = (int)(mix64(seed ^ mix64(ctr)) % (unsigned long long)n);
  const size_t ob = (size_t)mem * bm;
#pragma unroll
  for (int d = 0; d < kInPad; d++) {
    const bf16 v = X[(size_t)src * kInPad + d];
    Xb[(ob + r) * kInPad + d] = v;
    Xbt[(size_t)mem * kInPad * bm + (size_t)d * bm + r] = v;
  }
#pragma unroll
  for (int d = 0; d < kOut; d++) Tb[(ob + r) * kOut + d] = T[(size_t)src * kOut + d];
}

__global__ void loss_kernel(const float* __restrict__ Y, const float* __restrict__ Tb,
                            const float* __restrict__ w, int bm, bf16* __restrict__ dY,
                            bf16* __restrict__ dYt, float* __restrict__ dYft, double* loss,
                            unsigned* status) {
  const int r = blockIdx.x * blockDim.x + threadIdx.x, mem = blockIdx.y;
  double acc = 0.0;
  if (r < bm) {
    const size_t row = (size_t)mem * bm + r;
    const float inv = 2.0f / (float)(bm * kOut);
#pragma unroll
    for (int d = 0; d < kOutPad; d++) {
      float g = 0.0f;
      if (d < kOut) {
        const float diff = Y[row * kOutPad + d] - Tb[row * kOut + d];
        acc += (double)w[d] * diff * diff;
        g = inv * w[d] * diff;
      }
      const bf16 gb = __float2bfloat16_rn(g);
      dY[row * kOutPad + d] = gb;
      dYt[(size_t)mem * kOutPad * bm + (size_t)d * bm + r] = gb;
      dYft[(size_t)mem * kOutPad * bm + (size_t)d * bm + r] = g;
    }
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(loss + mem, acc / (double)(bm * kOut));
    if (!isfinite(acc)) atomicOr(status, kStatusNonFinite);
  }
}

template <typename T>
__device__ __forceinline__ float to_f(T v);
template <>
__device__ __forceinline__ float to_f<float>(float v) {
  return v;
}
template <>
__device__ __forceinline__ float to_f<bf16>(bf16 v) {
  return __bfloat162float(v);
}

// one warp per (member, row)
template <typename T>
__global__ void rowsum_kernel(const T* __restrict__ in, int rows, int cols, int ld, long long sin_,
                              float* __restrict__ out, long long sout) {
  const int row = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  const int mem = blockIdx.y;
  if (row >= rows) return;
  const T* p = in + mem * sin_ + (size_t)row * ld;
  float acc = 0.0f;
  for (int c = lane; c < cols; c += 32) acc += to_f<T>(p[c]);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) out[mem * sout + row] = acc;
}

// Locate flat parameter index i of a member: layer, and whether a weight
// (row r, column c) or a bias.
__device__ __forceinline__ void locate(const Layout& L, long long i, int& l, int& r, int& c,
                                       bool& weight) {
  l = 0;
#pragma unroll
  for (int k = 1; k <= kHidden; k++)
    if (i >= L.w_off[k]) l = k;
  if (i < L.b_off[l]) {
    weight = true;
    const long long j = i - L.w_off[l];
    r = (int)(j / L.nin[l]);
    c = (int)(j % L.nin[l]);
  } else {
    weight = false;
    r = (int)(i - L.b_off[l]);
    c = 0;
  }
}

// d_sched (may be null): {first step, number of steps} of the current
// training call; lr then decays along a half cosine, lr (1 + cos(pi s / S)) / 2
// at its step s of S.
__global__ void adam_kernel(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                            float* __restrict__ v, const Layout L, int members, float lr,
                            float beta1, float beta2, float eps, const long long* __restrict__ d_step,
                            const long long* __restrict__ d_sched, bf16* __restrict__ Wb,
                            bf16* __restrict__ WbT) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= L.total * members) return;
  if (d_sched && d_sched[1] > 0) {
    const float frac = (float)(*d_step - d_sched[0]) / (float)d_sched[1];
    lr *= 0.5f * (1.0f + cospif(fminf(fmaxf(frac, 0.0f), 1.0f)));
  }
  const float t = (float)(*d_step + 1);
  const float bc1 = 1.0f - powf(beta1, t), bc2 = 1.0f - powf(beta2, t);
  const float gi = g[i];
  const float mi = beta1 * m[i] + (1.0f - beta1) * gi;
  const float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  p[i] = pi;
  const long long mem = i / L.total, k = i % L.total;
  int l, r, c;
  bool weight;
  locate(L, k, l, r, c, weight);
  if (weight) {
    const bf16 b = __float2bfloat16_rn(pi);
    Wb[i] = b;
    WbT[mem * L.total + L.w_off[l] + (long long)c * L.nout[l] + r] = b;
  }
}

__global__ void cast_params_kernel(const float* __restrict__ p, const Layout L, int members,
                                   bf16* __restrict__ Wb, bf16* __restrict__ WbT) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= L.total * members) return;
  const long long mem = i / L.total, k = i % L.total;
  int l, r, c;
  bool weight;
  locate(L, k, l, r, c, weight);
  if (weight) {
    const bf16 b = __float2bfloat16_rn(p[i]);
    Wb[i] = b;
    WbT[mem * L.total + L.w_off[l] + (long long)c * L.nout[l] + r] = b;
  }
}

__global__ void advance_step_kernel(long long* d_step) { *d_step += 1; }

__global__ void decode_kernel(const float* __restrict__ Y, int n, int members, const Xform yf,
                              float* __restrict__ mean, float* __restrict__ sd) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= n) return;
#pragma unroll
  for (int d = 0; d < kOut; d++) {
    double s = 0.0, s2 = 0.0;
    for (int mem = 0; mem < members; mem++) {
      float v = Y[((size_t)mem * n + q) * kOutPad + d] * yf.scale[d] + yf.mean[d];
      if ((yf.log_mask >> d) & 1) v = expf(v);
      s += v;
      s2 += (double)v * v;
    }
    const double mu = s / members;
    mean[(size_t)q * kOut + d] = (float)mu;
    sd[(size_t)q * kOut + d] = (float)sqrt(fmax(s2 / members - mu * mu, 0.0));
  }
}

constexpr int kGateTile = 512;

__global__ void gate_kernel(const float* __restrict__ x, const float* __restrict__ Xq, int n,
                            const float* __restrict__ Xtrain, int nt, const float* __restrict__ lo,
                            const float* __restrict__ hi, float nn_cut,
                            const float* __restrict__ mean, const float* __restrict__ sd,
                            float tau, float tau_v, int* __restrict__ accept,
                            float* __restrict__ nn_dist) {
  __shared__ float tile[kGateTile * kIn];
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  float xq[kIn];
  bool inbox = q < n;
#pragma unroll
  for (int d = 0; d < kIn; d++) {
    xq[d] = q < n ? Xq[(size_t)q * kIn + d] : 0.0f;
    if (q < n) {
      const float raw = x[(size_t)q * kIn + d];
      inbox = inbox && raw >= lo[d] && raw <= hi[d];
    }
  }
  float best = 3.0e38f;
  for (int t0 = 0; t0 < nt; t0 += kGateTile) {
    const int cnt = min(kGateTile, nt - t0);
    __syncthreads();
    for (int k = threadIdx.x; k < cnt * kIn; k += blockDim.x) tile[k] = Xtrain[(size_t)t0 * kIn + k];
    __syncthreads();
    for (int j = 0; j < cnt; j++) {
      float d2 = 0.0f;
#pragma unroll
      for (int d = 0; d < kIn; d++) {
        const float e = xq[d] - tile[j * kIn + d];
        d2 += e * e;
      }
      best = fminf(best, d2);
    }
  }
  if (q >= n) return;
  const float nn = sqrtf(best);
  nn_dist[q] = nn;
  bool ok = inbox && nn <= nn_cut;
#pragma unroll
  for (int d = 0; d < 2; d++) {
    const float mu = mean[(size_t)q * kOut + d], s = sd[(size_t)q * kOut + d];
    ok = ok && isfinite(mu) && s <= (d == 0 ? tau : tau_v) * fabsf(mu);
  }
  accept[q] = ok ? 1 : 0;
}

inline unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

}  // namespace

cudaError_t launch_prep_inputs(const float* x, int n, const Xform& xf, bf16* X, float* Xf,
                               cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  prep_inputs_kernel<<<blocks(n, 128), 128, 0, s>>>(x, n, xf, X, Xf);
  return cudaGetLastError();
}

cudaError_t launch_prep_targets(const float* y, int n, const Xform& yf, float* T, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  prep_targets_kernel<<<blocks(n, 128), 128, 0, s>>>(y, n, yf, T);
  return cudaGetLastError();
}

cudaError_t launch_gather(const bf16* X, const float* T, int n, int bm, int members,
                          unsigned long long seed, const long long* d_step, bf16* Xb, bf16* Xbt,
                          float* Tb, cudaStream_t s) {
  gather_kernel<<<dim3(blocks(bm, 128), members), 128, 0, s>>>(X, T, n, bm, seed, d_step, Xb, Xbt,
                                                                Tb);
  return cudaGetLastError();
}

cudaError_t launch_loss(const float* Y, const float* Tb, const float* w, int bm, int members,
                        bf16* dY, bf16* dYt, float* dYft, double* loss, unsigned* status,
                        cudaStream_t s) {
  loss_kernel<<<dim3(blocks(bm, 128), members), 128, 0, s>>>(Y, Tb, w, bm, dY, dYt, dYft, loss,
                                                              status);
  return cudaGetLastError();
}

cudaError_t launch_rowsum_bf16(const bf16* in, int rows, int cols, int ld, long long sin_,
                               float* out, long long sout, int members, cudaStream_t s) {
  rowsum_kernel<bf16><<<dim3(blocks(rows, 8), members), 256, 0, s>>>(in, rows, cols, ld, sin_, out,
                                                                     sout);
  return cudaGetLastError();
}

cudaError_t launch_rowsum_f32(const float* in, int rows, int cols, int ld, long long sin_,
                              float* out, long long sout, int members, cudaStream_t s) {
  rowsum_kernel<float><<<dim3(blocks(rows, 8), members), 256, 0, s>>>(in, rows, cols, ld, sin_, out,
                                                                      sout);
  return cudaGetLastError();
}

cudaError_t launch_adam(float* p, const float* g, float* m, float* v, const Layout& L, int members,
                        float lr, float beta1, float beta2, float eps, const long long* d_step,
                        const long long* d_sched, bf16* Wb, bf16* WbT, cudaStream_t s) {
  adam_kernel<<<blocks(L.total * members, 256), 256, 0, s>>>(p, g, m, v, L, members, lr, beta1,
                                                              beta2, eps, d_step, d_sched, Wb, WbT);
  return cudaGetLastError();
}

__global__ void schedule_begin_kernel(const long long* __restrict__ d_step, long long* d_sched,
                                      long long steps) {
  d_sched[0] = *d_step;
  d_sched[1] = steps;
}

cudaError_t launch_schedule_begin(const long long* d_step, long long* d_sched, long long steps,
                                  cudaStream_t s) {
  schedule_begin_kernel<<<1, 1, 0, s>>>(d_step, d_sched, steps);
  return cudaGetLastError();
}

cudaError_t launch_cast_params(const float* p, const Layout& L, int members, bf16* Wb, bf16* WbT,
                               cudaStream_t s) {
  cast_params_kernel<<<blocks(L.total * members, 256), 256, 0, s>>>(p, L, members, Wb, WbT);
  return cudaGetLastError();
}

cudaError_t launch_advance_step(long long* d_step, cudaStream_t s) {
  advance_step_kernel<<<1, 1, 0, s>>>(d_step);
  return cudaGetLastError();
}

cudaError_t launch_decode(const float* Y, int n, int members, const Xform& yf, float* mean,
                          float* sd, cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  decode_kernel<<<blocks(n, 128), 128, 0, s>>>(Y, n, members, yf, mean, sd);
  return cudaGetLastError();
}

cudaError_t launch_gate(const float* x, const float* Xq, int n, const float* Xtrain, int nt,
                        const float* lo, const float* hi, float nn_cut, const float* mean,
                        const float* sd, float tau, float tau_v, int* accept, float* nn_dist,
                        cudaStream_t s) {
  if (n <= 0) return cudaSuccess;
  gate_kernel<<<blocks(n, 128), 128, 0, s>>>(x, Xq, n, Xtrain, nt, lo, hi, nn_cut, mean, sd, tau,
                                             tau_v, accept, nn_dist);
  return cudaGetLastError();
}

}  // namespace sg
