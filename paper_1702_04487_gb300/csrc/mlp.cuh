// Internal declarations of the surrogate network's kernels (BF16 tensor-core
// GEMM with fused epilogues, loss, bias gradients, Adam, input/output
// transforms, the acceptance gate).  Shared by mlp_kernels.cu and the host
// API in surrogate_api.cu.
#pragma once
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace sg {

typedef __nv_bfloat16 bf16;

// Status bits written by the kernels.
constexpr unsigned kStatusTimeout = 1u;   // an mbarrier wait ran out of iterations
constexpr unsigned kStatusNonFinite = 2u; // the loss met NaN or Inf

// Epilogues of C = A B^T (A: M x K, B: N x K, both K contiguous).
enum Epi {
  EPI_F32 = 0,        // Cf = acc                                   (weight gradients)
  EPI_BIAS_F32 = 1,   // Cf = acc + bias                            (output layer)
  EPI_BIAS_GELU = 2,  // z = acc + bias; Zout = z (optional);
                      // Cb = gelu(z) (optional), Ct = gelu(z)^T (optional)
  EPI_GELU_BWD = 3    // v = acc * gelu'(aux); Cb = v, Ct = v^T       (back-propagation)
};

// One GEMM, batched over grid.z (ensemble members) with element strides.
struct GemmArgs {
  const bf16* A;
  const bf16* B;
  int lda, ldb;
  int M, N, K;
  int epi;
  const float* bias;
  const float* aux;
  int ldaux;
  float* Cf;
  int ldcf;
  bf16* Cb;
  int ldcb;
  bf16* Ct;
  int ldct;
  float* Zout;
  int ldz;
  long long sA, sB, sBias, sAux, sCf, sCb, sCt, sZ;  // per-member strides (elements)
  unsigned* status;
};

// Requirements (checked by the host API): K, lda, ldb multiples of 8;
// output leading dimensions multiples of 8; 16-byte aligned base pointers.
cudaError_t launch_gemm(const GemmArgs& a, int members, cudaStream_t s);
size_t gemm_smem_bytes(int bn);

constexpr int kIn = 7, kInPad = 16, kOut = 4, kOutPad = 16, kHidden = 4;

// Per-feature transform: v -> ((log v if the bit is set) - mean) / scale.
struct Xform {
  float mean[kInPad];
  float scale[kInPad];
  int log_mask;
  int dim;
};

// Raw rows x [n][7] -> transformed BF16 rows X [n][16] (columns 7.. zero)
// and FP32 transformed copy Xf [n][7] (either may be null).
cudaError_t launch_prep_inputs(const float* x, int n, const Xform& xf, bf16* X, float* Xf,
                               cudaStream_t s);
// Raw targets y [n][4] -> transformed FP32 T [n][4].
cudaError_t launch_prep_targets(const float* y, int n, const Xform& yf, float* T, cudaStream_t s);
// Minibatch of `bm` rows per member drawn with replacement by a
// counter-based hash of (seed, member, step, row): Xb [m][bm][16], Xbt
// [m][16][bm], Tb [m][bm][4].
cudaError_t launch_gather(const bf16* X, const float* T, int n, int bm, int members,
                          unsigned long long seed, const long long* d_step, bf16* Xb, bf16* Xbt,
                          float* Tb, cudaStream_t s);
// Loss 1/(bm*4) sum w (y - t)^2 of every member: dY = 2 w (y - t) / (bm*4)
// as BF16 [m][bm][16] and its transpose [m][16][bm], FP32 transpose
// dYft [m][16][bm]; the loss sum is added to loss[member] (FP64).
cudaError_t launch_loss(const float* Y, const float* Tb, const float* w, int bm, int members,
                        bf16* dY, bf16* dYt, float* dYft, double* loss, unsigned* status,
                        cudaStream_t s);
// out[m][r] = sum_c in[m][r][c] for rows r < rows, c < cols (row length ld).
cudaError_t launch_rowsum_bf16(const bf16* in, int rows, int cols, int ld, long long sin_,
                               float* out, long long sout, int members, cudaStream_t s);
cudaError_t launch_rowsum_f32(const float* in, int rows, int cols, int ld, long long sin_,
                              float* out, long long sout, int members, cudaStream_t s);

// Parameter block of one member: for each layer l, Wt_l [out][in] then b_l [out].
struct Layout {
  int nin[kHidden + 1], nout[kHidden + 1];
  long long w_off[kHidden + 1], b_off[kHidden + 1];
  long long total;
};
// Adam (bias-corrected, step t = *d_step + 1) on every parameter of every
// member, then BF16 copies: Wb (same layout) and WbT (layer-wise transposes).
// d_sched (may be null): {first step, step count} of the current training
// call, over which lr decays along a half cosine.
cudaError_t launch_adam(float* p, const float* g, float* m, float* v, const Layout& L, int members,
                        float lr, float beta1, float beta2, float eps, const long long* d_step,
                        const long long* d_sched, bf16* Wb, bf16* WbT, cudaStream_t s);
// d_sched = {*d_step, steps}: the start of a training call of `steps` steps.
cudaError_t launch_schedule_begin(const long long* d_step, long long* d_sched, long long steps,
                                  cudaStream_t s);
// BF16 copies of the parameters without an update.
cudaError_t launch_cast_params(const float* p, const Layout& L, int members, bf16* Wb, bf16* WbT,
                               cudaStream_t s);
cudaError_t launch_advance_step(long long* d_step, cudaStream_t s);
// Member outputs Y [m][n][16] -> inverse-transformed outcomes, their mean
// and standard deviation over members: mean [n][4], std [n][4].
cudaError_t launch_decode(const float* Y, int n, int members, const Xform& yf, float* mean,
                          float* sd, cudaStream_t s);
// Acceptance gate: inside the per-feature box [lo, hi] of the training
// inputs, nearest training point (transformed space) within nn_cut, and
// relative ensemble spread sd/|mean| of outcome 0 below tau and of
// outcome 1 below tau_v.
cudaError_t launch_gate(const float* x, const float* Xq, int n, const float* Xtrain, int nt,
                        const float* lo, const float* hi, float nn_cut, const float* mean,
                        const float* sd, float tau, float tau_v, int* accept, float* nn_dist,
                        cudaStream_t s);

}  // namespace sg
