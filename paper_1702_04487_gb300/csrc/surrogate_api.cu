// Host side of the surrogate: ensemble parameters, training step (captured
// once as a CUDA graph and replayed), prediction with the acceptance gate,
// and the C ABI of include/surrogate.h.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/surrogate.h"
#include "mlp.cuh"

using namespace sg;

namespace {

thread_local char g_err[512] = "";

ij_status fail(ij_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

#define CUDA_TRY(x)                                                                  \
  do {                                                                               \
    cudaError_t e_ = (x);                                                            \
    if (e_ != cudaSuccess) return fail(IJ_ERR_CUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
  } while (0)

unsigned long long mix64(unsigned long long z) {
  z += 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

}  // namespace

struct sg_handle_s {
  sg_config cfg;
  int K = 1, H = 16, bm = 16;
  Layout L;
  cudaStream_t stream = nullptr;
  ij_alloc_fn alloc = nullptr;
  ij_free_fn free_fn = nullptr;
  void* ctx = nullptr;
  std::vector<void*> blocks;
  // parameters [K][P]
  float *p = nullptr, *g = nullptr, *m = nullptr, *v = nullptr;
  bf16 *Wb = nullptr, *WbT = nullptr;
  // transforms and gate
  Xform xin, xout;
  float tau = 0.01f, tau_v = 0.01f, nn_cut = 0.0f;
  float lo[kIn], hi[kIn];
  float *d_lo = nullptr, *d_hi = nullptr, *d_w = nullptr;
  // training data
  int n_train = 0;
  bf16* X = nullptr;
  float *T = nullptr, *Xf = nullptr;
  // minibatch workspace
  bf16 *Xb = nullptr, *Xbt = nullptr;
  float* Tb = nullptr;
  float* Z[kHidden] = {};
  bf16* Ha[kHidden] = {};
  bf16* Ht[kHidden] = {};
  float* Y = nullptr;
  bf16 *dY = nullptr, *dYt = nullptr;
  float* dYft = nullptr;
  bf16* dZ[2] = {};
  bf16* dZt[2] = {};
  double* d_loss = nullptr;
  unsigned* d_status = nullptr;
  long long* d_step = nullptr;
  long long* d_sched = nullptr;  // {first step, steps} of the current sg_train call
  cudaStream_t cap = nullptr;
  cudaGraphExec_t gexec = nullptr;
  // inference workspace (grown on demand)
  int q_cap = 0;
  float *q_x = nullptr, *q_xf = nullptr, *q_y = nullptr, *q_mean = nullptr, *q_sd = nullptr,
        *q_nn = nullptr;
  bf16 *q_x16 = nullptr, *q_h[2] = {};
  int* q_acc = nullptr;

  void* dalloc(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    void* ptr = nullptr;
    if (alloc)
      ptr = alloc(bytes, ctx);
    else if (cudaMalloc(&ptr, bytes) != cudaSuccess)
      ptr = nullptr;
    if (ptr) blocks.push_back(ptr);
    return ptr;
  }
  void release() {
    if (stream) cudaStreamSynchronize(stream); else cudaDeviceSynchronize();
    if (gexec) cudaGraphExecDestroy(gexec);
    if (cap) cudaStreamDestroy(cap);
    for (void* b : blocks) {
      if (free_fn) free_fn(b, ctx); else cudaFree(b);
    }
    blocks.clear();
  }
};

namespace {

Layout make_layout(int H) {
  Layout L;
  const int nin[kHidden + 1] = {kInPad, H, H, H, H};
  const int nout[kHidden + 1] = {H, H, H, H, kOutPad};
  long long off = 0;
  for (int l = 0; l <= kHidden; l++) {
    L.nin[l] = nin[l];
    L.nout[l] = nout[l];
    L.w_off[l] = off;
    off += (long long)nin[l] * nout[l];
    L.b_off[l] = off;
    off += nout[l];
  }
  L.total = off;
  return L;
}

GemmArgs gemm_args() {
  GemmArgs a;
  memset(&a, 0, sizeof(a));
  return a;
}

ij_status status_check(sg_handle h) {
  unsigned st = 0;
  CUDA_TRY(cudaMemcpyAsync(&st, h->d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (st & kStatusTimeout)
    return fail(IJ_ERR_TIMEOUT, "a tensor-core completion wait ran out of its iteration limit");
  if (st & kStatusNonFinite) return fail(IJ_ERR_NUMERIC, "non-finite training loss");
  return IJ_OK;
}

// Forward pass of every member on the minibatch buffers (training layout).
cudaError_t enqueue_forward_train(sg_handle h, int bm, cudaStream_t s) {
  const int H = h->H, K = h->K;
  const long long P = h->L.total;
  cudaError_t e = cudaSuccess;
  for (int l = 0; l <= kHidden && e == cudaSuccess; l++) {
    GemmArgs a = gemm_args();
    a.status = h->d_status;
    a.B = h->Wb + h->L.w_off[l];
    a.sB = P;
    a.ldb = h->L.nin[l];
    a.bias = h->p + h->L.b_off[l];
    a.sBias = P;
    a.M = bm;
    a.N = h->L.nout[l];
    a.K = h->L.nin[l];
    if (l == 0) {
      a.A = h->Xb;
      a.lda = kInPad;
      a.sA = (long long)bm * kInPad;
    } else {
      a.A = h->Ha[l - 1];
      a.lda = H;
      a.sA = (long long)bm * H;
    }
    if (l < kHidden) {
      a.epi = EPI_BIAS_GELU;
      a.Zout = h->Z[l];
      a.ldz = H;
      a.sZ = (long long)bm * H;
      a.Cb = h->Ha[l];
      a.ldcb = H;
      a.sCb = (long long)bm * H;
      a.Ct = h->Ht[l];
      a.ldct = bm;
      a.sCt = (long long)H * bm;
    } else {
      a.epi = EPI_BIAS_F32;
      a.Cf = h->Y;
      a.ldcf = kOutPad;
      a.sCf = (long long)bm * kOutPad;
    }
    e = launch_gemm(a, K, s);
  }
  return e;
}

// Loss and backward pass into h->g (all members).
cudaError_t enqueue_backward(sg_handle h, int bm, cudaStream_t s) {
  const int H = h->H, K = h->K;
  const long long P = h->L.total;
  cudaError_t e = launch_loss(h->Y, h->Tb, h->d_w, bm, K, h->dY, h->dYt, h->dYft, h->d_loss,
                              h->d_status, s);
  if (e != cudaSuccess) return e;
  // output layer: gW5 = dY^T H4, gb5 = column sums of dY
  {
    GemmArgs a = gemm_args();
    a.status = h->d_status;
    a.epi = EPI_F32;
    a.A = h->dYt;
    a.lda = bm;
    a.sA = (long long)kOutPad * bm;
    a.B = h->Ht[kHidden - 1];
    a.ldb = bm;
    a.sB = (long long)H * bm;
    a.M = kOutPad;
    a.N = H;
    a.K = bm;
    a.Cf = h->g + h->L.w_off[kHidden];
    a.ldcf = H;
    a.sCf = P;
    if ((e = launch_gemm(a, K, s)) != cudaSuccess) return e;
    if ((e = launch_rowsum_f32(h->dYft, kOutPad, bm, bm, (long long)kOutPad * bm,
                               h->g + h->L.b_off[kHidden], P, K, s)) != cudaSuccess)
      return e;
  }
  // dZ of the last hidden layer: (dY W5) * gelu'(Z4)
  int cur = 0;
  {
    GemmArgs a = gemm_args();
    a.status = h->d_status;
    a.epi = EPI_GELU_BWD;
    a.A = h->dY;
    a.lda = kOutPad;
    a.sA = (long long)bm * kOutPad;
    a.B = h->WbT + h->L.w_off[kHidden];
    a.ldb = kOutPad;
    a.sB = P;
    a.M = bm;
    a.N = H;
    a.K = kOutPad;
    a.aux = h->Z[kHidden - 1];
    a.ldaux = H;
    a.sAux = (long long)bm * H;
    a.Cb = h->dZ[cur];
    a.ldcb = H;
    a.sCb = (long long)bm * H;
    a.Ct = h->dZt[cur];
    a.ldct = bm;
    a.sCt = (long long)H * bm;
    if ((e = launch_gemm(a, K, s)) != cudaSuccess) return e;
  }
  for (int l = kHidden - 1; l >= 0; l--) {
    // weight gradient of layer l: dZ_l^T times the layer's input
    GemmArgs a = gemm_args();
    a.status = h->d_status;
    a.epi = EPI_F32;
    a.A = h->dZt[cur];
    a.lda = bm;
    a.sA = (long long)H * bm;
    if (l == 0) {
      a.B = h->Xbt;
      a.sB = (long long)kInPad * bm;
    } else {
      a.B = h->Ht[l - 1];
      a.sB = (long long)H * bm;
    }
    a.ldb = bm;
    a.M = H;
    a.N = h->L.nin[l];
    a.K = bm;
    a.Cf = h->g + h->L.w_off[l];
    a.ldcf = h->L.nin[l];
    a.sCf = P;
    if ((e = launch_gemm(a, K, s)) != cudaSuccess) return e;
    if ((e = launch_rowsum_bf16(h->dZt[cur], H, bm, bm, (long long)H * bm, h->g + h->L.b_off[l], P,
                                K, s)) != cudaSuccess)
      return e;
    if (l == 0) break;
    // dZ_{l-1} = (dZ_l W_l) * gelu'(Z_{l-1})
    GemmArgs b = gemm_args();
    b.status = h->d_status;
    b.epi = EPI_GELU_BWD;
    b.A = h->dZ[cur];
    b.lda = H;
    b.sA = (long long)bm * H;
    b.B = h->WbT + h->L.w_off[l];
    b.ldb = H;
    b.sB = P;
    b.M = bm;
    b.N = H;
    b.K = H;
    b.aux = h->Z[l - 1];
    b.ldaux = H;
    b.sAux = (long long)bm * H;
    b.Cb = h->dZ[cur ^ 1];
    b.ldcb = H;
    b.sCb = (long long)bm * H;
    b.Ct = h->dZt[cur ^ 1];
    b.ldct = bm;
    b.sCt = (long long)H * bm;
    if ((e = launch_gemm(b, K, s)) != cudaSuccess) return e;
    cur ^= 1;
  }
  return cudaSuccess;
}

cudaError_t enqueue_train_step(sg_handle h, cudaStream_t s) {
  cudaError_t e = launch_gather(h->X, h->T, h->n_train, h->bm, h->K, h->cfg.seed ^ 0x5EEDull,
                                h->d_step, h->Xb, h->Xbt, h->Tb, s);
  if (e == cudaSuccess) e = enqueue_forward_train(h, h->bm, s);
  if (e == cudaSuccess) e = enqueue_backward(h, h->bm, s);
  if (e == cudaSuccess)
    e = launch_adam(h->p, h->g, h->m, h->v, h->L, h->K, h->cfg.lr, h->cfg.beta1, h->cfg.beta2,
                    h->cfg.eps, h->d_step, h->cfg.lr_cosine ? h->d_sched : nullptr, h->Wb, h->WbT,
                    s);
  if (e == cudaSuccess) e = launch_advance_step(h->d_step, s);
  return e;
}

// Transform (mean, scale) of each column of a [n][dim] host array.
void fit_xform(const float* a, int n, int dim, int log_mask, Xform& xf) {
  memset(&xf, 0, sizeof(xf));
  xf.log_mask = log_mask;
  xf.dim = dim;
  for (int d = 0; d < dim; d++) {
    double s = 0, s2 = 0;
    for (int i = 0; i < n; i++) {
      double v = a[(size_t)i * dim + d];
      if ((log_mask >> d) & 1) v = log(v);
      s += v;
      s2 += v * v;
    }
    const double mu = s / n, var = std::max(s2 / n - mu * mu, 0.0);
    xf.mean[d] = (float)mu;
    xf.scale[d] = var > 1e-24 ? (float)sqrt(var) : 1.0f;
  }
  for (int d = dim; d < kInPad; d++) xf.scale[d] = 1.0f;
}

ij_status ensure_query(sg_handle h, int n) {
  if (n <= h->q_cap) return IJ_OK;
  const size_t nn = (size_t)n, K = h->K, H = h->H;
  h->q_x = (float*)h->dalloc(nn * kIn * 4);
  h->q_xf = (float*)h->dalloc(nn * kIn * 4);
  h->q_x16 = (bf16*)h->dalloc(nn * kInPad * 2);
  h->q_h[0] = (bf16*)h->dalloc(K * nn * H * 2);
  h->q_h[1] = (bf16*)h->dalloc(K * nn * H * 2);
  h->q_y = (float*)h->dalloc(K * nn * kOutPad * 4);
  h->q_mean = (float*)h->dalloc(nn * kOut * 4);
  h->q_sd = (float*)h->dalloc(nn * kOut * 4);
  h->q_nn = (float*)h->dalloc(nn * 4);
  h->q_acc = (int*)h->dalloc(nn * 4);
  if (!h->q_x || !h->q_xf || !h->q_x16 || !h->q_h[0] || !h->q_h[1] || !h->q_y || !h->q_mean ||
      !h->q_sd || !h->q_nn || !h->q_acc)
    return fail(IJ_ERR_OOM, "device allocation of the query workspace failed");
  h->q_cap = n;
  return IJ_OK;
}

}  // namespace

extern "C" {

ij_status sg_create(const sg_config* cfg, ij_alloc_fn alloc, ij_free_fn free_fn, void* ctx,
                    void* stream, sg_handle* out) {
  if (!out) return fail(IJ_ERR_PARAM, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(IJ_ERR_PARAM, "cfg is NULL");
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(IJ_ERR_PARAM, "alloc and free must both be set or both be NULL");
  if (cfg->members < 1 || cfg->members > 8) return fail(IJ_ERR_PARAM, "members must be in 1..8");
  if (cfg->hidden < 16 || cfg->hidden > 256 || cfg->hidden % 16)
    return fail(IJ_ERR_PARAM, "hidden must be a multiple of 16 in 16..256");
  if (cfg->batch < 16 || cfg->batch > 65536 || cfg->batch % 16)
    return fail(IJ_ERR_PARAM, "batch must be a multiple of 16 in 16..65536");
  if (!(cfg->lr > 0) || !(cfg->beta1 >= 0 && cfg->beta1 < 1) || !(cfg->beta2 >= 0 && cfg->beta2 < 1) ||
      !(cfg->eps > 0))
    return fail(IJ_ERR_PARAM, "Adam settings out of range");
  if (cfg->lr_cosine != 0 && cfg->lr_cosine != 1) return fail(IJ_ERR_PARAM, "lr_cosine must be 0 or 1");
  sg_handle h = new sg_handle_s();
  h->cfg = *cfg;
  h->K = cfg->members;
  h->H = cfg->hidden;
  h->bm = cfg->batch;
  h->L = make_layout(h->H);
  h->alloc = alloc;
  h->free_fn = free_fn;
  h->ctx = ctx;
  h->stream = (cudaStream_t)stream;
  auto bail = [&](ij_status st) {
    h->release();
    delete h;
    return st;
  };
  const size_t KP = (size_t)h->K * h->L.total, K = h->K, H = h->H, bm = h->bm;
  h->p = (float*)h->dalloc(KP * 4);
  h->g = (float*)h->dalloc(KP * 4);
  h->m = (float*)h->dalloc(KP * 4);
  h->v = (float*)h->dalloc(KP * 4);
  h->Wb = (bf16*)h->dalloc(KP * 2);
  h->WbT = (bf16*)h->dalloc(KP * 2);
  h->Xb = (bf16*)h->dalloc(K * bm * kInPad * 2);
  h->Xbt = (bf16*)h->dalloc(K * bm * kInPad * 2);
  h->Tb = (float*)h->dalloc(K * bm * kOut * 4);
  for (int l = 0; l < kHidden; l++) {
    h->Z[l] = (float*)h->dalloc(K * bm * H * 4);
    h->Ha[l] = (bf16*)h->dalloc(K * bm * H * 2);
    h->Ht[l] = (bf16*)h->dalloc(K * bm * H * 2);
  }
  h->Y = (float*)h->dalloc(K * bm * kOutPad * 4);
  h->dY = (bf16*)h->dalloc(K * bm * kOutPad * 2);
  h->dYt = (bf16*)h->dalloc(K * bm * kOutPad * 2);
  h->dYft = (float*)h->dalloc(K * bm * kOutPad * 4);
  for (int j = 0; j < 2; j++) {
    h->dZ[j] = (bf16*)h->dalloc(K * bm * H * 2);
    h->dZt[j] = (bf16*)h->dalloc(K * bm * H * 2);
  }
  h->d_loss = (double*)h->dalloc(K * 8);
  h->d_status = (unsigned*)h->dalloc(4);
  h->d_step = (long long*)h->dalloc(8);
  h->d_sched = (long long*)h->dalloc(16);
  h->d_lo = (float*)h->dalloc(kIn * 4);
  h->d_hi = (float*)h->dalloc(kIn * 4);
  h->d_w = (float*)h->dalloc(kOut * 4);
  for (void* b : {(void*)h->p, (void*)h->g, (void*)h->m, (void*)h->v, (void*)h->Wb, (void*)h->WbT,
                  (void*)h->Xb, (void*)h->Xbt, (void*)h->Tb, (void*)h->Y, (void*)h->dY,
                  (void*)h->dYt, (void*)h->dYft, (void*)h->d_loss, (void*)h->d_status,
                  (void*)h->d_step, (void*)h->d_sched, (void*)h->d_lo, (void*)h->d_hi,
                  (void*)h->d_w})
    if (!b) return bail(fail(IJ_ERR_OOM, "device allocation failed"));
  for (int l = 0; l < kHidden; l++)
    if (!h->Z[l] || !h->Ha[l] || !h->Ht[l]) return bail(fail(IJ_ERR_OOM, "device allocation failed"));
  for (int j = 0; j < 2; j++)
    if (!h->dZ[j] || !h->dZt[j]) return bail(fail(IJ_ERR_OOM, "device allocation failed"));
  // He-uniform initialisation on the host (once), zero biases and padding
  std::vector<float> init(KP, 0.0f);
  for (int mem = 0; mem < h->K; mem++)
    for (int l = 0; l <= kHidden; l++) {
      const int fan_in = l == 0 ? kIn : h->H;
      const double bound = sqrt(6.0 / fan_in);
      for (int r = 0; r < h->L.nout[l]; r++)
        for (int c = 0; c < h->L.nin[l]; c++) {
          if ((l == 0 && c >= kIn) || (l == kHidden && r >= kOut)) continue;
          const long long idx = h->L.w_off[l] + (long long)r * h->L.nin[l] + c;
          const unsigned long long u =
              mix64(cfg->seed ^ mix64(((unsigned long long)mem << 40) ^ (unsigned long long)idx));
          const double U = (double)(u >> 11) * (1.0 / 9007199254740992.0);
          init[(size_t)mem * h->L.total + idx] = (float)((2.0 * U - 1.0) * bound);
        }
    }
  cudaStream_t s = h->stream;
  CUDA_TRY(cudaMemcpyAsync(h->p, init.data(), KP * 4, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemsetAsync(h->g, 0, KP * 4, s));
  CUDA_TRY(cudaMemsetAsync(h->m, 0, KP * 4, s));
  CUDA_TRY(cudaMemsetAsync(h->v, 0, KP * 4, s));
  CUDA_TRY(cudaMemsetAsync(h->d_status, 0, 4, s));
  CUDA_TRY(cudaMemsetAsync(h->d_step, 0, 8, s));
  CUDA_TRY(cudaMemsetAsync(h->d_sched, 0, 16, s));
  CUDA_TRY(cudaMemcpyAsync(h->d_w, cfg->out_weight, kOut * 4, cudaMemcpyHostToDevice, s));
  CUDA_TRY(launch_cast_params(h->p, h->L, h->K, h->Wb, h->WbT, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  memset(&h->xin, 0, sizeof(Xform));
  memset(&h->xout, 0, sizeof(Xform));
  for (int d = 0; d < kInPad; d++) h->xin.scale[d] = h->xout.scale[d] = 1.0f;
  *out = h;
  return IJ_OK;
}

ij_status sg_set_data(sg_handle h, const float* x, const float* y, int n) {
  if (!h || !x || !y) return fail(IJ_ERR_PARAM, "null argument");
  if (n < 2) return fail(IJ_ERR_PARAM, "n must be >= 2");
  for (long long i = 0; i < (long long)n * kIn; i++)
    if (!isfinite(x[i]) || (((h->cfg.log_inputs >> (i % kIn)) & 1) && !(x[i] > 0)))
      return fail(IJ_ERR_PARAM, "input row %lld: non-finite or non-positive under a log", i / kIn);
  for (long long i = 0; i < (long long)n * kOut; i++)
    if (!isfinite(y[i]) || (((h->cfg.log_outputs >> (i % kOut)) & 1) && !(y[i] > 0)))
      return fail(IJ_ERR_PARAM, "outcome row %lld: non-finite or non-positive under a log",
                  i / kOut);
  fit_xform(x, n, kIn, h->cfg.log_inputs, h->xin);
  fit_xform(y, n, kOut, h->cfg.log_outputs, h->xout);
  for (int d = 0; d < kIn; d++) {
    h->lo[d] = h->hi[d] = x[d];
    for (int i = 1; i < n; i++) {
      h->lo[d] = std::min(h->lo[d], x[(size_t)i * kIn + d]);
      h->hi[d] = std::max(h->hi[d], x[(size_t)i * kIn + d]);
    }
  }
  // leave-one-out nearest-neighbour distances in transformed input space
  std::vector<double> xt((size_t)n * kIn);
  for (int i = 0; i < n; i++)
    for (int d = 0; d < kIn; d++) {
      double v = x[(size_t)i * kIn + d];
      if ((h->cfg.log_inputs >> d) & 1) v = log(v);
      xt[(size_t)i * kIn + d] = (v - h->xin.mean[d]) / h->xin.scale[d];
    }
  std::vector<double> nn(n, 1e300);
  for (int i = 0; i < n; i++)
    for (int j = i + 1; j < n; j++) {
      double d2 = 0;
      for (int d = 0; d < kIn; d++) {
        const double e = xt[(size_t)i * kIn + d] - xt[(size_t)j * kIn + d];
        d2 += e * e;
      }
      nn[i] = std::min(nn[i], d2);
      nn[j] = std::min(nn[j], d2);
    }
  std::sort(nn.begin(), nn.end());
  h->nn_cut = (float)(2.0 * sqrt(nn[(size_t)((n - 1) * 0.95)]));

  cudaStream_t s = h->stream;
  if (n > h->n_train) {
    h->X = (bf16*)h->dalloc((size_t)n * kInPad * 2);
    h->T = (float*)h->dalloc((size_t)n * kOut * 4);
    h->Xf = (float*)h->dalloc((size_t)n * kIn * 4);
    if (!h->X || !h->T || !h->Xf) return fail(IJ_ERR_OOM, "device allocation of the data failed");
  }
  // raw rows staged in the query workspace
  ij_status st = ensure_query(h, n);
  if (st != IJ_OK) return st;
  CUDA_TRY(cudaMemcpyAsync(h->q_x, x, (size_t)n * kIn * 4, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(h->q_mean, y, (size_t)n * kOut * 4, cudaMemcpyHostToDevice, s));
  CUDA_TRY(launch_prep_inputs(h->q_x, n, h->xin, h->X, h->Xf, s));
  CUDA_TRY(launch_prep_targets(h->q_mean, n, h->xout, h->T, s));
  CUDA_TRY(cudaMemcpyAsync(h->d_lo, h->lo, kIn * 4, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(h->d_hi, h->hi, kIn * 4, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  h->n_train = n;
  if (h->gexec) {  // the captured step bakes in n_train
    cudaGraphExecDestroy(h->gexec);
    h->gexec = nullptr;
  }
  return IJ_OK;
}

ij_status sg_train(sg_handle h, int steps, double* loss) {
  if (!h) return fail(IJ_ERR_PARAM, "null handle");
  if (steps < 0) return fail(IJ_ERR_PARAM, "steps < 0");
  if (h->n_train < 2) return fail(IJ_ERR_STATE, "no training data (sg_set_data)");
  if (!h->gexec) {
    if (!h->cap) CUDA_TRY(cudaStreamCreateWithFlags(&h->cap, cudaStreamNonBlocking));
    CUDA_TRY(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    cudaError_t e = cudaMemsetAsync(h->d_loss, 0, h->K * 8, h->cap);
    if (e == cudaSuccess) e = enqueue_train_step(h, h->cap);
    cudaGraph_t gr = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(h->cap, &gr);
    if (e != cudaSuccess || e2 != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      return fail(IJ_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    e = cudaGraphInstantiate(&h->gexec, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) return fail(IJ_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  }
  if (h->cfg.lr_cosine && steps > 0)
    CUDA_TRY(launch_schedule_begin(h->d_step, h->d_sched, steps, h->stream));
  for (int i = 0; i < steps; i++) CUDA_TRY(cudaGraphLaunch(h->gexec, h->stream));
  ij_status st = status_check(h);
  if (st != IJ_OK) return st;
  if (loss) {
    std::vector<double> l(h->K);
    CUDA_TRY(cudaMemcpy(l.data(), h->d_loss, h->K * 8, cudaMemcpyDeviceToHost));
    double s = 0;
    for (double v : l) s += v;
    *loss = steps > 0 ? s / h->K : 0.0;
  }
  return IJ_OK;
}

ij_status sg_predict(sg_handle h, const float* x, int n, float* mean, float* sd, int* accept,
                     int on_device) {
  if (!h || !x) return fail(IJ_ERR_PARAM, "null argument");
  if (n < 0) return fail(IJ_ERR_PARAM, "n < 0");
  if (n == 0) return IJ_OK;
  if (accept && h->n_train < 2) return fail(IJ_ERR_STATE, "the gate needs training data");
  ij_status st = ensure_query(h, n);
  if (st != IJ_OK) return st;
  cudaStream_t s = h->stream;
  const float* dx = x;
  if (!on_device) {
    CUDA_TRY(cudaMemcpyAsync(h->q_x, x, (size_t)n * kIn * 4, cudaMemcpyHostToDevice, s));
    dx = h->q_x;
  }
  CUDA_TRY(launch_prep_inputs(dx, n, h->xin, h->q_x16, h->q_xf, s));
  const int H = h->H;
  const long long P = h->L.total;
  for (int l = 0; l <= kHidden; l++) {
    GemmArgs a = gemm_args();
    a.status = h->d_status;
    a.B = h->Wb + h->L.w_off[l];
    a.sB = P;
    a.ldb = h->L.nin[l];
    a.bias = h->p + h->L.b_off[l];
    a.sBias = P;
    a.M = n;
    a.N = h->L.nout[l];
    a.K = h->L.nin[l];
    if (l == 0) {
      a.A = h->q_x16;
      a.lda = kInPad;
      a.sA = 0;  // one input for every member
    } else {
      a.A = h->q_h[(l - 1) & 1];
      a.lda = H;
      a.sA = (long long)n * H;
    }
    if (l < kHidden) {
      a.epi = EPI_BIAS_GELU;
      a.Cb = h->q_h[l & 1];
      a.ldcb = H;
      a.sCb = (long long)n * H;
    } else {
      a.epi = EPI_BIAS_F32;
      a.Cf = h->q_y;
      a.ldcf = kOutPad;
      a.sCf = (long long)n * kOutPad;
    }
    CUDA_TRY(launch_gemm(a, h->K, s));
  }
  CUDA_TRY(launch_decode(h->q_y, n, h->K, h->xout, h->q_mean, h->q_sd, s));
  if (accept)
    CUDA_TRY(launch_gate(dx, h->q_xf, n, h->Xf, h->n_train, h->d_lo, h->d_hi, h->nn_cut, h->q_mean,
                         h->q_sd, h->tau, h->tau_v, h->q_acc, h->q_nn, s));
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (mean) CUDA_TRY(cudaMemcpyAsync(mean, h->q_mean, (size_t)n * kOut * 4, kind, s));
  if (sd) CUDA_TRY(cudaMemcpyAsync(sd, h->q_sd, (size_t)n * kOut * 4, kind, s));
  if (accept) CUDA_TRY(cudaMemcpyAsync(accept, h->q_acc, (size_t)n * 4, kind, s));
  return status_check(h);
}

ij_status sg_set_gate(sg_handle h, float tau, float tau_v, float nn_cut) {
  if (!h) return fail(IJ_ERR_PARAM, "null handle");
  if (!(tau > 0) || !(tau_v > 0)) return fail(IJ_ERR_PARAM, "tau and tau_v must be > 0");
  h->tau = tau;
  h->tau_v = tau_v;
  if (nn_cut > 0) h->nn_cut = nn_cut;
  return IJ_OK;
}

ij_status sg_param_count(sg_handle h, long long* count) {
  if (!h || !count) return fail(IJ_ERR_PARAM, "null argument");
  *count = h->L.total;
  return IJ_OK;
}

ij_status sg_get_params(sg_handle h, int member, float* out) {
  if (!h || !out) return fail(IJ_ERR_PARAM, "null argument");
  if (member < 0 || member >= h->K) return fail(IJ_ERR_PARAM, "member out of range");
  CUDA_TRY(cudaMemcpyAsync(out, h->p + (size_t)member * h->L.total, h->L.total * 4,
                           cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return IJ_OK;
}

ij_status sg_set_params(sg_handle h, int member, const float* in) {
  if (!h || !in) return fail(IJ_ERR_PARAM, "null argument");
  if (member < 0 || member >= h->K) return fail(IJ_ERR_PARAM, "member out of range");
  CUDA_TRY(cudaMemcpyAsync(h->p + (size_t)member * h->L.total, in, h->L.total * 4,
                           cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(launch_cast_params(h->p, h->L, h->K, h->Wb, h->WbT, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return IJ_OK;
}

ij_status sg_get_transform(sg_handle h, float* in_mean, float* in_scale, float* out_mean,
                           float* out_scale) {
  if (!h) return fail(IJ_ERR_PARAM, "null handle");
  for (int d = 0; d < kIn; d++) {
    if (in_mean) in_mean[d] = h->xin.mean[d];
    if (in_scale) in_scale[d] = h->xin.scale[d];
  }
  for (int d = 0; d < kOut; d++) {
    if (out_mean) out_mean[d] = h->xout.mean[d];
    if (out_scale) out_scale[d] = h->xout.scale[d];
  }
  return IJ_OK;
}

ij_status sg_gradients(sg_handle h, const float* x, const float* y, int n, float* grads,
                       double* loss) {
  if (!h || !x || !y || !grads) return fail(IJ_ERR_PARAM, "null argument");
  if (n < 16 || n % 16 || n > h->bm) return fail(IJ_ERR_PARAM, "n must be a multiple of 16, <= batch");
  cudaStream_t s = h->stream;
  ij_status st = ensure_query(h, n);
  if (st != IJ_OK) return st;
  bf16* x16 = h->q_x16;
  float* t = h->q_sd;
  CUDA_TRY(cudaMemcpyAsync(h->q_x, x, (size_t)n * kIn * 4, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(h->q_mean, y, (size_t)n * kOut * 4, cudaMemcpyHostToDevice, s));
  CUDA_TRY(launch_prep_inputs(h->q_x, n, h->xin, x16, nullptr, s));
  CUDA_TRY(launch_prep_targets(h->q_mean, n, h->xout, t, s));
  // every member sees the same rows: replicate them into the minibatch layout
  for (int mem = 0; mem < h->K; mem++) {
    CUDA_TRY(cudaMemcpyAsync(h->Xb + (size_t)mem * n * kInPad, x16, (size_t)n * kInPad * 2,
                             cudaMemcpyDeviceToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(h->Tb + (size_t)mem * n * kOut, t, (size_t)n * kOut * 4,
                             cudaMemcpyDeviceToDevice, s));
  }
  // transpose of the input rows: one column at a time
  for (int mem = 0; mem < h->K; mem++)
    for (int d = 0; d < kInPad; d++)
      CUDA_TRY(cudaMemcpy2DAsync(h->Xbt + (size_t)mem * kInPad * n + (size_t)d * n, 2, x16 + d,
                                 kInPad * 2, 2, n, cudaMemcpyDeviceToDevice, s));
  CUDA_TRY(cudaMemsetAsync(h->d_loss, 0, h->K * 8, s));
  CUDA_TRY(enqueue_forward_train(h, n, s));
  CUDA_TRY(enqueue_backward(h, n, s));
  st = status_check(h);
  if (st != IJ_OK) return st;
  CUDA_TRY(cudaMemcpy(grads, h->g, (size_t)h->K * h->L.total * 4, cudaMemcpyDeviceToHost));
  if (loss) CUDA_TRY(cudaMemcpy(loss, h->d_loss, h->K * 8, cudaMemcpyDeviceToHost));
  return IJ_OK;
}

ij_status sg_destroy(sg_handle h) {
  if (!h) return IJ_OK;
  h->release();
  delete h;
  return IJ_OK;
}

const char* sg_last_error(void) { return g_err; }

ij_status sg_gemm_bf16(const void* A, int lda, const void* B, int ldb, int M, int N, int K,
                       float* C, int ldc, void* stream) {
  if (!A || !B || !C) return fail(IJ_ERR_PARAM, "null pointer");
  if (M < 1 || N < 1 || K < 1) return fail(IJ_ERR_PARAM, "M, N, K must be >= 1");
  if (K % 8 || lda % 8 || ldb % 8 || lda < K || ldb < K || ldc < N)
    return fail(IJ_ERR_PARAM, "K, lda, ldb must be multiples of 8, lda, ldb >= K, ldc >= N");
  if (((uintptr_t)A | (uintptr_t)B) & 15) return fail(IJ_ERR_PARAM, "A and B must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  unsigned* status = nullptr;
  CUDA_TRY(cudaMallocAsync((void**)&status, sizeof(unsigned), s));
  CUDA_TRY(cudaMemsetAsync(status, 0, sizeof(unsigned), s));
  GemmArgs a = gemm_args();
  a.A = (const bf16*)A;
  a.B = (const bf16*)B;
  a.lda = lda;
  a.ldb = ldb;
  a.M = M;
  a.N = N;
  a.K = K;
  a.epi = EPI_F32;
  a.Cf = C;
  a.ldcf = ldc;
  a.status = status;
  CUDA_TRY(launch_gemm(a, 1, s));
  unsigned st = 0;
  CUDA_TRY(cudaMemcpyAsync(&st, status, sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaFreeAsync(status, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  if (st & kStatusTimeout) return fail(IJ_ERR_TIMEOUT, "tensor-core completion wait timed out");
  return IJ_OK;
}

}  // extern "C"
