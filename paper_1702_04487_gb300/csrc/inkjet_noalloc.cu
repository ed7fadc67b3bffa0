// ij_step_noalloc: one time step of one lattice between caller-owned device
// buffers, with no device allocation.
//
// Who needs it: a caller that may not allocate device memory at the point
// where it steps the lattice -- for example a plugin living inside another
// framework that owns every byte of the device through its own pool, or a
// solver loop that must keep a fixed memory footprint (no allocator calls,
// whose latency and fragmentation it cannot bound).  ij_create would
// allocate the lattice, its descriptors and its diagnostics scratch; this
// entry point takes the populations from the caller and keeps everything
// else in a fixed file-scope device array.
//
// The array below is sized for one lattice of at most kMaxRows rows and
// kMaxItems work items; every GPU that loads the library holds it (about
// 0.7 MB) until the process exits.  All calls on a device share it and it
// keeps the last call's contents, so each call clears the parts that must
// start at zero, and calls whose GPU work overlaps (for example on two
// streams) race on it.
//
// Host side: the descriptor and the work list are built in static host
// buffers under one mutex and handed to cudaMemcpyAsync, which has consumed
// a pageable source by the time it returns; so no host heap is touched
// either, and concurrent host threads serialise on the mutex.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "inkjet.h"
#include "lbm2d.cuh"

namespace {

using namespace ij;

constexpr int kMaxRows = 8192;
constexpr int kMaxItems = 16384;
constexpr int kChunk = 64;  // rows per work item, as in ij_create
constexpr int kMaxDevices = 64;

constexpr size_t a256(size_t v) { return (v + 255) & ~(size_t)255; }
constexpr size_t kOffInst = 0;
constexpr size_t kOffItems = kOffInst + a256(sizeof(Inst));
constexpr size_t kOffT = kOffItems + a256((size_t)kMaxItems * sizeof(Item));
constexpr size_t kOffStatus = kOffT + 256;
constexpr size_t kOffRows = kOffStatus + 256;
constexpr size_t kOffSums = kOffRows + a256(3 * (size_t)kMaxRows * sizeof(double));
constexpr size_t kOffDstate = kOffSums + 256;
constexpr size_t kOffHist = kOffDstate + 256;
constexpr size_t kScratchBytes = kOffHist + a256(kRec * sizeof(double));

// Descriptor, work list, time, numeric flag and FP64 diagnostics scratch.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;                          // guards g_base and the staging below
unsigned char* g_base[kMaxDevices] = {};  // device address of g_scratch per device
Item g_items[kMaxItems];                  // host staging of the work list (static, no heap)

// Device address of g_scratch on the current device, looked up once per
// device (the host-side name of the array is not a device address).  The
// caller holds g_mu.  A stream that belongs to another device is refused:
// its kernels would run there against this device's scratch address.
ij_status scratch_base(cudaStream_t stream, unsigned char** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return report(IJ_ERR_CUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return report(IJ_ERR_CUDA, "device ordinal out of range");
  if (stream) {
    int sdev = -1;
    e = cudaStreamGetDevice(stream, &sdev);
    if (e != cudaSuccess) return report(IJ_ERR_CUDA, cudaGetErrorString(e));
    if (sdev != dev)
      return report(IJ_ERR_PARAM,
                    "ij_step_noalloc: the stream belongs to another device; make that device "
                    "current first");
  }
  if (!g_base[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) return report(IJ_ERR_CUDA, "cudaGetSymbolAddress of the scratch failed");
    e = set_step_smem_limit();
    if (e != cudaSuccess) return report(IJ_ERR_CUDA, cudaGetErrorString(e));
    g_base[dev] = static_cast<unsigned char*>(p);
  }
  *out = g_base[dev];
  return IJ_OK;
}

}  // namespace

extern "C" ij_status ij_step_noalloc(const ij_params* params, long long t, const float* f_in,
                                     const float* g_in, float* f_out, float* g_out,
                                     double* record_out, unsigned* status_out, void* stream) {
  if (!params || !f_in || !g_in || !f_out || !g_out)
    return report(IJ_ERR_PARAM, "ij_step_noalloc: params and the four population buffers are required");
  if (t < 0) return report(IJ_ERR_PARAM, "ij_step_noalloc: t < 0");
  if (f_in == f_out || g_in == g_out)
    return report(IJ_ERR_PARAM, "ij_step_noalloc: input and output buffers must differ");
  ij_status st = validate_params(*params, 0);
  if (st != IJ_OK) return st;
  const ij_params& p = *params;
  if (p.dim == 3) return report(IJ_ERR_PARAM, "ij_step_noalloc: 2-D lattices only");
  if (p.precision != IJ_FP32)
    return report(IJ_ERR_PARAM, "ij_step_noalloc: FP32 storage only");
  if (p.ny > kMaxRows)
    return report(IJ_ERR_PARAM, "ij_step_noalloc: ny exceeds the fixed scratch limit of 8192 rows");
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  std::lock_guard<std::mutex> lock(g_mu);
  // work list: the same strips and row chunks ij_create builds for one lattice
  Inst I = derive_params(p);
  const int n_items = make_items(I, 0, kChunk, g_items, kMaxItems);
  if (n_items < 0)
    return report(IJ_ERR_PARAM, "ij_step_noalloc: lattice needs more than the fixed 16384 work items");
  unsigned char* base = nullptr;
  st = scratch_base(s, &base);
  if (st != IJ_OK) return st;

  I.f[t & 1] = const_cast<float*>(f_in);
  I.g[t & 1] = const_cast<float*>(g_in);
  I.f[(t + 1) & 1] = f_out;
  I.g[(t + 1) & 1] = g_out;
  I.rows = reinterpret_cast<double*>(base + kOffRows);
  I.sums = reinterpret_cast<double*>(base + kOffSums);
  I.hist = reinterpret_cast<double*>(base + kOffHist);
  I.dstate = reinterpret_cast<double*>(base + kOffDstate);
  I.status = reinterpret_cast<unsigned*>(base + kOffStatus);
  const Inst* d_inst = reinterpret_cast<const Inst*>(base + kOffInst);
  const Item* d_items = reinterpret_cast<const Item*>(base + kOffItems);
  long long* d_t = reinterpret_cast<long long*>(base + kOffT);
  const double dinit[8] = {0, 0, 0, -1, 0, 0, 0, 0};
  const bool diag = record_out != nullptr;
#define NOALLOC_TRY(expr)                                              \
  do {                                                                 \
    cudaError_t e_ = (expr);                                           \
    if (e_ != cudaSuccess) return report(IJ_ERR_CUDA, cudaGetErrorString(e_)); \
  } while (0)
  NOALLOC_TRY(cudaMemcpyAsync(base + kOffInst, &I, sizeof(Inst), cudaMemcpyHostToDevice, s));
  NOALLOC_TRY(cudaMemcpyAsync(base + kOffItems, g_items, (size_t)n_items * sizeof(Item),
                              cudaMemcpyHostToDevice, s));
  NOALLOC_TRY(cudaMemcpyAsync(d_t, &t, sizeof(long long), cudaMemcpyHostToDevice, s));
  // what must start at zero: the numeric flag, and for a record the row and
  // lattice sums and the breakup state of the previous call
  NOALLOC_TRY(cudaMemsetAsync(base + kOffStatus, 0, sizeof(unsigned), s));
  if (diag) {
    NOALLOC_TRY(cudaMemsetAsync(base + kOffRows, 0, 3 * (size_t)p.ny * sizeof(double), s));
    NOALLOC_TRY(cudaMemsetAsync(base + kOffSums, 0, 4 * sizeof(double), s));
    NOALLOC_TRY(cudaMemcpyAsync(base + kOffDstate, dinit, sizeof(dinit), cudaMemcpyHostToDevice, s));
  }
  NOALLOC_TRY(launch_step(d_inst, d_items, n_items, kStepThreads,
                          (n_items + kStepThreads / 32 - 1) / (kStepThreads / 32), d_t, 0, diag,
                          step_prefetch_for(kStepThreads), false, p.nx % 2 != 0, s));
  if (diag) {
    NOALLOC_TRY(launch_finalize(d_inst, 1, d_t, s));
    NOALLOC_TRY(cudaMemcpyAsync(record_out, base + kOffHist, kRec * sizeof(double),
                                cudaMemcpyDeviceToDevice, s));
  }
  // the step kernel stops writing a lattice once its flag is set, so the
  // caller must learn of it to discard a partly written output
  if (status_out)
    NOALLOC_TRY(cudaMemcpyAsync(status_out, base + kOffStatus, sizeof(unsigned),
                                cudaMemcpyDeviceToDevice, s));
#undef NOALLOC_TRY
  return IJ_OK;
}
