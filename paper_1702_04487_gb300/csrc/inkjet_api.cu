// Host side of libinkjet.so: parameter validation and derivation, device
// memory, work lists and launches of the 2-D step (include/inkjet.h).
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "inkjet.h"
#include "lbm2d.cuh"
#include "lbm3d.cuh"

namespace ij {
cudaError_t set_step_smem_limit();
}

using namespace ij;

namespace {

thread_local char g_err[512] = "";

ij_status fail(ij_status st, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return st;
}

#define CUDA_TRY(expr)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess) return fail(IJ_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

// Contact angle -> wetting potential Omega by bisection on Cahn's relation
// cos(theta) = ((1 + Omega)^1.5 - (1 - Omega)^1.5) / 2, Omega in [-1, 1].
double omega_from_theta(double theta_deg) {
  const double target = cos(theta_deg * M_PI / 180.0);
  double lo = -1.0, hi = 1.0;
  for (int it = 0; it < 200; it++) {
    double mid = 0.5 * (lo + hi);
    double v = 0.5 * (pow(1.0 + mid, 1.5) - pow(1.0 - mid, 1.5));
    if (v < target) lo = mid; else hi = mid;
  }
  double om = 0.5 * (lo + hi);
  if (fabs(theta_deg - 90.0) == 0.0) om = 0.0;
  return om;
}

// Lattices launched together: same block size; rows split into chunks of
// `chunk`, populations staged `prefetch` rows ahead.
struct Bucket {
  int nthreads;
  int first, count;  // range in the item array
  int grid;
  int chunk, prefetch;
};

}  // namespace

struct ij_handle_s {
  int n_inst = 0;
  // 3-D handles: per-lattice descriptors; `inst` then holds each lattice's
  // diagnostics descriptor over its z planes (ny = nz) for the shared
  // record kernel and the observation calls
  bool is3d = false;
  bool fp16 = false;  // 2-D lattices in FP16 storage
  bool odd = false;   // some 2-D lattice has an odd nx (column-by-column copies)
  std::vector<Inst3> inst3;
  Inst3* d_inst3 = nullptr;
  std::vector<Item3> items3;  // work items of the 3-D step (all lattices)
  Item3* d_items3 = nullptr;
  size_t items3_cap = 0;
  float* stage = nullptr;  // FP32 staging of exported / imported states (3-D, 2-D FP16)
  size_t stage_floats = 0;
  std::vector<ij_params> params;
  std::vector<Inst> inst;
  std::vector<Item> items;
  std::vector<Bucket> buckets;
  size_t items_cap = 0;  // capacity of d_items
  Inst* d_inst = nullptr;
  Item* d_items = nullptr;
  long long* d_t = nullptr;
  unsigned* d_status = nullptr;  // [n_inst] numeric flags, one per lattice
  unsigned* h_status = nullptr;  // pinned mirror, refreshed after each ij_step
  long long t = 0;
  long long launches = 0;
  int diag_every = 0;
  bool poisoned = false;
  cudaStream_t stream = nullptr;
  ij_alloc_fn alloc = nullptr;
  ij_free_fn free_fn = nullptr;
  void* ctx = nullptr;
  std::vector<void*> blocks;
  // CUDA graph of one diagnostics period (diag_every steps, or 16); the
  // diagnostics record runs on a branch (cap_stream2) beside the next steps
  cudaStream_t cap_stream = nullptr, cap_stream2 = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int graph_steps = 0;
  long long graph_launches = 0;  // kernels per graph launch
  bool use_graph = true;
  void drop_graph() {
    if (gexec) cudaGraphExecDestroy(gexec);
    gexec = nullptr;
  }
  // optional CUDA-event timing of the step-kernel launches
  bool timing = false;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
  double timed_ms = 0.0;
  long long timed_launches = 0;
  cudaEvent_t get_event() {
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  void drain_events() {
    for (auto& pr : events) {
      float ms = 0.0f;
      if (cudaEventSynchronize(pr.second) == cudaSuccess &&
          cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess)
        timed_ms += ms;
      cudaEventDestroy(pr.first);
      cudaEventDestroy(pr.second);
    }
    events.clear();
  }

  void* dalloc(size_t bytes) {
    bytes = (bytes + 255) & ~(size_t)255;
    void* p = nullptr;
    if (alloc) {
      p = alloc(bytes, ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
      p = nullptr;
    }
    if (p) blocks.push_back(p);
    return p;
  }
  void release() {
    if (stream) cudaStreamSynchronize(stream); else cudaDeviceSynchronize();
    drain_events();
    drop_graph();
    if (cap_stream) cudaStreamDestroy(cap_stream);
    if (cap_stream2) cudaStreamDestroy(cap_stream2);
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    cap_stream = cap_stream2 = nullptr;
    ev_fork = ev_join = nullptr;
    for (void* p : blocks) {
      if (free_fn) free_fn(p, ctx); else cudaFree(p);
    }
    blocks.clear();
    if (h_status) cudaFreeHost(h_status);
    h_status = nullptr;
  }
};

static_assert(sizeof(ij_obs) == kRec * sizeof(double), "ij_obs is one diagnostics record");

namespace {

ij_status validate(const ij_params& p, int k) {
  if (p.nx < 1 || p.ny < 1) return fail(IJ_ERR_PARAM, "lattice %d: nx, ny must be >= 1", k);
  if ((long long)p.nx * p.ny > (1LL << 31) / 9)
    return fail(IJ_ERR_PARAM, "lattice %d: nx*ny too large for 32-bit plane indexing", k);
  if (!(p.rho_ink > p.rho_air) || !(p.rho_air > 0))
    return fail(IJ_ERR_PARAM, "lattice %d: need rho_ink > rho_air > 0", k);
  if (!(p.sigma > 0) || !(p.width_W > 0) || !(p.tau_phi > 0))
    return fail(IJ_ERR_PARAM, "lattice %d: sigma, width_W, tau_phi must be > 0", k);
  if (!(p.nu_ink > 0) || !(p.nu_air > 0))
    return fail(IJ_ERR_PARAM, "lattice %d: viscosities must be > 0", k);
  if (!(p.theta_deg >= 0 && p.theta_deg <= 180))
    return fail(IJ_ERR_PARAM, "lattice %d: theta_deg must be in [0, 180]", k);
  if (p.geometry < 0 || p.geometry > 2) return fail(IJ_ERR_PARAM, "lattice %d: bad geometry", k);
  if (p.axial_bc < 0 || p.axial_bc > 2) return fail(IJ_ERR_PARAM, "lattice %d: bad axial_bc", k);
  if (p.init_kind < 0 || p.init_kind > 3) return fail(IJ_ERR_PARAM, "lattice %d: bad init_kind", k);
  const int dim = p.dim == 0 ? 2 : p.dim;
  if (dim != 2 && dim != 3) return fail(IJ_ERR_PARAM, "lattice %d: dim must be 2 or 3", k);
  if (p.precision != IJ_FP32 && p.precision != IJ_FP16_STORE)
    return fail(IJ_ERR_PARAM, "lattice %d: precision must be IJ_FP32 or IJ_FP16_STORE", k);
  if (dim == 2 && p.precision == IJ_FP16_STORE && p.nx % 2 != 0)
    return fail(IJ_ERR_PARAM, "lattice %d: 2-D FP16 storage needs an even nx", k);
  if (dim == 3) {
    if (p.nz < 1) return fail(IJ_ERR_PARAM, "lattice %d: nz must be >= 1", k);
    if (p.precision == IJ_FP16_STORE && p.nx % 2 != 0)
      return fail(IJ_ERR_PARAM, "lattice %d: 3-D FP16 storage needs an even nx", k);
    if (p.nz > 65533 || p.ny > 262140)  // grid limits of the 32 x 4 x 1 blocks
      return fail(IJ_ERR_PARAM, "lattice %d: nz must be <= 65533 and ny <= 262140", k);
    if ((long long)p.nx * p.ny * p.nz > (1LL << 31) / 19)
      return fail(IJ_ERR_PARAM, "lattice %d: nx*ny*nz too large", k);
    if (p.geometry == IJ_GEOM_NOZZLE &&
        (p.nozzle_width < 1 || p.wall_thickness < 1 || p.nozzle_length < 0 ||
         2 * (p.nozzle_width + p.wall_thickness) + 4 > std::min(p.nx, p.ny)))
      return fail(IJ_ERR_PARAM, "lattice %d: round nozzle (radius + wall, plus 2 cells) must fit in nx, ny", k);
    if (p.geometry == IJ_GEOM_PLATE && (p.wall_thickness < 1 || p.wall_thickness >= p.nz))
      return fail(IJ_ERR_PARAM, "lattice %d: plate thickness must be in [1, nz)", k);
  }
  if (p.T1 < 0 || p.T2 < 0 || p.T_idle < 0) return fail(IJ_ERR_PARAM, "lattice %d: negative durations", k);
  if (p.diag_every < 0) return fail(IJ_ERR_PARAM, "lattice %d: diag_every < 0", k);
  if (dim == 2 && p.geometry == IJ_GEOM_NOZZLE) {
    if (p.nozzle_width < 1 || p.wall_thickness < 1 || p.nozzle_length < 0 ||
        p.nozzle_width + 2 * p.wall_thickness > p.nx)
      return fail(IJ_ERR_PARAM, "lattice %d: nozzle (width + 2 walls) must fit in nx", k);
  }
  if (dim == 2 && p.geometry == IJ_GEOM_PLATE && (p.wall_thickness < 1 || p.wall_thickness >= p.ny))
    return fail(IJ_ERR_PARAM, "lattice %d: plate thickness must be in [1, ny)", k);
  return IJ_OK;
}

// Derived constants of one lattice (free energy, relaxation, wetting).
Inst derive(const ij_params& p) {
  Inst I;
  memset(&I, 0, sizeof(I));
  I.nx = p.nx;
  I.ny = p.ny;
  I.geom = p.geometry;
  I.cx0 = (p.nx - p.nozzle_width) / 2;
  I.cx1 = I.cx0 + p.nozzle_width;
  I.L = p.nozzle_length;
  I.wt = p.wall_thickness;
  I.bc = p.axial_bc;
  I.init_kind = p.init_kind;
  I.fp16 = (p.dim == 0 || p.dim == 2) && p.precision == IJ_FP16_STORE;
  const double phis = 0.5 * (p.rho_ink - p.rho_air), n0 = 0.5 * (p.rho_ink + p.rho_air);
  const double A = 3.0 * p.sigma / (8.0 * p.width_W * phis * phis * phis * phis);
  const double kappa = 3.0 * p.sigma * p.width_W / (4.0 * phis * phis);
  const double q = 1.0 / (p.tau_phi + 0.5);
  const double gamma = p.gamma > 0 ? p.gamma : 0.04 / kappa;
  const double h = omega_from_theta(p.theta_deg) * phis * phis * sqrt(2.0 * kappa * A);
  I.phis = (float)phis;
  I.inv_phis = (float)(1.0 / phis);
  I.A4 = (float)(4.0 * A);
  I.kappa = (float)kappa;
  I.hk = (float)(h / kappa);
  I.q = (float)q;
  I.omq = 1.0f - I.q;  // exact in FP32 (q in [1/2, 1]), so (1-q) + q == 1 there too
  I.n0 = (float)n0;
  I.inv_tphi = (float)(1.0 / p.tau_phi);
  I.gamma = (float)gamma;
  I.inv2q = (float)(1.0 / (2.0 * q));
  I.nu_air = (float)p.nu_air;
  I.dnu = (float)(p.nu_ink - p.nu_air);
  I.F0 = (float)p.F0;
  I.Fneg = (float)p.F_neg;
  I.T1 = p.T1;
  I.T2 = p.T2;
  I.Tidle = p.T_idle;
  I.d_phis = phis;
  I.d_n0 = n0;
  I.d_A = A;
  I.d_kappa = kappa;
  I.d_h = h;
  I.d_gamma = gamma;
  I.d_q = q;
  I.d_W = p.width_W;
  I.init_x = p.init_x;
  I.init_y = p.init_y;
  I.init_r = p.init_r;
  I.jitter = p.jitter;
  I.seed = p.seed;
  const bool nozzle = p.geometry == IJ_GEOM_NOZZLE;
  I.y_exit = nozzle ? p.nozzle_length : 0;
  I.y_scan = nozzle ? p.nozzle_length - p.nozzle_length / 2 : 0;
  I.vmin = nozzle ? (double)p.nozzle_width : 1.0;
  return I;
}

// Derived constants of one 3-D lattice (same closure as derive()).
Inst3 derive3(const ij_params& p) {
  const Inst I2 = derive(p);
  Inst3 I;
  memset(&I, 0, sizeof(I));
  I.nx = p.nx;
  I.ny = p.ny;
  I.nz = p.nz;
  I.geom = p.geometry;
  I.L = p.nozzle_length;
  I.wt = p.wall_thickness;
  I.bc = p.axial_bc;
  I.fp16 = p.precision == IJ_FP16_STORE;
  I.cx = 0.5f * (p.nx - 1);
  I.cy = 0.5f * (p.ny - 1);
  I.R2 = (float)p.nozzle_width * (float)p.nozzle_width;
  I.Ro2 = (float)(p.nozzle_width + p.wall_thickness) * (float)(p.nozzle_width + p.wall_thickness);
  I.phis = I2.phis;
  I.inv_phis = I2.inv_phis;
  I.A4 = I2.A4;
  I.kappa = I2.kappa;
  I.hk = I2.hk;
  I.q = I2.q;
  I.omq = I2.omq;
  I.inv_tphi = I2.inv_tphi;
  I.gamma = I2.gamma;
  I.inv2q = I2.inv2q;
  I.nu_air = I2.nu_air;
  I.dnu = I2.dnu;
  I.F0 = I2.F0;
  I.Fneg = I2.Fneg;
  I.n0 = I2.n0;
  I.T1 = p.T1;
  I.T2 = p.T2;
  I.Tidle = p.T_idle;
  I.d_phis = I2.d_phis;
  I.d_n0 = I2.d_n0;
  I.d_A = I2.d_A;
  I.d_kappa = I2.d_kappa;
  I.d_h = I2.d_h;
  I.d_gamma = I2.d_gamma;
  I.d_q = I2.d_q;
  I.d_W = I2.d_W;
  I.init_x = p.init_x;
  I.init_y = p.init_y;
  I.init_z = p.init_z;
  I.init_r = p.init_r;
  I.jitter = p.jitter;
  I.init_kind = p.init_kind;
  I.seed = p.seed;
  return I;
}

// Every lattice runs in the one bucket of kStepThreads-thread blocks (one
// warp per work item).
int block_size_for(const Inst&) { return kStepThreads; }

// Rows of one strip that run the wall paths (wetting ghosts, bounce-back):
// rows below the first row whose stencil no longer reaches a solid cell.
int strip_wall_rows(const Inst& I, const Item& it) {
  const int x0 = it.xs - it.halo, x1 = it.xs + it.nout + it.halo;  // columns held
  if (I.geom == GEOM_NOZZLE) {
    // either wall band [cx0 - wt, cx0) or [cx1, cx1 + wt) among them (or a
    // wrapped copy of it)
    for (int sh = -I.nx; sh <= I.nx; sh += I.nx) {
      const int a = x0 + sh, b = x1 + sh;
      if ((b > I.cx0 - I.wt && a < I.cx0) || (b > I.cx1 && a < I.cx1 + I.wt))
        return std::min(I.ny, I.L + 2);
    }
    return 0;
  }
  if (I.geom == GEOM_PLATE) return std::min(I.ny, I.wt + 2);
  return 0;
}

// Cost-balanced work list (chunk <= 0).  The cost of a strip row is 1, or
// 1 + kWallCost for a row that runs the wall paths (measured: a wall-strip
// row takes 2.0-2.2 times a fluid one).  With S the number of work items the
// GPU runs at once (SMs x resident blocks), the body of every strip -- a
// fraction beta of its cost, from its first row -- is cut into pieces of
// equal cost near beta C / S (C the total cost), S pieces in all, so that the
// body is one wave of items that finish together; the rest of each strip
// becomes a tail of short pieces listed after all bodies, which the SMs
// that finish first take up.  Variants: chunk 0 (beta 7/8, tail pieces of a
// sixth of a body piece), -1 (beta 1, no tail), -2 (beta 3/4, tail pieces of
// an eighth), -3 .. -5 (beta 1, pieces for 2 .. 4 full waves).
constexpr double kWallCost = 1.2;

void balanced_items(ij_handle h, const Bucket& b, int slots) {
  const int variant = -b.chunk;
  // variants 3..5: the whole strip in equal pieces making 2..4 full waves
  const int waves = variant >= 3 ? variant - 1 : 1;
  slots *= waves;
  const double beta = variant == 0 ? 0.875 : (variant == 2 ? 0.75 : 1.0);
  const double tail_div = variant == 2 ? 8.0 : 6.0;
  struct Strip { Item it; int wall; double cost; };
  std::vector<Strip> strips;
  double C = 0.0;
  for (int k = 0; k < h->n_inst; k++) {
    const Inst& I = h->inst[k];
    const int n = items_per_range(I, I.ny, 0, I.ny, false);
    const size_t at = h->items.size();
    h->items.resize(at + n);
    make_items_range(I, k, I.ny, 0, I.ny, h->items.data() + at, n, false);
    for (int j = 0; j < n; j++) {
      Strip st;
      st.it = h->items[at + j];
      st.wall = strip_wall_rows(I, st.it);
      st.cost = I.ny + kWallCost * st.wall;
      C += st.cost;
      strips.push_back(st);
    }
    h->items.resize(at);
  }
  const double T = beta * C / std::max(1, slots);  // body piece cost
  // pieces per strip body, summing to exactly `slots` (largest remainders
  // get the extra pieces; at least one per strip): one more item than the
  // GPU holds would wait for a whole piece and double the step
  std::vector<int> nb(strips.size());
  std::vector<std::pair<double, size_t>> rem;
  long long total = 0;
  for (size_t i = 0; i < strips.size(); i++) {
    const double raw = strips[i].cost * slots / C;
    nb[i] = std::max(1, (int)floor(raw));
    total += nb[i];
    rem.push_back({raw - floor(raw), i});
  }
  std::sort(rem.begin(), rem.end(), [](const std::pair<double, size_t>& a,
                                       const std::pair<double, size_t>& b) { return a.first > b.first; });
  for (size_t j = 0; j < rem.size() && total < slots; j++, total++) nb[rem[j].second]++;
  // row at which the cumulative cost of a strip reaches c
  auto row_at = [](const Strip& st, double c) -> int {
    const double cw = (1.0 + kWallCost) * st.wall;
    const double y = c <= cw ? c / (1.0 + kWallCost) : st.wall + (c - cw);
    return std::max(0, std::min(st.it.ch, (int)lround(y)));
  };
  std::vector<Item> tail;
  // body pieces, listed round-robin over the strips (piece j of every strip,
  // then piece j + 1), so that each wave spans every strip
  std::vector<std::vector<Item>> pieces(strips.size());
  int max_pieces = 0;
  for (size_t i = 0; i < strips.size(); i++) {
    const Strip& st = strips[i];
    const double body = beta * st.cost;
    const int yb = beta >= 1.0 ? st.it.ch : std::max(1, row_at(st, body));
    int y = 0;
    for (int j = 1; j <= nb[i] && y < yb; j++) {
      const int ye = j == nb[i] ? yb : std::min(yb, std::max(y + 1, row_at(st, body * j / nb[i])));
      Item it = st.it;
      it.y0 = y;
      it.ch = ye - y;
      pieces[i].push_back(it);
      y = ye;
    }
    max_pieces = std::max(max_pieces, (int)pieces[i].size());
    const int tn = std::max(4, (int)lround(T / tail_div));  // rows per tail piece
    for (; y < st.it.ch; y += tn) {
      Item it = st.it;
      it.y0 = y;
      it.ch = std::min(tn, st.it.ch - y);
      tail.push_back(it);
    }
  }
  for (int j = 0; j < max_pieces; j++)
    for (size_t i = 0; i < strips.size(); i++)
      if (j < (int)pieces[i].size()) h->items.push_back(pieces[i][j]);
  h->items.insert(h->items.end(), tail.begin(), tail.end());
}

void build_items(ij_handle h) {
  std::vector<Bucket> old = h->buckets;
  h->items.clear();
  h->buckets.clear();
  Bucket b{kStepThreads, 0, 0, 0, 0, step_prefetch_for(kStepThreads)};
  for (const Bucket& o : old)
    if (o.nthreads == kStepThreads) {
      b.chunk = o.chunk;
      b.prefetch = o.prefetch;
    }
  if (b.chunk <= 0) {
    balanced_items(h, b, step_slots(b.prefetch, h->fp16, h->odd));
  } else {
    // The last eighth of every lattice's rows is cut into chunks a quarter as
    // long, and those items go last: the final wave of blocks is made of short
    // items, so SMs run out of work together.
    const int tail_chunk = std::max(4, b.chunk / 4);
    size_t n_body = 0;  // items before the tail
    for (int pass = 0; pass < 2; pass++) {
      if (pass == 1) n_body = h->items.size();
      for (int k = 0; k < h->n_inst; k++) {
        const Inst& I = h->inst[k];
        const int split = I.ny - I.ny / 8;
        const int ya = pass == 0 ? 0 : split, yb = pass == 0 ? split : I.ny;
        const int ch = pass == 0 ? b.chunk : tail_chunk;
        const int n = items_per_range(I, ch, ya, yb, true);
        const size_t at = h->items.size();
        h->items.resize(at + n);
        make_items_range(I, k, ch, ya, yb, h->items.data() + at, n, true);
      }
    }
    // Items of nozzle-wall strips below the nozzle exit cost more per row
    // (wetting ghosts, bounce-back): they go first, cut into chunks a quarter
    // as long, so that no SM is left with a long one of them at the end.
    auto costly = [&](const Item& it) {
      const Inst& I = h->inst[it.inst];
      if (it.half || I.geom != GEOM_NOZZLE || it.y0 > I.L + 1) return false;
      const int x0 = it.xs - it.halo, x1 = it.xs + it.nout + it.halo;  // columns held
      // either wall band [cx0 - wt, cx0) or [cx1, cx1 + wt) among them
      return (x1 > I.cx0 - I.wt && x0 < I.cx0) || (x1 > I.cx1 && x0 < I.cx1 + I.wt);
    };
    const size_t n_costly =
        std::stable_partition(h->items.begin(), h->items.begin() + n_body, costly) -
        h->items.begin();
    if (n_costly > 0) {
      std::vector<Item> split;
      for (size_t i = 0; i < n_costly; i++) {
        const Item& it = h->items[i];
        for (int y = it.y0; y < it.y0 + it.ch; y += tail_chunk) {
          Item c = it;
          c.y0 = y;
          c.ch = std::min(tail_chunk, it.y0 + it.ch - y);
          split.push_back(c);
        }
      }
      split.insert(split.end(), h->items.begin() + n_costly, h->items.end());
      h->items.swap(split);
    }
  }
  b.count = (int)h->items.size();
  // one block per item: the block scheduler hands new blocks to SMs as
  // they free up (measured faster than blocks of several items, which hold
  // their slot until the slowest finishes, and than a persistent grid)
  b.grid = (b.count + kStepThreads / 32 - 1) / (kStepThreads / 32);
  h->buckets.push_back(b);
}

// Upload the work list, growing the device copy when needed (the captured
// graph bakes the list in, so it is rebuilt on the next ij_step).
ij_status upload_items(ij_handle h) {
  h->drop_graph();
  if (h->items.size() > h->items_cap) {
    Item* p = (Item*)h->dalloc(h->items.size() * sizeof(Item));
    if (!p) return fail(IJ_ERR_OOM, "device allocation of the work list failed");
    h->d_items = p;  // the old list stays owned by the handle until destroy
    h->items_cap = h->items.size();
  }
  cudaError_t e = cudaMemcpyAsync(h->d_items, h->items.data(), h->items.size() * sizeof(Item),
                                  cudaMemcpyHostToDevice, h->stream);
  if (e != cudaSuccess) return fail(IJ_ERR_CUDA, "work list upload: %s", cudaGetErrorString(e));
  return IJ_OK;
}

ij_status check_handle(ij_handle h) {
  if (!h) return fail(IJ_ERR_PARAM, "null handle");
  return IJ_OK;
}

// One 3-D time step on stream s (time d_t[0] + t_off): the fused step of
// every lattice (with plane sums when diag), the wetting ghosts of the new
// phi, the flip of the current buffers.  The diagnostics record is the
// caller's.
cudaError_t enqueue_step3(ij_handle h, cudaStream_t s, int t_off, bool diag, long long* n) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (h->timing) {
    e0 = h->get_event();
    e1 = h->get_event();
    cudaEventRecord(e0, s);
  }
  cudaError_t e = launch_step3(h->d_inst3, h->d_items3, (int)h->items3.size(), h->n_inst, h->d_t,
                               t_off, diag, h->fp16, s);
  (*n)++;
  if (h->timing) {
    cudaEventRecord(e1, s);
    h->events.push_back({e0, e1});
    h->timed_launches++;
  }
  if (e != cudaSuccess) return e;
  e = launch_ghost3(h->d_inst3, h->inst3.data(), h->n_inst, true, s);
  (*n)++;
  if (e != cudaSuccess) return e;
  e = launch_flip3(h->d_inst3, h->n_inst, s);
  (*n)++;
  return e;
}

ij_status one_step(ij_handle h) {
  const bool diag = h->diag_every > 0 && h->t % h->diag_every == 0;
  if (h->is3d) {
    long long n = 0;
    CUDA_TRY(enqueue_step3(h, h->stream, 0, diag, &n));
    h->launches += n;
    if (diag) {
      CUDA_TRY(launch_finalize(h->d_inst, h->n_inst, h->d_t, h->stream));
      h->launches++;
    }
    CUDA_TRY(launch_advance(h->d_t, 1, h->stream));
    h->launches++;
    h->t++;
    return IJ_OK;
  }
  for (const Bucket& b : h->buckets) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (h->timing) {
      e0 = h->get_event();
      e1 = h->get_event();
      CUDA_TRY(cudaEventRecord(e0, h->stream));
    }
    CUDA_TRY(launch_step(h->d_inst, h->d_items + b.first, b.count, b.nthreads, b.grid, h->d_t, 0,
                         diag, b.prefetch, h->fp16, h->odd, h->stream));
    h->launches++;
    if (h->timing) {
      CUDA_TRY(cudaEventRecord(e1, h->stream));
      h->events.push_back({e0, e1});
      h->timed_launches++;
    }
  }
  if (diag) {
    CUDA_TRY(launch_finalize(h->d_inst, h->n_inst, h->d_t, h->stream));
    h->launches++;
  }
  CUDA_TRY(launch_advance(h->d_t, 1, h->stream));
  h->launches++;
  h->t++;
  return IJ_OK;
}

// Capture one diagnostics period into a graph: the step kernels of every
// bucket with time offsets 0..P-1 (offset 0 with diagnostics when enabled),
// the record kernel after the first step, and one advance of the time by P.
// The record kernel runs on a branch of its own beside steps 1..P-1: it
// reads only the FP64 row and lattice sums of step 0 (and resets them) and
// the time, which those steps do not touch; the branch joins before the
// advance of the time.
ij_status build_graph(ij_handle h) {
  h->drop_graph();
  const int P = h->diag_every > 0 ? h->diag_every : 16;
  if (!h->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&h->cap_stream, cudaStreamNonBlocking));
  if (!h->cap_stream2) CUDA_TRY(cudaStreamCreateWithFlags(&h->cap_stream2, cudaStreamNonBlocking));
  if (!h->ev_fork) CUDA_TRY(cudaEventCreateWithFlags(&h->ev_fork, cudaEventDisableTiming));
  if (!h->ev_join) CUDA_TRY(cudaEventCreateWithFlags(&h->ev_join, cudaEventDisableTiming));
  cudaStream_t cs = h->cap_stream;
  bool branched = false;
  CUDA_TRY(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  long long n = 0;
  cudaError_t e = cudaSuccess;
  for (int j = 0; j < P && e == cudaSuccess; j++) {
    const bool diag = h->diag_every > 0 && j == 0;
    if (h->is3d) {
      e = enqueue_step3(h, cs, j, diag, &n);
    } else {
      for (const Bucket& b : h->buckets) {
        e = launch_step(h->d_inst, h->d_items + b.first, b.count, b.nthreads, b.grid, h->d_t, j,
                        diag, b.prefetch, h->fp16, h->odd, cs);
        n++;
        if (e != cudaSuccess) break;
      }
    }
    if (diag && e == cudaSuccess) {
      e = cudaEventRecord(h->ev_fork, cs);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(h->cap_stream2, h->ev_fork, 0);
      if (e == cudaSuccess) e = launch_finalize(h->d_inst, h->n_inst, h->d_t, h->cap_stream2);
      if (e == cudaSuccess) e = cudaEventRecord(h->ev_join, h->cap_stream2);
      branched = e == cudaSuccess;
      n++;
    }
  }
  if (branched && e == cudaSuccess) e = cudaStreamWaitEvent(cs, h->ev_join, 0);
  if (e == cudaSuccess) {
    e = launch_advance(h->d_t, P, cs);
    n++;
  }
  cudaGraph_t g = nullptr;
  cudaError_t e2 = cudaStreamEndCapture(cs, &g);
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(IJ_ERR_CUDA, "graph capture: %s", cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&h->gexec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) return fail(IJ_ERR_CUDA, "graph instantiate: %s", cudaGetErrorString(e));
  h->graph_steps = P;
  h->graph_launches = n;
  return IJ_OK;
}

// Work items of the 3-D step and their upload (the device array grows only).
ij_status upload_items3(ij_handle h) {
  const int n = make_items3(h->inst3.data(), h->n_inst, h->buckets[0].chunk, nullptr);
  h->items3.resize(n);
  make_items3(h->inst3.data(), h->n_inst, h->buckets[0].chunk, h->items3.data());
  if ((size_t)n > h->items3_cap) {
    h->d_items3 = (Item3*)h->dalloc(n * sizeof(Item3));
    if (!h->d_items3) return fail(IJ_ERR_OOM, "device allocation of 3-D work items failed");
    h->items3_cap = n;
  }
  Bucket& b = h->buckets[0];
  b.count = n;
  CUDA_TRY(cudaMemcpyAsync(h->d_items3, h->items3.data(), n * sizeof(Item3), cudaMemcpyHostToDevice,
                           h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  h->drop_graph();
  return IJ_OK;
}

constexpr int kChunk3Default = 80;  // planes of a 3-D work item before tuning

// Allocate and initialise the lattices of a 3-D handle: per lattice two
// state buffers (f, g_1..6 in the storage format, g_0 and phi with its
// wetting ghosts in FP32), the list of ghost cells, the diagnostics over z
// planes.
ij_status create3(ij_handle h) {
  const int count = h->n_inst;
  h->is3d = true;
  for (int k = 1; k < count; k++)
    if (h->params[k].precision != h->params[0].precision)
      return fail(IJ_ERR_PARAM, "all 3-D lattices of a batch must share the precision");
  h->fp16 = h->params[0].precision == IJ_FP16_STORE;
  cudaError_t e3 = set_step3_smem_limit();
  if (e3 != cudaSuccess) return fail(IJ_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e3));
  h->inst3.resize(count);
  h->inst.resize(count);
  std::vector<int> ghosts;
  for (int k = 0; k < count; k++) {
    const ij_params& p = h->params[k];
    Inst3 I = derive3(p);
    const size_t N = (size_t)p.nx * p.ny * p.nz, NE = (size_t)p.nx * p.ny * (p.nz + 4);
    const size_t es = I.fp16 ? 2 : 4;
    for (int b = 0; b < 2; b++) {
      // f of one buffer is also the FP64 scratch of the initial phi
      I.f[b] = h->dalloc(std::max(19 * N * es, N * sizeof(double)));
      I.g[b] = h->dalloc(6 * N * es);
      I.g0[b] = (float*)h->dalloc(N * sizeof(float));
      I.phi[b] = (float*)h->dalloc(NE * sizeof(float));
      if (!I.f[b] || !I.g[b] || !I.g0[b] || !I.phi[b])
        return fail(IJ_ERR_OOM, "device allocation of 3-D lattice %d failed", k);
    }
    I.n_ghost = ghost_cells3(I, nullptr);
    ghosts.resize(std::max(1, I.n_ghost));
    ghost_cells3(I, ghosts.data());
    I.ghost = (int*)h->dalloc(ghosts.size() * sizeof(int));
    if (!I.ghost) return fail(IJ_ERR_OOM, "device allocation of 3-D lattice %d failed", k);
    CUDA_TRY(cudaMemcpyAsync(I.ghost, ghosts.data(), ghosts.size() * sizeof(int),
                             cudaMemcpyHostToDevice, h->stream));
    CUDA_TRY(cudaStreamSynchronize(h->stream));  // ghosts is reused
    // the step never stores solid cells: they hold 0 in both buffers
    for (int b = 0; b < 2; b++) {
      CUDA_TRY(cudaMemsetAsync(I.f[b], 0, std::max(19 * N * es, N * sizeof(double)), h->stream));
      CUDA_TRY(cudaMemsetAsync(I.g[b], 0, 6 * N * es, h->stream));
      CUDA_TRY(cudaMemsetAsync(I.g0[b], 0, N * sizeof(float), h->stream));
      CUDA_TRY(cudaMemsetAsync(I.phi[b], 0, NE * sizeof(float), h->stream));
    }
    // diagnostics over z planes, in the 2-D descriptor the record kernel reads
    Inst D;
    memset(&D, 0, sizeof(D));
    D.nx = p.nx;
    D.ny = p.nz;
    const bool nozzle = p.geometry == IJ_GEOM_NOZZLE;
    D.y_exit = nozzle ? p.nozzle_length : 0;
    D.y_scan = nozzle ? p.nozzle_length - p.nozzle_length / 2 : 0;
    D.vmin = nozzle ? M_PI * p.nozzle_width * p.nozzle_width : 1.0;
    D.rows = (double*)h->dalloc(3 * (size_t)p.nz * sizeof(double));
    D.sums = (double*)h->dalloc(4 * sizeof(double));
    D.hist = (double*)h->dalloc((size_t)kHistCap * kRec * sizeof(double));
    D.dstate = (double*)h->dalloc(8 * sizeof(double));
    if (!D.rows || !D.sums || !D.hist || !D.dstate)
      return fail(IJ_ERR_OOM, "device allocation of 3-D lattice %d failed", k);
    I.rows = D.rows;
    I.sums = D.sums;
    h->inst3[k] = I;
    h->inst[k] = D;
  }
  h->d_inst3 = (Inst3*)h->dalloc(count * sizeof(Inst3));
  h->d_inst = (Inst*)h->dalloc(count * sizeof(Inst));
  h->d_t = (long long*)h->dalloc(sizeof(long long));
  h->d_status = (unsigned*)h->dalloc(count * sizeof(unsigned));
  int* d_cur = (int*)h->dalloc(count * sizeof(int));
  if (!h->d_inst3 || !h->d_inst || !h->d_t || !h->d_status || !d_cur)
    return fail(IJ_ERR_OOM, "device allocation of descriptors failed");
  for (int k = 0; k < count; k++) {
    h->inst3[k].status = h->inst[k].status = h->d_status + k;
    h->inst3[k].cur = d_cur + k;
  }
  if (cudaMallocHost((void**)&h->h_status, count * sizeof(unsigned)) != cudaSuccess)
    return fail(IJ_ERR_OOM, "pinned allocation failed");
  memset(h->h_status, 0, count * sizeof(unsigned));
  int dev = 0, sms = 1;
  CUDA_TRY(cudaGetDevice(&dev));
  CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  h->buckets.assign(1, Bucket{kStep3Threads, 0, 0, sms, kChunk3Default, 1});
  ij_status st = upload_items3(h);
  if (st != IJ_OK) return st;
  cudaStream_t s = h->stream;
  CUDA_TRY(cudaMemcpyAsync(h->d_inst3, h->inst3.data(), count * sizeof(Inst3), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(h->d_inst, h->inst.data(), count * sizeof(Inst), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemsetAsync(h->d_t, 0, sizeof(long long), s));
  CUDA_TRY(cudaMemsetAsync(h->d_status, 0, count * sizeof(unsigned), s));
  CUDA_TRY(cudaMemsetAsync(d_cur, 0, count * sizeof(int), s));
  const double dinit[8] = {0, 0, 0, -1, 0, 0, 0, 0};
  for (int k = 0; k < count; k++) {
    const Inst& D = h->inst[k];
    CUDA_TRY(cudaMemsetAsync(D.rows, 0, 3 * (size_t)D.ny * sizeof(double), s));
    CUDA_TRY(cudaMemsetAsync(D.sums, 0, 4 * sizeof(double), s));
    CUDA_TRY(cudaMemsetAsync(D.hist, 0, (size_t)kHistCap * kRec * sizeof(double), s));
    CUDA_TRY(cudaMemcpyAsync(D.dstate, dinit, sizeof(dinit), cudaMemcpyHostToDevice, s));
    CUDA_TRY(launch_init3(h->d_inst3, h->inst3[k], k, s));
    h->launches += 3;
    // the other buffer's f held the FP64 initial phi: clear it again
    const Inst3& J = h->inst3[k];
    const size_t N = (size_t)J.nx * J.ny * J.nz;
    CUDA_TRY(cudaMemsetAsync(J.f[1], 0, std::max(19 * N * (J.fp16 ? 2 : 4), N * sizeof(double)), s));
  }
  CUDA_TRY(cudaStreamSynchronize(s));
  return IJ_OK;
}

// FP32 staging buffer for exporting / importing a lattice's state (3-D, 2-D FP16).
ij_status ensure_stage(ij_handle h, size_t floats) {
  if (h->stage_floats >= floats) return IJ_OK;
  h->stage = (float*)h->dalloc(floats * sizeof(float));
  if (!h->stage) return fail(IJ_ERR_OOM, "device allocation of the staging buffer failed");
  h->stage_floats = floats;
  return IJ_OK;
}

// Absolute FP32 populations of a 3-D lattice: f [19][N], g [7][N].
ij_status get_state3(ij_handle h, int index, float* f, float* g, int on_device) {
  const Inst3& J = h->inst3[index];
  const size_t N = (size_t)J.nx * J.ny * J.nz;
  ij_status st = ensure_stage(h, 26 * N);
  if (st != IJ_OK) return st;
  CUDA_TRY(launch_export3(h->d_inst3, J, index, h->stage, h->stage + 19 * N, h->stream));
  h->launches++;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (f) CUDA_TRY(cudaMemcpyAsync(f, h->stage, 19 * N * sizeof(float), kind, h->stream));
  if (g) CUDA_TRY(cudaMemcpyAsync(g, h->stage + 19 * N, 7 * N * sizeof(float), kind, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return IJ_OK;
}

// Each 3-D lattice keeps its own current-buffer index, so setting one
// lattice's state and time needs no move of the others' state.
ij_status set_state3(ij_handle h, int index, const float* f, const float* g, long long t,
                     int on_device) {
  const Inst3& J = h->inst3[index];
  const size_t N = (size_t)J.nx * J.ny * J.nz;
  ij_status st = ensure_stage(h, 26 * N);
  if (st != IJ_OK) return st;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CUDA_TRY(cudaMemcpyAsync(h->stage, f, 19 * N * sizeof(float), kind, h->stream));
  CUDA_TRY(cudaMemcpyAsync(h->stage + 19 * N, g, 7 * N * sizeof(float), kind, h->stream));
  CUDA_TRY(launch_import3(h->d_inst3, J, index, h->stage, h->stage + 19 * N, h->stream));
  h->launches++;
  CUDA_TRY(cudaMemcpyAsync(h->d_t, &t, sizeof(long long), cudaMemcpyHostToDevice, h->stream));
  const double dinit[8] = {0, 0, 0, -1, 0, 0, 0, 0};
  for (int k = 0; k < h->n_inst; k++)
    CUDA_TRY(cudaMemcpyAsync(h->inst[k].dstate, dinit, sizeof(dinit), cudaMemcpyHostToDevice, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  h->t = t;
  h->drop_graph();
  return IJ_OK;
}

// Absolute FP32 populations of a 2-D lattice in FP16 storage, decoded
// through the staging buffer (the other time buffer is too small for FP32).
ij_status get_state16(ij_handle h, int index, float* f, float* g, int on_device) {
  const Inst& I = h->inst[index];
  const size_t N = (size_t)I.nx * I.ny;
  ij_status st = ensure_stage(h, 14 * N);
  if (st != IJ_OK) return st;
  CUDA_TRY(launch_convert16(h->d_inst, I, index, (int)(h->t & 1), h->stage, h->stage + 9 * N,
                            false, h->stream));
  h->launches++;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (f) CUDA_TRY(cudaMemcpyAsync(f, h->stage, 9 * N * sizeof(float), kind, h->stream));
  if (g) CUDA_TRY(cudaMemcpyAsync(g, h->stage + 9 * N, 5 * N * sizeof(float), kind, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return IJ_OK;
}

// Encode absolute FP32 populations into the FP16 state of time parity t.
ij_status set_state16(ij_handle h, int index, const float* f, const float* g, long long t,
                      int on_device) {
  const Inst& I = h->inst[index];
  const size_t N = (size_t)I.nx * I.ny;
  ij_status st = ensure_stage(h, 14 * N);
  if (st != IJ_OK) return st;
  const cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  CUDA_TRY(cudaMemcpyAsync(h->stage, f, 9 * N * sizeof(float), kind, h->stream));
  CUDA_TRY(cudaMemcpyAsync(h->stage + 9 * N, g, 5 * N * sizeof(float), kind, h->stream));
  CUDA_TRY(launch_convert16(h->d_inst, I, index, (int)(t & 1), h->stage, h->stage + 9 * N, true,
                            h->stream));
  h->launches++;
  return IJ_OK;
}

}  // namespace

namespace ij {
// Parameter validation and derivation shared with the allocation-free entry
// point (inkjet_noalloc.cu).
ij_status validate_params(const ij_params& p, int k) { return validate(p, k); }
Inst derive_params(const ij_params& p) { return derive(p); }
ij_status report(ij_status st, const char* msg) { return fail(st, "%s", msg); }
}  // namespace ij

extern "C" {

ij_status ij_create(const ij_params* params, int count, ij_alloc_fn alloc, ij_free_fn free_fn,
                    void* ctx, void* stream, ij_handle* out) {
  if (!out) return fail(IJ_ERR_PARAM, "out is NULL");
  *out = nullptr;
  if (!params || count < 1 || count > 65536) return fail(IJ_ERR_PARAM, "count must be in [1, 65536]");
  if ((alloc == nullptr) != (free_fn == nullptr))
    return fail(IJ_ERR_PARAM, "alloc and free callbacks must be both set or both NULL");
  int de = params[0].diag_every;
  for (int k = 0; k < count; k++) {
    ij_status st = validate(params[k], k);
    if (st != IJ_OK) return st;
    if (params[k].diag_every != de)
      return fail(IJ_ERR_PARAM, "all lattices of a batch must share diag_every");
  }
  ij_handle h = new (std::nothrow) ij_handle_s();
  if (!h) return fail(IJ_ERR_OOM, "host allocation failed");
  h->n_inst = count;
  h->params.assign(params, params + count);
  h->stream = (cudaStream_t)stream;

  h->alloc = alloc;
  h->free_fn = free_fn;
  h->ctx = ctx;
  h->diag_every = de;
  auto bail = [&](ij_status st) {
    h->release();
    delete h;
    return st;
  };
  cudaError_t e = set_step_smem_limit();
  if (e != cudaSuccess) return bail(fail(IJ_ERR_CUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e)));
  const int dim0 = params[0].dim == 0 ? 2 : params[0].dim;
  for (int k = 0; k < count; k++)
    if ((params[k].dim == 0 ? 2 : params[k].dim) != dim0)
      return bail(fail(IJ_ERR_PARAM, "all lattices of a batch must have the same dim"));
  if (dim0 == 3) {
    ij_status st3 = create3(h);
    if (st3 != IJ_OK) return bail(st3);
    *out = h;
    return IJ_OK;
  }
  // one step launch covers every lattice, so they share one storage format
  for (int k = 1; k < count; k++)
    if (params[k].precision != params[0].precision)
      return bail(fail(IJ_ERR_PARAM, "all 2-D lattices of a batch must share the precision"));
  h->fp16 = params[0].precision == IJ_FP16_STORE;
  for (int k = 0; k < count; k++)
    if (params[k].nx % 2 != 0) h->odd = true;
  h->inst.resize(count);
  for (int k = 0; k < count; k++) {
    Inst I = derive(params[k]);
    for (int b = 0; b < 2; b++) {
      I.f[b] = (float*)h->dalloc(state_bytes_f(I));
      I.g[b] = (float*)h->dalloc(state_bytes_g(I));
      if (!I.f[b] || !I.g[b]) return bail(fail(IJ_ERR_OOM, "device allocation of lattice %d failed", k));
    }
    I.rows = (double*)h->dalloc(3 * (size_t)I.ny * sizeof(double));
    I.sums = (double*)h->dalloc(4 * sizeof(double));
    I.hist = (double*)h->dalloc((size_t)kHistCap * kRec * sizeof(double));
    I.dstate = (double*)h->dalloc(8 * sizeof(double));
    if (!I.rows || !I.sums || !I.hist || !I.dstate)
      return bail(fail(IJ_ERR_OOM, "device allocation of diagnostics failed"));
    h->inst[k] = I;
  }
  build_items(h);
  h->d_inst = (Inst*)h->dalloc(count * sizeof(Inst));
  h->d_items = (Item*)h->dalloc(h->items.size() * sizeof(Item));
  h->items_cap = h->items.size();
  h->d_t = (long long*)h->dalloc(sizeof(long long));
  h->d_status = (unsigned*)h->dalloc(count * sizeof(unsigned));
  for (int k = 0; k < count && h->d_status; k++) h->inst[k].status = h->d_status + k;
  if (!h->d_inst || !h->d_items || !h->d_t || !h->d_status)
    return bail(fail(IJ_ERR_OOM, "device allocation of descriptors failed"));
  if (cudaMallocHost((void**)&h->h_status, count * sizeof(unsigned)) != cudaSuccess)
    return bail(fail(IJ_ERR_OOM, "pinned allocation failed"));
  memset(h->h_status, 0, count * sizeof(unsigned));
  cudaStream_t s = h->stream;
#define BAIL_CUDA(expr)                                                                       \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess) return bail(fail(IJ_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_))); \
  } while (0)
  BAIL_CUDA(cudaMemcpyAsync(h->d_inst, h->inst.data(), count * sizeof(Inst), cudaMemcpyHostToDevice, s));
  BAIL_CUDA(cudaMemcpyAsync(h->d_items, h->items.data(), h->items.size() * sizeof(Item),
                            cudaMemcpyHostToDevice, s));
  BAIL_CUDA(cudaMemsetAsync(h->d_t, 0, sizeof(long long), s));
  BAIL_CUDA(cudaMemsetAsync(h->d_status, 0, count * sizeof(unsigned), s));
  const double dinit[8] = {0, 0, 0, -1, 0, 0, 0, 0};
  for (int k = 0; k < count; k++) {
    const Inst& I = h->inst[k];
    BAIL_CUDA(cudaMemsetAsync(I.rows, 0, 3 * (size_t)I.ny * sizeof(double), s));
    BAIL_CUDA(cudaMemsetAsync(I.sums, 0, 4 * sizeof(double), s));
    BAIL_CUDA(cudaMemsetAsync(I.hist, 0, (size_t)kHistCap * kRec * sizeof(double), s));
    BAIL_CUDA(cudaMemcpyAsync(I.dstate, dinit, sizeof(dinit), cudaMemcpyHostToDevice, s));
    BAIL_CUDA(launch_init(h->d_inst, I, k, s));
    h->launches += 4;
  }
  BAIL_CUDA(cudaStreamSynchronize(s));
#undef BAIL_CUDA
  *out = h;
  return IJ_OK;
}

ij_status ij_step(ij_handle h, long long nsteps) {
  ij_status st = check_handle(h);
  if (st != IJ_OK) return st;
  if (nsteps < 0) return fail(IJ_ERR_PARAM, "nsteps < 0");
  if (!h->poisoned) {
    int flagged = 0;
    for (int k = 0; k < h->n_inst; k++) flagged += (h->h_status[k] & kStatusNumeric) != 0;
    h->poisoned = flagged == h->n_inst;
  }
  if (h->poisoned)
    return fail(IJ_ERR_NUMERIC, "every lattice of the handle has produced NaN or |u| > 0.3");
  long long left = nsteps;
  while (left > 0) {
    const int P = h->diag_every > 0 ? h->diag_every : 16;
    // whole diagnostics periods run as one graph launch (not while the
    // step kernels are being timed launch by launch)
    if (h->use_graph && !h->timing && left >= P && h->t % P == 0) {
      if (!h->gexec) {
        st = build_graph(h);
        if (st != IJ_OK) return st;
      }
      CUDA_TRY(cudaGraphLaunch(h->gexec, h->stream));
      h->launches += h->graph_launches;
      h->t += P;
      left -= P;
    } else {
      st = one_step(h);
      if (st != IJ_OK) return st;
      left--;
    }
  }
  CUDA_TRY(cudaMemcpyAsync(h->h_status, h->d_status, h->n_inst * sizeof(unsigned),
                           cudaMemcpyDeviceToHost, h->stream));
  return IJ_OK;
}

ij_status ij_observe(ij_handle h, int index, ij_obs* out, float* phi_out, int phi_on_device) {
  ij_status st = check_handle(h);
  if (st != IJ_OK) return st;
  if (index < 0 || index >= h->n_inst) return fail(IJ_ERR_PARAM, "index out of range");
  const Inst& I = h->inst[index];
  if (phi_out && h->is3d) {
    const Inst3& J = h->inst3[index];
    const size_t N3 = (size_t)J.nx * J.ny * J.nz;
    if (!phi_on_device) {
      st = ensure_stage(h, N3);
      if (st != IJ_OK) return st;
    }
    float* dst = phi_on_device ? phi_out : h->stage;
    CUDA_TRY(launch_phi3(h->d_inst3, J, index, dst, h->stream));
    h->launches++;
    if (!phi_on_device)
      CUDA_TRY(cudaMemcpyAsync(phi_out, dst, N3 * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  } else if (phi_out) {
    const size_t N = (size_t)I.nx * I.ny;
    float* dst = phi_on_device ? phi_out : h->inst[index].f[(h->t + 1) & 1];
    CUDA_TRY(launch_phi(h->d_inst, I, index, h->d_t, dst, h->stream));
    h->launches++;
    if (!phi_on_device)
      CUDA_TRY(cudaMemcpyAsync(phi_out, dst, N * sizeof(float), cudaMemcpyDeviceToHost, h->stream));
  }
  unsigned status = 0;
  double dstate[8];
  CUDA_TRY(cudaMemcpyAsync(&status, h->d_status + index, sizeof(unsigned), cudaMemcpyDeviceToHost,
                           h->stream));
  CUDA_TRY(cudaMemcpyAsync(dstate, I.dstate, sizeof(dstate), cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (out) {
    long long cnt = (long long)dstate[4];
    if (cnt <= 0) {
      memset(out, 0, sizeof(*out));
      out->step = -1;
      out->breakup_step = -1;
    } else {
      CUDA_TRY(cudaMemcpy(out, I.hist + ((cnt - 1) % kHistCap) * kRec, sizeof(ij_obs),
                          cudaMemcpyDeviceToHost));
    }
  }
  if (status & kStatusNumeric)
    return fail(IJ_ERR_NUMERIC, "lattice %d produced NaN or |u| > 0.3 and is frozen", index);
  return IJ_OK;
}

ij_status ij_history(ij_handle h, int index, double* out, int max_records, int* count) {
  ij_status st = check_handle(h);
  if (st != IJ_OK) return st;
  if (index < 0 || index >= h->n_inst) return fail(IJ_ERR_PARAM, "index out of range");
  const Inst& I = h->inst[index];
  double dstate[8];
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  CUDA_TRY(cudaMemcpy(dstate, I.dstate, sizeof(dstate), cudaMemcpyDeviceToHost));
  long long cnt = (long long)dstate[4];
  long long held = std::min<long long>(cnt, kHistCap);
  if (count) *count = (int)held;
  if (out && max_records > 0) {
    long long first = cnt - held;
    long long n = std::min<long long>(held, max_records);
    for (long long r = 0; r < n; r++)
      CUDA_TRY(cudaMemcpy(out + r * kRec, I.hist + ((first + r) % kHistCap) * kRec,
                          kRec * sizeof(double), cudaMemcpyDeviceToHost));
  }
  return IJ_OK;
}

ij_status ij_get_state(ij_handle h, int index, float* f, float* g, int on_device) {
  ij_status st = check_handle(h);
  if (st != IJ_OK) return st;
  if (index < 0 || index >= h->n_inst) return fail(IJ_ERR_PARAM, "index out of range");
  if (h->is3d) return get_state3(h, index, f, g, on_device);
  if (h->fp16) return get_state16(h, index, f, g, on_device);
  const Inst& I = h->inst[index];
  const size_t N = (size_t)I.nx * I.ny;
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (f) {
    // the stored deviations become absolute populations on the way out; the
    // buffer of the other time parity is free between steps and stages them
    float* stage = on_device ? f : I.f[(h->t + 1) & 1];
    CUDA_TRY(launch_f_export(h->d_inst, I, index, I.f[h->t & 1], stage, h->stream));
    h->launches++;
    if (!on_device)
      CUDA_TRY(cudaMemcpyAsync(f, stage, 9 * N * sizeof(float), kind, h->stream));
  }
  if (g) CUDA_TRY(cudaMemcpyAsync(g, I.g[h->t & 1], 5 * N * sizeof(float), kind, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  return IJ_OK;
}

ij_status ij_set_state(ij_handle h, int index, const float* f, const float* g, long long t,
                       int on_device) {
  ij_status st = check_handle(h);
  if (st != IJ_OK) return st;
  if (index < 0 || index >= h->n_inst) return fail(IJ_ERR_PARAM, "index out of range");
  if (t < 0) return fail(IJ_ERR_PARAM, "t < 0");
  if (h->poisoned) return fail(IJ_ERR_STATE, "handle is poisoned");
  if (!f || !g) return fail(IJ_ERR_PARAM, "f and g are required");
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  if (h->is3d) return set_state3(h, index, f, g, t, on_device);
  cudaMemcpyKind kind = on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  // all lattices share the time: move the others' state to the new parity
  if ((t & 1) != (h->t & 1)) {
    for (int k = 0; k < h->n_inst; k++) {
      if (k == index) continue;
      const Inst& J = h->inst[k];
      CUDA_TRY(cudaMemcpyAsync(J.f[t & 1], J.f[h->t & 1], state_bytes_f(J), cudaMemcpyDeviceToDevice, h->stream));
      CUDA_TRY(cudaMemcpyAsync(J.g[t & 1], J.g[h->t & 1], state_bytes_g(J), cudaMemcpyDeviceToDevice, h->stream));
    }
  }
  const Inst& I = h->inst[index];
  if (h->fp16) {
    st = set_state16(h, index, f, g, t, on_device);
    if (st != IJ_OK) return st;
  } else {
    const size_t N = (size_t)I.nx * I.ny;
    CUDA_TRY(cudaMemcpyAsync(I.f[(t + 1) & 1], f, 9 * N * sizeof(float), kind, h->stream));
    CUDA_TRY(launch_f_import(h->d_inst, I, index, I.f[(t + 1) & 1], I.f[t & 1], h->stream));
    h->launches++;
    CUDA_TRY(cudaMemcpyAsync(I.g[t & 1], g, 5 * N * sizeof(float), kind, h->stream));
  }
  CUDA_TRY(cudaMemcpyAsync(h->d_t, &t, sizeof(long long), cudaMemcpyHostToDevice, h->stream));
  const double dinit[8] = {0, 0, 0, -1, 0, 0, 0, 0};
  for (int k = 0; k < h->n_inst; k++) {
    const Inst& J = h->inst[k];
    CUDA_TRY(cudaMemcpyAsync(J.dstate, dinit, sizeof(dinit), cudaMemcpyHostToDevice, h->stream));
  }
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  h->t = t;
  return IJ_OK;
}

ij_status ij_time(ij_handle h, long long* t) {
  ij_status st = check_handle(h);
  if (st != IJ_OK) return st;
  if (!t) return fail(IJ_ERR_PARAM, "t is NULL");
  *t = h->t;
  return IJ_OK;
}

ij_status ij_launch_count(ij_handle h, long long* launches) {
  ij_status st = check_handle(h);
  if (st != IJ_OK) return st;
  if (!launches) return fail(IJ_ERR_PARAM, "launches is NULL");
  *launches = h->launches;
  return IJ_OK;
}

ij_status ij_kernel_timing(ij_handle h, int enable, double* total_ms, long long* launches) {
  ij_status st = check_handle(h);
  if (st != IJ_OK) return st;
  h->drain_events();
  if (total_ms) *total_ms = h->timed_ms;
  if (launches) *launches = h->timed_launches;
  if (enable >= 0) {
    h->timing = enable != 0;
    h->timed_ms = 0.0;
    h->timed_launches = 0;
  }
  return IJ_OK;
}

ij_status ij_tune(ij_handle h, int block_size, int chunk, int prefetch) {
  ij_status st = check_handle(h);
  if (st != IJ_OK) return st;
  if (h->is3d) {
    // the z chunk of the 3-D work items; one block size, no prefetch depth
    if (chunk < 1 || prefetch != 1 || (block_size > 0 && block_size != kStep3Threads))
      return fail(IJ_ERR_PARAM, "3-D handles take chunk >= 1, prefetch 1, block size %d", kStep3Threads);
    h->buckets[0].chunk = chunk;
    CUDA_TRY(cudaStreamSynchronize(h->stream));
    return upload_items3(h);
  }
  if (chunk < -5 || prefetch < 1 || prefetch > kMaxPrefetch)
    return fail(IJ_ERR_PARAM, "chunk must be >= -5 and prefetch in 1..%d", kMaxPrefetch);
  bool found = false;
  for (Bucket& b : h->buckets)
    if (block_size <= 0 || b.nthreads == block_size) {
      found = true;
    }
  for (Bucket& b : h->buckets)
    if (block_size <= 0 || b.nthreads == block_size) {
      b.chunk = chunk;
      b.prefetch = prefetch;
    }
  if (!found) return fail(IJ_ERR_PARAM, "no lattice of the handle runs with %d threads", block_size);
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  build_items(h);
  return upload_items(h);
}

}  // extern "C"

namespace {

// The z chunk of the 3-D work items with the shortest step (trial launches
// read the state at t and write only the other buffer, without diagnostics
// or ghosts: the state is unchanged).
ij_status autotune3(ij_handle h, int reps) {
  static const int kChunks3[] = {8, 12, 16, 20, 24, 32, 40, 48, 64, 80, 96, 128, 160, 256};
  int max_nz = 1;
  for (const Inst3& I : h->inst3) max_nz = std::max(max_nz, I.nz);
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  float best = 1e30f;
  int best_chunk = h->buckets[0].chunk;
  ij_status st = IJ_OK;
  for (int chunk : kChunks3) {
    if (chunk > 2 * max_nz) continue;
    h->buckets[0].chunk = chunk;
    st = upload_items3(h);
    if (st != IJ_OK) break;
    const int n = (int)h->items3.size();
    cudaError_t e = launch_step3(h->d_inst3, h->d_items3, n, h->n_inst, h->d_t, 0, false, h->fp16,
                                 h->stream);  // warm-up
    if (e == cudaSuccess) e = cudaEventRecord(e0, h->stream);
    for (int r = 0; r < reps && e == cudaSuccess; r++)
      e = launch_step3(h->d_inst3, h->d_items3, n, h->n_inst, h->d_t, 0, false, h->fp16, h->stream);
    if (e == cudaSuccess) e = cudaEventRecord(e1, h->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e != cudaSuccess) {
      st = fail(IJ_ERR_CUDA, "3-D autotune: %s", cudaGetErrorString(e));
      break;
    }
    h->launches += reps + 1;
    if (ms < best) {
      best = ms;
      best_chunk = chunk;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (st != IJ_OK) return st;
  h->buckets[0].chunk = best_chunk;
  return upload_items3(h);
}

}  // namespace

extern "C" {

ij_status ij_autotune(ij_handle h, int reps) {
  ij_status st = check_handle(h);
  if (st != IJ_OK) return st;
  if (reps < 1) return fail(IJ_ERR_PARAM, "reps must be >= 1");
  if (h->poisoned) return fail(IJ_ERR_STATE, "handle is poisoned");
  if (h->is3d) return autotune3(h, reps);
  // row chunks, then the cost-balanced variants (chunk <= 0)
  static const int kChunks[] = {8,   16,  24,  32,  40,  48, 56, 64, 72, 80, 88, 96, 104,
                                112, 120, 128, 160, 192, 256, 0,  -1, -2, -3, -4, -5};
  cudaEvent_t e0, e1;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  // Trial launches read the state at t and write only the other time buffer
  // (without diagnostics), so the state is unchanged; t does not advance.
  for (size_t bi = 0; bi < h->buckets.size(); bi++) {
    const int nt = h->buckets[bi].nthreads;
    int max_ny = 1;
    for (int k = 0; k < h->n_inst; k++)
      if (block_size_for(h->inst[k]) == nt) max_ny = std::max(max_ny, h->inst[k].ny);
    float best = 1e30f;
    int best_chunk = h->buckets[bi].chunk, best_pf = h->buckets[bi].prefetch;
    for (int pf = 1; pf <= kMaxPrefetch; pf++)
      for (int chunk : kChunks) {
        if (chunk > 2 * max_ny && chunk > 0) continue;
        h->buckets[bi].chunk = chunk;
        h->buckets[bi].prefetch = pf;
        build_items(h);
        st = upload_items(h);
        if (st != IJ_OK) { cudaEventDestroy(e0); cudaEventDestroy(e1); return st; }
        const Bucket& b = h->buckets[bi];
        CUDA_TRY(launch_step(h->d_inst, h->d_items + b.first, b.count, nt, b.grid, h->d_t, 0,
                             false, pf, h->fp16, h->odd, h->stream));  // warm-up
        CUDA_TRY(cudaEventRecord(e0, h->stream));
        for (int r = 0; r < reps; r++)
          CUDA_TRY(launch_step(h->d_inst, h->d_items + b.first, b.count, nt, b.grid, h->d_t, 0,
                               false, pf, h->fp16, h->odd, h->stream));
        CUDA_TRY(cudaEventRecord(e1, h->stream));
        CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.0f;
        CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        h->launches += reps + 1;
        if (ms < best) {
          best = ms;
          best_chunk = chunk;
          best_pf = pf;
        }
      }
    h->buckets[bi].chunk = best_chunk;
    h->buckets[bi].prefetch = best_pf;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  build_items(h);
  return upload_items(h);
}

ij_status ij_use_graph(ij_handle h, int enable) {
  ij_status st = check_handle(h);
  if (st != IJ_OK) return st;
  h->use_graph = enable != 0;
  return IJ_OK;
}

ij_status ij_get_tuning(ij_handle h, int bucket, int* block_size, int* chunk, int* prefetch,
                        int* items) {
  ij_status st = check_handle(h);
  if (st != IJ_OK) return st;
  if (bucket < 0 || bucket >= (int)h->buckets.size()) return fail(IJ_ERR_PARAM, "no such bucket");
  const Bucket& b = h->buckets[bucket];
  if (block_size) *block_size = b.nthreads;
  if (chunk) *chunk = b.chunk;
  if (prefetch) *prefetch = b.prefetch;
  if (items) *items = b.count;
  return IJ_OK;
}

ij_status ij_destroy(ij_handle h) {
  if (!h) return IJ_OK;
  h->release();
  delete h;
  return IJ_OK;
}

const char* ij_last_error(void) { return g_err; }

}  // extern "C"
