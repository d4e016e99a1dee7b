// Host orchestration and C ABI of libpbs.
//
// Per Bloch vector k the iteration follows Algorithm 2 of the paper (Section 4):
//   R = A E - M E Lambda                   (FP64, Lambda = Rayleigh quotients)
//   W = B R                                (V-cycle for A + mu M, Section 5)
//   [E, W] <- projected off the gradients  (nodal V-cycles on L^* M L, Section 4/5)
//   Rayleigh-Ritz on span(E, W, P)         (Grams + small dense eigensolve, FP64)
//   E <- lowest p Ritz vectors, P <- new search direction
// until every wanted band has ||A e - lambda M e||_2 <= tol * lambda ||M e||_2.
// Along a k-path the first block of every k after the first comes from
// Rayleigh-Ritz of the new pencil on the span of up to three previous bases
// (Section 6).  The span of (E, W, P) equals the paper's span of
// (E_hat, E^(m), E^(m-1)) with E_hat = E - W; using W and the implicit
// direction P keeps the trial basis well conditioned.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <functional>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"
#include "pbs.h"

namespace pbs {

static thread_local std::string g_last_error;
thread_local KernelTimer* g_timer = nullptr;
static std::atomic<unsigned long long> g_launches{0}, g_df_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long delta) { g_launches.fetch_add((unsigned long long)delta, std::memory_order_relaxed); }
void count_df_launch() { g_df_launches.fetch_add(1, std::memory_order_relaxed); }

bool verbose_enabled() {
  static const bool v = std::getenv("PBS_VERBOSE") != nullptr;
  return v;
}

void timer_begin(int cls, cudaStream_t s, double work) {
  KernelTimer* t = g_timer;
  if (!t || !(t->mask & (1u << cls))) return;
  t->open = (t->seen[cls]++ % t->every) == 0;
  if (!t->open) return;
  std::pair<cudaEvent_t, cudaEvent_t> ev;
  if (!t->pool.empty()) {
    ev = t->pool.back();
    t->pool.pop_back();
  } else {
    PBS_CUDA(cudaEventCreate(&ev.first));
    PBS_CUDA(cudaEventCreate(&ev.second));
  }
  PBS_CUDA(cudaEventRecord(ev.first, s));
  t->pending.push_back(TimedLaunch{cls, work, ev.first, ev.second});
}

void timer_end(int cls, cudaStream_t s) {
  KernelTimer* t = g_timer;
  if (!t || !(t->mask & (1u << cls)) || !t->open || t->pending.empty()) return;
  t->open = false;
  PBS_CUDA(cudaEventRecord(t->pending.back().stop, s));
}

void timer_collect() {
  KernelTimer* t = g_timer;
  if (!t) return;
  for (auto& l : t->pending) {
    PBS_CUDA(cudaEventSynchronize(l.stop));
    float ms = 0.f;
    PBS_CUDA(cudaEventElapsedTime(&ms, l.start, l.stop));
    t->total_ms[l.cls] += ms;
    t->work[l.cls] += l.work;
    t->launches[l.cls] += 1;
    t->pool.push_back({l.start, l.stop});
  }
  t->pending.clear();
}

void fail(int status, const std::string& what) { throw Error{status, what}; }

void set_last_error(const std::string& what) { g_last_error = what; }

void check_cuda(cudaError_t e, const char* what) {
  if (e != cudaSuccess) {
    const int status = e == cudaErrorMemoryAllocation ? PBS_ENOMEM : PBS_ECUDA;
    fail(status, std::string(what) + ": " + cudaGetErrorString(e));
  }
}

void* DevMem::alloc(size_t bytes) {
  if (bytes == 0) bytes = 16;
  bytes = (bytes + 255) & ~size_t(255);
  if (fail_in_ > 0 && --fail_in_ == 0) fail(PBS_ENOMEM, "device allocation failed (injected)");
  if (budget_ && used_ + bytes > budget_) fail(PBS_ENOMEM, "device memory budget exceeded");
  void* p = nullptr;
  const cudaError_t e = cudaMalloc(&p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(PBS_ENOMEM, std::string("cudaMalloc: ") + cudaGetErrorString(e));
  }
  live_.push_back({p, bytes});
  used_ += bytes;
  return p;
}

void DevMem::free(void* p) {
  if (!p) return;
  for (size_t i = 0; i < live_.size(); ++i) {
    if (live_[i].first == p) {
      used_ -= live_[i].second;
      live_.erase(live_.begin() + i);
      cudaFree(p);
      return;
    }
  }
}

namespace {

uint64_t fnv1a(const void* data, size_t bytes, uint64_t h = 1469598103934665603ull) {
  const unsigned char* p = (const unsigned char*)data;
  for (size_t i = 0; i < bytes; ++i) {
    h ^= p[i];
    h *= 1099511628211ull;
  }
  return h;
}

__global__ void k_hash_eps(const double* __restrict__ eps, long n, unsigned long long* out) {
  unsigned long long h = 0;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x) {
    unsigned long long v = (unsigned long long)__double_as_longlong(eps[t]);
    v ^= (unsigned long long)t * 0x9e3779b97f4a7c15ull;
    v *= 0xbf58476d1ce4e5b9ull;
    v ^= v >> 31;
    h += v;
  }
  atomicAdd(out, h);
}

__global__ void k_rq(const double* __restrict__ parts, double* __restrict__ lam, int n) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < n) lam[c] = parts[2 * c + 1] / parts[2 * c];
}

template <class T> __global__ void k_axpy(cx<T>* __restrict__ y, const cx<T>* __restrict__ x, long n) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    y[t] = y[t] + x[t];
}

__global__ void k_sub_from(const double2* __restrict__ e, double2* __restrict__ w, long n) {  // w = e - w
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    w[t] = e[t] - w[t];
}

// Per-iteration trace on stderr when the environment sets PBS_VERBOSE (diagnostics only).
bool verbose() {
  static const bool v = std::getenv("PBS_VERBOSE") != nullptr;
  return v;
}

inline unsigned nblocks(long n) { return (unsigned)std::min<long>(std::max<long>((n + 255) / 256, 1), 4096); }

}  // namespace

// CUDA graphs of the iteration's multigrid sequences (projections and the
// preconditioner), captured on their second occurrence within a solve and replayed
// afterwards: one graph launch instead of tens of kernel launches per sequence.
// A graph is keyed by everything its launches depend on (pointers, column counts,
// cycles, the k = 0 deflation) and lives until the solve ends.
struct GraphCache {
  struct Entry {
    cudaGraphExec_t exec = nullptr;
    long kernels = 0;  // kernels per replay (for the launch counter)
  };
  std::map<std::string, Entry> graphs;
  std::map<std::string, int> seen;
  void clear() {
    for (auto& kv : graphs) cudaGraphExecDestroy(kv.second.exec);
    graphs.clear();
    seen.clear();
  }
  ~GraphCache() { clear(); }
};

// Batched solver workspace: G groups (Bloch vectors in flight) of p columns.
// The iteration's four blocks of G p columns live in one allocation of four
// quarters: [E P | W R] or [W R | E P] (`half` says which).  E and P stay adjacent
// (they are projected together), and the update writes P_new over R and E_new over
// W, after which the halves swap roles: no second copy of the block is kept.
// Group g's columns of a role start at g p.  Multigrid work (edge V-cycles, nodal
// projection) covers at most `chunk` columns at a time and exists only in the
// arithmetic of the precision policy in use.
struct Work {
  int G = 0, p = 0, prec = -1, chunk = 0;
  long D = 0, N = 0, hist_cols = 0;
  double2* blk = nullptr;
  int half = 0;
  double2 *init = nullptr, *hist = nullptr;
  double2 *GM = nullptr, *GA = nullptr, *C = nullptr, *rr_scr = nullptr, *gpart = nullptr;
  long gpart_cap = 0;
  double *theta = nullptr, *lam = nullptr, *parts = nullptr, *norms = nullptr, *rq = nullptr;
  int* info = nullptr;
  float2 *r32 = nullptr, *w32 = nullptr;
  void *nb = nullptr, *nx = nullptr, *nr = nullptr, *nd = nullptr;  // nodal vectors, chunk columns
  MgWork<float> e32, n32;
  MgWork<double> e64, n64;
  std::vector<void*> allocs;
  std::shared_ptr<GraphCache> graphs = std::make_shared<GraphCache>();
  long block() const { return (long)G * p * D; }
  double2* E() const { return blk + 2L * half * block(); }
  double2* P() const { return E() + block(); }
  double2* W() const { return blk + 2L * (1 - half) * block(); }
  double2* R() const { return W() + block(); }
};

}  // namespace pbs

using namespace pbs;

namespace pbs {

// One submitted path (pbs_submit): its inputs, copied at submission, and results.
struct Job {
  uint64_t id = 0;
  double a = 0, b = 0;
  int n = 0, m = 0, nk = 0;
  std::vector<double> eps, ks;
  pbs_opts o{};
  double est = 0;     // admission estimate, device bytes
  uint64_t gkey = 0;  // geometry key (permittivity, cell, mesh, mu, coarsest): slot affinity
  std::chrono::steady_clock::time_point t_submit, t_start, t_done;
  std::vector<double> lam, res;
  std::vector<int> iters;
  int status = PBS_OK;
  std::string err;
  bool started = false, done = false;
  int bypassed = 0;                // later jobs admitted before this one while it waited at the head
  std::atomic<bool> cancel{false};  // checked by the solver between iterations
};

// A serving slot: a child engine (own stream, resident hierarchy and workspace)
// driven by its own host thread, so that the jobs of different slots overlap on
// the device.
struct Slot {
  pbs_ctx* eng = nullptr;
  std::thread th;
  std::shared_ptr<Job> job;  // running job, null when idle
  double held = 0;           // bytes charged: the running job's estimate, or what stays resident when idle
  uint64_t resident = 0;     // geometry key of the resident hierarchy (0: none)
  bool evict = false;        // asked to free its resident hierarchy and workspace
};

// Continuous batching of path jobs: a queue in submission order and `nslots`
// slots.  A slot takes the first queued job that fits the memory the running jobs
// and the idle slots' resident data leave free (preferring, among the first few,
// a job whose geometry is resident in it); a job at the head that does not fit
// waits (idle slots are asked to free what they keep resident) and is passed by
// later jobs at most 2 nslots times.
struct Server {
  std::mutex m;
  std::condition_variable cv_work, cv_done;
  std::deque<std::shared_ptr<Job>> queue;
  std::map<uint64_t, std::shared_ptr<Job>> jobs;
  uint64_t next_id = 1;
  int nslots = 4;
  std::vector<std::unique_ptr<Slot>> slots;
  bool started = false, stop = false;
  double cap = 0;  // device bytes the jobs may hold together
};

}  // namespace pbs

struct pbs_ctx {
  std::mutex gpu_mu;  // every call that uses the context's device state holds it
  pbs::Server srv;
  int device = 0;
  cudaStream_t stream = nullptr;
  DevMem mem;
  Hierarchy H;
  bool have_h = false;
  int coarsest = 0;
  KData K;
  Work W;
  bool have_w = false;
  KernelTimer timer;
  double* d_eps_in = nullptr;  // device copy of the latest host permittivity array
  long d_eps_len = 0;
  const std::atomic<bool>* cancel = nullptr;  // set while a serving slot runs a job
  std::chrono::steady_clock::time_point t_created = std::chrono::steady_clock::now();
  explicit pbs_ctx(size_t budget) : mem(budget) {}
};

namespace {

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    cudaGetDevice(&prev);
    if (prev != dev) PBS_CUDA(cudaSetDevice(dev));
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

// Installs the context's kernel timer for the duration of an ABI call.
struct TimerScope {
  explicit TimerScope(pbs_ctx* ctx) { g_timer = ctx->timer.mask ? &ctx->timer : nullptr; }
  ~TimerScope() {
    try {
      timer_collect();
    } catch (...) {
    }
    g_timer = nullptr;
  }
};

// Frees the solver workspace, also one whose allocation failed part of the way.
void free_work(pbs_ctx* ctx) {
  for (void* p : ctx->W.allocs) ctx->mem.free(p);
  free_mg_work(ctx->mem, ctx->W.e32);
  free_mg_work(ctx->mem, ctx->W.n32);
  free_mg_work(ctx->mem, ctx->W.e64);
  free_mg_work(ctx->mem, ctx->W.n64);
  ctx->W.graphs->clear();
  ctx->W = Work();
  ctx->have_w = false;
}

void validate_opts(const pbs_opts& o) {
  if (o.nev < 1 || o.block < o.nev || o.block > kMaxBlock) fail(PBS_EINVAL, "need 1 <= nev <= block <= 32");
  if (o.max_iter < 0) fail(PBS_EINVAL, "max_iter must be >= 0");
  if (o.precision != PBS_FP64 && o.precision != PBS_MIXED) fail(PBS_EINVAL, "unknown precision");
  if (o.span < 1 || o.span > 3) fail(PBS_EINVAL, "span must be 1, 2 or 3");
  if (!(o.tol > 0)) fail(PBS_EINVAL, "tol must be positive");
  if (o.nu_pre < 0 || o.nu_post < 0 || o.nu_pre + o.nu_post < 1) fail(PBS_EINVAL, "need nu_pre + nu_post >= 1");
  if (o.coarsest < 2) fail(PBS_EINVAL, "coarsest must be >= 2");
  if (o.nodal_cycles < 1) fail(PBS_EINVAL, "nodal_cycles must be >= 1");
  if (o.extrap_depth < 0 || o.extrap_depth > 3) fail(PBS_EINVAL, "extrap_depth must be 0..3");
  if (o.kbatch < 1 || o.kbatch > 256) fail(PBS_EINVAL, "kbatch must be 1..256");
  if (o.start != PBS_START_RANDOM && o.start != PBS_START_NESTED) fail(PBS_EINVAL, "unknown start");
}

void validate_mesh(double a, double b, int n, int m) {
  if (!(a > 0) || !(b > 0) || !std::isfinite(a) || !std::isfinite(b)) fail(PBS_EINVAL, "a, b must be positive");
  if (n < 4 || m < 4 || (n & 1) || (m & 1)) fail(PBS_EINVAL, "n, m must be even and >= 4");
  if ((long)n * m > (1L << 28)) fail(PBS_EINVAL, "mesh too large");
}

double effective_mu(const pbs_opts& o, double a, double b) { return o.mu > 0 ? o.mu : 1.0 / (a * b); }

// Make the context's hierarchy match (geometry, mu, coarsest); eps on the device.
void ensure_hierarchy(pbs_ctx* ctx, double a, double b, int n, int m, const double* d_eps, uint64_t eps_hash, double mu,
                      int coarsest) {
  uint64_t key = eps_hash;
  key = fnv1a(&a, sizeof a, key);
  key = fnv1a(&b, sizeof b, key);
  key = fnv1a(&n, sizeof n, key);
  key = fnv1a(&m, sizeof m, key);
  key = fnv1a(&mu, sizeof mu, key);
  key = fnv1a(&coarsest, sizeof coarsest, key);
  if (ctx->have_h && ctx->H.key == key) return;
  free_work(ctx);  // workspaces depend on the hierarchy sizes
  if (ctx->have_h) free_hierarchy(ctx->mem, ctx->H);
  free_kdata(ctx->mem, ctx->K);
  ctx->have_h = false;
  ctx->H = Hierarchy();
  ctx->H.a = a;
  ctx->H.b = b;
  ctx->H.n = n;
  ctx->H.m = m;
  ctx->H.mu = mu;
  try {
    build_hierarchy(ctx->mem, ctx->H, d_eps, coarsest, ctx->stream);
  } catch (...) {
    free_hierarchy(ctx->mem, ctx->H);  // what was allocated before the failure
    ctx->H = Hierarchy();
    throw;
  }
  ctx->H.key = key;
  ctx->coarsest = coarsest;
  ctx->have_h = true;
}

// Upload host eps (hashing it first) and make the hierarchy resident.
void ensure_hierarchy_host(pbs_ctx* ctx, const pbs_geom* g, double mu, int coarsest) {
  validate_mesh(g->a, g->b, g->n, g->m);
  if (!g->eps) fail(PBS_EINVAL, "eps is NULL");
  const long N = (long)g->n * g->m;
  const uint64_t h = fnv1a(g->eps, N * sizeof(double));
  // the permittivity is an input of every call: it is copied each time, and the
  // resident hierarchy is rebuilt only when geometry, mu or coarsest changed
  if (ctx->d_eps_len != N) {
    ctx->mem.free(ctx->d_eps_in);
    ctx->d_eps_in = nullptr;
    ctx->d_eps_len = 0;
    ctx->d_eps_in = (double*)ctx->mem.alloc(N * sizeof(double));
    ctx->d_eps_len = N;
  }
  PBS_CUDA(cudaMemcpyAsync(ctx->d_eps_in, g->eps, N * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
  ensure_hierarchy(ctx, g->a, g->b, g->n, g->m, ctx->d_eps_in, h, mu, coarsest);
  PBS_CUDA(cudaStreamSynchronize(ctx->stream));
}

uint64_t device_eps_hash(pbs_ctx* ctx, const double* d_eps, long N) {
  unsigned long long* d_h = (unsigned long long*)ctx->mem.alloc(sizeof(unsigned long long));
  unsigned long long h = 0;
  PBS_CUDA(cudaMemsetAsync(d_h, 0, sizeof h, ctx->stream));
  k_hash_eps<<<nblocks(N), 256, 0, ctx->stream>>>(d_eps, N, d_h);
  PBS_LAUNCHED();
  PBS_CUDA(cudaMemcpyAsync(&h, d_h, sizeof h, cudaMemcpyDeviceToHost, ctx->stream));
  PBS_CUDA(cudaStreamSynchronize(ctx->stream));
  ctx->mem.free(d_h);
  return h;
}


// Multigrid work of one chunk is kept near chunk_bytes: 8 GiB, or an eighth of the
// context's device budget when that is smaller.  With D edges and N nodes a column
// needs about 2 D FP32 values for the preconditioner's FP32 copies (mixed), 4 D
// values of V-cycle work and 8 N values of nodal work, in the policy's precision.
double chunk_bytes(size_t budget) {
  const double cap = 8.0 * (1ull << 30);
  return budget > 0 ? std::min(cap, (double)budget / 8.0) : cap;
}

int chunk_columns(double D, double N, int p, int q, long want, int prec, double bytes) {
  const double c = prec == PBS_MIXED ? 8.0 : 16.0;
  const double per = (prec == PBS_MIXED ? 2.0 * D * 8.0 : 0.0) + 4.0 * D * c + 8.0 * N * c;
  long k = (long)(bytes / per);
  k -= k % p;
  k = std::max<long>(k, q);
  return (int)std::min<long>(k, std::max<long>(want, q));
}

// Work for G groups of p columns under precision policy `prec`, with `hist_cols`
// columns of extrapolation history.
void ensure_work(pbs_ctx* ctx, int p, int G, int prec, long hist_cols) {
  Work& W = ctx->W;
  const Hierarchy& H = ctx->H;
  if (ctx->have_w && W.p == p && W.G == G && W.prec == prec && W.hist_cols >= hist_cols &&
      W.D == H.lev[0].D() && W.N == H.lev[0].N())
    return;
  free_work(ctx);
  W.G = G;
  W.p = p;
  W.prec = prec;
  W.D = H.lev[0].D();
  W.N = H.lev[0].N();
  W.hist_cols = hist_cols;
  W.half = 0;
  const int q = 3 * p;
  auto A = [&](size_t bytes) {
    void* ptr = ctx->mem.alloc(bytes);
    W.allocs.push_back(ptr);
    return ptr;
  };
  const long D = W.D, N = W.N, Gp = (long)G * p;
  const int ck = chunk_columns((double)D, (double)N, p, q, std::max<long>(2 * Gp, q), prec,
                               chunk_bytes(ctx->mem.budget()));
  W.chunk = ck;
  W.blk = (double2*)A(sizeof(double2) * D * 4 * Gp);
  W.init = (double2*)A(sizeof(double2) * D * q);
  if (hist_cols > 0) W.hist = (double2*)A(sizeof(double2) * D * hist_cols);
  W.GM = (double2*)A(sizeof(double2) * q * q * G);
  W.GA = (double2*)A(sizeof(double2) * q * q * G);
  W.C = (double2*)A(sizeof(double2) * q * p * G);
  W.rr_scr = (double2*)A(small_rr_scratch(q) * G);
  W.gpart_cap = std::max(gram_partials_size(N, q, G), gram_partials_size(N, q, 1));
  W.gpart = (double2*)A(sizeof(double2) * W.gpart_cap);
  W.theta = (double*)A(sizeof(double) * q * G);
  W.lam = (double*)A(sizeof(double) * std::max<long>(Gp, q));
  const long ncol = std::max<long>(3 * Gp, q);
  const long nblk = ((H.lev[0].n + 31) / 32) * ((H.lev[0].m + 7) / 8);
  W.parts = (double*)A(sizeof(double) * std::max<long>(2 * nblk * ncol, 4 * 64 * ncol));
  W.norms = (double*)A(sizeof(double) * 2 * ncol);
  W.rq = (double*)A(sizeof(double) * 2 * ncol);
  W.info = (int*)A(sizeof(int) * 8 * G);
  const size_t cxb = prec == PBS_MIXED ? sizeof(float2) : sizeof(double2);
  W.nb = A(cxb * N * ck);
  W.nx = A(cxb * N * ck);
  W.nr = A(cxb * N * ck);
  W.nd = A(cxb * N * ck);
  if (prec == PBS_MIXED) {
    W.r32 = (float2*)A(sizeof(float2) * D * ck);
    W.w32 = (float2*)A(sizeof(float2) * D * ck);
    alloc_mg_work<float>(ctx->mem, H, ck, false, W.e32);
    alloc_mg_work<float>(ctx->mem, H, ck, true, W.n32);
  } else {
    alloc_mg_work<double>(ctx->mem, H, ck, false, W.e64);
    alloc_mg_work<double>(ctx->mem, H, ck, true, W.n64);
  }
  PBS_CUDA(cudaMemsetAsync(W.blk, 0, sizeof(double2) * D * 4 * Gp, ctx->stream));
  ctx->have_w = true;
}

// --- steps of the iteration ---------------------------------------------------

template <class T> struct Bufs;
template <> struct Bufs<float> {
  static float2* nb(Work& W) { return (float2*)W.nb; }
  static float2* nx(Work& W) { return (float2*)W.nx; }
  static float2* nr(Work& W) { return (float2*)W.nr; }
  static float2* nd(Work& W) { return (float2*)W.nd; }
  static MgWork<float>& emg(Work& W) { return W.e32; }
  static MgWork<float>& nmg(Work& W) { return W.n32; }
};
template <> struct Bufs<double> {
  static double2* nb(Work& W) { return (double2*)W.nb; }
  static double2* nx(Work& W) { return (double2*)W.nx; }
  static double2* nr(Work& W) { return (double2*)W.nr; }
  static double2* nd(Work& W) { return (double2*)W.nd; }
  static MgWork<double>& emg(Work& W) { return W.e64; }
  static MgWork<double>& nmg(Work& W) { return W.n64; }
};

// X <- X - L phi with phi from `cycles` nodal V-cycles on L^* M L phi = L^* M X; the
// constant edge fields of k = 0 groups are removed as well (Section 4).  Column c
// belongs to group c / cpg of K.
template <class T>
void project(pbs_ctx* ctx, const pbs_opts& o, const KData& K, double2* X, int ncols, int cpg, int cycles,
             cudaStream_t s) {
  if (ncols <= 0) return;
  Work& W = ctx->W;
  const Hierarchy& H = ctx->H;
  const Level& L0 = H.lev[0];
  const long N = L0.N(), D = L0.D();
  cx<T>* rhs = (cx<T>*)Bufs<T>::nb(W);
  cx<T>* phi = (cx<T>*)Bufs<T>::nx(W);
  cx<T>* res = (cx<T>*)Bufs<T>::nr(W);
  cx<T>* dphi = (cx<T>*)Bufs<T>::nd(W);
  const bool dfa = o.precision == PBS_MIXED;
  lift_adj_mass<T>(L0, K.d_ph, cpg, X, D, rhs, N, ncols, dfa, s);
  nodal_vcycle<T>(H, K, Bufs<T>::nmg(W), 0, rhs, phi, N, ncols, cpg, o.nu_pre, o.nu_post, s);
  const bool guess = nodal_takes_guess<T>(H, 0, o.nu_pre, o.nu_post);
  for (int c = 1; c < cycles; ++c) {
    if (guess) {
      // the next cycle continues from phi: phi + B (rhs - P phi) in one sweep of kernels
      nodal_vcycle_from<T>(H, K, Bufs<T>::nmg(W), 0, rhs, phi, phi, N, ncols, cpg, o.nu_pre, o.nu_post, s);
      continue;
    }
    apply_nodal<T>(L0, K.d_ph, cpg, phi, res, rhs, N, ncols, T(-1), T(1), s);
    nodal_vcycle<T>(H, K, Bufs<T>::nmg(W), 0, res, dphi, N, ncols, cpg, o.nu_pre, o.nu_post, s);
    timer_begin(KC_NODE_APPLY, s, 3.0 * sizeof(cx<T>) * N * ncols);
    k_axpy<T><<<nblocks(N * ncols), 256, 0, s>>>(phi, dphi, N * ncols);
    timer_end(KC_NODE_APPLY, s);
    PBS_LAUNCHED();
  }
  sub_lift<T>(L0, K.d_ph, cpg, phi, N, X, D, ncols, s);
  if (K.any_gamma()) deflate_constants(L0, X, D, ncols, K.d_gamma, cpg, W.parts, s);
}

// Columns [0, ncols) in pieces of whole groups of cpg columns, at most the
// workspace's chunk per piece: f(first column, columns, view of K for the piece).
template <class F> void for_chunks(pbs_ctx* ctx, const KData& K, int ncols, int cpg, F&& f) {
  const int per = std::max(cpg, ctx->W.chunk - ctx->W.chunk % cpg);
  for (int c0 = 0; c0 < ncols; c0 += per) {
    const int nc = std::min(per, ncols - c0);
    if (c0 == 0 && nc == ncols) f(0, nc, K);
    else f(c0, nc, kdata_chunk(K, c0 / cpg));
  }
}

bool graphs_enabled() {
  static const bool on = [] {
    const char* v = std::getenv("PBS_GRAPHS");
    return !(v && std::strcmp(v, "0") == 0);
  }();
  return on;
}

// Runs f (launches on stream s only, no host synchronisation) directly the first
// time `key` is met, captured into a CUDA graph and replayed from the second time
// on.  Kernel timing (pbs_profile_enable) of a class launched inside the sequences
// times launches one by one, so then f runs directly.
template <class F> void run_graph(pbs_ctx* ctx, const std::string& key, cudaStream_t s, F&& f) {
  GraphCache& gc = *ctx->W.graphs;
  constexpr unsigned kInside = (1u << KC_EDGE_SMOOTH) | (1u << KC_NODE_SMOOTH) | (1u << KC_LIFT_ADJ_MASK) |
                               (1u << KC_EDGE_APPLY) | (1u << KC_EDGE_TAIL) | (1u << KC_NODE_TAIL) |
                               (1u << KC_SUB_LIFT) | (1u << KC_CONVERT) | (1u << KC_NODE_APPLY);
  if (!graphs_enabled() || (g_timer != nullptr && (g_timer->mask & kInside))) {
    f();
    return;
  }
  auto it = gc.graphs.find(key);
  if (it == gc.graphs.end()) {
    if (gc.seen[key]++ == 0) {
      f();  // first occurrence: lazy set-up (kernel attributes) happens outside any capture
      return;
    }
    const unsigned long long before = g_launches.load();
    PBS_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
    try {
      f();
    } catch (...) {
      cudaGraph_t broken = nullptr;
      cudaStreamEndCapture(s, &broken);
      if (broken) cudaGraphDestroy(broken);
      cudaGetLastError();
      throw;
    }
    cudaGraph_t graph = nullptr;
    PBS_CUDA(cudaStreamEndCapture(s, &graph));
    GraphCache::Entry e;
    e.kernels = (long)(g_launches.load() - before);
    count_launches(-e.kernels);  // nothing ran yet: the replays count
    const cudaError_t ie = cudaGraphInstantiate(&e.exec, graph, 0);
    cudaGraphDestroy(graph);
    PBS_CUDA(ie);
    it = gc.graphs.emplace(key, e).first;
  }
  PBS_CUDA(cudaGraphLaunch(it->second.exec, s));
  count_launches(it->second.kernels);
}

std::string graph_key(const char* what, const void* x, const void* y, int ncols, int cpg, int cycles, const KData& K,
                      int prec) {
  char buf[256];
  std::snprintf(buf, sizeof buf, "%s|%p|%p|%d|%d|%d|%p|%d|%d|%d", what, x, y, ncols, cpg, cycles, (const void*)K.d_ph,
                K.goff, K.any_gamma() ? 1 : 0, prec);
  return buf;
}

void project_dispatch(pbs_ctx* ctx, const pbs_opts& o, const KData& K, double2* X, int ncols, int cpg, int cycles,
                      cudaStream_t s) {
  if (cycles <= 0) cycles = o.nodal_cycles;
  const long D = ctx->W.D;
  for_chunks(ctx, K, ncols, cpg, [&](int c0, int nc, const KData& Kc) {
    if (o.precision == PBS_MIXED) project<float>(ctx, o, Kc, X + (long)c0 * D, nc, cpg, cycles, s);
    else project<double>(ctx, o, Kc, X + (long)c0 * D, nc, cpg, cycles, s);
  });
}

// W = B R (one edge V-cycle per column); under the mixed policy `r32` (when given)
// holds R in FP32 already (the mixed residual kernel's output), else R is converted
void precondition_dispatch(pbs_ctx* ctx, const pbs_opts& o, const KData& K, const double2* R, double2* Wout, int ncols,
                           int cpg, cudaStream_t s, const float2* r32 = nullptr) {
  Work& W = ctx->W;
  for_chunks(ctx, K, ncols, cpg, [&](int c0, int nc, const KData& Kc) {
    const double2* Rc = R + (long)c0 * W.D;
    double2* Wc = Wout + (long)c0 * W.D;
    if (o.precision == PBS_MIXED) {
      const float2* in = W.r32;
      if (r32) in = r32 + (long)c0 * W.D;
      else convert_d2f(Rc, W.r32, W.D * nc, s);
      edge_vcycle<float>(ctx->H, Kc, W.e32, 0, in, W.w32, W.D, nc, cpg, o.nu_pre, o.nu_post, s);
      convert_f2d(W.w32, Wc, W.D * nc, s);
    } else {
      edge_vcycle<double>(ctx->H, Kc, W.e64, 0, Rc, Wc, W.D, nc, cpg, o.nu_pre, o.nu_post, s);
    }
  });
}

// Nodal cycles for the iteration's projections.  The preconditioner maps a
// gradient left in an iterate to about -(lambda/mu) times itself (A + mu M acts
// as mu M on gradients), so iterates with large Rayleigh quotients need a more
// accurate projection: one extra cycle (contraction about 0.1 each) per two
// decades of lambda/mu.
int projection_cycles(const pbs_opts& o, double theta_max, double mu) {
  const double ratio = theta_max / mu;
  const int extra = ratio > 1.0 ? (int)std::floor(std::log10(ratio) / 2.0) : 0;
  return o.nodal_cycles + std::min(extra, 6);
}

// Rayleigh-Ritz of one group's pencil (view Kv) on the q contiguous columns S:
// the p lowest Ritz vectors go to dst; returns the largest |theta|.
double rr_single(pbs_ctx* ctx, const KData& Kv, const double2* S, int q, int p, double2* dst, bool dfa,
                 cudaStream_t s) {
  Work& W = ctx->W;
  const Level& L0 = ctx->H.lev[0];
  const Roles R{{S, S, S}, q, W.D};
  gram_groups(L0, Kv.d_ph, R, q, 1, W.GM, W.GA, W.gpart, W.gpart_cap, dfa, s);
  small_rr(W.GM, W.GA, q, p, W.C, W.theta, W.rr_scr, W.info, 1, dfa, s);
  int info[2] = {0, 0};
  std::vector<double> th(p);
  PBS_CUDA(cudaMemcpyAsync(info, W.info, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  PBS_CUDA(cudaMemcpyAsync(th.data(), W.theta, p * sizeof(double), cudaMemcpyDeviceToHost, s));
  PBS_CUDA(cudaStreamSynchronize(s));
  if (info[0] != 0)
    fail(PBS_ENUMERIC, info[0] == -2 ? "non-finite Gram matrix"
                                     : info[0] == -3 ? "Rayleigh-Ritz breakdown" : "trial space lost rank");
  block_update(R, q, W.C, q, (long)q * p, dst, W.D, p, nullptr, 0, W.D, 1, false, s);
  double tm = 0.0;
  for (double t : th) tm = std::max(tm, std::fabs(t));
  return tm;
}

// The FP64 residual of a band with eigenvalue lambda cannot go below about
// 0.1 u lambda_max / lambda (u = 2^-53; the curl-curl stencil's terms are up to
// lambda_max / lambda times larger than the result; measured 0.08 - 0.16 on rod
// crystals from 256^2 to 1024^2).  A band converges at max(tol, 0.5 u
// lambda_max / lambda); lambda_max is bounded by max(1/eps) 12 (1/h1^2 + 1/h2^2),
// the largest symbol value of the stencils.
double lambda_max_bound(const Hierarchy& H) {
  const Level& L = H.lev[0];
  return H.winv_max * 12.0 * (1.0 / (L.h1 * L.h1) + 1.0 / (L.h2 * L.h2));
}
double band_tol(double tol, double lam_max, double lam) {
  return std::max(tol, 0.5 * std::ldexp(1.0, -53) * lam_max / std::fabs(lam));
}

// Host-side state of one group (one Bloch vector in flight, one chain of the path).
struct Group {
  int chain = -1;  // chain being solved (index into the chain list)
  int t = 0;       // position in the chain
  int pos = 0;     // index of the Bloch vector being solved in the k list
  int it = 0;
  bool have_p = false, active = false, need_init = false;
  int nhist = 0;
  double theta_max = 1e300;
};

// Start block of group g into E_g (P_g zeroed): extrapolation from the group's history,
// else `init` (host, D x p) or a seeded random block smoothed by two steps E <- B M E.
void init_group(pbs_ctx* ctx, const pbs_opts& o, Group& gr, int g, const pbs_c64* init, cudaStream_t s,
                const double2* dev_init = nullptr) {
  Work& W = ctx->W;
  const int p = o.block;
  const long D = W.D;
  const KData Kv = kdata_view(ctx->K, g);
  double2* Eg = W.E() + (long)g * p * D;
  double2* Pg = W.P() + (long)g * p * D;
  const int depth = std::min(gr.nhist, o.extrap_depth);
  double tm;
  if (depth > 0) {
    // S = [E_{k-1}, E_{k-2}, ...] as stored coefficient vectors (Section 6)
    const int q = depth * p;
    PBS_CUDA(cudaMemcpyAsync(W.init, W.hist + (long)g * o.extrap_depth * p * D, sizeof(double2) * D * q,
                             cudaMemcpyDeviceToDevice, s));
    project_dispatch(ctx, o, Kv, W.init, q, q, projection_cycles(o, gr.theta_max, ctx->H.mu), s);
    tm = rr_single(ctx, Kv, W.init, q, p, Eg, o.precision == PBS_MIXED, s);
  } else if (dev_init) {
    // a block prolongated from a coarser mesh (nested iteration): project, Rayleigh-Ritz
    PBS_CUDA(cudaMemcpyAsync(W.init, dev_init, sizeof(double2) * D * p, cudaMemcpyDeviceToDevice, s));
    project_dispatch(ctx, o, Kv, W.init, p, p, projection_cycles(o, 1e300, ctx->H.mu), s);
    tm = rr_single(ctx, Kv, W.init, p, p, Eg, o.precision == PBS_MIXED, s);
  } else {
    double2* X0 = W.init;           // p columns
    double2* X1 = W.init + D * p;   // p columns
    if (init) PBS_CUDA(cudaMemcpyAsync(X0, init, sizeof(double2) * D * p, cudaMemcpyHostToDevice, s));
    else random_block(X0, D, D, p, o.seed, s);
    // A block unrelated to the spectrum has Rayleigh quotients near its top: two
    // inverse-iteration steps E <- B M E (each followed by the projection and
    // Rayleigh-Ritz) damp the high frequencies before the iteration starts.
    const int cyc = projection_cycles(o, 1e300, ctx->H.mu);
    project_dispatch(ctx, o, Kv, X0, p, p, cyc, s);
    rr_single(ctx, Kv, X0, p, p, X1, o.precision == PBS_MIXED, s);
    double2* Rg = W.R() + (long)g * p * D;
    for (int step = 0; step < 2; ++step) {
      apply_edge<double>(ctx->H.lev[0], Kv.d_ph, p, X1, Rg, nullptr, D, p, 0.0, 1.0, 0.0, nullptr, 0.0, s);
      precondition_dispatch(ctx, o, Kv, Rg, X0, p, p, s);
      project_dispatch(ctx, o, Kv, X0, p, p, cyc, s);
      tm = rr_single(ctx, Kv, X0, p, p, step == 1 ? Eg : X1, o.precision == PBS_MIXED, s);
    }
  }
  PBS_CUDA(cudaMemsetAsync(Pg, 0, sizeof(double2) * D * p, s));
  gr.theta_max = tm;
  gr.it = 0;
  gr.have_p = false;
  gr.need_init = false;
}

// Smoothed random starts of every group at once (the groups' first Bloch vectors at the
// start of a solve): the steps of init_group's random branch, each one launch over all
// G groups (columns of group g at g p, cpg = p), with the W, R and P quarters of the
// block as scratch.  E ends with the groups' start blocks, P zeroed.
void rr_groups(pbs_ctx* ctx, const double2* S, int p, double2* dst, bool dfa, std::vector<double>& theta_max,
               cudaStream_t s) {
  Work& W = ctx->W;
  const int G = W.G;
  const Level& L0 = ctx->H.lev[0];
  const Roles R{{S, S, S}, p, W.D};
  gram_groups(L0, ctx->K.d_ph, R, p, G, W.GM, W.GA, W.gpart, W.gpart_cap, dfa, s);
  small_rr(W.GM, W.GA, p, p, W.C, W.theta, W.rr_scr, W.info, G, dfa, s);
  std::vector<int> info(8 * G);
  std::vector<double> th((size_t)G * p);
  PBS_CUDA(cudaMemcpyAsync(info.data(), W.info, sizeof(int) * 8 * G, cudaMemcpyDeviceToHost, s));
  PBS_CUDA(cudaMemcpyAsync(th.data(), W.theta, sizeof(double) * G * p, cudaMemcpyDeviceToHost, s));
  PBS_CUDA(cudaStreamSynchronize(s));
  for (int g = 0; g < G; ++g) {
    if (info[8 * g] != 0)
      fail(PBS_ENUMERIC, info[8 * g] == -2 ? "non-finite Gram matrix"
                                           : info[8 * g] == -3 ? "Rayleigh-Ritz breakdown" : "trial space lost rank");
    double tm = 0.0;
    for (int j = 0; j < p; ++j) tm = std::max(tm, std::fabs(th[(size_t)g * p + j]));
    theta_max[g] = tm;
  }
  block_update(R, p, W.C, p, (long)p * p, dst, W.D, p, nullptr, 0, W.D, G, false, s);
}

void init_random_all(pbs_ctx* ctx, const pbs_opts& o, std::vector<Group>& gr, cudaStream_t s) {
  Work& W = ctx->W;
  const int p = o.block, G = W.G;
  const long D = W.D;
  const bool dfa = o.precision == PBS_MIXED;
  double2* X0 = W.W();  // G p columns each
  double2* X1 = W.R();
  double2* Y = W.P();
  for (int g = 0; g < G; ++g) random_block(X0 + (long)g * p * D, D, D, p, o.seed, s);
  const int cyc = projection_cycles(o, 1e300, ctx->H.mu);
  std::vector<double> tm(G, 0.0);
  project_dispatch(ctx, o, ctx->K, X0, G * p, p, cyc, s);
  rr_groups(ctx, X0, p, X1, dfa, tm, s);
  for (int step = 0; step < 2; ++step) {
    apply_edge<double>(ctx->H.lev[0], ctx->K.d_ph, p, X1, Y, nullptr, D, G * p, 0.0, 1.0, 0.0, nullptr, 0.0, s);
    precondition_dispatch(ctx, o, ctx->K, Y, X0, G * p, p, s);
    project_dispatch(ctx, o, ctx->K, X0, G * p, p, cyc, s);
    rr_groups(ctx, X0, p, step == 1 ? W.E() : X1, dfa, tm, s);
  }
  PBS_CUDA(cudaMemsetAsync(W.P(), 0, sizeof(double2) * D * G * p, s));
  for (int g = 0; g < G; ++g) {
    gr[g].theta_max = tm[g];
    gr[g].it = 0;
    gr[g].have_p = false;
    gr[g].need_init = false;
  }
}

struct PathResult {
  std::vector<double> lam, res;  // nk x nev
  std::vector<int> iters;
  bool all_converged = true;
};

// Solve the Bloch vectors ks[0..nk) as `nchains` contiguous chains, one group per
// chain iterating in lock-step (Algorithm 2 for every group at once); each k of a
// chain after its first starts from the extrapolation of that chain's previous
// bases (Section 6).  A group whose k converged records it and restarts on the next
// k of its chain while the other groups keep iterating.
const double2* nested_blocks(pbs_ctx* ctx, const pbs_opts& o, int G, const std::vector<double>& kfirst);

// A chain of Bloch vectors solved in order by one group (Section 6): `idx` indexes
// the k list; `seeds` (device blocks of p columns, newest first, at most
// extrap_depth) are the bases its first Bloch vector is extrapolated from (none:
// a start block); save[t] >= 0 copies the converged block of its t-th Bloch vector
// into slot save[t] of the caller's store (p columns per slot).
struct Chain {
  std::vector<int> idx;
  std::vector<const double2*> seeds;
  std::vector<int> save;
};

// Eigenvectors of selected Bloch vectors copied out as they converge: slot[k] >= 0
// sends the nev wanted columns of Bloch vector k, M-normalised, to host + slot[k] nev D.
struct VecOut {
  std::vector<int> slot;
  pbs_c64* host = nullptr;
};

// Solve every chain of the list with G groups in lock-step; a group whose chain is
// done takes the next chain of the list.
PathResult solve_chain_list(pbs_ctx* ctx, const pbs_opts& o, int nk, const double* ks, const std::vector<Chain>& chains,
                            int Gwant, const pbs_c64* init, const double2* dev_init, double2* store,
                            const VecOut* vout = nullptr);

PathResult solve_chains(pbs_ctx* ctx, const pbs_opts& o, int nk, const double* ks, int nchains, const pbs_c64* init,
                        const double2* dev_init = nullptr, const VecOut* vout = nullptr) {
  const int G = std::max(1, std::min(nchains, nk));
  std::vector<Chain> chains(G);
  for (int g = 0; g < G; ++g)
    for (int i = (int)((long)nk * g / G); i <= (int)((long)nk * (g + 1) / G) - 1; ++i) chains[g].idx.push_back(i);
  return solve_chain_list(ctx, o, nk, ks, chains, G, init, dev_init, nullptr, vout);
}

PathResult solve_chain_list(pbs_ctx* ctx, const pbs_opts& o, int nk, const double* ks, const std::vector<Chain>& chains,
                            int Gwant, const pbs_c64* init, const double2* dev_init, double2* store,
                            const VecOut* vout) {
  for (long t = 0; t < 2L * nk; ++t)
    if (!std::isfinite(ks[t])) fail(PBS_EINVAL, "Bloch vectors must be finite");
  cudaStream_t s = ctx->stream;
  const bool dfa = o.precision == PBS_MIXED;
  const int p = o.block, G = std::max(1, std::min<int>(Gwant, (int)chains.size()));
  alloc_kdata(ctx->mem, ctx->H, ctx->K, G);
  // history slots per group: the extrapolation depth, when some chain has a second
  // Bloch vector or seeds
  bool chained = false;
  for (const Chain& c : chains) chained = chained || c.idx.size() > 1 || !c.seeds.empty();
  chained = chained && o.extrap_depth > 0;
  ensure_work(ctx, p, G, o.precision, chained ? (long)o.extrap_depth * G * p : 0);
  Work& W = ctx->W;
  W.graphs->clear();  // graphs hold pointers of this solve's tables only
  const Level& L0 = ctx->H.lev[0];
  const long D = W.D, Gp = (long)G * p;
  const double mu = ctx->H.mu;
  PathResult out;
  out.lam.assign((long)nk * o.nev, 0.0);
  out.res.assign((long)nk * o.nev, 0.0);
  out.iters.assign(nk, 0);
  std::vector<Group> gr(G);
  std::vector<double> kfirst(2 * G);
  int next_chain = G;
  // the seeds of group g's chain become its history (newest first)
  auto seed_history = [&](int g) {
    Group& x = gr[g];
    x.nhist = 0;
    if (!W.hist) return;
    const Chain& c = chains[x.chain];
    const int ns = std::min<int>((int)c.seeds.size(), o.extrap_depth);
    double2* hg = W.hist + (long)g * o.extrap_depth * p * D;
    for (int t = 0; t < ns; ++t)
      PBS_CUDA(cudaMemcpyAsync(hg + D * p * t, c.seeds[t], sizeof(double2) * D * p, cudaMemcpyDeviceToDevice, s));
    x.nhist = ns;
  };
  for (int g = 0; g < G; ++g) {
    gr[g].chain = g;
    gr[g].t = 0;
    gr[g].pos = chains[g].idx[0];
    gr[g].active = true;
    kfirst[2 * g] = ks[2 * gr[g].pos];
    kfirst[2 * g + 1] = ks[2 * gr[g].pos + 1];
    set_group_k(ctx->mem, ctx->H, ctx->K, g, kfirst[2 * g], kfirst[2 * g + 1], s);
    seed_history(g);
  }
  // first Bloch vector of every chain: seeds, a given block, the nested iteration, or a
  // smoothed random start
  const double2* first = dev_init;
  if (!first && !init && o.start == PBS_START_NESTED) first = nested_blocks(ctx, o, G, kfirst);
  bool all_random = !first && !init;
  for (int g = 0; g < G && all_random; ++g) all_random = gr[g].nhist == 0;
  if (all_random && G > 1) {
    init_random_all(ctx, o, gr, s);  // every group from a smoothed random start, batched
  } else {
    for (int g = 0; g < G; ++g)
      init_group(ctx, o, gr[g], g, g == 0 ? init : nullptr, s, first ? first + (long)g * p * D : nullptr);
  }
  std::vector<double> h_norms(2 * Gp), h_lam(Gp);
  const double lam_max = lambda_max_bound(ctx->H);
  std::vector<int> h_info(8 * G);
  const int q = 3 * p;
  int Ga = G;       // groups in the launches: the active ones, moved to the front
  long Gpa = Gp;
  // group src's state into slot dst (whose own group is finished): E, P, the residual
  // of this round (FP32 R32 under the mixed policy), the history ring and the tables
  auto move_group = [&](int src, int dst, float2* R32) {
    const size_t cb = sizeof(double2) * D * p;
    const long so = (long)src * p * D, d0 = (long)dst * p * D;
    PBS_CUDA(cudaMemcpyAsync(W.E() + d0, W.E() + so, cb, cudaMemcpyDeviceToDevice, s));
    PBS_CUDA(cudaMemcpyAsync(W.P() + d0, W.P() + so, cb, cudaMemcpyDeviceToDevice, s));
    if (R32) PBS_CUDA(cudaMemcpyAsync(R32 + d0, R32 + so, sizeof(float2) * D * p, cudaMemcpyDeviceToDevice, s));
    else PBS_CUDA(cudaMemcpyAsync(W.R() + d0, W.R() + so, cb, cudaMemcpyDeviceToDevice, s));
    if (W.hist) {
      const long hs = (long)o.extrap_depth * p * D;
      PBS_CUDA(cudaMemcpyAsync(W.hist + dst * hs, W.hist + src * hs, sizeof(double2) * hs, cudaMemcpyDeviceToDevice, s));
    }
    copy_group_k(ctx->K, src, dst, s);
    gr[dst] = gr[src];
  };
  for (int round = 0;; ++round) {
    bool any = false;
    for (auto& x : gr) any = any || x.active;
    if (!any) break;
    if (ctx->cancel && ctx->cancel->load(std::memory_order_relaxed)) fail(PBS_ECANCELED, "job cancelled");
    int cyc = o.nodal_cycles;
    for (auto& x : gr)
      if (x.active) cyc = std::max(cyc, projection_cycles(o, x.theta_max, mu));
    // Rayleigh-Ritz prefers combinations whose leftover gradient lowers the quotient,
    // so E and P are cleaned before the residual (Section 4, null-space elimination)
    if (round > 0) {
      // E and P are adjacent quarters: one pass while every group is launched, else two
      if (Ga == G) {
        run_graph(ctx, graph_key("project", W.E(), nullptr, 2 * (int)Gpa, p, cyc, ctx->K, o.precision), s,
                  [&] { project_dispatch(ctx, o, ctx->K, W.E(), 2 * (int)Gpa, p, cyc, s); });
      } else {
        for (double2* X : {W.E(), W.P()})
          run_graph(ctx, graph_key("project", X, nullptr, (int)Gpa, p, cyc, ctx->K, o.precision), s,
                    [&] { project_dispatch(ctx, o, ctx->K, X, (int)Gpa, p, cyc, s); });
      }
    }
    // Rayleigh quotients in factored form, then the FP64 residual
    rayleigh_parts(L0, ctx->K.d_ph, p, W.E(), D, (int)Gpa, W.parts, W.rq, dfa, s);
    k_rq<<<nblocks(Gpa), 256, 0, s>>>(W.rq, W.lam, (int)Gpa);
    PBS_LAUNCHED();
    // mixed: R in FP32 over the first half of the R block (the preconditioner's input)
    float2* R32 = reinterpret_cast<float2*>(W.R());
    if (dfa) residual_mixed(L0, ctx->K.d_ph, p, W.E(), R32, D, (int)Gpa, W.lam, W.parts, W.norms, s);
    else residual(L0, ctx->K.d_ph, p, W.E(), W.R(), D, (int)Gpa, W.lam, W.parts, W.norms, s);
    PBS_CUDA(cudaMemcpyAsync(h_norms.data(), W.norms, 2 * Gpa * sizeof(double), cudaMemcpyDeviceToHost, s));
    PBS_CUDA(cudaMemcpyAsync(h_lam.data(), W.lam, Gpa * sizeof(double), cudaMemcpyDeviceToHost, s));
    PBS_CUDA(cudaStreamSynchronize(s));
    timer_collect();
    std::vector<char> cont(Ga, 0);
    for (int g = 0; g < Ga; ++g) {
      Group& x = gr[g];
      if (!x.active) continue;
      bool conv = true;
      double tm = 0.0;
      std::vector<double> res(o.nev);
      for (int j = 0; j < p; ++j) tm = std::max(tm, std::fabs(h_lam[(long)g * p + j]));
      for (int j = 0; j < o.nev; ++j) {
        const long c = (long)g * p + j;
        const double r = std::sqrt(h_norms[2 * c]) / (std::fabs(h_lam[c]) * std::sqrt(h_norms[2 * c + 1]));
        if (!std::isfinite(r) || !std::isfinite(h_lam[c])) fail(PBS_ENUMERIC, "non-finite residual");
        res[j] = r;
        conv = conv && r <= band_tol(o.tol, lam_max, h_lam[c]);
      }
      x.theta_max = tm;
      if (verbose()) {
        std::fprintf(stderr, "[pbs] g=%d k=(%.6f,%.6f) it=%d", g, ctx->K.k1[g], ctx->K.k2[g], x.it);
        for (int j = 0; j < p; ++j) {
          const long c = (long)g * p + j;
          std::fprintf(stderr, " %.10g/%.1e", h_lam[c],
                       std::sqrt(h_norms[2 * c]) / (std::fabs(h_lam[c]) * std::sqrt(h_norms[2 * c + 1])));
        }
        std::fprintf(stderr, "\n");
      }
      if (conv || x.it >= o.max_iter) {
        // reported eigenvalues: the wanted bands' Rayleigh quotients in FP64 (the
        // iteration's double-float quotients of the mixed policy carry about
        // sqrt(lambda_max / lambda) 2^-47 relative error, 5e-10 next to Gamma at 1024^2)
        std::vector<double> lam_out(o.nev);
        for (int j = 0; j < o.nev; ++j) lam_out[j] = h_lam[(long)g * p + j];
        if (dfa) {
          const KData Kv = kdata_view(ctx->K, g);
          rayleigh_parts(L0, Kv.d_ph, o.nev, W.E() + (long)g * p * D, D, o.nev, W.parts, W.rq, false, s);
          std::vector<double> rq(2 * o.nev);
          PBS_CUDA(cudaMemcpyAsync(rq.data(), W.rq, rq.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
          PBS_CUDA(cudaStreamSynchronize(s));
          for (int j = 0; j < o.nev; ++j) lam_out[j] = rq[2 * j + 1] / rq[2 * j];
        }
        for (int j = 0; j < o.nev; ++j) {
          out.lam[(long)x.pos * o.nev + j] = lam_out[j];
          out.res[(long)x.pos * o.nev + j] = res[j];
        }
        if (vout && vout->slot[x.pos] >= 0) {
          // M-normalised copy of the wanted columns (the iterate itself stays as it is)
          const KData Kv = kdata_view(ctx->K, g);
          double2* V = W.init;
          PBS_CUDA(cudaMemcpyAsync(V, W.E() + (long)g * p * D, sizeof(double2) * D * o.nev, cudaMemcpyDeviceToDevice, s));
          rayleigh_parts(L0, Kv.d_ph, o.nev, V, D, o.nev, W.parts, W.rq, false, s);
          std::vector<double> rq(2 * o.nev), sc(o.nev);
          PBS_CUDA(cudaMemcpyAsync(rq.data(), W.rq, rq.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
          PBS_CUDA(cudaStreamSynchronize(s));
          for (int j = 0; j < o.nev; ++j) sc[j] = 1.0 / std::sqrt(rq[2 * j]);
          PBS_CUDA(cudaMemcpyAsync(W.norms, sc.data(), o.nev * sizeof(double), cudaMemcpyHostToDevice, s));
          scale_columns(V, D, D, o.nev, W.norms, s);
          PBS_CUDA(cudaMemcpyAsync(vout->host + (long)vout->slot[x.pos] * o.nev * D, V, sizeof(double2) * D * o.nev,
                                   cudaMemcpyDeviceToHost, s));
          PBS_CUDA(cudaStreamSynchronize(s));
        }
        out.iters[x.pos] = x.it;
        if (!conv) out.all_converged = false;
        const Chain& ch = chains[x.chain];
        if (store && x.t < (int)ch.save.size() && ch.save[x.t] >= 0)
          PBS_CUDA(cudaMemcpyAsync(store + (long)ch.save[x.t] * p * D, W.E() + (long)g * p * D,
                                   sizeof(double2) * D * p, cudaMemcpyDeviceToDevice, s));
        const bool more = x.t + 1 < (int)ch.idx.size();
        // history ring of the chain (newest first; oldest slot first, so no copy overlaps)
        if (W.hist && more) {
          const int depth = o.extrap_depth;
          double2* hg = W.hist + (long)g * depth * p * D;
          const int keep = std::min(x.nhist, depth - 1);
          for (int slot = keep; slot >= 1; --slot)
            PBS_CUDA(cudaMemcpyAsync(hg + D * p * slot, hg + D * p * (slot - 1), sizeof(double2) * D * p,
                                     cudaMemcpyDeviceToDevice, s));
          PBS_CUDA(cudaMemcpyAsync(hg, W.E() + (long)g * p * D, sizeof(double2) * D * p, cudaMemcpyDeviceToDevice, s));
          x.nhist = std::min(x.nhist + 1, depth);
        }
        if (more) {
          x.t += 1;
          x.pos = ch.idx[x.t];
          x.need_init = true;
        } else if (next_chain < (int)chains.size()) {
          // the next chain of the list, started from its own seeds
          x.chain = next_chain++;
          x.t = 0;
          x.pos = chains[x.chain].idx[0];
          seed_history(g);
          x.need_init = true;
        } else {
          x.active = false;
        }
      } else {
        cont[g] = 1;
      }
    }
    // groups with nothing left to solve leave the launches: the last active group moves
    // into each hole below the new count (E, P, this round's residual, history, tables),
    // so the rest of this round and the later rounds cover the active groups only
    {
      int na = 0;
      for (int g = 0; g < Ga; ++g) na += gr[g].active ? 1 : 0;
      int src = Ga - 1;
      for (int dst = 0; dst < na; ++dst) {
        if (gr[dst].active) continue;
        while (!gr[src].active) --src;  // an active group above na exists for every hole below it
        move_group(src, dst, dfa ? reinterpret_cast<float2*>(W.R()) : nullptr);
        cont[dst] = cont[src];
        gr[src].active = false;
        --src;
      }
      Ga = na;
      Gpa = (long)Ga * p;
    }
    bool any_cont = false;
    for (char c : cont) any_cont = any_cont || c;
    if (any_cont) {
      // W = B R, projected; Gram matrices of [E, P, W] per group; Rayleigh-Ritz; update
      double2* Wd = W.W();
      run_graph(ctx, graph_key("precondition", W.R(), Wd, (int)Gpa, p, 0, ctx->K, o.precision), s,
                [&] { precondition_dispatch(ctx, o, ctx->K, W.R(), Wd, (int)Gpa, p, s, dfa ? R32 : nullptr); });
      if (o.span == 1) {  // PINVIT (Algorithm 1): the trial block is E_hat = E - B R alone
        k_sub_from<<<nblocks(D * Gpa), 256, 0, s>>>(W.E(), Wd, D * Gpa);
        PBS_LAUNCHED();
      }
      run_graph(ctx, graph_key("project", Wd, nullptr, (int)Gpa, p, cyc, ctx->K, o.precision), s,
                [&] { project_dispatch(ctx, o, ctx->K, Wd, (int)Gpa, p, cyc, s); });
      // trial block per group: [E, P, W] (span 3; P = 0 until a search direction
      // exists, and always for span 2, so its columns are dropped) or [E_hat] (span 1)
      const Roles trial = o.span == 1 ? Roles{{Wd, Wd, Wd}, p, D} : Roles{{W.E(), W.P(), W.W()}, p, D};
      const int qt = o.span == 1 ? p : q;
      gram_groups(L0, ctx->K.d_ph, trial, qt, Ga, W.GM, W.GA, W.gpart, W.gpart_cap, dfa, s);
      small_rr(W.GM, W.GA, qt, p, W.C, W.theta, W.rr_scr, W.info, Ga, dfa, s);
      PBS_CUDA(cudaMemcpyAsync(h_info.data(), W.info, sizeof(int) * 8 * Ga, cudaMemcpyDeviceToHost, s));
      PBS_CUDA(cudaStreamSynchronize(s));
      for (int g = 0; g < Ga; ++g) {
        if (!cont[g] || h_info[8 * g] == 0) continue;
        if (h_info[8 * g] == -2) fail(PBS_ENUMERIC, "non-finite Gram matrix");
        if (h_info[8 * g] == -3) fail(PBS_ENUMERIC, "Rayleigh-Ritz breakdown");
        if (o.span != 3 || !gr[g].have_p) fail(PBS_ENUMERIC, "trial space lost rank");
        // rank loss in the LOBPCG basis: restart this group without the search direction
        PBS_CUDA(cudaMemsetAsync(W.P() + (long)g * p * D, 0, sizeof(double2) * D * p, s));
        const KData Kv = kdata_view(ctx->K, g);
        const Roles tg{{W.E() + (long)g * p * D, W.P() + (long)g * p * D, W.W() + (long)g * p * D}, p, D};
        double2* GMg = W.GM + (long)g * q * q;
        double2* GAg = W.GA + (long)g * q * q;
        gram_groups(L0, Kv.d_ph, tg, q, 1, GMg, GAg, W.gpart, W.gpart_cap, dfa, s);
        small_rr(GMg, GAg, q, p, W.C + (long)g * q * p, W.theta + (long)g * q, W.rr_scr, W.info + 8 * g, 1, dfa, s);
        int inf2[2];
        PBS_CUDA(cudaMemcpyAsync(inf2, W.info + 8 * g, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
        PBS_CUDA(cudaStreamSynchronize(s));
        if (inf2[0] != 0) fail(PBS_ENUMERIC, "trial space lost rank");
      }
      if (o.span == 1) {
        // E_new = E_hat C over the old E (E_hat lives in W); P stays zero
        block_update(trial, p, W.C, p, (long)p * p, W.E(), D, p, nullptr, 0, D, Ga, false, s);
        PBS_CUDA(cudaMemsetAsync(W.P(), 0, sizeof(double2) * D * Gpa, s));
      } else {
        // P_new = [P, W] C[p:q] over R, E_new = E C[0:p] + P_new over W, then the
        // halves swap roles (new E, P = old W, R blocks)
        double2* P2 = W.R();
        double2* E2 = W.W();
        const Roles pw{{W.P(), W.W(), W.W()}, p, D};
        block_update(pw, 2 * p, W.C + p, q, (long)q * p, P2, D, p, nullptr, 0, D, Ga, dfa, s);
        const Roles ee{{W.E(), W.E(), W.E()}, p, D};
        block_update(ee, p, W.C, q, (long)q * p, E2, D, p, P2, D, D, Ga, false, s);
        W.half = 1 - W.half;
        if (o.span == 2) PBS_CUDA(cudaMemsetAsync(W.P(), 0, sizeof(double2) * D * Gpa, s));  // gradient method: no P
      }
      for (int g = 0; g < Ga; ++g)
        if (cont[g]) {
          gr[g].have_p = true;
          gr[g].it += 1;
        }
    }
    // groups that moved to their next Bloch vector
    for (int g = 0; g < Ga; ++g) {
      if (!gr[g].need_init) continue;
      set_group_k(ctx->mem, ctx->H, ctx->K, g, ks[2 * gr[g].pos], ks[2 * gr[g].pos + 1], s);
      init_group(ctx, o, gr[g], g, nullptr, s);
    }
  }
  return out;
}

// single-group tables for the operator entry points
// Nested iteration for the first Bloch vector of each chain (Section 6): the block
// iteration on the coarsest hierarchy level with at least 16 x 16 cells (the
// "direct" solve: run there to the requested tolerance), then level by level the
// converged blocks are prolongated by the natural embedding (Section 5) and iterated
// on the next finer mesh to a relative residual of 1e-3 (the mesh change itself
// moves eigenvectors by about that much), all chains together.  The coarse meshes
// carry the hierarchy's averaged 1/eps.  Returns the prolongated level-1 blocks on
// level 0 (G groups of p columns in the R block), or null when the mesh has no
// coarse level of that size (then random starts are used).
struct ChildCtxs {
  std::vector<pbs_ctx*> c;
  ~ChildCtxs() {
    for (pbs_ctx* x : c)
      if (x) pbs_destroy(x);
  }
};

const double2* nested_blocks(pbs_ctx* ctx, const pbs_opts& o, int G, const std::vector<double>& kfirst) {
  const Hierarchy& H = ctx->H;
  int lc = 0;
  for (int l = 1; l < H.nlev; ++l)
    if (H.lev[l].n >= 16 && H.lev[l].m >= 16) lc = l;
  if (lc == 0) return nullptr;
  cudaStream_t s = ctx->stream;
  Work& W = ctx->W;
  const int p = o.block;
  ChildCtxs kids;
  kids.c.assign(lc + 1, nullptr);
  const double2* prev = nullptr;  // prolongated blocks on level l (device), none on the coarsest
  for (int l = lc; l >= 1; --l) {
    const Level& L = H.lev[l];
    std::vector<double> winv(L.N()), eps(L.N());
    PBS_CUDA(cudaMemcpyAsync(winv.data(), L.winv64, sizeof(double) * L.N(), cudaMemcpyDeviceToHost, s));
    PBS_CUDA(cudaStreamSynchronize(s));
    for (long t = 0; t < L.N(); ++t) eps[t] = 1.0 / winv[t];
    if (pbs_create(&kids.c[l], ctx->device, 0) != PBS_OK) fail(PBS_ECUDA, "nested iteration: context");
    pbs_ctx* c = kids.c[l];
    const pbs_geom geom{H.a, H.b, L.n, L.m, eps.data()};
    pbs_opts ol = o;
    ol.start = PBS_START_RANDOM;
    ol.kbatch = G;
    ol.tol = l == lc ? o.tol : std::max(o.tol, 1e-3);
    ensure_hierarchy_host(c, &geom, H.mu, o.coarsest);
    solve_chains(c, ol, G, kfirst.data(), G, nullptr, prev);
    // natural embedding of the converged blocks into level l - 1, phases of each group
    PBS_CUDA(cudaStreamSynchronize(c->stream));
    prolong_edge<double>(H.lev[l - 1], L, ctx->K.d_ph, p, c->W.E(), L.D(), W.R(), H.lev[l - 1].D(), G * p, false,
                         s);
    PBS_CUDA(cudaStreamSynchronize(s));
    prev = W.R();
  }
  return W.R();
}

void set_single_k(pbs_ctx* ctx, double k1, double k2) {
  alloc_kdata(ctx->mem, ctx->H, ctx->K, 1);
  set_group_k(ctx->mem, ctx->H, ctx->K, 0, k1, k2, ctx->stream);
}

}  // namespace

namespace {
int run_guarded_impl(const std::function<void()>& f);

// Device bytes a path job needs on a context that holds nothing else: the
// geometry's hierarchy, the per-Bloch-vector coarsest factors and the solver
// workspace, as ensure_work and build_hierarchy allocate them (the nodal and edge
// multigrid work counted as 4/3 of three fine-level vectors per column).
double job_bytes(int n, int m, const pbs_opts& o, int nk, size_t budget) {
  const int nl = num_levels(n, m, o.coarsest);
  double hb = 0.0;
  for (int l = 0; l < nl; ++l) hb += (double)(n >> l) * (m >> l) * (8 + 4 + 48 + 24);
  const double N = (double)n * m, D = 2.0 * N;
  hb += 8.0 * N + 8.0 * N;  // level-0 double-float weights, device copy of eps
  const double Nc = (double)(n >> (nl - 1)) * (m >> (nl - 1)), Dc = 2.0 * Nc;
  const int G = std::max(1, std::min(o.kbatch, nk)), p = o.block, q = 3 * p;
  const double Gp = (double)G * p;
  const double kd = G * (Dc * Dc + Nc * Nc) * (16.0 + 8.0);
  const int ck = chunk_columns(D, N, p, q, (long)std::max<double>(2 * Gp, q), o.precision, chunk_bytes(budget));
  const double cxb = o.precision == PBS_MIXED ? 8.0 : 16.0;
  const bool chained = o.extrap_depth > 0 && nk > G;
  double wb = 16.0 * D * (4.0 * Gp + q) + (chained ? 16.0 * D * o.extrap_depth * Gp : 0.0);
  wb += 4.0 * N * ck * cxb + 4.0 * D * ck * cxb + 4.0 * N * ck * cxb;
  if (o.precision == PBS_MIXED) wb += 2.0 * D * ck * 8.0;
  wb += 16.0 * (3.0 * q * q * G) + 16.0 * (double)std::max(gram_partials_size((long)N, q, G),
                                                           gram_partials_size((long)N, q, 1)) +
        64.0 * D / 8.0 * std::max<double>(3 * Gp, q);
  return hb + kd + wb;
}

// Frees what an idle engine keeps resident (workspace, hierarchy, coarsest factors).
void release_engine(pbs_ctx* e) {
  std::lock_guard<std::mutex> g(e->gpu_mu);
  run_guarded_impl([&] {
    DeviceGuard dg(e->device);
    PBS_CUDA(cudaStreamSynchronize(e->stream));
    free_work(e);
    if (e->have_h) free_hierarchy(e->mem, e->H);
    e->have_h = false;
    e->H = Hierarchy();
    free_kdata(e->mem, e->K);
  });
}

// Next job for slot `me` (called with the server lock held); null when none fits now.
std::shared_ptr<Job> pick_job(Server& sv, Slot* me) {
  if (sv.queue.empty()) return nullptr;
  double others = 0.0, idle_resident = 0.0;
  for (auto& sl : sv.slots)
    if (sl.get() != me) {
      others += sl->held;
      if (!sl->job) idle_resident += sl->held;
    }
  auto fits = [&](const Job& j) { return others + j.est <= sv.cap; };
  const size_t window = std::min<size_t>(sv.queue.size(), 2 * (size_t)sv.nslots);
  std::shared_ptr<Job>& head = sv.queue.front();
  const bool head_only = head->bypassed >= 2 * sv.nslots;
  long pick = -1;
  if (fits(*head)) {
    pick = 0;
    // a job whose geometry is resident here saves a hierarchy build
    if (!head_only && head->gkey != me->resident)
      for (size_t i = 1; i < window; ++i)
        if (sv.queue[i]->gkey == me->resident && me->resident != 0 && fits(*sv.queue[i])) {
          pick = (long)i;
          break;
        }
  } else {
    // the head waits for memory: idle slots give up what they keep resident
    if (others - idle_resident + head->est <= sv.cap)
      for (auto& sl : sv.slots)
        if (sl.get() != me && !sl->job && sl->held > 0) sl->evict = true;
    if (!head_only)
      for (size_t i = 1; i < window; ++i)
        if (fits(*sv.queue[i])) {
          pick = (long)i;
          break;
        }
  }
  if (pick < 0) return nullptr;
  std::shared_ptr<Job> j = sv.queue[pick];
  if (pick > 0) head->bypassed += 1;
  sv.queue.erase(sv.queue.begin() + pick);
  return j;
}

// Host thread of one serving slot: runs jobs on the slot's engine as pbs_solve_path
// would and records their results and times.
void slot_loop(pbs_ctx* ctx, Slot* me) {
  cudaSetDevice(ctx->device);
  Server& sv = ctx->srv;
  std::unique_lock<std::mutex> lk(sv.m);
  for (;;) {
    if (sv.stop) return;
    if (me->evict) {
      me->evict = false;
      if (me->held > 0) {
        lk.unlock();
        release_engine(me->eng);
        lk.lock();
        me->held = (double)me->eng->mem.used();
        me->resident = 0;
        sv.cv_work.notify_all();
      }
      continue;
    }
    std::shared_ptr<Job> j = pick_job(sv, me);
    if (!j) {
      sv.cv_work.wait(lk);
      continue;
    }
    me->job = j;
    me->held = std::max(j->est, (double)me->eng->mem.used());
    j->started = true;
    j->t_start = std::chrono::steady_clock::now();
    if (!sv.queue.empty()) sv.cv_work.notify_all();  // another slot may take the next job
    lk.unlock();
    pbs_ctx* e = me->eng;
    int status = PBS_OK;
    const int rc = run_guarded_impl([&] {
      std::lock_guard<std::mutex> g(e->gpu_mu);
      DeviceGuard dg(e->device);
      TimerScope ts(e);
      e->cancel = &j->cancel;
      struct Reset {
        pbs_ctx* e;
        ~Reset() { e->cancel = nullptr; }
      } reset{e};
      const pbs_geom geom{j->a, j->b, j->n, j->m, j->eps.data()};
      ensure_hierarchy_host(e, &geom, effective_mu(j->o, j->a, j->b), j->o.coarsest);
      const PathResult r = solve_chains(e, j->o, j->nk, j->ks.data(), j->o.kbatch, nullptr);
      j->lam = r.lam;
      j->res = r.res;
      j->iters = r.iters;
      if (!r.all_converged) status = PBS_ENOCONV;
    });
    const std::string err = g_last_error;
    lk.lock();
    j->status = rc != PBS_OK ? rc : status;
    if (rc != PBS_OK) j->err = err;
    j->t_done = std::chrono::steady_clock::now();
    j->done = true;
    me->job.reset();
    me->held = (double)e->mem.used();
    me->resident = (rc == PBS_OK && e->have_h) ? j->gkey : 0;
    sv.cv_done.notify_all();
    sv.cv_work.notify_all();
  }
}

// Starts the slots of a context's server (first submission).
void start_server(pbs_ctx* ctx) {
  Server& sv = ctx->srv;
  if (sv.started) return;
  if (sv.cap <= 0) {
    DeviceGuard g(ctx->device);
    size_t fr = 0, tot = 0;
    PBS_CUDA(cudaMemGetInfo(&fr, &tot));
    sv.cap = ctx->mem.budget() > 0 ? (double)ctx->mem.budget() : 0.9 * (double)fr;
  }
  for (int i = 0; i < sv.nslots; ++i) {
    auto sl = std::make_unique<Slot>();
    pbs_ctx* e = nullptr;
    const int rc = pbs_create(&e, ctx->device, 0);
    if (rc != PBS_OK) fail(rc, "serving slot: " + std::string(pbs_last_error()));
    e->timer.mask = 0;
    sl->eng = e;
    sv.slots.push_back(std::move(sl));
  }
  for (auto& sl : sv.slots) sl->th = std::thread(slot_loop, ctx, sl.get());
  sv.started = true;
}
}  // namespace

namespace {
int run_guarded_impl(const std::function<void()>& f) {
  try {
    g_last_error.clear();
    f();
    return PBS_OK;
  } catch (const Error& e) {
    g_last_error = e.what;
    return e.status;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return PBS_ENOMEM;
  } catch (...) {
    g_last_error = "unexpected failure";
    return PBS_ECUDA;
  }
}
}  // namespace

extern "C" {

const char* pbs_strerror(int status) {
  switch (status) {
    case PBS_OK: return "ok";
    case PBS_EINVAL: return "invalid argument";
    case PBS_ENOMEM: return "out of device memory or over the budget";
    case PBS_ENOCONV: return "not converged within max_iter";
    case PBS_ENUMERIC: return "numerical breakdown";
    case PBS_ETIMEOUT: return "device wait timed out";
    case PBS_ECUDA: return "CUDA error";
    case PBS_ECANCELED: return "job cancelled";
    default: return "unknown status";
  }
}

const char* pbs_last_error(void) { return g_last_error.c_str(); }

void pbs_default_opts(pbs_opts* o) {
  if (!o) return;
  o->nev = 4;
  o->block = 6;
  o->max_iter = 400;
  o->precision = PBS_MIXED;
  o->span = 3;
  o->tol = 1e-8;
  o->mu = 0.0;
  o->nu_pre = 1;
  o->nu_post = 1;
  o->coarsest = 4;
  o->nodal_cycles = 2;
  o->extrap_depth = 3;
  o->seed = 0;
  o->kbatch = 1;
  o->start = PBS_START_RANDOM;
}

int pbs_num_levels(int n, int m, int coarsest) {
  if (n < 2 || m < 2 || coarsest < 2) return PBS_EINVAL;
  return num_levels(n, m, coarsest);
}

int pbs_create(pbs_ctx** ctx, int device, size_t hbm_budget_bytes) {
  if (!ctx) return PBS_EINVAL;
  *ctx = nullptr;
  return run_guarded_impl([&] {
    int count = 0;
    PBS_CUDA(cudaGetDeviceCount(&count));
    if (device < 0 || device >= count || device >= kMaxDevices) fail(PBS_EINVAL, "no such CUDA device");
    DeviceGuard g(device);
    std::unique_ptr<pbs_ctx> c(new pbs_ctx(hbm_budget_bytes));
    c->device = device;
    PBS_CUDA(cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking));
    *ctx = c.release();
  });
}

int pbs_destroy(pbs_ctx* ctx) {
  if (!ctx) return PBS_OK;
  {
    // running jobs finish; queued jobs are dropped
    std::lock_guard<std::mutex> lk(ctx->srv.m);
    ctx->srv.stop = true;
  }
  ctx->srv.cv_work.notify_all();
  for (auto& sl : ctx->srv.slots) {
    if (sl->th.joinable()) sl->th.join();
    pbs_destroy(sl->eng);
    sl->eng = nullptr;
  }
  ctx->srv.slots.clear();
  return run_guarded_impl([&] {
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    free_work(ctx);
    if (ctx->have_h) free_hierarchy(ctx->mem, ctx->H);
    free_kdata(ctx->mem, ctx->K);
    ctx->mem.free(ctx->d_eps_in);
    for (auto& ev : ctx->timer.pool) {
      cudaEventDestroy(ev.first);
      cudaEventDestroy(ev.second);
    }
    cudaStreamDestroy(ctx->stream);
    delete ctx;
  });
}


int pbs_solve_k(pbs_ctx* ctx, const pbs_geom* geom, const pbs_opts* opts, const double k[2], const pbs_c64* init,
                double* eigvals, double* resid, int* iters, pbs_c64* evecs) {
  if (!ctx || !geom || !opts || !k || !eigvals || !resid || !iters) return PBS_EINVAL;
  int status = PBS_OK;
  const int rc = run_guarded_impl([&] {
    std::lock_guard<std::mutex> ctx_lock(ctx->gpu_mu);
    DeviceGuard g(ctx->device);
    TimerScope ts(ctx);
    pbs_opts o = *opts;
    validate_opts(o);
    ensure_hierarchy_host(ctx, geom, effective_mu(o, geom->a, geom->b), o.coarsest);
    const PathResult r = solve_chains(ctx, o, 1, k, 1, init);
    for (int j = 0; j < o.nev; ++j) {
      eigvals[j] = r.lam[j];
      resid[j] = r.res[j];
    }
    *iters = r.iters[0];
    if (evecs) {
      // M-normalise the returned columns
      Work& W = ctx->W;
      std::vector<double> rq(2 * o.block), sc(o.block);
      rayleigh_parts(ctx->H.lev[0], ctx->K.d_ph, o.block, W.E(), W.D, o.block, W.parts, W.rq, o.precision == PBS_MIXED,
                     ctx->stream);
      PBS_CUDA(cudaMemcpyAsync(rq.data(), W.rq, 2 * o.block * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
      PBS_CUDA(cudaStreamSynchronize(ctx->stream));
      for (int j = 0; j < o.block; ++j) sc[j] = 1.0 / std::sqrt(rq[2 * j]);
      PBS_CUDA(cudaMemcpyAsync(W.lam, sc.data(), o.block * sizeof(double), cudaMemcpyHostToDevice, ctx->stream));
      scale_columns(W.E(), W.D, W.D, o.nev, W.lam, ctx->stream);
      PBS_CUDA(cudaMemcpyAsync(evecs, W.E(), sizeof(double2) * W.D * o.nev, cudaMemcpyDeviceToHost, ctx->stream));
      PBS_CUDA(cudaStreamSynchronize(ctx->stream));
    }
    if (!r.all_converged) status = PBS_ENOCONV;
  });
  return rc != PBS_OK ? rc : status;
}

int pbs_solve_path(pbs_ctx* ctx, const pbs_geom* geom, const pbs_opts* opts, int nk, const double* ks,
                   double* eigvals, double* resid, int* iters) {
  if (!ctx || !geom || !opts || nk < 0 || (nk > 0 && (!ks || !eigvals || !resid || !iters))) return PBS_EINVAL;
  int status = PBS_OK;
  const int rc = run_guarded_impl([&] {
    std::lock_guard<std::mutex> ctx_lock(ctx->gpu_mu);
    DeviceGuard g(ctx->device);
    TimerScope ts(ctx);
    validate_opts(*opts);
    if (nk == 0) return;
    ensure_hierarchy_host(ctx, geom, effective_mu(*opts, geom->a, geom->b), opts->coarsest);
    const PathResult r = solve_chains(ctx, *opts, nk, ks, opts->kbatch, nullptr);
    std::copy(r.lam.begin(), r.lam.end(), eigvals);
    std::copy(r.res.begin(), r.res.end(), resid);
    std::copy(r.iters.begin(), r.iters.end(), iters);
    if (!r.all_converged) status = PBS_ENOCONV;
  });
  return rc != PBS_OK ? rc : status;
}

int pbs_solve_path_vectors(pbs_ctx* ctx, const pbs_geom* geom, const pbs_opts* opts, int nk, const double* ks,
                           double* eigvals, double* resid, int* iters, int nsel, const int* sel, pbs_c64* evecs) {
  if (!ctx || !geom || !opts || nk < 0 || nsel < 0 || (nk > 0 && (!ks || !eigvals || !resid || !iters)) ||
      (nsel > 0 && (!sel || !evecs)))
    return PBS_EINVAL;
  int status = PBS_OK;
  const int rc = run_guarded_impl([&] {
    std::lock_guard<std::mutex> ctx_lock(ctx->gpu_mu);
    DeviceGuard g(ctx->device);
    TimerScope ts(ctx);
    validate_opts(*opts);
    VecOut vo;
    vo.slot.assign(nk, -1);
    vo.host = evecs;
    for (int t = 0; t < nsel; ++t) {
      if (sel[t] < 0 || sel[t] >= nk) fail(PBS_EINVAL, "selected Bloch vector out of range");
      if (vo.slot[sel[t]] >= 0) fail(PBS_EINVAL, "a Bloch vector is selected twice");
      vo.slot[sel[t]] = t;
    }
    if (nk == 0) return;
    ensure_hierarchy_host(ctx, geom, effective_mu(*opts, geom->a, geom->b), opts->coarsest);
    const PathResult r = solve_chains(ctx, *opts, nk, ks, opts->kbatch, nullptr, nullptr, nsel > 0 ? &vo : nullptr);
    std::copy(r.lam.begin(), r.lam.end(), eigvals);
    std::copy(r.res.begin(), r.res.end(), resid);
    std::copy(r.iters.begin(), r.iters.end(), iters);
    if (!r.all_converged) status = PBS_ENOCONV;
  });
  return rc != PBS_OK ? rc : status;
}

int pbs_solve_path_device(pbs_ctx* ctx, double a, double b, int n, int m, const double* d_eps, const pbs_opts* opts,
                          int nk, const double* d_ks, double* d_eigvals, double* d_resid, int* d_iters,
                          void* cuda_stream) {
  if (!ctx || !opts || nk < 0 || !d_eps || (nk > 0 && (!d_ks || !d_eigvals || !d_resid || !d_iters)))
    return PBS_EINVAL;
  int status = PBS_OK;
  const int rc = run_guarded_impl([&] {
    std::lock_guard<std::mutex> ctx_lock(ctx->gpu_mu);
    DeviceGuard g(ctx->device);
    TimerScope ts(ctx);
    validate_opts(*opts);
    validate_mesh(a, b, n, m);
    cudaStream_t us = (cudaStream_t)cuda_stream;
    // order the library stream after the caller's work on the inputs
    cudaEvent_t ev;
    PBS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    PBS_CUDA(cudaEventRecord(ev, us));
    PBS_CUDA(cudaStreamWaitEvent(ctx->stream, ev, 0));
    cudaEventDestroy(ev);
    if (nk == 0) return;
    const uint64_t h = device_eps_hash(ctx, d_eps, (long)n * m);
    ensure_hierarchy(ctx, a, b, n, m, d_eps, h, effective_mu(*opts, a, b), opts->coarsest);
    std::vector<double> ks(2 * nk);
    PBS_CUDA(cudaMemcpyAsync(ks.data(), d_ks, sizeof(double) * 2 * nk, cudaMemcpyDeviceToHost, ctx->stream));
    PBS_CUDA(cudaStreamSynchronize(ctx->stream));
    const PathResult r = solve_chains(ctx, *opts, nk, ks.data(), opts->kbatch, nullptr);
    PBS_CUDA(cudaMemcpyAsync(d_eigvals, r.lam.data(), sizeof(double) * r.lam.size(), cudaMemcpyHostToDevice, ctx->stream));
    PBS_CUDA(cudaMemcpyAsync(d_resid, r.res.data(), sizeof(double) * r.res.size(), cudaMemcpyHostToDevice, ctx->stream));
    PBS_CUDA(cudaMemcpyAsync(d_iters, r.iters.data(), sizeof(int) * r.iters.size(), cudaMemcpyHostToDevice, ctx->stream));
    PBS_CUDA(cudaStreamSynchronize(ctx->stream));
    if (!r.all_converged) status = PBS_ENOCONV;
  });
  return rc != PBS_OK ? rc : status;
}

int pbs_apply(pbs_ctx* ctx, const pbs_geom* geom, const pbs_opts* opts, int op, int level, const double k[2],
              int ncols, const pbs_c64* x, pbs_c64* y, void* cuda_stream) {
  if (!ctx || !geom || !opts || !k || ncols < 0) return PBS_EINVAL;
  if (ncols > 0 && (!x || !y)) return PBS_EINVAL;
  return run_guarded_impl([&] {
    std::lock_guard<std::mutex> ctx_lock(ctx->gpu_mu);
    DeviceGuard g(ctx->device);
    TimerScope ts(ctx);
    const pbs_opts& o = *opts;
    if (o.precision != PBS_FP64 && o.precision != PBS_MIXED) fail(PBS_EINVAL, "unknown precision");
    if (o.coarsest < 2 || o.nodal_cycles < 1 || o.nu_pre < 0 || o.nu_post < 0) fail(PBS_EINVAL, "bad multigrid options");
    ensure_hierarchy_host(ctx, geom, effective_mu(o, geom->a, geom->b), o.coarsest);
    const Hierarchy& H = ctx->H;
    if (level < 0 || level >= H.nlev) fail(PBS_EINVAL, "level out of range");
    const bool transfer = op == PBS_OP_PROLONG || op == PBS_OP_RESTRICT || op == PBS_OP_PROLONG_NODAL ||
                          op == PBS_OP_RESTRICT_NODAL;
    if (transfer && level + 1 >= H.nlev) fail(PBS_EINVAL, "no coarser level below `level`");
    if (op < PBS_OP_A || op > PBS_OP_LH_M) fail(PBS_EINVAL, "unknown operator");
    if (op == PBS_OP_PROJECT && level != 0) fail(PBS_EINVAL, "PROJECT acts on level 0");
    if (ncols == 0) return;
    set_single_k(ctx, k[0], k[1]);
    cudaStream_t us = (cudaStream_t)cuda_stream;
    cudaStream_t s = ctx->stream;
    cudaEvent_t ev;
    PBS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    PBS_CUDA(cudaEventRecord(ev, us));
    PBS_CUDA(cudaStreamWaitEvent(s, ev, 0));
    const Level& L = H.lev[level];
    const KData& K = ctx->K;
    const double mu = H.mu;
    const double2* X = (const double2*)x;
    double2* Y = (double2*)y;
    const long D = L.D(), N = L.N();
    const int cpg = ncols;
    switch (op) {
      case PBS_OP_A: apply_edge<double>(L, K.d_ph, cpg, X, Y, nullptr, D, ncols, 1.0, 0.0, 0.0, nullptr, 0.0, s); break;
      case PBS_OP_M: apply_edge<double>(L, K.d_ph, cpg, X, Y, nullptr, D, ncols, 0.0, 1.0, 0.0, nullptr, 0.0, s); break;
      case PBS_OP_A_MU_M: apply_edge<double>(L, K.d_ph, cpg, X, Y, nullptr, D, ncols, 1.0, mu, 0.0, nullptr, 0.0, s); break;
      case PBS_OP_C: apply_curl<double>(L, K.d_ph, cpg, X, D, Y, N, ncols, s); break;
      case PBS_OP_CH: apply_curl_adj<double>(L, K.d_ph, cpg, X, N, Y, D, ncols, s); break;
      case PBS_OP_L: apply_lift<double>(L, K.d_ph, cpg, X, N, Y, D, ncols, s); break;
      case PBS_OP_LH: apply_lift_adj<double>(L, K.d_ph, cpg, X, D, Y, N, ncols, s); break;
      case PBS_OP_P_NODAL: apply_nodal<double>(L, K.d_ph, cpg, X, Y, nullptr, N, ncols, 1.0, 0.0, s); break;
      case PBS_OP_LH_M:
        lift_adj_mass<double>(L, K.d_ph, cpg, X, D, Y, N, ncols, o.precision == PBS_MIXED, s);
        break;
      case PBS_OP_RESIDUAL: {
        // the iteration's residual kernel with Lambda = mu on every column; its
        // per-column norms go to scratch that lives for this call only
        const long nblk = ((L.n + 31) / 32) * ((L.m + 7) / 8);
        double* tmp = (double*)ctx->mem.alloc(sizeof(double) * (ncols + 2L * nblk * ncols + 2L * ncols));
        try {
          std::vector<double> lam(ncols, mu);
          PBS_CUDA(cudaMemcpyAsync(tmp, lam.data(), sizeof(double) * ncols, cudaMemcpyHostToDevice, s));
          residual(L, K.d_ph, cpg, X, Y, D, ncols, tmp, tmp + ncols, tmp + ncols + 2L * nblk * ncols, s);
          PBS_CUDA(cudaStreamSynchronize(s));
        } catch (...) {
          ctx->mem.free(tmp);
          throw;
        }
        ctx->mem.free(tmp);
        break;
      }
      case PBS_OP_PROLONG: {
        const Level& C = H.lev[level + 1];
        prolong_edge<double>(L, C, K.d_ph, cpg, X, C.D(), Y, D, ncols, false, s);
        break;
      }
      case PBS_OP_RESTRICT: {
        const Level& C = H.lev[level + 1];
        restrict_edge<double>(L, C, K.d_ph, cpg, X, D, Y, C.D(), ncols, s);
        break;
      }
      case PBS_OP_PROLONG_NODAL: {
        const Level& C = H.lev[level + 1];
        prolong_node<double>(L, C, K.d_ph, cpg, X, C.N(), Y, N, ncols, false, s);
        break;
      }
      case PBS_OP_RESTRICT_NODAL: {
        const Level& C = H.lev[level + 1];
        restrict_node<double>(L, C, K.d_ph, cpg, X, N, Y, C.N(), ncols, s);
        break;
      }
      case PBS_OP_VCYCLE_EDGE:
      case PBS_OP_VCYCLE_NODAL:
      case PBS_OP_PROJECT: {
        // temporary multigrid workspace for ncols columns
        const bool nodal = op == PBS_OP_VCYCLE_NODAL;
        const long len = nodal ? N : D;
        if (op == PBS_OP_PROJECT) {
          const int pw = std::max(1, (ncols + 2) / 3);
          if (pw > kMaxBlock) fail(PBS_EINVAL, "too many columns");
          ensure_work(ctx, pw, 1, o.precision, 0);
          PBS_CUDA(cudaMemcpyAsync(Y, X, sizeof(double2) * D * ncols, cudaMemcpyDeviceToDevice, s));
          project_dispatch(ctx, o, K, Y, ncols, ncols, o.nodal_cycles, s);
          PBS_CUDA(cudaStreamSynchronize(s));
          break;
        }
        if (o.precision == PBS_MIXED) {
          MgWork<float> w;
          float2* xf = (float2*)ctx->mem.alloc(sizeof(float2) * len * ncols);
          float2* yf = (float2*)ctx->mem.alloc(sizeof(float2) * len * ncols);
          try {
            alloc_mg_work<float>(ctx->mem, H, ncols, nodal, w);
            convert_d2f(X, xf, len * ncols, s);
            if (nodal) nodal_vcycle<float>(H, K, w, level, xf, yf, len, ncols, ncols, o.nu_pre, o.nu_post, s);
            else edge_vcycle<float>(H, K, w, level, xf, yf, len, ncols, ncols, o.nu_pre, o.nu_post, s);
            convert_f2d(yf, Y, len * ncols, s);
            PBS_CUDA(cudaStreamSynchronize(s));
          } catch (...) {
            free_mg_work<float>(ctx->mem, w);
            ctx->mem.free(xf);
            ctx->mem.free(yf);
            throw;
          }
          free_mg_work<float>(ctx->mem, w);
          ctx->mem.free(xf);
          ctx->mem.free(yf);
        } else {
          MgWork<double> w;
          try {
            alloc_mg_work<double>(ctx->mem, H, ncols, nodal, w);
            if (nodal) nodal_vcycle<double>(H, K, w, level, X, Y, len, ncols, ncols, o.nu_pre, o.nu_post, s);
            else edge_vcycle<double>(H, K, w, level, X, Y, len, ncols, ncols, o.nu_pre, o.nu_post, s);
            PBS_CUDA(cudaStreamSynchronize(s));
          } catch (...) {
            free_mg_work<double>(ctx->mem, w);
            throw;
          }
          free_mg_work<double>(ctx->mem, w);
        }
        break;
      }
      default: fail(PBS_EINVAL, "unknown operator");
    }
    // order the caller's stream after the library's work
    PBS_CUDA(cudaEventRecord(ev, s));
    PBS_CUDA(cudaStreamWaitEvent(us, ev, 0));
    PBS_CUDA(cudaStreamSynchronize(s));
    cudaEventDestroy(ev);
  });
}

int pbs_gram(pbs_ctx* ctx, const pbs_geom* geom, const double k[2], int q, const pbs_c64* S, pbs_c64* GM, pbs_c64* GA,
             int precision, void* cuda_stream) {
  if (!ctx || !geom || !k || q < 0 || q > kMaxTrial) return PBS_EINVAL;
  if (precision != PBS_FP64 && precision != PBS_MIXED) return PBS_EINVAL;
  if (q > 0 && (!S || !GM || !GA)) return PBS_EINVAL;
  return run_guarded_impl([&] {
    std::lock_guard<std::mutex> ctx_lock(ctx->gpu_mu);
    DeviceGuard g(ctx->device);
    TimerScope ts(ctx);
    if (q == 0) return;
    pbs_opts o;
    pbs_default_opts(&o);
    ensure_hierarchy_host(ctx, geom, effective_mu(o, geom->a, geom->b), o.coarsest);
    set_single_k(ctx, k[0], k[1]);
    const Level& L0 = ctx->H.lev[0];
    cudaStream_t s = ctx->stream;
    cudaEvent_t ev;
    PBS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    PBS_CUDA(cudaEventRecord(ev, (cudaStream_t)cuda_stream));
    PBS_CUDA(cudaStreamWaitEvent(s, ev, 0));
    cudaEventDestroy(ev);
    const long cap = gram_partials_size(L0.N(), q, 1);
    double2* part = (double2*)ctx->mem.alloc(sizeof(double2) * cap);
    try {
      const Roles R{{(const double2*)S, (const double2*)S, (const double2*)S}, q, L0.D()};
      gram_groups(L0, ctx->K.d_ph, R, q, 1, (double2*)GM, (double2*)GA, part, cap, precision == PBS_MIXED, s);
      PBS_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
      ctx->mem.free(part);
      throw;
    }
    ctx->mem.free(part);
  });
}

int pbs_m_householder(pbs_ctx* ctx, const pbs_geom* geom, const double k[2], int q, const pbs_c64* S, pbs_c64* E,
                      pbs_c64* R, void* cuda_stream) {
  if (!ctx || !geom || !k || q < 0 || q > kMaxTrial) return PBS_EINVAL;
  if (q > 0 && (!S || !E || !R)) return PBS_EINVAL;
  if (q > householder_max_columns(geom->n, geom->m)) return PBS_EINVAL;
  return run_guarded_impl([&] {
    std::lock_guard<std::mutex> ctx_lock(ctx->gpu_mu);
    DeviceGuard g(ctx->device);
    TimerScope ts(ctx);
    if (q == 0) return;
    pbs_opts o;
    pbs_default_opts(&o);
    ensure_hierarchy_host(ctx, geom, effective_mu(o, geom->a, geom->b), o.coarsest);
    set_single_k(ctx, k[0], k[1]);
    const Level& L0 = ctx->H.lev[0];
    cudaStream_t s = ctx->stream;
    cudaEvent_t ev;
    PBS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    PBS_CUDA(cudaEventRecord(ev, (cudaStream_t)cuda_stream));
    PBS_CUDA(cudaStreamWaitEvent(s, ev, 0));
    cudaEventDestroy(ev);
    void* work = ctx->mem.alloc(householder_work_bytes(L0.D(), q));
    try {
      m_householder(L0, ctx->K.d_ph, (const double2*)S, (double2*)E, (double2*)R, q, work, s);
      PBS_CUDA(cudaStreamSynchronize(s));
    } catch (...) {
      ctx->mem.free(work);
      throw;
    }
    ctx->mem.free(work);
  });
}

int pbs_rayleigh_ritz(pbs_ctx* ctx, const pbs_geom* geom, const pbs_opts* opts, const double k[2], int q,
                      const pbs_c64* S, int p, int project, double* theta, pbs_c64* X, void* cuda_stream) {
  if (!ctx || !geom || !opts || !k || q < 1 || p < 1 || p > q || p > kMaxBlock || !S || !theta || !X)
    return PBS_EINVAL;
  return run_guarded_impl([&] {
    std::lock_guard<std::mutex> ctx_lock(ctx->gpu_mu);
    DeviceGuard g(ctx->device);
    TimerScope ts(ctx);
    const pbs_opts& o = *opts;
    if (q > kMaxTrial) fail(PBS_EINVAL, "q too large");
    ensure_hierarchy_host(ctx, geom, effective_mu(o, geom->a, geom->b), o.coarsest);
    const int pw = std::max(p, (q + 2) / 3);
    if (pw > kMaxBlock) fail(PBS_EINVAL, "q too large");
    ensure_work(ctx, pw, 1, o.precision, 0);
    set_single_k(ctx, k[0], k[1]);
    cudaStream_t s = ctx->stream;
    cudaEvent_t ev;
    PBS_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    PBS_CUDA(cudaEventRecord(ev, (cudaStream_t)cuda_stream));
    PBS_CUDA(cudaStreamWaitEvent(s, ev, 0));
    cudaEventDestroy(ev);
    Work& W = ctx->W;
    PBS_CUDA(cudaMemcpyAsync(W.init, S, sizeof(double2) * W.D * q, cudaMemcpyDeviceToDevice, s));
    const KData Kv = kdata_view(ctx->K, 0);
    if (project) project_dispatch(ctx, o, Kv, W.init, q, q, o.nodal_cycles, s);
    rr_single(ctx, Kv, W.init, q, p, (double2*)X, o.precision == PBS_MIXED, s);
    PBS_CUDA(cudaMemcpyAsync(theta, W.theta, sizeof(double) * p, cudaMemcpyDeviceToHost, s));
    PBS_CUDA(cudaStreamSynchronize(s));
  });
}

static const char* kClassNames[KC_COUNT] = {"", "edge_smooth", "node_smooth", "gram", "small_rr", "residual",
                                             "block_update", "lift_adj_mass", "edge_apply", "edge_tail",
                                             "node_tail", "householder", "sub_lift", "convert", "node_apply"};

static int class_of(const char* name) {
  for (int c = 1; c < KC_COUNT; ++c)
    if (std::strcmp(name, kClassNames[c]) == 0) return c;
  return -1;
}

int pbs_profile_enable(pbs_ctx* ctx, const char* classes) {
  if (!ctx) return PBS_EINVAL;
  std::lock_guard<std::mutex> ctx_lock(ctx->gpu_mu);
  unsigned mask = 0;
  int every = 1;
  std::string spec = classes ? classes : "";
  const size_t slash = spec.find('/');
  if (slash != std::string::npos) {
    every = std::atoi(spec.c_str() + slash + 1);
    spec = spec.substr(0, slash);
    if (every < 1) {
      g_last_error = "sampling interval must be >= 1";
      return PBS_EINVAL;
    }
  }
  classes = spec.c_str();
  if (classes && *classes) {
    if (std::strcmp(classes, "all") == 0) {
      mask = ((1u << KC_COUNT) - 1) & ~1u;
    } else {
      std::string list(classes);
      size_t pos = 0;
      while (pos <= list.size()) {
        const size_t e = std::min(list.find(',', pos), list.size());
        const std::string name = list.substr(pos, e - pos);
        const int c = class_of(name.c_str());
        if (c < 0) {
          g_last_error = "unknown kernel class: " + name;
          return PBS_EINVAL;
        }
        mask |= 1u << c;
        pos = e + 1;
      }
    }
  }
  KernelTimer& t = ctx->timer;
  t.mask = mask;
  t.every = every;
  t.open = false;
  for (int c = 0; c < KC_COUNT; ++c) {
    t.seen[c] = 0;
    t.total_ms[c] = 0.0;
    t.work[c] = 0.0;
    t.launches[c] = 0;
  }
  return PBS_OK;
}

int pbs_profile_read(pbs_ctx* ctx, const char* kernel_class, double* total_ms, long* launches, double* work) {
  if (!ctx || !kernel_class || !total_ms || !launches || !work) return PBS_EINVAL;
  std::lock_guard<std::mutex> ctx_lock(ctx->gpu_mu);
  const int c = class_of(kernel_class);
  if (c < 0) return PBS_EINVAL;
  *total_ms = ctx->timer.total_ms[c];
  *launches = ctx->timer.launches[c];
  *work = ctx->timer.work[c];
  return PBS_OK;
}

unsigned long long pbs_launch_count(void) { return g_launches.load(); }

unsigned long long pbs_launch_count_df(void) { return g_df_launches.load(); }

int pbs_solve_grid(pbs_ctx* ctx, const pbs_geom* geom, const pbs_opts* opts, int kappa, double* ks_out,
                   double* eigvals, double* resid, int* iters) {
  if (!ctx || !geom || !opts || kappa < 2 || !eigvals || !resid || !iters) return PBS_EINVAL;
  int status = PBS_OK;
  const int rc = run_guarded_impl([&] {
    std::lock_guard<std::mutex> ctx_lock(ctx->gpu_mu);
    DeviceGuard g(ctx->device);
    TimerScope ts(ctx);
    const pbs_opts o = *opts;
    validate_opts(o);
    ensure_hierarchy_host(ctx, geom, effective_mu(o, geom->a, geom->b), o.coarsest);
    // k_ij = (pi/a (2 i/(kappa-1) - 1), pi/b (2 j/(kappa-1) - 1)), index j kappa + i (Section 6)
    const int K = kappa, nk = K * K, p = o.block;
    std::vector<double> ks(2L * nk);
    for (int j = 0; j < K; ++j)
      for (int i = 0; i < K; ++i) {
        ks[2L * (j * K + i)] = M_PI / geom->a * (2.0 * i / (K - 1) - 1.0);
        ks[2L * (j * K + i) + 1] = M_PI / geom->b * (2.0 * j / (K - 1) - 1.0);
      }
    if (ks_out) std::copy(ks.begin(), ks.end(), ks_out);
    // bases of the first three columns, kept for the vertical and the row extrapolations
    const int nc = std::min(3, K);
    const long D = ctx->H.lev[0].D();
    auto slot = [&](int i, int j) { return j * nc + i; };
    double2* store = (double2*)ctx->mem.alloc(sizeof(double2) * D * p * nc * K);
    auto at = [&](int i, int j) -> const double2* { return store + (long)slot(i, j) * p * D; };
    bool all_conv = true;
    auto merge = [&](const std::vector<Chain>& chains, const PathResult& r) {
      for (const Chain& c : chains)
        for (int k : c.idx) {
          for (int b = 0; b < o.nev; ++b) {
            eigvals[(long)k * o.nev + b] = r.lam[(long)k * o.nev + b];
            resid[(long)k * o.nev + b] = r.res[(long)k * o.nev + b];
          }
          iters[k] = r.iters[k];
        }
      all_conv = all_conv && r.all_converged;
    };
    try {
      // row 0, horizontally: k_00 from the start, k_i0 from up to three predecessors
      std::vector<Chain> row0(1);
      for (int i = 0; i < K; ++i) {
        row0[0].idx.push_back(i);
        row0[0].save.push_back(i < nc ? slot(i, 0) : -1);
      }
      merge(row0, solve_chain_list(ctx, o, nk, ks.data(), row0, 1, nullptr, nullptr, store));
      // columns 0..2, vertically from row 0
      std::vector<Chain> cols(nc);
      for (int i = 0; i < nc; ++i) {
        cols[i].seeds = {at(i, 0)};
        for (int j = 1; j < K; ++j) {
          cols[i].idx.push_back(j * K + i);
          cols[i].save.push_back(slot(i, j));
        }
      }
      if (K > 1) merge(cols, solve_chain_list(ctx, o, nk, ks.data(), cols, o.kbatch, nullptr, nullptr, store));
      // rows 1.., horizontally from k_2j, k_1j, k_0j (read the same way for j = 1, 2, where the
      // printed schedule leaves the order open)
      std::vector<Chain> rows;
      for (int j = 1; j < K && K > 3; ++j) {
        Chain c;
        c.seeds = {at(2, j), at(1, j), at(0, j)};
        for (int i = 3; i < K; ++i) c.idx.push_back(j * K + i);
        rows.push_back(c);
      }
      if (!rows.empty()) merge(rows, solve_chain_list(ctx, o, nk, ks.data(), rows, o.kbatch, nullptr, nullptr, store));
    } catch (...) {
      ctx->mem.free(store);
      throw;
    }
    ctx->mem.free(store);
    if (!all_conv) status = PBS_ENOCONV;
  });
  return rc != PBS_OK ? rc : status;
}

int pbs_job_bytes(int n, int m, const pbs_opts* opts, int nk, size_t* bytes) {
  if (!opts || !bytes || nk < 1) return PBS_EINVAL;
  return run_guarded_impl([&] {
    validate_opts(*opts);
    validate_mesh(1.0, 1.0, n, m);
    if (num_levels(n, m, opts->coarsest) < 1) fail(PBS_EINVAL, "invalid mesh for the hierarchy");
    *bytes = (size_t)job_bytes(n, m, *opts, nk, 0);
  });
}

int pbs_submit(pbs_ctx* ctx, const pbs_geom* geom, const pbs_opts* opts, int nk, const double* ks,
               uint64_t* job_id) {
  if (!ctx || !geom || !opts || nk < 1 || !ks || !job_id || !geom->eps) return PBS_EINVAL;
  return run_guarded_impl([&] {
    validate_opts(*opts);
    validate_mesh(geom->a, geom->b, geom->n, geom->m);
    if (num_levels(geom->n, geom->m, opts->coarsest) < 1) fail(PBS_EINVAL, "invalid mesh for the hierarchy");
    const long N = (long)geom->n * geom->m;
    for (long t = 0; t < N; ++t)
      if (!(geom->eps[t] > 0.0) || !std::isfinite(geom->eps[t])) fail(PBS_EINVAL, "eps must be finite and positive");
    for (long t = 0; t < 2L * nk; ++t)
      if (!std::isfinite(ks[t])) fail(PBS_EINVAL, "k must be finite");
    // admission: a job that alone exceeds what the jobs may hold is refused; others
    // wait in the queue until the running jobs leave room for them
    auto j = std::make_shared<Job>();
    j->est = job_bytes(geom->n, geom->m, *opts, nk, 0);
    j->a = geom->a;
    j->b = geom->b;
    j->n = geom->n;
    j->m = geom->m;
    j->nk = nk;
    j->eps.assign(geom->eps, geom->eps + N);
    j->ks.assign(ks, ks + 2L * nk);
    j->o = *opts;
    {
      const double mu = effective_mu(*opts, geom->a, geom->b);
      uint64_t key = fnv1a(geom->eps, N * sizeof(double));
      key = fnv1a(&j->a, sizeof j->a, key);
      key = fnv1a(&j->b, sizeof j->b, key);
      key = fnv1a(&j->n, sizeof j->n, key);
      key = fnv1a(&j->m, sizeof j->m, key);
      key = fnv1a(&mu, sizeof mu, key);
      key = fnv1a(&opts->coarsest, sizeof opts->coarsest, key);
      j->gkey = key | 1;
    }
    Server& sv = ctx->srv;
    {
      std::lock_guard<std::mutex> lk(sv.m);
      if (sv.stop) fail(PBS_EINVAL, "context is shutting down");
      start_server(ctx);
      if (j->est > sv.cap) fail(PBS_ENOMEM, "job needs more device memory than the context may use");
      j->id = sv.next_id++;
      j->t_submit = std::chrono::steady_clock::now();
      sv.jobs[j->id] = j;
      sv.queue.push_back(j);
    }
    sv.cv_work.notify_all();
    *job_id = j->id;
  });
}

int pbs_poll(pbs_ctx* ctx, uint64_t job_id, int* done) {
  if (!ctx || !done) return PBS_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->srv.m);
  auto it = ctx->srv.jobs.find(job_id);
  if (it == ctx->srv.jobs.end()) {
    g_last_error = "unknown job";
    return PBS_EINVAL;
  }
  *done = it->second->done ? 1 : 0;
  return PBS_OK;
}

int pbs_fetch(pbs_ctx* ctx, uint64_t job_id, double* eigvals, double* resid, int* iters, double* latency_s) {
  if (!ctx) return PBS_EINVAL;
  std::shared_ptr<Job> j;
  {
    std::unique_lock<std::mutex> lk(ctx->srv.m);
    auto it = ctx->srv.jobs.find(job_id);
    if (it == ctx->srv.jobs.end()) {
      g_last_error = "unknown job";
      return PBS_EINVAL;
    }
    j = it->second;
    ctx->srv.cv_done.wait(lk, [&] { return j->done; });
    ctx->srv.jobs.erase(it);
  }
  if (eigvals) std::copy(j->lam.begin(), j->lam.end(), eigvals);
  if (resid) std::copy(j->res.begin(), j->res.end(), resid);
  if (iters) std::copy(j->iters.begin(), j->iters.end(), iters);
  if (latency_s) *latency_s = std::chrono::duration<double>(j->t_done - j->t_submit).count();
  g_last_error = j->err;
  return j->status;
}

int pbs_cancel(pbs_ctx* ctx, uint64_t job_id) {
  if (!ctx) return PBS_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->srv.m);
  auto it = ctx->srv.jobs.find(job_id);
  if (it == ctx->srv.jobs.end()) {
    g_last_error = "unknown job";
    return PBS_EINVAL;
  }
  Job& j = *it->second;
  if (j.done) return PBS_OK;
  j.cancel.store(true);
  if (!j.started) {
    auto& q = ctx->srv.queue;
    for (auto qi = q.begin(); qi != q.end(); ++qi)
      if ((*qi)->id == job_id) {
        q.erase(qi);
        break;
      }
    j.status = PBS_ECANCELED;
    j.err = "job cancelled before it started";
    j.t_start = j.t_done = std::chrono::steady_clock::now();
    j.done = true;
    ctx->srv.cv_done.notify_all();
    ctx->srv.cv_work.notify_all();
  }
  return PBS_OK;
}

int pbs_job_times(pbs_ctx* ctx, uint64_t job_id, double* submit_s, double* start_s, double* done_s) {
  if (!ctx || !submit_s || !start_s || !done_s) return PBS_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->srv.m);
  auto it = ctx->srv.jobs.find(job_id);
  if (it == ctx->srv.jobs.end()) {
    g_last_error = "unknown job";
    return PBS_EINVAL;
  }
  const Job& j = *it->second;
  auto rel = [&](std::chrono::steady_clock::time_point t) {
    return std::chrono::duration<double>(t - ctx->t_created).count();
  };
  *submit_s = rel(j.t_submit);
  *start_s = j.started || j.done ? rel(j.t_start) : -1.0;
  *done_s = j.done ? rel(j.t_done) : -1.0;
  return PBS_OK;
}

int pbs_serve_slots(pbs_ctx* ctx, int slots) {
  if (!ctx || slots < 1 || slots > 64) return PBS_EINVAL;
  std::lock_guard<std::mutex> lk(ctx->srv.m);
  if (ctx->srv.started) {
    g_last_error = "the serving slots are already running";
    return PBS_EINVAL;
  }
  ctx->srv.nslots = slots;
  return PBS_OK;
}

int pbs_set_budget(pbs_ctx* ctx, size_t hbm_budget_bytes) {
  if (!ctx) return PBS_EINVAL;
  std::lock_guard<std::mutex> g(ctx->gpu_mu);
  ctx->mem.set_budget(hbm_budget_bytes);
  return PBS_OK;
}

int pbs_fail_alloc_after(pbs_ctx* ctx, int count) {
  if (!ctx || count < 0) return PBS_EINVAL;
  std::lock_guard<std::mutex> g(ctx->gpu_mu);
  ctx->mem.fail_after(count);
  return PBS_OK;
}

}  // extern "C"
