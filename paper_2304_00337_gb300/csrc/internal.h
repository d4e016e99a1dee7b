// Host-side declarations shared by the pbs translation units (not part of the ABI).
#pragma once
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <functional>
#include <mutex>
#include <string>
#include <utility>
#include <vector>

#include "common.cuh"
#include "pbs.h"

namespace pbs {

constexpr int kMaxLevels = 16;
constexpr int kMaxBlock = 32;        // block width p
constexpr int kMaxTrial = 3 * kMaxBlock;  // trial width q
constexpr int kMaxCoarseEdges = 1024;     // dense coarsest edge system (2 n_c m_c)

// Failure that the ABI layer turns into a status code.
struct Error {
  int status;
  std::string what;
};
[[noreturn]] void fail(int status, const std::string& what);
void check_cuda(cudaError_t e, const char* what);
#define PBS_CUDA(call) ::pbs::check_cuda((call), #call)
// Detail of a failure for pbs_last_error on the calling thread.
void set_last_error(const std::string& what);

// Runs a set-up step once per CUDA device and process, from any thread, with
// that device current: kernel attributes such as the dynamic shared-memory limit
// belong to a device, so each device a process drives gets its own call.  A step
// that throws leaves the device's flag unset (the next launch tries again).
constexpr int kMaxDevices = 64;
struct PerDeviceOnce {
  std::once_flag flag[kMaxDevices];
  template <class F> void operator()(F&& f) {
    int dev = 0;
    check_cuda(cudaGetDevice(&dev), "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) fail(PBS_ECUDA, "device index beyond the library's table of devices");
    std::call_once(flag[dev], std::forward<F>(f));
  }
};

// One level of the bisection hierarchy (Section 5).  Geometry only: the
// Bloch phases enter the kernels separately, so a level serves every k.
struct Level {
  int n = 0, m = 0;
  double h1 = 0, h2 = 0;
  double* winv64 = nullptr;  // 1/eps per cell (2x2 mean of the finer level's 1/eps)
  float* winv32 = nullptr;
  double* k3_64 = nullptr;   // per node: 6 entries of the inverse 3x3 patch block, SoA [6][N]
  float* k3_32 = nullptr;
  float2* wdf = nullptr;     // level 0: w = (1/eps) / (h1 h2) as double-float (hi, lo) per cell
  double wmax = 0;           // level 0: the largest w
  long N() const { return (long)n * m; }
  WtsDF wts_df() const { return WtsDF{wdf, n, m}; }
  long D() const { return 2L * n * m; }
  template <class T> Lvl<T> lvl() const { return Lvl<T>{n, m, T(h2 / h1), T(h1 / h2)}; }
  template <class T> Wts<T> wts() const;
};
template <> inline Wts<double> Level::wts<double>() const { return Wts<double>{winv64, n, m, 1.0 / (h1 * h2)}; }
template <> inline Wts<float> Level::wts<float>() const { return Wts<float>{winv32, n, m, float(1.0 / (h1 * h2))}; }

// Multigrid hierarchy of one geometry and regularisation mu.
struct Hierarchy {
  double a = 0, b = 0, mu = 0;
  double winv_max = 0;  // largest 1/eps on the finest level
  int n = 0, m = 0, nlev = 0;
  uint64_t key = 0;
  Level lev[kMaxLevels];
  std::vector<void*> allocs;
};

// Per-Bloch-vector data of `ngroups` groups (one Bloch vector each): phases,
// k = 0 flags and the factored coarsest systems.  The device phase and flag
// tables repeat the per-group entries three times, so that column c of any
// role-major block [E_all | P_all | W_all] with `cpg` columns per group finds
// its group's entry at c / cpg.
struct KData {
  int ngroups = 0;
  int Dc = 0, Nc = 0;
  double* d_ph = nullptr;      // 3 * ngroups entries of (alpha.re, alpha.im, beta.re, beta.im)
  int* d_gamma = nullptr;      // 3 * ngroups flags: 1 when both phases equal one (k = 0)
  double2* edge64 = nullptr;   // ngroups Cholesky factors (lower, column-major Dc x Dc) of A_c + mu M_c
  float2* edge32 = nullptr;
  double2* node64 = nullptr;   // ngroups factors of P_c (+ a constant-mode term at k = 0), Nc x Nc
  float2* node32 = nullptr;
  int* d_info = nullptr;       // status of the coarsest factorisations (2 ints)
  std::vector<double> k1, k2;  // host mirror
  std::vector<char> gamma;
  int goff = 0;                // chunk views: column c uses coarsest factors of group (c / cpg + goff) % ngroups
  bool owner = true;
  bool any_gamma() const {
    for (char g : gamma)
      if (g) return true;
    return false;
  }
};
// Device allocator with a byte budget.
class DevMem {
 public:
  explicit DevMem(size_t budget) : budget_(budget) {}
  void* alloc(size_t bytes);
  void free(void* p);
  size_t used() const { return used_; }
  size_t budget() const { return budget_; }  // 0 = no cap
  void set_budget(size_t b) { budget_ = b; }
  // failure injection: the count-th allocation from now fails with PBS_ENOMEM (0: off)
  void fail_after(int count) { fail_in_ = count; }

 private:
  size_t budget_, used_ = 0;
  int fail_in_ = 0;
  std::vector<std::pair<void*, size_t>> live_;
};

int num_levels(int n, int m, int coarsest);

// Optional CUDA-event timing of kernel classes on the stream they are launched
// on (enabled per context through pbs_profile_enable; off by default).  Each
// timed launch also adds its algorithmic work (bytes for streaming kernels,
// flops for arithmetic-bound ones) so the achieved rate can be derived.
enum KernelClass {
  KC_NONE = 0, KC_EDGE_SMOOTH, KC_NODE_SMOOTH, KC_GRAM, KC_SMALL_RR, KC_RESIDUAL, KC_BLOCK_UPDATE,
  KC_LIFT_ADJ_MASK, KC_EDGE_APPLY, KC_EDGE_TAIL, KC_NODE_TAIL, KC_HOUSEHOLDER, KC_SUB_LIFT, KC_CONVERT,
  KC_NODE_APPLY, KC_COUNT
};
struct TimedLaunch {
  int cls;
  double work;
  cudaEvent_t start, stop;
};
struct KernelTimer {
  unsigned mask = 0;  // bit c set: class c is timed
  int every = 1;      // time every `every`-th launch of a timed class
  long seen[KC_COUNT] = {};
  bool open = false;  // the latest begin was recorded
  double total_ms[KC_COUNT] = {};
  double work[KC_COUNT] = {};
  long launches[KC_COUNT] = {};
  std::vector<TimedLaunch> pending;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
};
extern thread_local KernelTimer* g_timer;
void timer_begin(int cls, cudaStream_t s, double work);
void timer_end(int cls, cudaStream_t s);
void timer_collect();  // after a stream synchronisation
// every kernel launch of the library is counted (process-wide); launches of kernels
// that compute in double-float arithmetic are counted a second time on their own
void count_launch();
void count_launches(long delta);  // kernels of a replayed CUDA graph
void count_df_launch();
bool verbose_enabled();  // PBS_VERBOSE set in the environment (diagnostic traces)
#define PBS_LAUNCHED()                 \
  do {                                 \
    ::pbs::count_launch();             \
    PBS_CUDA(cudaGetLastError());      \
  } while (0)

// ---- launch-configuration autotuner (tune.cu) ------------------------------
// Index of the fastest of `ncand` candidate configurations for `key`: measured on
// first use (run(c) launches candidate c on stream s; candidates are idempotent),
// then remembered for the process and in the tuning cache file.
int tune_pick(const std::string& key, int ncand, const std::function<void(int)>& run, cudaStream_t s);
std::string device_tag();  // device name and SM count, for tuning keys

// ---- hierarchy set-up (mg.cu) ---------------------------------------------
void build_hierarchy(DevMem& mem, Hierarchy& H, const double* d_eps, int coarsest, cudaStream_t s);
void free_hierarchy(DevMem& mem, Hierarchy& H);
void alloc_kdata(DevMem& mem, const Hierarchy& H, KData& K, int ngroups);
void set_group_k(DevMem& mem, const Hierarchy& H, KData& K, int g, double k1, double k2, cudaStream_t s);
// group src's tables (phases, k = 0 flags, coarsest factors, host mirror) copied into slot dst
void copy_group_k(KData& K, int src, int dst, cudaStream_t s);
KData kdata_view(const KData& K, int g);  // non-owning single-group view of group g
// non-owning view for a chunk of a role-major block starting at column group v0
// (phase and flag tables shifted by v0, factors selected with the matching offset)
KData kdata_chunk(const KData& K, int v0);
void free_kdata(DevMem& mem, KData& K);

// ---- operators (ops.cu); X, Y device blocks of ncols columns with stride ld ----
// Y = sB*B + sA*(A X) + (sM + sL*lam[c]) (M X)   (B, lam may be null)
template <class T>
void apply_edge(const Level& L, const double* d_ph, int cpg, const cx<T>* X, cx<T>* Y, const cx<T>* B, long ld,
                int ncols, T sA, T sM, T sL, const T* lam, T sB, cudaStream_t s);
template <class T>
void apply_curl(const Level& L, const double* d_ph, int cpg, const cx<T>* X, long ldx, cx<T>* Y, long ldy, int ncols,
                cudaStream_t s);
template <class T>
void apply_curl_adj(const Level& L, const double* d_ph, int cpg, const cx<T>* X, long ldx, cx<T>* Y, long ldy,
                    int ncols, cudaStream_t s);
template <class T>
void apply_lift(const Level& L, const double* d_ph, int cpg, const cx<T>* X, long ldx, cx<T>* Y, long ldy, int ncols,
                cudaStream_t s);
template <class T>
void apply_lift_adj(const Level& L, const double* d_ph, int cpg, const cx<T>* X, long ldx, cx<T>* Y, long ldy,
                    int ncols, cudaStream_t s);
// Y = sB*B + sP*(P X) on nodes
template <class T>
void apply_nodal(const Level& L, const double* d_ph, int cpg, const cx<T>* X, cx<T>* Y, const cx<T>* B, long ld,
                 int ncols, T sP, T sB, cudaStream_t s);
// edge transfer: fine level `f` (index l) <-> coarse level `c` (l+1)
template <class T>
void prolong_edge(const Level& f, const Level& c, const double* d_ph, int cpg, const cx<T>* Xc, long ldc, cx<T>* Yf,
                  long ldf, int ncols, bool accumulate, cudaStream_t s);
template <class T>
void restrict_edge(const Level& f, const Level& c, const double* d_ph, int cpg, const cx<T>* Xf, long ldf, cx<T>* Yc,
                   long ldc, int ncols, cudaStream_t s);
template <class T>
void prolong_node(const Level& f, const Level& c, const double* d_ph, int cpg, const cx<T>* Xc, long ldc, cx<T>* Yf,
                  long ldf, int ncols, bool accumulate, cudaStream_t s);
template <class T>
void restrict_node(const Level& f, const Level& c, const double* d_ph, int cpg, const cx<T>* Xf, long ldf, cx<T>* Yc,
                   long ldc, int ncols, cudaStream_t s);

// ---- multigrid (mg.cu) ----------------------------------------------------
// Workspace for V-cycles of up to `ncols` columns on levels 1..nlev-1 (+ level-0 residual).
template <class T> struct MgWork {
  cx<T>* x[kMaxLevels] = {};
  cx<T>* b[kMaxLevels] = {};
  cx<T>* r[kMaxLevels] = {};
  int ncols = 0;
};
template <class T> void alloc_mg_work(DevMem& mem, const Hierarchy& H, int ncols, bool nodal, MgWork<T>& w);
template <class T> void free_mg_work(DevMem& mem, MgWork<T>& w);
// Y = B X: one edge V-cycle for A + mu M started from zero (x, y on level `l0`).
// `cpg` columns per group: column c uses group (c / cpg) of the tables.
template <class T>
void edge_vcycle(const Hierarchy& H, const KData& K, MgWork<T>& w, int l0, const cx<T>* X, cx<T>* Y, long ld,
                 int ncols, int cpg, int nu_pre, int nu_post, cudaStream_t s);
template <class T>
void nodal_vcycle(const Hierarchy& H, const KData& K, MgWork<T>& w, int l0, const cx<T>* X, cx<T>* Y, long ld,
                  int ncols, int cpg, int nu_pre, int nu_post, cudaStream_t s);
// Y = X0 + B (X - P X0): one nodal V-cycle continuing from the iterate X0 (Y may be X0),
// for levels where nodal_takes_guess holds; the residual is formed inside the cycle
template <class T> bool nodal_takes_guess(const Hierarchy& H, int l0, int nu_pre, int nu_post);
template <class T>
void nodal_vcycle_from(const Hierarchy& H, const KData& K, MgWork<T>& w, int l0, const cx<T>* X, const cx<T>* X0,
                       cx<T>* Y, long ld, int ncols, int cpg, int nu_pre, int nu_post, cudaStream_t s);

// ---- dense block kernels (dense.cu) ---------------------------------------
// Every kernel below reads and writes FP64 blocks.  Where a `dfa` flag is given it
// selects the arithmetic: false = FP64, true = double-float on the FP32 pipe
// (about 2^-47 relative; the mixed-precision policy).  What writes the iterate or
// differences it through the curl-curl stencil (residual, E C, x - L phi) stays in
// FP64: a relative perturbation eta of the iterate moves the relative residual by
// about eta lambda_max / lambda.
void convert_d2f(const double2* X, float2* Y, long n, cudaStream_t s);
void convert_f2d(const float2* X, double2* Y, long n, cudaStream_t s);
// x <- x - L phi (FP64 x, phi in T), level 0
template <class T>
void sub_lift(const Level& L, const double* d_ph, int cpg, const cx<T>* Phi, long ldp, double2* X, long ldx, int ncols,
              cudaStream_t s);
// rhs = L^* M x  (FP64), stored in T
template <class T>
void lift_adj_mass(const Level& L, const double* d_ph, int cpg, const double2* X, long ldx, cx<T>* Rhs, long ldr,
                   int ncols, bool dfa, cudaStream_t s);
// subtract the x-edge mean and the y-edge mean of every column of a k = 0 group
// (flags d_gamma[c / cpg]; the deflation of the two constant fields)
void deflate_constants(const Level& L, double2* X, long ld, int ncols, const int* d_gamma, int cpg,
                       double* d_partials, cudaStream_t s);
// per column: out[2c] = e^* M e, out[2c+1] = (C e)^* W (C e)
void rayleigh_parts(const Level& L, const double* d_ph, int cpg, const double2* X, long ld, int ncols,
                    double* d_partials, double* d_out, bool dfa, cudaStream_t s);
// R = A E - lam M E in the mixed policy: FP64 curls, double-float rest, R stored in
// FP32 (the preconditioner's input); the same norms (level 0 only)
void residual_mixed(const Level& L, const double* d_ph, int cpg, const double2* E, float2* R, long ld, int ncols,
                    const double* d_lam, double* d_partials, double* d_out, cudaStream_t s);
// R = A E - lam M E; per column out[2c] = |R|^2, out[2c+1] = |M E|^2
void residual(const Level& L, const double* d_ph, int cpg, const double2* E, double2* R, long ld, int ncols,
              const double* d_lam, double* d_partials, double* d_out, cudaStream_t s);
// Columns of trial blocks held in up to three role arrays: column a of group g is
// b[a / pr] + (g * pr + a % pr) * ld.
struct Roles {
  const double2* b[3];
  int pr;
  long ld;
};
// Per group g (phases from entry g of d_ph): GM_g = S^* M S, GA_g = (C S)^* W (C S), q x q
// column-major at GM + g q^2, GA + g q^2.
void gram_groups(const Level& L, const double* d_ph, Roles roles, int q, int ngroups, double2* GM, double2* GA,
                 double2* d_partials, long partial_capacity, bool dfa, cudaStream_t s);
long gram_partials_size(long rows, int q, int ngroups);  // double2 elements
// The mixed policy's Gram on the tensor cores (gram_tc.cu): the partial sums of
// gram_groups' double-float kernel for q <= 48, from bf16 slices (Ozaki splitting).
bool gram_tc_supported(int q);
bool gram_on_tensor_cores();  // true when the environment sets PBS_GRAM=tc (then offered first)
void gram_tc(const Level& L, const double* d_ph, Roles roles, int q, int ngroups, int npart, double2* d_partials,
             cudaStream_t s);
// Rayleigh-Ritz in coefficient space for ngroups groups: C (q x p per group), theta (p per
// group), status in d_info[8 g], scratch small_rr_scratch(q) bytes per group; dfa selects
// double-float (mixed policy) instead of FP64 arithmetic
void small_rr(const double2* GM, const double2* GA, int q, int p, double2* C, double* theta, double2* scratch,
              int* d_info, int ngroups, bool dfa, cudaStream_t s);
size_t small_rr_scratch(int q);
// Y_g[:, j] = sum_i X_g[:, i] C_g[i, j] (+ Z_g[:, j]) for each group
// (dfa: double-float, for the search direction only; the iterate's update is FP64)
void block_update(Roles X, int q, const double2* C, int ldc, long cgs, double2* Y, long ldy, int p,
                  const double2* Z, long ldz, long rows, int ngroups, bool dfa, cudaStream_t s);
void random_block(double2* X, long ld, long rows, int ncols, uint64_t seed, cudaStream_t s);

// ---- generalised Householder orthonormalisation (householder.cu) ----------
// Q_q .. Q_1 S = P R, E = Q_1 .. Q_q P (Section 4); S, E: D x q (ld D), R: q x q
// column-major, all on the device; `work` holds householder_work_bytes(D, q).
int householder_max_columns(int n, int m);
size_t householder_work_bytes(long D, int q);
void m_householder(const Level& L0, const double* d_ph, const double2* S, double2* E, double2* R, int q, void* work,
                   cudaStream_t s);
void scale_columns(double2* X, long ld, long rows, int ncols, const double* d_scale, cudaStream_t s);

}  // namespace pbs
