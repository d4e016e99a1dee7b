// Geometric multigrid of Section 5: bisection hierarchy with Galerkin coarse
// operators, node-patch block Gauss-Seidel for A + mu M (edges), point
// Gauss-Seidel for P = L^* M L (nodes), dense Cholesky on the coarsest level.
//
// Coarse operators.  With the natural embedding as prolongation the Galerkin
// product P^* A_f P is the curl-curl matrix of the coarse mesh whose 1/eps is
// the mean of the four children's 1/eps, and P^* M_f P is the coarse mass
// matrix (the curl is constant per cell, so a coarse cell's energy is the sum
// of its children's).  Hence every level uses the same stencil code with its
// own 1/eps and mesh widths, and the Bloch phases are unchanged (the periods
// a, b are the same on every level).
//
// Patch solve.  The patch of node (i,j) holds its left, right, bottom and top
// edges (L, R, B, T).  In "ghost" coordinates (values read through the Bloch
// extension) the 4x4 block of A + mu M is real and independent of k:
//   K = sum_cells w_c v_c v_c^T + mu diag(m1, m1, m2, m2),  m1 = 2/3 h2/h1, m2 = 2/3 h1/h2,
//   v_SW = (1,0,-1,0), v_NW = (-1,0,0,-1), v_SE = (0,1,1,0), v_NE = (0,-1,0,1).
// The gradient g = (1,-1,1,-1) of the node's hat function satisfies K g =
// mu M_loc g, which makes K ill-conditioned for small mu (Section 5).  Following
// the paper's stable variant, T = [g, t_a, t_b, t_c] with the M_loc-orthogonal
// complement t_a = (1,1,0,0), t_b = (0,0,1,1), t_c = (m2,-m2,-m1,m1) gives
// T^T K T = diag(mu g^T M_loc g, K3), so K^{-1} r = g (g^T r)/(mu g^T M_loc g)
// + T3 K3^{-1} T3^T r.  K3^{-1} (3x3, symmetric) is stored per node and level.
//
// Colouring.  Nodes are processed by colour (i mod 2, j mod 2) in the order
// (0,0), (1,0), (0,1), (1,1) (pre-smoothing) and reversed (post-smoothing).
// Same-colour patches share no edge and are not coupled by A or M, so each
// colour is one parallel launch and equals the sequential block Gauss-Seidel
// sweep; the resulting V-cycle is Hermitian.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <type_traits>

#include "internal.h"
#include "mgpoint.cuh"
#include "nodal_tiles.cuh"

namespace pbs {

namespace {

constexpr int kBX = 32, kBY = 8;
constexpr int kColours[4][2] = {{0, 0}, {1, 0}, {0, 1}, {1, 1}};

// w = (1/eps) / (h1 h2) as a double-float pair per cell
__global__ void k_weights_df(const double* __restrict__ winv, double scale, float2* __restrict__ w, long N) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= N) return;
  const df v = df_from(scale * winv[t]);
  w[t] = make_float2(v.hi, v.lo);
}

__global__ void k_inv_eps(const double* __restrict__ eps, double* __restrict__ w64, float* __restrict__ w32, long N,
                          int* __restrict__ bad, unsigned long long* __restrict__ wmax) {
  const long t = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (t >= N) return;
  const double e = eps[t];
  if (!(e > 0.0) || !isfinite(e)) {
    atomicExch(bad, 1);
    w64[t] = 1.0;
    w32[t] = 1.0f;
    return;
  }
  w64[t] = 1.0 / e;
  w32[t] = float(1.0 / e);
  // positive doubles order like their bit patterns
  atomicMax(wmax, (unsigned long long)__double_as_longlong(1.0 / e));
}

__global__ void k_coarsen_w(const double* __restrict__ wf, int nf, double* __restrict__ wc, float* __restrict__ wc32,
                            int nc, int mc) {
  const int I = blockIdx.x * kBX + threadIdx.x, J = blockIdx.y * kBY + threadIdx.y;
  if (I >= nc || J >= mc) return;
  const long a = (long)(2 * J) * nf + 2 * I, b = a + nf;
  const double v = 0.25 * (wf[a] + wf[a + 1] + wf[b] + wf[b + 1]);
  wc[(long)J * nc + I] = v;
  wc32[(long)J * nc + I] = float(v);
}

// K3 = sum_c w_c u_c u_c^T + mu diag(2 m1, 2 m2, 2 m1 m2 s), u_c = T3^T v_c, s = m1 + m2
__global__ void k_patch_factors(const double* __restrict__ winv, int n, int m, double scale, double m1, double m2,
                                double mu, double* __restrict__ k64, float* __restrict__ k32) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y;
  if (i >= n || j >= m) return;
  const int im = (i + n - 1) % n, jm = (j + m - 1) % m;
  const double wSW = scale * winv[(long)jm * n + im], wNW = scale * winv[(long)j * n + im];
  const double wSE = scale * winv[(long)jm * n + i], wNE = scale * winv[(long)j * n + i];
  const double s = m1 + m2;
  const double u[4][3] = {{1, -1, s}, {-1, -1, -s}, {1, 1, -s}, {-1, 1, s}};
  const double w[4] = {wSW, wNW, wSE, wNE};
  double K[3][3] = {{mu * 2 * m1, 0, 0}, {0, mu * 2 * m2, 0}, {0, 0, mu * 2 * m1 * m2 * s}};
  for (int c = 0; c < 4; ++c)
    for (int a = 0; a < 3; ++a)
      for (int b = 0; b < 3; ++b) K[a][b] += w[c] * u[c][a] * u[c][b];
  // inverse via the adjugate (K3 is symmetric positive definite and well conditioned)
  const double c00 = K[1][1] * K[2][2] - K[1][2] * K[2][1];
  const double c01 = K[0][2] * K[2][1] - K[0][1] * K[2][2];
  const double c02 = K[0][1] * K[1][2] - K[0][2] * K[1][1];
  const double c11 = K[0][0] * K[2][2] - K[0][2] * K[2][0];
  const double c12 = K[0][2] * K[1][0] - K[0][0] * K[1][2];
  const double c22 = K[0][0] * K[1][1] - K[0][1] * K[1][0];
  const double det = K[0][0] * c00 + K[0][1] * (K[1][2] * K[2][0] - K[1][0] * K[2][2]) + K[0][2] * (K[1][0] * K[2][1] - K[1][1] * K[2][0]);
  const double id = 1.0 / det;
  const double inv[6] = {c00 * id, c01 * id, c02 * id, c11 * id, c12 * id, c22 * id};
  const long N = (long)n * m, e = (long)j * n + i;
  for (int q = 0; q < 6; ++q) {
    k64[q * N + e] = inv[q];
    k32[q * N + e] = float(inv[q]);
  }
}

// Dense coarsest-level matrices, column-major: column `col` = operator applied to unit vector `col`.
__global__ void k_assemble_edge(Lvl<double> L, Wts<double> w, double mu, const double* ph, double2* K) {  // ph: the group's entry
  const int Nc = L.n * L.m, Dc = 2 * Nc;
  const int row = blockIdx.x * blockDim.x + threadIdx.x, col = blockIdx.y;
  if (row >= Dc || col >= Dc) return;
  const UnitERd<double> r{L.n, L.m, col / Nc, col % Nc, load_ph<double>(ph, 0)};
  const int kind = row / Nc, e = row % Nc, i = e % L.n, j = e / L.n;
  double2 v = kind == 0 ? A_x<double>(r, w, i, j) + mu * M_x<double>(r, L, i, j)
                        : A_y<double>(r, w, i, j) + mu * M_y<double>(r, L, i, j);
  K[(long)col * Dc + row] = v;
}

__global__ void k_assemble_node(Lvl<double> L, const double* ph, double shift, double2* K) {
  const int Nc = L.n * L.m;
  const int row = blockIdx.x * blockDim.x + threadIdx.x, col = blockIdx.y;
  if (row >= Nc || col >= Nc) return;
  const UnitNRd<double> r{L.n, L.m, col, load_ph<double>(ph, 0)};
  double2 v = P_at<double>(r, L, row % L.n, row / L.n);
  v.x += shift / Nc;  // k = 0: the constant mode gets eigenvalue `shift` (zero-mean solutions)
  K[(long)col * Nc + row] = v;
}

// In-place Cholesky (lower, column-major) of a Hermitian positive definite matrix; one block.
__global__ void k_cholesky(double2* A, int n, float2* A32, int* info) {
  __shared__ double piv;
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x == 0) {
      const double d = A[(long)k * n + k].x;
      piv = (d > 0.0 && isfinite(d)) ? sqrt(d) : -1.0;
      if (piv < 0 && *info == 0) *info = k + 1;
      A[(long)k * n + k] = make_double2(piv > 0 ? piv : 1.0, 0.0);
    }
    __syncthreads();
    const double p = piv > 0 ? piv : 1.0;
    for (int i = k + 1 + threadIdx.x; i < n; i += blockDim.x) {
      double2 v = A[(long)k * n + i];
      A[(long)k * n + i] = make_double2(v.x / p, v.y / p);
    }
    __syncthreads();
    const int rem = n - k - 1;
    for (long t = threadIdx.x; t < (long)rem * rem; t += blockDim.x) {
      const int jj = k + 1 + int(t / rem), ii = k + 1 + int(t % rem);
      if (ii < jj) continue;
      const double2 lik = A[(long)k * n + ii], ljk = A[(long)k * n + jj];
      double2 v = A[(long)jj * n + ii];
      // A[ii][jj] -= L[ii][k] * conj(L[jj][k])
      v.x -= lik.x * ljk.x + lik.y * ljk.y;
      v.y -= lik.y * ljk.x - lik.x * ljk.y;
      A[(long)jj * n + ii] = v;
    }
    __syncthreads();
  }
  for (long t = threadIdx.x; t < (long)n * n; t += blockDim.x) {
    const int jj = int(t / n), ii = int(t % n);
    const double2 v = ii >= jj ? A[t] : make_double2(0.0, 0.0);
    A[t] = v;
    A32[t] = make_float2(float(v.x), float(v.y));
  }
}

// Solve L L^* x = b for each column (one warp per column).
template <class T>
__global__ void k_chol_solve(const cx<T>* __restrict__ Lbase, int n, const cx<T>* __restrict__ B, long ldb,
                             cx<T>* __restrict__ X, long ldx, int ncols, int cpg, int ngroups, int goff) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (warp >= ncols) return;
  const cx<T>* Lf = Lbase + (long)((warp / cpg + goff) % ngroups) * n * n;
  chol_solve_warp<T>(Lf, n, B + warp * ldb, X + warp * ldx, lane);
}

// One colour of the node-patch block Gauss-Seidel sweep for A + mu M.
template <class T>
__global__ void k_edge_smooth(Lvl<T> L, Wts<T> w, const T* __restrict__ k3, T mu, const double* ph, int cpg,
                              cx<T>* X, const cx<T>* __restrict__ B, long ld, int ci, int cj) {
  const int i = 2 * (blockIdx.x * kBX + threadIdx.x) + ci, j = 2 * (blockIdx.y * kBY + threadIdx.y) + cj;
  const int c = blockIdx.z;
  if (i >= L.n || j >= L.m) return;
  const Ph<T> p = load_ph<T>(ph, c / cpg);
  const ERd<T> r{X + c * ld, L.n, L.m, p};
  const ERd<T> rb{B + c * ld, L.n, L.m, p};
  if (inside(i, j, L.n, L.m, 1, 1))
    edge_smooth_at<T>(L, inner<T>(w), k3, mu, p, inner_e<T>(X + c * ld, L.n, L.m), inner_e<T>(B + c * ld, L.n, L.m),
                      X + c * ld, i, j);
  else
    edge_smooth_at<T>(L, w, k3, mu, p, r, rb, X + c * ld, i, j);
}

// One colour of point Gauss-Seidel for P = L^* M L.
template <class T>
__global__ void k_node_smooth(Lvl<T> L, const double* ph, int cpg, cx<T>* X, const cx<T>* __restrict__ B, long ld,
                              int ci, int cj) {
  const int i = 2 * (blockIdx.x * kBX + threadIdx.x) + ci, j = 2 * (blockIdx.y * kBY + threadIdx.y) + cj;
  const int c = blockIdx.z;
  if (i >= L.n || j >= L.m) return;
  const NRd<T> r{X + c * ld, L.n, L.m, load_ph<T>(ph, c / cpg)};
  if (inside(i, j, L.n, L.m, 1, 1))
    node_smooth_at<T>(L, inner_n<T>(X + c * ld, L.n), X + c * ld, B + c * ld, i, j);
  else
    node_smooth_at<T>(L, r, X + c * ld, B + c * ld, i, j);
}

// ---- fused coarse-level V-cycles ---------------------------------------------
// The levels from `top` down to the coarsest run as one kernel: one CTA per
// column walks the rest of the V-cycle (zero, pre-smoothing by colour, residual
// and restriction on the way down; the coarsest triangular solves; prolongation
// and post-smoothing on the way up) with block-wide barriers between the steps.
// Every point update is the function the one-launch-per-step kernels call, in
// the same colour order, so the result is the one of the unfused V-cycle.
// The level vectors live in shared memory for the whole cycle: x on every tail
// level, b below the top one (the top right-hand side is read in place) and one
// residual buffer of the top level's size; the top x is written out at the end.
template <class T> struct TailLevel {
  Lvl<T> L;
  Wts<T> w;     // edge cycles only
  const T* k3;  // edge cycles only
  int sx, sb;   // shared-memory offsets (elements) of x and b; sb unused at the top
};
template <class T> struct TailArgs {
  int nl;  // levels in the tail, the last one the coarsest
  TailLevel<T> lev[kMaxLevels];
  int sr;           // shared-memory offset of the residual buffer
  int sf;           // shared-memory offset of the column's coarsest factor (leading dimension nfac + 1), or -1
  const cx<T>* b0;  // top level right-hand sides and solutions, columns at stride ld0
  cx<T>* x0;
  long ld0, len0;   // len0: values per top-level column
  const double* ph;
  int cpg;
  const cx<T>* factor;  // per-group coarsest Cholesky factors (nfac x nfac)
  int nfac, ngroups, goff;
  T mu;
  int nu_pre, nu_post;
};
constexpr int kTailThreads = 512;
constexpr long kTailMaxNodes = 4096;        // a level joins the tail when it has at most this many nodes
constexpr int kTailSmemBytes = 200 * 1024;  // and the tail's shared-memory vectors fit in this

template <class T> __device__ __forceinline__ const cx<T>* tail_b(const TailArgs<T>& a, cx<T>* sm, int l, int c) {
  return l == 0 ? a.b0 + c * a.ld0 : sm + a.lev[l].sb;
}

// Copy of the column's coarsest factor into shared memory (the block's first barrier
// orders it before the solve).
template <class T> __device__ __forceinline__ void stage_factor(const TailArgs<T>& a, const cx<T>* F, cx<T>* sm) {
  if (a.sf < 0) return;
  const int n = a.nfac;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) sm[a.sf + (t / n) * (n + 1) + t % n] = F[t];
}

// Range [lo, hi) of lattice steps a (point i0 + s a, 0 <= a < na) whose point lies in [ilo, ihi].
__device__ __forceinline__ void lattice_range(int i0, int s, int na, int ilo, int ihi, int& lo, int& hi) {
  lo = ilo <= i0 ? 0 : min(na, (ilo - i0 + s - 1) / s);
  hi = ihi < i0 ? 0 : min(na, (ihi - i0) / s + 1);
  hi = max(hi, lo);
}

// Calls f(i, j, inner) for every point (i0 + s a, j0 + s b), 0 <= a < na, 0 <= b < nb,
// spread over the block's threads: first the points with i in [ilo, ihi] and j in
// [jlo, jhi] (inner = true), then the frame around them, so that only the warp at
// the seam mixes the two kinds.
template <class F>
__device__ __forceinline__ void for_lattice(int i0, int j0, int s, int na, int nb, int ilo, int ihi, int jlo, int jhi,
                                            F&& f) {
  int alo, ahi, blo, bhi;
  lattice_range(i0, s, na, ilo, ihi, alo, ahi);
  lattice_range(j0, s, nb, jlo, jhi, blo, bhi);
  const int nai = ahi - alo, nbi = bhi - blo, nin = nai * nbi;
  const int nrows = (nb - nbi) * na, total = na * nb;
  for (int t = threadIdx.x; t < total; t += blockDim.x) {
    int a, b;
    if (t < nin) {
      a = alo + t % nai;
      b = blo + t / nai;
    } else if (t - nin < nrows) {  // whole rows below and above the inner block
      const int u = t - nin, r = u / na;
      a = u % na;
      b = r < blo ? r : bhi + (r - blo);
    } else {  // the side pieces of the inner rows
      const int u = t - nin - nrows, w = na - nai, k = u % w;
      b = blo + u / w;
      a = k < alo ? k : ahi + (k - alo);
    }
    f(i0 + s * a, j0 + s * b, t < nin);
  }
}

template <class T>
__global__ void __launch_bounds__(kTailThreads) k_node_tail(TailArgs<T> a) {
  extern __shared__ float4 fine_sm[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(fine_sm);
  const int c = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const Ph<T> p = load_ph<T>(a.ph, c / a.cpg);
  const cx<T>* F = a.factor + (long)((c / a.cpg + a.goff) % a.ngroups) * a.nfac * a.nfac;
  stage_factor<T>(a, F, sm);
  // colour q of (0,0), (1,0), (0,1), (1,1); inner nodes have all neighbours on the level
  auto sweep = [&](const Lvl<T>& L, cx<T>* x, const cx<T>* b, int q) {
    const int ci = q & 1, cj = q >> 1;
    const NRdPlain<T> rx{x, L.n, L.m, p};
    for_lattice(ci, cj, 2, (L.n - ci + 1) / 2, (L.m - cj + 1) / 2, 1, L.n - 2, 1, L.m - 2, [&](int i, int j, bool in) {
      if (in)
        node_smooth_at<T>(L, inner_n<T>(x, L.n), x, b, i, j);
      else
        node_smooth_at<T>(L, rx, x, b, i, j);
    });
    __syncthreads();
  };
  cx<T>* r = sm + a.sr;
  for (int l = 0; l < a.nl - 1; ++l) {
    const Lvl<T> L = a.lev[l].L;
    const int N = L.n * L.m;
    cx<T>* x = sm + a.lev[l].sx;
    const cx<T>* b = tail_b(a, sm, l, c);
    for (int t = tid; t < N; t += nt) x[t] = czero<T>();
    __syncthreads();
    for (int it = 0; it < a.nu_pre; ++it)
      for (int q = 0; q < 4; ++q) sweep(L, x, b, q);
    const NRdPlain<T> rx{x, L.n, L.m, p};
    for_lattice(0, 0, 1, L.n, L.m, 1, L.n - 2, 1, L.m - 2, [&](int i, int j, bool in) {
      r[j * L.n + i] = in ? apply_nodal_at<T>(L, inner_n<T>(x, L.n), b, T(-1), T(1), i, j)
                          : apply_nodal_at<T>(L, rx, b, T(-1), T(1), i, j);
    });
    __syncthreads();
    // restriction at (I, J) reads fine nodes 2I-1 .. 2I+1
    const Lvl<T> C = a.lev[l + 1].L;
    cx<T>* bc = sm + a.lev[l + 1].sb;
    const NRdPlain<T> rr{r, L.n, L.m, p};
    for_lattice(0, 0, 1, C.n, C.m, 1, (L.n - 2) / 2, 1, (L.m - 2) / 2, [&](int I, int J, bool in) {
      bc[J * C.n + I] = in ? restrict_node_at<T>(inner_n<T>(r, L.n), I, J) : restrict_node_at<T>(rr, I, J);
    });
    __syncthreads();
  }
  if (tid < 32) {
    const int l = a.nl - 1;
    if (a.sf >= 0)
      chol_solve_warp_cols<T>(sm + a.sf, a.nfac + 1, a.nfac, tail_b(a, sm, l, c), sm + a.lev[l].sx, tid);
    else
      chol_solve_warp<T>(F, a.nfac, tail_b(a, sm, l, c), sm + a.lev[l].sx, tid);
  }
  __syncthreads();
  for (int l = a.nl - 2; l >= 0; --l) {
    const Lvl<T> L = a.lev[l].L, C = a.lev[l + 1].L;
    cx<T>* x = sm + a.lev[l].sx;
    const cx<T>* b = tail_b(a, sm, l, c);
    const cx<T>* xc = sm + a.lev[l + 1].sx;
    const NRdPlain<T> rc{xc, C.n, C.m, p};
    // prolongation at fine (i, j) reads coarse nodes i/2 .. i/2 + 1
    for_lattice(0, 0, 1, L.n, L.m, 0, 2 * C.n - 3, 0, 2 * C.m - 3, [&](int i, int j, bool in) {
      const int e = j * L.n + i;
      x[e] = x[e] + (in ? prolong_node_at<T>(inner_n<T>(xc, C.n), i, j) : prolong_node_at<T>(rc, i, j));
    });
    __syncthreads();
    for (int it = 0; it < a.nu_post; ++it)
      for (int q = 3; q >= 0; --q) sweep(L, x, b, q);
  }
  const cx<T>* x = sm + a.lev[0].sx;
  for (long t = tid; t < a.len0; t += nt) a.x0[c * a.ld0 + t] = x[t];
}

template <class T>
__global__ void __launch_bounds__(kTailThreads) k_edge_tail(TailArgs<T> a) {
  extern __shared__ float4 fine_sm[];
  cx<T>* sm = reinterpret_cast<cx<T>*>(fine_sm);
  const int c = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const Ph<T> p = load_ph<T>(a.ph, c / a.cpg);
  const cx<T>* F = a.factor + (long)((c / a.cpg + a.goff) % a.ngroups) * a.nfac * a.nfac;
  stage_factor<T>(a, F, sm);
  // colour q of (0,0), (1,0), (0,1), (1,1); inner patches have all their edges and cells on the level
  auto sweep = [&](const TailLevel<T>& TL, cx<T>* x, const cx<T>* b, int q) {
    const Lvl<T>& L = TL.L;
    const int ci = q & 1, cj = q >> 1;
    const ERdPlain<T> rx{x, L.n, L.m, p};
    const ERdPlain<T> rb{b, L.n, L.m, p};
    for_lattice(ci, cj, 2, (L.n - ci + 1) / 2, (L.m - cj + 1) / 2, 1, L.n - 2, 1, L.m - 2, [&](int i, int j, bool in) {
      if (in)
        edge_smooth_at<T>(L, inner<T>(TL.w), TL.k3, a.mu, p, inner_e<T>(x, L.n, L.m), inner_e<T>(b, L.n, L.m), x, i,
                          j);
      else
        edge_smooth_at<T>(L, TL.w, TL.k3, a.mu, p, rx, rb, x, i, j);
    });
    __syncthreads();
  };
  cx<T>* r = sm + a.sr;
  for (int l = 0; l < a.nl - 1; ++l) {
    const TailLevel<T> TL = a.lev[l];
    const Lvl<T> L = TL.L;
    const int N = L.n * L.m;
    cx<T>* x = sm + TL.sx;
    const cx<T>* b = tail_b(a, sm, l, c);
    for (int t = tid; t < 2 * N; t += nt) x[t] = czero<T>();
    __syncthreads();
    for (int it = 0; it < a.nu_pre; ++it)
      for (int q = 0; q < 4; ++q) sweep(TL, x, b, q);
    const ERdPlain<T> rx{x, L.n, L.m, p};
    for_lattice(0, 0, 1, L.n, L.m, 1, L.n - 2, 1, L.m - 2, [&](int i, int j, bool in) {
      cx<T> yx, yy;
      if (in)
        apply_edge_at<T>(L, inner<T>(TL.w), inner_e<T>(x, L.n, L.m), b, T(-1), -a.mu, T(1), i, j, yx, yy);
      else
        apply_edge_at<T>(L, TL.w, rx, b, T(-1), -a.mu, T(1), i, j, yx, yy);
      r[j * L.n + i] = yx;
      r[N + j * L.n + i] = yy;
    });
    __syncthreads();
    // restriction at (I, J) reads fine edges with indices 2I-1 .. 2I+1
    const Lvl<T> C = a.lev[l + 1].L;
    const int Nc = C.n * C.m;
    cx<T>* bc = sm + a.lev[l + 1].sb;
    const ERdPlain<T> rr{r, L.n, L.m, p};
    for_lattice(0, 0, 1, C.n, C.m, 1, (L.n - 2) / 2, 1, (L.m - 2) / 2, [&](int I, int J, bool in) {
      cx<T> vx, vy;
      if (in)
        restrict_edge_at<T>(inner_e<T>(r, L.n, L.m), I, J, vx, vy);
      else
        restrict_edge_at<T>(rr, I, J, vx, vy);
      bc[J * C.n + I] = vx;
      bc[Nc + J * C.n + I] = vy;
    });
    __syncthreads();
  }
  if (tid < 32) {
    const int l = a.nl - 1;
    if (a.sf >= 0)
      chol_solve_warp_cols<T>(sm + a.sf, a.nfac + 1, a.nfac, tail_b(a, sm, l, c), sm + a.lev[l].sx, tid);
    else
      chol_solve_warp<T>(F, a.nfac, tail_b(a, sm, l, c), sm + a.lev[l].sx, tid);
  }
  __syncthreads();
  for (int l = a.nl - 2; l >= 0; --l) {
    const TailLevel<T> TL = a.lev[l];
    const Lvl<T> L = TL.L, C = a.lev[l + 1].L;
    const int N = L.n * L.m;
    cx<T>* x = sm + TL.sx;
    const cx<T>* b = tail_b(a, sm, l, c);
    const cx<T>* xc = sm + a.lev[l + 1].sx;
    const ERdPlain<T> rc{xc, C.n, C.m, p};
    // prolongation at fine (i, j) reads coarse edges with indices i/2 .. i/2 + 1
    for_lattice(0, 0, 1, L.n, L.m, 0, 2 * C.n - 3, 0, 2 * C.m - 3, [&](int i, int j, bool in) {
      cx<T> vx, vy;
      if (in)
        prolong_edge_at<T>(inner_e<T>(xc, C.n, C.m), i, j, vx, vy);
      else
        prolong_edge_at<T>(rc, i, j, vx, vy);
      const int e = j * L.n + i;
      x[e] = x[e] + vx;
      x[N + e] = x[N + e] + vy;
    });
    __syncthreads();
    for (int it = 0; it < a.nu_post; ++it)
      for (int q = 3; q >= 0; --q) sweep(TL, x, b, q);
  }
  const cx<T>* x = sm + a.lev[0].sx;
  for (long t = tid; t < a.len0; t += nt) a.x0[c * a.ld0 + t] = x[t];
}

template <class T> const cx<T>* edge_factor(const KData& K);
template <> const double2* edge_factor<double>(const KData& K) { return K.edge64; }
template <> const float2* edge_factor<float>(const KData& K) { return K.edge32; }
template <class T> const cx<T>* node_factor(const KData& K);
template <> const double2* node_factor<double>(const KData& K) { return K.node64; }
template <> const float2* node_factor<float>(const KData& K) { return K.node32; }
template <class T> const T* k3_of(const Level& L);
template <> const double* k3_of<double>(const Level& L) { return L.k3_64; }
template <> const float* k3_of<float>(const Level& L) { return L.k3_32; }

// Algorithmic bytes of one colour launch: every x value is read once (the
// patch residuals need the neighbours), the colour's edges (half of them) read b
// and write x, plus the colour's patch factors (6 reals per node) and 1/eps.
template <class T> double smooth_bytes(const Level& L, int ncols) {
  const double c = 2.0 * sizeof(T), D = (double)L.D(), N = (double)L.N();
  return ncols * (c * D + 2 * c * D / 2) + 6.0 * sizeof(T) * N / 4 + sizeof(T) * N;
}
// point smoother: read x once, read b and write x on a quarter of the nodes
template <class T> double node_smooth_bytes(const Level& L, int ncols) {
  const double c = 2.0 * sizeof(T), N = (double)L.N();
  return ncols * (c * N + 2 * c * N / 4);
}

inline dim3 half_grid(int n, int m, int ncols) {
  return dim3(((n + 1) / 2 + kBX - 1) / kBX, ((m + 1) / 2 + kBY - 1) / kBY, ncols);
}

}  // namespace

int num_levels(int n, int m, int coarsest) {
  if (n < 2 || m < 2 || coarsest < 2) return PBS_EINVAL;
  int L = 1;
  while (n % 2 == 0 && m % 2 == 0 && n / 2 >= coarsest && m / 2 >= coarsest && L < kMaxLevels) {
    n /= 2;
    m /= 2;
    ++L;
  }
  return L;
}

void build_hierarchy(DevMem& mem, Hierarchy& H, const double* d_eps, int coarsest, cudaStream_t s) {
  H.nlev = num_levels(H.n, H.m, coarsest);
  if (H.nlev < 1) fail(-1, "invalid mesh for the hierarchy");
  int* d_bad = (int*)mem.alloc(2 * sizeof(unsigned long long));
  unsigned long long* d_wmax = (unsigned long long*)d_bad + 1;
  H.allocs.push_back(d_bad);
  PBS_CUDA(cudaMemsetAsync(d_bad, 0, 2 * sizeof(unsigned long long), s));
  int n = H.n, m = H.m;
  for (int l = 0; l < H.nlev; ++l) {
    Level& L = H.lev[l];
    L.n = n;
    L.m = m;
    L.h1 = H.a / n;
    L.h2 = H.b / m;
    const long N = (long)n * m;
    L.winv64 = (double*)mem.alloc(N * sizeof(double));
    L.winv32 = (float*)mem.alloc(N * sizeof(float));
    L.k3_64 = (double*)mem.alloc(6 * N * sizeof(double));
    L.k3_32 = (float*)mem.alloc(6 * N * sizeof(float));
    H.allocs.insert(H.allocs.end(), {L.winv64, L.winv32, L.k3_64, L.k3_32});
    if (l == 0) {
      k_inv_eps<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(d_eps, L.winv64, L.winv32, N, d_bad, d_wmax);
    } else {
      const Level& F = H.lev[l - 1];
      k_coarsen_w<<<dim3((n + kBX - 1) / kBX, (m + kBY - 1) / kBY), dim3(kBX, kBY), 0, s>>>(F.winv64, F.n, L.winv64,
                                                                                           L.winv32, n, m);
    }
    PBS_LAUNCHED();
    if (l == 0) {
      L.wdf = (float2*)mem.alloc(N * sizeof(float2));
      H.allocs.push_back(L.wdf);
      k_weights_df<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(L.winv64, 1.0 / (L.h1 * L.h2), L.wdf, N);
      PBS_LAUNCHED();
    }
    const double m1 = 2.0 / 3.0 * L.h2 / L.h1, m2 = 2.0 / 3.0 * L.h1 / L.h2;
    k_patch_factors<<<dim3((n + kBX - 1) / kBX, (m + kBY - 1) / kBY), dim3(kBX, kBY), 0, s>>>(
        L.winv64, n, m, 1.0 / (L.h1 * L.h2), m1, m2, H.mu, L.k3_64, L.k3_32);
    PBS_LAUNCHED();
    n /= 2;
    m /= 2;
  }
  int bad = 0;
  unsigned long long wmax = 0;
  PBS_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
  PBS_CUDA(cudaMemcpyAsync(&wmax, d_wmax, sizeof(wmax), cudaMemcpyDeviceToHost, s));
  PBS_CUDA(cudaStreamSynchronize(s));
  if (bad) fail(-1, "eps must be finite and positive");
  std::memcpy(&H.winv_max, &wmax, sizeof(double));
  H.lev[0].wmax = H.winv_max / (H.lev[0].h1 * H.lev[0].h2);
  const Level& C = H.lev[H.nlev - 1];
  if (C.D() > kMaxCoarseEdges) fail(-1, "coarsest level too large for the dense solve (raise coarsest or use sides with more factors of 2)");
}

void free_hierarchy(DevMem& mem, Hierarchy& H) {
  for (void* p : H.allocs) mem.free(p);
  H.allocs.clear();
  H.nlev = 0;
}

void alloc_kdata(DevMem& mem, const Hierarchy& H, KData& K, int ngroups) {
  const Level& C = H.lev[H.nlev - 1];
  const int Dc = (int)C.D(), Nc = (int)C.N();
  if (K.ngroups == ngroups && K.Dc == Dc && K.d_info) return;
  free_kdata(mem, K);
  KData k;  // filled completely before it replaces K: a failed allocation leaves K empty
  k.owner = true;
  try {
    k.d_ph = (double*)mem.alloc(12ull * ngroups * sizeof(double));
    k.d_gamma = (int*)mem.alloc(3ull * ngroups * sizeof(int));
    k.edge64 = (double2*)mem.alloc((size_t)ngroups * Dc * Dc * sizeof(double2));
    k.edge32 = (float2*)mem.alloc((size_t)ngroups * Dc * Dc * sizeof(float2));
    k.node64 = (double2*)mem.alloc((size_t)ngroups * Nc * Nc * sizeof(double2));
    k.node32 = (float2*)mem.alloc((size_t)ngroups * Nc * Nc * sizeof(float2));
    k.d_info = (int*)mem.alloc(2 * sizeof(int));
  } catch (...) {
    free_kdata(mem, k);
    throw;
  }
  k.ngroups = ngroups;
  k.Dc = Dc;
  k.Nc = Nc;
  k.k1.assign(ngroups, 0.0);
  k.k2.assign(ngroups, 0.0);
  k.gamma.assign(ngroups, 0);
  K = k;
}

void set_group_k(DevMem& mem, const Hierarchy& H, KData& K, int g, double k1, double k2, cudaStream_t s) {
  if (g < 0 || g >= K.ngroups) fail(PBS_EINVAL, "group out of range");
  double ph[4] = {std::cos(k1 * H.a), std::sin(k1 * H.a), std::cos(k2 * H.b), std::sin(k2 * H.b)};
  const bool gamma = std::hypot(ph[0] - 1.0, ph[1]) < 1e-14 && std::hypot(ph[2] - 1.0, ph[3]) < 1e-14;
  if (gamma) {  // the exact phases at the lattice points
    ph[0] = 1.0; ph[1] = 0.0; ph[2] = 1.0; ph[3] = 0.0;
  }
  K.k1[g] = k1;
  K.k2[g] = k2;
  K.gamma[g] = gamma;
  const int gi = gamma ? 1 : 0;
  for (int rep = 0; rep < 3; ++rep) {
    const long e = (long)rep * K.ngroups + g;
    PBS_CUDA(cudaMemcpyAsync(K.d_ph + 4 * e, ph, 4 * sizeof(double), cudaMemcpyHostToDevice, s));
    PBS_CUDA(cudaMemcpyAsync(K.d_gamma + e, &gi, sizeof(int), cudaMemcpyHostToDevice, s));
  }
  const Level& C = H.lev[H.nlev - 1];
  const int Dc = K.Dc, Nc = K.Nc;
  double2* e64 = K.edge64 + (size_t)g * Dc * Dc;
  float2* e32 = K.edge32 + (size_t)g * Dc * Dc;
  double2* n64 = K.node64 + (size_t)g * Nc * Nc;
  float2* n32 = K.node32 + (size_t)g * Nc * Nc;
  const double* gph = K.d_ph + 4 * g;
  int* d_info = K.d_info;
  PBS_CUDA(cudaMemsetAsync(d_info, 0, 2 * sizeof(int), s));
  k_assemble_edge<<<dim3((Dc + 127) / 128, Dc), 128, 0, s>>>(C.lvl<double>(), C.wts<double>(), H.mu, gph, e64);
  PBS_LAUNCHED();
  k_cholesky<<<1, 256, 0, s>>>(e64, Dc, e32, d_info);
  PBS_LAUNCHED();
  const double shift = gamma ? P_diag<double>(C.lvl<double>()) : 0.0;
  k_assemble_node<<<dim3((Nc + 127) / 128, Nc), 128, 0, s>>>(C.lvl<double>(), gph, shift, n64);
  PBS_LAUNCHED();
  k_cholesky<<<1, 256, 0, s>>>(n64, Nc, n32, d_info + 1);
  PBS_LAUNCHED();
  int info[2] = {0, 0};
  PBS_CUDA(cudaMemcpyAsync(info, d_info, 2 * sizeof(int), cudaMemcpyDeviceToHost, s));
  PBS_CUDA(cudaStreamSynchronize(s));
  if (info[0] || info[1]) fail(PBS_ENUMERIC, "coarsest-level Cholesky factorisation failed");
}

void copy_group_k(KData& K, int src, int dst, cudaStream_t s) {
  if (src < 0 || dst < 0 || src >= K.ngroups || dst >= K.ngroups) fail(PBS_EINVAL, "group out of range");
  if (src == dst) return;
  K.k1[dst] = K.k1[src];
  K.k2[dst] = K.k2[src];
  K.gamma[dst] = K.gamma[src];
  for (int rep = 0; rep < 3; ++rep) {
    const long es = (long)rep * K.ngroups + src, ed = (long)rep * K.ngroups + dst;
    PBS_CUDA(cudaMemcpyAsync(K.d_ph + 4 * ed, K.d_ph + 4 * es, 4 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    PBS_CUDA(cudaMemcpyAsync(K.d_gamma + ed, K.d_gamma + es, sizeof(int), cudaMemcpyDeviceToDevice, s));
  }
  const size_t de = (size_t)K.Dc * K.Dc, dn = (size_t)K.Nc * K.Nc;
  PBS_CUDA(cudaMemcpyAsync(K.edge64 + dst * de, K.edge64 + src * de, de * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  PBS_CUDA(cudaMemcpyAsync(K.edge32 + dst * de, K.edge32 + src * de, de * sizeof(float2), cudaMemcpyDeviceToDevice, s));
  PBS_CUDA(cudaMemcpyAsync(K.node64 + dst * dn, K.node64 + src * dn, dn * sizeof(double2), cudaMemcpyDeviceToDevice, s));
  PBS_CUDA(cudaMemcpyAsync(K.node32 + dst * dn, K.node32 + src * dn, dn * sizeof(float2), cudaMemcpyDeviceToDevice, s));
}

KData kdata_view(const KData& K, int g) {
  KData v;
  v.ngroups = 1;
  v.Dc = K.Dc;
  v.Nc = K.Nc;
  v.d_ph = K.d_ph + 4 * g;
  v.d_gamma = K.d_gamma + g;
  v.edge64 = K.edge64 + (size_t)g * K.Dc * K.Dc;
  v.edge32 = K.edge32 + (size_t)g * K.Dc * K.Dc;
  v.node64 = K.node64 + (size_t)g * K.Nc * K.Nc;
  v.node32 = K.node32 + (size_t)g * K.Nc * K.Nc;
  v.d_info = K.d_info;
  v.k1 = {K.k1[g]};
  v.k2 = {K.k2[g]};
  v.gamma = {K.gamma[g]};
  v.owner = false;
  return v;
}

KData kdata_chunk(const KData& K, int v0) {
  KData v;
  v.ngroups = K.ngroups;
  v.Dc = K.Dc;
  v.Nc = K.Nc;
  v.d_ph = K.d_ph + 4L * v0;
  v.d_gamma = K.d_gamma + v0;
  v.edge64 = K.edge64;
  v.edge32 = K.edge32;
  v.node64 = K.node64;
  v.node32 = K.node32;
  v.d_info = K.d_info;
  v.k1 = K.k1;
  v.k2 = K.k2;
  v.gamma = K.gamma;
  v.goff = (K.goff + v0) % K.ngroups;
  v.owner = false;
  return v;
}

void free_kdata(DevMem& mem, KData& K) {
  if (K.owner)
    for (void* p : {(void*)K.d_ph, (void*)K.d_gamma, (void*)K.edge64, (void*)K.edge32, (void*)K.node64,
                    (void*)K.node32, (void*)K.d_info})
      if (p) mem.free(p);
  K = KData();
}

template <class T> void alloc_mg_work(DevMem& mem, const Hierarchy& H, int ncols, bool nodal, MgWork<T>& w) {
  free_mg_work<T>(mem, w);
  w.ncols = ncols;
  for (int l = 0; l < H.nlev; ++l) {
    const long len = nodal ? H.lev[l].N() : H.lev[l].D();
    const size_t bytes = (size_t)len * ncols * sizeof(cx<T>);
    w.r[l] = (cx<T>*)mem.alloc(bytes);
    if (l > 0) {
      w.x[l] = (cx<T>*)mem.alloc(bytes);
      w.b[l] = (cx<T>*)mem.alloc(bytes);
    }
  }
}

template <class T> void free_mg_work(DevMem& mem, MgWork<T>& w) {
  for (int l = 0; l < kMaxLevels; ++l) {
    for (cx<T>** p : {&w.x[l], &w.b[l], &w.r[l]}) {
      if (*p) mem.free(*p);
      *p = nullptr;
    }
  }
  w.ncols = 0;
}

namespace {

// Columns of `len` values at stride ld set to zero (one call when they are contiguous).
template <class T> void zero_columns(cx<T>* x, long ld, long len, int ncols, cudaStream_t s) {
  if (ld == len) {
    PBS_CUDA(cudaMemsetAsync(x, 0, (size_t)len * ncols * sizeof(cx<T>), s));
  } else {
    for (int c = 0; c < ncols; ++c) PBS_CUDA(cudaMemsetAsync(x + c * ld, 0, len * sizeof(cx<T>), s));
  }
}

// Shared-memory elements of a fused tail from level l: x on every level, b below
// the top one and a residual buffer of the top level's size.
inline long tail_smem_elems(const Hierarchy& H, int l, bool nodal) {
  auto len = [&](int k) { return nodal ? H.lev[k].N() : H.lev[k].D(); };
  long e = 2 * len(l);
  for (int k = l + 1; k < H.nlev; ++k) e += 2 * len(k);
  return e;
}

// The fused tail covers level l and everything below when l is not the coarsest,
// has at most kTailMaxNodes nodes and its vectors fit in shared memory.
template <class T> bool tail_from(const Hierarchy& H, int l, bool nodal) {
  return l < H.nlev - 1 && H.lev[l].N() <= kTailMaxNodes &&
         tail_smem_elems(H, l, nodal) * (long)sizeof(cx<T>) <= kTailSmemBytes;
}
template <class T> void set_tail_smem() {
  static PerDeviceOnce once;
  once([] {
    PBS_CUDA(cudaFuncSetAttribute(k_node_tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTailSmemBytes));
    PBS_CUDA(cudaFuncSetAttribute(k_edge_tail<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, kTailSmemBytes));
  });
}

// Algorithmic bytes of a fused tail: the top right-hand sides in and solutions
// out, the patch factors of its edge levels and the coarsest factors of the
// groups its columns belong to (the level vectors stay on chip).
template <class T> double tail_bytes(const Hierarchy& H, int l, int ncols, int cpg, bool nodal) {
  const Level& L = H.lev[l];
  const Level& C = H.lev[H.nlev - 1];
  const double len = nodal ? (double)L.N() : (double)L.D(), nfac = nodal ? (double)C.N() : (double)C.D();
  double b = 2.0 * len * ncols * sizeof(cx<T>) + nfac * nfac * sizeof(cx<T>) * ((ncols + cpg - 1) / cpg);
  if (!nodal)
    for (int k = l; k < H.nlev - 1; ++k) b += 6.0 * sizeof(T) * H.lev[k].N();
  return b;
}

// The tiled fine-level nodal kernels need the halo to wrap at most once (sides of at
// least one tile plus both halos) and at most three sweeps per side.
constexpr int kFineMaxNu = 3;
constexpr size_t kSmemOptIn = 232448;  // largest dynamic shared memory a CTA may opt into (227 KB)
inline bool fine_fits(const Level& L, int ft) {
  const int need = ft + 8 * kFineMaxNu + 3;
  return L.n >= need && L.m >= need;
}
inline bool fine_tiled(const Level& L, int nu_pre, int nu_post) {
  return nu_pre >= 1 && nu_post >= 1 && nu_pre <= kFineMaxNu && nu_post <= kFineMaxNu && fine_fits(L, 32);
}
// shared memory of the tiled kernels for tile side ft and nu sweeps
template <class T> size_t fine_down_smem(int ft, int nu) {
  const size_t W = ft + 8 * nu + 3;
  return 2 * W * W * sizeof(cx<T>);
}
template <class T> size_t fine_up_smem(int ft, int nu) {
  const size_t W = ft + 8 * nu, Wc = W / 2 + 1;
  return (2 * W * W + Wc * Wc) * sizeof(cx<T>);
}
// the largest of fn(nu) over the sweep counts whose shared memory fits a CTA
template <class F> size_t fine_smem_cap(F&& fn) {
  size_t m = 0;
  for (int nu = 1; nu <= kFineMaxNu; ++nu)
    if (fn(nu) <= kSmemOptIn) m = std::max(m, fn(nu));
  return m;
}
template <class T, int FT> void set_fine_smem() {
  static PerDeviceOnce once;
  once([] {
    PBS_CUDA(cudaFuncSetAttribute(k_node_down<T, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)fine_smem_cap([](int nu) { return fine_down_smem<T>(FT, nu); })));
    PBS_CUDA(cudaFuncSetAttribute(k_node_up<T, FT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)fine_smem_cap([](int nu) { return fine_up_smem<T>(FT, nu); })));
  });
}
// shared memory of the register-blocked steps (FP32, one sweep per side)
template <int FT, int NT> void set_fine_rb_smem() {
  static PerDeviceOnce once;
  once([] {
    PBS_CUDA(cudaFuncSetAttribute(k_node_down_rb<FT, NT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)RbDown<FT, NT, 1>::smem));
    PBS_CUDA(cudaFuncSetAttribute(k_node_up_rb<FT, NT, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)RbUp<FT, NT, 1>::smem));
  });
}
// launch shapes of the tiled steps offered to the autotuner: (tile side, threads,
// register-blocked); the first one fits every level the tiled path takes, the
// register-blocked ones run FP32 cycles with one sweep per side
struct FineShape {
  int ft, nt;
  bool rb;
};
constexpr FineShape kFineShapes[] = {{32, 256, false}, {64, 512, false}, {64, 256, false},
                                     {32, 256, true},  {64, 512, true},  {32, 128, true}};
constexpr int kNumFineShapes = 6;
template <class T>
int fine_shapes(const Level& L, int nu, bool down, FineShape* out) {
  int n = 0;
  for (const FineShape& f : kFineShapes) {
    if (f.rb && (!std::is_same<T, float>::value || nu != 1)) continue;
    const size_t sm = f.rb ? 0 : down ? fine_down_smem<T>(f.ft, nu) : fine_up_smem<T>(f.ft, nu);
    if (fine_fits(L, f.ft) && sm <= kSmemOptIn) out[n++] = f;
  }
  return n;
}
// algorithmic bytes of a tiled step: each level vector read or written once
// (down: b in, x and the coarse right-hand side out; up: b, x, the coarse
// correction in, x out)
template <class T> double fine_bytes(const Level& L, int ncols, int, bool down) {
  const double v = (double)L.N() * ncols * sizeof(cx<T>);
  return down ? 2.25 * v : 3.25 * v;
}

template <class T> std::string fine_key(const Level& L, int ncols, int cpg) {
  return std::to_string(L.n) + "x" + std::to_string(L.m) + "|c" + std::to_string(ncols) + "|g" +
         std::to_string(cpg) + "|" + (sizeof(T) == 4 ? "f32" : "f64") + "|" + device_tag();
}

template <class T, int FT>
void launch_node_down(const Level& L, const Level& C, const KData& K, MgWork<T>& w, int l, const cx<T>* b,
                      const cx<T>* x0, long ld, int ncols, int cpg, int nu, int nt, cudaStream_t s) {
  set_fine_smem<T, FT>();
  const dim3 grid((L.n + FT - 1) / FT, (L.m + FT - 1) / FT, ncols);
  k_node_down<T, FT><<<grid, nt, fine_down_smem<T>(FT, nu), s>>>(L.lvl<T>(), C.n, C.m, K.d_ph, cpg, b, ld, x0, ld,
                                                                  w.r[l], L.N(), w.b[l + 1], C.N(), nu);
  PBS_LAUNCHED();
}

template <class T, int FT>
void launch_node_up(const Level& L, const Level& C, const KData& K, MgWork<T>& w, int l, const cx<T>* b, cx<T>* x,
                    long ld, int ncols, int cpg, int nu, int nt, cudaStream_t s) {
  set_fine_smem<T, FT>();
  const dim3 grid((L.n + FT - 1) / FT, (L.m + FT - 1) / FT, ncols);
  k_node_up<T, FT><<<grid, nt, fine_up_smem<T>(FT, nu), s>>>(L.lvl<T>(), C.n, C.m, K.d_ph, cpg, b, ld, w.r[l], L.N(),
                                                              w.x[l + 1], C.N(), x, ld, nu);
  PBS_LAUNCHED();
}

template <int FT, int NT>
void launch_node_down_rb(const Level& L, const Level& C, const KData& K, MgWork<float>& w, int l, const float2* b,
                         const float2* x0, long ld, int ncols, int cpg, cudaStream_t s) {
  set_fine_rb_smem<FT, NT>();
  const dim3 grid((L.n + FT - 1) / FT, (L.m + FT - 1) / FT, ncols);
  k_node_down_rb<FT, NT, 1><<<grid, NT, RbDown<FT, NT, 1>::smem, s>>>(L.lvl<float>(), C.n, C.m, K.d_ph, cpg, b, ld,
                                                                      x0, ld, w.r[l], L.N(), w.b[l + 1], C.N());
  PBS_LAUNCHED();
}

template <int FT, int NT>
void launch_node_up_rb(const Level& L, const Level& C, const KData& K, MgWork<float>& w, int l, const float2* b,
                       float2* x, long ld, int ncols, int cpg, cudaStream_t s) {
  set_fine_rb_smem<FT, NT>();
  const dim3 grid((L.n + FT - 1) / FT, (L.m + FT - 1) / FT, ncols);
  k_node_up_rb<FT, NT, 1><<<grid, NT, RbUp<FT, NT, 1>::smem, s>>>(L.lvl<float>(), C.n, C.m, K.d_ph, cpg, b, ld,
                                                                  w.r[l], L.N(), w.x[l + 1], C.N(), x, ld);
  PBS_LAUNCHED();
}

// the register-blocked steps exist in FP32 only (fine_shapes offers them nowhere else)
template <class T>
void launch_rb(bool down, const FineShape& f, const Level& L, const Level& C, const KData& K, MgWork<T>& w, int l,
               const cx<T>* b, const cx<T>* x0, cx<T>* x, long ld, int ncols, int cpg, cudaStream_t s) {
  if constexpr (std::is_same<T, float>::value) {
    const bool s32 = f.ft == 32 && f.nt == 256, s64 = f.ft == 64 && f.nt == 512, t32 = f.ft == 32 && f.nt == 128;
    if (!s32 && !s64 && !t32) fail(-1, "nodal step: no register-blocked kernel for this shape");
    if (down) {
      if (s64) launch_node_down_rb<64, 512>(L, C, K, w, l, b, x0, ld, ncols, cpg, s);
      else if (s32) launch_node_down_rb<32, 256>(L, C, K, w, l, b, x0, ld, ncols, cpg, s);
      else launch_node_down_rb<32, 128>(L, C, K, w, l, b, x0, ld, ncols, cpg, s);
    } else {
      if (s64) launch_node_up_rb<64, 512>(L, C, K, w, l, b, x, ld, ncols, cpg, s);
      else if (s32) launch_node_up_rb<32, 256>(L, C, K, w, l, b, x, ld, ncols, cpg, s);
      else launch_node_up_rb<32, 128>(L, C, K, w, l, b, x, ld, ncols, cpg, s);
    }
  } else {
    fail(-1, "nodal step: register-blocked kernels run FP32 only");
  }
}

template <class T>
TailArgs<T> tail_args(const Hierarchy& H, const KData& K, int l, const cx<T>* b, cx<T>* x, long ld, int cpg,
                      int nu_pre, int nu_post, bool nodal, size_t* smem) {
  TailArgs<T> a{};
  a.nl = H.nlev - l;
  int off = 0;
  for (int k = 0; k < a.nl; ++k) {
    const Level& L = H.lev[l + k];
    const int len = (int)(nodal ? L.N() : L.D());
    TailLevel<T>& t = a.lev[k];
    t.L = L.lvl<T>();
    t.w = L.wts<T>();
    t.k3 = k3_of<T>(L);
    t.sx = off;
    off += len;
    if (k > 0) {
      t.sb = off;
      off += len;
    }
  }
  a.len0 = nodal ? H.lev[l].N() : H.lev[l].D();
  a.sr = off;
  off += (int)a.len0;
  const Level& Cst0 = H.lev[H.nlev - 1];
  const long nf = nodal ? Cst0.N() : Cst0.D();
  a.sf = -1;
  if ((off + nf * (nf + 1)) * (long)sizeof(cx<T>) <= kTailSmemBytes) {
    a.sf = off;
    off += (int)(nf * (nf + 1));
  }
  *smem = (size_t)off * sizeof(cx<T>);
  a.b0 = b;
  a.x0 = x;
  a.ld0 = ld;
  a.ph = K.d_ph;
  a.cpg = cpg;
  const Level& Cst = H.lev[H.nlev - 1];
  a.factor = nodal ? node_factor<T>(K) : edge_factor<T>(K);
  a.nfac = (int)(nodal ? Cst.N() : Cst.D());
  a.ngroups = K.ngroups;
  a.goff = K.goff;
  a.mu = T(H.mu);
  a.nu_pre = nu_pre;
  a.nu_post = nu_post;
  return a;
}

template <class T>
void edge_cycle(const Hierarchy& H, const KData& K, MgWork<T>& w, int l, const cx<T>* b, cx<T>* x, long ld, int ncols,
                int cpg, int nu_pre, int nu_post, cudaStream_t s) {
  const Level& L = H.lev[l];
  if (l == H.nlev - 1) {
    k_chol_solve<T><<<(ncols * 32 + 127) / 128, 128, 0, s>>>(edge_factor<T>(K), (int)L.D(), b, ld, x, ld, ncols, cpg,
                                                             K.ngroups, K.goff);
    PBS_LAUNCHED();
    return;
  }
  if (tail_from<T>(H, l, false)) {
    size_t smem = 0;
    const TailArgs<T> ta = tail_args<T>(H, K, l, b, x, ld, cpg, nu_pre, nu_post, false, &smem);
    set_tail_smem<T>();
    timer_begin(KC_EDGE_TAIL, s, tail_bytes<T>(H, l, ncols, cpg, false));
    k_edge_tail<T><<<ncols, kTailThreads, smem, s>>>(ta);
    timer_end(KC_EDGE_TAIL, s);
    PBS_LAUNCHED();
    return;
  }
  zero_columns<T>(x, ld, L.D(), ncols, s);
  const Lvl<T> lv = L.lvl<T>();
  const Wts<T> wt = L.wts<T>();
  const T mu = T(H.mu);
  for (int it = 0; it < nu_pre; ++it)
    for (int q = 0; q < 4; ++q) {
      timer_begin(KC_EDGE_SMOOTH, s, smooth_bytes<T>(L, ncols));
      k_edge_smooth<T><<<half_grid(L.n, L.m, ncols), dim3(kBX, kBY), 0, s>>>(lv, wt, k3_of<T>(L), mu, K.d_ph, cpg, x,
                                                                             b, ld, kColours[q][0], kColours[q][1]);
      timer_end(KC_EDGE_SMOOTH, s);
      PBS_LAUNCHED();
    }
  const Level& C = H.lev[l + 1];
  const long ldc = C.D();
  apply_edge<T>(L, K.d_ph, cpg, x, w.r[l], b, ld, ncols, T(-1), -mu, T(0), nullptr, T(1), s);
  restrict_edge<T>(L, C, K.d_ph, cpg, w.r[l], ld, w.b[l + 1], ldc, ncols, s);
  edge_cycle<T>(H, K, w, l + 1, w.b[l + 1], w.x[l + 1], ldc, ncols, cpg, nu_pre, nu_post, s);
  prolong_edge<T>(L, C, K.d_ph, cpg, w.x[l + 1], ldc, x, ld, ncols, true, s);
  for (int it = 0; it < nu_post; ++it)
    for (int q = 3; q >= 0; --q) {
      timer_begin(KC_EDGE_SMOOTH, s, smooth_bytes<T>(L, ncols));
      k_edge_smooth<T><<<half_grid(L.n, L.m, ncols), dim3(kBX, kBY), 0, s>>>(lv, wt, k3_of<T>(L), mu, K.d_ph, cpg, x,
                                                                             b, ld, kColours[q][0], kColours[q][1]);
      timer_end(KC_EDGE_SMOOTH, s);
      PBS_LAUNCHED();
    }
}

// A nodal cycle can continue from a given iterate when its top level runs the tiled steps
// (whose first kernel stages the iterate as it stages the right-hand side).
template <class T> bool takes_guess(const Hierarchy& H, int l, int nu_pre, int nu_post) {
  return l < H.nlev - 1 && !tail_from<T>(H, l, true) && fine_tiled(H.lev[l], nu_pre, nu_post);
}

template <class T>
void node_cycle(const Hierarchy& H, const KData& K, MgWork<T>& w, int l, const cx<T>* b, cx<T>* x, long ld, int ncols,
                int cpg, int nu_pre, int nu_post, cudaStream_t s, const cx<T>* x0 = nullptr) {
  const Level& L = H.lev[l];
  if (x0 && !takes_guess<T>(H, l, nu_pre, nu_post)) fail(-1, "nodal cycle: initial iterate on an untiled level");
  if (l == H.nlev - 1) {
    k_chol_solve<T><<<(ncols * 32 + 127) / 128, 128, 0, s>>>(node_factor<T>(K), (int)L.N(), b, ld, x, ld, ncols, cpg,
                                                             K.ngroups, K.goff);
    PBS_LAUNCHED();
    return;
  }
  if (tail_from<T>(H, l, true)) {
    size_t smem = 0;
    const TailArgs<T> ta = tail_args<T>(H, K, l, b, x, ld, cpg, nu_pre, nu_post, true, &smem);
    set_tail_smem<T>();
    timer_begin(KC_NODE_TAIL, s, tail_bytes<T>(H, l, ncols, cpg, true));
    k_node_tail<T><<<ncols, kTailThreads, smem, s>>>(ta);
    timer_end(KC_NODE_TAIL, s);
    PBS_LAUNCHED();
    return;
  }
  if (fine_tiled(L, nu_pre, nu_post)) {
    const Level& C = H.lev[l + 1];
    const auto down = [&](const FineShape& f) {
      if (f.rb) launch_rb<T>(true, f, L, C, K, w, l, b, x0, nullptr, ld, ncols, cpg, s);
      else if (f.ft == 64) launch_node_down<T, 64>(L, C, K, w, l, b, x0, ld, ncols, cpg, nu_pre, f.nt, s);
      else launch_node_down<T, 32>(L, C, K, w, l, b, x0, ld, ncols, cpg, nu_pre, f.nt, s);
    };
    const auto up = [&](const FineShape& f) {
      if (f.rb) launch_rb<T>(false, f, L, C, K, w, l, b, nullptr, x, ld, ncols, cpg, s);
      else if (f.ft == 64) launch_node_up<T, 64>(L, C, K, w, l, b, x, ld, ncols, cpg, nu_post, f.nt, s);
      else launch_node_up<T, 32>(L, C, K, w, l, b, x, ld, ncols, cpg, nu_post, f.nt, s);
    };
    FineShape fd[kNumFineShapes], fu[kNumFineShapes];
    const int nd = fine_shapes<T>(L, nu_pre, true, fd), nup = fine_shapes<T>(L, nu_post, false, fu);
    // both steps are idempotent (the down step reads b, the up step b, its saved
    // pre-smoothed x and the coarse correction, and neither writes what it reads)
    const std::string key = fine_key<T>(L, ncols, cpg);
    const int pd = tune_pick("node_down|" + key + "|nu" + std::to_string(nu_pre), nd, [&](int c) { down(fd[c]); }, s);
    timer_begin(KC_NODE_SMOOTH, s, fine_bytes<T>(L, ncols, nu_pre, true));
    down(fd[pd]);
    timer_end(KC_NODE_SMOOTH, s);
    node_cycle<T>(H, K, w, l + 1, w.b[l + 1], w.x[l + 1], C.N(), ncols, cpg, nu_pre, nu_post, s);
    const int pu = tune_pick("node_up|" + key + "|nu" + std::to_string(nu_post), nup, [&](int c) { up(fu[c]); }, s);
    timer_begin(KC_NODE_SMOOTH, s, fine_bytes<T>(L, ncols, nu_post, false));
    up(fu[pu]);
    timer_end(KC_NODE_SMOOTH, s);
    return;
  }
  zero_columns<T>(x, ld, L.N(), ncols, s);
  const Lvl<T> lv = L.lvl<T>();
  for (int it = 0; it < nu_pre; ++it)
    for (int q = 0; q < 4; ++q) {
      timer_begin(KC_NODE_SMOOTH, s, node_smooth_bytes<T>(L, ncols));
      k_node_smooth<T><<<half_grid(L.n, L.m, ncols), dim3(kBX, kBY), 0, s>>>(lv, K.d_ph, cpg, x, b, ld,
                                                                             kColours[q][0], kColours[q][1]);
      timer_end(KC_NODE_SMOOTH, s);
      PBS_LAUNCHED();
    }
  const Level& C = H.lev[l + 1];
  const long ldc = C.N();
  apply_nodal<T>(L, K.d_ph, cpg, x, w.r[l], b, ld, ncols, T(-1), T(1), s);
  restrict_node<T>(L, C, K.d_ph, cpg, w.r[l], ld, w.b[l + 1], ldc, ncols, s);
  node_cycle<T>(H, K, w, l + 1, w.b[l + 1], w.x[l + 1], ldc, ncols, cpg, nu_pre, nu_post, s);
  prolong_node<T>(L, C, K.d_ph, cpg, w.x[l + 1], ldc, x, ld, ncols, true, s);
  for (int it = 0; it < nu_post; ++it)
    for (int q = 3; q >= 0; --q) {
      timer_begin(KC_NODE_SMOOTH, s, node_smooth_bytes<T>(L, ncols));
      k_node_smooth<T><<<half_grid(L.n, L.m, ncols), dim3(kBX, kBY), 0, s>>>(lv, K.d_ph, cpg, x, b, ld,
                                                                             kColours[q][0], kColours[q][1]);
      timer_end(KC_NODE_SMOOTH, s);
      PBS_LAUNCHED();
    }
}

}  // namespace

template <class T>
void edge_vcycle(const Hierarchy& H, const KData& K, MgWork<T>& w, int l0, const cx<T>* X, cx<T>* Y, long ld,
                 int ncols, int cpg, int nu_pre, int nu_post, cudaStream_t s) {
  if (ncols <= 0) return;
  if (ncols > w.ncols) fail(-1, "multigrid workspace too small");
  edge_cycle<T>(H, K, w, l0, X, Y, ld, ncols, cpg, nu_pre, nu_post, s);
}

template <class T>
void nodal_vcycle(const Hierarchy& H, const KData& K, MgWork<T>& w, int l0, const cx<T>* X, cx<T>* Y, long ld,
                  int ncols, int cpg, int nu_pre, int nu_post, cudaStream_t s) {
  if (ncols <= 0) return;
  if (ncols > w.ncols) fail(-1, "multigrid workspace too small");
  node_cycle<T>(H, K, w, l0, X, Y, ld, ncols, cpg, nu_pre, nu_post, s);
}

template <class T> bool nodal_takes_guess(const Hierarchy& H, int l0, int nu_pre, int nu_post) {
  return takes_guess<T>(H, l0, nu_pre, nu_post);
}

template <class T>
void nodal_vcycle_from(const Hierarchy& H, const KData& K, MgWork<T>& w, int l0, const cx<T>* X, const cx<T>* X0,
                       cx<T>* Y, long ld, int ncols, int cpg, int nu_pre, int nu_post, cudaStream_t s) {
  if (ncols <= 0) return;
  if (ncols > w.ncols) fail(-1, "multigrid workspace too small");
  node_cycle<T>(H, K, w, l0, X, Y, ld, ncols, cpg, nu_pre, nu_post, s, X0);
}

#define PBS_INST_MG(T)                                                                                            \
  template bool nodal_takes_guess<T>(const Hierarchy&, int, int, int);                                            \
  template void nodal_vcycle_from<T>(const Hierarchy&, const KData&, MgWork<T>&, int, const cx<T>*, const cx<T>*, \
                                     cx<T>*, long, int, int, int, int, cudaStream_t);                             \
  template void alloc_mg_work<T>(DevMem&, const Hierarchy&, int, bool, MgWork<T>&);                               \
  template void free_mg_work<T>(DevMem&, MgWork<T>&);                                                             \
  template void edge_vcycle<T>(const Hierarchy&, const KData&, MgWork<T>&, int, const cx<T>*, cx<T>*, long, int, \
                               int, int, int, cudaStream_t);                                                      \
  template void nodal_vcycle<T>(const Hierarchy&, const KData&, MgWork<T>&, int, const cx<T>*, cx<T>*, long, int, \
                                int, int, int, cudaStream_t);
PBS_INST_MG(double)
PBS_INST_MG(float)

}  // namespace pbs
