// Matrix-free operators of the Bloch discretisation (Section 3) and the grid
// transfers of the bisection hierarchy (Section 5).  One thread per mesh
// index (i, j) and column; a column's Bloch phases come from its group
// (column / cpg) in the phase table.
#include "internal.h"
#include "mgpoint.cuh"

namespace pbs {

namespace {

constexpr int kBX = 32, kBY = 8;

inline dim3 grid2(int n, int m, int ncols) { return dim3((n + kBX - 1) / kBX, (m + kBY - 1) / kBY, ncols); }

template <class T>
__global__ void k_apply_edge(Lvl<T> L, Wts<T> w, const double* ph, int cpg, const cx<T>* __restrict__ X,
                             cx<T>* __restrict__ Y, const cx<T>* __restrict__ B, long ld, T sA, T sM, T sL,
                             const T* __restrict__ lam, T sB) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, c = blockIdx.z;
  if (i >= L.n || j >= L.m) return;
  const ERd<T> r{X + c * ld, L.n, L.m, load_ph<T>(ph, c / cpg)};
  const long N = (long)L.n * L.m, e = (long)j * L.n + i;
  const T s = sM + (lam ? sL * lam[c] : T(0));
  cx<T> yx, yy;
  if (inside(i, j, L.n, L.m, 1, 1))
    apply_edge_at<T>(L, inner<T>(w), inner_e<T>(X + c * ld, L.n, L.m), B ? B + c * ld : nullptr, sA, s, sB, i, j, yx,
                     yy);
  else
    apply_edge_at<T>(L, w, r, B ? B + c * ld : nullptr, sA, s, sB, i, j, yx, yy);
  Y[c * ld + e] = yx;
  Y[c * ld + N + e] = yy;
}

template <class T>
__global__ void k_curl(Lvl<T> L, const double* ph, int cpg, const cx<T>* __restrict__ X, long ldx,
                       cx<T>* __restrict__ Y, long ldy) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, c = blockIdx.z;
  if (i >= L.n || j >= L.m) return;
  const ERd<T> r{X + c * ldx, L.n, L.m, load_ph<T>(ph, c / cpg)};
  Y[c * ldy + (long)j * L.n + i] = curl_at<T>(r, i, j);
}

// C^* t: x-edge (i,j) = t(i,j-1) - t(i,j); y-edge (i,j) = t(i,j) - t(i-1,j)
template <class T>
__global__ void k_curl_adj(Lvl<T> L, const double* ph, int cpg, const cx<T>* __restrict__ X, long ldx,
                           cx<T>* __restrict__ Y, long ldy) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, c = blockIdx.z;
  if (i >= L.n || j >= L.m) return;
  const Ph<T> p = load_ph<T>(ph, c / cpg);
  const cx<T>* t = X + c * ldx;
  const long N = (long)L.n * L.m, e = (long)j * L.n + i;
  const cx<T> t0 = t[e];
  Y[c * ldy + e] = gread<T>(t, i, j - 1, L.n, L.m, p) - t0;
  Y[c * ldy + N + e] = t0 - gread<T>(t, i - 1, j, L.n, L.m, p);
}

// L phi: x-edge (i,j) = phi(i+1,j) - phi(i,j); y-edge (i,j) = phi(i,j+1) - phi(i,j)
template <class T>
__global__ void k_lift(Lvl<T> L, const double* ph, int cpg, const cx<T>* __restrict__ X, long ldx,
                       cx<T>* __restrict__ Y, long ldy) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, c = blockIdx.z;
  if (i >= L.n || j >= L.m) return;
  const Ph<T> p = load_ph<T>(ph, c / cpg);
  const cx<T>* f = X + c * ldx;
  const long N = (long)L.n * L.m, e = (long)j * L.n + i;
  const cx<T> f0 = f[e];
  Y[c * ldy + e] = gread<T>(f, i + 1, j, L.n, L.m, p) - f0;
  Y[c * ldy + N + e] = gread<T>(f, i, j + 1, L.n, L.m, p) - f0;
}

// L^* u at node (i,j) = u_x(i-1,j) - u_x(i,j) + u_y(i,j-1) - u_y(i,j)
template <class T>
__global__ void k_lift_adj(Lvl<T> L, const double* ph, int cpg, const cx<T>* __restrict__ X, long ldx,
                           cx<T>* __restrict__ Y, long ldy) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, c = blockIdx.z;
  if (i >= L.n || j >= L.m) return;
  const ERd<T> r{X + c * ldx, L.n, L.m, load_ph<T>(ph, c / cpg)};
  Y[c * ldy + (long)j * L.n + i] = r.x(i - 1, j) - r.x(i, j) + r.y(i, j - 1) - r.y(i, j);
}

template <class T>
__global__ void k_apply_nodal(Lvl<T> L, const double* ph, int cpg, const cx<T>* __restrict__ X,
                              cx<T>* __restrict__ Y, const cx<T>* __restrict__ B, long ld, T sP, T sB) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, c = blockIdx.z;
  if (i >= L.n || j >= L.m) return;
  const NRd<T> r{X + c * ld, L.n, L.m, load_ph<T>(ph, c / cpg)};
  Y[c * ld + (long)j * L.n + i] = inside(i, j, L.n, L.m, 1, 1)
                                      ? apply_nodal_at<T>(L, inner_n<T>(X + c * ld, L.n), B ? B + c * ld : nullptr,
                                                          sP, sB, i, j)
                                      : apply_nodal_at<T>(L, r, B ? B + c * ld : nullptr, sP, sB, i, j);
}

// Natural embedding of coarse edges (Section 5): a fine edge lying on a coarse
// edge takes 1/2 of it; a fine edge on the midline of a coarse cell takes 1/4
// of each of the two parallel coarse edges bounding that cell.
template <class T>
__global__ void k_prolong_edge(int nf, int mf, int nc, int mc, const double* ph, int cpg,
                               const cx<T>* __restrict__ Xc, long ldc, cx<T>* __restrict__ Yf, long ldf,
                               int accumulate) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, c = blockIdx.z;
  if (i >= nf || j >= mf) return;
  const ERd<T> rc{Xc + c * ldc, nc, mc, load_ph<T>(ph, c / cpg)};
  const long Nf = (long)nf * mf, e = (long)j * nf + i;
  cx<T> vx, vy;
  if (inside(i >> 1, j >> 1, nc, mc, 0, 1))
    prolong_edge_at<T>(inner_e<T>(Xc + c * ldc, nc, mc), i, j, vx, vy);
  else
    prolong_edge_at<T>(rc, i, j, vx, vy);
  cx<T>* yf = Yf + c * ldf;
  if (accumulate) {
    yf[e] = yf[e] + vx;
    yf[Nf + e] = yf[Nf + e] + vy;
  } else {
    yf[e] = vx;
    yf[Nf + e] = vy;
  }
}

// Adjoint of the embedding (conjugate phases through the ghost reads).
template <class T>
__global__ void k_restrict_edge(int nf, int mf, int nc, int mc, const double* ph, int cpg,
                                const cx<T>* __restrict__ Xf, long ldf, cx<T>* __restrict__ Yc, long ldc) {
  const int I = blockIdx.x * kBX + threadIdx.x, J = blockIdx.y * kBY + threadIdx.y, c = blockIdx.z;
  if (I >= nc || J >= mc) return;
  const ERd<T> r{Xf + c * ldf, nf, mf, load_ph<T>(ph, c / cpg)};
  cx<T> vx, vy;
  if (inside(2 * I, 2 * J, nf, mf, 1, 1))
    restrict_edge_at<T>(inner_e<T>(Xf + c * ldf, nf, mf), I, J, vx, vy);
  else
    restrict_edge_at<T>(r, I, J, vx, vy);
  const long Nc = (long)nc * mc, e = (long)J * nc + I;
  Yc[c * ldc + e] = vx;
  Yc[c * ldc + Nc + e] = vy;
}

// Bilinear embedding of coarse nodal functions.
template <class T>
__global__ void k_prolong_node(int nf, int mf, int nc, int mc, const double* ph, int cpg,
                               const cx<T>* __restrict__ Xc, long ldc, cx<T>* __restrict__ Yf, long ldf,
                               int accumulate) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, c = blockIdx.z;
  if (i >= nf || j >= mf) return;
  const NRd<T> rc{Xc + c * ldc, nc, mc, load_ph<T>(ph, c / cpg)};
  const cx<T> v = prolong_node_at<T>(rc, i, j);
  const long e = (long)j * nf + i;
  cx<T>* yf = Yf + c * ldf;
  yf[e] = accumulate ? yf[e] + v : v;
}

template <class T>
__global__ void k_restrict_node(int nf, int mf, int nc, int mc, const double* ph, int cpg,
                                const cx<T>* __restrict__ Xf, long ldf, cx<T>* __restrict__ Yc, long ldc) {
  const int I = blockIdx.x * kBX + threadIdx.x, J = blockIdx.y * kBY + threadIdx.y, c = blockIdx.z;
  if (I >= nc || J >= mc) return;
  const NRd<T> rf{Xf + c * ldf, nf, mf, load_ph<T>(ph, c / cpg)};
  Yc[c * ldc + (long)J * nc + I] = restrict_node_at<T>(rf, I, J);
}

}  // namespace

template <class T>
void apply_edge(const Level& L, const double* d_ph, int cpg, const cx<T>* X, cx<T>* Y, const cx<T>* B, long ld,
                int ncols, T sA, T sM, T sL, const T* lam, T sB, cudaStream_t s) {
  if (ncols <= 0) return;
  k_apply_edge<T><<<grid2(L.n, L.m, ncols), dim3(kBX, kBY), 0, s>>>(L.lvl<T>(), L.wts<T>(), d_ph, cpg, X, Y, B, ld,
                                                                      sA, sM, sL, lam, sB);
  PBS_LAUNCHED();
}

template <class T>
void apply_curl(const Level& L, const double* d_ph, int cpg, const cx<T>* X, long ldx, cx<T>* Y, long ldy, int ncols,
                cudaStream_t s) {
  if (ncols <= 0) return;
  k_curl<T><<<grid2(L.n, L.m, ncols), dim3(kBX, kBY), 0, s>>>(L.lvl<T>(), d_ph, cpg, X, ldx, Y, ldy);
  PBS_LAUNCHED();
}

template <class T>
void apply_curl_adj(const Level& L, const double* d_ph, int cpg, const cx<T>* X, long ldx, cx<T>* Y, long ldy,
                    int ncols, cudaStream_t s) {
  if (ncols <= 0) return;
  k_curl_adj<T><<<grid2(L.n, L.m, ncols), dim3(kBX, kBY), 0, s>>>(L.lvl<T>(), d_ph, cpg, X, ldx, Y, ldy);
  PBS_LAUNCHED();
}

template <class T>
void apply_lift(const Level& L, const double* d_ph, int cpg, const cx<T>* X, long ldx, cx<T>* Y, long ldy, int ncols,
                cudaStream_t s) {
  if (ncols <= 0) return;
  k_lift<T><<<grid2(L.n, L.m, ncols), dim3(kBX, kBY), 0, s>>>(L.lvl<T>(), d_ph, cpg, X, ldx, Y, ldy);
  PBS_LAUNCHED();
}

template <class T>
void apply_lift_adj(const Level& L, const double* d_ph, int cpg, const cx<T>* X, long ldx, cx<T>* Y, long ldy,
                    int ncols, cudaStream_t s) {
  if (ncols <= 0) return;
  k_lift_adj<T><<<grid2(L.n, L.m, ncols), dim3(kBX, kBY), 0, s>>>(L.lvl<T>(), d_ph, cpg, X, ldx, Y, ldy);
  PBS_LAUNCHED();
}

template <class T>
void apply_nodal(const Level& L, const double* d_ph, int cpg, const cx<T>* X, cx<T>* Y, const cx<T>* B, long ld,
                 int ncols, T sP, T sB, cudaStream_t s) {
  if (ncols <= 0) return;
  timer_begin(KC_NODE_APPLY, s, (B ? 3.0 : 2.0) * sizeof(cx<T>) * L.N() * ncols);  // read x (and b), write y
  k_apply_nodal<T><<<grid2(L.n, L.m, ncols), dim3(kBX, kBY), 0, s>>>(L.lvl<T>(), d_ph, cpg, X, Y, B, ld, sP, sB);
  timer_end(KC_NODE_APPLY, s);
  PBS_LAUNCHED();
}

template <class T>
void prolong_edge(const Level& f, const Level& c, const double* d_ph, int cpg, const cx<T>* Xc, long ldc, cx<T>* Yf,
                  long ldf, int ncols, bool accumulate, cudaStream_t s) {
  if (ncols <= 0) return;
  k_prolong_edge<T><<<grid2(f.n, f.m, ncols), dim3(kBX, kBY), 0, s>>>(f.n, f.m, c.n, c.m, d_ph, cpg, Xc, ldc, Yf, ldf,
                                                                        accumulate ? 1 : 0);
  PBS_LAUNCHED();
}

template <class T>
void restrict_edge(const Level& f, const Level& c, const double* d_ph, int cpg, const cx<T>* Xf, long ldf, cx<T>* Yc,
                   long ldc, int ncols, cudaStream_t s) {
  if (ncols <= 0) return;
  k_restrict_edge<T><<<grid2(c.n, c.m, ncols), dim3(kBX, kBY), 0, s>>>(f.n, f.m, c.n, c.m, d_ph, cpg, Xf, ldf, Yc,
                                                                         ldc);
  PBS_LAUNCHED();
}

template <class T>
void prolong_node(const Level& f, const Level& c, const double* d_ph, int cpg, const cx<T>* Xc, long ldc, cx<T>* Yf,
                  long ldf, int ncols, bool accumulate, cudaStream_t s) {
  if (ncols <= 0) return;
  k_prolong_node<T><<<grid2(f.n, f.m, ncols), dim3(kBX, kBY), 0, s>>>(f.n, f.m, c.n, c.m, d_ph, cpg, Xc, ldc, Yf, ldf,
                                                                        accumulate ? 1 : 0);
  PBS_LAUNCHED();
}

template <class T>
void restrict_node(const Level& f, const Level& c, const double* d_ph, int cpg, const cx<T>* Xf, long ldf, cx<T>* Yc,
                   long ldc, int ncols, cudaStream_t s) {
  if (ncols <= 0) return;
  k_restrict_node<T><<<grid2(c.n, c.m, ncols), dim3(kBX, kBY), 0, s>>>(f.n, f.m, c.n, c.m, d_ph, cpg, Xf, ldf, Yc,
                                                                         ldc);
  PBS_LAUNCHED();
}

#define PBS_INST_OPS(T)                                                                                             \
  template void apply_edge<T>(const Level&, const double*, int, const cx<T>*, cx<T>*, const cx<T>*, long, int, T, T, \
                              T, const T*, T, cudaStream_t);                                                          \
  template void apply_curl<T>(const Level&, const double*, int, const cx<T>*, long, cx<T>*, long, int, cudaStream_t); \
  template void apply_curl_adj<T>(const Level&, const double*, int, const cx<T>*, long, cx<T>*, long, int,           \
                                  cudaStream_t);                                                                      \
  template void apply_lift<T>(const Level&, const double*, int, const cx<T>*, long, cx<T>*, long, int, cudaStream_t); \
  template void apply_lift_adj<T>(const Level&, const double*, int, const cx<T>*, long, cx<T>*, long, int,           \
                                  cudaStream_t);                                                                      \
  template void apply_nodal<T>(const Level&, const double*, int, const cx<T>*, cx<T>*, const cx<T>*, long, int, T, T, \
                               cudaStream_t);                                                                         \
  template void prolong_edge<T>(const Level&, const Level&, const double*, int, const cx<T>*, long, cx<T>*, long,    \
                                int, bool, cudaStream_t);                                                             \
  template void restrict_edge<T>(const Level&, const Level&, const double*, int, const cx<T>*, long, cx<T>*, long,   \
                                 int, cudaStream_t);                                                                  \
  template void prolong_node<T>(const Level&, const Level&, const double*, int, const cx<T>*, long, cx<T>*, long,    \
                                int, bool, cudaStream_t);                                                             \
  template void restrict_node<T>(const Level&, const Level&, const double*, int, const cx<T>*, long, cx<T>*, long,   \
                                 int, cudaStream_t);
PBS_INST_OPS(double)
PBS_INST_OPS(float)

}  // namespace pbs
