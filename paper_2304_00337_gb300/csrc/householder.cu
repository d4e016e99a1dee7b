// Generalised (M-)Householder orthonormalisation of a block (Section 4): the
// reflections Q_i = I - 2 v_i v_i^* M / (v_i^* M v_i) with Q_q ... Q_1 S = P R,
// P the prescribed M-orthonormal basis of scaled unit x-edge vectors, and
// E = Q_1 ... Q_q P.  FP64 throughout, one Bloch vector, columns of D edges.
//
// Step i of the factorisation (no host synchronisation inside):
//   k_hh_perp    y := column i; twice y -= P_k (P_k^* M y), k < i, adding the
//                coefficients to R[k, i] (P_k^* M y is one mass-stencil value);
//   k_hh_mnorm   partial sums of y^* M y;
//   k_hh_sigma   ||y||_M, gamma = P_i^* M y, sigma = -||y||_M gamma/|gamma|,
//                R[i, i] = sigma, v_i = y - sigma P_i (in place of column i),
//                v_i^* M v_i = 2 ||y||_M^2 + 2 ||y||_M |gamma|;
//   k_hh_mdots   partial sums of v_i^* M y_j for the later columns j;
//   k_hh_update  their fixed-order totals, c_j = 2 v_i^* M y_j / v_i^* M v_i,
//                and y_j -= c_j v_i.
// E starts as P and takes the reflections q .. 1 (the last two kernels on
// columns i .. q-1: Q_i keeps P_k for k < i).  A step whose y is exactly zero
// (rank loss) keeps Q_i = I and R[i, i] = 0.
#include <algorithm>

#include "internal.h"
#include "mgpoint.cuh"

namespace pbs {

namespace {

constexpr int kHT = 256;             // threads per block of the streaming kernels
constexpr int kHBlocks = 2 * 152;    // blocks of the reductions (fixed: fixed summation order)
constexpr int kHCols = 8;            // later columns per block row of the dot kernel

// x-edge of prescribed vector k: (k mod n, 2 (k div n)), index j n + i
__device__ __forceinline__ long pivot_edge(int k, int n) { return (long)(2 * (k / n)) * n + k % n; }

// (M y) at x-edge (i, j); a plain reader, since the callers write y between reads
__device__ __forceinline__ double2 mass_x_at(const double2* y, const Lvl<double>& L, const Ph<double>& p, int i,
                                             int j) {
  const ERdPlain<double> r{y, L.n, L.m, p};
  return M_x<double>(r, L, i, j);
}

// (M y) at edge e (x-edges first)
__device__ __forceinline__ double2 mass_at(const ERd<double>& r, const Lvl<double>& L, long e, long N) {
  if (e < N) return M_x<double>(r, L, int(e % L.n), int(e / L.n));
  const long f = e - N;
  return M_y<double>(r, L, int(f % L.n), int(f / L.n));
}

__device__ __forceinline__ double2 cconj_mul(double2 a, double2 b) {  // conj(a) b
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
// acc + conj(a) b as four fused multiply-adds (the FP64 pipe is the bound)
__device__ __forceinline__ double2 cconj_fma(double2 a, double2 b, double2 acc) {
  return make_double2(fma(a.x, b.x, fma(a.y, b.y, acc.x)), fma(a.x, b.y, fma(-a.y, b.x, acc.y)));
}
// x - c v as four fused multiply-adds
__device__ __forceinline__ double2 cfms(double2 x, double2 c, double2 v) {
  return make_double2(fma(-c.x, v.x, fma(c.y, v.y, x.x)), fma(-c.x, v.y, fma(-c.y, v.x, x.y)));
}

// Fixed-order block sum of a complex value; result valid in thread 0.
__device__ __forceinline__ double2 block_sum_c(double2 v) {
  __shared__ double2 red[kHT / 32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double2 s = make_double2(0, 0);
  if (threadIdx.x == 0)
    for (int k = 0; k < kHT / 32; ++k) s = s + red[k];
  return s;
}

// Two passes of y -= P_k (P_k^* M y), k < i; thread k owns pivot k.  Pivots share
// no mass-matrix entry, so a thread's stencil never reads another pivot's edge.
__global__ void k_hh_perp(Lvl<double> L, const double* ph, double2* Y, long ld, int i, double2* R, int q) {
  const Ph<double> p = load_ph<double>(ph, 0);
  const double s = sqrt(2.0 / 3.0 * L.mx);  // P_k = e_{j_k} / s
  double2* y = Y + (long)i * ld;
  const int k = threadIdx.x;
  for (int pass = 0; pass < 2; ++pass) {
    if (k < i) {
      const long e = pivot_edge(k, L.n);
      const double2 my = mass_x_at(y, L, p, int(e % L.n), int(e / L.n));
      const double2 c = make_double2(my.x / s, my.y / s);
      R[(long)i * q + k] = R[(long)i * q + k] + c;
      y[e] = y[e] - make_double2(c.x / s, c.y / s);
    }
    __syncthreads();
  }
}

// partial sums of y^* M y, y = column i
__global__ void __launch_bounds__(kHT) k_hh_mnorm(Lvl<double> L, const double* ph, const double2* Y, long ld, int i,
                                                  double2* part) {
  const Ph<double> p = load_ph<double>(ph, 0);
  const double2* y = Y + (long)i * ld;
  const ERd<double> r{y, L.n, L.m, p};
  const long N = (long)L.n * L.m, D = 2 * N;
  double2 acc = make_double2(0, 0);
  for (long e = blockIdx.x * (long)kHT + threadIdx.x; e < D; e += (long)gridDim.x * kHT)
    acc = acc + cconj_mul(y[e], mass_at(r, L, e, N));
  const double2 t = block_sum_c(acc);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

// sigma, R[i, i], v_i (in place of column i) and v_i^* M v_i (0: Q_i = I)
__global__ void k_hh_sigma(Lvl<double> L, const double* ph, double2* Y, long ld, int i, const double2* part,
                           int nparts, double2* R, int q, double* vmv) {
  if (threadIdx.x != 0) return;
  const Ph<double> p = load_ph<double>(ph, 0);
  const double s = sqrt(2.0 / 3.0 * L.mx);
  double nn = 0.0;
  for (int b = 0; b < nparts; ++b) nn += part[b].x;
  const double nrm = sqrt(fmax(nn, 0.0));
  double2* y = Y + (long)i * ld;
  const long e = pivot_edge(i, L.n);
  const double2 my = mass_x_at(y, L, p, int(e % L.n), int(e / L.n));
  const double2 gamma = make_double2(my.x / s, my.y / s);
  const double ag = hypot(gamma.x, gamma.y);
  const double2 u = ag > 0.0 ? make_double2(gamma.x / ag, gamma.y / ag) : make_double2(1.0, 0.0);
  const double2 sigma = make_double2(-nrm * u.x, -nrm * u.y);
  const double w = 2.0 * nrm * nrm + 2.0 * nrm * ag;
  if (!(nrm > 0.0) || !(w > 0.0) || !isfinite(w)) {
    R[(long)i * q + i] = make_double2(0, 0);
    vmv[i] = 0.0;
    return;
  }
  R[(long)i * q + i] = sigma;
  y[e] = y[e] - make_double2(sigma.x / s, sigma.y / s);
  vmv[i] = w;
}

// partial sums of v^* M x_j = (M v)^* x_j for columns j0 + blockIdx.y kHCols + t
__global__ void __launch_bounds__(kHT) k_hh_mdots(Lvl<double> L, const double* ph, const double2* V,
                                                  const double2* X, long ld, int j0, int j1, const double* vmv,
                                                  int i, double2* part) {
  if (vmv[i] == 0.0) return;
  __shared__ double2 red[kHT / 32][kHCols];
  const Ph<double> p = load_ph<double>(ph, 0);
  const ERd<double> r{V, L.n, L.m, p};
  const long N = (long)L.n * L.m, D = 2 * N;
  const int jb = j0 + blockIdx.y * kHCols, nj = min(kHCols, j1 - jb);
  double2 acc[kHCols];
#pragma unroll
  for (int t = 0; t < kHCols; ++t) acc[t] = make_double2(0, 0);
  for (long e = blockIdx.x * (long)kHT + threadIdx.x; e < D; e += (long)gridDim.x * kHT) {
    const double2 mv = mass_at(r, L, e, N);
#pragma unroll
    for (int t = 0; t < kHCols; ++t)
      if (t < nj) acc[t] = cconj_fma(mv, X[(long)(jb + t) * ld + e], acc[t]);
  }
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int t = 0; t < kHCols; ++t) {
    for (int o = 16; o > 0; o >>= 1) {
      acc[t].x += __shfl_xor_sync(0xffffffffu, acc[t].x, o);
      acc[t].y += __shfl_xor_sync(0xffffffffu, acc[t].y, o);
    }
    if (lane == 0) red[w][t] = acc[t];
  }
  __syncthreads();
  if (threadIdx.x < nj) {
    double2 sum = make_double2(0, 0);
    for (int k = 0; k < kHT / 32; ++k) sum = sum + red[k][threadIdx.x];
    part[(long)(jb - j0 + threadIdx.x) * gridDim.x + blockIdx.x] = sum;
  }
}

// x_j -= c_j v for column j = j0 + blockIdx.y, c_j = 2 (v^* M x_j) / (v^* M v) from the
// nparts partial sums (fixed order, the same in every block of the column)
__global__ void __launch_bounds__(kHT) k_hh_update(const double2* V, double2* X, long ld, long D, int j0,
                                                   const double2* part, int nparts, const double* vmv, int i) {
  if (vmv[i] == 0.0) return;
  __shared__ double2 red[kHT / 32];
  __shared__ double2 coef;
  const int j = j0 + blockIdx.y;
  double2 s = make_double2(0, 0);
  for (int b = threadIdx.x; b < nparts; b += kHT) s = s + part[(long)blockIdx.y * nparts + b];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    s.x += __shfl_xor_sync(0xffffffffu, s.x, o);
    s.y += __shfl_xor_sync(0xffffffffu, s.y, o);
  }
  if (lane == 0) red[w] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double2 t = make_double2(0, 0);
    for (int k = 0; k < kHT / 32; ++k) t = t + red[k];
    const double f = 2.0 / vmv[i];
    coef = make_double2(f * t.x, f * t.y);
  }
  __syncthreads();
  const double2 c = coef;
  double2* x = X + (long)j * ld;
  for (long e = blockIdx.x * (long)kHT + threadIdx.x; e < D; e += (long)gridDim.x * kHT) {
    x[e] = cfms(x[e], c, V[e]);
  }
}

// E = P: zero columns with 1/s at the pivots
__global__ void k_hh_basis(Lvl<double> L, double2* E, long ld, int q) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k < q) E[(long)k * ld + pivot_edge(k, L.n)] = make_double2(1.0 / sqrt(2.0 / 3.0 * L.mx), 0.0);
}

// apply Q_i (vector in column i of V) to columns j0 .. j1-1 of X; about two blocks
// per SM in each launch
void reflect_columns(const Level& L0, const double* d_ph, const double2* V, double2* X, long ld, int j0, int j1,
                     const double* vmv, int i, double2* part, cudaStream_t s) {
  if (j1 <= j0) return;
  const int nc = j1 - j0, nchunk = (nc + kHCols - 1) / kHCols;
  const int nparts = std::max(1, kHBlocks / nchunk), ub = std::max(1, 2 * kHBlocks / nc);
  const Lvl<double> lv = L0.lvl<double>();
  timer_begin(KC_HOUSEHOLDER, s, 16.0 * L0.D() * (nc + 1));
  k_hh_mdots<<<dim3(nparts, nchunk), kHT, 0, s>>>(lv, d_ph, V, X, ld, j0, j1, vmv, i, part);
  timer_end(KC_HOUSEHOLDER, s);
  PBS_LAUNCHED();
  timer_begin(KC_HOUSEHOLDER, s, 16.0 * L0.D() * (2 * nc + 1));
  k_hh_update<<<dim3(ub, nc), kHT, 0, s>>>(V, X, ld, L0.D(), j0, part, nparts, vmv, i);
  timer_end(KC_HOUSEHOLDER, s);
  PBS_LAUNCHED();
}

}  // namespace

int householder_max_columns(int n, int m) { return n * (m / 2); }

size_t householder_work_bytes(long D, int q) {
  return sizeof(double2) * ((size_t)D * q + (size_t)kHBlocks * (q + 1)) + sizeof(double) * q;
}

void m_householder(const Level& L0, const double* d_ph, const double2* S, double2* E, double2* R, int q, void* work,
                   cudaStream_t s) {
  if (q <= 0) return;
  if (q > householder_max_columns(L0.n, L0.m)) fail(PBS_EINVAL, "m_householder: more columns than prescribed vectors");
  const long D = L0.D();
  double2* Y = (double2*)work;
  double2* part = Y + D * q;
  double* vmv = (double*)(part + (long)kHBlocks * (q + 1));
  const Lvl<double> lv = L0.lvl<double>();
  PBS_CUDA(cudaMemcpyAsync(Y, S, sizeof(double2) * D * q, cudaMemcpyDeviceToDevice, s));
  PBS_CUDA(cudaMemsetAsync(R, 0, sizeof(double2) * q * q, s));
  for (int i = 0; i < q; ++i) {
    if (i > 0) {
      k_hh_perp<<<1, ((i + 31) / 32) * 32, 0, s>>>(lv, d_ph, Y, D, i, R, q);
      PBS_LAUNCHED();
    }
    k_hh_mnorm<<<kHBlocks, kHT, 0, s>>>(lv, d_ph, Y, D, i, part);
    PBS_LAUNCHED();
    k_hh_sigma<<<1, 32, 0, s>>>(lv, d_ph, Y, D, i, part, kHBlocks, R, q, vmv);
    PBS_LAUNCHED();
    reflect_columns(L0, d_ph, Y + (long)i * D, Y, D, i + 1, q, vmv, i, part, s);
  }
  PBS_CUDA(cudaMemsetAsync(E, 0, sizeof(double2) * D * q, s));
  k_hh_basis<<<(q + 127) / 128, 128, 0, s>>>(lv, E, D, q);
  PBS_LAUNCHED();
  for (int i = q - 1; i >= 0; --i) reflect_columns(L0, d_ph, Y + (long)i * D, E, D, i, q, vmv, i, part, s);
}

}  // namespace pbs
