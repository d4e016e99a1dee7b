// Per-point bodies of the multigrid steps (Section 5): point and patch
// Gauss-Seidel updates, level residuals, grid transfers and the coarsest
// triangular solves.  The one-launch-per-step kernels (ops.cu, mg.cu) and the
// fused coarse-level V-cycle kernels (mg.cu) call the same functions, so both
// schedules perform the same arithmetic on every point.
//
// Readers come in two kinds: the __restrict__ ones of common.cuh for kernels
// that never write what they read, and the plain ones below for fused kernels
// that rewrite their buffers between block-wide barriers (a read-only cache path
// would not see those writes).
#pragma once
#include "common.cuh"

namespace pbs {

template <class T>
__device__ __forceinline__ cx<T> gread_plain(const cx<T>* f, int i, int j, int n, int m, const Ph<T>& p) {
  bool w = false;
  cx<T> ph = mk<T>(T(1), T(0));
  if (i < 0) {
    i += n;
    ph = conj(p.al);
    w = true;
  } else if (i >= n) {
    i -= n;
    ph = p.al;
    w = true;
  }
  if (j < 0) {
    j += m;
    ph = cmul(ph, conj(p.be));
    w = true;
  } else if (j >= m) {
    j -= m;
    ph = cmul(ph, p.be);
    w = true;
  }
  cx<T> v = f[(long)j * n + i];
  return w ? cmul(v, ph) : v;
}

template <class T> struct NRdPlain {
  const cx<T>* X;
  int n, m;
  Ph<T> p;
  __device__ __forceinline__ cx<T> v(int i, int j) const { return gread_plain<T>(X, i, j, n, m, p); }
};
template <class T> struct ERdPlain {
  const cx<T>* X;
  int n, m;
  Ph<T> p;
  __device__ __forceinline__ cx<T> x(int i, int j) const { return gread_plain<T>(X, i, j, n, m, p); }
  __device__ __forceinline__ cx<T> y(int i, int j) const { return gread_plain<T>(X + (long)n * m, i, j, n, m, p); }
};

// Readers without the Bloch extension, for stencils that stay inside the level:
// there the extended readers return the stored value unchanged, so a point
// computed through these gives the same result without the wrap tests.
template <class T> struct NRdIn {
  const cx<T>* X;
  int n;
  __device__ __forceinline__ cx<T> v(int i, int j) const { return X[(long)j * n + i]; }
};
template <class T> struct ERdIn {
  const cx<T>* X;
  int n;
  long N;
  __device__ __forceinline__ cx<T> x(int i, int j) const { return X[(long)j * n + i]; }
  __device__ __forceinline__ cx<T> y(int i, int j) const { return X[N + (long)j * n + i]; }
};
template <class T> struct WtsIn {
  const T* winv;
  int n;
  T scale;
  __device__ __forceinline__ T operator()(int i, int j) const { return scale * winv[(long)j * n + i]; }
};
template <class T> __device__ __forceinline__ WtsIn<T> inner(const Wts<T>& w) { return WtsIn<T>{w.winv, w.n, w.scale}; }
template <class T> __device__ __forceinline__ NRdIn<T> inner_n(const cx<T>* X, int n) { return NRdIn<T>{X, n}; }
template <class T> __device__ __forceinline__ ERdIn<T> inner_e(const cx<T>* X, int n, int m) {
  return ERdIn<T>{X, n, (long)n * m};
}
// the neighbourhood [i - lo, i + hi] x [j - lo, j + hi] lies inside an n x m level
__device__ __forceinline__ bool inside(int i, int j, int n, int m, int lo, int hi) {
  return i >= lo && j >= lo && i + hi < n && j + hi < m;
}

// ---- nodal (P = L^* M L) ----------------------------------------------------

// point Gauss-Seidel update of node (i,j); r reads x
template <class T, class R>
__device__ __forceinline__ void node_smooth_at(const Lvl<T>& L, const R& r, cx<T>* x, const cx<T>* b, int i, int j) {
  const long e = (long)j * L.n + i;
  const cx<T> res = b[e] - P_at<T>(r, L, i, j);
  x[e] = x[e] + (T(1) / P_diag<T>(L)) * res;
}

// sP (P x)(i,j) + sB b(i,j)
template <class T, class R>
__device__ __forceinline__ cx<T> apply_nodal_at(const Lvl<T>& L, const R& r, const cx<T>* b, T sP, T sB, int i,
                                                int j) {
  cx<T> y = sP * P_at<T>(r, L, i, j);
  if (b) y = y + sB * b[(long)j * L.n + i];
  return y;
}

// bilinear embedding: fine node (i,j) from coarse reader rc (nc x mc)
template <class T, class R> __device__ __forceinline__ cx<T> prolong_node_at(const R& rc, int i, int j) {
  const int I = i >> 1, J = j >> 1;
  if (!(i & 1) && !(j & 1)) return rc.v(I, J);
  if ((i & 1) && !(j & 1)) return T(0.5) * (rc.v(I, J) + rc.v(I + 1, J));
  if (!(i & 1) && (j & 1)) return T(0.5) * (rc.v(I, J) + rc.v(I, J + 1));
  return T(0.25) * (rc.v(I, J) + rc.v(I + 1, J) + rc.v(I, J + 1) + rc.v(I + 1, J + 1));
}

// adjoint of the bilinear embedding: coarse node (I,J) from fine reader rf
template <class T, class R> __device__ __forceinline__ cx<T> restrict_node_at(const R& rf, int I, int J) {
  cx<T> acc = czero<T>();
#pragma unroll
  for (int dj = -1; dj <= 1; ++dj) {
#pragma unroll
    for (int di = -1; di <= 1; ++di) {
      const T wgt = (di == 0 ? T(1) : T(0.5)) * (dj == 0 ? T(1) : T(0.5));
      acc = acc + wgt * rf.v(2 * I + di, 2 * J + dj);
    }
  }
  return acc;
}

// ---- edges (A + mu M) -------------------------------------------------------

// (sA A + s M) x + sB b at x-edge and y-edge (i,j)
template <class T, class R, class W>
__device__ __forceinline__ void apply_edge_at(const Lvl<T>& L, const W& w, const R& r, const cx<T>* B, T sA, T s,
                                              T sB, int i, int j, cx<T>& yx, cx<T>& yy) {
  const long N = (long)L.n * L.m, e = (long)j * L.n + i;
  yx = czero<T>();
  yy = czero<T>();
  if (sA != T(0)) {
    yx = sA * A_x<T>(r, w, i, j);
    yy = sA * A_y<T>(r, w, i, j);
  }
  if (s != T(0)) {
    yx = yx + s * M_x<T>(r, L, i, j);
    yy = yy + s * M_y<T>(r, L, i, j);
  }
  if (B) {
    yx = yx + sB * B[e];
    yy = yy + sB * B[N + e];
  }
}

// Block Gauss-Seidel update of the patch of node (i,j) (its edges L, R, B, T);
// r reads x, rb reads b; K3^{-1} of the node in k3 (SoA [6][N]).
template <class T, class R, class RB, class W>
__device__ __forceinline__ void edge_smooth_at(const Lvl<T>& L, const W& w, const T* k3, T mu, const Ph<T>& p,
                                               const R& r, const RB& rb, cx<T>* X, int i, int j) {
  // residual b - (A + mu M) x on the patch, in ghost coordinates
  const cx<T> rL = rb.x(i - 1, j) - (A_x<T>(r, w, i - 1, j) + mu * M_x<T>(r, L, i - 1, j));
  const cx<T> rR = rb.x(i, j) - (A_x<T>(r, w, i, j) + mu * M_x<T>(r, L, i, j));
  const cx<T> rB = rb.y(i, j - 1) - (A_y<T>(r, w, i, j - 1) + mu * M_y<T>(r, L, i, j - 1));
  const cx<T> rT = rb.y(i, j) - (A_y<T>(r, w, i, j) + mu * M_y<T>(r, L, i, j));
  const T m1 = T(2.0 / 3.0) * L.mx, m2 = T(2.0 / 3.0) * L.my;
  const cx<T> s0 = (T(1) / (mu * T(2) * (m1 + m2))) * (rL - rR + rB - rT);
  const cx<T> ya = rL + rR, yb = rB + rT, yc = m2 * (rL - rR) + m1 * (rT - rB);
  const long N = (long)L.n * L.m, e = (long)j * L.n + i;
  const T K00 = k3[e], K01 = k3[N + e], K02 = k3[2 * N + e], K11 = k3[3 * N + e], K12 = k3[4 * N + e],
          K22 = k3[5 * N + e];
  const cx<T> za = K00 * ya + K01 * yb + K02 * yc;
  const cx<T> zb = K01 * ya + K11 * yb + K12 * yc;
  const cx<T> zc = K02 * ya + K12 * yb + K22 * yc;
  const cx<T> dL = s0 + za + m2 * zc, dR = za - m2 * zc - s0;
  const cx<T> dB = s0 + zb - m1 * zc, dT = zb + m1 * zc - s0;
  cx<T>* Xx = X;
  cx<T>* Xy = X + N;
  Xx[e] = Xx[e] + dR;
  Xy[e] = Xy[e] + dT;
  // a ghost-coordinate change d of an edge read as conj(alpha) x is alpha d in storage
  if (i > 0) Xx[e - 1] = Xx[e - 1] + dL;
  else Xx[(long)j * L.n + L.n - 1] = Xx[(long)j * L.n + L.n - 1] + cmul(p.al, dL);
  if (j > 0) Xy[e - L.n] = Xy[e - L.n] + dB;
  else Xy[(long)(L.m - 1) * L.n + i] = Xy[(long)(L.m - 1) * L.n + i] + cmul(p.be, dB);
}

// Natural embedding (Section 5) at fine edge index (i,j): a fine edge on a coarse
// edge takes 1/2 of it, one on a coarse cell's midline 1/4 of each of the two
// parallel coarse edges bounding that cell.  rc reads the coarse vector.
template <class T, class R>
__device__ __forceinline__ void prolong_edge_at(const R& rc, int i, int j, cx<T>& vx, cx<T>& vy) {
  {
    const int I = i >> 1;
    if ((j & 1) == 0) vx = T(0.5) * rc.x(I, j >> 1);
    else vx = T(0.25) * (rc.x(I, j >> 1) + rc.x(I, (j >> 1) + 1));
  }
  {
    const int J = j >> 1;
    if ((i & 1) == 0) vy = T(0.5) * rc.y(i >> 1, J);
    else vy = T(0.25) * (rc.y(i >> 1, J) + rc.y((i >> 1) + 1, J));
  }
}

// adjoint of the embedding at coarse index (I,J); rf reads the fine vector
template <class T, class R>
__device__ __forceinline__ void restrict_edge_at(const R& rf, int I, int J, cx<T>& vx, cx<T>& vy) {
  const int i = 2 * I, j = 2 * J;
  vx = T(0.5) * (rf.x(i, j) + rf.x(i + 1, j)) +
       T(0.25) * (rf.x(i, j + 1) + rf.x(i + 1, j + 1) + rf.x(i, j - 1) + rf.x(i + 1, j - 1));
  vy = T(0.5) * (rf.y(i, j) + rf.y(i, j + 1)) +
       T(0.25) * (rf.y(i + 1, j) + rf.y(i + 1, j + 1) + rf.y(i - 1, j) + rf.y(i - 1, j + 1));
}

// ---- coarsest level ----------------------------------------------------------

// Solve L L^* x = b with the lower Cholesky factor Lf (column-major n x n), by one
// warp (all 32 lanes call it); x and b may not alias.
template <class T>
__device__ __forceinline__ void chol_solve_warp(const cx<T>* Lf, int n, const cx<T>* b, cx<T>* x, int lane) {
  // forward: L y = b  (y stored in x)
  for (int i = 0; i < n; ++i) {
    cx<T> acc = czero<T>();
    for (int k = lane; k < i; k += 32) acc = acc + cmul(Lf[(long)k * n + i], x[k]);
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) {
      const T d = Lf[(long)i * n + i].x;
      const cx<T> v = b[i] - acc;
      x[i] = mk<T>(v.x / d, v.y / d);
    }
    __syncwarp();
  }
  // backward: L^* x = y
  for (int i = n - 1; i >= 0; --i) {
    cx<T> acc = czero<T>();
    for (int k = i + 1 + lane; k < n; k += 32) acc = acc + cmulc(Lf[(long)i * n + k], x[k]);
    for (int o = 16; o > 0; o >>= 1) {
      acc.x += __shfl_xor_sync(0xffffffffu, acc.x, o);
      acc.y += __shfl_xor_sync(0xffffffffu, acc.y, o);
    }
    if (lane == 0) {
      const T d = Lf[(long)i * n + i].x;
      const cx<T> v = x[i] - acc;
      x[i] = mk<T>(v.x / d, v.y / d);
    }
    __syncwarp();
  }
}

// The same solve with the factor in shared memory at leading dimension ld (n + 1
// keeps both a column and a row of it free of bank conflicts), both triangular
// sweeps in column order: once x_k is known, its multiple of column k of L (row
// k of L^*) leaves the remaining right-hand side, so a step is one division and
// one strided update with no reduction.
template <class T>
__device__ __forceinline__ void chol_solve_warp_cols(const cx<T>* Lf, int ld, int n, const cx<T>* b, cx<T>* x,
                                                     int lane) {
  for (int j = lane; j < n; j += 32) x[j] = b[j];
  __syncwarp();
  // forward: L y = b  (y stored in x)
  for (int k = 0; k < n; ++k) {
    const T d = Lf[k * ld + k].x;
    const cx<T> v = x[k];
    const cx<T> y = mk<T>(v.x / d, v.y / d);
    for (int j = k + 1 + lane; j < n; j += 32) x[j] = x[j] - cmul(Lf[k * ld + j], y);
    __syncwarp();
    if (lane == 0) x[k] = y;
    __syncwarp();
  }
  // backward: L^* x = y, (L^*)(i,k) = conj(L(k,i)) = conj(Lf[i ld + k])
  for (int k = n - 1; k >= 0; --k) {
    const T d = Lf[k * ld + k].x;
    const cx<T> v = x[k];
    const cx<T> xk = mk<T>(v.x / d, v.y / d);
    for (int i = lane; i < k; i += 32) x[i] = x[i] - cmulc(Lf[i * ld + k], xk);
    __syncwarp();
    if (lane == 0) x[k] = xk;
    __syncwarp();
  }
}

}  // namespace pbs
