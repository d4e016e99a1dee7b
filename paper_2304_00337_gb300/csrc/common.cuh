// Device-side building blocks shared by the pbs kernels: complex arithmetic on
// float2/double2, the Bloch "ghost" readers and the edge / nodal stencils.
//
// Discretisation (Boerm, Koehl, Talebi, arXiv:2304.00337, Section 3), written
// zero-based: x-edge (i,j) = [i h1,(i+1) h1] x {j h2}, y-edge (i,j) =
// {i h1} x [j h2,(j+1) h2], cell (i,j) = [i h1,(i+1) h1] x [j h2,(j+1) h2],
// node (i,j) = (i h1, j h2).  Every field (edge, cell or node) is extended
// quasi-periodically: an index j >= m reads beta * f(j - m), j < 0 reads
// conj(beta) * f(j + m), and likewise in i with alpha (alpha = exp(i k1 a),
// beta = exp(i k2 b), Section 1 eq. bloch_boundary).  With that extension every
// operator of the paper is a plain constant-coefficient stencil:
//   curl of cell (i,j):  c = x(i,j+1) - x(i,j) - y(i+1,j) + y(i,j)
//   A = C^* W C,  W = diag(1/(eps_c h1 h2))
//   (M u)_x(i,j) = (h2/h1) [2/3 u_x(i,j) + 1/6 (u_x(i,j+1) + u_x(i,j-1))]
//   (M u)_y(i,j) = (h1/h2) [2/3 u_y(i,j) + 1/6 (u_y(i+1,j) + u_y(i-1,j))]
//   (L phi)_x(i,j) = phi(i+1,j) - phi(i,j),  (L phi)_y(i,j) = phi(i,j+1) - phi(i,j)
// (the stencils follow from the element integrals of the basis functions).
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

#include "df32.cuh"

namespace pbs {

template <class T> struct cx_of;
template <> struct cx_of<double> { using type = double2; };
template <> struct cx_of<float> { using type = float2; };
template <> struct cx_of<df> { using type = dcx; };
template <class T> using cx = typename cx_of<T>::type;

template <class T> __host__ __device__ __forceinline__ cx<T> mk(T r, T i) {
  cx<T> z;
  z.x = r;
  z.y = i;
  return z;
}
template <class T> __host__ __device__ __forceinline__ cx<T> czero() { return mk<T>(T(0), T(0)); }
__host__ __device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__host__ __device__ __forceinline__ double2 operator-(double2 a) { return make_double2(-a.x, -a.y); }
__host__ __device__ __forceinline__ float2 operator-(float2 a) { return make_float2(-a.x, -a.y); }
__host__ __device__ __forceinline__ double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__host__ __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// conj(a) * b
__host__ __device__ __forceinline__ double2 cmulc(double2 a, double2 b) {
  return make_double2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x);
}
__host__ __device__ __forceinline__ double2 conj(double2 a) { return make_double2(a.x, -a.y); }
__host__ __device__ __forceinline__ float2 conj(float2 a) { return make_float2(a.x, -a.y); }
__host__ __device__ __forceinline__ double nrm2(double2 a) { return a.x * a.x + a.y * a.y; }
__host__ __device__ __forceinline__ float nrm2(float2 a) { return a.x * a.x + a.y * a.y; }

template <class T> __device__ __forceinline__ cx<T> to_cx(double2 v) { return mk<T>(T(v.x), T(v.y)); }
template <class T> __device__ __forceinline__ cx<T> to_cx(float2 v) { return mk<T>(T(v.x), T(v.y)); }

// Bloch phases of one column group: device array of 4 doubles per group
// (alpha.re, alpha.im, beta.re, beta.im).
template <class T> struct Ph {
  cx<T> al, be;
};
template <class T> __device__ __forceinline__ cx<T> ph_as(double re, double im);
template <class T> __device__ __forceinline__ Ph<T> load_ph(const double* ph, int group) {
  Ph<T> p;
  p.al = ph_as<T>(ph[4 * group + 0], ph[4 * group + 1]);
  p.be = ph_as<T>(ph[4 * group + 2], ph[4 * group + 3]);
  return p;
}

// Quasi-periodic read of a scalar field f on an n x m index grid; (i, j) may lie
// one step outside [0,n) x [0,m) in each direction.
template <class T>
__device__ __forceinline__ cx<T> gread(const cx<T>* __restrict__ f, int i, int j, int n, int m, const Ph<T>& p) {
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

// FP64 storage read in arithmetic T (double: as is; df: split by integer operations;
// float: rounded).
template <class T> __device__ __forceinline__ cx<T> ld_as(const double2* p);
template <> __device__ __forceinline__ double2 ld_as<double>(const double2* p) { return *p; }
template <> __device__ __forceinline__ dcx ld_as<df>(const double2* p) { return dcx_split(*p); }
template <> __device__ __forceinline__ float2 ld_as<float>(const double2* p) {
  const double2 v = *p;
  return make_float2(d2f_rn(v.x), d2f_rn(v.y));
}
template <class T> __device__ __forceinline__ T ld_scalar(double d);
template <> __device__ __forceinline__ double ld_scalar<double>(double d) { return d; }
template <> __device__ __forceinline__ df ld_scalar<df>(double d) { return df_split(d); }
__device__ __forceinline__ double2 to_d2(double2 v) { return v; }
__device__ __forceinline__ double2 to_d2(dcx v) { return dcx_to(v); }
__device__ __forceinline__ double to_double(double v) { return v; }
__device__ __forceinline__ double to_double(df v) { return df_to(v); }
template <class T> __device__ __forceinline__ T narrow(double v) { return T(v); }
template <> __device__ __forceinline__ float narrow<float>(double v) { return d2f_rn(v); }
template <class T> __device__ __forceinline__ T narrow(df v);
template <> __device__ __forceinline__ float narrow<float>(df v) { return df_to_float(v); }
template <> __device__ __forceinline__ double narrow<double>(df v) { return df_to(v); }
// exact widening of a stored value to the arithmetic type
template <class T> __device__ __forceinline__ cx<T> widen(float2 v);
template <> __device__ __forceinline__ double2 widen<double>(float2 v) {
  return make_double2(f2d_exact(v.x), f2d_exact(v.y));
}
template <> __device__ __forceinline__ dcx widen<df>(float2 v) {
  return dcx_make(df_make(v.x, 0.0f), df_make(v.y, 0.0f));
}
template <class T> __device__ __forceinline__ cx<T> widen(double2 v);
template <> __device__ __forceinline__ double2 widen<double>(double2 v) { return v; }
template <> __device__ __forceinline__ dcx widen<df>(double2 v) { return dcx_split(v); }

// Phases in the arithmetic of a kernel
template <class T> __device__ __forceinline__ cx<T> ph_as(double re, double im);
template <> __device__ __forceinline__ double2 ph_as<double>(double re, double im) { return make_double2(re, im); }
template <> __device__ __forceinline__ float2 ph_as<float>(double re, double im) {
  return make_float2(d2f_rn(re), d2f_rn(im));
}
template <> __device__ __forceinline__ dcx ph_as<df>(double re, double im) {
  return dcx_make(df_split(re), df_split(im));
}

// gread of FP64 storage in arithmetic T
template <class T>
__device__ __forceinline__ cx<T> gread_d(const double2* __restrict__ f, int i, int j, int n, int m, const Ph<T>& p) {
  bool w = false;
  cx<T> ph = mk<T>(T(1.0), T(0.0));
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
  const cx<T> v = ld_as<T>(f + (long)j * n + i);
  return w ? cmul(v, ph) : v;
}
// Reader of an FP64 edge vector in arithmetic T
template <class T> struct ERdD {
  const double2* __restrict__ X;
  int n, m;
  Ph<T> p;
  __device__ __forceinline__ cx<T> x(int i, int j) const { return gread_d<T>(X, i, j, n, m, p); }
  __device__ __forceinline__ cx<T> y(int i, int j) const { return gread_d<T>(X + (long)n * m, i, j, n, m, p); }
};

// The same away from the boundary (no wrap, no phase): the caller checks that every
// read stays inside the level.
template <class T> struct ERdDIn {
  const double2* __restrict__ X;
  int n;
  long N;
  __device__ __forceinline__ cx<T> x(int i, int j) const { return ld_as<T>(X + (long)j * n + i); }
  __device__ __forceinline__ cx<T> y(int i, int j) const { return ld_as<T>(X + N + (long)j * n + i); }
};

// Reader of one edge vector from memory (x-edges at X, y-edges at X + n*m).
template <class T> struct ERd {
  const cx<T>* __restrict__ X;
  int n, m;
  Ph<T> p;
  __device__ __forceinline__ cx<T> x(int i, int j) const { return gread<T>(X, i, j, n, m, p); }
  __device__ __forceinline__ cx<T> y(int i, int j) const { return gread<T>(X + (long)n * m, i, j, n, m, p); }
};

// Reader of a unit edge vector (kind 0 = x, 1 = y; index j*n+i): assembles
// columns of the coarsest-level matrices with the same stencil code.
template <class T> struct UnitERd {
  int n, m, kind, idx;
  Ph<T> p;
  __device__ __forceinline__ cx<T> at(int k, int i, int j) const {
    cx<T> ph = mk<T>(T(1), T(0));
    if (i < 0) { i += n; ph = conj(p.al); } else if (i >= n) { i -= n; ph = p.al; }
    if (j < 0) { j += m; ph = cmul(ph, conj(p.be)); } else if (j >= m) { j -= m; ph = cmul(ph, p.be); }
    return (k == kind && j * n + i == idx) ? ph : czero<T>();
  }
  __device__ __forceinline__ cx<T> x(int i, int j) const { return at(0, i, j); }
  __device__ __forceinline__ cx<T> y(int i, int j) const { return at(1, i, j); }
};

// Cellwise weights w = (1/eps) / (h1 h2), periodic (no phase: eps is periodic).
template <class T> struct Wts {
  const T* __restrict__ winv;  // 1/eps per cell of this level
  int n, m;
  T scale;  // 1 / (h1 h2)
  __device__ __forceinline__ T operator()(int i, int j) const {
    if (i < 0) i += n; else if (i >= n) i -= n;
    if (j < 0) j += m; else if (j >= m) j -= m;
    return scale * winv[(long)j * n + i];
  }
};

// The same weights as double-floats, pre-scaled by 1 / (h1 h2) (level 0 only).
struct WtsDF {
  const float2* __restrict__ w;  // (hi, lo) per cell
  int n, m;
  __device__ __forceinline__ df operator()(int i, int j) const {
    if (i < 0) i += n; else if (i >= n) i -= n;
    if (j < 0) j += m; else if (j >= m) j -= m;
    const float2 v = w[(long)j * n + i];
    return df_make(v.x, v.y);
  }
};

// Level geometry constants.
template <class T> struct Lvl {
  int n, m;
  T mx;  // h2/h1: mass and curl-curl scaling along x-edges
  T my;  // h1/h2
};

template <class T, class R> __device__ __forceinline__ cx<T> curl_at(const R& r, int i, int j) {
  return r.x(i, j + 1) - r.x(i, j) - r.y(i + 1, j) + r.y(i, j);
}
// (A u) at x-edge (i,j): top of cell (i,j-1), bottom of cell (i,j)
template <class T, class R, class W> __device__ __forceinline__ cx<T> A_x(const R& r, const W& w, int i, int j) {
  return w(i, j - 1) * curl_at<T>(r, i, j - 1) - w(i, j) * curl_at<T>(r, i, j);
}
// (A u) at y-edge (i,j): right of cell (i-1,j), left of cell (i,j)
template <class T, class R, class W> __device__ __forceinline__ cx<T> A_y(const R& r, const W& w, int i, int j) {
  return w(i, j) * curl_at<T>(r, i, j) - w(i - 1, j) * curl_at<T>(r, i - 1, j);
}
template <class T, class R> __device__ __forceinline__ cx<T> M_x(const R& r, const Lvl<T>& L, int i, int j) {
  return L.mx * (T(2.0 / 3.0) * r.x(i, j) + T(1.0 / 6.0) * (r.x(i, j + 1) + r.x(i, j - 1)));
}
template <class T, class R> __device__ __forceinline__ cx<T> M_y(const R& r, const Lvl<T>& L, int i, int j) {
  return L.my * (T(2.0 / 3.0) * r.y(i, j) + T(1.0 / 6.0) * (r.y(i + 1, j) + r.y(i - 1, j)));
}

// Nodal operator P = L^* M L (the Bloch Q1 Laplacian, Section 5):
//   (h2/h1)/6 [-1 2 -1]_x (x) [1 4 1]_y + (h1/h2)/6 [1 4 1]_x (x) [-1 2 -1]_y
template <class T> struct NRd {
  const cx<T>* __restrict__ X;
  int n, m;
  Ph<T> p;
  __device__ __forceinline__ cx<T> v(int i, int j) const { return gread<T>(X, i, j, n, m, p); }
};
template <class T> struct UnitNRd {
  int n, m, idx;
  Ph<T> p;
  __device__ __forceinline__ cx<T> v(int i, int j) const {
    cx<T> ph = mk<T>(T(1), T(0));
    if (i < 0) { i += n; ph = conj(p.al); } else if (i >= n) { i -= n; ph = p.al; }
    if (j < 0) { j += m; ph = cmul(ph, conj(p.be)); } else if (j >= m) { j -= m; ph = cmul(ph, p.be); }
    return (j * n + i == idx) ? ph : czero<T>();
  }
};
template <class T, class R> __device__ __forceinline__ cx<T> P_at(const R& r, const Lvl<T>& L, int i, int j) {
  cx<T> acc_x = czero<T>(), acc_y = czero<T>();
#pragma unroll
  for (int d = -1; d <= 1; ++d) {
    const T wgt = d == 0 ? T(4) : T(1);
    acc_x = acc_x + wgt * (T(2) * r.v(i, j + d) - r.v(i - 1, j + d) - r.v(i + 1, j + d));
    acc_y = acc_y + wgt * (T(2) * r.v(i + d, j) - r.v(i + d, j - 1) - r.v(i + d, j + 1));
  }
  return (L.mx * T(1.0 / 6.0)) * acc_x + (L.my * T(1.0 / 6.0)) * acc_y;
}
template <class T> __host__ __device__ __forceinline__ T P_diag(const Lvl<T>& L) {
  return T(4.0 / 3.0) * (L.mx + L.my);
}

}  // namespace pbs
