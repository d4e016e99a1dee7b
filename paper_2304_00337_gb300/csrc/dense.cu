// Block kernels of the eigen-iteration (Section 4): FP64 residuals and
// Rayleigh quotients, the projection's right-hand side and update, the block
// Gram matrices, the small dense Rayleigh-Ritz step and the block update.
// Reductions are two-stage with a fixed summation order (deterministic).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <type_traits>

#include "df32.cuh"
#include "internal.h"
#include "mgpoint.cuh"

namespace pbs {

namespace {

constexpr int kBX = 32, kBY = 8, kThreads = kBX * kBY;

inline dim3 grid2(int n, int m, int ncols) { return dim3((n + kBX - 1) / kBX, (m + kBY - 1) / kBY, ncols); }

// Block-wide sum of two doubles; result valid in thread 0.
__device__ __forceinline__ void block_sum2(double& a, double& b) {
  __shared__ double sa[32], sb[32];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, o);
    b += __shfl_xor_sync(0xffffffffu, b, o);
  }
  if (lane == 0) {
    sa[wid] = a;
    sb[wid] = b;
  }
  __syncthreads();
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
  if (wid == 0) {
    a = lane < nw ? sa[lane] : 0.0;
    b = lane < nw ? sb[lane] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
  }
}

__device__ __forceinline__ df shfl_df(df v, int o) {
  return df_make(__shfl_xor_sync(0xffffffffu, v.hi, o), __shfl_xor_sync(0xffffffffu, v.lo, o));
}

// Block-wide sum of two double-floats (fixed order); result valid in thread 0.
__device__ __forceinline__ void block_sum2(df& a, df& b) {
  __shared__ df sa[32], sb[32];
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, lane = tid & 31, wid = tid >> 5;
  for (int o = 16; o > 0; o >>= 1) {
    a = a + df_make(__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o));
    b = b + df_make(__shfl_xor_sync(0xffffffffu, b.hi, o), __shfl_xor_sync(0xffffffffu, b.lo, o));
  }
  if (lane == 0) {
    sa[wid] = a;
    sb[wid] = b;
  }
  __syncthreads();
  const int nw = (blockDim.x * blockDim.y + 31) >> 5;
  if (wid == 0) {
    a = lane < nw ? sa[lane] : df_zero();
    b = lane < nw ? sb[lane] : df_zero();
    for (int o = 16; o > 0; o >>= 1) {
      a = a + df_make(__shfl_xor_sync(0xffffffffu, a.hi, o), __shfl_xor_sync(0xffffffffu, a.lo, o));
      b = b + df_make(__shfl_xor_sync(0xffffffffu, b.hi, o), __shfl_xor_sync(0xffffffffu, b.lo, o));
    }
  }
}

// partials: [ncols][nblk][2] -> out [ncols][2], fixed order
__global__ void k_finalize2(const double* __restrict__ part, int nblk, double* __restrict__ out) {
  const int c = blockIdx.x;
  double a = 0, b = 0;
  for (int t = threadIdx.x; t < nblk; t += blockDim.x) {
    a += part[((long)c * nblk + t) * 2];
    b += part[((long)c * nblk + t) * 2 + 1];
  }
  block_sum2(a, b);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    out[2 * c] = a;
    out[2 * c + 1] = b;
  }
}

// The mass matrix in factored form (Gram matrices, Rayleigh quotients).  Along an edge set the mass
// matrix is mx tridiag(1/6, 2/3, 1/6) with Bloch wrap (x-edges couple in j, y-edges
// in i), and tridiag(1/6, 2/3, 1/6) = B^* B for the bidiagonal B with diagonal alpha
// and upper diagonal beta, alpha = (1 + 1/sqrt(3))/2, beta = (1 - 1/sqrt(3))/2
// (alpha^2 + beta^2 = 2/3, alpha beta = 1/6; the wrap entry carries the phase).  So
// S^* M S = (B S)^* (B S) with z_x(i,j) = sqrt(mx) (alpha x(i,j) + beta x(i,j+1))
// and z_y(i,j) = sqrt(my) (alpha y(i,j) + beta y(i+1,j)): two staged arrays read
// on both sides of the product instead of x, y and M x, M y.
struct MassFactor {
  df ax, bx, ay, by;  // sqrt(mx) alpha, sqrt(mx) beta, sqrt(my) alpha, sqrt(my) beta
};
MassFactor mass_factor(const Level& L) {
  const double r3 = 1.0 / std::sqrt(3.0), al = 0.5 * (1.0 + r3), be = 0.5 * (1.0 - r3);
  const double sx = std::sqrt(L.h2 / L.h1), sy = std::sqrt(L.h1 / L.h2);
  return MassFactor{df(sx * al), df(sx * be), df(sy * al), df(sy * be)};
}

// The kernels below read and write FP64 blocks; V is the arithmetic: double
// (plain FP64) or df (double-float on the FP32 pipe, about 2^-47 relative).

template <class V, class W>
__global__ void k_rayleigh_parts(Lvl<V> L, W w, MassFactor mf, const double* ph, int cpg,
                                 const double2* __restrict__ X, long ld, double* __restrict__ part) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, c = blockIdx.z;
  V den = V(0.0), num = V(0.0);
  if constexpr (std::is_same<V, df>::value) {
    // double-float: e^* M e = |z_x|^2 + |z_y|^2 (factored mass), and plain reads where
    // the stencil stays inside the level
    const auto parts = [&](const auto& r) {
      const dcx x0 = r.x(i, j), x1 = r.x(i, j + 1), y0 = r.y(i, j), y1 = r.y(i + 1, j);
      den = nrm2(mf.ax * x0 + mf.bx * x1) + nrm2(mf.ay * y0 + mf.by * y1);
      num = w(i, j) * nrm2(x1 - x0 - y1 + y0);  // curl_at's order
    };
    if (i < L.n && j < L.m) {
      if (inside(i, j, L.n, L.m, 1, 1)) parts(ERdDIn<df>{X + c * ld, L.n, (long)L.n * L.m});
      else parts(ERdD<df>{X + c * ld, L.n, L.m, load_ph<df>(ph, c / cpg)});
    }
  } else if (i < L.n && j < L.m) {
    const ERdD<V> r{X + c * ld, L.n, L.m, load_ph<V>(ph, c / cpg)};
    const cx<V> mx = M_x<V>(r, L, i, j), my = M_y<V>(r, L, i, j);
    const cx<V> ex = r.x(i, j), ey = r.y(i, j);
    den = ex.x * mx.x + ex.y * mx.y + ey.x * my.x + ey.y * my.y;
    num = w(i, j) * nrm2(curl_at<V>(r, i, j));
  }
  block_sum2(den, num);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const int nblk = gridDim.x * gridDim.y, b = blockIdx.y * gridDim.x + blockIdx.x;
    part[((long)c * nblk + b) * 2] = to_double(den);
    part[((long)c * nblk + b) * 2 + 1] = to_double(num);
  }
}

// R = A E - lam M E in FP64 in every precision policy: the iterate enters through
// a stencil whose terms are up to lambda_max / lambda larger than the result, so
// a perturbation of the stored vector of relative size eta moves the relative
// residual by about eta lambda_max / lambda (1.6e7 at 256 x 256 next to Gamma),
// which only FP64's 1.1e-16 keeps well under a tolerance of 1e-8.
// FP64 issues slowly on this GPU, so the kernel spends as few FP64 operations as
// it can: each CTA forms H = w curl once per cell of its 32 x 8 tile and of a
// one-cell halo below and to the left (shared memory), A_x = H(i,j-1) - H(i,j),
// A_y = H(i,j) - H(i-1,j), and the mass stencil is (h2/h1)/6 (4 x0 + x+ + x-).
// Reader of a tile region staged in shared memory (origin (oi, oj), row widths wx, wy).
template <class V> struct TileERd {  // edge values of a tile region, x-edge (i, j) at sx[(j - oj) wx + i - oi]
  const cx<V>* sx;
  const cx<V>* sy;
  int oi, oj, wx, wy;
  __device__ __forceinline__ cx<V> x(int i, int j) const { return sx[(j - oj) * wx + (i - oi)]; }
  __device__ __forceinline__ cx<V> y(int i, int j) const { return sy[(j - oj) * wy + (i - oi)]; }
};

// Bloch phase of an index one step outside the level, formed in the order the
// extended readers use.
__device__ __forceinline__ double2 bloch_phase(int i, int j, int n, int m, const Ph<double>& p) {
  double2 ph = make_double2(1.0, 0.0);
  if (i < 0) ph = conj(p.al);
  else if (i >= n) ph = p.al;
  if (j < 0) ph = cmul(ph, conj(p.be));
  else if (j >= m) ph = cmul(ph, p.be);
  return ph;
}

// Stage the edges of one field around a tile: region element (a, b), a < w, b < h,
// is edge (i0 - 1 + a, j0 - 1 + b) of the field at F (n x m); only a <= amax and
// b <= bmax are read.  Edges inside the level are copied; those one step outside
// (only on the region's ring) are read through the Bloch extension by one thread
// each, so the phase products are not spread over every element.
__device__ __forceinline__ void stage_field(const double2* __restrict__ F, int n, int m, const Ph<double>& p,
                                            int i0, int j0, int w, int h, int amax, int bmax, double2* S) {
  const int tid = threadIdx.y * blockDim.x + threadIdx.x, nt = blockDim.x * blockDim.y;
  for (int t = tid; t < w * h; t += nt) {
    const int a = t % w, b = t / w, i = i0 - 1 + a, j = j0 - 1 + b;
    if (a <= amax && b <= bmax && i >= 0 && i < n && j >= 0 && j < m) S[t] = F[(long)j * n + i];
  }
  // ring: rows b = 0 and b = bmax (a = 0 .. amax), columns a = 0 and a = amax (b = 1 .. bmax - 1)
  const int ring = 2 * (amax + 1) + 2 * max(bmax - 1, 0);
  for (int t = tid; t < ring; t += nt) {
    int a, b;
    if (t < 2 * (amax + 1)) {
      a = t % (amax + 1);
      b = t < amax + 1 ? 0 : bmax;
    } else {
      const int u = t - 2 * (amax + 1);
      a = u % 2 == 0 ? 0 : amax;
      b = 1 + u / 2;
    }
    const int i = i0 - 1 + a, j = j0 - 1 + b;
    if (i >= 0 && i < n && j >= 0 && j < m) continue;
    const int ii = i < 0 ? i + n : (i >= n ? i - n : i), jj = j < 0 ? j + m : (j >= m ? j - m : j);
    S[b * w + a] = cmul(F[(long)jj * n + ii], bloch_phase(i, j, n, m, p));
  }
}

// The tile's work with a reader r and weights w (the Bloch-extended ones, or the
// direct ones on tiles whose reads all stay inside the level).
template <class Rd, class Wt>
__device__ __forceinline__ void residual_tile(const Lvl<double>& L, const Wt& w, const Rd& r, double l,
                                              double2* __restrict__ Rc, double& rr, double& mm) {
  __shared__ double2 Hs[kBY + 1][kBX + 1];  // cell (i0 - 1 + a, j0 - 1 + b) at Hs[b][a]
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i0 = blockIdx.x * kBX, j0 = blockIdx.y * kBY;
  const int i = i0 + tx, j = j0 + ty;
  const bool in = i < L.n && j < L.m;
  if (in) Hs[ty + 1][tx + 1] = w(i, j) * curl_at<double>(r, i, j);
  if (ty == 0 && i < L.n) Hs[0][tx + 1] = w(i, j0 - 1) * curl_at<double>(r, i, j0 - 1);
  if (tx == 0 && j < L.m) Hs[ty + 1][0] = w(i0 - 1, j) * curl_at<double>(r, i0 - 1, j);
  __syncthreads();
  if (in) {
    const double sx = L.mx * (1.0 / 6.0), sy = L.my * (1.0 / 6.0);
    const double2 x0 = r.x(i, j), x1 = r.x(i, j + 1), x2 = r.x(i, j - 1);
    const double2 y0 = r.y(i, j), y1 = r.y(i + 1, j), y2 = r.y(i - 1, j);
    const double2 mx = make_double2(sx * fma(4.0, x0.x, x1.x + x2.x), sx * fma(4.0, x0.y, x1.y + x2.y));
    const double2 my = make_double2(sy * fma(4.0, y0.x, y1.x + y2.x), sy * fma(4.0, y0.y, y1.y + y2.y));
    const double2 h = Hs[ty + 1][tx + 1], hb = Hs[ty][tx + 1], hl = Hs[ty + 1][tx];
    const double2 rx = make_double2(fma(-l, mx.x, hb.x - h.x), fma(-l, mx.y, hb.y - h.y));
    const double2 ry = make_double2(fma(-l, my.x, h.x - hl.x), fma(-l, my.y, h.y - hl.y));
    const long N = (long)L.n * L.m, e = (long)j * L.n + i;
    Rc[e] = rx;
    Rc[N + e] = ry;
    rr = fma(rx.x, rx.x, fma(rx.y, rx.y, fma(ry.x, ry.x, ry.y * ry.y)));
    mm = fma(mx.x, mx.x, fma(mx.y, mx.y, fma(my.x, my.x, my.y * my.y)));
  }
}

__global__ void __launch_bounds__(kBX * kBY) k_residual(Lvl<double> L, Wts<double> w, const double* ph, int cpg,
                                                         const double2* __restrict__ E, double2* __restrict__ R,
                                                         long ld, const double* __restrict__ lam,
                                                         double* __restrict__ part) {
  const int i0 = blockIdx.x * kBX, j0 = blockIdx.y * kBY, c = blockIdx.z;
  double rr = 0, mm = 0;
  // every read of the tile (indices i0 - 1 .. i0 + kBX, j0 - 1 .. j0 + kBY) inside the level
  if (i0 >= 1 && j0 >= 1 && i0 + kBX < L.n && j0 + kBY < L.m) {
    residual_tile(L, WtsIn<double>{w.winv, w.n, w.scale}, ERdIn<double>{E + c * ld, L.n, (long)L.n * L.m},
                  lam[c], R + c * ld, rr, mm);
  } else {
    // tiles at the level's edges: x-edges (i0 - 1 .. i0 + nx - 1, j0 - 1 .. j0 + ny) and y-edges
    // (i0 - 1 .. i0 + nx, j0 - 1 .. j0 + ny - 1) staged with their Bloch phases
    constexpr int WX = kBX + 1, WY = kBX + 2;
    __shared__ double2 sx[(kBY + 2) * WX], sy[(kBY + 1) * WY];
    const int nx = min(kBX, L.n - i0), ny = min(kBY, L.m - j0);
    const Ph<double> p = load_ph<double>(ph, c / cpg);
    const double2* Ec = E + c * ld;
    stage_field(Ec, L.n, L.m, p, i0, j0, WX, kBY + 2, nx, ny + 1, sx);
    stage_field(Ec + (long)L.n * L.m, L.n, L.m, p, i0, j0, WY, kBY + 1, nx + 1, ny, sy);
    __syncthreads();
    residual_tile(L, w, TileERd<double>{sx, sy, i0 - 1, j0 - 1, WX, WY}, lam[c], R + c * ld, rr, mm);
  }
  block_sum2(rr, mm);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const int nblk = gridDim.x * gridDim.y, b = blockIdx.y * gridDim.x + blockIdx.x;
    part[((long)c * nblk + b) * 2] = rr;
    part[((long)c * nblk + b) * 2 + 1] = mm;
  }
}

// The same residual for the mixed policy, whose preconditioner reads it in FP32.
// The curls c = x(i,j+1) - x(i,j) - y(i+1,j) + y(i,j) are formed in FP64: they are
// where the stencil cancels (neighbouring values of a smooth iterate nearly agree),
// and their FP64 rounding is the floor every policy shares.  Everything after them -
// H = w c, the differences of H, the mass stencil and R = A e - lambda M e - is
// double-float: those steps see the curls and the iterate's values themselves, so a
// relative rounding of 2^-47 there moves the relative residual by about 2^-47 (H
// differences: 2^-47 sqrt(lambda_max / lambda), 1e-10 next to Gamma at 1024^2), far
// below any tolerance.  R is stored rounded to FP32 and the norms |R|^2, |M e|^2 are
// summed per thread in FP32 and across the block in FP64 (the convergence test needs
// a few digits of them).  FP64 work: the curls only (about 7 operations per node
// against about 45 in the all-FP64 kernel).
template <class Rd>
__device__ __forceinline__ void residual_tile_mixed(const Lvl<df>& L, const WtsDF& w, const Rd& r, df l,
                                                    float2* __restrict__ Rc, double& rr, double& mm) {
  __shared__ dcx Hs[kBY + 1][kBX + 1];  // cell (i0 - 1 + a, j0 - 1 + b) at Hs[b][a]
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int i0 = blockIdx.x * kBX, j0 = blockIdx.y * kBY;
  const int i = i0 + tx, j = j0 + ty;
  const bool in = i < L.n && j < L.m;
  if (in) Hs[ty + 1][tx + 1] = w(i, j) * dcx_split(curl_at<double>(r, i, j));
  if (ty == 0 && i < L.n) Hs[0][tx + 1] = w(i, j0 - 1) * dcx_split(curl_at<double>(r, i, j0 - 1));
  if (tx == 0 && j < L.m) Hs[ty + 1][0] = w(i0 - 1, j) * dcx_split(curl_at<double>(r, i0 - 1, j));
  __syncthreads();
  if (in) {
    const df sx = L.mx * df(1.0 / 6.0), sy = L.my * df(1.0 / 6.0), four = df(4.0);
    const dcx x0 = dcx_split(r.x(i, j)), x1 = dcx_split(r.x(i, j + 1)), x2 = dcx_split(r.x(i, j - 1));
    const dcx y0 = dcx_split(r.y(i, j)), y1 = dcx_split(r.y(i + 1, j)), y2 = dcx_split(r.y(i - 1, j));
    const dcx mx = sx * (four * x0 + (x1 + x2));
    const dcx my = sy * (four * y0 + (y1 + y2));
    const dcx h = Hs[ty + 1][tx + 1], hb = Hs[ty][tx + 1], hl = Hs[ty + 1][tx];
    const dcx rx = (hb - h) - l * mx;
    const dcx ry = (h - hl) - l * my;
    const long N = (long)L.n * L.m, e = (long)j * L.n + i;
    const float2 fx = make_float2(df_to_float(rx.x), df_to_float(rx.y));
    const float2 fy = make_float2(df_to_float(ry.x), df_to_float(ry.y));
    Rc[e] = fx;
    Rc[N + e] = fy;
    const float r2 = fmaf(fx.x, fx.x, fmaf(fx.y, fx.y, fmaf(fy.x, fy.x, fy.y * fy.y)));
    const float mxf = df_to_float(mx.x), mxi = df_to_float(mx.y), myf = df_to_float(my.x), myi = df_to_float(my.y);
    const float m2 = fmaf(mxf, mxf, fmaf(mxi, mxi, fmaf(myf, myf, myi * myi)));
    rr = f2d_exact(r2);
    mm = f2d_exact(m2);
  }
}

__global__ void __launch_bounds__(kBX * kBY) k_residual_mixed(Lvl<df> L, WtsDF w, const double* ph, int cpg,
                                                               const double2* __restrict__ E, float2* __restrict__ R,
                                                               long ld, const double* __restrict__ lam,
                                                               double* __restrict__ part) {
  const int i0 = blockIdx.x * kBX, j0 = blockIdx.y * kBY, c = blockIdx.z;
  double rr = 0, mm = 0;
  const df l = df_split(lam[c]);
  if (i0 >= 1 && j0 >= 1 && i0 + kBX < L.n && j0 + kBY < L.m) {
    residual_tile_mixed(L, w, ERdIn<double>{E + c * ld, L.n, (long)L.n * L.m}, l, R + c * ld, rr, mm);
  } else {
    constexpr int WX = kBX + 1, WY = kBX + 2;
    __shared__ double2 sx[(kBY + 2) * WX], sy[(kBY + 1) * WY];
    const int nx = min(kBX, L.n - i0), ny = min(kBY, L.m - j0);
    const Ph<double> p = load_ph<double>(ph, c / cpg);
    const double2* Ec = E + c * ld;
    stage_field(Ec, L.n, L.m, p, i0, j0, WX, kBY + 2, nx, ny + 1, sx);
    stage_field(Ec + (long)L.n * L.m, L.n, L.m, p, i0, j0, WY, kBY + 1, nx + 1, ny, sy);
    __syncthreads();
    residual_tile_mixed(L, w, TileERd<double>{sx, sy, i0 - 1, j0 - 1, WX, WY}, l, R + c * ld, rr, mm);
  }
  block_sum2(rr, mm);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const int nblk = gridDim.x * gridDim.y, b = blockIdx.y * gridDim.x + blockIdx.x;
    part[((long)c * nblk + b) * 2] = rr;
    part[((long)c * nblk + b) * 2 + 1] = mm;
  }
}

// rhs(i,j) = (L^* M x)(i,j) = (Mx)_x(i-1,j) - (Mx)_x(i,j) + (Mx)_y(i,j-1) - (Mx)_y(i,j),
// computed in V and stored in T.  A CTA stages the edge values its 32 x 8 nodes
// read (converted to V once), forms each mass-stencil value once in shared
// memory, then combines them; the stencil functions and the order of the sums
// are those of the per-node formula.
template <class V, class T>
__global__ void __launch_bounds__(kBX * kBY) k_lift_adj_mass(Lvl<V> L, const double* ph, int cpg,
                                                             const double2* __restrict__ X, long ldx,
                                                             cx<T>* __restrict__ Y, long ldy) {
  constexpr int WX = kBX + 1, WY = kBX + 2;
  __shared__ cx<V> sx[(kBY + 2) * WX];  // x-edges (i0 - 1 + a, j0 - 1 + b)
  __shared__ cx<V> sy[(kBY + 1) * WY];  // y-edges (i0 - 1 + a, j0 - 1 + b)
  __shared__ cx<V> mxs[kBY * WX];       // (Mx)_x(i0 - 1 + a, j0 + b)
  __shared__ cx<V> mys[(kBY + 1) * kBX];  // (Mx)_y(i0 + a, j0 - 1 + b)
  const int i0 = blockIdx.x * kBX, j0 = blockIdx.y * kBY, c = blockIdx.z;
  const int tid = threadIdx.y * kBX + threadIdx.x, nt = kBX * kBY;
  const int nx = min(kBX, L.n - i0), ny = min(kBY, L.m - j0);  // nodes of the tile inside the level
  const double2* xc = X + c * ldx;
  const long N = (long)L.n * L.m;
  // the values the tile's nodes read: x-edges a <= nx, b <= ny + 1; y-edges a <= nx + 1, b <= ny
  if (i0 >= 1 && j0 >= 1 && i0 + kBX < L.n && j0 + kBY < L.m) {
    for (int t = tid; t < (kBY + 2) * WX; t += nt)
      sx[t] = ld_as<V>(xc + (long)(j0 - 1 + t / WX) * L.n + (i0 - 1 + t % WX));
    for (int t = tid; t < (kBY + 1) * WY; t += nt)
      sy[t] = ld_as<V>(xc + N + (long)(j0 - 1 + t / WY) * L.n + (i0 - 1 + t % WY));
  } else {
    const ERdD<V> r{xc, L.n, L.m, load_ph<V>(ph, c / cpg)};
    for (int t = tid; t < (kBY + 2) * WX; t += nt) {
      const int a = t % WX, b = t / WX;
      if (a <= nx && b <= ny + 1) sx[t] = r.x(i0 - 1 + a, j0 - 1 + b);
    }
    for (int t = tid; t < (kBY + 1) * WY; t += nt) {
      const int a = t % WY, b = t / WY;
      if (a <= nx + 1 && b <= ny) sy[t] = r.y(i0 - 1 + a, j0 - 1 + b);
    }
  }
  __syncthreads();
  const TileERd<V> tr{sx, sy, i0 - 1, j0 - 1, WX, WY};
  for (int t = tid; t < kBY * WX; t += nt) {
    const int a = t % WX, b = t / WX;
    if (a <= nx && b < ny) mxs[t] = M_x<V>(tr, L, i0 - 1 + a, j0 + b);
  }
  for (int t = tid; t < (kBY + 1) * kBX; t += nt) {
    const int a = t % kBX, b = t / kBX;
    if (a < nx && b <= ny) mys[t] = M_y<V>(tr, L, i0 + a, j0 - 1 + b);
  }
  __syncthreads();
  const int a = threadIdx.x, b = threadIdx.y;
  if (a >= nx || b >= ny) return;
  const cx<V> v = mxs[b * WX + a] - mxs[b * WX + a + 1] + mys[b * kBX + a] - mys[(b + 1) * kBX + a];
  Y[c * ldy + (long)(j0 + b) * L.n + i0 + a] = mk<T>(narrow<T>(v.x), narrow<T>(v.y));
}

// x <- x - L phi, in FP64 in every precision policy (it writes the iterate; see
// k_residual); phi differences of FP32 values are exact in FP64
template <class T>
__global__ void k_sub_lift(int n, int m, const double* ph, int cpg, const cx<T>* __restrict__ Phi, long ldp,
                           double2* __restrict__ X, long ldx) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, c = blockIdx.z;
  if (i >= n || j >= m) return;
  const cx<T>* f = Phi + c * ldp;
  const long N = (long)n * m, e = (long)j * n + i;
  double2* x = X + c * ldx;
  // phi in FP64 (widened exactly by integer operations)
  auto at = [&](int ii, int jj) -> double2 { return widen<double>(f[(long)jj * n + ii]); };
  const double2 f0 = at(i, j);
  if (i + 1 < n && j + 1 < m) {  // no wrap: the common case, without phase products
    x[e] = x[e] - (at(i + 1, j) - f0);
    x[N + e] = x[N + e] - (at(i, j + 1) - f0);
    return;
  }
  // read phi in FP64 through the Bloch extension
  const Ph<double> p = load_ph<double>(ph, c / cpg);
  auto rd = [&](int ii, int jj) -> double2 {
    double2 ph1 = make_double2(1, 0);
    bool wr = false;
    if (ii >= n) { ii -= n; ph1 = p.al; wr = true; }
    if (jj >= m) { jj -= m; ph1 = cmul(ph1, p.be); wr = true; }
    const double2 d = at(ii, jj);
    return wr ? cmul(d, ph1) : d;
  };
  x[e] = x[e] - (rd(i + 1, j) - f0);
  x[N + e] = x[N + e] - (rd(i, j + 1) - f0);
}

// per column sums of the x-edge and y-edge values (for the constant-field deflation at k = 0)
__global__ void k_edge_sums(long N, const double2* __restrict__ X, long ld, double* __restrict__ part, int nblk,
                            const int* __restrict__ gamma, int cpg) {
  const int c = blockIdx.y;
  if (!gamma[c / cpg]) return;
  double sx_re = 0, sx_im = 0, sy_re = 0, sy_im = 0;
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < N; t += (long)gridDim.x * blockDim.x) {
    const double2 a = X[c * ld + t], b = X[c * ld + N + t];
    sx_re += a.x; sx_im += a.y; sy_re += b.x; sy_im += b.y;
  }
  block_sum2(sx_re, sx_im);
  __syncthreads();
  block_sum2(sy_re, sy_im);
  if (threadIdx.x == 0) {
    double* o = part + ((long)c * nblk + blockIdx.x) * 4;
    o[0] = sx_re; o[1] = sx_im; o[2] = sy_re; o[3] = sy_im;
  }
}

__global__ void k_edge_sub_means(long N, double2* __restrict__ X, long ld, const double* __restrict__ part, int nblk,
                                 const int* __restrict__ gamma, int cpg) {
  const int c = blockIdx.y;
  if (!gamma[c / cpg]) return;
  __shared__ double mean[4];
  if (threadIdx.x < 4) {
    double s = 0;
    for (int b = 0; b < nblk; ++b) s += part[((long)c * nblk + b) * 4 + threadIdx.x];
    mean[threadIdx.x] = s / double(N);
  }
  __syncthreads();
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < N; t += (long)gridDim.x * blockDim.x) {
    X[c * ld + t].x -= mean[0];
    X[c * ld + t].y -= mean[1];
    X[c * ld + N + t].x -= mean[2];
    X[c * ld + N + t].y -= mean[3];
  }
}

__global__ void k_d2f(const double2* __restrict__ X, float2* __restrict__ Y, long n) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    Y[t] = make_float2(d2f_rn(X[t].x), d2f_rn(X[t].y));
}
__global__ void k_f2d(const float2* __restrict__ X, double2* __restrict__ Y, long n) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    Y[t] = make_double2(f2d_exact(X[t].x), f2d_exact(X[t].y));
}

// ---- block Gram matrices of a trial block, fused with the stencils ---------
// For group g (blockIdx.y) and trial columns a, b (a <= b):
//   GM[a][b] = sum_edges conj(s_a) (M s_b),   GA[a][b] = sum_cells w |..| conj(c_a) c_b,  c = C s
// Each block takes chunks of kGramRows nodes; for every trial column it stages
// the node's x- and y-edge values, (M s) at those edges and the curl of the
// node's cell in shared memory, then accumulates its share of the q(q+1)/2
// entries.  Trial column a of group g lives at roles.b[a / pr] + (g pr + a % pr) ld.
constexpr int kGramRows = 16;
constexpr int kGramAcc = 20;  // accumulators per thread: q(q+1)/2 <= 20 * 256 for q <= 100

__device__ __forceinline__ const double2* role_col(const Roles& R, int g, int a) {
  const int r = a / R.pr;  // selects rather than an indexed load keep R out of local memory
  const double2* base = r == 0 ? R.b[0] : (r == 1 ? R.b[1] : R.b[2]);
  return base + ((long)g * R.pr + a % R.pr) * R.ld;
}

__global__ void __launch_bounds__(256) k_gram_fused(Lvl<double> L, Wts<double> w, const double* ph, Roles roles, int q,
                                                    double2* __restrict__ part, int npart) {
  extern __shared__ double2 sm[];
  const int g = blockIdx.y;
  const long N = (long)L.n * L.m;
  double2* sx = sm;                      // [q][kGramRows]
  double2* sy = sx + q * kGramRows;
  double2* mx = sy + q * kGramRows;
  double2* my = mx + q * kGramRows;
  double2* cc = my + q * kGramRows;      // w-scaled curl in cc_w, plain curl in cc
  double2* cw = cc + q * kGramRows;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ne = q * (q + 1) / 2;
  const Ph<double> p = load_ph<double>(ph, g);
  int ea[kGramAcc], eb[kGramAcc];
  double2 am[kGramAcc], aa[kGramAcc];
#pragma unroll
  for (int k = 0; k < kGramAcc; ++k) {
    am[k] = make_double2(0, 0);
    aa[k] = make_double2(0, 0);
    const int e = tid + k * nt;
    int ai = 0, bi = 0;
    if (e < ne) {  // column-major upper triangle: e = b(b+1)/2 + a
      bi = int((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
      while ((bi + 1) * (bi + 2) / 2 <= e) ++bi;
      while (bi * (bi + 1) / 2 > e) --bi;
      ai = e - bi * (bi + 1) / 2;
    }
    ea[k] = ai;
    eb[k] = bi;
  }
  const long nchunks = (N + kGramRows - 1) / kGramRows;
  for (long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const long r0 = ch * kGramRows;
    __syncthreads();
    for (int t = tid; t < q * kGramRows; t += nt) {
      const int col = t / kGramRows, rr = t % kGramRows;
      const long node = r0 + rr;
      double2 vx = make_double2(0, 0), vy = vx, vmx = vx, vmy = vx, vc = vx, vcw = vx;
      if (node < N) {
        const int i = int(node % L.n), j = int(node / L.n);
        const ERd<double> rd{role_col(roles, g, col), L.n, L.m, p};
        vx = rd.x(i, j);
        vy = rd.y(i, j);
        vmx = M_x<double>(rd, L, i, j);
        vmy = M_y<double>(rd, L, i, j);
        vc = curl_at<double>(rd, i, j);
        vcw = w(i, j) * vc;
      }
      sx[col * kGramRows + rr] = vx;
      sy[col * kGramRows + rr] = vy;
      mx[col * kGramRows + rr] = vmx;
      my[col * kGramRows + rr] = vmy;
      cc[col * kGramRows + rr] = vc;
      cw[col * kGramRows + rr] = vcw;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kGramAcc; ++k) {
      if (tid + k * nt < ne) {
        const int ia = ea[k] * kGramRows, ib = eb[k] * kGramRows;
        double2 sM = am[k], sA = aa[k];
#pragma unroll 4
        for (int rr = 0; rr < kGramRows; ++rr) {
          const double2 u = sx[ia + rr], v = mx[ib + rr], u2 = sy[ia + rr], v2 = my[ib + rr];
          sM.x = fma(u.x, v.x, fma(u.y, v.y, sM.x));
          sM.y = fma(u.x, v.y, fma(-u.y, v.x, sM.y));
          sM.x = fma(u2.x, v2.x, fma(u2.y, v2.y, sM.x));
          sM.y = fma(u2.x, v2.y, fma(-u2.y, v2.x, sM.y));
          const double2 c1 = cc[ia + rr], c2 = cw[ib + rr];
          sA.x = fma(c1.x, c2.x, fma(c1.y, c2.y, sA.x));
          sA.y = fma(c1.x, c2.y, fma(-c1.y, c2.x, sA.y));
        }
        am[k] = sM;
        aa[k] = sA;
      }
    }
  }
  double2* pm = part + ((long)g * npart + blockIdx.x) * 2 * ne;
#pragma unroll
  for (int k = 0; k < kGramAcc; ++k) {
    const int e = tid + k * nt;
    if (e < ne) {
      pm[e] = am[k];
      pm[ne + e] = aa[k];
    }
  }
}

// The same partial sums in double-float on the FP32 pipe.  Trial columns are
// padded to qp = TS ceil(q/TS) and taken in tiles of TS; thread (slot, phase)
// accumulates the TS x TS tile `slot` (tiles I <= J, J-major; blockIdx.z selects
// which 256/P tiles this block holds) of GM and GA over rows phase, phase + P, ...
// of each staged chunk, with Dot2 accumulators folded once per chunk.  The P
// phases of a tile sit in one warp and are combined by shuffles in a fixed order.
constexpr int kGdRows = 16;  // rows (nodes) per staged chunk
constexpr int kGdTile = 2;   // tile side: 2 x 2 entries of GM and GA per thread (80 registers, 3 CTAs per SM)

__device__ __forceinline__ void mac_conj(acc2& re, acc2& im, const dcx& a, const dcx& b) {
  // += conj(a) b
  dot2(re, a.x, b.x);
  dot2(re, a.y, b.y);
  dot2(im, a.x, b.y);
  dot2_neg(im, a.y, b.x);
}

// The four staged values (z_x, z_y, curl, w curl) of a node whose stencil reaches
// across the level's boundary (Bloch extension), written at out, out + stride,
// out + 2 stride, out + 3 stride.  Out of line: few nodes take it, and the common
// interior path keeps its registers.
__device__ __noinline__ void gram_stage_boundary(const double2* X, Lvl<df> L, WtsDF w, MassFactor mf,
                                                 const double* ph, int g, int i, int j, dcx* out, int stride) {
  const ERdD<df> rd{X, L.n, L.m, load_ph<df>(ph, g)};
  const dcx x0 = rd.x(i, j), x1 = rd.x(i, j + 1), y0 = rd.y(i, j), y1 = rd.y(i + 1, j);
  out[0] = mf.ax * x0 + mf.bx * x1;
  out[stride] = mf.ay * y0 + mf.by * y1;
  const dcx vc = x1 - x0 - y1 + y0;  // curl_at's order
  out[2 * stride] = vc;
  out[3 * stride] = w(i, j) * vc;
}

template <int P, int TS>
__global__ void __launch_bounds__(256, 3) k_gram_df(Lvl<df> L, WtsDF w, MassFactor mf, const double* ph, Roles roles,
                                                 int q, int qp, int lds, int rows, double2* __restrict__ part,
                                                 int npart) {
  extern __shared__ float4 smf[];
  dcx* zx = reinterpret_cast<dcx*>(smf);  // [rows][lds] each, columns qp .. lds-1 unused
  dcx* zy = zx + rows * lds;
  dcx* cc = zy + rows * lds;
  dcx* cw = cc + rows * lds;
  const int g = blockIdx.y;
  const int tid = threadIdx.x;
  const int T3 = qp / TS, ntile = T3 * (T3 + 1) / 2;
  const int slot = blockIdx.z * (256 / P) + tid / P, phase = tid % P;
  const bool active = slot < ntile;
  int I = 0, J = 0;
  if (active) {
    J = int((sqrtf(8.0f * slot + 1.0f) - 1.0f) * 0.5f);
    while ((J + 1) * (J + 2) / 2 <= slot) ++J;
    while (J * (J + 1) / 2 > slot) --J;
    I = slot - J * (J + 1) / 2;
  }
  const dcx z = dcx_make(df_zero(), df_zero());
  for (int t = tid; t < rows * (qp - q); t += blockDim.x) {
    const int e = (t / (qp - q)) * lds + q + t % (qp - q);
    zx[e] = z; zy[e] = z; cc[e] = z; cw[e] = z;
  }
  acc2 mre[TS * TS], mim[TS * TS], are[TS * TS], aim[TS * TS];
#pragma unroll
  for (int k = 0; k < TS * TS; ++k) {
    mre[k] = acc2_zero(); mim[k] = acc2_zero(); are[k] = acc2_zero(); aim[k] = acc2_zero();
  }
  const long N = (long)L.n * L.m;
  const long nchunks = (N + rows - 1) / rows;
  for (long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const long r0 = ch * rows;
    __syncthreads();
    for (int t = tid; t < q * rows; t += blockDim.x) {
      const int col = t / rows, rr = t % rows;
      const long node = r0 + rr;
      const int e = rr * lds + col;
      const int i = int(node % L.n), j = int(node / L.n);
      if (node < N && inside(i, j, L.n, L.m, 1, 1)) {
        // the stencil's reads stay inside the level: no Bloch extension
        const ERdDIn<df> rd{role_col(roles, g, col), L.n, N};
        const dcx x0 = rd.x(i, j), x1 = rd.x(i, j + 1), y0 = rd.y(i, j), y1 = rd.y(i + 1, j);
        zx[e] = mf.ax * x0 + mf.bx * x1;
        zy[e] = mf.ay * y0 + mf.by * y1;
        const dcx vc = x1 - x0 - y1 + y0;  // curl_at's order
        cc[e] = vc;
        cw[e] = w(i, j) * vc;
      } else if (node < N) {
        gram_stage_boundary(role_col(roles, g, col), L, w, mf, ph, g, i, j, zx + e, rows * lds);
      } else {
        zx[e] = z; zy[e] = z; cc[e] = z; cw[e] = z;
      }
    }
    __syncthreads();
    if (active) {
      // the M sums take two row streams per node (x and y edges), the A sums one
      // (curls); the streams of a matrix are consecutive rows of one loop
      for (int rr = phase; rr < rows; rr += P) {
        const int ra = rr * lds + TS * I, rb = rr * lds + TS * J;
#pragma unroll 1
        for (int st = 0; st < 2; ++st) {
          const dcx* A = st == 0 ? zx : zy;  // (B S)^* (B S): both sides from one array
          const dcx* B = A;
          dcx a[TS], b[TS];
#pragma unroll
          for (int k = 0; k < TS; ++k) { a[k] = A[ra + k]; b[k] = B[rb + k]; }
#pragma unroll
          for (int k = 0; k < TS; ++k)
#pragma unroll
            for (int l = 0; l < TS; ++l) mac_conj(mre[TS * k + l], mim[TS * k + l], a[k], b[l]);
        }
        dcx a[TS], b[TS];
#pragma unroll
        for (int k = 0; k < TS; ++k) { a[k] = cc[ra + k]; b[k] = cw[rb + k]; }
#pragma unroll
        for (int k = 0; k < TS; ++k)
#pragma unroll
          for (int l = 0; l < TS; ++l) mac_conj(are[TS * k + l], aim[TS * k + l], a[k], b[l]);
      }
#pragma unroll
      for (int k = 0; k < TS * TS; ++k) {
        dot2_fold(mre[k]); dot2_fold(mim[k]); dot2_fold(are[k]); dot2_fold(aim[k]);
      }
    }
  }
  const int ne = q * (q + 1) / 2;
  double2* pm = part + ((long)g * npart + blockIdx.x) * 2 * ne;
#pragma unroll
  for (int k = 0; k < TS * TS; ++k) {
    df v[4] = {acc2_df(mre[k]), acc2_df(mim[k]), acc2_df(are[k]), acc2_df(aim[k])};
#pragma unroll
    for (int o = 1; o < P; o <<= 1)
#pragma unroll
      for (int t = 0; t < 4; ++t) v[t] = v[t] + shfl_df(v[t], o);
    const int a = TS * I + k / TS, b = TS * J + k % TS;
    if (active && phase == 0 && a < q && b < q && a <= b) {
      const int e = b * (b + 1) / 2 + a;
      pm[e] = make_double2(df_to(v[0]), df_to(v[1]));
      pm[ne + e] = make_double2(df_to(v[2]), df_to(v[3]));
    }
  }
}

// sum partials in fixed order; write full Hermitian q x q (column-major) per group
__global__ void k_gram_finalize(const double2* __restrict__ part, int npart, int q, double2* __restrict__ GM,
                                double2* __restrict__ GA) {
  const int g = blockIdx.y;
  const int ne = q * (q + 1) / 2;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < 2 * ne; e += gridDim.x * blockDim.x) {
    double2 s = make_double2(0, 0);
    for (int pp = 0; pp < npart; ++pp) {
      const double2 v = part[((long)g * npart + pp) * 2 * ne + e];
      s.x += v.x;
      s.y += v.y;
    }
    const int ee = e < ne ? e : e - ne;
    double2* G = (e < ne ? GM : GA) + (long)g * q * q;
    int bi = int((sqrt(8.0 * ee + 1.0) - 1.0) * 0.5);
    while ((bi + 1) * (bi + 2) / 2 <= ee) ++bi;
    while (bi * (bi + 1) / 2 > ee) --bi;
    const int ai = ee - bi * (bi + 1) / 2;
    if (ai == bi) s.y = 0.0;
    G[ai + (long)bi * q] = s;
    G[bi + (long)ai * q] = conj(s);
  }
}

// ---- small dense Rayleigh-Ritz (one block) -------------------------------
// Given the Gram matrices GM = S^* M S and GA = S^* A S of a trial block S
// (q columns), find the p smallest Ritz pairs (Section 4, eq. ritz_eigenvalue):
//  1. scale to unit diagonal (FP64), Cholesky GM = R^* R dropping directions
//     whose pivot falls below kDropTol (a span that lost rank);
//  2. T = R^{-1} by Gauss-Jordan elimination, H = T^* GA T;
//  3. Householder reduction H = Q Tr Q^*, Tr Hermitian tridiagonal, made real
//     by a diagonal unitary scaling;
//  4. the p smallest eigenvalues of Tr by multisection on Sturm counts, their
//     eigenvectors by inverse iteration (re-orthogonalised inside clusters);
//  5. back-transformation and C = D T Q U.
// Steps 2-5 run in the arithmetic R: FP64 under the plain policy, double-float
// (about 48 bits, FP32 pipe) under the mixed one, where the coefficients only need
// ~1e-14 accuracy (Ritz values and residuals are recomputed in FP64 from the
// updated block) and a serial chain of FP64 instructions is what limited this
// one-block kernel on GB300.
constexpr double kDropTol = 1e-12;  // relative pivot below which a trial direction is dropped
constexpr int kRRThreads = 512;
constexpr int kRRWarps = kRRThreads / 32;

// Arithmetic of the small dense solve: R = df (double-float on the FP32 pipe,
// the mixed policy) or double (plain FP64).  Ar<R> names the operations the
// kernel needs on reals and on complex values C of that precision.
// (operators as hidden friends, found by argument-dependent lookup only, so they
// do not hide the namespace's operators on double2 and the double-float types)
struct cd {
  double re, im;
  friend __device__ __forceinline__ cd operator+(cd a, cd b) { return cd{a.re + b.re, a.im + b.im}; }
  friend __device__ __forceinline__ cd operator-(cd a, cd b) { return cd{a.re - b.re, a.im - b.im}; }
  friend __device__ __forceinline__ cd operator-(cd a) { return cd{-a.re, -a.im}; }
  friend __device__ __forceinline__ cd operator*(cd a, cd b) {
    return cd{a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
  }
};

template <class R> struct Ar;
template <> struct Ar<df> {
  using C = cdf;
  using lead_t = float;  // leading part: comparisons, magnitudes and pivot limits
  static __device__ __forceinline__ df mk(float v) { return df_make(v, 0.0f); }
  static __device__ __forceinline__ df zero() { return df_zero(); }
  static __device__ __forceinline__ float lead(df a) { return a.hi; }
  static __device__ __forceinline__ double to(df a) { return df_to(a); }
  static __device__ __forceinline__ df sqrt(df a) { return df_sqrt(a); }
  static __device__ __forceinline__ bool lt(df a, df b) { return df_lt(a, b); }
  static __device__ __forceinline__ df mulf(df a, float b) { return df_mul_f(a, b); }
  static __device__ __forceinline__ df xshfl(df v, int o) { return shfl_df(v, o); }
  static __device__ __forceinline__ df ishfl(df v, int src) {
    return df_make(__shfl_sync(0xffffffffu, v.hi, src), __shfl_sync(0xffffffffu, v.lo, src));
  }
  static __device__ __forceinline__ C cmk(df r, df i) { return cdf_make(r, i); }
  static __device__ __forceinline__ C czero() { return cdf_zero(); }
  static __device__ __forceinline__ C cfrom(double2 v) { return cdf_from(v); }
  static __device__ __forceinline__ double2 cto(C z) { return cdf_to(z); }
  static __device__ __forceinline__ C conj(C a) { return cdf_conj(a); }
  static __device__ __forceinline__ C mulc(C a, C b) { return cdf_mulc(a, b); }
  static __device__ __forceinline__ C scale(C a, df s) { return cdf_scale(a, s); }
  static __device__ __forceinline__ df norm2(C a) { return cdf_norm2(a); }
};
template <> struct Ar<double> {
  using C = cd;
  using lead_t = double;
  static __device__ __forceinline__ double mk(double v) { return v; }
  static __device__ __forceinline__ double zero() { return 0.0; }
  static __device__ __forceinline__ double lead(double a) { return a; }
  static __device__ __forceinline__ double to(double a) { return a; }
  static __device__ __forceinline__ double sqrt(double a) { return a > 0.0 ? ::sqrt(a) : 0.0; }
  static __device__ __forceinline__ bool lt(double a, double b) { return a < b; }
  static __device__ __forceinline__ double mulf(double a, float b) { return a * (double)b; }
  static __device__ __forceinline__ double xshfl(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
  static __device__ __forceinline__ double ishfl(double v, int src) { return __shfl_sync(0xffffffffu, v, src); }
  static __device__ __forceinline__ C cmk(double r, double i) { return cd{r, i}; }
  static __device__ __forceinline__ C czero() { return cd{0.0, 0.0}; }
  static __device__ __forceinline__ C cfrom(double2 v) { return cd{v.x, v.y}; }
  static __device__ __forceinline__ double2 cto(C z) { return make_double2(z.re, z.im); }
  static __device__ __forceinline__ C conj(C a) { return cd{a.re, -a.im}; }
  static __device__ __forceinline__ C mulc(C a, C b) { return cd{a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re}; }
  static __device__ __forceinline__ C scale(C a, double s) { return cd{a.re * s, a.im * s}; }
  static __device__ __forceinline__ double norm2(C a) { return a.re * a.re + a.im * a.im; }
};

template <class R> __device__ __forceinline__ R warp_sum_r(R v) {
  for (int o = 16; o > 0; o >>= 1) v = v + Ar<R>::xshfl(v, o);
  return v;
}
template <class R> __device__ __forceinline__ typename Ar<R>::C warp_sum_c(typename Ar<R>::C v) {
  for (int o = 16; o > 0; o >>= 1) v = v + Ar<R>::cmk(Ar<R>::xshfl(v.re, o), Ar<R>::xshfl(v.im, o));
  return v;
}
// block-wide sum (all threads participate; result in every thread)
template <class R> __device__ __forceinline__ R block_sum_r(R v, R* red) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  v = warp_sum_r<R>(v);
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  R t = Ar<R>::zero();
  for (int w = 0; w < kRRWarps; ++w) t = t + red[w];
  return t;
}

// number of eigenvalues of the real symmetric tridiagonal (a, e^2) below x
template <class R, class P> __device__ int sturm_count_r(const R* a, const R* e2, int n, R x, P pivmin) {
  using A = Ar<R>;
  int cnt = 0;
  R d = a[0] - x;
  if (fabs(A::lead(d)) < pivmin) d = A::mk(-pivmin);
  if (A::lead(d) < 0) ++cnt;
  for (int i = 1; i < n; ++i) {
    d = (a[i] - x) - e2[i - 1] / d;
    if (fabs(A::lead(d)) < pivmin) d = A::mk(-pivmin);
    if (A::lead(d) < 0) ++cnt;
  }
  return cnt;
}

template <class R>
__global__ void __launch_bounds__(kRRThreads) k_small_rr(const double2* __restrict__ GM, const double2* __restrict__ GA,
                                                         int q, int p, double2* __restrict__ Cout,
                                                         double* __restrict__ theta_out, double2* __restrict__ scr,
                                                         int* __restrict__ info, int in_smem, int* __restrict__ phase_out,
                                                         long scr_stride) {
  using A = Ar<R>;
  using C = typename A::C;
  using LT = typename A::lead_t;
  extern __shared__ double2 dsm[];
  {  // group blockIdx.x: its own Gram matrices, outputs and scratch
    const long g = blockIdx.x;
    GM += g * q * q;
    GA += g * q * q;
    Cout += g * q * p;
    theta_out += g * p;
    scr += g * scr_stride;
    info += 8 * g;
    if (phase_out) phase_out += 8 * g;
  }
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nw = kRRWarps;
  const long qq = (long)q * q;
  C* G = (C*)(in_smem ? dsm : scr);  // M-Gram -> R -> Y
  C* H = G + qq;                        // A-Gram -> H -> reflectors
  C* T = H + qq;                        // R^{-1}
  C* U = T + qq;                        // q x p eigenvectors
  __shared__ double d[kMaxTrial];         // column scales (FP64)
  __shared__ int s_keep[kMaxTrial];
  __shared__ R ta[kMaxTrial], te[kMaxTrial], te2[kMaxTrial], tbeta[kMaxTrial];
  __shared__ C talpha[kMaxTrial], tphase[kMaxTrial], tvec[kMaxTrial], tp[kMaxTrial];
  __shared__ R lam[kMaxBlock], lo_s[kMaxBlock], hi_s[kMaxBlock];
  __shared__ R Z[kMaxTrial * kMaxBlock];  // real eigenvectors of the tridiagonal, column j at j*q
  __shared__ int s_r, s_bad, s_cnt[kRRThreads];
  __shared__ R s_piv, s_red[kRRWarps];
  long long t_phase[8];
  t_phase[0] = clock64();

  // 1. scaling (FP64) and conversion
  for (int i = tid; i < q; i += nt) {
    const double g = GM[(long)i * q + i].x;
    d[i] = (g > 0.0 && isfinite(g)) ? 1.0 / sqrt(g) : 0.0;
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (long t = tid; t < qq; t += nt) {
    const int i = int(t % q), j = int(t / q);
    const double sc = d[i] * d[j];
    const double2 gm = GM[t], ga = GA[t];
    if (!isfinite(gm.x) || !isfinite(gm.y) || !isfinite(ga.x) || !isfinite(ga.y)) s_bad = 1;
    G[t] = A::cfrom(sc * gm);
    H[t] = A::cfrom(sc * ga);
    T[t] = A::czero();
  }
  __syncthreads();
  // Cholesky with dropping: R row k stored in G[j*q + k] (j >= k).  A dropped
  // direction becomes a decoupled unit row and column of R and an isolated Ritz
  // value above every kept one.
  for (int k = 0; k < q; ++k) {
    if (tid == 0) {
      const R pv = G[(long)k * q + k].re;
      const bool keep = d[k] > 0.0 && A::to(pv) > kDropTol && isfinite(A::lead(pv));
      s_keep[k] = keep;
      s_piv = keep ? A::mk(1.0f) / A::sqrt(pv) : A::zero();  // 1 / R_kk
    }
    __syncthreads();
    const R inv = s_piv;
    if (A::lead(inv) > 0.0f) {
      for (int j = k + tid; j < q; j += nt) G[(long)j * q + k] = A::scale(G[(long)j * q + k], inv);
      __syncthreads();
      const int rem = q - k - 1;
      for (long t = tid; t < (long)rem * rem; t += nt) {
        const int ii = k + 1 + int(t % rem), jj = k + 1 + int(t / rem);
        if (ii > jj) continue;
        G[(long)jj * q + ii] = G[(long)jj * q + ii] - A::mulc(G[(long)ii * q + k], G[(long)jj * q + k]);
      }
    } else {
      for (int j = tid; j < q; j += nt) {
        G[(long)j * q + k] = A::cmk(A::mk(j == k ? 1.0f : 0.0f), A::zero());
        if (j < k) G[(long)k * q + j] = A::czero();
        H[(long)j * q + k] = A::czero();
        H[(long)k * q + j] = A::czero();
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    int r = 0;
    for (int k = 0; k < q; ++k) r += s_keep[k];
    s_r = r;
  }
  __syncthreads();
  if (s_r < p || s_bad) {
    if (tid == 0) {
      info[0] = s_bad ? -2 : -1;
      info[1] = s_r;
    }
    return;
  }
  const int r = q;
  t_phase[1] = clock64();
  // 2a. T = R^{-1}, column c solving R t = e_c by back substitution, one warp per
  //     column: lanes hold the right-hand side rows; at step k the owner of row k
  //     divides by R[k][k], broadcasts t_k, and every lane removes R[m][k] t_k from
  //     its rows m < k (R[m][k] = G[k q + m]).  Rows above c of T stay zero.
  {
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int kSlots = (kMaxTrial + 31) / 32;
    for (int c = warp; c < r; c += kRRWarps) {
      C bv[kSlots];
#pragma unroll
      for (int sl = 0; sl < kSlots; ++sl)
        bv[sl] = A::cmk(A::mk(lane + 32 * sl == c ? 1.0f : 0.0f), A::zero());
      for (int k = c; k >= 0; --k) {
        const int owner = k & 31, slot = k >> 5;
        C xk = A::czero();
#pragma unroll
        for (int sl = 0; sl < kSlots; ++sl)
          if (sl == slot && lane == owner) {
            const R rkk = G[(long)k * q + k].re;
            xk = A::cmk(bv[sl].re / rkk, bv[sl].im / rkk);
            T[(long)c * q + k] = xk;
          }
        xk = A::cmk(A::ishfl(xk.re, owner), A::ishfl(xk.im, owner));
#pragma unroll
        for (int sl = 0; sl < kSlots; ++sl) {
          const int m = lane + 32 * sl;
          if (m < k) bv[sl] = bv[sl] - G[(long)k * q + m] * xk;
        }
      }
    }
  }
  __syncthreads();
  // 2b. Y = A T into G (R is no longer needed), then H = T^* Y
  for (long t = tid; t < (long)r * r; t += nt) {
    const int i = int(t % r), c = int(t / r);
    C acc = A::czero();
    for (int m = 0; m <= c; ++m) acc = acc + H[(long)m * q + i] * T[(long)c * q + m];
    G[(long)c * q + i] = acc;
  }
  __syncthreads();
  for (long t = tid; t < (long)r * r; t += nt) {
    const int i = int(t % r), c = int(t / r);
    C acc = A::czero();
    for (int m = 0; m <= i; ++m) acc = acc + A::mulc(T[(long)i * q + m], G[(long)c * q + m]);
    H[(long)c * q + i] = acc;
  }
  __syncthreads();
  // exact Hermitian symmetry, and an isolated value for dropped directions
  for (long t = tid; t < (long)r * r; t += nt) {
    const int i = int(t % r), c = int(t / r);
    if (i < c) {
      const C up = H[(long)c * q + i], lo = H[(long)i * q + c];
      const R half = A::mk(0.5f);
      const C m = A::cmk((up.re + lo.re) * half, (up.im - lo.im) * half);
      H[(long)c * q + i] = m;
      H[(long)i * q + c] = A::conj(m);
    } else if (i == c) {
      H[(long)c * q + i].im = A::zero();
    }
  }
  __syncthreads();
  // Gershgorin row sums of the kept rows (in te, which the reduction below fills
  // before it is used again), then the bound by one thread
  for (int i = tid; i < r; i += nt) {
    R rs = A::zero();
    if (s_keep[i])
      for (int j = 0; j < r; ++j) rs = rs + A::sqrt(A::norm2(H[(long)j * q + i]));
    te[i] = rs;
  }
  __syncthreads();
  if (tid == 0) {
    R bound = A::zero();
    for (int i = 0; i < r; ++i)
      if (A::lt(bound, te[i])) bound = te[i];
    for (int i = 0; i < r; ++i)
      if (!s_keep[i]) H[(long)i * q + i] = A::cmk(bound + bound + A::mk(1.0f), A::zero());
  }
  __syncthreads();
  t_phase[2] = clock64();
  // 3. Householder tridiagonalisation; reflector k acts on rows/cols k+1..r-1 and is
  //    stored in column k below the diagonal (v, with v_0 = x_0 - alpha) and tbeta[k]
  for (int k = 0; k + 2 < r; ++k) {
    const int m = r - k - 1;
    R s2 = A::zero();
    for (int i = tid; i < m; i += nt) s2 = s2 + A::norm2(H[(long)k * q + k + 1 + i]);
    s2 = block_sum_r<R>(s2, s_red);
    if (tid == 0) {
      const R sigma = A::sqrt(s2);
      const C x0 = H[(long)k * q + k + 1];
      const R ax0 = A::sqrt(A::norm2(x0));
      C ph = A::lead(ax0) > 0.0f ? A::cmk(x0.re / ax0, x0.im / ax0) : A::cmk(A::mk(1.0f), A::zero());
      if (A::lead(sigma) > 0.0f) {
        const C alpha = -A::scale(ph, sigma);
        talpha[k] = alpha;
        tbeta[k] = A::mk(1.0f) / (sigma * (sigma + ax0));
        H[(long)k * q + k + 1] = x0 - alpha;
      } else {
        talpha[k] = x0;
        tbeta[k] = A::zero();
      }
    }
    __syncthreads();
    const R beta = tbeta[k];
    if (A::lead(beta) != 0.0f) {
      // p = beta * Hsub v (rows by warps, columns by lanes)
      for (int i = warp; i < m; i += nw) {
        C acc = A::czero();
        for (int j = lane; j < m; j += 32) acc = acc + H[(long)(k + 1 + j) * q + k + 1 + i] * H[(long)k * q + k + 1 + j];
        acc = warp_sum_c<R>(acc);
        if (lane == 0) tp[i] = A::scale(acc, beta);
      }
      __syncthreads();
      // K = beta/2 v^* p (real for Hermitian H); w = p - K v
      R kk = A::zero();
      for (int i = tid; i < m; i += nt) kk = kk + A::mulc(H[(long)k * q + k + 1 + i], tp[i]).re;
      kk = block_sum_r<R>(kk, s_red);
      const R K = kk * beta * A::mk(0.5f);
      for (int i = tid; i < m; i += nt) tvec[i] = tp[i] - A::scale(H[(long)k * q + k + 1 + i], K);
      __syncthreads();
      // Hsub -= v w^* + w v^*
      for (long t = tid; t < (long)m * m; t += nt) {
        const int i = int(t % m), j = int(t / m);
        const C vi = H[(long)k * q + k + 1 + i], vj = H[(long)k * q + k + 1 + j];
        C h = H[(long)(k + 1 + j) * q + k + 1 + i];
        h = h - vi * A::conj(tvec[j]) - tvec[i] * A::conj(vj);
        H[(long)(k + 1 + j) * q + k + 1 + i] = h;
      }
    }
    __syncthreads();
  }
  // real tridiagonal: diagonal ta, off-diagonal te = |alpha|, phases tphase
  if (tid == 0) {
    C ph = A::cmk(A::mk(1.0f), A::zero());
    for (int k = 0; k < r; ++k) {
      ta[k] = H[(long)k * q + k].re;
      tphase[k] = ph;
      if (k + 1 < r) {
        const C al = (k + 2 < r) ? talpha[k] : H[(long)k * q + k + 1];
        const R aa = A::sqrt(A::norm2(al));
        te[k] = aa;
        te2[k] = aa * aa;
        if (A::lead(aa) > 0.0f) ph = ph * A::cmk(al.re / aa, al.im / aa);
      }
    }
  }
  __syncthreads();
  t_phase[3] = clock64();
  // 4a. multisection: each warp refines one wanted eigenvalue at a time, its 32
  //     lanes evaluating the Sturm count at 32 interior points of the bracket
  R lo = A::zero(), hi = A::zero();
  for (int k = 0; k < r; ++k) {
    const R rad = (k > 0 ? te[k - 1] : A::zero()) + (k + 1 < r ? te[k] : A::zero());
    const R l = ta[k] - rad, h = ta[k] + rad;
    if (k == 0 || A::lt(l, lo)) lo = l;
    if (k == 0 || A::lt(hi, h)) hi = h;
  }
  const LT tnorm = fmax(fabs(A::lead(lo)), fabs(A::lead(hi))) + LT(1e-30);
  // Sturm pivots below pivmin are replaced by -pivmin: e^2 / pivmin stays far below the float range
  const LT pivmin = fmax(LT(1e-30) * tnorm * tnorm, LT(1e-36));
  // inverse iteration: pivots are kept above the accuracy of the shift, so a solve
  // grows the vector by at most ~1e14 and never leaves the float range
  const LT pivmin_ii = LT(1e-14) * tnorm;
  for (int j = warp; j < p; j += nw) {
    R a0 = lo - A::mk(1e-6f * tnorm), b0 = hi + A::mk(1e-6f * tnorm);
    for (int it = 0; it < 24; ++it) {
      const R w = b0 - a0;
      if (A::to(w) <= 4e-15 * (double)tnorm) break;
      const R x = a0 + A::mulf(w, float(lane + 1) / 33.0f);
      const int cnt = sturm_count_r<R>(ta, te2, r, x, pivmin);
      // new bracket: largest point with count <= j, smallest with count > j
      const unsigned below = __ballot_sync(0xffffffffu, cnt <= j);
      const int nb = __popc(below);  // points 0..nb-1 have count <= j (counts increase with x)
      const R xa = A::ishfl(x, nb > 0 ? nb - 1 : 0);
      const R xb = A::ishfl(x, nb < 32 ? nb : 31);
      if (nb > 0) a0 = xa;
      if (nb < 32) b0 = xb;
    }
    if (lane == 0) {
      lam[j] = (a0 + b0) * A::mk(0.5f);
      lo_s[j] = a0;
      hi_s[j] = b0;
    }
  }
  __syncthreads();
  t_phase[4] = clock64();
  // 4b. inverse iteration on Tr - lam_j I (Gaussian elimination with partial
  //     pivoting, factored once), one thread per eigenvalue; cluster members
  //     re-orthogonalised after every sweep
  R u0[kMaxTrial], u1[kMaxTrial], u2[kMaxTrial], mult[kMaxTrial];
  bool swp[kMaxTrial];
  if (tid < p) {
    const R shift = lam[tid];
    R d0 = ta[0] - shift, s1 = r > 1 ? te[0] : A::zero();
    for (int i = 0; i < r; ++i) {
      const R below_sub = i + 1 < r ? te[i] : A::zero();
      const R below_diag = i + 1 < r ? ta[i + 1] - shift : A::zero();
      const R below_sup = i + 2 < r ? te[i + 1] : A::zero();
      if (i + 1 < r && fabs(A::lead(below_sub)) > fabs(A::lead(d0))) {
        swp[i] = true;
        u0[i] = below_sub;
        u1[i] = below_diag;
        u2[i] = below_sup;
        const R mlt = d0 / below_sub;
        mult[i] = mlt;
        d0 = s1 - mlt * below_diag;
        s1 = -(mlt * below_sup);
      } else {
        swp[i] = false;
        R dd = d0;
        if (fabs(A::lead(dd)) < pivmin_ii) dd = A::mk(A::lead(dd) < 0.0f ? -pivmin_ii : pivmin_ii);
        u0[i] = dd;
        u1[i] = s1;
        u2[i] = A::zero();
        const R mlt = i + 1 < r ? below_sub / dd : A::zero();
        mult[i] = mlt;
        d0 = below_diag - mlt * s1;
        s1 = below_sup;
      }
    }
  }
  for (int sweep = 0; sweep < 4; ++sweep) {
    if (tid < p) {
      const int j = tid;
      R* z = Z + j * q;
      if (sweep == 0)
        for (int i = 0; i < r; ++i) z[i] = A::mk(1.0f + 0.37f * __sinf(1.7f * (i + 1) * (j + 1)));
      for (int i = 0; i + 1 < r; ++i) {
        if (swp[i]) {
          const R t0 = z[i];
          z[i] = z[i + 1];
          z[i + 1] = t0 - mult[i] * z[i];
        } else {
          z[i + 1] = z[i + 1] - mult[i] * z[i];
        }
      }
      for (int i = r - 1; i >= 0; --i) {
        R v = z[i];
        if (i + 1 < r) v = v - u1[i] * z[i + 1];
        if (i + 2 < r) v = v - u2[i] * z[i + 2];
        R dd = u0[i];
        if (fabs(A::lead(dd)) < pivmin_ii) dd = A::mk(A::lead(dd) < 0.0f ? -pivmin_ii : pivmin_ii);
        z[i] = v / dd;
      }
      LT zmax = 0;
      for (int i = 0; i < r; ++i) zmax = fmax(zmax, fabs(A::lead(z[i])));
      const float sc = zmax > 0 ? float(1.0 / zmax) : 1.0f;
      R nrm = A::zero();
      for (int i = 0; i < r; ++i) {
        z[i] = A::mulf(z[i], sc);
        nrm = nrm + z[i] * z[i];
      }
      const R inv = A::mk(1.0f) / A::sqrt(nrm);
      for (int i = 0; i < r; ++i) z[i] = z[i] * inv;
    }
    __syncthreads();
    // modified Gram-Schmidt against earlier vectors whose eigenvalues lie within
    // 1e-3 |T| (the usual reorthogonalisation window of inverse iteration);
    // warp 0, lanes over the components
    if (warp == 0) {
      for (int j = 1; j < p; ++j) {
        R* zj = Z + j * q;
        bool touched = false;
        for (int c = 0; c < j; ++c) {
          if (A::to(lam[j] - lam[c]) > 1e-3 * (double)tnorm) continue;
          const R* zc = Z + c * q;
          R dot = A::zero();
          for (int i = lane; i < r; i += 32) dot = dot + zc[i] * zj[i];
          dot = warp_sum_r<R>(dot);
          for (int i = lane; i < r; i += 32) zj[i] = zj[i] - dot * zc[i];
          __syncwarp();
          touched = true;
        }
        if (touched) {
          R nrm = A::zero();
          for (int i = lane; i < r; i += 32) nrm = nrm + zj[i] * zj[i];
          nrm = warp_sum_r<R>(nrm);
          const R inv = A::mk(1.0f) / A::sqrt(nrm);
          for (int i = lane; i < r; i += 32) zj[i] = zj[i] * inv;
          __syncwarp();
        }
      }
    }
    __syncthreads();
  }
  t_phase[5] = clock64();
  // 5. back-transformation u_j = Q (phase * z_j), then C = D T u (one warp per vector)
  for (int j = warp; j < p; j += nw) {
    C* u = U + (long)j * q;
    for (int i = lane; i < r; i += 32) u[i] = A::scale(tphase[i], Z[j * q + i]);
    __syncwarp();
    for (int k = r - 3; k >= 0; --k) {
      const R beta = tbeta[k];
      if (A::lead(beta) == 0.0f) continue;
      const int m = r - k - 1;
      C acc = A::czero();
      for (int i = lane; i < m; i += 32) acc = acc + A::mulc(H[(long)k * q + k + 1 + i], u[k + 1 + i]);
      acc = warp_sum_c<R>(acc);
      const C f = A::scale(acc, beta);
      for (int i = lane; i < m; i += 32) u[k + 1 + i] = u[k + 1 + i] - H[(long)k * q + k + 1 + i] * f;
      __syncwarp();
    }
    for (int i = lane; i < q; i += 32) {
      C acc = A::czero();
      for (int m = i; m < r; ++m) acc = acc + T[(long)m * q + i] * u[m];
      Cout[(long)j * q + i] = s_keep[i] ? d[i] * A::cto(acc) : make_double2(0, 0);
    }
  }
  for (int j = tid; j < p; j += nt) theta_out[j] = A::to(lam[j]);
  __syncthreads();
  // a non-finite coefficient means a breakdown: report it instead of passing it on
  int bad = 0;
  for (long t = tid; t < (long)q * p; t += nt) {
    const double2 c = Cout[t];
    bad |= !(isfinite(c.x) && isfinite(c.y));
  }
  for (int j = tid; j < p; j += nt) bad |= !isfinite(theta_out[j]);
  bad = __syncthreads_or(bad);
  t_phase[6] = clock64();
  if (tid == 0) {
    info[0] = bad ? -3 : 0;
    info[1] = s_r;
    if (phase_out)
      for (int ph = 0; ph < 6; ++ph) phase_out[ph] = (int)((t_phase[ph + 1] - t_phase[ph]) / 1000);
  }
}

// Y[:, j] = sum_i X[:, i] C[i, j] (+ Z[:, j]) for group blockIdx.y: trial column i
// of the group at role_col(X, g, i); output column j at Y + (g p + j) ldy;
// C of group g at C + g cgs (column-major, leading dimension ldc).  PB >= p
// accumulators per thread: the smallest instance that holds p keeps the register
// count (and so the number of resident warps) down.
template <int PB>
__global__ void __launch_bounds__(256, PB <= 12 ? 3 : 1)
    k_block_update(Roles X, int q, const double2* __restrict__ C, int ldc, long cgs, double2* __restrict__ Y, long ldy,
                   int p, const double2* __restrict__ Z, long ldz, long rows) {
  extern __shared__ double2 cs[];  // [p][q]
  const int g = blockIdx.y;
  const double2* Cg = C + g * cgs;
  for (int t = threadIdx.x; t < p * q; t += blockDim.x) cs[t] = Cg[(long)(t / q) * ldc + (t % q)];
  __syncthreads();
  double2* Yg = Y + (long)g * p * ldy;
  const double2* Zg = Z ? Z + (long)g * p * ldz : nullptr;
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < rows; r += (long)gridDim.x * blockDim.x) {
    double2 acc[PB];
#pragma unroll
    for (int j = 0; j < PB; ++j) acc[j] = make_double2(0, 0);
    for (int i = 0; i < q; ++i) {
      const double2 x = role_col(X, g, i)[r];
#pragma unroll
      for (int j = 0; j < PB; ++j) {
        if (j < p) {
          const double2 c = cs[j * q + i];
          acc[j].x = fma(x.x, c.x, fma(-x.y, c.y, acc[j].x));
          acc[j].y = fma(x.x, c.y, fma(x.y, c.x, acc[j].y));
        }
      }
    }
#pragma unroll
    for (int j = 0; j < PB; ++j) {
      if (j < p) {
        double2 v = acc[j];
        if (Zg) v = v + Zg[(long)j * ldz + r];
        Yg[(long)j * ldy + r] = v;
      }
    }
  }
}

// The same product in double-float (compensated Dot2 sums, folded every 8 trial
// columns; PB >= p accumulator pairs per thread).  Used for the search direction
// P = [P, W] C only: its rounding, 2^-47 |P|, reaches the iterate through
// E C + P, where it is 2^-47 |P| / |E| relative, far below the FP64 rounding of
// E C once the steps have become small.
template <int PB>
__global__ void __launch_bounds__(256, PB <= 12 ? 3 : 1)
    k_block_update_df(Roles X, int q, const double2* __restrict__ C, int ldc, long cgs, double2* __restrict__ Y,
                      long ldy, int p, const double2* __restrict__ Z, long ldz, long rows) {
  extern __shared__ float4 csf[];
  dcx* cs = reinterpret_cast<dcx*>(csf);  // [p][q]
  const int g = blockIdx.y;
  const double2* Cg = C + g * cgs;
  for (int t = threadIdx.x; t < p * q; t += blockDim.x) cs[t] = dcx_split(Cg[(long)(t / q) * ldc + (t % q)]);
  __syncthreads();
  double2* Yg = Y + (long)g * p * ldy;
  const double2* Zg = Z ? Z + (long)g * p * ldz : nullptr;
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < rows; r += (long)gridDim.x * blockDim.x) {
    acc2 re[PB], im[PB];
#pragma unroll
    for (int j = 0; j < PB; ++j) {
      re[j] = acc2_zero();
      im[j] = acc2_zero();
    }
    for (int i = 0; i < q; ++i) {
      const dcx x = dcx_split(role_col(X, g, i)[r]);
#pragma unroll
      for (int j = 0; j < PB; ++j) {
        if (j < p) {
          const dcx c = cs[j * q + i];
          dot2(re[j], x.x, c.x);
          dot2_neg(re[j], x.y, c.y);
          dot2(im[j], x.x, c.y);
          dot2(im[j], x.y, c.x);
        }
      }
      if ((i & 7) == 7) {
#pragma unroll
        for (int j = 0; j < PB; ++j) {
          dot2_fold(re[j]);
          dot2_fold(im[j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < PB; ++j) {
      if (j < p) {
        dcx v = dcx_make(acc2_df(re[j]), acc2_df(im[j]));
        if (Zg) v = v + dcx_split(Zg[(long)j * ldz + r]);
        Yg[(long)j * ldy + r] = dcx_to(v);
      }
    }
  }
}

__device__ __forceinline__ uint64_t mix64(uint64_t z) {
  z += 0x9e3779b97f4a7c15ull;
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}

__global__ void k_random(double2* X, long ld, long rows, uint64_t seed) {
  const int c = blockIdx.y;
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < rows; r += (long)gridDim.x * blockDim.x) {
    const uint64_t h1 = mix64(seed ^ mix64((uint64_t)c * 0x100000001b3ull + (uint64_t)r));
    const uint64_t h2 = mix64(h1);
    const double u1 = ((h1 >> 11) + 1) * (1.0 / 9007199254740993.0);
    const double u2 = (h2 >> 11) * (1.0 / 9007199254740992.0);
    const double rad = sqrt(-2.0 * log(u1));
    double sn, cs;
    sincospi(2.0 * u2, &sn, &cs);
    X[c * ld + r] = make_double2(rad * cs, rad * sn);
  }
}

__global__ void k_scale_cols(double2* X, long ld, long rows, const double* __restrict__ sc) {
  const int c = blockIdx.y;
  const double s = sc[c];
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < rows; r += (long)gridDim.x * blockDim.x)
    X[c * ld + r] = s * X[c * ld + r];
}

inline unsigned blocks_for(long n, int per = 256, unsigned cap = 4096) {
  long b = (n + per - 1) / per;
  if (b < 1) b = 1;
  return (unsigned)(b > cap ? cap : b);
}

}  // namespace

void convert_d2f(const double2* X, float2* Y, long n, cudaStream_t s) {
  if (n <= 0) return;
  timer_begin(KC_CONVERT, s, 24.0 * n);
  k_d2f<<<blocks_for(n), 256, 0, s>>>(X, Y, n);
  timer_end(KC_CONVERT, s);
  PBS_LAUNCHED();
}
void convert_f2d(const float2* X, double2* Y, long n, cudaStream_t s) {
  if (n <= 0) return;
  timer_begin(KC_CONVERT, s, 24.0 * n);
  k_f2d<<<blocks_for(n), 256, 0, s>>>(X, Y, n);
  timer_end(KC_CONVERT, s);
  PBS_LAUNCHED();
}

template <class T>
void sub_lift(const Level& L, const double* d_ph, int cpg, const cx<T>* Phi, long ldp, double2* X, long ldx, int ncols,
              cudaStream_t s) {
  if (ncols <= 0) return;
  // read phi, read and write x
  timer_begin(KC_SUB_LIFT, s, (sizeof(cx<T>) * (double)L.N() + 32.0 * L.D()) * ncols);
  k_sub_lift<T><<<grid2(L.n, L.m, ncols), dim3(kBX, kBY), 0, s>>>(L.n, L.m, d_ph, cpg, Phi, ldp, X, ldx);
  timer_end(KC_SUB_LIFT, s);
  PBS_LAUNCHED();
}

template <class T>
void lift_adj_mass(const Level& L, const double* d_ph, int cpg, const double2* X, long ldx, cx<T>* Rhs, long ldr,
                   int ncols, bool dfa, cudaStream_t s) {
  if (ncols <= 0) return;
  timer_begin(KC_LIFT_ADJ_MASK, s, (16.0 * L.D() + 2.0 * sizeof(T) * L.N()) * ncols);
  const dim3 g = grid2(L.n, L.m, ncols);
  if (dfa) {
    k_lift_adj_mass<df, T><<<g, dim3(kBX, kBY), 0, s>>>(L.lvl<df>(), d_ph, cpg, X, ldx, Rhs, ldr);
    count_df_launch();
  } else
    k_lift_adj_mass<double, T><<<g, dim3(kBX, kBY), 0, s>>>(L.lvl<double>(), d_ph, cpg, X, ldx, Rhs, ldr);
  timer_end(KC_LIFT_ADJ_MASK, s);
  PBS_LAUNCHED();
}

void deflate_constants(const Level& L, double2* X, long ld, int ncols, const int* d_gamma, int cpg,
                       double* d_partials, cudaStream_t s) {
  if (ncols <= 0) return;
  const int nblk = 64;
  k_edge_sums<<<dim3(nblk, ncols), 256, 0, s>>>(L.N(), X, ld, d_partials, nblk, d_gamma, cpg);
  PBS_LAUNCHED();
  k_edge_sub_means<<<dim3(nblk, ncols), 256, 0, s>>>(L.N(), X, ld, d_partials, nblk, d_gamma, cpg);
  PBS_LAUNCHED();
}

void rayleigh_parts(const Level& L, const double* d_ph, int cpg, const double2* X, long ld, int ncols,
                    double* d_partials, double* d_out, bool dfa, cudaStream_t s) {
  if (ncols <= 0) return;
  const dim3 g = grid2(L.n, L.m, ncols);
  if (dfa) {
    k_rayleigh_parts<df><<<g, dim3(kBX, kBY), 0, s>>>(L.lvl<df>(), L.wts_df(), mass_factor(L), d_ph, cpg, X, ld,
                                                     d_partials);
    count_df_launch();
  } else
    k_rayleigh_parts<double><<<g, dim3(kBX, kBY), 0, s>>>(L.lvl<double>(), L.wts<double>(), mass_factor(L), d_ph,
                                                         cpg, X, ld, d_partials);
  PBS_LAUNCHED();
  k_finalize2<<<ncols, 256, 0, s>>>(d_partials, g.x * g.y, d_out);
  PBS_LAUNCHED();
}

void residual_mixed(const Level& L, const double* d_ph, int cpg, const double2* E, float2* R, long ld, int ncols,
                    const double* d_lam, double* d_partials, double* d_out, cudaStream_t s) {
  if (ncols <= 0) return;
  const dim3 g = grid2(L.n, L.m, ncols);
  timer_begin(KC_RESIDUAL, s, 24.0 * L.D() * ncols);  // read E (16 B), write R (8 B) per edge DOF
  k_residual_mixed<<<g, dim3(kBX, kBY), 0, s>>>(L.lvl<df>(), L.wts_df(), d_ph, cpg, E, R, ld, d_lam, d_partials);
  timer_end(KC_RESIDUAL, s);
  PBS_LAUNCHED();
  count_df_launch();
  k_finalize2<<<ncols, 256, 0, s>>>(d_partials, g.x * g.y, d_out);
  PBS_LAUNCHED();
}

void residual(const Level& L, const double* d_ph, int cpg, const double2* E, double2* R, long ld, int ncols,
              const double* d_lam, double* d_partials, double* d_out, cudaStream_t s) {
  if (ncols <= 0) return;
  const dim3 g = grid2(L.n, L.m, ncols);
  timer_begin(KC_RESIDUAL, s, 32.0 * L.D() * ncols);
  k_residual<<<g, dim3(kBX, kBY), 0, s>>>(L.lvl<double>(), L.wts<double>(), d_ph, cpg, E, R, ld, d_lam, d_partials);
  timer_end(KC_RESIDUAL, s);
  PBS_LAUNCHED();
  k_finalize2<<<ncols, 256, 0, s>>>(d_partials, g.x * g.y, d_out);
  PBS_LAUNCHED();
}

// Partial blocks per group: enough to fill the GPU, and enough that no block sums
// more than kGramChunksPerBlock chunks of rows.  The double-float kernel keeps its
// sums as float pairs whose trailing parts collect rounding errors; a bounded row
// count per block keeps that error at a few units of 2^-48 whatever the mesh size
// and the number of Bloch vectors in flight (unbounded, 64 groups on a 512^2 mesh
// left about 1e-10 and the iteration stalled).
constexpr long kGramChunksPerBlock = 64;

int gram_partials(long rows, int ngroups) {
  const long chunks = (rows + kGramRows - 1) / kGramRows;
  long per = (2 * 152 + ngroups - 1) / ngroups;
  if (per < 8) per = 8;
  per = std::max(per, (chunks + kGramChunksPerBlock - 1) / kGramChunksPerBlock);
  return (int)(chunks < per ? chunks : per);
}

// Row stride of the staged arrays: qp, or (pad) the next stride that is 1 mod 8 in
// 16-byte elements, i.e. 4 banks mod 32.  With two row phases per tile (P = 2) the
// eight threads of a quarter-warp then read eight disjoint groups of four banks.
inline int gram_lds(int qp, bool pad) { return pad ? qp + ((1 - qp) % 8 + 8) % 8 : qp; }

template <int P, int TS> void launch_gram_df(const Level& L, const double* d_ph, Roles roles, int q, int ngroups,
                                             int npart, bool pad, double2* d_partials, cudaStream_t s) {
  static PerDeviceOnce once;
  once([] {
    PBS_CUDA(cudaFuncSetAttribute(k_gram_df<P, TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  4 * (kMaxTrial + TS + 8) * kGdRows * (int)sizeof(dcx)));
  });
  const int qp = TS * ((q + TS - 1) / TS), T = qp / TS, ntile = T * (T + 1) / 2, per = 256 / P;
  const int lds = gram_lds(qp, pad);
  const size_t smem = 4ull * lds * kGdRows * sizeof(dcx);
  k_gram_df<P, TS><<<dim3(npart, ngroups, (ntile + per - 1) / per), 256, smem, s>>>(
      L.lvl<df>(), L.wts_df(), mass_factor(L), d_ph, roles, q, qp, lds, kGdRows, d_partials, npart);
}

template <int TS> void gram_df_dispatch(const Level& L, const double* d_ph, Roles roles, int q, int ngroups, int npart,
                                        bool pad, double2* d_partials, cudaStream_t s) {
  const int T = (q + TS - 1) / TS, ntile = T * (T + 1) / 2;
  if (ntile <= 16) launch_gram_df<16, TS>(L, d_ph, roles, q, ngroups, npart, pad, d_partials, s);
  else if (ntile <= 32) launch_gram_df<8, TS>(L, d_ph, roles, q, ngroups, npart, pad, d_partials, s);
  else if (ntile <= 64) launch_gram_df<4, TS>(L, d_ph, roles, q, ngroups, npart, pad, d_partials, s);
  else launch_gram_df<2, TS>(L, d_ph, roles, q, ngroups, npart, pad, d_partials, s);
}

// Tuning keys count the groups of a launch in powers of two: the engine's launches
// shrink group by group as Bloch vectors converge, and one choice serves each range.
int group_bucket(int ngroups) {
  int b = 1;
  while (b < ngroups) b *= 2;
  return b;
}

void gram_groups(const Level& L, const double* d_ph, Roles roles, int q, int ngroups, double2* GM, double2* GA,
                 double2* d_partials, long partial_capacity, bool dfa, cudaStream_t s) {
  if (q <= 0 || ngroups <= 0) return;
  if (q > kMaxTrial) fail(PBS_EINVAL, "trial block too wide");
  const int ne = q * (q + 1) / 2;
  const int np0 = gram_partials(L.N(), ngroups);
  // variants: the kernel (tensor cores or double-float, mixed policy) and the number
  // of partial blocks per group; the autotuner picks among them on first use
  struct Variant {
    int kernel;  // 0: FP64, 1: double-float, 2: tensor cores
    int npart;
    bool pad;  // double-float kernel: bank-spread row stride of the staged arrays
  };
  Variant var[6];
  int nvar = 0;
  if (dfa && gram_tc_supported(q) && gram_on_tensor_cores()) {
    // offered first: with tuning off (PBS_TUNE=0) the tensor-core kernel runs
    var[nvar++] = {2, np0, false};
    var[nvar++] = {2, 2 * np0, false};
  }
  const int kern = dfa ? 1 : 0;
  var[nvar++] = {kern, np0, false};
  var[nvar++] = {kern, 2 * np0, false};
  if (dfa) {
    var[nvar++] = {kern, np0, true};
    var[nvar++] = {kern, 2 * np0, true};
  }
  auto fits = [&](const Variant& v) { return (long)ngroups * v.npart * 2 * ne <= partial_capacity; };
  if (!fits(var[0])) fail(PBS_EINVAL, "gram partials buffer too small");
  auto launch = [&](const Variant& v) {
    if (v.kernel == 2) {
      gram_tc(L, d_ph, roles, q, ngroups, v.npart, d_partials, s);
      count_df_launch();
    } else if (v.kernel == 1) {
      gram_df_dispatch<kGdTile>(L, d_ph, roles, q, ngroups, v.npart, v.pad, d_partials, s);
      count_df_launch();
    } else {
      static PerDeviceOnce once;
      once([] {
        PBS_CUDA(cudaFuncSetAttribute(k_gram_fused, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      6 * kMaxTrial * kGramRows * (int)sizeof(double2)));
      });
      const size_t smem = 6ull * q * kGramRows * sizeof(double2);
      k_gram_fused<<<dim3(v.npart, ngroups), 256, smem, s>>>(L.lvl<double>(), L.wts<double>(), d_ph, roles, q,
                                                              d_partials, v.npart);
    }
    PBS_LAUNCHED();
    k_gram_finalize<<<dim3((2 * ne + 255) / 256, ngroups), 256, 0, s>>>(d_partials, v.npart, q, GM, GA);
    PBS_LAUNCHED();
  };
  int pick = 0;
  if (nvar > 1) {
    const std::string key = std::string(dfa ? "gram_df" : "gram") + std::to_string(nvar) + "|" +
                            std::to_string(L.n) + "x" + std::to_string(L.m) + "|q" + std::to_string(q) + "|g" +
                            std::to_string(group_bucket(ngroups)) + "|" + device_tag();
    // a candidate whose partial sums do not fit the buffer runs the first one instead
    pick = tune_pick(key, nvar, [&](int c) { launch(fits(var[c]) ? var[c] : var[0]); }, s);
    if (!fits(var[pick])) pick = 0;
  }
  timer_begin(KC_GRAM, s, 8.0 * ne * 3.0 * L.N() * ngroups);  // flops: three complex MACs per entry and node
  launch(var[pick]);
  timer_end(KC_GRAM, s);
}

long gram_partials_size(long rows, int q, int ngroups) {
  // partial sums for up to twice the default split (a tuning candidate)
  return 2L * ngroups * gram_partials(rows, ngroups) * q * (q + 1);
}

bool gram_on_tensor_cores() {
  // PBS_GRAM=tc offers the tensor-core kernel to the autotuner (opt-in); the default
  // is the double-float kernel
  static const bool tc = [] {
    const char* v = std::getenv("PBS_GRAM");
    return v && std::strcmp(v, "tc") == 0;
  }();
  return tc;
}

size_t small_rr_scratch(int q) { return (3ull * q * q + (size_t)q * kMaxBlock) * sizeof(double2) + 64; }

void small_rr(const double2* GM, const double2* GA, int q, int p, double2* C, double* theta, double2* scratch,
              int* d_info, int ngroups, bool dfa, cudaStream_t s) {
  if (q > kMaxTrial || p > q || p < 1 || p > kMaxBlock || ngroups < 1) fail(PBS_EINVAL, "small_rr: bad sizes");
  const size_t dyn = (3ull * q * q + (size_t)q * p) * sizeof(double2);
  const int in_smem = dyn <= 150 * 1024 ? 1 : 0;
  static PerDeviceOnce once;
  once([] {
    PBS_CUDA(cudaFuncSetAttribute(k_small_rr<df>, cudaFuncAttributeMaxDynamicSharedMemorySize, 150 * 1024));
    PBS_CUDA(cudaFuncSetAttribute(k_small_rr<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, 150 * 1024));
  });
  const long stride = (long)(small_rr_scratch(q) / sizeof(double2));
  timer_begin(KC_SMALL_RR, s, 8.0 * 3.0 * q * q * q * ngroups);  // flops, order of magnitude
  int* phases = verbose_enabled() ? d_info + 2 : nullptr;
  if (dfa) {
    k_small_rr<df><<<ngroups, kRRThreads, in_smem ? dyn : 0, s>>>(GM, GA, q, p, C, theta, scratch, d_info, in_smem,
                                                                  phases, stride);
    count_df_launch();
  } else {
    k_small_rr<double><<<ngroups, kRRThreads, in_smem ? dyn : 0, s>>>(GM, GA, q, p, C, theta, scratch, d_info,
                                                                      in_smem, phases, stride);
  }
  timer_end(KC_SMALL_RR, s);
  PBS_LAUNCHED();
  if (verbose_enabled()) {
    int h[8] = {};
    PBS_CUDA(cudaMemcpyAsync(h, d_info, sizeof h, cudaMemcpyDeviceToHost, s));
    PBS_CUDA(cudaStreamSynchronize(s));
    std::fprintf(stderr, "[pbs] small_rr q=%d p=%d groups=%d info=%d rank=%d kcycles: chol %d solves %d householder %d bisect %d invit %d back %d\n",
                 q, p, ngroups, h[0], h[1], h[2], h[3], h[4], h[5], h[6], h[7]);
  }
}

template <int PB> void launch_update_df(Roles X, int q, const double2* C, int ldc, long cgs, double2* Y, long ldy,
                                        int p, const double2* Z, long ldz, long rows, dim3 grid, cudaStream_t s) {
  static PerDeviceOnce once;
  once([] {
    PBS_CUDA(cudaFuncSetAttribute(k_block_update_df<PB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kMaxBlock * kMaxTrial * (int)sizeof(dcx)));
  });
  k_block_update_df<PB><<<grid, 256, (size_t)p * q * sizeof(dcx), s>>>(X, q, C, ldc, cgs, Y, ldy, p, Z, ldz, rows);
}

template <int PB> void launch_update(Roles X, int q, const double2* C, int ldc, long cgs, double2* Y, long ldy, int p,
                                     const double2* Z, long ldz, long rows, dim3 grid, cudaStream_t s) {
  static PerDeviceOnce once;
  once([] {
    PBS_CUDA(cudaFuncSetAttribute(k_block_update<PB>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kMaxBlock * kMaxTrial * (int)sizeof(double2)));
  });
  k_block_update<PB><<<grid, 256, (size_t)p * q * sizeof(double2), s>>>(X, q, C, ldc, cgs, Y, ldy, p, Z, ldz, rows);
}

void block_update(Roles X, int q, const double2* C, int ldc, long cgs, double2* Y, long ldy, int p,
                  const double2* Z, long ldz, long rows, int ngroups, bool dfa, cudaStream_t s) {
  if (p <= 0 || rows <= 0 || ngroups <= 0) return;
  if (p > kMaxBlock) fail(PBS_EINVAL, "block_update: p too large");
  const long base = std::max<long>(1, blocks_for(rows, 256, 2 * 152 * 4) / ngroups);
  auto launch = [&](long per) {
    const dim3 grid((unsigned)per, ngroups);
    if (dfa) {
      if (p <= 8) launch_update_df<8>(X, q, C, ldc, cgs, Y, ldy, p, Z, ldz, rows, grid, s);
      else if (p <= 12) launch_update_df<12>(X, q, C, ldc, cgs, Y, ldy, p, Z, ldz, rows, grid, s);
      else if (p <= 16) launch_update_df<16>(X, q, C, ldc, cgs, Y, ldy, p, Z, ldz, rows, grid, s);
      else launch_update_df<32>(X, q, C, ldc, cgs, Y, ldy, p, Z, ldz, rows, grid, s);
      count_df_launch();
    } else {
      if (p <= 8) launch_update<8>(X, q, C, ldc, cgs, Y, ldy, p, Z, ldz, rows, grid, s);
      else if (p <= 12) launch_update<12>(X, q, C, ldc, cgs, Y, ldy, p, Z, ldz, rows, grid, s);
      else if (p <= 16) launch_update<16>(X, q, C, ldc, cgs, Y, ldy, p, Z, ldz, rows, grid, s);
      else launch_update<32>(X, q, C, ldc, cgs, Y, ldy, p, Z, ldz, rows, grid, s);
    }
    PBS_LAUNCHED();
  };
  // grid width: every row's result is the same whatever the grid (no cross-block
  // sums), so the autotuner's choice changes the time only
  const long cand[3] = {base, std::max<long>(1, base / 2), 2 * base};
  const std::string key = std::string(dfa ? "update_df" : "update") + "|" + std::to_string(rows) + "|q" +
                          std::to_string(q) + "|p" + std::to_string(p) + "|g" + std::to_string(group_bucket(ngroups)) + "|" +
                          device_tag();
  const int pick = tune_pick(key, 3, [&](int c) { launch(cand[c]); }, s);
  timer_begin(KC_BLOCK_UPDATE, s, 8.0 * q * p * rows * ngroups);  // flops
  launch(cand[pick]);
  timer_end(KC_BLOCK_UPDATE, s);
}

void random_block(double2* X, long ld, long rows, int ncols, uint64_t seed, cudaStream_t s) {
  if (ncols <= 0) return;
  k_random<<<dim3(blocks_for(rows, 256, 1024), ncols), 256, 0, s>>>(X, ld, rows, seed);
  PBS_LAUNCHED();
}

void scale_columns(double2* X, long ld, long rows, int ncols, const double* d_scale, cudaStream_t s) {
  if (ncols <= 0) return;
  k_scale_cols<<<dim3(blocks_for(rows, 256, 1024), ncols), 256, 0, s>>>(X, ld, rows, d_scale);
  PBS_LAUNCHED();
}

}  // namespace pbs

// ---------------------------------------------------------------------------
// Allocation-free Rayleigh-Ritz step (pbs_small_rr_noalloc in pbs.h).
//
// The scratch of the small dense solve lives in this file-scope device array,
// sized for the largest trial block the library supports (q = 96, p = 32):
// 3 q^2 + q p complex doubles, about 480 KB, held by every GPU that loads the
// library until the process exits.  Host code cannot use the array's name as a
// device address, so its address is looked up once per device with
// cudaGetSymbolAddress while that device is current.
// ---------------------------------------------------------------------------
#include <mutex>

namespace {
constexpr int kNoAllocQ = pbs::kMaxTrial, kNoAllocP = pbs::kMaxBlock;
static __device__ __align__(256) double2 g_small_rr_scratch[3 * kNoAllocQ * kNoAllocQ + kNoAllocQ * kNoAllocP + 8];
std::mutex g_scratch_mutex;
void* g_scratch_addr[pbs::kMaxDevices] = {};

int noalloc_fail(int status, const std::string& what) {
  pbs::set_last_error(what);
  return status;
}
}  // namespace

extern "C" int pbs_small_rr_noalloc(const pbs_c64* GM, const pbs_c64* GA, int q, int p, pbs_c64* C, double* theta,
                                    int* info, void* cuda_stream) {
  using namespace pbs;
  set_last_error("");
  if (!GM || !GA || !C || !theta || !info) return noalloc_fail(PBS_EINVAL, "a device pointer is NULL");
  if (q < 1 || q > kNoAllocQ || p < 1 || p > q || p > kNoAllocP)
    return noalloc_fail(PBS_EINVAL, "need 1 <= q <= 96 and 1 <= p <= min(q, 32)");
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return noalloc_fail(PBS_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return noalloc_fail(PBS_ECUDA, "device index beyond the library's table");
  // an error left by earlier work on this thread is reported as such and not cleared
  e = cudaPeekAtLastError();
  if (e != cudaSuccess)
    return noalloc_fail(PBS_ECUDA, std::string("an earlier CUDA error is pending: ") + cudaGetErrorString(e));
  void* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_addr[dev]) {
      // set-up on the first call on this device (with the device current)
      e = cudaGetSymbolAddress(&g_scratch_addr[dev], g_small_rr_scratch);
      if (e != cudaSuccess) {
        g_scratch_addr[dev] = nullptr;
        return noalloc_fail(PBS_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      }
    }
    scratch = g_scratch_addr[dev];
  }
  k_small_rr<df><<<1, kRRThreads, 0, (cudaStream_t)cuda_stream>>>((const double2*)GM, (const double2*)GA, q, p,
                                                                (double2*)C, theta, (double2*)scratch, info, 0,
                                                                nullptr, 0);
  count_launch();
  count_df_launch();
  e = cudaGetLastError();  // nothing was pending before the launch: this is the launch's own status
  if (e != cudaSuccess) return noalloc_fail(PBS_ECUDA, std::string("k_small_rr launch: ") + cudaGetErrorString(e));
  return PBS_OK;
}

namespace pbs {

template void sub_lift<double>(const Level&, const double*, int, const double2*, long, double2*, long, int,
                               cudaStream_t);
template void sub_lift<float>(const Level&, const double*, int, const float2*, long, double2*, long, int,
                              cudaStream_t);
template void lift_adj_mass<double>(const Level&, const double*, int, const double2*, long, double2*, long, int, bool,
                                    cudaStream_t);
template void lift_adj_mass<float>(const Level&, const double*, int, const double2*, long, float2*, long, int, bool,
                                   cudaStream_t);

}  // namespace pbs
