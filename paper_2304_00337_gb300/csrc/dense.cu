// Block kernels of the eigen-iteration (Section 4): FP64 residuals and
// Rayleigh quotients, the projection's right-hand side and update, the block
// Gram matrices, the small dense Rayleigh-Ritz step and the block update.
// Reductions are two-stage with a fixed summation order (deterministic).
#include <algorithm>
#include <cmath>

#include "internal.h"

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

__global__ void k_rayleigh_parts(Lvl<double> L, Wts<double> w, const double* ph, int cpg, const double2* __restrict__ X,
                                 long ld, double* __restrict__ part) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, c = blockIdx.z;
  double den = 0, num = 0;
  if (i < L.n && j < L.m) {
    const ERd<double> r{X + c * ld, L.n, L.m, load_ph<double>(ph, c / cpg)};
    const double2 mx = M_x<double>(r, L, i, j), my = M_y<double>(r, L, i, j);
    const double2 ex = r.x(i, j), ey = r.y(i, j);
    den = ex.x * mx.x + ex.y * mx.y + ey.x * my.x + ey.y * my.y;
    num = w(i, j) * nrm2(curl_at<double>(r, i, j));
  }
  block_sum2(den, num);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const int nblk = gridDim.x * gridDim.y, b = blockIdx.y * gridDim.x + blockIdx.x;
    part[((long)c * nblk + b) * 2] = den;
    part[((long)c * nblk + b) * 2 + 1] = num;
  }
}

__global__ void k_residual(Lvl<double> L, Wts<double> w, const double* ph, int cpg, const double2* __restrict__ E,
                           double2* __restrict__ R, long ld, const double* __restrict__ lam, double* __restrict__ part) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, c = blockIdx.z;
  double rr = 0, mm = 0;
  if (i < L.n && j < L.m) {
    const ERd<double> r{E + c * ld, L.n, L.m, load_ph<double>(ph, c / cpg)};
    const double l = lam[c];
    const double2 mx = M_x<double>(r, L, i, j), my = M_y<double>(r, L, i, j);
    const double2 rx = A_x<double>(r, w, i, j) - l * mx, ry = A_y<double>(r, w, i, j) - l * my;
    const long N = (long)L.n * L.m, e = (long)j * L.n + i;
    R[c * ld + e] = rx;
    R[c * ld + N + e] = ry;
    rr = nrm2(rx) + nrm2(ry);
    mm = nrm2(mx) + nrm2(my);
  }
  block_sum2(rr, mm);
  if (threadIdx.x == 0 && threadIdx.y == 0) {
    const int nblk = gridDim.x * gridDim.y, b = blockIdx.y * gridDim.x + blockIdx.x;
    part[((long)c * nblk + b) * 2] = rr;
    part[((long)c * nblk + b) * 2 + 1] = mm;
  }
}

// rhs(i,j) = (L^* M x)(i,j) = (Mx)_x(i-1,j) - (Mx)_x(i,j) + (Mx)_y(i,j-1) - (Mx)_y(i,j)
template <class T>
__global__ void k_lift_adj_mass(Lvl<double> L, const double* ph, int cpg, const double2* __restrict__ X, long ldx,
                                cx<T>* __restrict__ Y, long ldy) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, c = blockIdx.z;
  if (i >= L.n || j >= L.m) return;
  const ERd<double> r{X + c * ldx, L.n, L.m, load_ph<double>(ph, c / cpg)};
  const double2 v = M_x<double>(r, L, i - 1, j) - M_x<double>(r, L, i, j) + M_y<double>(r, L, i, j - 1) -
                    M_y<double>(r, L, i, j);
  Y[c * ldy + (long)j * L.n + i] = mk<T>(T(v.x), T(v.y));
}

// x <- x - L phi
template <class T>
__global__ void k_sub_lift(int n, int m, const double* ph, int cpg, const cx<T>* __restrict__ Phi, long ldp,
                           double2* __restrict__ X, long ldx) {
  const int i = blockIdx.x * kBX + threadIdx.x, j = blockIdx.y * kBY + threadIdx.y, c = blockIdx.z;
  if (i >= n || j >= m) return;
  const Ph<double> p = load_ph<double>(ph, c / cpg);
  const cx<T>* f = Phi + c * ldp;
  const long N = (long)n * m, e = (long)j * n + i;
  // read phi in FP64 through the Bloch extension
  auto rd = [&](int ii, int jj) -> double2 {
    double2 ph1 = make_double2(1, 0);
    bool wr = false;
    if (ii >= n) { ii -= n; ph1 = p.al; wr = true; }
    if (jj >= m) { jj -= m; ph1 = cmul(ph1, p.be); wr = true; }
    const cx<T> v = f[(long)jj * n + ii];
    const double2 d = make_double2(double(v.x), double(v.y));
    return wr ? cmul(d, ph1) : d;
  };
  const double2 f0 = rd(i, j);
  double2* x = X + c * ldx;
  x[e] = x[e] - (rd(i + 1, j) - f0);
  x[N + e] = x[N + e] - (rd(i, j + 1) - f0);
}

// per column sums of the x-edge and y-edge values (for the constant-field deflation at k = 0)
__global__ void k_edge_sums(long N, const double2* __restrict__ X, long ld, double* __restrict__ part, int nblk) {
  const int c = blockIdx.y;
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

__global__ void k_edge_sub_means(long N, double2* __restrict__ X, long ld, const double* __restrict__ part, int nblk) {
  const int c = blockIdx.y;
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
    Y[t] = make_float2(float(X[t].x), float(X[t].y));
}
__global__ void k_f2d(const float2* __restrict__ X, double2* __restrict__ Y, long n) {
  for (long t = blockIdx.x * (long)blockDim.x + threadIdx.x; t < n; t += (long)gridDim.x * blockDim.x)
    Y[t] = make_double2(double(X[t].x), double(X[t].y));
}

// ---- tall-skinny Gram: G[a][b] = sum_r conj(X[r][a]) wt[r] Y[r][b], a <= b ----
constexpr int kGramRows = 32;
constexpr int kGramAcc = 20;  // accumulators per thread: q(q+1)/2 <= 20 * 256 for q <= 100

__global__ void __launch_bounds__(256) k_gram_ts(const double2* __restrict__ X, long ldx, const double2* __restrict__ Y,
                                                 long ldy, int q, long rows, const double* __restrict__ winv,
                                                 double wscale, double2* __restrict__ part) {
  extern __shared__ double2 sm[];
  double2* xs = sm;                       // [q][kGramRows]
  double2* ys = sm + q * kGramRows;       // [q][kGramRows]
  const int tid = threadIdx.x, nt = blockDim.x;
  const int ne = q * (q + 1) / 2;
  int ea[kGramAcc], eb[kGramAcc];
  double2 acc[kGramAcc];
#pragma unroll
  for (int k = 0; k < kGramAcc; ++k) {
    acc[k] = make_double2(0, 0);
    const int e = tid + k * nt;
    int a = 0, b = 0;
    if (e < ne) {  // column-major upper triangle: e = b(b+1)/2 + a
      b = int((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
      while ((b + 1) * (b + 2) / 2 <= e) ++b;
      while (b * (b + 1) / 2 > e) --b;
      a = e - b * (b + 1) / 2;
    }
    ea[k] = a;
    eb[k] = b;
  }
  const long nchunks = (rows + kGramRows - 1) / kGramRows;
  for (long ch = blockIdx.x; ch < nchunks; ch += gridDim.x) {
    const long r0 = ch * kGramRows;
    __syncthreads();
    for (int t = tid; t < q * kGramRows; t += nt) {
      const int col = t / kGramRows, rr = t % kGramRows;
      const long r = r0 + rr;
      double2 xv = make_double2(0, 0), yv = make_double2(0, 0);
      if (r < rows) {
        xv = X[col * ldx + r];
        yv = Y[col * ldy + r];
        if (winv) yv = (wscale * winv[r]) * yv;
      }
      xs[col * kGramRows + rr] = xv;
      ys[col * kGramRows + rr] = yv;
    }
    __syncthreads();
#pragma unroll
    for (int k = 0; k < kGramAcc; ++k) {
      if (tid + k * nt < ne) {
        const double2* xa = xs + ea[k] * kGramRows;
        const double2* yb = ys + eb[k] * kGramRows;
        double2 s = acc[k];
#pragma unroll 8
        for (int rr = 0; rr < kGramRows; ++rr) {
          const double2 u = xa[rr], v = yb[rr];
          s.x = fma(u.x, v.x, fma(u.y, v.y, s.x));
          s.y = fma(u.x, v.y, fma(-u.y, v.x, s.y));
        }
        acc[k] = s;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < kGramAcc; ++k) {
    const int e = tid + k * nt;
    if (e < ne) part[(long)blockIdx.x * ne + e] = acc[k];
  }
}

// sum partials in fixed order; write full Hermitian q x q (column-major), optionally accumulating
__global__ void k_gram_finalize(const double2* __restrict__ part, int npart, int q, double2* __restrict__ G,
                                int accumulate) {
  const int ne = q * (q + 1) / 2;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < ne; e += gridDim.x * blockDim.x) {
    double2 s = make_double2(0, 0);
    for (int p = 0; p < npart; ++p) {
      const double2 v = part[(long)p * ne + e];
      s.x += v.x;
      s.y += v.y;
    }
    int b = int((sqrt(8.0 * e + 1.0) - 1.0) * 0.5);
    while ((b + 1) * (b + 2) / 2 <= e) ++b;
    while (b * (b + 1) / 2 > e) --b;
    const int a = e - b * (b + 1) / 2;
    if (accumulate) {
      s = s + G[a + (long)b * q];
    }
    if (a == b) s.y = 0.0;
    G[a + (long)b * q] = s;
    G[b + (long)a * q] = conj(s);
  }
}

// ---- small dense Rayleigh-Ritz (one block) -------------------------------
// scratch layout (double2 unless noted), q <= kMaxTrial:
//   G [q*q]  scaled M-Gram, overwritten by its Cholesky rows R (upper)
//   A [q*q]  scaled A-Gram
//   T [q*q]  R_K^{-1} (r x r, upper)
//   Y [q*q]  work
//   H [q*q]  T^* A_K T, diagonalised in place
//   V [q*q]  Jacobi eigenvectors
//   d [q] (double) column scales, keep [q] (int), theta [q] (double)
constexpr double kDropTol = 1e-12;  // relative pivot below which a trial direction is dropped

__device__ __forceinline__ double2 ldg2(const double2* p) { return *p; }

__global__ void __launch_bounds__(256) k_small_rr(const double2* __restrict__ GM, const double2* __restrict__ GA, int q,
                                                  int p, double2* __restrict__ Cout, double* __restrict__ theta_out,
                                                  double2* __restrict__ scr, int* __restrict__ info) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const long qq = (long)q * q;
  double2 *G = scr, *A = scr + qq, *T = scr + 2 * qq, *Y = scr + 3 * qq, *H = scr + 4 * qq, *V = scr + 5 * qq;
  double* d = (double*)(scr + 6 * qq);
  int* kidx = (int*)(d + q);
  __shared__ int s_r, s_bad;
  __shared__ double s_piv;
  __shared__ int s_keep[kMaxTrial];
  // 1. scale to unit diagonal
  for (int i = tid; i < q; i += nt) {
    const double g = GM[(long)i * q + i].x;
    d[i] = (g > 0.0 && isfinite(g)) ? 1.0 / sqrt(g) : 0.0;
  }
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (long t = tid; t < qq; t += nt) {
    const int i = int(t % q), j = int(t / q);
    const double s = d[i] * d[j];
    const double2 gm = GM[t], ga = GA[t];
    if (!isfinite(gm.x) || !isfinite(gm.y) || !isfinite(ga.x) || !isfinite(ga.y)) s_bad = 1;
    G[t] = s * gm;
    A[t] = s * ga;
  }
  __syncthreads();
  // 2. Cholesky G = R^* R (R upper, rows stored in G) with dropping of dependent directions
  for (int k = 0; k < q; ++k) {
    if (tid == 0) {
      const double pv = G[(long)k * q + k].x;
      const bool keep = d[k] > 0.0 && pv > kDropTol && isfinite(pv);
      s_keep[k] = keep;
      s_piv = keep ? sqrt(pv) : 0.0;
    }
    __syncthreads();
    const double piv = s_piv;
    if (piv > 0.0) {
      for (int j = k + tid; j < q; j += nt) {  // row k of R
        const double2 v = G[(long)j * q + k];
        G[(long)j * q + k] = make_double2(v.x / piv, v.y / piv);
      }
      __syncthreads();
      const int rem = q - k - 1;
      for (long t = tid; t < (long)rem * rem; t += nt) {
        const int ii = k + 1 + int(t % rem), jj = k + 1 + int(t / rem);
        if (ii > jj) continue;
        // G[ii][jj] -= conj(R[k][ii]) R[k][jj]
        const double2 rki = G[(long)ii * q + k], rkj = G[(long)jj * q + k];
        G[(long)jj * q + ii] = G[(long)jj * q + ii] - cmulc(rki, rkj);
      }
    } else {
      for (int j = k + tid; j < q; j += nt) G[(long)j * q + k] = make_double2(0, 0);
    }
    __syncthreads();
  }
  if (tid == 0) {
    int r = 0;
    for (int k = 0; k < q; ++k)
      if (s_keep[k]) kidx[r++] = k;
    s_r = r;
  }
  __syncthreads();
  const int r = s_r;
  if (r < p || s_bad) {
    if (tid == 0) {
      info[0] = s_bad ? -2 : -1;
      info[1] = r;
    }
    return;
  }
  // 3. T = R_K^{-1}: columns in parallel, back substitution
  for (int c = tid; c < r; c += nt) {
    for (int i = r - 1; i >= 0; --i) {
      double2 s = make_double2(i == c ? 1.0 : 0.0, 0.0);
      for (int k = i + 1; k <= c; ++k) s = s - cmul(G[(long)kidx[k] * q + kidx[i]], T[(long)c * q + k]);
      const double dii = G[(long)kidx[i] * q + kidx[i]].x;
      T[(long)c * q + i] = i > c ? make_double2(0, 0) : make_double2(s.x / dii, s.y / dii);
    }
  }
  __syncthreads();
  // 4. H = T^* A_K T
  for (long t = tid; t < (long)r * r; t += nt) {
    const int i = int(t % r), c = int(t / r);
    double2 s = make_double2(0, 0);
    for (int k = 0; k <= c; ++k) s = s + cmul(A[(long)kidx[k] * q + kidx[i]], T[(long)c * q + k]);
    Y[(long)c * q + i] = s;
  }
  __syncthreads();
  for (long t = tid; t < (long)r * r; t += nt) {
    const int i = int(t % r), c = int(t / r);
    double2 s = make_double2(0, 0);
    for (int k = 0; k <= i; ++k) s = s + cmulc(T[(long)i * q + k], Y[(long)c * q + k]);
    H[(long)c * q + i] = s;
    V[(long)c * q + i] = make_double2(i == c ? 1.0 : 0.0, 0.0);
  }
  __syncthreads();
  for (long t = tid; t < (long)r * r; t += nt) {  // exact Hermitian symmetry
    const int i = int(t % r), c = int(t / r);
    if (i < c) {
      const double2 u = H[(long)c * q + i], l = H[(long)i * q + c];
      H[(long)c * q + i] = make_double2(0.5 * (u.x + l.x), 0.5 * (u.y - l.y));
      H[(long)i * q + c] = make_double2(0.5 * (u.x + l.x), -0.5 * (u.y - l.y));
    } else if (i == c) {
      H[(long)c * q + i].y = 0.0;
    }
  }
  __syncthreads();
  // 5. cyclic Jacobi with a round-robin (parallel) ordering
  __shared__ int s_pp[kMaxTrial / 2 + 1], s_qq[kMaxTrial / 2 + 1];
  __shared__ double s_c[kMaxTrial / 2 + 1], s_s[kMaxTrial / 2 + 1];
  __shared__ double2 s_w[kMaxTrial / 2 + 1];
  __shared__ double s_off, s_dg;
  __shared__ double s_poff[256], s_pdg[256];
  const int rr = (r % 2) ? r + 1 : r;  // with a dummy player when r is odd
  const int npair = rr / 2;
  for (int sweep = 0; sweep < 60 && r > 1; ++sweep) {
    // convergence test (fixed summation order: per-thread partials, then thread 0)
    double off = 0, dg = 0;
    for (long t = tid; t < (long)r * r; t += nt) {
      const int i = int(t % r), c = int(t / r);
      if (i < c) off += nrm2(H[(long)c * q + i]);
      else if (i == c) dg += H[(long)c * q + i].x * H[(long)c * q + i].x;
    }
    s_poff[tid] = off;
    s_pdg[tid] = dg;
    __syncthreads();
    if (tid == 0) {
      double so = 0, sd = 0;
      for (int t = 0; t < nt; ++t) {
        so += s_poff[t];
        sd += s_pdg[t];
      }
      s_off = so;
      s_dg = sd;
    }
    __syncthreads();
    if (!(s_off > 1e-34 * s_dg)) break;
    for (int step = 0; step < rr - 1; ++step) {
      for (int k = tid; k < npair; k += nt) {
        int a, b;
        if (k == 0) { a = rr - 1; b = step; }
        else { a = (step + k) % (rr - 1); b = (step - k + rr - 1) % (rr - 1); }
        if (a > b) { const int t2 = a; a = b; b = t2; }
        s_pp[k] = a;
        s_qq[k] = b;
        double c = 1.0, s = 0.0;
        double2 w = make_double2(1, 0);
        if (b < r) {
          const double2 h = H[(long)b * q + a];
          const double ah = sqrt(nrm2(h));
          if (ah > 0.0) {
            const double app = H[(long)a * q + a].x, aqq = H[(long)b * q + b].x;
            const double th = (aqq - app) / (2.0 * ah);
            const double t = (th >= 0 ? 1.0 : -1.0) / (fabs(th) + sqrt(th * th + 1.0));
            c = 1.0 / sqrt(t * t + 1.0);
            s = t * c;
            w = make_double2(h.x / ah, -h.y / ah);  // conj(h)/|h|
          }
        }
        s_c[k] = c;
        s_s[k] = s;
        s_w[k] = w;
      }
      __syncthreads();
      // columns: H <- H J, V <- V J, J = [[c, s], [-s w, c w]] with w = conj(h)/|h|
      for (long t = tid; t < (long)npair * r; t += nt) {
        const int k = int(t / r), row = int(t % r);
        const int a = s_pp[k], b = s_qq[k];
        if (b >= r || s_s[k] == 0.0) continue;
        const double c = s_c[k], s = s_s[k];
        const double2 w = s_w[k];
        const double2 ha = H[(long)a * q + row], hb = cmul(w, H[(long)b * q + row]);
        H[(long)a * q + row] = c * ha - s * hb;
        H[(long)b * q + row] = s * ha + c * hb;
        const double2 va = V[(long)a * q + row], vb = cmul(w, V[(long)b * q + row]);
        V[(long)a * q + row] = c * va - s * vb;
        V[(long)b * q + row] = s * va + c * vb;
      }
      __syncthreads();
      // rows: H <- J^* H
      for (long t = tid; t < (long)npair * r; t += nt) {
        const int k = int(t / r), col = int(t % r);
        const int a = s_pp[k], b = s_qq[k];
        if (b >= r || s_s[k] == 0.0) continue;
        const double c = s_c[k], s = s_s[k];
        const double2 wc = conj(s_w[k]);
        const double2 ha = H[(long)col * q + a], hb = cmul(wc, H[(long)col * q + b]);
        H[(long)col * q + a] = c * ha - s * hb;
        H[(long)col * q + b] = s * ha + c * hb;
      }
      __syncthreads();
      for (int k = tid; k < npair; k += nt) {
        const int a = s_pp[k], b = s_qq[k];
        if (b >= r || s_s[k] == 0.0) continue;
        H[(long)b * q + a] = make_double2(0, 0);
        H[(long)a * q + b] = make_double2(0, 0);
        H[(long)a * q + a].y = 0.0;
        H[(long)b * q + b].y = 0.0;
      }
      __syncthreads();
    }
  }
  // 6. sort Ritz values ascending
  __shared__ int s_ord[kMaxTrial];
  if (tid == 0) {
    for (int i = 0; i < r; ++i) s_ord[i] = i;
    for (int i = 1; i < r; ++i) {
      const int v = s_ord[i];
      const double key = H[(long)v * q + v].x;
      int j = i - 1;
      while (j >= 0 && H[(long)s_ord[j] * q + s_ord[j]].x > key) {
        s_ord[j + 1] = s_ord[j];
        --j;
      }
      s_ord[j + 1] = v;
    }
  }
  __syncthreads();
  // 7. C[:, j] = D T V[:, ord[j]] (rows of dropped directions are zero)
  for (long t = tid; t < (long)q * p; t += nt) {
    const int row = int(t % q), j = int(t / q);
    Cout[(long)j * q + row] = make_double2(0, 0);
  }
  __syncthreads();
  for (long t = tid; t < (long)r * p; t += nt) {
    const int i = int(t % r), j = int(t / r);
    const int col = s_ord[j];
    double2 s = make_double2(0, 0);
    for (int k = i; k < r; ++k) s = s + cmul(T[(long)k * q + i], V[(long)col * q + k]);
    Cout[(long)j * q + kidx[i]] = d[kidx[i]] * s;
  }
  for (int j = tid; j < p; j += nt) theta_out[j] = H[(long)s_ord[j] * q + s_ord[j]].x;
  if (tid == 0) {
    info[0] = 0;
    info[1] = r;
  }
}

// Y[:, j] = sum_i X[:, i] C[i, j] (+ Z[:, j])
__global__ void __launch_bounds__(256) k_block_update(const double2* __restrict__ X, long ldx, int q,
                                                      const double2* __restrict__ C, int ldc, double2* __restrict__ Y,
                                                      long ldy, int p, const double2* __restrict__ Z, long ldz,
                                                      long rows) {
  extern __shared__ double2 cs[];  // [p][q]
  for (int t = threadIdx.x; t < p * q; t += blockDim.x) cs[t] = C[(long)(t / q) * ldc + (t % q)];
  __syncthreads();
  for (long r = blockIdx.x * (long)blockDim.x + threadIdx.x; r < rows; r += (long)gridDim.x * blockDim.x) {
    double2 acc[kMaxBlock];
#pragma unroll
    for (int j = 0; j < kMaxBlock; ++j) acc[j] = make_double2(0, 0);
    for (int i = 0; i < q; ++i) {
      const double2 x = X[(long)i * ldx + r];
#pragma unroll
      for (int j = 0; j < kMaxBlock; ++j) {
        if (j < p) {
          const double2 c = cs[j * q + i];
          acc[j].x = fma(x.x, c.x, fma(-x.y, c.y, acc[j].x));
          acc[j].y = fma(x.x, c.y, fma(x.y, c.x, acc[j].y));
        }
      }
    }
#pragma unroll
    for (int j = 0; j < kMaxBlock; ++j) {
      if (j < p) {
        double2 v = acc[j];
        if (Z) v = v + Z[(long)j * ldz + r];
        Y[(long)j * ldy + r] = v;
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
  k_d2f<<<blocks_for(n), 256, 0, s>>>(X, Y, n);
  PBS_LAUNCHED();
}
void convert_f2d(const float2* X, double2* Y, long n, cudaStream_t s) {
  if (n <= 0) return;
  k_f2d<<<blocks_for(n), 256, 0, s>>>(X, Y, n);
  PBS_LAUNCHED();
}

template <class T>
void sub_lift(const Level& L, const double* d_ph, int cpg, const cx<T>* Phi, long ldp, double2* X, long ldx, int ncols,
              cudaStream_t s) {
  if (ncols <= 0) return;
  k_sub_lift<T><<<grid2(L.n, L.m, ncols), dim3(kBX, kBY), 0, s>>>(L.n, L.m, d_ph, cpg, Phi, ldp, X, ldx);
  PBS_LAUNCHED();
}

template <class T>
void lift_adj_mass(const Level& L, const double* d_ph, int cpg, const double2* X, long ldx, cx<T>* Rhs, long ldr,
                   int ncols, cudaStream_t s) {
  if (ncols <= 0) return;
  timer_begin(KC_LIFT_ADJ_MASK, s, (16.0 * L.D() + 2.0 * sizeof(T) * L.N()) * ncols);
  k_lift_adj_mass<T><<<grid2(L.n, L.m, ncols), dim3(kBX, kBY), 0, s>>>(L.lvl<double>(), d_ph, cpg, X, ldx, Rhs, ldr);
  timer_end(KC_LIFT_ADJ_MASK, s);
  PBS_LAUNCHED();
}

void deflate_constants(const Level& L, double2* X, long ld, int ncols, double* d_partials, cudaStream_t s) {
  if (ncols <= 0) return;
  const int nblk = 64;
  k_edge_sums<<<dim3(nblk, ncols), 256, 0, s>>>(L.N(), X, ld, d_partials, nblk);
  PBS_LAUNCHED();
  k_edge_sub_means<<<dim3(nblk, ncols), 256, 0, s>>>(L.N(), X, ld, d_partials, nblk);
  PBS_LAUNCHED();
}

void rayleigh_parts(const Level& L, const double* d_ph, int cpg, const double2* X, long ld, int ncols,
                    double* d_partials, double* d_out, cudaStream_t s) {
  if (ncols <= 0) return;
  const dim3 g = grid2(L.n, L.m, ncols);
  k_rayleigh_parts<<<g, dim3(kBX, kBY), 0, s>>>(L.lvl<double>(), L.wts<double>(), d_ph, cpg, X, ld, d_partials);
  PBS_LAUNCHED();
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

int gram_partials(long rows) {
  long b = (rows + kGramRows - 1) / kGramRows;
  return (int)(b < 2 * 152 ? b : 2 * 152);
}

void gram(const Level& L, const double* d_ph, int cpg, const double2* S, long ld, int q, double2* GM, double2* GA,
          double2* work, double2* d_partials, int npart, cudaStream_t s) {
  if (q <= 0) return;
  if (q > kMaxTrial) fail(PBS_EINVAL, "trial block too wide");
  const long D = L.D(), N = L.N();
  double2* MS = work;            // D x q
  double2* CS = work + D * q;    // N x q
  apply_edge<double>(L, d_ph, cpg, S, MS, nullptr, ld, q, 0.0, 1.0, 0.0, nullptr, 0.0, s);
  // MS uses stride ld (same as S); CS stride N
  apply_curl<double>(L, d_ph, cpg, S, ld, CS, N, q, s);
  const size_t smem = 2ull * q * kGramRows * sizeof(double2);
  static bool attr = false;
  if (!attr) {
    PBS_CUDA(cudaFuncSetAttribute(k_gram_ts, cudaFuncAttributeMaxDynamicSharedMemorySize, 2 * kMaxTrial * kGramRows * (int)sizeof(double2)));
    attr = true;
  }
  const int ne = q * (q + 1) / 2;
  const int npM = std::min(npart, gram_partials(D));
  timer_begin(KC_GRAM, s, 8.0 * ne * D);  // flops: one complex MAC per entry and row
  k_gram_ts<<<npM, 256, smem, s>>>(S, ld, MS, ld, q, D, nullptr, 0.0, d_partials);
  timer_end(KC_GRAM, s);
  PBS_LAUNCHED();
  k_gram_finalize<<<(ne + 255) / 256, 256, 0, s>>>(d_partials, npM, q, GM, 0);
  PBS_LAUNCHED();
  const int npA = std::min(npart, gram_partials(N));
  timer_begin(KC_GRAM, s, 8.0 * ne * N);
  k_gram_ts<<<npA, 256, smem, s>>>(CS, N, CS, N, q, N, L.winv64, 1.0 / (L.h1 * L.h2), d_partials);
  timer_end(KC_GRAM, s);
  PBS_LAUNCHED();
  k_gram_finalize<<<(ne + 255) / 256, 256, 0, s>>>(d_partials, npA, q, GA, 0);
  PBS_LAUNCHED();
}

size_t small_rr_scratch(int q) { return (6ull * q * q + q) * sizeof(double2) + (size_t)q * sizeof(int) + 64; }

void small_rr(const double2* GM, const double2* GA, int q, int p, double2* C, double* theta, double2* scratch,
              int* d_info, cudaStream_t s) {
  if (q > kMaxTrial || p > q || p < 1) fail(PBS_EINVAL, "small_rr: bad sizes");
  timer_begin(KC_SMALL_RR, s, 8.0 * 6.0 * q * q * q);  // flops, order of magnitude
  k_small_rr<<<1, 256, 0, s>>>(GM, GA, q, p, C, theta, scratch, d_info);
  timer_end(KC_SMALL_RR, s);
  PBS_LAUNCHED();
}

void block_update(const double2* X, long ldx, int q, const double2* C, int ldc, double2* Y, long ldy, int p,
                  const double2* Z, long ldz, long rows, cudaStream_t s) {
  if (p <= 0 || rows <= 0) return;
  if (p > kMaxBlock) fail(PBS_EINVAL, "block_update: p too large");
  const size_t smem = (size_t)p * q * sizeof(double2);
  static bool attr = false;
  if (!attr) {
    PBS_CUDA(cudaFuncSetAttribute(k_block_update, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  kMaxBlock * kMaxTrial * (int)sizeof(double2)));
    attr = true;
  }
  timer_begin(KC_BLOCK_UPDATE, s, 8.0 * q * p * rows);  // flops
  k_block_update<<<blocks_for(rows, 256, 2 * 152 * 4), 256, smem, s>>>(X, ldx, q, C, ldc, Y, ldy, p, Z, ldz, rows);
  timer_end(KC_BLOCK_UPDATE, s);
  PBS_LAUNCHED();
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

template void sub_lift<double>(const Level&, const double*, int, const double2*, long, double2*, long, int, cudaStream_t);
template void sub_lift<float>(const Level&, const double*, int, const float2*, long, double2*, long, int, cudaStream_t);
template void lift_adj_mass<double>(const Level&, const double*, int, const double2*, long, double2*, long, int,
                                    cudaStream_t);
template void lift_adj_mass<float>(const Level&, const double*, int, const double2*, long, float2*, long, int,
                                   cudaStream_t);

}  // namespace pbs
