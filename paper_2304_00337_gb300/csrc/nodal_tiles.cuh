// Tiled fine-level steps of the nodal multigrid cycle (Section 5): one kernel
// for pre-smoothing, residual and restriction ("down"), one for prolongation
// and post-smoothing ("up").  Included by mg.cu; the kernels use nothing but
// the per-point bodies of mgpoint.cuh.
#pragma once
#include "mgpoint.cuh"

namespace pbs {

// ---- tiled fine-level nodal steps ------------------------------------------------
// On levels too large for the fused tail, the pre-smoothing, residual and
// restriction of the nodal cycle run as one kernel ("down") and the prolongation
// and post-smoothing as another ("up").  A CTA owns an FT x FT tile of fine nodes of
// one column and keeps a halo in shared memory wide enough that every colour step
// can be carried out there: colour step s of S = 4 nu needs the previous state one
// node further out, so the region shrinks by one ring per step.  Nodes outside the
// level are read through the Bloch extension and keep their colour (the sides are
// even), so the redundant halo work reproduces the neighbours' values exactly.
// The node updates use the per-node formulas of the step-by-step kernels.
// The tile side FT (32 or 64) and the block size are launch choices (the
// autotuner picks per level, column count and precision): a larger tile
// recomputes a smaller share of halo nodes but holds more shared memory.
constexpr int kFineMaxThreads = 512;

// reader of a shared-memory region whose element (0,0) is global node (oa, ob)
template <class T> struct NRdSm {
  const cx<T>* s;
  int W, oa, ob;
  __device__ __forceinline__ cx<T> v(int i, int j) const { return s[(j - ob) * W + (i - oa)]; }
};

// (u, v) with t = v w + u, 0 <= u < w, for 0 <= t < 2^16 and w >= 1: the float quotient
// (t + 1/2) / w lies at least 1/(2w) from an integer and is off by at most
// (t/w) 2^-23 (two roundings), i.e. by at most t 2^-22 <= 1/64 of that distance, so its
// truncation is exact (an integer division by a run-time w costs ~20 instructions)
__device__ __forceinline__ void split_index(int t, int w, float inv_w, int& u, int& v) {
  v = (int)(((float)t + 0.5f) * inv_w);
  u = t - v * w;
}

// colour q nodes (global parity (q & 1, q >> 1)) of the region rows/cols [r0, r1) in
// region coordinates, the region's global origin being (oa, ob)
template <class T, class F>
__device__ __forceinline__ void for_colour(int q, int r0, int r1, int oa, int ob, F&& f) {
  const int pa = ((q & 1) - oa) & 1, pb = ((q >> 1) - ob) & 1;
  const int a0 = r0 + ((pa - r0) & 1), b0 = r0 + ((pb - r0) & 1);
  const int na = (r1 - a0 + 1) / 2, nb = (r1 - b0 + 1) / 2;
  const float inv = 1.0f / (float)na;
  for (int t = threadIdx.x; t < na * nb; t += blockDim.x) {
    int u, v;
    split_index(t, na, inv, u, v);
    f(a0 + 2 * u, b0 + 2 * v);
  }
}

// Stage a W x W region of a node field whose element (0,0) is node (oa, ob): direct reads
// when the region lies inside the level, else through the Bloch extension.
template <class T>
__device__ __forceinline__ void stage_region(const cx<T>* __restrict__ f, int oa, int ob, int W, int n, int m,
                                             const Ph<T>& p, cx<T>* S) {
  const float inv = 1.0f / (float)W;
  const bool in = oa >= 0 && ob >= 0 && oa + W <= n && ob + W <= m;
  for (int t = threadIdx.x; t < W * W; t += blockDim.x) {
    int u, v;
    split_index(t, W, inv, u, v);
    S[t] = in ? f[(long)(ob + v) * n + oa + u] : gread<T>(f, oa + u, ob + v, n, m, p);
  }
}

template <class T, int FT>
__global__ void __launch_bounds__(kFineMaxThreads) k_node_down(Lvl<T> L, int nc, int mc, const double* ph, int cpg,
                                                            const cx<T>* __restrict__ B, long ldb,
                                                            const cx<T>* __restrict__ X0, long ld0,
                                                            cx<T>* __restrict__ Xs, long lds, cx<T>* __restrict__ Bc,
                                                            long ldc, int nu) {
  extern __shared__ float4 fine_sm[];
  // rows/cols [lo-2, lo+T+1) hold x after the last colour step (the residual reads
  // them); step s works on that range widened by 4 nu - 1 - s rings and reads one
  // ring further, so the region adds 4 nu + 2 rings below and 4 nu + 1 above
  const int lo = 4 * nu + 2, W = FT + 8 * nu + 3;
  cx<T>* sx = reinterpret_cast<cx<T>*>(fine_sm);
  cx<T>* sb = sx + W * W;
  const int c = blockIdx.z, tid = threadIdx.x, nt = blockDim.x;
  const int i0 = blockIdx.x * FT, j0 = blockIdx.y * FT, oa = i0 - lo, ob = j0 - lo;
  const Ph<T> p = load_ph<T>(ph, c / cpg);
  const cx<T>* b = B + c * ldb;
  stage_region<T>(b, oa, ob, W, L.n, L.m, p, sb);
  // the smoothing starts from X0 where one is given (a cycle that continues from an
  // iterate: the same steps as a zero start on the residual b - P X0, plus X0)
  if (X0) stage_region<T>(X0 + c * ld0, oa, ob, W, L.n, L.m, p, sx);
  else
    for (int t = tid; t < W * W; t += nt) sx[t] = czero<T>();
  __syncthreads();
  const NRdSm<T> rs{sx, W, oa, ob};
  for (int it = 0; it < nu; ++it)
    for (int q = 0; q < 4; ++q) {
      const int e = 4 * nu - 1 - (4 * it + q);  // rings beyond what the residual needs
      for_colour<T>(q, lo - 2 - e, lo + FT + 1 + e, oa, ob, [&](int a, int bb) {
        const int k = bb * W + a;
        const cx<T> res = sb[k] - P_at<T>(rs, L, oa + a, ob + bb);
        sx[k] = sx[k] + (T(1) / P_diag<T>(L)) * res;
      });
      __syncthreads();
    }
  // residual b - P x in place on the fine nodes the restriction reads
  for (int t = tid; t < (FT + 1) * (FT + 1); t += nt) {
    const int a = lo - 1 + t % (FT + 1), bb = lo - 1 + t / (FT + 1), k = bb * W + a;
    cx<T> y = T(-1) * P_at<T>(rs, L, oa + a, ob + bb);
    y = y + T(1) * sb[k];
    sb[k] = y;
  }
  __syncthreads();
  const NRdSm<T> rr{sb, W, oa, ob};
  for (int t = tid; t < (FT / 2) * (FT / 2); t += nt) {
    const int I = i0 / 2 + t % (FT / 2), J = j0 / 2 + t / (FT / 2);
    if (I < nc && J < mc) Bc[c * ldc + (long)J * nc + I] = restrict_node_at<T>(rr, I, J);
  }
  for (int t = tid; t < FT * FT; t += nt) {
    const int i = i0 + t % FT, j = j0 + t / FT;
    if (i < L.n && j < L.m) Xs[c * lds + (long)j * L.n + i] = sx[(lo + t / FT) * W + lo + t % FT];
  }
}

template <class T, int FT>
__global__ void __launch_bounds__(kFineMaxThreads) k_node_up(Lvl<T> L, int nc, int mc, const double* ph, int cpg,
                                                          const cx<T>* __restrict__ B, long ldb,
                                                          const cx<T>* __restrict__ Xs, long lds,
                                                          const cx<T>* __restrict__ Xc, long ldc,
                                                          cx<T>* __restrict__ X, long ldx, int nu) {
  extern __shared__ float4 fine_sm[];
  // step s works on the tile widened by 4 nu - 1 - s rings and reads one ring further;
  // the coarse nodes the region's prolongation reads (origin (oa/2, ob/2), W/2 + 1
  // per side, oa and ob even) are staged first
  const int lo = 4 * nu, W = FT + 8 * nu, Wc = W / 2 + 1;
  cx<T>* sx = reinterpret_cast<cx<T>*>(fine_sm);
  cx<T>* sb = sx + W * W;
  cx<T>* sc = sb + W * W;
  const int c = blockIdx.z, tid = threadIdx.x, nt = blockDim.x;
  const int i0 = blockIdx.x * FT, j0 = blockIdx.y * FT, oa = i0 - lo, ob = j0 - lo;
  const Ph<T> p = load_ph<T>(ph, c / cpg);
  const cx<T>* b = B + c * ldb;
  const cx<T>* xs = Xs + c * lds;
  const cx<T>* xc = Xc + c * ldc;
  stage_region<T>(xc, oa >> 1, ob >> 1, Wc, nc, mc, p, sc);
  stage_region<T>(b, oa, ob, W, L.n, L.m, p, sb);
  stage_region<T>(xs, oa, ob, W, L.n, L.m, p, sx);
  __syncthreads();
  const NRdSm<T> rc{sc, Wc, oa >> 1, ob >> 1};
  {
    const float inv = 1.0f / (float)W;
    for (int t = tid; t < W * W; t += nt) {
      int u, v;
      split_index(t, W, inv, u, v);
      sx[t] = sx[t] + prolong_node_at<T>(rc, oa + u, ob + v);
    }
  }
  __syncthreads();
  const NRdSm<T> rs{sx, W, oa, ob};
  for (int it = 0; it < nu; ++it)
    for (int q = 3; q >= 0; --q) {
      const int e = 4 * nu - 1 - (4 * it + 3 - q);
      for_colour<T>(q, lo - e, lo + FT + e, oa, ob, [&](int a, int bb) {
        const int k = bb * W + a;
        const cx<T> res = sb[k] - P_at<T>(rs, L, oa + a, ob + bb);
        sx[k] = sx[k] + (T(1) / P_diag<T>(L)) * res;
      });
      __syncthreads();
    }
  for (int t = tid; t < FT * FT; t += nt) {
    const int i = i0 + t % FT, j = j0 + t / FT;
    if (i < L.n && j < L.m) X[c * ldx + (long)j * L.n + i] = sx[(lo + t / FT) * W + lo + t % FT];
  }
}


// ---- register-blocked variants (FP32, one sweep per side) ---------------------
// The same two steps with the work split by 2 x 2 node blocks.  Region node (a, b)
// lives in shared memory in colour plane (a & 1) + 2 (b & 1), at position
// (b >> 1) H + (a >> 1) of that plane (H = W / 2; the region origins are even, so a
// plane holds one colour).  Thread t owns the blocks t, t + NT, ... of the H x H
// block grid: it keeps their four node values and right-hand sides in registers and
// writes each value it updates to its plane.  A colour update then takes four of
// its nine stencil values from the thread's own registers (the node itself and the
// three other colours of its block) and the other five from the planes, where
// consecutive threads read consecutive words; the right-hand side never enters
// shared memory.  The colour order, the rings each step covers and every node's
// expression are those of k_node_down / k_node_up, on the same operands, so the
// variants give the same results bit for bit.

// reader of the 2 x 2 block whose even node is region node (2 bu, 2 bv); offsets
// (i, j) count from that node, the block's own nodes come from registers
template <class T> struct BlkRd {
  const cx<T>* s;  // four planes of P = H * H values
  int H, P, bu, bv;
  cx<T> r00, r10, r01, r11;
  __device__ __forceinline__ cx<T> v(int i, int j) const {
    if (i == 0 && j == 0) return r00;
    if (i == 1 && j == 0) return r10;
    if (i == 0 && j == 1) return r01;
    if (i == 1 && j == 1) return r11;
    return s[((i & 1) | ((j & 1) << 1)) * P + (bv + (j >> 1)) * H + bu + (i >> 1)];
  }
};
// the four coarse values one fine 2 x 2 block is prolongated from, (I, J) in {0, 1}^2
template <class T> struct QuadRd {
  cx<T> c00, c10, c01, c11;
  __device__ __forceinline__ cx<T> v(int I, int J) const { return J ? (I ? c11 : c01) : (I ? c10 : c00); }
};

// Node (i, j) of a field on an n x m level: a direct read when the caller knows the
// region lies inside the level, else through the Bloch extension (the same value).
template <class T>
__device__ __forceinline__ cx<T> node_val(const cx<T>* __restrict__ f, bool in, int i, int j, int n, int m,
                                          const Ph<T>& p) {
  return in ? f[(long)j * n + i] : gread<T>(f, i, j, n, m, p);
}

template <int FT, int NT, int NU> struct RbDown {
  static constexpr int lo = 4 * NU + 2;      // k_node_down's margin below the tile
  static constexpr int W = FT + 8 * NU + 4;  // its region plus one unread ring (even)
  static constexpr int H = W / 2, P = H * H, KB = (P + NT - 1) / NT;
  static constexpr size_t smem = 2 * (size_t)W * W * sizeof(float2);  // x and the residual
  // even tile sides, margin and width: region coordinates keep the parity (colour) of
  // the level's, and the region splits into whole 2 x 2 blocks
  static_assert(FT % 2 == 0 && lo % 2 == 0 && W % 2 == 0, "register-blocked down step: odd tile geometry");
};
template <int FT, int NT, int NU> struct RbUp {
  static constexpr int lo = 4 * NU, W = FT + 8 * NU;
  static constexpr int H = W / 2, P = H * H, KB = (P + NT - 1) / NT;
  static constexpr size_t smem = (size_t)W * W * sizeof(float2);  // x
  static_assert(FT % 2 == 0 && lo % 2 == 0 && W % 2 == 0, "register-blocked up step: odd tile geometry");
};

template <int FT, int NT, int NU>
__global__ void __launch_bounds__(NT) k_node_down_rb(Lvl<float> L, int nc, int mc, const double* ph, int cpg,
                                                    const float2* __restrict__ B, long ldb,
                                                    const float2* __restrict__ X0, long ld0,
                                                    float2* __restrict__ Xs, long lds, float2* __restrict__ Bc,
                                                    long ldc) {
  using T = float;
  using S = RbDown<FT, NT, NU>;
  constexpr int lo = S::lo, W = S::W, H = S::H, P = S::P, KB = S::KB;
  extern __shared__ float4 fine_sm[];
  cx<T>* sx = reinterpret_cast<cx<T>*>(fine_sm);
  cx<T>* sr = sx + 4 * P;
  const int c = blockIdx.z, tid = threadIdx.x;
  const int i0 = blockIdx.x * FT, j0 = blockIdx.y * FT, oa = i0 - lo, ob = j0 - lo;
  const Ph<T> p = load_ph<T>(ph, c / cpg);
  const cx<T>* b = B + c * ldb;
  const cx<T>* x0 = X0 ? X0 + c * ld0 : nullptr;
  const bool in = oa >= 0 && ob >= 0 && oa + W <= L.n && ob + W <= L.m;
  const T inv = T(1) / P_diag<T>(L);
  int bu[KB], bv[KB];
  cx<T> xr[KB][4], br[KB][4];
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    const int t = tid + k * NT;
    bu[k] = t % H;
    bv[k] = t / H;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      xr[k][q] = czero<T>();
      br[k][q] = czero<T>();
      if (t < P) {
        const int a = oa + 2 * bu[k] + (q & 1), bb = ob + 2 * bv[k] + (q >> 1);
        br[k][q] = node_val<T>(b, in, a, bb, L.n, L.m, p);
        // a cycle that continues from an iterate starts the smoothing from it
        if (x0) xr[k][q] = node_val<T>(x0, in, a, bb, L.n, L.m, p);
        sx[q * P + t] = xr[k][q];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < NU; ++it)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int e = 4 * NU - 1 - (4 * it + q), r0 = lo - 2 - e, r1 = lo + FT + 1 + e;
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        const int t = tid + k * NT, a = 2 * bu[k] + (q & 1), bb = 2 * bv[k] + (q >> 1);
        if (t < P && a >= r0 && a < r1 && bb >= r0 && bb < r1) {
          const BlkRd<T> rd{sx, H, P, bu[k], bv[k], xr[k][0], xr[k][1], xr[k][2], xr[k][3]};
          const cx<T> res = br[k][q] - P_at<T>(rd, L, q & 1, q >> 1);
          xr[k][q] = xr[k][q] + inv * res;
          sx[q * P + t] = xr[k][q];
        }
      }
      __syncthreads();
    }
  // residual b - P x (over b in the registers) on the nodes [lo - 1, lo + FT - 1] the
  // restriction reads; the even node of a block is read by its own block only
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    const int t = tid + k * NT;
    if (t < P) {
      const BlkRd<T> rd{sx, H, P, bu[k], bv[k], xr[k][0], xr[k][1], xr[k][2], xr[k][3]};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int a = 2 * bu[k] + (q & 1), bb = 2 * bv[k] + (q >> 1);
        if (a >= lo - 1 && a <= lo + FT - 1 && bb >= lo - 1 && bb <= lo + FT - 1) {
          cx<T> y = T(-1) * P_at<T>(rd, L, q & 1, q >> 1);
          y = y + T(1) * br[k][q];
          br[k][q] = y;
          if (q) sr[q * P + t] = y;
        }
      }
    }
  }
  __syncthreads();
  // restriction to the coarse node on each tile block's even node; the tile's x
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    const int t = tid + k * NT, tu = bu[k] - lo / 2, tv = bv[k] - lo / 2;
    if (t < P && tu >= 0 && tu < FT / 2 && tv >= 0 && tv < FT / 2) {
      const BlkRd<T> rr{sr, H, P, bu[k], bv[k], br[k][0], br[k][1], br[k][2], br[k][3]};
      const int I = i0 / 2 + tu, J = j0 / 2 + tv;
      if (I < nc && J < mc) Bc[c * ldc + (long)J * nc + I] = restrict_node_at<T>(rr, 0, 0);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + 2 * tu + (q & 1), j = j0 + 2 * tv + (q >> 1);
        if (i < L.n && j < L.m) Xs[c * lds + (long)j * L.n + i] = xr[k][q];
      }
    }
  }
}

template <int FT, int NT, int NU>
__global__ void __launch_bounds__(NT) k_node_up_rb(Lvl<float> L, int nc, int mc, const double* ph, int cpg,
                                                  const float2* __restrict__ B, long ldb,
                                                  const float2* __restrict__ Xs, long lds,
                                                  const float2* __restrict__ Xc, long ldc, float2* __restrict__ X,
                                                  long ldx) {
  using T = float;
  using S = RbUp<FT, NT, NU>;
  constexpr int lo = S::lo, W = S::W, H = S::H, P = S::P, KB = S::KB;
  extern __shared__ float4 fine_sm[];
  cx<T>* sx = reinterpret_cast<cx<T>*>(fine_sm);
  const int c = blockIdx.z, tid = threadIdx.x;
  const int i0 = blockIdx.x * FT, j0 = blockIdx.y * FT, oa = i0 - lo, ob = j0 - lo, ca = oa >> 1, cb = ob >> 1;
  const Ph<T> p = load_ph<T>(ph, c / cpg);
  const cx<T>* b = B + c * ldb;
  const cx<T>* xs = Xs + c * lds;
  const cx<T>* xc = Xc + c * ldc;
  const bool in = oa >= 0 && ob >= 0 && oa + W <= L.n && ob + W <= L.m;
  const bool cin = ca >= 0 && cb >= 0 && ca + H + 1 <= nc && cb + H + 1 <= mc;
  const T inv = T(1) / P_diag<T>(L);
  int bu[KB], bv[KB];
  cx<T> xr[KB][4], br[KB][4];
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    const int t = tid + k * NT;
    bu[k] = t % H;
    bv[k] = t / H;
    QuadRd<T> cq{czero<T>(), czero<T>(), czero<T>(), czero<T>()};
    if (t < P) {
      const int I = ca + bu[k], J = cb + bv[k];
      cq = QuadRd<T>{node_val<T>(xc, cin, I, J, nc, mc, p), node_val<T>(xc, cin, I + 1, J, nc, mc, p),
                     node_val<T>(xc, cin, I, J + 1, nc, mc, p), node_val<T>(xc, cin, I + 1, J + 1, nc, mc, p)};
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      xr[k][q] = czero<T>();
      br[k][q] = czero<T>();
      if (t < P) {
        const int a = oa + 2 * bu[k] + (q & 1), bb = ob + 2 * bv[k] + (q >> 1);
        br[k][q] = node_val<T>(b, in, a, bb, L.n, L.m, p);
        xr[k][q] = node_val<T>(xs, in, a, bb, L.n, L.m, p) + prolong_node_at<T>(cq, q & 1, q >> 1);
        sx[q * P + t] = xr[k][q];
      }
    }
  }
  __syncthreads();
#pragma unroll
  for (int it = 0; it < NU; ++it)
#pragma unroll
    for (int q = 3; q >= 0; --q) {
      const int e = 4 * NU - 1 - (4 * it + 3 - q), r0 = lo - e, r1 = lo + FT + e;
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        const int t = tid + k * NT, a = 2 * bu[k] + (q & 1), bb = 2 * bv[k] + (q >> 1);
        if (t < P && a >= r0 && a < r1 && bb >= r0 && bb < r1) {
          const BlkRd<T> rd{sx, H, P, bu[k], bv[k], xr[k][0], xr[k][1], xr[k][2], xr[k][3]};
          const cx<T> res = br[k][q] - P_at<T>(rd, L, q & 1, q >> 1);
          xr[k][q] = xr[k][q] + inv * res;
          sx[q * P + t] = xr[k][q];
        }
      }
      __syncthreads();
    }
#pragma unroll
  for (int k = 0; k < KB; ++k) {
    const int t = tid + k * NT, tu = bu[k] - lo / 2, tv = bv[k] - lo / 2;
    if (t < P && tu >= 0 && tu < FT / 2 && tv >= 0 && tv < FT / 2)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = i0 + 2 * tu + (q & 1), j = j0 + 2 * tv + (q >> 1);
        if (i < L.n && j < L.m) X[c * ldx + (long)j * L.n + i] = xr[k][q];
      }
  }
}

}  // namespace pbs
