// Block Gram matrices on the tensor cores (the mixed policy's Gram, Section 4).
//
// GM = S^* M S and GA = (C S)^* W (C S) are sums over the mesh of products of
// values that need about 2^-47 relative accuracy (the double-float kernel's level).
// Written with real operands, X = [Re u | Im u] and Y = [Re v | Im v] (u = S,
// v = M S for GM; u = C S, v = W C S for GA), both products are P = X^T Y over
// the rows (edges, or cells):
//   G_re[a][b] = P[a][b] + P[h+a][h+b],   G_im[a][b] = P[a][h+b] - P[h+a][b]
// (h = the padded half width).  P is evaluated with the splitting of Ozaki,
// Ogita, Oishi and Rump (2012): every value, scaled by a power of two 2^-e
// shared by its column over the chunk's rows, is written as a sum of six
// bfloat16 slices, x = sum_i X_i, X_i = x_i 2^-8(i+1) with integer digits x_i
// (|x_0| <= 256, |x_i| <= 128 after rounding to nearest), so that every slice
// product X_i Y_j is exact in FP32 and a sum of 64 of them stays exact as long as
// i + j <= 2.  The tensor cores (mma.sync m16n8k16, bf16 in, FP32 accumulate)
// form the 21 slice products with i + j <= 5: the leading groups (i + j = 0, 1,
// 2) in exact FP32 accumulators, the rest (whose rounding is 2^-24 of terms
// already 2^-24 smaller) in one plain FP32 accumulator, all folded into
// double-float sums after every chunk.  The dropped products (i + j >= 6)
// and the slicing leave about 2^-48 of the scaled magnitudes per term.
//
// The scale of a column is a power of two above its largest magnitude over the
// chunk's rows, so each value keeps about 48 bits relative to its chunk's largest
// one (as the double-float kernel keeps 48 bits of every value); the curls of a
// smooth field are far smaller than the field itself, and a scale taken from a
// bound such as 4 max|u| would cost them a dozen bits.
//
// A block takes one product (GM or GA) of one group over a contiguous range of
// nodes, staging chunks of 16 nodes (the stencils M s and C s in double-float, as
// in the double-float kernel), then their slices, in shared memory; each warp multiplies
// one 16-row strip of P against up to NT 8-column tiles.  Tiles holding only
// entries below the diagonal of each of the four h x h blocks of P are skipped
// (the Gram matrices are Hermitian).
#include <cuda_bf16.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "mgpoint.cuh"

namespace pbs {
namespace {

constexpr int kTcNodes = 16;               // nodes per staged chunk
constexpr int kTcSlices = 6;               // bf16 slices per value
constexpr int kTcMaxHalf = 48;             // padded half width h (q <= 48)
constexpr int kTcMaxTasks = 16;            // warps per block
constexpr int kTcRowsGM = 2 * kTcNodes;    // GM rows per chunk: x-edge and y-edge of every node
constexpr int kTcStride = kTcRowsGM + 8;   // shared row stride (bf16): 80 bytes, conflict-free ldmatrix

// One warp's share of P: rows [16 mt, 16 mt + 16) and the 8-column tiles nt[0..nn).
constexpr int kTcMaxNT = 4;
struct TcTask {
  unsigned char mt, nn, nt[kTcMaxNT];
};
struct TcTasks {
  TcTask t[kTcMaxTasks];
  int count;
};

__device__ __forceinline__ const double2* tc_col(const Roles& R, int g, int a) {
  const int r = a / R.pr;
  const double2* base = r == 0 ? R.b[0] : (r == 1 ? R.b[1] : R.b[2]);
  return base + ((long)g * R.pr + a % R.pr) * R.ld;
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const unsigned (&a)[4], unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}
__device__ __forceinline__ void ldsm_x4(unsigned (&r)[4], const void* p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(s));
}
__device__ __forceinline__ void ldsm_x2(unsigned& r0, unsigned& r1, const void* p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x2.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(s));
}

// 2^k as a float (k within the normal range), exact
__device__ __forceinline__ float pow2f(int k) { return __int_as_float((k + 127) << 23); }

// Six bf16 slices of a double-float value v with |v| < 2^e: slice i holds
// x_i 2^(e - 8(i+1)) relative to the unscaled value; stored without the 2^e
// (which the block applies to P at the end).
__device__ __forceinline__ void split_store(df v, int e, __nv_bfloat16* dst, int slice_stride) {
  const float sc = pow2f(8 - e);  // scaled by 2^-e, times 256 for the first digit
  float hi = v.hi * sc, lo = v.lo * sc;
#pragma unroll
  for (int i = 0; i < kTcSlices; ++i) {
    const float d = rintf(hi);
    // true slice value d 2^-8(i+1): exact in bf16 (|d| <= 256 is an 8-bit integer times a power of two)
    dst[i * slice_stride] = __float2bfloat16_rn(d * pow2f(-8 * (i + 1)));
    const df r = quick_two_sum(hi - d, lo);  // hi - d is exact
    hi = r.hi * 256.0f;
    lo = r.lo * 256.0f;
  }
}

// exponent e with |v| < 2^e for every double-float v whose leading part is at most
// m in magnitude (|v| <= m (1 + 2^-23)); 0 for an all-zero column.  Clamped so that
// the float scalings by 2^(8-e) and 2^(ex+ey) stay in range.
__device__ __forceinline__ int chunk_exp(float m) {
  if (!(m > 0.0f)) return 0;
  int e;
  frexpf(m * 1.0000002f, &e);
  return max(-60, min(60, e));
}

// grid: (npart, ngroups, 2); blockIdx.z = 0: GM, 1: GA.  H = padded half width.
// Every chunk is scaled on its own: the largest magnitude of each operand column over
// the chunk's rows sets its power of two, so the slices carry the chunk's own values
// to 2^-48 (the accuracy of the double-float kernel's terms), and the chunk's slice
// products are folded into the double-float sums with that chunk's scales.
template <int H, int NT>
__global__ void __launch_bounds__(NT == 3 ? kTcMaxTasks * 32 : 384) k_gram_tc(Lvl<df> L, WtsDF w, const double* ph,
                                                                            Roles roles, int q, TcTasks tasks,
                                                                            double2* __restrict__ part, int npart) {
  extern __shared__ float4 tc_sm[];
  constexpr int W2 = 2 * H;           // real columns of X and Y
  constexpr int SL = W2 * kTcStride;  // bf16 elements of one slice of one operand
  __nv_bfloat16* sX = reinterpret_cast<__nv_bfloat16*>(tc_sm);  // [slice][W2][stride]
  __nv_bfloat16* sY = sX + kTcSlices * SL;
  dcx* su = reinterpret_cast<dcx*>(sY + kTcSlices * SL);  // [a][row] chunk values (X operand)
  dcx* sv = su + H * kTcRowsGM;                            // [a][row] (Y operand)
  __shared__ int ex[kTcMaxHalf], ey[kTcMaxHalf];
  const int g = blockIdx.y, prod = blockIdx.z;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const Ph<df> p = load_ph<df>(ph, g);
  const long N = (long)L.n * L.m;
  const long nchunks = (N + kTcNodes - 1) / kTcNodes;
  const long per = (nchunks + npart - 1) / npart;
  const long c_begin = blockIdx.x * per, c_end = min(nchunks, c_begin + per);
  const long r_end = min(N, c_end * kTcNodes);
  const int rows = prod == 0 ? kTcRowsGM : kTcNodes;  // rows per chunk
  // padding columns (a >= q) stay zero in every slice
  for (int t = tid; t < 2 * kTcSlices * SL; t += nt) sX[t] = __float2bfloat16_rn(0.0f);

  const bool active = warp < tasks.count;
  TcTask tk{0, 0, {0, 0, 0, 0}};
  if (active) tk = tasks.t[warp];
  df sum[NT][4];  // P entries of the warp's tiles
#pragma unroll
  for (int t = 0; t < NT; ++t)
#pragma unroll
    for (int k = 0; k < 4; ++k) sum[t][k] = df_zero();

  for (long ch = c_begin; ch < c_end; ++ch) {
    const long r0 = ch * kTcNodes;
    __syncthreads();  // the previous chunk's slices and scales are no longer read
    // 1. the chunk's operand values (stencils in double-float)
    for (int t = tid; t < q * kTcNodes; t += nt) {
      const int a = t / kTcNodes, rr = t % kTcNodes;
      const long node = r0 + rr;
      const dcx z = dcx_make(df_zero(), df_zero());
      dcx u0 = z, u1 = z, v0 = z, v1 = z;
      if (node < r_end) {
        const int i = int(node % L.n), j = int(node / L.n);
        const ERdD<df> rd{tc_col(roles, g, a), L.n, L.m, p};
        if (prod == 0) {
          u0 = rd.x(i, j);
          u1 = rd.y(i, j);
          v0 = M_x<df>(rd, L, i, j);
          v1 = M_y<df>(rd, L, i, j);
        } else {
          u0 = curl_at<df>(rd, i, j);
          v0 = w(i, j) * u0;
        }
      }
      if (prod == 0) {
        su[a * kTcRowsGM + 2 * rr] = u0;
        su[a * kTcRowsGM + 2 * rr + 1] = u1;
        sv[a * kTcRowsGM + 2 * rr] = v0;
        sv[a * kTcRowsGM + 2 * rr + 1] = v1;
      } else {
        su[a * kTcRowsGM + rr] = u0;
        sv[a * kTcRowsGM + rr] = v0;
      }
    }
    __syncthreads();
    // 2. column scales of the chunk: one warp per operand column (rows <= 32 = lanes)
    for (int c = warp; c < 2 * q; c += nt / 32) {
      const dcx* col = (c < q ? su : sv) + (c % q) * kTcRowsGM;
      float m = 0.0f;
      if (lane < rows) m = fmaxf(fabsf(col[lane].x.hi), fabsf(col[lane].y.hi));
      for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
      if (lane == 0) (c < q ? ex : ey)[c % q] = chunk_exp(m);
    }
    for (int a = q + tid; a < H; a += nt) {
      ex[a] = 0;
      ey[a] = 0;
    }
    __syncthreads();
    // 3. slices
    for (int t = tid; t < q * rows; t += nt) {
      const int a = t / rows, r = t % rows;
      const dcx u = su[a * kTcRowsGM + r], v = sv[a * kTcRowsGM + r];
      split_store(u.x, ex[a], sX + a * kTcStride + r, SL);
      split_store(u.y, ex[a], sX + (H + a) * kTcStride + r, SL);
      split_store(v.x, ey[a], sY + a * kTcStride + r, SL);
      split_store(v.y, ey[a], sY + (H + a) * kTcStride + r, SL);
    }
    __syncthreads();
    // 4. slice products on the tensor cores, folded with the chunk's scales
    if (active) {
      float acc[4][NT][4];  // [group: i+j = 0, 1, 2, >= 3][tile][fragment]
#pragma unroll
      for (int s2 = 0; s2 < 4; ++s2)
#pragma unroll
        for (int t = 0; t < NT; ++t)
#pragma unroll
          for (int k = 0; k < 4; ++k) acc[s2][t][k] = 0.0f;
      for (int k0 = 0; k0 < rows; k0 += 16) {
        unsigned A[kTcSlices][4];
#pragma unroll
        for (int i = 0; i < kTcSlices; ++i)
          ldsm_x4(A[i], sX + i * SL + (16 * tk.mt + (lane & 15)) * kTcStride + k0 + (lane >> 4) * 8);
#pragma unroll
        for (int j = 0; j < kTcSlices; ++j) {
#pragma unroll
          for (int t = 0; t < NT; ++t) {
            if (t >= tk.nn) break;
            unsigned b0, b1;
            ldsm_x2(b0, b1, sY + j * SL + (8 * tk.nt[t] + (lane & 7)) * kTcStride + k0 + ((lane >> 3) & 1) * 8);
#pragma unroll
            for (int i = 0; i + j < kTcSlices; ++i) {
              const int grp = i + j < 3 ? i + j : 3;
              mma_bf16(acc[grp][t], A[i], b0, b1);
            }
          }
        }
      }
      // the groups i + j <= 2 are exact; the rest carries 2^-24 of its (2^-24 smaller) value
#pragma unroll
      for (int t = 0; t < NT; ++t) {
        if (t >= tk.nn) break;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int row = 16 * tk.mt + (lane >> 2) + (k >= 2 ? 8 : 0);
          const int col = 8 * tk.nt[t] + 2 * (lane & 3) + (k & 1);
          const float sc = pow2f(ex[row % H] + ey[col % H]);
#pragma unroll
          for (int s2 = 0; s2 < 4; ++s2) sum[t][k] = sum[t][k] + df_make(acc[s2][t][k] * sc, 0.0f);
        }
      }
    }
  }
  __syncthreads();
  // 5. P in shared memory as FP64, then the partial sums
  double* Ps = reinterpret_cast<double*>(tc_sm);  // [W2][W2]
  if (active) {
#pragma unroll
    for (int t = 0; t < NT; ++t) {
      if (t >= tk.nn) break;
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        const int row = 16 * tk.mt + (lane >> 2) + (k >= 2 ? 8 : 0);
        const int col = 8 * tk.nt[t] + 2 * (lane & 3) + (k & 1);
        Ps[row * W2 + col] = df_to(sum[t][k]);
      }
    }
  }
  __syncthreads();
  const int ne = q * (q + 1) / 2;
  double2* pm = part + ((long)g * npart + blockIdx.x) * 2 * ne + (prod == 0 ? 0 : ne);
  for (int e = tid; e < ne; e += nt) {
    int b = int((sqrtf(8.0f * e + 1.0f) - 1.0f) * 0.5f);
    while ((b + 1) * (b + 2) / 2 <= e) ++b;
    while (b * (b + 1) / 2 > e) --b;
    const int a = e - b * (b + 1) / 2;
    const double re = Ps[a * W2 + b] + Ps[(H + a) * W2 + H + b];
    const double im = Ps[a * W2 + H + b] - Ps[(H + a) * W2 + b];
    pm[e] = make_double2(re, im);
  }
}

// Warp tasks for a padded half width h: the 16-row strips of P and, per strip, the
// 8-column tiles holding entries a <= b (a < q, b < q) of a block.
TcTasks make_tasks(int h, int q, int per_task) {
  TcTasks T{};
  const int w2 = 2 * h;
  for (int mt = 0; mt < w2 / 16; ++mt) {
    const int a0 = (16 * mt) % h;
    if (a0 >= q) continue;
    std::vector<int> cols;
    for (int ntl = 0; ntl < w2 / 8; ++ntl) {
      const int b0 = (8 * ntl) % h;
      if (b0 >= q || a0 > b0 + 7) continue;
      cols.push_back(ntl);
    }
    for (size_t s = 0; s < cols.size(); s += per_task) {
      if (T.count >= kTcMaxTasks) fail(PBS_EINVAL, "tensor-core Gram: too many tiles");
      TcTask& t = T.t[T.count++];
      t.mt = (unsigned char)mt;
      t.nn = (unsigned char)std::min<size_t>(per_task, cols.size() - s);
      for (int u = 0; u < t.nn; ++u) t.nt[u] = (unsigned char)cols[s + u];
    }
  }
  return T;
}

template <int H> size_t tc_smem() {
  const size_t slices = 2ull * kTcSlices * 2 * H * kTcStride * sizeof(__nv_bfloat16);
  const size_t stage = 2ull * H * kTcRowsGM * sizeof(dcx);
  const size_t pmat = (size_t)(2 * H) * (2 * H) * sizeof(double);
  return std::max(slices + stage, pmat);
}

template <int H, int NT>
void launch_tc(const Level& L, const double* d_ph, Roles roles, int q, int ngroups, int npart, double2* d_partials,
               cudaStream_t s) {
  static PerDeviceOnce once;
  once([] {
    PBS_CUDA(cudaFuncSetAttribute(k_gram_tc<H, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)tc_smem<H>()));
  });
  const TcTasks tasks = make_tasks(H, q, NT);
  k_gram_tc<H, NT><<<dim3(npart, ngroups, 2), 32 * tasks.count, tc_smem<H>(), s>>>(
      L.lvl<df>(), L.wts_df(), d_ph, roles, q, tasks, d_partials, npart);
}

}  // namespace

bool gram_tc_supported(int q) { return q >= 1 && q <= kTcMaxHalf; }

void gram_tc(const Level& L, const double* d_ph, Roles roles, int q, int ngroups, int npart, double2* d_partials,
             cudaStream_t s) {
  if (q <= 16) launch_tc<16, 3>(L, d_ph, roles, q, ngroups, npart, d_partials, s);
  else if (q <= 32) launch_tc<32, 3>(L, d_ph, roles, q, ngroups, npart, d_partials, s);
  else if (q <= 48) launch_tc<48, 4>(L, d_ph, roles, q, ngroups, npart, d_partials, s);
  else fail(PBS_EINVAL, "tensor-core Gram: q > 48");
}

}  // namespace pbs
