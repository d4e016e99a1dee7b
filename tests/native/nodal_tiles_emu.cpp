// Host emulation of the tiled nodal multigrid kernels (csrc/nodal_tiles.cuh).
//
// The kernels are compiled here by the host compiler as plain C++ (the CUDA
// qualifiers expand to nothing outside nvcc) and run CTA by CTA: every CUDA
// thread is a host thread, and the threads of a CTA take turns in a fixed order,
// each running from one barrier to the next while the others wait.  A kernel
// whose threads never read, between two barriers, a shared-memory word that
// another thread writes there gives the same result in every order; the checks
// below run the register-blocked kernels in ascending and descending thread
// order.  Dynamic shared memory is one static array: before each CTA the part
// beyond the launch's size is poisoned for AddressSanitizer (this file is built
// with -fsanitize=address) and the rest is filled with NaN, so a read past the
// launch's shared memory stops the run and a read of a word no thread wrote shows
// up as NaN in the results.  Every device array is a heap block of its exact size.
//
// Checked, bit for bit: k_node_down_rb against k_node_down and k_node_up_rb
// against k_node_up (one sweep per side, FP32) on several levels, Bloch vectors
// and tile shapes.  Checked against whole-level colour sweeps: k_node_down and
// k_node_up with one to three sweeps per side in FP32 and FP64 (bit for bit on
// tiles whose region lies inside the level, to rounding elsewhere).  Prints "ok"
// on success.
#include <cuda_runtime.h>
#include <sched.h>
#include <sanitizer/asan_interface.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <random>
#include <semaphore>
#include <thread>
#include <vector>

// ---- stand-ins for the device built-ins the headers name ---------------------
// IEEE single-precision operations with round-to-nearest (the host's arithmetic);
// the nodal kernels call none of them, the headers only need them declared.
inline float __fadd_rn(float a, float b) { return a + b; }
inline float __fsub_rn(float a, float b) { return a - b; }
inline float __fmul_rn(float a, float b) { return a * b; }
inline float __fmaf_rn(float a, float b, float c) { return std::fma(a, b, c); }
inline float __fdiv_rn(float a, float b) { return a / b; }
inline float __fsqrt_rn(float a) { return std::sqrt(a); }
inline int __clz(int x) { return x == 0 ? 32 : __builtin_clz((unsigned)x); }
inline void __syncwarp(unsigned = 0xffffffffu) {}
template <class V> V __shfl_xor_sync(unsigned, V v, int) { return v; }
inline long long __double_as_longlong(double d) {
  long long u;
  std::memcpy(&u, &d, sizeof u);
  return u;
}
inline double __longlong_as_double(long long u) {
  double d;
  std::memcpy(&d, &u, sizeof d);
  return d;
}
inline float __uint_as_float(unsigned u) {
  float f;
  std::memcpy(&f, &u, sizeof f);
  return f;
}
inline unsigned __float_as_uint(float f) {
  unsigned u;
  std::memcpy(&u, &f, sizeof u);
  return u;
}
#define __launch_bounds__(...)

// CUDA thread and block indices of the running emulated thread
thread_local uint3 threadIdx;
thread_local uint3 blockIdx;
thread_local dim3 blockDim;

// Turn-taking between the threads of one CTA: the thread holding the turn runs
// until its next barrier (or its end) and hands the turn to the next thread of
// the order; after the last one the first thread of the order runs again.
struct Turns {
  std::vector<int> order;
  std::vector<std::unique_ptr<std::binary_semaphore>> sem;
  size_t pos = 0;
  explicit Turns(std::vector<int> o) : order(std::move(o)) {
    for (size_t i = 0; i < order.size(); ++i) sem.emplace_back(new std::binary_semaphore(0));
  }
  void pass() {
    pos = (pos + 1) % order.size();
    sem[order[pos]]->release();
  }
};
thread_local Turns* tl_turns;
void __syncthreads() {
  tl_turns->pass();
  tl_turns->sem[threadIdx.x]->acquire();
}

namespace pbs {
constexpr size_t kEmuSmem = 232448;
alignas(16) float4 fine_sm[kEmuSmem / sizeof(float4)];
}  // namespace pbs

#include "nodal_tiles.cuh"

using namespace pbs;

// Run kernel body f on grid (gx, gy, gz) with nt threads per CTA and smem bytes of
// dynamic shared memory, the threads of a CTA taking turns in ascending (or, with
// reverse set, descending) order.  The same host threads run the CTAs one after
// the other: the end of a CTA is one more turn of every thread, and the first
// thread of the order resets the shared memory before each CTA.
void reset_smem(size_t smem) {
  char* base = reinterpret_cast<char*>(fine_sm);
  ASAN_UNPOISON_MEMORY_REGION(base, kEmuSmem);
  float* fs = reinterpret_cast<float*>(base);
  for (size_t i = 0; i < smem / sizeof(float); ++i) fs[i] = std::nanf("");
  ASAN_POISON_MEMORY_REGION(base + smem, kEmuSmem - smem);
}

template <class F>
void launch(int gx, int gy, int gz, int nt, size_t smem, bool reverse, F&& f) {
  if (smem > kEmuSmem) {
    std::fprintf(stderr, "shared memory %zu beyond the emulated %zu\n", smem, kEmuSmem);
    std::exit(1);
  }
  std::vector<int> order(nt);
  for (int t = 0; t < nt; ++t) order[t] = reverse ? nt - 1 - t : t;
  Turns turns(order);
  std::vector<std::thread> th;
  th.reserve(nt);
  for (int t = 0; t < nt; ++t)
    th.emplace_back([&, t] {
      threadIdx = make_uint3(t, 0, 0);
      blockDim = dim3(nt, 1, 1);
      tl_turns = &turns;
      turns.sem[t]->acquire();
      for (int z = 0; z < gz; ++z)
        for (int y = 0; y < gy; ++y)
          for (int x = 0; x < gx; ++x) {
            blockIdx = make_uint3(x, y, z);
            if (t == turns.order[0]) reset_smem(smem);
            f();
            __syncthreads();  // the CTA ends for every thread before the next one starts
          }
      turns.pass();
    });
  turns.sem[order[0]]->release();
  for (auto& t : th) t.join();
  ASAN_UNPOISON_MEMORY_REGION(reinterpret_cast<char*>(fine_sm), kEmuSmem);
}

// one case: an n x m level (coarse level n/2 x m/2), ncols columns in groups of cpg
// with their own Bloch phases
struct Case {
  int n, m, ncols, cpg;
  double a, b;
  std::vector<double> k;  // k1, k2 per group
  bool x0;                // the down step continues from an iterate
};

using Vec = std::vector<float2>;

Vec random_vec(size_t len, std::mt19937_64& g) {
  std::normal_distribution<float> d(0.0f, 1.0f);
  Vec v(len);
  for (auto& z : v) z = make_float2(d(g), d(g));
  return v;
}

bool same(const Vec& x, const Vec& y, const char* what, const Case& cs, int ft, int nt, bool rev) {
  for (size_t i = 0; i < x.size(); ++i) {
    if (!std::isfinite(x[i].x) || !std::isfinite(x[i].y) || std::memcmp(&x[i], &y[i], sizeof(float2)) != 0) {
      std::printf("MISMATCH %s n=%d m=%d ft=%d nt=%d reverse=%d x0=%d at %zu: (%.9g, %.9g) vs (%.9g, %.9g)\n", what,
                  cs.n, cs.m, ft, nt, (int)rev, (int)cs.x0, i, x[i].x, x[i].y, y[i].x, y[i].y);
      return false;
    }
  }
  return true;
}

template <int FT, int NT>
bool check_shape(const Case& cs) {
  constexpr int NU = 1;
  const int n = cs.n, m = cs.m, nc = n / 2, mc = m / 2;
  const long N = (long)n * m, Nc = (long)nc * mc;
  if (n < FT + 27 || m < FT + 27) return true;  // the tiled path's size condition
  const double h1 = cs.a / n, h2 = cs.b / m;
  const Lvl<float> L{n, m, (float)(h2 / h1), (float)(h1 / h2)};
  const int ngroups = (cs.ncols + cs.cpg - 1) / cs.cpg;
  std::vector<double> ph(4 * ngroups);
  for (int g = 0; g < ngroups; ++g) {
    const double ta = cs.k[2 * g] * cs.a, tb = cs.k[2 * g + 1] * cs.b;
    ph[4 * g + 0] = std::cos(ta);
    ph[4 * g + 1] = std::sin(ta);
    ph[4 * g + 2] = std::cos(tb);
    ph[4 * g + 3] = std::sin(tb);
  }
  std::mt19937_64 g(1234u + 7u * n + 13u * m + FT + NT);
  const Vec B = random_vec(N * cs.ncols, g), X0 = random_vec(N * cs.ncols, g), Xc = random_vec(Nc * cs.ncols, g);
  const float2* x0 = cs.x0 ? X0.data() : nullptr;
  const int gx = (n + FT - 1) / FT, gy = (m + FT - 1) / FT;

  // reference: the kernels of the GPU path (one thread order; they are checked on the GPU)
  Vec xs_ref(N * cs.ncols), bc_ref(Nc * cs.ncols), x_ref(N * cs.ncols);
  launch(gx, gy, cs.ncols, NT, 2 * (size_t)(FT + 11) * (FT + 11) * sizeof(float2), false, [&] {
    k_node_down<float, FT>(L, nc, mc, ph.data(), cs.cpg, B.data(), N, x0, N, xs_ref.data(), N, bc_ref.data(), Nc, NU);
  });
  launch(gx, gy, cs.ncols, NT, (2 * (size_t)(FT + 8) * (FT + 8) + (size_t)((FT + 8) / 2 + 1) * ((FT + 8) / 2 + 1)) *
                                   sizeof(float2),
         false, [&] {
           k_node_up<float, FT>(L, nc, mc, ph.data(), cs.cpg, B.data(), N, X0.data(), N, Xc.data(), Nc,
                                x_ref.data(), N, NU);
         });
  bool ok = true;
  for (int rev = 0; rev < 2; ++rev) {
    Vec xs(N * cs.ncols), bc(Nc * cs.ncols), x(N * cs.ncols);
    launch(gx, gy, cs.ncols, NT, RbDown<FT, NT, NU>::smem, rev, [&] {
      k_node_down_rb<FT, NT, NU>(L, nc, mc, ph.data(), cs.cpg, B.data(), N, x0, N, xs.data(), N, bc.data(), Nc);
    });
    launch(gx, gy, cs.ncols, NT, RbUp<FT, NT, NU>::smem, rev, [&] {
      k_node_up_rb<FT, NT, NU>(L, nc, mc, ph.data(), cs.cpg, B.data(), N, X0.data(), N, Xc.data(), Nc, x.data(), N);
    });
    ok = same(xs, xs_ref, "down x", cs, FT, NT, rev) && ok;
    ok = same(bc, bc_ref, "down coarse rhs", cs, FT, NT, rev) && ok;
    ok = same(x, x_ref, "up x", cs, FT, NT, rev) && ok;
  }
  return ok;
}

// ---- the plain tiled steps against whole-level sweeps, 1 to 3 sweeps per side ----
// The whole-level steps below run the same per-node expressions (P_at, the update,
// the residual, restrict_node_at, prolong_node_at) over the level in colour order,
// reading across the boundary through the Bloch extension.  A tile whose region
// lies inside the level reads no Bloch phase, so its outputs must agree bit for
// bit; elsewhere the tile's halo carries phase products of staged values instead
// of phase products of updated values, and the two agree to rounding.

template <class T> using CVec = std::vector<cx<T>>;

template <class T> CVec<T> random_cvec(size_t len, std::mt19937_64& g) {
  std::normal_distribution<double> d(0.0, 1.0);
  CVec<T> v(len);
  for (auto& z : v) z = mk<T>(T(d(g)), T(d(g)));
  return v;
}

template <class T> void level_sweep(const Lvl<T>& L, const Ph<T>& p, const cx<T>* b, cx<T>* x, int q) {
  const NRdPlain<T> r{x, L.n, L.m, p};
  for (int j = q >> 1; j < L.m; j += 2)
    for (int i = q & 1; i < L.n; i += 2) {
      const long e = (long)j * L.n + i;
      const cx<T> res = b[e] - P_at<T>(r, L, i, j);
      x[e] = x[e] + (T(1) / P_diag<T>(L)) * res;
    }
}

template <class T>
void level_down(const Lvl<T>& L, int nc, int mc, const Ph<T>& p, const cx<T>* b, const cx<T>* x0, int nu, cx<T>* x,
                cx<T>* bc) {
  const long N = (long)L.n * L.m;
  for (long e = 0; e < N; ++e) x[e] = x0 ? x0[e] : czero<T>();
  for (int it = 0; it < nu; ++it)
    for (int q = 0; q < 4; ++q) level_sweep<T>(L, p, b, x, q);
  CVec<T> r(N);
  const NRdPlain<T> rx{x, L.n, L.m, p};
  for (int j = 0; j < L.m; ++j)
    for (int i = 0; i < L.n; ++i) {
      const long e = (long)j * L.n + i;
      cx<T> y = T(-1) * P_at<T>(rx, L, i, j);
      y = y + T(1) * b[e];
      r[e] = y;
    }
  const NRdPlain<T> rr{r.data(), L.n, L.m, p};
  for (int J = 0; J < mc; ++J)
    for (int I = 0; I < nc; ++I) bc[(long)J * nc + I] = restrict_node_at<T>(rr, I, J);
}

template <class T>
void level_up(const Lvl<T>& L, int nc, int mc, const Ph<T>& p, const cx<T>* b, const cx<T>* xs, const cx<T>* xc,
              int nu, cx<T>* x) {
  const NRdPlain<T> rc{xc, nc, mc, p};
  for (int j = 0; j < L.m; ++j)
    for (int i = 0; i < L.n; ++i) {
      const long e = (long)j * L.n + i;
      x[e] = xs[e] + prolong_node_at<T>(rc, i, j);
    }
  for (int it = 0; it < nu; ++it)
    for (int q = 3; q >= 0; --q) level_sweep<T>(L, p, b, x, q);
}

// got against want on one column: bit for bit where inner(i, j), else within tol of
// the column's largest value
template <class T, class F>
bool agree(const cx<T>* got, const cx<T>* want, int n, int m, F&& inner, double tol, const char* what, int nu, int ft) {
  double mx = 0;
  long ninner = 0;
  for (long e = 0; e < (long)n * m; ++e) mx = std::max(mx, (double)std::hypot(want[e].x, want[e].y));
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < n; ++i) ninner += inner(i, j) ? 1 : 0;
  if (ninner == 0 || ninner == (long)n * m) {
    std::printf("CASE %s nu=%d ft=%d n=%d m=%d has %ld of %ld values on inner tiles (needs both kinds)\n", what,
                nu, ft, n, m, ninner, (long)n * m);
    return false;
  }
  for (int j = 0; j < m; ++j)
    for (int i = 0; i < n; ++i) {
      const long e = (long)j * n + i;
      const double d = std::hypot((double)got[e].x - want[e].x, (double)got[e].y - want[e].y);
      const bool bits = std::memcmp(&got[e], &want[e], sizeof(cx<T>)) == 0;
      if (!std::isfinite(d) || (inner(i, j) ? !bits : d > tol * mx)) {
        std::printf("MISMATCH %s (%s) nu=%d ft=%d n=%d m=%d at (%d, %d): diff %.3g of %.3g (inner %d)\n", what,
                    sizeof(T) == 4 ? "f32" : "f64", nu, ft, n, m, i, j, d, mx, (int)inner(i, j));
        return false;
      }
    }
  return true;
}

template <class T, int FT>
bool check_sweeps(int n, int m, double a, double b, double k1, double k2, bool with_x0, int nu) {
  constexpr int NT = 64;  // the plain kernels stride their loops by the block size
  const int nc = n / 2, mc = m / 2;
  const long N = (long)n * m, Nc = (long)nc * mc;
  const int Wd = FT + 8 * nu + 3, Wu = FT + 8 * nu, Wc = Wu / 2 + 1;
  const size_t smem_d = 2 * (size_t)Wd * Wd * sizeof(cx<T>);
  const size_t smem_u = (2 * (size_t)Wu * Wu + (size_t)Wc * Wc) * sizeof(cx<T>);
  if (n < FT + 27 || m < FT + 27 || smem_d > kEmuSmem || smem_u > kEmuSmem) return true;  // not offered
  const double h1 = a / n, h2 = b / m;
  const Lvl<T> L{n, m, T(h2 / h1), T(h1 / h2)};
  const double ph[4] = {std::cos(k1 * a), std::sin(k1 * a), std::cos(k2 * b), std::sin(k2 * b)};
  const Ph<T> p = load_ph<T>(ph, 0);
  std::mt19937_64 g(99u + 3u * n + 5u * m + FT + 17u * nu);
  const CVec<T> B = random_cvec<T>(N, g), X0 = random_cvec<T>(N, g), Xc = random_cvec<T>(Nc, g);
  const cx<T>* x0 = with_x0 ? X0.data() : nullptr;
  const int gx = (n + FT - 1) / FT, gy = (m + FT - 1) / FT;
  CVec<T> xs(N), bc(Nc), x(N), xs_w(N), bc_w(Nc), x_w(N);
  launch(gx, gy, 1, NT, smem_d, false, [&] {
    k_node_down<T, FT>(L, nc, mc, ph, 1, B.data(), N, x0, N, xs.data(), N, bc.data(), Nc, nu);
  });
  launch(gx, gy, 1, NT, smem_u, false, [&] {
    k_node_up<T, FT>(L, nc, mc, ph, 1, B.data(), N, X0.data(), N, Xc.data(), Nc, x.data(), N, nu);
  });
  level_down<T>(L, nc, mc, p, B.data(), x0, nu, xs_w.data(), bc_w.data());
  level_up<T>(L, nc, mc, p, B.data(), X0.data(), Xc.data(), nu, x_w.data());
  // a tile is inner when its region (down: margin 4 nu + 2 below, width Wd; up: margin
  // 4 nu, width Wu, and its coarse region) lies inside the level
  const auto down_in = [&](int i, int j) {
    const int oa = (i / FT) * FT - (4 * nu + 2), ob = (j / FT) * FT - (4 * nu + 2);
    return oa >= 0 && ob >= 0 && oa + Wd <= n && ob + Wd <= m;
  };
  const auto coarse_in = [&](int I, int J) { return down_in(2 * I, 2 * J); };
  const auto up_in = [&](int i, int j) {
    const int oa = (i / FT) * FT - 4 * nu, ob = (j / FT) * FT - 4 * nu;
    return oa >= 0 && ob >= 0 && oa + Wu <= n && ob + Wu <= m && oa / 2 + Wc <= nc && ob / 2 + Wc <= mc;
  };
  const double tol = sizeof(T) == 4 ? 2e-5 : 1e-13;
  bool ok = agree<T>(xs.data(), xs_w.data(), n, m, down_in, tol, "down x", nu, FT);
  ok = agree<T>(bc.data(), bc_w.data(), nc, mc, coarse_in, tol, "down coarse rhs", nu, FT) && ok;
  ok = agree<T>(x.data(), x_w.data(), n, m, up_in, tol, "up x", nu, FT) && ok;
  return ok;
}

int main() {
  // one core: the threads of a CTA run one at a time anyway, and a hand-over
  // between threads on one core is a plain context switch
  cpu_set_t one;
  CPU_ZERO(&one);
  if (sched_getaffinity(0, sizeof one, &one) == 0) {
    for (int cpu = 0; cpu < CPU_SETSIZE; ++cpu)
      if (CPU_ISSET(cpu, &one)) {
        CPU_ZERO(&one);
        CPU_SET(cpu, &one);
        sched_setaffinity(0, sizeof one, &one);
        break;
      }
  }
  const double pi = 3.14159265358979323846;
  std::vector<Case> cases = {
      // generic Bloch vectors (two groups), a rectangle with a partial last row of tiles
      {96, 64, 3, 2, 1.0, 0.5, {0.4, -1.3, 2.1, 0.7}, false},
      {96, 64, 3, 2, 1.0, 0.5, {0.4, -1.3, 2.1, 0.7}, true},
      // 64 x 64 tiles: a partial second column of tiles, Gamma and the zone corner
      {160, 96, 2, 1, 1.0, 0.75, {0.0, 0.0, pi, pi / 0.75}, true},
      {128, 128, 2, 2, 1.0, 1.0, {pi, pi, 0.0, 0.0}, false},
  };
  bool ok = true;
  for (const Case& cs : cases) {
    ok = check_shape<32, 256>(cs) && ok;
    ok = check_shape<32, 128>(cs) && ok;
    ok = check_shape<64, 512>(cs) && ok;
  }
  for (int nu = 1; nu <= 3; ++nu) {
    // levels with tiles on both sides of the boundary: 32 x 32 tiles on 128 x 96, 64 x 64
    // tiles on 192 x 160 (a partial last row), Gamma and generic Bloch vectors
    ok = check_sweeps<float, 32>(128, 96, 1.0, 0.5, 0.4, -1.3, true, nu) && ok;
    ok = check_sweeps<double, 32>(128, 96, 1.0, 0.5, 0.4, -1.3, false, nu) && ok;
    ok = check_sweeps<float, 64>(192, 160, 1.0, 1.0, 0.0, 0.0, false, nu) && ok;
    ok = check_sweeps<double, 64>(192, 160, 1.0, 1.0, 2.2, -0.9, true, nu) && ok;
  }
  std::printf(ok ? "ok\n" : "FAILED\n");
  return ok ? 0 : 1;
}
