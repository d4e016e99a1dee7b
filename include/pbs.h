/*
 * pbs.h - C ABI of the GB300 photonic band-structure library (libpbs.so).
 *
 * Computes the smallest non-zero eigenvalues of the 2-D curl-curl Maxwell
 * operator with Bloch boundary conditions, discretised with lowest-order
 * Nedelec edge elements on a regular n x m mesh of the periodic cell
 * [0,a] x [0,b] (Boerm, Koehl, Talebi, "Computing Maxwell eigenmodes with Bloch
 * boundary conditions", arXiv:2304.00337):
 *
 *   curl (1/eps) curl u = lambda u        (Section 1, eq. maxwell)
 *   u1(x1,b) = exp(i k2 b) u1(x1,0),  u2(a,x2) = exp(i k1 a) u2(0,x2)
 *                                         (Section 1, eq. bloch_boundary)
 *   A e = lambda M e                      (Section 1, eq. matrix; Section 3)
 *
 * All arithmetic runs in the library's CUDA kernels on one GPU; there is no
 * CPU fallback. Functions return 0 (PBS_OK) or a negative status; nothing is
 * thrown across the ABI. The library never frees caller memory. Host buffers
 * passed in are read or written only during the call. Device pointers are
 * plain CUDA device addresses on the context's device.
 *
 * Vector conventions (shared by every entry point):
 *  - complex numbers are interleaved (re, im) doubles (pbs_c64);
 *  - level l of the multigrid hierarchy has n_l = n >> l, m_l = m >> l,
 *    N_l = n_l * m_l cells (= nodes) and D_l = 2 N_l edges;
 *  - edge vectors: x-edges first, then y-edges; x-edge (i,j) is the segment
 *    [i h1,(i+1) h1] x {j h2} at index j*n_l + i, y-edge (i,j) is
 *    {i h1} x [j h2,(j+1) h2] at index N_l + j*n_l + i;  h1 = a/n_l, h2 = b/m_l;
 *    an edge coefficient is the line integral of the tangential component
 *    (Section 3, basis b_{x,i}, b_{y,i});
 *  - node (i,j) at (i h1, j h2) and cell (i,j) both have index j*n_l + i;
 *  - a block of `ncols` vectors is column-major: column c starts at c*len;
 *  - permittivity: one sample per finest-level cell, eps[j*n + i] > 0, taken
 *    at the cell centre (the reading of the paper's "standard quadrature" for
 *    a cellwise-constant 1/eps, Section 5).
 *
 * Environment (read once per process; none changes a result beyond rounding):
 *  - PBS_TUNE=0: no launch tuning, the first candidate of every choice;
 *  - PBS_TUNE_CACHE=<file>: where tuned choices are kept (default
 *    $HOME/.cache/pbs_tune.json); PBS_TUNE_FORCE=<prefix>=<i>,...: choice i for
 *    every tuning key with that prefix (tests);
 *  - PBS_GRAM=tc: offer the tensor-core Gram kernel to the tuner;
 *  - PBS_GRAPHS=0: no CUDA-graph replays of the multigrid sequences;
 *  - PBS_VERBOSE: per-iteration traces on stderr (synchronises the stream).
 */
#ifndef PBS_H
#define PBS_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define PBS_API __attribute__((visibility("default")))
#else
#define PBS_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ---------------------------------------------------- */
#define PBS_OK 0
#define PBS_EINVAL (-1)   /* invalid argument or unsupported size           */
#define PBS_ENOMEM (-2)   /* device allocation failed or over the budget    */
#define PBS_ENOCONV (-3)  /* max_iter reached; outputs filled with the last iterate */
#define PBS_ENUMERIC (-4) /* non-finite values or a breakdown of the small dense solves */
#define PBS_ETIMEOUT (-5) /* a bounded device wait gave up                 */
#define PBS_ECUDA (-6)    /* a CUDA runtime call failed                     */
#define PBS_ECANCELED (-7) /* the serving job was cancelled (pbs_cancel)    */

/* ---- precision policies (Section 4/5 preconditioner precision) -------- */
#define PBS_FP64 0  /* every kernel in FP64 ("plain"), the small Rayleigh-Ritz
                       eigensolve included; no double-float kernel runs
                       (pbs_launch_count_df does not move)                    */
#define PBS_MIXED 1 /* FP32 multigrid V-cycles and nodal cycles; the Gram
                       matrices, the Rayleigh quotients of the iteration, the
                       projection right-hand side L^* M x, the search direction
                       P and the small Rayleigh-Ritz eigensolve in double-float
                       arithmetic on the FP32 pipe (FP64 storage, about 2^-47
                       relative rounding); FP64 for everything that writes the
                       iterate or differences it through the curl-curl stencil
                       (residual A E - M E Lambda, E update, x - L phi) and for
                       the reported eigenvalues (FP64 Rayleigh quotients of the
                       converged block)                                       */

/* ---- operators for pbs_apply ----------------------------------------- */
#define PBS_OP_A 0             /* edge -> edge: y = A x  (Section 3)            */
#define PBS_OP_M 1             /* edge -> edge: y = M x                         */
#define PBS_OP_A_MU_M 2        /* edge -> edge: y = (A + mu M) x (Section 5)    */
#define PBS_OP_C 3             /* edge -> cell: y = C x, (Cx)_c = int_c scurl x */
#define PBS_OP_CH 4            /* cell -> edge: y = C^* x                       */
#define PBS_OP_L 5             /* node -> edge: y = L x, gradient lifting (eq. potential_discrete) */
#define PBS_OP_LH 6            /* edge -> node: y = L^* x                       */
#define PBS_OP_P_NODAL 7       /* node -> node: y = L^* M L x (Section 5)       */
#define PBS_OP_PROLONG 8       /* edge level l+1 -> level l: natural embedding (Section 5) */
#define PBS_OP_RESTRICT 9      /* edge level l -> level l+1: adjoint of the embedding */
#define PBS_OP_PROLONG_NODAL 10   /* node level l+1 -> level l                  */
#define PBS_OP_RESTRICT_NODAL 11  /* node level l -> level l+1                  */
#define PBS_OP_VCYCLE_EDGE 12  /* edge -> edge: y = B x, one V(nu_pre,nu_post) cycle for A + mu M */
#define PBS_OP_VCYCLE_NODAL 13 /* node -> node: y = B_P x, one V-cycle for L^* M L */
#define PBS_OP_PROJECT 14      /* edge -> edge: y = x - L phi, phi from nodal_cycles V-cycles on
                                  L^* M L phi = L^* M x (Section 4); at k = 0 the two constant
                                  edge fields are also M-projected out          */
#define PBS_OP_RESIDUAL 15     /* edge -> edge: y = A x - mu M x by the FP64 residual kernel of the
                                  iteration (R = A E - M E Lambda, Algorithm 2, with every
                                  Lambda entry equal to opts->mu)               */
#define PBS_OP_LH_M 16         /* edge -> node: y = L^* M x, the right-hand side of the projection
                                  (Section 4), in the arithmetic of opts->precision (FP64, or
                                  double-float under PBS_MIXED)                 */

typedef struct pbs_ctx pbs_ctx; /* opaque; owns every device allocation of the library */

typedef struct {
  double re, im;
} pbs_c64;

/* Periodic cell and mesh (Section 1 periods a, b; Section 3 mesh n x m). */
typedef struct {
  double a, b;       /* cell sizes, > 0                                     */
  int n, m;          /* cells per direction, even, >= 4                     */
  const double *eps; /* host, n*m samples (index j*n+i), > 0; copied at call */
} pbs_geom;

/* Solver options; pbs_default_opts fills documented defaults. */
typedef struct {
  int nev;          /* wanted bands (smallest non-zero eigenvalues), >= 1          */
  int block;        /* block width p (wanted + throw-away vectors, Section 7), nev <= block <= 32
                       (the trial block [E, W, P] then has at most 96 columns, the size
                       the one-CTA small dense eigensolve holds on chip)              */
  int max_iter;     /* iteration limit per Bloch vector (default 400)              */
  int precision;    /* PBS_FP64 or PBS_MIXED (default PBS_MIXED)                   */
  int span;         /* trial space of the Rayleigh-Ritz step (Section 4): 1 = PINVIT,
                       span(E - W) (Algorithm 1); 2 = gradient method, span(E, W);
                       3 = LOBPCG, span(E, W, P) (Algorithm 2; default 3); W is the
                       preconditioned residual, P the previous search direction    */
  double tol;       /* convergence: ||A e - lambda M e||_2 / (lambda ||M e||_2) <= tol on
                       the nev wanted bands (default 1e-8).  A band whose FP64
                       rounding floor is higher converges at
                       max(tol, 0.5 * 2^-53 * lambda_max / lambda), lambda_max =
                       max(1/eps) * 12 (1/h1^2 + 1/h2^2) (small lambda on fine
                       meshes, e.g. band 1 next to Gamma at 1024^2)             */
  double mu;        /* regularisation A + mu M of the preconditioner (Section 5); <= 0 selects 1/(a b) */
  int nu_pre;       /* pre-smoothing sweeps (default 1)                            */
  int nu_post;      /* post-smoothing sweeps (default 1)                           */
  int coarsest;     /* coarsen while both sides are even and >= 2*coarsest (default 4, >= 2) */
  int nodal_cycles; /* nodal V-cycles per projection (default 2)                   */
  int extrap_depth; /* previous bases used for the initial guess along a path, 0..3 (default 3) */
  uint64_t seed;    /* seed of the random initial block when no guess is given     */
  int kbatch;       /* Bloch vectors in flight along a path (default 1): the path is split
                       into kbatch contiguous chains solved in lock-step, one block of
                       `block` columns each, every launch covering all of them; each chain
                       extrapolates along its own segment (Section 6)                 */
  int start;        /* first Bloch vector of each chain when no init block is given:
                       PBS_START_RANDOM (default): seeded random block smoothed by two
                       preconditioned inverse-iteration steps; PBS_START_NESTED: the
                       nested iteration of Section 6 (solve on the coarsest hierarchy
                       mesh with at least 16 x 16 cells, prolongate the block level by
                       level, iterate each finer mesh to relative residual 1e-3)     */
} pbs_opts;

/* ---- starts (pbs_opts.start) ------------------------------------------ */
#define PBS_START_RANDOM 0
#define PBS_START_NESTED 1

/* Create a context on CUDA device `device`. `hbm_budget_bytes` caps the
 * library's device allocations (0 = no cap beyond free memory); the multigrid
 * work of the solver is then sized for chunks of at most an eighth of it (of
 * 8 GiB without a cap), so more Bloch vectors in flight fit at a small cost in
 * launches.  Contexts on different devices may live in one process; each
 * device gets its kernel attributes raised on its first launch there. */
PBS_API int pbs_create(pbs_ctx **ctx, int device, size_t hbm_budget_bytes);

/* Free every device allocation of the context and the context itself. NULL is a no-op. */
PBS_API int pbs_destroy(pbs_ctx *ctx);

/* Fill `o` with the defaults listed in pbs_opts. */
PBS_API void pbs_default_opts(pbs_opts *o);

/* Number of multigrid levels the hierarchy rule gives for (n, m, coarsest), or PBS_EINVAL. */
PBS_API int pbs_num_levels(int n, int m, int coarsest);

/*
 * Smallest non-zero eigenpairs at one Bloch vector k (Section 4, Algorithm 2
 * with the multigrid preconditioner of Section 5 and null-space elimination of
 * Section 4).  At k = 0 (both phases equal to one) the two constant edge fields
 * are deflated as well, so the reported values are the smallest non-zero ones.
 *   k       host, 2 doubles (k1, k2)
 *   init    host, D*block complex values (column-major) or NULL for a seeded
 *           random start
 *   eigvals host out, nev ascending Rayleigh quotients
 *   resid   host out, nev relative residuals (see pbs_opts.tol)
 *   iters   host out, iterations performed
 *   evecs   host out, D*nev complex (column-major, M-orthonormal) or NULL
 * Returns PBS_ENOCONV (outputs filled) when max_iter is reached.
 */
PBS_API int pbs_solve_k(pbs_ctx *ctx, const pbs_geom *geom, const pbs_opts *opts, const double k[2],
                const pbs_c64 *init, double *eigvals, double *resid, int *iters, pbs_c64 *evecs);

/*
 * A sequence of Bloch vectors solved in order; each one after the first starts
 * from the Rayleigh-quotient-minimising extrapolation of up to extrap_depth
 * previous bases (Section 6).  ks: host nk*2; eigvals, resid: host nk*nev;
 * iters: host nk.  Returns the first non-OK status met (later k still solved).
 */
PBS_API int pbs_solve_path(pbs_ctx *ctx, const pbs_geom *geom, const pbs_opts *opts, int nk, const double *ks,
                   double *eigvals, double *resid, int *iters);

/*
 * pbs_solve_path with the eigenvectors of selected Bloch vectors: sel (host, nsel
 * distinct indices into ks) picks them; evecs (host, nsel * nev * D complex) gets,
 * for selection t, the nev wanted eigenvectors of Bloch vector sel[t] at
 * evecs + t nev D (column-major, M-normalised: e^* M e = 1), copied when that
 * Bloch vector converges.  The computation is the one of pbs_solve_path: eigvals,
 * resid and iters are identical.  nsel = 0 is pbs_solve_path.
 */
PBS_API int pbs_solve_path_vectors(pbs_ctx *ctx, const pbs_geom *geom, const pbs_opts *opts, int nk, const double *ks,
                                   double *eigvals, double *resid, int *iters, int nsel, const int *sel,
                                   pbs_c64 *evecs);

/*
 * The kappa x kappa Brillouin-zone sample of Section 6,
 *   k_ij = (pi/a (2 i/(kappa-1) - 1), pi/b (2 j/(kappa-1) - 1)),  i, j in [0, kappa),
 * with the paper's extrapolation schedule: k_00 from the start block (opts->start),
 * row 0 horizontally (k_i0 from up to three predecessors in the row), columns 0, 1, 2
 * vertically from row 0, and every other k_ij horizontally from k_{i-3..i-1, j} (the
 * paper leaves rows 1 and 2 beyond column 2 unstated; read as horizontal).  The rows
 * beyond column 2 are independent chains and run opts->kbatch at a time.
 * Outputs (host, index j*kappa + i): ks (kappa^2 * 2, may be NULL), eigvals and resid
 * (kappa^2 * nev), iters (kappa^2).  kappa >= 2.  Returns PBS_ENOCONV (outputs
 * filled) when some Bloch vector reached max_iter.
 */
PBS_API int pbs_solve_grid(pbs_ctx *ctx, const pbs_geom *geom, const pbs_opts *opts, int kappa, double *ks,
                           double *eigvals, double *resid, int *iters);

/*
 * Same as pbs_solve_path with every array on the device: d_eps (n*m doubles),
 * d_ks (nk*2), d_eigvals (nk*nev), d_resid (nk*nev), d_iters (nk ints); the
 * work is issued on `cuda_stream` (a cudaStream_t, NULL = legacy default) and
 * the call returns after it finished.  The hierarchy of a geometry stays
 * resident in the context between calls.
 */
PBS_API int pbs_solve_path_device(pbs_ctx *ctx, double a, double b, int n, int m, const double *d_eps,
                          const pbs_opts *opts, int nk, const double *d_ks, double *d_eigvals,
                          double *d_resid, int *d_iters, void *cuda_stream);

/*
 * Apply one operator of the discretisation or the multigrid (PBS_OP_*) to
 * `ncols` columns.  x, y: device, interleaved complex FP64, lengths given by
 * the operator and `level`; x and y must not overlap. mu, nu_pre, nu_post,
 * coarsest, nodal_cycles and precision are taken from `opts`.
 */
PBS_API int pbs_apply(pbs_ctx *ctx, const pbs_geom *geom, const pbs_opts *opts, int op, int level, const double k[2],
              int ncols, const pbs_c64 *x, pbs_c64 *y, void *cuda_stream);

/*
 * Block Gram matrices of the pencil at k (Section 4, used by Rayleigh-Ritz):
 * GM = S^* M S and GA = (C S)^* W (C S) = S^* A S, W = diag(1/(eps_c h1 h2)).
 * S: device D x q; GM, GA: device q x q column-major.  `precision` selects the
 * arithmetic: PBS_FP64, or PBS_MIXED = double-float on the FP32 pipe (about
 * 2^-47 relative rounding, compensated sums), the arithmetic the mixed policy
 * uses inside the solver.  Inputs and outputs are FP64 either way.
 */
PBS_API int pbs_gram(pbs_ctx *ctx, const pbs_geom *geom, const double k[2], int q, const pbs_c64 *S, pbs_c64 *GM,
             pbs_c64 *GA, int precision, void *cuda_stream);

/*
 * Generalised Householder orthonormalisation (Section 4): reflections
 * Q_i = I - 2 v_i v_i^* M / (v_i^* M v_i) with Q_q ... Q_1 S = P R, where P is
 * the prescribed M-orthonormal basis of scaled unit vectors of the x-edges
 * (k mod n, 2 (k div n)), k = 0 .. q-1 (they share no mass-matrix entry), and
 * R is upper triangular; E = Q_1 ... Q_q P is M-orthonormal and S = E R.  When
 * S loses rank the matching diagonal entries of R vanish (exactly zero columns
 * leave Q_i = I) and E still is M-orthonormal with span(S) inside span(E).
 * S, E: device D x q column-major (leading dimension D = 2 n m); R: device
 * q x q column-major; FP64; S is not modified and must not overlap E or R.
 * q <= 96 and q <= n * floor(m / 2), else PBS_EINVAL.  Work space (about D q
 * complex doubles) comes from the context's budget for the duration of the call.
 */
PBS_API int pbs_m_householder(pbs_ctx *ctx, const pbs_geom *geom, const double k[2], int q, const pbs_c64 *S,
                              pbs_c64 *E, pbs_c64 *R, void *cuda_stream);

/*
 * Rayleigh-Ritz of the pencil on span(S) (Section 4, eq. ritz_eigenvalue):
 * the p smallest Ritz values (host `theta`) and M-orthonormal Ritz vectors
 * (device X, D x p).  With project != 0 the columns of S are first projected
 * off the gradients (and at k = 0 the constant fields) with opts->nodal_cycles
 * nodal V-cycles, which is the extrapolation step of Section 6. S is not modified.
 */
PBS_API int pbs_rayleigh_ritz(pbs_ctx *ctx, const pbs_geom *geom, const pbs_opts *opts, const double k[2], int q,
                      const pbs_c64 *S, int p, int project, double *theta, pbs_c64 *X, void *cuda_stream);

/*
 * Diagnostics: time every launch of the listed kernel classes with a pair of
 * CUDA events on the stream it is launched on (the library's stream).
 * `classes` is "all" or a comma-separated list of "edge_smooth",
 * "node_smooth", "gram", "small_rr", "residual", "block_update",
 * "lift_adj_mass", "edge_apply", "edge_tail", "node_tail", "householder",
 * "sub_lift" (x - L phi), "convert" (binary64 <-> binary32 copies), "node_apply"
 * (nodal operator applications and updates of the projection),
 * optionally followed by "/N" to time only every N-th launch
 * of each listed class; NULL or "" switches timing off.  Enabling resets the
 * counters.  pbs_profile_read returns, for one class, the summed device time
 * (ms), the number of timed launches and their summed algorithmic work (bytes
 * moved for the streaming kernels, flops for "gram", "small_rr" and
 * "block_update") since then.
 */
PBS_API int pbs_profile_enable(pbs_ctx *ctx, const char *classes);
PBS_API int pbs_profile_read(pbs_ctx *ctx, const char *kernel_class, double *total_ms, long *launches,
                             double *work);

/* Number of CUDA kernels the library has launched in this process. */
PBS_API unsigned long long pbs_launch_count(void);

/* Number of those launches whose kernel computes in double-float arithmetic on
 * the FP32 pipe (Gram, Rayleigh quotients, L^* M x, search direction and small
 * Rayleigh-Ritz of the mixed policy, and pbs_small_rr_noalloc).  A PBS_FP64
 * solve leaves it unchanged. */
PBS_API unsigned long long pbs_launch_count_df(void);

/*
 * Serving: paths of Bloch vectors (Section 6) submitted as independent requests
 * and solved with continuous batching.  No counterpart in the paper; it exists so
 * that many jobs can share one device.  The context runs `slots` serving slots
 * (pbs_serve_slots, default 4), each an engine with its own CUDA stream, resident
 * multigrid hierarchy and workspace, driven by its own host thread, so the jobs of
 * different slots overlap on the device.  A free slot takes the first queued job
 * that fits the device memory the running jobs and the idle slots' resident data
 * leave (the context's budget, or 90% of the free device memory at the first
 * submission when the budget is 0); among the first 2 slots queued jobs it prefers
 * one whose geometry it already holds.  A job at the head of the queue that does
 * not fit waits (idle slots free what they keep resident) and is passed by later
 * jobs at most 2 slots times.  Every job runs the computation of pbs_solve_path on
 * its own data, so its results do not depend on what else runs (bit for bit: the
 * kernels are deterministic).  Synchronous calls on the context use the context's
 * own engine and do not wait for jobs.
 *
 * pbs_job_bytes: device bytes a path job of nk Bloch vectors on an n x m mesh with
 *   these options needs on an engine that holds nothing else (hierarchy, coarsest
 *   factors, solver workspace; the admission estimate).
 * pbs_submit: copies geom (including eps), opts and ks (host, nk*2) and queues the
 *   job; returns at once with *job_id.  PBS_EINVAL for invalid input (checked at
 *   submission, eps and ks included), PBS_ENOMEM when the job alone needs more than
 *   the jobs may hold together.
 * pbs_poll: *done = 1 once the job has finished (successfully or not), else 0.
 * pbs_fetch: waits until the job has finished, copies its results (host,
 *   nk*nev eigvals and resid, nk iters; any may be NULL) and the latency from
 *   submission to completion in seconds (may be NULL), forgets the job and
 *   returns its status (the pbs_solve_path status, or PBS_ECANCELED;
 *   pbs_last_error in the calling thread then describes a failure).  Unknown ids
 *   give PBS_EINVAL.
 * pbs_cancel: a queued job is removed at once; a running job stops at its next
 *   iteration boundary (no kernel is interrupted); either way it finishes with
 *   PBS_ECANCELED.  A finished job is left as it is (PBS_OK).
 * pbs_job_times: seconds since the context's creation at which the job was
 *   submitted, started on a slot and finished (-1 for what has not happened yet);
 *   valid until pbs_fetch.
 * pbs_serve_slots: number of serving slots (1..64), before the first submission.
 * pbs_destroy lets running jobs finish and drops queued ones.
 */
PBS_API int pbs_job_bytes(int n, int m, const pbs_opts *opts, int nk, size_t *bytes);
PBS_API int pbs_submit(pbs_ctx *ctx, const pbs_geom *geom, const pbs_opts *opts, int nk, const double *ks,
                       uint64_t *job_id);
PBS_API int pbs_poll(pbs_ctx *ctx, uint64_t job_id, int *done);
PBS_API int pbs_fetch(pbs_ctx *ctx, uint64_t job_id, double *eigvals, double *resid, int *iters,
                      double *latency_s);
PBS_API int pbs_cancel(pbs_ctx *ctx, uint64_t job_id);
PBS_API int pbs_job_times(pbs_ctx *ctx, uint64_t job_id, double *submit_s, double *start_s, double *done_s);
PBS_API int pbs_serve_slots(pbs_ctx *ctx, int slots);

/*
 * Change the byte budget of the context's own allocations (0 = no cap).  Memory
 * already held stays; an allocation that would exceed the new budget fails with
 * PBS_ENOMEM, after which the context remains usable (a later call with a larger
 * budget succeeds).  Serving jobs are admitted against the budget the context had
 * at its first submission.
 */
PBS_API int pbs_set_budget(pbs_ctx *ctx, size_t hbm_budget_bytes);

/*
 * Failure injection for tests: the count-th device allocation of the context's
 * own engine from now fails as if the device were out of memory (PBS_ENOMEM from
 * the call that makes it; the context stays usable).  0 switches it off.
 */
PBS_API int pbs_fail_alloc_after(pbs_ctx *ctx, int count);

/*
 * Allocation-free Rayleigh-Ritz step.  No counterpart in the paper: it exists
 * for callers that cannot call cudaMalloc, because all of their device memory
 * is owned by another allocator (a framework's caching allocator or a fixed
 * arena) or because their process forbids new device allocations once it is
 * running.  Given the Gram matrices GM = S^* M S and GA = S^* A S of a trial
 * block (for example from pbs_gram), it computes the p smallest Ritz values
 * (`theta`, ascending) and the coefficient matrix C (q x p, column-major) with
 * X = S C M-orthonormal Ritz vectors - the same computation as the
 * coefficient step inside pbs_rayleigh_ritz.
 *   GM, GA  device, q x q column-major Hermitian;  C device q x p;
 *   theta   device, p doubles;  info device, 2 ints: info[0] = 0 on success,
 *           -1 if the span has fewer than p independent directions, -2 if an
 *           input is not finite, -3 if the eigensolve broke down; info[1] =
 *           numerical rank of the span.
 * Limits: 1 <= q <= 96, 1 <= p <= min(q, 32); larger sizes return PBS_EINVAL.
 * The kernel runs on `cuda_stream` on whichever device is current; the call
 * needs no context and is not tied to the device of any pbs_create.  It returns
 * after the launch, without waiting for it.  Failures set pbs_last_error; an
 * error already pending on the calling thread (from earlier CUDA work) is
 * reported as PBS_ECUDA without launching and is left in place.  It allocates nothing: its work
 * space is a fixed device array of about 480 KB compiled into the library and
 * held by every GPU that loads it until the process exits.  The first call on a
 * device looks up that array's device address, so make the first call on each
 * device before any stream capture.  Every call on a device shares the one
 * array: calls whose kernels may overlap on the GPU (different streams without
 * ordering) race and give wrong results; serialise them.  No element of the
 * array has to start at zero: everything read is written first by the same call.
 */
PBS_API int pbs_small_rr_noalloc(const pbs_c64 *GM, const pbs_c64 *GA, int q, int p, pbs_c64 *C, double *theta,
                                 int *info, void *cuda_stream);

/* Static description of a status code. */
PBS_API const char *pbs_strerror(int status);

/* Detail of the last failure on the calling thread ("" if none). */
PBS_API const char *pbs_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PBS_H */
