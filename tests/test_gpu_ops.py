"""GPU parity of the operators, transfers, V-cycles, projection, Gram and Rayleigh-Ritz steps.

Every call goes through the C ABI (``pbs_apply``, ``pbs_gram``,
``pbs_rayleigh_ritz``) on seeded inputs; expected values come from the CPU
oracle on the same inputs.  Bars: operator applications <= 1e-13 relative
(2-norm per column on small ragged meshes; entry by entry, relative to the
column's largest entry, on a mesh with interior tiles), FP64 V-cycles <= 1e-11
and projection <= 1e-12 (same algorithm, different summation order), FP32
cycles <= 1e-5 where the cycle is well conditioned (mu = lambda_max / 1000).
At the solver's mu = 0.7 an FP32 cycle inherits the cycle's own rounding
amplification (the oracle's output moves by up to 1.7e4 ulp under a one-ulp
input perturbation at 128 x 64), so that comparison's bar is twice that
amplification times 2^-24.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2304_00337_gb300 as pbs  # noqa: E402
import pbs_inputs as gi  # noqa: E402
from oracle import fem, multigrid as mg, extrapolation as ex, eigen  # noqa: E402

pytestmark = pytest.mark.gpu

# (a, b, n, m, k): tiles of the kernels are 32 x 8 threads, so 48 x 20 leaves ragged tails
CASES = [
    (1.0, 1.0, 16, 16, (0.3, -0.2)),
    (1.0, 20 / 48, 48, 20, (2.1, 0.7)),
    (1.0, 1.0, 8, 8, (0.0, 0.0)),
    (1.0, 1.0, 16, 16, (np.pi, np.pi)),
    (1.3, 0.7, 24, 12, (-1.1, 3.0)),
]
MU = 0.7
NCOLS = 3


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with pbs.Context(0) as c:
        yield c


def _eps(n, m, seed=11):
    return np.random.default_rng(seed).uniform(1.0, 9.0, (m, n))


def _block(ncols, size, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal((ncols, size)) + 1j * r.standard_normal((ncols, size))


def _dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _apply(ctx, geom, op, x, out_len, k, level=0, **o):
    xd = _dev(x)
    yd = torch.zeros((x.shape[0], out_len), dtype=torch.complex128, device="cuda")
    opts = pbs.default_opts(mu=MU, **o)
    ctx.apply(geom, op, xd.data_ptr(), yd.data_ptr(), x.shape[0], k=k, level=level, opts=opts,
              stream=torch.cuda.current_stream())
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _rel(got, want):
    return np.max(np.linalg.norm(got - want, axis=1) / np.maximum(np.linalg.norm(want, axis=1), 1e-300))


def _bars(fn, x):
    """FP64 and FP32 bars for a linear solver step.  The oracle's own output is
    moved by a one-ulp (2^-53) relative perturbation of its input; that change
    divided by 2^-53 is the rounding amplification of the step, which grows with
    the condition of the level operators.  Bars: 1e-12 (FP64) and 1e-5 (FP32), or
    twice the amplification times the unit roundoff, whichever is larger."""
    y = fn(x)
    d = x * (1 + 2.0 ** -53 * np.random.default_rng(99).standard_normal(x.shape))
    amp = np.linalg.norm(fn(d) - y) / np.linalg.norm(y) / 2.0 ** -53
    return max(1e-12, 2 * amp * 2.0 ** -53), max(1e-5, 2 * amp * 2.0 ** -24)


def _entrywise(got, want):
    """Largest entry error of each column relative to the column's largest entry."""
    return np.max(np.abs(got - want).max(axis=1) / np.maximum(np.abs(want).max(axis=1), 1e-300))


def _coarse_eps(eps):
    inv = 1.0 / eps
    return 1.0 / (0.25 * (inv[0::2, 0::2] + inv[1::2, 0::2] + inv[0::2, 1::2] + inv[1::2, 1::2]))


@pytest.mark.parametrize("a,b,n,m,k", CASES)
def test_edge_and_nodal_operators(ctx, a, b, n, m, k):
    eps = _eps(n, m)
    geom = pbs.Geometry(eps, a, b)
    ops = fem.assemble(fem.Mesh(a, b, n, m), eps, k)
    N, D = n * m, 2 * n * m
    x = _block(NCOLS, D, 1)
    xn = _block(NCOLS, N, 2)
    A, M, C, L, P = ops["A"], ops["M"], ops["C"], ops["L"], ops["P"]
    checks = [
        ("A", x, D, A @ x.T),
        ("M", x, D, M @ x.T),
        ("A_MU_M", x, D, (A + MU * M) @ x.T),
        ("C", x, N, C @ x.T),
        ("CH", xn, D, C.conj().T @ xn.T),
        ("L", xn, D, L @ xn.T),
        ("LH", x, N, L.conj().T @ x.T),
        ("P_NODAL", xn, N, P @ xn.T),
    ]
    for op, inp, olen, want in checks:
        got = _apply(ctx, geom, op, inp, olen, k)
        assert _rel(got, want.T) <= 1e-13, op


# 128 x 96 cells on 32 x 8 thread tiles (4 x 12 tiles, 20 of them interior, i.e. no
# read through the Bloch extension): every operator, the iteration's FP64 residual
# kernel and the projection right-hand side L^* M x, entry by entry
@pytest.mark.parametrize("k", [(0.9, -2.3), (0.0, 0.0), (np.pi, -np.pi)])
def test_operators_entrywise_interior_tiles(ctx, k):
    a, b, n, m = 1.0, 0.75, 128, 96
    eps = _eps(n, m, seed=17)
    geom = pbs.Geometry(eps, a, b)
    ops = fem.assemble(fem.Mesh(a, b, n, m), eps, k)
    N, D = n * m, 2 * n * m
    x = _block(NCOLS, D, 21)
    xn = _block(NCOLS, N, 22)
    A, M, C, L, P = ops["A"], ops["M"], ops["C"], ops["L"], ops["P"]
    checks = [
        ("A", x, D, A @ x.T, {}),
        ("M", x, D, M @ x.T, {}),
        ("A_MU_M", x, D, (A + MU * M) @ x.T, {}),
        ("C", x, N, C @ x.T, {}),
        ("CH", xn, D, C.conj().T @ xn.T, {}),
        ("L", xn, D, L @ xn.T, {}),
        ("LH", x, N, L.conj().T @ x.T, {}),
        ("P_NODAL", xn, N, P @ xn.T, {}),
        ("RESIDUAL", x, D, (A - MU * M) @ x.T, {}),
        ("LH_M", x, N, L.conj().T @ (M @ x.T), dict(precision=pbs.PBS_FP64)),
        ("LH_M", x, N, L.conj().T @ (M @ x.T), dict(precision=pbs.PBS_MIXED)),
    ]
    for op, inp, olen, want, o in checks:
        got = _apply(ctx, geom, op, inp, olen, k, **o)
        assert _entrywise(got, want.T) <= 1e-13, (op, o)


@pytest.mark.parametrize("a,b,n,m,k", [CASES[0], CASES[1], CASES[3]])
def test_transfers_and_coarse_level_operators(ctx, a, b, n, m, k):
    eps = _eps(n, m)
    geom = pbs.Geometry(eps, a, b)
    fine = fem.Mesh(a, b, n, m)
    coarse = fine.coarse()
    Pe = fem.edge_prolongation(fine, coarse, k)
    Pn = fem.nodal_prolongation(fine, coarse, k)
    xc = _block(NCOLS, coarse.D, 3)
    xf = _block(NCOLS, fine.D, 4)
    assert _rel(_apply(ctx, geom, "PROLONG", xc, fine.D, k), (Pe @ xc.T).T) <= 1e-14
    assert _rel(_apply(ctx, geom, "RESTRICT", xf, coarse.D, k), (Pe.conj().T @ xf.T).T) <= 1e-14
    xcn = _block(NCOLS, coarse.N, 5)
    xfn = _block(NCOLS, fine.N, 6)
    assert _rel(_apply(ctx, geom, "PROLONG_NODAL", xcn, fine.N, k), (Pn @ xcn.T).T) <= 1e-14
    assert _rel(_apply(ctx, geom, "RESTRICT_NODAL", xfn, coarse.N, k), (Pn.conj().T @ xfn.T).T) <= 1e-14
    # level-1 operators = coarse assembly with the children's mean 1/eps
    oc = fem.assemble(coarse, _coarse_eps(eps), k)
    got = _apply(ctx, geom, "A_MU_M", xc, coarse.D, k, level=1)
    assert _rel(got, ((oc["A"] + MU * oc["M"]) @ xc.T).T) <= 1e-13
    got = _apply(ctx, geom, "P_NODAL", xcn, coarse.N, k, level=1)
    assert _rel(got, (oc["P"] @ xcn.T).T) <= 1e-13


# levels with at most 4096 nodes run as one fused kernel; 96 x 48 (4608 nodes) runs
# its top level step by step and the rest fused; 128 x 64 runs its top nodal level as
# the tiled down/up kernels (both sides at least 59); the smaller cases fused throughout.
# Inputs are of the class the solver feeds the cycles: residuals of iterates that are
# M-orthogonal to the gradients, b = M (x - L phi) with L^* b = 0.
@pytest.mark.parametrize("a,b,n,m,k", [CASES[0], CASES[1], CASES[2], CASES[3], (1.0, 0.5, 96, 48, (0.4, -1.3)),
                                       (1.0, 0.5, 128, 64, (-0.8, 2.2))])
def test_vcycles_match_reference(ctx, a, b, n, m, k):
    eps = _eps(n, m)
    geom = pbs.Geometry(eps, a, b)
    mesh = fem.Mesh(a, b, n, m)
    ops = fem.assemble(mesh, eps, k)
    x = _block(2, mesh.D, 7)
    x = (ops["M"] @ mg.project_exact(ops, x.T)).T
    levels = mg.edge_hierarchy(mesh, eps, k, MU, 4)
    want = np.stack([mg.edge_vcycle(levels, x[c]) for c in range(2)])
    got = _apply(ctx, geom, "VCYCLE_EDGE", x, mesh.D, k, precision=pbs.PBS_FP64)
    assert _rel(got, want) <= 1e-11
    _, bar32 = _bars(lambda v: mg.edge_vcycle(levels, v), x[0])
    got32 = _apply(ctx, geom, "VCYCLE_EDGE", x, mesh.D, k, precision=pbs.PBS_MIXED)
    assert _rel(got32, want) <= bar32
    # a well-conditioned cycle (mu = lambda_max / 1000: amplification about 50 ulp) holds the
    # FP32 kernels to a fixed bar; a wrong colour order on any tile moves the result at O(1)
    mu_w = 12.0 * (1.0 / mesh.h1 ** 2 + 1.0 / mesh.h2 ** 2) / 1000.0
    lw = mg.edge_hierarchy(mesh, eps, k, mu_w, 4)
    want = np.stack([mg.edge_vcycle(lw, x[c]) for c in range(2)])
    for prec, bar in ((pbs.PBS_FP64, 1e-12), (pbs.PBS_MIXED, 1e-5)):
        xd = _dev(x)
        yd = torch.zeros_like(xd)
        ctx.apply(geom, "VCYCLE_EDGE", xd.data_ptr(), yd.data_ptr(), 2, k=k,
                  opts=pbs.default_opts(mu=mu_w, precision=prec), stream=torch.cuda.current_stream())
        torch.cuda.synchronize()
        assert _rel(yd.cpu().numpy(), want) <= bar, prec
    nlev = mg.nodal_hierarchy(mesh, eps, k, 4)
    xn = _block(2, mesh.N, 8)
    if fem.is_gamma(*fem.bloch_phases(k, a, b)):
        xn -= xn.mean(axis=1, keepdims=True)
    want = np.stack([mg.nodal_vcycle(nlev, xn[c]) for c in range(2)])
    got = _apply(ctx, geom, "VCYCLE_NODAL", xn, mesh.N, k, precision=pbs.PBS_FP64)
    assert _rel(got, want) <= 1e-11
    got32 = _apply(ctx, geom, "VCYCLE_NODAL", xn, mesh.N, k, precision=pbs.PBS_MIXED)
    assert _rel(got32, want) <= 1e-5


@pytest.mark.parametrize("a,b,n,m,k", [CASES[0], CASES[2], CASES[4]])
@pytest.mark.parametrize("cycles", [1, 3])
def test_projection_matches_reference(ctx, a, b, n, m, k, cycles):
    eps = _eps(n, m)
    geom = pbs.Geometry(eps, a, b)
    mesh = fem.Mesh(a, b, n, m)
    ops = fem.assemble(mesh, eps, k)
    nlev = mg.nodal_hierarchy(mesh, eps, k, 4)
    x = _block(3, mesh.D, 9)
    want = mg.project_approx(ops, nlev, x.T, cycles).T
    got = _apply(ctx, geom, "PROJECT", x, mesh.D, k, precision=pbs.PBS_FP64, nodal_cycles=cycles)
    assert _rel(got, want) <= 1e-12
    got32 = _apply(ctx, geom, "PROJECT", x, mesh.D, k, precision=pbs.PBS_MIXED, nodal_cycles=cycles)
    assert _rel(got32, want) <= 1e-5


# The tiled nodal steps on meshes where every launch shape the autotuner may pick fits
# (32 x 32 tiles of 256 threads, 64 x 64 tiles of 512 or 256 threads, and for FP32 cycles
# the register-blocked steps on 32 x 32 tiles of 256 or 128 threads and 64 x 64 tiles of
# 512): 192 x 96 has a partial last row of 64 x 64 tiles, 128 x 128 at Gamma whole ones
# and the constant remainder.  Run as they are here (the tuned shape) and with each shape
# forced below (FP64 cycles, which have the first three shapes only, tune the others).
@pytest.mark.parametrize("a,b,n,m,k", [(1.0, 0.5, 192, 96, (0.4, -1.3)), (1.0, 1.0, 128, 128, (0.0, 0.0))])
def test_nodal_cycle_and_projection_on_large_tiles(ctx, a, b, n, m, k):
    eps = _eps(n, m)
    geom = pbs.Geometry(eps, a, b)
    mesh = fem.Mesh(a, b, n, m)
    nlev = mg.nodal_hierarchy(mesh, eps, k, 4)
    xn = _block(2, mesh.N, 12)
    # at Gamma the nodal operator annihilates the constants on every level, and the
    # cycle's output is compared modulo them (the projection's L phi does not see them)
    gamma = fem.is_gamma(*fem.bloch_phases(k, a, b))
    if gamma:
        xn -= xn.mean(axis=1, keepdims=True)

    def mod(y):
        return y - y.mean(axis=1, keepdims=True) if gamma else y
    want = mod(np.stack([mg.nodal_vcycle(nlev, xn[c]) for c in range(2)]))
    assert _rel(mod(_apply(ctx, geom, "VCYCLE_NODAL", xn, mesh.N, k, precision=pbs.PBS_FP64)), want) <= 1e-11
    assert _rel(mod(_apply(ctx, geom, "VCYCLE_NODAL", xn, mesh.N, k, precision=pbs.PBS_MIXED)), want) <= 1e-5
    ops = fem.assemble(mesh, eps, k)
    x = _block(2, mesh.D, 13)
    want = mg.project_approx(ops, nlev, x.T, 2).T
    assert _rel(_apply(ctx, geom, "PROJECT", x, mesh.D, k, precision=pbs.PBS_FP64, nodal_cycles=2), want) <= 1e-12
    assert _rel(_apply(ctx, geom, "PROJECT", x, mesh.D, k, precision=pbs.PBS_MIXED, nodal_cycles=2), want) <= 1e-5


@pytest.mark.parametrize("shape", [0, 1, 2, 3, 4, 5])
def test_nodal_tile_shapes_in_child_processes(shape):
    # each launch shape of the tiled nodal steps forced (PBS_TUNE_FORCE) in a child process:
    # the cycle and projection cases above, and with the 64 x 64 tiles of 512 threads (plain
    # and register-blocked) the 256 x 256 rod path (levels 256 and 128 tiled) against the
    # oracle's stored eigenvalues
    import os
    import subprocess
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    tests = [os.path.join(here, "test_gpu_ops.py") + "::test_nodal_cycle_and_projection_on_large_tiles"]
    if shape in (1, 4):
        tests.append(os.path.join(here, "test_gpu_eigen.py") + "::test_rod256_path_full_size")
    env = dict(os.environ, PBS_TUNE_FORCE=f"node_down={shape},node_up={shape}")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider", *tests],
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]


# mixed policy: the double-float kernel (q = 12 .. 60); 128 x 96 has interior tiles and
# chunks that end inside a row
@pytest.mark.parametrize("precision", [pbs.PBS_FP64, pbs.PBS_MIXED])
@pytest.mark.parametrize("a,b,n,m,k,q", [CASES[1] + (30,), CASES[2] + (30,), CASES[1] + (12,), CASES[1] + (48,),
                                         CASES[1] + (60,), (1.0, 0.75, 128, 96, (0.9, -2.3), 30)])
def test_gram_matches_oracle(ctx, a, b, n, m, k, q, precision):
    eps = _eps(n, m)
    geom = pbs.Geometry(eps, a, b)
    ops = fem.assemble(fem.Mesh(a, b, n, m), eps, k)
    S = _block(q, geom.D, 10)
    # columns of very different sizes (as in a trial block [E, P, W] near convergence)
    S *= np.logspace(0, -9, q)[:, None]
    Sd = _dev(S)
    GM = torch.zeros((q, q), dtype=torch.complex128, device="cuda")
    GA = torch.zeros((q, q), dtype=torch.complex128, device="cuda")
    ctx.gram(geom, k, q, Sd.data_ptr(), GM.data_ptr(), GA.data_ptr(), torch.cuda.current_stream(),
             precision=precision)
    torch.cuda.synchronize()
    gm = GM.cpu().numpy().T  # column-major on the device
    ga = GA.cpu().numpy().T
    wm, wa = ex.grams(ops, S.T)
    # FP64: rounding ~1e-16 per term; mixed: inputs split to 2^-47 relative, stencils
    # and compensated (or sliced) sums add a few units of that.  Entry (a, b) is held to
    # 1e-13 of sqrt(G_aa G_bb), the scale of its terms (columns differ by up to 1e9)
    for got, want in ((gm, wm), (ga, wa)):
        d = np.sqrt(np.real(np.diag(want)))
        assert np.all(np.abs(got - want) <= 1e-13 * np.outer(d, d)), (q, precision)
    assert np.array_equal(gm, gm.conj().T) and np.array_equal(ga, ga.conj().T)


def test_tensor_core_gram_in_a_child_process():
    # the tensor-core Gram (bf16 slices, opt-in) is selected per process: a child process with
    # PBS_GRAM=tc and tuning off runs the Gram parity cases above on it, and the mixed 64 x 64
    # rod path against the oracle's stored values with it inside the iteration
    import os
    import subprocess
    import sys
    here = os.path.dirname(os.path.abspath(__file__))
    env = dict(os.environ, PBS_GRAM="tc", PBS_TUNE="0")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-p", "no:cacheprovider",
                        os.path.join(here, "test_gpu_ops.py") + "::test_gram_matches_oracle",
                        os.path.join(here, "test_gpu_eigen.py") + "::test_rod64_path_with_extrapolation"],
                       env=env, capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stdout[-3000:] + r.stderr[-2000:]


@pytest.mark.parametrize("precision", [pbs.PBS_FP64, pbs.PBS_MIXED])
@pytest.mark.parametrize("k", [(0.3, 0.1), (0.0, 0.0)])
def test_rayleigh_ritz_and_extrapolation(ctx, k, precision):
    n = 16
    eps = gi.rod_eps(n, n)
    geom = pbs.Geometry(eps)
    ks = [np.array(k) + d for d in (np.array([0.2, 0.1]), np.array([0.4, 0.2]))]
    prev = [eigen.solve_k(1, 1, n, n, eps, kk, 6, "dense")[1] for kk in ks]
    ops = fem.assemble(fem.Mesh(1, 1, n, n), eps, k)
    S = np.concatenate(prev, axis=1)  # (D, 12)
    Sd = _dev(S.T)
    X = torch.zeros((6, geom.D), dtype=torch.complex128, device="cuda")
    # plain Rayleigh-Ritz on the span
    th_want, _ = ex.rayleigh_ritz(ops, S, 6)
    th = ctx.rayleigh_ritz(geom, pbs.default_opts(precision=precision), k, 12, Sd.data_ptr(), 6, False,
                           X.data_ptr(), torch.cuda.current_stream())
    assert np.allclose(th, th_want, rtol=1e-11)
    Xh = X.cpu().numpy().T
    GM, GA = ex.grams(ops, Xh)
    assert np.allclose(GM, np.eye(6), atol=1e-10)
    assert np.allclose(np.real(np.diag(GA)), th_want, rtol=1e-10)
    # extrapolation: projection off the gradients first (Section 6)
    th_want, _ = ex.extrapolate(ops, prev, 6)
    th = ctx.rayleigh_ritz(geom, pbs.default_opts(precision=precision, nodal_cycles=14), k, 12, Sd.data_ptr(), 6,
                           True, X.data_ptr(), torch.cuda.current_stream())
    # mixed: the nodal cycles run in FP32 and leave ~1e-7 of the gradient part,
    # which moves the Ritz values at second order
    assert np.allclose(th, th_want, rtol=1e-10 if precision == pbs.PBS_FP64 else 1e-9)


def test_empty_and_invalid_calls(ctx):
    geom = pbs.Geometry(_eps(16, 16))
    x = torch.zeros((1, geom.D), dtype=torch.complex128, device="cuda")
    ctx.apply(geom, "A", x.data_ptr(), x.data_ptr(), 0, k=(0.1, 0.2))  # ncols = 0: no-op
    with pytest.raises(pbs.PbsError) as e:
        ctx.apply(geom, "PROLONG", x.data_ptr(), x.data_ptr(), 1, level=2)  # no level below the coarsest
    assert e.value.status == pbs.PBS_EINVAL
    with pytest.raises(pbs.PbsError) as e:
        ctx.solve_k(pbs.Geometry(_eps(15, 16)), dict(nev=2, block=4), (0.1, 0.1))  # odd side
    assert e.value.status == pbs.PBS_EINVAL
    bad = _eps(16, 16)
    bad[3, 4] = -1.0
    with pytest.raises(pbs.PbsError) as e:
        ctx.solve_k(pbs.Geometry(bad), dict(nev=2, block=4), (0.1, 0.1))
    assert e.value.status == pbs.PBS_EINVAL
    with pytest.raises(pbs.PbsError) as e:
        ctx.solve_k(geom, dict(nev=2, block=40), (0.1, 0.1))
    assert e.value.status == pbs.PBS_EINVAL


def test_max_size_operators_on_plane_waves(ctx):
    # 4096 x 4096 (33.5M edges): a discrete Bloch plane wave with eps = 1 is a generalised
    # eigenvector, A x = lambda M x, with lambda from the closed form; A L phi = 0 for any phi.
    n = 4096
    geom = pbs.Geometry(gi.const_eps(n, n, 1.0))
    k = (0.37, -1.21)
    p, q = 3, 5
    h = 1.0 / n
    t1, t2 = (k[0] + 2 * np.pi * p) * h, (k[1] + 2 * np.pi * q) * h
    s1, s2 = np.sin(t1 / 2), np.sin(t2 / 2)
    # rank-one curl-curl symbol 4w a a^T with a = (s2, -s1); eigenvector M^{-1} a of the pencil
    mx, my = (2 + np.cos(t2)) / 3, (2 + np.cos(t1)) / 3
    i = torch.arange(n, dtype=torch.float64, device="cuda")
    J, I = torch.meshgrid(i, i, indexing="ij")
    ex_ = (s2 / mx * torch.exp(1j * (t1 * (I + 0.5) + t2 * J))).reshape(-1)
    ey_ = (-s1 / my * torch.exp(1j * (t1 * I + t2 * (J + 0.5)))).reshape(-1)
    x = torch.cat([ex_, ey_]).reshape(1, -1).contiguous()
    del ex_, ey_
    lam = 6 * (1 - np.cos(t1)) / (h * h * (2 + np.cos(t1))) + 6 * (1 - np.cos(t2)) / (h * h * (2 + np.cos(t2)))
    y = torch.empty_like(x)
    z = torch.empty_like(x)
    opts = pbs.default_opts(mu=MU)
    ctx.apply(geom, "A", x.data_ptr(), y.data_ptr(), 1, k=k, opts=opts)
    ctx.apply(geom, "M", x.data_ptr(), z.data_ptr(), 1, k=k, opts=opts)
    torch.cuda.synchronize()
    rel = (torch.linalg.vector_norm(y - lam * z) / torch.linalg.vector_norm(y)).item()
    assert rel < 1e-9  # rounding of a 33.5M-entry stencil at lambda ~ 1e3
    del y, z
    phi = torch.exp(1j * (k[0] * I * h + k[1] * J * h)).reshape(1, -1).contiguous() * (1 + 0.5j)
    g = torch.empty_like(x)
    ctx.apply(geom, "L", phi.data_ptr(), g.data_ptr(), 1, k=k, opts=opts)
    ag = torch.empty_like(x)
    ctx.apply(geom, "A", g.data_ptr(), ag.data_ptr(), 1, k=k, opts=opts)
    torch.cuda.synchronize()
    assert (torch.linalg.vector_norm(ag) / torch.linalg.vector_norm(g)).item() < 1e-12 * 8 / h ** 2


@pytest.mark.parametrize("precision", [pbs.PBS_FP64, pbs.PBS_MIXED])
def test_rayleigh_ritz_drops_dependent_directions(ctx, precision):
    # a span given twice (second copy mixed by a random matrix) has rank 6: the
    # Cholesky step must drop the dependent half and return the Ritz pairs of the span
    n = 16
    eps = gi.rod_eps(n, n)
    geom = pbs.Geometry(eps)
    k = (0.9, -0.4)
    ops = fem.assemble(fem.Mesh(1, 1, n, n), eps, k)
    r = np.random.default_rng(21)
    V = eigen.eigs_dense(ops, 6)[1] + 1e-3 * (r.standard_normal((geom.D, 6)) + 1j * r.standard_normal((geom.D, 6)))
    mix = r.standard_normal((6, 6)) + 1j * r.standard_normal((6, 6))
    S = np.concatenate([V, V @ mix], axis=1)
    want, _ = ex.rayleigh_ritz(ops, V, 6)
    Sd = _dev(S.T)
    X = torch.zeros((6, geom.D), dtype=torch.complex128, device="cuda")
    th = ctx.rayleigh_ritz(geom, pbs.default_opts(precision=precision), k, 12, Sd.data_ptr(), 6, False,
                           X.data_ptr(), torch.cuda.current_stream())
    assert np.allclose(th, want, rtol=1e-9)
