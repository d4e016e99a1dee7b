"""GPU parity of the generalised Householder orthonormalisation (Section 4) through ``pbs_m_householder``.

Expected values come from ``oracle.householder`` on the same seeded blocks.
E and R are compared entry by entry (same algorithm, different summation order
in the M-norms and M-inner products: bar 1e-11 of the largest entry); the
rank-loss cases, whose reflections past the lost column are built from
rounding noise on both sides, are checked by the properties the paper states
(E^* M E = I, span(S) inside span(E)) and by R up to that column.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2304_00337_gb300 as pbs  # noqa: E402
import pbs_inputs as gi  # noqa: E402
from oracle import fem  # noqa: E402
from oracle.householder import m_householder, pivots  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with pbs.Context(0) as c:
        yield c


def _run(ctx, geom, k, S):
    """S: (q, D) rows = columns of the D x q block; returns E (q, D) and R (q x q)."""
    q, D = S.shape
    Sd = torch.from_numpy(np.ascontiguousarray(S)).cuda()
    Ed = torch.zeros((q, D), dtype=torch.complex128, device="cuda")
    Rd = torch.zeros((q, q), dtype=torch.complex128, device="cuda")
    ctx.m_householder(geom, k, q, Sd.data_ptr(), Ed.data_ptr(), Rd.data_ptr(), torch.cuda.current_stream())
    torch.cuda.synchronize()
    assert np.array_equal(Sd.cpu().numpy(), S)  # S is not modified
    return Ed.cpu().numpy(), Rd.cpu().numpy().T


# (a, b, n, m, k, q): ragged sizes, k = 0, a corner of the zone, q at the
# pivot limit n * floor(m / 2)
CASES = [
    (1.0, 20 / 48, 48, 20, (2.1, 0.7), 12),
    (1.0, 1.0, 16, 16, (0.0, 0.0), 30),
    (1.0, 1.0, 16, 16, (np.pi, np.pi), 7),
    (1.3, 0.7, 24, 14, (-1.1, 3.0), 30),
    (1.0, 0.75, 8, 6, (0.4, -2.0), 24),
    (1.0, 1.0, 32, 8, (1.0, 1.0), 1),
]


@pytest.mark.parametrize("a,b,n,m,k,q", CASES)
def test_matches_oracle(ctx, a, b, n, m, k, q):
    eps = np.random.default_rng(5).uniform(1.0, 9.0, (m, n))
    geom = pbs.Geometry(eps, a, b)
    M = fem.assemble(fem.Mesh(a, b, n, m), eps, k)["M"]
    S = gi.random_block(geom.D, q, seed=21)
    E, R = _run(ctx, geom, k, S)
    We, Wr, _ = m_householder(M, S.T, pivots(n, m, q))
    assert np.abs(R - Wr).max() <= 1e-11 * np.abs(Wr).max()
    assert np.abs(E - We.T).max() <= 1e-11 * np.abs(We).max()
    assert np.abs(E.conj() @ (M @ E.T) - np.eye(q)).max() <= 1e-12


def test_rank_loss(ctx):
    a, b, n, m, k, q = 1.0, 1.0, 16, 12, (0.6, -0.9), 8
    eps = np.random.default_rng(6).uniform(1.0, 9.0, (m, n))
    geom = pbs.Geometry(eps, a, b)
    M = fem.assemble(fem.Mesh(a, b, n, m), eps, k)["M"]
    S = gi.random_block(geom.D, q, seed=22)
    S[3] = 0.5 * S[0] + (0.25 - 1.5j) * S[1]  # dependent up to rounding
    S[6] = 0.0  # exactly zero
    E, R = _run(ctx, geom, k, S)
    _, Wr, _ = m_householder(M, S.T, pivots(n, m, q))
    scale = np.abs(Wr).max()
    assert np.abs(R[:, :3] - Wr[:, :3]).max() <= 1e-11 * scale
    assert np.abs(R[:3, 3] - Wr[:3, 3]).max() <= 1e-11 * scale
    assert abs(R[3, 3]) <= 1e-13 * scale and R[6, 6] == 0
    assert np.all(np.tril(R, -1) == 0)
    assert np.abs(E.conj() @ (M @ E.T) - np.eye(q)).max() <= 1e-12
    # span(S) inside span(E), and S = E R
    proj = (E.T @ (E.conj() @ (M @ S.T))).T
    assert np.abs(proj - S).max() <= 1e-12 * np.abs(S).max()
    assert np.abs((E.T @ R).T - S).max() <= 1e-12 * np.abs(S).max()


def test_full_size_bench_block(ctx):
    """256 x 256 rod crystal, 30 columns (the trial width of the bench's iteration) at X."""
    n = m = 256
    k = (np.pi, 0.0)
    eps = gi.rod_eps(n, m, radius=0.2, eps_rod=8.9)
    geom = pbs.Geometry(eps)
    M = fem.assemble(fem.Mesh(1.0, 1.0, n, m), eps, k)["M"]
    q = 30
    S = gi.random_block(geom.D, q, seed=23)
    E, R = _run(ctx, geom, k, S)
    We, Wr, _ = m_householder(M, S.T, pivots(n, m, q))
    assert np.abs(R - Wr).max() <= 1e-11 * np.abs(Wr).max()
    assert np.abs(E - We.T).max() <= 1e-11 * np.abs(We).max()
    assert np.abs(E.conj() @ (M @ E.T) - np.eye(q)).max() <= 1e-12


def test_invalid_widths(ctx):
    eps = np.ones((6, 8))
    geom = pbs.Geometry(eps)
    S = torch.zeros((25, geom.D), dtype=torch.complex128, device="cuda")
    E = torch.zeros_like(S)
    R = torch.zeros((25, 25), dtype=torch.complex128, device="cuda")
    with pytest.raises(pbs.PbsError):
        ctx.m_householder(geom, (0.1, 0.2), 25, S.data_ptr(), E.data_ptr(), R.data_ptr())  # 25 > 8 * 3
    ctx.m_householder(geom, (0.1, 0.2), 0, S.data_ptr(), E.data_ptr(), R.data_ptr())  # empty: no work
