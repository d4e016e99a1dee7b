"""Pins for the oracle's discretisation (Section 3 of the paper) against facts outside the oracle.

Each test checks the assembled matrices against something the paper or the
mathematics fixes independently: hand-integrated element values, Stokes'
theorem on smooth Bloch fields, the discrete de Rham property ``A L = 0``
(eq. potential_discrete), Hermitian/definite structure (Section 1), and the
Galerkin identities of the nested hierarchy (Section 5).
"""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import fem
from oracle.multigrid import level_meshes
import pbs_inputs as gi

CASES = [  # (a, b, n, m, k)
    (1.0, 1.0, 8, 8, (0.7, -0.4)),
    (1.0, 1.3, 6, 4, (2.9, 1.1)),
    (0.8, 1.0, 4, 6, (0.0, 0.0)),
    (1.0, 1.0, 6, 6, (np.pi, np.pi)),
]


def _rand_eps(n, m, seed=3):
    return np.random.default_rng(seed).uniform(1.0, 9.0, (m, n))


def test_paper_dof_count():
    # Section 8: a 1024x1024 mesh carries 2,097,152 Nedelec basis functions.
    txt = open(__file__.replace("test_oracle_fem.py", "golden/paper_sizes.txt")).read()
    want = int([l for l in txt.splitlines() if l.startswith("edge_dofs_1024x1024")][0].split()[1])
    assert fem.Mesh(1.0, 1.0, 1024, 1024).D == want == 2097152


@pytest.mark.parametrize("a,b,n,m,k", CASES)
def test_mass_entries_hand_integrals(a, b, n, m, k):
    # int b_x b_x over the two cells sharing an x-edge: (1/h1^2) * h1 * 2 * h2/3 = (2/3) h2/h1;
    # neighbours across one cell: (1/h1^2) * h1 * h2/6; x and y functions are orthogonal.
    mesh = fem.Mesh(a, b, n, m)
    ops = fem.assemble(mesh, _rand_eps(n, m), k)
    M = ops["M"].toarray()
    h1, h2, N = mesh.h1, mesh.h2, mesh.N
    al, be = ops["alpha"], ops["beta"]
    for (i, j) in [(0, 0), (n - 1, m - 1), (1, 2)]:
        ex = j * n + i
        assert np.isclose(M[ex, ex], 2 / 3 * h2 / h1, rtol=1e-14)
        up = ((j + 1) % m) * n + i
        ph = be if j == m - 1 else 1.0  # the edge above wraps to row 0 with beta
        assert np.isclose(M[ex, up], ph * h2 / h1 / 6, rtol=1e-13)
        ey = N + j * n + i
        assert np.isclose(M[ey, ey], 2 / 3 * h1 / h2, rtol=1e-14)
        rt = N + j * n + (i + 1) % n
        ph = al if i == n - 1 else 1.0
        assert np.isclose(M[ey, rt], ph * h1 / h2 / 6, rtol=1e-13)
    assert np.abs(M[:N, N:]).max() == 0.0


def _exact_edge_dofs(mesh, k, c1, c2):
    """Line integrals of u = exp(i k.x) (c1, c2) along every edge (closed form)."""
    n, m, h1, h2 = mesh.n, mesh.m, mesh.h1, mesh.h2
    jj, ii = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    x0, y0 = ii.ravel() * h1, jj.ravel() * h2

    def seg(kk, s0, h):
        return np.exp(1j * kk * s0) * (np.exp(1j * kk * h) - 1) / (1j * kk)

    ux = c1 * np.exp(1j * k[1] * y0) * seg(k[0], x0, h1)
    uy = c2 * np.exp(1j * k[0] * x0) * seg(k[1], y0, h2)
    return np.concatenate([ux, uy])


@pytest.mark.parametrize("a,b,n,m", [(1.0, 1.0, 8, 8), (1.0, 1.3, 6, 4), (0.7, 1.0, 5, 7)])
def test_curl_matches_stokes_on_bloch_plane_wave(a, b, n, m):
    # u = exp(i k.x)(c1,c2) satisfies the Bloch conditions (eq. bloch_boundary);
    # its edge DOFs are exact line integrals, and the discrete curl of a cell must
    # equal the integral of scurl u = d2 u1 - d1 u2 over the cell (Stokes).
    k = (0.9 / a, -1.7 / b)
    mesh = fem.Mesh(a, b, n, m)
    ops = fem.assemble(mesh, np.ones((m, n)), k)
    c1, c2 = 0.3 - 0.8j, 1.1 + 0.2j
    dofs = _exact_edge_dofs(mesh, k, c1, c2)
    jj, ii = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    x0, y0 = ii.ravel() * mesh.h1, jj.ravel() * mesh.h2

    def seg(kk, s0, h):
        return np.exp(1j * kk * s0) * (np.exp(1j * kk * h) - 1) / (1j * kk)

    cell_int = 1j * (k[1] * c1 - k[0] * c2) * seg(k[0], x0, mesh.h1) * seg(k[1], y0, mesh.h2)
    got = ops["C"] @ dofs
    assert np.allclose(got, cell_int, rtol=1e-12, atol=1e-14)


@pytest.mark.parametrize("a,b,n,m", [(1.0, 1.0, 8, 8), (1.0, 1.3, 6, 4), (0.7, 1.0, 5, 7)])
def test_lifting_is_exact_gradient_of_bloch_function(a, b, n, m):
    # phi = exp(i k.x) * (2 + cos(2 pi x1/a) sin(2 pi x2/b)) satisfies the scalar Bloch
    # conditions (eq. bloch_scalar); the DOF of grad phi on an edge is phi(end) - phi(start),
    # which L applied to the nodal samples must reproduce exactly (eq. potential_discrete).
    k = (1.3 / a, 0.4 / b)
    mesh = fem.Mesh(a, b, n, m)
    ops = fem.assemble(mesh, np.ones((m, n)), k)

    def phi(x1, x2):
        return np.exp(1j * (k[0] * x1 + k[1] * x2)) * (2 + np.cos(2 * np.pi * x1 / a) * np.sin(2 * np.pi * x2 / b))

    jj, ii = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    x0, y0 = ii.ravel() * mesh.h1, jj.ravel() * mesh.h2
    samples = phi(x0, y0)
    want = np.concatenate([phi(x0 + mesh.h1, y0) - phi(x0, y0), phi(x0, y0 + mesh.h2) - phi(x0, y0)])
    assert np.allclose(ops["L"] @ samples, want, rtol=1e-13, atol=1e-13)


@pytest.mark.parametrize("a,b,n,m,k", CASES)
def test_discrete_de_rham(a, b, n, m, k):
    ops = fem.assemble(fem.Mesh(a, b, n, m), _rand_eps(n, m), k)
    scale = abs(ops["A"]).max()
    assert abs(ops["C"] @ ops["L"]).max() < 1e-13
    assert abs(ops["A"] @ ops["L"]).max() < 1e-13 * scale


@pytest.mark.parametrize("a,b,n,m,k", CASES)
def test_hermitian_and_definite(a, b, n, m, k):
    ops = fem.assemble(fem.Mesh(a, b, n, m), _rand_eps(n, m), k)
    A, M = ops["A"].toarray(), ops["M"].toarray()
    assert abs(A - A.conj().T).max() < 1e-13 * abs(A).max()
    assert abs(M - M.conj().T).max() < 1e-15 * abs(M).max() + 1e-16
    ea = np.linalg.eigvalsh(A)
    em = np.linalg.eigvalsh(M)
    assert ea.min() > -1e-12 * ea.max()
    assert em.min() > 0
    # A is the factored form C^* W C (the two are assembled by different integrals)
    C = ops["C"].toarray()
    assert abs(A - C.conj().T @ (ops["w"][:, None] * C)).max() < 1e-13 * abs(A).max()


@pytest.mark.parametrize("gamma", [False, True])
def test_null_space_dimension(gamma):
    # ker A = gradients (n*m-dimensional) for k != 0; at k = 0 the constant potential is
    # lost and the two constant edge fields are added (Lemma 2, k = 0 case): n*m + 1.
    n, m = 6, 4
    k = (0.0, 0.0) if gamma else (0.5, 0.2)
    ops = fem.assemble(fem.Mesh(1.0, 1.0, n, m), _rand_eps(n, m), k)
    lam = sla.eigh(ops["A"].toarray(), ops["M"].toarray(), eigvals_only=True)
    zeros = np.sum(np.abs(lam) < 1e-10 * lam.max())
    assert zeros == n * m + (1 if gamma else 0)


@pytest.mark.parametrize("a,b,n,m,k", [(1.0, 1.0, 8, 8, (0.7, -0.4)), (1.0, 1.3, 8, 4, (2.9, 1.1)),
                                       (1.0, 1.0, 8, 8, (0.0, 0.0))])
def test_galerkin_coarse_operators(a, b, n, m, k):
    # Section 5: the natural embedding makes P^* A_f P the stiffness matrix of the coarse
    # mesh; with a cellwise constant curl this is the coarse assembly with 1/eps averaged
    # over the four children, and P^* M_f P is the coarse mass matrix.
    fine = fem.Mesh(a, b, n, m)
    coarse = fine.coarse()
    eps = _rand_eps(n, m)
    of = fem.assemble(fine, eps, k)
    inv = 1.0 / eps
    inv_c = 0.25 * (inv[0::2, 0::2] + inv[1::2, 0::2] + inv[0::2, 1::2] + inv[1::2, 1::2])
    oc = fem.assemble(coarse, 1.0 / inv_c, k)
    P = fem.edge_prolongation(fine, coarse, k)
    Ac = (P.conj().T @ of["A"] @ P).toarray()
    Mc = (P.conj().T @ of["M"] @ P).toarray()
    assert abs(Ac - oc["A"].toarray()).max() < 1e-12 * abs(Ac).max()
    assert abs(Mc - oc["M"].toarray()).max() < 1e-14 * abs(Mc).max()
    # nodal embedding: gradient of an embedded function = embedded gradient, and the
    # Galerkin nodal operator equals the coarse L^* M L
    Pn = fem.nodal_prolongation(fine, coarse, k)
    assert abs(of["L"] @ Pn - P @ oc["L"]).max() < 1e-14
    Pc = (Pn.conj().T @ of["P"] @ Pn).toarray()
    assert abs(Pc - oc["P"].toarray()).max() < 1e-13 * abs(Pc).max()


def test_embedding_weights_by_hand():
    # A coarse x-edge function contributes 1/2 to each fine edge on it and 1/4 to each fine
    # edge on the midlines of its two cells (linear profile across the cell).
    fine, coarse = fem.Mesh(1.0, 1.0, 8, 8), fem.Mesh(1.0, 1.0, 4, 4)
    k = (0.3, 0.9)
    P = fem.edge_prolongation(fine, coarse, k).toarray()
    be = np.exp(1j * k[1])
    col = 0 * 4 + 1  # coarse x-edge (1, 0): on the wrap row
    nz = {int(r): P[r, col] for r in np.nonzero(np.abs(P[:, col]) > 0)[0]}
    want = {0 * 8 + 2: 0.5, 0 * 8 + 3: 0.5, 1 * 8 + 2: 0.25, 1 * 8 + 3: 0.25,
            7 * 8 + 2: 0.25 * be, 7 * 8 + 3: 0.25 * be}
    assert set(nz) == set(want)
    for r, v in want.items():
        assert np.isclose(nz[r], v, rtol=1e-14)


def test_level_rule():
    assert [(m.n, m.m) for m in level_meshes(fem.Mesh(1, 1, 256, 256), 4)][-1] == (4, 4)
    assert [(m.n, m.m) for m in level_meshes(fem.Mesh(1, 1, 48, 32), 4)] == [(48, 32), (24, 16), (12, 8), (6, 4)]
    assert len(level_meshes(fem.Mesh(1, 1, 6, 6), 4)) == 1


def test_rod_generator_shape_and_symmetry():
    eps = gi.rod_eps(32, 32)
    assert eps.shape == (32, 32)
    assert np.array_equal(eps, eps.T) and np.array_equal(eps, eps[::-1]) and np.array_equal(eps, eps[:, ::-1])
    assert set(np.unique(eps)) == {1.0, 8.9}
