"""Pins of the generalised Householder oracle (Section 4) against mathematics it must satisfy.

* with M = I and the first q unit vectors as P it is the textbook Householder QR:
  |R| equals numpy's R entry by entry;
* M-QR is unique up to a diagonal unitary, so |R| equals the upper Cholesky factor
  of the M-Gram S^* M S (an independent construction);
* E^* M E = I, E R = S, R upper triangular, every Q_i an M-selfadjoint involution;
* rank loss: a dependent column gives R[i, i] ~ 0, a zero column R[i, i] = 0, and
  E stays M-orthonormal with span(S) inside span(E).
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from oracle import fem
from oracle.householder import basis_P, m_householder, pivots, reflect

pytestmark = pytest.mark.filterwarnings("ignore::scipy.sparse.SparseEfficiencyWarning")


def _rand(shape, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(shape) + 1j * r.standard_normal(shape)


def _mass(n, m, k, seed=0):
    mesh = fem.Mesh(1.0, 0.75, n, m)
    eps = 1.0 + 9.0 * np.random.default_rng(seed).random(n * m)
    return fem.assemble(mesh, eps, k)["M"]


def test_identity_metric_is_textbook_qr():
    D, q = 40, 6
    S = _rand((D, q), 1)
    E, R, _ = m_householder(sp.identity(D, format="csr", dtype=complex), S, np.arange(q))
    _, Rn = np.linalg.qr(S)
    assert np.allclose(np.abs(R), np.abs(Rn), rtol=0, atol=1e-12 * np.abs(Rn).max())
    assert np.allclose(E.conj().T @ E, np.eye(q), atol=1e-13)
    assert np.allclose(E @ R, S, atol=1e-13 * np.abs(S).max())


@pytest.mark.parametrize("n,m,k,q", [(8, 6, (0.7, -1.9), 5), (6, 5, (3.1, 0.4), 9), (12, 8, (0.0, 0.0), 12)])
def test_mass_metric_factorisation(n, m, k, q):
    M = _mass(n, m, k)
    piv = pivots(n, m, q)
    P, _ = basis_P(M, piv)
    assert np.allclose(P.conj().T @ (M @ P), np.eye(q), atol=1e-14)
    S = _rand((M.shape[0], q), 2)
    E, R, refl = m_householder(M, S, piv)
    assert np.allclose(E.conj().T @ (M @ E), np.eye(q), atol=1e-13)
    assert np.allclose(E @ R, S, atol=1e-13 * np.abs(S).max())
    assert np.all(np.tril(R, -1) == 0)
    Rc = sla.cholesky(S.conj().T @ (M @ S), lower=False)
    assert np.allclose(np.abs(R), np.abs(Rc), rtol=0, atol=1e-12 * np.abs(Rc).max())
    # every reflection is an M-selfadjoint involution; applied in order they give P R
    D = M.shape[0]
    Y = S.copy()
    for v, vMv in refl:
        Q = reflect(M, v, vMv, np.eye(D))
        assert np.allclose(Q @ Q, np.eye(D), atol=1e-12)
        MQ = M @ Q
        assert np.allclose(MQ, MQ.conj().T, atol=1e-12)
        Y = reflect(M, v, vMv, Y)
    assert np.allclose(Y, P @ R, atol=1e-12 * np.abs(S).max())


def test_span_matches_gram_projector():
    M = _mass(10, 8, (1.3, 2.2))
    q = 7
    S = _rand((M.shape[0], q), 3)
    E, _, _ = m_householder(M, S, pivots(10, 8, q))
    G = S.conj().T @ (M @ S)
    proj_S = S @ np.linalg.solve(G, S.conj().T @ M.toarray())
    proj_E = E @ (E.conj().T @ M.toarray())
    assert np.allclose(proj_E, proj_S, atol=1e-11)


def test_rank_loss_extends_the_basis():
    n, m, q = 8, 6, 6
    M = _mass(n, m, (0.5, 0.25))
    S = _rand((M.shape[0], q), 4)
    S[:, 2] = 0.3 * S[:, 0] - (1.0 - 2.0j) * S[:, 1]  # dependent up to rounding
    S[:, 4] = 0.0  # exactly zero
    E, R, refl = m_householder(M, S, pivots(n, m, q))
    scale = np.abs(R).max()
    assert abs(R[2, 2]) <= 1e-13 * scale
    assert R[4, 4] == 0 and refl[4] is None
    assert np.allclose(E.conj().T @ (M @ E), np.eye(q), atol=1e-12)
    # span(S) inside span(E): the M-orthogonal projection onto span(E) keeps S
    assert np.allclose(E @ (E.conj().T @ (M @ S)), S, atol=1e-12 * np.abs(S).max())


def test_pivot_limits():
    assert list(pivots(4, 5, 8)) == [0, 1, 2, 3, 8, 9, 10, 11]
    with pytest.raises(ValueError):
        pivots(4, 5, 9)
    M = _mass(4, 5, (0.9, -0.3))
    P, _ = basis_P(M, pivots(4, 5, 8))
    assert np.allclose(P.conj().T @ (M @ P), np.eye(8), atol=1e-14)
