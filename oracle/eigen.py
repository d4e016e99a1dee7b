"""Smallest non-zero eigenpairs of the Bloch pencil ``A e = lambda M e`` (ORACLE, test infrastructure).

What the GPU iteration converges to has a plain definition: the ``count``
smallest eigenvalues of ``(A(k), M(k))`` on the M-orthogonal complement of
``ker A`` (Section 1, eq. matrix; Section 4 on eliminating the null space).
This module computes that definition directly:

* ``eigs_dense``: ``scipy.linalg.eigh`` of the assembled pencil; the zero
  cluster (``N`` eigenvalues for ``k != 0``, ``N + 1`` at ``k = 0``) is removed
  and its size checked.
* ``eigs_reduced``: brute force through the cell-based reduced operator
  ``W^{1/2} C M^{-1} C^* W^{1/2}`` whose non-zero spectrum equals the pencil's.
* ``eigs_sparse``: ARPACK shift-invert at ``sigma = 0`` on the pencil
  constrained to ``L^* M e = 0`` (plus the two constant edge fields at
  ``k = 0``), one sparse LU of the saddle-point matrix.
* ``rayleigh``: factored Rayleigh quotients ``(Ce)^* W (Ce) / e^* M e``.
* ``closed_form_eps_const``: the exact discrete spectrum for constant ``eps``
  (symbol of the stencils on discrete plane waves).
* ``certify_pairs``: a posteriori checks of given approximate eigenpairs on the
  assembled pencil (residuals, the constraint ``L^* M e = 0``, M-orthonormality
  and the residual-over-gap bound on each eigenvalue), for meshes too large for
  a direct solve.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import Mesh, assemble, is_gamma

__all__ = ["closed_form_eps_const", "eigs_dense", "eigs_reduced", "eigs_sparse",
           "rayleigh", "solve_k", "null_dimension", "certify_pairs"]


def closed_form_eps_const(a: float, b: float, n: int, m: int, eps: float, k, count: int) -> np.ndarray:
    """Exact non-zero spectrum of the discrete pencil for constant ``eps``.

    On a discrete Bloch plane wave with angles ``theta = (k + 2 pi (p/a, q/b)) * (h1, h2)``
    (``p in [0,n)``, ``q in [0,m)``) the curl-curl symbol has rank one and the
    mass symbol is ``diag((h2/h1)(2+cos t2)/3, (h1/h2)(2+cos t1)/3)``; the
    non-zero generalised eigenvalue is
    ``(1/eps) [6 (1-cos t1) / (h1^2 (2+cos t1)) + 6 (1-cos t2) / (h2^2 (2+cos t2))]``.
    The wave with both angles zero (only at ``k = 0``) gives the extra zero.
    """
    h1, h2 = a / n, b / m
    p = np.arange(n)
    q = np.arange(m)
    t1 = (k[0] + 2 * np.pi * p / a) * h1
    t2 = (k[1] + 2 * np.pi * q / b) * h2
    # 1 - cos t written as 2 sin^2(t/2): the same value without the cancellation
    # that costs u / (t^2 / 2) relative accuracy for small angles (fine meshes near k = 0)
    f1 = 12 * np.sin(t1 / 2) ** 2 / (h1 ** 2 * (2 + np.cos(t1)))
    f2 = 12 * np.sin(t2 / 2) ** 2 / (h2 ** 2 * (2 + np.cos(t2)))
    lam = (f1[None, :] + f2[:, None]).ravel() / eps
    lam = np.sort(lam)
    # drop exact zeros (the constant wave at k = 0)
    scale = lam.max()
    lam = lam[lam > 1e-12 * scale]
    return lam[:count]


def null_dimension(n: int, m: int, gamma: bool) -> int:
    """Dimension of ``ker A``: the ``n*m`` gradients, plus the two constant fields at k = 0
    minus the constant potential (whose gradient vanishes)."""
    return n * m + (1 if gamma else 0)


def rayleigh(ops, X: np.ndarray) -> np.ndarray:
    """Rayleigh quotients of the columns of ``X`` (shape ``(D, q)``) in factored form.

    ``e^* A e`` is evaluated as ``sum_c w_c |(Ce)_c|^2`` (non-negative terms) to
    avoid the cancellation of ``e^*(Ae)``.
    """
    CX = ops["C"] @ X
    num = np.einsum("c,cq->q", ops["w"], np.abs(CX) ** 2)
    den = np.real(np.einsum("dq,dq->q", X.conj(), ops["M"] @ X))
    return num / den


def _normalize_M(ops, X):
    nrm = np.sqrt(np.real(np.einsum("dq,dq->q", X.conj(), ops["M"] @ X)))
    return X / nrm


def eigs_dense(ops, count: int, vectors: bool = True):
    """Dense generalised Hermitian eigensolve; removes and checks the zero cluster."""
    mesh: Mesh = ops["mesh"]
    A = ops["A"].toarray()
    M = ops["M"].toarray()
    lam, V = sla.eigh(A, M)
    nz = null_dimension(mesh.n, mesh.m, is_gamma(ops["alpha"], ops["beta"]))
    # the zero cluster is separated from the smallest positive eigenvalue by many orders
    gap_ok = abs(lam[nz - 1]) < 1e-10 * lam[-1] and lam[nz] > 1e-10 * lam[-1]
    if not gap_ok:
        raise RuntimeError("eigs_dense: unexpected size of the zero cluster")
    lam = lam[nz:nz + count]
    V = V[:, nz:nz + count]
    if not vectors:
        return lam
    V = _normalize_M(ops, V)
    return rayleigh(ops, V), V


def eigs_reduced(ops, count: int) -> np.ndarray:
    """Brute force via ``K = W^{1/2} C M^{-1} C^* W^{1/2}`` (dense, cell-based).

    For ``A = C^* W C`` the non-zero eigenvalues of ``(A, M)`` coincide with the
    non-zero eigenvalues of ``K`` (same non-zero spectrum as ``M^{-1} C^* W C``).
    """
    C = ops["C"].toarray()
    sw = np.sqrt(ops["w"])
    Minv_Ch = sla.solve(ops["M"].toarray(), C.conj().T, assume_a="her")
    K = (sw[:, None] * (C @ Minv_Ch)) * sw[None, :]
    K = 0.5 * (K + K.conj().T)
    lam = np.linalg.eigvalsh(K)
    lam = lam[lam > 1e-10 * lam[-1]]
    return lam[:count]


def _constraint_matrix(ops):
    """Rows ``B`` with ``ker B`` = M-orthogonal complement of ``ker A``.

    ``k != 0``: ``B = L^* M``.  ``k = 0``: ``L 1 = 0`` makes one row of ``L^* M``
    redundant (row 0 is dropped) and the constant edge fields ``z_x, z_y``
    (in ``ker A`` but not gradients, Lemma 2 case k = 0) add two rows.
    """
    L, M = ops["L"], ops["M"]
    B = (L.conj().T @ M).tocsr()
    if is_gamma(ops["alpha"], ops["beta"]):
        N = ops["mesh"].N
        zx = np.concatenate([np.ones(N), np.zeros(N)])
        zy = np.concatenate([np.zeros(N), np.ones(N)])
        Z = sp.csr_matrix(np.vstack([(M @ zx).conj(), (M @ zy).conj()]))
        B = sp.vstack([B[1:], Z]).tocsr()
    return B


def eigs_sparse(ops, count: int, tol: float = 1e-14, ncv: int | None = None, seed: int = 7):
    """ARPACK shift-invert (sigma = 0) on the constrained pencil.

    ``OPinv(f)`` returns ``x`` from the saddle-point system
    ``[[A, B^*], [B, 0]] [x; y] = [f; 0]``, i.e. the inverse of ``A`` on
    ``ker B`` (where ``A`` is definite).  In ARPACK's generalised mode 3 its
    largest eigenvalues ``1/lambda`` belong to the smallest non-zero
    ``lambda``; directions outside ``ker B`` are mapped to zero.  Eigenvalues
    are then refined as factored Rayleigh quotients.
    """
    A, M = ops["A"].tocsc(), ops["M"].tocsc()
    B = _constraint_matrix(ops)
    r = B.shape[0]
    K = sp.bmat([[A, B.conj().T], [B, None]], format="csc")
    lu = spla.splu(K, permc_spec="COLAMD", diag_pivot_thresh=0.1)
    D = A.shape[0]

    def solve(f):
        rhs = np.concatenate([f, np.zeros(r, complex)])
        return lu.solve(rhs)[:D]

    OPinv = spla.LinearOperator((D, D), matvec=solve, dtype=complex)
    rng = np.random.default_rng(seed)
    v0 = solve(M @ (rng.standard_normal(D) + 1j * rng.standard_normal(D)))
    nev = count + 2
    ncv = ncv or max(2 * nev + 1, 24)
    vals, vecs = spla.eigsh(A, k=nev, M=M, sigma=0.0, OPinv=OPinv, which="LM",
                            tol=tol, ncv=ncv, v0=v0)
    order = np.argsort(vals)
    vecs = _normalize_M(ops, vecs[:, order[:count]])
    return rayleigh(ops, vecs), vecs


def solve_k(a: float, b: float, n: int, m: int, eps, k, count: int, method: str = "auto"):
    """Assemble and return ``(eigenvalues, M-normalised eigenvectors, ops)`` at one Bloch vector."""
    ops = assemble(Mesh(a, b, n, m), eps, k)
    if method == "auto":
        method = "dense" if 2 * n * m <= 2048 else "sparse"
    if method == "dense":
        lam, V = eigs_dense(ops, count)
    else:
        lam, V = eigs_sparse(ops, count)
    return lam, V, ops


def _cg(M, r, iters: int = 60):
    """``M^-1 r`` by plain conjugate gradients (M Hermitian positive definite, well conditioned)."""
    x = np.zeros_like(r)
    res = r.copy()
    p = res.copy()
    rr = np.real(np.vdot(res, res))
    r0 = rr
    for _ in range(iters):
        if rr <= 1e-32 * r0:
            break
        Mp = M @ p
        alpha = rr / np.real(np.vdot(p, Mp))
        x += alpha * p
        res -= alpha * Mp
        rn = np.real(np.vdot(res, res))
        p = res + (rn / rr) * p
        rr = rn
    return x


def certify_pairs(ops, lam, V, cluster_rtol: float = 1e-6):
    """A posteriori certificate of approximate eigenpairs ``(lam[j], V[:, j])`` of the pencil.

    For a Hermitian pencil with ``M`` positive definite and an M-normalised vector
    ``e`` with Rayleigh quotient ``rho`` and residual ``r = A e - rho M e``, some
    eigenvalue lies within ``eta = ||r||_{M^-1}`` of ``rho``; if the interval
    ``(rho - delta, rho + delta)`` holds no other eigenvalue, the distance shrinks
    to ``eta^2 / delta`` (Kato-Temple).  Values closer than ``cluster_rtol``
    (relative) form a cluster (degenerate bands) and share the gap ``delta`` from
    the cluster to the nearest other value of ``lam``, with ``eta^2`` summed over
    the cluster.  The gap is taken between the given values: the bound says each
    value is that close to an eigenvalue of the pencil, not which one.

    Returns a dict of arrays over the columns: ``rq`` (factored Rayleigh quotients),
    ``res`` (``||A e - lam M e||_2 / (lam ||M e||_2)``), ``constraint``
    (``||L^* M e||_2 / (||L||_1 ||M e||_2)``, zero on ``(ker A)^{perp M}``),
    ``bound`` (the residual-over-gap bound, relative to ``lam``) and the scalar
    ``orth`` (``max |V^* M V - I|``).
    """
    A, M, L = ops["A"], ops["M"], ops["L"]
    V = np.asarray(V, complex)
    lam = np.asarray(lam, float)
    MV = M @ V
    G = V.conj().T @ MV
    orth = float(np.abs(G - np.eye(V.shape[1])).max())
    rq = rayleigh(ops, V)
    R = A @ V - MV * lam[None, :]
    res = np.linalg.norm(R, axis=0) / (np.abs(lam) * np.linalg.norm(MV, axis=0))
    lnorm = float(np.abs(L).sum(axis=0).max())  # ||L||_1: the largest column sum
    constraint = np.linalg.norm(L.conj().T @ MV, axis=0) / (lnorm * np.linalg.norm(MV, axis=0))
    # ||r||_{M^-1}^2 = r^* M^-1 r with the vector normalised in the M-norm; M^-1 r by
    # conjugate gradients (the 1-D mass stencils [1/6, 2/3, 1/6] give cond(M) <= 3)
    eta2 = np.array([np.real(np.vdot(R[:, j], _cg(M, R[:, j]))) for j in range(V.shape[1])])
    eta2 /= np.real(np.einsum("dq,dq->q", V.conj(), MV))
    order = np.argsort(lam)
    bound = np.zeros_like(lam)
    j = 0
    while j < len(order):
        c = [order[j]]
        while j + len(c) < len(order) and lam[order[j + len(c)]] - lam[c[-1]] <= cluster_rtol * abs(lam[c[-1]]):
            c.append(order[j + len(c)])
        others = [lam[t] for t in order if t not in c]
        lo, hi = min(lam[c]), max(lam[c])
        delta = min([abs(x - lo) if x < lo else abs(x - hi) for x in others], default=np.inf)
        e2 = eta2[c].sum()
        for t in c:
            bound[t] = min(np.sqrt(e2), e2 / delta) / abs(lam[t])
        j += len(c)
    return dict(rq=rq, res=res, constraint=constraint, bound=bound, orth=orth)
