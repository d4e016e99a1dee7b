"""Reference multigrid for ``A + mu M`` (edges) and ``P = L^* M L`` (nodes) - ORACLE, test infrastructure.

Follows Section 5 of the paper ("Geometric multigrid method") step by step,
with assembled sparse matrices and plain loops:

* hierarchy by bisection; prolongation = natural embedding of the coarse
  space (``fem.edge_prolongation`` / ``fem.nodal_prolongation``); coarse
  matrices by the Galerkin product ``P^* K P``;
* edge smoother: block Gauss-Seidel over the overlapping node patches (the four
  edges at a node, periodicity included), each patch system solved exactly;
* nodal smoother: point Gauss-Seidel;
* coarsest level: dense direct solve.

Readings where the paper is silent (shared with the GPU path as a
specification, not as code):

* nodes are visited colour by colour, colour ``(i mod 2, j mod 2)`` in the
  order (0,0), (1,0), (0,1), (1,1) for pre-smoothing and the reverse order
  for post-smoothing, so the cycle is a symmetric (Hermitian) operator;
  within a colour nodes are visited in increasing index (same-colour patches
  are uncoupled, so the order inside a colour does not change the result);
* V(nu_pre, nu_post) cycle started from zero;
* levels: coarsen while both sides are even and at least ``2*coarsest``;
* at k = 0 the nodal system is singular (constants); the coarsest nodal solve
  returns the minimum-norm (zero-mean) solution.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from .fem import Mesh, assemble, edge_prolongation, nodal_prolongation, is_gamma

__all__ = ["level_meshes", "edge_hierarchy", "nodal_hierarchy", "edge_vcycle", "nodal_vcycle",
           "edge_patch", "COLOUR_ORDER", "project_exact", "project_approx"]

COLOUR_ORDER = ((0, 0), (1, 0), (0, 1), (1, 1))


def level_meshes(mesh: Mesh, coarsest: int):
    """Meshes of the bisection hierarchy, finest first."""
    out = [mesh]
    while True:
        f = out[-1]
        if f.n % 2 or f.m % 2 or f.n // 2 < coarsest or f.m // 2 < coarsest:
            break
        out.append(f.coarse())
    return out


def edge_patch(mesh: Mesh, i: int, j: int):
    """Global DOFs of the node patch at ``(i, j)``: left, right, bottom, top edges."""
    n, m, N = mesh.n, mesh.m, mesh.N
    return np.array([j * n + (i - 1) % n, j * n + i, N + ((j - 1) % m) * n + i, N + j * n + i])


def edge_hierarchy(mesh: Mesh, eps, k, mu: float, coarsest: int):
    """Levels ``[{mesh, K, P}]``: ``K = A + mu M`` on the finest level, Galerkin products below.

    ``P`` of level ``l`` maps level ``l+1`` (coarse) to level ``l``.
    """
    ops = assemble(mesh, eps, k)
    meshes = level_meshes(mesh, coarsest)
    K = (ops["A"] + mu * ops["M"]).tocsr()
    levels = []
    for li, msh in enumerate(meshes):
        lev = dict(mesh=msh, K=K)
        if li + 1 < len(meshes):
            P = edge_prolongation(msh, meshes[li + 1], k)
            lev["P"] = P
            K = (P.conj().T @ K @ P).tocsr()
        levels.append(lev)
    levels[-1]["dense"] = levels[-1]["K"].toarray()
    return levels


def nodal_hierarchy(mesh: Mesh, eps, k, coarsest: int):
    """Levels for ``P = L^* M L`` (the nodal Bloch Laplacian), Galerkin products below."""
    ops = assemble(mesh, eps, k)
    meshes = level_meshes(mesh, coarsest)
    K = ops["P"].tocsr()
    levels = []
    for li, msh in enumerate(meshes):
        lev = dict(mesh=msh, K=K)
        if li + 1 < len(meshes):
            Pn = nodal_prolongation(msh, meshes[li + 1], k)
            lev["P"] = Pn
            K = (Pn.conj().T @ K @ Pn).tocsr()
        levels.append(lev)
    levels[-1]["dense"] = levels[-1]["K"].toarray()
    levels[-1]["gamma"] = is_gamma(ops["alpha"], ops["beta"])
    return levels


def _nodes_of_colour(mesh: Mesh, colour):
    ci, cj = colour
    return [(i, j) for j in range(cj, mesh.m, 2) for i in range(ci, mesh.n, 2)]


def edge_smooth(level, x, b, order):
    """One block Gauss-Seidel sweep over node patches, colours in ``order``."""
    K = level["K"]
    msh = level["mesh"]
    for colour in order:
        for (i, j) in _nodes_of_colour(msh, colour):
            idx = edge_patch(msh, i, j)
            r = b[idx] - K[idx, :] @ x
            Kl = K[idx, :][:, idx].toarray()
            x[idx] += np.linalg.solve(Kl, r)
    return x


def nodal_smooth(level, x, b, order):
    """One point Gauss-Seidel sweep, colours in ``order``."""
    K = level["K"]
    msh = level["mesh"]
    diag = K.diagonal()
    for colour in order:
        for (i, j) in _nodes_of_colour(msh, colour):
            g = j * msh.n + i
            r = b[g] - (K[g, :] @ x)[0]
            x[g] += r / diag[g]
    return x


def _coarse_solve(level, b, singular=False):
    Kd = level["dense"]
    if singular:
        return np.linalg.lstsq(Kd, b, rcond=None)[0]
    return sla.solve(Kd, b, assume_a="her")


def edge_vcycle(levels, b, nu_pre: int = 1, nu_post: int = 1, li: int = 0):
    """``x = B b``: one V(nu_pre, nu_post) cycle for ``A + mu M`` from ``x = 0``."""
    lev = levels[li]
    if li == len(levels) - 1:
        return _coarse_solve(lev, b)
    x = np.zeros_like(b)
    for _ in range(nu_pre):
        edge_smooth(lev, x, b, COLOUR_ORDER)
    r = b - lev["K"] @ x
    xc = edge_vcycle(levels, lev["P"].conj().T @ r, nu_pre, nu_post, li + 1)
    x += lev["P"] @ xc
    for _ in range(nu_post):
        edge_smooth(lev, x, b, COLOUR_ORDER[::-1])
    return x


def nodal_vcycle(levels, b, nu_pre: int = 1, nu_post: int = 1, li: int = 0):
    """``x = B_P b``: one V(nu_pre, nu_post) cycle for the nodal operator from ``x = 0``."""
    lev = levels[li]
    if li == len(levels) - 1:
        return _coarse_solve(lev, b, singular=levels[-1]["gamma"])
    x = np.zeros_like(b)
    for _ in range(nu_pre):
        nodal_smooth(lev, x, b, COLOUR_ORDER)
    r = b - lev["K"] @ x
    xc = nodal_vcycle(levels, lev["P"].conj().T @ r, nu_pre, nu_post, li + 1)
    x += lev["P"] @ xc
    for _ in range(nu_post):
        nodal_smooth(lev, x, b, COLOUR_ORDER[::-1])
    return x


def _gamma_fields(mesh: Mesh):
    N = mesh.N
    zx = np.concatenate([np.ones(N), np.zeros(N)])
    zy = np.concatenate([np.zeros(N), np.ones(N)])
    return zx, zy


def project_exact(ops, U):
    """Exact M-orthogonal projection of the columns of ``U`` off ``ker A`` (Section 4).

    Solves ``L^* M L phi = L^* M u`` and returns ``u - L phi``; at ``k = 0`` the
    two constant edge fields are M-projected out as well (the first option of
    Section 4 for the k = 0 remainder).
    """
    L, M, P = ops["L"], ops["M"], ops["P"]
    U = np.array(U, dtype=complex, copy=True)
    rhs = L.conj().T @ (M @ U)
    gamma = is_gamma(ops["alpha"], ops["beta"])
    if gamma:
        phi = np.linalg.lstsq(P.toarray(), rhs, rcond=None)[0] if P.shape[0] <= 4096 else \
            _singular_solve(P, rhs)
    else:
        phi = spla.spsolve(P.tocsc(), rhs)
    phi = phi.reshape(rhs.shape)
    U -= L @ phi
    if gamma:
        for z in _gamma_fields(ops["mesh"]):
            Mz = M @ z
            coef = (Mz.conj() @ U) / np.real(Mz.conj() @ z)
            U -= np.outer(z, coef) if U.ndim == 2 else z * coef
    return U


def _singular_solve(P, rhs):
    """Zero-mean solution of the consistent singular system ``P phi = rhs`` (constants span the kernel)."""
    N = P.shape[0]
    one = np.ones(N) / np.sqrt(N)
    Preg = (P + sp.csr_matrix(np.outer(one, one))).tocsc()
    return spla.spsolve(Preg, rhs)


def project_approx(ops, nodal_levels, U, cycles: int, nu_pre: int = 1, nu_post: int = 1):
    """Approximate projection: ``cycles`` nodal V-cycles on ``P phi = L^* M u`` from ``phi = 0``,
    then ``u - L phi`` (and the k = 0 constant-field removal), column by column."""
    L, M, P = ops["L"], ops["M"], ops["P"]
    U = np.array(U, dtype=complex, copy=True)
    cols = U if U.ndim == 2 else U[:, None]
    out = np.empty_like(cols)
    gamma = is_gamma(ops["alpha"], ops["beta"])
    for c in range(cols.shape[1]):
        u = cols[:, c].copy()
        rhs = L.conj().T @ (M @ u)
        phi = np.zeros_like(rhs)
        for _ in range(cycles):
            phi += nodal_vcycle(nodal_levels, rhs - P @ phi, nu_pre, nu_post)
        u -= L @ phi
        if gamma:
            for z in _gamma_fields(ops["mesh"]):
                Mz = M @ z
                u -= z * ((Mz.conj() @ u) / np.real(Mz.conj() @ z))
        out[:, c] = u
    return out if U.ndim == 2 else out[:, 0]
