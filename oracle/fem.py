"""Bloch-twisted Nedelec / Q1 discretisation, assembled from element integrals.

ORACLE - test infrastructure only. Plain FP64 NumPy/SciPy; shares no code with
the CUDA path. Follows Section 3 ("Discretization") of Boerm, Koehl, Talebi,
"Computing Maxwell eigenmodes with Bloch boundary conditions" (arXiv:2304.00337).

Zero-based translation of the paper's one-based definitions (Section 3):

* cell ``(i, j)`` is ``[i h1, (i+1) h1] x [j h2, (j+1) h2]``, ``h1 = a/n``, ``h2 = b/m``;
* x-edge ``(i, j)`` is the segment ``[i h1, (i+1) h1] x {j h2}``; its basis
  function rises over the cell below and falls over the cell above.  For
  ``j = 0`` the cell below is the top row ``j = m-1`` and carries the factor
  ``beta = exp(i k2 b)`` (the paper's case ``i2 = m``);
* y-edge ``(i, j)`` is ``{i h1} x [j h2, (j+1) h2]``; the cell to its left for
  ``i = 0`` is column ``n-1`` with the factor ``alpha = exp(i k1 a)``.  (The
  paper prints a stray third component in the first case of ``b_{y,i}``; the
  two-component reading is used.)
* node ``(i, j)`` sits at ``(i h1, j h2)``; the one-dimensional hat of node
  ``i = 0`` carries ``alpha`` on its rising piece ``[(n-1) h1, a]``.

DOF numbering: x-edge ``(i,j) -> j*n + i``; y-edge ``(i,j) -> N + j*n + i``;
node / cell ``(i,j) -> j*n + i`` with ``N = n*m``.

The DOF of an edge is the line integral of the tangential component along the
edge instance inside ``[0,a] x [0,b]``.  Matrices (Section 3, "The matrices"):
``A[r,c] = a(b_r, b_c)``, ``M[r,c] = m(b_r, b_c)`` with the sesquilinear forms of
eq. (variational); ``C[cell, e] = int_cell scurl b_e`` so that ``A = C^* W C``
with ``W = diag(1/(eps_c h1 h2))``; ``L[e, node]`` holds the DOFs of the
gradient of a nodal basis function (eq. potential_discrete).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

__all__ = ["Mesh", "bloch_phases", "x_edge_basis", "y_edge_basis", "nodal_basis",
           "assemble", "edge_prolongation", "nodal_prolongation", "is_gamma"]

# two-point Gauss rule on [0, 1]: exact for cubic integrands
_GX = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
_GW = np.array([0.5, 0.5])


class Mesh:
    """Regular ``n x m`` mesh of the cell ``[0,a] x [0,b]`` (Section 3)."""

    def __init__(self, a: float, b: float, n: int, m: int):
        if n < 2 or m < 2:
            raise ValueError("need n, m >= 2")
        self.a, self.b, self.n, self.m = float(a), float(b), int(n), int(m)
        self.h1, self.h2 = self.a / n, self.b / m
        self.N = n * m
        self.D = 2 * self.N

    def coarse(self) -> "Mesh":
        """Mesh of the next coarser level (bisection hierarchy, Section 5)."""
        if self.n % 2 or self.m % 2:
            raise ValueError("mesh cannot be coarsened")
        return Mesh(self.a, self.b, self.n // 2, self.m // 2)


def bloch_phases(k, a: float, b: float):
    """``alpha = exp(i k1 a)``, ``beta = exp(i k2 b)`` (Section 1, eq. bloch_boundary)."""
    return np.exp(1j * k[0] * a), np.exp(1j * k[1] * b)


def is_gamma(alpha: complex, beta: complex, tol: float = 1e-14) -> bool:
    """True when both phases equal one, i.e. the Bloch vector is a lattice point (k = 0)."""
    return abs(alpha - 1.0) < tol and abs(beta - 1.0) < tol


def _cell_of(x, h, count):
    c = np.floor(x / h).astype(np.int64)
    return np.clip(c, 0, count - 1)


def x_edge_basis(mesh: Mesh, alpha, beta, i, j, x1, x2):
    """Value ``(v1, v2)`` and scalar curl of the x-edge function ``b_{x,(i,j)}`` at ``(x1, x2)``.

    Arrays broadcast together.  The point is located in the cell given by
    ``floor`` of its coordinates (a point on a cell boundary is taken in the
    cell above / to the right; the functions are tangentially continuous).
    """
    n, m, h1, h2 = mesh.n, mesh.m, mesh.h1, mesh.h2
    i, j, x1, x2 = np.broadcast_arrays(np.asarray(i), np.asarray(j), np.asarray(x1, float), np.asarray(x2, float))
    ci = _cell_of(x1, h1, n)
    cj = _cell_of(x2, h2, m)
    t = x2 / h2
    v1 = np.zeros(i.shape, complex)
    curl = np.zeros(i.shape, complex)
    col = ci == i
    # paper case i2 < m  ->  zero-based j >= 1
    inner = j >= 1
    rise = col & inner & (cj == j - 1)
    fall = col & inner & (cj == j)
    v1[rise] = (t[rise] - (j[rise] - 1)) / h1
    curl[rise] = 1.0 / (h1 * h2)
    v1[fall] = ((j[fall] + 1) - t[fall]) / h1
    curl[fall] = -1.0 / (h1 * h2)
    # paper case i2 = m  ->  zero-based j = 0, wrapping over the top row with beta
    wrap = j == 0
    rise = col & wrap & (cj == m - 1)
    fall = col & wrap & (cj == 0)
    v1[rise] = beta * (t[rise] - (m - 1)) / h1
    curl[rise] = beta / (h1 * h2)
    v1[fall] = (1.0 - t[fall]) / h1
    curl[fall] = -1.0 / (h1 * h2)
    return v1, np.zeros_like(v1), curl


def y_edge_basis(mesh: Mesh, alpha, beta, i, j, x1, x2):
    """Value ``(v1, v2)`` and scalar curl of the y-edge function ``b_{y,(i,j)}`` at ``(x1, x2)``.

    ``scurl u = d2 u1 - d1 u2`` (Section 1), so a y-edge function rising in x1
    has curl ``-1/(h1 h2)`` times its phase.
    """
    n, m, h1, h2 = mesh.n, mesh.m, mesh.h1, mesh.h2
    i, j, x1, x2 = np.broadcast_arrays(np.asarray(i), np.asarray(j), np.asarray(x1, float), np.asarray(x2, float))
    ci = _cell_of(x1, h1, n)
    cj = _cell_of(x2, h2, m)
    t = x1 / h1
    v2 = np.zeros(i.shape, complex)
    curl = np.zeros(i.shape, complex)
    row = cj == j
    inner = i >= 1
    rise = row & inner & (ci == i - 1)
    fall = row & inner & (ci == i)
    v2[rise] = (t[rise] - (i[rise] - 1)) / h2
    curl[rise] = -1.0 / (h1 * h2)
    v2[fall] = ((i[fall] + 1) - t[fall]) / h2
    curl[fall] = 1.0 / (h1 * h2)
    wrap = i == 0
    rise = row & wrap & (ci == n - 1)
    fall = row & wrap & (ci == 0)
    v2[rise] = alpha * (t[rise] - (n - 1)) / h2
    curl[rise] = -alpha / (h1 * h2)
    v2[fall] = (1.0 - t[fall]) / h2
    curl[fall] = 1.0 / (h1 * h2)
    return np.zeros_like(v2), v2, curl


def _hat(x, i, h, count, phase):
    """One-dimensional Bloch hat of node ``i`` (Section 3, phi_{x,i} / phi_{y,j}).

    Pieces are tried in order (rising, then falling); at a shared breakpoint
    both give the same value, so the first match is taken.
    """
    x, i = np.broadcast_arrays(np.asarray(x, float), np.asarray(i))
    out = np.zeros(x.shape, complex)
    done = np.zeros(x.shape, bool)
    s = x / h
    inner = i >= 1
    # node i >= 1: rising on [(i-1)h, ih], falling on [ih, (i+1)h]
    r = inner & (s >= i - 1) & (s <= i)
    out[r] = s[r] - (i[r] - 1); done |= r
    f = inner & ~done & (s >= i) & (s <= i + 1)
    out[f] = (i[f] + 1) - s[f]; done |= f
    # node 0 (the paper's i = n): rising piece next to the far boundary carries the phase
    w = i == 0
    r = w & ~done & (s >= count - 1) & (s <= count)
    out[r] = phase * (s[r] - (count - 1)); done |= r
    f = w & ~done & (s >= 0) & (s <= 1)
    out[f] = 1.0 - s[f]
    return out


def nodal_basis(mesh: Mesh, alpha, beta, i, j, x1, x2):
    """Bloch Q1 nodal function ``varphi_(i,j)(x) = phi_{x,i}(x1) phi_{y,j}(x2)`` (Section 3)."""
    return _hat(x1, i, mesh.h1, mesh.n, alpha) * _hat(x2, j, mesh.h2, mesh.m, beta)


def _edge_ids(mesh: Mesh):
    n, m = mesh.n, mesh.m
    jj, ii = np.meshgrid(np.arange(m), np.arange(n), indexing="ij")
    return ii.ravel(), jj.ravel()


def _eval_edge(mesh, alpha, beta, kind, i, j, x1, x2):
    if kind == 0:
        return x_edge_basis(mesh, alpha, beta, i, j, x1, x2)
    return y_edge_basis(mesh, alpha, beta, i, j, x1, x2)


def assemble(mesh: Mesh, eps, k):
    """Assemble the Galerkin matrices for permittivity samples ``eps`` and Bloch vector ``k``.

    ``eps`` holds one sample per cell (shape ``(m, n)`` or flat ``j*n+i``);
    ``1/eps`` is constant on each cell (the reading of the paper's "standard
    quadrature" for a piecewise-constant permittivity).  Per cell the four
    edge functions with support there are integrated with a 2x2 Gauss rule
    (exact: the integrands are at most bilinear products).

    Returns a dict with sparse ``A, M, C, L, P`` (``P = L^* M L``), the diagonal
    weights ``w`` (``A = C^* diag(w) C``), the phases and the mesh.
    """
    n, m, h1, h2, N = mesh.n, mesh.m, mesh.h1, mesh.h2, mesh.N
    eps = np.asarray(eps, float).reshape(-1)
    if eps.size != N or np.any(~(eps > 0)):
        raise ValueError("eps must hold n*m positive samples")
    alpha, beta = bloch_phases(k, mesh.a, mesh.b)
    ci, cj = _edge_ids(mesh)  # cells, same enumeration
    cell = cj * n + ci
    area = h1 * h2
    # the four edges touching each cell: (kind, i, j, global index)
    slots = [
        (0, ci, cj, cj * n + ci),                                  # bottom x-edge
        (0, ci, (cj + 1) % m, ((cj + 1) % m) * n + ci),            # top x-edge
        (1, ci, cj, N + cj * n + ci),                              # left y-edge
        (1, (ci + 1) % n, cj, N + cj * n + (ci + 1) % n),          # right y-edge
    ]
    vals = []  # per slot: list over gauss points of (v1, v2, curl)
    for (kind, si, sj, _) in slots:
        per_g = []
        for g1 in range(2):
            for g2 in range(2):
                x1 = (ci + _GX[g1]) * h1
                x2 = (cj + _GX[g2]) * h2
                per_g.append((_GW[g1] * _GW[g2],) + _eval_edge(mesh, alpha, beta, kind, si, sj, x1, x2))
        vals.append(per_g)
    rows, cols, av, mv = [], [], [], []
    crow, ccol, cv = [], [], []
    inv_eps = 1.0 / eps[cell]
    for s in range(4):
        gs = slots[s][3]
        # C[cell, e] = integral of the curl over the cell
        cint = sum(wg * cu for (wg, _, _, cu) in vals[s]) * area
        crow.append(cell); ccol.append(gs); cv.append(cint)
        for t in range(4):
            gt = slots[t][3]
            mint = np.zeros(N, complex)
            aint = np.zeros(N, complex)
            for (ws, v1s, v2s, cus), (_, v1t, v2t, cut) in zip(vals[s], vals[t]):
                mint += ws * (np.conj(v1s) * v1t + np.conj(v2s) * v2t)
                aint += ws * np.conj(cus) * cut
            rows.append(gs); cols.append(gt)
            mv.append(mint * area)
            av.append(aint * area * inv_eps)
    rows = np.concatenate(rows); cols = np.concatenate(cols)
    D = mesh.D
    A = sp.csr_matrix((np.concatenate(av), (rows, cols)), shape=(D, D))
    M = sp.csr_matrix((np.concatenate(mv), (rows, cols)), shape=(D, D))
    C = sp.csr_matrix((np.concatenate(cv), (np.concatenate(crow), np.concatenate(ccol))), shape=(N, D))
    A.eliminate_zeros(); M.eliminate_zeros(); C.eliminate_zeros()
    w = inv_eps / area
    L = _lifting(mesh, alpha, beta)
    P = (L.conj().T @ M @ L).tocsr()
    return dict(mesh=mesh, k=np.asarray(k, float), alpha=alpha, beta=beta, eps=eps,
                A=A, M=M, C=C, w=w, L=L, P=P)


def _lifting(mesh: Mesh, alpha, beta):
    """``L[e, node]`` = DOF of ``grad varphi_node`` on edge ``e``.

    The DOF of a gradient is a line integral, i.e. the difference of the nodal
    function between the edge's end and start point.  Candidate nodes are the
    3x3 neighbourhoods of both end points; entries that vanish are dropped.
    """
    n, m, h1, h2, N = mesh.n, mesh.m, mesh.h1, mesh.h2, mesh.N
    ei, ej = _edge_ids(mesh)
    rows, cols, vals = [], [], []
    for kind in (0, 1):
        if kind == 0:
            s1, s2 = ei * h1, ej * h2
            e1, e2 = (ei + 1) * h1, ej * h2
            off = 0
        else:
            s1, s2 = ei * h1, ej * h2
            e1, e2 = ei * h1, (ej + 1) * h2
            off = N
        for di in (-1, 0, 1, 2):
            for dj in (-1, 0, 1, 2):
                ni = (ei + di) % n
                nj = (ej + dj) % m
                v = nodal_basis(mesh, alpha, beta, ni, nj, e1, e2) - nodal_basis(mesh, alpha, beta, ni, nj, s1, s2)
                nz = np.abs(v) > 0
                rows.append(off + (ej * n + ei)[nz]); cols.append((nj * n + ni)[nz]); vals.append(v[nz])
    L = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(mesh.D, N))
    # candidate sets overlap when n or m is small; each (edge, node) value is kept once
    return _unique_max(L)


def edge_prolongation(fine: Mesh, coarse: Mesh, k):
    """Natural embedding of the coarse edge space into the fine one (Section 5).

    ``P[f, c]`` = DOF of the coarse basis function ``c`` on fine edge ``f``,
    i.e. the line integral of its tangential component (2-point Gauss along
    the fine edge).  Candidate coarse edges: both orientations in a 3x3 block
    of coarse indices around the fine edge.
    """
    if fine.n != 2 * coarse.n or fine.m != 2 * coarse.m:
        raise ValueError("bisection hierarchy expected")
    alpha, beta = bloch_phases(k, fine.a, fine.b)
    n, h1, h2, N = fine.n, fine.h1, fine.h2, fine.N
    fi, fj = _edge_ids(fine)
    rows, cols, vals = [], [], []
    for fkind in (0, 1):
        for ckind in (0, 1):
            for dI in (-1, 0, 1):
                for dJ in (-1, 0, 1):
                    I = (fi // 2 + dI) % coarse.n
                    J = (fj // 2 + dJ) % coarse.m
                    acc = np.zeros(fi.shape, complex)
                    for g, wg in zip(_GX, _GW):
                        if fkind == 0:
                            x1, x2 = (fi + g) * h1, fj * h2
                        else:
                            x1, x2 = fi * h1, (fj + g) * h2
                        v1, v2, _ = _eval_edge(coarse, alpha, beta, ckind, I, J, x1, x2)
                        acc += wg * (v1 * h1 if fkind == 0 else v2 * h2)
                    nz = np.abs(acc) > 1e-300
                    rows.append(fkind * N + (fj * n + fi)[nz])
                    cols.append(ckind * coarse.N + (J * coarse.n + I)[nz])
                    vals.append(acc[nz])
    P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(fine.D, coarse.D))
    P = _unique_max(P)
    return P


def _unique_max(P):
    """Candidate blocks overlap on small meshes: keep one copy of each (row, col) entry."""
    P = P.tocoo()
    key = P.row.astype(np.int64) * P.shape[1] + P.col
    _, first = np.unique(key, return_index=True)
    return sp.csr_matrix((P.data[first], (P.row[first], P.col[first])), shape=P.shape)


def nodal_prolongation(fine: Mesh, coarse: Mesh, k):
    """Natural embedding of the coarse Q1 space: ``P[f, c] = varphi_c(x_f)`` at fine node ``x_f``."""
    if fine.n != 2 * coarse.n or fine.m != 2 * coarse.m:
        raise ValueError("bisection hierarchy expected")
    alpha, beta = bloch_phases(k, fine.a, fine.b)
    fi, fj = _edge_ids(fine)
    x1, x2 = fi * fine.h1, fj * fine.h2
    rows, cols, vals = [], [], []
    for dI in (-1, 0, 1, 2):
        for dJ in (-1, 0, 1, 2):
            I = (fi // 2 + dI) % coarse.n
            J = (fj // 2 + dJ) % coarse.m
            v = nodal_basis(coarse, alpha, beta, I, J, x1, x2)
            nz = np.abs(v) > 0
            rows.append((fj * fine.n + fi)[nz]); cols.append((J * coarse.n + I)[nz]); vals.append(v[nz])
    P = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(fine.N, coarse.N))
    return _unique_max(P)
