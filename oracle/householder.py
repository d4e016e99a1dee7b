"""Generalised (M-)Householder orthonormalisation - ORACLE, test infrastructure.

Section 4 orthonormalises the iteration block with generalised reflections
``Q_i = I - 2 v_i v_i^* M / (v_i^* M v_i)``, chosen so that
``Q_q ... Q_1 S = P R`` with ``R`` upper triangular and ``P`` a prescribed
M-orthonormal basis of canonical M-unit vectors with disjoint supports; the
result is ``E = Q_1 ... Q_q P``, M-orthonormal by construction, ``S = E R``, and
when ``S`` loses rank ``E`` still is M-orthonormal and its range contains that
of ``S`` (the basis is extended implicitly).  Plain numpy in FP64, one column
at a time in the order the paper describes; only ``tests/`` and the bench's
CPU leg use this module.

Readings where the paper is silent:

* ``P``: the scaled unit vectors of x-edges ``(k mod n, 2 (k div n))``; x-edges
  on one row, and on rows two apart, share no mass-matrix entry, so these are
  M-orthonormal (``pivots``).
* Step ``i`` works on ``y``, column ``i`` after the first ``i - 1`` reflections:
  ``y_perp = y - sum_{k<i} P_k (P_k^* M y)``, taken twice (a second pass on
  ``y_perp``; the coefficients of both passes add up to ``R[k, i]``), so that
  ``y_perp`` is M-orthogonal to the earlier ``P_k`` to rounding relative to its
  own size even when it is short (rank loss),
  ``gamma = P_i^* M y_perp``, ``sigma = -||y_perp||_M gamma / |gamma|``
  (``-||y_perp||_M`` when ``gamma = 0``; the sign avoids cancellation in ``v``),
  ``R[i, i] = sigma`` and ``v_i = y_perp - sigma P_i``.  Since ``v_i`` is
  M-orthogonal to ``P_1 .. P_{i-1}`` the reflection keeps the earlier columns,
  and ``y_perp^* M (sigma P_i)`` is real, so ``Q_i`` maps ``y_perp`` to
  ``sigma P_i`` and ``y`` to ``P R[:, i]``.
* ``y_perp = 0`` (exact rank loss): ``Q_i = I`` and ``R[i, i] = 0``.
"""
from __future__ import annotations

import numpy as np

__all__ = ["pivots", "basis_P", "m_householder", "reflect"]


def pivots(n: int, m: int, q: int) -> np.ndarray:
    """Edge indices of the prescribed basis: x-edge ``(k mod n, 2 (k div n))`` is index ``j n + i``."""
    rows = m // 2
    if q > n * rows:
        raise ValueError(f"at most {n * rows} prescribed vectors on a {n} x {m} mesh")
    k = np.arange(q)
    return (2 * (k // n)) * n + k % n


def basis_P(M, piv: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """Dense ``P`` (scaled unit vectors at ``piv``) and the scales ``s_k = sqrt(M[j_k, j_k])``."""
    D = M.shape[0]
    s = np.sqrt(np.real(np.asarray(M[piv, piv]).ravel()))
    P = np.zeros((D, len(piv)), complex)
    P[piv, np.arange(len(piv))] = 1.0 / s
    return P, s


def reflect(M, v: np.ndarray, vMv: float, X: np.ndarray) -> np.ndarray:
    """``Q X = X - 2 v (v^* M X) / (v^* M v)`` for the reflection of ``v``."""
    return X - np.outer(v, 2.0 * (v.conj() @ (M @ X)) / vMv)


def m_householder(M, S: np.ndarray, piv: np.ndarray):
    """Return ``E, R, refl`` with ``Q_q..Q_1 S = P R``, ``E = Q_1..Q_q P``; ``refl[i] = (v_i, v_i^* M v_i)`` or None."""
    S = np.asarray(S, complex)
    D, q = S.shape
    P, s = basis_P(M, piv)
    Y = S.copy()
    R = np.zeros((q, q), complex)
    refl = []
    for i in range(q):
        y = Y[:, i]
        My = M @ y
        y_perp = y.copy()
        for k in range(i):
            R[k, i] = My[piv[k]] / s[k]  # P_k^* M y
            y_perp = y_perp - P[:, k] * R[k, i]
        # second pass: the first leaves P-components of the size of the rounding of y,
        # which would dominate a short y_perp (rank loss)
        My = M @ y_perp
        for k in range(i):
            c = My[piv[k]] / s[k]
            R[k, i] += c
            y_perp = y_perp - P[:, k] * c
        nrm = np.sqrt(max(np.real(np.vdot(y_perp, M @ y_perp)), 0.0))
        if nrm == 0.0:
            refl.append(None)
            continue
        gamma = (M @ y_perp)[piv[i]] / s[i]  # P_i^* M y_perp
        sigma = -nrm * (gamma / abs(gamma) if gamma != 0 else 1.0)
        R[i, i] = sigma
        v = y_perp - sigma * P[:, i]
        vMv = np.real(np.vdot(v, M @ v))
        refl.append((v, vMv))
        if i + 1 < q:
            Y[:, i + 1:] = reflect(M, v, vMv, Y[:, i + 1:])
    E = P.copy()
    for i in reversed(range(q)):
        if refl[i] is not None:
            v, vMv = refl[i]
            E = reflect(M, v, vMv, E)
    return E, R, refl
