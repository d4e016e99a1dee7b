"""Rayleigh-Ritz on a span and the Rayleigh-quotient extrapolation (ORACLE, test infrastructure).

Section 4 (eq. ritz_eigenvalue, Algorithm 2) and Section 6 ("Extrapolation"):
given previously computed bases ``E_1 .. E_e`` (coefficient vectors reused as
they are under the new Bloch vector), the initial guess for the new ``k`` is
spanned by the ``p`` smallest non-zero minima of the Rayleigh quotient of the
new pencil on ``span(E_1 .. E_e)``.  "Non-zero" is realised by removing the
null space first: the span is projected M-orthogonally off ``ker A`` exactly
(``multigrid.project_exact``), then a dense generalised Hermitian eigensolve of
the projected Gram matrices gives the Ritz pairs.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from .multigrid import project_exact

__all__ = ["grams", "rayleigh_ritz", "extrapolate"]


def grams(ops, S: np.ndarray):
    """``G_M = S^* M S`` and ``G_A = (C S)^* W (C S)`` for a block ``S`` of shape ``(D, q)``."""
    MS = ops["M"] @ S
    CS = ops["C"] @ S
    GM = S.conj().T @ MS
    GA = CS.conj().T @ (ops["w"][:, None] * CS)
    return GM, GA


def rayleigh_ritz(ops, S: np.ndarray, p: int, drop: float = 1e-12):
    """Ritz values and M-orthonormal Ritz vectors of the pencil on ``span(S)`` (no projection).

    Directions of ``S`` whose M-Gram eigenvalue is below ``drop`` times the
    largest are discarded before the reduced eigensolve (rank-deficient spans).
    """
    GM, GA = grams(ops, S)
    GM = 0.5 * (GM + GM.conj().T)
    GA = 0.5 * (GA + GA.conj().T)
    s, V = np.linalg.eigh(GM)
    keep = s > drop * s.max()
    T = V[:, keep] / np.sqrt(s[keep])
    H = T.conj().T @ GA @ T
    H = 0.5 * (H + H.conj().T)
    theta, U = np.linalg.eigh(H)
    X = S @ (T @ U[:, :p])
    return theta[:p], X


def extrapolate(ops, prev_bases, p: int):
    """Initial block for the pencil ``ops`` from earlier bases (Section 6).

    ``prev_bases``: list of ``(D, p_i)`` arrays (most recent first).  Returns the
    ``p`` smallest Ritz values and the corresponding M-orthonormal vectors of
    the exactly projected span.
    """
    S = np.concatenate([np.asarray(E) for E in prev_bases], axis=1)
    S = project_exact(ops, S)
    return rayleigh_ritz(ops, S, p)
