"""Pins for Rayleigh-Ritz / extrapolation (Sections 4 and 6): Courant-Fischer and exactness."""
import numpy as np

from oracle import fem, eigen, extrapolation as ex
import pbs_inputs as gi

N_SIDE = 16


def _path_bases(count=6):
    eps = gi.rod_eps(N_SIDE, N_SIDE)
    ks = gi.gxmg_path(31)
    out = []
    for k in ks[1:4]:
        lam, V, ops = eigen.solve_k(1, 1, N_SIDE, N_SIDE, eps, k, count, "dense")
        out.append((lam, V, ops))
    return out


def test_ritz_values_bound_eigenvalues_and_deeper_spans_are_tighter():
    (l1, V1, _), (l2, V2, _), (l3, V3, ops3) = _path_bases()
    th1, _ = ex.extrapolate(ops3, [V2], 6)
    th2, _ = ex.extrapolate(ops3, [V2, V1], 6)
    assert np.all(th1 >= l3 * (1 - 1e-12))
    assert np.all(th2 >= l3 * (1 - 1e-12))
    assert np.all(th2 <= th1 * (1 + 1e-12))


def test_rayleigh_ritz_exact_on_invariant_subspace():
    (_, _, _), (_, _, _), (l3, V3, ops3) = _path_bases()
    mix = np.random.default_rng(0).standard_normal((6, 6)) + 1j * np.random.default_rng(1).standard_normal((6, 6))
    th, X = ex.rayleigh_ritz(ops3, V3 @ mix, 6)
    assert np.allclose(th, l3, rtol=1e-11)
    GM, _ = ex.grams(ops3, X)
    assert np.allclose(GM, np.eye(6), atol=1e-10)
