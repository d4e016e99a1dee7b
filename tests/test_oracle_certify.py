"""Pins of ``oracle.eigen.certify_pairs`` (the a posteriori check used where the
mesh is too large for a direct solve) against exact eigenpairs from the dense
solve and against perturbations whose effect is known."""
import numpy as np

import pbs_inputs as gi
from oracle import eigen, fem


def _pairs(n=16, k=(0.7, -0.3), count=6):
    eps = gi.rod_eps(n, n)
    ops = fem.assemble(fem.Mesh(1.0, 1.0, n, n), eps, k)
    lam, V = eigen.eigs_dense(ops, count)
    return ops, lam, V


def test_exact_pairs_certify_tightly():
    ops, lam, V = _pairs()
    c = eigen.certify_pairs(ops, lam, V)
    assert np.allclose(c["rq"], lam, rtol=1e-12)
    assert c["res"].max() < 1e-10 and c["orth"] < 1e-12
    assert c["constraint"].max() < 1e-10  # dense eigh: rounding ~ u lambda_max / lambda
    assert c["bound"].max() < 1e-12


def test_bound_holds_for_perturbed_vectors():
    # Kato-Temple: the Rayleigh quotient of a perturbed eigenvector is within the
    # bound of the exact eigenvalue.  A perturbation by higher eigenvectors moves the
    # quotient at second order and so does the bound (within the ratio of the
    # perturbation's eigenvalue distance to the gap); white noise (every frequency up
    # to lambda_max) still satisfies it
    ops, lam12, V12 = _pairs(count=12)
    lam, V = lam12[:6], V12[:, :6]
    r = np.random.default_rng(3)
    for size in (1e-3, 1e-5):
        W = V + size * V12[:, 6:12] @ (r.standard_normal((6, 6)) + 1j * r.standard_normal((6, 6)))
        W /= np.sqrt(np.real(np.einsum("dq,dq->q", W.conj(), ops["M"] @ W)))
        rq = eigen.rayleigh(ops, W)
        c = eigen.certify_pairs(ops, rq, W)
        err = np.abs(rq - lam) / lam
        assert np.all(err <= c["bound"] * (1 + 1e-9))
        assert np.all(c["bound"] <= 100 * err)  # second order, like the true error
        N = W + size * (r.standard_normal(V.shape) + 1j * r.standard_normal(V.shape))
        rq = eigen.rayleigh(ops, N)
        c = eigen.certify_pairs(ops, rq, N)
        assert np.all(np.abs(rq - lam) / lam <= c["bound"] * (1 + 1e-9))


def test_gradients_and_wrong_values_are_flagged():
    ops, lam, V = _pairs()
    # a gradient part violates the constraint L^* M e = 0
    phi = np.random.default_rng(5).standard_normal(ops["mesh"].N)
    W = V.copy()
    W[:, 0] += 1e-3 * (ops["L"] @ phi)
    c = eigen.certify_pairs(ops, eigen.rayleigh(ops, W), W)
    assert c["constraint"][0] > 1e-6 and c["constraint"][1:].max() < 1e-10
    # a value that is not the vector's eigenvalue leaves a large residual
    bad = lam.copy()
    bad[2] *= 1.01
    c = eigen.certify_pairs(ops, bad, V)
    assert c["res"][2] > 1e-3 and np.delete(c["res"], 2).max() < 1e-10


def test_degenerate_cluster_at_gamma():
    # at k = 0 the C4v rod crystal has degenerate pairs: the cluster shares one gap
    ops, lam, V = _pairs(k=(0.0, 0.0), count=6)
    c = eigen.certify_pairs(ops, lam, V)
    assert c["bound"].max() < 1e-12
