"""Pins for the oracle's eigensolves against the closed-form spectrum, brute force and symmetry."""
import numpy as np
import pytest

from oracle import fem, eigen
import pbs_inputs as gi

# Closed-form values for a=b=1, eps=1 (symbol of the stencils on discrete plane waves),
# quoted to 12 digits.
C1_32 = [3.084777829520, 22.863651398372, 32.767981202876, 52.546854771728, 52.636262412399]
C1_8 = [3.092684301946, 23.473204407063, 33.908319785757, 54.288839890874]


def test_closed_form_reproduces_quoted_values():
    k = (np.pi / 2, np.pi / 4)
    assert np.allclose(eigen.closed_form_eps_const(1, 1, 32, 32, 1.0, k, 5), C1_32, rtol=1e-12)
    assert np.allclose(eigen.closed_form_eps_const(1, 1, 8, 8, 1.0, k, 4), C1_8, rtol=1e-12)
    lam = eigen.closed_form_eps_const(1, 1, 8, 8, 1.0, (np.pi, 0.0), 6)
    assert np.allclose(lam[:2], 9.997080656247, rtol=1e-12)
    assert np.allclose(lam[2:6], 51.543648677132, rtol=1e-12)


@pytest.mark.parametrize("a,b,n,m,eps,k", [
    (1.0, 1.0, 32, 32, 1.0, (np.pi / 2, np.pi / 4)),   # the 32x32 homogeneous case
    (1.0, 1.0, 8, 8, 1.0, (np.pi, 0.0)),                # degenerate zone-boundary point
    (1.0, 1.3, 12, 8, 2.5, (0.4, -1.9)),                # rectangular cells, eps != 1
    (1.0, 1.0, 8, 8, 1.0, (0.0, 0.0)),                  # Gamma: one extra zero
])
def test_dense_assembly_matches_closed_form(a, b, n, m, eps, k):
    ops = fem.assemble(fem.Mesh(a, b, n, m), np.full((m, n), eps), k)
    lam = eigen.eigs_dense(ops, 8, vectors=False)
    want = eigen.closed_form_eps_const(a, b, n, m, eps, k, 8)
    assert np.allclose(lam, want, rtol=1e-10)


@pytest.mark.parametrize("k", [(0.3, 0.1), (0.0, 0.0), (np.pi, np.pi), (np.pi, 0.0)])
def test_three_eigen_routes_agree(k):
    n = 16
    ops = fem.assemble(fem.Mesh(1, 1, n, n), gi.rod_eps(n, n), k)
    ld = eigen.eigs_dense(ops, 8)[0]
    lr = eigen.eigs_reduced(ops, 8)
    ls = eigen.eigs_sparse(ops, 8)[0]
    assert np.allclose(ld, lr, rtol=1e-10)
    assert np.allclose(ls, lr, rtol=1e-11)


def test_k_minus_k_symmetry():
    # A(-k) = conj(A(k)), M(-k) = conj(M(k)) -> identical spectra
    n = 12
    eps = np.random.default_rng(5).uniform(1, 10, (n, n))
    k = (0.77, -1.3)
    a = eigen.eigs_sparse(fem.assemble(fem.Mesh(1, 1, n, n), eps, k), 6)[0]
    b = eigen.eigs_sparse(fem.assemble(fem.Mesh(1, 1, n, n), eps, (-k[0], -k[1])), 6)[0]
    assert np.allclose(a, b, rtol=1e-12)


def test_c4v_symmetry_of_rod_crystal():
    n = 16
    eps = gi.rod_eps(n, n)
    k = (0.9, 0.35)
    vals = [eigen.eigs_sparse(fem.assemble(fem.Mesh(1, 1, n, n), eps, kk), 6)[0]
            for kk in (k, (k[1], k[0]), (-k[0], k[1]))]
    assert np.allclose(vals[0], vals[1], rtol=1e-11)
    assert np.allclose(vals[0], vals[2], rtol=1e-11)


def test_rayleigh_quotients_and_residuals_of_sparse_eigenpairs():
    n = 24
    ops = fem.assemble(fem.Mesh(1, 1, n, n), gi.rod_eps(n, n), (0.5, 0.2))
    lam, V = eigen.eigs_sparse(ops, 6)
    R = ops["A"] @ V - (ops["M"] @ V) * lam
    rel = np.linalg.norm(R, axis=0) / (lam * np.linalg.norm(ops["M"] @ V, axis=0))
    assert rel.max() < 1e-9
    assert np.abs(ops["L"].conj().T @ (ops["M"] @ V)).max() < 1e-10


def test_second_order_discretisation_error():
    # eps = 1: the discrete eigenvalue of the lowest plane wave tends to |k|^2 with O(h^2)
    k = (0.6, 0.3)
    errs = [abs(eigen.closed_form_eps_const(1, 1, n, n, 1.0, k, 1)[0] - (k[0] ** 2 + k[1] ** 2))
            for n in (8, 16, 32)]
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5
