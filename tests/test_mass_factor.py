"""The factored mass form used by the double-float Gram and Rayleigh-quotient kernels.

Those kernels form x^* M y as (B x)^* (B y): along each edge set the mass matrix is
a scaled Bloch-periodic tridiag(1/6, 2/3, 1/6) (x-edges couple in j, y-edges in i),
which equals B^* B for B with diagonal alpha and upper diagonal beta,
alpha = (1 + 1/sqrt(3))/2, beta = (1 - 1/sqrt(3))/2, the wrap entry carrying the
Bloch phase.  Checked here against the oracle's assembled mass matrix (element
integrals of the Section 3 basis), so that a wrong coefficient, scale, phase or
coupling direction in the factor fails on the CPU."""
import numpy as np
import pytest

from oracle import fem


def _factor(mesh, alpha_ph, beta_ph):
    n, m, N = mesh.n, mesh.m, mesh.n * mesh.m
    r3 = 1.0 / np.sqrt(3.0)
    a, b = 0.5 * (1.0 + r3), 0.5 * (1.0 - r3)
    sx, sy = np.sqrt(mesh.h2 / mesh.h1), np.sqrt(mesh.h1 / mesh.h2)
    B = np.zeros((2 * N, 2 * N), dtype=complex)
    for j in range(m):
        for i in range(n):
            e = j * n + i
            # z_x(i, j) = sqrt(h2/h1) (alpha x(i, j) + beta x(i, j + 1)), x(i, m) = beta_ph x(i, 0)
            B[e, e] += sx * a
            B[e, ((j + 1) % m) * n + i] += sx * b * (beta_ph if j == m - 1 else 1.0)
            # z_y(i, j) = sqrt(h1/h2) (alpha y(i, j) + beta y(i + 1, j)), y(n, j) = alpha_ph y(0, j)
            B[N + e, N + e] += sy * a
            B[N + e, N + j * n + (i + 1) % n] += sy * b * (alpha_ph if i == n - 1 else 1.0)
    return B


@pytest.mark.parametrize("a,b,n,m,k", [
    (1.0, 1.0, 6, 6, (0.4, -1.1)),
    (1.3, 0.7, 6, 5, (2.0, 0.9)),
    (1.0, 1.0, 4, 4, (0.0, 0.0)),
    (1.0, 1.0, 8, 4, (np.pi, np.pi)),
    (1.0, 0.5, 4, 2, (0.7, 3.1)),
])
def test_mass_equals_factor_product(a, b, n, m, k):
    mesh = fem.Mesh(a, b, n, m)
    eps = np.random.default_rng(3).uniform(1.0, 9.0, (m, n))  # M does not depend on eps
    ops = fem.assemble(mesh, eps, k)
    M = ops["M"].toarray()
    B = _factor(mesh, np.exp(1j * k[0] * a), np.exp(1j * k[1] * b))
    assert np.max(np.abs(M - B.conj().T @ B)) <= 1e-14 * np.max(np.abs(M))


def test_factor_coefficients():
    r3 = 1.0 / np.sqrt(3.0)
    a, b = 0.5 * (1.0 + r3), 0.5 * (1.0 - r3)
    assert abs(a * a + b * b - 2.0 / 3.0) <= 1e-16 and abs(a * b - 1.0 / 6.0) <= 1e-16
