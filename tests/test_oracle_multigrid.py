"""Pins for the reference multigrid (Section 5): invariants of the algorithm, not its speed.

The paper prints no contraction factors, so the cycle's quality is not pinned
against the paper; these tests pin what the algorithm must satisfy: the
iterated cycle converges to the direct solution, the symmetric cycle is
Hermitian, each patch solve is exact and same-colour patches are uncoupled.
"""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem, multigrid as mg
import pbs_inputs as gi


def _rng_vec(size, seed):
    r = np.random.default_rng(seed)
    return r.standard_normal(size) + 1j * r.standard_normal(size)


@pytest.mark.parametrize("n,m,k", [(16, 16, (0.3, -0.2)), (16, 8, (0.0, 0.0)), (16, 16, (np.pi, np.pi))])
def test_edge_vcycle_converges_to_direct_solution(n, m, k):
    # b = m/n keeps the cells square (patch smoothers lose robustness on stretched cells)
    mesh = fem.Mesh(1.0, m / n, n, m)
    levs = mg.edge_hierarchy(mesh, gi.rod_eps(n, m, 1.0, m / n), k, 1.0, 4)
    K = levs[0]["K"]
    b = _rng_vec(mesh.D, 1)
    xs = spla.spsolve(K.tocsc(), b)
    x = np.zeros_like(b)
    for _ in range(30):
        x += mg.edge_vcycle(levs, b - K @ x)
    assert np.linalg.norm(x - xs) < 1e-8 * np.linalg.norm(xs)


@pytest.mark.parametrize("k", [(0.3, -0.2), (0.0, 0.0)])
def test_cycles_are_hermitian(k):
    n = 16
    mesh = fem.Mesh(1.0, 1.0, n, n)
    eps = gi.rod_eps(n, n)
    levs = mg.edge_hierarchy(mesh, eps, k, 1.0, 4)
    x, y = _rng_vec(mesh.D, 2), _rng_vec(mesh.D, 3)
    l, r = np.vdot(y, mg.edge_vcycle(levs, x)), np.vdot(mg.edge_vcycle(levs, y), x)
    assert abs(l - r) < 1e-12 * abs(l)
    nl = mg.nodal_hierarchy(mesh, eps, k, 4)
    x, y = _rng_vec(mesh.N, 4), _rng_vec(mesh.N, 5)
    if k == (0.0, 0.0):
        x -= x.mean(); y -= y.mean()
    l, r = np.vdot(y, mg.nodal_vcycle(nl, x)), np.vdot(mg.nodal_vcycle(nl, y), x)
    assert abs(l - r) < 1e-12 * abs(l)


def test_colour_step_solves_every_patch_of_that_colour_exactly():
    n = 8
    mesh = fem.Mesh(1.0, 1.0, n, n)
    levs = mg.edge_hierarchy(mesh, gi.rod_eps(n, n), (0.4, 0.9), 0.7, 4)
    K = levs[0]["K"]
    b = _rng_vec(mesh.D, 6)
    x = _rng_vec(mesh.D, 7)
    for colour in mg.COLOUR_ORDER:
        mg.edge_smooth(levs[0], x, b, (colour,))
        r = b - K @ x
        for (i, j) in [(i, j) for j in range(colour[1], n, 2) for i in range(colour[0], n, 2)]:
            idx = mg.edge_patch(mesh, i, j)
            assert np.abs(r[idx]).max() < 1e-10 * np.abs(b).max()


@pytest.mark.parametrize("n,m,k", [(16, 16, (0.3, -0.2)), (16, 8, (0.0, 0.0))])
def test_nodal_vcycle_converges(n, m, k):
    mesh = fem.Mesh(1.0, m / n, n, m)
    nl = mg.nodal_hierarchy(mesh, gi.rod_eps(n, m, 1.0, m / n), k, 4)
    P = nl[0]["K"]
    b = _rng_vec(mesh.N, 8)
    if k == (0.0, 0.0):
        b -= b.mean()
    x = np.zeros_like(b)
    for _ in range(10):
        x += mg.nodal_vcycle(nl, b - P @ x)
    assert np.linalg.norm(b - P @ x) < 1e-7 * np.linalg.norm(b)


@pytest.mark.parametrize("k", [(0.3, -0.2), (0.0, 0.0)])
def test_projection_exact_and_approximate(k):
    n = 16
    mesh = fem.Mesh(1.0, 1.0, n, n)
    eps = gi.rod_eps(n, n)
    ops = fem.assemble(mesh, eps, k)
    U = np.stack([_rng_vec(mesh.D, s) for s in (10, 11)], axis=1)
    Up = mg.project_exact(ops, U)
    # result is M-orthogonal to all gradients and differs from U by a gradient (+ constants at Gamma)
    assert np.abs(ops["L"].conj().T @ (ops["M"] @ Up)).max() < 1e-10 * np.abs(U).max()
    assert np.allclose(ops["A"] @ Up, ops["A"] @ U, rtol=1e-10, atol=1e-9)
    if k == (0.0, 0.0):
        assert abs(Up[: mesh.N].sum()) < 1e-9 and abs(Up[mesh.N:].sum()) < 1e-9
    nl = mg.nodal_hierarchy(mesh, eps, k, 4)
    Ua = mg.project_approx(ops, nl, U, cycles=8)
    assert np.linalg.norm(Ua - Up) < 1e-7 * np.linalg.norm(Up)
