"""Full-size workloads of the larger configurations.

* 1024 x 1024 (2,097,152 edge unknowns) with all 64 Bloch vectors of a
  Gamma-X-M-Gamma path in flight at once (block 10, 8 bands; no extrapolation
  chain exists when every Bloch vector starts together):
  - eps = 1: the discrete spectrum is known in closed form (the stencils' symbol
    on discrete plane waves), so every eigenvalue of every Bloch vector is checked;
  - the rod crystal (eps 8.9, r = 0.2a): mixed and FP64 agree per eigenvalue, and
    the eigenpairs returned next to Gamma, at X and at M are certified by the
    oracle on its own assembled matrices (residual, the gradient constraint,
    M-orthonormality and the residual-over-gap bound on every eigenvalue): the
    oracle's direct solve does not finish at this size.
* 4096 x 4096 (33.5M edge unknowns), 16 seeded disks, 12 bands, block 16: the
  mixed policy against the all-FP64 one per eigenvalue.
Bands next to Gamma converge at the FP64 rounding floor 0.5 u lambda_max /
lambda where that exceeds tol (band 1 at the first path points here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2304_00337_gb300 as pbs  # noqa: E402
import pbs_inputs as gi  # noqa: E402
from oracle import eigen, fem  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with pbs.Context(0) as c:
        yield c


def test_1024_path_64_in_flight_closed_form(ctx):
    n, nk, nev = 1024, 64, 8
    geom = pbs.Geometry(gi.const_eps(n, n))
    ks = gi.gxmg_path(nk)
    lam, res, iters = ctx.solve_path(geom, dict(nev=nev, block=10, kbatch=nk), ks)
    lam_max = 12.0 * 2 * n * n  # max(1/eps) 12 (1/h1^2 + 1/h2^2)
    floor = 0.5 * 2.0 ** -53 * lam_max / lam
    assert np.all(res <= np.maximum(1e-8, floor))
    for i, k in enumerate(ks):
        want = eigen.closed_form_eps_const(1, 1, n, n, 1.0, k, nev)
        assert np.max(np.abs(lam[i] - want) / want) <= 1e-9, (i, k)


def _band_tol(eps, n, m, lam, a=1.0, b=1.0, tol=1e-8):
    lam_max = np.max(1.0 / eps) * 12.0 * ((n / a) ** 2 + (m / b) ** 2)
    return np.maximum(tol, 0.5 * 2.0 ** -53 * lam_max / lam)


def test_1024_rod_path_64_in_flight_certified(ctx):
    n, nk, nev = 1024, 64, 8
    eps = gi.rod_eps(n, n)
    geom = pbs.Geometry(eps)
    ks = gi.gxmg_path(nk)
    sel = [1, 21, 42]  # next to Gamma, X, M (21 steps per leg)
    o = dict(nev=nev, block=10, kbatch=nk)
    lam, res, _, V = ctx.solve_path_vectors(geom, o, ks, sel)
    lam64, res64, _ = ctx.solve_path(geom, dict(o, precision=pbs.PBS_FP64), ks)
    assert np.all(res <= _band_tol(eps, n, n, lam)) and np.all(res64 <= _band_tol(eps, n, n, lam64))
    # error of the mixed policy against the all-FP64 path, per eigenvalue
    assert np.max(np.abs(lam - lam64) / lam64) <= 1e-10
    for t, i in enumerate(sel):
        ops = fem.assemble(fem.Mesh(1.0, 1.0, n, n), eps, ks[i])
        c = eigen.certify_pairs(ops, lam[i], V[t].T)
        assert np.max(np.abs(c["rq"] - lam[i]) / lam[i]) <= 1e-12, i
        # the oracle's FP64 residual carries its own rounding floor of the same size
        assert np.all(c["res"] <= 2.0 * _band_tol(eps, n, n, lam[i])), i
        assert c["constraint"].max() <= 1e-10 and c["orth"] <= 1e-10, i
        assert c["bound"].max() <= 1e-10, i


def test_4096_disks_mixed_vs_fp64(ctx):
    n, nev = 4096, 12
    eps = gi.disks_eps(n, n, seed=0)
    geom = pbs.Geometry(eps)
    ks = gi.gxmg_path(16)[[7]]  # between X and M
    o = dict(nev=nev, block=16)
    lam, res, _ = ctx.solve_path(geom, o, ks)
    lam64, res64, _ = ctx.solve_path(geom, dict(o, precision=pbs.PBS_FP64), ks)
    assert np.all(res <= _band_tol(eps, n, n, lam)) and np.all(res64 <= _band_tol(eps, n, n, lam64))
    assert np.max(np.abs(lam - lam64) / lam64) <= 1e-10
