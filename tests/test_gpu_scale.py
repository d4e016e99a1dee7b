"""Full-size workloads of the larger configurations, pinned where the
mathematics gives exact answers.

1024 x 1024 (2,097,152 edge unknowns) with all 64 Bloch vectors of a
Gamma-X-M-Gamma path in flight at once (block 10, 8 bands, mixed policy; no
extrapolation chain exists when every Bloch vector starts together): with
eps = 1 the discrete spectrum is known in closed form (the stencils' symbol on
discrete plane waves), so every eigenvalue of every Bloch vector is checked.
Bands next to Gamma converge at the FP64 rounding floor 0.5 u lambda_max /
lambda where that exceeds tol (band 1 at the first path points here)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2304_00337_gb300 as pbs  # noqa: E402
import pbs_inputs as gi  # noqa: E402
from oracle import eigen  # noqa: E402

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
