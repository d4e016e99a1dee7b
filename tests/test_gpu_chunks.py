"""The solver's multigrid work is split into chunks of whole groups when the
columns in flight need more than the chunk size (8 GiB, or an eighth of the
context's device budget).  Each column's arithmetic does not depend on how the
columns are grouped into launches, so a path solved with small chunks must equal
the one solved in a single chunk bit for bit."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2304_00337_gb300 as pbs  # noqa: E402
import pbs_inputs as gi  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("precision", [pbs.PBS_MIXED, pbs.PBS_FP64])
def test_chunked_multigrid_work_gives_identical_paths(precision):
    # 64 x 64, block 6, 5 chains of 2 Bloch vectors: 30 columns per role.  A 96 MB
    # budget gives 18-column chunks (3 groups), so the projection of [E | P] runs as
    # 18 + 18 + 18 + 6 columns (the third chunk straddles E and P) and the
    # preconditioner as 18 + 12.
    geom = pbs.Geometry(gi.rod_eps(64, 64))
    ks = gi.gxmg_path(10)
    opts = dict(nev=4, block=6, kbatch=5, precision=precision)
    with pbs.Context(0) as c:
        want = c.solve_path(geom, opts, ks)
    with pbs.Context(0, hbm_budget_bytes=96 * 2 ** 20) as c:
        got = c.solve_path(geom, opts, ks)
    for w, g in zip(want, got):
        assert np.array_equal(w, g)
    assert np.all(want[1] <= 1e-8)
