"""Failure handling through the C ABI, injected on the host (no device fault is
provoked): a failed device allocation, non-finite inputs, a budget shrunk between
calls, and a cancelled job.  Each returns its documented status and leaves the
context usable."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2304_00337_gb300 as pbs  # noqa: E402
import pbs_inputs as gi  # noqa: E402

pytestmark = pytest.mark.gpu

OPTS = dict(nev=4, block=6, tol=1e-8)


@pytest.fixture(scope="module")
def built():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_injected_allocation_failure(built):
    geom = pbs.Geometry(gi.rod_eps(64, 64))
    ks = gi.gxmg_path(4)
    with pbs.Context(0) as c:
        want = c.solve_path(geom, OPTS, ks)
        for nth in (1, 3, 7):
            with pbs.Context(0) as d:
                d.fail_alloc_after(nth)
                with pytest.raises(pbs.PbsError) as e:
                    d.solve_path(geom, OPTS, ks)
                assert e.value.status == pbs.PBS_ENOMEM and "injected" in pbs.last_error()
                got = d.solve_path(geom, OPTS, ks)  # usable afterwards, same results
                assert all(np.array_equal(a, b) for a, b in zip(want, got))


def test_non_finite_inputs(built):
    n = 32
    ks = gi.gxmg_path(4)
    with pbs.Context(0) as c:
        for bad in (np.nan, np.inf, -np.inf, 0.0):
            eps = gi.rod_eps(n, n)
            eps[3, 7] = bad
            with pytest.raises(pbs.PbsError) as e:
                c.solve_path(pbs.Geometry(eps), OPTS, ks)
            assert e.value.status == pbs.PBS_EINVAL
        geom = pbs.Geometry(gi.rod_eps(n, n))
        kbad = ks.copy()
        kbad[2, 1] = np.nan
        with pytest.raises(pbs.PbsError) as e:
            c.solve_path(geom, OPTS, kbad)
        assert e.value.status == pbs.PBS_EINVAL
        init = gi.random_block(geom.D, OPTS["block"], seed=1)
        init[2, 100] = np.nan
        with pytest.raises(pbs.PbsError) as e:
            c.solve_k(geom, OPTS, (0.3, 0.2), init=init)
        assert e.value.status == pbs.PBS_ENUMERIC
        lam, res, _ = c.solve_path(geom, OPTS, ks)  # still usable
        assert np.all(res <= OPTS["tol"])


def test_budget_shrunk_between_calls(built):
    geom = pbs.Geometry(gi.rod_eps(64, 64))
    ks = gi.gxmg_path(4)
    with pbs.Context(0) as c:
        want = c.solve_path(geom, OPTS, ks)
        c.set_budget(1 << 20)  # the resident workspace stays; a new one cannot be allocated
        again = c.solve_path(geom, OPTS, ks)
        assert all(np.array_equal(a, b) for a, b in zip(want, again))
        with pytest.raises(pbs.PbsError) as e:
            c.solve_path(geom, dict(OPTS, block=8), ks)
        assert e.value.status == pbs.PBS_ENOMEM
        c.set_budget(0)
        lam, res, _ = c.solve_path(geom, dict(OPTS, block=8), ks)
        assert np.all(res <= OPTS["tol"])
