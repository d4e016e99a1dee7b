"""Serving entry points (pbs_submit / pbs_poll / pbs_fetch) through the C ABI.

Jobs run the same computation as pbs_solve_path, one after another on the
context's host thread, so their results must equal the synchronous call's
bit for bit (the solver is deterministic)."""
import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import paper_2304_00337_gb300 as pbs  # noqa: E402
import pbs_inputs as gi  # noqa: E402

pytestmark = pytest.mark.gpu

OPTS = dict(nev=4, block=6, tol=1e-8)


@pytest.fixture(scope="module")
def ctx():
    import __graft_entry__ as ge
    ge.build()
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with pbs.Context(0) as c:
        yield c


def _jobs():
    # (geometry, opts, k list): rod paths on two meshes (one with two chains in
    # flight) and a disk crystal in plain FP64
    return [
        (pbs.Geometry(gi.rod_eps(32, 32)), dict(OPTS), gi.gxmg_path(7)),
        (pbs.Geometry(gi.rod_eps(64, 64)), dict(OPTS, kbatch=2), gi.gxmg_path(10)),
        (pbs.Geometry(gi.disks_eps(48, 48, seed=2, ndisks=3)), dict(OPTS, precision=pbs.PBS_FP64), gi.gxmg_path(4)),
    ]


def test_jobs_equal_synchronous_paths(ctx):
    jobs = _jobs()
    ids = [ctx.submit(g, o, ks) for g, o, ks in jobs]
    assert len(set(ids)) == len(ids)
    results = {}
    deadline = time.time() + 300
    while len(results) < len(ids) and time.time() < deadline:
        for i in ids:
            if i not in results and ctx.poll(i):
                results[i] = ctx.fetch(i)
        time.sleep(0.01)
    assert len(results) == len(ids)
    for i, (g, o, ks) in zip(ids, jobs):
        ev, rs, it, lat = results[i]
        want_ev, want_rs, want_it = ctx.solve_path(g, o, ks)
        assert np.array_equal(ev, want_ev) and np.array_equal(rs, want_rs) and np.array_equal(it, want_it)
        assert np.all(rs <= o["tol"]) and lat > 0.0


def test_fetch_waits_and_fifo_latency(ctx):
    g, o, ks = _jobs()[1]
    a = ctx.submit(g, o, ks)
    b = ctx.submit(g, o, ks[:4])
    ev_b, _, _, lat_b = ctx.fetch(b)  # waits; b ran after a
    ev_a, _, _, lat_a = ctx.fetch(a)
    assert ev_b.shape == (4, o["nev"]) and ev_a.shape == (len(ks), o["nev"])
    assert lat_b > lat_a * 0.9  # b waited for a in the queue
    # the two jobs split their paths into different chains; converged values agree
    assert np.allclose(ev_b, ev_a[:4], rtol=1e-9)


def test_unknown_and_invalid_jobs(ctx):
    with pytest.raises(pbs.PbsError) as e:
        ctx.poll(123456789)
    assert e.value.status == pbs.PBS_EINVAL
    with pytest.raises(pbs.PbsError) as e:
        ctx.fetch(987654321)
    assert e.value.status == pbs.PBS_EINVAL
    bad = gi.rod_eps(32, 32)
    bad[5, 5] = -2.0
    with pytest.raises(pbs.PbsError) as e:
        ctx.submit(pbs.Geometry(bad), OPTS, gi.gxmg_path(4))
    assert e.value.status == pbs.PBS_EINVAL
    with pytest.raises(pbs.PbsError) as e:
        ctx.submit(pbs.Geometry(gi.rod_eps(32, 32)), dict(OPTS, block=2), gi.gxmg_path(4))  # block < nev
    assert e.value.status == pbs.PBS_EINVAL


def test_admission_refuses_jobs_over_budget():
    need = pbs.job_bytes(256, 256, OPTS, 4)
    with pbs.Context(0, hbm_budget_bytes=need // 4) as c:
        with pytest.raises(pbs.PbsError) as e:
            c.submit(pbs.Geometry(gi.rod_eps(256, 256)), OPTS, gi.gxmg_path(4))
        assert e.value.status == pbs.PBS_ENOMEM
    with pbs.Context(0, hbm_budget_bytes=2 * need) as c:  # the estimate is enough to run it
        j = c.submit(pbs.Geometry(gi.rod_eps(256, 256)), OPTS, gi.gxmg_path(4))
        ev, rs, it, lat = c.fetch(j)
        assert np.all(rs <= OPTS["tol"])


def test_destroy_with_queued_jobs_and_sync_calls_in_between():
    c = pbs.Context(0)
    g, o, ks = _jobs()[1]
    ids = [c.submit(g, o, ks) for _ in range(4)]
    ev, rs, it = c.solve_path(g, o, ks[:4])  # waits for the job in progress, then runs
    assert np.all(rs <= o["tol"])
    c.close()  # the running job finishes, the queued ones are dropped; no hang
    assert ids
