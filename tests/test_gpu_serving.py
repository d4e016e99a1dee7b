"""Serving entry points (pbs_submit / pbs_poll / pbs_fetch / pbs_cancel) through the C ABI.

Jobs run the same computation as pbs_solve_path on the engines of the
context's serving slots, several at once, so their results must equal the
synchronous call's bit for bit (the solver is deterministic), alone and in a
mix of overlapping jobs; admission waits for memory instead of refusing."""
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


def test_fetch_waits_and_fifo_latency():
    # one slot: jobs run one after another in submission order
    with pbs.Context(0) as c:
        c.serve_slots(1)
        g, o, ks = _jobs()[1]
        a = c.submit(g, o, ks)
        b = c.submit(g, o, ks[:4])
        ev_b, _, _, lat_b = c.fetch(b)  # waits; b ran after a
        ev_a, _, _, lat_a = c.fetch(a)
        assert ev_b.shape == (4, o["nev"]) and ev_a.shape == (len(ks), o["nev"])
        assert lat_b > lat_a * 0.9  # b waited for a in the queue
        # the two jobs split their paths into different chains; converged values agree
        assert np.allclose(ev_b, ev_a[:4], rtol=1e-9)


def _overlap(t, u):
    return t[1] < u[2] and u[1] < t[2]


def test_overlapping_jobs_match_alone():
    # continuous batching: three slots run three jobs at once (their run intervals
    # overlap) and each job's results equal the ones it gets alone, bit for bit
    mix = [
        (pbs.Geometry(gi.rod_eps(128, 128)), dict(OPTS, kbatch=2), gi.gxmg_path(10)),
        (pbs.Geometry(gi.disks_eps(96, 96, seed=4, ndisks=5)), dict(OPTS, nev=6, block=8), gi.gxmg_path(13)),
        (pbs.Geometry(gi.rod_eps(64, 64, radius=0.3, eps_rod=12.0)), dict(OPTS, precision=pbs.PBS_FP64),
         gi.gxmg_path(16)),
    ]
    with pbs.Context(0) as c:
        c.serve_slots(3)
        alone = []
        for g, o, ks in mix:
            j = c.submit(g, o, ks)
            ev, rs, it, _ = c.fetch(j)
            alone.append((ev, rs, it))
        ids = [c.submit(g, o, ks) for g, o, ks in mix]
        while not all(c.poll(j) for j in ids):
            time.sleep(0.005)
        times = [c.job_times(j) for j in ids]
        together = [c.fetch(j)[:3] for j in ids]
    for (ev, rs, it), (ev2, rs2, it2) in zip(alone, together):
        assert np.array_equal(ev, ev2) and np.array_equal(rs, rs2) and np.array_equal(it, it2)
    assert _overlap(times[0], times[1]) and _overlap(times[0], times[2])


def test_admission_waits_for_memory():
    # a budget that holds one job at a time: the others wait in the queue (none is
    # refused) and the run intervals do not overlap
    g, o, ks = (pbs.Geometry(gi.rod_eps(128, 128)), dict(OPTS), gi.gxmg_path(7))
    need = pbs.job_bytes(128, 128, o, len(ks))
    with pbs.Context(0, hbm_budget_bytes=int(1.5 * need)) as c:
        c.serve_slots(3)
        ids = [c.submit(g, o, ks) for _ in range(3)]
        while not all(c.poll(j) for j in ids):
            time.sleep(0.005)
        times = sorted(c.job_times(j) for j in ids)
        res = [c.fetch(j) for j in ids]
    assert all(np.array_equal(r[0], res[0][0]) for r in res)
    for t, u in zip(times, times[1:]):
        assert not _overlap(t, u)


def test_cancel_queued_and_running():
    with pbs.Context(0) as c:
        c.serve_slots(1)
        big = c.submit(pbs.Geometry(gi.rod_eps(256, 256)), dict(OPTS), gi.gxmg_path(31))
        queued = c.submit(pbs.Geometry(gi.rod_eps(32, 32)), OPTS, gi.gxmg_path(4))
        last = c.submit(pbs.Geometry(gi.rod_eps(32, 32)), OPTS, gi.gxmg_path(7))
        c.cancel(queued)
        with pytest.raises(pbs.PbsError) as e:
            c.fetch(queued)
        assert e.value.status == pbs.PBS_ECANCELED
        while c.job_times(big)[1] < 0:  # wait until it runs
            time.sleep(0.002)
        c.cancel(big)
        t0 = time.time()
        with pytest.raises(pbs.PbsError) as e:
            c.fetch(big)
        assert e.value.status == pbs.PBS_ECANCELED and time.time() - t0 < 5.0
        ev, rs, it, _ = c.fetch(last)  # the queue goes on
        assert np.all(rs <= OPTS["tol"])



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
    # a job that alone needs more than the context may hold is refused at submission
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
