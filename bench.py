"""Throughput of Bloch-path eigensolves on one GB300 (k-point eigensolves per second).

Workload (one "step", default ``--workload c3``): the square-lattice rod crystal
(eps = 8.9 rod of radius 0.2a in air, cell-centre samples) on a 1024 x 1024 mesh
(2,097,152 complex edge unknowns), 64 Bloch vectors along Gamma-X-M-Gamma all in
flight at once (one block of 10 vectors each, every kernel launch covering all 64),
the 8 smallest non-zero eigenvalues of each converged to a relative residual
<= 1e-8 (or the FP64 rounding floor 0.5 u lambda_max / lambda where that is higher:
band 1 next to Gamma).  ``--workload c2`` is the 256 x 256 path of 31 Bloch vectors
(four chains with Rayleigh-quotient extrapolation), ``c4`` the 4096 x 4096 field of
16 seeded disks (12 bands, block 16, 16 Bloch vectors).

``value``: mixed precision (FP32 multigrid and nodal projection; double-float Gram,
Rayleigh quotients and small Rayleigh-Ritz; FP64 residual, update and reported
eigenvalues), inputs and outputs resident on the device (``pbs_solve_path_device``);
``plain_fp64`` is the same workload with every kernel in FP64, and the per-band
difference of the two policies' eigenvalues is reported.  ``e2e``: the host-buffer
entry point ``pbs_solve_path`` with the permittivity copied from pinned host memory
and the results copied back in every step.  L2 is flushed (a 512 MiB write) before
every timed step (the c3 step's blocks, 86 GB, exceed it anyway).  The c3 line also
carries the c2 workload (value, plain FP64 and the error of both policies against the
oracle's stored eigenvalues).

``--impl reference`` times the CPU oracle (SciPy) on a bounded sample instead.
"""
from __future__ import annotations

import argparse
import json
import os
import resource
import statistics
import subprocess
import tempfile
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

TOL = 1e-8
METRIC = "k-point eigensolves/s at resid<=1e-8 (mixed; plain FP64 alongside)"
UNIT = "k-points/s"
# path workloads: mesh, Bloch vectors, bands, block, Bloch vectors in flight, permittivity
WORKLOADS = {
    "c2": dict(n=256, nk=31, nev=8, block=10, kbatch=4, eps="rod",
               text="rod crystal eps=8.9 r=0.2a, 256x256 Nedelec edges (131072 DOF), 31 k-points Gamma-X-M-Gamma, "
                    "8 bands, block 10, tol 1e-8, 4 chains with extrapolation depth 3"),
    "c3": dict(n=1024, nk=64, nev=8, block=10, kbatch=64, eps="rod",
               text="rod crystal eps=8.9 r=0.2a, 1024x1024 Nedelec edges (2097152 DOF), 64 k-points Gamma-X-M-Gamma "
                    "all in flight, 8 bands, block 10, tol 1e-8"),
    "c4": dict(n=4096, nk=16, nev=12, block=16, kbatch=2, eps="disks",
               text="16 seeded disks (r U(0.05,0.15)a, eps U(2,13), background 1), 4096x4096 Nedelec edges "
                    "(33554432 DOF), 16 k-points Gamma-X-M-Gamma, 12 bands, block 16, tol 1e-8, 2 chains"),
}
GOLDEN_C2 = os.path.join(ROOT, "tests", "golden", "rod256_path31.txt")
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
SAMPLE_EVERY = 16  # the dominant kernel is timed on every 16th launch inside the timed region
GRAM_DRAM_BYTES = 256.6e6  # measured per batched k_gram_df launch at 256x256 (4 groups of 30 columns)
FP64_PEAK_TFLOPS = 1.2  # 152 SMs x 4 FP64 flop/clk x ~1.98 GHz; measured 1.20 TFLOP/s with an FMA-chain probe
# Double-float kernels (mixed policy) run on the FP32 pipe: 152 SMs x 128 lanes x 1.98 GHz
# instructions/s, and a compensated complex multiply-add (8 algorithmic flops) takes 48 of them.
DF_PEAK_TFLOPS = 152 * 128 * 1.98e9 * 8 / 48 / 1e12


def workload_inputs(name: str):
    """Permittivity samples and Bloch vectors of a path workload (seeded, synthetic)."""
    import pbs_inputs as gi
    w = WORKLOADS[name]
    n = w["n"]
    eps = gi.rod_eps(n, n) if w["eps"] == "rod" else gi.disks_eps(n, n, seed=0)
    return eps, gi.gxmg_path(w["nk"])


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    return rank, ws


class Ranks:
    """The replica ranks of a run: one process per GPU, each solving the whole workload
    (weak scaling, no data-path collective); torch.distributed only for the barrier
    around the timed region and the maximum of the per-rank times."""

    def __init__(self, ws: int, device):
        self.ws = ws
        self.device = device

    def barrier(self):
        if self.ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def max(self, x: float) -> float:
        if self.ws == 1:
            return x
        import torch
        import torch.distributed as dist
        t = torch.tensor([x], dtype=torch.float64, device=self.device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())


def job_throughput(ws: int, units_per_rank: int, ms_max: float) -> float:
    """Whole-job units per second: every rank's units over the slowest rank's time."""
    return ws * units_per_rank / (ms_max / 1e3)


def _peaks():
    try:
        return json.load(open(PEAKS_PATH)), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        # the raw samples go to PBS_CLOCKS_DIR (default: the system's temporary directory)
        base = os.environ.get("PBS_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(base, f"clocks_{os.getpid()}.csv")

    def start(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader",
                                          "-i", str(self.dev), "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["clock sampling unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1].split()[0]))
                smax.append(float(parts[2].split()[0]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _oracle_kpoint_seconds(n: int, eps_kind: str, k) -> float:
    """Wall time of the oracle's solve of one Bloch vector (assembly + constrained sparse
    shift-invert eigensolve) on an n x n mesh of the workload's crystal."""
    import pbs_inputs as gi
    from oracle import fem, eigen
    eps = gi.rod_eps(n, n) if eps_kind == "rod" else gi.disks_eps(n, n, seed=0)
    t0 = time.perf_counter()
    ops = fem.assemble(fem.Mesh(1.0, 1.0, n, n), eps, k)
    eigen.eigs_sparse(ops, 8)
    return time.perf_counter() - t0


def oracle_sample_kps(name: str, seconds_budget: float = 20.0):
    """CPU oracle (SciPy shift-invert on the assembled pencil) on a bounded sample of the workload.

    Up to 256 x 256 the sample solves Bloch vectors of the workload's path on its own mesh
    until the budget is spent.  On larger meshes one Bloch vector takes far longer than the
    budget (512 x 512 ran for more than an hour on 8 host cores), so the sample solves the
    path's second Bloch vector on the same crystal at 64 x 64 and 128 x 128 and
    extrapolates to the workload's mesh with the growth t ~ D^alpha measured between the
    two; the direct solve's fill grows faster than that, so the extrapolated CPU time is a
    lower bound and the CPU rate an upper bound."""
    w = WORKLOADS[name]
    eps_kind = w["eps"]
    r0 = resource.getrusage(resource.RUSAGE_SELF)
    t0 = time.perf_counter()
    if w["n"] <= 256:
        import pbs_inputs as gi
        ks = gi.gxmg_path(w["nk"])
        done = 0
        for k in ks[1:]:
            _oracle_kpoint_seconds(w["n"], eps_kind, k)
            done += 1
            if time.perf_counter() - t0 > seconds_budget:
                break
        wall = time.perf_counter() - t0
        value = done / wall
        sample = f"{done} of the {w['nk']} k-points on the workload's mesh"
    else:
        import pbs_inputs as gi
        k = gi.gxmg_path(w["nk"])[1]
        t_a = _oracle_kpoint_seconds(64, eps_kind, k)
        t_b = _oracle_kpoint_seconds(128, eps_kind, k)
        alpha = max(1.0, np.log(t_b / t_a) / np.log(4.0))
        t_n = t_b * (w["n"] / 128.0) ** (2 * alpha)
        wall = time.perf_counter() - t0
        value = 1.0 / t_n
        sample = (f"one Bloch vector on the same crystal at 64x64 ({t_a:.2f} s) and 128x128 ({t_b:.2f} s), "
                  f"extrapolated to {w['n']}x{w['n']} with t ~ D^{alpha:.2f} ({t_n:.0f} s per k-point; "
                  "a lower bound: the direct solve's fill grows faster)")
    r1 = resource.getrusage(resource.RUSAGE_SELF)
    cpu = (r1.ru_utime - r0.ru_utime) + (r1.ru_stime - r0.ru_stime)
    return {"value": value, "unit": UNIT, "cores": max(1, round(cpu / wall)), "kind": "oracle",
            "sample": f"{sample}; {wall:.1f} s wall, {cpu:.1f} s CPU on {os.cpu_count()} host cores"}


def run_reference(args):
    rank, ws = _dist()
    if rank != 0:
        return
    name = args.workload
    w = WORKLOADS[name]
    per_step = []
    samples = []
    for s in range(args.warmup + args.steps):
        cb = oracle_sample_kps(name, seconds_budget=5.0)
        if s >= args.warmup:
            per_step.append(cb["value"])
            samples.append(cb)
    value = float(np.mean(per_step))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * w["nk"] / value, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["text"], "grid": f"{w['n']}x{w['n']}", "k_points": w["nk"], "bands": w["nev"],
                       "block": w["block"], "tol": TOL,
                       "sample": "each step a bounded oracle sample of the workload (see cpu_baseline.sample)"},
            "cpu_baseline": {"kind": "oracle", "cores": samples[-1]["cores"], "sample": samples[-1]["sample"],
                             "value": value, "unit": UNIT},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _opts(pbs, name, prec):
    w = WORKLOADS[name]
    return pbs.default_opts(nev=w["nev"], block=w["block"], tol=TOL, precision=prec, max_iter=400,
                            kbatch=w["kbatch"])


def _band_tol(eps, n, lam):
    lam_max = float(np.max(1.0 / eps)) * 12.0 * 2.0 * n * n
    return np.maximum(TOL, 0.5 * 2.0 ** -53 * lam_max / lam)


def c2_leg(pbs, dev, stream):
    """The 256 x 256 path (31 Bloch vectors, four chains): mixed and plain FP64 k-points/s
    (one warm and one timed step each) and both policies' per-band error against the
    oracle's stored eigenvalues."""
    import torch
    eps, ks = workload_inputs("c2")
    want = np.loadtxt(GOLDEN_C2)[:, 2:]
    d_eps = torch.from_numpy(eps.copy()).to(dev)
    d_ks = torch.from_numpy(ks.copy()).to(dev)
    nk, nev = len(ks), WORKLOADS["c2"]["nev"]
    d_ev = torch.zeros((nk, nev), dtype=torch.float64, device=dev)
    d_rs = torch.zeros_like(d_ev)
    d_it = torch.zeros(nk, dtype=torch.int32, device=dev)
    out = {"workload": WORKLOADS["c2"]["text"]}
    with pbs.Context(dev.index or 0) as ctx:
        for label, prec in (("mixed", pbs.PBS_MIXED), ("plain_fp64", pbs.PBS_FP64)):
            def step():
                ctx.solve_path_device(1.0, 1.0, 256, 256, d_eps.data_ptr(), _opts(pbs, "c2", prec), nk,
                                      d_ks.data_ptr(), d_ev.data_ptr(), d_rs.data_ptr(), d_it.data_ptr(), stream)
            step()
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step()
            e1.record(stream)
            torch.cuda.synchronize(dev)
            lam = d_ev.cpu().numpy()
            rel = np.abs(lam - want) / want
            out[label] = {"value": nk / (e0.elapsed_time(e1) / 1e3), "unit": UNIT,
                          "max_rel_err_vs_oracle_per_band": rel.max(axis=0).tolist(),
                          "max_resid": float(d_rs.max().item())}
    return out


def run_ours(args):
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_2304_00337_gb300 as pbs

    name = args.workload
    w = WORKLOADS[name]
    n, nk, nev = w["n"], w["nk"], w["nev"]
    rank, ws = _dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    ranks = Ranks(ws, dev)
    barrier, max_over_ranks = ranks.barrier, ranks.max

    eps, ks = workload_inputs(name)
    d_eps = torch.from_numpy(eps.copy()).to(dev)
    d_ks = torch.from_numpy(ks.copy()).to(dev)
    d_ev = torch.zeros((nk, nev), dtype=torch.float64, device=dev)
    d_rs = torch.zeros_like(d_ev)
    d_it = torch.zeros(nk, dtype=torch.int32, device=dev)
    flush = torch.empty(512 * 2 ** 20 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    ctx = pbs.Context(local)

    def step(prec):
        ctx.solve_path_device(1.0, 1.0, n, n, d_eps.data_ptr(), _opts(pbs, name, prec), nk, d_ks.data_ptr(),
                              d_ev.data_ptr(), d_rs.data_ptr(), d_it.data_ptr(), stream)

    def timed(prec, steps, profile=None):
        times = []
        launches0 = pbs.launch_count()
        if profile:
            ctx.profile_enable(profile)
        for _ in range(steps):
            flush.fill_(1.0)
            torch.cuda.synchronize(dev)
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            step(prec)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            barrier()
            times.append(e0.elapsed_time(e1))
        launches = pbs.launch_count() - launches0
        return times, launches

    # warm-up; the first warm-up step also measures every kernel class's share
    ctx.profile_enable("all")
    step(pbs.PBS_MIXED)
    torch.cuda.synchronize(dev)
    classes = ["edge_smooth", "node_smooth", "gram", "small_rr", "residual", "block_update", "lift_adj_mass",
               "edge_tail", "node_tail", "sub_lift", "convert", "node_apply"]
    shares = {c: ctx.profile_read(c) for c in classes}
    ctx.profile_enable(None)
    for _ in range(max(0, args.warmup - 1)):
        step(pbs.PBS_MIXED)
    torch.cuda.synchronize(dev)
    dominant = max(classes, key=lambda c: shares[c][0])

    clocks = ClockSampler(local)
    clocks.start()
    t_mixed, launches = timed(pbs.PBS_MIXED, args.steps, profile=f"{dominant}/{SAMPLE_EVERY}")
    clk = clocks.stop()
    dom_ms, dom_n, dom_work = ctx.profile_read(dominant)
    ctx.profile_enable(None)
    lam_mixed = d_ev.cpu().numpy()
    rs = d_rs.cpu().numpy()
    its = d_it.cpu().numpy()
    ok = bool(np.all(rs <= _band_tol(eps, n, lam_mixed)))

    # end to end through the host-buffer entry point (pinned host eps, results copied back)
    h_eps = torch.empty((n, n), dtype=torch.float64, pin_memory=True)
    h_eps.copy_(torch.from_numpy(eps))
    geom = pbs.Geometry(h_eps.numpy())
    e2e_steps = 1 if name != "c2" else args.steps
    e2e_t = []
    for _ in range(e2e_steps):
        flush.fill_(1.0)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        lam_h, res_h, it_h = ctx.solve_path(geom, _opts(pbs, name, pbs.PBS_MIXED), ks)
        e2e_t.append((time.perf_counter() - t0) * 1e3)

    # plain FP64 on the same workload (one step; its first call also allocates the FP64 workspace)
    t_fp64, _ = timed(pbs.PBS_FP64, 1 if name != "c2" else max(1, min(args.steps, 2)))
    lam_fp64 = d_ev.cpu().numpy()
    rs64 = d_rs.cpu().numpy()
    ctx.close()
    del ctx

    ms_step = max_over_ranks(float(np.sum(t_mixed)) / args.steps)
    ms_fp64 = max_over_ranks(float(np.sum(t_fp64)) / len(t_fp64))
    ms_e2e = max_over_ranks(float(np.sum(e2e_t)) / len(e2e_t))
    value = job_throughput(ws, nk, ms_step)
    c2 = c2_leg(pbs, dev, stream) if name == "c3" and rank == 0 else None
    if rank != 0:
        return
    peaks, peak_kind = _peaks()
    df_classes = {"gram", "small_rr"}  # double-float arithmetic under the mixed policy
    fp64_classes = {"block_update"}
    if dominant in df_classes:
        achieved = dom_work / (dom_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": DF_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / DF_PEAK_TFLOPS, "traffic": None, "kernel": dominant,
                "peak_kind": "derived double-float rate on the FP32 pipe (152 SMs x 128 lanes x 1.98 GHz, "
                             "48 FP32 instructions per 8-flop compensated complex multiply-add)"}
    elif dominant in fp64_classes:
        achieved = dom_work / (dom_ms / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / FP64_PEAK_TFLOPS, "traffic": None, "kernel": dominant,
                "peak_kind": "derived FP64 rate (152 SMs x 4 flop/clk x 1.98 GHz, matches a measured FMA probe)"}
    else:
        achieved = dom_work / (dom_ms / 1e3) / 1e9
        roof = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": None, "kernel": dominant,
                "peak_kind": f"{peak_kind} hbm_gbs"}
    roof["avg_launch_us"] = 1e3 * dom_ms / max(dom_n, 1)
    roof["launches_timed"] = dom_n
    roof["timing"] = f"CUDA events on the library stream around every {SAMPLE_EVERY}th launch in the timed steps"
    roof["share_of_kernel_time"] = shares[dominant][0] / sum(v[0] for v in shares.values())
    cb = oracle_sample_kps(name, seconds_budget=20.0) if ws == 1 else None
    rel = np.abs(lam_mixed - lam_fp64) / lam_fp64
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c128 storage; FP64 residual and update; double-float (FP32 pipe) Gram, Rayleigh quotients "
                 "and small Rayleigh-Ritz; c64 FP32 multigrid", "data": "synthetic",
        "config": {"workload": w["text"], "grid": f"{n}x{n}", "k_points": nk, "bands": nev, "block": w["block"],
                   "tol": TOL, "k_points_in_flight": w["kbatch"], "precision": "mixed",
                   "l2": "flushed (512 MiB write) before every timed step", "replicas": ws},
        "converged": ok, "max_resid": float(rs.max()), "iters_per_k": its.tolist(),
        "plain_fp64": {"value": job_throughput(ws, nk, ms_fp64), "unit": UNIT, "ms_per_step": ms_fp64,
                       "steps": len(t_fp64), "max_resid": float(rs64.max()),
                       "converged": bool(np.all(rs64 <= _band_tol(eps, n, lam_fp64)))},
        "max_rel_err_mixed_vs_fp64_per_band": rel.max(axis=0).tolist(),
        "clocks": clk,
        "e2e": {"value": job_throughput(ws, nk, ms_e2e), "unit": UNIT, "steps": e2e_steps,
                "h2d_bytes_per_step": int(eps.nbytes + ks.nbytes),
                "d2h_bytes_per_step": int(lam_h.nbytes + res_h.nbytes + it_h.nbytes)},
        "gpu_launches": int(launches),
        "gpu_launches_note": f"library kernel launches in the {args.steps} timed steps (pbs_launch_count)",
        "roofline": roof,
        "kernel_time_ms_per_class_warmup": {c: round(v[0], 3) for c, v in shares.items()},
        "achieved_per_class_warmup": per_class_rates(shares, peaks["hbm_gbs"]),
        "cpu_baseline": cb,
    }
    if c2 is not None:
        line["c2"] = c2
    print(json.dumps(line), flush=True)


def once_run(name: str, fp64_k: int) -> None:
    """One timed solve of a path workload in the mixed policy and one in plain FP64 (on the
    first ``fp64_k`` Bloch vectors of the path, all of them when 0), for workloads too long
    for repeated timing (c4: about 16 GB per Bloch vector).  CUDA events around each call
    on the caller's stream, inputs resident; the workspace of each policy is allocated by a
    short solve (one more Bloch vector than are in flight) first.  One JSON line:
    k-points/s of both policies, iterations, residuals and the per-band relative difference
    of the eigenvalues at the shared Bloch vectors."""
    import torch
    import __graft_entry__ as ge
    ge.build()
    import paper_2304_00337_gb300 as pbs
    w = WORKLOADS[name]
    n, nev = w["n"], w["nev"]
    eps, ks = workload_inputs(name)
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    d_eps = torch.from_numpy(eps.copy()).to(dev)
    out = {}
    lam = {}
    with pbs.Context(0) as ctx:
        for label, prec, kk in (("mixed", pbs.PBS_MIXED, ks), ("plain_fp64", pbs.PBS_FP64,
                                                               ks[:fp64_k] if fp64_k else ks)):
            nk = len(kk)
            d_ks = torch.from_numpy(np.ascontiguousarray(kk)).to(dev)
            d_ev = torch.zeros((nk, nev), dtype=torch.float64, device=dev)
            d_rs = torch.zeros_like(d_ev)
            d_it = torch.zeros(nk, dtype=torch.int32, device=dev)
            o = _opts(pbs, name, prec)
            o.kbatch = min(w["kbatch"], nk)

            def run(count):
                ctx.solve_path_device(1.0, 1.0, n, n, d_eps.data_ptr(), o, count, d_ks.data_ptr(), d_ev.data_ptr(),
                                      d_rs.data_ptr(), d_it.data_ptr(), stream)
            run(min(nk, o.kbatch + 1))  # hierarchy, workspace (with the chains' history), tuning
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run(nk)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1)
            ev = d_ev.cpu().numpy()
            rs = d_rs.cpu().numpy()
            lam[label] = ev
            out[label] = {"value": nk / (ms / 1e3), "unit": UNIT, "seconds": ms / 1e3, "k_points": nk,
                          "iters_per_k": d_it.cpu().numpy().tolist(), "max_resid": float(rs.max()),
                          "converged": bool(np.all(rs <= _band_tol(eps, n, ev)))}
    m = lam["plain_fp64"].shape[0]
    rel = np.abs(lam["mixed"][:m] - lam["plain_fp64"]) / lam["plain_fp64"]
    print(json.dumps({"metric": METRIC, "value": out["mixed"]["value"], "unit": UNIT, "higher_is_better": True,
                      "n_gpus": 1, "data": "synthetic", "mixed": out["mixed"], "plain_fp64": out["plain_fp64"],
                      "max_rel_err_mixed_vs_fp64_per_band": rel.max(axis=0).tolist(),
                      "eigenvalues_mixed": lam["mixed"].tolist(),
                      "config": {"workload": w["text"], "grid": f"{n}x{n}", "k_points_in_flight": w["kbatch"],
                                 "timing": "one solve per policy (CUDA events), after a short set-up solve"}}),
          flush=True)


def profile_run(name: str, nk: int, precision: str):
    """One untimed solve of the first ``nk`` Bloch vectors of a workload (a small case for ncu)."""
    import __graft_entry__ as ge
    ge.build()
    import paper_2304_00337_gb300 as pbs
    w = WORKLOADS[name]
    eps, ks = workload_inputs(name)
    geom = pbs.Geometry(eps)
    prec = pbs.PBS_MIXED if precision == "mixed" else pbs.PBS_FP64
    o = _opts(pbs, name, prec)
    o.kbatch = min(w["kbatch"], nk)
    with pbs.Context(0) as ctx:
        lam, res, it = ctx.solve_path(geom, o, ks[:nk])
    print(f"profile-run ok: {name}, {nk} k-points, iterations {it.tolist()}, max resid {res.max():.2e}", flush=True)


def serving_bench(njobs: int, grids, slots: int, rate_factor: float) -> None:
    """Serving workload: a seeded stream of rod-crystal path jobs (radius U(0.1, 0.45) a,
    eps U(2, 13), 6-12 bands with two throw-away vectors, 10-64 Bloch vectors on
    Gamma-X-M-Gamma, meshes drawn from ``grids``) submitted through pbs_submit at Poisson
    arrival times, at ``rate_factor`` of the saturation rate measured in a closed-loop
    warm-up, into a context with ``slots`` serving slots (continuous batching: jobs that
    arrive while others run are admitted as slots and memory free up).  Prints one JSON
    line with the p50 / p99 latency from submission to completion and the k-points/s."""
    import __graft_entry__ as ge
    ge.build()
    import paper_2304_00337_gb300 as pbs
    import pbs_inputs as gi
    jobs = gi.serving_jobs(njobs, seed=0, rate_per_s=1.0, grids=tuple(grids))

    def args_of(j):
        geom = pbs.Geometry(gi.rod_eps(j["grid"], j["grid"], radius=j["radius"], eps_rod=j["eps_rod"]))
        o = pbs.default_opts(nev=j["bands"], block=j["block"], tol=TOL, kbatch=min(8, j["nk"]))
        return geom, o, gi.gxmg_path(j["nk"])

    prepared = [args_of(j) for j in jobs]
    with pbs.Context(0) as ctx:
        ctx.serve_slots(slots)
        # closed loop: the first 2 slots jobs, all submitted at once, give the saturation rate
        warm = prepared[:2 * slots]
        t0 = time.perf_counter()
        ids = [ctx.submit(*a) for a in warm]
        for i in ids:
            ctx.fetch(i)
        rate = rate_factor * len(warm) / (time.perf_counter() - t0)
        # open loop: Poisson arrivals (the stream's unit-rate arrival times scaled to `rate`)
        start = time.perf_counter()
        ids = []
        for j, a in zip(jobs, prepared):
            due = start + j["arrival_s"] / rate
            now = time.perf_counter()
            if due > now:
                time.sleep(due - now)
            ids.append(ctx.submit(*a))
        while not all(ctx.poll(i) for i in ids):
            time.sleep(0.01)
        times = [ctx.job_times(i) for i in ids]
        res = [ctx.fetch(i, allow_noconv=True) for i in ids]
        wall = time.perf_counter() - start
    lat = np.array([r[3] for r in res])
    ok = all(np.all(r[1] <= 1e-6) for r in res)
    kpts = sum(j["nk"] for j in jobs)
    # concurrency: the mean number of jobs running, from their start and finish times
    busy = sum(t[2] - t[1] for t in times)
    span = max(t[2] for t in times) - min(t[1] for t in times)
    by_grid = {}
    for j, l in zip(jobs, lat):
        by_grid.setdefault(j["grid"], []).append(l)
    print(json.dumps({
        "metric": "serving latency p50 (submission to completion)", "value": float(np.percentile(lat, 50)),
        "unit": "s", "higher_is_better": False, "p99_s": float(np.percentile(lat, 99)),
        "mean_s": float(lat.mean()), "jobs": njobs, "arrival_rate_per_s": rate,
        "throughput_jobs_per_s": njobs / wall, "throughput_kpoints_per_s": kpts / wall,
        "mean_jobs_running": busy / span, "converged": bool(ok), "wall_s": wall,
        "p50_s_by_grid": {str(g): float(np.percentile(v, 50)) for g, v in sorted(by_grid.items())},
        "data": "synthetic", "n_gpus": 1,
        "config": {"workload": f"rod-crystal path jobs, Poisson arrivals at {rate_factor} x saturation",
                   "grids": list(grids), "bands": "6-12 (+2 throw-away)", "k_points_per_job": "10-64",
                   "seed": 0, "slots": slots, "k_points_in_flight_per_job": "min(8, nk)"}}), flush=True)


def grid_bench(kappa: int, n: int) -> None:
    """The paper's Brillouin-zone workload (Section 8: rod eps = 11.56, r = 0.18 a, 16 bands
    with 8 throw-away vectors, kappa x kappa sample with the Section 6 schedule) on an
    n x n mesh, at the paper's tolerance 1e-2 and at 1e-8.  One JSON line: k-points/s
    and the iterations per Bloch vector (the paper reports fewer than 4 at 1e-2)."""
    import __graft_entry__ as ge
    ge.build()
    import paper_2304_00337_gb300 as pbs
    import pbs_inputs as gi
    geom = pbs.Geometry(gi.rod_eps(n, n, radius=0.18, eps_rod=11.56))
    out = {}
    with pbs.Context(0) as ctx:
        for tol in (1e-2, 1e-8):
            o = pbs.default_opts(nev=16, block=24, tol=tol, kbatch=4)
            ctx.solve_grid(geom, o, 4)  # warm-up (hierarchy, workspace)
            t0 = time.perf_counter()
            ks, lam, res, it = ctx.solve_grid(geom, o, kappa)
            dt = time.perf_counter() - t0
            out[f"tol_{tol:g}"] = {"seconds": dt, "kpoints_per_s": kappa * kappa / dt,
                                   "iters_first_k": int(it[0]), "iters_mean_others": float(np.mean(it[1:])),
                                   "iters_max_others": int(np.max(it[1:])),
                                   "iters_p50_others": float(np.median(it[1:])),
                                   "max_resid": float(res.max())}
    print(json.dumps({"metric": "Brillouin-zone grid k-points/s (tol 1e-8)",
                      "value": out["tol_1e-08"]["kpoints_per_s"], "unit": "k-points/s", "higher_is_better": True,
                      "n_gpus": 1, "data": "synthetic", "results": out,
                      "config": {"workload": f"rod eps=11.56 r=0.18a, {n}x{n}, {kappa}x{kappa} k-points, "
                                             "16 bands + 8 throw-away, Section 6 extrapolation schedule",
                                 "k_points_in_flight": 4, "precision": "mixed"}}), flush=True)


def throwaway_bench(n: int) -> None:
    """Section 7 experiment: eps = 100 in the disk |x - (1/2, 1/2)| <= 1/3, 1 elsewhere;
    16 wanted bands plus 1..16 throw-away vectors, at k = (pi/2, pi/4) on an n x n mesh
    (the paper names neither), for the paper's preconditioned block inverse iteration
    (span 1) and LOBPCG (span 3), tolerance 1e-8 on the wanted bands only.  One JSON
    line: iterations, time and the observed convergence factor per iteration,
    (1e-8)^(1/iterations), for each count of throw-away vectors."""
    import __graft_entry__ as ge
    ge.build()
    import paper_2304_00337_gb300 as pbs
    import pbs_inputs as gi
    geom = pbs.Geometry(gi.rod_eps(n, n, radius=1.0 / 3.0, eps_rod=100.0))
    k = (np.pi / 2, np.pi / 4)
    rows = []
    with pbs.Context(0) as ctx:
        ctx.solve_k(geom, dict(nev=16, block=17, tol=1e-4), k, allow_noconv=True)  # warm-up
        for span in (1, 3):
            for extra in (1, 2, 4, 8, 16):
                o = dict(nev=16, block=16 + extra, span=span, max_iter=2000, seed=0)
                t0 = time.perf_counter()
                lam, res, it, _ = ctx.solve_k(geom, o, k, allow_noconv=True)
                dt = time.perf_counter() - t0
                rows.append({"span": span, "throw_away": extra, "iterations": int(it), "seconds": dt,
                             "rate_per_iteration": float(1e-8 ** (1.0 / max(int(it), 1))),
                             "max_resid": float(res.max())})
    best = min((r for r in rows if r["span"] == 3), key=lambda r: r["seconds"])
    print(json.dumps({"metric": "throw-away study: fastest LOBPCG solve (16 bands)", "value": best["seconds"],
                      "unit": "s", "higher_is_better": False, "n_gpus": 1, "data": "synthetic", "results": rows,
                      "config": {"workload": f"eps=100 disk r=1/3, {n}x{n}, k=(pi/2,pi/4), 16 bands",
                                 "precision": "mixed", "tol": 1e-8}}), flush=True)


def per_class_rates(shares: dict, hbm_gbs: float) -> dict:
    """Achieved rate of every timed kernel class in the first warm-up step: algorithmic
    bytes per second (and the fraction of the measured HBM copy bandwidth) for the
    streaming classes, algorithmic flops per second for the arithmetic-bound ones."""
    out = {}
    for c, (ms, n, work) in shares.items():
        if ms <= 0 or n <= 0:
            continue
        if c in ("gram", "small_rr", "block_update"):
            out[c] = {"tflops": work / (ms * 1e-3) / 1e12, "ms": round(ms, 3), "launches": int(n)}
        else:
            gbs = work / (ms * 1e-3) / 1e9
            out[c] = {"gbs": gbs, "frac_hbm": gbs / hbm_gbs, "ms": round(ms, 3), "launches": int(n)}
    return out


def householder_bench(n: int, q: int, reps: int) -> None:
    """The generalised Householder orthonormalisation of Section 4 (``pbs_m_householder``) on
    the bench geometry: a seeded D x q block (q = 30, the trial width of the path's iteration)
    of the 256x256 rod crystal at X.  One JSON line: factorisations/s (CUDA events around
    ``reps`` calls on the caller's stream, inputs resident), the streaming kernels' achieved
    bandwidth, and the oracle's time for one factorisation on the host cores."""
    import __graft_entry__ as ge
    ge.build()
    import torch
    import paper_2304_00337_gb300 as pbs
    import pbs_inputs as gi
    from oracle import fem
    from oracle.householder import m_householder, pivots
    eps = gi.rod_eps(n, n, radius=0.2, eps_rod=8.9)
    geom = pbs.Geometry(eps)
    k = (np.pi, 0.0)
    S = gi.random_block(geom.D, q, seed=23)
    Sd = torch.from_numpy(S).cuda()
    Ed = torch.zeros_like(Sd)
    Rd = torch.zeros((q, q), dtype=torch.complex128, device="cuda")
    st = torch.cuda.current_stream()
    with pbs.Context(0) as ctx:
        for _ in range(3):
            ctx.m_householder(geom, k, q, Sd.data_ptr(), Ed.data_ptr(), Rd.data_ptr(), st)
        ctx.profile_enable("householder")
        launches0 = pbs.launch_count()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(st)
        for _ in range(reps):
            ctx.m_householder(geom, k, q, Sd.data_ptr(), Ed.data_ptr(), Rd.data_ptr(), st)
        t1.record(st)
        torch.cuda.synchronize()
        ms = t0.elapsed_time(t1) / reps
        launches = (pbs.launch_count() - launches0) // reps
        kms, klaunch, kbytes = ctx.profile_read("householder")
    peaks, peak_kind = _peaks()
    gbs = kbytes / (kms * 1e-3) / 1e9 if kms > 0 else 0.0
    # FP64 flops of the timed kernels per call: the dot kernel evaluates the mass
    # stencil (12 flops an edge) and one complex multiply-add (8) per later column,
    # the update one complex multiply-add per later column; reflections of the
    # factorisation act on q-1-i columns, those that form E on q-i
    D = geom.D
    ncs = [q - 1 - i for i in range(q) if q - 1 - i > 0] + [q - i for i in range(q)]
    flops = sum(D * (12 + 16 * nc) for nc in ncs) * reps
    tflops = flops / (kms * 1e-3) / 1e12 if kms > 0 else 0.0
    c0 = time.perf_counter()
    M = fem.assemble(fem.Mesh(1.0, 1.0, n, n), eps, k)["M"]
    m_householder(M, S.T, pivots(n, n, q))
    cpu_s = time.perf_counter() - c0
    print(json.dumps({
        "metric": "M-Householder block orthonormalisations/s", "value": 1e3 / ms, "unit": "factorisations/s",
        "higher_is_better": True, "n_gpus": 1, "ms_per_factorisation": ms, "gpu_launches_per_call": int(launches),
        "dtype": "c128 (FP64)", "data": "synthetic",
        "roofline": {"bound": "alu", "achieved": tflops, "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": tflops / FP64_PEAK_TFLOPS, "traffic": None,
                     "kernel": "k_hh_mdots + k_hh_update (reflection of the later columns)",
                     "peak_kind": "FP64 rate (152 SMs x 4 FP64 flop/clk; 1.20 TFLOP/s measured with an FMA-chain probe)",
                     "hbm_achieved_gbs": gbs, "hbm_peak_gbs": peaks["hbm_gbs"], "hbm_peak_kind": peak_kind,
                     "note": "working set (S copy and E, 2 x 63 MB) is about the L2 size: partly L2-resident",
                     "launches_timed": int(klaunch)},
        "cpu_baseline": {"value": 1.0 / cpu_s, "unit": "factorisations/s", "cores": os.cpu_count(),
                         "kind": "oracle", "sample": "one factorisation of the same block, incl. mass assembly"},
        "config": {"workload": f"rod eps=8.9 r=0.2a, {n}x{n} (D = {geom.D}), {q} columns, k = X",
                   "precision": "fp64"}}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--profile-run", type=int, default=0, metavar="NK",
                    help="solve the first NK k-points of the workload once (no timing) - the small case for ncu")
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--workload", default="c3",
                    choices=sorted(WORKLOADS) + ["serving", "grid", "throwaway", "householder"],
                    help="c3: the headline 1024x1024 path with 64 k-points in flight (default); c2: 256x256 "
                         "path; c4: 4096x4096 disks; serving: the job-stream latency line; grid: the paper's "
                         "kappa x kappa Brillouin-zone workload")
    ap.add_argument("--kappa", type=int, default=30, help="grid workload: k-points per direction")
    ap.add_argument("--grid-n", type=int, default=256, help="grid workload: cells per direction")
    ap.add_argument("--jobs", type=int, default=200, help="jobs of the serving workload")
    ap.add_argument("--serve-grids", default="128,256,512,1024,2048", help="serving workload: mesh sizes")
    ap.add_argument("--slots", type=int, default=4, help="serving workload: serving slots")
    ap.add_argument("--rate", type=float, default=0.8, help="serving workload: arrival rate / saturation rate")
    ap.add_argument("--once", action="store_true",
                    help="one timed solve per policy (workloads too long for repeated timing, e.g. c4)")
    ap.add_argument("--fp64-k", type=int, default=0, help="--once: Bloch vectors of the FP64 solve (0: all)")
    args = ap.parse_args()
    if args.workload == "serving" and args.impl == "ours":
        serving_bench(args.jobs, [int(g) for g in args.serve_grids.split(",")], args.slots, args.rate)
        return
    if args.workload == "grid" and args.impl == "ours":
        grid_bench(args.kappa, args.grid_n)
        return
    if args.workload == "throwaway" and args.impl == "ours":
        throwaway_bench(128)
        return
    if args.workload == "householder" and args.impl == "ours":
        householder_bench(256, 30, 10)
        return
    if args.workload not in WORKLOADS:
        print(json.dumps({"impl": args.impl, "unavailable": f"no reference arm for the {args.workload} workload"}))
        return
    if args.profile_run:
        profile_run(args.workload, args.profile_run, args.precision)
        return
    if args.once and args.impl == "ours":
        once_run(args.workload, args.fp64_k)
        return
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
