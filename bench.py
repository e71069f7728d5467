"""Throughput benchmark of the GB300 EC-PIC hot path (particle-steps/s).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

A "step" is one time step of the whole hot path -- gather, leapfrog push,
walls, null-collision MCC, fixed-point deposit, Poisson and field, the counting
sort every 16 steps -- for every live particle of the workload.  Inputs are
synthetic and seeded (``paper_2308_13092_gb300.inputs``); no dataset exists.

Headline workload ("batched"): 256 independent RF-CCP runs drawn from
``default_rng(0)`` -- cells logU[64,1024], particles logU[1e4,1e6] split
between electrons and 4 amu ions, V0 logU[100,500] V, p logU[10,100] mTorr,
dx U[0.5,1] mm, n0 = 1e14, dt = 1/(400 f) -- all resident on the GPU and
advanced together, one launch per kernel phase, replayed from CUDA graphs.
About 5.5e7 particles (1.5 GB of particle state, far above the 129 MB L2).

Also reported (same JSON line):
  single_run  the 1024-cell, 524,288-particle resolved discharge alone (its
              29 MB state fits in L2, so L2 is flushed before every timed step);
  one_by_one  the same batched manifest run one run at a time (a sample);
  served      a Poisson stream of run requests admitted by device memory,
              with p50/p99 completion latency, against one-at-a-time service;
  e2e         the batched job through the public API from host configs to
              host diagnostics, whole jobs of 5 RF periods (2000 steps).
The timed window holds whole sort cycles: the autotuner picks the sort
cadence K among the divisors of --steps (4..64), the warm-up runs on to a sort
boundary, and the window's per-kernel device times come from CUDA events
recorded inside the very graph replays that advance the runs (phase timing),
so that pass + collision + field + sort add up to the timed step.
For N > 1 (torchrun) each rank runs its own manifest (seed = rank); value =
all ranks' particle-steps / max over ranks of the time.  --impl reference
times the FP64 CPU oracle on the host cores (a thread per core, each stepping
its own runs of a sample of the same workload).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

from paper_2308_13092_gb300 import inputs as I  # noqa: E402

# Algorithmic HBM bytes per particle-step of the fused pass: read cell, xi,
# vx, vy, vz (4 B each) and the 8 B id = 28 B, write cell, xi, vx = 12 B.
BYTES_PER_PARTICLE_STEP = 40
METRIC = "particle-steps/s"
N_RUNS = 256
AUTOTUNE_STEPS = 64  # steps per autotuner trial (two per candidate) before the warm-up
E2E_STEPS = 2000  # end-to-end job length: 5 RF periods at 400 steps per period
SAMPLE_EVERY = 40  # energy-sample cadence of the manifest runs: 1/10 RF period

# DRAM traffic of k_pass measured with ncu (dram__bytes_read.sum +
# dram__bytes_write.sum of one stepping launch on the 64-run manifest, see
# profiles/k_pass_batched64.md), per particle-step.  It is reported only while
# the kernel sources' code (comments and whitespace aside) hashes to the
# measured version; after any change to the code the traffic is unknown
# (null) until it is measured again.
TRAFFIC = {"sources_sha256": "97d3f44d0645effc5e7448ce61f66f70aefea41fc9a25ca91342ee7782d3395a",
           "dram_bytes_per_particle_step": 570.325e6 / 14.3047e6}


def kernel_code(text):
    """The code of a CUDA source without its comments and with whitespace
    collapsed, so that edits to comments leave the traffic pin valid."""
    import re
    text = re.sub(r"/\*.*?\*/", " ", text, flags=re.S)
    text = re.sub(r"//[^\n]*", " ", text)
    return " ".join(text.split())


def kernel_sources_sha256():
    import hashlib
    h = hashlib.sha256()
    for f in ("kernels.cu", "ecpic_dev.cuh"):
        with open(os.path.join(ROOT, "paper_2308_13092_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(kernel_code(fh.read()).encode())
    return h.hexdigest()


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=400)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--runs", type=int, default=N_RUNS)
    ap.add_argument("--scale", type=float, default=1.0, help="particle-count scale")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="engine defaults (sort every 16 steps, automatic grid) instead of the autotuner")
    ap.add_argument("--no-extras", action="store_true",
                    help="headline only (no single-run, one-by-one, served, e2e)")
    return ap.parse_args()


def autotune_steps(per_trial, Ks=(8, 16, 32, 64), grids=5, sample_every=SAMPLE_EVERY):
    """Steps the autotuner advances the runs: every (K, grid) pair is tried
    twice; per trial, K steps to start the cadence and max(per_trial, 2K)
    rounded up to whole cycles of both the sort and the energy sample (the
    sort cycle alone where their common multiple exceeds 8x that)."""
    total = 0
    for K in Ks:
        want = max(per_trial, 2 * K)
        cyc = K
        if sample_every > 0:
            lcm = K * sample_every // math.gcd(K, sample_every)
            cyc = lcm if lcm <= 8 * want else K
        total += K + -(-want // cyc) * cyc
    return 2 * grids * total


def sample_steps(k0, steps, every=SAMPLE_EVERY):
    """Energy-sample steps among the `steps` steps from level k0: the push of
    level k samples when (k + 1) % every == 0."""
    if every <= 0:
        return 0
    return sum(1 for k in range(k0, k0 + steps) if (k + 1) % every == 0)


def combine_ranks(ms, ps):
    """Whole-job figures of a weak-scaling replica run: the slowest rank's
    time and the particle-steps of all ranks (host-side gloo reductions; the
    ranks share no data)."""
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    p = torch.tensor([float(ps)], dtype=torch.float64)
    dist.all_reduce(p, op=dist.ReduceOp.SUM)
    return float(t.item()), float(p.item())


def dist_env():
    return (int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")),
            int(os.environ.get("LOCAL_RANK", "0")))


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        return json.load(open(p)).get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


def manifest(rank, args, steps):
    runs = I.batched_manifest(args.runs, seed=rank, steps=steps, scale=args.scale)
    for r in runs:
        r.sample_every = SAMPLE_EVERY
    return runs


class Clocks:
    """nvidia-smi sampling during the timed region."""

    def __init__(self, index):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={index}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
                pw.append(float(parts[3]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(pw) if pw else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------------ oracle arm
def host_threads():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_parallel(cfgs, threads, warmup, steps, budget_s, warm_budget_s=20.0):
    """The FP64 C oracle as it stands, on `threads` host threads: thread t
    steps the runs t, t + threads, ... of `cfgs` (ctypes releases the GIL
    inside every oracle call, and runs share no state), `warmup` untimed steps,
    then up to `steps` timed steps each, stopping once `budget_s` seconds have
    passed.  Particle-steps count the live particles at the start of every
    step.  Returns (particle-steps/s, particle-steps, timed steps of the
    slowest thread, runs used, warm-up steps done)."""
    import threading
    from concurrent.futures import ThreadPoolExecutor
    from helpers import oracle_from_config
    threads = max(1, min(threads, len(cfgs)))
    bar = threading.Barrier(threads)
    t0 = [0.0]

    def work(t):
        mine = [oracle_from_config(c) for c in cfgs[t::threads]]
        tw = time.perf_counter()
        warm = 0
        for _ in range(warmup):
            for o in mine:
                o.step(1, allow_capacity=True)
            warm += 1
            if time.perf_counter() - tw > warm_budget_s:
                break
        if bar.wait() == 0:
            t0[0] = time.perf_counter()
        bar.wait()
        ps, done = 0, 0
        for _ in range(steps):
            for o in mine:
                ps += sum(s["n"] for s in o.counters()["species"])
                o.step(1, allow_capacity=True)
            done += 1
            if time.perf_counter() - t0[0] > budget_s:
                break
        t1 = time.perf_counter()
        for o in mine:
            o.close()
        return ps, done, t1, len(mine), warm

    with ThreadPoolExecutor(threads) as ex:
        res = list(ex.map(work, range(threads)))
    wall = max(r[2] for r in res) - t0[0]
    ps = sum(r[0] for r in res)
    return (ps / wall, ps, min(r[1] for r in res), sum(r[3] for r in res),
            min(r[4] for r in res))


def cpu_baseline_block(cfgs, budget_s=10.0, steps=400):
    """Oracle baseline on the manifest: all host cores (a thread each over
    independent runs) and one core, each for about `budget_s` seconds of
    stepping after loading."""
    nthr = host_threads()
    v_all, ps_all, st_all, used_all, _ = oracle_parallel(cfgs[: 2 * nthr], nthr, 0, steps, budget_s)
    v_one, ps_one, st_one, used_one, _ = oracle_parallel(cfgs[:2], 1, 0, steps, budget_s)
    return {"value": v_all, "unit": "particle-steps/s", "cores": nthr, "kind": "oracle",
            "sample": f"first {used_all} runs of the batched manifest, {st_all}+ steps each "
                      f"({ps_all:.3g} particle-steps), FP64, {nthr} host threads (one per core, "
                      f"each stepping its own runs)",
            "single_core": {"value": v_one, "cores": 1, "particle_steps": ps_one,
                            "sample": f"first {used_one} runs of the manifest, {st_one} steps each"}}


def run_reference(args, rank, world):
    if rank != 0:
        return
    cfgs = manifest(0, args, steps=args.warmup + args.steps)
    nthr = host_threads()
    # a bounded sample: two runs per host thread, the timed steps stopping
    # after 120 s of host time so that the default run ends within minutes
    sample = cfgs[: min(2 * nthr, len(cfgs))]
    v, ps, done, used, warm = oracle_parallel(sample, nthr, args.warmup, args.steps, 120.0)
    wall_ms = ps / v * 1e3
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "particle-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "steps_timed": done,
            "warmup_done": warm,
            "ms_per_step": wall_ms / max(1, done), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"batched RF-CCP manifest ({len(cfgs)} runs); FP64 CPU oracle "
                                   f"on the first {used} runs, {nthr} host threads"},
            "cpu_baseline": {"value": v, "unit": "particle-steps/s", "cores": min(nthr, used),
                             "kind": "oracle",
                             "sample": f"{used} runs of the batched manifest, {done} steps each "
                                       f"after {warm} warm-up, {ps:.3g} particle-steps"},
            "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ GPU arms
def pump_until_done(eng, chunk=200):
    while True:
        r, q = eng.pump(chunk)
        if r == 0 and q == 0:
            return


def single_run_block(torch, ecpic, stream, device, steps=100, warmup=10):
    cfg = I.config_resolved(seed=11)
    cfg.sample_every = 20
    run = ecpic.Run.from_config(cfg, device=device, stream=stream.cuda_stream)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def l2_flush():
        flush.zero_()
        flush.sum()

    with torch.cuda.stream(stream):
        # sort cadence (divisors of the timed steps) and pass grid from the
        # library's autotuner, as for the batched line
        tuned = run.autotune(16, ks=sort_cadences(steps))
        run.set_phase_timing(True)  # per-phase events inside the replayed steps
        for _ in range(warmup):
            l2_flush()
            run.step(1)
        run.sync()
        run.phase_times()  # clear the warm-up's sums
        ps0 = run.diagnostics(profiles=False)
        n0 = sum(s["n"] for s in ps0["species"])
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(steps)]
        for k in range(steps):
            l2_flush()
            evs[k][0].record(stream)
            run.step(1)
            evs[k][1].record(stream)
        stream.synchronize()
        run.sync()
        n1 = sum(s["n"] for s in run.diagnostics(profiles=False)["species"])
        ms = float(sum(a.elapsed_time(b) for a, b in evs))
        prof = run.phase_times()  # the timed steps' own phases
    run.close()
    del flush
    v = 0.5 * (n0 + n1) * steps / (ms * 1e-3)
    return {"value": v, "unit": "particle-steps/s", "ms_per_step": ms / steps,
            "workload": f"{cfg.name}: {cfg.N} uniform cells, {cfg.n_particles} particles",
            "l2": "flushed before every timed step",
            "pass_ms_avg": prof["pass_ms"] / max(1, prof["launches"][0]),
            "field_ms_avg": prof["field_ms"] / max(1, prof["launches"][1]),
            "collide_ms_avg": prof["collide_ms"] / max(1, prof["launches"][3]),
            "sort_ms_per_step": prof["sort_ms"] / max(1, prof["steps"]),
            "steps_timed": prof["steps"], "sort_every": tuned["sort_every"],
            "pass_ctas": tuned["pass_ctas"] or "auto"}


def one_by_one_block(ecpic, cfgs, stream, device, n_runs=12, steps=200):
    """The manifest one run at a time through the engine (a sample)."""
    rng = np.random.default_rng(5)
    pick = rng.choice(len(cfgs), min(n_runs, len(cfgs)), replace=False)
    eng = ecpic.Engine(device=device, stream=stream.cuda_stream, max_slots=1, max_cells=1024)
    t = 0.0
    ps = 0
    for i in pick:
        c = cfgs[i]
        tk = eng.submit(c, n_steps=steps)
        eng.pump(0)  # admit and load
        s0 = eng.stats()["particle_steps"]
        t0 = time.perf_counter()
        pump_until_done(eng, chunk=steps)
        t += time.perf_counter() - t0
        ps += eng.poll(tk)["particle_steps"]
        eng.release(tk)
        del s0
    eng.close()
    return {"value": ps / t, "unit": "particle-steps/s", "runs": int(len(pick)),
            "steps_per_run": steps,
            "what": "sampled runs of the batched manifest, each alone (wall clock per run)"}


def appendix_b_block(ecpic, stream, device, steps=100_000, chunks=10):
    """App. B sweep as one batch: EC and MC, collisionless periodic Table 1
    plasma on 2048 cells of dx/lambda_De = 0.5..16, dt = 0.1/w_pe, 10,000/w_pe.
    Heating = relative change of the total energy W = KE + FE from the first
    sample (t = 100/w_pe); KE alone beside it.  Wall clock of the whole batch."""
    cfgs = I.appendix_b_sweep(steps=steps, sample_every=steps // (10 * chunks))
    eng = ecpic.Engine(device=device, stream=stream.cuda_stream, max_slots=len(cfgs),
                       max_cells=2048, species_per_run=1)
    tks = [eng.submit(c) for c in cfgs]
    eng.pump(0)
    W0, K0, dK, series = {}, {}, {}, {c.name: [] for c in cfgs}
    t0 = time.perf_counter()
    ps0 = eng.stats()["particle_steps"]
    done = 0
    first = steps // (10 * chunks)
    for k in range(chunks + 1):
        n = first if k == 0 else steps // chunks - (first if k == 1 else 0)
        eng.pump(n)
        done += n
        for c, tk in zip(cfgs, tks):
            d = eng.poll(tk, diagnostics=True)["diag"]
            w, ke = float(d["ke"].sum() + d["fe"]), float(d["ke"].sum())
            if k == 0:
                W0[c.name], K0[c.name] = w, ke
            else:
                series[c.name].append(round(w / W0[c.name] - 1.0, 6))
            if k == chunks:
                dK[c.name] = round(ke / K0[c.name] - 1.0, 6)
    wall = time.perf_counter() - t0
    ps = eng.stats()["particle_steps"] - ps0
    eng.close()
    return {"value": ps / wall, "unit": "particle-steps/s", "runs": len(cfgs), "steps": done,
            "cells": 2048, "ppc": 64,
            "dW_over_W": series, "dKE_over_KE_final": dK,
            "what": "App. B sweep (EC and MC at dx/lambda_De 0.5-16) as one batch; "
                    "relative total-energy change every 1000/w_pe from t = 100/w_pe"}


def served_block(ecpic, stream, device, capacity, n_req=2000, rho=0.7, slots=256, n_alone=256):
    """Poisson arrivals of CCP run requests (sizes as in the batched manifest,
    5..50 RF periods at 1/10 of the steps), continuous batching vs one at a
    time; completion latency = finish - arrival.  Throughput is reported over
    the whole stream (first arrival to last completion: it includes the
    ramp-up from an empty GPU and the drain after the last arrival) and
    sustained, over the arrival window (from the arrival of the first quarter
    of the requests to the last arrival), from the engine's particle-step
    count sampled after every pump.  The stream holds as many requests as
    the served workload (2000), so that the arrival window is many request
    lifetimes long; one at a time serves only the first ``n_alone`` of them,
    with the same arrival times (it is overloaded at these rates, so its
    latencies grow with the stream's length; ``n_alone`` = 0 leaves it out).
    The engine holds up to ``slots`` runs, by default as many as the batched
    line keeps resident."""
    reqs = I.served_stream(n_req, seed=1, rate=1.0)
    for r in reqs:
        r.config.n_steps = max(40, r.config.n_steps // 10)
        I.with_headroom(r.config, I.growth_headroom(r.config.n_steps))
        r.config.sample_every = SAMPLE_EVERY
    work = np.mean([r.config.n_particles * r.config.n_steps for r in reqs])
    rate = rho * capacity / work
    arr = np.cumsum(np.random.default_rng(2).exponential(1.0 / rate, n_req))

    def serve(max_slots, n):
        eng = ecpic.Engine(device=device, stream=stream.cuda_stream, max_slots=max_slots,
                           max_cells=1024, mem_budget=64 << 30)
        t0 = time.perf_counter()
        pending = list(range(n))
        live = {}
        done = {}
        samples = []  # (time, particle-steps done) after every pump
        while len(done) < n:
            now = time.perf_counter() - t0
            while pending and arr[pending[0]] <= now:
                i = pending.pop(0)
                live[eng.submit(reqs[i].config)] = i
            if not live:
                time.sleep(max(0.0, arr[pending[0]] - now))
                continue
            eng.pump(40)
            now = time.perf_counter() - t0
            samples.append((now, eng.stats()["particle_steps"]))
            for tk in list(live):
                st = eng.poll(tk)
                if st["state"] == 2 or st["state"] < 0:
                    done[live.pop(tk)] = (now, st["particle_steps"])
                    eng.release(tk)
        total = time.perf_counter() - t0
        eng.close()
        lat = np.array([done[i][0] - arr[i] for i in range(n)])
        ps = sum(v[1] for v in done.values())
        t_a, t_b = float(arr[n // 4]), float(arr[n - 1])
        win = [(t, p) for t, p in samples if t_a <= t <= t_b]
        sustained = None
        if len(win) >= 2 and win[-1][0] > win[0][0]:
            sustained = (win[-1][1] - win[0][1]) / (win[-1][0] - win[0][0])
        return {"requests": n, "p50_s": float(np.percentile(lat, 50)),
                "p99_s": float(np.percentile(lat, 99)),
                "particle_steps_per_s": ps / total, "wall_s": total,
                "sustained_particle_steps_per_s": sustained,
                "sustained_window_s": [t_a, t_b]}

    mix = serve(slots, n_req)
    alone = serve(1, min(n_alone, n_req)) if n_alone > 0 else None
    sus = mix["sustained_particle_steps_per_s"]
    return {"requests": n_req, "load": rho, "arrival_rate_per_s": rate,
            "continuous_batching": mix, "one_at_a_time": alone,
            "sustained_over_batched": None if sus is None else sus / capacity,
            "slots": slots,
            "what": "Poisson arrivals; admitted by device memory as slots free; steps/10 of "
                    "the full request lengths; sustained = over the arrival window; one at "
                    "a time on the stream's first requests"}


def e2e_block(ecpic, cfgs, stream, device, steps):
    """Whole batched job through the public API: host configs in, host
    diagnostics out, wall clock."""
    import torch
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    eng = ecpic.Engine(device=device, stream=stream.cuda_stream, max_slots=len(cfgs),
                       max_cells=1024)
    h2d = 0
    tickets = []
    for c in cfgs:
        tickets.append(eng.submit(c, n_steps=steps))
        h2d += c.edges.nbytes + sum(p.sigma.nbytes for p in c.processes) + 512
    pump_until_done(eng, chunk=steps)
    ps = 0
    d2h = 0
    for tk, c in zip(tickets, cfgs):
        r = eng.poll(tk, diagnostics=True, profiles=True)
        ps += r["particle_steps"]
        d2h += 8 * (c.N + 1) * (4 * len(c.species) + 1) + 1024
    dt = time.perf_counter() - t0
    eng.close()
    return {"value": ps / dt, "unit": "particle-steps/s",
            "h2d_bytes_per_step": int(h2d / steps), "d2h_bytes_per_step": int(d2h / steps),
            "steps": steps,
            "what": f"ecpic_engine_submit of {len(cfgs)} host configs (particles loaded on the GPU), "
                    f"pump to completion ({steps} steps = {steps // 400} RF periods each), "
                    "ecpic_engine_poll of every run's diagnostics; wall clock"}


def sort_cadences(steps, lo=4, hi=64, want=(8, 16, 32, 64)):
    """Sort cadences for the autotuner that divide the timed window, so that
    it holds whole sort cycles: the divisors of `steps` in [lo, hi], at most
    one per wanted value (the nearest on a log scale)."""
    divs = [k for k in range(lo, min(hi, steps) + 1) if steps % k == 0]
    if not divs:
        return [steps] if steps <= 4096 else [hi]
    pick = []
    for w in want:
        k = min(divs, key=lambda d: abs(np.log(d / w)))
        if k not in pick:
            pick.append(k)
    return sorted(pick)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        return run_reference(args, rank, world)

    import torch
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("gloo")
    torch.cuda.set_device(local)
    from paper_2308_13092_gb300 import ecpic
    ecpic.lib(build_if_missing=True)
    stream = torch.cuda.Stream()

    ks = sort_cadences(args.steps)
    # every run outlives the autotuner's trials, the warm-up (with its
    # alignment to a sort boundary), the timed window and the plain-graph
    # check window, so none retires inside them
    total = (args.warmup + max(ks) + 2 * args.steps + autotune_steps(AUTOTUNE_STEPS, Ks=ks) + 256)
    cfgs = manifest(rank, args, total)
    eng = ecpic.Engine(device=local, stream=stream.cuda_stream, max_slots=len(cfgs),
                       max_cells=1024)
    tickets = [eng.submit(c) for c in cfgs]
    eng.pump(0)  # admit and load everything
    # sort cadence and pass grid from the autotuner (its trials are steps of
    # the same runs, before the warm-up)
    if args.no_autotune:
        K = ks[0] if 16 not in ks else 16
        tuned = {"sort_every": K, "pass_ctas": 0}
        eng.tune(0, K)
    else:
        tuned = eng.autotune(AUTOTUNE_STEPS, ks=ks)
    K = tuned["sort_every"]
    # phase timing on before the warm-up, so that its graphs are built there
    eng.set_phase_timing(True)
    eng.pump(args.warmup)
    since = eng.sort_state()["since_sort"]
    align = (K - since) % K
    if align:
        eng.pump(align)  # on to a sort boundary
    assert eng.sort_state()["since_sort"] == 0
    eng.phase_times()  # clear the warm-up's sums
    # energy-sample steps in the window (every run steps in lockstep from its
    # admission): the pass of level k samples when (k + 1) % SAMPLE_EVERY == 0
    k0 = eng.poll(tickets[0], diagnostics=True)["diag"]["step"]
    samples = sample_steps(k0, args.steps)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ps0 = eng.stats()["particle_steps"]
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    ev0.record(stream)
    eng.pump(args.steps)
    ev1.record(stream)
    ev1.synchronize()
    torch.cuda.synchronize()
    ck = clocks.stop()
    ms = ev0.elapsed_time(ev1)
    ps = eng.stats()["particle_steps"] - ps0
    ph = eng.phase_times()  # the window's own replays
    sorts = ph["sorts"]
    assert ph["steps"] == args.steps, ph
    assert sorts == args.steps // K and args.steps % K == 0, (sorts, args.steps, K)
    # the same window length with the plain graphs (no phase events), as a
    # check that the events do not slow the steps
    eng.set_phase_timing(False)
    eng.pump(K)  # rebuild the plain graphs outside the check window
    assert eng.sort_state()["since_sort"] == 0
    ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ps2 = eng.stats()["particle_steps"]
    ev2.record(stream)
    eng.pump(args.steps)
    ev3.record(stream)
    ev3.synchronize()
    ms_plain = ev2.elapsed_time(ev3)
    ps_plain = eng.stats()["particle_steps"] - ps2
    retired = eng.stats()["runs_finished"]  # 0: every run stepped through both windows
    eng.close()

    if world > 1:
        ms, ps = combine_ranks(ms, ps)

    value = ps / (ms * 1e-3)
    hbm, peak_kind = peaks()
    nst = max(1, ph["launches"][0])
    pass_ms = ph["pass_ms"] / nst
    field_ms = ph["field_ms"] / max(1, ph["launches"][1])
    collide_ms = ph["collide_ms"] / max(1, ph["launches"][3])
    sort_ms_step = ph["sort_ms"] / max(1, ph["steps"])
    phase_sum = pass_ms + field_ms + collide_ms + sort_ms_step
    bytes_per_launch = BYTES_PER_PARTICLE_STEP * ps / max(1, args.steps) / world
    achieved = bytes_per_launch / (pass_ms * 1e-3) / 1e9
    traffic = None
    if kernel_sources_sha256() == TRAFFIC["sources_sha256"]:
        traffic = TRAFFIC["dram_bytes_per_particle_step"] * ps / max(1, args.steps) / world

    extras = {}
    if rank == 0 and not args.no_extras:
        extras["single_run"] = single_run_block(torch, ecpic, stream, local)
        # 200-step jobs: configs sized for 200 steps
        short = manifest(rank, args, 200)
        extras["one_by_one"] = one_by_one_block(ecpic, short, stream, local)
        extras["served"] = served_block(ecpic, stream, local, capacity=value / max(1, world))
        extras["served_load_0.9"] = served_block(ecpic, stream, local,
                                                 capacity=value / max(1, world), rho=0.9)
        # the same stream with a quarter of the slots: the queue builds and
        # the smaller resident population steps less efficiently
        extras["served_load_0.9_slots64"] = served_block(ecpic, stream, local,
                                                         capacity=value / max(1, world), rho=0.9,
                                                         slots=64, n_alone=0)
        extras["appendix_b"] = appendix_b_block(ecpic, stream, local)
        # whole jobs of 5 RF periods (2000 steps), the shortest request length
        # of the served stream
        e2e = e2e_block(ecpic, manifest(rank, args, E2E_STEPS), stream, local, steps=E2E_STEPS)
    else:
        e2e = None
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        cpu = cpu_baseline_block(cfgs)

    if rank == 0:
        n_part = sum(c.n_particles for c in cfgs)
        line = {
            "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"batched: {len(cfgs)} independent 1D3V EC-PIC RF-CCP runs "
                                   f"(seeded manifest), {n_part} initial particles, cells "
                                   f"{min(c.N for c in cfgs)}-{max(c.N for c in cfgs)}",
                       "runs_per_gpu": len(cfgs),
                       "l2": f"inputs larger than L2 ({28e-9 * ps / max(1, args.steps) / world:.1f} GB "
                             f"of particle records live per GPU and step, 28 B each)",
                       "sort_every": K, "sort_cadences_tried": ks,
                       "sorts_in_window": sorts,
                       "sample_steps_in_window": samples,
                       "warmup_steps_run": args.warmup + align,
                       "pass_ctas": tuned["pass_ctas"] or "auto",
                       "tuning": "defaults" if args.no_autotune else
                                 "autotuner (sort cadence x pass grid) before the warm-up",
                       "sample_every": 40, "scheme": "EC",
                       "arithmetic": "FP32 particles, FP64 field solve",
                       "runs_retired_before_window_end": retired},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": traffic, "kernel": "k_pass",
                         "traffic_unit": "bytes per launch (DRAM read + write)",
                         "peak_kind": f"{peak_kind} (MEASURED_PEAKS.json hbm_gbs)",
                         "bytes_per_particle_step": BYTES_PER_PARTICLE_STEP,
                         "timing": "CUDA events recorded by the timed window's own graph "
                                   "replays after every kernel phase",
                         "pass_ms_avg": pass_ms, "field_ms_avg": field_ms,
                         "field_us_per_run": 1e3 * field_ms / len(cfgs),
                         "collide_ms_avg": collide_ms, "sort_ms_per_step": sort_ms_step,
                         "phase_sum_ms_per_step": phase_sum,
                         "phase_sum_over_step": phase_sum / (ms / args.steps),
                         "pass_share": pass_ms / phase_sum},
            "plain_graph_check": {"ms_per_step": ms_plain / args.steps,
                                  "value": ps_plain / (ms_plain * 1e-3),
                                  "what": "the next window of the same length replayed from "
                                          "the step graphs without phase events"},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(sum(ph["launches"])),
            "clocks": ck,
        }
        line.update(extras)
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
