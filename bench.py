"""Throughput benchmark of the GB300 EC-PIC hot path (particle-steps/s).

python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                [--workload resolved]

A "step" is one time step of the whole hot path (gather, push, walls, MCC,
deposit, field; the counting sort every 16 steps) over every live particle of
the workload.  Inputs are synthetic and seeded (``paper_2308_13092_gb300.inputs``).

Workload "resolved": one 1D3V RF-CCP, 1024 uniform cells at dx = lambda_De,
256 particles/cell/species (524,288 particles), 300 V, 30 mTorr, w_pe dt = 0.2.
Its particle state (29 MB) fits in the 129 MB L2, so L2 is flushed (a 512 MB
write) before every timed step and each step is timed alone with CUDA events.

For N > 1 (torchrun) every rank steps an independent replica of the workload
(different seed); value = all ranks' particle-steps / max over ranks of the
time.  --impl reference times the FP64 CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2308_13092_gb300 import inputs as I  # noqa: E402

BYTES_PER_PARTICLE_STEP = 40  # 28 B read (cell, xi, vx, vy, vz, id) + 12 B written
METRIC = "particle-steps/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="resolved", choices=["resolved"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload_config(name, rank):
    if name == "resolved":
        return I.config_resolved(seed=1000 + rank)
    raise ValueError(name)


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


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
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_rate(cfg, budget_s=12.0, max_steps=10_000):
    """The FP64 C oracle, as it stands, on one host core: particle-steps/s over
    a bounded number of steps of the same workload."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from helpers import oracle_from_config
    o = oracle_from_config(cfg)
    t0 = time.perf_counter()
    ps = 0
    steps = 0
    while steps < max_steps:
        c = o.counters()
        live = sum(s["n"] for s in c["species"])
        o.step(1, allow_capacity=True)
        ps += live
        steps += 1
        if time.perf_counter() - t0 > budget_s:
            break
    dt = time.perf_counter() - t0
    return ps / dt, steps, ps


def run_reference(args, rank, world):
    if rank != 0:
        return
    cfg = workload_config(args.workload, 0)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from helpers import oracle_from_config
    o = oracle_from_config(cfg)
    for _ in range(args.warmup):
        o.step(1, allow_capacity=True)
    t0 = time.perf_counter()
    ps = 0
    for _ in range(args.steps):
        ps += sum(s["n"] for s in o.counters()["species"])
        o.step(1, allow_capacity=True)
    dt = time.perf_counter() - t0
    v = ps / dt
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "particle-steps/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": dt * 1e3 / max(1, args.steps), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": f"{args.workload}: {cfg.name}, {cfg.N} cells, "
                                   f"{cfg.n_particles} particles, FP64 CPU oracle"},
            "cpu_baseline": {"value": v, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} steps of the full workload after "
                                       f"{args.warmup} warm-up steps"},
            "e2e": {"value": v, "unit": "particle-steps/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


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

    cfg = workload_config(args.workload, rank)
    cfg.sample_every = 20
    stream = torch.cuda.Stream()
    run = ecpic.Run.from_config(cfg, device=local, stream=stream.cuda_stream)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")

    def live():
        return sum(s["n"] for s in run.diagnostics(profiles=False)["species"])

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            run.step(1)
        stream.synchronize()
        run.sync()

        # ---- timed region: each step alone, L2 flushed before it
        n0 = live()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
               for _ in range(args.steps)]
        counts = []
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
        clocks = Clocks(local)
        for k in range(args.steps):
            flush.zero_()
            evs[k][0].record(stream)
            run.step(1)
            evs[k][1].record(stream)
        stream.synchronize()
        torch.cuda.synchronize()
        ck = clocks.stop()
        run.sync()
        n1 = live()
        step_ms = [a.elapsed_time(b) for a, b in evs]
        total_ms = float(sum(step_ms))
        # live particles at the start of each step: interpolate the start/end
        # counts (they change by < 1% over the window)
        particle_steps = 0.5 * (n0 + n1) * args.steps

        # ---- per-kernel device time on the same stream, same workload
        prof = {"pass_ms": 0.0, "field_ms": 0.0, "sort_ms": 0.0, "launches": [0, 0, 0]}
        nprof = min(args.steps, 100)
        live_prof = 0
        for _ in range(nprof):
            flush.zero_()
            live_prof += live()
            p = run.profile_step(1)
            for k in ("pass_ms", "field_ms", "sort_ms"):
                prof[k] += p[k]
            prof["launches"] = [a + b for a, b in zip(prof["launches"], p["launches"])]

    if world > 1:
        import torch.distributed as dist
        t = torch.tensor([total_ms], dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
        ps = torch.tensor([particle_steps], dtype=torch.float64)
        dist.all_reduce(ps, op=dist.ReduceOp.SUM)
        particle_steps = float(ps.item())

    value = particle_steps / (total_ms * 1e-3)
    hbm, peak_kind = peaks()
    pass_avg_ms = prof["pass_ms"] / max(1, prof["launches"][0])
    per_launch_bytes = BYTES_PER_PARTICLE_STEP * live_prof / max(1, nprof)
    achieved = per_launch_bytes / (pass_avg_ms * 1e-3) / 1e9
    kernels_per_step = (prof["launches"][0] + prof["launches"][1] + prof["launches"][2]) / max(1, nprof)

    # ---- end to end through the C ABI with host buffers (pinned)
    e2e = None
    if rank == 0:
        e2e = end_to_end(cfg, local, stream, n_steps=min(args.steps, 100))

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        v, st, ps = oracle_rate(cfg)
        cpu = {"value": v, "unit": "particle-steps/s", "cores": 1, "kind": "oracle",
               "sample": f"{st} steps ({ps:.3g} particle-steps) of the same workload on one "
                         f"host core, FP64"}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "particle-steps/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": f"{args.workload}: {cfg.name}, {cfg.N} uniform cells, "
                                   f"{cfg.n_particles} particles (2 species), EC, 300 V, 30 mTorr",
                       "runs": world, "l2": "flushed (512 MB write) before every timed step",
                       "sort_every": 16, "sample_every": cfg.sample_every},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                         "frac": achieved / hbm, "traffic": None,
                         "kernel": "k_pass", "peak_kind": peak_kind,
                         "bytes_per_particle_step": BYTES_PER_PARTICLE_STEP,
                         "pass_ms_avg": pass_avg_ms,
                         "field_ms_avg": prof["field_ms"] / max(1, prof["launches"][1]),
                         "sort_ms_per_step": prof["sort_ms"] / max(1, nprof)},
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": int(round(kernels_per_step * args.steps)),
            "clocks": ck,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def end_to_end(cfg, device, stream, n_steps):
    """Particle-steps/s through the public API: the initial state is uploaded
    from pinned host buffers, then every step is ecpic_step(1) followed by a
    device-to-host read of the run's diagnostics (ecpic_diagnostics)."""
    import torch
    from paper_2308_13092_gb300 import ecpic
    run = ecpic.Run.from_config(cfg, device=device, stream=stream.cuda_stream)
    host = []
    for s in range(len(cfg.species)):
        p = run.get_particles(s)
        pinned = {}
        for k, a in p.items():
            t = torch.empty(a.size, dtype={np.int32: torch.int32, np.float32: torch.float32,
                                           np.uint64: torch.int64}[a.dtype.type], pin_memory=True)
            t.numpy()[:] = a.view(t.numpy().dtype)
            pinned[k] = t.numpy().view(a.dtype)
        host.append(pinned)
    h2d = sum(a.nbytes for p in host for a in p.values())
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for s, p in enumerate(host):
        run.set_particles(s, p["cell"], p["xi"], p["vx"], p["vy"], p["vz"], p["id"])
    ps = 0
    d2h = 0
    for _ in range(n_steps):
        run.step(1)
        d = run.diagnostics(profiles=False)
        ps += sum(s["n"] for s in d["species"])
        d2h += 1024
    dt = time.perf_counter() - t0
    run.close()
    return {"value": ps / dt, "unit": "particle-steps/s",
            "h2d_bytes_per_step": int(h2d / n_steps), "d2h_bytes_per_step": 1024,
            "what": "set_particles from pinned host buffers, then per step ecpic_step(1) + "
                    "ecpic_diagnostics (synchronising D2H read)"}


if __name__ == "__main__":
    main()
