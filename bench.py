"""Benchmark: walker-steps/s and % of HBM roofline for node2vec walks on an
R-MAT scale-22 graph on one GB300.

Workload (one bench step = three walks, one per (p, q)):
  graph    undirected R-MAT s22, edge factor 16, (a,b,c) = (.57,.19,.19),
           symmetrised, duplicates and self-loops removed, sorted int32 CSR,
           h ~ U(0,1] FP32 (generator seed 1, weight seed 2)
  walkers  one per node (W = 4,194,304), length 80, seed 42, cost-model mode
  (p, q)   (1, 1), (4, 0.25), (0.25, 4)

`value` is walker-steps (hops actually taken) per second with the graph and
the start array resident in HBM; `e2e` is the same metric through
fw_walk_host with pinned host buffers (start upload and row download inside
the timed region).  `roofline` relates the algorithmic bytes of the walk
kernel (byte model counted by the kernel's counting build) to its CUDA-event
time and the measured HBM copy bandwidth.  `cpu_baseline` is the CPU oracle
timed on a bounded sample of the same workload on the host cores.

Run: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
For N > 1 launch with torchrun; every rank walks its own replica of the
workload with its own random streams (weak scaling, no data-path collective).
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np

PQ = [(1.0, 1.0), (4.0, 0.25), (0.25, 4.0)]
LENGTH = 80
SEED = 42
WORKLOAD = ("node2vec on undirected R-MAT s22 ef16 (a=.57,b=c=.19), 4,194,304 nodes, h~U(0,1] FP32, "
            "one walker per node, length 80, (p,q) in {(1,1),(4,.25),(.25,4)}, cost-model mode")
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "walk_kernel_s22_node2vec.md")


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0, help="target CPU work of the oracle sample")
    ap.add_argument("--scale", type=int, default=22, help="R-MAT scale (22 = the benchmark workload; smaller "
                    "scales are for profiling captures)")
    ap.add_argument("--pq", action="append", default=None, help="restrict to one (p,q), e.g. --pq 4,0.25")
    ap.add_argument("--no-e2e", action="store_true")
    a = ap.parse_args()
    global PQ
    if a.pq:
        PQ = [tuple(float(x) for x in s.split(",")) for s in a.pq]
    return a


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def source_digest():
    from paper_2512_00705_gb300 import _build
    return _build._inputs_digest()[:16]


def read_traffic():
    """ncu DRAM bytes per hop recorded for the current kernel source, else None."""
    try:
        txt = open(TRAFFIC_FILE).read()
    except OSError:
        return None
    vals = {}
    for line in txt.splitlines():
        line = line.strip().strip("`")
        if ":" in line:
            k, v = line.split(":", 1)
            vals[k.strip().lstrip("- ")] = v.strip()
    try:
        if vals.get("source_digest") != source_digest():
            return None
        return {pq: float(vals[f"dram_bytes_per_hop_p{pq[0]:g}_q{pq[1]:g}"]) for pq in PQ}
    except (KeyError, ValueError):
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ["clocks.sm", "clocks.max.sm", "power.draw", "clocks_event_reasons.hw_slowdown",
              "clocks_event_reasons.hw_thermal_slowdown", "clocks_event_reasons.sw_thermal_slowdown",
              "clocks_event_reasons.sw_power_cap"]

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + ",".join(self.FIELDS),
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) != len(self.FIELDS):
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[3:]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def oracle_sample(g, cpu_seconds, threads):
    """Time the CPU oracle on a seeded sample of the workload's walkers."""
    import oracle
    rng = np.random.default_rng(7)
    nonzero = np.nonzero(np.diff(g.offsets) > 0)[0]
    # calibrate on a small sample, then size the timed sample to ~cpu_seconds
    cal = rng.choice(nonzero, 64, replace=False).astype(np.int32)
    t0 = time.perf_counter()
    hops = 0
    for (p, q) in PQ:
        _, h = oracle.walk(g, cal, LENGTH, "node2vec", p, q, seed=SEED, threads=threads)
        hops += h
    dt = max(time.perf_counter() - t0, 1e-3)
    per_walker = dt / (64 * len(PQ))
    nw = int(max(64, min(len(nonzero), cpu_seconds / per_walker / len(PQ))))
    starts = rng.choice(nonzero, nw, replace=False).astype(np.int32)
    t0 = time.perf_counter()
    hops = 0
    for (p, q) in PQ:
        _, h = oracle.walk(g, starts, LENGTH, "node2vec", p, q, seed=SEED, threads=threads)
        hops += h
    dt = time.perf_counter() - t0
    return hops / dt, nw, hops, dt


def run_reference(args):
    """The reference arm: the CPU oracle (exact inverse-CDF walks) timed on the
    host cores, each bench step a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2512_00705_gb300 import synth
    import oracle
    oracle.build()
    g = synth.workload_graph("s22")
    threads = os.cpu_count() or 1
    per_step = max(2.0, min(20.0, 60.0 / max(1, args.steps + args.warmup)))
    rates = []
    for i in range(args.warmup + args.steps):
        rate, nw, hops, dt = oracle_sample(g, per_step, threads)
        if i >= args.warmup:
            rates.append((rate, nw, hops, dt))
    value = sum(r[2] for r in rates) / sum(r[3] for r in rates)
    nw = rates[-1][1]
    line = {"metric": "walker-steps/sec", "value": value, "unit": "walker-steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000.0 * sum(r[3] for r in rates) / len(rates), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "sample": f"{nw} seeded non-isolated walkers x 80 hops x 3 (p,q) per step"},
            "cpu_baseline": {"value": value, "unit": "walker-steps/s", "cores": threads, "kind": "oracle",
                             "sample": f"{nw} seeded walkers x 80 hops x 3 (p,q)"},
            "e2e": {"value": value, "unit": "walker-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    from paper_2512_00705_gb300 import _build, synth
    from paper_2512_00705_gb300 import flexiwalk as fw
    _build.build()

    if args.scale == 22:
        g = synth.workload_graph("s22")
    else:
        g = synth.rmat(args.scale, 16, 0.57, 0.19, 0.19, seed=1)
        g.h = synth.edge_weights(g, "uniform01", seed=2)
    G = fw.Graph(g)
    n = g.n
    stream = torch.cuda.current_stream()
    starts = torch.arange(n, dtype=torch.int32, device=dev)
    out = torch.empty((n, LENGTH + 1), dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    base = rank * n  # each rank's replica uses its own random streams

    def walk(p, q, flags=0):
        G.walk(starts, LENGTH, "node2vec", p=p, q=q, mode="auto", seed=SEED, flags=flags, walker_base=base, out=out)

    # counted run: hops and algorithmic bytes per launch (untimed)
    counts = {}
    for (p, q) in PQ:
        G.reset_counters()
        walk(p, q, fw.FLAG_COUNTERS)
        counts[(p, q)] = G.counters()
    hops_per_step = sum(c["hops"] for c in counts.values())
    bytes_per_step = sum(c["bytes"] for c in counts.values())

    for _ in range(args.warmup):
        for (p, q) in PQ:
            walk(p, q)
    torch.cuda.synchronize()

    sampler = ClockSampler(local)
    sampler.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = fw.fw_launch_count()
    per_launch = {pq: [] for pq in PQ}
    step_ms = []
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)  # evict L2 between steps (256 MiB > 129 MB L2), outside the timed events
        evs = []
        for (p, q) in PQ:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            walk(p, q)
            e1.record(stream)
            evs.append(((p, q), e0, e1))
        torch.cuda.synchronize()
        tot = 0.0
        for pq, e0, e1 in evs:
            t = e0.elapsed_time(e1)
            per_launch[pq].append(t)
            tot += t
        step_ms.append(tot)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    wall = time.perf_counter() - wall0
    launches = fw.fw_launch_count() - launches0
    clocks = sampler.stop()
    G.check()

    ms_per_step = sum(step_ms) / len(step_ms)
    if world > 1:
        t = torch.tensor([ms_per_step], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms_per_step = float(t.item())
    value = world * hops_per_step / (ms_per_step / 1000.0)

    # ---- e2e through the host-buffer entry point (pinned buffers)
    e2e_line = None
    if not args.no_e2e:
        starts_h = torch.arange(n, dtype=torch.int32).pin_memory()
        out_h = torch.empty((n, LENGTH + 1), dtype=torch.int32).pin_memory()
        e2e_ms = []
        for i in range(2 + max(2, args.steps // 2)):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for (p, q) in PQ:
                G.walk_host(starts_h, LENGTH, "node2vec", p=p, q=q, mode="auto", seed=SEED, walker_base=base,
                            out=out_h)
            dt = (time.perf_counter() - t0) * 1000.0
            if i >= 2:
                e2e_ms.append(dt)
        e2e_step = statistics.median(e2e_ms)
        # sanity: host rows equal device rows for the last (p, q)
        walk(*PQ[-1])
        torch.cuda.synchronize()
        assert torch.equal(out.cpu(), out_h), "host-buffer walk differs from device walk"
        e2e_line = {"value": world * hops_per_step / (e2e_step / 1000.0), "unit": "walker-steps/s",
                    "h2d_bytes_per_step": len(PQ) * n * 4, "d2h_bytes_per_step": len(PQ) * n * (LENGTH + 1) * 4}

    # ---- roofline of the walk kernel
    peak, peak_kind = measured_peaks()
    kern_ms = sum(sum(v) for v in per_launch.values()) / args.steps
    achieved = bytes_per_step / (kern_ms / 1000.0) / 1e9
    traffic = read_traffic() if args.scale == 22 else None
    traffic_per_launch = None
    if traffic is not None:
        traffic_per_launch = sum(traffic[pq] * counts[pq]["hops"] for pq in PQ) / len(PQ)

    line = {
        "metric": "walker-steps/sec", "value": value, "unit": "walker-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD if args.scale == 22 and len(PQ) == 3 else
                   f"node2vec R-MAT s{args.scale} ef16 (profiling case), (p,q)={PQ}", "walkers": n, "walk_length": LENGTH, "edges": g.e,
                   "hops_per_step": hops_per_step, "l2": "256 MiB write between steps; graph and rows > L2",
                   "per_pq_ms": {f"p{p:g}_q{q:g}": statistics.median(per_launch[(p, q)]) for (p, q) in PQ},
                   "per_pq_hops": {f"p{p:g}_q{q:g}": counts[(p, q)]["hops"] for (p, q) in PQ},
                   "wall_s": wall},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic_per_launch,
                     "peak_kind": peak_kind, "kernel": "walk_kernel<1,false>",
                     "algorithmic_bytes_per_launch": bytes_per_step / len(PQ),
                     "avg_launch_ms": kern_ms / len(PQ)},
        "e2e": e2e_line,
        "gpu_launches": launches,
        "clocks": clocks,
        "counters": {f"p{p:g}_q{q:g}": counts[(p, q)] for (p, q) in PQ},
    }
    if rank == 0 and not args.no_cpu_baseline and args.scale == 22:
        import oracle
        oracle.build()
        threads = os.cpu_count() or 1
        rate, nw, hops, dt = oracle_sample(g, args.cpu_seconds, threads)
        line["cpu_baseline"] = {"value": rate, "unit": "walker-steps/s", "cores": threads, "kind": "oracle",
                                "sample": f"{nw} seeded non-isolated walkers x 80 hops x 3 (p,q), {dt:.1f} s"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    G.close()
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
