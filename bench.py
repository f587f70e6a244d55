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
import ctypes
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
TRAFFIC_FILE = os.path.join(ROOT, "profiles", "walk_kernel_s20_node2vec_traffic.md")
SUBSET = 65536  # the fixed seeded walker subset the CPU oracle is timed on


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
    ap.add_argument("--no-extras", action="store_true", help="walk suite: leave out the batched, served and "
                    "metapath measurements that the default line carries (N = 1 only)")
    ap.add_argument("--suite", default="walk", choices=["walk", "batch", "serve", "metapath", "skew", "ablation"],
                    help="walk: the headline node2vec s22 line; batch: 64 mixed jobs on skewed R-MAT s24, "
                    "batched vs one launch per job; serve: Poisson query stream on s22, continuous batching vs "
                    "serial calls; metapath: metapath walks on R-MAT s23; skew: Pareto / degree-based weights on "
                    "s22, cost model vs eRJS-only / eRVS-only / random / degree-rule selection; ablation: the "
                    "headline s22 walk for node2vec (weighted and unweighted), weighted and second-order PageRank, "
                    "cost model vs eRJS-only / eRVS-only")
    ap.add_argument("--cost-ratio", type=float, default=None, help="walk suite: use this r of Eq. (runtime) for "
                    "every (p,q) instead of tuning it (profiling captures)")
    ap.add_argument("--mode", default="auto", choices=["auto", "rjs", "rvs", "exact"],
                    help="walk suite: sampler mode (auto = the cost model; the others force one sampler, for "
                    "profiling captures)")
    ap.add_argument("--int8", action="store_true", help="walk suite: store the weights as 8-bit codes "
                    "(fw_graph_quantize_weights) before tuning and timing")
    ap.add_argument("--duration", type=float, default=10.0, help="serve suite: seconds of offered load")
    ap.add_argument("--rate", type=float, default=2000.0, help="serve suite: mean arrivals per second")
    ap.add_argument("--max-waves", type=int, default=8, help="serve suite: concurrent waves (streams) of the server")
    ap.add_argument("--large-query-steps", type=int, default=0,
                    help="serve suite: the server's size-class threshold on W x L (0: one class, arrival order)")
    ap.add_argument("--no-serial", action="store_true", help="serve suite: skip the serial comparison (for "
                    "arrival rates far above what serial calls sustain, e.g. capacity runs)")
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
    """Digest of the walk kernel's sources (profiles of the kernel are keyed to it)."""
    from paper_2512_00705_gb300 import _build
    return _build.walk_kernel_digest()[:16]


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


def cpu_info():
    """CPU model and logical CPU count of this host."""
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.split(":")[0].strip() == "Model name":
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for line in open("/proc/cpuinfo"):
                if line.lower().startswith(("model name", "cpu part")):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return {"model": model or "unknown", "nproc": os.cpu_count() or 1}


def subset_starts(g):
    """The fixed seeded subset of SUBSET non-isolated s22 walkers (numpy PCG64
    seed 7 permutation of the nodes with neighbours, first SUBSET)."""
    rng = np.random.default_rng(7)
    return rng.permutation(np.nonzero(np.diff(g.offsets) > 0)[0]).astype(np.int32)[:SUBSET]


def oracle_sample(g, cpu_seconds, threads):
    """Time the CPU oracle (exact inverse-CDF walks, 80 hops, the three (p, q))
    on the first nw walkers of the fixed subset, nw grown (at most SUBSET)
    until one timed pass takes about `cpu_seconds`.  Returns (walker-steps/s,
    nw, hops, seconds)."""
    import oracle
    sub = subset_starts(g)
    nw = 64
    while True:
        starts = sub[:nw]
        t0 = time.perf_counter()
        hops = 0
        for (p, q) in PQ:
            _, h = oracle.walk(g, starts, LENGTH, "node2vec", p, q, seed=SEED, threads=threads)
            hops += h
        dt = time.perf_counter() - t0
        if dt >= 0.6 * cpu_seconds or nw >= len(sub):
            return hops / dt, nw, hops, dt
        nw = int(min(len(sub), nw * max(2.0, 1.2 * cpu_seconds / max(dt, 1e-3))))


def cpu_baseline(g, cpu_seconds):
    """The oracle on all host cores and on one core, each on a prefix of the
    fixed subset sized to about `cpu_seconds` (one core: half of that)."""
    threads = os.cpu_count() or 1
    rate, nw, hops, dt = oracle_sample(g, cpu_seconds, threads)
    rate1, nw1, hops1, dt1 = oracle_sample(g, 0.5 * cpu_seconds, 1)
    info = cpu_info()
    return {"value": rate, "unit": "walker-steps/s", "cores": threads, "kind": "oracle",
            "sample": f"walkers 0..{nw - 1} of the fixed seeded {SUBSET}-walker s22 subset (non-isolated nodes, "
                      f"permutation seed 7) x 80 hops x 3 (p,q): {hops} hops in {dt:.1f} s",
            "single_core": {"value": rate1, "unit": "walker-steps/s", "cores": 1,
                            "sample": f"walkers 0..{nw1 - 1} of the same subset: {hops1} hops in {dt1:.1f} s"},
            "cpu_model": info["model"], "nproc": info["nproc"]}


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
            "config": {"workload": WORKLOAD, "sample": f"walkers 0..{nw - 1} of the fixed seeded {SUBSET}-walker "
                                                      "s22 subset x 80 hops x 3 (p,q) per step"},
            "cpu_baseline": {"value": value, "unit": "walker-steps/s", "cores": threads, "kind": "oracle",
                             "sample": f"walkers 0..{nw - 1} of the fixed seeded {SUBSET}-walker s22 subset "
                                       "x 80 hops x 3 (p,q)", "cpu_model": cpu_info()["model"]},
            "e2e": {"value": value, "unit": "walker-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ====================================================================== suites
def _hops(rows):
    import torch
    return int((rows[:, 1:] >= 0).sum().item()) if isinstance(rows, torch.Tensor) else int((rows[:, 1:] >= 0).sum())


def _line(metric, value, unit, args, extra):
    line = {"metric": metric, "value": value, "unit": unit, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic"}
    line.update(extra)
    print(json.dumps(line), flush=True)


def batch_result(warmup, steps):
    """64 independent jobs on a skewed R-MAT s24 graph (a=.7, b=c=.1, edge
    factor 24): start sets log-uniform in [1K, 1M] walkers, lengths uniform
    in {5..80}, algorithms node2vec (p, q log-uniform in [0.25, 4]) /
    metapath (schema 0-1-2-3-4) / weighted, autotuned per algorithm; one
    batched launch (a replayed CUDA-graph plan) against one fw_walk launch
    per job on the same stream.  Returns the result as a dict."""
    import torch
    from paper_2512_00705_gb300 import _build, synth
    from paper_2512_00705_gb300 import flexiwalk as fw
    _build.build()
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    g = synth.workload_graph("s24_skew")
    gen_s = time.perf_counter() - t0
    G = fw.Graph(g)
    ratios = {a: G.autotune(a, p=1.0, q=1.0, schema=[0, 1, 2, 3, 4] if a == "metapath" else None, method=1)
              for a in ["node2vec", "metapath", "weighted"]}
    rng = np.random.default_rng(44)
    specs = []
    for j in range(64):
        algo = ["node2vec", "metapath", "weighted"][j % 3]
        w = int(np.exp(rng.uniform(np.log(1e3), np.log(1e6))))
        sp = dict(algo=algo, w=w, L=int(rng.integers(5, 81)), seed=1000 + j,
                  starts=torch.from_numpy(synth.random_starts(g.n, w, seed=500 + j)).cuda())
        if algo == "node2vec":
            sp["p"], sp["q"] = [float(np.exp(rng.uniform(np.log(0.25), np.log(4.0)))) for _ in range(2)]
        sp["out"] = torch.empty((w, sp["L"] + 1), dtype=torch.int32, device="cuda")
        specs.append(sp)

    def kw(sp):
        d = {"seed": sp["seed"]}
        if "p" in sp:
            d["p"], d["q"] = sp["p"], sp["q"]
        if sp["algo"] == "metapath":
            d["schema"] = [0, 1, 2, 3, 4]
        return d

    jobs = [fw.make_job(sp["starts"], sp["L"], sp["algo"], sp["out"], **kw(sp)) for sp in specs]
    plan = fw.BatchPlan(G, jobs)  # hand-set launch shape (defaults), r from the sweep

    def per_job():
        for sp in specs:
            G.walk(sp["starts"], sp["L"], sp["algo"], out=sp["out"], **kw(sp))

    def timed(fn):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        fn()
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1)

    for _ in range(warmup):
        per_job()
        plan.launch()
    torch.cuda.synchronize()
    per_ms, bat_ms = [], []
    for _ in range(steps):
        per_ms.append(timed(per_job))
        ref = [sp["out"].clone() for sp in specs]
        bat_ms.append(timed(plan.launch))
    same = all(torch.equal(r, sp["out"]) for r, sp in zip(ref, specs))
    hops = sum(_hops(sp["out"]) for sp in specs)
    per, bat = statistics.median(per_ms), statistics.median(bat_ms)
    plan.close()
    # the autotuner's launch shape (fw_autotune method 2) per algorithm, then the same batch again
    t_tune = time.perf_counter()
    tuned = {a: G.autotune(a, p=1.0, q=1.0, schema=[0, 1, 2, 3, 4] if a == "metapath" else None, method=2)
             for a in ["node2vec", "metapath", "weighted"]}
    tune_s = time.perf_counter() - t_tune
    info = G.info
    shapes = {a: {"r": tuned[a], "lane_max_degree": info["lane_max_degrees"][fw.ALGO[a]],
                  "rjs_batch": info["rjs_batches"][fw.ALGO[a]], "trial_budget": info["trial_budgets"][fw.ALGO[a]]}
              for a in tuned}
    jobs2 = [fw.make_job(sp["starts"], sp["L"], sp["algo"], sp["out"], **kw(sp)) for sp in specs]
    plan2 = fw.BatchPlan(G, jobs2)
    for _ in range(warmup):
        plan2.launch()
    torch.cuda.synchronize()
    tuned_ms = []
    for _ in range(steps):
        tuned_ms.append(timed(plan2.launch))
    same2 = all(torch.equal(r, sp["out"]) for r, sp in zip(ref, specs))
    plan2.close()
    tun = statistics.median(tuned_ms)
    res = {"value": hops / (min(bat, tun) / 1e3), "unit": "walker-steps/s", "ms_per_step": min(bat, tun),
           "hand_set_shape": {"value": hops / (bat / 1e3), "ms_per_step": bat,
                              "shape": {"lane_max_degree": 8, "rjs_batch": 2, "trial_budget": 1.0}},
           "autotuned_shape": {"value": hops / (tun / 1e3), "ms_per_step": tun, "per_algorithm": shapes,
                               "tuning_s": tune_s, "rows_identical": same2},
           "per_job": {"value": hops / (per / 1e3), "ms_per_step": per, "launches": 64},
           "batched_over_per_job": per / min(bat, tun), "autotuned_over_hand_set": bat / tun, "rows_identical": same,
           "config": {"workload": "64 jobs on skewed R-MAT s24 ef24 (a=.7,b=c=.1), W log-U[1K,1M], L U{5..80}, "
                                  "node2vec/metapath/weighted mixed; batched = one replayed CUDA-graph plan",
                      "nodes": g.n, "edges": g.e, "max_degree": int(G.info["max_degree"]),
                      "walkers": sum(sp["w"] for sp in specs), "hops_per_step": hops, "generation_s": gen_s,
                      "cost_ratios": ratios, "steps": steps, "warmup": warmup}}
    G.close()
    return res


def run_batch(args):
    r = batch_result(args.warmup, args.steps)
    _line("walker-steps/sec (batched)", r["value"], "walker-steps/s", args,
          {k: v for k, v in r.items() if k not in ("value", "unit")})


def metapath_result(warmup, steps):
    """Metapath walks (schema 0-1-2-3-4, cyclic) on R-MAT s23 ef16 with
    lognormal(0,1) weights and labels U{0..4}: 2M random starts, length 5
    and 40.  Returns the result as a dict."""
    import torch
    from paper_2512_00705_gb300 import _build, synth
    from paper_2512_00705_gb300 import flexiwalk as fw
    _build.build()
    torch.cuda.set_device(0)
    g = synth.workload_graph("s23_meta")
    G = fw.Graph(g)
    starts = torch.from_numpy(synth.random_starts(g.n, 2_000_000, seed=43)).cuda()
    r_meta = G.autotune("metapath", schema=[0, 1, 2, 3, 4], method=1)
    res = {}
    for L in (5, 40):
        out = torch.empty((starts.numel(), L + 1), dtype=torch.int32, device="cuda")
        for _ in range(warmup):
            G.walk(starts, L, "metapath", schema=[0, 1, 2, 3, 4], out=out, seed=SEED, cost_ratio=r_meta)
        ms = []
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            G.walk(starts, L, "metapath", schema=[0, 1, 2, 3, 4], out=out, seed=SEED, cost_ratio=r_meta)
            e1.record()
            torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        G.reset_counters()  # counted run (untimed): sampler shares and algorithmic bytes
        G.walk(starts, L, "metapath", schema=[0, 1, 2, 3, 4], out=out, seed=SEED, cost_ratio=r_meta,
               flags=fw.FLAG_COUNTERS)
        c = G.counters()
        res[L] = (_hops(out), statistics.median(ms), c)
    hops = sum(h for h, _, _ in res.values())
    tot = sum(t for _, t, _ in res.values())
    per_len = {}
    for L, (h, t, c) in res.items():
        per_len[str(L)] = {"hops": h, "ms": t, "walker_steps_per_s": h / (t / 1e3),
                           "rjs_share": c["rjs_steps"] / max(1, c["hops"]),
                           "rjs_trials_per_rjs_step": c["rjs_trials"] / max(1, c["rjs_steps"]),
                           "rvs_items_per_rvs_step": c["rvs_items"] / max(1, c["rvs_steps"]),
                           "dead_ends": c["dead_ends"], "algorithmic_bytes_per_hop": c["bytes"] / max(1, c["hops"]),
                           "algorithmic_GBps": c["bytes"] / (t / 1e3) / 1e9}
    G.close()
    return {"value": hops / (tot / 1e3), "unit": "walker-steps/s", "ms_per_step": tot,
            "config": {"workload": "metapath 0-1-2-3-4 on R-MAT s23 ef16, h~lognormal(0,1), labels U{0..4}, "
                                   "2M random starts (seed 43), L=5 and L=40", "nodes": g.n, "edges": g.e,
                       "cost_ratio": r_meta, "steps": steps, "warmup": warmup, "per_length": per_len}}


def run_metapath(args):
    r = metapath_result(args.warmup, args.steps)
    _line("walker-steps/sec (metapath)", r["value"], "walker-steps/s", args,
          {k: v for k, v in r.items() if k not in ("value", "unit")})


class _ServeClient:
    """Client side of the serving measurement: a Poisson stream of walk
    queries against the resident graph, W log-uniform in [1, 1e5] walkers,
    length uniform in {10..100}, algorithm uniform over node2vec (p=2,
    q=0.5) / metapath (0-1-2-3-4) / weighted; host buffers from pinned
    pools.  Latency = completion - arrival."""

    def __init__(self, G, g):
        import torch
        from paper_2512_00705_gb300 import synth
        self.G, self.g = G, g
        self.pool_words = 4 * 100_000 + 1
        self.starts_pool = torch.from_numpy(synth.random_starts(g.n, self.pool_words, seed=46)).pin_memory().numpy()
        # 16 GiB of pinned rows; a query takes the next range, reused once it completes (at 70 % of
        # capacity the ring turns over in about 0.2 s, so a slow query does not hold up later ones)
        self.ring_words = 1 << 32
        self.ring = torch.empty(self.ring_words, dtype=torch.int32, pin_memory=True).numpy()

    @staticmethod
    def queries(rate, duration, seed):
        rng = np.random.default_rng(seed)
        n = max(1, int(rate * duration))
        arrivals = np.cumsum(rng.exponential(1.0 / rate, n))
        W = np.exp(rng.uniform(0, np.log(1e5), n)).astype(np.int64)
        Ls = rng.integers(10, 101, n)
        algos = rng.integers(0, 3, n)
        return arrivals, W, Ls, algos

    def run(self, mode, rate, duration, seed=45, max_waves=8, count=None, large_query_steps=None):
        """Offer the query stream to the server (batched submit / poll calls,
        hops counted on the device) or to serial fw_walk_host calls."""
        from concurrent.futures import ThreadPoolExecutor
        from paper_2512_00705_gb300 import flexiwalk as fw
        arrivals, W, Ls, algos = self.queries(rate, duration, seed)
        count = len(arrivals) if count is None else min(count, len(arrivals))
        arrivals, W, Ls, algos = arrivals[:count], W[:count], Ls[:count], algos[:count]
        words = W * (Ls + 1)
        # rows go to a pinned ring, allocated in arrival order; query i may be
        # submitted once every earlier query whose range it reuses is done
        offs = np.zeros(count, dtype=np.int64)
        head = 0
        for i in range(count):
            if head + words[i] > self.ring_words:
                head = 0
            offs[i] = head
            head += words[i]
        ends = offs + words
        # the queries of the previous pass over the ring whose ranges overlap query i's
        # (within a pass offsets increase, so they form one index range [klo, khi))
        pass_start = np.nonzero(offs == 0)[0]
        klo = np.zeros(count, dtype=np.int64)
        khi = np.zeros(count, dtype=np.int64)
        for p_ in range(1, len(pass_start)):
            a0, a1 = pass_start[p_ - 1], pass_start[p_]
            b1 = pass_start[p_ + 1] if p_ + 1 < len(pass_start) else count
            idx = np.arange(a1, b1)
            klo[idx] = a0 + np.searchsorted(ends[a0:a1], offs[idx], side="right")
            khi[idx] = np.maximum(a0, a0 + np.searchsorted(offs[a0:a1], ends[idx], side="left"))
        # query i waits until every query below khi[i] is done: those overlapping it in the
        # previous pass and everything of the passes before (long finished in practice)
        names = ["node2vec", "metapath", "weighted"]

        def kw(i):
            d = {"seed": int(1000 + i)}
            if algos[i] == 0:
                d["p"], d["q"] = 2.0, 0.5
            if algos[i] == 1:
                d["schema"] = [0, 1, 2, 3, 4]
            return d

        starts_v = [self.starts_pool[(i * 7919) % (self.pool_words - W[i]):][:W[i]] for i in range(count)]
        outs_v = [self.ring[offs[i]:offs[i] + words[i]].reshape(W[i], Ls[i] + 1) for i in range(count)]
        lat = np.zeros(count)
        done = np.zeros(count, dtype=bool)

        prefix = [0]  # every query below prefix[0] is done

        def ring_free(i):
            while prefix[0] < count and done[prefix[0]]:
                prefix[0] += 1
            return prefix[0] >= khi[i]

        if mode == "server":
            jobs = (fw.fw_job * count)()
            for i in range(count):
                jobs[i] = fw.make_host_query(starts_v[i], int(Ls[i]), names[algos[i]], outs_v[i], **kw(i))
            srv = fw.Server(self.G, mem_budget=8 << 30, max_waves=max_waves, large_query_steps=large_query_steps)
            jsize = ctypes.sizeof(fw.fw_job)
            tickets = np.zeros(count, dtype=np.uint64)
            lag = np.zeros(count)
            nxt, ndone = 0, 0
            t_base = time.perf_counter()
            while ndone < count:
                now = time.perf_counter() - t_base
                hi = int(np.searchsorted(arrivals, now, side="right"))
                j = nxt
                while j < hi and ring_free(j):
                    j += 1
                if j > nxt:
                    sub = (fw.fw_job * (j - nxt)).from_address(ctypes.addressof(jobs) + nxt * jsize)
                    tickets[nxt:j] = srv.submit_many(sub)
                    lag[nxt:j] = (time.perf_counter() - t_base) - arrivals[nxt:j]
                    nxt = j
                pend = np.nonzero(~done[:nxt])[0]
                if len(pend):
                    d, l_ms, st = srv.poll_many(tickets[pend])
                    fin = pend[d.astype(bool)]
                    if np.any(st[d.astype(bool)] != 0):
                        raise RuntimeError("a served query failed")
                    done[fin] = True
                    lat[fin] = lag[fin] * 1e3 + l_ms[d.astype(bool)]
                    ndone += len(fin)
                if nxt < count and ndone < count and not len(pend):
                    time.sleep(max(0.0, min(0.0005, arrivals[nxt] - (time.perf_counter() - t_base))))
            wall = time.perf_counter() - t_base
            stats = srv.stats()
            srv.close()
            hops = int(stats["walker_steps"])
        else:
            counter = ThreadPoolExecutor(max_workers=8)

            def row_hops(rows):
                # -1 marks the steps after a dead end; the start column is never -1
                return rows.shape[0] * (rows.shape[1] - 1) - int(np.count_nonzero(rows[:, 1:] < 0))

            futs = []
            t_base = time.perf_counter()
            for i in range(count):
                while time.perf_counter() - t_base < arrivals[i]:
                    pass
                self.G.walk_host(starts_v[i], int(Ls[i]), names[algos[i]], out=outs_v[i], **kw(i))
                lat[i] = (time.perf_counter() - t_base - arrivals[i]) * 1e3
                done[i] = True
                futs.append(counter.submit(row_hops, outs_v[i]))
            wall = time.perf_counter() - t_base
            hops = sum(f.result() for f in futs)
            counter.shutdown()
            stats = None
        # offered load: the steps the queries actually took (a dead end ends a walker early) over the
        # arrival span; the nominal figure counts W x L per query
        span = max(float(arrivals[-1]), 1e-9)
        self.last = {"latency_ms": lat, "W": W, "L": Ls, "algo": algos, "arrival_s": arrivals}  # per query
        r = {"queries": count, "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
             "mean_ms": float(lat.mean()), "walker_steps_per_s": hops / wall, "wall_s": wall, "hops": hops,
             "arrival_span_s": span, "backlog_ms": (wall - span) * 1e3,
             "offered_walker_steps_per_s": hops / span,
             "offered_nominal_walker_steps_per_s": float((W * Ls).sum() / span)}
        if stats:
            r.update({"waves": stats["waves"], "queries_per_wave": stats["queries_per_wave"],
                      "peak_inflight_waves": stats["peak_inflight_waves"],
                      "submit_lag_p99_ms": float(np.percentile(lag, 99)) * 1e3,
                      "server_queue_p50_ms": stats["queue_p50_ms"], "server_queue_p99_ms": stats["queue_p99_ms"],
                      "server_wave_p50_ms": stats["wave_p50_ms"], "server_wave_p99_ms": stats["wave_p99_ms"],
                      "server_enqueue_ms_per_wave": stats["enqueue_ms_per_wave"],
                      "copies_per_query": stats["copies"] / max(1, count)})
        return r


def _device_rate(G, cl, rate, duration, seed, hops, nstreams=8, per_batch=64):
    """The queries of a served stream walked straight from device memory, in
    arrival order, as plain batches of `per_batch` (fw_walk_batch) spread
    round-robin over `nstreams` streams: no host copies, no server.  What the
    GPU does with this mix when nothing but the walks runs, batched the way
    the server's waves are.  Rows of each stream's batches share one device
    buffer (overwritten); `hops` is the walker-step count of the same queries
    (their rows are identical to the server's, so the served run's count)."""
    import torch
    from paper_2512_00705_gb300 import flexiwalk as fw
    arrivals, W, Ls, algos = cl.queries(rate, duration, seed)
    count = len(arrivals)
    names = ["node2vec", "metapath", "weighted"]
    pool = torch.from_numpy(np.ascontiguousarray(cl.starts_pool)).cuda()
    words = (W * (Ls + 1)).astype(np.int64)
    nb = (count + per_batch - 1) // per_batch
    most = int(max(words[b * per_batch:(b + 1) * per_batch].sum() for b in range(nb)))
    streams = [torch.cuda.Stream() for _ in range(nstreams)]
    bufs = [torch.empty(most, dtype=torch.int32, device="cuda") for _ in range(nstreams)]
    batches = []
    for b in range(nb):
        buf, pos, js = bufs[b % nstreams], 0, []
        for i in range(b * per_batch, min(count, (b + 1) * per_batch)):
            off = (i * 7919) % (cl.pool_words - W[i])
            out = buf[pos:pos + words[i]].view(int(W[i]), int(Ls[i]) + 1)
            pos += int(words[i])
            d = {"seed": int(1000 + i)}
            if algos[i] == 0:
                d["p"], d["q"] = 2.0, 0.5
            if algos[i] == 1:
                d["schema"] = [0, 1, 2, 3, 4]
            js.append(fw.make_job(pool[off:off + W[i]], int(Ls[i]), names[algos[i]], out, **d))
        batches.append(js)
    fw.fw_walk_batch(G.handle, batches[0], stream=streams[0])  # warm-up
    torch.cuda.synchronize()
    main = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(main)
    for st in streams:
        st.wait_event(e0)
    for b, js in enumerate(batches):
        fw.fw_walk_batch(G.handle, js, stream=streams[b % nstreams])
    for st in streams:
        main.wait_stream(st)
    e1.record(main)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    del bufs
    return {"walker_steps_per_s": hops / (ms / 1e3), "queries": count, "hops": hops, "ms": ms,
            "batches": nb, "streams": nstreams}


def serve_result(G, g, rate=2000.0, duration=10.0, max_waves=8, serial=True, capacity=True, large_query_steps=0):
    """Continuous batching (fw_server) against serial fw_walk_host calls on the
    same arrival sequence at `rate` queries/s for `duration` s; then the
    server's capacity (throughput when 60x the rate arrives for 1 s: the
    same 20x-rate query count, so the queue builds up and the server drains
    it at its own pace) and its p50 / p99 at 70 % and 50 % of that capacity
    (5 s each).  Returns a dict."""
    ratios = {"node2vec": G.autotune("node2vec", p=2.0, q=0.5, method=1),
              "metapath": G.autotune("metapath", schema=[0, 1, 2, 3, 4], method=1),
              "weighted": G.autotune("weighted", method=1)}
    cl = _ServeClient(G, g)
    lqs = large_query_steps
    cl.run("server", rate, duration, max_waves=max_waves, count=400, large_query_steps=lqs)  # warm-up, discarded
    out = {"server": cl.run("server", rate, duration, max_waves=max_waves, large_query_steps=lqs)}
    if serial:
        out["serial"] = cl.run("serial", rate, duration)
    res = {"value": out["server"]["walker_steps_per_s"], "unit": "walker-steps/s",
           "config": {"workload": f"Poisson {rate:g}/s for {duration:g} s (shortened from 60 s) on R-MAT s22; "
                                  "W log-U[1,1e5], L U{10..100}, node2vec(2,.5)/metapath/weighted",
                      "cost_ratios": ratios, "max_waves": max_waves, "large_query_steps": large_query_steps},
           "serving": out,
           "p99_server_over_serial": (out["server"]["p99_ms"] / out["serial"]["p99_ms"]) if serial else None,
           "steps_server_over_serial": (out["server"]["walker_steps_per_s"] / out["serial"]["walker_steps_per_s"])
           if serial else None}
    if capacity:
        sat = cl.run("server", 60.0 * rate, 1.0, seed=47, max_waves=max_waves, large_query_steps=lqs)
        cap = sat["walker_steps_per_s"]
        res["device_rate_same_queries"] = _device_rate(G, cl, 60.0 * rate, 1.0, 47, sat["hops"], max_waves)
        # queries per second at 70 % of capacity, from the steps a query of this mix actually takes
        rate70 = 0.7 * cap / (sat["hops"] / sat["queries"])
        at70 = cl.run("server", rate70, 5.0, seed=48, max_waves=max_waves, large_query_steps=lqs)
        at50 = cl.run("server", rate70 * 5.0 / 7.0, 5.0, seed=49, max_waves=max_waves, large_query_steps=lqs)
        res["capacity"] = {"walker_steps_per_s": cap, "saturated_run": sat,
                           "saturated": bool(sat["offered_walker_steps_per_s"] >= 1.5 * cap),
                           "over_device_rate": cap / res["device_rate_same_queries"]["walker_steps_per_s"],
                           "rate_at_70pct": rate70,
                           "at_70pct": at70,
                           "at_70pct_load": at70["offered_walker_steps_per_s"] / cap,
                           "at_50pct": at50,
                           "rate_saturates": bool(out["server"]["offered_walker_steps_per_s"] >= 0.95 * cap)}
    return res


def run_serve(args):
    import torch
    from paper_2512_00705_gb300 import _build, synth
    from paper_2512_00705_gb300 import flexiwalk as fw
    _build.build()
    torch.cuda.set_device(0)
    g = synth.workload_graph("s22")
    G = fw.Graph(g)
    r = serve_result(G, g, args.rate, args.duration, args.max_waves, serial=not args.no_serial,
                     large_query_steps=args.large_query_steps)
    G.close()
    _line("walker-steps/sec (served)", r["value"], "walker-steps/s", args,
          dict({k: v for k, v in r.items() if k not in ("value", "unit")}, ms_per_step=None))


def run_skew(args):
    """Weight skew (Sec. 5.2 power-law / degree-based weights, Sec. 5.3-5.4
    ablations): the s22 structure with classical Pareto weights (x_m = 1,
    shape alpha in {1, 1.5, 2, 3, 4}), degree-based weights h(v, u) = d(u),
    U(0,1] weights and no weights (h = 1); weighted node2vec p = 2, q = 0.5;
    2^18 random starts x 40 hops per run.  For each weight set: the cost
    model (profiled r, and the sweep's r) against eRJS-only, eRVS-only,
    random and degree-rule (< 1K -> eRVS) selection, with the share of steps
    the cost model gave eRJS; then the weights as 8-bit codes (Sec. 6.2
    extension), re-tuned, under the cost model."""
    import torch
    from paper_2512_00705_gb300 import _build, synth
    from paper_2512_00705_gb300 import flexiwalk as fw
    _build.build()
    torch.cuda.set_device(0)
    base = synth.rmat(22, 16, 0.57, 0.19, 0.19, seed=1)
    starts = torch.from_numpy(synth.random_starts(base.n, 1 << 18, seed=47)).cuda()
    L = 40
    out = torch.empty((starts.numel(), L + 1), dtype=torch.int32, device="cuda")
    sets = [(f"pareto{a:g}", synth.edge_weights(base, "pareto", a, seed=2)) for a in (1.0, 1.5, 2.0, 3.0, 4.0)]
    sets.append(("degree", synth.degree_weights(base)))
    sets.append(("uniform01", synth.edge_weights(base, "uniform01", seed=2)))
    sets.append(("unweighted", None))
    res = {}
    for name, h in sets:
        G = fw.Graph(synth.Csr(base.offsets, base.cols, h))
        r_sweep = G.autotune("node2vec", p=2.0, q=0.5, method=1)
        r = G.autotune("node2vec", p=2.0, q=0.5, method=0)
        row = {"cost_ratio_profiled": r, "cost_ratio_sweep": r_sweep}
        # method 2 (r and launch shape), tuned afresh `reps` times: the spread shows how stable it is
        shape_runs = []
        for _ in range(3 if name == "pareto1" else 1):
            r2 = G.autotune("node2vec", p=2.0, q=0.5, method=2)
            inf = G.info
            shape_runs.append({"r": r2, "lane_max_degree": inf["lane_max_degrees"][1],
                               "rjs_batch": inf["rjs_batches"][1], "trial_budget": inf["trial_budgets"][1]})
        row["shape_tuning"] = shape_runs
        for mode in ["auto", "auto_sweep"] + [f"auto_shape{k}" for k in range(len(shape_runs))] + \
                ["rjs", "rvs", "random", "degree"]:
            shp = {}
            if mode.startswith("auto_shape"):
                sr = shape_runs[int(mode[len("auto_shape"):])]
                rr = sr["r"]
                shp = {k: sr[k] for k in ("lane_max_degree", "rjs_batch", "trial_budget")}
            else:
                rr = r_sweep if mode == "auto_sweep" else r
                shp = {"lane_max_degree": 8, "rjs_batch": 2, "trial_budget": 1.0}
            md = "auto" if mode.startswith("auto") else mode
            def go(flags=0):
                G.walk(starts, L, "node2vec", p=2.0, q=0.5, mode=md, cost_ratio=rr, seed=SEED, flags=flags, out=out,
                       **shp)
            go()
            ms = []
            for _ in range(max(1, args.steps)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                go()
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            row[f"{mode}_ms"] = statistics.median(ms)
            if mode == "auto":
                G.reset_counters()
                go(fw.FLAG_COUNTERS)
                c = G.counters()
                row["hops"] = c["hops"]
                row["rjs_share"] = c["rjs_steps"] / max(1, c["hops"])
                row["rjs_trials_per_rjs_step"] = c["rjs_trials"] / max(1, c["rjs_steps"])
        if h is not None:
            # the same weights as 8-bit codes: re-tuned, cost model only
            row["int8_max_scale"] = G.quantize_weights()
            r8 = G.autotune("node2vec", p=2.0, q=0.5, method=1)
            row["cost_ratio_sweep_int8"] = r8
            for md in ("auto", "rvs"):  # eRVS-only: scans read 1-byte weights
                G.walk(starts, L, "node2vec", p=2.0, q=0.5, mode=md, cost_ratio=r8, seed=SEED, out=out)
                ms = []
                for _ in range(max(1, args.steps)):
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record()
                    G.walk(starts, L, "node2vec", p=2.0, q=0.5, mode=md, cost_ratio=r8, seed=SEED, out=out)
                    e1.record()
                    torch.cuda.synchronize()
                    ms.append(e0.elapsed_time(e1))
                row[f"{md}_int8_ms"] = statistics.median(ms)
            # weights below half a step of their row's scale are stored as code 1
            sv = G.weight_scales().cpu().numpy()[np.repeat(np.arange(base.n), np.diff(base.offsets))]
            row["int8_clamped_share"] = float(np.mean(h.astype(np.float64) < 0.5 * sv))
        row["auto_speedup_vs_best_single"] = min(row["rjs_ms"], row["rvs_ms"]) / row["auto_ms"]
        row["auto_sweep_speedup_vs_best_single"] = min(row["rjs_ms"], row["rvs_ms"]) / row["auto_sweep_ms"]
        row["auto_shape_speedup_vs_best_single"] = [min(row["rjs_ms"], row["rvs_ms"]) / row[f"auto_shape{k}_ms"]
                                                    for k in range(len(shape_runs))]
        row["auto_speedup_vs_random"] = row["random_ms"] / row["auto_ms"]
        row["auto_speedup_vs_degree_rule"] = row["degree_ms"] / row["auto_ms"]
        res[name] = row
        G.close()
    hops = sum(r_["hops"] for r_ in res.values())
    tot = sum(r_["auto_ms"] for r_ in res.values())
    _line("walker-steps/sec (skewed weights, cost model)", hops / (tot / 1e3), "walker-steps/s", args, {
        "ms_per_step": tot,
        "config": {"workload": "weighted node2vec p=2 q=0.5 on R-MAT s22 structure, Pareto(alpha), degree-based, "
                               "U(0,1] and no weights, 2^18 random starts x 40 hops"},
        "skew": res})


def run_ablation(args):
    """Sampler ablation at the headline size (Sec. 5.3): R-MAT s22 with
    h ~ U(0,1], one walker per node, 80 hops.  node2vec at the three (p, q)
    with the weights and with h = 1 (unweighted, Sec. 5.1), the weighted
    first-order walk, and second-order PageRank (Eq. 2ndpr, gamma = 0.2).
    Each case: the cost model with the sweep-tuned r against eRJS-only and
    eRVS-only (eRVS-only once timed: a single launch takes seconds)."""
    import torch
    from paper_2512_00705_gb300 import _build, synth
    from paper_2512_00705_gb300 import flexiwalk as fw
    _build.build()
    torch.cuda.set_device(0)
    g = synth.workload_graph("s22")
    G = fw.Graph(g)
    starts = torch.arange(g.n, dtype=torch.int32, device="cuda")
    out = torch.empty((g.n, LENGTH + 1), dtype=torch.int32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    U = fw.FLAG_UNWEIGHTED
    cases = [("node2vec", p, q, 0) for (p, q) in PQ] + [("node2vec", p, q, U) for (p, q) in PQ] + \
            [("weighted", 1.0, 1.0, 0), ("pagerank2", 1.0, 1.0, 0)]
    res = {}
    for algo, p, q, flags in cases:
        name = f"{algo}" + (f"_p{p:g}_q{q:g}" if algo == "node2vec" else "") + ("_unweighted" if flags else "")
        r = G.autotune(algo, p=p, q=q, flags=flags, method=1)
        row = {"cost_ratio": r}

        def go(mode):
            G.walk(starts, LENGTH, algo, p=p, q=q, mode=mode, cost_ratio=r, seed=SEED, flags=flags, out=out)

        for mode in ("auto", "rjs", "rvs"):
            go(mode)
            reps = 1 if mode == "rvs" else max(1, args.steps)
            ms = []
            for _ in range(reps):
                flush.fill_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                go(mode)
                e1.record()
                torch.cuda.synchronize()
                ms.append(e0.elapsed_time(e1))
            row[f"{mode}_ms"] = statistics.median(ms)
            if mode == "auto":
                G.reset_counters()
                G.walk(starts, LENGTH, algo, p=p, q=q, mode="auto", cost_ratio=r, seed=SEED,
                       flags=flags | fw.FLAG_COUNTERS, out=out)
                c = G.counters()
                row["hops"] = c["hops"]
                row["rjs_share"] = c["rjs_steps"] / max(1, c["hops"])
        row["walker_steps_per_s"] = row["hops"] / (row["auto_ms"] / 1e3)
        row["auto_vs_best_single"] = min(row["rjs_ms"], row["rvs_ms"]) / row["auto_ms"]
        res[name] = row
    G.close()
    hops = sum(r_["hops"] for r_ in res.values())
    tot = sum(r_["auto_ms"] for r_ in res.values())
    _line("walker-steps/sec (sampler ablation, s22)", hops / (tot / 1e3), "walker-steps/s", args, {
        "ms_per_step": tot,
        "config": {"workload": "R-MAT s22 ef16, h~U(0,1] or h=1, one walker per node, 80 hops: node2vec x3 (p,q) "
                               "weighted and unweighted, weighted walk, second-order PageRank gamma=0.2; cost model "
                               "(sweep r) vs eRJS-only vs eRVS-only",
                   "l2": "256 MiB write before every timed launch; graph and rows > L2"},
        "ablation": res})


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.suite == "batch":
        return run_batch(args)
    if args.suite == "metapath":
        return run_metapath(args)
    if args.suite == "serve":
        return run_serve(args)
    if args.suite == "skew":
        return run_skew(args)
    if args.suite == "ablation":
        return run_ablation(args)
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
    if args.int8:
        G.quantize_weights()
    n = g.n
    stream = torch.cuda.current_stream()
    from paper_2512_00705_gb300 import sharding
    if world == 1:
        starts = torch.arange(n, dtype=torch.int32, device=dev)
        wids = None
    else:
        # weak scaling: `world` replicas of the workload, spread over the GPUs by
        # a hash of the start node (Sec. 5.6); a query's global index is its stream id
        glob = np.tile(np.arange(n, dtype=np.int32), world)
        idx = sharding.shard(glob, rank, world)
        starts = torch.from_numpy(glob[idx]).to(dev)
        wids = torch.from_numpy(idx.astype(np.int32)).to(dev)
    nw = starts.numel()
    out = torch.empty((nw, LENGTH + 1), dtype=torch.int32, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)

    # tuning before sampling, reported and not timed: r of Eq. (runtime) per (p, q) from the
    # autotuner's sample-walk sweep; the Sec. 5.1 profiling kernels' r is reported beside it
    if args.cost_ratio is None:
        t_prof = time.perf_counter()
        ratio_profiled = {(p, q): G.autotune("node2vec", p=p, q=q, method=0) for (p, q) in PQ}
        profile_ms = (time.perf_counter() - t_prof) * 1e3
        t_prof = time.perf_counter()
        ratio = {(p, q): G.autotune("node2vec", p=p, q=q, method=1) for (p, q) in PQ}
        sweep_ms = (time.perf_counter() - t_prof) * 1e3
    else:
        ratio = {pq: args.cost_ratio for pq in PQ}
        ratio_profiled, profile_ms, sweep_ms = {pq: None for pq in PQ}, 0.0, 0.0

    def walk(p, q, flags=0):
        r = ratio[(p, q)]
        if wids is None:
            G.walk(starts, LENGTH, "node2vec", p=p, q=q, mode=args.mode, seed=SEED, flags=flags, cost_ratio=r, out=out)
        else:
            G.walk_ids(starts, wids, LENGTH, "node2vec", p=p, q=q, mode=args.mode, seed=SEED, flags=flags,
                       cost_ratio=r, out=out)

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

    ms_per_step = sharding.max_over_ranks(sum(step_ms) / len(step_ms))
    hops_all = hops_per_step
    if world > 1:
        t = torch.tensor([float(hops_per_step)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
        hops_all = int(t.item())
    value = hops_all / (ms_per_step / 1000.0)

    # ---- e2e through the host-buffer entry point (pinned buffers)
    e2e_line = None
    if not args.no_e2e and args.mode == "auto":
        starts_h = starts.cpu().pin_memory()
        out_h = torch.empty((nw, LENGTH + 1), dtype=torch.int32).pin_memory()
        e2e_ms = []
        for i in range(2 + max(4, args.steps)):  # 2 warm-up steps, then the median of the rest
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for (p, q) in PQ:
                G.walk_host(starts_h, LENGTH, "node2vec", p=p, q=q, mode="auto", seed=SEED, cost_ratio=ratio[(p, q)],
                            out=out_h)
            dt = (time.perf_counter() - t0) * 1000.0
            if i >= 2:
                e2e_ms.append(dt)
        e2e_step = statistics.median(e2e_ms)
        # sanity: host rows equal device rows for the last (p, q) (same random streams)
        p_, q_ = PQ[-1]
        G.walk(starts, LENGTH, "node2vec", p=p_, q=q_, mode="auto", seed=SEED, cost_ratio=ratio[(p_, q_)], out=out)
        torch.cuda.synchronize()
        assert torch.equal(out.cpu(), out_h), "host-buffer walk differs from device walk"
        e2e_ms_all = sharding.max_over_ranks(e2e_step)
        e2e_line = {"value": hops_all / (e2e_ms_all / 1000.0), "unit": "walker-steps/s",
                    "h2d_bytes_per_step": len(PQ) * nw * 4, "d2h_bytes_per_step": len(PQ) * nw * (LENGTH + 1) * 4,
                    "ms_per_step": e2e_step, "ms_per_step_min_max": [min(e2e_ms), max(e2e_ms)]}

    # ---- random-access ceiling of the device memory (the walk kernel's operative roof):
    # dependent 32-byte gathers over a 4 GiB table
    table = torch.empty(4 << 30, dtype=torch.uint8, device=dev)
    gather_ceiling = fw.fw_gather_ceiling(table)
    del table
    torch.cuda.empty_cache()

    # ---- roofline of the walk kernel
    peak, peak_kind = measured_peaks()
    kern_ms = sum(sum(v) for v in per_launch.values()) / args.steps
    achieved = bytes_per_step / (kern_ms / 1000.0) / 1e9
    # the survey's byte model of the method: 16 B per walker-step (offsets, bound scalar, row write), 64 B per
    # eRJS trial (a column sector and a weight sector), 32 B per membership probe, 8 B per eRVS item (col + h)
    survey_bytes = sum(16 * c["hops"] + 64 * c["rjs_trials"] + 32 * c["probes"] + 8 * c["rvs_items"]
                       for c in counts.values())
    achieved_survey = survey_bytes / (kern_ms / 1000.0) / 1e9
    # DRAM bytes per hop from the ncu capture of the R-MAT s20 case (same kernel source), times this run's hops
    traffic = read_traffic() if args.scale == 22 and not args.int8 else None
    traffic_per_launch = None
    if traffic is not None:
        traffic_per_launch = sum(traffic[pq] * counts[pq]["hops"] for pq in PQ) / len(PQ)

    line = {
        "metric": "walker-steps/sec", "value": value, "unit": "walker-steps/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": (WORKLOAD if args.scale == 22 and len(PQ) == 3 and args.mode == "auto" else
                                f"node2vec R-MAT s{args.scale} ef16 (profiling case), (p,q)={PQ}, mode {args.mode}")
                   + ("; weights stored as 8-bit codes x FP32 scale" if args.int8 else ""), "walkers": n * world,
                   "walkers_per_gpu": nw, "sharding": "replicas of the workload hashed by start node" if world > 1
                   else "none", "walk_length": LENGTH, "edges": g.e,
                   "hops_per_step": hops_all, "l2": "256 MiB write between steps; graph and rows > L2",
                   "cost_ratio": {f"p{p:g}_q{q:g}": ratio[(p, q)] for (p, q) in PQ},
                   "cost_ratio_profiled": {f"p{p:g}_q{q:g}": ratio_profiled[(p, q)] for (p, q) in PQ},
                   "profile_ms": profile_ms, "sweep_ms": sweep_ms, "preprocess_ms": G.info["preprocess_ms"],
                   "per_pq_ms": {f"p{p:g}_q{q:g}": statistics.median(per_launch[(p, q)]) for (p, q) in PQ},
                   "per_pq_hops": {f"p{p:g}_q{q:g}": counts[(p, q)]["hops"] for (p, q) in PQ},
                   "wall_s": wall},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic_per_launch,
                     # DRAM bytes ncu measured per launch over the same launch time: the bandwidth the
                     # random gathers actually draw (each 32-byte access fetches 64-128 bytes)
                     "traffic_GBps": (traffic_per_launch / (kern_ms / len(PQ) / 1000.0) / 1e9
                                      if traffic_per_launch else None),
                     "traffic_frac": (traffic_per_launch / (kern_ms / len(PQ) / 1000.0) / 1e9 / peak
                                      if traffic_per_launch else None),
                     "peak_kind": peak_kind, "kernel": "walk_kernel<1, 0, 1, 0> (single job, uncounted, node2vec, no hub sharing)",
                     "algorithmic_bytes_per_launch": bytes_per_step / len(PQ),
                     "byte_model": "this engine's accesses: 32 B per node record, eRJS edge record and membership "
                                   "probe; 4 B per row entry; eRVS items 8 B",
                     "achieved_survey_model": achieved_survey, "frac_survey_model": achieved_survey / peak,
                     "survey_bytes_per_launch": survey_bytes / len(PQ),
                     "survey_byte_model": "16 B per walker-step + 64 B per eRJS trial + 32 B per membership probe "
                                          "+ 8 B per eRVS item, from the counted trials, probes and items",
                     "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per hop on the R-MAT s20 "
                                       "case of the same kernel source, times this launch's hops",
                     "avg_launch_ms": kern_ms / len(PQ)},
        "roofline_random_access": {
            "bound": "dram_random_access", "unit": "G sector accesses/s",
            "achieved": bytes_per_step / 32.0 / (kern_ms / 1000.0) / 1e9,
            "peak": gather_ceiling / 1e9, "frac": bytes_per_step / 32.0 / (kern_ms / 1000.0) / gather_ceiling,
            "peak_kind": "measured in this run by fw_gather_ceiling (dependent 32-B gathers, 4 GiB table, "
                         "5x256 threads per SM; the rate is flat from 5 to 8 blocks per SM)",
            "note": "algorithmic bytes are sector-granular (32 B per random access), so bytes/32 = accesses"},
        "e2e": e2e_line,
        "gpu_launches": launches,
        "clocks": clocks,
        "counters": {f"p{p:g}_q{q:g}": counts[(p, q)] for (p, q) in PQ},
    }
    # ---- batched, served and metapath workloads (single GPU only; graphs of their own except serving)
    if world == 1 and not args.no_extras and args.scale == 22 and len(PQ) == 3 and args.mode == "auto":
        t_x = time.perf_counter()
        line["serving"] = serve_result(G, g, rate=2000.0, duration=10.0, max_waves=args.max_waves)
        G.close()
        del out, flush, starts
        torch.cuda.empty_cache()
        line["metapath"] = metapath_result(2, 3)
        torch.cuda.empty_cache()
        line["batched"] = batch_result(2, 3)
        torch.cuda.empty_cache()
        line["extras_wall_s"] = time.perf_counter() - t_x
    else:
        G.close()
    if rank == 0 and not args.no_cpu_baseline and args.scale == 22:
        import oracle
        oracle.build()
        line["cpu_baseline"] = cpu_baseline(g, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
