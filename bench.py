"""Benchmark: exact k-clique counting (4- and 5-cliques) on the Chung-Lu
power-law graph (1M vertices, 10M edges, exponent 2.1, max weight 20K).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = counting every 4-clique and every 5-clique of the resident graph
(one launch of the persistent clique kernel computes both).  Prints one JSON
line on rank 0.  ``--impl reference`` times the plain CPU oracle (textbook
oriented clique lister) on a bounded sample of start vertices instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthgraph as sg  # noqa: E402

WORKLOAD = "kclique_chunglu_n1M_m10M_g2.1"
# ncu figures of k_count_clique on this workload (profiles/k_count_clique_chunglu_n1M_m10M.md),
# valid only for the kernel source they were taken on
NCU_CLIQUE = {"source_sha16": "9aa03cc35376c69d", "dram_bytes_per_launch": 89225984,
              "l2_bytes_per_launch": 5841528672, "issue_active_frac": 0.691, "inst_executed_frac": 0.690}
METRIC = "exact pattern matches/sec"
UNIT = "matches/s"
CLIQUE_SIZES = (4, 5)
CPU_SAMPLE_SOURCES = 100_000


def workload_config(g):
    return {"workload": WORKLOAD,
            "graph": {"generator": "chung_lu", "n": g.n, "m": g.m, "gamma": 2.1,
                      "max_weight": 20000, "max_degree": int(g.meta["max_degree"]),
                      "seed": int(g.meta["seed"])},
            "patterns": [f"{k}-clique" for k in CLIQUE_SIZES]}


# --------------------------------------------------------------- clocks ----

class ClockSampler:
    """Clock / throttle-reason sampling during the timed region: NVML in
    process, else nvidia-smi.  Reads settings only; changes none."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.nvml = None
        self.proc = None
        self.lines: list[str] = []

    def _start_nvml(self) -> bool:
        """In-process NVML sampling every 20 ms (enough samples even in a
        sub-second timed region); the GPU is the one CUDA sees, found by its
        PCI bus id.  Returns False (nothing started) on any NVML problem."""
        try:
            import pynvml
            import torch
            pynvml.nvmlInit()
        except Exception:
            return False
        try:
            p = torch.cuda.get_device_properties(self.gpu)
            try:
                h = pynvml.nvmlDeviceGetHandleByPciBusId(
                    f"{p.pci_domain_id:08x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0")
            except Exception:
                h = pynvml.nvmlDeviceGetHandleByIndex(self.gpu)
            reasons = None  # the newer name first; older drivers only have the second
            for name in ("nvmlDeviceGetCurrentClocksEventReasons", "nvmlDeviceGetCurrentClocksThrottleReasons"):
                fn = getattr(pynvml, name, None)
                try:
                    if fn is not None:
                        fn(h)
                        reasons = fn
                        break
                except Exception:
                    continue
            if reasons is None:
                raise RuntimeError("no clock-reason query")
            smax = float(pynvml.nvmlDeviceGetMaxClockInfo(h, pynvml.NVML_CLOCK_SM))
            pynvml.nvmlDeviceGetClockInfo(h, pynvml.NVML_CLOCK_SM)
        except Exception:
            try:
                pynvml.nvmlShutdown()
            except Exception:
                pass
            return False
        self.nvml_samples: list[tuple[float, int]] = []
        self.nvml_stop = threading.Event()

        def loop():
            while not self.nvml_stop.is_set():
                try:
                    self.nvml_samples.append((float(pynvml.nvmlDeviceGetClockInfo(h, pynvml.NVML_CLOCK_SM)),
                                              int(reasons(h))))
                except Exception:
                    break
                self.nvml_stop.wait(0.02)

        self.nvml = (pynvml, smax)
        self.thread = threading.Thread(target=loop, daemon=True)
        self.thread.start()
        return True

    def _stop_nvml(self) -> dict:
        pynvml, smax = self.nvml
        self.nvml_stop.set()
        self.thread.join(timeout=5)
        try:
            pynvml.nvmlShutdown()
        except Exception:
            pass
        bits = {"sw_power_cap": 0x4, "hw_slowdown": 0x8, "sw_thermal_slowdown": 0x20, "hw_thermal_slowdown": 0x40}
        sm = [c for c, _ in self.nvml_samples]
        seen = set()
        for _, r in self.nvml_samples:
            seen |= {name for name, b in bits.items() if r & b}
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax, "reasons": sorted(seen),
                "samples": len(sm), "source": "nvml, 20 ms"}

    def start(self):
        if self._start_nvml():
            return
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except OSError:
            self.proc = None

    def wait_ready(self, timeout: float = 2.0):
        """Wait (bounded) until the sampler has produced its first sample."""
        t = time.perf_counter()
        while time.perf_counter() - t < timeout:
            if self.nvml is not None or self.proc is None or self.lines or self.proc.poll() is not None:
                return
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def stop(self, window=None) -> dict:
        """Stop sampling; with window = (t0, t1) in time.perf_counter()
        seconds keep the samples that arrived in it (plus a 0.25 s grace for
        the output delay), or every sample if none did."""
        if self.nvml is not None:
            return self._stop_nvml()
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        lines = [ln for t, ln in self.lines if window is None or window[0] <= t <= window[1] + 0.25]
        in_window = bool(lines) and window is not None
        if not lines:
            lines = [ln for _, ln in self.lines]
        for line in lines:
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for name, val in zip(names, f[5:9]):
                if val.lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm), "source": "nvidia-smi, 50 ms",
                "window": "timed region" if in_window else "whole sampling run"}


# --------------------------------------------------------------- helpers ---

def algorithmic_bytes(g, rank: np.ndarray, kmin: int) -> int:
    """Bytes of adjacency operands the clique plan's level-1 set operations
    read in one launch: for every start vertex v with at least kmin-1
    higher-ranked neighbours, its out-list N+(v) plus the out-list of every
    u in N+(v) except the first (row 0 of the sub-graph has no bits), plus
    the 16-byte vertex record of every start vertex."""
    deg = np.diff(g.offsets)
    src = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    dst = g.adj.astype(np.int64)
    out = rank[dst] < rank[src]
    dplus = np.bincount(src[out], minlength=g.n).astype(np.int64)
    s, d = src[out], dst[out]
    active = dplus[s] >= kmin - 1
    s, d = s[active], d[active]
    total = int(dplus[dplus >= kmin - 1].sum()) + int(dplus[d].sum())
    # remove the first out-neighbour (smallest rank) of every active start
    if s.size:
        order = np.lexsort((rank[d], s))
        s, d = s[order], d[order]
        first = np.ones(s.size, dtype=bool)
        first[1:] = s[1:] != s[:-1]
        total -= int(dplus[d[first]].sum())
    return 4 * total + 16 * g.n


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, x: float, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(world, x: float, device=None) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t)
    return float(t.item())


# --------------------------------------------------------------- CPU arm ---

def cpu_oracle_rate(g, steps: int, seed: int = 7, sources: int = CPU_SAMPLE_SOURCES):
    """Oracle lister on `steps` seeded samples of `sources` start vertices."""
    import oracle
    rng = np.random.default_rng(seed)
    total, secs = 0, 0.0
    for _ in range(steps):
        src = np.sort(rng.choice(g.n, sources, replace=False)).astype(np.int32)
        t = time.perf_counter()
        for k in CLIQUE_SIZES:
            total += oracle.kcliques(g, k, sources=src)
        secs += time.perf_counter() - t
    return total / secs, total, secs


def run_reference(args):
    world, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    g = sg.workload_graph(2)
    cores = os.cpu_count()
    cpu_oracle_rate(g, max(1, min(args.warmup, 1)))  # warm-up (page-in, build)
    rate, total, secs = cpu_oracle_rate(g, args.steps, seed=11)
    sample = (f"{CPU_SAMPLE_SOURCES} seeded random start vertices per step (of {g.n}); "
              f"4- and 5-cliques whose lowest (degree, id) vertex is sampled")
    line = {"impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int32",
            "data": "synthetic", "config": workload_config(g),
            "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- GPU arm ---

def run_ours(args):
    import torch
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2004_02369_b300 as pg

    g = sg.workload_graph(2)
    stream = torch.cuda.current_stream(dev)
    G = pg.Graph.from_synth(g, stream=stream)
    plans = [pg.Plan(k, sg.clique_edges(k), name=f"{k}-clique") for k in CLIQUE_SIZES]
    counts = torch.zeros(2 * len(plans), dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 126 MB L2

    def step():
        pg.count_async(G, plans, counts, kernel=args.kernel, stream=stream)

    # launch parameters chosen by measurement on this graph (the autotuned
    # persistent variant); the search is not part of the timed steps
    if args.tuning_json:
        fixed = json.loads(open(args.tuning_json).read() if os.path.exists(args.tuning_json) else args.tuning_json)
        pg.set_tuning(G, stream=stream, **fixed)
        tune = {"chosen": pg.get_tuning(G), "fixed": True}
    else:
        tune = pg.autotune(G, plans, stream=stream) if args.autotune and args.kernel == 0 else None

    clocks = ClockSampler(local)  # running before the timed region starts
    clocks.start()
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    expect = pg.decode_counts(counts)
    clocks.wait_ready()
    times = []
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        flush.zero_()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        step()
        e.record(stream)
        times.append((s, e))
    torch.cuda.synchronize()
    barrier(world)
    wall = time.perf_counter() - t0
    clk = clocks.stop(window=(t0, t0 + wall))
    ms = [s.elapsed_time(e) for s, e in times]
    got = pg.decode_counts(counts)
    if got != expect:
        raise SystemExit(f"counts changed between steps: {expect} -> {got}")
    matches = sum(got)
    ms_step = float(np.mean(ms))
    ms_step_max = max_over_ranks(world, ms_step, dev)
    value = sum_over_ranks(world, matches, dev) / (ms_step_max / 1e3)

    if args.only_kernel:
        if rank == 0:
            print(json.dumps({"only_kernel": True, "ms_per_step": ms_step, "counts": got}), flush=True)
        return 0

    # ---- end to end: host CSR in pinned memory -> load -> count -> host ----
    off_h = torch.from_numpy(g.offsets).pin_memory()
    adj_h = torch.from_numpy(g.adj).pin_memory()
    e2e_ms = []
    for it in range(1 + max(1, min(args.steps, 3))):
        torch.cuda.synchronize()
        t = time.perf_counter()
        off_d = off_h.to(dev, non_blocking=True)
        adj_d = adj_h.to(dev, non_blocking=True)
        G2 = pg.Graph(off_d, adj_d, stream=stream)
        pg.count_async(G2, plans, counts, kernel=args.kernel, stream=stream)
        host = counts.cpu()
        dt = (time.perf_counter() - t) * 1e3
        G2.close()
        del off_d, adj_d
        if pg.decode_counts(host) != expect:
            raise SystemExit("end-to-end counts differ")
        if it > 0:
            e2e_ms.append(dt)
    e2e = {"value": matches / (np.mean(e2e_ms) / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(g.offsets.nbytes + g.adj.nbytes),
           "d2h_bytes_per_step": int(counts.numel() * 8),
           "ms_per_step": float(np.mean(e2e_ms)),
           "includes": "pinned H2D of the CSR, validation + degree relabel on device, count, D2H"}

    # ---- one-pattern-per-launch plain interpreter, for comparison ----------
    plain = None
    if args.compare_plain and rank == 0:
        pc = torch.zeros(2, dtype=torch.int64, device=dev)
        per = {}
        for p in plans:
            pg.count_async(G, [p], pc, kernel=pg.KERNEL_CLIQUE_PLAIN, stream=stream)  # warm
            torch.cuda.synchronize()
            flush.zero_()
            s = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            s.record(stream)
            pg.count_async(G, [p], pc, kernel=pg.KERNEL_CLIQUE_PLAIN, stream=stream)
            e.record(stream)
            torch.cuda.synchronize()
            assert pg.decode_counts(pc)[0] == expect[plans.index(p)]
            per[p.name] = s.elapsed_time(e)
        tot = sum(per.values())
        plain = {"kernel": "plan interpreter, one warp per start vertex, one launch per pattern",
                 "ms_per_step": tot, "value": matches / (tot / 1e3), "per_pattern_ms": per,
                 "speedup_of_value": (matches / (ms_step / 1e3)) / (matches / (tot / 1e3))}

    if rank != 0:
        return 0
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm_peak = float(peaks.get("hbm_gbs", 6400.0))
    alg = algorithmic_bytes(g, G.rank(), min(CLIQUE_SIZES))
    achieved = alg / (ms_step / 1e3) / 1e9
    import hashlib
    src = os.path.join(ROOT, "paper_2004_02369_b300", "csrc", "count_clique.cu")
    sha16 = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    ncu_valid = sha16 == NCU_CLIQUE["source_sha16"]
    traffic = args.traffic if args.traffic is not None else (NCU_CLIQUE["dram_bytes_per_launch"] if ncu_valid else None)
    roofline = {"bound": "hbm", "kernel": "k_count_clique", "achieved": achieved, "peak": hbm_peak,
                "unit": "GB/s", "frac": achieved / hbm_peak,
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "algorithmic_bytes_per_launch": alg, "traffic": traffic,
                "ncu": ({"l2_bytes_per_launch": NCU_CLIQUE["l2_bytes_per_launch"],
                         "issue_active_frac": NCU_CLIQUE["issue_active_frac"],
                         "inst_executed_frac_of_peak": NCU_CLIQUE["inst_executed_frac"],
                         "note": "graph is L2-resident; the kernel is instruction-issue bound"}
                        if ncu_valid else None)}

    cpu_rate, _, cpu_secs = cpu_oracle_rate(g, 1)
    cfg = workload_config(g)
    cfg.update({"kernel": {0: "auto (persistent bitmap clique kernel)", 3: "clique"}.get(args.kernel, str(args.kernel)),
                "autotune": tune,
                "l2": "256 MiB buffer written between timed steps (not timed)",
                "counts": {p.name: c for p, c in zip(plans, got)}})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step_max, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": cfg, "e2e": e2e, "gpu_launches": args.steps,
            "roofline": roofline, "clocks": clk,
            "cpu_baseline": {"value": cpu_rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{CPU_SAMPLE_SOURCES} seeded random start vertices, 4- and 5-cliques, "
                                       f"{cpu_secs:.1f} s"},
            "plain_one_pattern_per_launch": plain,
            "wall_s_timed": wall}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- other workloads ---

def _events_ms(fn, stream, reps=1):
    import torch
    s = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    s.record(stream)
    for _ in range(reps):
        fn()
    e.record(stream)
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def run_motif3(args):
    """Induced triangles and wedges on ER G(2000, 0.005): launch-latency
    bound, so microseconds per two-pattern batch, with and without CUDA-graph
    replay of the captured batch launch."""
    import torch
    import paper_2004_02369_b300 as pg
    torch.cuda.set_device(0)
    g = sg.workload_graph(1)
    G = pg.Graph.from_synth(g)
    plans = [pg.Plan.from_dict(p) for p in sg.motif3_patterns()]
    batch = pg.Batch(plans)
    out = torch.zeros(4, dtype=torch.int64, device="cuda")
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        for _ in range(5):
            pg.count_batch(G, batch, out, stream=side)
        reps = 200
        eager_us = 1e3 * _events_ms(lambda: pg.count_batch(G, batch, out, stream=side), side, reps)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            pg.count_batch(G, batch, out, stream=side)
        graph.replay()
        graph_us = 1e3 * _events_ms(graph.replay, side, reps)
    torch.cuda.synchronize()
    counts = pg.decode_counts(out)
    line = {"metric": "microseconds per batch of induced 3-motifs", "value": graph_us, "unit": "us",
            "higher_is_better": False, "data": "synthetic", "n_gpus": 1,
            "config": {"workload": "motif3_er_n2000_p0.005", "m": g.m,
                       "patterns": ["induced_triangle", "induced_wedge"]},
            "eager_us": eager_us, "cuda_graph_us": graph_us,
            "counts": {"induced_triangle": counts[0], "induced_wedge": counts[1]}}
    print(json.dumps(line), flush=True)
    return 0


def run_motif4(args):
    """The six induced 4-motifs of R-MAT scale 20 in one fused launch."""
    import torch
    import paper_2004_02369_b300 as pg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    res = {}
    for sd in ([4, 0] if not args.motif4_small else [4]):
        g = sg.workload_graph(3, scale_down=sd)
        G = pg.Graph.from_synth(g)
        plans = [pg.Plan.from_dict(p) for p in sg.motif4_patterns()]
        out = torch.zeros(12, dtype=torch.int64, device="cuda")
        b = pg.Batch(plans)
        pg.count_batch(G, b, out)
        fused = _events_ms(lambda: pg.count_batch(G, b, out), stream)
        counts = pg.decode_counts(out)
        tune = None
        if args.autotune:
            tune = pg.autotune(G, plans, sample_stride=8 if sd > 0 else 64)
            tuned = _events_ms(lambda: pg.count_batch(G, b, out), stream)
            if pg.decode_counts(out) != counts:
                raise SystemExit("counts changed under tuned launch parameters")
            tune["full_launch_ms_default"] = fused
            tune["full_launch_ms_tuned"] = tuned
            fused = tuned  # the parameters now in effect
        row = {"n": g.n, "m": g.m, "fused_batched_ms": fused, "autotune": tune,
               "counts": dict(zip([p["name"] for p in sg.motif4_patterns()], counts)),
               "matches_per_s": sum(counts) / (fused / 1e3)}
        if sd > 0:
            sep = 0.0
            o = torch.zeros(2, dtype=torch.int64, device="cuda")
            for pl in plans:
                sep += _events_ms(lambda: pg.count_async(G, [pl], o, kernel=pg.KERNEL_GENERIC), stream)
            row["six_separate_launches_ms"] = sep
        res[f"rmat_scale{20 - sd}"] = row
    full = res.get("rmat_scale20") or res["rmat_scale16"]
    line = {"metric": "exact pattern matches/sec", "value": full["matches_per_s"], "unit": "matches/s",
            "data": "synthetic", "n_gpus": 1,
            "config": {"workload": "motif4_induced_rmat_scale20_ef16"}, "results": res}
    print(json.dumps(line), flush=True)
    return 0


def run_motif5(args):
    """The 21 induced 5-vertex motifs of R-MAT scale 12 in one fused launch
    against one launch per motif."""
    import torch
    import paper_2004_02369_b300 as pg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    g = sg.workload_graph(3, scale_down=8)
    G = pg.Graph.from_synth(g)
    pats = pg.generate_all(5, vertex_induced=True)
    plans = [pg.Plan.from_dict(p) for p in pats]
    out = torch.zeros(2 * len(plans), dtype=torch.int64, device="cuda")
    b = pg.Batch(plans)
    pg.count_batch(G, b, out)
    fused = _events_ms(lambda: pg.count_batch(G, b, out), stream)
    counts = pg.decode_counts(out)
    o = torch.zeros(2, dtype=torch.int64, device="cuda")
    per = []
    for p, pl in zip(pats, plans):
        per.append({"edges": p["edges"], "count": counts[len(per)],
                    "ms": _events_ms(lambda: pg.count_async(G, [pl], o, kernel=pg.KERNEL_GENERIC), stream)})
    sep = sum(x["ms"] for x in per)
    print(json.dumps({"workload": "motif5_induced_rmat_scale12_ef16", "data": "synthetic", "n_gpus": 1,
                      "n": g.n, "m": g.m, "patterns": len(plans), "fused_batched_ms": fused,
                      "separate_launches_ms": sep, "per_pattern_interpreter": per, "matches": sum(counts),
                      "matches_per_s": sum(counts) / (fused / 1e3)}), flush=True)
    return 0


def run_lmotif3(args):
    """Labeled 3-motifs with label discovery on the Chung-Lu 500K / 5M graph
    with Zipf labels over 20."""
    import torch
    import paper_2004_02369_b300 as pg
    torch.cuda.set_device(0)
    g = sg.workload_graph(4)
    G = pg.Graph.from_synth(g)
    pg.labeled_motif3(G)  # warm
    times = []
    for _ in range(3):
        torch.cuda.synchronize()
        t = time.perf_counter()
        got = pg.labeled_motif3(G)
        times.append((time.perf_counter() - t) * 1e3)
    matches = sum(got.values())
    print(json.dumps({"workload": "labeled_motif3_chunglu_n500K_m5M_zipf20", "data": "synthetic", "n_gpus": 1,
                      "ms_wall": min(times), "labeled_patterns": len(got), "matches": matches,
                      "triangles": sum(v for (sh, _), v in got.items() if sh == "triangle"),
                      "matches_per_s": matches / (min(times) / 1e3)}), flush=True)
    return 0


def run_exists(args):
    """Existence queries with early termination on the 1M-vertex Chung-Lu graph:
    time to a verdict against the full count."""
    import torch
    import paper_2004_02369_b300 as pg
    torch.cuda.set_device(0)
    g = sg.workload_graph(2)
    G = pg.Graph.from_synth(g)
    res = {}
    for k in (4, 5, 6):
        plan = pg.Plan(k, sg.clique_edges(k))
        pg.count_until(G, plan, 1)  # warm
        t = time.perf_counter()
        got, reached = pg.count_until(G, plan, 1)
        t_exists = (time.perf_counter() - t) * 1e3
        pg.count(G, [plan])
        t = time.perf_counter()
        full = pg.count(G, [plan])[0]
        t_full = (time.perf_counter() - t) * 1e3
        res[f"{k}-clique"] = {"exists": reached, "found_before_stop": got, "ms_to_verdict": t_exists,
                              "full_count": full, "ms_full_count": t_full}
    pg.clustering_coefficient_above(G, 0.01)
    t = time.perf_counter()
    ans, tri, w = pg.clustering_coefficient_above(G, 0.01)
    res["clustering_coefficient_above_0.01"] = {"answer": bool(ans), "triangles_counted": tri, "wedges": w,
                                               "ms": (time.perf_counter() - t) * 1e3}
    print(json.dumps({"workload": "existence_queries_chunglu_n1M_m10M", "data": "synthetic", "n_gpus": 1,
                      "results": res}), flush=True)
    return 0


def run_fsm(args):
    """Frequent labeled patterns (1..3 edges, MNI >= 1000) on Chung-Lu 500K."""
    import torch
    import paper_2004_02369_b300 as pg
    torch.cuda.set_device(0)
    g = sg.workload_graph(4)
    G = pg.Graph.from_synth(g)
    pg.fsm(G, threshold=1000)
    torch.cuda.synchronize()
    t = time.perf_counter()
    freq = pg.fsm(G, threshold=1000)
    dt = time.perf_counter() - t
    by_shape = {}
    for (shape, _), v in freq.items():
        by_shape[shape] = by_shape.get(shape, 0) + 1
    line = {"metric": "FSM wall seconds (all labeled patterns <= 3 edges, MNI >= 1000)", "value": dt,
            "unit": "s", "higher_is_better": False, "data": "synthetic", "n_gpus": 1,
            "config": {"workload": "fsm_chunglu_n500K_m5M_g2.3_zipf20", "threshold": 1000},
            "frequent": len(freq), "frequent_by_shape": by_shape}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------- serving ---

def run_serving(args):
    """Poisson stream of count queries over a resident R-MAT graph: batched
    continuous serving vs the same kernels one query at a time."""
    import torch
    import paper_2004_02369_b300 as pg
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    scale = args.serve_scale
    g = sg.workload_graph(5, scale_down=22 - scale)
    G = pg.Graph.from_synth(g)
    # unlabeled 5-cycles take minutes alone on power-law hubs: they are
    # calibrated alone (alone_ms) and drawn only in their labeled form
    qs = sg.serving_queries(args.serve_n, seed=sg.SEED_BASE + 55, labeled_only=("C5",))
    types = sorted({q["name"] for q in qs})

    # per-type service time alone (first call compiles / sizes scratch)
    alone_ms = {}
    for name in types:
        q = next(x for x in qs if x["name"] == name)
        plan = pg.Plan.from_dict(q)
        pg.count(G, [plan])
        t = time.perf_counter()
        pg.count(G, [plan])
        alone_ms[name] = (time.perf_counter() - t) * 1e3

    def log(msg):
        print(f"[serving {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)

    log(f"graph n={g.n} m={g.m}; {len(qs)} queries; per-type alone ms {alone_ms}")

    def drive(server, arrivals):
        t0 = time.perf_counter()
        tickets = []
        for q, a in zip(qs, arrivals):
            while time.perf_counter() - t0 < a:
                time.sleep(min(2e-4, max(0.0, a - (time.perf_counter() - t0))))
            tickets.append(server.submit(q))
        server.drain(args.serve_timeout)
        res = {r["ticket"]: r for r in server.poll(len(qs) + 10)}
        out = [res[t] for t in tickets]
        lat = np.array([r["t_done"] - r["t_submit"] for r in out]) * 1e3
        span = max(r["t_done"] for r in out) - min(r["t_submit"] for r in out)
        return out, {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "mean_ms": float(lat.mean()), "queries_per_s": len(out) / span,
                     "batches": server.stats()["batches"]}

    # serial capacity: closed loop, everything submitted at t = 0
    srv = pg.Server(G, serial=True)
    base, cal = drive(srv, np.zeros(len(qs)))
    srv.close()
    capacity = cal["queries_per_s"]
    log(f"serial capacity {capacity:.1f} queries/s ({cal})")
    want = [r["count"] for r in base]
    runs = []
    for f in args.serve_lambdas:
        arrivals = sg.poisson_arrivals(len(qs), f * capacity, seed=sg.SEED_BASE + int(100 * f))
        row = {"lambda_x_capacity": f, "rate_qps": f * capacity}
        for mode, kw in (("serial", dict(serial=True)), ("batched", dict(n_streams=4, max_batch=32))):
            srv = pg.Server(G, **kw)
            out, st = drive(srv, arrivals)
            srv.close()
            log(f"lambda {f} {mode}: {st}")
            if [r["count"] for r in out] != want:
                raise SystemExit(f"serving counts differ from one-at-a-time ({mode}, lambda {f})")
            row[mode] = st
        runs.append(row)
    line = {"metric": "serving p50/p99 latency and queries/s, batched vs one query at a time",
            "unit": "ms, queries/s", "n_gpus": 1, "data": "synthetic",
            "config": {"workload": f"serving_rmat_scale{scale}_ef16_labels8",
                       "graph": {"n": g.n, "m": g.m, "max_degree": int(g.meta["max_degree"])},
                       "queries": len(qs), "types": types, "labeled_fraction": 0.1,
                       "labeled_only": ["C5"],
                       "arrivals": "Poisson, rate = lambda x measured serial capacity",
                       "batched": "4 streams, up to 32 queries per launch"},
            "serial_capacity_qps": capacity, "alone_ms": alone_ms, "runs": runs,
            "mix_equals_alone": True}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--kernel", type=int, default=0, help="PG_KERNEL_* (0 = auto)")
    ap.add_argument("--no-compare-plain", dest="compare_plain", action="store_false")
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the default launch parameters")
    ap.add_argument("--workload", choices=["cliques", "serving", "motif3", "motif4", "motif5", "lmotif3", "fsm", "exists"],
                    default="cliques")
    ap.add_argument("--motif4-small", action="store_true", help="skip the full-size motif run")
    ap.add_argument("--serve-scale", type=int, default=16, help="R-MAT scale of the serving graph")
    ap.add_argument("--serve-n", type=int, default=300, help="queries per arrival rate")
    ap.add_argument("--serve-lambdas", type=float, nargs="+", default=[0.5, 0.9, 1.5])
    ap.add_argument("--serve-timeout", type=float, default=600.0, help="seconds to wait for a run's results")
    ap.add_argument("--tuning-json", default=None,
                    help="launch parameters (JSON object or file) applied instead of the autotuner")
    ap.add_argument("--only-kernel", action="store_true",
                    help="time the counting steps only (for profiler runs)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="dram bytes per launch from an ncu capture of this kernel")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "serving":
        return run_serving(args)
    if args.workload == "motif3":
        return run_motif3(args)
    if args.workload == "motif4":
        return run_motif4(args)
    if args.workload == "fsm":
        return run_fsm(args)
    if args.workload == "exists":
        return run_exists(args)
    if args.workload == "motif5":
        return run_motif5(args)
    if args.workload == "lmotif3":
        return run_lmotif3(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
