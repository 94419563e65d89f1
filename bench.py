"""Benchmark: exact k-clique counting (4- and 5-cliques) on the Chung-Lu
power-law graph (1M vertices, 10M edges, exponent 2.1, max weight 20K).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = counting every 4-clique and every 5-clique of the resident graph
(one launch of the persistent clique kernel computes both).  With N GPUs
every rank holds the graph and counts the start vertices of degree rank
r = rank (mod N); one exact sum of the 128-bit counters gives the whole
count, so `value` = all matches / the slowest rank's time.  Prints one JSON
line on rank 0, with the other workloads (induced 3- and 4-motifs, FSM,
14-clique existence, serving) as extra keys under "configs" at N = 1.
``--impl reference`` times the plain CPU oracle (textbook oriented clique
lister) on a bounded sample of start vertices instead.
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
# per-kernel figures of one ncu capture each (DRAM bytes per launch, issue
# rate), keyed by kernel and valid only for the kernel source they were
# taken on
NCU_RECORDS = os.path.join(ROOT, "profiles", "ncu_kernels.json")
CSRC = os.path.join(ROOT, "paper_2004_02369_b300", "csrc")
GOLDEN = os.path.join(ROOT, "tests", "golden", "workload_counts.json")
METRIC = "exact pattern matches/sec"
UNIT = "matches/s"
CLIQUE_SIZES = (4, 5)
CPU_SAMPLE_SOURCES = 100_000
SM_MAX_MHZ = 2032  # maximum SM clock of the B300 (nvidia-smi clocks.max.sm)


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


def log(msg: str):
    """Progress on stderr (the JSON line stays alone on stdout)."""
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def ncu_record(kernel: str):
    """The ncu figures of `kernel` if they were taken on its current source
    (sha256 prefix of the .cu file named in the record), else None."""
    import hashlib
    try:
        rec = json.load(open(NCU_RECORDS))[kernel]
    except (OSError, KeyError, ValueError):
        return None
    src = os.path.join(CSRC, rec["source"])
    if hashlib.sha256(open(src, "rb").read()).hexdigest()[:16] != rec["source_sha16"]:
        return None
    return rec


def golden_counts(name: str) -> dict:
    return {k: int(v) for k, v in json.load(open(GOLDEN))[name]["counts"].items()}


def measured_peaks() -> dict:
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


def hbm_roofline(kernel: str, alg_bytes: int, ms: float, per_launch_note: str, extra=None) -> dict:
    peaks = measured_peaks()
    peak = float(peaks.get("hbm_gbs", 6400.0))
    achieved = alg_bytes / (ms / 1e3) / 1e9
    rec = ncu_record(kernel)
    out = {"bound": "hbm", "kernel": kernel, "achieved": achieved, "peak": peak, "unit": "GB/s",
           "frac": achieved / peak, "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
           "frac_of_nominal_7700": achieved / 7700.0,
           "algorithmic_bytes_per_launch": int(alg_bytes), "algorithmic_bytes": per_launch_note,
           "traffic": rec["dram_bytes_per_launch"] if rec and "dram_bytes_per_launch" in rec else None}
    if rec:
        out["ncu"] = {k: v for k, v in rec.items() if k not in ("source", "source_sha16", "command")}
    if extra:
        out.update(extra)
    return out


def issue_roofline(rec, ms: float, dev, max_mhz=None):
    """Instruction-issue roofline of an issue-bound kernel: its warp
    instructions per launch (from the ncu record, when it matches the
    current source) over the CUDA-event time, against one warp instruction
    per cycle per SM sub-partition (4 per SM) at the maximum SM clock."""
    import torch
    if not rec or "warp_instructions_per_launch" not in rec:
        return None
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(max_mhz or SM_MAX_MHZ)
    peak = sms * 4 * mhz * 1e6
    achieved = rec["warp_instructions_per_launch"] / (ms / 1e3)
    return {"bound": "issue", "achieved": achieved, "peak": peak, "unit": "warp instructions/s",
            "frac": achieved / peak, "peak_source": f"{sms} SMs x 4 issue slots x {mhz:.0f} MHz (maximum SM clock)",
            "instructions_source": "ncu smsp__inst_executed.sum of one launch"}


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


def sum_counts_over_ranks(world, counts, device=None) -> list[int]:
    """Exact sum over ranks of non-negative integer counts below 2^128:
    each count travels as four 32-bit limbs in int64 lanes (sums of up to
    2^31 ranks cannot overflow), recombined after the all-reduce."""
    if world == 1:
        return [int(c) for c in counts]
    import torch
    import torch.distributed as dist
    limbs = [[(int(c) >> (32 * j)) & 0xFFFFFFFF for j in range(4)] for c in counts]
    t = torch.tensor(limbs, dtype=torch.int64, device=device)
    dist.all_reduce(t)
    return [sum(int(x) << (32 * j) for j, x in enumerate(row)) for row in t.cpu().tolist()]


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

def _pinned(a: np.ndarray) -> np.ndarray:
    """A page-locked copy of a host array (numpy view of pinned memory)."""
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).pin_memory().numpy()


def run_ours(args):
    import torch
    world, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    import paper_2004_02369_b300 as pg

    g = sg.workload_graph(2)
    log("graph generated")
    stream = torch.cuda.current_stream(dev)
    G = pg.Graph.from_synth(g, stream=stream)
    if world > 1:
        pg.set_partition(G, rank, world)  # start vertices of rank r = rank (mod world)
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

    log(f"tuned: {tune['chosen'] if tune else None}")
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
    total = sum_counts_over_ranks(world, got, dev)
    gold = golden_counts("cliques")
    if total != [gold[f"{k}-clique"] for k in CLIQUE_SIZES]:
        raise SystemExit(f"counts differ from the oracle's: {total}")
    matches = sum(total)
    ms_step = float(np.mean(ms))
    ms_step_max = max_over_ranks(world, ms_step, dev)
    value = matches / (ms_step_max / 1e3)

    if args.only_kernel:
        if rank == 0:
            print(json.dumps({"only_kernel": True, "ms_per_step": ms_step, "counts": got}), flush=True)
        return 0

    log(f"timed steps: {ms_step:.3f} ms")
    # ---- end to end through the C-ABI with host buffers: pinned CSR ->
    # pg_load_graph (the library's own H2D, validation, degree relabel) ->
    # pg_count (launch, D2H) -> exact sum over ranks
    off_h, adj_h = _pinned(g.offsets), _pinned(g.adj)
    e2e_ms = []
    for it in range(1 + max(1, min(args.steps, 3))):
        barrier(world)
        torch.cuda.synchronize()
        t = time.perf_counter()
        G2 = pg.Graph(off_h, adj_h, stream=stream)
        pg.set_tuning(G2, stream=stream, **pg.get_tuning(G))
        if world > 1:
            pg.set_partition(G2, rank, world)
        host = pg.count(G2, plans, stream=stream)
        host_total = sum_counts_over_ranks(world, host, dev)
        dt = (time.perf_counter() - t) * 1e3
        G2.close()
        if host_total != total:
            raise SystemExit("end-to-end counts differ")
        if it > 0:
            e2e_ms.append(max_over_ranks(world, dt, dev))
    e2e = {"value": matches / (np.mean(e2e_ms) / 1e3), "unit": UNIT,
           "h2d_bytes_per_step": int(g.offsets.nbytes + g.adj.nbytes),
           "d2h_bytes_per_step": int(16 * len(plans)),
           "ms_per_step": float(np.mean(e2e_ms)),
           "includes": "pg_load_graph from pinned host CSR (H2D, validation, degree relabel), "
                       "launch-parameter copy, pg_count (count, D2H), sum over ranks"}

    log(f"e2e: {e2e['ms_per_step']:.2f} ms")
    # ---- plain one-pattern-per-launch forms on the same GPU --------------
    plain = interp = None
    if args.compare_plain and rank == 0 and world == 1:
        plain = _per_pattern(pg, G, plans, expect, pg.KERNEL_CLIQUE_NONPERSISTENT, stream, flush, matches)
        plain["kernel"] = ("k-clique bitmap kernel without persistence: one warp per start vertex (one CTA per "
                           "heavy start vertex), one launch pair per pattern")
        plain["speedup_of_value"] = plain["ms_per_step"] / ms_step
        log(f"plain non-persistent: {plain['ms_per_step']:.2f} ms")
        interp = _per_pattern(pg, G, plans, expect, pg.KERNEL_CLIQUE_PLAIN, stream, flush, matches)
        log(f"interpreter per pattern: {interp['ms_per_step']:.2f} ms")
        interp["kernel"] = ("plan interpreter (sorted-list set operations, 16-byte driver loads), one warp per "
                            "start vertex, one launch per pattern")
        interp["speedup_of_value"] = interp["ms_per_step"] / ms_step

    if rank != 0:
        return 0
    alg = algorithmic_bytes(g, G.rank(), min(CLIQUE_SIZES))
    rec = ncu_record("k_count_clique")
    roofline = hbm_roofline(
        "k_count_clique", alg // max(world, 1), ms_step_max,
        "4 B x (out-list of every start vertex + out-lists of its out-neighbours but the first): the operands "
        "of the level-1 intersections; deeper levels are word ANDs of on-chip bitmap rows",
        {"issue_active_frac": rec.get("issue_active_frac") if rec else None,
         "note": "graph L2-resident; the kernel is bound by instruction issue (issue_active_frac of the "
                 "SM issue slots, ncu)"})
    # every set operation of the two plans, all levels (the device operand
    # walk over the same prefixes as the plan interpreter)
    t = time.perf_counter()
    ops_bytes = [pg.plan_operand_bytes(G, p, stream=stream) for p in plans]
    all_bytes = sum(b for b, _ in ops_bytes)
    log(f"operand walk: {all_bytes / 1e9:.1f} GB in {time.perf_counter() - t:.1f} s")
    roofline["all_levels"] = {
        "algorithmic_bytes_per_launch": all_bytes, "set_operations": sum(o for _, o in ops_bytes),
        "achieved": all_bytes / (ms_step_max / 1e3) / 1e9, "unit": "GB/s",
        "frac": all_bytes / (ms_step_max / 1e3) / 1e9 / roofline["peak"],
        "algorithmic_bytes": "4 B x every partial-order-bounded operand slice of every set operation of the "
                             "4- and 5-clique plans, all levels (pg_plan_operand_bytes); this kernel does the "
                             "levels below the first as on-chip bitmap ANDs, so the fraction can pass 1"}
    roofline["issue"] = issue_roofline(rec, ms_step_max, dev, (clk or {}).get("sm_max_mhz"))
    extra = run_extra_configs(args, pg, dev, G) if (args.extra and world == 1) else None
    cpu_rate, _, cpu_secs = cpu_oracle_rate(g, 1)
    cfg = workload_config(g)
    cfg.update({"kernel": {0: "auto (persistent bitmap clique kernel)", 3: "clique"}.get(args.kernel, str(args.kernel)),
                "autotune": tune,
                "parallelism": f"start vertices dealt round-robin by degree rank over {world} GPU(s), exact "
                               "sum of the 128-bit counters" if world > 1 else "one GPU",
                "l2": "256 MiB buffer written between timed steps (not timed)",
                "counts": {p.name: c for p, c in zip(plans, total)}, "counts_match_oracle": True})
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step_max, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "int32", "data": "synthetic",
            "config": cfg, "e2e": e2e, "gpu_launches": args.steps,
            "roofline": roofline, "clocks": clk,
            "cpu_baseline": {"value": cpu_rate, "unit": UNIT, "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{CPU_SAMPLE_SOURCES} seeded random start vertices, 4- and 5-cliques, "
                                       f"{cpu_secs:.1f} s"},
            "plain_one_pattern_per_launch": plain,
            "interpreter_one_pattern_per_launch": interp,
            "configs": extra,
            "wall_s_timed": wall}
    print(json.dumps(line), flush=True)
    return 0


def _per_pattern(pg, G, plans, expect, kernel, stream, flush, matches):
    """One launch (pair) per pattern with `kernel`, CUDA events per pattern."""
    import torch
    pc = torch.zeros(2, dtype=torch.int64, device=flush.device)
    per = {}
    for i, p in enumerate(plans):
        pg.count_async(G, [p], pc, kernel=kernel, stream=stream)  # warm
        torch.cuda.synchronize()
        flush.zero_()
        s = torch.cuda.Event(enable_timing=True)
        e = torch.cuda.Event(enable_timing=True)
        s.record(stream)
        pg.count_async(G, [p], pc, kernel=kernel, stream=stream)
        e.record(stream)
        torch.cuda.synchronize()
        if pg.decode_counts(pc)[0] != expect[i]:
            raise SystemExit(f"{p.name}: kernel {kernel} count differs")
        per[p.name] = s.elapsed_time(e)
    tot = sum(per.values())
    return {"ms_per_step": tot, "value": matches / (tot / 1e3), "per_pattern_ms": per}


# --------------------------------------------------------------- other configs ---

def _events(stream):
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def _timed(fn, stream, flush=None, reps=1) -> float:
    """Device milliseconds of fn() per call on `stream` (CUDA events),
    flushing L2 before the timed region when `flush` is given."""
    import torch
    torch.cuda.synchronize()
    if flush is not None:
        flush.zero_()
    s, e = _events(stream)
    s.record(stream)
    for _ in range(reps):
        fn()
    e.record(stream)
    torch.cuda.synchronize()
    return s.elapsed_time(e) / reps


def _e2e(pg, g, call, reps=3) -> dict:
    """End to end through the C-ABI with host buffers: pinned CSR (and
    labels) -> pg_load_graph -> call(graph) (launches and D2H) -> graph
    freed; mean wall milliseconds over reps after one warm-up."""
    import torch
    off_h, adj_h = _pinned(g.offsets), _pinned(g.adj)
    lab_h = None if g.labels is None else _pinned(g.labels)
    ms = []
    for it in range(reps + 1):
        torch.cuda.synchronize()
        t = time.perf_counter()
        G = pg.Graph(off_h, adj_h, lab_h)
        res = call(G)
        dt = (time.perf_counter() - t) * 1e3
        G.close()
        if it:
            ms.append(dt)
    h2d = int(g.offsets.nbytes + g.adj.nbytes + (0 if g.labels is None else g.labels.nbytes))
    return {"ms": float(np.mean(ms)), "h2d_bytes_per_step": h2d, "result": res}


def _cfg_motif3(pg, dev) -> dict:
    """Induced triangles and wedges on ER G(2000, 0.005): launch-latency
    bound; microseconds per two-pattern batch, eager and CUDA-graph replay."""
    import torch
    g = sg.workload_graph(1)
    G = pg.Graph.from_synth(g)
    plans = [pg.Plan.from_dict(p) for p in sg.motif3_patterns()]
    batch = pg.Batch(plans)
    out = torch.zeros(4, dtype=torch.int64, device=dev)
    side = torch.cuda.Stream()
    with torch.cuda.stream(side):
        for _ in range(5):
            pg.count_batch(G, batch, out, stream=side)
        eager_us = 1e3 * _timed(lambda: pg.count_batch(G, batch, out, stream=side), side, reps=200)
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=side):
            pg.count_batch(G, batch, out, stream=side)
        graph.replay()
        graph_us = 1e3 * _timed(graph.replay, side, reps=200)
    torch.cuda.synchronize()
    got = pg.decode_counts(out)
    gold = golden_counts("motif3")
    ok = got == [gold["induced_triangle"], gold["induced_wedge"]]
    e2e = _e2e(pg, g, lambda G2: pg.count(G2, plans))
    if e2e["result"] != got:
        raise SystemExit("motif3 end-to-end counts differ")
    adj_bytes = int(g.adj.nbytes + 16 * g.n)
    return {"workload": "motif3_er_n2000_p0.005", "metric": "microseconds per batch of induced 3-motifs",
            "unit": "us", "higher_is_better": False, "value": graph_us, "eager_us": eager_us,
            "cuda_graph_us": graph_us, "counts": {"induced_triangle": got[0], "induced_wedge": got[1]},
            "counts_match_oracle": ok, "gpu_launches_per_batch": 2,
            "e2e": {"value": 1e3 * e2e["ms"], "unit": "us", "h2d_bytes_per_step": e2e["h2d_bytes_per_step"],
                    "d2h_bytes_per_step": 32, "includes": "pg_load_graph from pinned host CSR, pg_count, D2H"},
            "roofline": hbm_roofline("k_count_batched", adj_bytes, graph_us / 1e3,
                                     "every adjacency list and vertex record read once (lower bound)",
                                     {"note": "launch-latency bound: 2 kernels of a few microseconds"})}


def c4_increments(g, rank):
    """Adjacency elements the 4-cycle co-degree kernel reads: for every
    anchor w and neighbour a ranked after w, the suffix of adj(a) ranked
    after w, plus the anchors' own neighbour suffixes."""
    deg = np.diff(g.offsets)
    src = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    rs, rd = rank[src].astype(np.int64), rank[g.adj.astype(np.int64)].astype(np.int64)
    o = np.lexsort((rd, rs))
    RS, RD = rs[o], rd[o]
    off = np.zeros(g.n + 1, np.int64)
    np.add.at(off, RS + 1, 1)
    off = np.cumsum(off)
    pos = np.arange(RS.size) - off[RS]
    lower = RD < RS                      # edge (a -> w) with w ranked before a
    above = (off[RS + 1] - off[RS]) - pos - 1
    return int(above[lower].sum()) + int(lower.sum())


def _cfg_motif4(pg, dev, args) -> dict:
    """The six induced 4-vertex motifs of R-MAT scale 20 in one fused launch
    (anti-edges expanded into edge-induced terms; the 4-cycle term by the
    co-degree kernel, cliques by the clique kernel, the rest on the prefix
    tree)."""
    import torch
    g = sg.workload_graph(3)
    G = pg.Graph.from_synth(g)
    pats = sg.motif4_patterns()
    plans = [pg.Plan.from_dict(p) for p in pats]
    batch = pg.Batch(plans)
    out = torch.zeros(12, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    tune = pg.autotune(G, plans, sample_stride=64) if args.autotune else None
    pg.count_batch(G, batch, out)
    fused_ms = min(_timed(lambda: pg.count_batch(G, batch, out), stream, flush) for _ in range(2))
    got = pg.decode_counts(out)
    gold = golden_counts("motif4")
    ok = got == [gold[p["name"]] for p in pats]
    c4 = pg.Batch([pg.Plan(4, sg.cycle_edges(4))])
    c4_out = torch.zeros(2, dtype=torch.int64, device=dev)
    pg.count_batch(G, c4, c4_out)
    c4_ms = _timed(lambda: pg.count_batch(G, c4, c4_out), stream, flush)
    # the prefix-tree kernel's part of the step: the other edge-induced terms
    tree = pg.Batch([pg.Plan(4, sg.MOTIF4_SHAPES[k]) for k in ("path", "star", "tailed_triangle", "diamond")])
    tree_out = torch.zeros(8, dtype=torch.int64, device=dev)
    pg.count_batch(G, tree, tree_out)
    tree_ms = _timed(lambda: pg.count_batch(G, tree, tree_out), stream, flush)
    matches = sum(got)
    e2e = _e2e(pg, g, lambda G2: pg.count(G2, plans), reps=2)
    if e2e["result"] != got:
        raise SystemExit("motif4 end-to-end counts differ")
    inc = c4_increments(g, G.rank())
    return {"workload": "motif4_induced_rmat_scale20_ef16", "metric": METRIC, "unit": UNIT, "value": matches / (fused_ms / 1e3),
            "ms": fused_ms, "counts": dict(zip([p["name"] for p in pats], got)), "counts_match_oracle": ok,
            "graph": {"n": g.n, "m": g.m}, "autotune": tune, "edge_induced_4cycle_ms": c4_ms,
            "e2e": {"value": matches / (e2e["ms"] / 1e3), "unit": UNIT, "ms": e2e["ms"],
                    "h2d_bytes_per_step": e2e["h2d_bytes_per_step"], "d2h_bytes_per_step": 96,
                    "includes": "pg_load_graph from pinned host CSR, pg_count (batch build, launches, D2H)"},
            "roofline": hbm_roofline("k_c4_tiled", 4 * inc, c4_ms,
                                     "4 B x adjacency elements the co-degree pass reads (neighbour suffixes "
                                     "above each anchor); timed: the 4-cycle term alone",
                                     {"share_of_fused_step": c4_ms / fused_ms,
                                      "dominant_kernel": {
                                          "kernel": "k_count_batched", "ms": tree_ms,
                                          "share_of_fused_step": tree_ms / fused_ms,
                                          "terms": "edge-induced path, star, tailed triangle, diamond",
                                          "bound": "latency of the binary-search loads of its set operations "
                                                   "(graph L2-resident; ncu in profiles/)"}})}


def fsm_bytes(g) -> int:
    """Bytes the FSM row kernel reads and writes: per vertex its record, label
    masks and list; per neighbour w its record, masks and list, a 16-byte
    mask per element of adj(w) (path ends), and the smaller list of the
    triangle test; one row of membership words written and read once."""
    deg = np.diff(g.offsets).astype(np.int64)
    src = np.repeat(np.arange(g.n, dtype=np.int64), deg)
    dw = deg[g.adj.astype(np.int64)]
    nl = int(g.labels.max()) + 1
    words = 1 + 3 * nl + 4 * nl * nl
    return int(g.n * 32 + 4 * deg.sum() + 32 * deg.sum() + 20 * dw.sum() + 4 * np.minimum(deg[src], dw).sum()
               + 2 * 4 * words * g.n)


def _cfg_fsm(pg, dev) -> dict:
    """Labeled FSM with MNI support >= 1000, 1..3 edges, on Chung-Lu 500K / 5M
    with Zipf labels over 20 (synchronous call: wall milliseconds)."""
    import torch
    g = sg.workload_graph(4)
    G = pg.Graph.from_synth(g)
    pg.fsm(G, threshold=1000)
    ms = []
    for _ in range(3):
        torch.cuda.synchronize()
        t = time.perf_counter()
        freq = pg.fsm(G, threshold=1000)
        ms.append((time.perf_counter() - t) * 1e3)
    want = {}
    for key, v in golden_counts("fsm").items():
        shape, labels = key.split(":")
        want[(shape, tuple(int(x) for x in labels.split(",")))] = v
    e2e = _e2e(pg, g, lambda G2: len(pg.fsm(G2, threshold=1000)), reps=2)
    by_shape = {}
    for (shape, _), _v in freq.items():
        by_shape[shape] = by_shape.get(shape, 0) + 1
    return {"workload": "fsm_chunglu_n500K_m5M_g2.3_zipf20", "metric": "FSM milliseconds (labeled patterns <= 3 "
            "edges, MNI >= 1000)", "unit": "ms", "higher_is_better": False, "value": min(ms),
            "frequent": len(freq), "frequent_by_shape": by_shape, "counts_match_oracle": freq == want,
            "e2e": {"value": e2e["ms"], "unit": "ms", "h2d_bytes_per_step": e2e["h2d_bytes_per_step"],
                    "d2h_bytes_per_step": 32 * len(freq),
                    "includes": "pg_load_graph from pinned host CSR and labels, pg_fsm (host scan of the label "
                                "histogram, kernels, D2H, sort)"},
            "roofline": hbm_roofline("k_fsm_rows", fsm_bytes(g), min(ms),
                                     "vertex and neighbour records, lists, per-element label masks of the 2-hop "
                                     "scan, rows written and read once; timed: the whole synchronous call",
                                     {"note": "the call's wall time includes host steps"})}


def _cfg_exists(pg, G, budget_ms: float = 30000.0) -> dict:
    """Existence queries with early termination on the 1M-vertex Chung-Lu graph
    (the paper's 14-clique existence query, and 6- and 10-cliques), each
    under a device work budget: a query that neither finds a match nor
    exhausts the search within it is reported as undetermined."""
    import torch
    res = {}
    pg.set_time_budget(G, budget_ms)
    try:
        for k in (4, 5, 6, 10, 14):
            plan = pg.Plan(k, sg.clique_edges(k))
            r = {}
            # the first call sizes scratch and sets kernel attributes; a
            # query that reached a verdict is timed again warm
            for key in ("ms_to_verdict_first_call", "ms_to_verdict"):
                torch.cuda.synchronize()
                t = time.perf_counter()
                try:
                    got, reached = pg.count_until(G, plan, 1)
                    r.update({"exists": reached, "found_before_stop": got, key: (time.perf_counter() - t) * 1e3})
                except pg.PgError as e:
                    if e.code != pg.PG_ETIMEOUT:
                        raise
                    r = {"exists": None, "undetermined_within_ms": budget_ms}
                    break
            res[f"{k}-clique"] = r
            log(f"exists {k}-clique: {r}")
    finally:
        pg.set_time_budget(G, 0)
    return {"workload": "existence_chunglu_n1M_m10M", "results": res, "budget_ms": budget_ms,
            "note": "wall milliseconds of the synchronous pg_count_until (launch, stop flag, D2H); "
                    "cliques run on the k-clique kernel with cardinality pruning; found_before_stop "
                    "is the count published when the stop flag was seen"}


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
    import torch
    import paper_2004_02369_b300 as pg
    torch.cuda.set_device(0)
    print(json.dumps(_cfg_motif3(pg, torch.device("cuda", 0))), flush=True)
    return 0


def run_motif4(args):
    """The six induced 4-motifs of R-MAT scale 20 in one fused launch."""
    import torch
    import paper_2004_02369_b300 as pg
    torch.cuda.set_device(0)
    stream = torch.cuda.current_stream()
    res = {}
    for scale in (args.motif4_scales if not args.motif4_small else [16]):
        sd = 20 - scale
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
            tune = pg.autotune(G, plans, sample_stride=8 if scale <= 16 else 64)
            tuned = _events_ms(lambda: pg.count_batch(G, b, out), stream)
            if pg.decode_counts(out) != counts:
                raise SystemExit("counts changed under tuned launch parameters")
            tune["full_launch_ms_default"] = fused
            tune["full_launch_ms_tuned"] = tuned
            fused = tuned  # the parameters now in effect
        row = {"n": g.n, "m": g.m, "fused_batched_ms": fused, "autotune": tune,
               "counts": dict(zip([p["name"] for p in sg.motif4_patterns()], counts)),
               "matches_per_s": sum(counts) / (fused / 1e3)}
        if scale <= 16:
            sep = 0.0
            o = torch.zeros(2, dtype=torch.int64, device="cuda")
            for pl in plans:
                sep += _events_ms(lambda: pg.count_async(G, [pl], o, kernel=pg.KERNEL_GENERIC), stream)
            row["six_separate_launches_ms"] = sep
        if args.motif4_terms:
            # the edge-induced terms the induced motifs expand into, each alone
            terms = {}
            o = torch.zeros(2, dtype=torch.int64, device="cuda")
            for name, edges in sg.MOTIF4_SHAPES.items():
                tb = pg.Batch([pg.Plan(4, edges)])
                pg.count_batch(G, tb, o)
                terms[name] = _events_ms(lambda: pg.count_batch(G, tb, o), stream)
            row["edge_induced_terms_ms"] = terms
        res[f"rmat_scale{scale}"] = row
    full = res[f"rmat_scale{max(int(x) for x in (args.motif4_scales if not args.motif4_small else [16]))}"]
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
    import torch
    import paper_2004_02369_b300 as pg
    torch.cuda.set_device(0)
    print(json.dumps(_cfg_fsm(pg, torch.device("cuda", 0))), flush=True)
    return 0


# --------------------------------------------------------------- serving ---

def serving_run(pg, scale: int, n_queries: int, lambdas, timeout_s: float, labeled_only=("C5",),
                query_timeout_s: float = 0.0, alone_only: bool = False, alone_budget_ms: float = 0.0,
                types=None, alone_fractions=(1.0,)) -> dict:
    """Poisson streams of count queries over a resident R-MAT graph (the
    serving mix of cliques, stars, paths, cycles and tailed triangles, 10%
    labeled over 8 labels): continuous batching (4 streams, up to 32 queries
    per launch) against the same kernels one query at a time; every result
    of the mix equals the query's count alone."""
    import torch
    dev = torch.device("cuda", torch.cuda.current_device())
    g = sg.workload_graph(5, scale_down=22 - scale)
    G = pg.Graph.from_synth(g)
    qs = sg.serving_queries(n_queries, seed=sg.SEED_BASE + 55, labeled_only=labeled_only, types=types)
    types = sorted({q["name"] for q in qs})

    def log(msg):
        print(f"[serving {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)

    # per-type service time alone (first call compiles / sizes scratch);
    # with alone_budget_ms a type that runs longer is reported as over it
    alone_ms = {}
    if alone_budget_ms:
        pg.set_time_budget(G, alone_budget_ms)
    for name in types:
        q = next(x for x in qs if x["name"] == name)
        plan = pg.Plan.from_dict(q)
        try:
            pg.count(G, [plan])
            t = time.perf_counter()
            pg.count(G, [plan])
            alone_ms[name] = (time.perf_counter() - t) * 1e3
        except pg.PgError as e:
            if e.code != pg.PG_ETIMEOUT:
                raise
            alone_ms[name] = f"> {alone_budget_ms:.0f}"
        log(f"alone {name}: {alone_ms[name]}")
    pg.set_time_budget(G, 0)

    log(f"graph n={g.n} m={g.m}; {len(qs)} queries; per-type alone ms {alone_ms}")
    if alone_only:
        done = [alone_ms[q["name"]] for q in qs if not isinstance(alone_ms[q["name"]], str)]
        return {"workload": f"serving_rmat_scale{scale}_ef16_labels8", "graph": {"n": g.n, "m": g.m},
                "alone_ms": alone_ms, "alone_budget_ms": alone_budget_ms,
                "mix_mean_alone_ms_of_measured": float(np.mean(done)) if done else None}

    def drive(server, arrivals, closed=False):
        # closed: each query is submitted when the previous one is done
        t0 = time.perf_counter()
        tickets, res = [], {}
        for q, a in zip(qs, arrivals):
            while time.perf_counter() - t0 < a:
                time.sleep(min(2e-4, max(0.0, a - (time.perf_counter() - t0))))
            tickets.append(server.submit(q))
            if closed:
                server.drain(timeout_s)
                res.update({r["ticket"]: r for r in server.poll(10)})
        server.drain(timeout_s)
        res.update({r["ticket"]: r for r in server.poll(len(qs) + 10)})
        out = [res[t] for t in tickets]
        lat = np.array([r["t_done"] - r["t_submit"] for r in out]) * 1e3
        span = max(r["t_done"] for r in out) - min(r["t_submit"] for r in out)
        return out, {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                     "mean_ms": float(lat.mean()), "queries_per_s": len(out) / span,
                     "batches": server.stats()["batches"],
                     "timed_out": sum(1 for r in out if r["status"] == pg.PG_ETIMEOUT)}

    # serial capacity: closed loop, one query at a time (so that a query time
    # limit counts only the query's own run)
    srv = pg.Server(G, serial=True, query_timeout_s=query_timeout_s)
    base, cal = drive(srv, np.zeros(len(qs)), closed=True)
    srv.close()
    capacity = cal["queries_per_s"]
    log(f"serial capacity {capacity:.1f} queries/s ({cal})")
    ok_status = (pg.PG_OK, pg.PG_ETIMEOUT) if query_timeout_s > 0 else (pg.PG_OK,)
    if any(r["status"] not in ok_status for r in base):
        raise SystemExit("a serving query failed when run one at a time")
    want = [r["count"] if r["status"] == pg.PG_OK else None for r in base]
    runs = []
    for f in lambdas:
        arrivals = sg.poisson_arrivals(len(qs), f * capacity, seed=sg.SEED_BASE + int(100 * f))
        row = {"lambda_x_capacity": f, "rate_qps": f * capacity}
        modes = [("serial", dict(serial=True))]
        for fr in alone_fractions:
            modes.append(("batched" if fr == 1.0 else f"batched_alone_sm{fr:g}",
                          dict(n_streams=4, max_batch=32, alone_sm_fraction=fr)))
        for mode, kw in modes:
            srv = pg.Server(G, query_timeout_s=query_timeout_s, **kw)
            out, st = drive(srv, arrivals)
            srv.close()
            log(f"lambda {f} {mode}: {st}")
            got = [r["count"] if r["status"] == pg.PG_OK else None for r in out]
            if any(x is not None and w is not None and x != w for x, w in zip(got, want)):
                raise SystemExit(f"serving counts differ from one-at-a-time ({mode}, lambda {f})")
            st["compared_with_alone"] = sum(1 for x, w in zip(got, want) if x is not None and w is not None)
            row[mode] = st
        runs.append(row)
    return {"workload": f"serving_rmat_scale{scale}_ef16_labels8",
            "metric": "serving p50/p99 latency and queries/s, batched vs one query at a time",
            "unit": "ms, queries/s",
            "graph": {"n": g.n, "m": g.m, "max_degree": int(g.meta["max_degree"])},
            "queries": len(qs), "types": types, "labeled_fraction": 0.1, "labeled_only": list(labeled_only),
            "arrivals": "Poisson, rate = lambda x measured serial capacity",
            "batched": "4 streams, up to 32 queries per launch; a pattern's first query and patterns longer "
                       "than 20 ms alone run alone (with the waiting queries of the same pattern) on at most 3 "
                       "streams, on all SMs unless the mode name gives a share", "serial_capacity_qps": capacity,
            "alone_ms": alone_ms, "runs": runs, "mix_equals_alone": True,
            "query_timeout_s": query_timeout_s}


def run_extra_configs(args, pg, dev, G_cliques) -> dict:
    t = time.perf_counter()
    out = {}
    for name, fn in (("motif3_er2000", lambda: _cfg_motif3(pg, dev)), ("motif4_rmat20", lambda: _cfg_motif4(pg, dev, args)),
                     ("fsm_chunglu500k", lambda: _cfg_fsm(pg, dev)), ("exists_chunglu1M", lambda: _cfg_exists(pg, G_cliques))):
        log(f"config {name} ...")
        out[name] = fn()
        log(f"config {name} done")
    if args.serve_n > 0:
        out[f"serving_rmat{args.serve_scale}"] = serving_run(pg, args.serve_scale, args.serve_n, args.serve_lambdas,
                                                             args.serve_timeout)
    out["wall_s"] = time.perf_counter() - t
    return out


def run_serving(args):
    import torch
    import paper_2004_02369_b300 as pg
    torch.cuda.set_device(0)
    line = serving_run(pg, args.serve_scale, args.serve_n, args.serve_lambdas, args.serve_timeout,
                       labeled_only=tuple(args.serve_labeled_only), query_timeout_s=args.serve_query_timeout,
                       alone_only=args.serve_alone_only, alone_budget_ms=args.serve_alone_budget_ms,
                       types=args.serve_types, alone_fractions=tuple(args.serve_alone_fractions))
    line.update({"n_gpus": 1, "data": "synthetic"})
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
    ap.add_argument("--motif4-scales", type=int, nargs="+", default=[16, 20], help="R-MAT scales of the motif run")
    ap.add_argument("--motif4-terms", action="store_true", help="also time each edge-induced 4-vertex term alone")
    ap.add_argument("--no-extra", dest="extra", action="store_false",
                    help="only the k-clique headline (no per-config keys)")
    ap.add_argument("--serve-scale", type=int, default=16, help="R-MAT scale of the serving graph")
    ap.add_argument("--serve-n", type=int, default=100, help="queries per arrival rate (0: no serving key)")
    ap.add_argument("--serve-labeled-only", nargs="*", default=["C5"],
                    help="query types drawn only in their labeled form")
    ap.add_argument("--serve-query-timeout", type=float, default=0.0, help="server query time limit (s)")
    ap.add_argument("--serve-alone-only", action="store_true", help="only each query type's time alone")
    ap.add_argument("--serve-alone-budget-ms", type=float, default=0.0,
                    help="device work budget of each alone measurement (0: none)")
    ap.add_argument("--serve-types", nargs="*", default=None, help="query types of the mix (default: all)")
    ap.add_argument("--serve-alone-fractions", type=float, nargs="+", default=[1.0],
                    help="SM shares of alone-running queries, one batched run each")
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
