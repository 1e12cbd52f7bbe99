"""Benchmark of the BITS hot path on B300 (one JSON line on stdout).

Headline workload (one "step"): bits_count of the learned-index workload at
scale -- 100,000,000 query intervals placed uniformly on a 3.0 Gbp line
against a resident database of 100,000,000 intervals (80 % from a mixture of
1000 Gaussians, 20 % uniform; lengths log-uniform in [50, 10^4]) with a
learned index of 2^16 linear leaves per sorted array -- Algorithm 2's
counting loop over Algorithm 1, per-query uint32 counts plus the uint64
total.  The headline is the fastest of the plain 16-ary search, the learned
index and the autotuned choice (bits_count's AUTO, whose records the line
also reports); all are timed and reported side by side (with merge path).
L2 is flushed before every timed step.

Also reported on the same line (most important last, so that a reader of
the line's tail sees them): the random-read rates the search kernels are
set against, the exome-vs-reads workload (200,000 queries vs 20,000,000
reads: count forms, host-buffer count, build, one-shot build+count,
projection, enumeration), the 64 x 32 all-pairs count (from the query sets'
intervals, and from databases on both sides) and Monte-Carlo screen, the
100M database build, the headline's forms, and the Monte-Carlo
significance test (100,000 intervals vs 1,000,000, 10,000 shuffles per
launch: shuffles/s, placements/s, its L2 and issue rooflines).  Parity is
checked in the run: every headline count of a 4M-query sample and the
sorted arrays against the CPU oracle, all 10,000 Monte-Carlo totals and all
2,048 all-pairs totals (both forms) against the oracle's stored values.

The CPU oracle is timed on this host (rank 0) by the protocol both arms
share: count of a 4,000,000-query sample of the headline against the
oracle-sorted database with all cores, of a 200,000-query sample
single-threaded, and the oracle's database sort (std::sort) of 10,000,000
of its intervals, each as mean and sd over 5 runs.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--detail PATH]

Under torchrun (N > 1) the headline's queries and the Monte-Carlo test's
shuffles are split across the ranks (each rank keeps its own copy of the
database; no collective inside the timed region), so the job's total work
is fixed and "scaling" is "strong"; value is all ranks' queries divided by
the slowest rank's time.  The other workloads run on rank 0 only.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.join(ROOT, "tests"))

METRIC = "queries/s and MC shuffles/s on 1 B300, learned-index vs binary-search, bit-exact"
HEADLINE = ("learned-index BITS at scale: 100,000,000 uniform queries vs 100,000,000 intervals "
            "(80% from 1000 Gaussians sigma U[1e3,1e6], 20% uniform) on a 3.0 Gbp line, lengths "
            "log-uniform [50,1e4], 2^16 linear leaves per sorted array")
SAMPLE_ALL, SAMPLE_ONE, SAMPLE_BUILD, PROTOCOL_RUNS = 4_000_000, 200_000, 10_000_000, 5


def config_dict(world: int) -> dict:
    """The headline's config, identical in both arms."""
    return {"workload": HEADLINE,
            "method": "fastest of plain 16-ary search, learned index and the autotuned choice "
                      "(all in forms)",
            "l2": "flushed (256 MB write) before every timed step; queries 800 MB > L2",
            "parallelism": f"dp{world}: queries and shuffles split across ranks, database "
                           "replicated, no collective in the timed region"}


def sig(x, digits: int = 4):
    """Round for the compact JSON line."""
    if x is None or isinstance(x, (bool, str)):
        return x
    if isinstance(x, dict):
        return {k: sig(v, digits) for k, v in x.items()}
    if isinstance(x, (list, tuple)):
        return [sig(v, digits) for v in x]
    if isinstance(x, int):
        return x
    return float(f"{x:.{digits}g}")


# ---------------------------------------------------------------------------- helpers

def env_rank():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), \
        int(os.environ.get("LOCAL_RANK", "0"))


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def tree_levels(n: int, top_log2: int = 12) -> int:
    """Levels of the 16-ary tree a search reads below the shared-memory top
    (one 64-byte node each) for a database of n intervals."""
    cap, length, levels = (1 << top_log2) - 1, n, 0
    while length > cap and levels < 5:
        length = (length + 15) // 16
        levels += 1
    return levels


def source_digest(paths):
    h = hashlib.sha256()
    for p in paths:
        with open(os.path.join(ROOT, p), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_value(profile: str, field: str, sources):
    """A number recorded in profiles/<profile>.md for this exact kernel source."""
    path = os.path.join(ROOT, "profiles", f"{profile}.md")
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"source_digest:\s*([0-9a-f]+)", text)
    t = re.search(field + r":\s*([0-9.eE+]+)", text)
    if not m or not t or m.group(1) != source_digest(sources):
        return None
    return float(t.group(1))


def mean_sd(xs):
    return {"mean": statistics.fmean(xs), "sd": statistics.stdev(xs) if len(xs) > 1 else 0.0,
            "runs": len(xs), "values": list(xs)}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons, sampled every 50 ms (read only)."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,utilization.gpu,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "50"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self, t0, t1):
        rows = []
        for ts, line in self.lines:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append((ts, float(parts[1]), float(parts[2]), float(parts[3]),
                             float(parts[4]), parts[5:9]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"]}
        inside = [r for r in rows if t0 - 0.25 <= r[0] <= t1 + 0.25]
        loaded = [r for r in inside if r[4] > 0] or inside or rows
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in loaded for i, v in enumerate(r[5])
                          if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in loaded),
                "sm_max_mhz": max(r[2] for r in loaded), "reasons": reasons,
                "samples": len(loaded), "samples_in_timed_region": len(inside)}


# ------------------------------------------------------------- the oracle protocol

def oracle_protocol(o, a4, b4, bs4, be4, cores: int) -> dict:
    """Both arms time the CPU oracle this way: count of a 4M-query sample of
    the headline against the oracle-sorted 100M database with all cores and
    of a 200k sample single-threaded, and the oracle's sort of 10M of the
    database's intervals (single-threaded std::sort of both words), each 5
    runs after one untimed run, as rates with mean and sd."""
    def rate(fn, units):
        fn()  # one untimed run first: page-ins and thread start-up
        xs = []
        for _ in range(PROTOCOL_RUNS):
            t = time.perf_counter()
            fn()
            xs.append(units / (time.perf_counter() - t))
        return mean_sd(xs)
    s_all, s_one, b_sub = a4[:SAMPLE_ALL], a4[:SAMPLE_ONE], b4[:SAMPLE_BUILD]
    return {
        "count_all_cores": rate(lambda: o.count_sorted(s_all, bs4, be4, threads=cores), SAMPLE_ALL),
        "count_one_thread": rate(lambda: o.count_sorted(s_one, bs4, be4, threads=1), SAMPLE_ONE),
        "build_one_thread": rate(lambda: o.build(b_sub), SAMPLE_BUILD),
        "units": "queries/s (count), intervals/s (build)",
        "cores": cores}


def cpu_baseline_from(proto: dict) -> dict:
    c = proto["count_all_cores"]
    return {"value": c["mean"], "unit": "queries/s", "cores": proto["cores"], "kind": "oracle",
            "sample": f"first {SAMPLE_ALL:,} headline queries against the full oracle-sorted "
                      f"database, std::thread over all cores, mean of {c['runs']} runs "
                      f"(sd {c['sd']:.3g}); single thread {proto['count_one_thread']['mean']:.3g} "
                      f"q/s; oracle sort {proto['build_one_thread']['mean']:.3g} intervals/s"}


# ------------------------------------------------------------------ reference arm

def run_reference(args):
    """The CPU oracle, as it stands, on this host's cores: same metric and config."""
    rank, world, _ = env_rank()
    if rank != 0:
        return
    import bits_synth
    import oracle
    o = oracle.get()
    a4, b4 = bits_synth.config4()
    bs4, be4 = o.build(b4)
    cores = os.cpu_count() or 1
    n_samples = a4.shape[0] // SAMPLE_ALL

    def step(i):
        k = i % n_samples
        o.count_sorted(a4[k * SAMPLE_ALL:(k + 1) * SAMPLE_ALL], bs4, be4, threads=cores)

    for i in range(args.warmup):
        step(i)
    times = []
    for i in range(args.steps):
        t = time.perf_counter()
        step(args.warmup + i)
        times.append(time.perf_counter() - t)
    per_step = statistics.fmean(times)
    qps = SAMPLE_ALL / per_step
    proto = oracle_protocol(o, a4, b4, bs4, be4, cores)
    cpu = cpu_baseline_from(proto)
    cpu["value"] = qps
    cpu["sample"] = (f"{SAMPLE_ALL:,} headline queries per step (a different slice each step) "
                     "against the full oracle-sorted database, all cores")
    line = {
        "impl": "reference", "metric": METRIC, "value": qps, "unit": "queries/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": per_step * 1e3, "higher_is_better": True,
        "scaling": "strong", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": config_dict(world), "cpu_baseline": cpu,
        "e2e": {"value": qps, "unit": "queries/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
        "protocol": sig(proto),
    }
    print(json.dumps(line))


# -------------------------------------------------------------------------- our arm

def read_tuning(path: str) -> list:
    """The autotuner's records of this run (BITS_AUTOTUNE_CACHE lines)."""
    if not os.path.exists(path):
        return []
    out = []
    for ln in open(path).read().splitlines():
        f = ln.split()
        if len(f) >= 6:
            out.append({"kind": f[1], "log2_queries": int(f[2]), "log2_db": int(f[3]),
                        "flags": int(f[4]), "values": [int(x) for x in f[5:]]})
    return out


def run_ours(args):
    # The autotuner records its choices in a fresh file for this run; the
    # line reports them (kind "count": method, top raise, threads per CTA;
    # "mc": shuffles and intervals per work unit, top raise; "allpairs":
    # queries per work unit).
    tune_path = os.path.join("/tmp", f"bits_autotune_{os.getpid()}.txt")
    if os.path.exists(tune_path):
        os.remove(tune_path)
    os.environ["BITS_AUTOTUNE_CACHE"] = tune_path
    import torch

    import bits_synth
    import goldens
    import oracle
    import paper_1208_3407_b300 as bits
    from paper_1208_3407_b300 import probe, sharding

    rank, world, local = env_rank()
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    lead = rank == 0
    dev = torch.device("cuda", local)
    hbm_peak, peak_kind = peaks()
    o = oracle.get()
    cores = os.cpu_count() or 1

    def barrier():
        if dist is not None:
            dist.barrier()

    def max_over_ranks(x: float) -> float:
        if dist is None:
            return x
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        return float(t.item())

    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)  # 256 MB > L2
    stream = torch.cuda.current_stream()

    def to_dev(x):
        return torch.from_numpy(np.ascontiguousarray(x, dtype=np.uint32)).to(dev)

    def timed(fn, steps, warmup, all_ranks=True):
        """Mean device ms of fn over `steps` runs (L2 flushed before each),
        the kernels it launched per step, and the host time window."""
        for _ in range(warmup):
            fn()
        torch.cuda.synchronize()
        if all_ranks:
            barrier()
        torch.cuda.synchronize()
        l0 = bits.kernel_launches()
        ms = 0.0
        t0 = time.time()
        for _ in range(steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            ms += e0.elapsed_time(e1)
        torch.cuda.synchronize()
        t1 = time.time()
        if all_ranks:
            barrier()
            return max_over_ranks(ms / steps), (bits.kernel_launches() - l0) / steps, (t0, t1)
        return ms / steps, (bits.kernel_launches() - l0) / steps, (t0, t1)

    # Random 64-byte node reads: from DRAM (4 GiB buffer) -- the bound of the
    # searches on databases larger than L2 -- and from L2 (32 MiB buffer), the
    # bound of the Monte-Carlo kernels; best of three each.
    rand_peak = max(probe.probe_random_reads(4 << 30, 1 << 25, device=dev) for _ in range(3))
    l2_peak = max(probe.probe_random_reads(32 << 20, 1 << 25, device=dev) for _ in range(3))
    torch.cuda.empty_cache()

    vis = os.environ.get("CUDA_VISIBLE_DEVICES", "").split(",")[0]
    sampler = ClockSampler(int(vis) if vis.isdigit() else local)
    sampler.start()
    detail = {}

    # ================= headline: 100M queries vs 100M intervals ================
    a4_np, b4_np = bits_synth.config4()
    n4 = a4_np.shape[0]
    lo4, hi4 = sharding.shard_bounds(n4, rank, world)
    b4 = to_dev(b4_np)
    # Five builds of the 100M database, alternately with and without the
    # learned index; the first (which also grows the memory pool) is not
    # timed, the last is kept for the counts.
    build4 = []
    for i in range(5):
        rmi = i % 2 == 0
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        d = bits.Database(b4, rmi_leaves_log2=16 if rmi else 0)
        e1.record(stream)
        e1.synchronize()
        if i > 0:
            build4.append((int(rmi), e0.elapsed_time(e1)))
        if i < 4:
            d.free()
    db4 = d                                             # plain levels + learned index
    del b4
    a4 = to_dev(a4_np[lo4:hi4])
    n_mine = hi4 - lo4
    c4 = torch.empty(n_mine, dtype=torch.uint32, device=dev)
    t4 = torch.empty(1, dtype=torch.uint64, device=dev)
    forms = {}
    totals4 = {}
    for name, m, per_query in (("search", bits.METHOD_SEARCH, True),
                               ("rmi", bits.METHOD_RMI, True),
                               ("mergepath", bits.METHOD_MERGEPATH, True),
                               ("search_total_only", bits.METHOD_SEARCH, False)):
        out_c = c4 if per_query else False
        ms, launches, _ = timed(lambda m=m, out_c=out_c: db4.count(a4, counts=out_c, total=t4,
                                                                   method=m, check=False),
                                args.steps, args.warmup)
        totals4[name] = int(t4.cpu().numpy()[0])
        forms[name] = {"ms": ms, "queries_per_s": n4 / (ms * 1e-3), "gpu_launches": launches}
    db4.check()
    assert len(set(totals4.values())) == 1, totals4
    db4.count(a4, counts=c4, total=t4, check=True)           # AUTO: tunes this size class
    auto_ms, _, _ = timed(lambda: db4.count(a4, counts=c4, total=t4, check=False), args.steps,
                          args.warmup)
    forms["auto"] = {"ms": auto_ms, "queries_per_s": n4 / (auto_ms * 1e-3)}
    head = min(("search", "rmi", "auto"), key=lambda k: forms[k]["ms"])
    head_m = {"search": bits.METHOD_SEARCH, "rmi": bits.METHOD_RMI, "auto": bits.METHOD_AUTO}[head]
    head_ms, launches, window = timed(lambda: db4.count(a4, counts=c4, total=t4, method=head_m,
                                                        check=False), args.steps, args.warmup)
    db4.check()
    clocks = sampler.summary(*window)
    combined = sharding.combine_totals(int(t4.cpu().numpy()[0])) if dist else \
        int(t4.cpu().numpy()[0])

    # Parity of the headline against the oracle: the sorted arrays, and every
    # count of the first 4M queries (the oracle sorts the database itself).
    parity = {}
    bs4 = be4 = None
    if lead:
        bs4, be4 = o.build(b4_np)
        gs, ge = db4.sorted_arrays()
        parity["headline_sorted_arrays"] = bool(np.array_equal(gs.cpu().numpy(), bs4) and
                                                np.array_equal(ge.cpu().numpy(), be4))
        k = min(SAMPLE_ALL, n_mine)
        oc, _ = o.count_sorted(a4_np[lo4:lo4 + k], bs4, be4, threads=cores)
        parity["headline_counts_4m_sample"] = bool(np.array_equal(c4[:k].cpu().numpy(), oc))
    if dist is not None and lead:
        full = torch.empty(1, dtype=torch.uint64, device=dev)
        db4.count(to_dev(a4_np), counts=False, total=full, method=bits.METHOD_SEARCH)
        parity["sharded_total_equals_single_gpu"] = int(full.cpu().numpy()[0]) == combined

    # End to end through the C ABI with host buffers: bits_count_host reads the
    # page-locked queries and writes the page-locked counts in place over the
    # bus and copies the total back -- every byte crosses inside the timed step.
    a_host = torch.from_numpy(np.ascontiguousarray(a4_np[lo4:hi4])).pin_memory()
    counts_host = torch.zeros(n_mine, dtype=torch.uint32).pin_memory()
    total_host = torch.zeros(1, dtype=torch.uint64).pin_memory()

    # Host buffers: the plain search and the learned index read and write
    # them in place over the bus (merge path would stage them).  The faster
    # of the plain search and the headline's method is reported.
    e2e_forms = {}
    for name, m in (("search_in_place", bits.METHOD_SEARCH), ("headline_method", head_m)):
        if name == "headline_method" and head_m == bits.METHOD_SEARCH:
            continue
        ms, l, _ = timed(lambda m=m: db4.count_host(a_host, counts=counts_host, total=total_host,
                                                     method=m, check=False), args.steps, args.warmup)
        e2e_forms[name] = (ms, l)
    e2e_name = min(e2e_forms, key=lambda k: e2e_forms[k][0])
    e2e_ms, e2e_launches = e2e_forms[e2e_name]
    # The host link's own rate for the same bytes: a copy-engine transfer of
    # the page-locked queries into device memory (the bound of the call
    # above, whose 8-byte query reads dominate its traffic).
    q_dev = torch.empty_like(a_host, device=dev)
    link_ms, _, _ = timed(lambda: q_dev.copy_(a_host, non_blocking=True), 3, 2)
    link_gbs = a_host.numel() * 4 / (link_ms * 1e-3) / 1e9
    del q_dev
    db4.check()
    parity["headline_host_buffers"] = bool(
        np.array_equal(counts_host.numpy(), c4.cpu().numpy()) and
        int(total_host.numpy()[0]) == int(t4.cpu().numpy()[0]))
    del a_host, counts_host

    rmi_src = ["paper_1208_3407_b300/csrc/search.cuh", "paper_1208_3407_b300/csrc/rmi_search.cuh",
               "paper_1208_3407_b300/csrc/rmi.cu"]
    search_src = ["paper_1208_3407_b300/csrc/search.cuh", "paper_1208_3407_b300/csrc/count.cu"]
    tuned_auto = [r for r in read_tuning(tune_path)
                  if r["kind"] == "count" and r["flags"] >> 2 == 0 and r["log2_queries"] == 27]
    head_method = head if head != "auto" else \
        ({1: "search", 2: "rmi", 3: "mergepath"}.get(tuned_auto[0]["values"][0], "search")
         if tuned_auto else "search")
    kernel = "k_count_rmi" if head_method == "rmi" else "k_count_search"
    src = rmi_src if head_method == "rmi" else search_src
    # DRAM bytes per query from the ncu capture named in profiles/ (valid
    # while the kernel's sources are unchanged), times this rank's queries.
    traffic_q = profiled_value(f"{kernel}_100m", "dram_bytes_per_query", src)
    achieved = 76.0 * n4 / (head_ms * 1e-3) / 1e9
    roofline = {"bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                "frac": achieved / hbm_peak,
                "traffic": traffic_q * n_mine if traffic_q else None,
                "peak_source": peak_kind, "kernel": kernel,
                "algorithmic_bytes_per_query": 76}
    random_access = {"bound": "random 64-B node reads from DRAM (probe, 4 GiB)",
                     "achieved": 2.0 * n4 / (head_ms * 1e-3), "peak": rand_peak,
                     "unit": "nodes/s", "frac": 2.0 * n4 / (head_ms * 1e-3) / rand_peak,
                     "nodes_per_query": 2}
    db4.free()
    del a4, c4

    # ================= Monte-Carlo significance test (config of Table 1) ========
    g3, a3_np, b3_np = bits_synth.config3()
    co_np, cl_np = bits_synth.mc_contig_table(g3)
    db3 = bits.Database(to_dev(b3_np), rmi_leaves_log2=16)
    a3, co, cl = to_dev(a3_np), to_dev(co_np), to_dev(cl_np)
    n_sh = 10_000
    s0, s1 = sharding.shuffle_range(n_sh, rank, world)
    totals3 = torch.empty(max(s1 - s0, 1), dtype=torch.uint64, device=dev)
    mc_forms = {}
    mc_windows = {}
    gobs, gk, _, gtot = goldens.read_mc_fullsize()
    for name, m in (("search", bits.METHOD_SEARCH), ("rmi", bits.METHOD_RMI)):
        def mc_step(m=m):
            db3.mc(a3, co, cl, seed=7, shuffle_begin=s0, shuffle_end=s1, totals=totals3, method=m)

        ms, l, win = timed(mc_step, args.steps, args.warmup)
        mc_windows[name] = win
        mc_forms[name] = {"ms": ms, "shuffles_per_s": n_sh / (ms * 1e-3),
                          "placements_per_s": n_sh * a3_np.shape[0] / (ms * 1e-3),
                          "gpu_launches": l}
        if dist is not None:
            tot, st = sharding.sharded_mc(db3, a3, co, cl, seed=7, n_shuffles=n_sh, method=m)
            t_all, k_all, obs_all = tot.cpu().numpy(), st["k_ge"], st["observed"]
        else:
            _, obs_all, k_all, _ = db3.mc(a3, co, cl, seed=7, shuffle_end=n_sh, totals=totals3,
                                          method=m)
            t_all = totals3.cpu().numpy()
        parity[f"mc_{name}_all_10000_totals"] = bool(
            np.array_equal(t_all, gtot) and obs_all == gobs and k_all == gk)
    best_mc = min(mc_forms, key=lambda k: mc_forms[k]["ms"])
    mc_src = ["paper_1208_3407_b300/csrc/mc.cu", "paper_1208_3407_b300/csrc/mc_unit.cuh",
              "paper_1208_3407_b300/csrc/search.cuh", "paper_1208_3407_b300/csrc/philox.cuh"]
    wi = profiled_value("k_mc_search", "warp_instructions_per_launch", mc_src)
    nodes_pp = 2 * tree_levels(b3_np.shape[0])
    mc_l2 = {"bound": "random 64-B node reads from L2 (probe, 32 MiB)",
             "achieved": nodes_pp * n_sh * a3_np.shape[0] / (mc_forms["search"]["ms"] * 1e-3),
             "peak": l2_peak, "unit": "nodes/s", "nodes_per_placement": nodes_pp}
    mc_l2["frac"] = mc_l2["achieved"] / l2_peak
    db3.free()
    del a3, co, cl, totals3

    # ================= rank 0 only: the other workloads ==========================
    sections = {}
    if lead:
        sections = other_workloads(args, bits, bits_synth, goldens, o, torch, dev, to_dev,
                                   timed, flush, stream, hbm_peak, l2_peak, parity, detail)
    sampler.stop()

    def issue_roofline(warp_instr, ms, window):
        ck = sampler.summary(*window)
        mhz = ck.get("sm_mhz") or clocks.get("sm_mhz")
        if warp_instr is None or not mhz:
            return None
        peak = 148 * 4 * mhz * 1e6
        ach = warp_instr / (ms * 1e-3)
        return {"bound": "alu", "achieved": ach, "peak": peak, "unit": "warp-instructions/s",
                "frac": ach / peak, "sm_mhz": mhz}

    mc_issue = issue_roofline(wi, mc_forms["search"]["ms"], mc_windows["search"])

    # ================= CPU baseline: the oracle protocol ==========================
    cpu = proto = None
    if lead:
        proto = oracle_protocol(o, a4_np, b4_np, bs4, be4, cores)
        cpu = cpu_baseline_from(proto)

    value = n4 / (head_ms * 1e-3)
    line = {
        "metric": METRIC, "value": value, "unit": "queries/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": head_ms,
        "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "u32",
        "data": "synthetic (seeded generator; the paper's datasets are not available)",
        "config": config_dict(world),
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": {"value": n4 / (e2e_ms * 1e-3), "unit": "queries/s",
                "h2d_bytes_per_step": int(n4 * 8), "d2h_bytes_per_step": int(n4 * 4 + 8),
                "ms_per_step": e2e_ms, "gpu_launches": e2e_launches,
                "call": "bits_count_host on page-locked queries and counts (read and written "
                        "in place by the search kernel over the bus) + the total copied back",
                "form": e2e_name, "forms_ms": sig({k: v[0] for k, v in e2e_forms.items()}),
                "host_link": sig({"h2d_gbs": link_gbs, "h2d_ms_for_queries": link_ms,
                                  "frac": link_ms / e2e_ms,
                                  "what": "copy-engine transfer of the same page-locked "
                                          "queries to the device, timed alone"})},
        "gpu_launches": launches,
        "clocks": clocks,
        "headline_form": head,
        "roofline_random_access": sig(random_access),
        "probe": sig({"dram_nodes_per_s": rand_peak, "l2_nodes_per_s": l2_peak}),
    }
    line.update(sig(sections))
    line["build_100m_ms"] = sig({"plain": statistics.fmean(t for r, t in build4 if not r),
                                 "with_learned_index": statistics.fmean(t for r, t in build4 if r)})
    line["protocol"] = sig(proto) if proto else None
    # The line carries the autotuner's choices for the headline and exome
    # counts, the Monte-Carlo test and the all-pairs screen; every record of
    # the run (per-method records and the screen's per-database counts) goes
    # to the detail file.
    tuning_all = read_tuning(tune_path)
    line["tuning"] = [r for r in tuning_all if r["kind"] != "count" or (
        r["flags"] >> 2 == 0 and (r["log2_queries"], r["log2_db"]) in ((27, 27), (18, 25)))]
    detail["tuning_all"] = tuning_all
    line["forms"] = sig({k: {"ms": v["ms"], "qps": v["queries_per_s"]} for k, v in forms.items()})
    line["mc"] = sig({
        "workload": "100k x 1M, 10,000 shuffles per launch (Table 1 corner)",
        "shuffles_per_s": mc_forms[best_mc]["shuffles_per_s"],
        "placements_per_s": mc_forms[best_mc]["placements_per_s"], "form": best_mc,
        "forms": {k: {"ms": v["ms"], "shuffles_per_s": v["shuffles_per_s"]}
                  for k, v in mc_forms.items()},
        "roofline_l2_frac": mc_l2["frac"],
        "roofline_issue_frac": mc_issue["frac"] if mc_issue else None,
        "paper": "357 shuffles/s (Table 1, 1e5 x 1e4, 2012 GPU)"})
    line["parity"] = parity
    detail.update({"line": line, "forms_full": forms, "mc_forms": mc_forms, "mc_l2": mc_l2,
                   "mc_issue": mc_issue, "protocol": proto, "build4": build4})
    if lead:
        if args.detail:
            with open(args.detail, "w") as f:
                json.dump(detail, f, indent=1, default=str)
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()


def other_workloads(args, bits, bits_synth, goldens, o, torch, dev, to_dev, timed, flush, stream,
                    hbm_peak, l2_peak, parity, detail):
    """Exome-vs-reads count forms, build, one-shot, host buffers, projection and
    enumeration; the 10k x 10k count; the 64 x 32 all-pairs count and screen."""
    out = {}
    # ---- 10,000 x 10,000 on one 1 Mbp contig (launch-bound) -------------------
    a1_np, b1_np = bits_synth.config1()
    db1 = bits.Database(to_dev(b1_np))
    a1 = to_dev(a1_np)
    c1 = torch.empty(a1_np.shape[0], dtype=torch.uint32, device=dev)
    t1 = torch.empty(1, dtype=torch.uint64, device=dev)
    ms1, _, _ = timed(lambda: db1.count(a1, counts=c1, total=t1, method=bits.METHOD_SEARCH,
                                        check=False), args.steps, args.warmup, all_ranks=False)
    oc1, _ = o.count_brute(a1_np, b1_np)
    parity["small_10k_brute_force"] = bool(np.array_equal(c1.cpu().numpy(), oc1))
    db1.free()
    out["small_10k_us"] = ms1 * 1e3

    # ---- exome-vs-reads: 200,000 queries vs 20,000,000 reads ------------------
    genome, a_np, b_np = bits_synth.config2()
    n_a, n_b = a_np.shape[0], b_np.shape[0]
    a, b = to_dev(a_np), to_dev(b_np)
    builds = []
    for i in range(args.warmup + args.steps):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        d = bits.Database(b)
        e1.record(stream)
        e1.synchronize()
        if i >= args.warmup:
            builds.append(e0.elapsed_time(e1))
        d.free()
    build_ms = statistics.fmean(builds)
    one_c = torch.empty(n_a, dtype=torch.uint32, device=dev)
    one_t = torch.empty(1, dtype=torch.uint64, device=dev)

    def one_shot():
        d = bits.Database(b)
        d.count(a, counts=one_c, total=one_t, method=bits.METHOD_SEARCH, check=False)
        d.free()

    one_ms, _, _ = timed(one_shot, args.steps, args.warmup, all_ranks=False)
    db = bits.Database(b, rmi_leaves_log2=16)
    counts = torch.empty(n_a, dtype=torch.uint32, device=dev)
    total = torch.empty(1, dtype=torch.uint64, device=dev)
    ex_forms = {}
    for name, m in (("search", bits.METHOD_SEARCH), ("rmi", bits.METHOD_RMI)):
        ms, _, _ = timed(lambda m=m: db.count(a, counts=counts, total=total, method=m,
                                              check=False), args.steps, args.warmup,
                         all_ranks=False)
        ex_forms[name] = ms
    db.check()
    idx = np.random.default_rng(0).choice(n_a, size=256, replace=False)
    oc, _ = o.count_brute(a_np[idx], b_np)
    parity["exome_counts_256_brute_force"] = bool(np.array_equal(counts.cpu().numpy()[idx], oc))
    a_host = torch.from_numpy(a_np.astype(np.uint32)).pin_memory()
    ch = torch.zeros(n_a, dtype=torch.uint32).pin_memory()
    th = torch.zeros(1, dtype=torch.uint64).pin_memory()
    host_ms, _, _ = timed(lambda: db.count_host(a_host, counts=ch, total=th,
                                                method=bits.METHOD_SEARCH, check=False),
                          args.steps, args.warmup, all_ranks=False)
    db.free()
    ex = {"count_us": {k: v * 1e3 for k, v in ex_forms.items()},
          "count_qps": n_a / (min(ex_forms.values()) * 1e-3),
          "host_buffers_us": host_ms * 1e3, "build_20m_ms": build_ms,
          "build_keys_per_s": 2 * n_b / (build_ms * 1e-3),
          # 36 B per key (four 8-bit passes of 8 B plus the split's 4 B) against
          # the copy bandwidth; the passes are bound by shared memory, not HBM
          "build_hbm_frac": 36.0 * 2 * n_b / (build_ms * 1e-3) / 1e9 / hbm_peak,
          "one_shot_ms": one_ms}

    # projection of 20M chromosome-local closed reads (12 B read + 8 B written each)
    pc_np, ps_np, pe_np = bits_synth.local_intervals(genome, n_b, seed=5, lo=100, hi=100,
                                                     closed=True)
    pc, ps, pe = to_dev(pc_np), to_dev(ps_np), to_dev(pe_np)
    pco, pcl = to_dev(genome.offsets), to_dev(genome.lengths)
    p_out = torch.empty((n_b, 2), dtype=torch.uint32, device=dev)
    proj_ms, _, _ = timed(lambda: bits.project(ps, pe, contig=pc, contig_off=pco, contig_len=pcl,
                                               closed=True, out=p_out),
                          args.steps, args.warmup, all_ranks=False)
    pidx = np.random.default_rng(1).choice(n_b, size=4096, replace=False)
    exp_p, _ = o.project(pc_np[pidx], ps_np[pidx], pe_np[pidx], genome.offsets, genome.lengths,
                         closed=True)
    parity["projection_4096_sample"] = bool(np.array_equal(p_out.cpu().numpy()[pidx], exp_p))
    ex["project_ms"] = proj_ms
    ex["project_hbm_frac"] = 20.0 * n_b / (proj_ms * 1e-3) / 1e9 / hbm_peak
    del pc, ps, pe, p_out

    # enumeration of every intersecting pair
    db_en = bits.Database(b, enumerate=True)
    en_ms, _, _ = timed(lambda: db_en.enumerate(a, check=False), args.steps, args.warmup,
                        all_ranks=False)
    off_g, pairs_g = db_en.enumerate(a)
    eidx = np.random.default_rng(2).choice(n_a, size=64, replace=False)
    eoff, epairs = o.enumerate_scan(a_np[eidx], b_np)
    off_np, pairs_np = off_g.cpu().numpy(), pairs_g.cpu().numpy()
    ok = True
    for k, i in enumerate(eidx):
        ok &= bool(np.array_equal(pairs_np[int(off_np[i]):int(off_np[i + 1]), 1],
                                  epairs[int(eoff[k]):int(eoff[k + 1]), 1]))
    parity["enumeration_64_queries"] = ok
    ex["enumerate_ms"] = en_ms
    ex["enumerate_pairs_per_s"] = int(off_np[-1]) / (en_ms * 1e-3)
    db_en.free()
    del off_g, pairs_g, a, b
    out["exome"] = ex

    # ---- all-pairs: 64 query sets x 32 databases ------------------------------
    g5, a5_np, b5_np = bits_synth.config5()
    dbs5 = [bits.Database(to_dev(x), rmi_leaves_log2=16) for x in b5_np]
    a5 = [to_dev(x) for x in a5_np]
    m5 = torch.empty((len(a5), len(dbs5)), dtype=torch.uint64, device=dev)
    bits.count_matrix(dbs5, a5, out=m5)          # autotunes and captures the graph
    ms5, _, _ = timed(lambda: bits.count_matrix(dbs5, a5, out=m5), max(3, min(args.steps, 5)), 3,
                      all_ranks=False)
    parity["allpairs_all_2048_totals"] = bool(np.array_equal(m5.cpu().numpy(),
                                                             goldens.read_allpairs_fullsize()))
    n_q5 = sum(x.shape[0] for x in a5_np)
    ap_nodes = sum(x.shape[0] * 2 * tree_levels(y.shape[0]) for x in a5_np for y in b5_np)
    out["allpairs"] = {"ms": ms5, "pair_counts_per_s": n_q5 * len(dbs5) / (ms5 * 1e-3),
                       "roofline_l2_frac": ap_nodes / (ms5 * 1e-3) / l2_peak}
    # The same matrix with the 64 query sets built as databases too
    # (bits_count_matrix_db): each pair counted from its smaller side's sorted
    # keys.  The sets' builds are setup, timed on their own.
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    adbs5 = [bits.Database(x) for x in a5]
    e1.record(stream)
    e1.synchronize()
    build_sets_ms = e0.elapsed_time(e1)
    m5d = torch.empty_like(m5)
    bits.count_matrix_db(adbs5, dbs5, out=m5d)   # tunes and captures the graph
    ms5d, _, _ = timed(lambda: bits.count_matrix_db(adbs5, dbs5, out=m5d),
                       max(3, min(args.steps, 5)), 3, all_ranks=False)
    parity["allpairs_db_all_2048_totals"] = bool(np.array_equal(m5d.cpu().numpy(),
                                                                goldens.read_allpairs_fullsize()))
    n_keys5 = sum(min(x.shape[0], y.shape[0]) for x in a5_np for y in b5_np)
    out["allpairs"]["from_databases"] = {
        "ms": ms5d, "build_query_sets_ms": build_sets_ms,
        "pair_counts_per_s": n_q5 * len(dbs5) / (ms5d * 1e-3),
        # each pair's smaller side, merged or searched against the larger
        "key_pairs": n_keys5, "key_pairs_per_s": n_keys5 / (ms5d * 1e-3)}
    for d in adbs5:
        d.free()
    del adbs5, m5d
    # ---- Monte-Carlo screen over the same sets: 4 shuffles per step -------------
    co5, cl5 = bits_synth.mc_contig_table(g5)
    dco5, dcl5 = to_dev(co5), to_dev(cl5)
    nsh5 = 4
    scr = (torch.empty((len(a5), len(dbs5)), dtype=torch.uint64, device=dev),
           torch.empty((len(a5), len(dbs5), nsh5), dtype=torch.uint64, device=dev),
           torch.empty((len(a5), len(dbs5), 8), dtype=torch.uint64, device=dev))

    def screen_step():
        bits.mc_matrix(dbs5, a5, dco5, dcl5, seed=17, shuffle_end=nsh5, out=scr)

    screen_step()
    ms_scr, _, _ = timed(screen_step, 3, 3, all_ranks=False)
    for d in dbs5:
        d.check()
    i_s = int(np.argmin([x.shape[0] for x in a5_np]))
    bs5, be5 = o.build(b5_np[7])
    ot, oo, _, _ = o.mc(a5_np[i_s], co5, cl5, bs5, be5, seed=17, s_begin=0, s_end=nsh5,
                        threads=os.cpu_count() or 1, set_index=i_s)
    parity["screen_sample_pair"] = bool(np.array_equal(scr[1][i_s, 7].cpu().numpy(), ot) and
                                        int(scr[0][i_s, 7].cpu()) == oo)
    out["mc_screen"] = {"ms": ms_scr,
                        "placements_per_s": n_q5 * len(dbs5) * nsh5 / (ms_scr * 1e-3)}
    for d in dbs5:
        d.free()
    detail["other"] = out
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--detail", default=None, help="also write every measured number here")
    args = ap.parse_args()
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
