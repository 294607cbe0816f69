"""Benchmark of the Motifs-k hot path on GB300.

A step is one pass of the whole path over one batch: randomise R null graphs,
rebuild their CSRs, plan, enumerate + classify + count every connected k-set of
the original and the R nulls in one launch, z-scores.  The default workload is
the k=5 null-model batch (directed Chung-Lu n=1,500, m=6,000, gamma 2.2, 10%
reciprocal, plus 256 arc-swap nulls with 10*m attempts each, seeds 1..256).

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import synthetic as syn  # noqa: E402

# Root sample the CPU oracle times (k-sets whose smallest vertex is in it):
# about 7-12 s of oracle work on 16 host cores for the two null-model
# workloads (1.3e8 and 2.1e7 k-sets), the whole graph for the small ones.
CPU_SAMPLE = {"nullmodel_k5": (30, 200), "nullmodel_k6": (60, 200), "chunglu_k4": (0, 2000),
              "uniform_k3": (0, 300)}
INT32_LANES_PER_SM = 128


def _peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            return json.load(f), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            threading.Thread(target=self._read, daemon=True).start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ------------------------------------------------------------------ reference arm (oracle)


def run_reference(args, world, rank):
    import oracle

    if rank != 0:
        return
    w = syn.WORKLOADS[args.workload]
    k = w["k"]
    g = syn.workload_graph(args.workload)
    a, b = CPU_SAMPLE[args.workload]
    roots = np.arange(a, min(b, g.n))
    cores = oracle.default_threads()
    for _ in range(args.warmup):
        oracle.count_roots(g, k, roots)
    times, sets = [], 0
    for _ in range(args.steps):
        t0 = time.perf_counter()
        _, sets = oracle.count_roots(g, k, roots)
        times.append(time.perf_counter() - t0)
    total = sum(times)
    value = sets * args.steps / total
    sample = (f"k-sets of the original graph whose smallest vertex is in [{a},{b}) "
              f"({sets} sets per step)")
    line = {"impl": "reference", "metric": "k-subgraphs classified/s", "value": value,
            "unit": "subgraphs/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1000 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
            "config": _config(args, w, world),
            "cpu_baseline": {"value": value, "unit": "subgraphs/s", "cores": cores,
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "subgraphs/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def _strip_comments(src: str) -> str:
    """C/C++ source without comments and with whitespace runs collapsed (string
    and character literals kept), so that a comment-only edit keeps the hash."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if src.startswith("//", i):
            j = src.find("\n", i)
            i = n if j < 0 else j
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
            out.append(" ")
        elif c in "\"'":
            j = i + 1
            while j < n and src[j] != c:
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        else:
            out.append(c)
            i += 1
    return " ".join("".join(out).split())


def _kernel_source_hash() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in ("count.cu", "count.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_1804_09741_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(_strip_comments(fh.read()).encode())
    return h.hexdigest()[:16]


COUNTERS_JSON = os.path.join(ROOT, "profiles", "k_count_counters.json")


def _captured(kind, method, workload, nulls):
    """An ncu capture of one k_count launch recorded in profiles/k_count_counters.json
    (entries keyed by what was captured: `kind` "traffic" for the full-size DRAM
    bytes, "gather" for the small-case load and reduction counters), only if it
    was taken from the current kernel source and the same launch; else None."""
    if not os.path.exists(COUNTERS_JSON):
        return None
    with open(COUNTERS_JSON) as f:
        entries = json.load(f).get("captures", [])
    src = _kernel_source_hash()
    for e in entries:
        if (e.get("kind") == kind and e.get("method") == method and e.get("workload") == workload
                and e.get("nulls") == nulls and e.get("source") == src):
            return e
    return None


def _captured_traffic(method, workload, nulls):
    """DRAM bytes per k_count launch (dram__bytes_read.sum + dram__bytes_write.sum)
    of a full-size capture of the current kernel, else None."""
    e = _captured("traffic", method, workload, nulls)
    return None if e is None else int(e["dram_bytes"])


def _config(args, w, world):
    nulls = w.get("nulls", 0) if args.nulls is None else args.nulls
    c = {"workload": args.workload, "k": w["k"], "n": w["n"], "m": w["m"],
         "gamma": w.get("gamma"), "dmax": w.get("dmax"), "reciprocity": w.get("recip"),
         "null_graphs": nulls, "swaps_per_null": 10 * w["m"] if nulls else 0,
         "graphs_per_step": 1 + nulls, "parallelism": f"replicas{world}",
         "null_model": getattr(args, "null_model", "arcswap"),
         "l2": "flushed between timed steps (256 MiB write)", "method": args.method}
    if getattr(args, "compact_table", False):
        c["table"] = "compact (199 x 2^18 slots)"
    return c


# ------------------------------------------------------------------ our arm


def run_ours(args, world, rank, local):
    import torch

    import paper_1804_09741_gb300 as mt
    from paper_1804_09741_gb300 import shard

    torch.cuda.set_device(local)
    mt.load_library()
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = syn.WORKLOADS[args.workload]
    k = w["k"]
    R = w.get("nulls", 0) if args.nulls is None else args.nulls
    g = syn.workload_graph(args.workload)
    stream = torch.cuda.current_stream()

    t0 = time.perf_counter()
    table = mt.table_build(k, compact=args.compact_table)
    table_ms = 1000 * (time.perf_counter() - t0)
    dg = mt.graph_from(g)
    C = table.num_classes
    seeds = shard.rank_seeds(R, rank) if R else None
    swaps = 10 * g.m

    method = mt.METHOD_CELLS if args.method == "cells" else mt.METHOD_ENUMERATE
    tuning = mt.make_tuning(method=method) if method else None
    tuned = None
    if R and not args.no_autotune:
        from paper_1804_09741_gb300 import autotune
        t_tune = time.perf_counter()
        tp = autotune.tune_batch(dg, table, g, swaps, probe_nulls=16, method=method,
                                 cache_path=None)
        tuning = mt.make_tuning(0.0, tp.warps_per_block, tp.split_scale, tp.stack_cap, method)
        tuned = {"warps_per_block": tp.warps_per_block, "split_scale": tp.split_scale,
                 "stack_cap": tp.stack_cap, "probe_count_ms": tp.ms,
                 "tune_s": time.perf_counter() - t_tune,
                 "source": "autotuner: 16-null probe batch, 8 candidates"}
    null_model = 1 if args.null_model == "dyad" else 0
    if R:
        batch = mt.Batch(dg, table, R, swaps, tuning, null_model=null_model)
        hists = torch.empty((R + 1, C), dtype=torch.int64, device="cuda")
        z = torch.empty(C, dtype=torch.float64, device="cuda")

        def step():
            batch.run(seeds, hists, z)
        launches_per_step = 9
    else:
        hists = torch.empty(C, dtype=torch.int64, device="cuda")

        def step():
            if tuning is None:
                mt.count(dg, table, hists)
            else:
                mt.count_tuned(dg, table, out=hists, method=method)
        launches_per_step = 5

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    subgraphs_per_step = int(mt.to_numpy_u64(hists).astype(np.uint64).sum())
    if R:
        assert batch.error() == 0, "device stack overflow"

    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    count_ms = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = ClockSampler(local)
    clocks.start()
    for i in range(args.steps):
        flush.fill_(i & 0xFF)
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        if R:
            count_ms.append(batch.phase_ms()[1])
    torch.cuda.synchronize()
    clk = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    all_subgraphs = subgraphs_per_step  # per step, all ranks (their null graphs differ)
    if dist:
        tt = torch.tensor([total_ms], device="cuda")
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        total_ms = float(tt.item())
        ts = torch.tensor([subgraphs_per_step], dtype=torch.int64, device="cuda")
        dist.all_reduce(ts, op=dist.ReduceOp.SUM)
        all_subgraphs = int(ts.item())
        dist.barrier()
    value = all_subgraphs * args.steps / (total_ms / 1000.0)

    # end to end through the public API with host buffers: load the graph from
    # host CSR, run the one-shot batch into host histograms and z-scores.
    e2e = None
    if not args.no_e2e:  # every rank its own batch; the slowest rank's time counts
        # inputs in pinned host memory, as a caller streaming graphs would keep them
        rp_t = torch.empty(g.n + 1, dtype=torch.int32, pin_memory=True)
        col_t = torch.empty(max(g.m, 1), dtype=torch.int32, pin_memory=True)
        rp_t.numpy()[:] = g.row_ptr
        col_t.numpy()[:g.m] = g.col
        rp, col = rp_t.numpy(), col_t.numpy()[:g.m]
        e2e_times = []
        if dist:
            dist.barrier()
        for _ in range(2):
            torch.cuda.synchronize()
            t1 = time.perf_counter()
            gg = mt.graph_load_csr(g.n, rp, col)
            if R:
                hh, zz = mt.count_batch(gg, table, seeds, swaps)
            else:
                hh = mt.count_host(gg, table)
            torch.cuda.synchronize()
            e2e_times.append(time.perf_counter() - t1)
            gg.free()
        assert int(hh.sum()) == subgraphs_per_step
        h2d = world * (rp.nbytes + col.nbytes + (seeds.nbytes if R else 0))
        d2h = world * ((R + 1) * C * 8 + (C * 8 if R else 0))
        e2e_s = min(e2e_times)
        if dist:
            te = torch.tensor([e2e_s], dtype=torch.float64, device="cuda")
            dist.all_reduce(te, op=dist.ReduceOp.MAX)
            e2e_s = float(te.item())
        e2e = {"value": all_subgraphs / e2e_s, "unit": "subgraphs/s",
               "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
               "ms_per_step": 1000 * e2e_s}

    cpu = None
    if not args.no_cpu_baseline and rank == 0 and world == 1:
        import oracle
        a, b = CPU_SAMPLE[args.workload]
        t1 = time.perf_counter()
        _, sets = oracle.count_roots(g, k, np.arange(a, min(b, g.n)))
        dt = time.perf_counter() - t1
        cpu = {"value": sets / dt, "unit": "subgraphs/s", "cores": oracle.default_threads(),
               "kind": "oracle",
               "sample": f"k-sets of the original graph with smallest vertex in [{a},{b}): "
                         f"{sets} sets in {dt:.1f} s"}

    peaks, src = _peaks()
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    sms = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = sms * INT32_LANES_PER_SM * sm_mhz * 1e6 / 1e12  # Tops/s
    roofline = None
    if R and count_ms:
        cm = statistics.mean(count_ms)
        ops = ops_per_subgraph(k) * subgraphs_per_step
        achieved = ops / (cm / 1000.0) / 1e12
        roofline = {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "Tops/s",
                    "frac": achieved / alu_peak,
                    "traffic": _captured_traffic(args.method, args.workload, R),
                    "kernel": "k_count (enumerate+classify+count)", "kernel_ms": cm,
                    "ops_per_subgraph": ops_per_subgraph(k),
                    "peak_source": f"{sms} SMs (device query) x {INT32_LANES_PER_SM} int32 lanes "
                                   f"x {sm_mhz} MHz ({src} sm_max_mhz)"}

    extra = {}
    if (rank == 0 and not args.no_extra and args.workload == "nullmodel_k5" and args.nulls is None
            and args.method == "enumerate" and args.null_model == "arcswap"):
        extra["plain_vs_batched"] = measure_plain_vs_batched(
            mt, torch, dg, table, g, (1 + R) / (total_ms / args.steps / 1000.0))
        extra["k3_uniform_latency"] = measure_single("uniform_k3", mt, torch)
        extra["k4_chunglu_plain"] = measure_single("chunglu_k4", mt, torch)
        extra["k6_batch"] = measure_k6(mt, torch)
        dyad = measure_batch_method(mt, torch, "nullmodel_k5", table, method=0, null_model=1)
        dyad["metric"] = "k-subgraphs classified/s"
        dyad["note"] = "same k=5 batch with the dyad-preserving null model (reciprocity kept)"
        extra["dyad_null_model"] = dyad
        extra["cells_method"] = {
            "k5_batch": measure_batch_method(mt, torch, "nullmodel_k5", table),
            "k6_batch": measure_batch_method(mt, torch, "nullmodel_k6", None),
            "note": "same workloads counted with MT_METHOD_CELLS (Algorithm 1 of Sec. 3: the "
                    "last two vertices counted per cell pair); histograms identical"}
        extra["serving"] = measure_serving(mt, torch, {5: table})
        extra["serving_cells"] = measure_serving(mt, torch, {5: table}, method=1)

    gar = None
    if rank == 0 and R and count_ms:
        sub_rate = subgraphs_per_step / (statistics.mean(count_ms) / 1000.0)
        gar = _ceilings(mt, k, sub_rate, args.method, args.workload)

    if rank == 0:
        line = {"metric": "k-subgraphs classified/s", "value": value, "unit": "subgraphs/s",
                "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": total_ms / args.steps, "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "int64",
                "data": "synthetic (seeded Chung-Lu digraph and arc-swap nulls)",
                "config": _config(args, w, world),
                "subgraphs_per_step": subgraphs_per_step,
                "graphs_per_s": (1 + R) * args.steps * world / (total_ms / 1000.0),
                "table_build_ms": table_ms,
                "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e,
                "gpu_launches": launches_per_step * args.steps, "clocks": clk}
        line["config"]["tuning"] = tuned or "automatic"
        line["gather_atomic_roofline"] = gar
        line.update(extra)
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _timed(torch, fn, steps, flush):
    """Device time (ms) of `steps` calls of fn, L2 flushed before each call."""
    stream = torch.cuda.current_stream()
    total = 0.0
    for i in range(steps):
        flush.fill_(i & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        fn()
        b.record(stream)
        b.synchronize()
        total += a.elapsed_time(b)
    return total


def _ceilings(mt, k, sub_rate, method="enumerate", workload=None):
    """The count kernel's global-memory work against the measured ceilings of
    random 4 B reads from a table of 2^(k(k-1)) words (the k-vertex table) and
    random 64-bit atomic adds into the class count's power of two of counters.

    The kernel does not read the table once per subgraph: it reads once per
    group of equal keys.  So the reads and reductions it actually issues per
    classified subgraph come from an ncu capture of the current kernel
    (global-load and global-reduction sectors of one launch of a smaller batch
    that takes the same code path, profiles/k_count_counters.json), and the fraction is issued sectors/s over
    the probe's random reads/s (each probe read touches one sector)."""
    table_words = 1 << (k * (k - 1))
    hist_words = 1 << (int(syn_classes(k)) - 1).bit_length()
    gps, aps = mt.probe_rates(table_words, hist_words)
    out = {"gather_peak_per_s": gps, "atomic_peak_per_s": aps,
           "kernel_subgraphs_per_s": sub_rate, "table_bytes": 4 * table_words,
           "hist_counters": hist_words}
    cap = _captured("gather", method, workload, None) if workload else None
    if cap is None:
        out["issued"] = None
        out["note"] = ("no ncu capture of the current kernel for this workload: reads and adds "
                       "issued per subgraph unknown")
        return out
    ld = cap["global_ld_sectors"] / cap["subgraphs"]
    red = cap["global_red_sectors"] / cap["subgraphs"]
    out["issued"] = {"global_ld_sectors_per_subgraph": ld, "global_red_sectors_per_subgraph": red,
                     "global_ld_requests_per_subgraph": cap["global_ld_requests"] / cap["subgraphs"],
                     "global_red_requests_per_subgraph": cap["global_red_requests"] / cap["subgraphs"],
                     "capture": cap["case"]}
    out["frac_of_gather"] = ld * sub_rate / gps
    out["frac_of_atomic"] = red * sub_rate / aps if red > 0 else 0.0
    out["note"] = ("issued global-load and global-reduction sectors per classified subgraph "
                   "(ncu, a smaller batch on the same code path) x the kernel's subgraphs/s, over the "
                   "measured random-read and random-atomic rates (mt_probe_rates, this run); "
                   + cap.get("reading", ""))
    return out


def syn_classes(k):
    return {3: 13, 4: 199, 5: 9364, 6: 1530843}[k]


def measure_single(name, mt, torch, calls=200, warmup=20):
    """One plain count of a small workload graph, the way a caller makes it:
    single-call latency (host clock, p50/p99) with the graph resident on the
    device and the histogram copied to a host buffer, the same end to end from
    the host CSR (load, count, histogram back, free), and the device-timed rate
    of the count alone (CUDA events, L2 flushed before each call)."""
    w = syn.WORKLOADS[name]
    g = syn.workload_graph(name)
    t = mt.table_build(w["k"])
    dg = mt.graph_from(g)
    out = torch.empty(t.num_classes, dtype=torch.int64, device="cuda")
    for _ in range(warmup):
        mt.count_host(dg, t)
    sub = int(mt.count_host(dg, t).sum())
    lat = []
    for _ in range(calls):
        t0 = time.perf_counter()
        mt.count_host(dg, t)
        lat.append(1000 * (time.perf_counter() - t0))
    lat_e2e = []
    for _ in range(calls):
        t0 = time.perf_counter()
        gg = mt.graph_load_csr(g.n, g.row_ptr, g.col)
        h = mt.count_host(gg, t)
        gg.free()
        lat_e2e.append(1000 * (time.perf_counter() - t0))
    assert int(h.sum()) == sub
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    steps = 20
    ms = _timed(torch, lambda: mt.count(dg, t, out), steps, flush)
    res = {"config": f"{name}: n={w['n']} m={w['m']} k={w['k']}", "subgraphs_per_call": sub,
           "device_subgraphs_per_s": sub * steps / (ms / 1000.0), "device_ms_per_call": ms / steps,
           "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
           "subgraphs_per_s_at_p50": sub / (np.percentile(lat, 50) / 1000.0),
           "e2e_p50_ms": float(np.percentile(lat_e2e, 50)),
           "e2e_p99_ms": float(np.percentile(lat_e2e, 99)),
           "note": "p50/p99: mt_count into a host buffer on a resident graph (plan, enumerate, copy "
                   "back, synchronise); e2e: mt_graph_load_csr + mt_count + free per call"}
    dg.free()
    t.free()
    return res


def measure_k6(mt, torch, steps=3, warmup=3, nplain=16):
    """The k=6 null-model batch: Chung-Lu n=800, m=3,200 plus 64 nulls; and the
    plain path on the same kind of graphs (one mt_count launch per graph: the
    original and `nplain` nulls made beforehand by mt_randomize)."""
    w = syn.WORKLOADS["nullmodel_k6"]
    g = syn.workload_graph("nullmodel_k6")
    t0 = time.perf_counter()
    t = mt.table_build(6)
    table_ms = 1000 * (time.perf_counter() - t0)
    dg = mt.graph_from(g)
    R = w["nulls"]
    b = mt.Batch(dg, t, R, 10 * g.m, _autotuned(mt, dg, t, g, 0))
    seeds = np.arange(1, R + 1, dtype=np.uint64)
    hists = torch.empty((R + 1, t.num_classes), dtype=torch.int64, device="cuda")
    z = torch.empty(t.num_classes, dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        b.run(seeds, hists, z)
    torch.cuda.synchronize()
    sub = int(mt.to_numpy_u64(hists).sum())
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ms = 0.0
    count_ms = []
    for _ in range(steps):
        ms += _timed(torch, lambda: b.run(seeds, hists, z), 1, flush)
        count_ms.append(b.phase_ms()[1])
    cm = statistics.mean(count_ms)
    out = {"value": sub * steps / (ms / 1000.0), "unit": "subgraphs/s",
           "graphs_per_s": (R + 1) * steps / (ms / 1000.0), "ms_per_step": ms / steps,
           "count_kernel_ms": cm, "subgraphs_per_step": sub, "graphs_per_step": R + 1,
           "table_build_ms": table_ms,
           "gather_atomic_roofline": _ceilings(mt, 6, sub / (cm / 1000.0), "enumerate",
                                               "nullmodel_k6"),
           "config": "Chung-Lu n=800 m=3200 gamma 2.5 dmax 40 r 0.10 + 64 nulls, k=6"}
    ref = mt.to_numpy_u64(hists).copy()
    b.free()
    # plain: one launch per graph on the same table
    out["plain_vs_batched"] = measure_plain_vs_batched(mt, torch, dg, t, g, out["graphs_per_s"],
                                                       nplain)
    t.free()
    # the same batch with the compact k = 6 table (208 MB instead of 4 GiB)
    t0 = time.perf_counter()
    tc = mt.table_build(6, compact=True)
    ctable_ms = 1000 * (time.perf_counter() - t0)
    bc = mt.Batch(dg, tc, R, 10 * g.m, _autotuned(mt, dg, tc, g, 0))
    for _ in range(warmup):
        bc.run(seeds, hists, z)
    torch.cuda.synchronize()
    assert bc.error() == 0 and np.array_equal(mt.to_numpy_u64(hists), ref)
    ms = 0.0
    count_ms = []
    for _ in range(steps):
        ms += _timed(torch, lambda: bc.run(seeds, hists, z), 1, flush)
        count_ms.append(bc.phase_ms()[1])
    out["compact_table"] = {"value": sub * steps / (ms / 1000.0), "unit": "subgraphs/s",
                            "ms_per_step": ms / steps, "count_kernel_ms": statistics.mean(count_ms),
                            "table_bytes": 199 * (1 << 18) * 4 + 4096 * 2 + 4096 * 256,
                            "table_build_ms": ctable_ms, "histograms_equal": True}
    bc.free()
    tc.free()
    return out


def _autotuned(mt, dg, t, g, method):
    from paper_1804_09741_gb300 import autotune
    tp = autotune.tune_batch(dg, t, g, 10 * g.m, probe_nulls=16, method=method, cache_path=None)
    return mt.make_tuning(0.0, tp.warps_per_block, tp.split_scale, tp.stack_cap, method)


def measure_batch_method(mt, torch, name, table, method=1, steps=3, warmup=3, null_model=0):
    """A null-model batch counted with another counting method or null model."""
    w = syn.WORKLOADS[name]
    g = syn.workload_graph(name)
    own = table is None
    t = mt.table_build(w["k"]) if own else table
    dg = mt.graph_from(g)
    R = w["nulls"]
    b = mt.Batch(dg, t, R, 10 * g.m, _autotuned(mt, dg, t, g, method), null_model=null_model)
    seeds = np.arange(1, R + 1, dtype=np.uint64)
    hists = torch.empty((R + 1, t.num_classes), dtype=torch.int64, device="cuda")
    z = torch.empty(t.num_classes, dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        b.run(seeds, hists, z)
    torch.cuda.synchronize()
    assert b.error() == 0
    sub = int(mt.to_numpy_u64(hists).sum())
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    count_ms = []

    def one():
        b.run(seeds, hists, z)
    ms = 0.0
    for i in range(steps):
        ms += _timed(torch, one, 1, flush)
        count_ms.append(b.phase_ms()[1])
    out = {"metric": "k-subgraphs counted/s", "value": sub * steps / (ms / 1000.0),
           "unit": "subgraphs/s", "graphs_per_s": (R + 1) * steps / (ms / 1000.0),
           "ms_per_step": ms / steps, "count_kernel_ms": statistics.mean(count_ms),
           "subgraphs_per_step": sub}
    b.free()
    if own:
        t.free()
    return out


def measure_plain_vs_batched(mt, torch, dg, table, g, batched_graphs_per_s, nplain=16):
    """One launch per graph (mt_count on the original and `nplain` null graphs
    made by mt_randomize) against the batched step's graphs/s.  The plain time
    excludes making the null graphs; the batched time includes it."""
    graphs = [dg] + [mt.randomize(dg, s, 10 * g.m) for s in range(1, nplain + 1)]
    out = torch.empty(table.num_classes, dtype=torch.int64, device="cuda")
    for gr in graphs:
        mt.count(gr, table, out)
    torch.cuda.synchronize()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    it = iter(range(10**9))
    ms = _timed(torch, lambda: mt.count(graphs[next(it) % len(graphs)], table, out),
                len(graphs), flush)
    plain = len(graphs) / (ms / 1000.0)
    return {"plain_graphs_per_s": plain, "batched_graphs_per_s": batched_graphs_per_s,
            "batched_over_plain": batched_graphs_per_s / plain, "plain_graphs": len(graphs),
            "note": "plain = one mt_count launch per graph, null graphs made beforehand; "
                    "batched = randomise + rebuild + count + z in one captured step"}


def _work_bound(g, k):
    from math import comb
    s, d = g.arcs()
    deg = np.bincount(s, minlength=g.n) + np.bincount(d, minlength=g.n)
    return sum(comb(int(x), k - 1) for x in deg)


def serving_requests(num, seed):
    """Seeded request stream; requests whose work bound sum_v C(d_v, k-1)
    exceeds 2e9 are redrawn."""
    out, s = [], seed
    while len(out) < num:
        for k, g, _ in syn.serving_stream(num, s):
            if _work_bound(g, k) <= 2e9 and len(out) < num:
                out.append((k, g))
        s += 1
    return out


def measure_serving(mt, torch, have_tables, num=32, seed=0, method=0, round_cost=1.6e9):
    """Continuous-batching server on a seeded stream of mixed-k requests:
    closed-loop capacity first, then Poisson arrivals at 80% of it."""
    from paper_1804_09741_gb300.server import Server, poisson_arrivals, run_stream
    reqs = serving_requests(num, seed)
    tables = dict(have_tables)
    for k in (3, 4, 5, 6):
        if k not in tables:
            tables[k] = mt.table_build(k)
    srv = Server(tables, memory_budget=16 << 30, max_slots=32, round_cost=round_cost, method=method)
    run_stream(srv, reqs[:4])  # warm-up
    res, lat, wall = run_stream(srv, reqs)
    cap = num / wall
    rate = 0.8 * cap
    res, lat, wall2 = run_stream(srv, reqs, poisson_arrivals(num, rate, seed + 1))
    ok = all(r[0] == 2 for r in res)
    sub = sum(int(r[1].sum()) for r in res if r[1] is not None)
    srv.free()
    # the plain path on the same requests: load, one count launch, histogram
    # back to the host, one request after another
    def plain(k, g):
        dg = mt.graph_from(g)
        if method:
            h = mt.to_numpy_u64(mt.count_tuned(dg, tables[k], method=method))
        else:
            h = mt.count_host(dg, tables[k])
        dg.free()
        return h
    for k, g in reqs[:4]:
        plain(k, g)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    plain_ok = True
    for (k, g), r in zip(reqs, res):
        plain_ok &= r[1] is not None and np.array_equal(plain(k, g), r[1])
    plain_wall = time.perf_counter() - t0
    ks = [k for k, _ in reqs]
    return {"graphs_per_s": num / wall2, "capacity_graphs_per_s": cap,
            "plain_graphs_per_s": num / plain_wall, "served_over_plain": plain_wall / wall,
            "plain_equal": bool(plain_ok),
            "arrival_rate_per_s": rate, "p50_ms": float(np.percentile(lat, 50)),
            "p99_ms": float(np.percentile(lat, 99)), "subgraphs_per_s": sub / wall2,
            "requests": num, "round_cost": round_cost,
            "k_mix": {str(k): ks.count(k) for k in (3, 4, 5, 6)},
            "n_range": [int(min(g.n for _, g in reqs)), int(max(g.n for _, g in reqs))],
            "all_ok": ok, "method": "cells" if method else "enumerate"}


def ops_per_subgraph(k: int) -> int:
    """Algorithmic integer operations per classified k-subgraph: one table
    read, one histogram increment and the 2(k-1) direction-bit tests that fix
    the last vertex's arcs to the others (the enumeration's bookkeeping is not
    counted)."""
    return 2 + 2 * (k - 1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="nullmodel_k5", choices=sorted(syn.WORKLOADS))
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-autotune", action="store_true",
                    help="use the automatic launch instead of the autotuner's choice")
    ap.add_argument("--method", default="enumerate", choices=["enumerate", "cells"],
                    help="counting method of the main measurement (recorded in config)")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the k=6 batch, plain-vs-batched and serving measurements")
    ap.add_argument("--compact-table", action="store_true",
                    help="k=6 only: count with the compact table (recorded in config)")
    ap.add_argument("--null-model", default="arcswap", choices=["arcswap", "dyad"],
                    help="null graphs by degree-preserving arc swaps (default) or dyad-preserving "
                         "swaps (recorded in config)")
    ap.add_argument("--nulls", type=int, default=None,
                    help="number of null graphs (default: the workload's); smaller values make "
                         "the small cases profiled under ncu, recorded in config")
    args = ap.parse_args()
    world, rank, local = _dist()
    if args.impl == "reference":
        run_reference(args, world, rank)
    else:
        run_ours(args, world, rank, local)


if __name__ == "__main__":
    main()
