"""Benchmark: index creation (Kronecker-product CFPQ/RPQ) on GB300.

The default line (default): Dyck-4 CFPQ on a Zipf graph, n = 65536 -- the
largest of the five workloads, and the one whose closure has dense label
matrices, so that it compares the closure forms.  A step is one complete
index creation -- staging the edge list (device-resident), epsilon
initialisation and the fixpoint loop of Kronecker product, incremental
closure and extraction (Listing 1) -- with the default closure (AUTO:
bit-packed rows, tensor-core tiles for a nonterminal once its matrix is
dense).  ``value`` is queries per second over all ranks.  The same line
carries:

* ``closure_modes``: the bit-packed-only and tensor-core closures timed on
  the same query, each answer compared bit for bit with AUTO's;
* ``e2e``: the metric through the public C ABI with host buffers (edge list
  in, the answer's bit matrix out, every step);
* ``roofline`` (dominant kernel) and ``roofline_other``: the row gather
  against measured HBM bandwidth and the tile products against the FP8
  tensor peak, from CUDA events in a host-driven run of the same query;
* ``cpu_baseline``: Oracle B (the worklist oracle) on the same recipe at
  small n, extrapolated (the oracle cannot run this size in minutes).

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
Under torchrun (N > 1) every rank runs its own query (independent queries,
no collective on the data path) and rank 0 prints the line.

The other workloads print their own line with ``--workload``:
  rpq        the regular query (ab)*c | a*b*, n = 8192, 8 out-edges;
  cycles     two coprime cycles (126 vertices, S -> a S b | a b): latency,
             microseconds per fixpoint iteration;
  dyck_modes Dyck-4 at any n (--dyck-n), closure modes side by side;
  batched    512 (graph, RSM) queries in one batch vs one at a time;
  served     resident 32768-vertex graph, Poisson arrivals, p50/p99 latency;
  sources    multiple-source RPQ (1, 16, 256 sources) against the full run;
  paths      all-path extraction (vs -> vf, at most L edges) after index
             creation, against Oracle C on the same calls.
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
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2103_14688_gb300 import workloads as W  # noqa: E402

METRIC = "CFPQ queries/s & closure Bool-GOPS, tensor-core/batched vs bit-packed, bit-exact"
UNIT = "queries/s"
WORKLOAD = "rpq_abc_n8192_deg8"
FP8_PER_BF16 = 2.0  # nominal dense tensor rates: FP8 4.5 PFLOP/s vs bf16 2.25 PFLOP/s
FP4_PER_BF16 = 6.0  # nominal dense FP4 13.5 PFLOP/s vs bf16 2.25 PFLOP/s
# one K stage of a 128 x 256 tile, 128 deep (an FP4 stage of a 256 x 192 tile,
# 256 deep, is counted as three of these)
TILE_FLOP_PER_KSTAGE = 2.0 * 128 * 256 * 128


def _config(n, deg, flush):
    return {"workload": WORKLOAD, "query": W.ABC_REGEX, "rsm_states": 8, "n": n, "out_degree": deg,
            "labels": 3, "graph": "uniform targets, uniform labels, seeded PCG64",
            "l2": flush, "step": "stage edge list (device) + full fixpoint"}


def _dyck_config(n, flush):
    return {"workload": f"dyck4_zipf_n{n}", "query": "S -> S S | o_i c_i | o_i S c_i (i = 1..4)",
            "rsm_states": 11, "n": n, "out_degree": "Zipf(2.1) on 1..192, mean 3", "labels": 8,
            "graph": "uniform targets, labels uniform over o1..o4, c1..c4, seeded PCG64",
            "closure": "AUTO", "l2": flush, "step": "stage edge list (device) + full fixpoint"}


def _peaks():
    """Measured device peaks (MEASURED_PEAKS.json), else the fallback figures."""
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d.get("bf16_tflops_sustained", d["bf16_tflops"])),
                "kind": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0, "kind": "fallback"}


def _host_info():
    """Host cores and CPU model of the machine the CPU baseline runs on."""
    model = None
    try:
        for ln in open("/proc/cpuinfo"):
            if ln.lower().startswith(("model name", "cpu part", "hardware")):
                model = ln.split(":", 1)[1].strip()
                break
    except OSError:
        pass
    try:
        import platform
        arch = platform.machine()
    except Exception:
        arch = None
    return {"nproc": os.cpu_count(), "cpu_model": model, "arch": arch}


class ClockSampler:
    """nvidia-smi clock and throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int):
        self.device = device
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
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
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def run_rpq(args):
    import torch
    from paper_2103_14688_gb300 import cfpq

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    from paper_2103_14688_gb300 import shard
    n, deg = args.n, 8
    # independent queries per rank (weak scaling; no collective on the data path)
    g, r = W.rpq_abc(n=n, out_deg=deg, seed=shard.rank_seed(W.SEED_BASE + 2, rank))
    m = g.m
    d_src = torch.from_numpy(g.src.astype(np.int32)).to(dev)
    d_lbl = torch.from_numpy(g.lbl.astype(np.int32)).to(dev)
    d_dst = torch.from_numpy(g.dst.astype(np.int32)).to(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    ctx = cfpq.Context(device=local)
    ctx.load_rsm(r)

    def step_device():
        ctx.load_graph_device(n, 3, d_src, d_lbl, d_dst)
        return ctx.run()

    for _ in range(args.warmup):
        step_device()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    times = []
    last = None
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        last = step_device()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = float(np.mean(times))
    total_ms = shard.max_over_ranks(float(np.sum(times)), dist, dev)
    value = ws * args.steps / (total_ms / 1000.0)
    stats = last

    # parity spot-check of the timed configuration (8 sampled rows, oracle-free:
    # the answer of the empty word is the diagonal, and each row is non-empty)
    bits = ctx.reachable_bits(0)
    assert bits.diagonal().all()

    # closure Bool-GOPS: executed = OR-AND operations of the source-row ORs
    # (one per bit of a padded row); paper accounting (Theorem 2) = one
    # length-|Q|n vector operation per M3 edge and per closure bit,
    # W = (nnz(M3) + nnz(C3)) * |Q|n, an equivalent-work count far above it
    cbits, m3bits = ctx.count_index()
    Nq = r.n_states * n
    work = (cbits + m3bits) * Nq
    gops = work / (step_ms / 1000.0) / 1e9
    exec_gops = stats.row_ors * (stats.row_bytes * 8) / (step_ms / 1000.0) / 1e9

    # end to end through the ABI: host (pinned) edge list in, answer bits out
    h_src = torch.from_numpy(g.src.astype(np.int32)).pin_memory()
    h_lbl = torch.from_numpy(g.lbl.astype(np.int32)).pin_memory()
    h_dst = torch.from_numpy(g.dst.astype(np.int32)).pin_memory()
    wn = (n + 63) // 64
    out_bits = torch.empty(n * wn, dtype=torch.int64).pin_memory()
    lib = ctx.lib
    import ctypes

    def step_e2e():
        u32 = ctypes.POINTER(ctypes.c_uint32)
        rc = lib.cfpq_load_graph(ctx.h, n, 3, m, ctypes.cast(h_src.data_ptr(), u32), ctypes.cast(h_lbl.data_ptr(), u32),
                                 ctypes.cast(h_dst.data_ptr(), u32))
        assert rc == 0, rc
        st = cfpq.cfpq_run_stats()
        rc = lib.cfpq_run(ctx.h, ctypes.byref(st))
        assert rc == 0, rc
        rc = lib.cfpq_get_reachable_bits(ctx.h, 0, ctypes.c_void_p(out_bits.data_ptr()))
        assert rc == 0, rc

    for _ in range(max(1, args.warmup)):
        step_e2e()
    barrier()
    e_times = []
    for _ in range(args.steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step_e2e()
        e_times.append((time.perf_counter() - t0) * 1000.0)
    barrier()
    e_total = shard.max_over_ranks(float(np.sum(e_times)), dist, dev)
    e2e_value = ws * args.steps / (e_total / 1000.0)
    e2e_equal = bool((out_bits.numpy().view(np.uint64).reshape(n, wn) == ctx.reachable_words(0)).all())

    # roofline of the dominant kernel (closure pass): per-launch CUDA events in a
    # host-driven profiling run of the same workload on the same stream
    pctx = cfpq.Context(device=local, loop_mode=cfpq.CFPQ_LOOP_HOST, profile=1)
    pctx.load_rsm(r)
    pctx.load_graph_device(n, 3, d_src, d_lbl, d_dst)
    pctx.run()
    ps = pctx.run()
    alg_bytes = (ps.row_ors + 2 * ps.rows_changed) * ps.row_bytes
    launches = max(1, ps.closure_launches)
    per_launch_bytes = alg_bytes / launches
    per_launch_s = ps.ms_closure / 1000.0 / launches
    achieved = per_launch_bytes / per_launch_s / 1e9
    pk = _peaks()
    peak, peak_kind = pk["hbm_gbs"], pk["kind"]
    traffic = _traffic_from_profiles("k_gather_rpq_abc_n8192")
    staging_kernels = 10
    gpu_launches = args.steps * (stats.gpu_launches + staging_kernels)

    # the same query with the closure products on the tensor cores (0/1 FP8),
    # for comparison: bit-exact, timed once after a warm-up run
    modes = None
    if not args.no_extras:
        tctx = cfpq.Context(device=local, closure_mode=cfpq.CFPQ_CLOSURE_TC_FP8)
        tctx.load_rsm(r)
        tctx.load_graph_device(n, 3, d_src, d_lbl, d_dst)
        tctx.run()
        t0 = torch.cuda.Event(enable_timing=True)
        t1 = torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        tctx.load_graph_device(n, 3, d_src, d_lbl, d_dst)
        tst = tctx.run()
        t1.record(stream)
        t1.synchronize()
        modes = {"bitpacked_ms_per_query": step_ms, "tc_fp8_ms_per_query": t0.elapsed_time(t1),
                 "tc_fp8_tiles": tst.tile_mmas,
                 "tc_equals_bitpacked": bool((tctx.reachable_words(0) == ctx.reachable_words(0)).all())}
        tctx.close()

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": _config(n, deg, "256 MiB L2 flush before every timed step; closure blocks 208 MiB > L2"),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 3 * 4 * m,
                "d2h_bytes_per_step": n * wn * 8, "matches_device_result": e2e_equal},
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "cfpq::k_gather<2>",
                     "peak_source": f"{peak_kind} hbm_gbs", "launches_timed": launches,
                     "algorithmic_bytes_per_launch": per_launch_bytes, "ms_per_launch": per_launch_s * 1e3},
        "closure_bool_gops": exec_gops,
        "closure_bool_gops_paper_accounting": gops,
        "closure_work_W": work,
        "index": {"closure_bits": cbits, "m3_bits": m3bits, "answer_pairs": int(bits.sum()),
                  "iterations": stats.iterations, "passes": stats.rounds, "blocks": stats.closure_blocks,
                  "row_ors": stats.row_ors, "rows_changed": stats.rows_changed},
        "gpu_launches": gpu_launches,
        "closure_modes": modes,
        "clocks": clk,
        "wall_s": wall,
    }
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline_rpq(g, r)
    if rank == 0:
        print(json.dumps(line), flush=True)
    ctx.close()
    pctx.close()
    if dist:
        dist.destroy_process_group()


def _roofline_gather(st, peaks, n):
    """Row gather: algorithmic bytes = every source row ORed read once, every
    changed output row read and written once, over the gather launches' event
    time, against the measured HBM copy bandwidth."""
    alg = (st.row_ors + 2 * st.rows_changed) * st.row_bytes
    launches = max(1, st.gather_launches)
    sec = max(st.ms_gather, 1e-9) / 1e3
    achieved = alg / sec / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": _traffic_from_profiles(f"k_gather_dyck4_n{n}"),
            "kernel": "cfpq::k_gather (row gather)", "peak_source": f"{peaks['kind']} hbm_gbs (burst copy)",
            "launches_timed": launches, "algorithmic_bytes_per_launch": alg / launches,
            "ms_per_launch": st.ms_gather / launches,
            "accounting": "(source rows ORed + 2 x output rows changed) x row bytes"}


def _roofline_tiles(st, peaks, n, fp4=False, nv=False):
    """Tile products: dense 0/1 multiply-adds over the compacted inner
    dimension (2 x 128 x 256 x 128 per K stage) over the product launches'
    event time, against the peak of the tiles' format (measured sustained
    bf16 x the nominal FP8/bf16 or FP4/bf16 ratio: the kernel runs inside a
    long step)."""
    flop = st.tile_kstages * TILE_FLOP_PER_KSTAGE
    launches = max(1, st.tile_launches)
    sec = max(st.ms_tile_products, 1e-9) / 1e3
    achieved = flop / sec / 1e12
    ratio, fmt = (FP4_PER_BF16, "FP4") if fp4 else (FP8_PER_BF16, "FP8")
    peak = peaks["bf16_tflops_sustained"] * ratio
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak,
            "traffic": _traffic_from_profiles(f"k_tc_product_tma_{'fp4_' if fp4 else ''}dyck4_n{n}"),
            "kernel": "cfpq::k_tc_product_tma (tcgen05 " + (("kind::mxf4nvf4" if nv else "kind::mxf4") + ", 0/1 E2M1"
                                                           if fp4 else "kind::f8f6f4") + ")",
            "peak_source": f"{peaks['kind']} bf16_tflops_sustained x {ratio} (nominal {fmt}/bf16)",
            "launches_timed": launches, "flop_per_launch": flop / launches,
            "ms_per_launch": st.ms_tile_products / launches,
            "accounting": "tile K stages x 2 x 128 x 256 x 128 (inner dimension compacted to the dirty rows)"}


def run_dyck(args):
    """The default line: Dyck-4 CFPQ on the Zipf graph (n = 65536 by default)."""
    import ctypes
    import torch
    from paper_2103_14688_gb300 import cfpq, shard

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dist = None
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)

    def barrier():
        if dist:
            dist.barrier()
        torch.cuda.synchronize()

    n = args.dyck_n
    # independent queries per rank (weak scaling; no collective on the data path)
    g, r = W.dyck_zipf(n, seed=shard.rank_seed(W.SEED_BASE + 3, rank))
    m, nt = g.m, g.n_terminals
    d_src, d_lbl, d_dst = (torch.from_numpy(np.asarray(a).astype(np.int32)).to(dev) for a in (g.src, g.lbl, g.dst))
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream(dev)

    ctx = cfpq.Context(device=local)  # AUTO closure, device-side loop
    ctx.load_rsm(r)

    def step_device():
        ctx.load_graph_device(n, nt, d_src, d_lbl, d_dst)
        return ctx.run()

    for _ in range(args.warmup):
        step_device()
    barrier()
    clocks = ClockSampler(local)
    clocks.start()
    times, last = [], None
    t_wall = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        last = step_device()
        e1.record(stream)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    barrier()
    wall = time.perf_counter() - t_wall
    clk = clocks.stop()
    step_ms = float(np.mean(times))
    total_ms = shard.max_over_ranks(float(np.sum(times)), dist, dev)
    value = ws * args.steps / (total_ms / 1000.0)
    stats = last
    tuning = ctx.tune().as_dict()  # the autotuner's probe ran in the first warm-up step
    words = ctx.reachable_words(0)
    pairs = int(ctx.count_reachable(0))
    cbits, m3bits = ctx.count_index()
    Nq = r.n_states * n

    # end to end through the ABI: pinned host edge list in, answer bits out
    h = [torch.from_numpy(np.asarray(a).astype(np.int32)).pin_memory() for a in (g.src, g.lbl, g.dst)]
    wn = (n + 63) // 64
    out_bits = torch.empty(n * wn, dtype=torch.int64).pin_memory()
    lib = ctx.lib
    u32 = ctypes.POINTER(ctypes.c_uint32)

    def step_e2e():
        rc = lib.cfpq_load_graph(ctx.h, n, nt, m, *(ctypes.cast(a.data_ptr(), u32) for a in h))
        assert rc == 0, rc
        st = cfpq.cfpq_run_stats()
        rc = lib.cfpq_run(ctx.h, ctypes.byref(st))
        assert rc == 0, rc
        rc = lib.cfpq_get_reachable_bits(ctx.h, 0, ctypes.c_void_p(out_bits.data_ptr()))
        assert rc == 0, rc

    e_steps = max(1, min(args.steps, args.e2e_steps))
    step_e2e()
    barrier()
    e_times = []
    for _ in range(e_steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        step_e2e()
        e_times.append((time.perf_counter() - t0) * 1000.0)
    barrier()
    e_total = shard.max_over_ranks(float(np.sum(e_times)), dist, dev)
    e2e_value = ws * e_steps / (e_total / 1000.0)
    e2e_equal = bool((out_bits.numpy().view(np.uint64).reshape(n, wn) == words).all())
    ctx.close()

    # the same query with the other closure forms, each compared bit for bit
    modes = None
    if not args.no_extras:
        modes = {"auto_ms_per_query": step_ms, "auto_tile_products": stats.tile_mmas}
        for name, mode, fmt in (("bitpacked", cfpq.CFPQ_CLOSURE_BITPACKED, 0),
                                ("tc_fp8", cfpq.CFPQ_CLOSURE_TC_FP8, 0), ("tc_fp4", cfpq.CFPQ_CLOSURE_TC_FP4, 0),
                                ("auto_fp8_tiles", cfpq.CFPQ_CLOSURE_AUTO, cfpq.CFPQ_TILES_FP8)):
            mctx = cfpq.Context(device=local, closure_mode=mode, tile_format=fmt)
            mctx.load_rsm(r)
            mctx.load_graph_device(n, nt, d_src, d_lbl, d_dst)
            mctx.run()  # warm-up: buffers, plan, CUDA graph
            flush.fill_(1)
            _, ms = _ctx_time(mctx, stream, lambda: (mctx.load_graph_device(n, nt, d_src, d_lbl, d_dst), mctx.run()))
            modes[f"{name}_ms_per_query"] = ms
            modes[f"{name}_equals_auto"] = bool((mctx.reachable_words(0) == words).all())
            mctx.close()
        modes["auto_speedup_vs_bitpacked"] = modes["bitpacked_ms_per_query"] / step_ms

    # rooflines: per-kernel CUDA events in a host-driven run of the same query
    pctx = cfpq.Context(device=local, loop_mode=cfpq.CFPQ_LOOP_HOST, profile=1)
    pctx.load_rsm(r)
    pctx.load_graph_device(n, nt, d_src, d_lbl, d_dst)
    pctx.run()
    ps = pctx.run()
    prof_equal = bool((pctx.reachable_words(0) == words).all())
    pctx.close()
    peaks = _peaks()
    roof_g = _roofline_gather(ps, peaks, n)
    # AUTO's tiles are the autotuner's kernel (E2M1 on GB300): its format sets the peak
    tiles_fp4 = tuning.get("tile_format") in (cfpq.CFPQ_TILES_FP4, cfpq.CFPQ_TILES_NVFP4)
    roof_t = (_roofline_tiles(ps, peaks, n, fp4=tiles_fp4, nv=tuning.get("tile_format") == cfpq.CFPQ_TILES_NVFP4)
              if ps.tile_launches else None)
    dominant, other = (roof_g, roof_t)
    if roof_t is not None and ps.ms_tile_products > ps.ms_gather:
        dominant, other = roof_t, roof_g
    staging_kernels = 10
    gpu_launches = args.steps * (stats.gpu_launches + staging_kernels)

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": step_ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "u64", "data": "synthetic",
        "config": _dyck_config(n, f"inputs larger than L2: {stats.device_bytes / 1e9:.1f} GB of closure state "
                                  f"per query (L2 129 MB), and a 256 MiB L2 flush before every timed step"),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 3 * 4 * m, "d2h_bytes_per_step": n * wn * 8,
                "steps": e_steps, "matches_device_result": e2e_equal},
        "roofline": dominant,
        "roofline_other": other,
        "closure_modes": modes,
        "autotune": tuning,
        "closure_time_split_ms": {"gather": ps.ms_gather, "tile_operands": ps.ms_tile_operands,
                                  "tile_products": ps.ms_tile_products, "host_loop_result_equal": prof_equal},
        "tile_operands": {"bytes_expanded": ps.tile_operand_bytes,
                          "write_gbs": ps.tile_operand_bytes / max(ps.ms_tile_operands, 1e-9) / 1e6,
                          "note": "0/1 operand bytes written by k_tc_a8/k_tc_b8 over the operand kernels' event time "
                                  "(which also lists the dirty rows and new-edge columns)"},
        "closure_bool_gops": stats.row_ors * stats.row_bytes * 8 / (step_ms / 1000.0) / 1e9,
        "closure_bool_gops_paper_accounting": (cbits + m3bits) * Nq / (step_ms / 1000.0) / 1e9,
        "tensor_tflops_issued": stats.tile_kstages * TILE_FLOP_PER_KSTAGE / (step_ms / 1000.0) / 1e12,
        "index": {"closure_bits": cbits, "m3_bits": m3bits, "answer_pairs": pairs, "edges": m,
                  "iterations": stats.iterations, "passes": stats.rounds, "blocks": stats.closure_blocks,
                  "row_ors": stats.row_ors, "rows_changed": stats.rows_changed, "tile_products": stats.tile_mmas,
                  "device_gb": stats.device_bytes / 1e9},
        "gpu_launches": gpu_launches,
        "clocks": clk,
        "wall_s": wall,
    }
    if rank == 0 and not args.no_extras:
        line["batched"] = batched_summary(args.batch, local)
        line["served"] = served_summary(args.served_lambda, args.served_horizon, local)
    if rank == 0 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline_dyck(n)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def batched_summary(count, device):
    """The batched workload (512 queries, n ~ U[256, 8192], 3-24 RSM states):
    one batch in AUTO and with bit-packed rows only, against the same
    queries one at a time; every batched answer compared with its solo run."""
    import torch
    from paper_2103_14688_gb300 import cfpq
    qs = W.batched_queries(count=count)

    split = {}

    def batch(mode, name):
        ctx = cfpq.Context(device=device, closure_mode=mode)
        ctx.batch_run(qs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        _, tot = ctx.batch_run(qs)
        torch.cuda.synchronize()
        el = time.perf_counter() - t0
        split[name] = {"setup_ms": tot.ms_setup, "loop_ms": tot.ms_loop, "passes": tot.rounds,
                       "gpu_launches": tot.gpu_launches, "tile_products": tot.tile_mmas}
        return ctx, el

    actx, at = batch(cfpq.CFPQ_CLOSURE_AUTO, "auto")
    bctx, bt = batch(cfpq.CFPQ_CLOSURE_BITPACKED, "bitpacked")
    solo = cfpq.Context(device=device)
    st, mism = 0.0, 0
    for i, (g, r) in enumerate(qs):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        solo.load_graph(g)
        solo.load_rsm(r)
        solo.run()
        torch.cuda.synchronize()
        st += time.perf_counter() - t0
        for b in range(r.n_boxes):
            want = solo.reachable_words(b)
            mism += int(not ((actx.batch_reachable_words(i, b) == want).all() and
                             (bctx.batch_reachable_words(i, b) == want).all()))
    # the plain bit-packed single-query path, one query at a time
    plain = cfpq.Context(device=device, closure_mode=cfpq.CFPQ_CLOSURE_BITPACKED)
    pt = 0.0
    for g, r in qs:
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        plain.load_graph(g)
        plain.load_rsm(r)
        plain.run()
        torch.cuda.synchronize()
        pt += time.perf_counter() - t0
    for c in (actx, bctx, solo, plain):
        c.close()
    return {"queries": len(qs), "batched_qps": len(qs) / at, "batched_bitpacked_qps": len(qs) / bt,
            "one_at_a_time_qps": len(qs) / st, "one_at_a_time_bitpacked_qps": len(qs) / pt,
            "speedup_vs_one_at_a_time": st / at, "speedup_vs_bitpacked_one_at_a_time": pt / at,
            "mismatches_vs_solo": mism, "split": split,
            "timing": "host clock around one batch_run after a warm-up batch; one at a time: AUTO and "
                      "bit-packed contexts, each query staged and run"}


def served_summary(lam, horizon, device):
    """The served workload (resident Zipf graph n = 32768, random RSMs with
    3-32 states, Poisson arrivals at `lam` per second for `horizon` s):
    queries/s and p50/p99 latency, and the same queries one at a time."""
    import torch
    from paper_2103_14688_gb300 import cfpq
    wl = W.serving_workload(lam=lam, n_queries=100000, horizon_s=horizon)
    srv = cfpq.Server(wl.graph, device=device)
    t_start = time.perf_counter()
    pending = list(zip(wl.arrivals.tolist(), wl.choice.tolist()))
    live, lat, i = {}, [], 0
    while i < len(pending) or live:
        now = time.perf_counter() - t_start
        while i < len(pending) and pending[i][0] <= now:
            live[srv.submit(wl.pool[pending[i][1]])] = pending[i][0]
            i += 1
        srv.step()
        now = time.perf_counter() - t_start
        for t in list(live):
            if srv.poll(t):
                lat.append(now - live.pop(t))
                srv.release(t)
        if not live and i < len(pending):
            time.sleep(max(0.0, min(0.001, pending[i][0] - now)))
    el = time.perf_counter() - t_start
    srv.close()
    solo_t = {}
    for name, mode in (("auto", cfpq.CFPQ_CLOSURE_AUTO), ("bitpacked", cfpq.CFPQ_CLOSURE_BITPACKED)):
        solo = cfpq.Context(device=device, closure_mode=mode)
        solo.load_graph(wl.graph)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for j in wl.choice.tolist():
            solo.load_rsm(wl.pool[j])
            solo.run()
        torch.cuda.synchronize()
        solo_t[name] = time.perf_counter() - t0
        solo.close()
    solo_s = solo_t["auto"]
    lat = np.array(lat)
    return {"lambda": lam, "horizon_s": horizon, "queries": int(len(lat)), "qps": len(lat) / el,
            "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
            "one_at_a_time_qps": len(wl.choice) / solo_s,
            "one_at_a_time_bitpacked_qps": len(wl.choice) / solo_t["bitpacked"]}


def _traffic_from_profiles(name):
    """DRAM read + write bytes per launch from the committed ncu summary
    profiles/<name>.json, when it was taken on the current source of the
    kernel's file; else None."""
    p = os.path.join(ROOT, "profiles", f"{name}.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
        from paper_2103_14688_gb300 import build as B
        import hashlib
        src = open(os.path.join(B.CSRC, d.get("source_file", "cfpq_kernels.cu")), "rb").read()
        if d.get("kernel_source_sha1") != hashlib.sha1(src).hexdigest():
            return None
        return d.get("dram_bytes_per_launch")
    except Exception:
        return None


def cpu_baseline_rpq(g, r):
    """Oracle A (Listing 1 with the closure recomputed from scratch every
    iteration) on the whole RPQ workload, its closure rows spread over every
    host core with OpenMP."""
    import oracle
    cores = os.cpu_count() or 1
    oracle.set_threads(cores)
    t0 = time.perf_counter()
    oracle.kron_fixpoint(g, r)
    dt = time.perf_counter() - t0
    oracle.set_threads(1)
    return {"value": 1.0 / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"Oracle A on the whole query (n = {g.n}), closure rows over {cores} threads, {dt:.1f} s",
            **_host_info()}


def dyck_oracle_seconds(n_target, sizes=(2048, 4096)):
    """Oracle B (worklist, one thread) on the Dyck-4 Zipf recipe at the given
    sizes, and the time extrapolated to n_target by the power law through
    the two largest: (seconds at n_target, per-size seconds, exponent)."""
    import oracle
    ts = {}
    for n in sizes:
        g, r = W.dyck_zipf(n)
        t0 = time.perf_counter()
        oracle.worklist_words(g, r)
        ts[n] = time.perf_counter() - t0
    a, b = sizes[-2], sizes[-1]
    k = float(np.log(ts[b] / ts[a]) / np.log(b / a))
    return ts[b] * (n_target / b) ** k, ts, k


def cpu_baseline_dyck(n):
    """The oracle on a bounded sample of the Dyck-4 workload: Oracle B cannot
    be restricted to a few source rows of a context-free query (every box
    call enters new vertices), so it runs the same recipe at n = 2048 and
    4096 and its time is extrapolated to n."""
    t, ts, k = dyck_oracle_seconds(n)
    return {"value": 1.0 / t, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"Oracle B on the same recipe at n = 2048 ({ts[2048]:.2f} s) and 4096 ({ts[4096]:.2f} s); "
                      f"time extrapolated to n = {n} as n^{k:.2f}: {t:.0f} s per query",
            **_host_info()}


def _ctx_time(ctx, stream, fn):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    out = fn()
    e1.record(stream)
    e1.synchronize()
    return out, e0.elapsed_time(e1)


def run_other(args):
    """The other configurations, one JSON line each (besides the default RPQ line)."""
    import torch
    from paper_2103_14688_gb300 import cfpq
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    line = {"workload": args.workload, "n_gpus": 1, "data": "synthetic"}
    # host-driven loop: one launch per kernel and pass, visible to profilers
    loop_mode = cfpq.CFPQ_LOOP_HOST if args.loop == "host" else cfpq.CFPQ_LOOP_DEVICE
    if args.loop == "host":
        line["loop"] = "host"
    if args.workload == "cycles":
        g, r = W.two_cycles(63, 64)
        ctx = cfpq.Context()
        ctx.load_graph(g)
        ctx.load_rsm(r)
        ctx.run()
        ts = []
        for _ in range(max(1, args.steps)):
            st, ms = _ctx_time(ctx, stream, ctx.run)
            ts.append(ms)
        ms = float(np.median(ts))
        ans = ctx.reachable_bits(0)
        line.update({"metric": "time per query (two coprime cycles, 4032-pair closed form)", "unit": "ms",
                     "value": ms, "higher_is_better": False, "iterations": st.iterations,
                     "us_per_iteration": 1000.0 * ms / st.iterations, "passes": st.rounds,
                     "pairs": int(ans.sum()), "closed_form_pairs": 4032})
    elif args.workload == "dyck_modes":
        g, r = W.dyck_zipf(args.dyck_n)
        res = {}
        all_modes = {"auto": (cfpq.CFPQ_CLOSURE_AUTO, 0), "bitpacked": (cfpq.CFPQ_CLOSURE_BITPACKED, 0),
                     "tc_fp8": (cfpq.CFPQ_CLOSURE_TC_FP8, 0), "tc_fp4": (cfpq.CFPQ_CLOSURE_TC_FP4, 0),
                     "auto_fp8": (cfpq.CFPQ_CLOSURE_AUTO, cfpq.CFPQ_TILES_FP8)}
        names = [m for m in args.modes.split(",") if m in all_modes]
        if args.no_extras:
            names = names[:1]
        for name in names:
            mode, fmt = all_modes[name]
            if name == "auto" and args.tile_format:
                fmt = args.tile_format
            ctx = cfpq.Context(closure_mode=mode, tile_format=fmt, loop_mode=loop_mode)
            ctx.load_graph(g)
            ctx.load_rsm(r)
            ctx.run()  # warm-up: planning, buffers, the loop's CUDA graph (and the autotuner's probe)
            st, ms = _ctx_time(ctx, stream, ctx.run)
            res[name] = {"ms": ms, "iterations": st.iterations, "passes": st.rounds, "row_ors": st.row_ors,
                         "tile_products": st.tile_mmas, "tile_kstages": st.tile_kstages,
                         "issued_tensor_tflop": st.tile_kstages * 2.0 * 128 * 256 * 128 / 1e12,
                         "pairs": ctx.count_reachable(0),
                         "executed_bool_gops": st.row_ors * st.row_bytes * 8 / (ms / 1e3) / 1e9,
                         "device_gb": st.device_bytes / 1e9,
                         "tile_products_per_iteration": st.tile_mmas / max(1, st.iterations)}
            # Theorem 2's work count, W = (nnz(M3) + nnz(C3)) * |Q|n
            cbits, m3bits = ctx.count_index()
            res[name].update({"closure_bits": cbits, "m3_bits": m3bits,
                              "closure_bool_gops_paper_accounting":
                                  (cbits + m3bits) * r.n_states * g.n / (ms / 1e3) / 1e9})
            res[name]["words"] = ctx.reachable_words(0)
            ctx.close()
        ref = res[names[0]]["words"]
        same = {k: bool((v["words"] == ref).all()) for k, v in res.items()}
        for v in res.values():
            v.pop("words", None)
        line.update({"metric": "Dyck-4 index creation time (second run of a context: set-up excluded)",
                     "unit": "ms", "value": res[names[0]]["ms"],
                     "higher_is_better": False, "n": g.n, "m": g.m, "modes": res,
                     f"modes_equal_{names[0]}": same})
    elif args.workload == "sources":
        # multiple-source runs: only rows reachable from the sources
        out = []
        for n, deg in ((8192, 8), (65536, 2)):
            g, r = W.rpq_abc(n=n, out_deg=deg)
            ctx = cfpq.Context()
            ctx.load_graph(g)
            ctx.load_rsm(r)
            ctx.run()
            st, ms_full = _ctx_time(ctx, stream, ctx.run)
            full = ctx.reachable_words(0)
            rows = {"n": n, "out_degree": deg, "full_ms": ms_full}
            for k in (1, 16, 256):
                src = list(range(0, n, n // k))[:k]
                ctx.run_sources(src)
                st, ms = _ctx_time(ctx, stream, lambda: ctx.run_sources(src))
                same = bool((ctx.reachable_words(0)[src] == full[src]).all())
                rows[f"sources_{k}"] = {"ms": ms, "speedup_vs_full": ms_full / ms, "rows_equal_full": same}
            out.append(rows)
            ctx.close()
        line.update({"metric": "multiple-source RPQ time (rows reachable from the sources only)", "unit": "ms",
                     "value": out[0]["sources_16"]["ms"], "higher_is_better": False, "graphs": out})
    elif args.workload == "paths":
        # all-path extraction after index creation: device backward layers
        # prune the host enumeration; Oracle C (all paths up to L, words
        # tested) timed on the same calls where it finishes quickly
        import oracle
        from collections import deque
        out = []
        for name, (g, r), lens in (("rpq_abc_n8192_deg8", W.rpq_abc(n=8192, out_deg=8), (4, 6, 8)),
                                   ("dyck4_zipf_n4096", W.dyck_zipf(n=4096), (4, 8, 12, 16))):
            ctx = cfpq.Context()
            ctx.load_graph(g)
            ctx.load_rsm(r)
            ctx.run()
            words = ctx.reachable_words(0)
            adj = [[] for _ in range(g.n)]
            for a, b in zip(np.asarray(g.src).tolist(), np.asarray(g.dst).tolist()):
                adj[a].append(b)
            rng = np.random.Generator(np.random.PCG64(2103_14688))
            for L in lens:
                pairs = []
                for vs in rng.permutation(g.n).tolist():
                    dist, dq = {vs: 0}, deque([vs])
                    while dq:
                        v = dq.popleft()
                        if dist[v] < L:
                            for w in adj[v]:
                                if w not in dist:
                                    dist[w] = dist[v] + 1
                                    dq.append(w)
                    near = [v for v in dist if (int(words[vs, v >> 6]) >> (v & 63)) & 1]
                    if near:
                        pairs.append((vs, int(rng.choice(near))))
                    if len(pairs) == 8:
                        break
                ts, npaths, same, ots = [], [], True, []
                for vs, vf in pairs:
                    t0 = time.perf_counter()
                    got, trunc = ctx.extract_paths(0, vs, vf, L)
                    ts.append(1e3 * (time.perf_counter() - t0))
                    npaths.append(len(got))
                    if sum(ots) < 20e3:
                        t0 = time.perf_counter()
                        want = oracle.brute_paths(g, r, 0, vs, vf, L, path_cap=1 << 20, edge_cap=1 << 26)
                        ots.append(1e3 * (time.perf_counter() - t0))
                        same &= got == want
                slow = max(ts) > 10e3
                out.append({"graph": name, "max_len": L, "pairs": len(pairs), "ms_median": float(np.median(ts)),
                            "ms_max": float(max(ts)), "paths_median": float(np.median(npaths)),
                            "paths_max": int(max(npaths)),
                            "oracle_ms_median": float(np.median(ots)) if ots else None,
                            "oracle_calls": len(ots), "equal_oracle": bool(same)})
                if slow:  # longer bounds would take longer still
                    break
            ctx.close()
        line.update({"metric": "all-path extraction time per (vs, vf) call (median, Dyck-4 at the largest bound)",
                     "unit": "ms", "value": out[-1]["ms_median"], "higher_is_better": False, "runs": out})
    elif args.workload == "batched":
        qs = W.batched_queries(count=args.batch)
        ctx = cfpq.Context()
        ctx.batch_run(qs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        per, tot = ctx.batch_run(qs)
        torch.cuda.synchronize()
        bt = time.perf_counter() - t0
        bits = [ctx.batch_reachable_bits(i, 0) for i in range(len(qs))]
        # the same batch with bit-packed rows only (no tensor-core tiles)
        bctx = cfpq.Context(closure_mode=cfpq.CFPQ_CLOSURE_BITPACKED)
        bctx.batch_run(qs)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        bctx.batch_run(qs)
        torch.cuda.synchronize()
        bp_t = time.perf_counter() - t0
        bp_same = all((bctx.batch_reachable_bits(i, 0) == bits[i]).all() for i in range(len(qs)))
        bctx.close()
        solo = cfpq.Context()
        st_s = 0.0
        mism = 0
        for i, (g, r) in enumerate(qs):
            torch.cuda.synchronize()
            a = time.perf_counter()
            solo.load_graph(g)
            solo.load_rsm(r)
            solo.run()
            torch.cuda.synchronize()
            st_s += time.perf_counter() - a
            mism += int(not (solo.reachable_bits(0) == bits[i]).all())
        line.update({"metric": "batched queries/s vs one at a time", "unit": "queries/s",
                     "value": len(qs) / bt, "higher_is_better": True, "queries": len(qs),
                     "one_at_a_time_qps": len(qs) / st_s, "speedup": st_s / bt, "mismatches_vs_solo": mism,
                     "batched_bitpacked_qps": len(qs) / bp_t, "bitpacked_equal": bool(bp_same),
                     "batch_setup_ms": tot.ms_setup, "batch_loop_ms": tot.ms_loop, "passes": tot.rounds,
                     "device_gb": tot.device_bytes / 1e9})
    elif args.workload == "served":
        out = []
        for lam in [float(x) for x in args.lambdas.split(",")]:
            wl = W.serving_workload(lam=lam, n_queries=args.served_queries, horizon_s=args.horizon)
            srv = cfpq.Server(wl.graph)
            t_start = time.perf_counter()
            pending = list(zip(wl.arrivals.tolist(), wl.choice.tolist()))
            live, lat, i, waits = {}, [], 0, 0
            while i < len(pending) or live:
                now = time.perf_counter() - t_start
                while i < len(pending) and pending[i][0] <= now:
                    live[srv.submit(wl.pool[pending[i][1]])] = pending[i][0]
                    i += 1
                _, wait = srv.step()
                waits += wait
                now = time.perf_counter() - t_start
                for t in list(live):
                    if srv.poll(t):
                        lat.append(now - live.pop(t))
                        srv.release(t)
                if not live and i < len(pending):
                    time.sleep(max(0.0, min(0.001, pending[i][0] - now)))
            el = time.perf_counter() - t_start
            lat = np.array(lat)
            out.append({"lambda": lam, "queries": int(len(lat)), "elapsed_s": el, "qps": len(lat) / el,
                        "p50_ms": float(np.percentile(lat, 50) * 1e3), "p99_ms": float(np.percentile(lat, 99) * 1e3),
                        "admission_waits": waits})
            srv.close()
        # the same pool of queries one at a time on the same resident graph
        wl = W.serving_workload(lam=100.0, n_queries=args.served_queries, horizon_s=args.horizon)
        k = min(200, len(wl.choice))
        solo_qps = {}
        for name, mode in (("auto", cfpq.CFPQ_CLOSURE_AUTO), ("bitpacked", cfpq.CFPQ_CLOSURE_BITPACKED)):
            solo = cfpq.Context(closure_mode=mode)
            solo.load_graph(wl.graph)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for j in wl.choice[:k].tolist():
                solo.load_rsm(wl.pool[j])
                solo.run()
            torch.cuda.synchronize()
            solo_qps[name] = k / (time.perf_counter() - t0)
            solo.close()
        line.update({"metric": "served queries/s and latency", "unit": "queries/s",
                     "value": max(o["qps"] for o in out), "higher_is_better": True, "n": 32768, "sweep": out,
                     "one_at_a_time_qps": solo_qps["auto"], "one_at_a_time_bitpacked_qps": solo_qps["bitpacked"],
                     "one_at_a_time_queries": k})
    print(json.dumps(line), flush=True)


def run_reference(args):
    """The oracle as the reference arm, on the host cores, for the same
    workload, metric and unit as the GPU line.  Each step is a bounded sample:
    for the Dyck-4 line, Oracle B on the same recipe at n = 2048 and 4096 with
    its time extrapolated to the benchmark's n; for the RPQ line, Oracle B
    from a random sample of source vertices (facts of different sources are
    independent), scaled by the sampled fraction."""
    ws, rank, _ = _dist()
    if rank != 0:
        return
    import oracle
    if args.workload == "rpq":
        g, r = W.rpq_abc(n=args.n, out_deg=8)
        n_s = args.cpu_sources
        rng = np.random.Generator(np.random.PCG64(1))

        def one():
            srcs = sorted(rng.choice(g.n, size=n_s, replace=False).tolist())
            t0 = time.perf_counter()
            oracle.worklist(g, r, sources=srcs)
            return (time.perf_counter() - t0) * g.n / n_s  # seconds per whole query

        sample = f"Oracle B from {n_s} random source vertices per step of {g.n}, scaled by the sampled fraction"
        config = _config(args.n, 8, "n/a (host)")
    else:
        n = args.dyck_n

        def one():
            return dyck_oracle_seconds(n)[0]

        sample = (f"Oracle B on the Dyck-4 Zipf recipe at n = 2048 and 4096 per step, time extrapolated to "
                  f"n = {n} by the power law through the two")
        config = _dyck_config(n, "n/a (host)")
    for _ in range(args.warmup):
        one()
    ts = [one() for _ in range(args.steps)]
    total = float(np.sum(ts))
    value = args.steps / total
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u64", "data": "synthetic",
            "config": config, "impl": "reference",
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample,
                             **_host_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--n", type=int, default=8192, help="rpq workload: vertices")
    ap.add_argument("--cpu-sources", type=int, default=512)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--workload", default="dyck",
                    choices=["dyck", "rpq", "cycles", "dyck_modes", "batched", "served", "sources", "paths"])
    ap.add_argument("--dyck-n", type=int, default=65536)
    ap.add_argument("--e2e-steps", type=int, default=5, help="end-to-end steps (at most --steps)")
    ap.add_argument("--batch", type=int, default=512)
    ap.add_argument("--served-lambda", type=float, default=100.0, help="default line: served probe arrival rate")
    ap.add_argument("--served-horizon", type=float, default=3.0, help="default line: served probe seconds")
    ap.add_argument("--lambdas", default="10,30,100,300,1000")
    ap.add_argument("--horizon", type=float, default=60.0, help="served workload: seconds of arrivals per lambda")
    ap.add_argument("--served-queries", type=int, default=2000, help="served workload: arrivals per lambda (cap)")
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--loop", default="device", choices=["device", "host"],
                    help="dyck_modes workload: fixpoint loop in a CUDA graph (device) or one launch per pass (host)")
    ap.add_argument("--tile-format", type=int, default=0,
                    help="dyck_modes workload: tile_format of the auto mode (0 = the autotuner's choice; "
                         "1 FP8, 2 FP4, 3 FP8 128-row tiles: no autotuner probe in the process)")
    ap.add_argument("--modes", default="auto,bitpacked,tc_fp8,tc_fp4,auto_fp8",
                    help="dyck_modes workload: closure modes to run (the first is the line's value)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "dyck":
        run_dyck(args)
    elif args.workload == "rpq":
        run_rpq(args)
    else:
        run_other(args)


if __name__ == "__main__":
    main()
