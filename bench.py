#!/usr/bin/env python3
"""Benchmark: bulk MTGP32 generation on GB300.

Default workload (N = 1): 10 000 streams of one Mexp 11213 parameter set,
output counts floor(2^U), U ~ Uniform[10, 22] (seed 7), about 5.04e9 uint32
numbers (20 GB) per step.  A step is one replay of a recorded plan: a CUDA
graph holding one persistent work-stealing launch over all streams.  Output
(20 GB per step) is far larger than L2; in addition a 256 MiB buffer is
rewritten between timed steps.

Prints one JSON line (rank 0).  Under torchrun each rank runs its own
instance of the workload (distinct stream seeds) on its own GPU; no data
crosses ranks (weak scaling); the elapsed time is the max over ranks.

--impl reference times the CPU oracle on the host cores instead (bounded
samples of the same workload per step).
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
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1501_07701_gb300 import dist as mdist  # noqa: E402
from paper_1501_07701_gb300 import workloads  # noqa: E402

METRIC = "Gnumbers/s and % of HBM-write roofline, bit-exact; serving p50/p99 latency"
UNIT = "Gnumbers/s"
# device source of each generation kernel (a recorded DRAM traffic figure is
# used only while these still hash to the value it was taken on)
KERNEL_SOURCES = {
    "mtgp_fast_kernel": ["paper_1501_07701_gb300/csrc/mtgp_fast.cuh"],
}
KERNEL_NAMES = {0: "mtgp_fast_kernel", 1: "mtgp_ring_kernel"}
FORMATS = {"u32": 0, "f12": 1, "f01": 2}


def kernel_source_hash(kernel: str = "mtgp_fast_kernel") -> str:
    h = hashlib.sha256()
    for rel in KERNEL_SOURCES.get(kernel, []):
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def recorded_traffic(kernel: str, workload_name: str):
    """DRAM bytes per launch of the uneven workload from the committed ncu
    summary of that kernel, if it was taken on the current kernel source;
    else None."""
    if workload_name != "uneven":
        return None
    path = os.path.join(ROOT, "profiles", kernel.replace("mtgp_", "") + "_uneven_traffic.md")
    try:
        txt = open(path).read()
    except OSError:
        return None
    m_b = re.search(r"traffic_bytes_per_launch:\s*([0-9.eE+]+)", txt)
    m_h = re.search(r"kernel_source_sha256_16:\s*([0-9a-f]+)", txt)
    if not (m_b and m_h) or m_h.group(1) != kernel_source_hash(kernel):
        return None
    return float(m_b.group(1))


def workload(name: str, rank: int, streams: int = 0, count: int = 0, param_sets: int = 0,
             generator: str = "", mexp: int = 0):
    """Seeds and counts of a named workload; `generator` replaces the MTGP32
    label in the description (the comparison generator runs the same shapes)
    and `mexp` the workload's MTGP exponent."""
    gen = generator or "MTGP32 Mexp %d" % (mexp or workloads.MEXP_MAIN)
    if name == "uneven":
        w = workloads.uneven()
        desc = "uneven: 10000 %s streams, counts floor(2^U), U~U[10,22] (seed 7)" % gen
        if streams:
            w = {"mexp": w["mexp"], "seeds": w["seeds"][:streams], "counts": w["counts"][:streams]}
            desc = "uneven subset: first %d of the 10000 %s streams" % (streams, gen)
    elif name == "single":
        w = workloads.single()
        desc = "single: 1 %s stream (seed 1) x 2^20" % gen
    elif name == "equal":
        w = workloads.equal(streams or 4096, count or (1 << 18))
        desc = "equal: %d %s streams x %d" % (streams or 4096, gen, count or (1 << 18))
    elif name.startswith("long"):
        w = workloads.long_streams(int(name[4:]))
        desc = "long: 1024 %s streams x 2^20" % (generator or "MTGP32 Mexp " + name[4:])
    else:
        raise SystemExit("unknown workload " + name)
    if mexp:
        w["mexp"] = mexp
    w["seeds"] = mdist.weak_seeds(w["seeds"], rank)
    w["param_seeds"] = None
    if param_sets:
        n_sets = min(param_sets, w["seeds"].size)
        w["param_seeds"] = workloads.param_seeds(w["seeds"].size, n_sets)
        desc += "; %d parameter sets, stream s uses set s mod %d" % (n_sets, n_sets)
    return w, desc


def oracle_params_of(w):
    """Oracle parameter set of every stream (one shared set, or per stream)."""
    import oracle
    if w.get("param_seeds") is None:
        p = oracle.params_generate(w["mexp"], workloads.PARAM_SEED)
        return lambda s: p
    cache = {}

    def get(s):
        k = int(w["param_seeds"][s])
        if k not in cache:
            cache[k] = oracle.params_generate(w["mexp"], k)
        return cache[k]
    return get


def rank_workload(args, rank: int, world: int):
    """This rank's share of the job.  weak: its own instance of the workload
    (stream seeds shifted by rank), so per-GPU work is fixed as ranks are
    added; strong: the contiguous range of one instance's streams that
    dist.strong_range gives this rank, so the job's work is fixed."""
    if getattr(args, "rank_split", "weak") == "strong" and world > 1:
        w, desc = workload(args.workload, 0, args.streams, args.count, args.param_sets,
                           mexp=args.mexp)
        a, b = mdist.strong_range(w["seeds"].size, rank, world)
        w = dict(w, seeds=w["seeds"][a:b], counts=w["counts"][a:b],
                 param_seeds=None if w["param_seeds"] is None else w["param_seeds"][a:b])
        desc += "; split into %d contiguous stream ranges, one per GPU" % world
        return w, desc
    return workload(args.workload, rank, args.streams, args.count, args.param_sets, mexp=args.mexp)


class bracket:
    """Barrier + device synchronisation on entry and on exit of the timed
    region, so every rank starts and ends it together."""

    def __init__(self, dist, sync):
        self.dist, self.sync = dist, sync

    def __enter__(self):
        if self.dist:
            self.dist.barrier()
        self.sync()
        return self

    def __exit__(self, *exc):
        self.sync()
        if self.dist:
            self.dist.barrier()
        return False


def job_rate(local_numbers: int, local_elapsed: float, device=None):
    """Whole-job throughput over all ranks: the numbers every rank produced
    divided by the slowest rank's elapsed time.  Returns (Gnumbers/s,
    elapsed max over ranks, numbers summed over ranks)."""
    elapsed = mdist.max_over_ranks(local_elapsed, device=device)
    numbers = mdist.sum_over_ranks(float(local_numbers), device=device)
    return numbers / elapsed / 1e9, elapsed, numbers


class ClockSampler:
    """nvidia-smi clock / throttle-reason samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.proc = None
        self.gpu = gpu_index

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
                power.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm),
                "power_w_max": max(power) if power else None}


def oracle_rate(w, budget_s: float, threads: int, max_batch=1 << 26, seed=0, mt_params=None):
    """Times the CPU oracle on a bounded random sample of the workload's
    streams: whole streams in random order, in batches of at most max_batch
    numbers (outputs discarded batch by batch), until budget_s seconds of
    oracle time have been spent.  Returns (numbers/s, numbers, seconds,
    streams).  With mt_params (an oracle.mt parameter set) the original-MT
    oracle is timed instead."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    if mt_params is not None:
        import oracle.mt as gen_oracle
        p_of = lambda s: mt_params  # noqa: E731
    else:
        gen_oracle = oracle
        p_of = oracle_params_of(w)
    per_stream = w.get("param_seeds") is not None
    pool = ThreadPoolExecutor(threads) if per_stream else None
    order = np.random.default_rng(seed).permutation(w["seeds"].size)
    done, t_all, used, k = 0, 0.0, 0, 0
    while t_all < budget_s and k < order.size:
        batch, acc = [], 0
        while k < order.size and len(batch) < 4 * threads and (
                acc == 0 or acc + int(w["counts"][order[k]]) <= max_batch):
            batch.append(int(order[k]))
            acc += int(w["counts"][order[k]])
            k += 1
        states = [gen_oracle.init_state(p_of(i), int(w["seeds"][i])) for i in batch]
        t0 = time.perf_counter()
        if per_stream:   # each stream with its own set, streams spread over the host threads
            list(pool.map(lambda a: oracle.generate(p_of(a[0]), a[1], int(w["counts"][a[0]])),
                          zip(batch, states)))
        else:
            gen_oracle.generate_many(p_of(0), np.stack(states), np.arange(len(batch)),
                                     w["counts"][batch], 0, threads)
        t_all += time.perf_counter() - t0
        done += acc
        used += len(batch)
    if pool:
        pool.shutdown()
    return done / t_all, done, t_all, used


def run_reference(args, rank, world):
    if rank != 0:
        return
    threads = os.cpu_count() or 1
    w, desc = workload(args.workload, 0, args.streams, args.count, args.param_sets, mexp=args.mexp)
    # each step: a bounded sample sized so the whole run stays within ~2 minutes
    per_step = min(10.0, max(0.05, 100.0 / max(1, args.steps + args.warmup)))
    vals, secs, nums = [], [], []
    for step in range(args.warmup + args.steps):
        r, n, t, ns = oracle_rate(w, per_step, threads, seed=step)
        if step >= args.warmup:
            vals.append(r)
            secs.append(t)
            nums.append(n)
    value = sum(nums) / sum(secs) / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(secs) / len(secs),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic", "config": {"workload": desc, "format": "u32",
                                        "sample": "random streams per step, ~%.2f s each" % per_step},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle",
                         "sample": "%d numbers over %d steps of random whole streams" % (
                             sum(nums), len(nums))},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def run_ours(args, rank, world, local_rank):
    import torch
    from paper_1501_07701_gb300 import mtgp
    from paper_1501_07701_gb300.build import build
    build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    w, desc = rank_workload(args, rank, world)
    counts = w["counts"]
    total = int(counts.sum())
    stream = torch.cuda.Stream()
    if w["param_seeds"] is None:
        params = mtgp.mtgp_params_generate(w["mexp"], workloads.PARAM_SEED)
        st = mtgp.mtgp_init_statuses(params, w["seeds"], stream)
    else:
        uniq, set_of = np.unique(w["param_seeds"], return_inverse=True)
        sets = [mtgp.mtgp_params_generate(w["mexp"], int(k)) for k in uniq]
        st = mtgp.mtgp_init_statuses_multi(sets, set_of.astype(np.uint32), w["seeds"], stream)
    out = torch.empty(total, dtype=torch.int32, device=dev)
    ids = np.arange(w["seeds"].size, dtype=np.uint32)
    if args.config:
        cv = [int(v) for v in args.config.split(",")] + [0, 0]
        mtgp.mtgp_set_launch_config(st, warps_per_cta=cv[0], words_per_lane=cv[1],
                                    coop_percent=cv[2], ctas_per_sm=cv[3], kernel=cv[4])
    fmt = FORMATS[args.format]
    plan = mtgp.mtgp_plan_create(st, ids, counts, fmt, out)
    max_piece = split_piece(args.split, total, torch.cuda.get_device_properties(dev).multi_processor_count)
    if max_piece:
        mtgp.mtgp_plan_set_split(plan, max_piece)
    tuned = None
    if not args.no_autotune and not args.config:
        tuned = mtgp.mtgp_plan_autotune(plan)
    info = mtgp.mtgp_plan_get_info(plan)

    # bit-exact spot check of the first launch against the oracle (rank 0)
    bit_exact = None
    states0 = mtgp.mtgp_get_statuses(st, stream) if rank == 0 else None
    flush = torch.empty(64 << 20, dtype=torch.int32, device=dev)   # 256 MiB > L2
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            mtgp.mtgp_plan_launch(plan, stream)
            if _ == 0 and rank == 0:
                stream.synchronize()
                bit_exact = spot_check(w, counts, out, states0, fmt)
            flush.fill_(1)
    stream.synchronize()

    # timed region
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    smi_index = cvd.split(",")[local_rank] if cvd else str(local_rank)
    clocks = ClockSampler(smi_index)
    clocks.start()
    time.sleep(0.3)   # let the sampler start
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    with bracket(dist, torch.cuda.synchronize):
        t0.record(stream)
        with torch.cuda.stream(stream):
            for i in range(args.steps):
                ev[i][0].record(stream)
                mtgp.mtgp_plan_launch(plan, stream)
                ev[i][1].record(stream)
                flush.fill_(i)
        t1.record(stream)
    clk = clocks.stop()
    kern_ms = [a.elapsed_time(b) for a, b in ev]
    value, elapsed, _ = job_rate(total * args.steps, t0.elapsed_time(t1) / 1e3, device=dev)

    # roofline of the dominant kernel (the persistent generation kernel)
    peak, peak_src = hbm_peak()
    n_words = mtgp.mtgp_streams_info(st)[1]
    alg_bytes = 4.0 * total + 8.0 * n_words * info["n_items"]
    kern_avg = sum(kern_ms) / len(kern_ms) / 1e3
    kname = KERNEL_NAMES.get(info["config"]["kernel"], "?")
    achieved = alg_bytes / kern_avg / 1e9

    # quality statistics of the last timed launch's output (tests 35 and 100, Sec. 4.2),
    # taken before the bandwidth check below overwrites the buffer
    qual = None
    if rank == 0 and args.quality:
        qual = quality_stats(mtgp, torch, out, counts, stream)
        qual["fused"] = measure_fused_stats(mtgp, torch, st, ids, counts, out, stream, flush,
                                            total / kern_avg / 1e9)

    # self-measured write-only bandwidth (fill of the output buffer)
    wb_a, wb_b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(stream):
        out.fill_(0)
        wb_a.record(stream)
        for _ in range(3):
            out.fill_(7)
        wb_b.record(stream)
    stream.synchronize()
    write_gbs = 3 * 4.0 * total / (wb_a.elapsed_time(wb_b) / 1e3) / 1e9

    # end to end through the public API: host output buffer, copies inside
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(mtgp, torch, st, ids, counts, stream, args)

    per_stream = None
    if rank == 0 and args.workload == "uneven" and not args.no_extra:
        per_stream = measure_per_stream_launches(mtgp, torch, st, w, out, stream, flush)

    configs = None
    if rank == 0 and not args.no_extra:
        del plan
        configs = measure_configs(mtgp, torch, dev, stream, flush)

    serving = None
    if rank == 0 and args.serving_seconds > 0:
        plan = None
        serving = measure_serving(mtgp, torch, args)

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        r, n, t, ns = oracle_rate(w, args.cpu_seconds, threads)
        cpu = {"value": r / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "%d random whole streams of the workload, %d numbers, %.1f s" % (ns, n, t)}

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "strong" if args.rank_split == "strong" else "weak",
            "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": desc, "numbers_per_step_per_gpu": total, "format": args.format,
                       "parallelism": ("1 GPU" if world == 1 else
                                       "one contiguous stream range per GPU" if args.rank_split == "strong"
                                       else "independent streams per GPU"),
                       "l2": "20 GB written per step (> 129 MB L2) plus a 256 MiB rewrite "
                             "between timed steps",
                       "launch": info["config"], "grid_ctas": info["grid_ctas"],
                       "split": {"max_piece": info["max_piece"], "streams": info["n_split_streams"],
                                 "jumps_per_launch": info["n_jumps"], "items": info["n_items"]},
                       "coop_streams": info["n_coop"], "regs_per_thread": info["regs_per_thread"],
                       "resident_ctas_per_sm": info["resident_ctas_per_sm"],
                       "autotuned": tuned is not None},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": recorded_traffic(kname, args.workload),
                         "peak_source": peak_src + " (MEASURED_PEAKS.json hbm_gbs)"
                         if peak_src == "measured" else "fallback 6.8 TB/s",
                         "algorithmic_bytes_per_launch": alg_bytes,
                         "kernel_ms_avg": 1e3 * kern_avg,
                         "kernel": kname},
            "write_only_fill_gbs": write_gbs,
            "clocks": clk,
            "e2e": e2e,
            "gpu_launches": args.steps * info["kernel_launches"],
            "bit_exact_sample": bit_exact,
            "one_launch_per_stream": per_stream,
            "configs": configs,
            "serving": serving,
            "quality": qual,
            "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def split_piece(spec: str, total: int, sms: int) -> int:
    """Piece length for --split: 0 (off), an explicit count, 'auto' -- the
    numbers per warp slot at 16 warps per SM, so that no piece outlasts an
    even share of the launch at that residency -- or 'autoW', the launch cut
    into W pieces per SM (for short states, whose best residency is higher:
    'auto48' is half a warp slot's share at 24 warps per SM)."""
    if spec in ("", "0"):
        return 0
    if spec == "auto":
        return max(64, -(-total // (sms * 16)))
    if spec.startswith("auto"):
        return max(64, -(-total // (sms * int(spec[4:]))))
    return max(64, int(spec))


def hbm_peak():
    """The measured copy bandwidth (MEASURED_PEAKS.json hbm_gbs), else the
    6.8 TB/s fallback; returns (GB/s, "measured" | "fallback")."""
    try:
        peak = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))).get("hbm_gbs")
    except (OSError, ValueError):
        peak = None
    return (peak, "measured") if peak else (6800.0, "fallback")


def quality_stats(mtgp, torch, out, counts, stream):
    """Pooled statistics of tests 35 and 100 (Sec. 4.2) over a launch's
    output, with the rate of each reduction kernel."""
    from paper_1501_07701_gb300 import quality
    total = int(counts.sum())
    bounds = quality.default_hamming_bounds(1200, 4)
    q0, q1, q2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
    q0.record(stream)
    hist = mtgp.mtgp_gap_histogram(out, counts, r=25, b=5, t=128, stream=stream)
    q1.record(stream)
    tab = mtgp.mtgp_hamming_pairs(out, counts, r=25, s=5, L=1200, bounds=bounds, stream=stream)
    q2.record(stream)
    stream.synchronize()
    g = quality.gap_test(hist.sum(axis=0), b=5)
    hm = quality.hamming_test(tab.sum(axis=0), L=1200, bounds=bounds)
    return {"gap_test": {"r": 25, "beta": "1/32", "t": 128,
                         "gnum_s": total / (q0.elapsed_time(q1) * 1e6), "pooled": g},
            "hamming_indep": {"r": 25, "s": 5, "L": 1200, "classes": len(bounds) + 1,
                              "gnum_s": total / (q1.elapsed_time(q2) * 1e6), "pooled": hm}}


def measure_fused_stats(mtgp, torch, st, ids, counts, out, stream, flush, gen_rate, steps=5):
    """Generation with both statistics fused in (mtgp_plan_set_stats, the
    parameters of quality_stats): per-launch rate over `steps` launches
    (CUDA events, the L2 rewrite between launches as in the timed region)
    at 8 and 16 warps per SM, and at 16 with the longest requests split into
    pieces of two lengths (statistics stitched across pieces), next to
    generation alone timed the same way.  Each shape's counts of its last
    launch are compared with the standalone reductions over its output."""
    from paper_1501_07701_gb300 import quality
    bounds = quality.default_hamming_bounds(1200, 4)
    total = int(counts.sum())
    saved = mtgp.mtgp_get_launch_config(st)
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    piece = split_piece("auto", total, sms)
    by_res = {}
    try:
        # 8 and 16 warps per SM (one or two 8-warp CTAs), and 16 with the longest
        # requests split into pieces (stitched statistics); the fastest is reported
        for label, ctas, max_piece in (("8", 1, 0), ("16", 2, 0), ("16 split %d" % piece, 2, piece),
                                       ("16 split %d" % (piece // 2), 2, piece // 2)):
            mtgp.mtgp_set_launch_config(st, **dict(saved, warps_per_cta=8, ctas_per_sm=ctas))
            plan = mtgp.mtgp_plan_create(st, ids, counts, FORMATS["u32"], out)
            try:
                mtgp.mtgp_plan_set_stats(plan, gap=(25, 5, 128), hamming=(25, 5, 1200, bounds))
                if max_piece:
                    mtgp.mtgp_plan_set_split(plan, max_piece)
            except mtgp.MtgpError as e:
                return {"unavailable": str(e)}
            info = mtgp.mtgp_plan_get_info(plan)
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for _ in range(steps)]
            with torch.cuda.stream(stream):
                for _ in range(2):
                    mtgp.mtgp_plan_launch(plan, stream)
                    flush.fill_(2)
                for i in range(steps):
                    ev[i][0].record(stream)
                    mtgp.mtgp_plan_launch(plan, stream)
                    ev[i][1].record(stream)
                    flush.fill_(i)
            stream.synchronize()
            ms = [a.elapsed_time(b) for a, b in ev]
            hist, tab = mtgp.mtgp_plan_read_stats(plan, stream)
            sh = mtgp.mtgp_gap_histogram(out, counts, r=25, b=5, t=128, stream=stream)
            stab = mtgp.mtgp_hamming_pairs(out, counts, r=25, s=5, L=1200, bounds=bounds, stream=stream)
            by_res[label] = {
                "gnum_s": total / (sum(ms) / len(ms) / 1e3) / 1e9,
                "launch_ms": [round(v, 3) for v in ms], "grid_ctas": info["grid_ctas"],
                "warps_per_sm": 8 * info["resident_ctas_per_sm"], "max_piece": info["max_piece"],
                "jumps_per_launch": info["n_jumps"], "kernel_launches": info["kernel_launches"],
                "regs_per_thread": info["regs_per_thread"],
                "counts_equal_standalone": bool(np.array_equal(hist, sh) and np.array_equal(tab, stab)),
                "pooled": (hist.sum(axis=0), tab.sum(axis=0))}
            del plan
    finally:
        mtgp.mtgp_set_launch_config(st, **saved)
    best = max(by_res, key=lambda k: by_res[k]["gnum_s"])
    b = by_res[best]
    hs, ts = b.pop("pooled")
    for v in by_res.values():
        v.pop("pooled", None)
    return {"gnum_s": b["gnum_s"], "generation_alone_gnum_s": gen_rate, "ratio": b["gnum_s"] / gen_rate,
            "best": best, "steps": steps, "kernel": "mtgp_fused_kernel",
            "by_launch_shape": by_res,
            "counts_equal_standalone": all(v["counts_equal_standalone"] for v in by_res.values()),
            "pooled_gap": quality.gap_test(hs, b=5),
            "pooled_hamming": quality.hamming_test(ts, L=1200, bounds=bounds)}


def run_mt(args, rank, world, local_rank):
    """The comparison generator of Sec. 5.3 (the original Mersenne Twister)
    on the same workload shapes: one mtgp_mt_generate launch per step."""
    import torch
    import oracle.mt as omt
    from paper_1501_07701_gb300 import mtgp
    from paper_1501_07701_gb300.build import build
    build()
    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
    if args.mt_p == 19937:
        q, oq, label = mtgp.mtgp_mt_params_mt19937(), omt.params_mt19937(), "MT19937"
    else:
        q = mtgp.mtgp_mt_params_generate(args.mt_p, workloads.PARAM_SEED)
        oq = omt.params_generate(args.mt_p, workloads.PARAM_SEED)
        label = "original-MT p %d (seed-generated set)" % args.mt_p
    w, desc = workload(args.workload, rank, args.streams, args.count, generator=label)
    counts = w["counts"]
    total = int(counts.sum())
    stream = torch.cuda.Stream()
    mt = mtgp.mtgp_mt_init(q, w["seeds"], stream)
    out = torch.empty(total, dtype=torch.int32, device=dev)
    ids = np.arange(w["seeds"].size, dtype=np.uint32)
    fmt = FORMATS[args.format]
    bit_exact = None
    states0 = mtgp.mtgp_mt_get_statuses(mt, stream) if rank == 0 else None
    flush = torch.empty(64 << 20, dtype=torch.int32, device=dev)   # 256 MiB > L2
    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            mtgp.mtgp_mt_generate(mt, ids, counts, fmt, out, stream)
            if i == 0 and rank == 0:
                stream.synchronize()
                offs = np.concatenate([[0], np.cumsum(counts.astype(np.int64))])
                bit_exact = True
                for s in sorted({int(np.argmax(counts)), 0, counts.size - 1, counts.size // 2}):
                    ref, _ = omt.generate(oq, states0[s], int(counts[s]), fmt)
                    got = out[int(offs[s]):int(offs[s + 1])].cpu().numpy().view(np.uint32)
                    bit_exact = bit_exact and bool(np.array_equal(ref, got))
            flush.fill_(1)
    mtgp.mtgp_mt_check(mt, stream)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    cvd = os.environ.get("CUDA_VISIBLE_DEVICES", "")
    clocks = ClockSampler(cvd.split(",")[local_rank] if cvd else str(local_rank))
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    with torch.cuda.stream(stream):
        for i in range(args.steps):
            ev[i][0].record(stream)
            mtgp.mtgp_mt_generate(mt, ids, counts, fmt, out, stream)
            ev[i][1].record(stream)
            flush.fill_(i)
    t1.record(stream)
    stream.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = clocks.stop()
    elapsed = mdist.max_over_ranks(t0.elapsed_time(t1) / 1e3, device=dev)
    kern_avg = sum(a.elapsed_time(b) for a, b in ev) / len(ev) / 1e3
    value = total * args.steps * world / elapsed / 1e9
    peak, peak_src = hbm_peak()
    alg_bytes = 4.0 * total + 8.0 * oq.n * ids.size
    achieved = alg_bytes / kern_avg / 1e9
    qual = quality_stats(mtgp, torch, out, counts, stream) if rank == 0 and args.quality else None
    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        threads = os.cpu_count() or 1
        r, n, t, ns = oracle_rate(w, args.cpu_seconds, threads, mt_params=oq)
        cpu = {"value": r / 1e9, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "%d random whole streams of the workload, %d numbers, %.1f s" % (ns, n, t)}
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
            "data": "synthetic", "generator": label, "params": oq.as_dict(),
            "config": {"workload": desc, "numbers_per_step_per_gpu": total, "format": args.format,
                       "l2": "output > 129 MB L2 plus a 256 MiB rewrite between timed steps",
                       "launch": "mtgp_mt_generate per step (work table upload + one kernel)"},
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": None,
                         "peak_source": peak_src, "algorithmic_bytes_per_launch": alg_bytes,
                         "kernel_ms_avg": 1e3 * kern_avg, "kernel": "mt_gen_kernel"},
            "clocks": clk, "e2e": None, "gpu_launches": args.steps,
            "bit_exact_sample": bit_exact, "quality": qual, "cpu_baseline": cpu,
        }
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def run_quality_sweep(args):
    """Sec. 5.3 restated on this library: many parameter sets of MTGP and of
    the original MT at the same period 2^p, one stream per set from seed
    status 0 (Sec. 5.1), each stream's output put through the statistics of
    tests 35 and 100 on the GPU; the line reports the fraction of sets whose
    p-values stay inside [0.001, 0.999] (TestU01's suspect bounds).  The
    sets are seed-generated, not made by the dynamic creators, and the
    statistics are this library's restatement, not TestU01's."""
    import torch
    import oracle
    import oracle.mt as omt
    from paper_1501_07701_gb300 import mtgp, quality
    from paper_1501_07701_gb300.build import build
    build()
    torch.cuda.set_device(0)
    S, C, p = args.quality_sweep, args.sweep_count, args.mexp or 3217
    SB = min(S, args.sweep_batch)   # sets per launch (bounds the output buffer)
    bounds = quality.default_hamming_bounds(1200, 4)
    out = torch.empty(SB * C, dtype=torch.int32, device="cuda")
    inside = lambda v: 1e-3 <= v <= 1.0 - 1e-3  # noqa: E731
    res = {}
    for gen in ("mtgp", "mt"):
        pg, ph = np.zeros(S), np.zeros(S)
        gen_ms = stats_ms = 0.0
        exact = True
        for k0 in range(0, S, SB):
            nb = min(SB, S - k0)
            counts = np.full(nb, C, np.uint64)
            ids = np.arange(nb, dtype=np.uint32)
            seeds = np.zeros(nb, np.uint32)
            if gen == "mtgp":
                sets = [mtgp.mtgp_params_generate(p, k0 + k) for k in range(nb)]
                st = mtgp.mtgp_init_statuses_multi(sets, ids, seeds)
            else:
                sets = [mtgp.mtgp_mt_params_generate(p, k0 + k) for k in range(nb)]
                st = mtgp.mtgp_mt_init_multi(sets, ids, seeds)
            torch.cuda.synchronize()
            e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
            e0.record()
            if gen == "mtgp":
                mtgp.mtgp_generate_u32(st, ids, counts, out)
            else:
                mtgp.mtgp_mt_generate(st, ids, counts, mtgp.MTGP_U32, out)
            e1.record()
            hist = mtgp.mtgp_gap_histogram(out, counts, r=25, b=5, t=128)
            tab = mtgp.mtgp_hamming_pairs(out, counts, r=25, s=5, L=1200, bounds=bounds)
            e2.record()
            torch.cuda.synchronize()
            gen_ms += e0.elapsed_time(e1)
            stats_ms += e1.elapsed_time(e2)
            # bit-exact check of the first 2^16 outputs of three sets per batch against the oracles
            for k in sorted({0, nb // 2, nb - 1}):
                if gen == "mtgp":
                    q = oracle.params_generate(p, k0 + k)
                    ref, _ = oracle.generate(q, oracle.init_state(q, 0), min(C, 1 << 16))
                else:
                    q = omt.params_generate(p, k0 + k)
                    ref, _ = omt.generate(q, omt.init_state(q, 0), min(C, 1 << 16))
                got = out[k * C:k * C + ref.size].cpu().numpy().view(np.uint32)
                exact = exact and bool(np.array_equal(got, ref))
            for i in range(nb):
                pg[k0 + i] = quality.gap_test(hist[i], b=5)["p_value"]
                ph[k0 + i] = quality.hamming_test(tab[i], L=1200, bounds=bounds)["p_value"]
            del st
        ok_g = np.array([inside(v) for v in pg])
        ok_h = np.array([inside(v) for v in ph])
        res[gen] = {"sets": S, "pass_gap": float(ok_g.mean()), "pass_hamming": float(ok_h.mean()),
                    "pass_both": float((ok_g & ok_h).mean()),
                    "gap_p_below_1e-3": int((pg < 1e-3).sum()),
                    "hamming_p_below_1e-3": int((ph < 1e-3).sum()),
                    "failing_gap_sets": [int(i) for i in np.nonzero(~ok_g)[0]],
                    "failing_hamming_sets": [int(i) for i in np.nonzero(~ok_h)[0]],
                    "gen_gnum_s": S * C / (gen_ms * 1e6), "stats_ms": stats_ms,
                    "bit_exact_sample": exact}
    print(json.dumps({"quality_sweep": {"period_exponent": p, "numbers_per_set": C,
                                        "seed_status": 0, "tests": "gap r=25 b=5 t=128; "
                                        "Hamming pairs r=25 s=5 L=1200, 4 classes",
                                        "suspect_bounds": [1e-3, 1 - 1e-3], **res}}), flush=True)


def spot_check(w, counts, out, states0, fmt):
    """Whole outputs of a few streams of the first launch vs the oracle."""
    import oracle
    p_of = oracle_params_of(w)
    offs = np.concatenate([[0], np.cumsum(counts.astype(np.int64))])
    pick = sorted({int(np.argmax(counts)), 0, counts.size - 1, counts.size // 2})
    for s in pick:
        ref, _ = oracle.generate(p_of(s), states0[s], int(counts[s]), fmt)
        got = out[int(offs[s]):int(offs[s + 1])].cpu().numpy().view(np.uint32)
        if not np.array_equal(ref, got):
            return False
    return True


def measure_e2e(mtgp, torch, st, ids, counts, stream, args):
    total = int(counts.sum())
    try:
        host = torch.empty(total, dtype=torch.int32, pin_memory=True)
    except RuntimeError as e:
        return {"value": None, "unit": UNIT, "error": "pinned host buffer: %s" % str(e)[:120]}
    h2d = ids.nbytes + counts.nbytes
    fmt = FORMATS[args.format]
    mtgp.mtgp_generate_to_host(st, ids, counts, fmt, host, 0, stream)   # warm-up
    per = []
    t0 = time.perf_counter()
    for _ in range(args.e2e_steps):
        ts = time.perf_counter()
        mtgp.mtgp_generate_to_host(st, ids, counts, fmt, host, 0, stream)
        per.append(total / (time.perf_counter() - ts) / 1e9)
    dt = time.perf_counter() - t0
    # the device-to-host link is the bound; its rate varies with other
    # traffic to host memory, so the per-step rates are reported as well
    return {"value": total * args.e2e_steps / dt / 1e9, "unit": UNIT,
            "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": 4 * total,
            "steps": args.e2e_steps, "per_step_gnum_s": [round(v, 2) for v in per],
            "api": "mtgp_generate_to_host (pinned host output)"}


def measure_per_stream_launches(mtgp, torch, st, w, out, stream, flush):
    """The uneven workload without batching: one mtgp_generate_u32 call per
    stream, in stream order on one CUDA stream (each call uploads a
    one-stream work table and launches one kernel), timed with CUDA events
    over the whole sequence; whole outputs of a few streams are checked
    against the oracle."""
    counts = w["counts"]
    n = counts.size
    offs = np.concatenate([[0], np.cumsum(counts.astype(np.int64))])
    states0 = mtgp.mtgp_get_statuses(st, stream)
    flush.fill_(3)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t_host = time.perf_counter()
    e0.record(stream)
    for i in range(n):
        mtgp.mtgp_generate_u32(st, np.array([i], np.uint32), counts[i:i + 1],
                               out[int(offs[i]):int(offs[i + 1])], stream)
    e1.record(stream)
    stream.synchronize()
    t_host = time.perf_counter() - t_host
    sec = e0.elapsed_time(e1) / 1e3
    mtgp.mtgp_check(st, stream)
    exact = spot_check(w, counts, out, states0, 0)
    total = int(counts.sum())
    return {"launches": n, "gnum_s": total / sec / 1e9, "ms": 1e3 * sec,
            "host_s": t_host, "bit_exact_sample": exact,
            "how": "mtgp_generate_u32 once per stream, stream order, one CUDA stream"}


# (label, workload, format, split, mexp) of the other configurations measured
# beside the uneven headline: one stream of 2^20 numbers (unsplit, and in 64
# pieces started by jumps), 4096 x 2^18 at Mexp 11213, 1024 x 2^20 at Mexp
# 23209 and 44497 in the three output formats, and the uneven workload at
# the paper's exponent 3217 (unsplit and split).
EXTRA_CONFIGS = [("single stream x 2^20, Mexp 11213, u32", "single", "u32", "0", 0),
                 ("single stream x 2^20, Mexp 11213, u32, 64 pieces", "single", "u32", "16384", 0),
                 ("equal 4096 x 2^18, Mexp 11213, u32", "equal", "u32", "0", 0)] + [
    ("long 1024 x 2^20, Mexp %d, %s" % (m, f), "long%d" % m, f, "0", 0)
    for m in (23209, 44497) for f in ("u32", "f12", "f01")] + [
    ("uneven 10 000 streams, Mexp 3217, u32", "uneven", "u32", "0", 3217),
    ("uneven 10 000 streams, Mexp 3217, u32, split in pieces of total / (48 x SMs)", "uneven", "u32",
     "auto48", 3217)]


def measure_configs(mtgp, torch, dev, stream, flush, steps=5, warmup=3):
    """Each configuration as the headline is measured: an autotuned plan
    (one persistent graph-replayed launch), L2 rewritten between launches,
    CUDA events around each launch; the first launch's whole outputs of the
    first, middle and last streams are checked against the oracle."""
    peak, _ = hbm_peak()
    res = []
    buf = None
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    for label, name, fmt_name, split, mexp in EXTRA_CONFIGS:
        w, desc = workload(name, 0, mexp=mexp)
        counts = w["counts"]
        total = int(counts.sum())
        if buf is None or buf.numel() < total:
            buf = torch.empty(total, dtype=torch.int32, device=dev)
        out = buf[:total]
        fmt = FORMATS[fmt_name]
        params = mtgp.mtgp_params_generate(w["mexp"], workloads.PARAM_SEED)
        st = mtgp.mtgp_init_statuses(params, w["seeds"], stream)
        ids = np.arange(counts.size, dtype=np.uint32)
        plan = mtgp.mtgp_plan_create(st, ids, counts, fmt, out)
        max_piece = split_piece(split, total, sms)
        if max_piece:
            mtgp.mtgp_plan_set_split(plan, max_piece)
        mtgp.mtgp_plan_autotune(plan)
        info = mtgp.mtgp_plan_get_info(plan)
        states0 = mtgp.mtgp_get_statuses(st, stream)
        exact = None
        with torch.cuda.stream(stream):
            for i in range(warmup):
                mtgp.mtgp_plan_launch(plan, stream)
                if i == 0:
                    stream.synchronize()
                    exact = spot_check(w, counts, out, states0, fmt)
                flush.fill_(i)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
              for _ in range(steps)]
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0.record(stream)
        with torch.cuda.stream(stream):
            for i in range(steps):
                ev[i][0].record(stream)
                mtgp.mtgp_plan_launch(plan, stream)
                ev[i][1].record(stream)
                flush.fill_(i)
        t1.record(stream)
        stream.synchronize()
        mtgp.mtgp_check(st, stream)
        kern = sum(a.elapsed_time(b) for a, b in ev) / steps / 1e3
        n_words = mtgp.mtgp_streams_info(st)[1]
        alg = 4.0 * total + 8.0 * n_words * counts.size
        res.append({"config": label, "workload": desc, "format": fmt_name, "numbers": total,
                    "gnum_s": total * steps / (t0.elapsed_time(t1) / 1e3) / 1e9,
                    "kernel_ms_avg": 1e3 * kern, "frac": alg / kern / 1e9 / peak,
                    "launch": info["config"], "bit_exact_sample": exact,
                    "split": {"max_piece": info["max_piece"], "jumps_per_launch": info["n_jumps"]}})
        del plan, st
    return res


def verify_serving_prefix(mtgp, tr, n_streams, budget=1_200_000_000, max_piece=0):
    """Replays the prefix of the serving trace whose results fit the 8 GiB
    arena at once, through continuous batching (split ticks when max_piece),
    recording every result's arena offset; then checks every request of the
    prefix against the oracle's replay of its stream's requests alone and in
    order, and every final state."""
    import oracle
    from concurrent.futures import ThreadPoolExecutor
    cum = np.cumsum(tr["counts"].astype(np.int64))
    n = int(np.searchsorted(cum, budget))
    t, ids, counts, fmts = tr["t"][:n], tr["ids"][:n], tr["counts"][:n], tr["fmt"][:n]
    params = mtgp.mtgp_params_generate(workloads.MEXP_MAIN, workloads.PARAM_SEED)
    st = mtgp.mtgp_init_statuses(params, np.arange(n_streams, dtype=np.uint32))
    states0 = mtgp.mtgp_get_statuses(st)
    srv = mtgp.mtgp_server_create(st, arena_bytes=8 << 30, max_inflight=4, max_piece=max_piece)
    _, offs, _ = mtgp.mtgp_server_run_trace(srv, t, ids, counts, fmts, mode=0, record=True)
    arena = mtgp.mtgp_server_read(srv, 0, int((offs + counts).max()))
    op = oracle.params_generate(workloads.MEXP_MAIN, workloads.PARAM_SEED)
    per = {}
    for j in range(n):
        per.setdefault(int(ids[j]), []).append(j)

    def replay(sid):
        s = states0[sid].copy()
        good = True
        for j in per[sid]:
            ref, s = oracle.generate(op, s, int(counts[j]), int(fmts[j]))
            good = good and bool(np.array_equal(arena[int(offs[j]):int(offs[j]) + int(counts[j])],
                                                ref))
        return good, s

    final = states0.copy()
    ok = True
    with ThreadPoolExecutor(os.cpu_count() or 4) as ex:
        for sid, (good, s) in zip(per, ex.map(replay, list(per))):
            ok = ok and good
            final[sid] = s
    ok = ok and bool(np.array_equal(mtgp.mtgp_get_statuses(st), final))
    srv.close()
    st.close()
    return {"requests": n, "arrivals_s": float(t[-1]), "numbers": int(counts.sum()),
            "bit_exact": ok}


def measure_serving(mtgp, torch, args):
    """Continuous batching vs one launch per request: on the serving trace
    (50 000 requests/s, which overloads the one-launch-per-request arm), and
    on a trace at a rate that arm sustains (its latencies are then service
    times, not backlog).  A third arm batches continuously with requests
    longer than --serving-piece numbers cut into pieces started by exact
    jumps (config max_piece).  Each arm's host time per launch (work-table
    build, upload and kernel launch) is reported beside its latencies."""
    rate_lo, secs_lo = 20000.0, min(5.0, args.serving_seconds)
    traces = [("offered_50k_req_s", workloads.serving_trace(duration_s=args.serving_seconds),
               50000.0, args.serving_seconds),
              ("sustained_20k_req_s", workloads.serving_trace(duration_s=secs_lo, rate=rate_lo),
               rate_lo, secs_lo)]
    n_streams = traces[0][1]["n_streams"]
    params = mtgp.mtgp_params_generate(workloads.MEXP_MAIN, workloads.PARAM_SEED)
    st = mtgp.mtgp_init_statuses(params, np.arange(n_streams, dtype=np.uint32))
    srv = mtgp.mtgp_server_create(st, arena_bytes=8 << 30, max_inflight=4)
    srv_split = None
    if args.serving_piece:
        srv_split = mtgp.mtgp_server_create(st, arena_bytes=8 << 30, max_inflight=4,
                                            max_piece=args.serving_piece)
    res = {"workload": "65536 resident Mexp 11213 streams; Poisson arrivals (seed 11); "
                       "k = floor(2^U), U~U[8,20]; u32 or f32[0,1); arena (admission cap) 8 GiB",
           "split_piece": args.serving_piece}
    arms = [(srv, 0, "continuous_batching"), (srv, 1, "one_launch_per_request")]
    if srv_split:
        arms.append((srv_split, 0, "continuous_batching_split"))
    for key, tr, rate, secs in traces:
        r = {"rate_req_s": rate, "seconds": secs, "requests": int(tr["t"].size),
             "offered_gnum_s": float(tr["counts"].sum()) / secs / 1e9}
        for server, mode, name in arms:
            lat, _, stats = mtgp.mtgp_server_run_trace(server, tr["t"], tr["ids"], tr["counts"],
                                                       tr["fmt"], mode=mode)
            r[name] = {"p50_ms": 1e3 * float(np.percentile(lat, 50)),
                       "p99_ms": 1e3 * float(np.percentile(lat, 99)),
                       "mean_ms": 1e3 * float(lat.mean()),
                       "gnum_s": stats["numbers"] / stats["elapsed"] / 1e9,
                       "kernel_launches": int(stats["ticks"]), "elapsed_s": stats["elapsed"],
                       "host_us_per_launch": 1e6 * stats["launch_host_s"] / max(1, stats["ticks"]),
                       "jumps": int(stats["jumps"])}
        res[key] = r
    if srv_split:
        srv_split.close()
    srv.close()
    st.close()
    if not args.no_serving_parity:
        res["parity_prefix"] = verify_serving_prefix(mtgp, traces[0][1], n_streams)
        if args.serving_piece:
            res["parity_prefix_split"] = verify_serving_prefix(mtgp, traces[0][1], n_streams,
                                                               max_piece=args.serving_piece)
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="uneven", help="uneven | single | equal | long23209 | long44497")
    ap.add_argument("--format", default="u32", choices=sorted(FORMATS),
                    help="u32, f12 (float32 [1,2)) or f01 (float32 [0,1))")
    ap.add_argument("--streams", type=int, default=0, help="equal workload: stream count")
    ap.add_argument("--count", type=int, default=0, help="equal workload: numbers per stream")
    ap.add_argument("--param-sets", type=int, default=0,
                    help="one parameter set per stream group: K distinct sets, stream s uses set "
                         "s mod K (0 = one shared set)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--serving-seconds", type=float, default=10.0,
                    help="length of the serving trace (0 = skip the serving measurement)")
    ap.add_argument("--serving-piece", type=int, default=1 << 16,
                    help="serving arm with requests longer than this cut into pieces started by "
                         "jumps (server max_piece; 0 = no such arm)")
    ap.add_argument("--config", default="",
                    help="force warps_per_cta,words_per_lane,coop_percent[,ctas_per_sm[,kernel]] "
                         "(skips autotuning)")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-quality", dest="quality", action="store_false",
                    help="skip the gap and Hamming-weight statistics over the generated output")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extra", action="store_true",
                    help="skip the equal/long workloads and the one-launch-per-stream comparison")
    ap.add_argument("--no-serving-parity", action="store_true",
                    help="skip the oracle replay of the serving trace's prefix")
    ap.add_argument("--split", default="0",
                    help="cut streams longer than this many numbers into pieces started by exact "
                         "jumps (mtgp_plan_set_split); 'auto' = the numbers per warp slot at 16 warps "
                         "per SM; 'autoW' = the launch cut into W pieces per SM; 0 = off")
    ap.add_argument("--ranks", dest="rank_split", default="weak", choices=["weak", "strong"],
                    help="N > 1: weak = one workload instance per GPU; strong = one instance cut "
                         "into contiguous stream ranges")
    ap.add_argument("--mexp", type=int, default=0,
                    help="MTGP exponent of the workload (0 = the workload's own, 11213 for uneven)")
    ap.add_argument("--generator", default="mtgp", choices=["mtgp", "mt"],
                    help="mt: the original Mersenne Twister of Sec. 5.3 on the same workload")
    ap.add_argument("--quality-sweep", type=int, default=0,
                    help="S > 0: tests 35 and 100 over S parameter sets of MTGP and of the original "
                         "MT at period 2^mexp (default 3217), one stream each (Sec. 5.3)")
    ap.add_argument("--sweep-count", type=int, default=1 << 24, help="numbers per set in the sweep")
    ap.add_argument("--sweep-batch", type=int, default=1000, help="sets per launch in the sweep")
    ap.add_argument("--mt-p", type=int, default=3217,
                    help="exponent of the original-MT set (19937 = MT19937, else seed-generated)")
    args = ap.parse_args()
    if args.warmup < 3:
        raise SystemExit("--warmup must be >= 3")
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world != args.gpus:
        raise SystemExit("--gpus %d but WORLD_SIZE %d: launch N > 1 with torchrun" % (args.gpus, world))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
    elif args.quality_sweep:
        run_quality_sweep(args)
    elif args.generator == "mt":
        run_mt(args, rank, world, local_rank)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
