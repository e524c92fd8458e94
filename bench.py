#!/usr/bin/env python
"""Benchmark: exact Jones-polynomial evaluation of the 64-knot random grid-walk workload.

Workload ("scale"): 64 random grid-walk knots, grid side L=40, seeds 1..64 (rank r of
N uses seeds 64r+1..64r+64), each redrawn until it has 100..400 crossings, random
over/under per crossing; every knot is evaluated at q = 2, 3, 5 (t = i, e^{i pi/3},
(3+sqrt 5)/2).  One step = Z(q) and V_K(t(q)) for all 64 x 3 = 192 (knot, q) pairs, all
on the GPU through libpk.  `value` is knot evaluations per second (one knot = one
(knot, q) pair), whole job, in the headline precision (split FP32 by default), with
every plan's program resident in HBM (one workspace per plan) and the 192 plans'
launch sequences replayed as independent branches of one CUDA graph; L2 is flushed
between steps.  The same workload is then run once in
complex64 and once in complex128; the relative error of every evaluation against
complex128 is reported.

The default line also carries the in-step roofline (one replay of the same graph with an
event pair around every launch, read per kernel class), the CPU oracle on the host cores
(single-core and all-core on one identical sample), and two further workloads measured on
the same GPU: `batch` (4096 small knots in one persistent launch) and `grad` (the reverse
pass of one 300-crossing knot).

--impl reference times the CPU oracle (complex128 spin elimination in numpy, one
evaluation per process on all host cores) on a bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

T0 = time.perf_counter()
SM_COUNT, FP32_LANES, SM_MAX_GHZ = 152, 128, 2.070
FP32_CORE_TFLOPS = SM_COUNT * FP32_LANES * 2 * SM_MAX_GHZ / 1e3   # FMA = 2 flops
FP32_ISSUE_TOPS = SM_COUNT * FP32_LANES * SM_MAX_GHZ / 1e3         # FP32 instructions
FF_INSTR_PER_CMAC = 48   # float-float complex multiply-add: 4 x (two-product + TwoSum)
FP64_TFLOPS = 1.25       # GB300 FP64 rate
TC_PAIRS = 15            # BF16 digit pairs per real multiply-add on the tensor cores (5 digits)


def log(msg):
    print(f"[bench {time.perf_counter() - T0:7.1f}s] {msg}", file=sys.stderr, flush=True)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="split", choices=["split", "c64", "c128"])
    ap.add_argument("--skip-compare", action="store_true",
                    help="omit the complex64 / complex128 comparison passes")
    ap.add_argument("--qs", default="2,3,5")
    ap.add_argument("--knots", type=int, default=64, help="knots per GPU (64 = the workload)")
    ap.add_argument("--first", type=int, default=0,
                    help="index of the first knot taken from the rank's workload (profiling subsets)")
    ap.add_argument("--skip-cpu", action="store_true", help="omit the oracle baseline")
    ap.add_argument("--skip-extra", action="store_true",
                    help="omit the batch and grad workloads of the default line")
    ap.add_argument("--refine", type=int, default=8,
                    help="subtree reconfiguration of the cheapest candidate orders, frontiers of "
                         "up to this many subtrees (pk_plan_opts.refine; 0 = off)")
    ap.add_argument("--restarts", type=int, default=256,
                    help="min-fill restarts per plan (planning effort; plans are built once, "
                         "before the timed region, on all host cores)")
    ap.add_argument("--workload", default="scale", choices=["scale", "batch", "large"],
                    help="scale: 64 knots at q=2,3,5 (default); batch: 4096 knots at q=3 "
                         "in one persistent launch; large: 8 knots of 600-1000 crossings and "
                         "their Reidemeister-moved copies")
    ap.add_argument("--large-budget", type=float, default=5e13,
                    help="large workload: complex multiply-adds allowed per evaluation")
    return ap.parse_args()


KNOTS_PER_RANK = 64
METRIC = "knot evaluations per second (exact Z(q), V_K(t(q))), split-FP32 vs complex128"
ORACLE_MAX_ENTRIES = 1 << 24   # CPU samples: largest oracle factor after a spin is summed out


def shard_seeds(rank, n=KNOTS_PER_RANK):
    """Seeds of rank r's knots: 64r+1 .. 64r+64 (weak scaling: fixed work per GPU, no
    knot shared between ranks)."""
    return [KNOTS_PER_RANK * rank + s for s in range(1, n + 1)]


def workload(rank, n=KNOTS_PER_RANK):
    import knotgen as kg
    return [kg.random_grid_knot(40, s, True, 100, 400) for s in shard_seeds(rank, n)]


def max_over_ranks(x, dist, device):
    """The largest of every rank's x (the step time of the slowest rank); x itself when
    running alone."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(world, units_per_rank, step_ms):
    """Whole-job throughput: the units all ranks processed per second of the slowest."""
    return world * units_per_rank / (step_ms / 1000.0)


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "_fallback": True}


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self, dev):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits",
                                       "-lms", "200", "-i", str(dev)], stdout=self.f,
                                      stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
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
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def _oracle_one(job):
    """One (knot, q) evaluation by the CPU oracle in a worker process: min-fill spin
    order (oracle.order), Z by spin elimination, V = A(q) Z.  Returns (key, seconds) or
    (key, None) when a factor would exceed ORACLE_MAX_ENTRIES entries (q^(w-1) for a bucket
    of w spins)."""
    sys.path.insert(0, ROOT)
    import oracle
    from oracle.order import min_fill_order
    key, pd, outer, q = job
    t0 = time.perf_counter()
    g = oracle.tait_graph(pd, outer=outer)
    order, w = min_fill_order(g.n_v, g.edges, q, restarts=4)
    if q ** (w - 1) > ORACLE_MAX_ENTRIES:
        return key, None
    z = oracle.z_complex(g.n_v, g.edges, q, order=order, sum_inside=True)
    oracle.jones_from_z(z, g, q)
    return key, time.perf_counter() - t0


def _oracle_pool(procs):
    """A spawn pool of single-threaded oracle workers (numpy's BLAS held to one thread
    per process, so `procs` is the number of cores used)."""
    import multiprocessing as mp
    for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
        os.environ[v] = "1"
    return mp.get_context("spawn").Pool(procs)


def oracle_jobs(knots, qs):
    return [(f"{gk.seed}@q{q}", gk.pd, gk.outer, q) for gk in knots for q in qs]


def cpu_oracle_baseline(knots, qs, budget_s=12.0):
    """The oracle as it stands on the host cores: a sample of the workload chosen in
    workload order by a single-core run of about budget_s seconds, then the same sample
    on all cores (one evaluation per process).  Evaluations too wide for the oracle
    (a factor above ORACLE_MAX_ENTRIES entries) are skipped and counted."""
    jobs = oracle_jobs(knots, qs)
    sample, skipped, t_single = [], 0, 0.0
    with _oracle_pool(1) as pool:
        t0 = time.perf_counter()
        for job, (key, dt) in zip(jobs, pool.imap(_oracle_one, jobs)):
            if dt is None:
                skipped += 1
            else:
                sample.append(job)
            if time.perf_counter() - t0 > budget_s:
                pool.terminate()
                break
        t_single = time.perf_counter() - t0
    ncpu = os.cpu_count() or 1
    with _oracle_pool(ncpu) as pool:
        pool.map(_oracle_one, sample[:ncpu])          # workers import numpy first
        t0 = time.perf_counter()
        pool.map(_oracle_one, sample, chunksize=1)
        t_all = time.perf_counter() - t0
    n = len(sample)
    text = (f"the first {n + skipped} (knot, q) evaluations in workload order "
            f"({jobs[0][0]}..{sample[-1][0] if sample else '-'}), {skipped} skipped as needing an "
            f"oracle factor above 2^24 entries; {n} timed")
    return {"value": n / t_all, "unit": "knots/s", "cores": ncpu, "kind": "oracle",
            "sample": text, "single_core": {"value": n / t_single, "cores": 1},
            "all_core": {"value": n / t_all, "cores": ncpu}}


def run_reference(args):
    """The oracle as the reference arm: each step evaluates one bounded sample of the
    scale workload (the evaluations in workload order that fit the oracle and that an
    all-core warm-up finished within about 6 s) on all host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    qs = tuple(int(x) for x in args.qs.split(","))
    jobs = oracle_jobs(workload(0), qs)
    ncpu = os.cpu_count() or 1
    with _oracle_pool(ncpu) as pool:
        sample, skipped = [], 0
        t0 = time.perf_counter()
        for job, (key, dt) in zip(jobs, pool.imap(_oracle_one, jobs)):
            if dt is None:
                skipped += 1
            else:
                sample.append(job)
            if time.perf_counter() - t0 > 6.0:
                break
        for _ in range(max(0, args.warmup - 1)):
            pool.map(_oracle_one, sample, chunksize=1)
        times = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            pool.map(_oracle_one, sample, chunksize=1)
            times.append(time.perf_counter() - t0)
    step = sum(times) / len(times)
    v = len(sample) / step
    text = (f"{len(sample)} (knot, q) evaluations per step: the first that fit the oracle in "
            f"workload order ({sample[0][0]}..{sample[-1][0]}), {skipped} skipped as needing an "
            f"oracle factor above 2^24 entries")
    out = {"impl": "reference", "metric": METRIC,
           "value": v, "unit": "knots/s", "n_gpus": args.gpus, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": 1000 * step,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
           "data": "synthetic",
           "config": {"workload": "scale: 64 grid-walk knots L=40, 100-400 crossings, q in {2,3,5}",
                      "impl": "CPU oracle, numpy complex128 spin elimination, min-fill order, "
                              "one evaluation per process"},
           "cpu_baseline": {"value": v, "unit": "knots/s", "cores": ncpu, "kind": "oracle",
                            "sample": text},
           "e2e": {"value": v, "unit": "knots/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


# bound of each kernel class (see the design doc's kernel table): the tensor-core GEMM by the
# tensor pipe, the CUDA-core GEMM by its arithmetic units, everything else by HBM
CLASS_KERNEL = {"build": "k_build", "rows": "k_rows / k_outs / k_seg (fused permute-and-contract)",
                "splitk": "k_splitk", "results": "k_slice_result / k_sum_slices",
                "gemm": "k_gemm (tiled strided complex GEMM, CUDA cores)",
                "gemm_tc": "k_gemm_tc (complex GEMM on tcgen05 tensor cores, BF16 digit products)",
                "digits": "k_digits (operand digits for k_gemm_tc)"}
# DRAM traffic (ncu dram__bytes_read.sum + dram__bytes_write.sum) of one captured launch
# divided by that launch's algorithmic bytes as the library counts them (its storage type,
# 16 bytes per complex entry in split): the multiple applied to a class's average launch.
# Sources (the heaviest launch of each class in the workload, knot seed 11 at q = 5):
# tensor-core GEMM profiles/k_gemm_tc_split_q5_seed11.md (2.008 GB against (9.77 M + 9.77 M
# + 48.8 M) x 16 B), digits profiles/k_digits_split_q5_seed11.md (2.599 GB against the
# operands it reads, (48.8 M + 9.77 M) x 16 B).  The row kernels (2% of the step) have no
# capture of a launch large enough to leave its output in DRAM.
NCU_TRAFFIC_RATIO = {"gemm_tc": 2.008012 / 1.09375, "digits": 2.599281 / 0.9375}


def roofline_blocks(classes, prec, pk_, instep=None):
    """Per kernel class of the serialised event pass (launches one after another, a CUDA
    event pair around each, on the stream they are launched on): achieved = algorithmic
    bytes (or flops) per launch / average launch duration, against the measured peak.  The
    dominant class is the one with the largest GPU-fill-weighted time: each launch's
    duration times the share of the GPU's CTA slots it fills, which is what a launch costs
    the concurrent step (many plans' launches overlap there; a one-CTA launch costs almost
    nothing).  Algorithmic bytes follow the step definition e (|A| + |B| + |C|) with e = 8
    for complex64 and split storage, 16 for complex128 (the library counts the bytes of its
    storage type, 16 for split, so halved here)."""
    e_scale = 0.5 if prec == "split" else 1.0
    out = {}
    tot_fill = sum(d.get("fill_ms", 0.0) for d in classes.values()) or 1.0
    tot_ms = sum(d["ms"] for d in classes.values()) or 1.0
    for c, d in classes.items():
        if d["launches"] <= 0 or d["ms"] <= 0:
            continue
        avg_s = d["ms"] / d["launches"] / 1e3
        alg_bytes = d["bytes"] * e_scale / d["launches"]
        flops = 8.0 * d["cmacs"] / d["launches"]
        if c == "gemm_tc":
            burst = pk_["bf16_tflops"]
            peak = burst / TC_PAIRS
            ach = flops / avg_s / 1e12
            blk = {"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                   "peak_source": f"measured dense BF16 burst {burst} TFLOP/s (of measured, "
                                  f"MEASURED_PEAKS.json; the kernel is timed alone) / {TC_PAIRS} "
                                  f"BF16 digit-pair products per real multiply-add"}
        elif c == "gemm" and prec != "c128":
            peak = FP32_ISSUE_TOPS / FF_INSTR_PER_CMAC * 8 if prec == "split" else FP32_CORE_TFLOPS
            ach = flops / avg_s / 1e12
            blk = {"bound": "alu", "achieved": ach, "peak": peak, "unit": "TFLOP/s",
                   "peak_source": "derived from 152 SM x 128 FP32 lanes x 2.07 GHz"}
        else:
            peak = pk_["hbm_gbs"]
            ach = alg_bytes / avg_s / 1e9
            blk = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                   "peak_source": "measured copy bandwidth (of measured, MEASURED_PEAKS.json hbm_gbs)"}
        ratio = NCU_TRAFFIC_RATIO.get(c)
        blk.update({"frac": ach / peak, "kernel": CLASS_KERNEL[c],
                    "traffic": ratio * d["bytes"] / d["launches"] if ratio else None,
                    "traffic_unit": "bytes per launch (DRAM read + write)",
                    "launches": d["launches"], "avg_launch_us": 1e6 * avg_s,
                    "serialised_ms": d["ms"], "share_serialised": d["ms"] / tot_ms,
                    "fill_weighted_ms": d.get("fill_ms"),
                    "share_fill_weighted": d.get("fill_ms", 0.0) / tot_fill,
                    "alg_bytes_per_launch": alg_bytes, "flops_per_launch": flops,
                    "units": "algorithmic bytes e(|A|+|B|+|C|), e = 8 (complex64 / split) or 16 "
                             "(complex128); flops = 8 per complex multiply-add"})
        if instep and c in instep:
            blk["in_step_summed_ms"] = instep[c]["ms"]
        out[c] = blk
    dom = max(out, key=lambda c: out[c]["fill_weighted_ms"] or 0.0)
    return dict(out[dom], kernel_class=dom), out


def batch_workload(pk, ctx, stream, flush, args):
    """4096 grid-walk knots of 18..122 crossings at q = 3 in ONE persistent launch (a CUDA
    graph), split and complex128: device time per launch with inputs resident, and end to
    end per step: the knot-derived inputs (knot headers, initial-tensor recipes) from pinned
    memory, the launch, the results back; the plans' step records stay resident, as the
    scale workload's plans do (and, for comparison, with the whole image re-sent)."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    import knotgen as kg
    knots = kg.knot_suite("batch")
    t0 = time.perf_counter()
    kn = [pk.Knot.from_pd(ctx, k.pd, outer=k.outer) for k in knots]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        plans = list(ex.map(lambda k: pk.Plan(ctx, k, 3), kn))
    plan_s = time.perf_counter() - t0
    cm = sum(p.stats()["cmacs"] for p in plans)
    out, res = {"workload": "4096 grid-walk knots, 18-122 crossings (target uniform 20-120, L "
                            "from the target), q=3, one persistent launch in a CUDA graph",
                "plan_seconds": plan_s, "complex_macs_per_step": cm}, {}
    for pr in ("split", "c128"):
        b = pk.Batch(plans, pr)
        nbytes, upbytes = b.workspace_bytes()
        ws = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
        b.upload(ws)
        for _ in range(max(3, args.warmup)):
            b.launch(ws)
        torch.cuda.synchronize()
        times = []
        for _ in range(args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            b.launch(ws)
            e.record(stream)
            e.synchronize()
            times.append(a.elapsed_time(e))
        ms = sum(times) / len(times)
        res[pr] = b.download(ws)
        torch.cuda.synchronize()
        def e2e(upload):
            upload(ws)                  # one untimed pass
            b.launch(ws)
            b.download(ws)
            t1 = time.perf_counter()
            for _ in range(args.steps):
                upload(ws)
                b.launch(ws)
                b.download(ws)
            return 1e3 * (time.perf_counter() - t1) / args.steps

        inbytes = b.upload_inputs(ws)
        full_ms = e2e(b.upload)
        e2e_ms = e2e(b.upload_inputs)
        out[pr] = {"value": len(plans) / (ms / 1e3), "unit": "knots/s", "ms_per_step": ms,
                   "complex_tflops": 8 * cm / (ms / 1e3) / 1e12,
                   "e2e": {"value": len(plans) / (e2e_ms / 1e3), "unit": "knots/s",
                           "h2d_bytes_per_step": inbytes, "d2h_bytes_per_step": 32 * len(plans)},
                   "e2e_whole_image": {"value": len(plans) / (full_ms / 1e3), "unit": "knots/s",
                                       "h2d_bytes_per_step": upbytes,
                                       "d2h_bytes_per_step": 32 * len(plans)}}
        del ws, b
        torch.cuda.empty_cache()
    errs = [max(rel_err(z, zr), rel_err(v, vr)) for z, v, zr, vr in
            zip(res["split"][0], res["split"][1], res["c128"][0], res["c128"][1])]
    out["split"].update({"max_rel_err_vs_c128": max(errs),
                         "evaluations_over_1e-6": sum(x > 1e-6 for x in errs)})
    return out


def grad_workload(pk, ctx, stream, args):
    """The reverse pass of one 300-crossing grid-walk knot (L=53, seed 7) at q = 3 with
    intermediates checkpointed every 4th tree level: Z, d log Z over every edge weight and
    dV/dt per pk_grad call, complex128 and split; the split result against complex128."""
    import numpy as np
    import torch
    import knotgen as kg
    (gk,) = kg.knot_suite("grad")
    k = pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer)
    p = pk.Plan(ctx, k, 3, grad=True, checkpoint_stride=4)
    gs = p.grad_stats()
    out = {"workload": f"L=53 seed 7, {k.info()['n_c']} crossings, q=3, checkpoint stride 4",
           "complex_macs_per_call": gs["cmacs_forward"] + gs["cmacs_recompute"] + gs["cmacs_adjoint"],
           "steps_per_call": gs["steps_forward"] + gs["steps_recompute"] + gs["steps_adjoint"]}
    res = {}
    for pr in ("c128", "split"):
        ws = torch.empty(p.grad_workspace_bytes(pr), dtype=torch.uint8, device="cuda")
        for _ in range(3):
            res[pr] = pk.grad(p, pr, ws)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        n = max(3, args.steps)
        for _ in range(n):
            pk.grad(p, pr, ws)
        out[pr] = {"ms_per_call": 1e3 * (time.perf_counter() - t0) / n,
                   "note": "host clock around blocking pk_grad calls (results on the host)"}
        del ws
    d128, dsp = res["c128"][2], res["split"][2]
    out["split"]["max_rel_err_dlogz_vs_c128"] = float(np.max(np.abs(dsp - d128)) / np.max(np.abs(d128)))
    out["split"]["rel_err_dlogv_dt_vs_c128"] = abs(res["split"][3] - res["c128"][3]) / abs(res["c128"][3])
    return out


def rel_err(a, b):
    """|a - b| / |b| for two pk.Scaled values."""
    d = a.exp2 - b.exp2
    ma = a.mantissa * (2.0 ** d if d > -1000 else 0.0)
    return abs(ma - b.mantissa) / abs(b.mantissa) if b.mantissa != 0 else abs(ma)


def run_batch(args):
    """4096 grid-walk knots of 18..122 crossings at q = 3, all in one persistent launch
    (CUDA graph), in split FP32, complex128 and complex64; plus complex128 one knot at
    a time.  Errors against batched complex128."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import knotgen as kg
    import paper_1807_02119_gb300 as pk
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    ctx = pk.Context(local)
    stream = torch.cuda.current_stream()
    ctx.set_stream(stream.cuda_stream)
    knots = kg.knot_suite("batch")
    t0 = time.perf_counter()
    plans = [pk.Plan(ctx, pk.Knot.from_pd(ctx, k.pd, outer=k.outer), 3) for k in knots]
    plan_s = time.perf_counter() - t0
    log(f"planned {len(plans)} knots in {plan_s:.1f}s")
    cm = sum(p.stats()["cmacs"] for p in plans)
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    res, line = {}, {}
    for pr in ("split", "c128", "c64"):
        b = pk.Batch(plans, pr)
        ws = torch.empty(b.workspace_bytes()[0], dtype=torch.uint8, device="cuda")
        b.upload(ws)
        for _ in range(args.warmup):
            b.launch(ws)
        torch.cuda.synchronize()
        times = []
        clocks = Clocks(local) if pr == "split" else None
        for _ in range(args.steps):
            flush.zero_()
            a = torch.cuda.Event(enable_timing=True)
            e = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            b.launch(ws)
            e.record(stream)
            e.synchronize()
            times.append(a.elapsed_time(e))
        if clocks:
            line["clocks"] = clocks.stop()
        ms = sum(times) / len(times)
        res[pr] = b.download(ws)
        line[pr] = {"value": len(plans) / (ms / 1e3), "unit": "knots/s", "ms_per_step": ms,
                    "complex_tflops": 8 * cm / (ms / 1e3) / 1e12}
        if pr == "split":
            t1 = time.perf_counter()
            b.upload(ws)
            b.launch(ws)
            b.download(ws)
            line["e2e"] = {"value": len(plans) / (time.perf_counter() - t1), "unit": "knots/s",
                           "h2d_bytes_per_step": b.workspace_bytes()[1],
                           "d2h_bytes_per_step": 32 * len(plans)}
        del ws, b
        torch.cuda.empty_cache()
        log(f"batched {pr}: {ms:.2f} ms per 4096 knots")
    for pr in ("split", "c64"):
        errs = [max(rel_err(z, zr), rel_err(v, vr)) for z, v, zr, vr in
                zip(res[pr][0], res[pr][1], res["c128"][0], res["c128"][1])]
        line[pr].update({"max_rel_err_vs_c128": max(errs),
                         "evaluations_over_1e-6": sum(x > 1e-6 for x in errs)})
    # complex128 one knot at a time (the plain per-knot contraction)
    big = max(p.workspace_bytes("c128") for p in plans)
    ws = torch.empty(big + 256, dtype=torch.uint8, device="cuda")
    for p in plans[:16]:
        pk.evaluate(p, "c128", ws)
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    e = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for p in plans:
        pk.upload(p, "c128", ws)
        pk.launch(p, "c128", ws)
    e.record(stream)
    e.synchronize()
    ms = a.elapsed_time(e)
    line["c128_one_knot_per_launch_sequence"] = {"value": len(plans) / (ms / 1e3), "unit": "knots/s",
                                                 "ms_per_step": ms}
    out = {"metric": "knot evaluations per second, 4096 knots in one persistent launch",
           "value": line["split"]["value"], "unit": "knots/s", "n_gpus": 1, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": line["split"]["ms_per_step"],
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "split",
           "data": "synthetic",
           "config": {"workload": "batch: 4096 grid-walk knots, 18-122 crossings (target uniform "
                                  "20-120, L from the target), q=3, one persistent launch in a CUDA graph",
                      "plan_seconds": plan_s, "complex_macs_per_step": cm,
                      "l2": "flushed between steps (512 MB write)"},
           "precisions": line, "e2e": line.get("e2e"), "clocks": line.get("clocks")}
    print(json.dumps(out))


def run_large(args):
    """8 grid-walk knots of 600-1000 crossings (L=86) and a Reidemeister-moved copy of
    each, in split precision, one evaluation at a time: q = 2 for all, q = 3 where the
    plan fits the budget; q = 4 and 6 are reported with their planned work.  Checks that
    hold at any size: V = +-1 at q = 2, |V|^2 a power of 3 at q = 3, copy = original."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import knotgen as kg
    import paper_1807_02119_gb300 as pk
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    ctx = pk.Context(local)
    stream = torch.cuda.current_stream()
    ctx.set_stream(stream.cuda_stream)
    ctx.set_hbm_budget(int(180e9))          # the workload's device-memory budget
    pairs = list(zip(kg.knot_suite("large"), kg.knot_suite("large_moved")))
    evals, skipped, checks = [], [], []
    tot_ms = tot_cm = 0.0
    t_plan = time.perf_counter()
    work = []
    for i, (gk, mv) in enumerate(pairs):
        ks = [pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer), pk.Knot.from_pd(ctx, mv.pd)]
        for q in (2, 3, 4, 6):
            plans = []
            for kk in ks:
                try:
                    plans.append(pk.Plan(ctx, kk, q, restarts=512 if q == 3 else 64))
                except pk.PkError as e:
                    plans.append(None)
            cms = [p.stats()["cmacs"] if p else float("inf") for p in plans]
            if max(cms) > args.large_budget:
                # not run: the planned work (or, past the slice limit, the unsliced work of the
                # order search alone) and the seconds it would take at this run's rate
                feas = []
                for kk, p in zip(ks, plans):
                    if p is not None:
                        st = p.stats()
                        feas.append({"cmacs": st["cmacs"], "slices": st["n_slices"],
                                     "workspace_gb": st["workspace_split"] / 1e9})
                    else:
                        o = kk.order_stats(q, "fill_spin", 64)
                        feas.append({"cmacs": 2.0 ** o["log2_work"], "slices": None,
                                     "delta_h": o["delta_h"], "note": "more than 2^40 slices"})
                skipped.append({"knot": i, "q": q, "copies": feas})
                continue
            work.append((i, q, ks, plans))
    plan_s = time.perf_counter() - t_plan
    log(f"planned; {len(work)} (knot, q) pairs to run, {len(skipped)} over budget")
    for i, q, ks, plans in work:
        vs = []
        for which, p in zip(("original", "moved"), plans):
            ws = torch.empty(p.workspace_bytes("split") + 256, dtype=torch.uint8, device="cuda")
            pk.upload(p, "split", ws)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            pk.launch(p, "split", ws)
            b.record(stream)
            b.synchronize()
            ms = a.elapsed_time(b)
            z, v = pk.download(p, "split", ws)
            del ws
            torch.cuda.empty_cache()
            st = p.stats()
            tot_ms += ms
            tot_cm += st["cmacs"]
            vs.append(v)
            evals.append({"knot": i, "copy": which, "q": q, "crossings": ks[0 if which == "original" else 1].info()["n_c"],
                          "ms": ms, "cmacs": st["cmacs"], "slices": st["n_slices"],
                          "log2_max_elems": st["log2_max_elems"]})
            log(f"knot {i} {which} q={q}: {ms:.1f} ms, {st['cmacs']:.2e} cMACs")
        v0, v1 = vs
        if q == 2:
            ok = all(abs(abs(v.to_complex().real) - 1) < 1e-6 and abs(v.to_complex().imag) < 1e-6
                     for v in vs) and round(v0.to_complex().real) == round(v1.to_complex().real)
        else:
            l3 = (2 * math.log2(abs(v0.mantissa)) + 2 * v0.exp2) / math.log2(3)
            ok = abs(l3 - round(l3)) < 1e-5 and rel_err(v1, v0) < 1e-6
        checks.append({"knot": i, "q": q, "ok": bool(ok)})
    rate = tot_cm / (tot_ms / 1e3) if tot_ms > 0 else None     # complex MACs per second
    for sk in skipped:
        for f in sk["copies"]:
            f["est_seconds_at_this_rate"] = f["cmacs"] / rate if rate else None
    out = {"metric": "knot evaluations per second, 600-1000-crossing knots (split)",
           "value": len(evals) / (tot_ms / 1e3), "unit": "knots/s", "n_gpus": 1, "steps": 1,
           "warmup": 0, "ms_per_step": tot_ms, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "split", "data": "synthetic",
           "config": {"workload": "large: 8 grid-walk knots L=86, 600-1000 crossings, and a "
                                  "Reidemeister I/II-moved copy of each; q=2 all, q=3 within "
                                  f"{args.large_budget:.0e} complex multiply-adds; one "
                                  "evaluation at a time, the first launch of each plan timed; "
                                  "plans sliced to fit a 180 GB device-memory budget",
                      "plan_seconds": plan_s, "complex_macs": tot_cm,
                      "complex_tflops": 8 * tot_cm / (tot_ms / 1e3) / 1e12},
           "checks_passed": sum(c["ok"] for c in checks), "checks": checks,
           "evaluations": evals, "over_budget": skipped}
    print(json.dumps(out))


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batch":
        run_batch(args)
        return
    if args.workload == "large":
        run_large(args)
        return
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    import __graft_entry__
    __graft_entry__.build()
    import paper_1807_02119_gb300 as pk

    qs = tuple(int(x) for x in args.qs.split(","))
    knots = workload(rank)[args.first:args.first + args.knots]
    ctx = pk.Context(local)
    stream = torch.cuda.current_stream()
    ctx.set_stream(stream.cuda_stream)
    t0 = time.perf_counter()
    from concurrent.futures import ThreadPoolExecutor
    # reconfiguration ranks sequences by the split precision's tensor-core cost model
    refine = args.refine if args.precision == "split" else 0
    args.refine = refine
    kn = [pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer) for gk in knots]
    jobs = [(k, q) for k in kn for q in qs]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:   # planning is host C++
        plans = list(ex.map(lambda kq: pk.Plan(ctx, kq[0], kq[1], restarts=args.restarts,
                                                   refine=refine), jobs))
    plan_s = time.perf_counter() - t0
    log(f"planned {len(plans)} evaluations in {plan_s:.2f}s")
    stats = [p.stats() for p in plans]
    prec = args.precision
    dev = f"cuda:{local}"

    def workspaces(pr, pl=plans):
        """A full workspace per plan (program uploaded, resident in HBM)."""
        ws = [torch.empty(p.workspace_bytes(pr) + 256, dtype=torch.uint8, device=dev) for p in pl]
        for p, w in zip(pl, ws):
            pk.upload(p, pr, w)
        return ws

    def results(pr, ws, pl=plans):
        return [pk.download(p, pr, w) for p, w in zip(pl, ws)]

    # every plan's kernels recorded as an independent branch of one CUDA graph
    ws = workspaces(prec)
    group = pk.Group(plans, prec, ws)
    torch.cuda.synchronize()
    flush = torch.empty(512 * 1024 * 1024, dtype=torch.uint8, device=dev)
    log("workspaces and graph ready")

    # warm-up: W replays; then one sequential pass with an event pair around every launch
    # (serialised: comparable with the shares of ncu's launch list, not with the step)
    for _ in range(args.warmup):
        group.launch()
    torch.cuda.synchronize()
    prof = {}
    for p, w in zip(plans, ws):
        for kname, d in pk.profile(p, prec, w).items():
            acc = prof.setdefault(kname, {"ms": 0.0, "launches": 0.0, "cmacs": 0.0, "bytes": 0.0,
                                          "fill_ms": 0.0})
            for f in acc:
                acc[f] += d[f]
    group.launch()
    torch.cuda.synchronize()
    res_main = results(prec, ws)
    log("warm-up done")

    # timed region: K replays, L2 flushed between steps (outside the events)
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    times = []
    for _ in range(args.steps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        group.launch()
        b.record(stream)
        b.synchronize()
        times.append(a.elapsed_time(b))
    torch.cuda.synchronize()
    clk = clocks.stop()
    log(f"timed {args.steps} steps")
    step_ms = max_over_ranks(sum(times) / len(times), dist, dev)
    evals = len(plans)
    value = job_rate(world, evals, step_ms)

    # end to end through the public API, every step: every plan's knot-derived inputs
    # host->device from pinned memory (its initial-tensor recipes and slots; the
    # sequence-kernel step records stay resident like the rest of the plan's structure,
    # which its graph holds), the kernels, every scaled result device->host (one wait for
    # all); the mean over the same number of steps.  Also with every whole program re-sent.
    d2h = 32 * len(plans)

    def e2e(inputs_only):
        group.upload(inputs_only)          # one untimed pass
        group.launch()
        group.download()
        torch.cuda.synchronize()
        if dist:
            dist.barrier()
        t1 = time.perf_counter()
        for _ in range(args.steps):
            nb = group.upload(inputs_only)
            group.launch()
            group.download()
        return max_over_ranks((time.perf_counter() - t1) / args.steps, dist, dev), nb

    full_s, h2d_full = e2e(False)
    e2e_s, h2d = e2e(True)
    e2e_val = job_rate(world, evals, 1000.0 * e2e_s)
    log("end-to-end pass")

    # in-step profile: one replay of the same step as a graph with an event pair around
    # every launch (event-record nodes), so each launch's duration is taken while it runs
    # among the other plans' launches; on the same resident workspaces
    pgroup = pk.Group(plans, prec, ws, profiled=True)
    pgroup.launch()
    torch.cuda.synchronize()
    flush.zero_()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    a.record(stream)
    pgroup.launch()
    b.record(stream)
    b.synchronize()
    instep = pgroup.profile()
    instep_ms = a.elapsed_time(b)
    del pgroup, group, ws
    torch.cuda.empty_cache()
    log("in-step profile")
    roof, rooflines = roofline_blocks(prof, prec, peaks(), instep)

    # the same workload once in each other precision (same concurrent execution);
    # errors against complex128
    compare = {}
    res_by = {prec: res_main}
    if not args.skip_compare:
        # complex64 and complex128 keep GEMM-shaped row steps (N < 32) on the row kernel,
        # where the reconfigured sequences (ranked by the tensor-core cost model) are slow:
        # they run the same knots' plans without reconfiguration
        cplans = plans
        if args.refine > 0:
            with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
                cplans = list(ex.map(lambda kq: pk.Plan(ctx, kq[0], kq[1], restarts=args.restarts),
                                     jobs))
        for pr in ("c64", "c128"):
            if pr == prec:
                continue
            ws2 = workspaces(pr, cplans)
            g2 = pk.Group(cplans, pr, ws2)
            g2.launch()                         # loads the kernels
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            g2.launch()
            b.record(stream)
            b.synchronize()
            ms = max_over_ranks(a.elapsed_time(b), dist, dev)
            res_by[pr] = results(pr, ws2, cplans)
            compare[pr] = {"value": world * evals / (ms / 1000.0), "unit": "knots/s",
                           "ms_per_step": ms, "note": "one timed replay after a warm-up replay"
                           + ("; plans without subtree reconfiguration" if cplans is not plans else ""),
                           "complex_macs_per_step": sum(p.stats()["cmacs"] for p in cplans)}
            del g2, ws2
            torch.cuda.empty_cache()
            log(f"{pr} pass")
        if "c128" in res_by:
            for pr, res in res_by.items():
                if pr == "c128":
                    continue
                errs = [max(rel_err(z, zr), rel_err(v, vr))
                        for (z, v), (zr, vr) in zip(res, res_by["c128"])]
                entry = compare.setdefault(pr, {})
                entry.update({"max_rel_err_vs_c128": max(errs),
                              "median_rel_err_vs_c128": statistics.median(errs),
                              "evaluations_over_1e-6": sum(e > 1e-6 for e in errs)})

    extra = {}
    if not args.skip_extra and world == 1:
        extra["batch"] = batch_workload(pk, ctx, stream, flush, args)
        log("batch workload")
        extra["grad"] = grad_workload(pk, ctx, stream, args)
        log("grad workload")

    cpu = None
    if rank == 0 and world == 1 and not args.skip_cpu:
        log("cpu baseline")
        cpu = cpu_oracle_baseline(knots, qs)

    launches = sum(p.launches(prec) for p in plans) * args.steps
    tot_cmacs = sum(s["cmacs"] for s in stats)
    if rank == 0:
        out = {"metric": METRIC,
               "value": value, "unit": "knots/s", "n_gpus": world, "steps": args.steps,
               "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
               "scaling": "weak", "vs_baseline": None, "dtype": prec, "data": "synthetic",
               "config": {"workload": "scale: 64 random grid-walk knots per GPU, L=40, 100-400 crossings, "
                                      "random over/under, q in {2,3,5}; 192 (knot, q) evaluations per step",
                          "order": f"auto per knot (lowest estimated cost after slicing, {args.restarts} min-fill "
                                   f"restarts, subtree reconfiguration with up to {args.refine} subtrees)",
                          "l2": "flushed between steps (512 MB write)",
                          "tuning": dict(ctx.tuning(), source="compiled-in table written by "
                                         "paper_1807_02119_gb300/autotune.py"),
                          "plan_seconds": plan_s, "complex_macs_per_step": tot_cmacs,
                          "complex_tflops": 8 * tot_cmacs / (step_ms / 1e3) / 1e12},
               "roofline": roof, "rooflines": rooflines, "cpu_baseline": cpu,
               "e2e": {"value": e2e_val, "unit": "knots/s", "h2d_bytes_per_step": h2d,
                       "d2h_bytes_per_step": d2h},
               "e2e_whole_program": {"value": job_rate(world, evals, 1000.0 * full_s),
                                     "unit": "knots/s", "h2d_bytes_per_step": h2d_full,
                                     "d2h_bytes_per_step": d2h},
               "gpu_launches": launches, "clocks": clk,
               "kernel_classes_in_step": {"replay_ms": instep_ms, "classes": instep,
                                          "how": "one replay of the step's graph with an event "
                                                 "pair around every launch; ms = sum over launches "
                                                 "of each launch's duration"},
               "kernel_classes_serialised": {"classes": prof,
                                             "how": "every plan's launches one after another, "
                                                    "an event pair around each; fill_ms weights "
                                                    "each launch by the share of the GPU's CTA "
                                                    "slots it fills"},
               "precisions": compare, "workloads": extra}
        print(json.dumps(out))
    if dist:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
