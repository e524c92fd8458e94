"""Autotuner for the executor's launch shapes (pk_tuning), run on the target GPU.

Two sweeps, each timed with CUDA events on the stream the kernels run on, L2 flushed
before every timed launch, the fastest median kept:

* batch executor (`pk_batch_*`, one persistent launch for many knots): threads per CTA
  x contracted-index offsets kept in shared memory, on the 4096-knot batch workload
  (q = 3, split precision);
* sequence runs (consecutive small steps of a plan launched as one one-CTA kernel): the
  largest step, in outputs and in complex multiply-adds, that joins a run, on the 64-knot
  scale workload (q = 2, 3, 5; 192 plans replayed as one concurrent graph, split);
* the smallest contracted extent and column count from which row steps of GEMM shape
  also run on the tensor cores (split), on the same workload;
* the number of flush groups from which a tensor-core step runs one CTA per SM with two
  accumulator sets instead of two CTAs per SM with one, on the same workload;
* the planner's cost weights (a tensor-core multiply-add, an output entry) with which the
  candidate contraction orders are ranked, on the same workload.

Every candidate's results are checked against the first candidate's (same plans, same
precision) before its time counts.  The winners are written to csrc/tuned_table.h (the
defaults the library is compiled with) together with every measured time, and a copy of
the table goes to the output directory given by --out.

Usage (on a GPU): python -m paper_1807_02119_gb300.autotune [--out DIR] [--quick]
[--only tc_min_k,tc_db_groups] (--only: sweep just those scale-workload parameters, the
others keep the compiled-in table's values)
"""
from __future__ import annotations

import argparse
import datetime
import os
import statistics
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
TABLE = os.path.join(HERE, "csrc", "tuned_table.h")
RESTARTS = 256   # min-fill restarts per plan of the scale workload, as bench.py builds them
REFINE = 8       # subtree reconfiguration of the scale workload's plans, as bench.py

BATCH_THREADS = (128, 256, 512)
BATCH_KTAB = (512, 1024, 2048)
SEQ_OUTS = (1024, 2048, 4096, 8192)
SEQ_WORK = (1 << 12, 1 << 14, 1 << 16)
TC_MIN_K = (4, 8, 16)
TC_DB_GROUPS = (0, 2, 3, 4, 6)
TC_MIN_N = (8, 12, 16, 24, 32)
COST_GEMM = (50, 100, 150, 250, 400)
COST_OUT = (1000, 2000, 4000, 8000, 16000, 32000, 64000, 128000, 256000)
TC_WIDE_N = (16, 25, 50, 100, 1 << 30)
COST_TCIN = (0, 500, 1000, 2000, 4000, 8000, 16000)
TC_MIN_WORK = (0, 1 << 16, 1 << 18, 1 << 20, 1 << 22)
SCALE_PARAMS = {"tc_min_k": TC_MIN_K, "tc_min_n": TC_MIN_N, "tc_wide_n": TC_WIDE_N,
                "tc_db_groups": TC_DB_GROUPS, "cost_gemm_milli": COST_GEMM,
                "cost_out_milli": COST_OUT, "cost_tcin_milli": COST_TCIN,
                "tc_min_work": TC_MIN_WORK}


def _rel(a, b):
    d = a.exp2 - b.exp2
    ma = a.mantissa * (2.0 ** d if d > -1000 else 0.0)
    return abs(ma - b.mantissa) / abs(b.mantissa) if b.mantissa != 0 else abs(ma)


def _time(launch, stream, flush, reps):
    import torch
    for _ in range(3):
        launch()
    torch.cuda.synchronize()
    ts = []
    for _ in range(reps):
        flush.zero_()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        launch()
        b.record(stream)
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return statistics.median(ts)


def sweep_batch(pk, ctx, stream, flush, reps, log):
    import torch
    from concurrent.futures import ThreadPoolExecutor
    import knotgen as kg
    knots = kg.knot_suite("batch")
    kn = [pk.Knot.from_pd(ctx, k.pd, outer=k.outer) for k in knots]
    with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
        plans = list(ex.map(lambda k: pk.Plan(ctx, k, 3), kn))
    rows, ref, best = [], None, None
    for th in BATCH_THREADS:
        for kt in BATCH_KTAB:
            ctx.set_tuning(batch_threads=th, batch_ktab=kt)
            b = pk.Batch(plans, "split")
            ws = torch.empty(b.workspace_bytes()[0], dtype=torch.uint8, device="cuda")
            b.upload(ws)
            ms = _time(lambda: b.launch(ws), stream, flush, reps)
            z, v = b.download(ws)
            if ref is None:
                ref = z
            err = max(_rel(x, y) for x, y in zip(z, ref))
            ok = err <= 1e-6
            rows.append((th, kt, ms, ok))
            log(f"batch threads={th} ktab={kt}: {ms:.3f} ms ({len(plans) / ms * 1e3:.0f} knots/s)"
                f"{'' if ok else ' RESULTS DIFFER'}")
            if ok and (best is None or ms < best[2]):
                best = (th, kt, ms)
            del b, ws
            torch.cuda.empty_cache()
    return best, rows


def sweep_seq(pk, ctx, stream, flush, reps, log, quick):
    import torch
    from concurrent.futures import ThreadPoolExecutor
    import knotgen as kg
    knots = kg.knot_suite("scale")
    kn = [pk.Knot.from_pd(ctx, k.pd, outer=k.outer) for k in knots]
    jobs = [(k, q) for k in kn for q in (2, 3, 5)]
    rows, ref, best = [], None, None
    outs = SEQ_OUTS if not quick else (2048, 4096)
    works = SEQ_WORK if not quick else (1 << 12, 1 << 14)
    for so in outs:
        for sw in works:
            ctx.set_tuning(seq_outs=so, seq_work=sw)
            with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
                plans = list(ex.map(lambda j: pk.Plan(ctx, j[0], j[1], restarts=RESTARTS,
                                                          refine=REFINE), jobs))
            ws = [torch.empty(p.workspace_bytes("split") + 256, dtype=torch.uint8, device="cuda")
                  for p in plans]
            for p, w in zip(plans, ws):
                pk.upload(p, "split", w)
            g = pk.Group(plans, "split", ws)
            ms = _time(g.launch, stream, flush, reps)
            z = [pk.download(p, "split", w)[0] for p, w in zip(plans, ws)]
            if ref is None:
                ref = z
            err = max(_rel(x, y) for x, y in zip(z, ref))
            ok = err <= 1e-6
            launches = sum(p.launches("split") for p in plans)
            rows.append((so, sw, ms, ok, launches))
            log(f"sequence runs outs<={so} work<={sw}: {ms:.2f} ms per step, {launches} launches"
                f"{'' if ok else ' RESULTS DIFFER'}")
            if ok and (best is None or ms < best[2]):
                best = (so, sw, ms)
            del g, ws, plans
            torch.cuda.empty_cache()
    return best, rows


def sweep_scale_param(pk, ctx, stream, flush, reps, log, name):
    """One pk_tuning field over its candidates (SCALE_PARAMS) on the scale workload (split,
    192 plans replayed as one concurrent graph), the other fields as the context has them."""
    import torch
    from concurrent.futures import ThreadPoolExecutor
    import knotgen as kg
    knots = kg.knot_suite("scale")
    kn = [pk.Knot.from_pd(ctx, k.pd, outer=k.outer) for k in knots]
    jobs = [(k, q) for k in kn for q in (2, 3, 5)]
    rows, ref, best = [], None, None
    for tk in SCALE_PARAMS[name]:
        ctx.set_tuning(**{**ctx.tuning(), name: tk})
        with ThreadPoolExecutor(max_workers=os.cpu_count() or 1) as ex:
            plans = list(ex.map(lambda j: pk.Plan(ctx, j[0], j[1], restarts=RESTARTS,
                                                          refine=REFINE), jobs))
        ws = [torch.empty(p.workspace_bytes("split") + 256, dtype=torch.uint8, device="cuda")
              for p in plans]
        for p, w in zip(plans, ws):
            pk.upload(p, "split", w)
        g = pk.Group(plans, "split", ws)
        ms = _time(g.launch, stream, flush, reps)
        z = [pk.download(p, "split", w)[0] for p, w in zip(plans, ws)]
        if ref is None:
            ref = z
        ok = max(_rel(x, y) for x, y in zip(z, ref)) <= 1e-6
        rows.append((tk, ms, ok))
        log(f"{name} = {tk}: {ms:.2f} ms per step{'' if ok else ' RESULTS DIFFER'}")
        if ok and (best is None or ms < best[1]):
            best = (tk, ms)
        del g, ws, plans
        torch.cuda.empty_cache()
    return best, rows


PARAM_TITLES = {
    "tc_min_k": "Tensor cores for row steps of GEMM shape from this K",
    "tc_db_groups": "One CTA per SM, two accumulator sets, from this many flush groups (0: never)",
    "tc_min_n": "Tensor cores for row steps of GEMM shape from this many columns",
    "cost_gemm_milli": "Planner: cost of a tensor-core multiply-add (thousandths of a row one)",
    "cost_out_milli": "Planner: cost of an output entry (thousandths of a multiply-add)",
    "tc_wide_n": "Tensor cores for short-K (4 <= K < tc_min_k) row steps from this many columns",
    "cost_tcin_milli": "Planner: cost of a tensor-core step's operand entry (thousandths of a multiply-add)",
    "tc_min_work": "Tensor cores for row steps of GEMM shape from this many multiply-adds",
}


def write_table(path, tune, batch_rows, seq_rows, gpu, param_rows):
    when = datetime.datetime.now(datetime.timezone.utc).strftime("%Y-%m-%d %H:%M UTC")
    lines = ["// Executor launch shapes, written by paper_1807_02119_gb300/autotune.py from",
             f"// measurements on {gpu} ({when}); the library's defaults (pk_tuning_default).",
             "// Batch executor, 4096 knots at q = 3, split, one launch (median ms):"]
    for th, kt, ms, ok in batch_rows:
        lines.append(f"//   threads {th:4d}  ktab {kt:5d}  {ms:8.3f}{'' if ok else '  (results differ)'}")
    lines.append("// Sequence runs, 192 evaluations of the scale workload, split (median ms per step):")
    for so, sw, ms, ok, nl in seq_rows:
        lines.append(f"//   outs <= {so:5d}  work <= {sw:6d}  {ms:8.2f}  ({nl} launches)"
                     f"{'' if ok else '  (results differ)'}")
    for name, prow in param_rows.items():
        lines.append(f"// {PARAM_TITLES[name]}, split (median ms per step):")
        for tk, ms, ok in prow:
            lines.append(f"//   {name} = {tk:4d}  {ms:8.2f}{'' if ok else '  (results differ)'}")
    lines += ["#pragma once", '#include "pk.h"', "",
              "constexpr pk_tuning kTunedDefault = {" +
              f"{tune['batch_threads']}, {tune['batch_ktab']}, {tune['seq_outs']}, "
              f"{tune['seq_work']}, {tune['seq_k']}, {tune['tc_min_k']}, {tune['tc_db_groups']}, "
              f"{tune['tc_min_n']}, {tune['cost_gemm_milli']}, {tune['cost_out_milli']}, "
              f"{tune['tc_wide_n']}, {tune['cost_tcin_milli']}, {tune['tc_min_work']}" +
              "};", ""]
    with open(path, "w") as f:
        f.write("\n".join(lines))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=None, help="also copy the table here")
    ap.add_argument("--reps", type=int, default=7)
    ap.add_argument("--quick", action="store_true", help="a smaller sequence-run sweep")
    ap.add_argument("--only", default=None,
                    help="comma-separated scale-workload parameters to sweep alone")
    args = ap.parse_args()
    sys.path.insert(0, ROOT)
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_1807_02119_gb300 as pk

    def log(m):
        print(f"[autotune] {m}", flush=True)

    ctx = pk.Context(0)
    stream = torch.cuda.current_stream()
    ctx.set_stream(stream.cuda_stream)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda")
    tune = pk.default_tuning()
    gpu = torch.cuda.get_device_name(0)
    prows = {}
    if args.only:   # some scale parameters alone: the table is only written to --out
        ctx.set_tuning()
        for name in args.only.split(","):
            (best, _), prows[name] = sweep_scale_param(pk, ctx, stream, flush, args.reps, log, name)
            tune[name] = best
            ctx.set_tuning(**tune)
        if args.out:
            os.makedirs(args.out, exist_ok=True)
            write_table(os.path.join(args.out, "tuned_table.h"), tune, [], [], gpu, prows)
        log(f"chosen: {tune}")
        return
    (bt, bk, _), brows = sweep_batch(pk, ctx, stream, flush, args.reps, log)
    ctx.set_tuning()
    (so, sw, _), srows = sweep_seq(pk, ctx, stream, flush, args.reps, log, args.quick)
    tune.update(batch_threads=bt, batch_ktab=bk, seq_outs=so, seq_work=sw)
    ctx.set_tuning(**tune)
    for name in SCALE_PARAMS:
        (best, _), prows[name] = sweep_scale_param(pk, ctx, stream, flush, args.reps, log, name)
        tune[name] = best
        ctx.set_tuning(**tune)
    write_table(TABLE, tune, brows, srows, gpu, prows)
    if args.out:
        os.makedirs(args.out, exist_ok=True)
        write_table(os.path.join(args.out, "tuned_table.h"), tune, brows, srows, gpu, prows)
    log(f"chosen: {tune}")


if __name__ == "__main__":
    main()
