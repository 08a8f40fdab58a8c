"""Benchmark of the FastSTMF hot path on GB300: sweeps/s and max-plus Gop/s.

Workload (default): the gene-expression-scale job, R 1000 x 5000 FP32 with a
planted rank-10 tropical structure (0.5*log2(1+LogNormal(3,2)) factors),
N(0, 0.05) noise, 80% of entries given, rank 10 (synthetic stand-in for the
paper's TCGA matrices, which are not available).

A step is one sweep of Algorithm 3 (every row of the oriented R visited once:
candidate windows of F-ULF / F-URF updates, select, commit, refresh of the
product planes and statistics).  The run is one factorization: W untimed
warm-up sweeps from the Random Acol start, then K timed sweeps of the same
run, each bracketed by a barrier, a device synchronisation and CUDA events on
the library's stream; the L2 cache is flushed (a 256 MiB write) before each
timed sweep, outside its timed span.  The e2e figure is the same K sweeps
through the public API from pinned host buffers, with the job's upload of R
and the mask, its initialisation and the download of U, V inside the timed
region (the warm-up sweeps are timed apart and left out).

value = sweeps/s summed over ranks (independent replicas, weak scaling).
gops  = algorithmic max-plus operations of the sequential method per second:
        2 r N_obs per product refresh + 6 N_obs per candidate tried (up to the
        kept one); speculative window work is not counted.
Peaks are measured at run time by the library's microbenchmark
(stmf_peak_addmax): the 1:1 FP32 add+max mix, and the instruction mixes of
the two window-evaluation passes.

``--impl reference`` times the oracle (plain C, FP64 arithmetic rounded to
FP32, on all host cores) on the same workload: a step is one row of the sweep
that follows the W warm-up sweeps (the start state is the library's state
after W sweeps, mapped into the oracle's frame; without a GPU it is the
oracle's own initial state); one untimed row, then K timed rows;
value = rows/s / m sweeps/s.  The CPU baseline of the main arm times the
same rows (the first 20) from the same state.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import tempfile
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "FastSTMF sweeps/s & max-plus Gop/s (% FP32 peak); time-to-error vs plain"
# k_delta DRAM bytes per launch (read + write), ncu capture of the gene
# workload, valid for the kernel source it was taken on
# DRAM bytes per phase-2 launch from the ncu captures in profiles/ (gene
# workload, 64 candidates, cold), valid for the captured source only
EVAL_TRAFFIC = {"workload": "gene",
                "k_delta8": {"source_sha256_prefix": "4baf8c918da4073a", "bytes": 47.74e6}}
CPU_ROWS = 20   # rows of the CPU baseline (the reference arm's first rows)


def eval_traffic(workload_name, kernel):
    import hashlib
    rec = EVAL_TRAFFIC.get(kernel)
    src = os.path.join(ROOT, "paper_2205_06619_gb300", "csrc", "kernels_eval.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    if rec is None or sha != rec["source_sha256_prefix"] or workload_name != EVAL_TRAFFIC["workload"]:
        return None
    return rec["bytes"]


def measured_peaks(api):
    """Peaks in Top/s from the library's microbenchmark, best of 3 each:
    the 1:1 FADD/FMNMX stream, and the mixes of k_delta and k_res in their
    algorithmic operations per entry and candidate."""
    out = {}
    for name, mode in (("addmax_1to1", 0), ("k_delta_mix", 6), ("k_res_mix", 7)):
        out[name] = max(api.peak_addmax(mode, 20000) for _ in range(3)) / 1e3
    return out


def workload(name, seed):
    from paper_2205_06619_gb300 import synth
    if name == "gene":
        w = synth.workload_gene(seed)
        w["label"] = "gene-expression 1000x5000 rank-10, 80% given"
    elif name == "small":
        w = synth.workload_small(seed)
        w["label"] = "small 200x100 rank-3, 80% given"
    elif name == "large":
        w = synth.workload_large(seed)
        w["label"] = "large 4000x20000 rank-20, 50% given"
    else:
        raise SystemExit("unknown workload " + name)
    return w


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        # raw samples: $STMF_CLOCKS_DIR if set, else the system temporary directory
        d = os.environ.get("STMF_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, "clocks_bench_%d.csv" % os.getpid())

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1])); mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_rows(R, M, rank, seed, U_start, V_start, budget_s, min_rows=1, max_rows=None, warm_rows=0, threads=0):
    """Times the oracle's ByRow steps on the first rows of a sweep from a given
    state (caller orientation) on `threads` host threads (0: all cores);
    returns (rows, seconds, per-row times, threads used)."""
    import oracle as orc
    used = orc.set_threads(threads)
    st = orc.prepare(R, M, rank, seed=seed)
    assert not st["transposed"]
    Ri, Mi = st["R"], st["M"]
    perm = st["perm"]
    if U_start is not None:
        Ui = np.ascontiguousarray(U_start[perm], dtype=np.float64)
        Vi = np.ascontiguousarray(V_start, dtype=np.float64)
    else:
        Ui, Vi = st["U"], st["V"]
    f = orc.error(Ri, Mi, Ui, Vi)
    times = []
    i = 0
    for _ in range(warm_rows):
        _, f, _, _ = orc.row_step(Ri, Mi, Ui, Vi, i, f)
        i += 1
    t_all = time.perf_counter()
    while True:
        t = time.perf_counter()
        _, f, _, _ = orc.row_step(Ri, Mi, Ui, Vi, i, f)
        times.append(time.perf_counter() - t)
        i += 1
        if max_rows is not None and len(times) >= max_rows:
            break
        if len(times) >= min_rows and time.perf_counter() - t_all >= budget_s:
            break
        if i >= Ri.shape[0]:
            break
    return len(times), sum(times), times, used


def run_reference(args):
    """The oracle on the host cores, on the same workload (see module doc)."""
    rank_id = int(os.environ.get("RANK", "0"))
    if rank_id != 0:
        return
    w = workload(args.workload, args.seed)
    R, M, r = w["R"], w["mask"], w["rank"]
    U_start = V_start = None
    start = "the oracle's own initial state (sweep 0)"
    try:
        import torch
        if torch.cuda.is_available() and args.warmup > 0:
            from paper_2205_06619_gb300 import api
            fz = api.Factorization(torch.from_numpy(R).cuda(), api.pack_mask(M), rank=r, seed=args.seed)
            fz.run(args.warmup)
            U, V = fz.result()
            U_start, V_start = U.cpu().numpy().astype(np.float64), V.cpu().numpy().astype(np.float64)
            start = ("the state after %d sweeps (the warm-up sweeps of the library's arm, prepared on the GPU "
                     "and mapped into the oracle's frame)" % args.warmup)
            fz.close()
    except Exception as e:  # pragma: no cover - reported in the sample text
        start += " (GPU preparation failed: %s)" % e
    rows, secs, _, used = oracle_rows(R, M, r, args.seed, U_start, V_start, budget_s=0.0,
                                      min_rows=args.steps, max_rows=args.steps, warm_rows=min(args.warmup, 1))
    m = min(R.shape)
    value = rows / secs / m
    sample = ("%d timed rows (after %d untimed row) of the ByRow sweep of the %s job, from %s, on %d host "
              "threads (nproc %d); sweeps/s = rows/s / %d rows" % (rows, min(args.warmup, 1), w["label"], start,
                                                                  used, os.cpu_count() or 0, m))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / rows,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64->f32",
            "data": "synthetic", "config": {"workload": w["label"], "step": "one row of the sweep"},
            "cpu_baseline": {"value": value, "unit": "sweeps/s", "cores": used, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "sweeps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def progress(msg):
    """A progress line on stderr (a long run that is cut off still leaves its finished legs)."""
    print("[bench] " + msg, file=sys.stderr, flush=True)


def run_batch(args):
    """Many independent problems (the batched workload: 64 problems, rows
    U{100..2000}, columns U{200..8000}, ranks U{3..20}, given densities
    U[0.2, 0.9], generated as the small workload, 10 sweeps each).  The
    autotuner runs first, on jobs of 0 sweeps (its trials are cached per size
    class in the context).  Then, on a seeded subset of the problems at their
    stated sizes, one batched launch against one problem at a time through
    stmf_factorize; with --batch-whole also the whole batch in one launch
    (over an hour on one GB300 at full scale: the late sweeps of these sizes
    cost seconds each).  Decisions are identical, so the final errors are
    equal and the times are times to equal error."""
    import torch
    from paper_2205_06619_gb300 import api, synth
    rng = np.random.default_rng(args.seed)
    sc = args.batch_scale
    probs = []
    for q in range(args.batch_count):
        m = max(4, int(rng.integers(100, 2001) * sc)); n = max(4, int(rng.integers(200, 8001) * sc))
        r = int(rng.integers(3, 21)); d = float(rng.uniform(0.2, 0.9))
        sub = int(rng.integers(0, 2**31 - 1))
        R, M, _, _ = synth.uniform_planted(m, n, r, 0.01, d, sub)
        probs.append(dict(R=torch.from_numpy(R).cuda(), mask_words=api.pack_mask(M), rank=r, sweeps=10, seed=q,
                          m=m, n=n))
    torch.cuda.synchronize()
    subset = sorted(int(x) for x in np.random.default_rng(args.seed + 1).choice(
        len(probs), size=min(args.batch_subset, len(probs)), replace=False))
    sub = [probs[q] for q in subset]
    with ClockSampler(0) as clocks:
        t = time.perf_counter()
        _, tuned = api.factorize_batched([dict(p, sweeps=0) for p in probs], window=0)
        t_tune = time.perf_counter() - t
        progress("batch: autotuner %.1f s" % t_tune)
        whole = None
        if args.batch_whole:
            torch.cuda.synchronize()
            t = time.perf_counter()
            outs, _ = api.factorize_batched(probs, window=0)
            torch.cuda.synchronize()
            whole = {"seconds": time.perf_counter() - t, "sweeps": sum(p["sweeps"] for p in probs),
                     "equals_subset": None}
            progress("batch: whole batch in one launch %.1f s" % whole["seconds"])
        torch.cuda.synchronize()
        t = time.perf_counter()
        outs_sub, _ = api.factorize_batched(sub, window=0)
        torch.cuda.synchronize()
        t_batched_sub = time.perf_counter() - t
        progress("batch: subset %s batched %.1f s" % (subset, t_batched_sub))
        t = time.perf_counter()
        plain = [api.factorize(p["R"], p["mask_words"], rank=p["rank"], sweeps=p["sweeps"], seed=p["seed"])
                 for p in sub]
        torch.cuda.synchronize()
        t_plain_sub = time.perf_counter() - t
        progress("batch: subset one at a time %.1f s" % t_plain_sub)
    same = all(torch.equal(a[0], b[0]) and torch.equal(a[1], b[1]) for a, b in zip(outs_sub, plain))
    if whole is not None:
        whole["equals_subset"] = all(torch.equal(outs[q][0], outs_sub[i][0]) and
                                     torch.equal(outs[q][1], outs_sub[i][1]) for i, q in enumerate(subset))
    sweeps_sub = sum(p["sweeps"] for p in sub)
    entries = sum(p["m"] * p["n"] for p in probs)
    value, t_step = (whole["sweeps"] / whole["seconds"], whole["seconds"]) if whole else \
        (sweeps_sub / t_batched_sub, t_batched_sub)
    line = {"metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": 1, "steps": 1,
            "warmup": 0, "ms_per_step": 1e3 * t_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "batch of %d problems, rows U{100..2000}*%.2f, cols U{200..8000}*%.2f, "
                                   "rank U{3..20}, given U[0.2,0.9], 10 sweeps each (%.1f M entries in all)"
                                   % (args.batch_count, sc, sc, entries / 1e6),
                       "step": "the whole batch in one launch" if whole else
                               "problems %s of the batch in one launch" % subset},
            "subset": {"problems": subset, "shapes": [(p["m"], p["n"], p["rank"]) for p in sub],
                       "batched_seconds": t_batched_sub, "one_at_a_time_seconds": t_plain_sub,
                       "speedup_vs_one_at_a_time": t_plain_sub / t_batched_sub, "identical_results": same,
                       "launch_shapes": [(o[2]["eval_res_chunk"], o[2]["eval_delta_blocks"]) for o in outs_sub]},
            "whole_batch": whole, "autotuner_seconds": t_tune,
            "tuned_windows": sorted(set(tuned)), "clocks": clocks.summary()}
    print(json.dumps(line), flush=True)


def run_precision(args):
    """Candidate screening in packed FP16 with FP32 re-check (precision 1) vs
    the all-FP32 path (precision 0) on the 4000 x 20000 rank-20 workload, 50%
    given.  Both runs start from the same Random Acol state and make the same
    decisions; the final b-norm error of each is recomputed in FP64 by the
    oracle from the returned factors (the CPU leg)."""
    import torch
    from paper_2205_06619_gb300 import api, synth
    w = synth.workload_large(seed=args.seed)
    R_np, M_np, r = w["R"], w["mask"], w["rank"]
    Rg, Mw = torch.from_numpy(R_np).cuda(), api.pack_mask(M_np)
    stream = api.context().stream
    out = {}
    with ClockSampler(0) as clocks:
        for prec in (0, 1):
            fz = api.Factorization(Rg, Mw, rank=r, seed=args.seed, precision=prec)
            rep0 = fz.run(0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            rep1 = fz.run(args.steps)
            b.record(stream)
            torch.cuda.synchronize()
            U, V = fz.result()
            out[prec] = dict(seconds=a.elapsed_time(b) / 1e3, rep=rep1, rep0=rep0, U=U.cpu().numpy(),
                             V=V.cpu().numpy())
            fz.close()
    same = bool(np.array_equal(out[0]["U"], out[1]["U"]) and np.array_equal(out[0]["V"], out[1]["V"]))
    res = {}
    for prec in (0, 1):
        o = out[prec]
        d = {k: o["rep"][k] - o["rep0"][k] for k in ("eval_ns", "eval_launches", "candidates_issued",
                                                     "candidates_screened", "windows")}
        res["fp32" if prec == 0 else "fp16_screen"] = {
            "sweeps_per_s": args.steps / o["seconds"], "seconds": o["seconds"], "f_final": o["rep"]["f_final"],
            "eval_us_per_window": d["eval_ns"] / 1e3 / max(d["eval_launches"], 1),
            "candidates_issued": d["candidates_issued"], "candidates_screened": d["candidates_screened"],
            "screened_fraction": d["candidates_screened"] / max(d["candidates_issued"], 1)}
    cpu = None
    if not args.no_cpu_baseline:
        import oracle  # CPU leg: FP64 error of the returned factors
        t = time.perf_counter()
        for prec, key in ((0, "fp32"), (1, "fp16_screen")):
            f64 = oracle.error(R_np, M_np, out[prec]["U"].astype(np.float64), out[prec]["V"].astype(np.float64))
            res[key]["f_oracle_fp64"] = f64
            res[key]["rel_err_vs_oracle"] = abs(res[key]["f_final"] - f64) / f64
        secs = time.perf_counter() - t
        cpu = {"value": 2.0 / secs, "unit": "error evaluations/s", "cores": 1, "kind": "oracle",
               "sample": "FP64 b-norm error of both returned factorizations (4000x20000, rank 20), %.1f s" % secs}
    scr = res["fp16_screen"]
    line = {"metric": METRIC, "value": scr["sweeps_per_s"], "unit": "sweeps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": 0, "ms_per_step": 1e3 * out[1]["seconds"] / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f16 screen + f32 re-check", "data": "synthetic",
            "config": {"workload": "precision: 4000x20000 rank-20, 50% given, U*,V* ~ U[0,1) + N(0,0.01)",
                       "step": "one ByRow sweep from the Random Acol start", "l2": "inputs (1.3 GB) exceed L2"},
            "identical_decisions": same, "speedup_vs_fp32": res["fp32"]["seconds"] / scr["seconds"],
            "precision": res, "clocks": clocks.summary(), "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)


def run_selection(args):
    """The four selections of (j, k) within a row (Section "The ByRow
    strategy": TD_A as published, TD_B, TD, SEQ) and the ByElement strategy
    (STMF_ByElement_PermC_TD_W) on the gene-expression workload: sweeps/s over
    sweeps W..W+K-1 of one run each (CUDA events on the library's stream),
    with the error reached and the candidates tried; the ByMatrix strategy
    (STMF_ByMatrix_NoPerm_TD_W, one update per iteration): iterations/s over
    iterations W..W+100K-1.
    CPU leg: the oracle computing the same row's (j, k) order for each
    selection from the library's final state."""
    import torch
    from paper_2205_06619_gb300 import api, synth
    w = synth.workload_gene(seed=args.seed)
    R_np, M_np, r = w["R"], w["mask"], w["rank"]
    Rg, Mw = torch.from_numpy(R_np).cuda(), api.pack_mask(M_np)
    stream = api.context().stream
    res, last = {}, None
    runs = [("TD_A", dict(selection="TD_A")), ("TD_B", dict(selection="TD_B")), ("TD", dict(selection="TD")),
            ("SEQ", dict(selection="SEQ")), ("ByElement", dict(strategy="ByElement"))]
    with ClockSampler(0) as clocks:
        for sel, kw in runs:
            fz = api.Factorization(Rg, Mw, rank=r, seed=args.seed, **kw)
            fz.run(args.warmup)
            rep0 = fz.run(0)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            a.record(stream)
            rep1 = fz.run(args.steps)
            b.record(stream)
            torch.cuda.synchronize()
            secs = a.elapsed_time(b) / 1e3
            d = {k: rep1[k] - rep0[k] for k in ("candidates_tried", "candidates_issued", "accepted", "windows",
                                                "refreshes")}
            res[sel] = {"sweeps_per_s": args.steps / secs, "f_start": rep0["f_final"], "f_end": rep1["f_final"],
                        "f_init": rep1["f_init"],
                        "per_sweep": {k: v / args.steps for k, v in d.items()}}
            if sel == "TD_A":
                last = fz.result()
            fz.close()
        # ByMatrix: one update per iteration; 100 K iterations timed after W
        fz = api.Factorization(Rg, Mw, rank=r, seed=args.seed, strategy="ByMatrix")
        fz.run(args.warmup)
        rep0 = fz.run(0)
        nit = 100 * args.steps
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(stream)
        rep1 = fz.run(nit)
        b.record(stream)
        torch.cuda.synchronize()
        secs = a.elapsed_time(b) / 1e3
        d = {k: rep1[k] - rep0[k] for k in ("candidates_tried", "accepted", "windows")}
        res["ByMatrix"] = {"iterations_per_s": nit / secs, "iterations": nit, "f_start": rep0["f_final"],
                           "f_end": rep1["f_final"], "f_init": rep1["f_init"],
                           "per_iteration": {k: v / nit for k, v in d.items()}}
        fz.close()
    cpu = None
    if not args.no_cpu_baseline:
        import oracle   # CPU leg: the oracle's row orders from the library's TD_A state
        U, V = (x.cpu().numpy().astype(np.float64) for x in last)
        st = oracle.prepare(R_np, M_np, r, seed=args.seed)
        # the factors come back in the caller's frame; the oracle's frame is oriented and permuted
        Ui = U[st["perm"]]
        t = time.perf_counter()
        for sel in ("TD_A", "TD_B", "TD", "SEQ"):
            oracle.row_order(st["R"], st["M"], Ui, V, 0, selection=sel)
        secs = time.perf_counter() - t
        cpu = {"value": 4.0 / secs, "unit": "row orders/s", "cores": 1, "kind": "oracle",
               "sample": "the (j, k) order of row 0 for each of the 4 selections at 1000x5000, %.1f s" % secs}
    a_ = res["TD_A"]
    line = {"metric": METRIC, "value": a_["sweeps_per_s"], "unit": "sweeps/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 / a_["sweeps_per_s"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "selection: gene-expression 1000x5000 rank-10, 80% given, each selection of "
                                   "(j, k) of ByRow from the same Random Acol start, and ByElement (its PermC "
                                   "column order changes the Acol start)",
                       "step": "one ByRow sweep (sweeps W..W+K-1 of each run)", "l2": "not flushed"},
            "selections": res, "clocks": clocks.summary(), "cpu_baseline": cpu}
    print(json.dumps(line), flush=True)


def run_learned(args):
    """Learned initialisation vs Random Acol: sweeps and time to reach the
    plain method's final error on fresh matrices (same permutation for both)."""
    import torch
    from paper_2205_06619_gb300 import api, learned_init
    m, n = args.learned_m, args.learned_n
    T_sweeps = args.learned_sweeps
    t = time.perf_counter()
    X, T = learned_init.training_set(args.learned_train, m, n, 10, args.learned_train_sweeps or T_sweeps,
                                     seed=args.seed, target=args.learned_target)
    t_data = time.perf_counter() - t
    t = time.perf_counter()
    net, hist = learned_init.train(X, T, 10, epochs=args.learned_epochs, batch=256, lr=1e-3, seed=args.seed)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t
    rng = np.random.default_rng(args.seed + 12345)
    rows = []
    for q in range(args.learned_eval):
        R, M = learned_init.gene_like(m, n, int(rng.integers(0, 2**31 - 1)))
        Rg, Mw = torch.from_numpy(R).cuda(), api.pack_mask(M)
        perm = rng.permutation(min(m, n)).astype(np.int32)
        seed = int(rng.integers(0, 2**31 - 1))
        torch.cuda.synchronize()
        t = time.perf_counter()
        fz = api.Factorization(Rg, Mw, rank=10, seed=seed, perm=perm)
        rep = fz.run(T_sweeps)
        torch.cuda.synchronize()
        t_plain = time.perf_counter() - t
        f_target, f0_plain = rep["f_final"], rep["f_init"]
        fz.close()
        t = time.perf_counter()
        U_ref = None
        if args.learned_target == "sorted":   # Random Acol's start gives the components' order per row
            U_ref = api.factorize(Rg, Mw, rank=10, sweeps=0, seed=seed, perm=perm)[0]
        U0 = learned_init.predict_U(net, Rg, Mw, U_ref=U_ref)
        U0 = U0[torch.from_numpy(perm.astype(np.int64)).cuda()].contiguous()
        fz = api.Factorization(Rg, Mw, rank=10, seed=seed, perm=perm, U0=U0)
        f0_learn = fz.run(0)["f_init"]
        sw = 0
        while sw < 2 * T_sweeps:
            rep = fz.run(1)
            sw += 1
            if rep["f_final"] <= f_target:
                break
        torch.cuda.synchronize()
        t_learn = time.perf_counter() - t
        fz.close()
        rows.append(dict(f_target=f_target, f0_plain=f0_plain, f0_learned=f0_learn, sweeps_learned=sw,
                         reached=rep["f_final"] <= f_target, t_plain=t_plain, t_learned=t_learn,
                         f_learned_end=rep["f_final"]))
    ok = [r for r in rows if r["reached"]]
    # time-to-equal-error speedup per matrix; a learned run that does not reach
    # the plain error within 2T sweeps has no time to equal error: speedup 0
    speed = [r["t_plain"] / r["t_learned"] if r["reached"] else 0.0 for r in rows]
    line = {"metric": METRIC, "value": float(np.median(speed)),
            "unit": "time-to-equal-error speedup vs Random Acol (median over matrices; 0 where the learned "
                    "start does not reach the plain error within twice its sweeps)", "n_gpus": 1, "steps": len(rows),
            "warmup": 0, "higher_is_better": True, "dtype": "f32 (MLP: bf16 weights, f32 accumulation)",
            "data": "synthetic", "vs_baseline": None, "scaling": "weak",
            "config": {"workload": "learned init (%s targets): train on %d method factorizations of %dx%d "
                                   "rank-10 gene-like matrices (%d sweeps), evaluate on %d fresh ones against the "
                                   "plain method's error after %d sweeps" %
                                   (args.learned_target, args.learned_train, m, n,
                                    args.learned_train_sweeps or T_sweeps, args.learned_eval, T_sweeps)},
            "train": {"samples": int(X.shape[0]), "epochs": args.learned_epochs, "loss_first": hist[0],
                      "loss_last": hist[-1], "data_seconds": t_data, "train_seconds": t_train},
            "reached_fraction": len(ok) / len(rows),
            "speedup_mean": float(np.mean(speed)), "speedups": speed,
            "sweeps_to_equal_error_learned_mean": float(np.mean([r["sweeps_learned"] for r in rows])),
            "sweeps_plain": T_sweeps,
            "init_error_ratio_mean": float(np.mean([r["f0_learned"] / r["f0_plain"] for r in rows])),
            "per_matrix": rows}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20, help="timed sweeps")
    ap.add_argument("--warmup", type=int, default=5, help="untimed warm-up sweeps")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="gene",
                    choices=["gene", "small", "large", "batch", "learned", "precision", "selection"])
    ap.add_argument("--learned-train", type=int, default=200)
    ap.add_argument("--learned-eval", type=int, default=16)
    ap.add_argument("--learned-m", type=int, default=200)
    ap.add_argument("--learned-n", type=int, default=1000)
    ap.add_argument("--learned-sweeps", type=int, default=10)
    ap.add_argument("--learned-epochs", type=int, default=30)
    ap.add_argument("--learned-target", default="sorted", choices=["sorted", "canonical"])
    ap.add_argument("--learned-train-sweeps", type=int, default=0, help="sweeps of the training runs (0: as eval)")
    ap.add_argument("--batch-count", type=int, default=64)
    ap.add_argument("--batch-scale", type=float, default=1.0, help="size scale of the batch workload")
    ap.add_argument("--batch-subset", type=int, default=8, help="problems of the one-at-a-time comparison")
    ap.add_argument("--batch-whole", action="store_true", help="also time the whole batch in one launch")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--shapes", default="", help="launch shapes of the window evaluation: "
                                               "res_chunk,delta_blocks_per_sm[,delta_tile_rows] (0: default)")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        raise SystemExit("at least 3 warm-up sweeps are required")

    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batch":
        run_batch(args)
        return
    if args.workload == "learned":
        run_learned(args)
        return
    if args.workload == "selection":
        run_selection(args)
        return
    if args.workload == "precision":
        run_precision(args)
        return

    import torch
    from paper_2205_06619_gb300 import api

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank_id = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    # independent replicas: rank q factorizes its own seeded matrix
    w = workload(args.workload, args.seed + rank_id)
    R_np, M_np, r = w["R"], w["mask"], w["rank"]
    n_obs = int(M_np.sum())
    m_or = min(R_np.shape)
    R_host = torch.from_numpy(R_np).pin_memory()
    mask_words_host = api.pack_mask(M_np).cpu().pin_memory()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    ctx = api.context()
    stream = ctx.stream
    peaks = measured_peaks(api)

    # ---- the job through the public API; the timed sweeps inside it
    barrier()
    t_job = time.perf_counter()
    R_dev = R_host.to("cuda", non_blocking=True)
    mask_dev = mask_words_host.to("cuda", non_blocking=True)
    shapes = tuple(int(x) for x in args.shapes.split(",")) if args.shapes else None
    fz = api.Factorization(R_dev, mask_dev, rank=r, seed=args.seed + rank_id, shapes=shapes)
    torch.cuda.synchronize()
    t_apart = time.perf_counter()          # warm-up sweeps and the oracle's start state: not e2e
    for _ in range(args.warmup):
        fz.run(1)
    rep0 = fz.run(0)
    Uw, Vw = fz.result()
    U_w, V_w = Uw.cpu().numpy().astype(np.float64), Vw.cpu().numpy().astype(np.float64)
    torch.cuda.synchronize()
    t_apart = time.perf_counter() - t_apart
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    with ClockSampler(local) as clocks:
        for k in range(args.steps):
            flush.zero_()
            barrier()
            ev[k][0].record(stream)
            fz.run(1)
            ev[k][1].record(stream)
            barrier()
        torch.cuda.synchronize()
    times = [a.elapsed_time(b) / 1e3 for a, b in ev]
    rep1 = fz.report
    U, V = fz.result()
    U_h, V_h = U.cpu(), V.cpu()
    torch.cuda.synchronize()
    t_job = time.perf_counter() - t_job
    t_e2e = t_job - t_apart
    # training and prediction error of the returned factors: RMSE-A over the
    # given entries, RMSE-P over the 20% held out (Section "Evaluation metrics")
    rmse_a, rmse_p, n_a, n_p = api.rmse(R_dev, U, V, mask_dev)

    t_timed = sum(times)
    if dist is not None:
        tt = torch.tensor([t_timed, t_e2e], device="cuda", dtype=torch.float64)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        t_timed, t_e2e = float(tt[0]), float(tt[1])
    sweeps_all = args.steps * world
    value = sweeps_all / t_timed
    d = {k: rep1[k] - rep0[k] for k in ("candidates_tried", "candidates_issued", "accepted", "refreshes",
                                        "windows", "eval_ns", "eval_launches", "eval_candidates", "eval_res_ns",
                                        "eval_delta_ns", "candidates_discarded")}
    ops = 6.0 * n_obs * d["candidates_tried"] + 2.0 * r * n_obs * d["refreshes"]
    gops = ops / (t_timed / world) / 1e9 * world
    # algorithmic ops per given entry and candidate: phase 1 (residuation)
    # one sub + one min; phase 2 (error change) add, max, sub, accumulate
    ec = d["eval_candidates"]
    ach_res = (2.0 * n_obs * ec) / (d["eval_res_ns"] * 1e-9) / 1e12 if d["eval_res_ns"] else None
    ach_del = (4.0 * n_obs * ec) / (d["eval_delta_ns"] * 1e-9) / 1e12 if d["eval_delta_ns"] else None
    achieved = (6.0 * n_obs * ec) / (d["eval_ns"] * 1e-9) / 1e12 if d["eval_ns"] else None
    # the window evaluation's peak: 4 ops at the k_delta mix and 2 at the k_res mix per entry and candidate
    peak_eval = 6.0 / (4.0 / peaks["k_delta_mix"] + 2.0 / peaks["k_res_mix"])
    # per pipeline step: k_res, k_delta (window t), k_select (window t-1; it
    # also builds window t+1), k_seed (window t+1); a row takes one step more
    # than it decides windows; per row k_row_begin and the seeds of window 0;
    # per refresh k_stats, k_maxplus_planes, k_td_finalize, k_rank,
    # k_scatter_f; per sweep k_sweep_begin
    rows_visited = args.steps * m_or
    launches = 4 * (d["windows"] + rows_visited) + 2 * rows_visited + 5 * d["refreshes"] + args.steps

    if rank_id != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    heldout = {"rmse_a": rmse_a, "rmse_p": rmse_p, "given": n_a, "held_out": n_p,
               "after_sweeps": args.warmup + args.steps}
    cpu = None
    if not args.no_cpu_baseline:
        import oracle  # noqa: F401  (CPU baseline leg only)
        oa, op, _, _ = oracle.rmse(R_np, M_np, U_h.numpy().astype(np.float64), V_h.numpy().astype(np.float64))
        heldout.update(oracle_rmse_a=oa, oracle_rmse_p=op)
        rows, secs, _, used = oracle_rows(R_np, M_np, r, args.seed, U_w, V_w, budget_s=0.0, min_rows=CPU_ROWS,
                                          max_rows=CPU_ROWS)
        cpu = {"value": rows / secs / m_or, "unit": "sweeps/s", "cores": used, "kind": "oracle",
               "sample": "rows 0..%d of sweep %d of the same run, from the library's state after the %d warm-up "
                         "sweeps (the reference arm's start), oracle on %d host threads (nproc %d), %.1f s; "
                         "sweeps/s = rows/s / %d rows" % (rows - 1, args.warmup, args.warmup, used,
                                                          os.cpu_count() or 0, secs, m_or)}

    h2d = (R_np.nbytes + mask_words_host.numel() * 4) / args.steps
    d2h = (U_h.numel() + V_h.numel()) * 4 / args.steps
    rd = lambda x, n=4: None if x is None else round(x, n)   # noqa: E731
    line = {
        "metric": METRIC, "value": value, "unit": "sweeps/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * t_timed / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w["label"], "m": int(R_np.shape[0]), "n": int(R_np.shape[1]), "rank": r,
                   "given": n_obs, "step": "one ByRow sweep (sweeps %d..%d of one run)"
                                           % (args.warmup, args.warmup + args.steps - 1),
                   "l2": "flushed (256 MiB write) before every timed sweep",
                   "parallelism": "independent replicas" if world > 1 else "single GPU"},
        "gops": gops, "gops_frac_of_addmax_peak": gops / (peaks["addmax_1to1"] * 1e3),
        "steady_state": {"candidates_tried_per_sweep": d["candidates_tried"] / args.steps,
                         "candidates_per_row": d["candidates_tried"] / (args.steps * m_or),
                         "candidates_issued_per_sweep": d["candidates_issued"] / args.steps,
                         "accepted_per_sweep": d["accepted"] / args.steps,
                         "windows_per_row": d["windows"] / (args.steps * m_or),
                         "candidates_per_window": d["candidates_issued"] / max(d["windows"], 1),
                         "candidates_dropped_per_sweep": d["candidates_discarded"] / args.steps,
                         "launch_shapes": {"k_res_chunk": rep1["eval_res_chunk"],
                                           "k_delta_blocks": rep1["eval_delta_blocks"],
                                           "k_delta_tile_rows": rep1["eval_delta_rows"]},
                         "window_eval_share_of_sweep": d["eval_ns"] * 1e-9 / t_timed if world == 1 else None},
        "peaks_measured_Tops": {k: rd(v) for k, v in peaks.items()},
        "heldout_rmse": heldout,
        "roofline": {"kernel": "%s (phase 2 of a window: error changes of all its candidates)"
                               % ("k_delta8" if rep1["eval_delta_rows"] == 8 else "k_delta"),
                     "bound": "alu", "achieved": ach_del, "peak": peaks["k_delta_mix"], "unit": "Top/s",
                     "frac": ach_del / peaks["k_delta_mix"] if ach_del else None,
                     "peak_source": "measured at run time (stmf_peak_addmax mode 6: k_delta's instruction mix, "
                                    "4 algorithmic ops per entry and candidate)",
                     "frac_of_addmax_1to1": ach_del / peaks["addmax_1to1"] if ach_del else None,
                     "traffic": eval_traffic(args.workload, "k_delta8" if rep1["eval_delta_rows"] == 8 else "k_delta"),
                     "traffic_unit": "bytes per launch",
                     "launches": d["eval_launches"], "avg_launch_us": d["eval_delta_ns"] / 1e3 / max(d["eval_launches"], 1),
                     "candidates_per_launch": ec / max(d["eval_launches"], 1),
                     "ops_per_given_entry_per_candidate": 4,
                     "timing": "per-launch device time from %globaltimer (kernels run inside a CUDA graph)",
                     "phase1_k_res": {"achieved": ach_res, "peak": peaks["k_res_mix"],
                                      "frac": ach_res / peaks["k_res_mix"] if ach_res else None,
                                      "peak_source": "stmf_peak_addmax mode 7 (k_res's mix, 2 ops per entry)",
                                      "avg_launch_us": d["eval_res_ns"] / 1e3 / max(d["eval_launches"], 1),
                                      "ops_per_given_entry_per_candidate": 2},
                     "window_eval": {"achieved": achieved, "peak": peak_eval,
                                     "frac": achieved / peak_eval if achieved else None,
                                     "avg_us": d["eval_ns"] / 1e3 / max(d["eval_launches"], 1),
                                     "span": "k_res start to k_delta end, 6 ops per given entry per candidate"}},
        "e2e": {"value": args.steps * world / t_e2e, "unit": "sweeps/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "job": "the same %d sweeps through the public API from pinned host buffers, with the job's "
                       "upload of R and the mask, its initialisation and the download of U, V (%.2f s; the %d "
                       "warm-up sweeps, %.2f s, are left out)" % (args.steps, t_e2e, args.warmup, t_apart)},
        "gpu_launches": int(launches),
        "clocks": clocks.summary(),
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
