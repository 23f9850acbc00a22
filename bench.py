"""Benchmark of the BM-Global hot path on one GB300 (or N independent replicas).

Default (`--mode grad`): one step = one evaluation of the loss and both
gradients (bm_loss_grad: the SDDMM residual and the SpMMs R H and R^T W) on
the recommendation-scale workload (480,189 x 17,770, 100,480,507 Zipf(1.2)
ratings, lambda = 0.25, k = 64, FP32); `value` = observed entries per second
summed over replicas ("BM gradient nnz/s").  The line carries the roofline of
the dominant pass (against the FP32 ALU and HBM peaks and against the measured
gather roof of its index order), the whole call's fractions, the FP64
oracle's rate on the host cores, an end-to-end figure through host buffers,
and secondary figures: cycles of Algorithm 1 on the same handle, time to the
oracle's objective on the planted 500 x 300 problem, a serving sample.

`--mode cycle` times cycles of Algorithm 1 (3 BM iterations + 1 inexact PG
step) instead.  `--mode tto` times a solve to the FP64 oracle's objective on
the planted 500 x 300 problem; `--mode serve` measures the continuous-batching
server.  `--mode edm` times the distance-geometry loss/gradient and
`--mode edm_solve` the cycles of Algorithm 1 on the distance-geometry QSDP
(30,000-point chain); `--mode bcd` compares the column-block BM solver with
the PR+ BM phase.  `--impl reference` times the FP64 oracle on the host cores
on a bounded sample of the same workload.
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

WORKLOAD = "netflix"
K_BENCH = 64
LMSVD_TOL = 1e-5   # the library's default LmSVD stop tolerance (bm_default_options)


def _load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return d, "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def _clock_sampler(path):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    try:
        f = open(path, "w")
        return subprocess.Popen(["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "200"],
                                stdout=f, stderr=subprocess.DEVNULL), f
    except (OSError, FileNotFoundError):
        return None, None


def _clock_summary(path, dev):
    sm, mx, reasons = [], 0.0, set()
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    try:
        for line in open(path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9 or parts[0] != str(dev):
                continue
            try:
                sm.append(float(parts[1]))
                mx = max(mx, float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
    except OSError:
        pass
    return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx or None,
            "reasons": sorted(reasons), "samples": len(sm)}


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws > 1:
        import torch.distributed as dist
        if not dist.is_initialized():
            backend = "nccl"
            dist.init_process_group(backend=backend)
        return dist, dist.get_rank(), ws
    return None, 0, 1


def _reduce(dist, x, op):
    """All-reduce one host scalar over the replicas (NCCL on GPUs, gloo on CPU)."""
    if dist is None:
        return x
    import torch
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=op)
    return float(t.item())


def _maxall(dist, x):
    return x if dist is None else _reduce(dist, x, dist.ReduceOp.MAX)


def _sumall(dist, x):
    return x if dist is None else _reduce(dist, x, dist.ReduceOp.SUM)


def replica_throughput(dist, ms_per_step, units_per_step):
    """Whole-job figures of N independent replicas: the slowest rank's step
    time and the units all ranks processed per step over it."""
    ms = _maxall(dist, ms_per_step)
    units = _sumall(dist, float(units_per_step))
    return ms, units, units / (ms / 1e3)


def algorithmic_bytes(kernel, d, k, q, vb=4):
    """Algorithmic DRAM bytes of one launch (unique data each launch must move).

    grad_csr: col idx + value per entry (4 + vb B; vb = 1 with the one-byte
              value codec, else 4), residual write (4 B), W read, gW write
              (m*k*4 each), H read once (n*k*4).
    grad_csc: row idx + value (4 + vb B; the column pass writes no
              residual), H read, gH write, W read once.
    linesearch_csr: col idx + residual (8 B), W, DW (m*k*4 each), H, DH (n*k*4 each).
    spmm_csc / spmm_csr (prox): idx + residual value (8 B), gathered block
              read once (rows*q*4), output read + write (2*rows*q*4).
    """
    m, n, nnz = d["m"], d["n"], d["nnz"]
    if kernel == "grad_csr":
        return nnz * (8 + vb) + (2 * m + n) * k * 4
    if kernel == "grad_csc":
        return nnz * (4 + vb) + (2 * n + m) * k * 4
    if kernel == "linesearch_csr":
        return nnz * 8 + 2 * (m + n) * k * 4
    if kernel == "spmm_csc":
        return nnz * 8 + m * q * 4 + 2 * n * q * 4
    if kernel == "spmm_csr":
        return nnz * 8 + n * q * 4 + 2 * m * q * 4
    return None


def algorithmic_flops(kernel, d, k, q):
    nnz = d["nnz"]
    if kernel in ("grad_csr", "grad_csc"):
        return nnz * (4 * k + 2)
    if kernel == "linesearch_csr":
        return nnz * (6 * k + 8)
    if kernel in ("spmm_csc", "spmm_csr"):
        return nnz * 2 * q
    return None


def run_ours(args):
    import torch

    import paper_2204_14067_gb300 as B
    from synth import named_config, random_factors

    dist, rank, ws = _dist()
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    t_gen = time.time()
    p = named_config(args.config)
    t_gen = time.time() - t_gen
    opt = B.bm_default_options()
    opt.precision = args.precision
    opt.value_codec = args.codec
    opt.tensor_grams = args.tensor_grams
    if args.lmsvd_tol is not None:
        opt.lmsvd_tol = args.lmsvd_tol
    k_cap = min(p.k_max, 127)            # the library's rank cap (k_max + 1 vectors fit 128-wide rows)
    h = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, k_cap, opt)
    codec_on = B.bm_get_codes(h)[0]
    stream = torch.cuda.Stream()
    B.bm_set_stream(h, stream)
    d = B.bm_dims(h)
    k = min(args.k or K_BENCH, k_cap)
    W0, H0 = random_factors(p.m, p.n, k, seed=11, scale=0.1)
    B.bm_set_factors(h, k, W0, H0)
    # work-split autotuning of the sparse passes (panel order for L2 reuse)
    tune = None if args.no_tune else B.bm_autotune(h)

    gWd = torch.empty((p.m, k), dtype=torch.float32, device="cuda")
    gHd = torch.empty((p.n, k), dtype=torch.float32, device="cuda")
    # gather roof of the gradient passes: a gather-only pass over the same
    # index order (bm_gather_roof), outside the timed region
    gather = {nm: B.bm_gather_roof(h, nm) for nm in ("grad_csr", "grad_csc")} if args.mode == "grad" else {}

    def step():
        if args.mode == "grad":
            B.bm_loss_grad(h, gWd, gHd)
        else:
            B.bm_solve(h, max_outer=1, tol=0.0)   # one cycle of Algorithm 1

    def steps(count):
        # cycle mode: one bm_solve call of `count` cycles, as a solve runs them
        # (the call's closing objective evaluation is paid once, not per cycle)
        if args.mode == "grad":
            for _ in range(count):
                step()
        else:
            B.bm_solve(h, max_outer=count, tol=0.0)

    steps(args.warmup)
    torch.cuda.synchronize()
    if dist is not None:
        dist.barrier()
    clk_path = os.path.join(tempfile.gettempdir(), f"bm_bench_clocks_r{rank}_{os.getpid()}.csv")
    os.makedirs(os.path.dirname(clk_path), exist_ok=True)
    sampler, fh = _clock_sampler(clk_path)
    B.bm_profile_enable(h, True)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("timed")     # lets an ncu capture select the timed launches
    ev0.record(stream)
    steps(args.steps)
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    ms = ev0.elapsed_time(ev1)
    prof = B.bm_profile_read(h)
    B.bm_profile_enable(h, False)
    if sampler is not None:
        sampler.terminate()
        sampler.wait()
        fh.close()
    clocks = _clock_summary(clk_path, local)
    k_now = B.bm_dims(h)["k"]

    # end to end through the public API with host buffers, copies inside the
    # timed region: grad mode copies the factors in and both gradients out;
    # cycle mode copies the whole solve state (factors and the PG step's warm
    # start) in and out, so every cycle runs from the state the last one left
    Wh = np.ascontiguousarray(W0)
    Hh = np.ascontiguousarray(H0)
    e2e_steps = max(1, min(args.steps, 3))
    if args.mode == "cycle":
        # pinned host buffers for the state, sized for the largest rank
        state = torch.empty(B.bm_state_size(h) + (1 << 20), dtype=torch.uint8, pin_memory=True)
        n_state = B.bm_get_state(h, state)
    else:
        Wh = torch.from_numpy(Wh).pin_memory()
        Hh = torch.from_numpy(Hh).pin_memory()
        gW = torch.empty_like(Wh).pin_memory()
        gH = torch.empty_like(Hh).pin_memory()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2d = d2h = 0
    for _ in range(e2e_steps):
        if args.mode == "grad":
            B.bm_set_factors(h, k, Wh, Hh)
            B.bm_loss_grad(h, gW, gH)
            h2d = (Wh.numel() + Hh.numel()) * 4
            d2h = (gW.numel() + gH.numel()) * 4
        else:
            B.bm_set_state(h, state, n_state)
            B.bm_solve(h, max_outer=1, tol=0.0)
            h2d = n_state
            n_state = B.bm_get_state(h, state)
            d2h = n_state
    torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    # secondary figures of the default (gradient) run: cycles of Algorithm 1
    # on the same handle, time to the oracle's objective, a serving sample
    extra = {}
    if args.mode == "grad" and not args.no_extra:
        B.bm_solve(h, max_outer=2, tol=0.0)
        ev2, ev3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ev2.record(stream)
        B.bm_solve(h, max_outer=5, tol=0.0)
        ev3.record(stream)
        torch.cuda.synchronize()
        cyc_ms = ev2.elapsed_time(ev3) / 5
        extra["cycle"] = {"metric": "BM-Global cycle nnz/s", "value": p.nnz / (cyc_ms / 1e3), "unit": "nnz/s",
                          "ms_per_cycle": cyc_ms, "cycles": 5, "k_end": B.bm_dims(h)["k"],
                          "step": "3 BM iterations + 1 inexact PG step"}
    B.bm_destroy(h)
    if args.mode == "grad" and not args.no_extra:
        import types
        sub = types.SimpleNamespace(**vars(args))
        sub.steps, sub.warmup, sub.no_cpu = 1, 1, False
        t = run_tto(sub)
        extra["time_to_oracle"] = {"metric": t["metric"], "value": t["value"], "unit": "s",
                                   "workload": t["config"]["workload"], "cycles": t["config"]["cycles"],
                                   "final_rel": t["config"]["final_rel"], "e2e_s": t["e2e"]["value"],
                                   "oracle_s": (t["cpu_baseline"] or {}).get("value")}
        sub.serve_count = 16
        sub.serve_max_nnz = 1_000_000
        sv = run_serve(sub)
        extra["serving"] = {"metric": sv["metric"], "value": sv["value"], "unit": sv["unit"],
                            "workload": sv["config"]["workload"], "batched_bf16": sv["batched_bf16"],
                            "one_at_a_time_fp32": sv["one_at_a_time_fp32"], "final_objective": sv["final_objective"],
                            "oracle_check": sv["oracle_check"],
                            "saturation_solves_per_s": sv["saturation_solves_per_s"]}

    ms_step, total_units, value = replica_throughput(dist, ms / args.steps, p.nnz)
    e2e_val = _sumall(dist, float(p.nnz)) / _maxall(dist, e2e_s)
    if rank != 0:
        return None
    peaks, peak_kind = _load_peaks()
    # dominant kernel: the largest total device time among kernels with a work model
    # dominant kernel: the largest total device time among the passes whose
    # per-launch work is fixed (the q-wide SpMMs of the PG step run with two
    # block widths in one cycle, so one launch has no single work figure)
    modeled = {nm: v for nm, v in prof.items()
               if nm in ("grad_csr", "grad_csc", "linesearch_csr") and algorithmic_bytes(nm, d, 1, 1) is not None}
    top_all = max(prof.items(), key=lambda kv: kv[1][1])[0] if prof else None
    dom = max(modeled.items(), key=lambda kv: kv[1][1]) if modeled else (None, (0, 0.0))
    name, (launches, tot_ms) = dom
    q = k_now + 1
    kk = k_now if args.mode == "cycle" else k
    fl = algorithmic_flops(name, d, kk, q) if name else None
    by = algorithmic_bytes(name, d, kk, q, 1 if codec_on else 4) if name else None
    avg_s = (tot_ms / launches) / 1e3 if launches else None
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    n_sms = torch.cuda.get_device_properties(local).multi_processor_count
    alu_peak = n_sms * 128 * 2 * sm_max * 1e6 / 1e12  # FP32 FMA lanes x 2 flops x max SM clock, TFLOP/s
    roof = None
    if avg_s and fl is not None and by is not None:
        intensity = fl / by
        ridge = alu_peak * 1e12 / (float(peaks["hbm_gbs"]) * 1e9)
        # DRAM bytes of a full-size launch are not captured: the two DRAM
        # counters take two ncu passes, and multi-pass captures run on the
        # quarter-size case only (profiles/grad_sparse_netflix_quarter_k64.txt)
        traffic = None
        if intensity >= ridge:
            ach = fl / avg_s / 1e12
            roof = {"bound": "alu", "kernel": name, "achieved": ach, "peak": alu_peak, "unit": "TFLOP/s",
                    "frac": ach / alu_peak, "traffic": traffic,
                    "peak_source": f"derived: {n_sms} SMs (device attribute) x 128 FP32 lanes x 2 x {sm_max:.0f} MHz",
                    "hbm_achieved_gbs": by / avg_s / 1e9, "hbm_peak_gbs": float(peaks["hbm_gbs"]),
                    "hbm_frac": by / avg_s / 1e9 / float(peaks["hbm_gbs"]), "hbm_peak_source": peak_kind}
        else:
            ach = by / avg_s / 1e9
            roof = {"bound": "hbm", "kernel": name, "achieved": ach, "peak": float(peaks["hbm_gbs"]),
                    "unit": "GB/s", "frac": ach / float(peaks["hbm_gbs"]), "traffic": traffic,
                    "peak_source": peak_kind}
        roof["bytes_per_launch"] = by
        roof["flops_per_launch"] = fl
        roof["avg_launch_ms"] = avg_s * 1e3
        roof["top_kernel_overall"] = top_all
        roof["traffic_note"] = ("not captured at full size (two-pass counters); quarter-size case: "
                                "profiles/grad_sparse_netflix_quarter_k64.txt")
        if name in gather:
            # the pass gathers one FP32 row per entry; the measured roof is a
            # gather-only pass over the same index order
            g_ms, g_gbs = gather[name]
            gb = d["nnz"] * kk * 4
            roof["l2_gather"] = {"achieved_gbs": gb / avg_s / 1e9, "peak_gbs": g_gbs, "frac": g_ms / (avg_s * 1e3),
                                 "gathered_bytes_per_launch": gb,
                                 "peak_source": "measured: gather-only pass over the same index (bm_gather_roof)"}
    # the whole loss/gradient call (every pass it launches) against both roofs
    grad_call = None
    if args.mode == "grad":
        vb = 1 if codec_on else 4
        by_call = algorithmic_bytes("grad_csr", d, k, 0, vb) + algorithmic_bytes("grad_csc", d, k, 0, vb)
        fl_call = algorithmic_flops("grad_csr", d, k, 0) + algorithmic_flops("grad_csc", d, k, 0)
        s_call = ms_step / 1e3
        grad_call = {"ms": ms_step, "algorithmic_bytes": by_call, "flops": fl_call,
                     "hbm_gbs": by_call / s_call / 1e9,
                     "hbm_frac": by_call / s_call / 1e9 / float(peaks["hbm_gbs"]),
                     "alu_tflops": fl_call / s_call / 1e12, "alu_frac": fl_call / s_call / 1e12 / alu_peak,
                     "kernels": sorted(prof)}
        if gather:
            g_ms = sum(v[0] for v in gather.values())
            grad_call["l2_gather"] = {"gather_only_ms": g_ms, "frac": g_ms / ms_step,
                                      "gathered_bytes": 2 * d["nnz"] * k * 4,
                                      "note": "both passes gather one FP32 factor row per entry; the roof is the "
                                              "time of gather-only passes over the same index orders"}
    cpu = cpu_baseline(p, args.mode) if not args.no_cpu else None
    line = {
        "metric": "BM gradient nnz/s" if args.mode == "grad" else "BM-Global cycle nnz/s",
        "value": value,
        "unit": "nnz/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32" if args.precision == 0 else "bf16 gathers, f32 accumulation",
        "data": "synthetic",
        "config": {"workload": (f"{p.name}-shaped {p.m}x{p.n}, nnz={p.nnz}, Zipf(1.2), "
                                f"ratings {int(p.vals.min())}..{int(p.vals.max())}"),
                   "lambda": p.lam, "k": k, "k_end": k_now, "step": "3 BM iterations + 1 inexact PG step"
                   if args.mode == "cycle" else "one loss/gradient evaluation",
                   "parallelism": f"replicas x{ws}", "l2": "inputs larger than L2 (1.6 GB of index per pass)",
                   "generate_s": round(t_gen, 1),
                   "value_codec": "one byte per observed value" if codec_on else "fp32 values",
                   "work_split": ({nm: {"panels": v[0], "layout": "warp per segment" if v[3] else "group per segment"}
                                   for nm, v in tune.items()} if tune else "natural split, automatic layout")},
        "e2e": {"value": e2e_val, "unit": "nnz/s",
                "h2d_bytes_per_step": int(h2d),
                "d2h_bytes_per_step": int(d2h)},
        "gpu_launches": int(sum(v[0] for v in prof.values())) // max(1, args.steps) * args.steps,
        "kernels": {kname: {"launches": v[0], "ms": round(v[1], 4)} for kname, v in sorted(prof.items())},
        "roofline": roof,
        "gradient_call": grad_call,
        "secondary": extra or None,
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    return line


def _subproblem(p, target_nnz, seed=0):
    """A bounded sample of the workload: a random subset of the short side's
    indices (internal rows) with all of their observed entries."""
    rng = np.random.default_rng(seed)
    short_is_cols = p.n < p.m
    ids = p.cols if short_is_cols else p.rows
    count = p.n if short_is_cols else p.m
    deg = np.bincount(ids, minlength=count)
    order = rng.permutation(count)
    take = order[np.cumsum(deg[order]) <= target_nnz]
    keep = np.zeros(count, bool)
    keep[take] = True
    sel = keep[ids]
    remap = -np.ones(count, np.int64)
    remap[take] = np.arange(take.size)
    rows, cols = p.rows[sel], p.cols[sel]
    if short_is_cols:
        cols = remap[cols]
        return p.m, take.size, rows, cols, p.vals[sel]
    rows = remap[rows]
    return take.size, p.n, rows, cols, p.vals[sel]


def cpu_baseline(p, mode, target_nnz=400_000):
    """The FP64 oracle, as it stands, timed on this host on a bounded sample."""
    from oracle import bm_oracle as O
    from synth import random_factors
    m, n, rows, cols, vals = _subproblem(p, target_nnz)
    ix = O.build_index(m, n, rows, cols, vals.astype(np.float64))
    k = min(K_BENCH, ix.m)
    W, H = random_factors(ix.m, ix.n, k, seed=11, scale=0.1)
    W, H = W.astype(np.float64), H.astype(np.float64)
    opt = O.Options(lmsvd_tol=LMSVD_TOL)     # the library's default stop tolerance
    st = O.State(W=W, H=H, U_prev=O.orth(W)[0], U_prev2=None, u=None, psi=opt.psi0,
                 rank_hist=[k, k], prev_warm_cols=k + 1, t=0, bm_changed=True)
    t0 = time.perf_counter()
    reps = 0
    while True:
        if mode == "grad":
            O.loss_grad(ix, st.W, st.H, p.lam)
        else:
            st, _ = O.bm_phase(ix, st, p.lam, 3)
            st, _ = O.prox_step(ix, st, p.lam, p.k_max, opt)
        reps += 1
        el = time.perf_counter() - t0
        if el > 10.0 or reps >= 50:
            break
    return {"value": ix.nnz * reps / el, "unit": "nnz/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{ix.m}x{ix.n} sub-matrix with {ix.nnz} entries (random subset of the short side), "
                      f"{reps} {'gradient evaluations' if mode == 'grad' else 'cycles'}, {el:.1f} s"}


def run_reference(args):
    dist, rank, ws = _dist_cpu()
    if rank != 0:
        return None
    if args.mode not in ("grad", "cycle"):
        return {"impl": "reference",
                "unavailable": ("the reference arm (the FP64 oracle on the host cores) is timed for --mode grad "
                                "and --mode cycle; in tto, edm and edm_solve the oracle's own figure is the "
                                "line's cpu_baseline, serve and bcd have no oracle timing")}
    from synth import named_config
    p = named_config(args.config)
    from oracle import bm_oracle as O
    from synth import random_factors
    m, n, rows, cols, vals = _subproblem(p, 400_000)
    ix = O.build_index(m, n, rows, cols, vals.astype(np.float64))
    k = min(K_BENCH, ix.m)
    W, H = random_factors(ix.m, ix.n, k, seed=11, scale=0.1)
    opt = O.Options(lmsvd_tol=LMSVD_TOL)     # the library's default stop tolerance
    st = O.State(W=W.astype(np.float64), H=H.astype(np.float64), U_prev=O.orth(W.astype(np.float64))[0],
                 U_prev2=None, u=None, psi=opt.psi0, rank_hist=[k, k], prev_warm_cols=k + 1, t=0,
                 bm_changed=True)

    def step():
        nonlocal st
        if args.mode == "grad":
            O.loss_grad(ix, st.W, st.H, p.lam)
        else:
            st, _ = O.bm_phase(ix, st, p.lam, 3)
            st, _ = O.prox_step(ix, st, p.lam, p.k_max, opt)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    el = (time.perf_counter() - t0) / args.steps
    v = ix.nnz / el
    return {"impl": "reference", "metric": "BM gradient nnz/s" if args.mode == "grad" else "BM-Global cycle nnz/s",
            "value": v, "unit": "nnz/s", "n_gpus": ws, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": el * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic",
            "config": {"workload": (f"{p.name}-shaped {p.m}x{p.n}, nnz={p.nnz}, Zipf(1.2), "
                                    f"ratings {int(p.vals.min())}..{int(p.vals.max())}"),
                       "lambda": p.lam, "k": k,
                       "step": "3 BM iterations + 1 inexact PG step" if args.mode == "cycle"
                       else "one loss/gradient evaluation", "parallelism": "host cores, rank 0 only"},
            "cpu_baseline": {"value": v, "unit": "nnz/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": (f"each step on a {ix.m}x{ix.n} sub-matrix with {ix.nnz} entries (a "
                                        f"random subset of the short side with all its entries), scaled to nnz/s")},
            "e2e": {"value": v, "unit": "nnz/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def _read_golden_tiny():
    vals = {}
    for line in open(os.path.join(ROOT, "tests", "golden", "tiny_optimum.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, v = line.split()
        vals[k] = float(v)
    return vals["F_star"], int(vals["rank"])


def run_tto(args):
    """Time to the oracle's objective: wall time of bm_solve from X = 0 until
    F <= F*(1 + 1e-6) on the 500 x 300 planted problem, F* being the FP64
    oracle's converged objective (tests/golden/tiny_optimum.txt)."""
    import torch

    import paper_2204_14067_gb300 as B
    from synth import named_config

    F_star, rank = _read_golden_tiny()
    p = named_config("tiny")
    target = F_star * (1 + 1e-6)
    opts = B.bm_default_options()
    opts.step_rule = args.step_rule
    if args.lmsvd_tol is not None:
        opts.lmsvd_tol = args.lmsvd_tol
    runs = []
    for rep in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        h = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, 64, opts)
        t1 = time.perf_counter()
        r = B.bm_solve(h, max_outer=2000, tol=0.0, F_target=target)
        torch.cuda.synchronize()
        t2 = time.perf_counter()
        B.bm_get_factors(h, p.m, p.n)
        t3 = time.perf_counter()
        B.bm_destroy(h)
        if rep >= args.warmup:
            runs.append((t2 - t1, t3 - t0, r["outer"], r["F"], bool(r["converged"])))
    solve_s = statistics.median(x[0] for x in runs)
    e2e_s = statistics.median(x[1] for x in runs)
    cpu = None
    if not args.no_cpu:
        from oracle import bm_oracle as O
        ix = O.build_index(p.m, p.n, p.rows, p.cols, p.vals.astype(np.float64))
        t0 = time.perf_counter()
        if args.step_rule == 1:
            from oracle import sparsa_oracle as S
            _, Fh, _ = S.solve_bb(ix, p.lam, 8, 64, O.Options(lmsvd_tol=args.lmsvd_tol or LMSVD_TOL),
                                  S.BbOptions(), max_outer=2000, tol=0.0,
                                  F_target=target)
            cycles = len(Fh) - 1
        else:
            _, oi = O.solve(ix, p.lam, 8, 64, O.Options(lmsvd_tol=args.lmsvd_tol or LMSVD_TOL), max_outer=2000,
                            tol=0.0, F_target=target)
            cycles = oi.outer
        cpu = {"value": time.perf_counter() - t0, "unit": "s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"the same solve to the same target ({cycles} cycles)"}
    return {
        "metric": "time to oracle objective (relative 1e-6)", "value": solve_s, "unit": "s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": solve_s * 1e3, "higher_is_better": False,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "planted rank-5 500x300, 15,000 entries, lambda 0.5, k0 8, k_max 64",
                   "step_rule": "SpaRSA (BB + backtracking)" if args.step_rule == 1 else "fixed alpha 1.99",
                   "F_star": F_star, "oracle_rank": rank, "cycles": [x[2] for x in runs],
                   "converged": all(x[4] for x in runs), "final_rel": max((x[3] - F_star) / F_star for x in runs)},
        "e2e": {"value": e2e_s, "unit": "s", "h2d_bytes_per_step": int(p.nnz * 12),
                "d2h_bytes_per_step": int((p.m + p.n) * 64 * 4)},
        "cpu_baseline": cpu,
    }


def run_serve(args):
    """Continuous-batching serving on a prefix of the serving stream (m
    log-U[1k, 200k], n log-U[500, 20k], density log-U[0.1 %, 2 %], nnz up to
    --serve-max-nnz, planted rank 2..16): half the requests take lambda from the
    stream's grid {0.02 .. 0.5} max|A| (these run into the rank cap of 32), half
    from {3, 5, 8} max|A| (optimum below the cap: the solves converge).  First
    the capacity of one-at-a-time FP32 solves, then Poisson arrivals at 0.8 of
    it served by the batched BF16 server (FP32 refinement) and by the
    one-at-a-time FP32 server.  Final objectives of solves that converged in
    both are compared, and a sample of served solutions is re-evaluated and
    compared with the optimum by the FP64 oracle."""
    import torch

    import paper_2204_14067_gb300 as B
    from synth import serving_requests

    count = args.serve_count
    probs, _ = serving_requests(count=count, seed=4, max_nnz=args.serve_max_nnz or None, k_max=32,
                                lam_grid2=(3.0, 5.0, 8.0), share2=0.5)
    torch.cuda.synchronize()
    cap_outer = 60

    def serve(arrivals, **kw):
        s = B.bm_server_create(max_outer=cap_outer, tol=1e-7, keep_factors=1, **kw)
        try:
            t0 = time.perf_counter()
            ids = []
            for q, t in zip(probs, arrivals):
                d = t - (time.perf_counter() - t0)
                if d > 0:
                    time.sleep(d)
                ids.append(B.bm_server_submit(s, q.m, q.n, q.rows, q.cols, q.vals, q.lam, q.k_max))
            B.bm_server_drain(s, 3600.0)
            wall = time.perf_counter() - t0
            res = {r["id"]: r for r in B.bm_server_results(s)}
            err = B.binding.lib().bm_server_last_error(s)
            out = [res[i] for i in ids]
            facs = {}
            for j, (i, q) in enumerate(zip(ids, probs)):
                if out[j]["status"] == 0:
                    facs[j] = B.bm_server_factors(s, i, q.m, q.n)
            return out, wall, (err.decode() if err else ""), facs
        finally:
            B.bm_server_destroy(s)

    plain0, t_cap, _, _ = serve(np.zeros(count), max_active=1, precision=0, batched=0, workers=1)
    cap = count / t_cap
    # saturation throughput of the batched server (every request queued at 0)
    bat0, t_cap_b, _, _ = serve(np.zeros(count), max_active=16, precision=1, batched=1, workers=8)
    rate = 0.8 * cap
    rng = np.random.default_rng(123)
    arrivals = np.cumsum(rng.exponential(1.0 / rate, count))
    bat, wall_b, err_b, fb = serve(arrivals, max_active=16, precision=1, batched=1, workers=8)
    pla, wall_p, err_p, fp = serve(arrivals, max_active=1, precision=0, batched=0, workers=1)

    def stats(res, wall):
        lat = np.array([r["t_done"] - r["t_submit"] for r in res])
        return {"p50_s": float(np.percentile(lat, 50)), "p99_s": float(np.percentile(lat, 99)),
                "solves_per_s": len(res) / wall, "wall_s": wall,
                "errors": int(sum(r["status"] != 0 for r in res))}

    sb, sp = stats(bat, wall_b), stats(pla, wall_p)
    if err_b:
        sb["last_error"] = err_b
    if err_p:
        sp["last_error"] = err_p
    # equal final objective where both solves ended on the tolerance (a solve
    # that ran into the cycle cap stopped wherever it was)
    ok = [(j, a, b) for j, (a, b) in enumerate(zip(bat, pla)) if a["status"] == 0 and b["status"] == 0]
    conv = [(j, a, b) for j, a, b in ok if a["outer"] < cap_outer and b["outer"] < cap_outer]
    rel_conv = max((abs(a["F"] - b["F"]) / abs(b["F"]) for _, a, b in conv), default=None)
    objective = {"converged_in_both": len(conv),
                 "max_rel_diff_converged": rel_conv,
                 "hit_cycle_cap": {"batched_bf16": int(sum(a["outer"] >= cap_outer for _, a, _ in ok)),
                                   "one_at_a_time_fp32": int(sum(b["outer"] >= cap_outer for _, _, b in ok))}}
    # the oracle on a sample: the smallest converged requests
    check = None
    if not args.no_cpu and conv:
        from oracle import bm_oracle as O
        sample = sorted(conv, key=lambda t: probs[t[0]].rows.shape[0])[:3]
        rows_out = []
        for j, a, b in sample:
            q = probs[j]
            ix = O.build_index(q.m, q.n, q.rows, q.cols, q.vals.astype(np.float64))
            st, oi = O.solve(ix, q.lam, 8, q.k_max, O.Options(), max_outer=400, tol=1e-12)
            F_star = oi.F_hist[-1]
            ent = {"nnz": int(q.rows.shape[0]), "F_oracle_optimum": F_star}
            for tag, fac in (("batched_bf16", fb.get(j)), ("one_at_a_time_fp32", fp.get(j))):
                if fac is None:
                    continue
                W64, H64 = fac[0].astype(np.float64), fac[1].astype(np.float64)
                Wi, Hi = (H64, W64) if ix.transposed else (W64, H64)
                ent[tag + "_rel_to_optimum"] = (O.objective(ix, Wi, Hi, q.lam) - F_star) / F_star
            rows_out.append(ent)
        check = rows_out
    return {
        "metric": "serving solves/s (batched BF16 + FP32 refinement)", "value": sb["solves_per_s"],
        "unit": "solves/s", "n_gpus": 1, "steps": 1, "warmup": 0, "ms_per_step": wall_b * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16/f32", "data": "synthetic",
        "config": {"workload": f"first {count} requests of the serving stream: m log-U[1k,200k], n log-U[500,20k], "
                               f"density log-U[0.1%,2%], nnz <= {args.serve_max_nnz or 'density*m*n'}, planted rank "
                               "2..16, lambda {0.02..0.5} max|A| or (half the requests) {3,5,8} max|A|, k_max 32",
                   "arrival_rate_per_s": rate, "fp32_capacity_per_s": cap, "cycle_cap": cap_outer},
        "batched_bf16": sb, "one_at_a_time_fp32": sp, "final_objective": objective, "oracle_check": check,
        "saturation_solves_per_s": {"batched_bf16": count / t_cap_b, "one_at_a_time_fp32": cap},
    }


def run_edm(args):
    """Distance-geometry loss/gradient (Eq. EDM) on the 30,000-point chain,
    k = 16: one step = one bm_edm_loss_grad; value = pairs / s."""
    import torch

    import paper_2204_14067_gb300 as B
    from synth import self_avoiding_chain

    p = self_avoiding_chain(n=30_000, seed=3)
    k = 16
    lam = -10.0 * np.sqrt(p.n) / float(np.sum(p.d.astype(np.float64) ** 2))   # lambda of the conformation workload
    rng = np.random.default_rng(5)
    V = (p.X_true @ rng.standard_normal((3, k)) * 0.3 + 0.05 * rng.standard_normal((p.n, k))).astype(np.float32)
    h = B.bm_edm_create(p.n, p.i, p.j, p.d, lam, k)
    stream = torch.cuda.Stream()
    B.bm_edm_set_stream(h, stream)
    B.bm_edm_set_factor(h, k, V)
    gV = torch.empty((p.n, k), dtype=torch.float32, device="cuda")
    for _ in range(args.warmup):
        B.bm_edm_loss_grad(h, gV)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    ev0.record(stream)
    for _ in range(args.steps):
        B.bm_edm_loss_grad(h, gV)
    ev1.record(stream)
    torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    t0 = time.perf_counter()
    for _ in range(args.steps):
        B.bm_edm_set_factor(h, k, V)
        gh = np.empty_like(V)
        B.bm_edm_loss_grad(h, gh)
    e2e_s = (time.perf_counter() - t0) / args.steps
    B.bm_edm_destroy(h)
    pairs = p.npairs
    by = 2 * pairs * 8 + 2 * p.n * k * 4        # both directions: column + d^2 per stored pair; V in, gradient out
    fl = 2 * pairs * 6 * k                      # residual (3k) and gradient update (3k) per stored pair
    peaks, kind = _load_peaks()
    ach = by / (ms / 1e3) / 1e9
    cpu = None
    if not args.no_cpu:
        from oracle import bm_oracle as O
        V64 = V.astype(np.float64)
        t0 = time.perf_counter()
        reps = 0
        while time.perf_counter() - t0 < 10.0 and reps < 20:
            O.edm_loss_grad(V64, p.i, p.j, p.d, 1.0, lam)
            reps += 1
        el = time.perf_counter() - t0
        cpu = {"value": pairs * reps / el, "unit": "pairs/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"the full problem, {reps} evaluations, {el:.1f} s"}
    return {
        "metric": "EDM gradient pairs/s", "value": pairs / (ms / 1e3), "unit": "pairs/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"3-D self-avoiding chain, n = {p.n}, {pairs} pairs within 6.0, k = {k}",
                   "l2": "problem fits in L2 (about 30 MB): cached between steps"},
        "e2e": {"value": pairs / e2e_s, "unit": "pairs/s", "h2d_bytes_per_step": int(V.nbytes),
                "d2h_bytes_per_step": int(V.nbytes)},
        "roofline": {"bound": "hbm", "kernel": "edm", "achieved": ach, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                     "frac": ach / float(peaks["hbm_gbs"]), "traffic": None, "peak_source": kind,
                     "bytes_per_launch": by, "flops_per_launch": fl},
        "cpu_baseline": cpu,
    }


def edm_solve_bytes(kernel, n, npairs, ld, q):
    """Algorithmic bytes of one launch of the distance-geometry solve kernels
    (every pair is stored in both directions: 2 * npairs directed entries).

    edm_pass: column index, d^2 and weight per entry (12 B), V read and
              gradient write (n * ld * 4 each); the residual write of the PG
              step's call (4 B per entry) is not counted (the BM iterations,
              which dominate, do not write it).
    edm_ls:   column index, d^2 and weight per entry (12 B), V and D read
              (n * ld * 4 each).
    edm_lap:  column index + coefficient per entry (8 B), block read once
              (n * q * 4), output read + write (2 * n * q * 4).
    """
    E = 2 * npairs
    if kernel == "edm_pass":
        return E * 12 + 2 * n * ld * 4
    if kernel == "edm_ls":
        return E * 12 + 2 * n * ld * 4
    if kernel == "edm_lap":
        return E * 8 + 3 * n * q * 4
    return None


def run_edm_solve(args):
    """Algorithm 1 on the distance-geometry QSDP, the 30,000-point chain
    (about 450,000 pairs within 6.0), k_max = 16: one step = one cycle of
    30 BM iterations (PR+ with the exact quartic line search) and one inexact
    PG step (LmSVD on Z + sigma J, projection, rank rule).  The initial PG step
    from X = 0 and W warm-up cycles run before the timed region."""
    import torch

    import paper_2204_14067_gb300 as B
    from synth import self_avoiding_chain

    p = self_avoiding_chain(n=30_000, seed=3)
    k_max, epochs = 16, 30
    lam = -10.0 * np.sqrt(p.n) / float(np.sum(p.d.astype(np.float64) ** 2))   # lambda of the conformation workload
    h = B.bm_edm_create(p.n, p.i, p.j, p.d, lam, k_max)
    o = B.bm_default_options()
    o.bm_epochs = epochs
    B.bm_edm_set_options(h, o)
    stream = torch.cuda.Stream()
    B.bm_edm_set_stream(h, stream)
    t0 = time.perf_counter()
    init = B.bm_edm_init(h)
    init_s = time.perf_counter() - t0
    F_hist = [init["F"]]

    def cycle():
        B.bm_edm_bm_phase(h, epochs)
        return B.bm_edm_prox_step(h)

    for _ in range(args.warmup):
        F_hist.append(cycle()["F"])
    clk_path = os.path.join(tempfile.gettempdir(), f"bm_bench_clocks_edm_{os.getpid()}.csv")
    os.makedirs(os.path.dirname(clk_path), exist_ok=True)
    sampler, fh = _clock_sampler(clk_path)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    ev0.record(stream)
    infos = []
    for _ in range(args.steps):
        infos.append(cycle())
    ev1.record(stream)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_pop()
    ms = ev0.elapsed_time(ev1) / args.steps
    if sampler is not None:
        sampler.terminate()
        sampler.wait()
        fh.close()
    clocks = _clock_summary(clk_path, 0)
    F_hist += [x["F"] for x in infos]
    # kernel breakdown of the same cycles (events around every launch)
    B.bm_edm_profile_enable(h, True)
    for _ in range(args.steps):
        cycle()
    prof = B.bm_edm_profile_read(h)
    B.bm_edm_profile_enable(h, False)
    k_now = B.bm_edm_get_factor(h, p.n).shape[1]
    # end to end through the public API with host buffers: factor in, one cycle, factor out
    Vh = np.ascontiguousarray(B.bm_edm_get_factor(h, p.n))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        B.bm_edm_set_factor(h, Vh.shape[1], Vh)
        cycle()
        Vh = np.ascontiguousarray(B.bm_edm_get_factor(h, p.n))
    e2e_s = (time.perf_counter() - t0) / args.steps
    B.bm_edm_destroy(h)

    pairs = p.npairs
    ld = max(4, (k_now + 3) // 4 * 4)
    q = 2 * (k_max + 1)
    peaks, kind = _load_peaks()
    modeled = {nm: v for nm, v in prof.items() if edm_solve_bytes(nm, p.n, pairs, ld, q) is not None}
    top = max(modeled.items(), key=lambda kv: kv[1][1])[0] if modeled else None
    roof = None
    if top is not None:
        launches, tot = prof[top]
        by = edm_solve_bytes(top, p.n, pairs, ld, q if top != "edm_lap" else min(q, 128))
        avg = tot / max(1, launches)
        ach = by / (avg / 1e3) / 1e9
        traffic = None
        try:
            for line in open(os.path.join(ROOT, "profiles", "edm_pass_ls_chain30k_k16.txt")):
                if line.startswith(f"{top} dram_bytes_per_launch:"):
                    traffic = float(line.split(":", 1)[1].split()[0])
        except OSError:
            pass
        roof = {"bound": "hbm", "kernel": top, "achieved": ach, "peak": float(peaks["hbm_gbs"]), "unit": "GB/s",
                "frac": ach / float(peaks["hbm_gbs"]), "traffic": traffic, "peak_source": kind,
                "bytes_per_launch": by, "avg_launch_ms": avg,
                "note": "traffic: ncu DRAM bytes per launch (profiles/edm_pass_ls_chain30k_k16.txt)"}
    cpu = None
    if not args.no_cpu:
        from oracle import bm_oracle as O
        from oracle import edm_oracle as E
        i, j, d, w = E.pair_arrays(p.i, p.j, p.d, 1.0)
        alpha = 1.0 / E.lipschitz(p.n, i, j, w)
        V = Vh.astype(np.float64)
        st = E.EdmState(V=V, U=np.zeros((p.n, 0)), k_eig=min(k_max, V.shape[1] + 1))
        t0 = time.perf_counter()
        Vb, _ = E.bm_phase(st.V, i, j, d, w, lam, epochs)
        E.prox_step(E.EdmState(V=Vb, U=st.U, k_eig=st.k_eig), i, j, d, w, lam, alpha, k_max,
                    O.Options(lmsvd_tol=LMSVD_TOL))
        el = time.perf_counter() - t0
        cpu = {"value": 1.0 / el, "unit": "cycles/s", "cores": os.cpu_count(), "kind": "oracle",
               "sample": f"one cycle of the same workload from the GPU's last factor, {el:.1f} s"}
    return {
        "metric": "EDM Algorithm 1 cycles/s", "value": 1e3 / ms, "unit": "cycles/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"3-D self-avoiding chain, n = {p.n}, {pairs} pairs within 6.0, k_max = {k_max}",
                   "step": f"{epochs} BM iterations + 1 inexact PG step", "lambda": lam,
                   "l2": "problem fits in L2 (about 30 MB): cached between steps", "k_end": k_now,
                   "init_s": init_s, "F": [F_hist[0], F_hist[-1]],
                   "lmsvd_iters": [x["lmsvd_iters"] for x in infos], "ranks": [x["rank"] for x in infos]},
        "e2e": {"value": 1.0 / e2e_s, "unit": "cycles/s", "h2d_bytes_per_step": int(Vh.nbytes),
                "d2h_bytes_per_step": int(Vh.nbytes)},
        "gpu_launches": int(sum(v[0] for v in prof.values())),
        "kernels": {kname: {"launches": v[0], "ms": round(v[1], 4)} for kname, v in sorted(prof.items())},
        "roofline": roof,
        "gradient_call": grad_call,
        "secondary": extra or None,
        "cpu_baseline": cpu,
        "clocks": clocks,
    }


def run_bcd(args):
    """Column-block coordinate descent (the polyMF-SS form of the BM phase)
    against the full-gradient PR+ BM phase on the netflix-shaped workload, k =
    64, from the same factors: time per epoch (one sweep over the k column
    blocks, resp. one PR+ iteration) and the objective after each epoch."""
    import torch

    import paper_2204_14067_gb300 as B
    from synth import named_config, random_factors

    p = named_config(args.config)
    k = min(K_BENCH, p.k_max)
    W0, H0 = random_factors(p.m, p.n, k, seed=11, scale=0.1)
    out = {}
    for solver in ("pr_cg", "column_blocks"):
        opt = B.bm_default_options()
        opt.value_codec = args.codec
        opt.tensor_grams = args.tensor_grams
        h = B.bm_create(p.m, p.n, p.rows, p.cols, p.vals, p.lam, p.k_max, opt)
        stream = torch.cuda.Stream()
        B.bm_set_stream(h, stream)
        B.bm_set_factors(h, k, W0, H0)
        step = (lambda: B.bm_bcd_phase(h, 1)) if solver == "column_blocks" else (lambda: B.bm_bm_phase(h, 1))
        F = [B.bm_loss_grad(h)[1]]
        for _ in range(args.warmup):
            F.append(step())
        B.bm_profile_enable(h, True)
        torch.cuda.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ev0.record(stream)
        for _ in range(args.steps):
            F.append(step())
        ev1.record(stream)
        torch.cuda.synchronize()
        prof = B.bm_profile_read(h)
        B.bm_profile_enable(h, False)
        B.bm_destroy(h)
        out[solver] = {"ms_per_epoch": ev0.elapsed_time(ev1) / args.steps, "F": F,
                       "kernels": {kk: {"launches": v[0], "ms": round(v[1], 3)} for kk, v in sorted(prof.items())}}
    ms = out["column_blocks"]["ms_per_epoch"]
    # dominant kernel: the residual update fused with the next block's gradient,
    # 12 B per entry (index, residual read and write); the six column vectors it
    # reads are L2-resident
    kb = out["column_blocks"]["kernels"].get("bcd_update_spmv")
    roof = None
    if kb:
        peaks, kind = _load_peaks()
        by = p.nnz * 12
        avg = kb["ms"] / max(1, kb["launches"])
        ach = by / (avg / 1e3) / 1e9
        roof = {"bound": "hbm", "kernel": "bcd_update_spmv", "achieved": ach, "peak": float(peaks["hbm_gbs"]),
                "unit": "GB/s", "frac": ach / float(peaks["hbm_gbs"]), "traffic": None, "peak_source": kind,
                "bytes_per_launch": by, "avg_launch_ms": avg}
    return {
        "metric": "column-block BM sweep nnz/s", "value": p.nnz / (ms / 1e3), "unit": "nnz/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.config}-shaped, nnz={p.nnz}, k={k}, lambda={p.lam}",
                   "step": "one sweep over the k column blocks (column_blocks) / one PR+ iteration (pr_cg)"},
        "column_blocks": out["column_blocks"], "pr_cg": out["pr_cg"], "roofline": roof,
    }


def _dist_cpu():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    return None, int(os.environ.get("RANK", "0")), ws


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--mode", default="grad", choices=["cycle", "grad", "tto", "serve", "edm", "edm_solve", "bcd"])
    ap.add_argument("--precision", type=int, default=0, choices=[0, 1],
                    help="1: BF16 copies of the gathered factor rows (cycle and grad modes)")
    ap.add_argument("--serve-count", type=int, default=24)
    ap.add_argument("--serve-max-nnz", type=int, default=1_000_000,
                    help="cap on a serving request's entries (0: none, the stream's own sizes up to about 80M)")
    ap.add_argument("--k", type=int, default=0, help="factor rank (default 64; at most the workload's cap)")
    ap.add_argument("--lmsvd-tol", type=float, default=None,
                    help="LmSVD stop tolerance (cycle and tto modes; default: the library's)")
    ap.add_argument("--codec", type=int, default=1, choices=[0, 1],
                    help="1: one-byte codes for integer observed values in the loss/gradient passes")
    ap.add_argument("--step-rule", type=int, default=0, choices=[0, 1],
                    help="tto mode: 0 fixed PG step, 1 SpaRSA step rule")
    ap.add_argument("--config", default=WORKLOAD)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-tune", action="store_true", help="keep the natural work split (one panel)")
    ap.add_argument("--tensor-grams", type=int, default=1, choices=[0, 1],
                    help="plain Grams of the PG step on the tensor cores (1) or the FP32 pipes (0)")
    ap.add_argument("--no-extra", action="store_true",
                    help="grad mode: skip the secondary figures (cycle, time to oracle, serving sample)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        line = run_reference(args)
    elif args.mode == "tto":
        line = run_tto(args)
    elif args.mode == "serve":
        line = run_serve(args)
    elif args.mode == "edm":
        line = run_edm(args)
    elif args.mode == "edm_solve":
        line = run_edm_solve(args)
    elif args.mode == "bcd":
        line = run_bcd(args)
    else:
        line = run_ours(args)
    if line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
