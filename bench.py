#!/usr/bin/env python3
"""Converged plans/s of batched ADMM planning on one B300 (and N replicas).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--workload cfg0|cfg1|cfg2|cfg3]
    python bench.py --impl reference ...     # the FP64 CPU oracle on host cores

A step is one solve of the whole hot path over one batch of weightings: K
weightings of the 9x9 (cfg1) or 21x21 (cfg2) slider grid, iterated on the
device until every column meets the residual tolerance (1e-4), with the case
(A, S^{-1}) resident.  `value` = converged plans / device time of the timed
steps.  `e2e` times the whole C-ABI round trip per step from pinned host
buffers: create_case (phi host->device, assembly, scaling, S, Cholesky,
inverse), the solve, and fetch_times (device->host).

The workload is synthetic (seeded generator `synth.cases`): the paper's patient
cases are not public.  Multi-GPU runs are independent replicas (one case per
rank, no data-path collective): weak scaling.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOADS = {"cfg0": 0, "cfg1": 1, "cfg2": 2, "cfg3": 3}
METRIC = "converged plans/s (81 & 441 weightings) vs plain FP32 form; p50/p99 latency"
PAPER_ITERS = 3000          # fixed iterations per pass in the paper (Sec. 3.D)
RHO0_PER_BETA = 1.1e3       # Eq. rho_rule constant per unit of beta (re-tuned, Sec. 3.C)
PRECISIONS = {"bf16": 1, "bf16x3": 2}     # lgk PREC_* of the BF16 forms
PRECISION_NOTE = {
    "bf16": "A as 1 bf16 term (solves the LP of the rounded A), iterates 2 bf16 terms",
    "bf16x3": ("A as 2 bf16 terms, iterates 2 bf16 terms (3 products per GEMM); S^-1 and solve "
               "input 3 bf16 terms (6 products); fp32 accumulate")}


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return p["hbm_gbs"], p["bf16_tflops"], p["bf16_tflops_sustained"], "measured"
    except (OSError, KeyError, ValueError):
        return 6400.0, 1800.0, 1400.0, "fallback"


# bytes per entry of A each GEMM streams, per precision form
A_BYTES = {"bf16": 2, "bf16x3": 4}
# BF16 products per algorithmic product in the two A GEMMs, per form
GEMM_TERMS = {"bf16": 2, "bf16x3": 3}


def kernel_work(name, m, n, K, form="bf16x3", refine=False):
    """Work of one launch of an iteration kernel: (algorithmic bytes,
    algorithmic flops, executed tensor flops, executed bytes).

    Algorithmic = the per-unit figures of the method with A and the iterates
    entering the GEMMs as one BF16 term each (A read once per GEMM: 2mn
    bytes; iterates 2 bytes, FP32 state 4 bytes; the solve's operator as one
    FP32 m x m matrix).  Executed = what the chosen form moves and multiplies:
    A as 2 BF16 terms (4 bytes per entry) or 1 (2 bytes), the iterates as two
    BF16 terms, S^{-1} and the solve input as three."""
    a_exec, t = A_BYTES[form], GEMM_TERMS[form]
    if refine:               # light iterations: the high BF16 term of A, 2 products
        a_exec, t = 2, 2
    if name == "gemm1_lo":   # lo . R1_hi -> c1 (FP32), full iterations only; no algorithmic work
        return 0, 0, 2 * m * n * K, 2 * m * n + 2 * n * K + 4 * m * K
    if name == "gemm2_lo":   # lo^T . V_hi -> c2 (FP32)
        return 0, 0, 2 * m * n * K, 2 * m * n + 2 * m * K + 4 * n * K
    if name == "gemm1":      # A . R1 -> rhs (partial slots)
        return (2 * m * n + 2 * n * K + 4 * m * K, 2 * m * n * K, t * 2 * m * n * K,
                a_exec * m * n + 4 * n * K + 4 * m * K)
    if name == "solve":      # S^{-1} . rhs -> v (partial slots)
        return (4 * m * m + 4 * m * K + 4 * m * K, 2 * m * m * K, 6 * 2 * m * m * K,
                6 * m * m + 6 * m * K + 4 * m * K)
    if name == "gemm2":      # A^T . V, q1 read / write, R1 out
        return (2 * m * n + 2 * m * K + 10 * n * K, 2 * m * n * K, t * 2 * m * n * K,
                a_exec * m * n + 4 * m * K + 12 * n * K + (4 * n * K if refine else 0))
    if name in ("reduce_rhs", "reduce_solve"):
        return 16 * m * K, 0, 0, 16 * m * K
    if name == "q1_update":  # partial sums in, q1 r/w, R1 hi/lo out
        return 16 * n * K, 0, 0, 16 * n * K
    return 0, 0, 0, 0


class Clocks:
    """nvidia-smi samples (200 ms) during the timed region."""

    def __init__(self, idx):
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={idx}", f"--query-gpu={q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        self.p.wait()
        self.f.seek(0)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return rank, world, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allreduce_max(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def allreduce_sum(x, world):
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64,
                     device="cuda" if dist.get_backend() == "nccl" else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def knobs(args):
    """lgk_params fields the command line sets for every BF16 case."""
    return dict(solve_refine=args.solve_refine, setup_fp64=int(args.setup_fp64), rho_adapt=int(args.rho_adapt),
                l2_keep_inverse=int(args.l2_keep_inverse), gemm2_tile_rows=args.gemm2_rows)


def passes(st, ck, tol):
    if ck is None:                         # --no-check: the residual test alone
        return np.asarray(st["converged"], dtype=bool)
    return _passes(st, ck, tol)


def _passes(st, ck, tol):
    """Plans counted as converged: the device's residual test passed (relative
    residuals <= tol, FP32 partial sums) and the plan check confirms it on the
    LP itself: ||(A z1 - b)_+|| <= 2 tol (1 + ||A||_2) ||z|| (lgk_fetch_check's
    primal field).  A stop at residual tol bounds the left side by
    tol (1 + ||A||_2) max(||x||, ||z||) plus the x-step solve's own error
    ||rhs - S v||; the factor 2 allows that error up to the same size, while
    a stop reached with an inexact solve (the 9-target case without
    refinement: 1e-2 and above) fails."""
    return np.asarray(st["converged"], dtype=bool) & (ck["primal"] <= 2.0 * tol)


def make_inputs(cfg):
    from synth import cases as SC
    case = SC.workload_case(cfg)
    W = SC.slider_weights(SC.WORKLOADS[cfg]["grid"])
    return case, W


def oracle_iters(workload):
    """Mean iterations per plan of the FP64 oracle ADMM at tol 1e-4 on this
    workload, as recorded by tests/golden/make_oracle_iters.py (oracle only),
    or None if not recorded."""
    try:
        with open(os.path.join(ROOT, "tests", "golden", "oracle_iters.json")) as f:
            e = json.load(f)[workload]
        return float(e["mean_iters"]), e["sample"]
    except (OSError, KeyError, ValueError):
        return None


def iteration_basis(workload):
    """Iterations per plan by which both CPU figures extrapolate one timed
    oracle iteration: the oracle's own recorded mean, else the paper's fixed
    count (Sec. 3.D)."""
    rec = oracle_iters(workload)
    if rec:
        return rec[0], (f"the FP64 oracle's own mean of {rec[0]:.0f} iterations per plan at "
                        f"tol 1e-4 ({rec[1]}; tests/golden/oracle_iters.json)")
    return float(PAPER_ITERS), f"the paper's fixed {PAPER_ITERS} iterations (Sec. 3.D)"


def oracle_sample(case, W, iters_to_converge, basis, budget_s=30.0):
    """Time the FP64 oracle ADMM (as it stands) on the host cores: a bounded
    number of iterations over all K columns; per-iteration time is the
    difference to a zero-iteration run (which still forms and factors S)."""
    from oracle import admm as AD
    from oracle import lp as L
    from synth import cases as SC
    lp = L.precondition(L.assemble_case(case))
    b, l, u = L.bounds(lp, W)
    rho = L.rho_rule(W[:, 3], SC.W0_BOT, L.rho0_for(lp))
    t0 = time.perf_counter()
    AD.admm(lp.A, lp.c, b, l, u, rho, max_iter=0)
    t_setup = time.perf_counter() - t0
    n_it = 2
    t0 = time.perf_counter()
    AD.admm(lp.A, lp.c, b, l, u, rho, max_iter=n_it)
    t_run = time.perf_counter() - t0
    t_iter = max((t_run - t_setup) / n_it, 1e-9)
    K = W.shape[0]
    cores = len(os.sched_getaffinity(0))
    return dict(value=K / (t_iter * iters_to_converge), unit="plans/s", cores=cores,
                kind="oracle",
                sample=(f"FP64 oracle ADMM (numpy/LAPACK) on {case.name}, all {K} weightings, "
                        f"{n_it} iterations timed after S formation+Cholesky ({t_setup:.1f} s, "
                        f"excluded like the device's case set-up); {t_iter * 1e3:.1f} ms/iteration "
                        f"extrapolated to {basis}"))


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    cfg = WORKLOADS[args.workload]
    case, W = make_inputs(cfg)
    K = W.shape[0]
    from oracle import admm as AD
    from oracle import lp as L
    from synth import cases as SC
    lp = L.precondition(L.assemble_case(case))
    b, l, u = L.bounds(lp, W)
    rho = L.rho_rule(W[:, 3], SC.W0_BOT, L.rho0_for(lp))
    t0 = time.perf_counter()
    AD.admm(lp.A, lp.c, b, l, u, rho, max_iter=0)
    t_setup = time.perf_counter() - t0
    times = []
    for s in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        AD.admm(lp.A, lp.c, b, l, u, rho, max_iter=1)
        dt = time.perf_counter() - t0 - t_setup
        if s >= args.warmup:
            times.append(max(dt, 1e-9))
    t_iter = statistics.median(times)
    n_iters, basis = iteration_basis(args.workload)
    value = K / (t_iter * n_iters)
    cores = len(os.sched_getaffinity(0))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "plans/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": t_iter * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": workload_config(case, W, args),
            "cpu_baseline": {"value": value, "unit": "plans/s", "cores": cores, "kind": "oracle",
                             "sample": (f"one FP64 oracle ADMM iteration over all {K} weightings "
                                        f"per step (S formation+Cholesky, {t_setup:.1f} s, "
                                        f"subtracted), extrapolated to {basis}")},
            "e2e": {"value": value, "unit": "plans/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def workload_config(case, W, args):
    m, n = 25 * case.n_iso, case.n_pts + 8 * case.n_iso
    return {"workload": f"{case.name} (A {m}x{n}, K={W.shape[0]} weightings, tol {args.tol:g})",
            "m": m, "n": n, "K": int(W.shape[0]), "tol": args.tol,
            "precision": PRECISION_NOTE[args.precision] + (
                "; between residual tests (every 10 iterations) the heavy products use A's high term "
                "and add the low term's products from the last test iteration (lo_refresh)"
                if args.precision == "bf16x3" and not args.exact else ""),
            "solve_refine": args.solve_refine, "rho_adapt": bool(args.rho_adapt),
            "l2_keep_inverse": bool(args.l2_keep_inverse), "gemm2_tile_rows": args.gemm2_rows,
            "schur": "S = I + A A^T on " + ("FP64 CUDA cores" if args.setup_fp64 else "tensor cores (BF16 "
                                             "products, FP32 chunk sums, FP64 across chunks)"),
            "rho": "Eq. rho_rule, rho0 = 1100 beta", "l2": "inputs larger than L2 (A resident, "
            f"{A_BYTES[args.precision] * m * n / 1e6:.0f} MB > 126 MB)", "parallelism": "replicas"}


def kernel_hash():
    h = hashlib.sha256()
    for f in ("tc_gemm.cu", "tc_ptx.cuh", "iter_ctx.cuh", "iter.cu"):
        with open(os.path.join(ROOT, "paper_2509_08602_b300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def committed_traffic(kernel, workload, k_launch):
    """DRAM bytes per launch from a committed ncu summary of the same workload
    and launch width, if the kernel source is unchanged since it was taken."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        e = t[f"{workload}_k{k_launch}"][kernel]
        return e["bytes_per_launch"] if e.get("source_hash") == kernel_hash() else None
    except (OSError, KeyError, ValueError):
        return None


def run_ours(args, rank, world, local):
    import torch
    from paper_2509_08602_b300 import build
    if rank == 0:
        build.build()
    barrier(world)
    torch.cuda.set_device(local)
    from paper_2509_08602_b300 import lgk
    cfg = WORKLOADS[args.workload]
    case, W = make_inputs(cfg)
    K = W.shape[0]
    prec = PRECISIONS[args.precision]
    refine = args.precision == "bf16x3" and not args.exact
    # the timed solves run without per-kernel events (those split the
    # iteration graph and stop consecutive kernels from overlapping); the
    # per-kernel durations come from a profiled solve of the same batch
    params = lgk.default_params(precision=prec, device=local, profile=0, lo_refresh=int(refine),
                                check_every=args.check_every, **knobs(args))
    from synth import cases as SC
    cs = lgk.create_case(case.phi, case.kind, case.struct_id, case.n_iso, case.d_presc,
                         case.q_area, case.q_vol, case.d_ld1, case.d_ld2, case.phi_cal,
                         params=params)
    rule = dict(w0_bot=SC.W0_BOT, rho0=RHO0_PER_BETA * cs.beta, tol=args.tol,
                max_iter=args.max_iter)
    sw = args.stream_width
    if sw:
        # streaming: the slowest weightings (lowest BOT weight) enter first
        W = W[np.argsort(W[:, 3], kind="stable")]
    k_launch = min(sw, K) if sw else K         # columns one GEMM launch carries
    for _ in range(args.warmup):
        if sw:
            lgk.solve_stream(cs, W, None, width=sw, **rule)
        else:
            lgk.solve_weightings(cs, W, None, **rule).close()
    lgk.launch_count()
    barrier(world)
    torch.cuda.synchronize()
    clocks = Clocks(local)
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    prof = {k: [0.0, 0] for k in lgk.KERNELS}
    conv = 0
    iters = []
    lat = []
    ev0.record()
    t_host0 = time.perf_counter()
    r_last = None
    checks = []
    conv_flag = 0
    for _ in range(args.steps):
        t1 = time.perf_counter()
        if sw:
            st = lgk.solve_stream(cs, W, None, width=sw, check=not args.no_check, **rule)
            ck = st.get("check")
            lat.append(time.perf_counter() - t1)
        else:
            r = lgk.solve_weightings(cs, W, None, **rule)
            st = lgk.fetch_stats(r)
            ck = None if args.no_check else lgk.fetch_check(r)
            lat.append(time.perf_counter() - t1)
            if r_last is not None:
                r_last.close()
            r_last = r
        conv += int(passes(st, ck, args.tol).sum())
        conv_flag += int(np.asarray(st["converged"]).sum())
        iters.append(st["iters"])
        if ck is not None:
            checks.append(ck)
    ev1.record()
    torch.cuda.synchronize()
    barrier(world)
    launches = lgk.launch_count()
    clk = clocks.stop()
    host_s = time.perf_counter() - t_host0
    dev_s = ev0.elapsed_time(ev1) / 1e3
    # the library solves on its own stream; the host-blocking solve brackets it
    step_s = max(dev_s, host_s)
    t_max = allreduce_max(step_s, world)
    conv_all = allreduce_sum(conv, world)
    value = conv_all / t_max
    mean_iters = float(np.mean(np.concatenate(iters)))
    max_iters = int(max(int(i.max()) for i in iters))

    # per-kernel CUDA-event durations: one profiled solve of the same batch
    cs_p = lgk.create_case(case.phi, case.kind, case.struct_id, case.n_iso, case.d_presc,
                           case.q_area, case.q_vol, case.d_ld1, case.d_ld2, case.phi_cal,
                           params=lgk.default_params(precision=prec, device=local, profile=1,
                                                     lo_refresh=int(refine), check_every=args.check_every,
                                                     **knobs(args)))
    if sw:
        pr = lgk.solve_stream(cs_p, W, None, width=sw, profile=True, **rule)["profile"]
        prof_iters = pr["gemm1"][1]          # iterations of the whole stream (one GEMM1 each)
    else:
        r = lgk.solve_weightings(cs_p, W, None, **rule)
        pr = lgk.fetch_profile(r)
        prof_iters = int(lgk.fetch_stats(r)["iters"].max())
        r.close()
    for k, (ms, nl) in pr.items():
        prof[k][0] += ms
        prof[k][1] += nl
    cs_p.close()

    # e2e: pinned host inputs, create + solve + fetch per step
    phi_pinned = torch.empty(case.phi.shape, dtype=torch.float64, pin_memory=True).numpy()
    phi_pinned[...] = case.phi
    e2e_steps = max(1, min(args.steps, 3))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    conv_e2e = 0
    for _ in range(e2e_steps):
        c2 = lgk.create_case(phi_pinned, case.kind, case.struct_id, case.n_iso, case.d_presc,
                             case.q_area, case.q_vol, case.d_ld1, case.d_ld2, case.phi_cal,
                             params=lgk.default_params(precision=prec, device=local,
                                                       lo_refresh=int(refine),
                                                       check_every=args.check_every, **knobs(args)))
        if sw:
            s2 = lgk.solve_stream(c2, W, None, width=sw, check=True, **rule)
            t, tau = s2["t"], s2["tau"]
            conv_e2e += int(passes(s2, s2["check"], args.tol).sum())
        else:
            r = lgk.solve_weightings(c2, W, None, **rule)
            t, tau = lgk.fetch_times(r)
            conv_e2e += int(passes(lgk.fetch_stats(r), lgk.fetch_check(r), args.tol).sum())
            r.close()
        c2.close()
    torch.cuda.synchronize()
    e2e_s = allreduce_max(time.perf_counter() - t0, world)
    e2e_value = allreduce_sum(conv_e2e, world) / e2e_s
    h2d = case.phi.nbytes + case.kind.nbytes + case.struct_id.nbytes + W.nbytes
    d2h = t.nbytes + tau.nbytes

    out = None
    if rank == 0:
        # plain FP32 GPU form, same workload and tolerance (comparison form)
        fp32 = None
        if not args.no_fp32:
            c3 = lgk.create_case(case.phi, case.kind, case.struct_id, case.n_iso, case.d_presc,
                                 case.q_area, case.q_vol, case.d_ld1, case.d_ld2, case.phi_cal,
                                 params=lgk.default_params(precision=lgk.PREC_FP32, device=local))
            fp32 = fp32_form(lgk, c3, W, rule, sw, args.tol)
            fp32["ratio_over_fp32"] = (value / world) / fp32["value"] if fp32["value"] else None
            fp32["max_iter"] = args.max_iter
            c3.close()
        hbm, tf_burst, tf_sus, src = peaks()
        m, n = 25 * case.n_iso, case.n_pts + 8 * case.n_iso
        dom = max(prof, key=lambda k: prof[k][0])
        ms_avg = prof[dom][0] / max(prof[dom][1], 1)
        nbytes, flops, executed, xbytes = kernel_work(dom, m, n, k_launch, args.precision, refine)
        t_hbm = xbytes / (hbm * 1e9)
        t_tensor = executed / (tf_sus * 1e12)
        if t_hbm >= t_tensor:
            achieved = nbytes / (ms_avg / 1e3) / 1e9
            roof = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s"}
        else:
            achieved = flops / (ms_avg / 1e3) / 1e12
            roof = {"bound": "tensor", "achieved": achieved, "peak": tf_sus, "unit": "TFLOP/s",
                    "note": ("achieved counts algorithmic flops (2mnK); the kernel executes "
                             f"{executed / flops:.0f} BF16 products per algorithmic one")}
        roof["frac"] = roof["achieved"] / roof["peak"]
        roof["executed_tensor_frac"] = executed / (ms_avg / 1e3) / (tf_sus * 1e12)
        roof["executed_bytes_per_launch"] = xbytes
        roof["executed_hbm_frac"] = xbytes / (ms_avg / 1e3) / (hbm * 1e9)
        roof["traffic"] = committed_traffic(dom, args.workload, k_launch)
        roof["kernel"] = dom
        roof["peak_source"] = (f"{src} (MEASURED_PEAKS.json; hbm_gbs, bf16_tflops_sustained)"
                               if src == "measured" else "fallback")
        roof["algorithmic_bytes_per_launch"] = nbytes
        roof["algorithmic_flops_per_launch"] = flops
        roof["avg_launch_ms"] = ms_avg
        total_ms = sum(v[0] for v in prof.values())
        roof["kernel_share"] = {k: round(v[0] / total_ms, 4) for k, v in prof.items()}
        roof["timing"] = (f"CUDA events around every kernel of one profiled solve of the same workload "
                          f"and batching ({prof_iters} iterations); the timed steps run without them")
        # iterations per step: the batch runs until its slowest column stops;
        # a stream's count is that of its profiled run (the same schedule)
        roof["us_per_iteration_timed"] = t_max / args.steps / (prof_iters if sw else max_iters) * 1e6
        roof["us_per_iteration_profiled"] = total_ms / prof_iters * 1e3
        cpu = None
        if not args.no_cpu_baseline:
            n_iters, basis = iteration_basis(args.workload)
            cpu = oracle_sample(case, W, n_iters, basis)
        if not args.no_extras and r_last is None:     # streaming: one batch solve for the extras
            r_last = lgk.solve_weightings(cs, W, None, **rule)
        # the measurements beside the main line: a failure in one is recorded
        # in its key and does not take the main line down with it
        extra = {}

        def leg(name, fn):
            try:
                extra[name] = fn()
            except Exception as e:          # noqa: BLE001 (reported in the line)
                extra[name] = {"error": f"{type(e).__name__}: {e}"[:400]}

        if not args.no_extras:
            leg("plan_metrics", lambda: bench_metrics(lgk, case, r_last))
            leg("two_pass", lambda: bench_two_pass(lgk, case, W, args, local))
        if not args.no_k441 and args.workload == "cfg1":
            leg("k441", lambda: bench_k441(lgk, args, local))
        if not args.no_group and args.workload == "cfg1":
            leg("group", lambda: bench_group(lgk, args, local, with_cfg3=args.group_cfg3))
        if not args.no_serve and args.workload == "cfg1":
            def serving():
                sv = serve_run(lgk, args, local, n_cases=24, rate=1.0, workers=2)
                sv["note"] = ("a short stream of the serving workload (bench.py --serve N sweeps the "
                              "arrival rate); latency = submit to results")
                return sv
            leg("serving", serving)
        lat_ms = sorted(x * 1e3 for x in lat)
        out = {"metric": METRIC, "value": value, "unit": "plans/s", "n_gpus": world,
               "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max / args.steps * 1e3,
               "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
               "dtype": "bf16", "data": "synthetic (seeded generator; paper cases are not public)",
               "config": workload_config(case, W, args),
               "e2e": {"value": e2e_value, "unit": "plans/s", "h2d_bytes_per_step": int(h2d),
                       "d2h_bytes_per_step": int(d2h),
                       "note": "create_case from pinned host phi + solve + fetch_times"},
               "batching": (f"stream: {K} weightings through {sw} columns, each column refilled "
                            "with the next weighting (ascending w_BOT) when it stops" if sw else
                            f"one batch of {K} columns, run until every column stops"),
               "gpu_launches": int(launches),
               "clocks": clk, "roofline": roof, "cpu_baseline": cpu,
               "latency_ms": {"p50": lat_ms[len(lat_ms) // 2],
                              "p99": lat_ms[min(len(lat_ms) - 1, int(0.99 * len(lat_ms)))]},
               "mean_iters_per_plan": mean_iters, "max_iters": max_iters,
               "converged_fraction": conv / (K * args.steps),
               "residual_test_fraction": conv_flag / (K * args.steps),
               "fp64_check": check_summary(checks) if checks else None,
               "fp32_form": fp32, **extra}
        print(json.dumps(out), flush=True)
    if r_last is not None:
        r_last.close()
    cs.close()
    return 0


def bench_k441(lgk, args, local, width=128, steps=2, fp32_max_iter=4000):
    """The 441-weighting half of the metric: the 4-target 5000 x 61600 case,
    its 21 x 21 slider grid streamed through `width` columns (lowest w_BOT
    first), one untimed and `steps` timed streams on the device (case
    resident), plans counted with the FP64 check; e2e = create_case from
    pinned host phi + stream + times; and the plain FP32 form through the same
    width, bounded at fp32_max_iter iterations per weighting (it stalls above
    tol at this size)."""
    import torch
    from synth import cases as SC
    case, W = make_inputs(2)
    W = W[np.argsort(W[:, 3], kind="stable")]
    K = W.shape[0]
    prec = PRECISIONS[args.precision]
    refine = args.precision == "bf16x3" and not args.exact
    # the precision form of this case refines the x-update's solve (one step
    # per iteration): without it the explicit-inverse solve's error leaves
    # most plans' FP64 primal check above 2 tol although their residual
    # test passes
    kn = dict(knobs(args), solve_refine=max(1, args.solve_refine))
    params = lgk.default_params(precision=prec, device=local, lo_refresh=int(refine),
                                check_every=args.check_every, **kn)
    cs = lgk.create_case(case.phi, case.kind, case.struct_id, case.n_iso, case.d_presc, case.q_area,
                         case.q_vol, case.d_ld1, case.d_ld2, case.phi_cal, params=params)
    rule = dict(w0_bot=SC.W0_BOT, rho0=RHO0_PER_BETA * cs.beta, tol=args.tol, max_iter=args.max_iter)
    lgk.solve_stream(cs, W, None, width=width, **rule)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    conv, conv_flag, its, cks = 0, 0, [], []
    for _ in range(steps):
        st = lgk.solve_stream(cs, W, None, width=width, check=True, **rule)
        conv += int(passes(st, st["check"], args.tol).sum())
        conv_flag += int(np.asarray(st["converged"]).sum())
        its.append(st["iters"])
        cks.append(st["check"])
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / steps
    cs.close()
    phi_pinned = torch.empty(case.phi.shape, dtype=torch.float64, pin_memory=True).numpy()
    phi_pinned[...] = case.phi
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    c2 = lgk.create_case(phi_pinned, case.kind, case.struct_id, case.n_iso, case.d_presc, case.q_area,
                         case.q_vol, case.d_ld1, case.d_ld2, case.phi_cal, params=params)
    s2 = lgk.solve_stream(c2, W, None, width=width, check=True, **rule)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    conv_e2e = int(passes(s2, s2["check"], args.tol).sum())
    c2.close()
    fp32 = None
    if not args.no_fp32:
        c3 = lgk.create_case(case.phi, case.kind, case.struct_id, case.n_iso, case.d_presc,
                             case.q_area, case.q_vol, case.d_ld1, case.d_ld2, case.phi_cal,
                             params=lgk.default_params(precision=lgk.PREC_FP32, device=local))
        rule32 = dict(rule, max_iter=fp32_max_iter)
        t0 = time.perf_counter()
        s3 = lgk.solve_stream(c3, W, None, width=width, check=True, **rule32)
        d3 = time.perf_counter() - t0
        n3 = int(passes(s3, s3["check"], args.tol).sum())
        fp32 = {"value": n3 / d3, "unit": "plans/s", "converged": n3, "K": K,
                "max_iter": fp32_max_iter, "seconds": d3,
                "median_rel_pri": float(np.median(s3["rel_pri"])),
                "median_rel_dual": float(np.median(s3["rel_dual"])),
                "ratio_over_fp32": (conv / steps / dt) / (n3 / d3) if n3 else None}
        c3.close()
    it = np.concatenate(its)
    m, n = 25 * case.n_iso, case.n_pts + 8 * case.n_iso
    return {"workload": f"{case.name} (A {m}x{n}, K={K} weightings, tol {args.tol:g})",
            "value": conv / steps / dt, "unit": "plans/s", "converged": conv / steps, "K": K,
            "residual_test_passed": conv_flag / steps,
            "s_per_step": dt, "steps": steps, "batching": f"stream through {width} columns",
            "solve_refine": kn["solve_refine"],
            "mean_iters_per_plan": float(it.mean()), "max_iters": int(it.max()),
            "fp64_check": check_summary(cks),
            "e2e": {"value": conv_e2e / e2e_s, "unit": "plans/s", "seconds": e2e_s,
                    "h2d_bytes_per_step": int(case.phi.nbytes + case.kind.nbytes
                                              + case.struct_id.nbytes + W.nbytes),
                    "d2h_bytes_per_step": int(s2["t"].nbytes + s2["tau"].nbytes)},
            "fp32_form": fp32}


def bench_group(lgk, args, local, with_cfg3=False):
    """Co-scheduled cases (lgk_solve_group): the 3750 x 41200 case with its 81
    weightings and the 500 x 4660 sphere case with its 9 (and, with_cfg3, the
    9-target 8325 x 122664 case with its 441, all three refining the solve),
    each as one batch, every tensor-core product of an iteration one launch
    over all of them; against the same batches solved one after another.
    Plans are counted by the residual test and the FP64 check as in the main
    line; the group's plans equal the sequential ones bitwise (checked)."""
    import torch
    from synth import cases as SC
    cfgs = [1, 0] + ([3] if with_cfg3 else [])
    refine = args.precision == "bf16x3" and not args.exact
    kn = dict(knobs(args), refine_after=0)
    if with_cfg3:
        kn["solve_refine"] = max(1, args.solve_refine)
    prec = PRECISIONS[args.precision]
    cases, Ws, rho0 = [], [], []
    for c in cfgs:
        case, W = make_inputs(c)
        cs = lgk.create_case(case.phi, case.kind, case.struct_id, case.n_iso, case.d_presc, case.q_area,
                             case.q_vol, case.d_ld1, case.d_ld2, case.phi_cal,
                             params=lgk.default_params(precision=prec, device=local, lo_refresh=int(refine),
                                                       check_every=args.check_every, **kn))
        cases.append(cs)
        Ws.append(W)
        rho0.append(RHO0_PER_BETA * cs.beta)
    kw = dict(w0_bot=SC.W0_BOT, tol=args.tol, max_iter=args.max_iter)

    def counted(res):
        n = 0
        for r in res:
            n += int(passes(lgk.fetch_stats(r), lgk.fetch_check(r), args.tol).sum())
        return n

    for r in lgk.solve_group(cases, Ws, None, rho0=rho0, **kw):       # untimed: graphs, plans
        r.close()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    grp = lgk.solve_group(cases, Ws, None, rho0=rho0, **kw)
    torch.cuda.synchronize()
    t_group = time.perf_counter() - t0
    t0 = time.perf_counter()
    seq = [lgk.solve_weightings(c, W, None, rho0=r0, **kw) for c, W, r0 in zip(cases, Ws, rho0)]
    torch.cuda.synchronize()
    t_seq = time.perf_counter() - t0
    same = all(np.array_equal(lgk.fetch_stats(a)["obj"], lgk.fetch_stats(b)["obj"]) for a, b in zip(grp, seq))
    n_g, n_s = counted(grp), counted(seq)
    members = []
    for c, cs, W, r in zip(cfgs, cases, Ws, grp):
        st = lgk.fetch_stats(r)
        members.append({"case": f"{SC.WORKLOADS[c]['name']} (A {cs.m}x{cs.n})", "K": int(W.shape[0]),
                        "max_iters": int(st["iters"].max()), "mean_iters": float(st["iters"].mean())})
    for r in grp + seq:
        r.close()
    for cs in cases:
        cs.close()
    plans = sum(int(W.shape[0]) for W in Ws)
    return {"value": n_g / t_group, "unit": "plans/s", "plans": plans, "converged": n_g,
            "seconds": t_group, "sequential": {"value": n_s / t_seq, "seconds": t_seq, "converged": n_s},
            "speedup": t_seq / t_group, "bitwise_equal_to_sequential": bool(same), "members": members,
            "solve_refine": kn["solve_refine"],
            "note": "one batch per case; the group ends when its slowest member's slowest column stops"}


def check_summary(checks):
    """Worst values of the FP64 plan check over the timed steps."""
    ck = {k: np.concatenate([c[k] for c in checks]) for k in checks[0]}
    return {"max_primal": float(np.max(ck["primal"])), "max_abs_gap": float(np.max(np.abs(ck["gap"]))),
            "median_abs_gap": float(np.median(np.abs(ck["gap"]))), "max_infeas": float(np.max(ck["infeas"])),
            "max_hard": float(np.max(ck["hard"])), "max_bound": float(np.max(ck["bound"])),
            "note": "lgk_fetch_check per plan (FP64 A z1, A^T lam against the exact LP); a plan "
                    "counts as converged when its residual test passed and primal <= 2 tol; gap is "
                    "the FP64 duality gap of the plan (c^T z1 against the Sec. 2.A objective)"}


def fp32_form(lgk, c3, W, rule, sw, tol):
    """The plain FP32 GPU form (cuBLAS SGEMM, FP32 S^-1) on the same weightings
    and batching as the measured form (streamed through the same width, or one
    batch), so the ratio compares precision forms alone; one untimed run,
    then one timed.  Plans are counted as in the measured form."""
    def once():
        if sw:
            s3 = lgk.solve_stream(c3, W, None, width=sw, check=True, **rule)
            return s3, s3["check"]
        r = lgk.solve_weightings(c3, W, None, **rule)
        out = lgk.fetch_stats(r), lgk.fetch_check(r)
        r.close()
        return out
    once()
    t0 = time.perf_counter()
    s3, ck = once()
    dt = time.perf_counter() - t0
    n3 = int(passes(s3, ck, tol).sum())
    K = W.shape[0]
    return {"value": n3 / dt, "unit": "plans/s", "mean_iters": float(np.mean(s3["iters"])),
            "converged": n3, "K": K, "all_converged": n3 == K,
            "batching": f"stream through {sw} columns" if sw else f"one batch of {K}",
            "median_rel_pri": float(np.median(s3["rel_pri"])),
            "median_rel_dual": float(np.median(s3["rel_dual"]))}


def bench_metrics(lgk, case, res, reps=3):
    """Clinical metrics of all K plans on the device (lgk_fetch_metrics) on a
    2 mm evaluation grid over the targets' bounding box + 12 mm."""
    from synth import cases as SC
    pts, label, _ = SC.eval_grid(case, spacing=2.0, margin=12.0)
    phi_eval = SC.dose_rate(pts, case.iso)
    lgk.fetch_metrics(res, phi_eval, label)
    t0 = time.perf_counter()
    for _ in range(reps):
        met = lgk.fetch_metrics(res, phi_eval, label)
    dt = (time.perf_counter() - t0) / reps
    K, E, B = res.K, phi_eval.shape[0], phi_eval.shape[1]
    return {"ms_per_call": dt * 1e3, "ms_per_plan": dt * 1e3 / K, "n_eval": int(E), "K": int(K),
            "dose_fp64_gflops": 2.0 * K * E * B / dt / 1e9,
            "h2d_bytes": int(phi_eval.nbytes + label.nbytes),
            "coverage_range": [float(met["coverage"].min()), float(met["coverage"].max())],
            "bot_range": [float(met["bot"].min()), float(met["bot"].max())],
            "note": "FP64 doses phi_eval t (dominant), integer threshold counts, BOT; host phi_eval "
                    "uploaded inside each call"}


def bench_two_pass(lgk, case, W, args, local, reps=2, n_ld=1000, delta=(1.0, 0.5), seed=7):
    """Both passes of the two-pass optimisation (Sec. 2.C) through
    lgk_two_pass: pass-1 case + solve, low-dose volumes of all plans on the
    candidates (2 mm grid over the targets' box + 25 mm, outside the targets),
    Algorithm 1 (n_ld points per weighting and level), pass-2 case + masked
    solve.  Plus one run through the separate entry points for a breakdown."""
    from synth import cases as SC
    pts, label, _ = SC.eval_grid(case, spacing=2.0, margin=25.0)
    phi_cand = SC.dose_rate(pts[label < 0], case.iso)
    params = lgk.default_params(precision=PRECISIONS[args.precision], device=local,
                                lo_refresh=int(not args.exact), **knobs(args))
    kw = dict(phi_cand=phi_cand, delta_ld1=delta[0], delta_ld2=delta[1], n_ld1=n_ld, n_ld2=n_ld,
              seed=seed, w0_bot=SC.W0_BOT, rho0_per_beta=RHO0_PER_BETA, tol=args.tol,
              max_iter=args.max_iter, params=params)
    args_case = (case.phi, case.kind, case.struct_id, case.n_iso, case.d_presc, case.q_area,
                 case.q_vol, case.d_ld1, case.d_ld2, case.phi_cal, W)

    def once():
        r1, c2, r2, un = lgk.two_pass(*args_case, **kw)
        st = lgk.fetch_stats(r2)
        out = (int(st["converged"].sum()), int(st["iters"].max()), c2.n, [len(u) for u in un])
        r1.close(), r2.close(), c2.close()
        return out

    once()
    t0 = time.perf_counter()
    runs = [once() for _ in range(reps)]
    dt = (time.perf_counter() - t0) / reps
    conv = sum(r[0] for r in runs) / reps
    # breakdown through the separate entry points
    K = W.shape[0]
    tb = {}
    t = time.perf_counter()
    c1 = lgk.create_case(*args_case[:10], params=params)
    tb["setup1_s"] = time.perf_counter() - t
    t = time.perf_counter()
    r1 = lgk.solve_weightings(c1, W, None, w0_bot=SC.W0_BOT, rho0=RHO0_PER_BETA * c1.beta,
                              tol=args.tol, max_iter=args.max_iter)
    tb["solve1_s"] = time.perf_counter() - t
    t = time.perf_counter()
    member, count = lgk.low_dose_volumes(r1, phi_cand, (case.d_ld1, case.d_ld2), delta)
    tb["volumes_s"] = time.perf_counter() - t
    t = time.perf_counter()
    for l in range(2):
        lgk.sample_low_dose(member[l], [n_ld] * K, seed=seed, level=l)
    tb["sampling_s"] = time.perf_counter() - t
    r1.close(), c1.close()
    return {"value": conv / dt, "unit": "converged second-pass plans/s", "s_per_call": dt,
            "converged": conv, "K": K, "max_iters_pass2": runs[-1][1], "n_pass2": runs[-1][2],
            "union_points": runs[-1][3], "n_cand": int(phi_cand.shape[0]),
            "volume_sizes": [int(count.min()), int(count.max())], "breakdown": tb,
            "note": "end to end from host phi and candidates (both cases set up inside the call); "
                    "pass-2 case set-up and solve are the remainder of s_per_call"}


def serve_cases(n_req, seed=4000):
    """Serving workload: sizes log-uniform between the 8 mm sphere case
    (20 isocenters, 4500 points) and the 52 cm^3 ellipsoid case (150
    isocenters, 40000 points), 1 + floor(8u) targets, 81 or 441 weightings
    (p = 1/2); half of the cases get a follow-up request of 9 weightings (a
    3 x 3 slider refinement around the grid's centre) for the same case."""
    from synth import cases as SC
    rng = np.random.default_rng(seed)
    out = []
    for r in range(n_req):
        u = rng.uniform()
        n_iso = int(round(np.exp(np.log(20) + u * (np.log(150) - np.log(20)))))
        P = int(round(np.exp(np.log(4500) + u * (np.log(40000) - np.log(4500)))))
        nT = 1 + int(8 * rng.uniform())
        if nT == 1:
            targets = [(np.zeros(3), np.full(3, rng.uniform(6.0, 15.0)))]
        else:
            targets = SC._spheres(rng, nT, 3.0, 12.0, 60.0)
        n_t = int(0.3 * P)
        rest = P - n_t
        case = SC.make_case(targets, n_target_pts=n_t, n_ring=rest // 3, n_ld1=rest // 3,
                            n_ld2=rest - 2 * (rest // 3), n_iso=n_iso, seed=seed + 1 + r,
                            name=f"req{r}")
        grid = 9 if rng.uniform() < 0.5 else 21
        follow = None
        if rng.uniform() < 0.5:
            s = np.array([0.4, 0.5, 0.6])
            follow = np.array([(1.0, 1.0, a, SC.W0_BOT * 10.0 ** (3.0 * c)) for a in s for c in s])
        out.append((case, SC.slider_weights(grid), follow))
    return out


_SERVE_CACHE = {}


def serve_run(lgk, args, local, n_cases, rate, workers, width=32, seed=4000):
    """One Poisson stream of serving requests through lgk_server (continuous
    batching): every case is opened as a resident case with its initial
    request; a follow-up request for the same case arrives later in the
    stream and joins the case's running stream (or finds it resident and
    idle); a case is closed after its last request is submitted.  Returns
    throughput and latency figures."""
    import threading
    from synth import cases as SC
    key = (n_cases, seed)
    if key not in _SERVE_CACHE:                 # the same workload at every rate of a sweep
        _SERVE_CACHE[key] = serve_cases(n_cases + 3, seed=seed)
    reqs = _SERVE_CACHE[key]
    warm, reqs = reqs[:3], reqs[3:]
    srv = lgk.Server(workers=workers, tol=args.tol, max_iter=args.max_iter, w0_bot=SC.W0_BOT,
                     rho0_per_beta=RHO0_PER_BETA, stream_width=width,
                     params=lgk.default_params(device=local, **knobs(args)))

    def open_case(case):
        return srv.open(case.phi, case.kind, case.struct_id, case.n_iso, case.d_presc, case.q_area,
                        case.q_vol, case.d_ld1, case.d_ld2, case.phi_cal)

    # capacity from three cases served one at a time (untimed)
    service = []
    for case, W, _ in warm:
        t0 = time.perf_counter()
        cid = open_case(case)
        rid = srv.submit_to(cid, W)
        srv.close_case(cid)
        srv.wait(rid, case.n_iso, W.shape[0])
        service.append(time.perf_counter() - t0)
    cap = workers / float(np.mean(service))          # cases per second
    lam = rate * cap
    rng = np.random.default_rng(77)
    t_case = np.cumsum(rng.exponential(1.0 / lam, size=len(reqs)))
    events = []                                      # (time, kind, case index)
    for k, (case, W, follow) in enumerate(reqs):
        events.append((t_case[k], 0, k))
        if follow is not None:
            events.append((t_case[k] + rng.exponential(2.0 / lam), 1, k))
    events.sort()
    last = {}
    for e in events:
        last[e[2]] = e
    ids = []                                         # (request id, n_iso, K, kind)
    lock = threading.Lock()
    results = []
    cids = {}
    submitted = threading.Semaphore(0)

    def collector(n):
        for _ in range(n):
            submitted.acquire()
            with lock:
                rid, n_iso, K, kind = ids[len(results)]
            info = srv.wait(rid, n_iso, K)[0]
            with lock:
                results.append((kind, info))

    th = threading.Thread(target=collector, args=(len(events),))
    th.start()
    t0 = time.perf_counter()
    for ev in events:
        t_ev, kind, k = ev
        delay = t0 + t_ev - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        case, W, follow = reqs[k]
        if kind == 0:
            cids[k] = open_case(case)
        Wk = W if kind == 0 else follow
        rid = srv.submit_to(cids[k], Wk)
        if last[k] is ev:
            srv.close_case(cids[k])
        with lock:
            ids.append((rid, case.n_iso, Wk.shape[0], kind))
        submitted.release()
    th.join()
    makespan = time.perf_counter() - t0
    srv.close()
    lat = np.array([i["total_ms"] for _, i in results])
    lat_f = np.array([i["total_ms"] for kd, i in results if kd == 1])
    conv = sum(i["converged"] for _, i in results)
    n_plans = sum(i["K"] for _, i in results)
    return {"value": conv / makespan, "unit": "plans/s", "cases": len(reqs),
            "requests": len(results), "follow_ups": int(len(lat_f)), "workers": workers,
            "stream_width": width, "arrival_rate_cases_per_s": lam, "rate_vs_capacity": rate,
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99)),
                           "follow_up_p50": float(np.percentile(lat_f, 50)) if len(lat_f) else None,
                           "follow_up_p99": float(np.percentile(lat_f, 99)) if len(lat_f) else None,
                           "mean_queue": float(np.mean([i["queue_ms"] for _, i in results])),
                           "mean_setup": float(np.mean([i["setup_ms"] for _, i in results]))},
            "all_ok": all(i["status"] == 0 for _, i in results),
            "converged_fraction": conv / n_plans, "makespan_s": makespan}


def run_serve(args, rank, world, local):
    import torch
    from paper_2509_08602_b300 import build
    if rank == 0:
        build.build()
    barrier(world)
    torch.cuda.set_device(local)
    from paper_2509_08602_b300 import lgk
    rates = [float(x) for x in args.serve_rates.split(",")]
    sweep = [serve_run(lgk, args, local, args.serve, r, args.serve_workers) for r in rates]
    line = {"metric": "served converged plans/s; p50/p99 request latency",
            "value": max(x["value"] for x in sweep), "unit": "plans/s", "n_gpus": world,
            "sweep": sweep, "data": "synthetic", "dtype": "bf16",
            "config": {"workload": f"Poisson stream of {args.serve} cases (sizes log-uniform 500x4660 .. "
                                   "3750x41200, 1-8 targets, 81 or 441 weightings; half get a 9-weighting "
                                   "follow-up request for the same resident case)", "tol": args.tol,
                       "rates_vs_capacity": rates}}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="cfg1", choices=sorted(WORKLOADS))
    ap.add_argument("--tol", type=float, default=1e-4)
    ap.add_argument("--max-iter", type=int, default=20000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-fp32", action="store_true")
    ap.add_argument("--check-every", type=int, default=10,
                    help="iterations between residual tests (and low-term refreshes)")
    ap.add_argument("--exact", action="store_true",
                    help="both BF16 terms of A in every iteration (lo_refresh = 0)")
    ap.add_argument("--stream-width", type=int, default=32,
                    help="streaming solve: the workload's weightings through this many columns, "
                         "refilled as columns stop; 0: one batch of all weightings")
    ap.add_argument("--precision", default="bf16x3", choices=sorted(PRECISIONS),
                    help="BF16 form of A: bf16x3 (two BF16 terms; the plans match FP64), bf16 (one term)")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the device plan-metrics and two-pass measurements")
    ap.add_argument("--solve-refine", type=int, default=0,
                    help="refinement steps of the solve per iteration (lgk_params.solve_refine)")
    ap.add_argument("--setup-fp64", action="store_true",
                    help="form S = A A^T + I with FP64 products instead of the tensor cores")
    ap.add_argument("--rho-adapt", action="store_true",
                    help="per-column residual balancing of rho (lgk_params.rho_adapt)")
    ap.add_argument("--no-check", action="store_true",
                    help="count plans by the residual test alone (no FP64 check in the timed region)")
    ap.add_argument("--l2-keep-inverse", action="store_true",
                    help="keep S^-1 in a persisting L2 carve-out during solves (lgk_params.l2_keep_inverse)")
    ap.add_argument("--gemm2-rows", type=int, default=0, choices=[0, 128, 256],
                    help="GEMM2 tile height (lgk_params.gemm2_tile_rows; 0: as GEMM1)")
    ap.add_argument("--no-group", action="store_true",
                    help="skip the co-scheduled group measurement (lgk_solve_group) of the cfg1 line")
    ap.add_argument("--group-cfg3", action="store_true",
                    help="add the 9-target 8325 x 122664 case (441 weightings) to the group measurement")
    ap.add_argument("--no-k441", action="store_true",
                    help="skip the 441-weighting (5000 x 61600) measurement of the cfg1 line")
    ap.add_argument("--serve", type=int, default=0,
                    help="serving mode: number of requests of a Poisson stream")
    ap.add_argument("--serve-workers", type=int, default=2)
    ap.add_argument("--serve-rates", default="0.25,0.5,1,2",
                    help="arrival rates to sweep, as multiples of the measured capacity")
    ap.add_argument("--no-serve", action="store_true",
                    help="skip the short serving run of the cfg1 line")
    args = ap.parse_args()
    rank, world, local = dist_init()
    if args.impl == "reference":
        rc = run_reference(args, rank, world)
    elif args.serve:
        rc = run_serve(args, rank, world, local)
    else:
        rc = run_ours(args, rank, world, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return rc


if __name__ == "__main__":
    sys.exit(main())
