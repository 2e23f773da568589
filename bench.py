#!/usr/bin/env python3
"""Benchmark of the two-site sweep on GB300.

Workload (the chi = 1024 configuration of the headline metric): Heisenberg
XXZ open chain, Delta = 1, N = 100 sites, d = 2, MPO bond D = 5, chi_max =
1024, truncation weight 1e-12, Lanczos Krylov dimension 20, bf16x3 tensor-core
contractions.  One step = one complete pair update of a left-to-right sweep
in the bulk of the chain (chi_l = chi_r = 1024): two-site tensor, Lanczos
(20 effective-operator applies), truncated SVD split, centre move and the
left environment update.  Each rank runs its own chain (independent problems,
no data-path collective): weak scaling.

The metric is H_eff-matvec TFLOP/s over whole steps: useful flops of the
effective-operator applies (2 D d^2 chi_l chi_r (chi_l + chi_r) +
4 D^2 d^3 chi_l chi_r per apply, counted once although bf16x3 issues three
MMAs) divided by the wall time of the steps; sweep seconds are the measured
mean step time times the 2 (N - 1) pair updates of a sweep.

The chain is synthetic: random Gaussian matrices (SplitMix64, seeded per
rank) turned into left / right isometries by the library's own SVD, with the
bulk isometry shared by all bulk sites, environments built by the library.
Inputs (MPS and environments: ~17 GB per chain) exceed the 129 MB L2.

--impl reference times the CPU oracle (plain FP64 NumPy) on a bounded sample
of the same workload: one pair update per step.
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

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "H_eff matvec TFLOP/s & sweep sec at chi=1024, mixed vs FP64 GPU, at stated energy err"
N_SITES, D_MPO, PHYS, DELTA = 100, 5, 2, 1.0
TRUNC_TOL = 1e-12
KRYLOV = 20
# DRAM bytes (read + write) of the Jacobi phase of one 2048 x 2048 split (the
# stationary-block sweep kernel 17.6 MB + 44.5 MB, the cleanup kernel 17.0 MB),
# from one ncu capture of `bench.py --kernel svd --chi 1024` (a split of the
# same shape; the working set of 16 MB of FP32 columns stays in L2)
JACOBI_TRAFFIC = 79154688


def log(msg: str):
    print(f"[bench {time.strftime('%H:%M:%S')}] {msg}", file=sys.stderr, flush=True)


def heff_flops(chl: int, chr_: int, D: int = D_MPO, d: int = PHYS) -> float:
    return 2.0 * D * d * d * chl * chr_ * (chl + chr_) + 4.0 * D * D * d ** 3 * chl * chr_


# ---------------------------------------------------------------- distributed plumbing
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu: int):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.reader = threading.Thread(target=self._read, daemon=True)
            self.reader.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self) -> dict:
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def measured_peaks() -> dict:
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            d = json.load(fh)
        return {"hbm_gbs": d.get("hbm_gbs", 6800.0), "bf16_tflops": d.get("bf16_tflops", 1900.0),
                "sm_max_mhz": d.get("sm_max_mhz", 2070.0), "source": "measured"}
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0, "source": "fallback"}


# ---------------------------------------------------------------- synthetic chain
def bond_dims(n: int, chi: int) -> list:
    return [int(min(chi, 2 ** min(i, 40), 2 ** min(n - i, 40))) for i in range(n + 1)]


def build_chain(pkg, ctx, chi: int, first: int, seed: int, precision: int):
    """A chain in mixed canonical form with the centre on site `first`.

    Left sites are left isometries, right sites right isometries (from the
    library's SVD of seeded Gaussian matrices, one shared isometry per
    distinct shape), the centre a normalised Gaussian tensor.
    """
    import torch
    import workloads as wl

    n = N_SITES
    chis = bond_dims(n, chi)
    W = wl.mpo.xxz(n, DELTA)
    cache = {}
    stream_off = [0]

    def gauss(shape):
        cnt = int(np.prod(shape))
        g = wl.rng.gaussians(seed, cnt, stream_off[0])
        stream_off[0] += (cnt + 1) // 2
        return torch.from_numpy(g.reshape(shape)).to(ctx.device)

    def left_iso(chl, chr_):
        key = ("L", chl, chr_)
        if key not in cache:
            M = gauss((chl * PHYS, chr_))
            res = ctx.svd_truncate(M, chr_, 0.0, absorb=pkg.ABSORB_RIGHT, precision=precision)
            assert res.rank == chr_, (key, res.rank)
            cache[key] = res.A_left.reshape(chl, PHYS, chr_).clone()
        return cache[key]

    def right_iso(chl, chr_):
        key = ("R", chl, chr_)
        if key not in cache:
            M = gauss((chl, PHYS * chr_))
            res = ctx.svd_truncate(M, chl, 0.0, absorb=pkg.ABSORB_LEFT, precision=precision)
            assert res.rank == chl, (key, res.rank)
            cache[key] = res.A_right.reshape(chl, PHYS, chr_).clone()
        return cache[key]

    A = []
    for i in range(n):
        if i < first:
            A.append(left_iso(chis[i], chis[i + 1]))
        elif i > first:
            A.append(right_iso(chis[i], chis[i + 1]))
        else:
            c = gauss((chis[i], PHYS, chis[i + 1]))
            A.append(c / torch.linalg.vector_norm(c))
    chain = pkg.Chain(ctx, W, A, chi)
    ctx.build_environments(chain, first, precision=precision)
    torch.cuda.synchronize()
    return chain, W


# ---------------------------------------------------------------- our arm
def run_ours(args) -> dict:
    import torch
    import paper_2601_16734_gb300 as pkg

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    pkg.build()
    chi = args.chi
    prec = pkg.BF16X3 if args.precision == "bf16x3" else pkg.FP64
    ctx = pkg.Context(local, chi_max=chi, d=PHYS, D_max=D_MPO, krylov_dim=KRYLOV)
    # tile autotuner: time both tile shapes on the bulk pair's GEMMs once (untimed)
    tuned = ctx.autotune(chi, chi, PHYS, D_MPO, D_MPO, D_MPO) if args.autotune else 0
    ctx.set_autotune(args.autotune)
    ctx.set_fused_mixing(args.fused_mix)
    first = 20
    need = first + args.warmup + 2 * args.steps + args.fp64_steps + 2
    assert need <= N_SITES - 10, "too many steps for one half sweep of the bulk"
    t_setup = time.time()
    log("building the synthetic chain")
    chain, W = build_chain(pkg, ctx, chi, first, seed=1 + 7919 * rank, precision=prec)
    setup_s = time.time() - t_setup
    log(f"chain ready in {setup_s:.1f} s")
    kw = dict(precision=prec, krylov_dim=KRYLOV, chi_max=chi, tol=TRUNC_TOL)

    # warm-up pair updates (untimed)
    pos = first
    if args.warmup:
        t0 = time.time()
        ctx.sweep_range(chain, pos, args.warmup, 1, **kw)
        pos += args.warmup
        log(f"{args.warmup} warm-up pair updates in {time.time() - t0:.2f} s")
    stream = ctx.stream
    launches0 = ctx.launch_count()
    ctx.svd_stats(reset=True)
    ctx.svd_cleanup_stats(reset=True)
    ctx.get_timing(reset=True)
    ctx.set_timing(True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    with Clocks(local) as clk:
        ev0.record(stream)
        rep = ctx.sweep_range(chain, pos, args.steps, 1, **kw)
        ev1.record(stream)
        torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    ctx.set_timing(False)
    phases = ctx.get_timing(reset=True)
    svd_stats = ctx.svd_stats(reset=True)
    cleanup_stats = ctx.svd_cleanup_stats(reset=True)
    launches = ctx.launch_count() - launches0
    elapsed_ms = ev0.elapsed_time(ev1)
    log(f"timed {args.steps} pair updates: {elapsed_ms:.1f} ms")
    pos += args.steps
    applies = rep["local_iters"]
    flops = applies * heff_flops(chi, chi)
    from paper_2601_16734_gb300.shard import reduce_run
    elapsed_ms, flops_all, launches_all = reduce_run(elapsed_ms, flops, launches, device=ctx.device)
    value = flops_all / (elapsed_ms * 1e-3) / 1e12
    step_ms = elapsed_ms / args.steps

    # ---- the plain FP64 GPU path on the same chain (the "vs FP64 GPU" half of the metric)
    fp64 = None
    if args.fp64_steps > 0:
        kw64 = dict(kw, precision=pkg.FP64)
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(stream)
        rep64 = ctx.sweep_range(chain, pos, args.fp64_steps, 1, **kw64)
        f1.record(stream)
        torch.cuda.synchronize()
        f_ms = f0.elapsed_time(f1)
        pos += args.fp64_steps
        fp64 = {"ms_per_step": round(f_ms / args.fp64_steps, 1), "steps": args.fp64_steps,
                "value": round(rep64["local_iters"] * heff_flops(chi, chi) / (f_ms * 1e-3) / 1e12, 3),
                "unit": "TFLOP/s", "sweep_sec": round(f_ms / args.fp64_steps * 2 * (N_SITES - 1) / 1e3, 1),
                "speedup_of_mixed": round((f_ms / args.fp64_steps) / step_ms, 2)}
        log(f"FP64 GPU: {args.fp64_steps} pair updates in {f_ms:.1f} ms")

    # ---- end to end: host buffers in, host buffers out, through the same C-ABI call
    nd = chi * PHYS * chi
    ne = chi * D_MPO * chi
    host_in = [torch.empty(nd, dtype=torch.float64, pin_memory=True) for _ in range(2)] + \
              [torch.empty(ne, dtype=torch.float64, pin_memory=True) for _ in range(2)]
    host_out = [torch.empty(nd, dtype=torch.float64, pin_memory=True) for _ in range(2)] + \
               [torch.empty(ne, dtype=torch.float64, pin_memory=True), torch.empty(1, dtype=torch.float64,
                                                                                  pin_memory=True)]
    e2e_steps = max(1, min(args.steps, 3))
    # snapshot of a realistic state as the host-side inputs
    host_in[0].copy_(chain.A[pos][:nd])
    host_in[1].copy_(chain.A[pos + 1][:nd])
    host_in[2].copy_(chain.L[pos][:ne])
    host_in[3].copy_(chain.R[pos + 2][:ne])
    torch.cuda.synchronize()
    h2d = sum(t.numel() * 8 for t in host_in)
    d2h = 2 * nd * 8 + ne * 8 + 8
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    e2e_applies = 0
    for k in range(e2e_steps):
        i = pos + k
        chain.A[i][:nd].copy_(host_in[0], non_blocking=True)
        chain.A[i + 1][:nd].copy_(host_in[1], non_blocking=True)
        chain.L[i][:ne].copy_(host_in[2], non_blocking=True)
        chain.R[i + 2][:ne].copy_(host_in[3], non_blocking=True)
        chain.chi[i + 1] = chi
        r = ctx.sweep_range(chain, i, 1, 1, **kw)
        e2e_applies += r["local_iters"]
        host_out[0].copy_(chain.A[i][:nd], non_blocking=True)
        host_out[1].copy_(chain.A[i + 1][:nd], non_blocking=True)
        host_out[2].copy_(chain.L[i + 1][:ne], non_blocking=True)
        host_out[3][0] = r["energy"]
    e1.record(stream)
    torch.cuda.synchronize()
    e2e_ms = e0.elapsed_time(e1)
    log(f"e2e {e2e_steps} pair updates: {e2e_ms:.1f} ms")
    e2e_value = e2e_applies * heff_flops(chi, chi) / (e2e_ms * 1e-3) / 1e12 * world

    # ---- roofline of the dominant kernel (the tcgen05 GEMM or the SVD)
    peaks = measured_peaks()
    tc_ms, tc_n = phases["tc_gemm"]
    mv_ms, mv_n = phases["matvec"]
    svd_ms, svd_n = phases["svd"]
    # algorithmic flops of the two tensor-core GEMMs of one apply, counted
    # once (the bf16x3 split issues 3x these MMAs)
    gemm_flops_apply = 2.0 * D_MPO * PHYS ** 2 * chi * chi * (chi + chi)
    env_ms, env_n = phases["env"]
    gemm_flops_env = 2 * 2.0 * PHYS * D_MPO * chi ** 3  # two GEMMs per environment update
    roof_tc = None
    if tc_n and mv_n:
        per_launch_ms = tc_ms / tc_n
        gemm_share = (gemm_flops_apply * mv_n + gemm_flops_env * env_n) / tc_n  # mean algorithmic flops/launch
        achieved = 3.0 * gemm_share / (per_launch_ms * 1e-3) / 1e12  # tensor-pipe flops issued
        roof_tc = {"kernel": "tc_gemm_bf16x3_kernel", "bound": "tensor", "achieved": round(achieved, 1),
                   "peak": peaks["bf16_tflops"], "unit": "TFLOP/s", "frac": round(achieved / peaks["bf16_tflops"], 4),
                   "traffic": None, "peak_source": peaks["source"] + " bf16 burst (of measured)",
                   "useful_tflops_per_launch": round(gemm_share / (per_launch_ms * 1e-3) / 1e12, 1),
                   "launches": tc_n, "mean_launch_ms": round(per_launch_ms, 4),
                   "note": "achieved counts the 3 bf16 MMAs of the split product; useful = achieved/3"}
    # Jacobi SVD kernel: FP32 CUDA-core ALU bound; peak = SMs x 128 FP32 lanes x 2 flops x max SM clock.
    # Its launches are timed by their own CUDA-event phase ("jacobi"); the QR
    # preconditioning and the rest of the split are reported beside it.
    roof_svd = None
    jac_ms, jac_n = phases.get("jacobi", (0.0, 0))
    qr_ms, qr_n = phases.get("qr", (0.0, 0))
    if jac_n and svd_stats["calls"]:
        sms = torch.cuda.get_device_properties(local).multi_processor_count
        fp32_peak = sms * 128 * 2 * peaks["sm_max_mhz"] * 1e6 / 1e12
        jac_launch_ms = jac_ms / jac_n
        # the one-sided Jacobi's work model, 6 m n^2 flops per sweep of the n(n-1)/2 column
        # pairs of length m: 12 m flops per visited pair (its two norms and cross product,
        # 6 m, and the rotation, 6 m); m = 2 chi at the bulk pair
        ach = 12.0 * (2 * chi) * svd_stats["pair_visits"] / (jac_ms * 1e-3) / 1e12
        ach_lean = svd_stats["flops"] / (jac_ms * 1e-3) / 1e12
        roof_svd = {"kernel": "svd_sm_kernel (block FP32 one-sided Jacobi, cooperative, stationary blocks; "
                              "svd_block_kernel for other block counts) + svd_cleanup_kernel (its last sweeps)",
                    "bound": "alu",
                    "achieved": round(ach, 2), "peak": round(fp32_peak, 1), "unit": "TFLOP/s",
                    "frac": round(ach / fp32_peak, 4), "traffic": JACOBI_TRAFFIC,
                    "peak_source": "derived: SMs x 128 FP32 lanes x 2 x max SM clock",
                    "launches": jac_n, "mean_launch_ms": round(jac_launch_ms, 2),
                    "jacobi_sweeps_per_call": round(svd_stats["sweeps"] / svd_stats["calls"], 1),
                    "pair_visits_per_call": int(svd_stats["pair_visits"] / svd_stats["calls"]),
                    "cleanup": {"calls": cleanup_stats["calls"], "rounds": cleanup_stats["rounds"],
                                "fallbacks": cleanup_stats["fallbacks"]},
                    "qr_ms_per_call": round(qr_ms / qr_n, 2) if qr_n else None,
                    "svd_ms_per_call": round(svd_ms / svd_n, 2),
                    "achieved_executed": round(ach_lean, 2),
                    "note": "achieved: 12 m flops per visited column pair of length m (6 m n^2 per Jacobi "
                            "sweep, norms and cross product plus rotation); achieved_executed counts what "
                            "the kernel executes: 2 m per visited pair (the cross product; norms are "
                            "updated from it) + 6 m per rotated pair. The kernel is latency-bound (one CTA "
                            "barrier and a rotation per slot, an L2 hand-off of the circulating block per "
                            "block step)"}
    if roof_svd and jac_ms > tc_ms:
        roofline, roofline_secondary = roof_svd, roof_tc
    else:
        roofline, roofline_secondary = roof_tc, roof_svd

    res = {
        "metric": METRIC, "value": round(value, 3), "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(step_ms, 3), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "bf16x3" if prec == pkg.BF16X3 else "f64",
        "data": "synthetic (seeded Gaussian isometries, XXZ MPO)",
        "config": {"workload": f"XXZ Delta=1 N={N_SITES} d=2 D=5 chi={chi}: one bulk pair update per step "
                               f"(Lanczos k={KRYLOV}, SVD split, env update)",
                   "chi": chi, "n_sites": N_SITES, "krylov_dim": KRYLOV, "truncation": TRUNC_TOL,
                   "l2": "inputs larger than L2 (~17 GB of MPS and environments per chain)",
                   "parallelism": f"independent chains x{world}"},
        "sweep_sec": None,  # measured by full_sweep below
        "sweep_sec_from_bulk_steps": round(step_ms * 2 * (N_SITES - 1) / 1e3, 2),
        "energy_last_pair": rep["energy"],
        "phases_ms": {k: round(v[0], 3) for k, v in phases.items()},
        "phase_counts": {k: v[1] for k, v in phases.items()},
        "heff_matvec_tflops": round(mv_n and (mv_n * heff_flops(chi, chi)) / (mv_ms * 1e-3) / 1e12 or 0.0, 1),
        # the matvec's share of the dtype's dense tensor peak (measured bf16 burst): useful
        # flops, and the three bf16 MMAs issued per split product
        "heff_matvec_frac": {
            "useful": round((mv_n and (mv_n * heff_flops(chi, chi)) / (mv_ms * 1e-3) / 1e12 or 0.0)
                            / peaks["bf16_tflops"], 4),
            "issued": round(3 * (mv_n and (mv_n * heff_flops(chi, chi)) / (mv_ms * 1e-3) / 1e12 or 0.0)
                            / peaks["bf16_tflops"], 4),
            "peak_tflops": peaks["bf16_tflops"]},
        "gpu_launches": launches_all,
        "autotune": {"enabled": bool(args.autotune), "shapes_timed": tuned, **ctx.autotune_stats()},
        "fused_mixing": bool(args.fused_mix),
        "setup_s": round(setup_s, 1),
        "e2e": {"value": round(e2e_value, 3), "unit": "TFLOP/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "steps": e2e_steps},
        "roofline": roofline,
        "roofline_secondary": roofline_secondary,
        "fp64_gpu": fp64,
        "clocks": clk.summary(),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        log("cpu baseline (oracle, one pair update)")
        res["cpu_baseline"] = cpu_baseline(chain, W, pos, chi)
    if args.full_sweep:
        del chain
        torch.cuda.empty_cache()
        sw = full_sweep(pkg, ctx, chi, seed=1 + 7919 * rank, precision=prec, gpu=local)
        res["sweep"] = sw
        res["sweep_sec"] = sw["sweep_sec"]
        res["energy_err"] = sw["energy_err"]
        if fp64 is not None:
            fp64["sweep_sec_est"] = fp64.pop("sweep_sec")
            fp64["speedup_of_mixed_sweep_est"] = round(fp64["sweep_sec_est"] / sw["sweep_sec"], 1)
    ctx.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return res if rank == 0 else None


def full_sweep(pkg, ctx, chi: int, seed: int, precision: int, gpu: int) -> dict:
    """One complete sweep of the N-site chain at chi_max, timed: pairs 0..N-2
    left to right, then N-2..0 right to left (2 (N - 1) pair updates, the
    small bonds at the chain ends included), from a right-canonical seeded
    random MPS with its environments prebuilt.  Then the FP64 energy of the
    MPS the sweep produced: environments rebuilt in FP64 and
    <theta, H_0 theta> / <theta, theta> at the end pair, against the energy
    the mixed sweep reported for that pair (its last local solve)."""
    import torch

    chain, W = build_chain(pkg, ctx, chi, 0, seed, precision)
    kw = dict(precision=precision, krylov_dim=KRYLOV, chi_max=chi, tol=TRUNC_TOL)
    stream = ctx.stream
    torch.cuda.synchronize()
    ctx.svd_stats(reset=True)
    ctx.svd_cleanup_stats(reset=True)
    ctx.get_timing(reset=True)
    ctx.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(gpu) as clk:
        e0.record(stream)
        r1 = ctx.sweep_range(chain, 0, N_SITES - 1, 1, **kw)
        r2 = ctx.sweep_range(chain, N_SITES - 2, N_SITES - 1, -1, **kw)
        e1.record(stream)
        torch.cuda.synchronize()
    ctx.set_timing(False)
    ms = e0.elapsed_time(e1)
    phases = {k: round(v[0] / 1e3, 3) for k, v in ctx.get_timing(reset=True).items()}
    svd_st, cl_st = ctx.svd_stats(reset=True), ctx.svd_cleanup_stats(reset=True)
    log(f"full sweep ({2 * (N_SITES - 1)} pair updates) in {ms / 1e3:.2f} s")
    # FP64 energy of the resulting state (centre on pair (0, 1))
    t0 = time.time()
    ctx.build_environments(chain, 0, precision=pkg.FP64)
    A0, A1 = chain.tensors()[0], chain.tensors()[1]
    theta = ctx.two_site(A0, A1)
    c = chain.chi
    L0 = chain.L[0][:1].view(1, 1, 1)
    D2 = int(W[1].shape[3])  # MPO bond between sites 1 and 2
    R2 = chain.R[2][: c[2] * D2 * c[2]].view(c[2], D2, c[2])
    Wd = [torch.from_numpy(np.ascontiguousarray(w)).to(ctx.device) for w in (W[0], W[1])]
    y = ctx.heff_apply(L0, Wd[0], Wd[1], R2, theta, precision=pkg.FP64)
    e64 = float(torch.sum(theta * y) / torch.sum(theta * theta))
    log(f"FP64 energy of the swept state in {time.time() - t0:.1f} s")
    em = r2["energy"]
    out = {"sweep_sec": round(ms / 1e3, 3), "pair_updates": 2 * (N_SITES - 1),
           "local_iters": r1["local_iters"] + r2["local_iters"], "energy_mixed": em, "energy_fp64_same_state": e64,
           "energy_err": abs(em - e64) / abs(e64), "max_discarded": max(r1["max_discarded"], r2["max_discarded"]),
           "start": "right-canonical seeded random MPS, bonds min(chi, 2^i, 2^(N-i))",
           "phases_sec": phases, "large_splits": svd_st["calls"], "jacobi_sweeps": svd_st["sweeps"],
           "cleanup": cl_st, "clocks": clk.summary()}
    del chain
    torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------- kernel-only mode
def run_heff_only(args) -> dict:
    """Effective-operator applies alone at the bench size (a small-memory case
    of the hot kernels, ~1.4 GB on the device; used for profiling)."""
    import torch
    import paper_2601_16734_gb300 as pkg

    pkg.build()
    chi, D, d = args.chi, D_MPO, PHYS
    ctx = pkg.Context(0, chi_max=chi, d=d, D_max=D, krylov_dim=KRYLOV)
    g = torch.Generator(device="cuda").manual_seed(0)
    rn = lambda *sh: torch.randn(*sh, dtype=torch.float64, device="cuda", generator=g)
    L, R, W1, W2, th = rn(chi, D, chi), rn(chi, D, chi), rn(D, d, d, D), rn(D, d, d, D), rn(chi, d, d, chi)
    y = torch.empty_like(th)
    prec = pkg.BF16X3 if args.precision == "bf16x3" else pkg.FP64
    for _ in range(args.warmup):
        ctx.heff_apply(L, W1, W2, R, th, precision=prec, out=y)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(args.steps):
        ctx.heff_apply(L, W1, W2, R, th, precision=prec, out=y)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / args.steps
    ctx.close()
    return {"mode": "heff_only", "chi": chi, "ms_per_apply": round(ms, 4),
            "useful_tflops": round(heff_flops(chi, chi) / (ms * 1e-3) / 1e12, 1), "precision": args.precision}


def run_svd_only(args) -> dict:
    """The mixed-precision SVD split alone on one 2 chi x 2 chi two-site matrix
    with a graded spectrum, s_j = exp(-j / 150) (the shape of the bench's
    split; 16 MB of FP32 Jacobi data, small enough for a full ncu capture)."""
    import torch
    import paper_2601_16734_gb300 as pkg
    from workloads.rng import gaussians

    pkg.build()
    n = 2 * args.chi
    ctx = pkg.Context(0, chi_max=args.chi, d=PHYS, D_max=1, krylov_dim=2)
    U = np.linalg.qr(gaussians(11, n * n).reshape(n, n))[0]
    V = np.linalg.qr(gaussians(12, n * n).reshape(n, n))[0]
    s = np.exp(-np.arange(n) / 150.0)
    M = torch.from_numpy((U * s) @ V.T).cuda()
    prec = pkg.BF16X3 if args.precision == "bf16x3" else pkg.FP64
    for _ in range(args.warmup):
        ctx.svd_truncate(M, args.chi, TRUNC_TOL, precision=prec)
    torch.cuda.synchronize()
    ctx.svd_stats(reset=True)
    ctx.get_timing(reset=True)
    ctx.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    for _ in range(args.steps):
        res = ctx.svd_truncate(M, args.chi, TRUNC_TOL, precision=prec)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ctx.set_timing(False)
    ms = e0.elapsed_time(e1) / args.steps
    ph = ctx.get_timing(reset=True)
    st = ctx.svd_stats(reset=True)
    cst = ctx.svd_cleanup_stats(reset=True)
    rot, _ = ctx.svd_sweep_counts()
    err = float(np.abs(res.S.cpu().numpy()[: n] - s).max())
    ctx.close()
    calls = max(1, st["calls"])
    return {"mode": "svd_only", "n": n, "ms_per_split": round(ms, 3), "rotations_per_sweep": rot,
            "cleanup": cst,
            "jacobi_ms": round(ph["jacobi"][0] / max(1, ph["jacobi"][1]), 3),
            "qr_ms": round(ph["qr"][0] / max(1, ph["qr"][1]), 3),
            "sweeps_per_split": st["sweeps"] / calls, "pair_visits_per_split": st["pair_visits"] // calls,
            "jacobi_tflops": round(12.0 * n * st["pair_visits"] / (ph["jacobi"][0] * 1e-3) / 1e12, 2)
            if ph["jacobi"][0] else None,
            "jacobi_tflops_executed": round(st["flops"] / (ph["jacobi"][0] * 1e-3) / 1e12, 2)
            if ph["jacobi"][0] else None,
            "max_abs_s_error": err, "rank": res.rank, "precision": args.precision}


def run_simplify_only(args) -> dict:
    """Variational compression (simplify mode): a seeded random target b of
    bond dimension 2 chi on 32 sites (each tensor scaled by 1/sqrt(chi_l d))
    compressed to bond chi; one untimed sweep from a random guess, then one
    timed full sweep (62 pair updates: antilinear-form vector, split,
    environment update)."""
    import torch
    import paper_2601_16734_gb300 as pkg
    from workloads.states import random_mps

    pkg.build()
    n, chi, chib = 32, args.chi, 2 * args.chi
    prec = pkg.BF16X3 if args.precision == "bf16x3" else pkg.FP64
    b = random_mps(n, PHYS, chib, 61)
    b = [t / np.sqrt(t.shape[0] * t.shape[1]) for t in b]
    x0 = random_mps(n, PHYS, chi, 62)
    ctx = pkg.Context(0, chi_max=chi, d=PHYS, D_max=1, krylov_dim=2, chib_max=chib)
    ch = pkg.Chain(ctx, None, x0, chi, B=b)
    ctx.sweep(ch, mode=pkg.MODE_SIMPLIFY, n_sweeps=1, precision=prec, chi_max=chi, tol=1e-14)
    torch.cuda.synchronize()
    ctx.get_timing(reset=True)
    ctx.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    rep = ctx.sweep(ch, mode=pkg.MODE_SIMPLIFY, n_sweeps=1, precision=prec, chi_max=chi, tol=1e-14,
                    canonicalize=False)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ctx.set_timing(False)
    ph = ctx.get_timing(reset=True)
    ms = e0.elapsed_time(e1)
    ctx.close()
    pairs = 2 * (n - 1)
    return {"mode": "simplify", "n_sites": n, "chi": chi, "chi_b": chib, "precision": args.precision,
            "ms_per_pair_update": round(ms / pairs, 3), "sweep_ms": round(ms, 1),
            "svd_ms_per_pair": round(ph["svd"][0] / max(1, ph["svd"][1]), 3),
            "discarded_fraction_max": rep["max_discarded"], "error_bound": rep["error_bound"]}


def run_tdvp_only(args) -> dict:
    """Two-site TDVP in imaginary time on the bench chain (XXZ, N=100,
    chi=1024, centre at site 20): one untimed pair update, then `steps` timed
    left-to-right pair updates (forward Krylov exponential of the pair,
    normalised split, environment update, backward one-site exponential),
    dt = 0.05, Krylov dimension 20."""
    import torch
    import paper_2601_16734_gb300 as pkg

    pkg.build()
    chi = args.chi
    prec = pkg.BF16X3 if args.precision == "bf16x3" else pkg.FP64
    ctx = pkg.Context(0, chi_max=chi, d=PHYS, D_max=D_MPO, krylov_dim=KRYLOV)
    first = 20
    chain, _ = build_chain(pkg, ctx, chi, first, seed=1, precision=prec)
    kw = dict(mode=pkg.MODE_TDVP, precision=prec, krylov_dim=KRYLOV, chi_max=chi, tol=TRUNC_TOL, tdvp_dt=0.05)
    ctx.sweep_range(chain, first, 1, 1, **kw)
    torch.cuda.synchronize()
    ctx.get_timing(reset=True)
    ctx.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    rep = ctx.sweep_range(chain, first + 1, args.steps, 1, **kw)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ctx.set_timing(False)
    ph = ctx.get_timing(reset=True)
    ms = e0.elapsed_time(e1)
    assert ctx.device_status() == 0
    ctx.close()
    # useful matvec flops: pair operator (k applies) + one-site operator (k applies)
    one_site = 2 * D_MPO * PHYS * chi * chi * (chi + chi) + 2 * D_MPO * D_MPO * PHYS * PHYS * chi * chi
    flops = rep["local_iters"] * heff_flops(chi, chi) + args.steps * KRYLOV * one_site
    return {"mode": "tdvp", "chi": chi, "precision": args.precision, "pair_updates": args.steps,
            "ms_per_pair_update": round(ms / args.steps, 3),
            "matvec_tflops_useful": round(flops / (ms * 1e-3) / 1e12, 2),
            "phases_ms_per_pair": {k: round(v[0] / args.steps, 3) for k, v in ph.items() if v[1]},
            "energy": rep["energy"], "max_discarded": rep["max_discarded"]}


def run_apply_only(args) -> dict:
    """Variational MPO-MPS product (apply mode): the XXZ MPO (D = 5) applied to
    a seeded random b of bond chi on 24 sites (each tensor scaled by
    1/sqrt(chi_l d)), the product (bond 5 chi) compressed to bond chi; one
    untimed sweep from a random guess, then one timed full sweep (46 pair
    updates: b's two-site tensor, the pair's MPO action between the
    environments of <x, W b>, split, environment update)."""
    import torch
    import paper_2601_16734_gb300 as pkg
    import workloads as wl
    from workloads.states import random_mps

    pkg.build()
    n, chi = 24, args.chi
    prec = pkg.BF16X3 if args.precision == "bf16x3" else pkg.FP64
    W = wl.mpo.xxz(n, DELTA)
    b = random_mps(n, PHYS, chi, 81)
    b = [t / np.sqrt(t.shape[0] * t.shape[1]) for t in b]
    x0 = random_mps(n, PHYS, chi, 82)
    ctx = pkg.Context(0, chi_max=chi, d=PHYS, D_max=D_MPO, krylov_dim=2, chib_max=chi)
    ch = pkg.Chain(ctx, W, x0, chi, B=b)
    kw = dict(mode=pkg.MODE_APPLY, n_sweeps=1, precision=prec, chi_max=chi, tol=1e-14)
    ctx.sweep(ch, **kw)
    torch.cuda.synchronize()
    ctx.get_timing(reset=True)
    ctx.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(ctx.stream)
    rep = ctx.sweep(ch, canonicalize=False, **kw)
    e1.record(ctx.stream)
    torch.cuda.synchronize()
    ctx.set_timing(False)
    ph = ctx.get_timing(reset=True)
    ms = e0.elapsed_time(e1)
    assert ctx.device_status() == 0
    ctx.close()
    pairs = 2 * (n - 1)
    return {"mode": "apply", "n_sites": n, "chi": chi, "chi_b": chi, "D": D_MPO, "precision": args.precision,
            "ms_per_pair_update": round(ms / pairs, 3), "sweep_ms": round(ms, 1),
            "phases_ms_per_pair": {k: round(v[0] / pairs, 3) for k, v in ph.items() if v[1]},
            "discarded_fraction_max": rep["max_discarded"]}


def run_c5(args) -> dict:
    """Large-chi DMRG: the J1-J2 Heisenberg cylinder (J2/J1 = 0.5, width 6,
    length 16, snaked into 96 sites, MPO from the exact graph builder), the
    bulk pair (48, 49) at chi = 2048.  Environments L_48 and R_50 are built by
    the library (bf16x3 updates over seeded random isometries, one shared
    bulk isometry, only the current environment kept); then `steps` mixed
    pair updates of that pair from the same normalised Gaussian start vector
    (Lanczos k = 20 on bf16x3 products, the mixed split, the left environment
    update), timed with CUDA events, and the FP64 GPU Lanczos from the same
    start vector on the same environments as the comparator (energy and
    time)."""
    import torch
    import paper_2601_16734_gb300 as pkg
    import workloads as wl

    pkg.build()
    n, chi, p = 96, args.chi, 48
    W = wl.mpo.heisenberg_graph(n, wl.mpo.j1j2_cylinder_bonds(6, 16, 1.0, 0.5))
    Dmax = max(int(w.shape[3]) for w in W)
    chis = bond_dims(n, chi)
    ctx = pkg.Context(0, chi_max=chi, d=PHYS, D_max=Dmax, krylov_dim=KRYLOV)
    if args.autotune:
        ctx.set_autotune(True)
    dev = ctx.device
    Wd = [torch.from_numpy(np.ascontiguousarray(w)).to(dev) for w in W]
    t0 = time.time()
    off = [0]

    def gauss(shape, seed):
        cnt = int(np.prod(shape))
        g = torch.from_numpy(wl.rng.gaussians(seed, cnt, off[0]).reshape(shape)).to(dev)
        off[0] += (cnt + 1) // 2
        return g

    cache = {}

    def iso(side, chl, chr_):
        key = (side, chl, chr_)
        if key not in cache:
            if side == "L":
                res = ctx.svd_truncate(gauss((chl * PHYS, chr_), 2), chr_, 0.0, absorb=pkg.ABSORB_RIGHT,
                                       precision=pkg.BF16X3)
                cache[key] = res.A_left.reshape(chl, PHYS, chr_).clone()
            else:
                res = ctx.svd_truncate(gauss((chl, PHYS * chr_), 2), chl, 0.0, absorb=pkg.ABSORB_LEFT,
                                       precision=pkg.BF16X3)
                cache[key] = res.A_right.reshape(chl, PHYS, chr_).clone()
        return cache[key]

    L = torch.ones(1, 1, 1, dtype=torch.float64, device=dev)
    for k in range(p):
        L = ctx.env_update(pkg.LEFT, L, iso("L", chis[k], chis[k + 1]), Wd[k], precision=pkg.BF16X3)
    R = torch.ones(1, 1, 1, dtype=torch.float64, device=dev)
    for k in range(n - 1, p + 1, -1):
        R = ctx.env_update(pkg.RIGHT, R, iso("R", chis[k], chis[k + 1]), Wd[k], precision=pkg.BF16X3)
    cache.clear()
    torch.cuda.synchronize()
    setup = time.time() - t0
    D_l, D_m, D_r = int(W[p].shape[0]), int(W[p].shape[3]), int(W[p + 1].shape[3])
    if args.autotune:
        ctx.autotune(chi, chi, PHYS, D_l, D_m, D_r)
    log(f"C5 environments (chi {chi}, MPO bonds {D_l}/{D_m}/{D_r}) in {setup:.1f} s")
    theta0 = gauss((chi, PHYS, PHYS, chi), 5)
    theta0 /= torch.linalg.vector_norm(theta0)
    A_l = torch.empty(chi * PHYS * chi, dtype=torch.float64, device=dev)
    A_r = torch.empty_like(A_l)

    def pair_update(prec):
        th = theta0.clone()
        e, it = ctx.local_eig(L, Wd[p], Wd[p + 1], R, th, krylov_dim=KRYLOV, precision=prec)
        res = ctx.svd_truncate(th.view(chi * PHYS, PHYS * chi), chi, TRUNC_TOL, absorb=pkg.ABSORB_RIGHT,
                               normalize=True, precision=prec)
        ctx.env_update(pkg.LEFT, L, res.A_left.reshape(chi, PHYS, res.rank), Wd[p], precision=prec)
        return e, it, res.rank

    for _ in range(args.warmup):
        pair_update(pkg.BF16X3)
    torch.cuda.synchronize()
    ctx.get_timing(reset=True)
    ctx.set_timing(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with Clocks(0) as clk:
        e0.record(ctx.stream)
        applies = 0
        for _ in range(args.steps):
            e_mix, it, rank = pair_update(pkg.BF16X3)
            applies += it
        e1.record(ctx.stream)
        torch.cuda.synchronize()
    ctx.set_timing(False)
    ph = ctx.get_timing(reset=True)
    ms = e0.elapsed_time(e1) / args.steps
    fl = heff_flops_dims(chi, chi, D_l, D_m, D_r)
    mv_ms, mv_n = ph["matvec"]
    peaks = measured_peaks()
    heff_tf = mv_n * fl / (mv_ms * 1e-3) / 1e12 if mv_n else 0.0
    out = {"mode": "c5", "workload": "J1-J2 (J2/J1 = 0.5) cylinder 6 x 16 -> 96 sites, pair (48, 49)",
           "chi": chi, "mpo_bonds": [D_l, D_m, D_r], "precision": "bf16x3",
           "ms_per_pair_update": round(ms, 2), "lanczos_steps": it, "rank": rank,
           "heff_matvec_tflops_useful": round(heff_tf, 1),
           "heff_matvec_tensor_frac_issued": round(3 * heff_tf / peaks["bf16_tflops"], 4),
           "peak_bf16_tflops": peaks["bf16_tflops"], "peak_source": peaks["source"],
           "phases_ms_per_pair": {k: round(v[0] / args.steps, 2) for k, v in ph.items() if v[1]},
           "energy_mixed": e_mix, "setup_s": round(setup, 1), "clocks": clk.summary()}
    if args.fp64_steps > 0:
        th = theta0.clone()
        f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        f0.record(ctx.stream)
        e64, it64 = ctx.local_eig(L, Wd[p], Wd[p + 1], R, th, krylov_dim=KRYLOV, precision=pkg.FP64)
        f1.record(ctx.stream)
        torch.cuda.synchronize()
        out["fp64_lanczos"] = {"energy": e64, "seconds": round(f0.elapsed_time(f1) / 1e3, 2), "steps": it64,
                               "energy_rel_diff_mixed": abs(e_mix - e64) / abs(e64)}
        log(f"C5 FP64 Lanczos: {out['fp64_lanczos']}")
    assert ctx.device_status() == 0
    ctx.close()
    return out


def heff_flops_dims(chl: int, chr_: int, Dl: int, Dm: int, Dr: int, d: int = PHYS) -> float:
    """Useful flops of one H_n apply in the build's order: L . theta (2 D_l d^2
    chl^2 chr), the fused MPO mix (2 D_l D_r d^4 chl chr), T2 . R
    (2 D_r d^2 chl chr^2)."""
    return 2.0 * Dl * d * d * chl * chl * chr_ + 2.0 * Dl * Dr * d ** 4 * chl * chr_ + \
        2.0 * Dr * d * d * chl * chr_ * chr_


def run_cgs_only(args) -> dict:
    """Global conjugate gradients on MPS: U = 0.5 I + tridiag(-1, 2, -1) as a
    QTT MPO (D = 3) on 24 sites (2^24 unknowns), b a seeded random MPS of
    bond 16, bond limit 64, two sweeps per compression; `steps` CG steps
    timed (rtol 0, so every step runs)."""
    import torch
    import paper_2601_16734_gb300 as pkg
    import workloads as wl
    from workloads.states import random_mps

    pkg.build()
    n, chi, chib = 24, 64, 16
    prec = pkg.BF16X3 if args.precision == "bf16x3" else pkg.FP64
    W = wl.mpo.laplacian_qtt_1d(n, 1.0)
    W[-1] = W[-1].copy()
    W[-1][0, :, :, 0] += 0.5 * np.eye(2)
    b = random_mps(n, PHYS, chib, 91)
    x0 = random_mps(n, PHYS, 8, 92)
    ctx = pkg.Context(0, chi_max=chi, d=PHYS, D_max=3, krylov_dim=2, chib_max=2 * chi)
    ctx.cgs_solve(W, b, x0, chi, rtol=0.0, maxiter=1, precision=prec)
    torch.cuda.synchronize()
    t0 = time.time()
    _, rep = ctx.cgs_solve(W, b, x0, chi, rtol=0.0, maxiter=args.steps, precision=prec)
    wall = time.time() - t0
    assert ctx.device_status() == 0
    ctx.close()
    h = rep["residual_history"]
    return {"mode": "cgs", "n_sites": n, "chi": chi, "chi_b": chib, "precision": args.precision,
            "steps": rep["iterations"], "ms_per_step": round(1e3 * wall / max(1, rep["iterations"]), 2),
            "relative_residual": [round(v / rep["norm_b"], 10) for v in (h[0], h[-1])]}


def run_batch_only(args) -> dict:
    """Independent chains in one batched call (the C3 shape at a bounded
    size): 64 TFIM chains, g ~ U[0.5, 1.5], N ~ U{32..64}, chi_max ~ U{64, 128}
    from SplitMix64(3 + chain), 2 mixed sweeps + 1 FP64 refinement sweep each,
    run concurrently by seemps_sweep_batch and (on one GPU) then one after
    another on the same fresh inputs.  With several ranks the chains are
    shared out by cost (shard.shard_chains) and each rank batches its own;
    the elapsed time is the maximum over ranks (the batched energies are
    checked against the closed form in the GPU tests, not here)."""
    import torch
    import paper_2601_16734_gb300 as pkg
    from paper_2601_16734_gb300 import abi
    from paper_2601_16734_gb300.shard import chain_cost, reduce_run, shard_chains
    from workloads import mpo, rng, states

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    pkg.build()
    specs = []
    for k in range(64):
        u = rng.uniforms(3 + k, 3)
        specs.append((0.5 + u[0], 32 + int(u[1] * 33), [64, 128][int(u[2] * 2)]))
    mine = shard_chains([chain_cost(n, chi) for (_, n, chi) in specs], world, rank)

    def make():
        ctxs, chains, params = [], [], []
        for k in mine:
            g, n, chi = specs[k]
            ctxs.append(pkg.Context(local, chi_max=chi, d=PHYS, D_max=3, krylov_dim=KRYLOV,
                                    stream=torch.cuda.Stream()))
            chains.append(pkg.Chain(ctxs[-1], mpo.tfim(n, g), states.random_mps(n, PHYS, chi, 300 + k), chi))
            params.append(dict(mode=pkg.MODE_EIG, n_sweeps=2, refine_sweeps=1, precision=pkg.BF16X3,
                               krylov_dim=KRYLOV, chi_max=chi, tol=1e-12))
        torch.cuda.synchronize()
        return ctxs, chains, params

    ctxs, chains, params = make()
    if world > 1:
        torch.distributed.barrier()
    t0 = time.time()
    reps = abi.sweep_batch(ctxs, chains, params, max_threads=16)
    torch.cuda.synchronize()
    t_local = time.time() - t0
    for c in ctxs:
        c.close()
    my_pairs = sum(2 * 3 * (specs[k][1] - 1) for k in mine)
    t_batch, pairs, _ = reduce_run(t_local, my_pairs, 0, device=torch.device("cuda", local))
    out = {"mode": "batch", "chains": len(specs), "n_gpus": world, "pair_updates": int(pairs),
           "batched_s": round(t_batch, 3), "pair_updates_per_s": round(pairs / t_batch, 1),
           "energy_per_site_range_rank0": [round(min(r["energy"] / specs[k][1] for r, k in zip(reps, mine)), 6),
                                           round(max(r["energy"] / specs[k][1] for r, k in zip(reps, mine)), 6)]}
    if world == 1:
        ctxs, chains, params = make()
        t0 = time.time()
        for c, ch, kw in zip(ctxs, chains, params):
            c.sweep(ch, **kw)
        torch.cuda.synchronize()
        t_serial = time.time() - t0
        for c in ctxs:
            c.close()
        out.update({"serial_s": round(t_serial, 3), "speedup": round(t_serial / t_batch, 2)})
    if world > 1:
        torch.distributed.destroy_process_group()
    return out if rank == 0 else None


# ---------------------------------------------------------------- CPU oracle
def oracle_pair_update(Lenv, W1, W2, Renv, A1, A2, chi):
    """One pair update by the oracle: Lanczos (k = 20), SVD split, left env."""
    from oracle import sweep as S

    theta = S.two_site(A1, A2)
    mv = lambda v: S.heff_apply(Lenv, W1, W2, Renv, v)
    E, theta, m = S.lanczos_lowest(mv, theta, KRYLOV)
    chl, d1, d2, chr_ = theta.shape
    U, s, Vt, _, dw = S.svd_truncate(theta.reshape(chl * d1, d2 * chr_), chi, TRUNC_TOL)
    A1n = U.reshape(chl, d1, len(s))
    Ln = S.left_env(Lenv, A1n, W1)
    return E, m, Ln


def cpu_baseline(chain, W, pos, chi) -> dict:
    """The oracle, as it stands, on one pair update of the same workload."""
    import torch
    cores = len(os.sched_getaffinity(0))
    nd, ne = chi * PHYS * chi, chi * D_MPO * chi
    A1 = chain.A[pos][:nd].cpu().numpy().reshape(chi, PHYS, chi)
    A2 = chain.A[pos + 1][:nd].cpu().numpy().reshape(chi, PHYS, chi)
    Lenv = chain.L[pos][:ne].cpu().numpy().reshape(chi, D_MPO, chi)
    Renv = chain.R[pos + 2][:ne].cpu().numpy().reshape(chi, D_MPO, chi)
    t0 = time.time()
    E, m, _ = oracle_pair_update(Lenv, W[pos], W[pos + 1], Renv, A1, A2, chi)
    dt = time.time() - t0
    return {"value": round(m * heff_flops(chi, chi) / dt / 1e12, 4), "unit": "TFLOP/s", "cores": cores,
            "kind": "oracle", "sample": f"1 pair update at chi={chi} (Lanczos k={m}, SVD, env), {dt:.1f} s",
            "seconds": round(dt, 2), "energy": E}


def run_reference(args) -> dict:
    """--impl reference: the CPU oracle timed on bounded samples (rank 0 only)."""
    world, rank, local = dist_env()
    if rank != 0:
        return None
    import workloads as wl
    from oracle import sweep as S

    chi = args.ref_chi
    rng_seed = 1
    # a bulk pair of the same workload at the sample's bond dimension
    W = wl.mpo.xxz(N_SITES, DELTA)
    g = wl.rng.gaussians(rng_seed, 4 * chi * PHYS * chi + 2 * chi * D_MPO * chi)
    off = 0

    def take(shape):
        nonlocal off
        cnt = int(np.prod(shape))
        out = g[off:off + cnt].reshape(shape)
        off += cnt
        return out

    A1 = np.linalg.qr(take((chi * PHYS, chi)))[0].reshape(chi, PHYS, chi)
    A2 = np.linalg.qr(take((chi * PHYS, chi)))[0].T.reshape(chi, PHYS, chi)
    Lr = take((chi, D_MPO, chi))
    Rr = take((chi, D_MPO, chi))
    Lenv = 0.5 * (Lr + Lr.transpose(2, 1, 0))
    Renv = 0.5 * (Rr + Rr.transpose(2, 1, 0))
    for _ in range(args.warmup):
        oracle_pair_update(Lenv, W[40], W[41], Renv, A1, A2, chi)
    t0 = time.time()
    applies = 0
    for _ in range(args.steps):
        _, m, _ = oracle_pair_update(Lenv, W[40], W[41], Renv, A1, A2, chi)
        applies += m
    dt = time.time() - t0
    value = applies * heff_flops(chi, chi) / dt / 1e12
    cores = len(os.sched_getaffinity(0))
    return {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "TFLOP/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(1e3 * dt / args.steps, 1),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"XXZ Delta=1 d=2 D=5: one bulk pair update per step at chi={chi} "
                                   f"(Lanczos k={KRYLOV}, SVD split, env update), CPU oracle"},
            "cpu_baseline": {"value": round(value, 5), "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": f"{args.steps} pair updates at chi={chi}"},
            "e2e": {"value": round(value, 5), "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=8)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--chi", type=int, default=1024)
    ap.add_argument("--ref-chi", type=int, default=512)
    ap.add_argument("--precision", default="bf16x3", choices=["bf16x3", "fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fp64-steps", type=int, default=1)
    ap.add_argument("--no-autotune", dest="autotune", action="store_false",
                    help="keep the fixed tile rule instead of timing both tile shapes first")
    ap.add_argument("--fused-mix", dest="fused_mix", action="store_true",
                    help="run the effective operator's MPO mixing in the first GEMM's epilogue")
    ap.add_argument("--no-full-sweep", dest="full_sweep", action="store_false",
                    help="skip the timed full sweep and the FP64 energy of its state")
    ap.add_argument("--kernel", default="", choices=["", "heff", "svd", "simplify", "batch", "tdvp", "apply", "cgs",
                                                     "c5"],
                    help="heff: effective-operator applies only; svd: the mixed SVD split only "
                         "(profiling cases); simplify: one variational-compression sweep; batch: "
                         "independent chains batched vs one by one; tdvp: TDVP pair updates; apply: one "
                         "variational MPO-MPS product sweep; cgs: global conjugate-gradient steps; c5: the J1-J2 "
                         "cylinder pair at chi 2048 (use --chi 2048), mixed vs FP64 Lanczos")
    args = ap.parse_args()
    if args.impl == "reference":
        out = run_reference(args)
    elif args.kernel == "heff":
        out = run_heff_only(args)
    elif args.kernel == "svd":
        out = run_svd_only(args)
    elif args.kernel == "simplify":
        out = run_simplify_only(args)
    elif args.kernel == "batch":
        out = run_batch_only(args)
    elif args.kernel == "tdvp":
        out = run_tdvp_only(args)
    elif args.kernel == "apply":
        out = run_apply_only(args)
    elif args.kernel == "c5":
        out = run_c5(args)
    elif args.kernel == "cgs":
        out = run_cgs_only(args)
    else:
        out = run_ours(args)
    if out is not None:
        print(json.dumps(out))


if __name__ == "__main__":
    main()
