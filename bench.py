"""Benchmark: 2-D grid unbalanced OT, 256x256 images, KL lambda = 0.5 on both
marginals, eps-scaling 1e-1 -> 1e-3 (10 stages x 100 iterations, Sec. 4.4),
then iterations at eps = 1e-3 until the marginal violation is <= 1e-6.

One step = one complete solve through the C ABI (uot_solve) on synthetic
inputs resident in HBM.  Reported:
  value        Sinkhorn iterations per second (whole job, all ranks)
  ms_per_step  time to 1e-6 marginal violation (one solve)
  e2e          the same metric through uot_solve with host buffers: pinned
               host -> device copies of the inputs and the device -> host read
               of the potentials inside the timed region
  roofline     the dominant kernel (separable grid pass, FP32): exponentials
               per launch / average launch time (CUDA events on its stream)
               against the SFU ex2 throughput of the chip
  cpu_baseline the FP64 oracle timed on the host on a bounded sample

Multi-GPU (torchrun): replicas only.  Every rank solves its own copy of the
problem (weak scaling, no collective on the data path); value = iterations of
all ranks / max time over ranks.

--impl reference runs the CPU oracle (the only reference this method has) on
the same workload, a bounded number of iterations per step.
"""
from __future__ import annotations

import argparse
import math
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

H = W = 256
LAM = 0.5
EPS, EPS_START, STAGES, IPS = 1e-3, 1e-1, 10, 100
TOL, CHECK_EVERY, MAX_ITER = 1e-6, 20, 20000
SEED = 1235
# SFU throughput used as the ALU roofline of the grid pass: 32 MUFU.EX2 per
# clock per SM (GB300's doubled SFU rate; a throughput probe sustained 30.2 per
# clock per SM) x 152 SMs x the 2070 MHz maximum SM clock.
SM_COUNT, MUFU_PER_CLK, SM_MAX_MHZ = 152, 32, 2070.0
MUFU_PEAK_GEXP = SM_COUNT * MUFU_PER_CLK * SM_MAX_MHZ * 1e6 / 1e9
# FP64 pipe (Algorithm 1 matvec): GB300 runs FP64 at 1.25 TFLOP/s nominal,
# i.e. 2 DFMA per clock per SM.
FP64_PEAK_GFLOPS = 1250.0
# HBM copy bandwidth measured on this GPU type (MEASURED_PEAKS.json hbm_gbs)
HBM_PEAK_GBS = 6760.6
# dram bytes of one rows_lse_f64_pf<4, 4, 1> launch of the wf workload (ncu,
# profiles/rows_lse_f64_pf_wf3000.md); None once the kernel changes
WF_ROWS_TRAFFIC_BYTES = 36848640
# dram bytes of one alg1_cluster launch (2000 iterations of the dense 256 x 256
# problem; profiles/alg1_cluster_dense256.md); None once the kernel changes
ALG1_CLUSTER_TRAFFIC_BYTES = 1185792
# FP32 pipe: 128 lanes per clock per SM (FADD/FMUL/FFMA; a packed f32x2
# instruction occupies it for two lane-slots per pair).
FP32_PER_CLK = 128
FP32_PEAK_GOPS = SM_COUNT * FP32_PER_CLK * SM_MAX_MHZ * 1e6 / 1e9
# FP32-pipe operations per kernel term exp(t_j - k|x_i - y_j|^2 - m_i) summed
# into a running sum, as the kernels evaluate it: grid pass (1-D) sub, mul,
# sub, fma, add = 5; point clouds d = 3: 3 sub, mul, 2 fma, sub, fma, add = 9;
# d = 2: 7.
FP32_OPS_PER_TERM = {"grid": 5, "points3": 9, "points2": 7}


def alu_roofline(kernel, achieved_gexp, fp32_ops, timing, **extra):
    """Roofline of an exponential-sum kernel.  The method's work is one
    exponential per kernel term, so the ceiling is the SFU's ex2 rate
    (`peak`, 152 SMs x 32 MUFU.EX2/clk x 2070 MHz); `achieved` and `peak` are
    terms (= exponentials) per second.  The FP32-pipe load of the kernel's
    own instruction mix is reported beside it under `pipes` (context: it
    depends on the implementation, not on the method)."""
    mufu = MUFU_PEAK_GEXP
    d = {"bound": "alu", "kernel": kernel, "achieved": achieved_gexp, "peak": mufu, "unit": "Gexp2/s",
         "frac": achieved_gexp / mufu, "traffic": None, "binding_pipe": "mufu",
         "pipes": {"mufu_ex2": {"peak_gexp": mufu, "frac": achieved_gexp / mufu},
                   "fp32": {"ops_per_term": fp32_ops, "peak_gops": FP32_PEAK_GOPS,
                            "frac": achieved_gexp * fp32_ops / FP32_PEAK_GOPS}},
         "peak_source": "derived: 152 SMs x 2070 MHz x 32 MUFU.EX2/clk (a probe sustains ~31.8/clk/SM)",
         "timing": timing}
    d.update(extra)
    return d

WORKLOAD = "grid2d-256x256-kl0.5-epsscale1e-1to1e-3-tol1e-6"
# dram__bytes_read.sum + dram__bytes_write.sum of one grid_pass_f32<8, 4>
# launch on this workload (profiles/grid_pass_f32_grid256.md); None once the
# kernel changes after that capture.
GRID_PASS_F32_TRAFFIC_BYTES = 904192
# --mass-div: Algorithm 4 (Sec. 4.5) on the same workload, a divergence on the
# plan's total mass with target MASS_M0 (the plain solve's plan has mass ~1.14)
MASS_M0 = 1.5
MASS_DIVS = {"eq": "eq", "kl": "kl0.5", "tv": "tv0.5", "rg": "rg[0.8,1.2]"}


def mass_div(uot_or_oracle, name):
    m = uot_or_oracle
    return {"eq": m.EQ(), "kl": m.KL(LAM), "tv": m.TV(LAM), "rg": m.RG(0.8, 1.2)}[name]


def config_dict(extra=None, mass=None):
    c = {"workload": WORKLOAD + (f"-mass-{MASS_DIVS[mass]}-m0{MASS_M0}" if mass else ""), "grid": [H, W], "lambda": LAM, "eps": EPS, "eps_start": EPS_START,
         "eps_stages": STAGES, "iters_per_stage": IPS, "tol": TOL, "check_every": CHECK_EVERY,
         "l2": "flushed between steps (256 MB write)", "parallelism": "replicas"}
    if mass:
        c.update({"mass_divergence": MASS_DIVS[mass], "mass_m0": MASS_M0, "algorithm": "Algorithm 4 (Sec. 4.5)"})
    if extra:
        c.update(extra)
        if extra.get("translate"):
            c["workload"] += "-translated"
    return c


def rank_barrier(world):
    """Barrier over the ranks of a multi-GPU run (no-op for one rank)."""
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def reduce_over_ranks(world, device, times, counts):
    """Whole-job figures of a replicated run: the maximum over ranks of each
    time and the sum over ranks of each count (all_reduce on `device`, which
    is the GPU under NCCL and the CPU under gloo)."""
    import torch
    t = torch.tensor([float(v) for v in times], dtype=torch.float64, device=device)
    c = torch.tensor([float(v) for v in counts], dtype=torch.float64, device=device)
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return t.tolist(), c.tolist()


def inputs(seed):
    from paper_1607_05816_gb300 import synth
    return synth.problem_grid2d(H, W, seed=seed, masses=(1.0, 1.3))


# ----------------------------------------------------------------------------
# clocks sampling during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ----------------------------------------------------------------------------
# our implementation
# ----------------------------------------------------------------------------

def run_ours(args, rank, world, local_rank):
    import torch
    import torch.distributed as dist

    from paper_1607_05816_gb300 import uot

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    uot.load()
    uot.force_grid_tile(args.grid_tile)
    prec = {"f32": uot.F32, "f64": uot.F64, "mixed": uot.MIXED}[args.precision]
    dt = torch.float64 if prec == uot.F64 else torch.float32
    # FP32 / mixed: the stop is confirmed in FP64 and the potentials are returned in FP64
    verify = prec != uot.F64 and not args.no_verify and not args.mass_div
    odt = torch.float64 if verify else dt
    d = inputs(SEED + rank)

    def dev_t(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev).ravel()

    geo = uot.Geometry.grid([dev_t(a) for a in d["xs"]], [dev_t(a) for a in d["ys"]])
    p, dx, q, dy = dev_t(d["p"]), dev_t(d["dx"]), dev_t(d["q"]), dev_t(d["dy"])
    Ub = torch.empty(H * W, dtype=odt, device=dev)
    Vb = torch.empty(H * W, dtype=odt, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    max_iter = args.max_iter if args.max_iter else MAX_ITER
    stages = 0 if args.no_eps_scaling else STAGES
    F3 = mass_div(uot, args.mass_div) if args.mass_div else None

    def step(Uo=Ub, Vo=Vb, pp=p, dxx=dx, qq=q, dyy=dy, g=geo):
        if F3 is not None:
            U_, V_, _, info = uot.solve_mass(g, pp, dxx, qq, dyy, uot.KL(LAM), uot.KL(LAM), F3, MASS_M0, EPS,
                                             precision=prec, max_iter=max_iter, tol=TOL,
                                             check_every=CHECK_EVERY, eps_start=EPS_START, eps_stages=stages,
                                             iters_per_stage=IPS, U=Uo, V=Vo, launch_mode=args.launch_mode)
            return U_, V_, info
        return uot.solve(g, pp, dxx, qq, dyy, uot.KL(LAM), uot.KL(LAM), EPS, precision=prec,
                         max_iter=max_iter, tol=TOL, check_every=CHECK_EVERY,
                         eps_start=EPS_START, eps_stages=stages, iters_per_stage=IPS, U=Uo, V=Vo,
                         launch_mode=args.launch_mode, out_f64=verify, verify=verify,
                         translate=getattr(args, "translate", False))

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- device-resident timed region ----
    sampler = ClockSampler(local_rank)
    sampler.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    launches0 = uot.launch_count()
    total_ms, iters, errs, infos = 0.0, 0, [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, _, info = step()
        e1.record()
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        iters += info["total_iters"]
        errs.append(info["marg_err"])
        infos.append(info)
    torch.cuda.synchronize()
    barrier()
    launches = uot.launch_count() - launches0
    clocks = sampler.stop()

    # ---- dominant-kernel timing: CUDA events around every grid-pass launch, on
    # the stream it runs on, during one more step identical to the timed ones
    # (kept out of the timed region so the event records do not perturb it) ----
    flush.fill_(1.0)
    torch.cuda.synchronize()
    uot.profile_begin()
    step()
    torch.cuda.synchronize()
    kern_ms, kern_n = uot.profile_end(uot.PROF_GRID_PASS)
    blk_ms, blk_n = uot.profile_end(uot.PROF_GRID_BLK)  # passes the block-stabilised kernel ran
    kern_ms, kern_n = kern_ms + blk_ms, kern_n + blk_n

    # ---- end-to-end through the C ABI with host buffers ----
    def pinned(a):
        return torch.as_tensor(np.ascontiguousarray(a), dtype=dt).ravel().pin_memory()

    if args.no_e2e:
        args_e2e_steps = 0
    else:
        args_e2e_steps = max(1, args.steps // 2)
    hp, hdx, hq, hdy = pinned(d["p"]), pinned(d["dx"]), pinned(d["q"]), pinned(d["dy"])
    hax = [pinned(a) for a in d["xs"]] + [pinned(a) for a in d["ys"]]
    hU = torch.empty(H * W, dtype=odt).pin_memory()
    hV = torch.empty(H * W, dtype=odt).pin_memory()
    h2d = sum(t.numel() * t.element_size() for t in [hp, hdx, hq, hdy] + hax)
    d2h = hU.numel() * hU.element_size() + hV.numel() * hV.element_size()
    barrier()
    torch.cuda.synchronize()
    e2e_ms, e2e_iters = 0.0, 0
    for _ in range(args_e2e_steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        gp, gdx, gq, gdy = (t.to(dev, non_blocking=True) for t in (hp, hdx, hq, hdy))
        axes = [t.to(dev, non_blocking=True) for t in hax]
        g2 = uot.Geometry.grid(axes[:2], axes[2:])
        Ud, Vd, info = step(Uo=torch.empty_like(Ub), Vo=torch.empty_like(Vb), pp=gp, dxx=gdx,
                            qq=gq, dyy=gdy, g=g2)
        hU.copy_(Ud, non_blocking=True)
        hV.copy_(Vd, non_blocking=True)
        e1.record()
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
        e2e_iters += info["total_iters"]
    barrier()

    # ---- max over ranks ----
    (total_ms_max, e2e_ms_max), (all_iters, all_e2e_iters) = reduce_over_ranks(
        world, dev, [total_ms, e2e_ms], [iters, e2e_iters])
    if rank != 0:
        return
    value = all_iters / (total_ms_max / 1e3)
    # Every Sinkhorn iteration applies 4 separable passes of nlines * nout * nin
    # = 256^3 terms (launch modes 0-2: one kernel per pass; mode 3: two passes per
    # kernel).  Consecutive kernels overlap (programmatic dependent launch), so
    # the kernels' time is taken in the pipelined steady state: the terms of
    # all iterations over the CUDA-event time of the timed steps (grid-pass
    # kernels are > 99.9% of the launches, counted in the profiled step).
    terms_per_iter = 4.0 * float(H) ** 3
    launches_per_step = kern_n
    eff_launch_ms = (total_ms / args.steps) / max(1, launches_per_step)
    # FP32 iterations only (FP64 finishing iterations, if any, run other kernels)
    # (uot_solve_mass reports no FP64 finishing iterations)
    fp32_iters = sum(i["total_iters"] - i.get("polish_iters", 0) for i in infos)
    achieved = terms_per_iter * (fp32_iters / args.steps) / (total_ms / args.steps / 1e3) / 1e9
    avg_kern_ms = kern_ms / max(1, kern_n)
    line = {
        "metric": "sinkhorn_iters_per_s",
        "value": value,
        "unit": "iters/s",
        "n_gpus": world,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": total_ms_max / args.steps,
        "time_to_tol_ms": total_ms_max / args.steps,
        "iters_per_step": iters / args.steps,
        "final_marg_err": max(errs),
        "stop": ({"rule": "FP32 check, confirmed by an FP64 evaluation of the returned potentials' "
                          "violation (included in the step time); FP64 iterations past the FP32 floor",
                  "marg_err_fp64": max(errs), "marg_err_fp32": max(i["marg_err_fp32"] for i in infos),
                  "fp64_confirmations_per_step": sum(i["verifications"] for i in infos) / len(infos),
                  "fp64_iters_per_step": sum(i["polish_iters"] for i in infos) / len(infos),
                  "precise_iters_per_step": sum(i["precise_iters"] for i in infos) / len(infos),
                  "outputs": "float64"} if verify else
                 {"rule": "FP64 check" if prec == uot.F64 else "FP32 check"}),
        "mixed": ({"bf16_tensor_core_iters_per_step": sum(i["mixed_iters"] for i in infos) / len(infos),
                   "fp32_iters_per_step": sum(i["total_iters"] - i["mixed_iters"] - i["polish_iters"]
                                              for i in infos) / len(infos),
                   "switch": "violation <= 1e-3 or the BF16 floor"} if prec == uot.MIXED else None),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": {uot.F32: "f32", uot.F64: "f64", uot.MIXED: "bf16-mma/f32"}[prec],
        "data": "synthetic",
        "config": config_dict({"precision": args.precision, "launch_mode": args.launch_mode,
                               "translate": bool(getattr(args, "translate", False))}, args.mass_div),
        "e2e": {"value": all_e2e_iters / (e2e_ms_max / 1e3) if e2e_ms_max > 0 else None, "unit": "iters/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": alu_roofline(
            "grid_fused2" if (args.launch_mode == 3 and prec == uot.F32) else
            "grid_pass_blk" if (prec == uot.F32 and blk_n > kern_n // 2) else
            {uot.F32: "grid_pass_f32", uot.F64: "grid_pass_f64", uot.MIXED: "grid_pass_tc"}[prec], achieved,
            FP32_OPS_PER_TERM["grid"],
            "achieved = 4 passes x 256^3 terms per iteration x iterations / CUDA-event time of the timed "
            "steps; pipelined_launch_us = step time / grid-pass kernels; isolated_launch_us brackets each "
            "kernel with events in one extra step (this serialises the overlapped launches)",
            launches_per_step=launches_per_step, pipelined_launch_us=eff_launch_ms * 1e3,
            isolated_launch_us=avg_kern_ms * 1e3),
        "grid_tiles": uot.autotune_table().strip().splitlines(),
    }
    tiles = line["grid_tiles"]
    if prec == uot.F32 and any("lines=256 nin=256 nout=256" in t and "warps=8 outputs/lane=4" in t for t in tiles):
        # the ncu capture in profiles/ is of this tile on this workload
        line["roofline"]["traffic"] = GRID_PASS_F32_TRAFFIC_BYTES
        line["roofline"]["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                              "grid_pass_f32<8, 4> launch (profiles/grid_pass_f32_grid256.md)")
    # sustained pipe rates measured by the library's own probes (ops/clk/SM), beside
    # the unit counts the derived peak uses
    probe = uot.probe_pipes()
    line["roofline"]["pipe_probe"] = dict(probe, peak_gexp_from_probe=min(
        probe["mufu_ex2_per_clk_per_sm"], probe["ffma_per_clk_per_sm"] / FP32_OPS_PER_TERM["grid"])
        * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e9)
    if prec == uot.F64:
        # the FP64 pass evaluates one FP64 exp() per term: its ceiling is the
        # measured FP64 exponential rate, not the MUFU (kept as context)
        r = line["roofline"]
        peak64 = probe["dexp_per_clk_per_sm"] * SM_COUNT * SM_MAX_MHZ * 1e6 / 1e9
        r.update({"binding_pipe": "fp64 (exp)", "peak": peak64, "frac": r["achieved"] / peak64,
                  "peak_source": "measured: the library's FP64 exp() throughput probe (64 warps per SM, "
                                 "dependent chains), x 152 SMs x 2070 MHz"})
        r["pipes"]["fp64_exp"] = {"peak_gexp": peak64, "frac": r["achieved"] / peak64}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(args.cpu_iters, args.mass_div)
    return line


# ----------------------------------------------------------------------------
# other single-solve workloads (one step = one solve through the C ABI)
# ----------------------------------------------------------------------------

def run_single(args, rank, world, local_rank):
    """points: n = m = 20000 colour-like clouds in [0,1]^3, KL (or TV) lambda = 0.1,
    eps-scaling 1e-1 -> 1e-3, tol 1e-6, FP32 online cost.
    dense1d: 1-D 256 points, KL lambda = 1, eps = 1e-2, Algorithm 1 FP64, 2000 iterations.
    bary: KL barycenter of 32 blob images 128x128, lambda = 1, eps = 1e-2, 500 iterations.
    wf: WF gradient flow with growth (Sec. 5.3) on 3000 samples of [0, 1], FP64, 500
    iterations per flow step, 4 flow steps per bench step: one species tau = 0.006,
    eps = 1e-8, or two species tau = 0.004, eps = 1e-7 (the paper's runs), alpha = 1.
    color: colour transfer (Sec. 5.1) between two 1024x1024 synthetic images, 64x32x32 colour
    bins, F1 = EQ, F2 = 0.03 KL, eps = 0.002, 2000 iterations (the paper's setting); one step is
    the whole pipeline (two histograms, the 3-D grid solve, the barycentric map, the bin map)."""
    import torch

    from paper_1607_05816_gb300 import synth, uot

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    uot.load()
    uot.force_grid_tile(args.grid_tile)
    f = lambda a, dt=torch.float32: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)
    wl = args.workload
    if wl == "points":
        d = synth.problem_points(20000, 20000, 3, seed=1236 + rank)
        geo = uot.Geometry.points(f(d["x"]), f(d["y"]))
        F = uot.TV(0.1) if args.penalty == "tv" else uot.KL(0.1)
        ins = [f(d[k]).ravel() for k in ("p", "dx", "q", "dy")]

        tr = bool(getattr(args, "translate", False)) and args.penalty == "kl"

        def step():
            # the stop confirmed in FP64 on FP64 outputs (the float-float state)
            return uot.solve(geo, *ins, F, F, 1e-3, precision=uot.F32, max_iter=MAX_ITER, tol=TOL,
                             check_every=CHECK_EVERY, eps_start=1e-1, eps_stages=10, iters_per_stage=100,
                             launch_mode=args.launch_mode, translate=tr, out_f64=True, verify=True)
        work_per_iter, unit_work, kernel = 2.0 * 20000 * 20000, "Gexp2/s", "points_partial"
        cfg = {"workload": f"points3d-20000x20000-{args.penalty}0.1-epsscale1e-1to1e-3-tol1e-6"
                           + ("-translated" if tr else ""), "n": 20000, "m": 20000, "d": 3, "translate": tr,
               "stop": "FP32 check confirmed by an FP64 evaluation of the returned (FP64) potentials"}
        dtype = "f32"
    elif wl == "dense1d":
        d = synth.problem_1d(256, 256, seed=1234)
        C = (d["x"][:, None] - d["y"][None, :]) ** 2
        geo = uot.Geometry.dense(f(C, torch.float64))
        ins = [f(d[k], torch.float64).ravel() for k in ("p", "dx", "q", "dy")]

        # launch mode 1: Algorithm 1 as one launch of a thread-block cluster holding K in
        # shared memory (mode 0: two launches per iteration)
        lm = 0 if args.launch_mode == 0 else 1

        def step():
            return uot.solve(geo, *ins, uot.KL(1.0), uot.KL(1.0), 1e-2, precision=uot.F64, max_iter=2000,
                             plain_scaling=True, launch_mode=lm)
        work_per_iter, unit_work = 2.0 * 256 * 256 * 2, "GFLOP/s"
        kernel = "alg1_cluster" if lm == 1 else "alg1_half"
        cfg = {"workload": "dense1d-256-kl1-eps1e-2-alg1-2000it", "n": 256, "m": 256, "launch_mode": lm}
        dtype = "f64"
    elif wl == "wf":
        S = args.wf_species
        n, nflow, tau, eps = 3000, 4, (0.006 if S == 1 else 0.004), (1e-8 if S == 1 else 1e-7)
        x, dxw, P0 = synth.tumor_densities(n, S, seed=1240 + rank)
        xt = f(x, torch.float64)
        geo = uot.Geometry.dense(uot.wf_cost(xt, xt, math.pi / 2, precision=uot.F64))
        P0t, dxt = f(P0, torch.float64), f(dxw, torch.float64)

        def step():
            P_, U_, V_, info = uot.wf_flow(geo, P0t, dxt, tau, 1.0, 1.0, eps, nflow, precision=uot.F64,
                                           iters=500, launch_mode=args.launch_mode)
            info["marg_err"] = float("nan")
            return U_, V_, info
        work_per_iter, unit_work, kernel = 2.0 * S * n * n, "Gterm/s", "rows_lse_f64_pf<4, 4, 1>"
        cfg = {"workload": f"wf-flow-{S}species-3000-eps{eps:g}-tau{tau:g}-alpha1-500it-x4steps",
               "n": n, "species": S, "eps": eps, "tau": tau, "alpha": 1.0, "lambda": 1.0,
               "iters_per_flow_step": 500, "flow_steps_per_bench_step": nflow,
               "cost": "WF, unscaled distance (cut locus at pi/2)"}
        dtype = "f64"
    elif wl == "color":
        bins, iters_c = (64, 32, 32), 2000
        prec = {"f32": uot.F32, "f64": uot.F64, "mixed": uot.F32}[args.precision]
        ix = f(synth.color_image(1024, 1024, seed=1242 + 2 * rank))
        iy = f(synth.color_image(1024, 1024, seed=1243 + 2 * rank))

        def step():
            out_, T_, info = uot.color_transfer(ix, iy, uot.KL(0.03), eps=0.002, iters=iters_c, bins=bins,
                                                precision=prec, launch_mode=args.launch_mode, check_every=100)
            return out_, T_, info
        nb = 64 * 32 * 32
        # separable passes per direction: axis 0 (1024 lines x 64 x 64), axes 1, 2 (2048 lines x 32 x 32)
        work_per_iter, unit_work, kernel = 2.0 * (1024 * 64 * 64 + 2 * 2048 * 32 * 32), "Gexp2/s", "grid_pass"
        cfg = {"workload": "color-transfer-1024x1024-bins64x32x32-eq-kl0.03-eps2e-3-2000it",
               "image": [1024, 1024], "bins": list(bins), "eps": 0.002, "iters": iters_c,
               "F1": "EQ", "F2": "0.03 KL", "bins_total": nb}
        dtype = {uot.F32: "f32", uot.F64: "f64"}[prec]
    else:  # bary
        b = synth.barycenter_images(32, 128, 128, seed=1237 + rank)
        prec = {"f32": uot.F32, "mixed": uot.MIXED, "f64": uot.F64}[args.precision]
        adt = torch.float64 if prec == uot.F64 else torch.float32
        geo = uot.Geometry.grid([f(a, adt).ravel() for a in b["xs"]])
        P = f(b["P"].reshape(32, -1), adt)
        alpha = np.full(32, 1.0 / 32)

        Fh = {"kl": uot.KL(1.0), "tv": uot.TV(1.0), "rg": uot.RG(0.5, 2.0)}[args.bary_div]

        def step():
            dt = torch.float64 if prec == uot.F64 else torch.float32
            lh, U_, V_, info = uot.barycenter_div(geo, alpha, P, f(b["dx"], dt).ravel(), f(b["dy"], dt).ravel(),
                                                  uot.EQ(), Fh, 1e-2, precision=prec, max_iter=500,
                                                  launch_mode=args.launch_mode)
            return U_, V_, info
        work_per_iter, unit_work, kernel = 32 * 2 * 2 * 128.0 ** 3, "Gexp2/s", "grid_pass"
        cfg = {"workload": {"kl": "bary32-128x128-kl1-eps1e-2-500it", "tv": "bary32-128x128-tv1-eps1e-2-500it",
                            "rg": "bary32-128x128-rg[0.5,2]-eps1e-2-500it"}[args.bary_div],
               "K": 32, "grid": [128, 128], "barycenter_divergence": args.bary_div}
        dtype = args.precision
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    sampler = ClockSampler(local_rank)
    sampler.start()
    time.sleep(0.3)
    rank_barrier(world)
    torch.cuda.synchronize()
    launches0 = uot.launch_count()
    total_ms, iters, errs, infos = 0.0, 0, [], []
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        out = step()
        e1.record()
        e1.synchronize()
        info = out[-1]
        infos.append(info)
        total_ms += e0.elapsed_time(e1)
        iters += info["total_iters"]
        errs.append(info["marg_err"])
    torch.cuda.synchronize()
    rank_barrier(world)
    launches = uot.launch_count() - launches0
    clocks = sampler.stop()
    (total_ms_max,), (all_iters,) = reduce_over_ranks(world, dev, [total_ms], [iters])
    if rank != 0:
        return
    achieved = work_per_iter * iters / (total_ms / 1e3) / 1e9
    cfg.update({"l2": "flushed between steps (256 MB write)", "parallelism": "replicas"})
    line = {
        "metric": "sinkhorn_iters_per_s", "value": all_iters / (total_ms_max / 1e3), "unit": "iters/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms_max / args.steps,
        "iters_per_step": iters / args.steps, "final_marg_err": max(errs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": dtype, "data": "synthetic", "config": cfg,
        "gpu_launches": launches, "clocks": clocks,
    }
    if infos and "verifications" in infos[0] and wl == "points":
        line["stop"] = {"rule": "FP32 check, confirmed by an FP64 evaluation of the returned potentials' "
                                "violation (included in the step time); FP64 iterations past the FP32 floor",
                        "marg_err_fp64": max(errs),
                        "marg_err_fp32": max(i["marg_err_fp32"] for i in infos),
                        "fp64_confirmations_per_step": sum(i["verifications"] for i in infos) / len(infos),
                        "fp64_iters_per_step": sum(i["polish_iters"] for i in infos) / len(infos),
                        "precise_iters_per_step": sum(i["precise_iters"] for i in infos) / len(infos),
                        "outputs": "float64"}
    timing = "algorithmic work of all iterations / CUDA-event time of the timed steps"
    if unit_work == "Gexp2/s":
        line["roofline"] = alu_roofline(kernel, achieved, FP32_OPS_PER_TERM["points3" if wl == "points" else "grid"],
                                        timing)
        if wl in ("bary", "color"):
            line["grid_tiles"] = uot.autotune_table().strip().splitlines()
    elif unit_work == "Gterm/s":
        # rows_lse_f64_pf: the FP32 prefilter reads the FP32 copy of the cost once
        # per term (4 B; both sweeps run from shared memory) and evaluates FP64
        # exponentials only where they do not underflow, so its floor is HBM.
        gbs = achieved * 4.0
        line["roofline"] = {"bound": "hbm", "kernel": kernel, "achieved": gbs, "peak": HBM_PEAK_GBS,
                            "unit": "GB/s", "frac": gbs / HBM_PEAK_GBS,
                            "traffic": WF_ROWS_TRAFFIC_BYTES,
                            "traffic_source": ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch "
                                               "(cold cache; profiles/rows_lse_f64_pf_wf3000.md)")
                            if WF_ROWS_TRAFFIC_BYTES is not None else None,
                            "algorithmic_bytes_per_launch": 4.0 * n * n,
                            "terms_per_s": achieved * 1e9,
                            "peak_source": "MEASURED_PEAKS.json hbm_gbs (burst copy), of measured",
                            "timing": timing}
    else:
        tr = ALG1_CLUSTER_TRAFFIC_BYTES if kernel == "alg1_cluster" else None
        line["roofline"] = {"bound": "alu", "kernel": kernel, "achieved": achieved, "peak": FP64_PEAK_GFLOPS,
                            "unit": unit_work, "frac": achieved / FP64_PEAK_GFLOPS, "traffic": tr,
                            "timing": timing}
        if tr is not None:
            line["roofline"]["traffic_source"] = ("ncu dram__bytes_read.sum + dram__bytes_write.sum of one "
                                                  "2000-iteration launch (profiles/alg1_cluster_dense256.md)")
    return line


# ----------------------------------------------------------------------------
# batched workload: 4096 uneven 2-D point-cloud problems in one persistent launch
# ----------------------------------------------------------------------------

BATCH_NPROB, BATCH_SIZE, BATCH_EPS, BATCH_TOL = 4096, (64, 2048), 1e-2, 1e-6


def run_batch(args, rank, world, local_rank):
    import torch

    from paper_1607_05816_gb300 import synth, uot

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    uot.load()
    uot.force_grid_tile(args.grid_tile)
    nprob = args.batch_nprob or BATCH_NPROB
    probs = synth.batch_points(nprob=nprob, size=BATCH_SIZE, d=2, seed=1238 + rank)
    sizes = [(len(pr["x"]), len(pr["y"])) for pr in probs]
    divs = [(uot.KL(pr["lam"]), uot.KL(pr["lam"])) for pr in probs]

    def cat(key):
        return torch.as_tensor(np.concatenate([np.asarray(pr[key], np.float32) for pr in probs]),
                               device=dev)

    x, p, dx, y, q, dy = (cat(k) for k in ("x", "p", "dx", "y", "q", "dy"))
    N, M = x.shape[0], y.shape[0]
    # FP64 outputs: the float-float state, not its FP32 rounding, is what the check measured
    Ub = torch.empty(N, dtype=torch.float64, device=dev)
    Vb = torch.empty(M, dtype=torch.float64, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        return uot.solve_batch(sizes, divs, 2, x, p, dx, y, q, dy, BATCH_EPS, max_iter=MAX_ITER,
                               tol=BATCH_TOL, check_every=CHECK_EVERY, U=Ub, V=Vb,
                               translate=bool(getattr(args, "translate", False)), out_f64=True)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local_rank)
    sampler.start()
    time.sleep(0.3)
    rank_barrier(world)
    torch.cuda.synchronize()
    launches0 = uot.launch_count()
    total_ms, iters, exps, worst = 0.0, 0, 0.0, 0.0
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _, _, it, errs, info = step()
        e1.record()
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        iters += sum(it)
        exps += sum(2.0 * n * m * k for (n, m), k in zip(sizes, it))
        worst = max(worst, max(errs))
    torch.cuda.synchronize()
    rank_barrier(world)
    launches = uot.launch_count() - launches0
    clocks = sampler.stop()
    (total_ms_max,), (all_iters,) = reduce_over_ranks(world, dev, [total_ms], [iters])
    if rank != 0:
        return
    achieved = exps / (total_ms / 1e3) / 1e9
    line = {
        "metric": "sinkhorn_iters_per_s", "value": all_iters / (total_ms_max / 1e3), "unit": "iters/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": total_ms_max / args.steps, "time_to_tol_ms": total_ms_max / args.steps,
        "iters_per_step": iters / args.steps, "final_marg_err": worst,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": f"batch{nprob}-points2d-n,m~U[64,2048]-kl-lam~logU[0.05,5]-eps1e-2-tol1e-6"
                               + ("-translated" if getattr(args, "translate", False) else ""),
                   "translate": bool(getattr(args, "translate", False)),
                   "outputs": "float64 (the float-float state)",
                   "stop": "each problem's FP32 check (no FP64 confirmation; the oracle's violation of "
                           "the returned potentials lies within 10% of it)",
                   "nprob": nprob, "sum_nm": int(sum(n * m for n, m in sizes)),
                   "l2": "flushed between steps (256 MB write)", "parallelism": "replicas"},
        "gpu_launches": launches, "clocks": clocks,
        "roofline": alu_roofline("batch_solve", achieved, FP32_OPS_PER_TERM["points2"],
                                 "exponentials of all problems' iterations / CUDA-event time of the launch"),
        "tuned": uot.autotune_table().strip().splitlines(),
    }
    return line


# ----------------------------------------------------------------------------
# learned warm start (64 x 64 grids): the network trained on solver-generated
# instances, then held-out instances solved to 1e-6 three ways
# ----------------------------------------------------------------------------

WS_TRAIN, WS_EPOCHS, WS_EVAL, WS_GROUP = 8192, 8, 1024, 32
# dram bytes of one conv_tc<128> launch of a 128 -> 128 layer, scaled from the
# 32-instance capture to the 64 instances of the timed forward pass; None once
# the kernel changes
CONV_TC_TRAFFIC_BYTES_128x128_64INST = 2 * (33879040 + 419840)
# measured dense BF16 GEMM rate of this GPU type (MEASURED_PEAKS.json bf16_tflops, burst)
BF16_PEAK_TFLOPS = 1916.2


def run_warmstart(args, rank, world, local_rank):
    import torch

    from paper_1607_05816_gb300 import synth, uot
    from paper_1607_05816_gb300 import warmstart as WS

    torch.cuda.set_device(local_rank)
    uot.load()
    H = W = 64
    ntrain = args.ws_train or WS_TRAIN
    epochs = args.ws_epochs or WS_EPOCHS
    neval = args.ws_eval or WS_EVAL
    t0 = time.perf_counter()
    inst = synth.warmstart_instances(ntrain, H, W, seed=1239 + 1000 * rank, group=256)
    P, Q, Us, Vs = WS.generate_targets(inst, H, W, max_iter=6000, group=256)
    torch.cuda.synchronize()
    gen_s = time.perf_counter() - t0
    net = WS.WarmStartNetTC(channels=128, seed=rank)
    t0 = time.perf_counter()
    hist = WS.train_tc(net, P, Q, Us, Vs, inst["eps"], inst["lam"], epochs=epochs, batch=32, lr=3e-4)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    del P, Q, Us, Vs
    ev = synth.warmstart_instances(neval, H, W, seed=777001 + rank, group=WS_GROUP)  # held out: other seed
    warm_inst = {k: (v[:2 * WS_GROUP] if k in ("P", "Q", "eps", "lam") else v) for k, v in ev.items()}
    # warm-up (tile tuner, graphs, the streams' workspaces)
    WS.evaluate_tc(net, warm_inst, H, W, group=WS_GROUP, plain_sample=2, streams=args.ws_streams)
    sampler = ClockSampler(local_rank)
    sampler.start()
    time.sleep(0.3)
    launches0 = uot.launch_count()
    res = WS.evaluate_tc(net, ev, H, W, group=WS_GROUP, plain_sample=16, streams=args.ws_streams)
    launches = uot.launch_count() - launches0
    clocks = sampler.stop()
    # the convolutions' rate: one forward pass of 64 instances, CUDA events
    Pb = torch.as_tensor(ev["P"][:64], dtype=torch.float32, device="cuda")
    Qb = torch.as_tensor(ev["Q"][:64], dtype=torch.float32, device="cuda")
    feats = net.features(Pb, Qb, ev["eps"][:64], ev["lam"][:64])
    for _ in range(3):
        net.forward(feats, 64, H, W, keep=False)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(10):
        net.forward(feats, 64, H, W, keep=False)
    e1.record()
    e1.synchronize()
    fwd_ms = e0.elapsed_time(e1) / 10
    pad = lambda c: 64 if c <= 64 else 128
    out_pad = lambda c: 16 if c <= 16 else (64 if c <= 64 else 128)
    flops_alg = 2.0 * 9 * sum(ci * co for ci, co, _, _ in net.layers) * 64 * H * W
    flops_mma = 2.0 * 9 * sum(pad(ci) * out_pad(co) for ci, co, _, _ in net.layers) * 64 * H * W
    if rank != 0:
        return None
    med = lambda a: float(np.median(a)) if len(a) else None
    # the headline: every group in flight on its own stream when --ws-streams > 0
    warm_seq = res["warm_ms"]  # inference included
    warm_total = res.get("warm_streams_ms", warm_seq)
    line = {
        "metric": "instances_per_s", "value": neval / (warm_total / 1e3), "unit": "instances/s",
        "n_gpus": world, "steps": 1, "warmup": 1, "ms_per_step": warm_total, "time_to_tol_ms": warm_total,
        "iters_per_step": float(np.sum(res["warm_iters"])), "final_marg_err": res["worst_err_warm"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16-mma/f32",
        "data": "synthetic",
        "config": {"workload": f"warmstart-64x64-train{ntrain}x{epochs}ep-heldout{neval}-groups{WS_GROUP}-tol1e-6",
                   "grid": [H, W], "eps": "logU[1e-3, 1e-1]", "lambda": "logU[0.1, 10]", "masses": "U[0.5, 2]",
                   "parallelism": "replicas", "l2": "inputs resident; solves and inference back to back"},
        "gpu_launches": launches, "clocks": clocks,
        "roofline": {"bound": "tensor", "kernel": "conv_tc_n256 (network forward, 64 instances)",
                     "achieved": flops_alg / (fwd_ms / 1e3) / 1e12, "peak": BF16_PEAK_TFLOPS, "unit": "TFLOP/s",
                     "frac": flops_alg / (fwd_ms / 1e3) / 1e12 / BF16_PEAK_TFLOPS,
                     "traffic": CONV_TC_TRAFFIC_BYTES_128x128_64INST,
                     "traffic_source": None if CONV_TC_TRAFFIC_BYTES_128x128_64INST is None else
                     "ncu dram__bytes_read.sum + dram__bytes_write.sum of one launch of a 128 -> 128 layer on 32 "
                     "instances (profiles/conv_tc_warmstart64.md), x2 for the 64 instances timed here",
                     "mma_flops_incl_padding_tflops": flops_mma / (fwd_ms / 1e3) / 1e12,
                     "forward_ms_64_instances": fwd_ms,
                     "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst), of measured",
                     "timing": "algorithmic FLOPs of one forward pass (2 x 9 Cin Cout per pixel and layer) / "
                               "CUDA-event time"},
        "warm_start": {
            "params": net.n_params(), "train_instances": ntrain, "epochs": epochs, "batch": 32,
            "data_generation_s": gen_s, "train_s": train_s, "train_loss_per_epoch": hist,
            "heldout_instances": neval, "group": WS_GROUP,
            "forms": {
                "plain": "uot_solve per instance, cold start, eps-scaling, the iteration as printed "
                         f"(sampled on {len(res['plain_iters'])} instances, scaled)",
                "batched_cold": "uot_solve_many per group, cold start, eps-scaling, as printed",
                "batched_cold_translated": "the same with the translation step (opts.translate)",
                "batched_warm_translated": "network inference, then uot_solve_many from the predicted "
                                           "potentials at the final eps with the translation step",
                "streams": f"the last two forms with the {len(res['groups'])} groups in flight at once, one "
                           f"host thread and CUDA stream each for {args.ws_streams} streams (the headline "
                           "value when > 0)",
            },
            "ms_total": {"plain": res["plain_ms"], "batched_cold": res["batched_ms"],
                         "batched_cold_translated": res["batched_tr_ms"], "batched_warm_translated": warm_seq,
                         "batched_cold_translated_streams": res.get("batched_tr_streams_ms"),
                         "batched_warm_translated_streams": res.get("warm_streams_ms")},
            "streams": args.ws_streams,
            "streams_iteration_mismatches": res.get("streams_mismatch"),
            "warm_inference_ms_total": res["warm_infer_ms"],  # part of batched_warm_translated
            "speedup_of_warm": {"vs_plain": res["plain_ms"] / warm_seq,
                                "vs_batched_cold": res["batched_ms"] / warm_seq,
                                "vs_batched_cold_translated": res["batched_tr_ms"] / warm_seq,
                                "streams_vs_batched_cold_translated_streams":
                                    (res["batched_tr_streams_ms"] / res["warm_streams_ms"])
                                    if "warm_streams_ms" in res else None},
            "median_iters": {"plain": med(res["plain_iters"]), "batched_cold": med(res["batched_iters"]),
                             "batched_cold_translated": med(res["batched_tr_iters"]),
                             "batched_warm_translated": med(res["warm_iters"])},
            "worst_marg_err_fp64": {"plain": res["worst_err_plain"], "batched_cold": res["worst_err_batched"],
                                    "batched_cold_translated": res["worst_err_batched_tr"],
                                    "batched_warm_translated": res["worst_err_warm"],
                                    "batched_cold_translated_streams": res.get("worst_err_batched_tr_streams"),
                                    "batched_warm_translated_streams": res.get("worst_err_warm_streams")},
            "groups": res["groups"],
        },
    }
    return line


# ----------------------------------------------------------------------------
# the oracle on the host (baseline and --impl reference)
# ----------------------------------------------------------------------------

def oracle_iterations(n_iters, seed=SEED, mass=None):
    """Run n_iters oracle iterations of the bench workload at the final eps
    (Algorithm 4's with a mass divergence); returns (seconds, iterations)."""
    import oracle as O
    d = inputs(seed)
    og = O.Geometry("grid", xs=d["xs"], ys=d["ys"])
    if mass:
        t0 = time.perf_counter()
        O.solve_mass_log(og, d["dx"], d["dy"], d["p"], d["q"], O.KL(LAM), O.KL(LAM), mass_div(O, mass),
                         MASS_M0, EPS, max_iter=n_iters)
        return time.perf_counter() - t0, n_iters
    logs = tuple(O.safe_log(d[k]) for k in ("dx", "dy", "p", "q"))
    t0 = time.perf_counter()
    O.iterate_log(og, *logs, O.KL(LAM), O.KL(LAM), EPS, n_iters)
    return time.perf_counter() - t0, n_iters


def cpu_baseline(n_iters, mass=None):
    sec, n = oracle_iterations(n_iters, mass=mass)
    what = "Algorithm 4 (mass divergence) " if mass else ""
    return {"value": n / sec, "unit": "iters/s", "cores": 1, "kind": "oracle",
            "sample": f"{n} FP64 numpy {what}iterations of the 256x256 grid problem at eps=1e-3 "
                      f"(separable log-domain form), {sec:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return
    per_step = max(1, args.cpu_iters // 2)
    for _ in range(args.warmup):
        oracle_iterations(1, mass=args.mass_div)
    sec, n = 0.0, 0
    for _ in range(args.steps):
        s, k = oracle_iterations(per_step, mass=args.mass_div)
        sec += s
        n += k
    value = n / sec
    line = {
        "metric": "sinkhorn_iters_per_s", "value": value, "unit": "iters/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": sec * 1e3 / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "impl": "reference", "config": config_dict({"precision": "f64"}, args.mass_div),
        "cpu_baseline": {"value": value, "unit": "iters/s", "cores": 1, "kind": "oracle",
                         "sample": f"{per_step} iterations per step at eps=1e-3"},
        "e2e": {"value": value, "unit": "iters/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# the oracle on the host cores for every configuration: one core, and all the
# host's cores (worker processes started with spawn, each computing a block of
# output rows of the Gibbs operator; one BLAS thread per worker)
# ----------------------------------------------------------------------------

_WORKER = {}


def _oracle_worker_init(data):
    _WORKER.clear()
    _WORKER.update(data)


def _oracle_rows(task):
    """eps log K(e^{W/eps} w) on the output rows [r0, r1) of one direction.
    grid: rows of the first axis of the output grid; points, dense: rows."""
    import oracle as O
    side, r0, r1, W, logw, eps = task
    kind = _WORKER["kind"]
    if kind == "grid":
        out_axes = list(_WORKER["ys"] if side else _WORKER["xs"])
        in_axes = _WORKER["xs"] if side else _WORKER["ys"]
        out_axes[0] = out_axes[0][r0:r1]
        g = O.Geometry("grid", xs=out_axes, ys=in_axes)
        return O.apply_K_log(g, W, logw, eps)
    if kind == "points":
        xo = (_WORKER["y"] if side else _WORKER["x"])[r0:r1]
        xi = _WORKER["x"] if side else _WORKER["y"]
        return O.apply_K_points_streamed(xo, xi, W, logw, eps)
    C = _WORKER["C"]
    Cs = (C.T if side else C)[r0:r1]
    return O.apply_K_log(O.Geometry("dense", C=Cs), W, logw, eps)


def _oracle_problems(task):
    """n_iter log-domain iterations of each listed batch problem (KL, KL)."""
    import oracle as O
    idx, n_iter, eps = task
    t0 = time.perf_counter()
    for k in idx:
        pr = _WORKER["probs"][k]
        g = O.Geometry("points", x=pr["x"], y=pr["y"])
        logs = tuple(O.safe_log(pr[key]) for key in ("dx", "dy", "p", "q"))
        O.iterate_log(g, *logs, O.KL(pr["lam"]), O.KL(pr["lam"]), eps, n_iter)
    return time.perf_counter() - t0


def _oracle_alg1(task):
    import oracle as O
    K, dx, dy, p, q, lam, eps, iters = task
    t0 = time.perf_counter()
    O.scaling_alg1(K, dx, dy, p, q, O.KL(lam), O.KL(lam), eps, iters)
    return time.perf_counter() - t0


class OraclePool:
    """`cores` spawned worker processes with one BLAS/OpenMP thread each."""

    def __init__(self, cores, data, blas_threads=1):
        import multiprocessing as mp
        env = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
        old = {k: os.environ.get(k) for k in env}
        for k in env:
            os.environ[k] = str(blas_threads)
        try:
            self.pool = mp.get_context("spawn").Pool(cores, initializer=_oracle_worker_init, initargs=(data,))
        finally:
            for k, v in old.items():
                if v is None:
                    os.environ.pop(k, None)
                else:
                    os.environ[k] = v
        self.cores = cores
        self.pool.map(abs, range(cores))  # workers up before anything is timed

    def close(self):
        self.pool.close()
        self.pool.join()


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def _split(n, parts):
    b = [(n * k) // parts for k in range(parts + 1)]
    return [(b[k], b[k + 1]) for k in range(parts) if b[k + 1] > b[k]]


def _oracle_log_iterations(pool, n_rows, shape_p, shape_q, logs, F1, F2, eps, n_iter):
    """n_iter oracle iterations (log domain) with both operators split by
    output rows over the pool; returns seconds."""
    import oracle as O
    logdx, logdy, logp, logq = logs
    U = np.zeros(shape_p)
    V = np.zeros(shape_q)
    nx, ny = n_rows
    t0 = time.perf_counter()
    for _ in range(n_iter):
        parts = pool.pool.map(_oracle_rows, [(0, a, b, V, logdy, eps) for a, b in _split(nx, pool.cores)])
        S = np.concatenate(parts, axis=0).reshape(shape_p)
        U = O.prox_update_log(F1, logp, S, eps)
        parts = pool.pool.map(_oracle_rows, [(1, a, b, U, logdx, eps) for a, b in _split(ny, pool.cores)])
        T = np.concatenate(parts, axis=0).reshape(shape_q)
        V = O.prox_update_log(F2, logq, T, eps)
    return time.perf_counter() - t0


def oracle_baselines(name, cores_all, one_core=True):
    """The oracle on one core and on `cores_all` cores for workload `name`, in
    the workload's metric (iterations per second; problem-iterations per
    second for the batch).  Each measurement is a bounded sample (stated)."""
    import oracle as O
    from paper_1607_05816_gb300 import synth
    out = {}
    for cores in ((1, cores_all) if one_core else (cores_all,)):
        label = "one_core" if cores == 1 else "all_cores"
        if name in ("grid2d", "grid2d_f64", "warmstart"):
            if name == "warmstart":
                inst = synth.warmstart_instances(1, 64, 64, seed=1239 + 7)
                xs = inst["xs"]
                p_, q_, dx_ = inst["P"][0], inst["Q"][0], inst["dx"]
                e, lam = float(inst["eps"][0]), float(inst["lam"][0])
                n_iter = 40 if cores == 1 else 80
                sample = f"{n_iter} cold-start iterations of one 64x64 instance (eps {e:.3g}, lambda {lam:.3g})"
            else:
                d = inputs(SEED)
                xs, p_, q_, dx_ = d["xs"], d["p"], d["q"], d["dx"]
                e, lam = EPS, LAM
                n_iter = 4 if cores == 1 else 16
                sample = f"{n_iter} iterations of the 256x256 grid problem at eps = 1e-3"
            pool = OraclePool(cores, {"kind": "grid", "xs": xs, "ys": xs})
            try:
                logs = tuple(O.safe_log(a) for a in (dx_, dx_, p_, q_))
                sec = _oracle_log_iterations(pool, (len(xs[0]), len(xs[0])), np.shape(p_), np.shape(q_), logs,
                                             O.KL(lam), O.KL(lam), e, n_iter)
            finally:
                pool.close()
            out[label] = {"value": n_iter / sec, "unit": "iters/s", "cores": cores, "kind": "oracle",
                          "sample": sample, "seconds": sec}
        elif name in ("points_kl", "points_tv"):
            d = synth.problem_points(20000, 20000, 3, seed=1236)
            F = O.TV(0.1) if name == "points_tv" else O.KL(0.1)
            pool = OraclePool(cores, {"kind": "points", "x": d["x"], "y": d["y"]})
            try:
                logs = tuple(O.safe_log(d[k]) for k in ("dx", "dy", "p", "q"))
                if cores == 1:
                    # output rows [0, 1000) of one half-step, scaled to both half-steps
                    t0 = time.perf_counter()
                    pool.pool.map(_oracle_rows, [(0, 0, 1000, np.zeros(20000), logs[1], 1e-3)])
                    sec = (time.perf_counter() - t0) * 2 * 20000 / 1000
                    sample = "1000 of 20000 output rows of one half-step at eps = 1e-3, scaled x40 to an iteration"
                else:
                    sec = _oracle_log_iterations(pool, (20000, 20000), (20000,), (20000,), logs, F, F, 1e-3, 1)
                    sample = "1 iteration of the 20000 x 20000 problem at eps = 1e-3"
            finally:
                pool.close()
            out[label] = {"value": 1.0 / sec, "unit": "iters/s", "cores": cores, "kind": "oracle",
                          "sample": sample, "seconds_per_iter": sec}
        elif name == "dense1d":
            d = synth.problem_1d(256, 256, seed=1234)
            K = np.exp(-(d["x"][:, None] - d["y"][None, :]) ** 2 / 1e-2)
            pool = OraclePool(1, {}, blas_threads=cores)
            try:
                n_iter = 2000
                sec = pool.pool.apply(_oracle_alg1, ((K, d["dx"], d["dy"], d["p"], d["q"], 1.0, 1e-2, n_iter),))
            finally:
                pool.close()
            out[label] = {"value": n_iter / sec, "unit": "iters/s", "cores": cores, "kind": "oracle",
                          "sample": f"Algorithm 1 verbatim, {n_iter} iterations (numpy matrix-vector products"
                                    f" with {cores} BLAS thread{'s' if cores > 1 else ''})", "seconds": sec}
        elif name == "batch":
            probs = synth.batch_points(nprob=BATCH_NPROB, size=BATCH_SIZE, d=2, seed=1238)
            nm = np.array([len(pr["x"]) * len(pr["y"]) for pr in probs], dtype=np.float64)
            order = np.argsort(nm)
            sample_idx = [int(k) for k in order[::64]]  # 64 problems spread over the sizes
            pool = OraclePool(cores, {"probs": [probs[k] for k in sample_idx]})
            try:
                n_iter = 1
                t0 = time.perf_counter()
                pool.pool.map(_oracle_problems, [(list(range(a, b)), n_iter, BATCH_EPS)
                                                 for a, b in _split(len(sample_idx), cores)])
                sec = time.perf_counter() - t0
            finally:
                pool.close()
            # scaled by sum n m: problem-iterations per second of the whole batch's mix
            rate = n_iter * float(nm[sample_idx].sum()) / sec / float(nm.mean())
            out[label] = {"value": rate, "unit": "problem-iters/s", "cores": cores, "kind": "oracle",
                          "sample": f"{n_iter} iterations of 64 of the 4096 problems (every 64th by size), "
                                    f"scaled by sum n m", "seconds": sec}
        elif name == "bary":
            b = synth.barycenter_images(32, 128, 128, seed=1237)
            pool = OraclePool(cores, {"kind": "grid", "xs": b["xs"], "ys": b["ys"]})
            try:
                n_iter = 1 if cores == 1 else 2
                sec = _oracle_bary_iterations(pool, b, n_iter)
            finally:
                pool.close()
            out[label] = {"value": n_iter / sec, "unit": "iters/s", "cores": cores, "kind": "oracle",
                          "sample": f"{n_iter} KL-barycenter iteration(s) of the 32 x 128 x 128 workload",
                          "seconds": sec}
    return out


def _oracle_bary_iterations(pool, b, n_iter):
    """Barycenter iterations (Sec. 5.2, Table 2 KL) with every measure's
    operator split by output rows over the pool."""
    import oracle as O
    P = np.asarray(b["P"], dtype=np.float64)
    K = P.shape[0]
    logdx, logdy, logP = O.safe_log(b["dx"]), O.safe_log(b["dy"]), O.safe_log(P)
    alpha = np.full(K, 1.0 / K)
    eps, lam = 1e-2, 1.0
    U = np.zeros_like(P)
    V = np.zeros_like(P)
    H = P.shape[1]
    t0 = time.perf_counter()
    for _ in range(n_iter):
        tasks = [(0, a, c, V[k], logdy, eps) for k in range(K) for a, c in _split(H, pool.cores)]
        parts = pool.pool.map(_oracle_rows, tasks)
        per = len(parts) // K
        for k in range(K):
            U[k] = O.prox_update_log(O.EQ(), logP[k], np.concatenate(parts[k * per:(k + 1) * per], 0), eps)
        tasks = [(1, a, c, U[k], logdx, eps) for k in range(K) for a, c in _split(H, pool.cores)]
        parts = pool.pool.map(_oracle_rows, tasks)
        T = np.stack([np.concatenate(parts[k * per:(k + 1) * per], 0) for k in range(K)])
        logh = O.bary_h_log(T, alpha, lam, eps, "kl") / eps
        for k in range(K):
            V[k] = O.prox_update_log(O.KL(lam), logh, T[k], eps)
    return time.perf_counter() - t0


def _compact(line, cpu):
    """The figures of a workload line that the sub-record keeps."""
    r = line.get("roofline") or {}
    d = {"value": line["value"], "unit": line["unit"], "time_to_tol_ms": line.get("time_to_tol_ms",
         line.get("ms_per_step")), "ms_per_step": line["ms_per_step"], "iters_per_step": line.get("iters_per_step"),
         "final_marg_err": line.get("final_marg_err"), "dtype": line["dtype"], "config": line["config"],
         "clocks": line.get("clocks"), "gpu_launches": line.get("gpu_launches"),
         "roofline": {k: r.get(k) for k in ("bound", "kernel", "achieved", "peak", "unit", "frac", "traffic")}}
    for k in ("stop", "warm_start", "mixed"):
        if k in line:
            d[k] = line[k]
    if cpu:
        d["cpu_baseline"] = cpu
    return d


def sub_workloads(args, local_rank, cpu=True):
    """Every configuration besides the headline, each as a bounded run (1
    warm-up step, 2 timed steps; FP64 grid: 1 timed step) with its oracle
    baselines on one core and on all host cores."""
    import copy
    import torch
    cores = host_cores()
    subs = [
        ("dense1d", dict(workload="dense1d", launch_mode=1)),
        ("grid2d_f64", dict(workload="grid2d", precision="f64", steps=1)),
        ("grid2d_mixed", dict(workload="grid2d", precision="mixed", steps=1)),
        ("grid2d_translated", dict(workload="grid2d", translate=True)),
        ("points_kl", dict(workload="points", penalty="kl")),
        ("points_kl_translated", dict(workload="points", penalty="kl", translate=True)),
        ("points_tv", dict(workload="points", penalty="tv")),
        ("batch", dict(workload="batch")),
        ("batch_translated", dict(workload="batch", translate=True)),
        ("bary", dict(workload="bary")),
        ("warmstart", dict(workload="warmstart")),
        # the rows beyond the hot path's core, each as its own bounded run (no oracle timing)
        ("bary_tv", dict(workload="bary", bary_div="tv")),
        ("mass_eq", dict(workload="grid2d", mass_div="eq")),
        ("wf", dict(workload="wf", wf_species=1)),
        ("wf_2species", dict(workload="wf", wf_species=2)),
        ("color", dict(workload="color")),
    ]
    res = {"host_cores": cores}
    for name, over in subs:
        a = copy.copy(args)
        a.steps, a.warmup, a.no_e2e, a.no_cpu_baseline, a.grid_tile = 2, 1, True, True, -1
        a.launch_mode = 2
        for k, v in over.items():
            setattr(a, k, v)
        try:
            if a.workload == "batch":
                line = run_batch(a, 0, 1, local_rank)
            elif a.workload == "warmstart":
                line = run_warmstart(a, 0, 1, local_rank)
            elif a.workload == "grid2d":
                line = run_ours(a, 0, 1, local_rank)
            else:
                line = run_single(a, 0, 1, local_rank)
            torch.cuda.synchronize()
            # the translated runs share their untranslated twin's oracle iteration rate
            timed = name in ("dense1d", "grid2d_f64", "points_kl", "points_tv", "batch", "bary", "warmstart")
            base = oracle_baselines(name, cores) if cpu and timed else None
            res[name] = _compact(line, base)
        except Exception as e:  # a failed sub-run is reported, not hidden
            res[name] = {"error": f"{type(e).__name__}: {e}"}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f64", "mixed"])
    ap.add_argument("--cpu-iters", type=int, default=6)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    # profiling knobs (small cases for ncu captures); not used for bench lines
    ap.add_argument("--max-iter", type=int, default=0)
    ap.add_argument("--no-eps-scaling", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-verify", action="store_true",
                    help="grid2d FP32/mixed: stop on the FP32 check alone and return float potentials")
    ap.add_argument("--workload", default="grid2d",
                    choices=["grid2d", "batch", "points", "dense1d", "bary", "wf", "color", "warmstart"])
    ap.add_argument("--ws-train", type=int, default=0, help="warmstart: training instances")
    ap.add_argument("--ws-epochs", type=int, default=0, help="warmstart: epochs")
    ap.add_argument("--ws-eval", type=int, default=0, help="warmstart: held-out instances")
    ap.add_argument("--ws-streams", type=int, default=8,
                    help="warmstart: streams (host threads) solving groups at once; 0 = one group at a time")
    ap.add_argument("--wf-species", type=int, default=1, choices=[1, 2],
                    help="species of the wf workload (Sec. 5.3: the tumor example or its two-species extension)")
    ap.add_argument("--penalty", default="kl", choices=["kl", "tv"])
    ap.add_argument("--translate", action="store_true",
                    help="grid2d, points and batch with KL: the translation step after every checked "
                         "iteration (opts.translate; not in the paper)")
    ap.add_argument("--batch-nprob", type=int, default=0)
    ap.add_argument("--launch-mode", type=int, default=2, choices=[0, 1, 2, 3],
                    help="0 one launch per pass, 1 persistent solve, 2 CUDA-graph blocks, 3 fused pass pairs + graph blocks")
    ap.add_argument("--bary-div", default="kl", choices=["kl", "tv", "rg"],
                    help="barycenter divergence of the bary workload (Table 2 (ii), (iii), (iv))")
    ap.add_argument("--mass-div", default=None, choices=sorted(MASS_DIVS),
                    help="grid2d workload through Algorithm 4 with this divergence on the plan's total mass")
    ap.add_argument("--no-workloads", action="store_true",
                    help="grid2d: skip the other configurations' sub-record")
    ap.add_argument("--grid-tile", type=int, default=-1,
                    help="force one FP32 grid-pass tile shape (default: the tuner's choice)")
    args = ap.parse_args()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    try:
        if args.workload == "batch":
            line = run_batch(args, rank, world, local_rank)
        elif args.workload == "warmstart":
            line = run_warmstart(args, rank, world, local_rank)
        elif args.workload in ("points", "dense1d", "bary", "wf", "color"):
            line = run_single(args, rank, world, local_rank)
        else:
            line = run_ours(args, rank, world, local_rank)
            # every other configuration, measured in the same run (one GPU only)
            if world == 1 and line is not None and not args.no_workloads and not args.mass_div \
                    and args.precision == "f32" and not args.max_iter and not args.no_eps_scaling:
                line["workloads"] = sub_workloads(args, local_rank, cpu=not args.no_cpu_baseline)
                if not args.no_cpu_baseline:
                    line["cpu_baseline_all_cores"] = oracle_baselines("grid2d", host_cores(),
                                                                      one_core=False)["all_cores"]
        if line is not None:
            print(json.dumps(line), flush=True)
    finally:
        if world > 1:
            import torch.distributed as dist
            dist.destroy_process_group()


if __name__ == "__main__":
    main()
