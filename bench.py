"""Throughput of the StoMsFEM local-upscaling hot path on GB300.

One step = one batch of samples through the whole plain path:
coefficient sampling (xi -> a), simultaneous local upscaling of every
(sample, coarse cell) unit (a -> K_e, b_e), coarse assembly + solve and the
running Monte Carlo moments (K_e, b_e -> u, mean, M2).  The metric is
coarse elements (units) upscaled per second at H/h = 32 (the 1024^2 /
32^2 workload with per-cell oversampling 0..4), for the chosen precision
form, with the plain FP64 path measured in the same run for the speed-up
and the coarse-solution error of the chosen form against it.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
With N > 1 (torchrun), every rank processes its own samples (weak scaling,
no data-path collective); timing is the max over ranks.
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

from paper_1607_00693_gb300 import workloads as W  # noqa: E402

FORMS = {"fp64": 0, "fp32r": 1, "fp32": 2}

# Measured DRAM traffic per unit of the upscale kernel (ncu, 32 samples of
# the H/h = 32 workload, the forward-only and the back-substitution launches
# of one FP32 call), by library version and form: 0.6 and 0.7 share one
# kernel (counters taken on 0.6); 0.8 changed the factorisation window's
# layout and 0.9 the back substitution's end row (counters retaken on each;
# FP64 not retaken).
_TRAFFIC_06 = {"fp32": (0.051981e9 + 0.000175e9 + 7.110618e9 + 6.763874e9) / 32768,
               "fp64": (1.827271e9 + 1.937667e9) / 4096}
_TRAFFIC_08 = {"fp32": (0.051976e9 + 0.000239e9 + 7.124753e9 + 6.771178e9) / 32768}
_TRAFFIC_09 = {"fp32": (0.051979e9 + 0.000154e9 + 6.837680e9 + 6.506667e9) / 32768}
DRAM_BYTES_PER_UNIT = {("stomsfem-gb300 %s (sm_103a)" % v, f): b
                       for v, t in (("0.6", _TRAFFIC_06), ("0.7", _TRAFFIC_06), ("0.8", _TRAFFIC_08),
                                    ("0.9", _TRAFFIC_09))
                       for f, b in t.items()}
DTYPE = {"fp64": "f64", "fp32r": "f32 factor + f64 refinement", "fp32": "f32"}


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


def alu_peak_tflops(form, api=None):
    """(peak TFLOP/s, note) of the non-tensor FMA pipe the upscaling kernel's
    roofline is taken against: measured in this run by the library's FMA
    probe (stomsfem_selftest_fma_rate: FP32 chains for the FP32 forms, FP64
    for the FP64 form), else derived from unit counts and the maximum clock
    (152 SMs x 128 FP32 lanes x 2 flops; FP64 2 FMA/clk/SM)."""
    if api is not None:
        try:
            v = api.stomsfem_selftest_fma_rate(api.FP64 if form == "fp64" else api.FP32)
            return v, "measured in this run: FMA-chain probe (stomsfem_selftest_fma_rate, %s)" % (
                "FP64" if form == "fp64" else "FP32")
        except Exception:
            pass
    clk = _peaks().get("sm_max_mhz", 2070.0) * 1e6
    if form == "fp64":
        return 152 * 2 * 2 * clk / 1e12, "derived: 152 SMs x 2 FP64 FMA/clk x 2 flops x max clock"
    return 152 * 128 * 2 * clk / 1e12, "derived: 152 SMs x 128 FP32 lanes x 2 flops x max clock"


def unit_flops(nf, nc, ov, form, refine=2):
    """Algorithmic flops of one sample (all cells): banded Cholesky of each
    patch matrix, forward/back substitution of 3 right-hand sides, the
    refinement sweeps, the K_e/b_e accumulation (about 70 flops per fine
    element of the cell)."""
    rho = nf // nc
    tot = 0.0
    for cell in range(nc * nc):
        cx, cy = cell % nc, cell // nc
        o = int(ov[cell]) if ov is not None else 0
        x0, x1 = max(0, cx * rho - o), min(nf, (cx + 1) * rho + o)
        y0, y1 = max(0, cy * rho - o), min(nf, (cy + 1) * rho + o)
        mx, my = x1 - x0 - 1, y1 - y0 - 1
        n, b = mx * my, mx + 1
        k = np.arange(n)
        t = np.minimum(b, n - 1 - k).astype(np.float64)
        chol = float(np.sum(t * (t + 1) / 2))
        solve = 3.0 * 2.0 * float(np.sum(t))
        fl = 2.0 * (chol + solve)
        if form == "fp32r":
            fl += refine * (2.0 * 3 * 9 * n + 2.0 * solve)
        fl += 70.0 * rho * rho
        tot += fl
    return tot


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
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
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                smax = float(p[2])
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_oracle_step(w, xi, ov, nthreads=0):
    """The oracle on one batch: a from xi, per-unit MsFEM, coarse solve,
    moments.  Returns seconds."""
    import oracle
    t0 = time.perf_counter()
    a = oracle.sample_coef(w["nf"], w["field"], xi, nthreads=nthreads)
    Ke, be = oracle.upscale(w["nf"], w["nc"], w["f"], a, ov, nthreads=nthreads)
    u = oracle.coarse_solve(w["nc"], Ke, be)
    oracle.mc_moments(u)
    return time.perf_counter() - t0


def cpu_baseline(w, ov, samples=2, single_core_samples=2):
    """The oracle on the host cores, and on one core (a smaller sample of the
    same workload, timed after the all-core run; the OpenMP thread count is
    set back afterwards)."""
    import oracle
    oracle.build()
    cores = oracle.ncores()
    xi = W.draw_xi(w["field"], samples, w["seed"], w["dist"])
    dt = cpu_oracle_step(w, xi, ov, nthreads=cores)
    units = samples * w["nc"] ** 2
    out = {"value": units / dt, "unit": "units/s", "cores": cores, "kind": "oracle",
           "sample": "%d samples x %d cells of %s (FP64 oracle: a, cell problems, coarse solve), "
                     "%.1f s" % (samples, w["nc"] ** 2, w["name"], dt)}
    if single_core_samples > 0:
        xi1 = W.draw_xi(w["field"], single_core_samples, w["seed"], w["dist"], first=samples)
        dt1 = cpu_oracle_step(w, xi1, ov, nthreads=1)
        oracle.sample_coef(w["nf"], w["field"], xi1[:1], nthreads=cores)   # thread count back
        v1 = single_core_samples * w["nc"] ** 2 / dt1
        out["single_core"] = {"value": v1, "unit": "units/s",
                              "sample": "%d samples, 1 thread, %.1f s" % (single_core_samples, dt1)}
        out["sample"] += "; one core: %.0f units/s (%d samples, 1 thread, %.1f s)" % (v1, single_core_samples, dt1)
    return out


def run_reference(args, w, ov):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    oracle.build()
    S = args.ref_samples
    units = S * w["nc"] ** 2
    for i in range(args.warmup):
        cpu_oracle_step(w, W.draw_xi(w["field"], S, w["seed"], w["dist"], first=i * S), ov)
    tt = 0.0
    for i in range(args.steps):
        tt += cpu_oracle_step(w, W.draw_xi(w["field"], S, w["seed"], w["dist"],
                                           first=(args.warmup + i) * S), ov)
    value = units * args.steps / tt
    line = {"impl": "reference", "metric": "coarse elements upscaled/s at H/h=32",
            "value": value, "unit": "units/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * tt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w["name"], "nf": w["nf"], "nc": w["nc"],
                       "samples_per_step": S, "oversample": "0..4 per cell"},
            "cpu_baseline": {"value": value, "unit": "units/s", "cores": oracle.ncores(),
                             "kind": "oracle",
                             "sample": "%d samples x %d cells per step of %s" % (S, w["nc"] ** 2,
                                                                                w["name"])},
            "e2e": {"value": value, "unit": "units/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def _timed_call(stream, fn, reps=3):
    """CUDA-event time (ms) of fn() on `stream`, after one warm-up call."""
    import torch
    with torch.cuda.stream(stream):
        fn()
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn()
        e1.record(stream)
        stream.synchronize()
    return e0.elapsed_time(e1) / reps


def _coarse_err(api, g, Ka, ba, Kb, bb, dev):
    import torch
    S = Ka.shape[0]
    ua = torch.empty((S, (g.nc + 1) ** 2), dtype=torch.float64, device=dev)
    ub = torch.empty_like(ua)
    api.stomsfem_coarse_solve(g, Ka, ba, ua)
    api.stomsfem_coarse_solve(g, Kb, bb, ub)
    torch.cuda.synchronize()
    return float(((ua - ub).norm(dim=1) / ub.norm(dim=1)).max().item())


def shard(rank, ws, total, batch):
    """This rank's contiguous slice of the workload's sample stream: (first,
    count).  Every rank gets the same count (at least one batch), so per-GPU
    work is fixed as the GPU count grows (weak scaling).  Shards are
    disjoint while ws x count <= total; beyond that the last ranks take the
    workload's final slice again (every shard stays inside the workload)."""
    per_rank = max(batch, total // ws)
    if per_rank >= total:
        return 0, per_rank
    return min(rank * per_rank, total - per_rank), per_rank


def max_over_ranks(value, device=None):
    """Maximum of a float over all ranks (the slowest rank sets the time)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(value)
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def bench_pod(api, dev, stream, samples=None):
    """Reduced-basis form on its workload (64^2 fine, 8^2 coarse): offline
    basis from 200 training samples, online stage for 10^4 samples (the
    tensor-core W^T A W GEMM per cell + the reduced solves)."""
    import torch
    w = W.workload("pod_64")
    nf, nc = w["nf"], w["nc"]
    g = api.grid(nf, nc, w["f"])
    fld = api.field_from_dict(w["field"])
    rho = nf // nc
    Ns, S = w["train_samples"], samples or w["samples"]
    xtr = torch.from_numpy(W.draw_xi(w["field"], Ns, w["train_seed"])).to(dev)
    atr = torch.empty((Ns, nf, nf), dtype=torch.float64, device=dev)
    api.stomsfem_sample_coef(g, fld, xtr, atr)
    Ktr = torch.empty((Ns, nc * nc, 10), dtype=torch.float64, device=dev)
    btr = torch.empty((Ns, nc * nc, 4), dtype=torch.float64, device=dev)
    phi = torch.empty((Ns, nc * nc, 4, (rho + 1) ** 2), dtype=torch.float64, device=dev)
    api.stomsfem_upscale(g, atr, Ktr, btr, phi=phi)
    t0 = time.perf_counter()
    h, ranks = api.stomsfem_pod_build(g, phi, atr, tol=w["tol"], max_rank=27)
    t_build = time.perf_counter() - t0
    xi = torch.from_numpy(W.draw_xi(w["field"], S, w["seed"])).to(dev)
    a = torch.empty((S, nf, nf), dtype=torch.float64, device=dev)
    api.stomsfem_sample_coef(g, fld, xi, a)
    Ke = torch.empty((S, nc * nc, 10), dtype=torch.float64, device=dev)
    be = torch.empty_like(Ke[..., :4]).contiguous()
    Kp = torch.empty_like(Ke)
    bp = torch.empty_like(be)
    wsp = torch.empty(api.stomsfem_pod_workspace_size(h, S), dtype=torch.uint8, device=dev)
    _, rb = api.stomsfem_upscale_workspace_size(g, 0, api.FP64)
    wsu = torch.empty(rb, dtype=torch.uint8, device=dev)
    res = {"workload": "pod_64", "samples": S, "units": S * nc * nc, "build_s": t_build,
           "rank_min": int(min(ranks)), "rank_max": int(max(ranks)),
           "rank_mean": float(sum(ranks) / len(ranks))}
    ms_plain = _timed_call(stream, lambda: api.stomsfem_upscale(g, a, Kp, bp, workspace=wsu, stream=stream))
    res["fp64_plain_units_per_s"] = S * nc * nc / (ms_plain / 1e3)
    P0 = 4 + 27
    gemm_flops = 2.0 * S * nc * nc * 64 * (P0 * (P0 + 1) // 2)
    for refine in (0, 4):
        ms = _timed_call(stream, lambda: api.stomsfem_pod_upscale(h, g, a, Ke, be, refine_iters=refine,
                                                                  workspace=wsp, stream=stream))
        key = "refined%d" % refine
        err_k = float(((Ke - Kp).norm(dim=2) / Kp.norm(dim=2)).max().item())
        res[key] = {"units_per_s": S * nc * nc / (ms / 1e3), "ms": ms, "Ke_rel_vs_plain": err_k,
                    "coarse_rel_l2_vs_fp64": _coarse_err(api, g, Ke[:256].contiguous(),
                                                         be[:256].contiguous(), Kp[:256].contiguous(),
                                                         bp[:256].contiguous(), dev),
                    "tensor_tflops_lower_bound": gemm_flops / (ms / 1e3) / 1e12}
    # the same unrefined call with one BF16 product per K step instead of the
    # default BF16 pairs (three products)
    api.stomsfem_pod_set_gemm_split(h, 0)
    ms = _timed_call(stream, lambda: api.stomsfem_pod_upscale(h, g, a, Ke, be, refine_iters=0,
                                                              workspace=wsp, stream=stream))
    api.stomsfem_pod_set_gemm_split(h, 1)
    res["refined0_one_bf16_pass"] = {
        "units_per_s": S * nc * nc / (ms / 1e3), "ms": ms,
        "Ke_rel_vs_plain": float(((Ke - Kp).norm(dim=2) / Kp.norm(dim=2)).max().item()),
        "coarse_rel_l2_vs_fp64": _coarse_err(api, g, Ke[:256].contiguous(), be[:256].contiguous(),
                                             Kp[:256].contiguous(), bp[:256].contiguous(), dev)}
    api.stomsfem_pod_destroy(h)
    peaks = _peaks()
    res["roofline_note"] = ("GEMM flops of the whole call / whole-call time vs bf16 %.0f TFLOP/s "
                            "(measured burst): launch- and FP64-epilogue-bound at this size"
                            % peaks.get("bf16_tflops", 1900.0))
    return res, 4 + 3 * 3 * 4


def bench_contrast(api, dev, stream, batch=128, fp64_batch=8, n_train=24, n_sur_train=1024, sur_steps=20000):
    """The high-contrast comparison (contrast_2048: 2048^2 fine, 64^2 coarse,
    H/h = 32, contrast 10^4, xi ~ N(0,1), no oversampling): plain FP64, the
    FP32 form, FP32 + one refinement sweep (tuned plans, one graph per
    step) and the POD form (offline basis from n_train training samples in
    snapshot space; online BF16 tensor-core W^T A W with K = 1024 per cell
    and the FP32 reduced solves, no refinement) and the learned surrogate
    (per-family networks on the local variables at tau = 1e-3, at most 15
    per cell here; trained on n_sur_train samples from the plain FP32
    upscaler; alone and with the ensemble indicator) on the same GPU, each a
    whole step (sampling, upscaling, coarse solve), with the coarse error
    against plain FP64 on the first fp64_batch samples.  CUDA events, one
    warm-up step and two timed steps per arm."""
    import torch
    w = W.workload("contrast_2048")
    nf, nc = w["nf"], w["nc"]
    ncell = nc * nc
    nn = (nc + 1) ** 2
    rho = nf // nc
    g = api.grid(nf, nc, w["f"])
    fld = api.field_from_dict(w["field"])
    K = W.n_vars(w["field"])
    xi = torch.from_numpy(W.draw_xi(w["field"], batch, w["seed"], w["dist"])).to(dev)
    out = {"workload": "contrast_2048", "H_over_h": rho, "samples_per_step": batch, "fp64_samples": fp64_batch}

    def run_arm(form, Bs, refine=2):
        arm = PlanArm(api, g, fld, None, 0, Bs, form, nn, K, stream, dev, tune_xi=xi[:Bs], refine=refine)
        with torch.cuda.stream(stream):
            arm.step(xi[:Bs])
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(2):
                arm.step(xi[:Bs])
            e1.record(stream)
            stream.synchronize()
        ms = e0.elapsed_time(e1) / 2
        u = arm.u[:fp64_batch].cpu().numpy()
        info = arm.info()
        arm.close()
        return Bs * ncell / (ms / 1e3), u, info

    v64, u64, _ = run_arm("fp64", fp64_batch)
    out["fp64_units_per_s"] = v64

    def err(u):
        return float(np.max(np.linalg.norm(u - u64, axis=1) / np.linalg.norm(u64, axis=1)))

    v32, u32, info32 = run_arm("fp32", batch)
    out["fp32"] = {"units_per_s": v32, "speedup_vs_fp64": v32 / v64, "coarse_rel_l2_vs_fp64": err(u32),
                   "plan": info32}
    v32r, u32r, _ = run_arm("fp32r", batch, refine=1)
    out["fp32r_1_sweep"] = {"units_per_s": v32r, "speedup_vs_fp64": v32r / v64,
                            "coarse_rel_l2_vs_fp64": err(u32r)}
    # POD: offline from n_train FP64 snapshots, then the online step
    xtr = torch.from_numpy(W.draw_xi(w["field"], n_train, w["seed"] + 1000, w["dist"])).to(dev)
    atr = torch.empty((n_train, nf, nf), dtype=torch.float64, device=dev)
    api.stomsfem_sample_coef(g, fld, xtr, atr)
    Ktr = torch.empty((n_train, ncell, 10), dtype=torch.float64, device=dev)
    btr = torch.empty((n_train, ncell, 4), dtype=torch.float64, device=dev)
    phi = torch.empty((n_train, ncell, 4, (rho + 1) ** 2), dtype=torch.float64, device=dev)
    api.stomsfem_upscale(g, atr, Ktr, btr, phi=phi)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h, ranks = api.stomsfem_pod_build(g, phi, atr, tol=1e-6, max_rank=27)
    t_build = time.perf_counter() - t0
    del phi, Ktr, btr, atr
    a = torch.empty((batch, nf, nf), dtype=torch.float64, device=dev)
    Ke = torch.empty((batch, ncell, 10), dtype=torch.float64, device=dev)
    be = torch.empty((batch, ncell, 4), dtype=torch.float64, device=dev)
    u = torch.empty((batch, nn), dtype=torch.float64, device=dev)
    pst = torch.zeros((batch, ncell), dtype=torch.int32, device=dev)
    wsp = torch.empty(api.stomsfem_pod_workspace_size(h, batch), dtype=torch.uint8, device=dev)
    wsc = torch.empty(api.stomsfem_coarse_workspace_size(g, batch), dtype=torch.uint8, device=dev)

    def pod_step(ev=None):
        # the coefficient in FP32 arithmetic, as the FP32 form samples it (the
        # GEMM takes it as BF16 pairs, 16 bits)
        api.stomsfem_sample_coef_precision(g, fld, xi, a, precision=api.FP32, stream=stream)
        if ev is not None:
            ev[0].record(stream)
        api.stomsfem_pod_upscale(h, g, a, Ke, be, refine_iters=0, unit_status=pst, workspace=wsp, stream=stream)
        if ev is not None:
            ev[1].record(stream)
        api.stomsfem_coarse_solve(g, Ke, be, u, workspace=wsc, stream=stream)

    def two_steps(step):
        """(ms per whole step, ms of its upscaling call): one warm-up step,
        then two timed ones."""
        evs = []
        with torch.cuda.stream(stream):
            step()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(2):
                ev = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                evs.append(ev)
                step(ev)
            e1.record(stream)
            stream.synchronize()
        return e0.elapsed_time(e1) / 2, sum(a_.elapsed_time(b_) for a_, b_ in evs) / len(evs)

    ms, ms_up = two_steps(pod_step)
    P0 = 4 + int(max(ranks))
    Ppad = (P0 * (P0 + 1) // 2 + 15) // 16 * 16
    gemm_flops = 2.0 * batch * ncell * (rho * rho) * Ppad
    out["pod"] = {"units_per_s": batch * ncell / (ms / 1e3), "speedup_vs_fp64": batch * ncell / (ms / 1e3) / v64,
                  "coarse_rel_l2_vs_fp64": err(u[:fp64_batch].cpu().numpy()),
                  "train_samples": n_train, "build_s": t_build, "rank_min": int(min(ranks)),
                  "rank_max": int(max(ranks)), "rank_mean": float(sum(ranks) / len(ranks)),
                  "pod_upscale_ms": ms_up, "gemm_tensor_tflops_whole_call": gemm_flops / (ms_up / 1e3) / 1e12,
                  "failed_units": int((pst != 0).sum().item()),
                  "refinement": "none (FP64 refinement is offered for H/h <= 8)"}
    api.stomsfem_pod_destroy(h)
    del pst, wsp
    # learned surrogate: two networks per family (the second for the
    # ensemble indicator), trained on FP32 plain-upscaler pairs
    tau = 1e-3
    kv, _, _, nfam = api.stomsfem_local_vars(g, fld, tau)
    xs = torch.from_numpy(W.draw_xi(w["field"], n_sur_train, w["seed"] + 2000, w["dist"])).to(dev)
    As = torch.empty((n_sur_train, nf, nf), dtype=torch.float64, device=dev)
    api.stomsfem_sample_coef(g, fld, xs, As)
    Ks = torch.empty((n_sur_train, ncell, 10), dtype=torch.float64, device=dev)
    bs = torch.empty((n_sur_train, ncell, 4), dtype=torch.float64, device=dev)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    api.stomsfem_upscale(g, As, Ks, bs, precision=api.FP32)
    torch.cuda.synchronize()
    t_pairs = time.perf_counter() - t0
    hs, losses = [], []
    t0 = time.perf_counter()
    for rep in range(2):
        hh, _ = api.stomsfem_surrogate_create(g, fld, tau, api.xavier_weights(nfam, rep))
        losses.append(api.stomsfem_surrogate_train(hh, xs, As, Ks, bs, steps=sur_steps, lr=2e-3, lr_min=2e-5,
                                                   seed=w["seed"] + 7 + rep))
        hs.append(hh)
    t_train = (time.perf_counter() - t0) / 2
    del xs, As, Ks, bs
    fb = torch.empty((batch, ncell), dtype=torch.uint8, device=dev)

    def sur_arm(ws):
        def step(ev=None):
            # FP64 coefficient: the indicator's cell means and the fallback
            # upscaler read it
            api.stomsfem_sample_coef(g, fld, xi, a, stream=stream)
            if ev is not None:
                ev[0].record(stream)
            api.stomsfem_surrogate_infer(hs[0], g, xi, a, Ke, be, fb, workspace=ws, stream=stream)
            if ev is not None:
                ev[1].record(stream)
            api.stomsfem_coarse_solve(g, Ke, be, u, workspace=wsc, stream=stream)

        ms_, ms_inf = two_steps(step)
        v = batch * ncell / (ms_ / 1e3)
        return {"units_per_s": v, "speedup_vs_fp64": v / v64, "coarse_rel_l2_vs_fp64": err(u[:fp64_batch].cpu().numpy()),
                "infer_ms": ms_inf, "fallback_rate": float((fb != 0).double().mean().item()),
                "ensemble_fallback_rate": float((fb == 2).double().mean().item())}

    sur = {"tau": tau, "k_min": int(kv.min()), "k_max": int(kv.max()), "families": nfam,
           "train_samples": n_sur_train, "train_pairs": n_sur_train * ncell, "train_steps": sur_steps,
           "pairs_s": t_pairs, "train_s_per_network": t_train,
           "train_loss_last": float(losses[0][-50:].mean()),
           "single": sur_arm(torch.empty(api.stomsfem_surrogate_workspace_size(hs[0], batch), dtype=torch.uint8,
                                         device=dev))}
    ens_tol = 0.005
    api.stomsfem_surrogate_set_partner(hs[0], hs[1], ens_tol)
    sur["ensemble"] = dict(tol=ens_tol, **sur_arm(torch.empty(api.stomsfem_surrogate_workspace_size(hs[0], batch),
                                                              dtype=torch.uint8, device=dev)))
    for hh in hs:
        api.stomsfem_surrogate_destroy(hh)
    out["surrogate"] = sur
    out["note"] = ("random interpolation is not run here: its degree rule's tensor grids exceed the 2048 points "
                   "per family that the online kernel holds (46,656 for one family at eps = 1e-3, 3,888 at "
                   "eps = 0.1)")
    return out


def bench_pod_affine(api, dev, stream, samples=None):
    """Affine reduced basis (Sec. 3.2.2, Eqs. RBaffine, localAF) on the 64^2 /
    8^2 grid with the affine field: basis from 200 training samples, affine
    parts per cell, online stage for 10^4 samples straight from xi (no fine
    grid, no workspace) against plain FP64 upscaling of the same samples."""
    import torch
    w = W.workload("pod_affine_64")
    nf, nc = w["nf"], w["nc"]
    g = api.grid(nf, nc, w["f"])
    fld = api.field_from_dict(w["field"])
    rho = nf // nc
    Ns, S = w["train_samples"], samples or w["samples"]
    xtr = torch.from_numpy(W.draw_xi(w["field"], Ns, w["train_seed"])).to(dev)
    atr = torch.empty((Ns, nf, nf), dtype=torch.float64, device=dev)
    api.stomsfem_sample_coef(g, fld, xtr, atr)
    Ktr = torch.empty((Ns, nc * nc, 10), dtype=torch.float64, device=dev)
    btr = torch.empty((Ns, nc * nc, 4), dtype=torch.float64, device=dev)
    phi = torch.empty((Ns, nc * nc, 4, (rho + 1) ** 2), dtype=torch.float64, device=dev)
    api.stomsfem_upscale(g, atr, Ktr, btr, phi=phi)
    h, ranks = api.stomsfem_pod_build(g, phi, atr, tol=w["tol"], max_rank=27)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    api.stomsfem_pod_set_affine(h, g, fld, w["tau"], stream=stream)
    t_aff = time.perf_counter() - t0
    xi = torch.from_numpy(W.draw_xi(w["field"], S, w["seed"])).to(dev)
    a = torch.empty((S, nf, nf), dtype=torch.float64, device=dev)
    api.stomsfem_sample_coef(g, fld, xi, a)
    Ke = torch.empty((S, nc * nc, 10), dtype=torch.float64, device=dev)
    be = torch.empty((S, nc * nc, 4), dtype=torch.float64, device=dev)
    Kp, bp = torch.empty_like(Ke), torch.empty_like(be)
    _, rb = api.stomsfem_upscale_workspace_size(g, 0, api.FP64)
    wsu = torch.empty(rb, dtype=torch.uint8, device=dev)
    units = S * nc * nc
    ms = _timed_call(stream, lambda: api.stomsfem_pod_upscale_affine(h, g, xi, Ke, be, stream=stream))
    ms_plain = _timed_call(stream, lambda: api.stomsfem_upscale(g, a, Kp, bp, workspace=wsu, stream=stream))
    res = {"workload": "pod_affine_64", "samples": S, "units": units, "affine_parts_s": t_aff,
           "rank_mean": float(sum(ranks) / len(ranks)), "units_per_s": units / (ms / 1e3), "ms": ms,
           "fp64_plain_units_per_s": units / (ms_plain / 1e3), "speedup_vs_fp64": ms_plain / ms,
           "Ke_rel_vs_plain": float(((Ke - Kp).norm(dim=2) / Kp.norm(dim=2)).max().item()),
           "coarse_rel_l2_vs_fp64": _coarse_err(api, g, Ke[:256].contiguous(), be[:256].contiguous(),
                                                Kp[:256].contiguous(), bp[:256].contiguous(), dev)}
    api.stomsfem_pod_destroy(h)
    return res, 3 + 3


def bench_two_level(api, dev, stream, n0=10000, n1=256):
    """Two-level Monte Carlo (Eq. MCmean2level) on the 64^2 / 8^2 grid:
    N_0 = 10^4 coarse samples (random interpolation online + coarse solve),
    N_1 = 256 independent samples on both levels (fine Q1 FEM on the GPU
    and the coarse solution), against plain Monte Carlo with the same 256
    fine solves: the sampling standard deviation of the mean (root of the
    node-averaged variance of the estimator)."""
    import torch
    w = W.workload("ri_64")
    nf, nc = w["nf"], w["nc"]
    g = api.grid(nf, nc, w["f"])
    fld = api.field_from_dict(w["field"])
    nn = (nc + 1) ** 2
    h, _ = api.stomsfem_ri_build(g, fld, w["eps"], w["nu_max"], w["nodes"], stream=stream)

    def mom():
        return [torch.zeros(nn, dtype=torch.float64, device=dev), torch.zeros(nn, dtype=torch.float64, device=dev),
                torch.zeros(1, dtype=torch.float64, device=dev)]

    def coarse_ri(xi, S, m):
        Ke = torch.empty((S, nc * nc, 10), dtype=torch.float64, device=dev)
        be = torch.empty((S, nc * nc, 4), dtype=torch.float64, device=dev)
        fb = torch.empty((S, nc * nc), dtype=torch.uint8, device=dev)
        u = torch.empty((S, nn), dtype=torch.float64, device=dev)
        api.stomsfem_ri_upscale(h, g, xi, None, Ke, be, fb, stream=stream)
        api.stomsfem_coarse_solve(g, Ke, be, u, *m, stream=stream)
        return u

    x0 = torch.from_numpy(W.draw_xi(w["field"], n0, 501)).to(dev)
    x1 = torch.from_numpy(W.draw_xi(w["field"], n1, 502)).to(dev)
    a1 = torch.empty((n1, nf, nf), dtype=torch.float64, device=dev)
    uh = torch.empty((n1, (nf + 1) ** 2), dtype=torch.float64, device=dev)
    wsf = torch.empty(api.stomsfem_fine_fem_workspace_size(g, n1), dtype=torch.uint8, device=dev)
    d = torch.empty((n1, nn), dtype=torch.float64, device=dev)
    uhc = torch.empty((n1, nn), dtype=torch.float64, device=dev)
    m0, m1, mp = mom(), mom(), mom()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        coarse_ri(x0, n0, m0)
        e[1].record(stream)
        api.stomsfem_sample_coef(g, fld, x1, a1, stream=stream)
        api.stomsfem_fine_fem(g, a1, uh, workspace=wsf, stream=stream)
        uH1 = coarse_ri(x1, n1, [None, None, None])
        api.stomsfem_restrict_to_coarse(g, uh, d, u_coarse=uH1, stream=stream)
        api.stomsfem_mc_moments(d, *m1, stream=stream)
        e[2].record(stream)
        api.stomsfem_restrict_to_coarse(g, uh, uhc, stream=stream)
        api.stomsfem_mc_moments(uhc, *mp, stream=stream)
    stream.synchronize()
    sd2 = float(((m0[1] / n0 / n0) + (m1[1] / n1 / n1)).mean().sqrt().item())
    sdp = float((mp[1] / n1 / n1).mean().sqrt().item())
    diff = float(((m0[0] + m1[0]) - mp[0]).norm().item() / mp[0].norm().item())
    api.stomsfem_ri_destroy(h)
    return {"workload": "ri_64 grid, level 0 by random interpolation", "n0_coarse": n0, "n1_fine": n1,
            "level0_ms": e[0].elapsed_time(e[1]), "level1_ms": e[1].elapsed_time(e[2]),
            "fine_fem_samples_per_s": n1 / (e[1].elapsed_time(e[2]) / 1e3),
            "sd_of_mean_two_level": sd2, "sd_of_mean_plain_mc_same_fine_solves": sdp,
            "variance_reduction": (sdp / sd2) ** 2 if sd2 > 0 else None,
            "two_level_vs_plain_mean_rel": diff}


def bench_two_level_1024(api, dev, stream, ov, n0=512, n1=16, workload="upscale_1024"):
    """Two-level Monte Carlo (Eq. MCmean2level) on an H/h = 32 workload's
    grids (upscale_1024: 1024^2 / 32^2 with its oversampling; contrast_2048:
    2048^2 / 64^2, contrast 10^4, none): level 0, n0 samples through the
    FP32 upscaler and the coarse solve; level 1, n1 independent samples
    with the fine Q1 FEM (multigrid-preconditioned CG on the GPU) and their
    coarse solutions; against plain Monte Carlo with the same n1 fine solves."""
    import torch
    w = W.workload(workload)
    nf, nc = w["nf"], w["nc"]
    g = api.grid(nf, nc, w["f"])
    fld = api.field_from_dict(w["field"])
    nn = (nc + 1) ** 2
    ov_t = torch.from_numpy(ov).to(dev) if ov is not None else None
    mo = int(ov.max()) if ov is not None else 0

    def mom():
        return [torch.zeros(nn, dtype=torch.float64, device=dev), torch.zeros(nn, dtype=torch.float64, device=dev),
                torch.zeros(1, dtype=torch.float64, device=dev)]

    _, rb = api.stomsfem_upscale_workspace_size(g, mo, api.FP32)
    wsu = torch.empty(rb, dtype=torch.uint8, device=dev)

    def coarse(xi, S, m, a=None):
        if a is None:
            a = torch.empty((S, nf, nf), dtype=torch.float64, device=dev)
            api.stomsfem_sample_coef_precision(g, fld, xi, a, precision=api.FP32, stream=stream)
        Ke = torch.empty((S, nc * nc, 10), dtype=torch.float64, device=dev)
        be = torch.empty((S, nc * nc, 4), dtype=torch.float64, device=dev)
        u = torch.empty((S, nn), dtype=torch.float64, device=dev)
        api.stomsfem_upscale(g, a, Ke, be, oversample=ov_t, max_oversample=mo, precision=api.FP32,
                             workspace=wsu, stream=stream)
        api.stomsfem_coarse_solve(g, Ke, be, u, *m, stream=stream)
        return u

    x0 = torch.from_numpy(W.draw_xi(w["field"], n0, 601, w["dist"])).to(dev)
    x1 = torch.from_numpy(W.draw_xi(w["field"], n1, 602, w["dist"])).to(dev)
    a1 = torch.empty((n1, nf, nf), dtype=torch.float64, device=dev)
    uh = torch.empty((n1, (nf + 1) ** 2), dtype=torch.float64, device=dev)
    wsf = torch.empty(api.stomsfem_fine_fem_workspace_size(g, n1), dtype=torch.uint8, device=dev)
    d = torch.empty((n1, nn), dtype=torch.float64, device=dev)
    uhc = torch.empty((n1, nn), dtype=torch.float64, device=dev)
    m0, m1, mp = mom(), mom(), mom()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        coarse(x0, n0, m0)
        e[1].record(stream)
        api.stomsfem_sample_coef(g, fld, x1, a1, stream=stream)
        e[2].record(stream)
        api.stomsfem_fine_fem(g, a1, uh, workspace=wsf, stream=stream)
        e[3].record(stream)
        uH1 = coarse(x1, n1, [None, None, None], a=a1)
        api.stomsfem_restrict_to_coarse(g, uh, d, u_coarse=uH1, stream=stream)
        api.stomsfem_mc_moments(d, *m1, stream=stream)
        api.stomsfem_restrict_to_coarse(g, uh, uhc, stream=stream)
        api.stomsfem_mc_moments(uhc, *mp, stream=stream)
    stream.synchronize()
    sd2 = float(((m0[1] / n0 / n0) + (m1[1] / n1 / n1)).mean().sqrt().item())
    sdp = float((mp[1] / n1 / n1).mean().sqrt().item())
    fine_ms = e[2].elapsed_time(e[3])
    return {"workload": "%s grids (%d^2 fine, %d^2 coarse), level 0 by the FP32 upscaler" % (workload, nf, nc),
            "n0_coarse": n0, "n1_fine": n1, "level0_ms": e[0].elapsed_time(e[1]),
            "fine_fem_ms": fine_ms, "fine_fem_samples_per_s": n1 / (fine_ms / 1e3),
            "fine_fem_method": "CG (FP64) with a multigrid V-cycle (FP32) preconditioner",
            "sd_of_mean_two_level": sd2, "sd_of_mean_plain_mc_same_fine_solves": sdp,
            "variance_reduction": (sdp / sd2) ** 2 if sd2 > 0 else None}


def bench_surrogate(api, dev, stream, samples=None, steps=3000):
    """Learned-surrogate form (64^2 / 8^2 workload): training on 1563
    samples (10^5 cell pairs) from the plain upscaler, inference on 10^5
    fresh samples (6.4 M units) with indicator and fallback."""
    import torch
    w = W.workload("surrogate_64")
    nf, nc = w["nf"], w["nc"]
    g = api.grid(nf, nc, w["f"])
    fld = api.field_from_dict(w["field"])
    Ns, S = w["train_samples"], samples or w["samples"]
    xtr = torch.from_numpy(W.draw_xi(w["field"], Ns, w["train_seed"])).to(dev)
    atr = torch.empty((Ns, nf, nf), dtype=torch.float64, device=dev)
    api.stomsfem_sample_coef(g, fld, xtr, atr)
    Ktr = torch.empty((Ns, nc * nc, 10), dtype=torch.float64, device=dev)
    btr = torch.empty((Ns, nc * nc, 4), dtype=torch.float64, device=dev)
    api.stomsfem_upscale(g, atr, Ktr, btr)
    _, _, _, nfam = api.stomsfem_local_vars(g, fld, 1e-6)
    h, _ = api.stomsfem_surrogate_create(g, fld, 1e-6, api.xavier_weights(nfam, 0))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    loss = api.stomsfem_surrogate_train(h, xtr, atr, Ktr, btr, steps=steps, lr=2e-3, lr_min=2e-5,
                                        seed=w["train_seed"])
    t_train = time.perf_counter() - t0
    xi = torch.from_numpy(W.draw_xi(w["field"], S, w["seed"])).to(dev)
    a = torch.empty((S, nf, nf), dtype=torch.float64, device=dev)
    api.stomsfem_sample_coef(g, fld, xi, a)
    Ke = torch.empty((S, nc * nc, 10), dtype=torch.float64, device=dev)
    be = torch.empty((S, nc * nc, 4), dtype=torch.float64, device=dev)
    fb = torch.empty((S, nc * nc), dtype=torch.uint8, device=dev)
    Kp = torch.empty_like(Ke)
    bp = torch.empty_like(be)
    wss = torch.empty(api.stomsfem_surrogate_workspace_size(h, S), dtype=torch.uint8, device=dev)
    _, rb = api.stomsfem_upscale_workspace_size(g, 0, api.FP64)
    wsu = torch.empty(rb, dtype=torch.uint8, device=dev)
    units = S * nc * nc
    ms_inf = _timed_call(stream, lambda: api.stomsfem_surrogate_infer(h, g, xi, a, Ke, be, fb, workspace=wss,
                                                                      stream=stream))
    ms_plain = _timed_call(stream, lambda: api.stomsfem_upscale(g, a, Kp, bp, workspace=wsu, stream=stream))
    flops = 2.0 * units * (64 * 128 + 2 * 128 * 128 + 16 * 128)  # padded inputs, as computed
    res = {"workload": "surrogate_64", "train_pairs": Ns * nc * nc, "train_steps": steps,
           "train_s": t_train, "train_loss_first": float(loss[:10].mean()),
           "train_loss_last": float(loss[-50:].mean()), "families": nfam,
           "infer_units": units, "infer_units_per_s": units / (ms_inf / 1e3),
           "fp64_plain_units_per_s": units / (ms_plain / 1e3),
           "speedup_vs_fp64": ms_plain / ms_inf,
           "fallback_rate": float(fb.double().mean().item()),
           "coarse_rel_l2_vs_fp64": _coarse_err(api, g, Ke[:2000].contiguous(), be[:2000].contiguous(),
                                                Kp[:2000].contiguous(), bp[:2000].contiguous(), dev),
           "tensor_tflops_whole_call": flops / (ms_inf / 1e3) / 1e12,
           "tensor_peak_tflops": _peaks().get("bf16_tflops", 1900.0)}
    # the ensemble indicator: a second network from other initial weights
    # and minibatch draws, its disagreement above 2 % sending units back
    h2, _ = api.stomsfem_surrogate_create(g, fld, 1e-6, api.xavier_weights(nfam, 1))
    api.stomsfem_surrogate_train(h2, xtr, atr, Ktr, btr, steps=steps, lr=2e-3, lr_min=2e-5,
                                 seed=w["train_seed"] + 1)
    api.stomsfem_surrogate_set_partner(h, h2, 0.02)
    wss2 = torch.empty(api.stomsfem_surrogate_workspace_size(h, S), dtype=torch.uint8, device=dev)
    ms_ens = _timed_call(stream, lambda: api.stomsfem_surrogate_infer(h, g, xi, a, Ke, be, fb, workspace=wss2,
                                                                      stream=stream))
    res["ensemble"] = {"tol": 0.02, "units_per_s": units / (ms_ens / 1e3), "speedup_vs_fp64": ms_plain / ms_ens,
                       "fallback_rate": float((fb != 0).double().mean().item()),
                       "ensemble_fallback_rate": float((fb == 2).double().mean().item()),
                       "coarse_rel_l2_vs_fp64": _coarse_err(api, g, Ke[:2000].contiguous(), be[:2000].contiguous(),
                                                            Kp[:2000].contiguous(), bp[:2000].contiguous(), dev)}
    api.stomsfem_surrogate_destroy(h)
    api.stomsfem_surrogate_destroy(h2)
    return res, 6 * 4 + 8 + 9 * 4


def bench_ri(api, dev, stream, samples=None):
    """Random-interpolation form (Sec. 3.1, Algorithms 1-2) on the 64^2 / 8^2
    workload: offline collocation through the FP64 upscaler, online
    interpolation of K_e and b_e for 10^5 fresh samples (6.4 M units), the
    direct FP64 fallback armed (a given)."""
    import torch
    w = W.workload("ri_64")
    nf, nc = w["nf"], w["nc"]
    g = api.grid(nf, nc, w["f"])
    fld = api.field_from_dict(w["field"])
    S = samples or w["samples"]
    fam, _, nu, nfam, npts = api.stomsfem_ri_plan(g, fld, w["eps"], w["nu_max"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h, _ = api.stomsfem_ri_build(g, fld, w["eps"], w["nu_max"], w["nodes"], stream=stream)
    t_build = time.perf_counter() - t0
    xi = torch.from_numpy(W.draw_xi(w["field"], S, w["seed"])).to(dev)
    a = torch.empty((S, nf, nf), dtype=torch.float64, device=dev)
    api.stomsfem_sample_coef(g, fld, xi, a)
    Ke = torch.empty((S, nc * nc, 10), dtype=torch.float64, device=dev)
    be = torch.empty((S, nc * nc, 4), dtype=torch.float64, device=dev)
    fb = torch.empty((S, nc * nc), dtype=torch.uint8, device=dev)
    Kp = torch.empty_like(Ke)
    bp = torch.empty_like(be)
    wsr = torch.empty(api.stomsfem_ri_workspace_size(h, S), dtype=torch.uint8, device=dev)
    _, rb = api.stomsfem_upscale_workspace_size(g, 0, api.FP64)
    wsu = torch.empty(rb, dtype=torch.uint8, device=dev)
    units = S * nc * nc
    ms = _timed_call(stream, lambda: api.stomsfem_ri_upscale(h, g, xi, a, Ke, be, fb, workspace=wsr,
                                                             stream=stream))
    ms_plain = _timed_call(stream, lambda: api.stomsfem_upscale(g, a, Kp, bp, workspace=wsu, stream=stream))
    # algorithmic FP32 flops: 14 multiply-adds per grid point of the unit's family
    pts_cell = [int(np.prod(nu[c][nu[c] > 0] + 1)) for c in range(nc * nc)]
    flops = 2.0 * 14 * S * sum(pts_cell)
    peaks = _peaks()
    res = {"workload": "ri_64", "eps": w["eps"], "nu_max": w["nu_max"],
           "nodes": "legendre" if w["nodes"] == 1 else "chebyshev", "families": nfam,
           "grid_points": int(npts), "grid_points_per_unit_mean": float(np.mean(pts_cell)),
           "build_s": t_build, "units": units, "units_per_s": units / (ms / 1e3), "ms": ms,
           "fp64_plain_units_per_s": units / (ms_plain / 1e3), "speedup_vs_fp64": ms_plain / ms,
           "fallback_rate": float(fb.double().mean().item()),
           "Ke_rel_vs_plain": float(((Ke - Kp).norm(dim=2) / Kp.norm(dim=2)).max().item()),
           "coarse_rel_l2_vs_fp64": _coarse_err(api, g, Ke[:2000].contiguous(), be[:2000].contiguous(),
                                                Kp[:2000].contiguous(), bp[:2000].contiguous(), dev),
           "fp32_tflops_whole_call": flops / (ms / 1e3) / 1e12,
           "fp32_peak_tflops": alu_peak_tflops("fp32", api)[0],
           "fp32_frac_whole_call": flops / (ms / 1e3) / 1e12 / alu_peak_tflops("fp32", api)[0],
           "roofline_note": "FP32 ALU: 28 flops per grid point per unit over the whole call against "
                            "the peak derived from unit counts; HBM moves 113 B per unit (K_e, b_e, "
                            "flag) plus its share of xi, far below the ALU time"}
    api.stomsfem_ri_destroy(h)
    return res, 3 * 3 + 3  # (tiles, eval, fallback) x 3 timed calls + the FP64 comparison x 3


ENGINE_NAMES = {0: "auto", 1: "blocked_fma", 2: "tc_tf32x3", 3: "tc_tf32x2", 4: "wide_fma"}
ORDER_NAMES = {0: "cell", 1: "patch_size"}


class PlanArm:
    """The headline step through the library's plan: launch choices picked
    by its autotuner on the first batch (or fixed), then every step replayed
    as one captured CUDA graph.  Each step's batch is copied into the
    plan's fixed input buffer first (a device-to-device copy of the xi rows,
    part of the step), and the device time of its upscaling launches is read
    from the plan's timing events right after the step is queued."""

    def __init__(self, api, g, fld, ov_t, mo, Bs, form, nn, K, stream, dev, engine=None, tune_xi=None, refine=2):
        import torch
        self.api, self.stream, self.Bs = api, stream, Bs
        self.h = api.stomsfem_plan_create(g, fld, Bs, FORMS[form], oversample=ov_t, max_oversample=mo,
                                          refine_iters=refine)
        self.u = torch.empty((Bs, nn), dtype=torch.float64, device=dev)
        self.mean = torch.zeros(nn, dtype=torch.float64, device=dev)
        self.m2 = torch.zeros_like(self.mean)
        self.cnt = torch.zeros(1, dtype=torch.float64, device=dev)
        self.xd = torch.empty((Bs, K), dtype=torch.float64, device=dev)
        self.tune_ms = None
        with torch.cuda.stream(stream):
            if engine is None:
                self.xd.copy_(tune_xi)
                _, _, self.tune_ms = api.stomsfem_plan_tune(self.h, self.xd, self.u, stream=stream)
            else:
                api.stomsfem_plan_set_choice(self.h, 0, 1, engine)
        stream.synchronize()

    def step(self, xs):
        """Queue one step on xs (device [Bs][K]); returns the upscaling time (ms)."""
        self.xd.copy_(xs, non_blocking=True)
        self.api.stomsfem_plan_step(self.h, self.xd, self.u, self.mean, self.m2, self.cnt, stream=self.stream)
        return self.api.stomsfem_plan_upscale_ms(self.h)

    def info(self):
        bps, split, eng, order, ready, nbytes = self.api.stomsfem_plan_info(self.h)
        return {"blocks_per_sm": bps, "split_fp32": split, "engine": ENGINE_NAMES[eng],
                "order": ORDER_NAMES[order], "graph_ready": ready, "device_bytes": nbytes,
                "tune_best_ms": self.tune_ms}

    def launches_per_step(self, form, oversampled):
        """Kernels of one step: sampling, the upscaling launches (the
        cell-list kernel and one or two upscale_kernel launches), and the
        coarse assembly/solve, moments and count kernels."""
        _, split, _, order, _, _ = self.api.stomsfem_plan_info(self.h)
        if oversampled and form == "fp32" and split:
            n_up = 3
        elif oversampled and order == 1:
            n_up = 2
        else:
            n_up = 1
        return 1 + n_up + 3

    def close(self):
        self.api.stomsfem_plan_destroy(self.h)


def bench_engines(api, g, fld, ov_t, mo, B, nn, stream, dev, xs_for, u64, Bc):
    """The FP32 forms' factorisation engines A/B (CUDA events, the same
    batch through plans fixed to each engine, one untimed step then three
    timed, graph replay): units/s of the whole step and the coarse error
    against the plain FP64 step on the first Bc samples."""
    import torch
    out = {}
    if not api.stomsfem_plan_create:  # pragma: no cover
        return out
    for pname, prec, Bs in (("fp32", api.FP32, B), ("fp32r", api.FP32_REFINED, max(Bc, B // 4))):
        res = {}
        for eng, order in ((api.ENGINE_BLOCKED, 0), (api.ENGINE_BLOCKED, 1), (api.ENGINE_WIDE, 0),
                           (api.ENGINE_TC3, 0), (api.ENGINE_TC2, 0)):
            name = ENGINE_NAMES[eng] + ("" if order == 0 else "+" + ORDER_NAMES[order] + "_order")
            h = api.stomsfem_plan_create(g, fld, Bs, prec, oversample=ov_t, max_oversample=mo, refine_iters=2)
            try:
                api.stomsfem_plan_set_choice(h, 0, 1, eng, order)
            except Exception as e:  # not eligible for this grid
                api.stomsfem_plan_destroy(h)
                res[name] = {"unavailable": str(e)}
                continue
            u = torch.empty((Bs, nn), dtype=torch.float64, device=dev)
            xs = xs_for(0, Bs).contiguous()
            with torch.cuda.stream(stream):
                api.stomsfem_plan_step(h, xs, u, stream=stream)
                stream.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(3):
                    api.stomsfem_plan_step(h, xs, u, stream=stream)
                e1.record(stream)
                stream.synchronize()
            ms = e0.elapsed_time(e1) / 3
            ub = u[:Bc].cpu().numpy()
            err = float(np.max(np.linalg.norm(ub - u64[:Bc], axis=1) / np.linalg.norm(u64[:Bc], axis=1)))
            res[name] = {"units_per_s": Bs * g.nc * g.nc / (ms / 1e3), "ms_per_step": ms,
                         "coarse_rel_l2_vs_fp64": err}
            api.stomsfem_plan_destroy(h)
        out[pname] = dict(samples_per_step=Bs, **res)
    # the pipe rates the engines trade between (measured here)
    out["pipe_tflops"] = {"fp32_fma": api.stomsfem_selftest_fma_rate(api.FP32),
                          "mma_sync_tf32": api.stomsfem_selftest_mma_rate(0),
                          "mma_sync_bf16": api.stomsfem_selftest_mma_rate(1)}
    return out


def bench_mixed_bc(api, g, nn, stream, dev, K, b, pg, reps=5):
    """Coarse solve with mixed boundary data (Sec. 5.2, Eqs. xsquarewave /
    ysquarewave: the square-wave lines x = 0.1 and 0.9, zero flux on the
    rest of the boundary) on a step's own K_e and b_e, timed beside the
    plain zero-Dirichlet solve of the same batch."""
    import torch
    from paper_1607_00693_gb300 import workloads as W
    S = K.shape[0]
    dm_np, gv_np = W.mixed_bc(g.nc, axis="x")
    dm, gv = torch.from_numpy(dm_np).to(dev), torch.from_numpy(gv_np).to(dev)
    u = torch.empty((S, nn), dtype=torch.float64, device=dev)
    ws = torch.empty(api.stomsfem_coarse_bc_workspace_size(g, pg, S), dtype=torch.uint8, device=dev)
    if pg:
        ws0 = torch.empty(api.stomsfem_coarse_pg_workspace_size(g, S), dtype=torch.uint8, device=dev)
        plain = lambda: api.stomsfem_coarse_solve_pg(g, K, b, u, workspace=ws0, stream=stream)
    else:
        ws0 = torch.empty(api.stomsfem_coarse_workspace_size(g, S), dtype=torch.uint8, device=dev)
        plain = lambda: api.stomsfem_coarse_solve(g, K, b, u, workspace=ws0, stream=stream)
    mixed = lambda: api.stomsfem_coarse_solve_bc(g, pg, K, b, dm, gv, u, workspace=ws, stream=stream)

    def timed_ms(fn):
        with torch.cuda.stream(stream):
            fn()
            fn()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                fn()
            e1.record(stream)
            stream.synchronize()
        return e0.elapsed_time(e1) / reps

    ms0 = timed_ms(plain)
    ms = timed_ms(mixed)
    return {"form": "petrov_galerkin" if pg else "galerkin", "samples": S, "nodes": nn, "ms_per_call": ms,
            "samples_per_s": S / (ms / 1e3), "zero_dirichlet_ms_per_call": ms0,
            "finite": bool(torch.isfinite(u).all().item()), "gpu_launches_per_call": 1}


def bench_oscillatory(api, g, bf, ov_t, mo, precision, stream, reps=3):
    """Upscaling with the oscillatory boundary data of the cell problems (the
    MsFEM option of Sec. 5.3) on a step's own coefficient batch, timed
    beside the bilinear data through the same call, and how much it changes
    K_e."""
    import torch
    B = bf["a"].shape[0]
    ncell = g.nc * g.nc
    Ko, bo = torch.empty_like(bf["Ke"]), torch.empty_like(bf["be"])

    def timed_ms(bc, K, b):
        run = lambda: api.stomsfem_upscale_bc(g, False, bc, bf["a"], K, b, oversample=ov_t, max_oversample=mo,
                                              precision=precision, refine_iters=2, workspace=bf["wsu"],
                                              stream=stream)
        with torch.cuda.stream(stream):
            run()
            stream.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                run()
            e1.record(stream)
            stream.synchronize()
        return e0.elapsed_time(e1) / reps

    ms_b = timed_ms(api.BC_BILINEAR, bf["Ke"], bf["be"])
    ms_o = timed_ms(api.BC_OSCILLATORY, Ko, bo)
    rel = float(((Ko - bf["Ke"]).norm(dim=-1) / bf["Ke"].norm(dim=-1)).max())
    return {"samples": B, "units_per_s": B * ncell / (ms_o / 1e3), "ms_per_call": ms_o,
            "bilinear_ms_per_call": ms_b, "max_rel_change_of_Ke": rel,
            "finite": bool(torch.isfinite(Ko).all().item()), "gpu_launches_per_call": 1}


def bench_pg(api, g, fld, ov_t, mo, nf, ncell, nn, stream, dev, xs_for, B, Bc, u64_gal):
    """Petrov-Galerkin form (Eq. stiffness_local_petrov) of the FP32 step on
    the same workload: sample a, upscale with bilinear test functions (16
    entries per unit), non-symmetric coarse solve (banded LU) with moments.
    Its coarse error against the FP64 Petrov-Galerkin step, and how far the
    Petrov-Galerkin solution is from the Galerkin one (FP64 both)."""
    import torch

    def bufs(Bs, prec):
        _, rb = api.stomsfem_upscale_workspace_size(g, mo, prec)
        return dict(a=torch.empty((Bs, nf, nf), dtype=torch.float64, device=dev),
                    Ke=torch.empty((Bs, ncell, 16), dtype=torch.float64, device=dev),
                    be=torch.empty((Bs, ncell, 4), dtype=torch.float64, device=dev),
                    u=torch.empty((Bs, nn), dtype=torch.float64, device=dev),
                    wsu=torch.empty(rb, dtype=torch.uint8, device=dev),
                    wsc=torch.empty(api.stomsfem_coarse_pg_workspace_size(g, Bs), dtype=torch.uint8,
                                    device=dev),
                    mean=torch.zeros(nn, dtype=torch.float64, device=dev),
                    m2=torch.zeros(nn, dtype=torch.float64, device=dev),
                    cnt=torch.zeros(1, dtype=torch.float64, device=dev))

    def step(bf, xs, prec):
        api.stomsfem_sample_coef_precision(g, fld, xs, bf["a"], precision=api.FP32 if prec == api.FP32
                                           else api.FP64, stream=stream)
        api.stomsfem_upscale_pg(g, bf["a"], bf["Ke"], bf["be"], oversample=ov_t, max_oversample=mo,
                                precision=prec, workspace=bf["wsu"], stream=stream)
        api.stomsfem_coarse_solve_pg(g, bf["Ke"], bf["be"], bf["u"], bf["mean"], bf["m2"], bf["cnt"],
                                     workspace=bf["wsc"], stream=stream)

    bf = bufs(B, api.FP32)
    steps = 3
    with torch.cuda.stream(stream):
        for i in range(2):
            step(bf, xs_for(i, B), api.FP32)
        stream.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for i in range(steps):
            step(bf, xs_for(2 + i, B), api.FP32)
        e1.record(stream)
        stream.synchronize()
    ms = e0.elapsed_time(e1)
    mixed = bench_mixed_bc(api, g, nn, stream, dev, bf["Ke"], bf["be"], 1)
    del bf
    b32, b64 = bufs(Bc, api.FP32), bufs(Bc, api.FP64)
    with torch.cuda.stream(stream):
        step(b32, xs_for(0, Bc), api.FP32)
        step(b64, xs_for(0, Bc), api.FP64)
    stream.synchronize()
    u32, u64 = b32["u"].cpu().numpy(), b64["u"].cpu().numpy()
    rel = lambda x, y: float(np.max(np.linalg.norm(x - y, axis=1) / np.linalg.norm(y, axis=1)))
    return {"form": "fp32", "samples_per_step": B, "units_per_s": B * ncell * steps / (ms / 1e3),
            "ms_per_step": ms / steps, "coarse_rel_l2_vs_fp64_pg": rel(u32, u64),
            "pg_vs_galerkin_fp64_rel_l2": rel(u64, u64_gal[:Bc]),
            "gpu_launches_per_step": 7, "mixed_bc": mixed}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="fp32", choices=list(FORMS))
    ap.add_argument("--workload", default="upscale_1024")
    ap.add_argument("--batch", type=int, default=512, help="samples per step")
    ap.add_argument("--fp64-batch", type=int, default=32, help="samples per step of the FP64 arm")
    ap.add_argument("--ref-samples", type=int, default=8)
    ap.add_argument("--cpu-samples", type=int, default=96)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-extra-forms", action="store_true",
                    help="skip the reduced-basis, surrogate and interpolation measurements")
    ap.add_argument("--contrast-batch", type=int, default=128, help="samples per step of the contrast_2048 arms")
    ap.add_argument("--contrast-train", type=int, default=24, help="POD training samples on contrast_2048 (<= 24)")
    ap.add_argument("--contrast-sur-train", type=int, default=1024,
                    help="surrogate training samples on contrast_2048")
    ap.add_argument("--contrast-sur-steps", type=int, default=20000, help="surrogate training steps on contrast_2048")
    ap.add_argument("--sections", default="",
                    help="comma-separated subset of the extra sections (engines, petrov_galerkin, pod, surrogate, "
                         "ri, pod_affine, two_level_mc, two_level_mc_1024, two_level_mc_2048, contrast_2048, mixed_bc, "
                         "oscillatory_bc); default all")
    ap.add_argument("--pod-samples", type=int, default=None, help="online POD samples (default 10^4)")
    ap.add_argument("--sg-samples", type=int, default=None, help="surrogate inference samples (default 10^5)")
    ap.add_argument("--sg-steps", type=int, default=3000, help="surrogate training steps")
    ap.add_argument("--ri-samples", type=int, default=None, help="random-interpolation samples (default 10^5)")
    ap.add_argument("--pg-batch", type=int, default=128, help="samples per step of the Petrov-Galerkin arm")
    ap.add_argument("--fp32r-batch", type=int, default=64, help="samples per step of the FP32+refinement arm")
    ap.add_argument("--engine", default="tuned", choices=["tuned", "default", "blocked", "wide", "tc3", "tc2"],
                    help="factorisation engine of the FP32 forms in the timed steps (tuned: the plan's "
                         "autotuner picks the launch choices)")
    args = ap.parse_args()

    w = W.workload(args.workload)
    w["name"] = args.workload
    ov = W.draw_oversample(w["nc"], w["oversample"])
    if args.impl == "reference":
        return run_reference(args, w, ov)

    import torch
    from paper_1607_00693_gb300 import api

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(device=dev)

    nf, nc = w["nf"], w["nc"]
    ncell = nc * nc
    B = args.batch
    engine = {"tuned": None, "default": None, "blocked": api.ENGINE_BLOCKED, "wide": api.ENGINE_WIDE,
              "tc3": api.ENGINE_TC3, "tc2": api.ENGINE_TC2}[args.engine]
    g = api.grid(nf, nc, w["f"])
    fld = api.field_from_dict(w["field"])
    K = W.n_vars(w["field"])
    total = w["samples"]
    # this rank's samples: a contiguous shard of the workload's stream
    first, per_rank = shard(rank, ws, total, B)
    xi_host = W.draw_xi(w["field"], per_rank, w["seed"], w["dist"], first=first)
    xi = torch.from_numpy(xi_host).to(dev)
    ov_t = torch.from_numpy(ov).to(dev) if ov is not None else None
    mo = int(ov.max()) if ov is not None else 0
    nn = (nc + 1) ** 2

    def buffers(Bs, form):
        a = torch.empty((Bs, nf, nf), dtype=torch.float64, device=dev)
        Ke = torch.empty((Bs, ncell, 10), dtype=torch.float64, device=dev)
        be = torch.empty((Bs, ncell, 4), dtype=torch.float64, device=dev)
        u = torch.empty((Bs, nn), dtype=torch.float64, device=dev)
        _, rb = api.stomsfem_upscale_workspace_size(g, mo, FORMS[form])
        wsu = torch.empty(rb, dtype=torch.uint8, device=dev)
        wsc = torch.empty(api.stomsfem_coarse_workspace_size(g, Bs), dtype=torch.uint8, device=dev)
        mom = [torch.zeros(nn, dtype=torch.float64, device=dev) for _ in range(2)]
        cnt = torch.zeros(1, dtype=torch.float64, device=dev)
        return dict(a=a, Ke=Ke, be=be, u=u, wsu=wsu, wsc=wsc, mean=mom[0], m2=mom[1], cnt=cnt)

    def step(bf, xs, form, ev=None, refine=2, engine=None):
        # the FP32 form samples the coefficient in FP32 arithmetic too
        api.stomsfem_sample_coef_precision(g, fld, xs, bf["a"],
                                           precision=api.FP32 if form == "fp32" else api.FP64,
                                           stream=stream)
        if ev is not None:
            ev[0].record(stream)
        api.stomsfem_upscale(g, bf["a"], bf["Ke"], bf["be"], oversample=ov_t, max_oversample=mo,
                             precision=FORMS[form], refine_iters=refine, workspace=bf["wsu"], stream=stream,
                             engine=engine if form != "fp64" else None)  # None: the default
        if ev is not None:
            ev[1].record(stream)
        api.stomsfem_coarse_solve(g, bf["Ke"], bf["be"], bf["u"], bf["mean"], bf["m2"], bf["cnt"],
                                  workspace=bf["wsc"], stream=stream)

    def xs_for(i, Bs):
        s0 = (i * Bs) % max(1, per_rank - Bs + 1)
        return xi[s0:s0 + Bs]

    def barrier():
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()

    def timed(form, Bs, steps, warmup, clocks=None, refine=2, engine=None):
        bf = buffers(Bs, form)
        with torch.cuda.stream(stream):
            for i in range(warmup):
                step(bf, xs_for(i, Bs), form, refine=refine, engine=engine)
            stream.synchronize()
            barrier()
            torch.cuda.synchronize()
            evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                   for _ in range(steps)]
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            if clocks:
                clocks.start()
            e0.record(stream)
            for i in range(steps):
                step(bf, xs_for(warmup + i, Bs), form, evs[i], refine=refine, engine=engine)
            e1.record(stream)
            stream.synchronize()
            clk = clocks.stop() if clocks else None
            barrier()
            torch.cuda.synchronize()
        ms = max_over_ranks(e0.elapsed_time(e1), dev)
        up_ms = [a.elapsed_time(b) for a, b in evs]
        return ms, up_ms, clk, bf

    form = args.form
    # roofline denominator: the FMA pipe's peak, measured here before timing
    peak, peak_note = alu_peak_tflops(form, api)
    clocks = ClockSampler(local)
    # the headline: the step through a plan (autotuned launch choices, one
    # captured graph per step)
    arm = PlanArm(api, g, fld, ov_t, mo, B, form, nn, K, stream, dev,
                  engine=engine if args.engine not in ("tuned", "default") else
                  (api.ENGINE_AUTO if args.engine == "default" else None),
                  tune_xi=xs_for(0, B))
    with torch.cuda.stream(stream):
        for i in range(args.warmup):
            arm.step(xs_for(i, B))
        stream.synchronize()
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        clocks.start()
        e0.record(stream)
        up_ms = [arm.step(xs_for(args.warmup + i, B)) for i in range(args.steps)]
        e1.record(stream)
        stream.synchronize()
        clk = clocks.stop()
        barrier()
        torch.cuda.synchronize()
    ms = max_over_ranks(e0.elapsed_time(e1), dev)
    plan_info = arm.info()
    launches = arm.launches_per_step(form, ov is not None)
    units_step = B * ncell
    value = units_step * ws * args.steps / (ms / 1e3)
    fl = unit_flops(nf, nc, ov, form) * B
    up_avg = sum(up_ms) / len(up_ms)
    achieved = fl / (up_avg / 1e3) / 1e12
    # the same step by direct calls with the default launch choice
    msd, _, _, bf = timed(form, B, max(1, min(args.steps, 3)), 1,
                          engine=engine if args.engine not in ("tuned", "default") else None)
    value_direct = units_step * ws * max(1, min(args.steps, 3)) / (msd / 1e3)

    # the chosen form's coarse solution on the first batch (for its error)
    Bc = min(args.fp64_batch, B)
    with torch.cuda.stream(stream):
        arm.step(xs_for(0, B))
        stream.synchronize()
    uf = arm.u[:Bc].cpu().numpy()

    def plan_timed(form_, Bs, steps, warmup, refine=2):
        """A tuned plan of another form: warm-up, timed steps (CUDA events),
        then one step on the first batch, whose solutions stay in .u."""
        a = PlanArm(api, g, fld, ov_t, mo, Bs, form_, nn, K, stream, dev, tune_xi=xs_for(0, Bs), refine=refine)
        with torch.cuda.stream(stream):
            for i in range(warmup):
                a.step(xs_for(i, Bs))
            stream.synchronize()
            barrier()
            torch.cuda.synchronize()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            ups = [a.step(xs_for(warmup + i, Bs)) for i in range(steps)]
            t1.record(stream)
            stream.synchronize()
            a.step(xs_for(0, Bs))
            stream.synchronize()
        a.up_ms = sum(ups) / len(ups)
        return max_over_ranks(t0.elapsed_time(t1), dev), a

    # the plain FP64 arm (same path, FP64 throughout, its own tuned plan),
    # smaller batch
    steps_s = max(1, min(args.steps, 3))
    ms64, arm64 = plan_timed("fp64", args.fp64_batch, steps_s, 1)
    value64 = args.fp64_batch * ncell * ws * steps_s / (ms64 / 1e3)
    plan64 = arm64.info()
    u64 = arm64.u[:Bc].cpu().numpy()
    # the FP64 upscaling's own roofline (FP64 FMA pipe, measured here)
    peak64, _ = alu_peak_tflops("fp64", api)
    ach64 = unit_flops(nf, nc, ov, "fp64") * args.fp64_batch / (arm64.up_ms / 1e3) / 1e12
    roof64 = {"achieved": ach64, "peak": peak64, "unit": "TFLOP/s", "frac": ach64 / peak64,
              "upscale_ms": arm64.up_ms, "peak_note": "measured in this run: FMA-chain probe, FP64"}
    arm64.close()
    # coarse-solution error of the chosen form vs the FP64 path on the same samples
    err = float(np.max(np.linalg.norm(uf - u64, axis=1) / np.linalg.norm(u64, axis=1)))
    # the FP32 factor + FP64 refinement arm: the fewest sweeps (1, then 2)
    # that bring the coarse solution within 1e-10 of the FP64 path
    Br = min(args.fp32r_batch, args.fp64_batch)
    fp32r = {}
    for sweeps in (1, 2):
        ms32r, arm32r = plan_timed("fp32r", args.fp32r_batch, steps_s, 1, refine=sweeps)
        v = args.fp32r_batch * ncell * ws * steps_s / (ms32r / 1e3)
        e = float(np.max(np.linalg.norm(arm32r.u[:Br].cpu().numpy() - u64[:Br], axis=1) /
                         np.linalg.norm(u64[:Br], axis=1)))
        fp32r[sweeps] = (v, e, arm32r.info(),
                         unit_flops(nf, nc, ov, "fp32r", refine=sweeps) * args.fp32r_batch / (arm32r.up_ms / 1e3) / 1e12)
        arm32r.close()
    sweeps_chosen = 1 if fp32r[1][1] <= 1e-10 else 2
    value32r, err32r, plan32r, ach32r = fp32r[sweeps_chosen]

    e2e = None
    if not args.no_e2e:
        # end to end through the public calls (the plan): pinned host xi in,
        # u out, every step
        steps_e = args.steps
        xh = torch.from_numpy(xi_host[:B].copy()).pin_memory()
        uh = torch.empty((B, nn), dtype=torch.float64).pin_memory()
        with torch.cuda.stream(stream):
            arm.xd.copy_(xh, non_blocking=True)
            api.stomsfem_plan_step(arm.h, arm.xd, arm.u, arm.mean, arm.m2, arm.cnt, stream=stream)
            uh.copy_(arm.u, non_blocking=True)
            stream.synchronize()
            barrier()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for i in range(steps_e):
                arm.xd.copy_(xh, non_blocking=True)
                api.stomsfem_plan_step(arm.h, arm.xd, arm.u, arm.mean, arm.m2, arm.cnt, stream=stream)
                uh.copy_(arm.u, non_blocking=True)
            e1.record(stream)
            stream.synchronize()
        mse = max_over_ranks(e0.elapsed_time(e1), dev)
        e2e = {"value": units_step * ws * steps_e / (mse / 1e3), "unit": "units/s",
               "h2d_bytes_per_step": int(xh.numel() * 8), "d2h_bytes_per_step": int(uh.numel() * 8),
               "api": "stomsfem_plan_step (captured graph)"}
    merged = None
    if ws > 1:
        # the method's one exchange, after the timed region: every rank's
        # running moments gathered and folded into one set on each rank
        import torch.distributed as dist
        with torch.cuda.stream(stream):
            parts = []
            for t in (arm.mean, arm.m2, arm.cnt):
                lst = [torch.empty_like(t) for _ in range(ws)]
                dist.all_gather(lst, t)
                parts.append(lst)
            mean_t, m2_t, cnt_t = (parts[k][0].clone() for k in range(3))
            for r in range(1, ws):
                api.stomsfem_mc_merge(mean_t, m2_t, cnt_t, parts[0][r], parts[1][r], parts[2][r], stream=stream)
            stream.synchronize()
        merged = {"samples": int(cnt_t.item()), "ranks": ws}
    arm.close()

    extra = {}
    if not args.no_extra_forms:
        # the other forms and paths, each outside the headline's timed region
        # (--sections picks a subset by name)
        want = set(args.sections.split(",")) if args.sections else None
        counts = {}
        sections = [
            ("engines", lambda: bench_engines(api, g, fld, ov_t, mo, min(B, 256), nn, stream, dev, xs_for, u64,
                                              Bc)),
            ("petrov_galerkin", lambda: bench_pg(api, g, fld, ov_t, mo, nf, ncell, nn, stream, dev, xs_for,
                                                 args.pg_batch, Bc, u64)),
            ("pod", lambda: bench_pod(api, dev, stream, args.pod_samples)),
            ("surrogate", lambda: bench_surrogate(api, dev, stream, args.sg_samples, args.sg_steps)),
            ("ri", lambda: bench_ri(api, dev, stream, args.ri_samples)),
            ("pod_affine", lambda: bench_pod_affine(api, dev, stream, args.pod_samples)),
            ("two_level_mc", lambda: bench_two_level(api, dev, stream)),
            ("two_level_mc_1024", lambda: bench_two_level_1024(api, dev, stream, ov)),
            ("two_level_mc_2048", lambda: bench_two_level_1024(api, dev, stream, None, n0=128, n1=8,
                                                               workload="contrast_2048")),
            ("contrast_2048", lambda: bench_contrast(api, dev, stream, batch=args.contrast_batch,
                                                     n_train=args.contrast_train,
                                                     n_sur_train=args.contrast_sur_train,
                                                     sur_steps=args.contrast_sur_steps)),
            ("mixed_bc", lambda: bench_mixed_bc(api, g, nn, stream, dev, bf["Ke"], bf["be"], 0)),
            ("oscillatory_bc", lambda: dict(form=form, **bench_oscillatory(api, g, bf, ov_t, mo, FORMS[form],
                                                                           stream))),
        ]
        for name, fn in sections:
            if want is not None and name not in want:
                continue
            r = fn()
            if name in ("pod", "surrogate", "ri", "pod_affine"):
                r, counts[name] = r
            extra[name] = r
        # kernels of each form's own timed calls (outside the step's timed region)
        for k, n in counts.items():
            extra[k]["gpu_launches_timed_calls"] = n

    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, ov, args.cpu_samples)

    # DRAM bytes of one upscale launch: ncu's dram__bytes_read.sum +
    # dram__bytes_write.sum per unit on a 32-sample launch of the same kernel
    # (same library version), times the units of this launch; None when the
    # library differs from the one the counters were taken on
    per_unit = (DRAM_BYTES_PER_UNIT.get((api.stomsfem_version(), form))
                if args.workload == "upscale_1024" else None)
    traffic = per_unit * units_step if per_unit else None
    traffic_note = ("ncu counters of a 32-sample launch scaled by units (%.0f B/unit)" % per_unit
                    if per_unit else "no counters for this library version, form and workload")
    if rank == 0:
        line = {
            "metric": "coarse elements upscaled/s at H/h=32",
            "value": value, "unit": "units/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": DTYPE[form], "data": "synthetic",
            "config": {"workload": args.workload, "nf": nf, "nc": nc, "H_over_h": nf // nc,
                       "samples_per_step": B, "units_per_step": units_step,
                       "oversample": "0..4 per cell (seeded)", "form": form,
                       "engine": args.engine,
                       "plan": plan_info,
                       "direct_calls_units_per_s": round(value_direct, 1),
                       "l2": "inputs larger than L2 (a: %.1f GB per step)" % (B * nf * nf * 8 / 1e9),
                       "parallelism": "replicas (sample shards)" if ws > 1 else "single GPU"},
            "_forms": {"chosen": form, "chosen_units_per_s": value, "fp64_units_per_s": value64,
                      "speedup_vs_fp64": value / value64, "coarse_rel_l2_vs_fp64": err,
                      "fp32r_units_per_s": value32r, "fp32r_speedup_vs_fp64": value32r / value64,
                      "fp32r_coarse_rel_l2_vs_fp64": err32r, "fp32r_sweeps": sweeps_chosen,
                      "fp32r_by_sweeps": {str(k): {"units_per_s": v[0], "coarse_rel_l2_vs_fp64": v[1]}
                                          for k, v in fp32r.items()},
                      "plans": {"fp64": plan64, "fp32r": plan32r},
                      "fp64_roofline": roof64,
                      "fp32r_achieved_tflops": ach32r,
                      "fp32r_frac_of_fp32_peak": ach32r / peak},
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "traffic_note": traffic_note,
                         "kernel": "upscale_kernel (%s)" % form,
                         "peak_note": peak_note},
            "e2e": e2e,
            # the upscaling alone (coefficient resident in HBM): the plan's
            # events around its launches in every timed step
            "upscale_only": {"units_per_s": units_step * ws / (up_avg / 1e3), "ms_per_step": up_avg},
            # per step: sampling, upscaling (FP32 form with oversampling: a
            # cell-list kernel and two upscale launches), coarse solve, moments, count
            "gpu_launches": launches * args.steps,
            "moments_merged": merged,
            "clocks": clk,
            "cpu_baseline": cpu,
        }
        forms = line.pop("_forms")
        # the metric's comparison (chosen form vs plain FP64 at <= 1e-3
        # coarse error), compact, where the record of the line keeps it
        line["config"]["vs_plain_fp64"] = {"fp64_units_per_s": round(value64, 1),
                                          "speedup": round(value / value64, 2),
                                          "coarse_rel_l2": float("%.3g" % err),
                                          "fp32r_sweeps": sweeps_chosen,
                                          "fp32r_speedup": round(value32r / value64, 2)}
        line.update(extra)
        line["forms"] = forms   # last: the tail of the line
        print(json.dumps(line))
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
