"""Benchmark: events/s of maximum-likelihood position reconstruction.

Default workload (1 GPU): 8 x 8 SiPM array, per-sensor XY B-spline LRFs
(24 x 24 intervals), 10^6 synthetic events, plain FP32 contracting-grid
search 11 x 11 nodes x 8 grids.  One step = one reconstruction of all events
(signals already resident in HBM; 256 MB of signals, larger than the 129 MB
L2, so every step streams them from HBM).

  python bench.py [--gpus N --steps K --warmup W] [--impl reference]

Under torchrun each rank reconstructs its own 10^6 events (weak scaling, no
collective on the data path); value = all ranks' events / max-over-ranks time.
--impl reference times the FP64 CPU oracle on host cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "events/s of ML position reconstruction, plain CGS vs chosen form, same error"
SM_COUNT_NOMINAL = 152  # used only where no device can be queried
MUFU_PER_CLK_SM = 16  # 32-bit log2 per clock per SM (nominal)
FMA_PER_CLK_SM = 128  # FP32 fused multiply-adds per clock per SM (nominal)
# canonical FP32 multiply-adds per (node, sensor) evaluation of each search:
# B-spline tensor product, likelihood term and energy sum
F_FMA = {"radial": 19, "xy": 22, "xyz": 86, "local": 9, "composite": 41, "axial_z": 25, "sliced": 46,
         "xy_minimize": 70}


def sm_count() -> int:
    """Streaming multiprocessors of the current CUDA device (queried)."""
    try:
        import torch
        if torch.cuda.is_available():
            return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)
    except Exception:
        pass
    return SM_COUNT_NOMINAL


def alu_roofline(evals_per_s: float, kind: str, verbose: bool = True) -> dict:
    """Evaluation rate against min(FP32 FMA peak / F, log2 peak / 1): nominal
    per-SM rates x the device's SM count x the measured maximum SM clock."""
    pk, pk_kind = peaks()
    clk = float(pk.get("sm_max_mhz", 2070.0)) * 1e6
    sms = sm_count()
    fma_ceiling = sms * FMA_PER_CLK_SM * clk / F_FMA[kind]
    log_ceiling = sms * MUFU_PER_CLK_SM * clk
    peak = min(fma_ceiling, log_ceiling)
    out = {"bound": "alu", "achieved": evals_per_s / 1e12, "peak": peak / 1e12, "unit": "Teval/s",
           "frac": evals_per_s / peak, "frac_of_log2_peak": evals_per_s / log_ceiling}
    if verbose:
        out["peak_kind"] = (f"nominal {FMA_PER_CLK_SM} FMA and {MUFU_PER_CLK_SM} log2 per clock per SM x {sms} SMs "
                            f"(device) x {clk / 1e6:.0f} MHz ({pk_kind} max clock), F = {F_FMA[kind]} FMA per "
                            f"evaluation")
    return out
# DRAM bytes (read + write) per event of the headline kernel, from one ncu
# capture of it on 600 000 events of the same workload (156.46 MB read +
# 10.98 MB written); None once the kernel changes.
XY_TRAFFIC_PER_EVENT = (156464640 + 10975232) / 600_000
# thread-instructions the headline kernel issues per (node, sensor)
# evaluation (ncu smsp__thread_inst_executed.sum / evaluations of the same
# capture: 8.6601e11 / (600 000 x 121 x 8 x 64)); None once the kernel changes
XY_INST_PER_EVAL = 866006665465 / (600_000 * 121 * 8 * 64)


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


class ClockSampler:
    """nvidia-smi sampling of SM clock and throttle reasons during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.dev), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (FileNotFoundError, OSError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
            out, _ = self.proc.communicate()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for name, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(name)
        if not sm:
            return None
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": float(max(mx)), "reasons": sorted(reasons),
                "samples": len(sm)}


def rank_seed(base: int, rank: int) -> int:
    """Event seed of a rank: every rank reconstructs its own events."""
    return base + 7919 * rank


def max_over_ranks(x: float, device="cuda") -> float:
    """The largest x over all ranks (the job's wall time); x itself on one rank."""
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(n_per_rank: int, world: int, steps: int, seconds: float) -> float:
    """Whole-job events/s: the events all ranks processed over the slowest rank's time."""
    return n_per_rank * world * steps / seconds


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload():
    import synth.workloads
    return synth.workloads.get("sipm8x8_xy")


def cpu_oracle_rate(w, n_sample: int, seed: int, threads: int = 0):
    """Events/s of the FP64 oracle (as it stands) on a sample of the workload,
    on all host cores (threads = 0) or on `threads` threads."""
    import oracle
    pts, vals = w.fit_samples()
    coef, _, _ = oracle.lrf_fit(w.n_int, w.lo, w.hi, pts, vals)
    L = oracle.Lrf(oracle.XY, w.sensor_xy, w.n_int + (0,), w.lo + (0,), w.hi + (0,), coef)
    P = oracle.CgsParams(n_xy=w.n_xy, iters=w.iters, step_xy=w.step_xy, shrink=w.shrink)
    ev = w.events(n_sample, seed=seed)
    sig = ev.signals.astype(np.float64)
    all_cores = oracle.num_threads()
    if threads:
        oracle.set_num_threads(threads)
    try:
        used = oracle.num_threads()
        t0 = time.perf_counter()
        oracle.cgs(L, P, sig, gain_cog=w.gains)
        dt = time.perf_counter() - t0
    finally:
        if threads:
            oracle.set_num_threads(all_cores)
    return n_sample / dt, dt, used, (L, P, sig)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    w = workload()
    import oracle
    pts, vals = w.fit_samples()
    coef, _, _ = oracle.lrf_fit(w.n_int, w.lo, w.hi, pts, vals)
    L = oracle.Lrf(oracle.XY, w.sensor_xy, w.n_int + (0,), w.lo + (0,), w.hi + (0,), coef)
    P = oracle.CgsParams(n_xy=w.n_xy, iters=w.iters, step_xy=w.step_xy, shrink=w.shrink)
    n_step = args.ref_events
    ev = w.events(n_step * (args.warmup + args.steps), seed=w.event_seed)
    sig = ev.signals.astype(np.float64)
    for k in range(args.warmup):
        oracle.cgs(L, P, sig[k * n_step:(k + 1) * n_step], gain_cog=w.gains)
    t0 = time.perf_counter()
    for k in range(args.warmup, args.warmup + args.steps):
        oracle.cgs(L, P, sig[k * n_step:(k + 1) * n_step], gain_cog=w.gains)
    dt = time.perf_counter() - t0
    value = n_step * args.steps / dt
    sample = f"{n_step} events of the 10^6-event workload per step, FP64 C oracle with OpenMP"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_of(w, w.n_events),
        "cpu_baseline": {"value": value, "unit": "events/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "events/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def config_of(w, n_events):
    return {"workload": f"{w.name}: {w.n_sensors} sensors, XY B-spline LRF {w.n_int[0]}x{w.n_int[1]} intervals, "
                        f"{n_events} events, contracting grid {w.n_xy}x{w.n_xy} x {w.iters} grids",
            "n_events": n_events, "n_sensors": w.n_sensors, "grid": f"{w.n_xy}x{w.n_xy}", "iters": w.iters,
            "method": "plain FP32 contracting grids", "l2": "inputs larger than L2 (256 MB of signals per step)"}


def forms_comparison(args, ants, torch, ctx, stream):
    """Plain contracting grids vs the learned form (network start + 5x5x4
    refine + deviance fallback) on the 16x16 SiPM detector, same events."""
    import synth.workloads
    w = synth.workloads.get("sipm16x16_xy")
    t0 = time.perf_counter()
    det = ants.Detector(w.sensor_xy, w.gains)
    pts, vals = w.fit_samples()
    lrf = ants.Lrf.fit(ctx, det, ants.ANTS_LRF_XY, w.n_int, w.lo, w.hi, pts, vals)
    plain = ants.CgsParams(n_xy=w.n_xy, iters=w.iters, step_xy=w.step_xy, shrink=w.shrink)
    refine = ants.CgsParams(n_xy=5, iters=4, step_xy=0.5, shrink=0.5)
    # events from the library's GPU simulator (Poisson counts from the fitted LRFs)
    src = ants.SimParams("square", 24.0, 0.0, 0.0, 0.0, 0.0, 2000.0, 0.05, 0.0)
    tsig, truth = ants.simulate(ctx, lrf, src, args.train_events, seed=2001)
    mlp = ants.Mlp.create(ctx, w.n_sensors, 256, 25.6, float(np.log(2000.0)), 0.05, seed=2001)
    torch.cuda.synchronize()
    t_tr = time.perf_counter()
    rep = mlp.train(tsig, truth, ants.TrainParams(epochs=20, batch=1024, bf16=1, seed=2001))
    train_s = time.perf_counter() - t_tr  # the call is synchronous
    del tsig, truth
    csig, _ = ants.simulate(ctx, lrf, src, 20000, seed=2002)
    rc = ants.reconstruct(ctx, lrf, plain, csig)
    Dc = torch.empty(csig.shape[0], device="cuda")
    ants.ants_deviance(ctx.handle, lrf.handle, csig, rc.xyz, Dc)
    thr = float(np.quantile(Dc.cpu().numpy(), 0.995))
    sp = ants.seeded_params(mlp, refine, plain, deviance_max=thr, border_fallback=True, bf16=1)
    table = ants.LogTable(ctx, lrf, 64, 64)
    gp = table.params(ants.CgsParams(n_xy=7, iters=5, step_xy=0.8 / 3, shrink=0.5), top_k=8, nms_cells=1.5)
    sig, etruth = ants.simulate(ctx, lrf, src, args.forms_events, seed=3001)
    torch.cuda.synchronize()
    true_xy = etruth[:, :2].double().cpu().numpy()
    n = sig.shape[0]
    setup_s = time.perf_counter() - t0
    # candidates the precision form refines per event: the top-8 grid points
    # minus those within 1.5 cells of a better kept one (same rule as the library)
    _, ix8 = table.topk(sig, 8)
    gx, gy = (ix8 % 64).long(), (ix8 // 64).long()
    kept = torch.zeros(ix8.shape, dtype=torch.bool, device=ix8.device)
    kept[:, 0] = True
    for j in range(1, 8):
        ok = (ix8[:, j] >= 0) & (ix8[:, j] < 64 * 64)
        for q in range(j):
            near = torch.maximum((gx[:, j] - gx[:, q]).abs(), (gy[:, j] - gy[:, q]).abs()) <= 1.5
            ok &= ~(near & kept[:, q])
        kept[:, j] = ok
    kept_per_event = float(kept.sum()) / kept.shape[0]
    del ix8, gx, gy, kept
    out = {}
    # the precision form reads its signals as FP16 (photo-electron counts below
    # 2048 are exact in FP16, so all three forms see the same events)
    sig16 = sig.half()
    assert bool((sig16.float() == sig).all())
    mp = ants.MinimizeParams(max_iter=40, tol=1e-3)
    for name, method, params, s_in in (("plain", ants.ANTS_CGS_PLAIN, plain, sig),
                                       ("learned", ants.ANTS_MLP_SEEDED, sp, sig),
                                       ("precision", ants.ANTS_GEMM_TOPK, gp, sig16),
                                       ("minimize", ants.ANTS_MINIMIZE, mp, sig)):
        tr = name == "minimize"
        res = ants.reconstruct(ctx, lrf, params, s_in, method=method, stream=stream, want_trace=tr)
        for _ in range(2):
            ants.reconstruct(ctx, lrf, params, s_in, method=method, stream=stream, want_trace=tr)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.forms_steps):
            res = ants.reconstruct(ctx, lrf, params, s_in, method=method, stream=stream, want_trace=tr)
        e1.record(stream)
        torch.cuda.synchronize()
        dt = e0.elapsed_time(e1) / 1e3 / args.forms_steps
        d = res.xyz[:, :2].double().cpu().numpy() - true_xy
        err = np.sqrt((d ** 2).sum(1))
        st = res.status.cpu().numpy()
        fb_frac = float((st == ants.ANTS_EVT_FALLBACK).mean())
        trials = float(np.abs(res.trace[:, 0].cpu().numpy().astype(np.int64)).mean()) + 1.0 if tr else 0.0
        evals = n * {"plain": plain.n_xy ** 2 * plain.iters,
                     "learned": refine.n_xy ** 2 * refine.iters + fb_frac * plain.n_xy ** 2 * plain.iters,
                     "precision": kept_per_event * 7 * 7 * 5, "minimize": trials}[name] * w.n_sensors
        kind = {"plain": "xy", "minimize": "xy_minimize"}.get(name, "local")
        out[name] = {"events_per_s": n / dt, "ms_per_step": 1e3 * dt,
                     "evals_per_s": evals / dt,
                     "roofline": alu_roofline(evals / dt, kind),
                     "rms_dxy_mm": float(np.sqrt((err ** 2).mean())),
                     "median_dxy_mm": float(np.median(err)), "p95_dxy_mm": float(np.quantile(err, 0.95)),
                     "fallback_frac": fb_frac}
    out["minimize"]["mean_trials"] = trials - 1.0
    for k in ("learned", "precision", "minimize"):
        out[k]["speedup_vs_plain"] = out[k]["events_per_s"] / out["plain"]["events_per_s"]
        out[k]["rms_ratio_vs_plain"] = out[k]["rms_dxy_mm"] / out["plain"]["rms_dxy_mm"]
    out["precision"]["refines_per_event"] = kept_per_event
    # the precision form's tensor-core scan on its own (tcgen05 product + top-8)
    sc = torch.empty((n, 8), device="cuda")
    ix = torch.empty((n, 8), dtype=torch.int32, device="cuda")
    for _ in range(3):
        ants.ants_logtable_topk(ctx.handle, table.handle, sig, 8, sc, ix, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.forms_steps):
        ants.ants_logtable_topk(ctx.handle, table.handle, sig, 8, sc, ix, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) / 1e3 / args.forms_steps
    flop = 2.0 * n * 64 * 64 * w.n_sensors
    pk, pk_kind = peaks()
    peak = float(pk.get("bf16_tflops", 1900.0))
    out["precision"]["scan_roofline"] = {
        "kernel": "umma_tn_kernel<TOPK> (tcgen05 BF16 product, fused top-8)", "bound": "tensor",
        "achieved": flop / dt / 1e12, "peak": peak, "unit": "TFLOP/s", "frac": flop / dt / 1e12 / peak,
        "ms": 1e3 * dt, "flop_per_event": 2 * 64 * 64 * w.n_sensors,
        "peak_kind": f"{pk_kind} bf16 burst (cuBLAS 8192^3)"}
    del sc, ix, sig, sig16
    out["vs_oracle_fp64"] = forms_vs_oracle(args, ants, torch, ctx, w, lrf, (
        ("plain", ants.ANTS_CGS_PLAIN, plain), ("learned", ants.ANTS_MLP_SEEDED, sp),
        ("precision", ants.ANTS_GEMM_TOPK, gp), ("minimize", ants.ANTS_MINIMIZE, mp)), stream)
    return {"workload": f"{w.name}: 256 sensors, XY LRF 32x32, {n} events; plain {w.n_xy}x{w.n_xy}x{w.iters} vs "
                        f"MLP 256-256-256-3 (BF16, trained on the GPU on {args.train_events} events, "
                        f"{rep.epochs_run} epochs) + refine 5x5x4 + fallback at the 99.5 % deviance quantile; precision form: "
                        f"FP16 signals, 64x64 BF16 log-response table, tcgen05 top-8, suppression 1.5 cells, "
                        f"refine 7x7x5; continuous minimisation from the centroid (at most 40 trials, tol 1e-3 mm)",
            "training": {"events": args.train_events, "epochs": rep.epochs_run, "seconds": train_s,
                         "events_epochs_per_s": args.train_events * rep.epochs_run / train_s,
                         "best_monitor_mse": rep.best_monitor_mse,
                         "products": "BF16 tcgen05 (hidden layers, forward, backward, weight gradients)"},
            "short": f"{w.name}: 256 sensors, {n} events (same events for every form)",
            "setup_s": setup_s, "deviance_max": thr, **out}


def forms_vs_oracle(args, ants, torch, ctx, w, lrf, forms, stream):
    """Each form's position and energy error against the FP64 oracle's plain
    contracting-grid search (same grid as the plain form) on a sample of
    events drawn by the seeded numpy generator; the oracle's LRF is its own
    FP64 fit of the same samples the library's LRF was fitted to."""
    import oracle
    n = args.oracle_events
    ev = w.events(n, seed=4001)
    pts, vals = w.fit_samples()
    coef, _, _ = oracle.lrf_fit(w.n_int, w.lo, w.hi, pts, vals)
    L = oracle.Lrf(oracle.XY, w.sensor_xy, w.n_int + (0,), w.lo + (0.0,), w.hi + (0.0,), coef)
    P = oracle.CgsParams(n_xy=w.n_xy, iters=w.iters, step_xy=w.step_xy, shrink=w.shrink)
    t0 = time.perf_counter()
    ref = oracle.cgs(L, P, ev.signals.astype(np.float64), gain_cog=w.gains)
    t_or = time.perf_counter() - t0
    sig = torch.from_numpy(ev.signals).cuda()
    sig16 = sig.half()
    assert bool((sig16.float() == sig).all())  # counts below 2048: exact in FP16
    out = {"events": n, "oracle": f"FP64 plain {w.n_xy}x{w.n_xy}x{w.iters} search, {oracle.num_threads()} threads, "
                                  f"{t_or:.1f} s"}
    ok_ref = ref["status"] == 0
    for name, method, params in forms:
        r = ants.reconstruct(ctx, lrf, params, sig16 if method == ants.ANTS_GEMM_TOPK else sig, method=method,
                             stream=stream)
        torch.cuda.synchronize()
        xyz = r.xyz.double().cpu().numpy()
        E = r.E.double().cpu().numpy()
        ok = ok_ref & np.isfinite(xyz[:, 0]) & np.isfinite(E)
        d = np.hypot(xyz[ok, 0] - ref["xyz"][ok, 0], xyz[ok, 1] - ref["xyz"][ok, 1])
        dE = np.abs(E[ok] / ref["E"][ok] - 1.0)
        out[name] = {"rms_dxy_mm": float(np.sqrt((d ** 2).mean())), "p95_dxy_mm": float(np.quantile(d, 0.95)),
                     "max_dxy_mm": float(d.max()), "rms_dE_rel": float(np.sqrt((dE ** 2).mean())),
                     "p95_dE_rel": float(np.quantile(dE, 0.95)), "compared": int(ok.sum())}
    return out


def _g(x, digits=4):
    """x rounded to a few significant digits (compact JSON)."""
    return None if x is None else float(f"{x:.{digits}g}")


def forms_compact(f):
    """The forms comparison reduced to the numbers the metric needs: events/s
    of each form on the same events, RMS error against the truth, ratios to
    the plain search (same error: RMS ratio <= 1.02), each form's error
    against the FP64 oracle's plain search, and the tensor-core scan's
    roofline."""
    if f is None or "error" in f:
        return f
    c = {"workload": f["short"]}
    for k in ("plain", "learned", "precision", "minimize"):
        o = f[k]
        d = {"events_per_s": _g(o["events_per_s"]), "rms_dxy_mm": _g(o["rms_dxy_mm"])}
        if k != "plain":
            d.update(speedup=_g(o["speedup_vs_plain"], 3), rms_ratio=_g(o["rms_ratio_vs_plain"]),
                     same_error=bool(o["rms_ratio_vs_plain"] <= 1.02))
        d["roofline_frac"] = _g(o["roofline"]["frac"], 3)
        c[k] = d
    c["learned"]["fallback_frac"] = _g(f["learned"]["fallback_frac"], 3)
    c["learned"]["train_s"] = _g(f["training"]["seconds"], 3)
    sr = f["precision"]["scan_roofline"]
    c["precision"]["scan"] = {"tflops": _g(sr["achieved"]), "frac": _g(sr["frac"], 3), "ms": _g(sr["ms"])}
    vo = f["vs_oracle_fp64"]
    c["vs_oracle_fp64"] = {"events": vo["events"], **{
        k: {"rms_dxy_mm": _g(v["rms_dxy_mm"], 3), "p95_dxy_mm": _g(v["p95_dxy_mm"], 3),
            "rms_dE_rel": _g(v["rms_dE_rel"], 3)} for k, v in vo.items() if isinstance(v, dict)}}
    c["chosen"] = "learned"
    return c


def radial_run(args, ants, torch, ctx, stream):
    """19-PMT hexagonal detector with one radial LRF (9x9 grid, 6 grids):
    throughput on 10^6 events (the workload's 10^4 events take under a
    millisecond, too short to time) and accuracy against the true positions."""
    import synth.workloads
    w = synth.workloads.get("hex19_radial")
    det = ants.Detector(w.sensor_xy, w.gains)
    pts, vals = w.fit_samples()
    lrf = ants.Lrf.fit(ctx, det, ants.ANTS_LRF_RADIAL, w.n_int, w.lo, w.hi, pts, vals, shared=True)
    p = ants.CgsParams(n_xy=w.n_xy, iters=w.iters, step_xy=w.step_xy, shrink=w.shrink)
    out = {}
    for n in (w.n_events, 1_000_000):
        ev = w.events(n, seed=w.event_seed)
        sig = torch.from_numpy(ev.signals).cuda()
        for _ in range(3):
            res = ants.reconstruct(ctx, lrf, p, sig, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 5
        e0.record(stream)
        for _ in range(reps):
            res = ants.reconstruct(ctx, lrf, p, sig, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        dt = e0.elapsed_time(e1) / 1e3 / reps
        d = res.xyz[:, :2].double().cpu().numpy() - ev.xyz[:, :2]
        evals = n * w.n_xy * w.n_xy * w.iters * w.n_sensors
        out[str(n)] = {"events_per_s": n / dt, "ms_per_launch": 1e3 * dt, "evals_per_s": evals / dt,
                       "roofline": alu_roofline(evals / dt, "radial"),
                       "rms_dxy_mm": float(np.sqrt((d ** 2).sum(1).mean()))}
    return {"workload": "hex19_radial: 19 PMTs, hexagonal, pitch 30 mm, one radial LRF (20 intervals on [0,150] mm), "
                        "contracting grid 9x9 x 6 grids, plain FP32", **out}


def variants_run(args, ants, torch, ctx, stream):
    """Search variants (Sec. 5.1.2, 5.3) on the 8x8 SiPM workload, 10^6
    events: maximum likelihood through the per-node variant kernel, least
    squares, and maximum likelihood with the strongest-sensor start, signal
    and distance cuts and a passive sensor; events/s and the XY roofline."""
    import synth.workloads
    w = workload()
    det = ants.Detector(w.sensor_xy, w.gains)
    pts, vals = w.fit_samples()
    lrf = ants.Lrf.fit(ctx, det, ants.ANTS_LRF_XY, w.n_int, w.lo, w.hi, pts, vals)
    p = ants.CgsParams(n_xy=w.n_xy, iters=w.iters, step_xy=w.step_xy, shrink=w.shrink)
    n = 1_000_000
    ev = w.events(n, seed=w.event_seed)
    sig = torch.from_numpy(ev.signals).cuda()
    pas = np.zeros(w.n_sensors, dtype=np.uint8)
    pas[27] = 1
    cases = {"ml": ants.VariantParams(p),
             "ls": ants.VariantParams(p, criterion=ants.ANTS_CRIT_LS),
             "ml_max_sensor_cuts_passive": ants.VariantParams(p, start=ants.ANTS_START_MAX_SENSOR, min_signal=60.0,
                                                              max_distance=25.0, passive=pas)}
    out = {}
    evals = n * w.n_xy * w.n_xy * w.iters * w.n_sensors
    for name, vp in cases.items():
        for _ in range(2):
            res = ants.reconstruct(ctx, lrf, vp, sig, stream=stream, method=ants.ANTS_CGS_VARIANT)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(2):
            res = ants.reconstruct(ctx, lrf, vp, sig, stream=stream, method=ants.ANTS_CGS_VARIANT)
        e1.record(stream)
        torch.cuda.synchronize()
        dt = e0.elapsed_time(e1) / 1e3 / 2
        d = res.xyz[:, :2].double().cpu().numpy() - ev.xyz[:, :2]
        ok = res.status.cpu().numpy() == 0
        out[name] = {"events_per_s": n / dt, "ms_per_launch": 1e3 * dt,
                     "roofline": alu_roofline(evals / dt, "xy"),
                     "rms_dxy_mm": float(np.sqrt((d[ok] ** 2).sum(1).mean())), "ok_frac": float(ok.mean())}
    return {"workload": f"{w.name}: 64 sensors, XY LRF, {n} events, 11x11 x 8 grids; per-node variant kernel "
                        "(least squares evaluates every node twice); cuts: signal >= 60, within 25 mm of the "
                        "strongest sensor, sensor 27 passive", **out}


def minimize_run(args, ants, torch, ctx, stream):
    """The continuous minimisation (Sec. 5.1.2.1) on the 8x8 SiPM workload,
    10^6 events: from the centroid (maximum likelihood), and as a refine of
    shorter contracting grids (11x11 x 4 grids, then the minimisation from
    their result) beside the plain 11x11 x 8 search; events/s, RMS error,
    trials, and the rate of sensor evaluations with gradient against the ALU
    ceiling (70 FMA per evaluation: value and gradient of the tensor spline,
    the weights and their derivatives, the Fisher and gradient sums)."""
    w = workload()
    det = ants.Detector(w.sensor_xy, w.gains)
    pts, vals = w.fit_samples()
    lrf = ants.Lrf.fit(ctx, det, ants.ANTS_LRF_XY, w.n_int, w.lo, w.hi, pts, vals)
    n = 1_000_000
    ev = w.events(n, seed=w.event_seed)
    sig = torch.from_numpy(ev.signals).cuda()
    mp = ants.MinimizeParams(max_iter=40, tol=1e-3)
    short = ants.CgsParams(n_xy=w.n_xy, iters=4, step_xy=w.step_xy, shrink=w.shrink)
    plain = ants.CgsParams(n_xy=w.n_xy, iters=w.iters, step_xy=w.step_xy, shrink=w.shrink)
    trace = torch.empty((n, 1), dtype=torch.int16, device="cuda")
    xyz0 = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    E0, L0 = torch.empty(n, device="cuda"), torch.empty(n, device="cuda")
    st0 = torch.empty(n, dtype=torch.int32, device="cuda")

    def minimize(start=None):
        r = ants.Result(torch.empty((n, 3), device="cuda"), torch.empty(n, device="cuda"),
                        torch.empty(n, device="cuda"), torch.empty(n, dtype=torch.int32, device="cuda"), trace)
        ants.ants_reconstruct(ctx.handle, lrf.handle, ants.ANTS_MINIMIZE, mp, sig, w.n_sensors, r.xyz, r.E, r.logL,
                              r.status, start_xyz=start, trace=trace, stream=stream)
        return r

    def refine():
        ants.ants_reconstruct(ctx.handle, lrf.handle, ants.ANTS_CGS_PLAIN, short, sig, w.n_sensors, xyz0, E0, L0, st0,
                              stream=stream)
        return minimize(xyz0)

    def grid():
        return ants.reconstruct(ctx, lrf, plain, sig, stream=stream)

    out = {}
    for name, fn in (("from_centroid", minimize), ("grids_11x11x4_then_refine", refine), ("plain_11x11x8", grid)):
        for _ in range(2):
            res = fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 3
        e0.record(stream)
        for _ in range(reps):
            res = fn()
        e1.record(stream)
        torch.cuda.synchronize()
        dt = e0.elapsed_time(e1) / 1e3 / reps
        ok = res.status.cpu().numpy() == 0
        d = res.xyz[:, :2].double().cpu().numpy() - ev.xyz[:, :2]
        o = {"events_per_s": n / dt, "ms_per_launch": 1e3 * dt, "ok_frac": float(ok.mean()),
             "rms_dxy_mm": float(np.sqrt((d[ok] ** 2).sum(1).mean()))}
        if name != "plain_11x11x8":
            t = trace[:, 0].cpu().numpy().astype(np.int64)
            o["mean_trials"] = float(np.abs(t[ok]).mean())
            o["converged_frac"] = float((t[ok] > 0).mean())
            if name == "from_centroid":
                evals = float(np.abs(t[ok]).sum() + ok.sum()) * w.n_sensors  # the start's pass and one per trial
                o["roofline"] = alu_roofline(evals / dt, "xy_minimize")
        out[name] = o
    return {"workload": f"{w.name}: 64 sensors, XY LRF, {n} events; damped Fisher scoring (maximum likelihood, "
                        "E profiled), at most 40 trials, tol 1e-3 mm", **out}


def _optics_stack(ants, pre_reject=0):
    """A 4 x 4 SiPM array (pitch 8 mm, 6 mm windows) under a 2 mm light guide
    (n 1.5), a 10 mm scintillator (n 1.8, absorption 100 mm, Rayleigh 40 mm)
    and a 2 mm window (n 1.5) with a diffuse reflector on top; lateral walls
    at 20 mm, a partly absorbing, partly specular floor between the windows."""
    g = np.arange(4) * 8.0 - 12.0
    sxy = np.array([(x, y) for y in g for x in g])
    qe = 0.2 + 0.1 * np.random.default_rng(4).uniform(size=16)
    return ants.OpticsParams(z=(0.0, 2.0, 12.0, 14.0), n=(1.5, 1.8, 1.5), abs_len=(200.0, 100.0, 0.0),
                             ray_len=(0.0, 40.0, 0.0), sensor_xy=sxy, sensor_size=6.0, qe=qe, n_below=1.0,
                             n_above=1.0, half_x=20.0, half_y=20.0, p_abs=(0.3, 0.0, 0.0, 0.1),
                             p_spec=(0.2, 0.0, 0.0, 0.0), p_diff=(0.0, 0.0, 0.0, 0.9), n_sensor=1.5,
                             ang=[1.0, 0.98, 0.9, 0.7, 0.3], max_cycles=200, pre_reject=pre_reject), sxy


def optics_run(args, ants, torch, ctx, stream):
    """Optical photon transport (Sec. 4.2.3-4.2.6): photons/s of the FP32 and
    FP64 kernels (64 sources x 10^6 photons in the scintillator, with and
    without pre-rejection), then the chain the simulation serves: light
    response on a 17 x 17 grid of sources (2 x 10^5 photons each) -> XY LRFs
    fitted on the device -> 20000 events of 4000 photons traced by the same
    simulator and reconstructed (plain 11 x 11 x 8) with those LRFs."""
    P, sxy = _optics_stack(ants)
    Pr, _ = _optics_stack(ants, pre_reject=1)
    rng = np.random.default_rng(5)
    src = torch.tensor(np.stack([rng.uniform(-15, 15, 64), rng.uniform(-15, 15, 64), rng.uniform(2.5, 11.5, 64)],
                                1).astype(np.float32)).cuda()
    n_ph = 1_000_000
    counts = torch.empty((64, 16), dtype=torch.int32, device="cuda")
    out = {}
    for name, params, prec in (("fp32", P, ants.ANTS_F32), ("fp64", P, ants.ANTS_F64),
                               ("fp32_prereject", Pr, ants.ANTS_F32)):
        ants.ants_trace_photons(ctx.handle, params, src, n_ph, 1, prec, counts, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        reps = 2
        e0.record(stream)
        for r in range(reps):
            ants.ants_trace_photons(ctx.handle, params, src, n_ph, 2 + r, prec, counts, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        dt = e0.elapsed_time(e1) / 1e3 / reps
        out[name] = {"photons_per_s": 64 * n_ph / dt, "ms_per_launch": 1e3 * dt,
                     "detected_frac": float(counts.sum()) / (64 * n_ph)}
    # light response on a grid -> LRFs -> reconstruction of traced events
    t0 = time.perf_counter()
    gx = np.linspace(-16.0, 16.0, 17)
    grid = np.array([(x, y, 7.0) for y in gx for x in gx], dtype=np.float32)
    _, _, eta = ants.trace_photons(ctx, P, torch.from_numpy(grid).cuda(), 200_000, 11, want_eta=True)
    det = ants.Detector(sxy)
    lrf = ants.Lrf.fit(ctx, det, ants.ANTS_LRF_XY, (8, 8), (-16.0, -16.0), (16.0, 16.0), grid[:, :2].astype(np.float64),
                       eta.double().cpu().numpy())
    n_ev = 20000
    truth = np.stack([rng.uniform(-12, 12, n_ev), rng.uniform(-12, 12, n_ev), np.full(n_ev, 7.0)], 1).astype(np.float32)
    sig, _, _ = ants.trace_photons(ctx, P, torch.from_numpy(truth).cuda(), 4000, 12)
    res = ants.reconstruct(ctx, lrf, ants.CgsParams(n_xy=11, iters=8, step_xy=4.0, shrink=0.5), sig.float())
    torch.cuda.synchronize()
    ok = res.status.cpu().numpy() == 0
    d = res.xyz[:, :2].double().cpu().numpy() - truth[:, :2]
    out["physical_lrf_chain"] = {"grid_sources": int(grid.shape[0]), "photons_per_grid_source": 200_000,
                                 "events": n_ev, "photons_per_event": 4000,
                                 "mean_detected_per_event": float(sig.float().sum(1).mean()),
                                 "ok_frac": float(ok.mean()), "rms_dxy_mm": float(np.sqrt((d[ok] ** 2).sum(1).mean())),
                                 "seconds": time.perf_counter() - t0}
    return {"workload": "slab stack over 4 x 4 SiPMs (guide n 1.5 / scintillator n 1.8, absorption 100 mm, "
                        "Rayleigh 40 mm / window n 1.5, diffuse reflector), 64 sources x 10^6 photons per launch",
            **out}


def schemes_run(args, ants, torch, ctx, stream):
    """The other LRF schemes (Sec. 6.1.1, 6.1.2) on a 4 x 4 SiPM array (pitch
    6 mm), LRFs fitted on the GPU to the closed-form truth (composite: the
    axial truth with a 5 % smooth XY term; axial+z and sliced: the 3D truth
    over z in [0, 20] mm, 5 planes), 10^6 events simulated on the GPU from
    each, reconstructed by the per-node kernel (composite 9x9 x 7 grids,
    3D 7x7x5 x 5 grids)."""
    import synth
    sxy = synth.square_array(4, 6.0)
    g = synth.sensor_gains(16, 0.05, 3)
    det = ants.Detector(sxy)
    rng = np.random.default_rng(2)
    p2 = rng.uniform(-12.0, 12.0, (40000, 2))
    v2 = synth.truth_eta(sxy, g, p2) * (1.0 + 0.05 * np.cos(p2[:, :1] / 7.0) * np.sin(p2[:, 1:] / 5.0))
    p3 = np.concatenate([p2, rng.uniform(0.0, 20.0, (40000, 1))], 1)
    p3s = np.concatenate([p2, rng.integers(0, 5, (40000, 1)) * 5.0], 1)
    lrfs = {
        "composite": ants.Lrf.fit_scheme(ctx, det, ants.ANTS_LRF_COMPOSITE, (8, 8), (-12.0, -12.0), (12.0, 12.0),
                                         p2, v2, n_int_r=12, hi_r=40.0),
        "axial_z": ants.Lrf.fit_scheme(ctx, det, ants.ANTS_LRF_AXIAL_Z, (12, 6), (0.0, 0.0), (40.0, 20.0), p3,
                                       synth.truth_eta(sxy, g, p3)),
        "sliced": ants.Lrf.fit_scheme(ctx, det, ants.ANTS_LRF_SLICED, (8, 8), (-12.0, -12.0, 0.0),
                                      (12.0, 12.0, 20.0), p3s, synth.truth_eta(sxy, g, p3s), n_planes=5)}
    n = 1_000_000
    out = {}
    for name, lrf in lrfs.items():
        three = name != "composite"
        src = ants.SimParams("square", 8.0, 0.0, 0.0, 0.0, 20.0 if three else 0.0, 4000.0, 0.05, 0.0)
        sig, truth = ants.simulate(ctx, lrf, src, n, seed=77)
        if three:
            p = ants.CgsParams(n_xy=7, iters=5, step_xy=2.0, n_z=5, step_z=4.0, z0=10.0)
            nodes = 7 * 7 * 5
        else:
            p = ants.CgsParams(n_xy=9, iters=7, step_xy=2.0)
            nodes = 81
        for _ in range(2):
            res = ants.reconstruct(ctx, lrf, p, sig, stream=stream)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(2):
            res = ants.reconstruct(ctx, lrf, p, sig, stream=stream)
        e1.record(stream)
        torch.cuda.synchronize()
        dt = e0.elapsed_time(e1) / 1e3 / 2
        evals = n * nodes * p.iters * 16
        d = (res.xyz - truth[:, :3]).double()
        out[name] = {"events_per_s": n / dt, "ms_per_launch": 1e3 * dt, "roofline": alu_roofline(evals / dt, name),
                     "rms_dxy_mm": float((d[:, :2] ** 2).sum(1).mean().sqrt()),
                     "rms_dz_mm": float((d[:, 2] ** 2).mean().sqrt()) if three else None}
    return {"workload": "4x4 SiPMs, pitch 6 mm; 10^6 events per scheme simulated from its own LRFs; composite "
                        "9x9 x 7 grids, axial+z and sliced 7x7x5 x 5 grids; per-node kernel", **out}


def iterative_run(args, ants, torch, ctx, stream):
    """Iterative LRF reconstruction (Sec. 8) from a flood of 10^6 events of the
    19-PMT detector (relative gains N(1, 0.1^2), known): from a too-wide
    simulated guess of the group's radial profile (the truth form with
    r0 = 55 mm instead of 40 mm), `iter_cycles` cycles of reconstruct - chi2 -
    cuts - FP64 refit, all on the GPU.  Reported: events x cycles per second of
    the whole procedure, the time of each stage, and the position error of
    the final LRFs against that of the true LRFs."""
    import synth
    import synth.workloads
    w = synth.workloads.get("hex19_radial")
    gains = synth.sensor_gains(19, 0.1, 5)
    det = ants.Detector(w.sensor_xy, gains)
    pts, vals = w.fit_samples()
    R = ants.ANTS_LRF_RADIAL

    def group(values):
        c = ants.Lrf.fit(ctx, det, R, w.n_int, w.lo, w.hi, pts, values, shared=True).coefficients()
        return ants.Lrf.from_coefficients(ctx, det, R, w.n_int, w.lo, w.hi, c, shared=True, gain=gains)

    lt = group(vals)
    lrf0 = group(synth.eta_axial(pts[:, 0], r0=55.0)[:, None])
    n, cycles = args.iter_events, args.iter_cycles
    sig = torch.empty((n, 19), device="cuda")
    truth = torch.empty((n, 4), device="cuda")
    src = ants.SimParams("disk", 60.0, 0.0, 0.0, 0.0, 0.0, 1e4, 0.05, 0.1)
    ants.ants_simulate_events(ctx.handle, lt.handle, src, 4321, 0, sig, truth)
    p = ants.CgsParams(n_xy=w.n_xy, iters=w.iters, step_xy=w.step_xy, shrink=w.shrink)
    cuts = ants.EventCuts(chi2_max=25.0)

    def rms(lrf):
        res = ants.reconstruct(ctx, lrf, p, sig, stream=stream)
        return float(((res.xyz[:, :2] - truth[:, :2]) ** 2).sum(1).mean().sqrt())

    lrf0.iterate(sig, p, 1, cuts)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lf, stats = lrf0.iterate(sig, p, cycles, cuts)
    dt = time.perf_counter() - t0
    # the stages on their own: the reconstruction (CUDA events), the refit of
    # all events (synchronous call, wall clock)
    for _ in range(2):
        res = ants.reconstruct(ctx, lrf0, p, sig, stream=stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(3):
        res = ants.reconstruct(ctx, lrf0, p, sig, stream=stream)
    e1.record(stream)
    torch.cuda.synchronize()
    t_rec = e0.elapsed_time(e1) / 1e3 / 3
    t1 = time.perf_counter()
    lrf0.refit(sig, res.xyz, res.E)
    t_fit = time.perf_counter() - t1
    evals = n * w.n_xy * w.n_xy * w.iters * w.n_sensors
    e_true, e_start, e_final = rms(lt), rms(lrf0), rms(lf)
    # the same procedure with the continuous minimisation as the reconstruction
    mp = ants.MinimizeParams(max_iter=40, tol=1e-3)
    lrf0.iterate(sig, mp, 1, cuts)  # warm-up
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lm, stats_m = lrf0.iterate(sig, mp, cycles, cuts)
    dt_m = time.perf_counter() - t0
    e_min = rms(lm)
    return {"workload": f"hex19 flood: 19 PMTs, radial LRF group with known gains N(1, 0.1^2), {n} events in a "
                        f"60 mm disk (E = 1e4 +- 5 %, Poisson, single-p.e. spread 0.1); start: the truth form with "
                        f"r0 = 55 mm; {cycles} cycles of contracting grids 9x9x6 - Pearson chi2 <= 25 - FP64 refit",
            "events": n, "cycles": cycles, "events_cycles_per_s": n * cycles / dt, "ms_per_cycle": 1e3 * dt / cycles,
            "reconstruct_ms": 1e3 * t_rec, "refit_ms": 1e3 * t_fit,
            "reconstruct_share": t_rec * cycles / dt,
            "reconstruct_roofline": alu_roofline(evals / t_rec, "radial"),
            "rms_dxy_mm": {"true_lrf": e_true, "start": e_start, "final": e_final, "final_over_true": e_final / e_true},
            "last_cycle": stats[-1],
            "with_minimisation": {"events_cycles_per_s": n * cycles / dt_m, "ms_per_cycle": 1e3 * dt_m / cycles,
                                  "final_rms_dxy_mm": e_min, "final_over_true": e_min / e_true,
                                  "last_cycle": stats_m[-1]}}


def batched_run(args, ants, torch, ctx, stream):
    """Eight detectors with 3D LRFs (19..256 sensors, 3e6 events) in one
    persistent launch per step (CUDA graph), launch shape autotuned."""
    import synth.workloads
    ws = synth.workloads.batch8_xyz()
    t0 = time.perf_counter()
    items, keep, truths = [], [], []
    for k, w in enumerate(ws):
        det = ants.Detector(w.sensor_xy, w.gains)
        pts, vals = w.fit_samples(per_interval=2)
        lrf = ants.Lrf.fit(ctx, det, ants.ANTS_LRF_XYZ, w.n_int, w.lo, w.hi, pts, vals)
        ev = w.event
        src = ants.SimParams(ev["region"], ev["extent"], 0.0, 0.0, ev["z_range"][0], ev["z_range"][1], ev["e0"], 0.05,
                             0.0)
        n = w.n_events if args.batch_scale >= 1.0 else max(1, int(w.n_events * args.batch_scale))
        sig, truth = ants.simulate(ctx, lrf, src, n, seed=w.event_seed)
        p = ants.CgsParams(n_xy=w.n_xy, iters=w.iters, step_xy=w.step_xy, shrink=w.shrink, n_z=w.n_z,
                           step_z=w.step_z, z0=w.z0)
        items.append((lrf, p, sig, None))
        keep.append((det, lrf))
        truths.append(truth)
    plan = ants.BatchPlan(ctx, items)
    cfg = plan.autotune(None, events_per_item=2048)
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t0
    plan.run(stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.batch_steps):
        plan.run(stream)
    e1.record(stream)
    torch.cuda.synchronize()
    dt = e0.elapsed_time(e1) / 1e3 / args.batch_steps
    n_tot = sum(int(it[2].shape[0]) for it in items)
    evals = sum(int(it[2].shape[0]) * it[0].n_sensors * it[1].n_xy * it[1].n_xy * it[1].n_z * it[1].iters
                for it in items)
    per = []
    for w, o, tr in zip(ws, plan.outs, truths):
        d = (o.xyz - tr[:, :3]).double()
        per.append({"detector": w.name, "events": int(o.xyz.shape[0]),
                    "rms_dxy_mm": float(d[:, :2].pow(2).sum(1).mean().sqrt()),
                    "rms_dz_mm": float(d[:, 2].pow(2).mean().sqrt())})
    return {"workload": f"8 detectors, XYZ LRFs 16x16x8, {n_tot} events, grid 7x7x5 x 7, one persistent launch "
                        f"per step (CUDA graph)", "events_per_s": n_tot / dt, "ms_per_step": 1e3 * dt,
            "evals_per_s": evals / dt, "roofline": alu_roofline(evals / dt, "xyz"),
            "steps": args.batch_steps, "setup_s": setup_s,
            "autotuned": {"unit_events": cfg.unit_events, "warps_per_block": cfg.warps_per_block,
                          "blocks_per_sm": cfg.blocks_per_sm}, "detectors": per}


def run_ours(args):
    import torch

    import paper_1602_07247_gb300 as ants
    from paper_1602_07247_gb300 import _build

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.cuda.current_device()
    if not os.path.exists(_build.LIB):
        _build.build()
    w = workload()
    n = args.events or w.n_events
    ctx = ants.Context(dev)
    det = ants.Detector(w.sensor_xy, w.gains)
    pts, vals = w.fit_samples()
    lrf = ants.Lrf.fit(ctx, det, ants.ANTS_LRF_XY, w.n_int, w.lo, w.hi, pts, vals)  # FP64 fit on the GPU
    p = ants.CgsParams(n_xy=w.n_xy, iters=w.iters, step_xy=w.step_xy, shrink=w.shrink)
    ev = w.events(n, seed=rank_seed(w.event_seed, rank))
    sig = torch.from_numpy(ev.signals).cuda()
    xyz = torch.empty((n, 3), dtype=torch.float32, device="cuda")
    E = torch.empty(n, dtype=torch.float32, device="cuda")
    logL = torch.empty(n, dtype=torch.float32, device="cuda")
    status = torch.empty(n, dtype=torch.int32, device="cuda")
    stream = torch.cuda.current_stream()

    def step():
        ants.ants_reconstruct(ctx.handle, lrf.handle, ants.ANTS_CGS_PLAIN, p, sig, w.n_sensors, xyz, E, logL,
                              status, stream=stream)
        return ants.last_launch_count()

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    clocks = ClockSampler(dev)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    launches = 0
    ev0.record(stream)
    for _ in range(args.steps):
        launches += step()
    ev1.record(stream)
    torch.cuda.synchronize()
    barrier()
    clk = clocks.stop()
    dt = max_over_ranks(ev0.elapsed_time(ev1) / 1e3)
    value = job_rate(n, world, args.steps, dt)
    kernel_s = dt / args.steps  # one kernel launch per step

    # accuracy of this run (not timed): RMS |dxy| against the true positions
    d = xyz[:, :2].double().cpu().numpy() - ev.xyz[:, :2]
    rms = float(np.sqrt((d ** 2).sum(1).mean()))

    # end-to-end through host buffers (H2D signals, D2H results inside the timed region)
    sig_host = torch.from_numpy(ev.signals).pin_memory()
    outs = {k: torch.empty(shape, dtype=dt_).pin_memory() for k, shape, dt_ in
            (("xyz", (n, 3), torch.float32), ("E", (n,), torch.float32), ("logL", (n,), torch.float32),
             ("status", (n,), torch.int32))}

    def step_host():
        ants.ants_reconstruct_host(ctx.handle, lrf.handle, ants.ANTS_CGS_PLAIN, p, sig_host, w.n_sensors,
                                   outs["xyz"], outs["E"], outs["logL"], outs["status"])

    for _ in range(max(1, args.warmup // 2)):
        step_host()
    e2e_steps = max(3, args.steps // 3)
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step_host()
    t_e2e = max_over_ranks(time.perf_counter() - t0)
    e2e = {"value": job_rate(n, world, e2e_steps, t_e2e), "unit": "events/s",
           "h2d_bytes_per_step": int(sig_host.numel() * 4),
           "d2h_bytes_per_step": int(sum(v.numel() * v.element_size() for v in outs.values()))}

    if rank != 0:
        if world > 1:
            import torch.distributed as dist
            dist.barrier()  # rank 0 prints after the others are done with the GPU collectives
            dist.destroy_process_group()
        return 0
    evals = n * w.iters * w.n_xy * w.n_xy * w.n_sensors
    traffic = None if XY_TRAFFIC_PER_EVENT is None else XY_TRAFFIC_PER_EVENT * n
    roofline = {**alu_roofline(evals / kernel_s, "xy"), "traffic": traffic, "traffic_unit": "bytes per launch",
                "thread_inst_per_eval": XY_INST_PER_EVAL}
    cpu = None
    if not args.no_cpu_baseline:
        rate, secs, cores, _ = cpu_oracle_rate(w, args.cpu_events, seed=w.event_seed)
        n1 = max(64, args.cpu_events // 8)
        rate1, secs1, _, _ = cpu_oracle_rate(w, n1, seed=w.event_seed, threads=1)
        cpu = {"value": rate, "unit": "events/s", "cores": cores, "kind": "oracle",
               "sample": f"{args.cpu_events} events of this workload ({secs:.1f} s), FP64 C oracle, OpenMP",
               "single_thread": {"value": rate1, "unit": "events/s", "cores": 1,
                                 "sample": f"{n1} events ({secs1:.1f} s), one thread"}}
    def optional(fn, skip):
        if skip or world > 1:
            return None
        try:
            return fn(args, ants, torch, ctx, stream)
        except Exception as exc:  # the headline line must still be printed
            return {"error": f"{type(exc).__name__}: {exc}"}

    # every optional section is printed as a line of its own (key "section"),
    # before the headline, which is the last line and carries the forms
    # comparison in compact form
    forms = None
    for name, fn, skip in (("forms_16x16", forms_comparison, args.no_forms),
                           ("radial_hex19", radial_run, args.no_forms),
                           ("batched_3d", batched_run, args.no_batched),
                           ("iterative_lrf", iterative_run, args.no_iterative),
                           ("variants_8x8", variants_run, args.no_variants),
                           ("lrf_schemes_4x4", schemes_run, args.no_schemes),
                           ("minimize_8x8", minimize_run, args.no_minimize),
                           ("optics_4x4", optics_run, args.no_optics)):
        r = optional(fn, skip)
        if r is None:
            continue
        if name == "forms_16x16":
            forms = r
        print(json.dumps({"section": name, **r}), flush=True)
    line = {
        "metric": METRIC, "value": value, "unit": "events/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic", "config": config_of(w, n),
        "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clk, "gpu_launches": launches,
        "rms_dxy_mm": rms, "forms": forms_compact(forms),
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--events", type=int, default=0, help="override the event count (default: workload's)")
    ap.add_argument("--cpu-events", type=int, default=4096)
    ap.add_argument("--ref-events", type=int, default=1024)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true", help="skip the plain vs learned comparison")
    ap.add_argument("--forms-events", type=int, default=4_000_000)
    ap.add_argument("--forms-steps", type=int, default=3)
    ap.add_argument("--train-events", type=int, default=1_000_000)
    ap.add_argument("--oracle-events", type=int, default=20_000,
                    help="events of the forms' comparison with the FP64 oracle's plain search")
    ap.add_argument("--no-batched", action="store_true", help="skip the 8-detector 3D batched run")
    ap.add_argument("--no-iterative", action="store_true", help="skip the iterative LRF reconstruction")
    ap.add_argument("--no-variants", action="store_true", help="skip the search variants")
    ap.add_argument("--no-schemes", action="store_true", help="skip the composite, axial+z and sliced LRFs")
    ap.add_argument("--no-minimize", action="store_true", help="skip the continuous minimisation")
    ap.add_argument("--no-optics", action="store_true", help="skip the optical photon transport")
    ap.add_argument("--iter-events", type=int, default=1_000_000)
    ap.add_argument("--iter-cycles", type=int, default=6)
    ap.add_argument("--batch-steps", type=int, default=1)
    ap.add_argument("--batch-scale", type=float, default=1.0, help="fraction of each detector's events")
    args = ap.parse_args()
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
