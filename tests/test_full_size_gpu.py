"""Parity at the benchmark's full sizes, in its launch configurations, on
sampled events: the 8-detector XYZ batch (3.0e6 events, one persistent launch)
and the 16x16 SiPM forms (4e6 events: precision form on FP16 signals, learned
form).  Sampled rows are replayed by the oracle; where a form's parts are
needed (candidate lists, network seeds) they are recomputed for the sampled
rows alone, which is exact because every row's result depends on that row
only (checked bit for bit)."""
import numpy as np
import pytest

import oracle
import synth
import synth.workloads
from parity import compare, gpu_objects, oracle_lrf, to_numpy

pytestmark = pytest.mark.gpu


def test_batch_full_size_sampled():
    import torch
    import paper_1602_07247_gb300 as ants
    ctx = ants.Context(0)
    ws = synth.workloads.batch8_xyz()
    items, keep = [], []
    for w in ws:
        det = ants.Detector(w.sensor_xy, w.gains)
        pts, vals = w.fit_samples(per_interval=2)
        lrf = ants.Lrf.fit(ctx, det, ants.ANTS_LRF_XYZ, w.n_int, w.lo, w.hi, pts, vals)
        ev = w.event
        src = ants.SimParams(ev["region"], ev["extent"], 0.0, 0.0, ev["z_range"][0], ev["z_range"][1], ev["e0"],
                             0.05, 0.0)
        sig, _ = ants.simulate(ctx, lrf, src, w.n_events, seed=w.event_seed)
        p = ants.CgsParams(n_xy=w.n_xy, iters=w.iters, step_xy=w.step_xy, shrink=w.shrink, n_z=w.n_z,
                           step_z=w.step_z, z0=w.z0)
        items.append((lrf, p, sig, None))
        keep.append((w, det, lrf))
    assert sum(int(it[2].shape[0]) for it in items) == 3_000_000
    plan = ants.BatchPlan(ctx, items, want_trace=True)
    plan.autotune(None, events_per_item=1024)
    plan.run()
    torch.cuda.synchronize()
    rng = np.random.default_rng(11)
    for (w, det, lrf), (_, _, sig, _), out in zip(keep, items, plan.outs):
        L = oracle_lrf(w, lrf.coefficients())
        idx = np.sort(rng.choice(w.n_events, 16, replace=False))
        res = {k: v[idx] for k, v in to_numpy(out).items()}
        stats = compare(w, L, sig[idx].cpu().numpy(), res)
        print(w.name, stats)


@pytest.fixture(scope="module")
def forms16():
    import torch
    import paper_1602_07247_gb300 as ants
    ctx = ants.Context(0)
    w = synth.workloads.get("sipm16x16_xy")
    L = oracle_lrf(w)
    _, det, lrf, plain = gpu_objects(w, L, ctx)
    src = ants.SimParams("square", 24.0, 0.0, 0.0, 0.0, 0.0, 2000.0, 0.05, 0.0)
    sig, truth = ants.simulate(ctx, lrf, src, 4_000_000, seed=3001)
    return torch, ants, ctx, w, L, lrf, plain, src, sig, truth


def test_precision_form_full_size_sampled(forms16):
    torch, ants, ctx, w, L, lrf, plain, src, sig, truth = forms16
    table = ants.LogTable(ctx, lrf, 64, 64)
    refine = ants.CgsParams(n_xy=7, iters=5, step_xy=0.8 / 3)
    gp = table.params(refine, top_k=8, nms_cells=1.5)
    sig16 = sig.half()
    res = to_numpy(ants.reconstruct(ctx, lrf, gp, sig16, method=ants.ANTS_GEMM_TOPK))
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(12).choice(sig.shape[0], 40, replace=False))
    rows = sig[torch.from_numpy(idx).cuda()].contiguous()
    alone = to_numpy(ants.reconstruct(ctx, lrf, gp, rows.half(), method=ants.ANTS_GEMM_TOPK))
    for k in ("xyz", "E", "logL", "status"):
        assert np.array_equal(res[k][idx], alone[k]), k
    _, ix = table.topk(rows, 8)
    ix = ix.cpu().numpy()
    nx, x0, dx = 64, -25.6 + 0.4, 0.8
    P = oracle.CgsParams(n_xy=7, iters=5, step_xy=0.8 / 3)
    sig64 = rows.double().cpu().numpy()
    best = np.full(len(idx), -np.inf)
    for e in range(len(idx)):
        kept = []
        for g in ix[e]:
            if all(max(abs(g % nx - h % nx), abs(g // nx - h // nx)) > 1.5 for h in kept):
                kept.append(g)
        starts = np.array([[np.float32(x0 + dx * (g % nx)), np.float32(x0 + dx * (g // nx)), 0.0] for g in kept])
        r = oracle.cgs(L, P, np.repeat(sig64[e:e + 1], len(kept), 0), start_xyz=starts)
        best[e] = r["logL"].max()
    _, got = oracle.energy_logl_at(L, sig64, alone["xyz"])
    assert np.all(got >= best - (1e-5 * np.abs(best) + 5e-3)), (best - got).max()
    assert np.abs(alone["logL"] / got - 1.0).max() < 1e-5


def test_learned_form_full_size_sampled(forms16):
    torch, ants, ctx, w, L, lrf, plain, src, sig, truth = forms16
    tsig, ttruth = ants.simulate(ctx, lrf, src, 200_000, seed=2001)
    M = ants.Mlp.create(ctx, w.n_sensors, 256, 25.6, float(np.log(2000.0)), 0.05, seed=2001)
    M.train(tsig, ttruth, ants.TrainParams(epochs=4, batch=1024, bf16=1, seed=2001))
    csig, _ = ants.simulate(ctx, lrf, src, 20_000, seed=2002)
    rc = ants.reconstruct(ctx, lrf, plain, csig)
    Dc = torch.empty(csig.shape[0], device="cuda")
    ants.ants_deviance(ctx.handle, lrf.handle, csig, rc.xyz, Dc)
    thr = float(np.quantile(Dc.cpu().numpy(), 0.995))
    refine = ants.CgsParams(n_xy=5, iters=4, step_xy=0.5)
    sp = ants.seeded_params(M, refine, plain, deviance_max=thr, border_fallback=True, bf16=1)
    res = to_numpy(ants.reconstruct(ctx, lrf, sp, sig, method=ants.ANTS_MLP_SEEDED))
    torch.cuda.synchronize()
    idx = np.sort(np.random.default_rng(13).choice(sig.shape[0], 200, replace=False))
    rows = sig[torch.from_numpy(idx).cuda()].contiguous()
    _, seeds, _ = M.forward(rows, bf16=1)
    seeds = seeds.clamp(-25.6, 25.6)
    seeds[:, 2] = 0.0
    ref = to_numpy(ants.reconstruct(ctx, lrf, refine, rows, start_xyz=seeds.contiguous(), want_trace=True))
    full = to_numpy(ants.reconstruct(ctx, lrf, plain, rows, want_trace=True))
    kept = res["status"][idx] == ants.ANTS_EVT_OK
    fb = res["status"][idx] == ants.ANTS_EVT_FALLBACK
    assert kept.sum() > 150
    assert np.array_equal(res["xyz"][idx][kept], ref["xyz"][kept])
    assert np.array_equal(res["xyz"][idx][fb], full["xyz"][fb])
    print("refine", compare(w.with_(n_xy=5, iters=4, step_xy=0.5), L, rows.cpu().numpy(), ref,
                            start=seeds.double().cpu().numpy()))
    print("fallback fraction (full size)", float((res["status"] == ants.ANTS_EVT_FALLBACK).mean()))
