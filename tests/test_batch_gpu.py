"""Batched persistent reconstruction of several detectors in one launch
(radial, XY and XYZ LRFs mixed): every detector's results pass the same
oracle parity as separate launches; the captured graph reruns bit-identically;
the autotuner picks a launch shape and reuses its cache."""
import numpy as np
import pytest

import synth
import synth.workloads
from parity import compare, gpu_objects, oracle_lrf, to_numpy

pytestmark = pytest.mark.gpu


def test_batched_mixed_detectors(tmp_path):
    import torch
    assert torch.cuda.is_available()
    import paper_1602_07247_gb300 as ants
    ctx = ants.Context(0)
    ws = [synth.workloads.get("hex19_radial"), synth.workloads.get("sipm8x8_xy"), synth.workloads.get("sipm4x4_xyz")]
    bw = synth.workloads.batch8_xyz()
    ws.append(bw[0].with_(n_int=(8, 8, 4)))  # a hexagonal PMT array with a smaller 3D LRF
    counts = [301, 257, 199, 133]
    items, keep = [], []
    for w, n in zip(ws, counts):
        L = oracle_lrf(w) if w.lrf_type != "xyz" else None
        if L is None:
            pts, vals = w.fit_samples(per_interval=2)
            import oracle
            coef, _, _ = oracle.lrf_fit(w.n_int, w.lo, w.hi, pts, vals)
            L = oracle_lrf(w, coef)
        _, det, lrf, p = gpu_objects(w, L, ctx)
        ev = w.events(n, seed=40 + n)
        sig = torch.from_numpy(ev.signals).cuda()
        items.append((lrf, p, sig, None))
        keep.append((w, L, ev, det))
    plan = ants.BatchPlan(ctx, items, ants.BatchConfig(8, 4, 2), want_trace=True)
    plan.run()
    torch.cuda.synchronize()
    first = [to_numpy(o) for o in plan.outs]
    for (w, L, ev, det), res in zip(keep, first):
        stats = compare(w, L, ev.signals, res)
        print(w.name, stats)
    # graph rerun: identical
    plan.run()
    torch.cuda.synchronize()
    for a, o in zip(first, plan.outs):
        b = to_numpy(o)
        assert np.array_equal(a["xyz"], b["xyz"], equal_nan=True) and np.array_equal(a["trace"], b["trace"])
    # autotune (small per-item budget), then the cache answers without timing
    cache = str(tmp_path / "tune.txt")
    c1 = plan.autotune(cache, events_per_item=64)
    print("autotuned", c1.unit_events, c1.warps_per_block, c1.blocks_per_sm)
    c2 = plan.autotune(cache, events_per_item=64)
    assert (c1.unit_events, c1.warps_per_block, c1.blocks_per_sm) == (c2.unit_events, c2.warps_per_block,
                                                                        c2.blocks_per_sm)
    with open(cache) as f:
        assert len(f.readlines()) == 1
    plan.run()
    torch.cuda.synchronize()
    for a, o in zip(first, plan.outs):
        assert np.array_equal(a["xyz"], to_numpy(o)["xyz"], equal_nan=True)
