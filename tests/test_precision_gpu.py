"""Precision form on the GPU: log-response table against the FP64 oracle,
tensor-core top-K against an FP64 product of the same BF16 operands, and the
whole form against the oracle's refine of every candidate."""
import numpy as np
import pytest

import oracle
import synth
import synth.workloads
from parity import gpu_objects, oracle_lrf, oracle_params, to_numpy

pytestmark = pytest.mark.gpu


def bf16_round(x):
    """Round float32 to the nearest BF16 (ties to even) and back."""
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000
    return b.astype(np.uint32).view(np.float32)


@pytest.fixture(scope="module")
def setup16():
    import torch
    assert torch.cuda.is_available()
    import paper_1602_07247_gb300 as ants
    ctx = ants.Context(0)
    w = synth.workloads.get("sipm16x16_xy")
    L = oracle_lrf(w)
    _, det, lrf, plain = gpu_objects(w, L, ctx)
    table = ants.LogTable(ctx, lrf, 64, 64)
    return torch, ants, ctx, w, L, det, lrf, plain, table


def test_table_matches_oracle(setup16):
    torch, ants, ctx, w, L, det, lrf, plain, table = setup16
    T, m = table.values()
    To, mo = oracle.logtable(L, 64, 64)
    assert np.abs(m - mo).max() < 1e-4
    err = np.abs(T - To)
    assert np.all(err <= np.abs(To) * 2.0 ** -8 + 2e-4), err.max()


def test_topk_scores_match_fp64_product(setup16):
    torch, ants, ctx, w, L, det, lrf, plain, table = setup16
    ev = w.events(1037, seed=71)  # ragged against the 64-row tile
    sc, ix = table.topk(torch.from_numpy(ev.signals).cuda(), 8)
    sc, ix = sc.cpu().numpy(), ix.cpu().numpy()
    T, _ = table.values()  # the BF16 table values
    A = bf16_round(ev.signals).astype(np.float64)
    full = A @ T.astype(np.float64).T  # [n, 4096]
    bound = 256 * 2.0 ** -23 * (np.abs(A) @ np.abs(T.astype(np.float64)).T)
    rows = np.arange(ix.shape[0])[:, None]
    assert np.all(np.abs(sc - full[rows, ix]) <= bound[rows, ix] + 1e-6)
    assert np.all(np.diff(sc, axis=1) <= 0)
    kth = -np.sort(-full, axis=1)[:, 7]
    slack = bound.max(axis=1) * 2
    assert np.all(full[rows, ix] >= kth[:, None] - slack[:, None])


def test_precision_form_against_oracle_refines(setup16):
    torch, ants, ctx, w, L, det, lrf, plain, table = setup16
    refine = ants.CgsParams(n_xy=7, iters=5, step_xy=0.8 / 3)
    gp = table.params(refine, top_k=8, nms_cells=1.5)
    ev = w.events(301, seed=72)
    sig = torch.from_numpy(ev.signals).cuda()
    res = to_numpy(ants.reconstruct(ctx, lrf, gp, sig, method=ants.ANTS_GEMM_TOPK))
    _, ix = table.topk(sig, 8)
    ix = ix.cpu().numpy()
    T, _ = table.values()
    nx = 64
    x0, dx = -25.6 + 0.4, 0.8
    P = oracle.CgsParams(n_xy=7, iters=5, step_xy=0.8 / 3)
    sig64 = ev.signals.astype(np.float64)
    best_logl = np.full(len(ev.signals), -np.inf)
    for e in range(len(ev.signals)):
        kept = []
        for g in ix[e]:
            if all(max(abs(g % nx - h % nx), abs(g // nx - h // nx)) > 1.5 for h in kept):
                kept.append(g)
        starts = np.array([[np.float32(x0 + dx * (g % nx)), np.float32(x0 + dx * (g // nx)), 0.0] for g in kept])
        r = oracle.cgs(L, P, np.repeat(sig64[e:e + 1], len(kept), 0), start_xyz=starts)
        best_logl[e] = r["logL"].max()
    E, got_logl = oracle.energy_logl_at(L, sig64, res["xyz"])
    # the GPU's choice is (within FP32 noise) the best refine the oracle finds
    tol = 1e-5 * np.abs(best_logl) + 5e-3
    assert np.all(got_logl >= best_logl - tol), (best_logl - got_logl).max()
    assert np.abs(res["logL"] / got_logl - 1.0).max() < 1e-5
    full = to_numpy(ants.reconstruct(ctx, lrf, plain, sig))
    rms = lambda r: float(np.sqrt(((r["xyz"][:, :2] - ev.xyz[:, :2]) ** 2).sum(1).mean()))
    print("rms precision form", rms(res), "plain", rms(full))
    assert rms(res) <= 1.05 * rms(full)


def _check_topk(sig, T, sc, ix, k):
    """Scores equal the FP64 product of the BF16 operands within the FP32
    accumulation bound, lists are sorted, and no omitted column beats a kept one
    by more than that bound."""
    A = bf16_round(sig).astype(np.float64)
    full = A @ T.astype(np.float64).T
    bound = T.shape[1] * 2.0 ** -23 * (np.abs(A) @ np.abs(T.astype(np.float64)).T) + 1e-6
    rows = np.arange(ix.shape[0])[:, None]
    assert ix.shape[1] == k
    assert np.all((ix >= 0) & (ix < T.shape[0]))
    assert np.all(np.abs(sc - full[rows, ix]) <= bound[rows, ix])
    assert np.all(np.diff(sc, axis=1) <= 0)
    for r in range(ix.shape[0]):
        assert len(set(ix[r].tolist())) == k
    kth = -np.sort(-full, axis=1)[:, k - 1]
    assert np.all(full[rows, ix] >= kth[:, None] - 2 * bound.max(axis=1)[:, None])


@pytest.mark.parametrize("nx,ny,k,n", [(10, 10, 1, 1), (10, 10, 8, 129), (33, 31, 3, 300), (16, 16, 8, 257),
                                       (64, 64, 5, 128)])
def test_topk_edge_shapes_8x8(nx, ny, k, n):
    """K = 64 sensors; grids smaller than one 256-column tile, ragged against
    it, and exactly one tile; event counts of 1, one tile, and ragged."""
    import torch
    import paper_1602_07247_gb300 as ants
    ctx = ants.Context(0)
    w = synth.workloads.get("sipm8x8_xy")
    L = oracle_lrf(w)
    _, det, lrf, _ = gpu_objects(w, L, ctx)
    table = ants.LogTable(ctx, lrf, nx, ny)
    T, _ = table.values()
    assert T.shape == (nx * ny, 64)
    ev = w.events(n, seed=90 + nx + k)
    sc, ix = table.topk(torch.from_numpy(ev.signals).cuda(), k)
    _check_topk(ev.signals, T, sc.cpu().numpy(), ix.cpu().numpy(), k)
    assert ants.ants_ctx_fault(ctx.handle) == 0


def test_topk_many_bands_16x16(setup16):
    """More 128-row bands than SMs, so every block takes several bands in turn
    (the A chunks are refilled while the previous band's products finish)."""
    torch, ants, ctx, w, L, det, lrf, plain, table = setup16
    ev = w.events(152 * 128 * 2 + 77, seed=93)
    sig = torch.from_numpy(ev.signals).cuda()
    sc, ix = table.topk(sig, 8)
    sc, ix = sc.cpu().numpy(), ix.cpu().numpy()
    T, _ = table.values()
    pick = np.r_[0:200, len(ev.signals) - 300:len(ev.signals)]
    _check_topk(ev.signals[pick], T, sc[pick], ix[pick], 8)
    # every band agrees with a launch that sees it alone (no state leaks between bands)
    sc1, ix1 = table.topk(sig[-300:], 8)
    assert np.array_equal(ix1.cpu().numpy(), ix[-300:]) and np.array_equal(sc1.cpu().numpy(), sc[-300:])
    assert ants.ants_ctx_fault(ctx.handle) == 0


def test_fp16_signals_equal_their_fp32_values(setup16):
    """FP16 signals (the precision workload's storage type) give bit-identical
    results to the same values passed as FP32, for all three methods and the
    host-buffer path, across the 2^20-event conversion chunks' boundary logic."""
    torch, ants, ctx, w, L, det, lrf, plain, table = setup16
    ev = w.events(1531, seed=95)
    h = torch.from_numpy(ev.signals).cuda().to(torch.float16)
    f = h.float()
    gp = table.params(ants.CgsParams(n_xy=7, iters=5, step_xy=0.8 / 3), top_k=8, nms_cells=1.5)
    for params, method in ((plain, ants.ANTS_CGS_PLAIN), (gp, ants.ANTS_GEMM_TOPK)):
        a = to_numpy(ants.reconstruct(ctx, lrf, params, h, method=method))
        b = to_numpy(ants.reconstruct(ctx, lrf, params, f, method=method))
        for k in ("xyz", "E", "logL", "status"):
            assert np.array_equal(a[k], b[k], equal_nan=True), (method, k)
    hh = h.cpu().numpy()
    rh = ants.reconstruct_host(ctx, lrf, plain, hh)
    rf = ants.reconstruct_host(ctx, lrf, plain, hh.astype(np.float32))
    assert np.array_equal(rh.xyz, rf.xyz, equal_nan=True) and np.array_equal(rh.logL, rf.logL, equal_nan=True)
    with pytest.raises(ants.AntsError):
        ants.ants_reconstruct(ctx.handle, lrf.handle, ants.ANTS_CGS_PLAIN, plain, f, 256, *[torch.empty(
            s, device="cuda") for s in ((1531, 3), 1531, 1531)], torch.empty(1531, dtype=torch.int32, device="cuda"),
            signal_dtype=7)


def test_stalled_product_gives_up_and_the_context_recovers(setup16):
    """A tensor-core product whose producer never delivers stops after its
    bounded wait, reports through the fault word, and the next launch on the
    same context is correct (no GPU fault, trap or hang involved)."""
    torch, ants, ctx, w, L, det, lrf, plain, table = setup16
    ants.ants_selftest_stalled_product(ctx.handle)
    assert ants.ants_ctx_fault(ctx.handle) == 0
    ev = w.events(300, seed=97)
    sc, ix = table.topk(torch.from_numpy(ev.signals).cuda(), 8)
    T, _ = table.values()
    _check_topk(ev.signals, T, sc.cpu().numpy(), ix.cpu().numpy(), 8)


def test_host_buffer_path_precision_form(setup16):
    """The precision form through host buffers (chunks of 2^17 events run in
    turn) equals the device path bit for bit, also for FP16 host signals."""
    torch, ants, ctx, w, L, det, lrf, plain, table = setup16
    gp = table.params(ants.CgsParams(n_xy=7, iters=5, step_xy=0.8 / 3), top_k=8, nms_cells=1.5)
    ev = w.events(2500, seed=98)
    dev = to_numpy(ants.reconstruct(ctx, lrf, gp, torch.from_numpy(ev.signals).cuda(), method=ants.ANTS_GEMM_TOPK))
    host = ants.reconstruct_host(ctx, lrf, gp, ev.signals, method=ants.ANTS_GEMM_TOPK)
    for k in ("xyz", "E", "logL", "status"):
        assert np.array_equal(getattr(host, k), dev[k], equal_nan=True), k
    h16 = ants.reconstruct_host(ctx, lrf, gp, ev.signals.astype(np.float16), method=ants.ANTS_GEMM_TOPK)
    d16 = to_numpy(ants.reconstruct(ctx, lrf, gp, torch.from_numpy(ev.signals).cuda().half(),
                                    method=ants.ANTS_GEMM_TOPK))
    assert np.array_equal(h16.xyz, d16["xyz"], equal_nan=True)
