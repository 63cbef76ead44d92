"""GPU parity of the plain contracting-grid search against the FP64 oracle.

Bar (FP32 path): |dxyz| <= 1e-3 mm and |dlogL|/|logL| <= 1e-5 against the
FP64 search replayed along the GPU's chosen nodes, where every choice must
score within the tie tolerance tau = 8 * 2^-24 * sum_i |s_i ln p_i| of the
FP64 best node; events without such a tie must follow the oracle's own path
exactly."""
import numpy as np
import pytest

import oracle
import synth
import synth.workloads
from parity import compare, gpu_objects, oracle_lrf, to_numpy

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch_cuda():
    import torch
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    return torch


@pytest.fixture(scope="module")
def ctx(torch_cuda):
    import paper_1602_07247_gb300 as ants
    return ants.Context(0)


def run_gpu(torch, ctx, lrf, p, sig, start=None):
    import paper_1602_07247_gb300 as ants
    s = torch.from_numpy(np.ascontiguousarray(sig, dtype=np.float32)).cuda()
    st = None if start is None else torch.from_numpy(np.asarray(start, dtype=np.float32)).cuda()
    res = ants.reconstruct(ctx, lrf, p, s, start_xyz=st, want_trace=True)
    torch.cuda.synchronize()
    return to_numpy(res)


@pytest.mark.parametrize("name,n", [("hex19_radial", 2001), ("sipm8x8_xy", 1003)])
def test_lrf_eval_matches_oracle(torch_cuda, ctx, name, n):
    torch = torch_cuda
    w = synth.workloads.get(name)
    L = oracle_lrf(w)
    _, det, lrf, _ = gpu_objects(w, L, ctx)
    rng = np.random.default_rng(1)
    half = 70.0 if w.lrf_type == "radial" else 24.0
    pts = rng.uniform(-half, half, (n, 2))
    got = lrf.eval(torch.from_numpy(pts.astype(np.float32)).cuda()).cpu().numpy()
    want = oracle.lrf_eval(L, pts.astype(np.float32).astype(np.float64))
    assert np.array_equal(np.isnan(got), np.isnan(want))
    ok = ~np.isnan(want)
    assert np.abs(got[ok] / want[ok] - 1.0).max() < 2e-6


@pytest.mark.parametrize("name,n", [("hex19_radial", 3001), ("sipm8x8_xy", 1501)])
def test_cgs_parity(torch_cuda, ctx, name, n):
    w = synth.workloads.get(name)
    L = oracle_lrf(w)
    _, det, lrf, p = gpu_objects(w, L, ctx)
    ev = w.events(n)
    gpu = run_gpu(torch_cuda, ctx, lrf, p, ev.signals)
    stats = compare(w, L, ev.signals, gpu)
    print(name, stats)
    assert stats["n"] == n
    # at most 5 % of the events need a certified tie (the XY kernel scores its
    # narrow last grids with an accurate log2(1 + u) of u = eta/eta_c - 1)
    assert stats["tie_frac"] < 0.05


def test_cgs_parity_given_start(torch_cuda, ctx):
    w = synth.workloads.get("sipm8x8_xy").with_(n_xy=5, iters=4, step_xy=0.5)
    L = oracle_lrf(w)
    _, det, lrf, p = gpu_objects(w, L, ctx)
    ev = w.events(517, seed=77)
    start = ev.xyz.copy()
    start[:, :2] += np.random.default_rng(3).normal(0.0, 0.4, (517, 2))
    start = np.clip(start, -23.0, 23.0).astype(np.float32).astype(np.float64)
    start[:, 2] = 0.0
    gpu = run_gpu(torch_cuda, ctx, lrf, p, ev.signals, start=start)
    stats = compare(w, L, ev.signals, gpu, start=start)
    print(stats)


def test_event_status_edge_cases(torch_cuda, ctx):
    w = synth.workloads.get("sipm8x8_xy")
    L = oracle_lrf(w)
    _, det, lrf, p = gpu_objects(w, L, ctx)
    sig = w.events(40, seed=5).signals.copy()
    sig[0] = 0.0
    sig[1, 7] = -2.0
    sig[2, 9] = np.nan
    sig[3, 63] = np.inf
    sig[4, :] = 0.0
    sig[4, 27] = 50.0  # a single lit sensor
    gpu = run_gpu(torch_cuda, ctx, lrf, p, sig)
    assert list(gpu["status"][:4]) == [2, 3, 3, 3]
    assert np.all(gpu["trace"][:4] == -1)
    compare(w, L, sig, gpu)


def test_empty_and_single_event(torch_cuda, ctx):
    torch = torch_cuda
    import paper_1602_07247_gb300 as ants
    w = synth.workloads.get("hex19_radial")
    L = oracle_lrf(w)
    _, det, lrf, p = gpu_objects(w, L, ctx)
    res = ants.reconstruct(ctx, lrf, p, torch.empty((0, 19), device="cuda"))
    assert res.xyz.shape == (0, 3)
    ev = w.events(1, seed=9)
    gpu = run_gpu(torch, ctx, lrf, p, ev.signals)
    compare(w, L, ev.signals, gpu)


def test_noise_free_recovery_gpu(torch_cuda, ctx):
    """s = E eta(x_true) with x_true on the first grid: the GPU lands on x_true."""
    w = synth.workloads.get("sipm8x8_xy").with_(n_xy=9, iters=4, step_xy=1.5)
    L = oracle_lrf(w)
    _, det, lrf, p = gpu_objects(w, L, ctx)
    xt = np.array([[3.25, -2.5, 0.0], [-6.5, 4.75, 0.0], [0.5, 0.25, 0.0], [12.0, -9.5, 0.0]])
    off = np.array([[2, -1, 0], [-3, 4, 0], [0, 1, 0], [1, 1, 0]], dtype=float)
    start = xt - off * 1.5
    s = 3000.0 * oracle.lrf_eval(L, xt[:, :2])
    gpu = run_gpu(torch_cuda, ctx, lrf, p, s, start=start)
    assert np.abs(gpu["xyz"] - xt).max() < 1e-5
    assert np.abs(gpu["E"] / 3000.0 - 1.0).max() < 1e-5


def test_host_buffers_match_device(torch_cuda, ctx):
    import paper_1602_07247_gb300 as ants
    w = synth.workloads.get("sipm8x8_xy")
    L = oracle_lrf(w)
    _, det, lrf, p = gpu_objects(w, L, ctx)
    n = 300_000  # more than two pipeline chunks, ragged last chunk
    ev = w.events(n, seed=21)
    res_h = ants.reconstruct_host(ctx, lrf, p, ev.signals)
    sig = torch_cuda.from_numpy(ev.signals).cuda()
    res_d = to_numpy(ants.reconstruct(ctx, lrf, p, sig))
    assert np.array_equal(res_h.status, res_d["status"])
    assert np.array_equal(res_h.xyz.astype(np.float64), res_d["xyz"], equal_nan=True)
    assert np.array_equal(res_h.logL.astype(np.float64), res_d["logL"], equal_nan=True)


def test_lrf_save_load_roundtrip(torch_cuda, ctx, tmp_path):
    import paper_1602_07247_gb300 as ants
    w = synth.workloads.get("hex19_radial")
    L = oracle_lrf(w)
    _, det, lrf, p = gpu_objects(w, L, ctx)
    path = str(tmp_path / "lrf.bin")
    lrf.save(path)
    lrf2 = ants.Lrf.load(ctx, det, path)
    assert np.array_equal(lrf2.coefficients(), lrf.coefficients())
    ev = w.events(200, seed=4)
    sig = torch_cuda.from_numpy(ev.signals).cuda()
    a = to_numpy(ants.reconstruct(ctx, lrf, p, sig))
    b = to_numpy(ants.reconstruct(ctx, lrf2, p, sig))
    assert np.array_equal(a["xyz"], b["xyz"])


def test_argument_errors_before_launch(torch_cuda, ctx):
    import paper_1602_07247_gb300 as ants
    w = synth.workloads.get("hex19_radial")
    L = oracle_lrf(w)
    _, det, lrf, p = gpu_objects(w, L, ctx)
    sig = torch_cuda.zeros((4, 18), device="cuda")
    with pytest.raises(ants.AntsError) as e:
        ants.reconstruct(ctx, lrf, p, sig)
    assert e.value.code == -5
    bad = ants.CgsParams(n_xy=4, iters=3, step_xy=1.0)
    with pytest.raises(ants.AntsError) as e:
        ants.reconstruct(ctx, lrf, bad, torch_cuda.zeros((4, 19), device="cuda"))
    assert e.value.code == -1


def test_full_size_sampled(torch_cuda, ctx):
    """10^6 events of the 8x8 SiPM workload in the benchmark's launch
    configuration; 400 sampled events replayed by the oracle."""
    import paper_1602_07247_gb300 as ants
    w = synth.workloads.get("sipm8x8_xy")
    L = oracle_lrf(w)
    _, det, lrf, p = gpu_objects(w, L, ctx)
    ev = w.events()
    sig = torch_cuda.from_numpy(ev.signals).cuda()
    res = ants.reconstruct(ctx, lrf, p, sig, want_trace=True)
    torch_cuda.cuda.synchronize()
    idx = np.random.default_rng(0).choice(w.n_events, 400, replace=False)
    idx.sort()
    gpu = {k: v[idx] for k, v in to_numpy(res).items()}
    stats = compare(w, L, ev.signals[idx], gpu)
    print(stats)
    st = res.status.cpu().numpy()
    assert np.all(st == 0)
    d = res.xyz.cpu().numpy()[:, :2] - ev.xyz[:, :2]
    rms = float(np.sqrt((d ** 2).sum(1).mean()))
    print("rms |dxy| vs truth", rms)
    assert rms < 2.0


@pytest.mark.parametrize("n_xy", [5, 7, 9, 11, 13, 15])
@pytest.mark.parametrize("rows", [3, 4])
def test_cgs_xy_grid_sizes_and_odd_sensor_counts(torch_cuda, ctx, n_xy, rows):
    """Every templated grid size of the separable XY kernel; 9 sensors (odd:
    one padding sensor) and 16 sensors (even)."""
    sxy = synth.square_array(rows, 6.0)
    half = 3.0 * rows
    w = synth.workloads.sipm8x8_xy().with_(
        name="small", sensor_xy=sxy, gains=synth.sensor_gains(rows * rows, 0.05, 7), n_int=(12, 12),
        lo=(-half, -half), hi=(half, half), n_xy=n_xy, iters=5, step_xy=2.0 * half / (n_xy - 1),
        event=dict(region="square", extent=half - 3.0, e0=2500.0))
    L = oracle_lrf(w)
    _, det, lrf, p = gpu_objects(w, L, ctx)
    ev = w.events(333, seed=n_xy * 10 + rows)
    gpu = run_gpu(torch_cuda, ctx, lrf, p, ev.signals)
    stats = compare(w, L, ev.signals, gpu)
    print(n_xy, rows, stats)


def test_cgs_xy_table_in_global_memory(torch_cuda, ctx):
    """16 x 16 SiPMs: the 1.25 MB coefficient table exceeds shared memory and
    is read through L1/L2 instead."""
    w = synth.workloads.get("sipm16x16_xy")
    L = oracle_lrf(w)
    _, det, lrf, p = gpu_objects(w, L, ctx)
    ev = w.events(257, seed=5)
    gpu = run_gpu(torch_cuda, ctx, lrf, p, ev.signals)
    stats = compare(w, L, ev.signals, gpu)
    print(stats)


@pytest.mark.parametrize("side,pitch,n_int,n_xy,step", [
    (16, 3.2, 32, 5, 0.5), (15, 3.2, 30, 5, 0.3), (10, 6.0, 48, 5, 0.5), (7, 6.0, 48, 5, 0.4),
    (16, 3.2, 32, 7, 0.8 / 3), (15, 3.2, 30, 7, 0.25), (10, 6.0, 48, 7, 0.3), (7, 6.0, 48, 7, 0.25)])
def test_cgs_xy_patch_kernel(torch_cuda, ctx, side, pitch, n_int, n_xy, step):
    """5 x 5 and 7 x 7 grids on a coefficient table larger than shared memory
    take the patch kernel (a team of warps per event, one sensor pair per lane;
    7 x 7 grids in three groups of columns): 16 x 16 and 15 x 15 SiPMs (teams
    of four warps; 15 x 15 is odd: one padding sensor), 10 x 10 (two warps) and
    7 x 7 (one warp, odd) on fine knot grids; starts near the sources, on the
    edges and in the corners of the field of view, and a zero-signal event."""
    sxy = synth.square_array(side, pitch)
    half = 0.5 * pitch * side
    w = synth.workloads.sipm16x16_xy().with_(
        name=f"sipm{side}x{side}", sensor_xy=sxy, gains=synth.sensor_gains(side * side, 0.05, 9 + side),
        lo=(-half, -half), hi=(half, half), n_int=(n_int, n_int), n_xy=n_xy, iters=4, step_xy=step,
        event=dict(region="square", extent=half - 0.5 * pitch, e0=2000.0))
    L = oracle_lrf(w)
    _, det, lrf, p = gpu_objects(w, L, ctx)
    n = 301
    ev = w.events(n, seed=40 + side)
    sig = ev.signals.copy()
    sig[7] = 0.0
    rng = np.random.default_rng(side)
    start = ev.xyz.copy()
    start[:, :2] += rng.normal(0.0, 0.4, (n, 2))
    start[:8, :2] = [[half, half], [-half, -half], [half, -half], [-half, half], [half, 0.0], [0.0, -half],
                     [half - 0.2, half - 0.7], [0.0, 0.0]]
    # starts in single precision inside the box (25.6 rounds up in FP32)
    s32 = np.clip(start, -half, half).astype(np.float32)
    out = np.abs(s32.astype(np.float64)) > half
    s32[out] = np.nextafter(s32[out], np.float32(0.0))
    start = s32.astype(np.float64)
    start[:, 2] = 0.0
    gpu = run_gpu(torch_cuda, ctx, lrf, p, sig, start=start)
    assert gpu["status"][7] == 2
    stats = compare(w, L, sig, gpu, start=start)
    print(side, n_int, n_xy, step, stats)
    assert stats["tie_frac"] < 0.05


def test_cgs_xyz_parity(torch_cuda, ctx):
    w = synth.workloads.get("sipm4x4_xyz")
    L = oracle_lrf(w)
    _, det, lrf, p = gpu_objects(w, L, ctx)
    ev = w.events(401, seed=3)
    gpu = run_gpu(torch_cuda, ctx, lrf, p, ev.signals)
    stats = compare(w, L, ev.signals, gpu)
    print(stats)
    d = np.abs(gpu["xyz"] - ev.xyz)
    print("median |dx|, |dz| vs truth", np.median(d[:, 0]), np.median(d[:, 2]))


@pytest.mark.parametrize("n_xy,n_z,iters,step_xy,step_z", [
    (7, 5, 5, 4.0, 5.0),    # separable path, the workload's grid
    (5, 3, 6, 12.0, 10.0),  # separable, first grids wider than the whole lattice
    (7, 1, 4, 3.0, 0.0),    # separable with a single z plane (z stays at z0)
    (9, 5, 4, 3.0, 4.0),    # 405 nodes: per-node evaluation
])
def test_cgs_xyz_grids(torch_cuda, ctx, n_xy, n_z, iters, step_xy, step_z):
    """XYZ searches through both evaluation paths against the oracle."""
    w = synth.workloads.get("sipm4x4_xyz").with_(n_xy=n_xy, n_z=n_z, iters=iters, step_xy=step_xy, step_z=step_z)
    L = oracle_lrf(w)
    _, det, lrf, p = gpu_objects(w, L, ctx)
    ev = w.events(157, seed=11 + n_xy)
    gpu = run_gpu(torch_cuda, ctx, lrf, p, ev.signals)
    print(compare(w, L, ev.signals, gpu))
