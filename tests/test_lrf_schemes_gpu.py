"""Composite, axial+z and sliced LRF sets (Sec. 6.1.1, 6.1.2) on the GPU
against the FP64 oracle: evaluation, the device fits, the event simulator and
the contracting-grid reconstruction (replayed by the oracle under the tie
rule)."""
import numpy as np
import pytest

import oracle
import pins
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    import paper_1602_07247_gb300 as ants
    return ants.Context(0)


def _gpu(ctx, L):
    import paper_1602_07247_gb300 as ants
    det = ants.Detector(L.sensor_xy)
    if L.type == oracle.COMPOSITE:
        return ants.Lrf.from_scheme(ctx, det, L.type, L.n_int[:2], L.lo[:2], L.hi[:2], L.coef, n_int_r=L.n_int_r,
                                    hi_r=L.hi_r)
    if L.type == oracle.AXIAL_Z:
        return ants.Lrf.from_scheme(ctx, det, L.type, L.n_int[:2], L.lo[:2], L.hi[:2], L.coef)
    return ants.Lrf.from_scheme(ctx, det, L.type, L.n_int[:2], L.lo, L.hi, L.coef, n_planes=L.n_planes)


def _realistic():
    """Scheme LRFs of a 4 x 4 array (pitch 6 mm) fitted by the oracle to the
    closed-form truth: composite (axial truth plus a 5 % smooth XY term),
    axial+z and sliced (5 planes) from the 3D truth over z in [0, 20] mm."""
    sxy = synth.square_array(4, 6.0)
    g = synth.sensor_gains(16, 0.05, 3)
    rng = np.random.default_rng(2)
    p2 = rng.uniform(-12.0, 12.0, (20000, 2))
    v2 = synth.truth_eta(sxy, g, p2) * (1.0 + 0.05 * np.cos(p2[:, :1] / 7.0) * np.sin(p2[:, 1:] / 5.0))
    comp = oracle.lrf_fit_composite(sxy, p2, v2, 12, 40.0, (8, 8), (-12.0, -12.0), (12.0, 12.0))
    p3 = np.concatenate([p2, rng.uniform(0.0, 20.0, (20000, 1))], 1)
    v3 = synth.truth_eta(sxy, g, p3)
    az = oracle.lrf_fit_axial_z(sxy, p3, v3, (12, 6), 40.0, 0.0, 20.0)
    p3s = np.concatenate([p2, rng.integers(0, 5, (20000, 1)) * 5.0], 1)
    sl = oracle.lrf_fit_sliced(sxy, p3s, synth.truth_eta(sxy, g, p3s), (8, 8), (-12.0, -12.0), (12.0, 12.0), 5,
                               0.0, 20.0)
    return sxy, g, comp, az, sl, (p2, v2, p3, v3, p3s)


@pytest.fixture(scope="module")
def realistic():
    return _realistic()


@pytest.mark.parametrize("k", [0, 1, 2], ids=["composite", "axial_z", "sliced"])
def test_eval_matches_oracle(ctx, k):
    import torch
    sxy, comp, az, sl = pins._scheme_lrfs()
    L = (comp, az, sl)[k]
    lrf = _gpu(ctx, L)
    rng = np.random.default_rng(5)
    d = 2 if k == 0 else 3
    pts = np.concatenate([rng.uniform(-11.9, 11.9, (4000, 2)), rng.uniform(0.0, 20.0, (4000, 1))], 1)[:, :d]
    pts[:3, 2 if d == 3 else 0] = [0.0, 10.0, 20.0] if d == 3 else pts[:3, 0]  # planes and range ends
    got = lrf.eval(torch.from_numpy(pts.astype(np.float32)).cuda()).cpu().numpy()
    want = oracle.lrf_eval(L, pts.astype(np.float32).astype(np.float64))
    ok = np.isfinite(want)
    assert np.array_equal(ok, np.isfinite(got))
    err = np.abs(got[ok] - want[ok]).max() / np.abs(want[ok]).max()
    assert err < 2e-6, err


@pytest.mark.parametrize("k", [0, 1, 2], ids=["composite", "axial_z", "sliced"])
def test_fit_matches_oracle(ctx, realistic, k):
    import paper_1602_07247_gb300 as ants
    sxy, g, comp, az, sl, (p2, v2, p3, v3, p3s) = realistic
    det = ants.Detector(sxy)
    if k == 0:
        want = comp
        got = ants.Lrf.fit_scheme(ctx, det, ants.ANTS_LRF_COMPOSITE, (8, 8), (-12.0, -12.0), (12.0, 12.0), p2, v2,
                                  n_int_r=12, hi_r=40.0)
        q = np.random.default_rng(7).uniform(-11.0, 11.0, (500, 2))
    elif k == 1:
        want = az
        got = ants.Lrf.fit_scheme(ctx, det, ants.ANTS_LRF_AXIAL_Z, (12, 6), (0.0, 0.0), (40.0, 20.0), p3, v3)
        q = np.concatenate([np.random.default_rng(7).uniform(-11.0, 11.0, (500, 2)),
                            np.random.default_rng(8).uniform(0.0, 20.0, (500, 1))], 1)
    else:
        want = sl
        got = ants.Lrf.fit_scheme(ctx, det, ants.ANTS_LRF_SLICED, (8, 8), (-12.0, -12.0, 0.0), (12.0, 12.0, 20.0),
                                  p3s, synth.truth_eta(sxy, g, p3s), n_planes=5)
        q = np.concatenate([np.random.default_rng(7).uniform(-11.0, 11.0, (500, 2)),
                            np.random.default_rng(8).uniform(0.0, 20.0, (500, 1))], 1)
    c = got.coefficients()
    assert c.shape == want.coef.shape
    err = np.abs(c - want.coef).max() / np.abs(want.coef).max()
    assert err < 1e-8, err
    # the same set evaluated through the oracle from the GPU's coefficients
    G = oracle.Lrf(want.type, sxy, want.n_int, want.lo, want.hi, c, n_int_r=want.n_int_r, hi_r=want.hi_r,
                   n_planes=want.n_planes)
    assert np.abs(oracle.lrf_eval(G, q) - oracle.lrf_eval(want, q)).max() < 1e-9


@pytest.mark.parametrize("k", [0, 1, 2], ids=["composite", "axial_z", "sliced"])
def test_reconstruction_matches_oracle(ctx, realistic, k):
    """Events simulated by the oracle from each scheme, reconstructed on the
    GPU (plain method; 2D for composite, 3D for the others) and replayed by
    the oracle along the GPU's path."""
    import torch
    import paper_1602_07247_gb300 as ants
    sxy, g, comp, az, sl, _ = realistic
    L = (comp, az, sl)[k]
    lrf = _gpu(ctx, L)
    three = k > 0
    sig, tr = oracle.simulate(L, 40 + k, 0, 1500, region="square", extent=8.0, z_lo=0.0, z_hi=20.0 if three else 0.0,
                              e0=4000.0, e_spread=0.05)
    if three:
        P = oracle.CgsParams(n_xy=7, iters=6, step_xy=2.0, n_z=5, step_z=4.0, z0=10.0)
        p = ants.CgsParams(n_xy=7, iters=6, step_xy=2.0, n_z=5, step_z=4.0, z0=10.0)
    else:
        P = oracle.CgsParams(n_xy=9, iters=7, step_xy=2.0)
        p = ants.CgsParams(n_xy=9, iters=7, step_xy=2.0)
    res = ants.reconstruct(ctx, lrf, p, torch.from_numpy(sig.astype(np.float32)).cuda(), want_trace=True)
    torch.cuda.synchronize()
    rp = oracle.cgs_replay(L, P, sig.astype(np.float32).astype(np.float64), res.trace.cpu().numpy().astype(np.int32))
    st = res.status.cpu().numpy()
    assert np.array_equal(st, rp["status"])
    ok = st == 0
    assert ok.mean() > 0.98
    assert np.all(rp["n_bad"][ok] == 0), np.nonzero(rp["n_bad"])[0][:5]
    assert np.abs(res.xyz.cpu().numpy()[ok] - rp["xyz"][ok]).max() <= 1e-3
    assert np.abs(res.logL.cpu().numpy()[ok] / rp["logL"][ok] - 1).max() <= 1e-5
    err = np.sqrt(((res.xyz.cpu().numpy()[ok] - tr[ok, :3]) ** 2).sum(1).mean())
    print(["composite", "axial_z", "sliced"][k], "RMS |dxyz| vs truth", err, "ties", (rp["n_tie"][ok] > 0).mean())


def test_simulator_3d_schemes(ctx, realistic):
    import paper_1602_07247_gb300 as ants
    sxy, g, comp, az, sl, _ = realistic
    for L in (az, sl):
        lrf = _gpu(ctx, L)
        p = ants.SimParams("square", 8.0, 0.0, 0.0, 0.0, 20.0, 3000.0, 0.05, 0.0)
        s, t = ants.simulate(ctx, lrf, p, 3000, seed=11)
        os_, ot = oracle.simulate(L, 11, 0, 3000, region="square", extent=8.0, z_lo=0.0, z_hi=20.0, e0=3000.0,
                                  e_spread=0.05)
        assert np.abs(t.cpu().numpy()[:, :3] - ot[:, :3]).max() < 1e-4
        assert (np.abs(s.cpu().numpy() - os_) == 0).mean() > 0.999


def test_scheme_limits(ctx):
    import torch
    import paper_1602_07247_gb300 as ants
    sxy, comp, az, sl = pins._scheme_lrfs()
    lrf = _gpu(ctx, comp)
    with pytest.raises(ants.AntsError):
        lrf.save("/tmp/ants_scheme.lrf")
    with pytest.raises(ants.AntsError):
        ants.LogTable(ctx, lrf, 8, 8)
    sig = torch.ones((4, 4), device="cuda")
    with pytest.raises(ants.AntsError):
        lrf.refit(sig, torch.zeros((4, 3), device="cuda"), torch.ones(4, device="cuda"))
    det = ants.Detector(sxy)
    with pytest.raises(ants.AntsError):  # n_z > 1 needs a z coordinate
        ants.reconstruct(ctx, lrf, ants.CgsParams(n_xy=5, iters=2, step_xy=1.0, n_z=3, step_z=1.0), sig)
    with pytest.raises(ants.AntsError):
        ants.Lrf.from_scheme(ctx, det, ants.ANTS_LRF_SLICED, (4, 4), (-12.0, -12.0, 0.0), (12.0, 12.0, 20.0),
                             sl.coef, n_planes=1)
