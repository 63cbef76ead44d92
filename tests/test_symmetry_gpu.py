"""XY LRF classes by the array's symmetry (Sec. 6.2) on the GPU against
the FP64 oracle: the 8 x 8 SiPM array's ten classes, each one XY LRF in its
representative's frame, every sensor with its gain."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    assert torch.cuda.is_available()
    import paper_1602_07247_gb300 as ants
    ctx = ants.Context(0)
    sq = synth.square_array(8, 6.0)
    det = ants.Detector(sq)
    cl, op, k, c = det.symmetry(1e-6)
    # class LRFs: the representative's bump sampled on the knot grid, with
    # a non-symmetric modulation so that the operations matter
    n = 12
    kx = np.linspace(-24.0 - 2 * 48.0 / n, 24.0 + 2 * 48.0 / n, n + 3)  # approximately the knot centres
    X, Y = np.meshgrid(kx, kx)
    reps = [int(np.nonzero(cl == j)[0][0]) for j in range(k)]
    coef = np.stack([0.03 / (1 + ((X - sq[r, 0]) ** 2 + (Y - sq[r, 1]) ** 2) / 64.0) ** 1.5 *
                     (1.0 + 0.1 * np.sin(X / 7.0 + 0.3 * Y / 5.0)) for r in reps]).reshape(k, -1)
    gains = np.random.default_rng(9).uniform(0.9, 1.1, 64)
    L = oracle.Lrf(oracle.XY, sq, (n, n, 0), (-24.0, -24.0, 0.0), (24.0, 24.0, 0.0), coef, gain=gains, group=cl,
                   op=op, sym_c=c)
    lrf = ants.Lrf.from_symmetry(ctx, det, (n, n), (-24.0, -24.0), (24.0, 24.0), cl, op, c, coef, gains)
    return ctx, det, L, lrf, k


def test_symmetric_eval(setup):
    import torch
    ctx, det, L, lrf, k = setup
    assert k == 10
    pts = np.random.default_rng(2).uniform(-23.5, 23.5, (2000, 2)).astype(np.float32)
    got = lrf.eval(torch.from_numpy(pts).cuda()).cpu().numpy()
    want = oracle.lrf_eval(L, pts.astype(np.float64))
    ok = np.isfinite(want)
    assert np.array_equal(ok, np.isfinite(got))
    assert np.abs(got[ok] - want[ok]).max() <= 2e-6 * np.abs(want[ok]).max()


def test_symmetric_search_minimise_simulate(setup):
    import torch
    import paper_1602_07247_gb300 as ants
    ctx, det, L, lrf, k = setup
    sig, tr = oracle.simulate(L, 5, 0, 1500, region="square", extent=18.0, e0=3000.0, e_spread=0.05)
    sig = sig.astype(np.float32)
    p = ants.CgsParams(n_xy=11, iters=8, step_xy=4.8, shrink=0.5)
    res = ants.reconstruct(ctx, lrf, p, torch.from_numpy(sig).cuda(), want_trace=True)
    torch.cuda.synchronize()
    P = oracle.CgsParams(n_xy=11, iters=8, step_xy=4.8, shrink=0.5)
    rp = oracle.cgs_replay(L, P, sig.astype(np.float64), res.trace.cpu().numpy().astype(np.int32))
    st = res.status.cpu().numpy()
    assert np.array_equal(st, rp["status"])
    ok = st == 0
    assert ok.mean() > 0.95
    assert np.all(rp["n_bad"][ok] == 0)
    assert np.abs(res.xyz.cpu().numpy()[ok] - rp["xyz"][ok]).max() <= 1e-3
    assert np.abs(res.logL.cpu().numpy()[ok] / rp["logL"][ok] - 1).max() <= 1e-5
    rm = ants.reconstruct(ctx, lrf, ants.MinimizeParams(max_iter=40, tol=1e-4), torch.from_numpy(sig[:500]).cuda(),
                          want_trace=True, method=ants.ANTS_MINIMIZE)
    om = oracle.minimize(L, sig[:500].astype(np.float64), oracle.Variant(), oracle.Minimize(max_iter=40, tol=1e-4))
    conv = (rm.trace.cpu().numpy()[:, 0] > 0) & (om["n_iter"] > 0)
    assert conv.mean() > 0.95
    assert np.abs(rm.xyz.cpu().numpy()[conv] - om["xyz"][conv]).max() <= 1e-3
    sp = ants.SimParams("square", 18.0, 0.0, 0.0, 0.0, 0.0, 3000.0, 0.05, 0.0)
    s, t = ants.simulate(ctx, lrf, sp, 3000, seed=8)
    os_, ot = oracle.simulate(L, 8, 0, 3000, region="square", extent=18.0, e0=3000.0, e_spread=0.05)
    assert np.abs(t.cpu().numpy()[:, :2] - ot[:, :2]).max() < 1e-4
    assert (s.cpu().numpy() == os_).mean() > 0.999
    with pytest.raises(ants.AntsError):
        lrf.save("/tmp/ants_sym.lrf")


def test_symmetric_fit_matches_oracle(setup):
    """The class fit from samples (device FP64 fit of the mapped samples)
    against the oracle's."""
    import paper_1602_07247_gb300 as ants
    ctx, det, L, lrf, k = setup
    rng = np.random.default_rng(41)
    pts = rng.uniform(-24.0, 24.0, (4000, 2))
    vals = oracle.lrf_eval(L, pts) * rng.uniform(0.98, 1.02, (4000, 64))
    cl, op, _, c = det.symmetry(1e-6)
    got = ants.Lrf.fit_symmetric(ctx, det, (12, 12), (-24.0, -24.0), (24.0, 24.0), cl, op, c, pts, vals, L.gain)
    want = oracle.lrf_fit_symmetric(L.sensor_xy, cl, op, c, (12, 12), (-24.0, -24.0), (24.0, 24.0), pts, vals,
                                    gain=L.gain)
    cg = got.coefficients()
    assert cg.shape == want.coef.shape
    assert np.abs(cg - want.coef).max() <= 1e-9 * np.abs(want.coef).max()


def test_symmetric_refit_matches_oracle(setup):
    """The refit of the classes from reconstructed events (positions shifted
    by the seeded offsets) equals the oracle's class fit of the same samples."""
    import torch
    import paper_1602_07247_gb300 as ants
    ctx, det, L, lrf, k = setup
    sig, tr = oracle.simulate(L, 6, 0, 3000, region="square", extent=18.0, e0=3000.0, e_spread=0.05)
    sd = torch.from_numpy(sig.astype(np.float32)).cuda()
    p = ants.CgsParams(n_xy=11, iters=8, step_xy=4.8, shrink=0.5)
    res = ants.reconstruct(ctx, lrf, p, sd)
    keep = np.nonzero(res.status.cpu().numpy() == 0)[0].astype(np.int32)
    R = lrf.refit(sd, res.xyz, res.E, index=torch.from_numpy(keep).cuda(), shift_sigma=0.5, seed=4, cycle=2)
    xyz = res.xyz.cpu().numpy()[keep].astype(np.float64)
    xyz[:, :2] += oracle.shift_xy(4, 2, keep, 0.5)
    want = oracle.lrf_refit(L, sig[keep], xyz, res.E.cpu().numpy()[keep].astype(np.float64))
    c = R.coefficients()
    assert c.shape == want.coef.shape
    assert np.abs(c - want.coef).max() <= 1e-8 * np.abs(want.coef).max()
