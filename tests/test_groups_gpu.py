"""Grouped radial LRFs (Sec. 6.2) on the GPU against the FP64 oracle: the
19-PMT hexagon with its four rings, each ring one profile and every PMT its
own gain; evaluation, the contracting-grid search (replayed by the oracle
under the tie rule) and the event simulator."""
import numpy as np
import pytest

import oracle
import synth
import synth.workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    assert torch.cuda.is_available()
    import paper_1602_07247_gb300 as ants
    ctx = ants.Context(0)
    w = synth.workloads.get("hex19_radial")
    det = ants.Detector(w.sensor_xy, w.gains)
    g, k = det.rings(1.0)
    pts, vals = w.fit_samples()
    coef, _, _ = oracle.lrf_fit(w.n_int, w.lo, w.hi, pts, vals)
    rng = np.random.default_rng(6)
    rows = coef[0][None, :] * rng.uniform(0.9, 1.1, (k, 1))  # ring profiles differ in scale
    gains = rng.uniform(0.9, 1.1, 19)
    L = oracle.Lrf(oracle.RADIAL, w.sensor_xy, w.n_int + (0, 0), w.lo + (0, 0), w.hi + (0, 0), rows, gain=gains,
                   group=g)
    lrf = ants.Lrf.from_groups(ctx, det, w.n_int, w.lo, w.hi, g, rows, gains)
    return ctx, w, det, g, k, L, lrf


def test_grouped_eval(setup):
    import torch
    ctx, w, det, g, k, L, lrf = setup
    assert k == 4
    pts = np.random.default_rng(1).uniform(-80, 80, (3000, 2)).astype(np.float32)
    got = lrf.eval(torch.from_numpy(pts).cuda()).cpu().numpy()
    want = oracle.lrf_eval(L, pts.astype(np.float64))
    ok = np.isfinite(want)
    assert np.array_equal(ok, np.isfinite(got))
    assert np.abs(got[ok] - want[ok]).max() <= 2e-6 * np.abs(want[ok]).max()


def test_grouped_search_matches_oracle(setup):
    import torch
    import paper_1602_07247_gb300 as ants
    ctx, w, det, g, k, L, lrf = setup
    sig, tr = oracle.simulate(L, 17, 0, 3000, region="disk", extent=60.0, e0=1e4, e_spread=0.05)
    sig = sig.astype(np.float32)
    p = ants.CgsParams(n_xy=w.n_xy, iters=w.iters, step_xy=w.step_xy, shrink=w.shrink)
    res = ants.reconstruct(ctx, lrf, p, torch.from_numpy(sig).cuda(), want_trace=True)
    torch.cuda.synchronize()
    P = oracle.CgsParams(n_xy=w.n_xy, iters=w.iters, step_xy=w.step_xy, shrink=w.shrink)
    rp = oracle.cgs_replay(L, P, sig.astype(np.float64), res.trace.cpu().numpy().astype(np.int32), gain_cog=w.gains)
    st = res.status.cpu().numpy()
    assert np.array_equal(st, rp["status"])
    ok = st == 0
    assert np.all(rp["n_bad"][ok] == 0)
    assert np.abs(res.xyz.cpu().numpy()[ok] - rp["xyz"][ok]).max() <= 1e-3
    assert np.abs(res.logL.cpu().numpy()[ok] / rp["logL"][ok] - 1).max() <= 1e-5
    # the continuous minimisation reads the same grouped profiles
    rm = ants.reconstruct(ctx, lrf, ants.MinimizeParams(max_iter=40, tol=1e-4), torch.from_numpy(sig[:500]).cuda(),
                          want_trace=True, method=ants.ANTS_MINIMIZE)
    om = oracle.minimize(L, sig[:500].astype(np.float64), oracle.Variant(), oracle.Minimize(max_iter=40, tol=1e-4),
                         gain=w.gains)
    conv = (rm.trace.cpu().numpy()[:, 0] > 0) & (om["n_iter"] > 0)
    assert conv.mean() > 0.95
    assert np.abs(rm.xyz.cpu().numpy()[conv] - om["xyz"][conv]).max() <= 1e-3


def test_grouped_simulation_and_limits(setup):
    import paper_1602_07247_gb300 as ants
    ctx, w, det, g, k, L, lrf = setup
    sp = ants.SimParams("disk", 60.0, 0.0, 0.0, 0.0, 0.0, 1e4, 0.05, 0.0)
    s, t = ants.simulate(ctx, lrf, sp, 4000, seed=21)
    os_, ot = oracle.simulate(L, 21, 0, 4000, region="disk", extent=60.0, e0=1e4, e_spread=0.05)
    assert np.abs(t.cpu().numpy()[:, :2] - ot[:, :2]).max() < 1e-4
    assert (s.cpu().numpy() == os_).mean() > 0.999
    with pytest.raises(ants.AntsError):
        lrf.save("/tmp/ants_grouped.lrf")
    with pytest.raises(ants.AntsError):
        ants.Lrf.from_groups(ctx, det, w.n_int, w.lo, w.hi, np.full(19, 4), np.ones((4, 23)))


def test_grouped_refit_and_iteration(setup):
    """The refit of the rings from reconstructed events equals the oracle's
    FP64 refit of the same samples (profiles per ring, gains within rings);
    three cycles of the iteration from the true rings keep the events and
    stay at the truth's position error."""
    import torch
    import paper_1602_07247_gb300 as ants
    ctx, w, det, g, k, L, lrf = setup
    sig, tr = oracle.simulate(L, 33, 0, 3000, region="disk", extent=60.0, e0=1e4, e_spread=0.05)
    sd = torch.from_numpy(sig.astype(np.float32)).cuda()
    p = ants.CgsParams(n_xy=w.n_xy, iters=w.iters, step_xy=w.step_xy, shrink=w.shrink)
    res = ants.reconstruct(ctx, lrf, p, sd)
    keep = np.nonzero(res.status.cpu().numpy() == 0)[0].astype(np.int32)
    R = lrf.refit(sd, res.xyz, res.E, index=torch.from_numpy(keep).cuda(), refit_gains=True)
    want = oracle.lrf_refit(L, sig[keep], res.xyz.cpu().numpy()[keep].astype(np.float64),
                            res.E.cpu().numpy()[keep].astype(np.float64), refit_gains=True)
    c = R.coefficients()
    assert c.shape == want.coef.shape == (k, w.n_int[0] + 3)
    assert np.abs(c - want.coef).max() <= 1e-9 * np.abs(want.coef).max()
    assert np.abs(R.gains() - want.gain).max() <= 1e-9
    # the iteration on 10^5 simulated flood events (the ring of one sensor
    # needs the statistics)
    n = 100_000
    sp = ants.SimParams("disk", 60.0, 0.0, 0.0, 0.0, 0.0, 1e4, 0.05, 0.1)
    s2 = torch.empty((n, 19), device="cuda")
    truth = torch.empty((n, 4), device="cuda")
    ants.ants_simulate_events(ctx.handle, lrf.handle, sp, 77, 0, s2, truth)
    it, stats = lrf.iterate(s2, p, 3, ants.EventCuts(chi2_max=25.0), refit_gains=True)
    assert stats[-1]["n_kept"] > 0.95 * n
    err = lambda L: float(((ants.reconstruct(ctx, L, p, s2).xyz[:, :2] - truth[:, :2]) ** 2).sum(1).mean().sqrt())
    e_true, e_it = err(lrf), err(it)
    assert e_it < 1.03 * e_true, (e_it, e_true)
