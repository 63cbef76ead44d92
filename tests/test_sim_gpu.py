"""GPU event simulator against its FP64 oracle twin: the same Philox4x32-10
streams give the same sources and (up to rare FP32 rounding at a decision
boundary) the same Poisson counts; counts follow scipy's Poisson pmf."""
import numpy as np
import pytest

import oracle
import synth
import synth.workloads
from parity import gpu_objects, oracle_lrf

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch
    assert torch.cuda.is_available()
    import paper_1602_07247_gb300 as ants
    return torch, ants, ants.Context(0)


@pytest.mark.parametrize("name,region,extent,spe", [("sipm8x8_xy", "square", 21.0, 0.0),
                                                     ("hex19_radial", "disk", 60.0, 0.1),
                                                     ("sipm4x4_xyz", "square", 9.0, 0.0)])
def test_simulator_matches_oracle(env, name, region, extent, spe):
    torch, ants, ctx = env
    w = synth.workloads.get(name)
    L = oracle_lrf(w)
    _, det, lrf, _ = gpu_objects(w, L, ctx)
    zr = (0.0, 20.0) if w.lrf_type == "xyz" else (0.0, 0.0)
    e0 = 3000.0
    p = ants.SimParams(region, extent, 0.0, 0.0, zr[0], zr[1], e0, 0.05, spe)
    n, first = 4001, 123456
    sig, truth = ants.simulate(ctx, lrf, p, n, seed=99, first_event=first)
    osig, otruth = oracle.simulate(L, 99, first, n, region=region, extent=extent, z_lo=zr[0], z_hi=zr[1], e0=e0,
                                   e_spread=0.05, spe_sigma=spe)
    t = truth.cpu().numpy()
    assert np.abs(t[:, :3] - otruth[:, :3]).max() < 1e-4
    assert np.abs(t[:, 3] / otruth[:, 3] - 1.0).max() < 1e-6
    s = sig.cpu().numpy()
    same = np.abs(s - osig) <= (1e-3 * np.maximum(1.0, osig) if spe > 0 else 0.0)
    print(name, "identical fraction", same.mean())
    assert same.mean() > 0.999
    # counter-based: a split range reproduces the same events
    a, _ = ants.simulate(ctx, lrf, p, 1000, seed=99, first_event=first)
    b, _ = ants.simulate(ctx, lrf, p, 3001, seed=99, first_event=first + 1000)
    assert torch.equal(torch.cat([a, b]), sig)


@pytest.mark.parametrize("lam", [0.5, 5.0, 50.0, 500.0])
def test_poisson_distribution(env, lam):
    """A one-sensor detector with a constant LRF value c gives rate E c."""
    from scipy.stats import chi2, poisson
    torch, ants, ctx = env
    det = ants.Detector(np.zeros((1, 2)))
    c = 0.5
    lrf = ants.Lrf.from_coefficients(ctx, det, ants.ANTS_LRF_XY, (2, 2), (-10.0, -10.0), (10.0, 10.0),
                                     np.full((1, 25), c))
    p = ants.SimParams("square", 5.0, 0.0, 0.0, 0.0, 0.0, lam / c, 0.0, 0.0)
    sig, _ = ants.simulate(ctx, lrf, p, 200000, seed=5)
    x = sig.cpu().numpy()[:, 0].astype(np.float64)
    assert abs(x.mean() - lam) < 5 * np.sqrt(lam / x.size)
    assert abs(x.var() / lam - 1.0) < 0.02
    lo, hi = int(poisson.ppf(1e-5, lam)), int(poisson.ppf(1 - 1e-5, lam))
    edges = np.arange(lo, hi + 2)
    obs, _ = np.histogram(x, bins=edges)
    exp = x.size * poisson.pmf(edges[:-1], lam)
    keep = exp > 5
    stat = ((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    assert stat < chi2.ppf(0.999, keep.sum() - 1), stat
