"""GPU FP64 LRF fit against the oracle's FP64 fit (same samples)."""
import numpy as np
import pytest

import oracle
import synth
import synth.workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    import paper_1602_07247_gb300 as ants
    return ants.Context(0)


TYPES = {"radial": 1, "xy": 2, "xyz": 3}


@pytest.mark.parametrize("name", ["hex19_radial", "sipm8x8_xy", "sipm16x16_xy"])
def test_fit_matches_oracle(ctx, name):
    import paper_1602_07247_gb300 as ants
    w = synth.workloads.get(name)
    pts, vals = w.fit_samples()
    want, rc, _ = oracle.lrf_fit(w.n_int, w.lo, w.hi, pts, vals)
    det = ants.Detector(w.sensor_xy, w.gains)
    lrf = ants.Lrf.fit(ctx, det, TYPES[w.lrf_type], w.n_int, w.lo, w.hi, pts, vals, shared=w.shared)
    got = lrf.coefficients()
    assert got.shape == want.shape
    err = np.abs(got - want).max() / np.abs(want).max()
    print(name, "max rel coefficient difference", err)
    assert err < 1e-9
    assert lrf.ridge_used == 0.0
    # bitwise reproducible
    lrf2 = ants.Lrf.fit(ctx, det, TYPES[w.lrf_type], w.n_int, w.lo, w.hi, pts, vals, shared=w.shared)
    assert np.array_equal(lrf2.coefficients(), got)


def test_fit_tensor_3d_and_random_points(ctx):
    """Scattered samples of a smooth 3D function, on a small tricubic grid.
    Uneven sampling makes the normal matrix less well conditioned than on a
    regular grid, so the two FP64 solves (different summation orders) agree
    to ~1e-8 instead of ~1e-12."""
    import paper_1602_07247_gb300 as ants
    rng = np.random.default_rng(12)
    sxy = synth.square_array(2, 10.0)
    n_int, lo, hi = (5, 4, 3), (-12.0, -10.0, 0.0), (12.0, 10.0, 20.0)
    pts = np.stack([rng.uniform(lo[a], hi[a], 6000) for a in range(3)], axis=1)
    vals = np.stack([synth.eta_3d(np.hypot(pts[:, 0] - x, pts[:, 1] - y), pts[:, 2]) for x, y in sxy], axis=1)
    want, rc, _ = oracle.lrf_fit(n_int, lo, hi, pts, vals)
    det = ants.Detector(sxy)
    lrf = ants.Lrf.fit(ctx, det, 3, n_int, lo, hi, pts, vals)
    err = np.abs(lrf.coefficients() - want).max() / np.abs(want).max()
    assert err < 1e-7, err


def test_fit_ridge_fallback(ctx):
    """Samples only on half of the domain: the normal matrix is singular, so
    both fits retry with the same ridge; their fitted values agree."""
    import paper_1602_07247_gb300 as ants
    n_int, lo, hi = (10,), (0.0,), (100.0,)
    r = np.linspace(0.0, 45.0, 200)
    v = synth.eta_axial(r)
    want, rc, lam_o = oracle.lrf_fit(n_int, lo, hi, r[:, None], v)
    assert rc == 1
    det = ants.Detector(np.zeros((1, 2)))
    lrf = ants.Lrf.fit(ctx, det, 1, n_int, lo, hi, r[:, None], v, shared=True)
    assert lrf.ridge_used > 0.0 and abs(lrf.ridge_used / lam_o - 1.0) < 1e-12
    x = np.linspace(0.0, 45.0, 50)[:, None]
    a = oracle.spline_eval(n_int, lo, hi, want[0], x)
    b = oracle.spline_eval(n_int, lo, hi, lrf.coefficients()[0], x)
    assert np.abs(a - b).max() < 1e-6 * np.abs(a).max()
