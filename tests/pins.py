"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each pin takes ``mutant`` (0 = the real oracle; k > 0 = a build with one
planted mistake) and raises AssertionError when the oracle disagrees with
the fact.  tests/test_oracle_pins.py runs them on the real oracle;
tests/test_oracle_mutants.py checks that every planted mistake trips at
least one of them.  The facts are closed forms, textbook values, library
routines (scipy) and exhaustive search on tiny inputs.
"""
from __future__ import annotations

import math
import os
from fractions import Fraction

import numpy as np

import oracle
import synth
import synth.workloads

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _golden_bspline():
    rows = []
    with open(os.path.join(GOLDEN, "uniform_cubic_bspline.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if not line:
                continue
            parts = line.split()
            t = Fraction(int(parts[0]), int(parts[1]))
            b = [Fraction(p) for p in parts[2:6]]
            rows.append((t, b))
    return rows


# --------------------------------------------------------------------------
# B-spline basis
# --------------------------------------------------------------------------


def pin_bspline_golden(mutant=0):
    """Basis values on a span equal the closed-form uniform cubic segment
    polynomials (golden fractions), for the full and the local recursion."""
    n, lo, hi = 5, -1.0, 9.0  # h = 2
    for t, b in _golden_bspline():
        for span in (0, 2, 4):
            x = lo + 2.0 * (span + float(t))
            m, B = oracle.bspline_basis_all(n, lo, hi, x, mutant)
            j0, B4 = oracle.bspline_basis4(n, lo, hi, x, mutant)
            assert j0 == span, (j0, span)
            want = np.array([float(v) for v in b])
            assert np.allclose(B[span:span + 4], want, rtol=0, atol=1e-15), (B[span:span + 4], want)
            assert np.allclose(B4, want, rtol=0, atol=1e-15), (B4, want)
            assert np.all(np.delete(B, range(span, span + 4)) == 0.0)


def pin_partition_of_unity(mutant=0):
    """sum_j B_j(x) = 1 on [lo, hi], including both ends and the knots."""
    rng = np.random.default_rng(5)
    for n, lo, hi in ((1, 0.0, 1.0), (4, -3.0, 5.0), (20, 0.0, 150.0), (32, -25.6, 25.6)):
        xs = np.concatenate([rng.uniform(lo, hi, 50), np.linspace(lo, hi, n + 1)])
        for x in xs:
            m, B = oracle.bspline_basis_all(n, lo, hi, float(x), mutant)
            j0, B4 = oracle.bspline_basis4(n, lo, hi, float(x), mutant)
            assert abs(B.sum() - 1.0) < 1e-14, (n, x, B.sum())
            assert abs(B4.sum() - 1.0) < 1e-14, (n, x, B4.sum())
            assert np.all(B >= -1e-16) and np.all(B4 >= -1e-16)
        m, B = oracle.bspline_basis_all(n, lo, hi, hi + 1e-9, mutant)
        assert m == -1 and not B.any()


# --------------------------------------------------------------------------
# least-squares fit
# --------------------------------------------------------------------------


def _poly_nd(pts, coefs):
    v = np.zeros(pts.shape[0])
    for powers, c in coefs.items():
        term = np.full(pts.shape[0], c)
        for a, pw in enumerate(powers):
            term = term * pts[:, a] ** pw
        v += term
    return v


def pin_fit_reproduces_cubics(mutant=0):
    """Cubic splines reproduce (tensor) cubic polynomials exactly, so the
    least-squares fit of polynomial samples recovers them to rounding."""
    rng = np.random.default_rng(7)
    cases = [
        ((7,), (0.0,), (10.0,)),
        ((5, 6), (-3.0, -2.0), (4.0, 5.0)),
        ((3, 4, 2), (-1.0, 0.0, 0.0), (2.0, 3.0, 2.0)),
    ]
    for n_int, lo, hi in cases:
        d = len(n_int)
        coefs = {}
        for powers in np.ndindex(*([4] * d)):
            coefs[powers] = rng.uniform(-1.0, 1.0) / (1.0 + sum(powers)) ** 2
        pts = synth.grid_samples(n_int, lo, hi, per_interval=3)
        vals = _poly_nd(pts, coefs)
        coef, rc, lam = oracle.lrf_fit(n_int, lo, hi, pts, vals, mutant=mutant)
        assert rc == 0
        test = np.stack([rng.uniform(lo[a], hi[a], 300) for a in range(d)], axis=1)
        got = oracle.spline_eval(n_int, lo, hi, coef[0], test, mutant=mutant)
        want = _poly_nd(test, coefs)
        scale = np.abs(want).max()
        assert np.abs(got - want).max() < 1e-10 * max(scale, 1.0), (n_int, np.abs(got - want).max())


def pin_fit_h4_convergence(mutant=0):
    """The cubic-spline fit error of the smooth axial LRF falls as h^4:
    halving h cuts the maximum error by about 16."""
    r = np.linspace(0.0, 150.0, 3001)
    errs = []
    for n in (10, 20, 40):
        pts = synth.grid_samples((n,), (0.0,), (150.0,), per_interval=4)
        coef, rc, _ = oracle.lrf_fit((n,), (0.0,), (150.0,), pts, synth.eta_axial(pts[:, 0]), mutant=mutant)
        got = oracle.spline_eval((n,), (0.0,), (150.0,), coef[0], r[:, None], mutant=mutant)
        errs.append(np.abs(got - synth.eta_axial(r)).max())
    for a, b in zip(errs, errs[1:]):
        assert 10.0 < a / b < 24.0, errs


def pin_lrf_matches_closed_form(mutant=0):
    """Fitted LRFs evaluated through the sensor geometry reproduce the
    closed-form truth: axial (20 intervals on [0,150]) and per-sensor XY
    (24 x 24 on +-24 mm, off-centre sensors) within 1e-4 relative."""
    w = synth.workloads.get("hex19_radial")
    pts, vals = w.fit_samples()
    coef, _, _ = oracle.lrf_fit(w.n_int, w.lo, w.hi, pts, vals, mutant=mutant)
    L = oracle.Lrf(oracle.RADIAL, w.sensor_xy, w.n_int + (0, 0), w.lo + (0, 0), w.hi + (0, 0), coef,
                   shared=True)
    rng = np.random.default_rng(11)
    p = rng.uniform(-60, 60, (400, 2))
    got = oracle.lrf_eval(L, p, mutant=mutant)
    want = synth.truth_eta(w.sensor_xy, w.gains, p)
    assert np.nanmax(np.abs(got / want - 1.0)) < 1e-4
    w = synth.workloads.get("sipm8x8_xy")
    sel = [0, 9, 27, 62]  # corner, inner and edge sensors: no symmetry to hide a transposition
    sxy = w.sensor_xy[sel]
    g = w.gains[sel]
    pts = synth.grid_samples(w.n_int, w.lo, w.hi, 4)
    vals = synth.truth_eta(sxy, g, pts)
    coef, _, _ = oracle.lrf_fit(w.n_int, w.lo, w.hi, pts, vals, mutant=mutant)
    L = oracle.Lrf(oracle.XY, sxy, w.n_int + (0,), w.lo + (0,), w.hi + (0,), coef)
    p = rng.uniform(-24, 24, (400, 2))
    got = oracle.lrf_eval(L, p, mutant=mutant)
    want = synth.truth_eta(sxy, g, p)
    assert np.abs(got / want - 1.0).max() < 1e-4, np.abs(got / want - 1.0).max()


# --------------------------------------------------------------------------
# centroid
# --------------------------------------------------------------------------


def pin_cog(mutant=0):
    """COG of symmetric patterns is the array centre; one lit sensor gives
    its own position; mirrored signals give the mirrored COG; with two lit
    sensors and gains g_i, s_i = g_i w_i gives (X1 w1 + X2 w2)/(w1 + w2)."""
    sxy = synth.hex_array(2, 30.0)
    n = sxy.shape[0]
    c = oracle.cog(np.ones((1, n)), sxy, mutant=mutant)
    assert np.abs(c).max() < 1e-12
    r = np.hypot(sxy[:, 0], sxy[:, 1])
    c = oracle.cog(np.exp(-r / 30.0)[None, :], sxy, mutant=mutant)
    assert np.abs(c).max() < 1e-12
    for i in (0, 7, 18):
        s = np.zeros((1, n))
        s[0, i] = 123.0
        assert np.allclose(oracle.cog(s, sxy, mutant=mutant)[0], sxy[i], atol=1e-12)
    rng = np.random.default_rng(3)
    s = rng.uniform(1, 100, n)
    # mirror x -> -x maps sensor i to sensor j with X_j = -X_i, Y_j = Y_i
    perm = [int(np.argmin(np.hypot(sxy[:, 0] + sxy[i, 0], sxy[:, 1] - sxy[i, 1]))) for i in range(n)]
    s_m = np.empty(n)
    s_m[perm] = s
    c1 = oracle.cog(s[None], sxy, mutant=mutant)[0]
    c2 = oracle.cog(s_m[None], sxy, mutant=mutant)[0]
    assert abs(c1[0] + c2[0]) < 1e-12 and abs(c1[1] - c2[1]) < 1e-12
    gains = rng.uniform(0.5, 2.0, n)
    s = np.zeros((1, n))
    s[0, 3], s[0, 11] = gains[3] * 5.0, gains[11] * 15.0
    want = (sxy[3] * 5.0 + sxy[11] * 15.0) / 20.0
    assert np.allclose(oracle.cog(s, sxy, gains, mutant=mutant)[0], want, atol=1e-12)


# --------------------------------------------------------------------------
# likelihood and energy
# --------------------------------------------------------------------------


def _small_xy_lrf(mutant=0):
    sxy = synth.square_array(3, 8.0)
    g = np.linspace(0.9, 1.1, 9)
    n_int, lo, hi = (8, 8), (-16.0, -16.0), (16.0, 16.0)
    pts = synth.grid_samples(n_int, lo, hi, 4)
    coef, _, _ = oracle.lrf_fit(n_int, lo, hi, pts, synth.truth_eta(sxy, g, pts), mutant=mutant)
    return oracle.Lrf(oracle.XY, sxy, n_int + (0,), lo + (0,), hi + (0,), coef), g


def pin_energy_is_ml(mutant=0):
    """At fixed position the Poisson likelihood is maximised over E at
    E = sum s / sum eta (Sec. 5.1.2.2): the reported E beats E(1 +- 1e-3)."""
    L, _ = _small_xy_lrf(mutant)
    rng = np.random.default_rng(4)
    for _ in range(5):
        x = np.array([rng.uniform(-10, 10), rng.uniform(-10, 10), 0.0])
        s = rng.poisson(800 * synth.truth_eta(L.sensor_xy, np.ones(9), x[None, :2])[0]).astype(float)
        E, _ = oracle.energy_logl_at(L, s[None], x[None], mutant=mutant)
        l0 = oracle.logl_at_energy(L, s, x, E[0], mutant=mutant)
        for f in (1 - 1e-3, 1 + 1e-3):
            assert oracle.logl_at_energy(L, s, x, E[0] * f, mutant=mutant) < l0


def pin_logl_is_poisson(mutant=0):
    """The reported logL equals the sum of scipy's Poisson log-pmf at
    mu_i = E eta_i for integer signals."""
    from scipy.stats import poisson
    L, _ = _small_xy_lrf(mutant)
    rng = np.random.default_rng(8)
    for _ in range(5):
        x = np.array([rng.uniform(-10, 10), rng.uniform(-10, 10), 0.0])
        s = rng.poisson(500 * synth.truth_eta(L.sensor_xy, np.ones(9), x[None, :2])[0]).astype(float)
        s[2] = 0.0
        E, logL = oracle.energy_logl_at(L, s[None], x[None], mutant=mutant)
        eta = oracle.lrf_eval(L, x[None, :2], mutant=mutant)[0]
        want = poisson.logpmf(s, E[0] * eta).sum()
        assert abs(logL[0] - want) < 1e-9 * abs(want), (logL[0], want)


def pin_profile_identity(mutant=0):
    """max_E logL(x, E), found numerically by scipy, equals the searched
    objective F(x) = sum s ln eta - S ln H plus S ln S - S - sum lgamma(s+1)."""
    from scipy.optimize import minimize_scalar
    L, _ = _small_xy_lrf(mutant)
    rng = np.random.default_rng(9)
    for _ in range(4):
        x = np.array([rng.uniform(-10, 10), rng.uniform(-10, 10), 0.0])
        s = rng.poisson(700 * synth.truth_eta(L.sensor_xy, np.ones(9), x[None, :2])[0]).astype(float)
        S = s.sum()
        res = minimize_scalar(lambda E: -oracle.logl_at_energy(L, s, x, E, mutant=mutant),
                              bounds=(1.0, 1e5), method="bounded", options={"xatol": 1e-7})
        F = oracle.objective_at(L, s[None], x[None], mutant=mutant)[0]
        want = F + S * math.log(S) - S - sum(math.lgamma(v + 1.0) for v in s)
        assert abs(-res.fun - want) < 1e-6 * abs(want), (-res.fun, want)


# --------------------------------------------------------------------------
# contracting grids
# --------------------------------------------------------------------------


def pin_noise_free_recovery(mutant=0):
    """With s = E eta(x_true) (no noise) and x_true on a node of the first
    grid, the search lands exactly on x_true and E = E_true: by Gibbs'
    inequality sum s ln p, p = eta/H, is maximal only where p = s/S."""
    L, _ = _small_xy_lrf(mutant)
    P = oracle.CgsParams(n_xy=9, iters=6, step_xy=1.5)
    xt = np.array([[3.25, -2.5, 0.0], [-6.5, 4.75, 0.0], [0.5, 0.25, 0.0]])
    off = np.array([[2, -1, 0], [-3, 4, 0], [0, 1, 0]], dtype=float)
    start = xt - off * P.step_xy
    eta = oracle.lrf_eval(L, xt[:, :2], mutant=mutant)
    E_true = np.array([900.0, 1500.0, 4000.0])
    s = E_true[:, None] * eta
    r = oracle.cgs(L, P, s, start_xyz=start, mutant=mutant)
    assert np.all(r["status"] == 0)
    assert np.abs(r["xyz"] - xt).max() < 1e-12, r["xyz"]
    assert np.abs(r["E"] / E_true - 1.0).max() < 1e-12, r["E"]
    c = (P.n_xy - 1) // 2
    for e in range(3):
        k0 = (c + int(off[e, 1])) * P.n_xy + (c + int(off[e, 0]))
        assert r["trace"][e, 0] == k0
        assert np.all(r["trace"][e, 1:] == c * P.n_xy + c)
    # axial LRF on the PMT array, from the COG start of a central event
    w = synth.workloads.get("hex19_radial")
    pts, vals = w.fit_samples()
    coef, _, _ = oracle.lrf_fit(w.n_int, w.lo, w.hi, pts, vals, mutant=mutant)
    Lr = oracle.Lrf(oracle.RADIAL, w.sensor_xy, w.n_int + (0, 0), w.lo + (0, 0), w.hi + (0, 0), coef,
                    shared=True)
    Pr = oracle.CgsParams(n_xy=w.n_xy, iters=w.iters, step_xy=w.step_xy)
    xt = np.array([[7.5, -15.0, 0.0]])
    s = 1e4 * oracle.lrf_eval(Lr, xt[:, :2], mutant=mutant)
    r = oracle.cgs(Lr, Pr, s, start_xyz=xt - np.array([[1.0, 2.0, 0.0]]) * Pr.step_xy, mutant=mutant)
    assert np.abs(r["xyz"] - xt).max() < 1e-12 and abs(r["E"][0] / 1e4 - 1.0) < 1e-12


def pin_noise_free_recovery_3d(mutant=0):
    """The same Gibbs argument in 3D: an XYZ LRF, x_true on a node of the
    first x-y-z grid, noise-free signals -> exactly x_true and E_true."""
    import synth.workloads
    w = synth.workloads.get("sipm4x4_xyz")
    pts = synth.grid_samples(w.n_int, w.lo, w.hi, 2)
    vals = synth.truth_eta(w.sensor_xy, w.gains, pts)
    coef, _, _ = oracle.lrf_fit(w.n_int, w.lo, w.hi, pts, vals, mutant=mutant)
    L = oracle.Lrf(oracle.XYZ, w.sensor_xy, w.n_int, w.lo, w.hi, coef)
    P = oracle.CgsParams(n_xy=7, iters=4, step_xy=2.0, n_z=5, step_z=4.0)
    xt = np.array([[2.5, -3.0, 6.0], [-5.0, 1.5, 14.0]])
    off = np.array([[1, -2, -1], [-3, 0, 2]], dtype=float)
    start = xt - off * np.array([2.0, 2.0, 4.0])
    s = np.array([[1500.0], [2600.0]]) * oracle.lrf_eval(L, xt, mutant=mutant)
    r = oracle.cgs(L, P, s, start_xyz=start, mutant=mutant)
    assert np.abs(r["xyz"] - xt).max() < 1e-12, r["xyz"]
    assert np.abs(r["E"] / np.array([1500.0, 2600.0]) - 1.0).max() < 1e-12
    # flat index (iz, iy, ix) of the first choice
    k0 = [((2 + int(o[2])) * 7 + (3 + int(o[1]))) * 7 + (3 + int(o[0])) for o in off]
    assert list(r["trace"][:, 0]) == k0, (r["trace"][:, 0], k0)


def pin_cg_matches_brute_force(mutant=0):
    """On a tiny detector (2 x 2 sensors) the contracting-grid result is the
    global maximum found by exhaustive search on a fine grid."""
    sxy = synth.square_array(2, 10.0)
    g = np.array([1.0, 0.95, 1.05, 1.02])
    n_int, lo, hi = (10, 10), (-15.0, -15.0), (15.0, 15.0)
    pts = synth.grid_samples(n_int, lo, hi, 4)
    coef, _, _ = oracle.lrf_fit(n_int, lo, hi, pts, synth.truth_eta(sxy, g, pts, r0=20.0), mutant=mutant)
    L = oracle.Lrf(oracle.XY, sxy, n_int + (0,), lo + (0,), hi + (0,), coef)
    # sources inside the array, where four sensors pin the position; far
    # outside it the profiled likelihood has flat valleys and no unique max
    ev = synth.draw_events(sxy, g, 120, 77, region="square", extent=6.0, e0=4000.0, r0=20.0)
    P = oracle.CgsParams(n_xy=9, iters=8, step_xy=3.75)
    r = oracle.cgs(L, P, ev.signals, gain_cog=g, mutant=mutant)
    fine = 0.05
    xy, F = oracle.brute_force(L, ev.signals, (-15, 15), int(30 / fine) + 1, (-15, 15), int(30 / fine) + 1,
                               mutant=mutant)
    d = np.hypot(*(r["xyz"][:, :2] - xy).T)
    final = P.step_xy * P.shrink ** (P.iters - 1)
    ok = d <= 2.0 * (fine + final)
    assert ok.mean() >= 0.99, (ok.mean(), d.max())


def pin_ties_go_to_lowest_index(mutant=0):
    """With a single sensor, F = s ln eta - s ln eta = 0 exactly at every
    node, so all nodes tie; the search must take the lowest flat index (the
    (-,-) corner) on every grid."""
    sxy = np.array([[3.0, 1.0]])
    n_int, lo, hi = (4, 4), (-40.0, -40.0), (40.0, 40.0)
    coef = np.random.default_rng(2).uniform(0.5, 1.5, (1, 49))
    L = oracle.Lrf(oracle.XY, sxy, n_int + (0,), lo + (0,), hi + (0,), coef)
    P = oracle.CgsParams(n_xy=5, iters=4, step_xy=2.0)
    s = np.array([[37.0]])
    start = np.array([[1.0, -3.0, 0.0]])
    r = oracle.cgs(L, P, s, start_xyz=start, mutant=mutant)
    assert np.all(r["trace"] == 0), r["trace"]
    walk = -2.0 * P.step_xy * sum(P.shrink ** k for k in range(P.iters))
    assert np.allclose(r["xyz"][0, :2], start[0, :2] + walk, atol=1e-12)


def pin_domain(mutant=0):
    """Nodes outside the LRF's box score -inf: with every node tied, the
    search takes the lowest-index node inside the box (re-derived here by
    direct enumeration)."""
    sxy = np.array([[3.0, 1.0]])  # one sensor: every node ties exactly
    n_int, lo, hi = (4, 4), (-20.0, -20.0), (20.0, 20.0)
    coef = np.random.default_rng(6).uniform(0.5, 1.5, (1, 49))
    L = oracle.Lrf(oracle.XY, sxy, n_int + (0,), lo + (0,), hi + (0,), coef)
    P = oracle.CgsParams(n_xy=5, iters=5, step_xy=4.0)
    s = np.array([[42.0]])
    start = np.array([[-18.8, 17.0, 0.0]])
    r = oracle.cgs(L, P, s, start_xyz=start, mutant=mutant)
    cx, cy, st = start[0, 0], start[0, 1], P.step_xy
    for it in range(P.iters):
        pick = None
        for k in range(P.n_xy * P.n_xy):
            x = cx + (k % P.n_xy - 2) * st
            y = cy + (k // P.n_xy - 2) * st
            if -20.0 <= x <= 20.0 and -20.0 <= y <= 20.0:
                pick = (k, x, y)
                break
        assert r["trace"][0, it] == pick[0], (it, r["trace"][0], pick)
        cx, cy = pick[1], pick[2]
        st *= P.shrink
    assert abs(r["xyz"][0, 0] - cx) < 1e-12 and abs(r["xyz"][0, 1] - cy) < 1e-12


def pin_event_status(mutant=0):
    """Zero total signal -> zero-signal status; negative, NaN or infinite
    signals -> bad-signal status; outputs NaN for both."""
    L, _ = _small_xy_lrf(mutant)
    P = oracle.CgsParams(n_xy=5, iters=2, step_xy=1.0)
    s = np.full((5, 9), 10.0)
    s[0] = 0.0
    s[1, 3] = -1.0
    s[2, 4] = np.nan
    s[3, 5] = np.inf
    r = oracle.cgs(L, P, s, mutant=mutant)
    assert list(r["status"]) == [2, 3, 3, 3, 0]
    assert np.all(np.isnan(r["xyz"][:4])) and np.all(np.isnan(r["E"][:4]))
    assert np.all(np.isfinite(r["xyz"][4]))


def pin_replay(mutant=0):
    """Replaying the oracle's own path certifies it with no ties; a path
    that takes a clearly worse node is flagged."""
    L, g = _small_xy_lrf(mutant)
    ev = synth.draw_events(L.sensor_xy, g, 40, 5, region="square", extent=10.0, e0=2000.0)
    P = oracle.CgsParams(n_xy=7, iters=5, step_xy=2.0)
    r = oracle.cgs(L, P, ev.signals, gain_cog=g, mutant=mutant)
    rp = oracle.cgs_replay(L, P, ev.signals, r["trace"], gain_cog=g, mutant=mutant)
    assert np.all(rp["n_tie"] == 0) and np.all(rp["n_bad"] == 0)
    assert np.array_equal(rp["xyz"], r["xyz"]) and np.array_equal(rp["logL"], r["logL"])
    bad = r["trace"].copy()
    bad[:, 0] = np.where(bad[:, 0] == 0, 48, 0)  # a far corner instead of the best node
    rp = oracle.cgs_replay(L, P, ev.signals, bad, gain_cog=g, mutant=mutant)
    assert np.all(rp["n_bad"] >= 1)


# --------------------------------------------------------------------------
# learned proposal
# --------------------------------------------------------------------------


def _small_mlp(seed, n_in=6, n_hid=5, n_out=3, scale=0.7):
    rng = np.random.default_rng(seed)
    return oracle.Mlp(rng.normal(0, scale, (n_hid, n_in)), rng.normal(0, 0.3, n_hid),
                      rng.normal(0, scale, (n_hid, n_hid)), rng.normal(0, 0.3, n_hid),
                      rng.normal(0, scale, (n_out, n_hid)), rng.normal(0, 0.3, n_out))


def pin_gelu(mutant=0):
    """GELU(x) = x Phi(x): Phi from scipy's normal CDF; GELU(x) - GELU(-x) = x."""
    from scipy.stats import norm
    for x in (-3.0, -0.7, 0.0, 0.4, 1.3, 3.0):
        assert abs(oracle.gelu(x, mutant) - x * norm.cdf(x)) < 1e-14
        assert abs(oracle.gelu(x, mutant) - oracle.gelu(-x, mutant) - x) < 1e-14


def pin_mlp_forward(mutant=0):
    """With W1 = W2 = 0 the output is W3 GELU(b2) + b3 (GELU by scipy); the
    sum normalisation makes the output invariant to scaling all signals."""
    from scipy.stats import norm
    M = _small_mlp(3)
    M.W1[:] = 0.0
    M.W2[:] = 0.0
    sig = np.random.default_rng(1).uniform(1, 50, (4, 6))
    want = M.W3 @ (M.b2 * norm.cdf(M.b2)) + M.b3
    out = oracle.mlp_forward(M, sig, mutant)
    assert np.abs(out - want[None, :]).max() < 1e-12
    M = _small_mlp(4)
    a = oracle.mlp_forward(M, sig, mutant)
    b = oracle.mlp_forward(M, 7.5 * sig, mutant)
    assert np.abs(a - b).max() < 1e-12


def pin_mlp_gradient(mutant=0):
    """Back-propagated gradients of the mean squared error match central
    differences of the loss (relative error <= 1e-6)."""
    M = _small_mlp(5)
    rng = np.random.default_rng(6)
    sig = rng.uniform(1, 40, (7, 6))
    tgt = rng.normal(0, 1, (7, 3))
    loss, grads = oracle.mlp_loss_grad(M, sig, tgt, mutant)
    h = 1e-6
    for P, G in zip(M.params(), grads):
        flat, gflat = P.reshape(-1), G.reshape(-1)
        for idx in range(0, flat.size, max(1, flat.size // 6)):
            old = flat[idx]
            flat[idx] = old + h
            lp, _ = oracle.mlp_loss_grad(M, sig, tgt, mutant)
            flat[idx] = old - h
            lm, _ = oracle.mlp_loss_grad(M, sig, tgt, mutant)
            flat[idx] = old
            num = (lp - lm) / (2 * h)
            assert abs(num - gflat[idx]) <= 1e-6 * max(1e-3, abs(num)), (num, gflat[idx])


def pin_adam(mutant=0):
    """From m = v = 0 the first Adam step moves every parameter by
    -lr g / (|g| + eps); the second step follows the bias-corrected moments."""
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    p = np.array([1.0, 2.0, 3.0, 4.0])
    m, v = np.zeros(4), np.zeros(4)
    oracle.adam_step(p, g, m, v, 1, lr=0.01, mutant=mutant)
    want = np.array([1.0, 2.0, 3.0, 4.0]) - 0.01 * g / (np.abs(g) + 1e-8)
    assert np.abs(p - want).max() < 1e-12
    g2 = np.array([0.1, 0.1, 0.1, 0.1])
    m2 = 0.9 * (0.1 * g) + 0.1 * g2
    v2 = 0.999 * (0.001 * g * g) + 0.001 * g2 * g2
    want2 = want - 0.01 * (m2 / (1 - 0.81)) / (np.sqrt(v2 / (1 - 0.999 ** 2)) + 1e-8)
    oracle.adam_step(p, g2, m, v, 2, lr=0.01, mutant=mutant)
    assert np.abs(p - want2).max() < 1e-12


def pin_deviance(mutant=0):
    """The Poisson deviance is 0 for noise-free signals at the true position
    and positive elsewhere."""
    L, _ = _small_xy_lrf(mutant)
    xt = np.array([[2.0, -1.5, 0.0], [-4.0, 3.0, 0.0]])
    s = 1200.0 * oracle.lrf_eval(L, xt[:, :2], mutant=mutant)
    D = oracle.deviance_at(L, s, xt, mutant=mutant)
    assert np.abs(D).max() < 1e-9, D
    D2 = oracle.deviance_at(L, s, xt + np.array([[0.5, 0.0, 0.0]]), mutant=mutant)
    assert np.all(D2 > 1e-3)


# --------------------------------------------------------------------------
# simulation
# --------------------------------------------------------------------------


def pin_poisson_sampler(mutant=0):
    """Counts drawn by the oracle's sampler follow scipy's Poisson pmf
    (chi-squared test at 0.1 % per rate) for rates on both sides of the
    switch between inversion and transformed rejection, with the right mean
    and variance."""
    from scipy.stats import chi2, poisson
    for lam in (0.5, 5.0, 9.9, 10.0, 50.0, 500.0):
        x = oracle.poisson_draws(lam, 17, 40000, mutant)
        assert abs(x.mean() - lam) < 5 * np.sqrt(lam / x.size), (lam, x.mean())
        assert abs(x.var() / lam - 1.0) < 0.05, (lam, x.var())
        lo, hi = int(poisson.ppf(1e-4, lam)), int(poisson.ppf(1 - 1e-4, lam))
        edges = np.arange(lo, hi + 2)
        obs, _ = np.histogram(x, bins=edges)
        exp = x.size * poisson.pmf(edges[:-1], lam)
        keep = exp > 5
        stat = ((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum()
        assert stat < chi2.ppf(0.999, keep.sum() - 1), (lam, stat)


def pin_uniform_stream(mutant=0):
    """Philox outputs as uniforms: equal-probability bins pass a chi-squared
    test and neighbouring draws are uncorrelated; different counters give
    different blocks."""
    from scipy.stats import chi2
    u = []
    for e in range(20000):
        b = oracle.philox(1234567, (e, 0, 7, 0), mutant)
        u.extend(((b >> 8).astype(np.float64) + 0.5) / 16777216.0)
    u = np.array(u)
    obs, _ = np.histogram(u, bins=64, range=(0.0, 1.0))
    exp = u.size / 64
    assert ((obs - exp) ** 2 / exp).sum() < chi2.ppf(0.999, 63)
    assert abs(np.corrcoef(u[:-1], u[1:])[0, 1]) < 0.01
    assert not np.array_equal(oracle.philox(1, (0, 0, 0, 0)), oracle.philox(1, (1, 0, 0, 0)))
    assert not np.array_equal(oracle.philox(1, (0, 0, 0, 0)), oracle.philox(2, (0, 0, 0, 0)))


def pin_simulator(mutant=0):
    """Event simulation: sources uniform in the square (mean, variance a^2/3)
    and in the disk (r^2 uniform), energies uniform in e0 (1 +- spread), counts
    with mean E eta_i(source) and Poisson variance, plus N(1, sigma^2) per
    photo-electron when a single-p.e. spread is given (variance E eta (1 +
    sigma^2)); different first_event values continue one stream."""
    L, _ = _small_xy_lrf()
    a, e0, sp = 4.0, 800.0, 0.1
    sig, tr = oracle.simulate(L, 99, 0, 20000, region="square", extent=a, e0=e0, e_spread=sp, mutant=mutant)
    n = len(tr)
    for c in (0, 1):
        assert abs(tr[:, c].mean()) < 4 * a / np.sqrt(3 * n)
        assert abs(tr[:, c].var() / (a * a / 3) - 1) < 0.05
    assert tr[:, 0].min() >= -a and tr[:, 0].max() <= a
    assert tr[:, 3].min() >= e0 * (1 - sp) and tr[:, 3].max() <= e0 * (1 + sp)
    assert abs(tr[:, 3].mean() / e0 - 1) < 4 * sp / np.sqrt(3 * n)
    mu = tr[:, 3:4] * oracle.lrf_eval(L, tr[:, :2])
    z = (sig - mu) / np.sqrt(mu)
    assert np.all(np.abs(z.mean(0)) < 4 / np.sqrt(n)), z.mean(0)
    assert np.all(np.abs(z.var(0) - 1) < 0.05), z.var(0)
    assert np.array_equal(sig, np.round(sig))
    sd, td = oracle.simulate(L, 99, 0, 20000, region="disk", extent=a, e0=e0, e_spread=sp, mutant=mutant)
    r2 = (td[:, 0] ** 2 + td[:, 1] ** 2) / (a * a)
    assert r2.max() <= 1 + 1e-12 and abs(r2.mean() - 0.5) < 4 * np.sqrt(1 / 12 / n)
    ss, ts = oracle.simulate(L, 99, 0, 20000, region="square", extent=a, e0=e0, e_spread=sp, spe_sigma=0.3,
                             mutant=mutant)
    mu = ts[:, 3:4] * oracle.lrf_eval(L, ts[:, :2])
    assert np.all(np.abs((ss - mu).var(0) / (mu * 1.09).mean(0) - 1) < 0.08)
    s2, t2 = oracle.simulate(L, 99, 5000, 100, region="square", extent=a, e0=e0, e_spread=sp, mutant=mutant)
    assert np.array_equal(s2, sig[5000:5100]) and np.array_equal(t2, tr[5000:5100])


def pin_logtable_ranks_like_likelihood(mutant=0):
    """The table scores sum_i s_i T[g][i] differ from the profiled
    log-likelihood F(g) = sum s ln eta - S ln H by a constant per event, and
    every column of T averages to zero over the grid."""
    L, _ = _small_xy_lrf(mutant)
    T, m = oracle.logtable(L, 9, 7, mutant)
    assert np.abs(T.mean(axis=0)).max() < 1e-12
    rng = np.random.default_rng(31)
    sig = rng.poisson(900 * synth.truth_eta(L.sensor_xy, np.ones(9), rng.uniform(-8, 8, (5, 2)))).astype(float)
    gx = -16.0 + (np.arange(9) + 0.5) * 32.0 / 9
    gy = -16.0 + (np.arange(7) + 0.5) * 32.0 / 7
    pts = np.array([(x, y, 0.0) for y in gy for x in gx])
    for s in sig:
        F = oracle.objective_at(L, np.repeat(s[None], len(pts), 0), pts, mutant)
        d = s @ T.T - F
        assert np.abs(d - d[0]).max() < 1e-9 * max(1.0, np.abs(F).max())


# --------------------------------------------------------------------------
# event filters and iterative LRF reconstruction (Sec. 5.2, 6.2, 6.3, 8)
# --------------------------------------------------------------------------


def _hex19_truth(gain_sigma=0.1):
    """The 19-PMT radial group with relative gains N(1, gain_sigma^2)."""
    w = synth.workloads.get("hex19_radial")
    gains = synth.sensor_gains(19, gain_sigma, 5)
    pts, vals = w.fit_samples()
    coef, _, _ = oracle.lrf_fit(w.n_int, w.lo, w.hi, pts, vals)
    L = oracle.Lrf(oracle.RADIAL, w.sensor_xy, w.n_int + (0, 0), w.lo + (0, 0), w.hi + (0, 0), coef, shared=True,
                   gain=gains)
    return w, L, gains


def pin_chi2(mutant=0):
    """Pearson chi-squared: exactly 0 for noise-free signals at the true
    position and energy; for Poisson counts at the true position and energy
    each sensor's term (s - mu)^2 / mu has expectation 1, so chi2 * (n_s - 3)
    averages n_s; sensors outside the LRF's reach add nothing."""
    w, L, _ = _hex19_truth()
    rng = np.random.default_rng(3)
    n = 20000
    xy = rng.uniform(-40, 40, (n, 2))
    xyz = np.concatenate([xy, np.zeros((n, 1))], axis=1)
    E = rng.uniform(2000.0, 4000.0, n)
    mu = E[:, None] * oracle.lrf_eval(L, xy)
    assert np.abs(oracle.chi2_at(L, mu, xyz, E, mutant)).max() < 1e-18
    s = rng.poisson(mu).astype(np.float64)
    c = oracle.chi2_at(L, s, xyz, E, mutant) * (19 - 3)
    sd = np.sqrt((2.0 * 19 + (1.0 / mu).sum(1).mean()) / n)
    assert abs(c.mean() - 19.0) < 5 * sd, (c.mean(), sd)
    # a far point: sensors beyond the 150 mm profile contribute nothing
    far = np.array([[140.0, 0.0, 0.0]])
    m1 = 3000.0 * np.nan_to_num(oracle.lrf_eval(L, far[:, :2]))
    t = oracle.chi2_at(L, m1 + 1.0, far, np.array([3000.0]), mutant)[0] * 16
    inside = m1[0] > 0
    assert abs(t - (1.0 / m1[0][inside]).sum()) < 1e-9 * t
    assert np.isnan(oracle.chi2_at(L, s[:1], np.array([[np.nan, 0.0, 0.0]]), E[:1], mutant)[0])


def pin_event_filter(mutant=0):
    """Sec. 5.2 cuts: bounds are inclusive, every cut acts alone, failed or
    non-finite reconstructions never pass, and with every cut off every
    finished event passes."""
    xyz = np.array([[0.0, 0.0, 0.0], [3.0, 4.0, 0.0], [3.0, 4.0001, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0],
                    [0.0, 0.0, 0.0], [np.nan, 0.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0]])
    E = np.array([100.0, 100.0, 100.0, 50.0, 150.0, 100.0, 100.0, 100.0, 100.0])
    chi2 = np.array([1.0, 1.0, 1.0, 1.0, 1.0, 2.0, 1.0, 1.0, np.inf])
    ssum = np.array([10.0, 10.0, 10.0, 10.0, 10.0, 10.0, 10.0, 20.0, 10.0])
    st = np.array([0, 0, 0, 0, 0, 0, 0, 0, 0])
    f = oracle.event_filter
    C = oracle.EventCuts
    assert f(st, xyz, E, chi2, ssum, C(), mutant).tolist() == [1, 1, 1, 1, 1, 1, 0, 1, 0]
    assert f(st, xyz, E, chi2, ssum, C(r_max=5.0), mutant).tolist() == [1, 1, 0, 1, 1, 1, 0, 1, 0]
    assert f(st, xyz, E, chi2, ssum, C(e_lo=50.0, e_hi=100.0), mutant).tolist() == [1, 1, 1, 1, 0, 1, 0, 1, 0]
    assert f(st, xyz, E, chi2, ssum, C(chi2_max=1.0), mutant).tolist() == [1, 1, 1, 1, 1, 0, 0, 1, 0]
    assert f(st, xyz, E, chi2, ssum, C(sum_lo=5.0, sum_hi=10.0), mutant).tolist() == [1, 1, 1, 1, 1, 1, 0, 0, 0]
    assert f(st, xyz + [[1.0, 0.0, 0.0]], E, chi2, ssum, C(r_max=5.0, cx=1.0), mutant).tolist()[:3] == [1, 1, 0]
    st2 = st.copy()
    st2[0] = oracle.EVT_ZERO_SIGNAL
    assert not f(st2, xyz, E, chi2, ssum, C(), mutant)[0]


def pin_shift(mutant=0):
    """Random shifts: normal (Kolmogorov-Smirnov against scipy's normal CDF),
    mean 0, variance sigma^2, uncorrelated components; fixed by (seed, cycle,
    event) alone; another cycle gives independent draws."""
    from scipy.stats import kstest, norm
    ev = np.arange(50000) * 7 + 3
    d = oracle.shift_xy(11, 2, ev, 1.5, mutant)
    for c in (0, 1):
        assert abs(d[:, c].mean()) < 5 * 1.5 / np.sqrt(ev.size)
        assert abs(d[:, c].var() / 2.25 - 1) < 0.03
        assert kstest(d[:, c] / 1.5, norm.cdf).pvalue > 1e-4
    assert abs(np.corrcoef(d[:, 0], d[:, 1])[0, 1]) < 0.02
    assert np.array_equal(oracle.shift_xy(11, 2, ev[100:200], 1.5, mutant), d[100:200])
    d3 = oracle.shift_xy(11, 3, ev, 1.5, mutant)
    assert abs(np.corrcoef(d[:, 0], d3[:, 0])[0, 1]) < 0.02


def pin_lrf_refit_exact(mutant=0):
    """When the signals are exactly E times a spline on the LRF's own knot
    grid, the refit recovers that spline (least squares on consistent data):
    per-sensor XY LRFs, a radial group with known gains, per-sensor radial
    LRFs; with the group's profile fixed, the gain refit recovers planted
    gains, scaled to mean 1 with eta = g f unchanged (Sec. 6.2, 6.3)."""
    rng = np.random.default_rng(8)
    sxy = synth.square_array(2, 10.0)
    n_int, lo, hi = (5, 4, 0), (-12.0, -10.0, 0.0), (12.0, 10.0, 0.0)
    cx = rng.uniform(0.5, 2.0, (4, 8 * 7))
    Lxy = oracle.Lrf(oracle.XY, sxy, n_int, lo, hi, cx)
    xy = np.stack([rng.uniform(-12, 12, 3000), rng.uniform(-10, 10, 3000)], axis=1)
    xyz = np.concatenate([xy, np.zeros((3000, 1))], axis=1)
    E = rng.uniform(500, 1500, 3000)
    s = E[:, None] * oracle.lrf_eval(Lxy, xy, mutant)
    R = oracle.lrf_refit(Lxy, s, xyz, E, mutant=mutant)
    assert np.abs(R.coef - cx).max() < 1e-8 * np.abs(cx).max()
    w, Lt, gains = _hex19_truth()
    xy = rng.uniform(-60, 60, (2000, 2))
    xyz = np.concatenate([xy, np.zeros((2000, 1))], axis=1)
    E = rng.uniform(5000, 15000, 2000)
    s = E[:, None] * np.nan_to_num(oracle.lrf_eval(Lt, xy, mutant))
    # distances reach 134 mm: compare the profiles where samples exist (the
    # unsampled tail is set by the ridge fallback)
    rr = np.linspace(0.0, 130.0, 66)[:, None]
    prof = lambda c: oracle.spline_eval(Lt.n_int[:1], Lt.lo[:1], Lt.hi[:1], c, rr, mutant)
    ft = prof(Lt.coef[0])
    R = oracle.lrf_refit(Lt, s, xyz, E, mutant=mutant)
    assert np.abs(prof(R.coef[0]) - ft).max() < 1e-7 * ft.max()
    R2 = oracle.lrf_refit(Lt, s, xyz, E, shared=False, mutant=mutant)
    d = xyz[:, None, :2] - Lt.sensor_xy[None]
    r = np.sqrt((d ** 2).sum(-1))
    for i in (0, 7, 18):  # each sensor's unsampled tail takes the ridge fallback (~1e-6 effect)
        ok = rr[:, 0] <= r[:, i].max()
        assert np.abs(prof(R2.coef[i]) - gains[i] * ft)[ok].max() < 3e-6 * ft.max()
    L1 = oracle.Lrf(oracle.RADIAL, Lt.sensor_xy, Lt.n_int, Lt.lo, Lt.hi, Lt.coef, shared=True, gain=np.ones(19))
    s1 = E[:, None] * np.nan_to_num(oracle.lrf_eval(L1, xy, mutant)) * gains[None, :]
    R3 = oracle.lrf_refit(L1, s1, xyz, E, refit_gains=True, mutant=mutant)
    gm = gains.mean()
    assert abs(R3.gain.mean() - 1.0) < 1e-12
    assert np.abs(R3.gain - gains / gm).max() < 2e-3  # the profile absorbed the mean gain error
    g = oracle.gain_refit(20, 0.0, 150.0, Lt.coef, r, s / E[:, None], mutant)
    assert np.abs(g - gains).max() < 1e-10


def pin_iterative_lrf_converges(mutant=0):
    """Sec. 8 on a flood dataset (2000 events of the 19-PMT group, gains
    known): starting from a simulated guess of the profile that is too wide
    (the truth form with r0 = 55 mm instead of 40 mm), whose reconstruction
    errs by several mm, four cycles of reconstruct - refit bring the position
    error within 6 % of that with the true LRFs and the profile shape within
    3 % of the truth; every event stays in (no cut active), and the mean
    chi2 settles near 1."""
    w, Lt, gains = _hex19_truth()
    sig, tr = oracle.simulate(Lt, 78, 0, 2000, region="disk", extent=60.0, e0=1e4, e_spread=0.05, mutant=mutant)
    P = oracle.CgsParams(n_xy=w.n_xy, iters=w.iters, step_xy=w.step_xy, shrink=w.shrink)
    rms = lambda L: np.sqrt(((oracle.cgs(L, P, sig, mutant=mutant)["xyz"][:, :2] - tr[:, :2]) ** 2).sum(1).mean())
    pts, _ = w.fit_samples()
    c0, _, _ = oracle.lrf_fit(w.n_int, w.lo, w.hi, pts, synth.eta_axial(pts[:, 0], r0=55.0)[:, None], mutant=mutant)
    L0 = oracle.Lrf(oracle.RADIAL, Lt.sensor_xy, Lt.n_int, Lt.lo, Lt.hi, c0, shared=True, gain=gains.copy())
    e_true, e0 = rms(Lt), rms(L0)
    L, st = oracle.lrf_iterate(L0, P, sig, 4, oracle.EventCuts(), mutant=mutant)
    e4 = rms(L)
    assert e0 > 5 * e_true and e4 < 1.06 * e_true, (e_true, e0, e4)
    assert st[-1]["n_kept"] == 2000 and 0.9 < st[-1]["mean_chi2"] < 1.15, st[-1]
    rr = np.linspace(0.0, 100.0, 51)[:, None]
    f = oracle.spline_eval(L.n_int[:1], L.lo[:1], L.hi[:1], L.coef[0], rr)
    ft = oracle.spline_eval(Lt.n_int[:1], Lt.lo[:1], Lt.hi[:1], Lt.coef[0], rr)
    assert np.abs(f / f[0] - ft / ft[0]).max() < 0.03

# --------------------------------------------------------------------------
# search variants (Sec. 5.1.2, 5.3)
# --------------------------------------------------------------------------


def _variant_events(L, g, n, seed, extent=12.0, e0=2500.0):
    return synth.draw_events(L.sensor_xy, g, n, seed, region="square", extent=extent, e0=e0).signals


def pin_variant_defaults_and_passive(mutant=0):
    """With no option set the variant search is the plain search, bit for
    bit; a passive sensor (Sec. 5.3) gives exactly the search on the detector
    without that sensor (its LRF, signal and gain removed)."""
    L, g = _small_xy_lrf(mutant)
    P = oracle.CgsParams(n_xy=9, iters=6, step_xy=1.5)
    sig = _variant_events(L, g, 60, 5)
    a = oracle.cgs(L, P, sig, gain_cog=g, mutant=mutant)
    b = oracle.cgs_variant(L, P, sig, oracle.Variant(), gain=g, mutant=mutant)
    for k in ("xyz", "E", "logL", "status", "trace"):
        assert np.array_equal(a[k], b[k]), k
    keep = np.array([i for i in range(9) if i != 4])
    L2 = oracle.Lrf(oracle.XY, L.sensor_xy[keep], L.n_int, L.lo, L.hi, L.coef[keep])
    c = oracle.cgs(L2, P, sig[:, keep], gain_cog=g[keep], mutant=mutant)
    pas = np.zeros(9, dtype=int)
    pas[4] = 1
    sig_bad = sig.copy()
    sig_bad[:, 4] = -7.0  # a passive sensor's signal is never read
    d = oracle.cgs_variant(L, P, sig_bad, oracle.Variant(passive=pas), gain=g, mutant=mutant)
    for k in ("xyz", "E", "logL", "status", "trace"):
        assert np.array_equal(c[k], d[k]), k


def pin_variant_start_and_cuts(mutant=0):
    """The strongest-sensor start (Sec. 5.1.2.1) is the plain search started
    at the sensor with the largest s_i / g_i; the signal cut and the distance
    cut (Sec. 5.1.2) equal, event by event, the search with the cut sensors
    made passive, whenever the cut keeps the start sensor (the distance cut
    always does; the start is chosen before any cut)."""
    L, g = _small_xy_lrf(mutant)
    P = oracle.CgsParams(n_xy=9, iters=6, step_xy=1.5)
    sig = _variant_events(L, g, 40, 6)
    best = np.argmax(sig / g[None, :], axis=1)
    start = np.concatenate([L.sensor_xy[best], np.zeros((40, 1))], axis=1)
    a = oracle.cgs(L, P, sig, start_xyz=start, mutant=mutant)
    b = oracle.cgs_variant(L, P, sig, oracle.Variant(start=1), gain=g, mutant=mutant)
    for k in ("xyz", "E", "logL", "trace"):
        assert np.array_equal(a[k], b[k]), k
    thr, R = 100.0, 9.0
    n_sig = 0
    for e in range(40):
        s1 = sig[e:e + 1]
        cuts = [(dict(max_distance=R), np.hypot(*(L.sensor_xy - start[e, :2]).T) > R)]
        if s1[0, best[e]] >= thr:
            cuts.append((dict(min_signal=thr), s1[0] < thr))
            n_sig += 1
        for cut, pas in cuts:
            x = oracle.cgs_variant(L, P, s1, oracle.Variant(start=1, **cut), gain=g, mutant=mutant)
            y = oracle.cgs_variant(L, P, s1, oracle.Variant(start=1, passive=pas.astype(int)), gain=g, mutant=mutant)
            for k in ("xyz", "E", "logL", "trace"):
                assert np.array_equal(x[k], y[k], equal_nan=k != "trace"), (e, cut, k)
    assert n_sig >= 10, n_sig


def pin_least_squares(mutant=0):
    """Least-squares criterion (Sec. 5.1.2), read as Pearson's statistic with
    E = S / H: noise-free signals are recovered exactly (the statistic is 0
    only at the source; the strongest-sensor start puts the source on a node
    of the first grid), and on a tiny detector the contracting-grid result is
    the minimum of (H / S) sum s_i^2 / eta_i - S (the same statistic in
    another algebraic form) over an exhaustive fine grid."""
    L, g = _small_xy_lrf(mutant)
    P = oracle.CgsParams(n_xy=9, iters=6, step_xy=1.5)
    xt = np.array([[3.0, -1.5]])
    s = np.array([[2500.0]]) * oracle.lrf_eval(L, xt, mutant=mutant)
    assert np.argmax(s[0] / g) == 4  # the centre sensor, at (0, 0)
    v = oracle.cgs_variant(L, P, s, oracle.Variant(criterion=1, start=1), gain=g, mutant=mutant)
    assert v["status"][0] == 0
    assert np.abs(v["xyz"][0, :2] - xt[0]).max() < 1e-12 and abs(v["E"][0] / 2500.0 - 1) < 1e-12, v["xyz"]
    sxy = synth.square_array(2, 10.0)
    g4 = np.array([1.0, 0.95, 1.05, 1.02])
    n_int, lo, hi = (10, 10), (-15.0, -15.0), (15.0, 15.0)
    pts = synth.grid_samples(n_int, lo, hi, 4)
    coef, _, _ = oracle.lrf_fit(n_int, lo, hi, pts, synth.truth_eta(sxy, g4, pts, r0=20.0), mutant=mutant)
    L4 = oracle.Lrf(oracle.XY, sxy, n_int + (0,), lo + (0,), hi + (0,), coef)
    ev = synth.draw_events(sxy, g4, 60, 78, region="square", extent=6.0, e0=4000.0, r0=20.0)
    P4 = oracle.CgsParams(n_xy=9, iters=8, step_xy=3.75)
    x = oracle.cgs_variant(L4, P4, ev.signals, oracle.Variant(criterion=1), gain=g4, mutant=mutant)
    fine = 0.05
    gx = np.linspace(-15, 15, int(30 / fine) + 1)
    X, Y = np.meshgrid(gx, gx)
    grid = np.stack([X.ravel(), Y.ravel()], axis=1)
    eta = oracle.lrf_eval(L4, grid, mutant=mutant)
    H = eta.sum(1)
    ok = 0
    for e in range(60):
        sv = ev.signals[e]
        S = sv.sum()
        stat = H / S * (sv[None, :] ** 2 / eta).sum(1) - S
        bxy = grid[np.argmin(stat)]
        d = np.hypot(*(x["xyz"][e, :2] - bxy))
        ok += d <= 2.0 * (fine + P4.step_xy * P4.shrink ** (P4.iters - 1))
    assert ok / 60 >= 0.95, ok

# --------------------------------------------------------------------------
# LRF parameterisation schemes (Sec. 6.1.1, 6.1.2)
# --------------------------------------------------------------------------


def _scheme_lrfs(mutant=0, seed=4):
    """Small composite, axial+z and sliced LRF sets on a 2 x 2 array with
    random smooth coefficients (positive, order 1)."""
    rng = np.random.default_rng(seed)
    sxy = synth.square_array(2, 10.0)
    ca = np.stack([0.04 / (1 + (np.linspace(-7.5, 37.5, 10) / 20.0) ** 2) ** 1.5 for _ in range(4)])
    cxy = rng.uniform(-0.002, 0.002, (4, 9 * 9))
    comp = oracle.Lrf(oracle.COMPOSITE, sxy, (6, 6, 0), (-12.0, -12.0, 0.0), (12.0, 12.0, 0.0),
                      np.concatenate([ca, cxy], axis=1), n_int_r=7, hi_r=35.0)
    # axial+z: the closed-form 3D response (its width changes with z, so z is
    # identifiable) fitted on the (r, z) grid, times a per-sensor factor
    rz = synth.grid_samples((6, 5), (0.0, 0.0), (30.0, 20.0), 4)
    c1, _, _ = oracle.lrf_fit((6, 5), (0.0, 0.0), (30.0, 20.0), rz, synth.eta_3d(rz[:, 0], rz[:, 1], r0=15.0),
                              mutant=mutant)
    caz = c1 * rng.uniform(0.9, 1.1, (4, 1))
    az = oracle.Lrf(oracle.AXIAL_Z, sxy, (6, 5, 0), (0.0, 0.0, 0.0), (30.0, 20.0, 0.0), caz)
    csl = rng.uniform(0.5, 1.5, (4, 3 * 49)) * 0.01
    sl = oracle.Lrf(oracle.SLICED, sxy, (4, 4, 0), (-12.0, -12.0, 0.0), (12.0, 12.0, 20.0), csl, n_planes=3)
    return sxy, comp, az, sl


def pin_lrf_schemes_eval(mutant=0):
    """Composite = its axial part (as per-sensor radial LRFs) plus its XY
    part (as XY LRFs); axial+z = the two-dimensional spline of (r, z) evaluated
    by the plain tensor routine; sliced = the plane's XY LRF on each plane and
    the linear blend (1 - w) f_j + w f_{j+1} between planes."""
    sxy, comp, az, sl = _scheme_lrfs(mutant)
    rng = np.random.default_rng(9)
    p2 = rng.uniform(-11.0, 11.0, (50, 2))
    rad = oracle.Lrf(oracle.RADIAL, sxy, (7, 0, 0), (0.0, 0.0, 0.0), (35.0, 0.0, 0.0), comp.coef[:, :10])
    xy = oracle.Lrf(oracle.XY, sxy, (6, 6, 0), (-12.0, -12.0, 0.0), (12.0, 12.0, 0.0), comp.coef[:, 10:])
    want = oracle.lrf_eval(rad, p2, mutant) + oracle.lrf_eval(xy, p2, mutant)
    assert np.abs(oracle.lrf_eval(comp, p2, mutant) - want).max() < 1e-15
    p3 = np.concatenate([p2, rng.uniform(0.0, 20.0, (50, 1))], axis=1)
    got = oracle.lrf_eval(az, p3, mutant)
    d = p3[:, None, :2] - sxy[None]
    r = np.sqrt((d ** 2).sum(-1))
    for i in range(4):
        ref = oracle.spline_eval((6, 5), (0.0, 0.0), (30.0, 20.0), az.coef[i], np.stack([r[:, i], p3[:, 2]], 1))
        assert np.abs(got[:, i] - ref).max() < 1e-14
    planes = [oracle.Lrf(oracle.XY, sxy, (4, 4, 0), (-12.0, -12.0, 0.0), (12.0, 12.0, 0.0),
                         sl.coef[:, 49 * j:49 * (j + 1)]) for j in range(3)]
    f = [oracle.lrf_eval(P, p2, mutant) for P in planes]
    for z, w0, j in ((0.0, 1.0, 0), (10.0, 1.0, 1), (20.0, 1.0, 2), (2.5, 0.75, 0), (17.5, 0.25, 1)):
        v = oracle.lrf_eval(sl, np.concatenate([p2, np.full((50, 1), z)], 1), mutant)
        ref = w0 * f[j] + (1.0 - w0) * f[min(j + 1, 2)]
        assert np.abs(v - ref).max() < 1e-15, (z, np.abs(v - ref).max())


def pin_lrf_schemes_fit(mutant=0):
    """Fits of the schemes recover LRFs that lie in their spline spaces:
    axial+z from scattered (x, y, z) samples, sliced from samples on the
    planes; a composite fit of purely axial data reproduces it with a
    (numerically) zero XY part."""
    sxy, comp, az, sl = _scheme_lrfs(mutant)
    rng = np.random.default_rng(10)
    p3 = np.stack([rng.uniform(-12, 12, 4000), rng.uniform(-12, 12, 4000), rng.uniform(0, 20, 4000)], 1)
    F = oracle.lrf_fit_axial_z(sxy, p3, oracle.lrf_eval(az, p3, mutant), (6, 5), 30.0, 0.0, 20.0, mutant=mutant)
    q = np.stack([rng.uniform(-10, 10, 300), rng.uniform(-10, 10, 300), rng.uniform(0, 20, 300)], 1)
    # distances reach 24 of the profile's 30 mm: the unsampled tail takes the
    # ridge fallback, which moves the values near 0.05 by ~5e-9
    assert np.abs(oracle.lrf_eval(F, q, mutant) - oracle.lrf_eval(az, q, mutant)).max() < 5e-8
    pz = np.concatenate([p3[:, :2], rng.integers(0, 3, (4000, 1)) * 10.0], 1)
    G = oracle.lrf_fit_sliced(sxy, pz, oracle.lrf_eval(sl, pz, mutant), (4, 4), (-12.0, -12.0), (12.0, 12.0), 3,
                              0.0, 20.0, mutant=mutant)
    assert np.abs(oracle.lrf_eval(G, q, mutant) - oracle.lrf_eval(sl, q, mutant)).max() < 1e-9
    ax = oracle.Lrf(oracle.COMPOSITE, sxy, comp.n_int, comp.lo, comp.hi,
                    np.concatenate([comp.coef[:, :10], np.zeros((4, 81))], 1), n_int_r=7, hi_r=35.0)
    p2 = p3[:, :2]
    H = oracle.lrf_fit_composite(sxy, p2, oracle.lrf_eval(ax, p2, mutant), 7, 35.0, (6, 6), (-12.0, -12.0),
                                 (12.0, 12.0), mutant=mutant)
    # values where samples exist; the axial tail beyond r = 24 mm is set by
    # the ridge fallback, which leaves the XY part at the 1e-8 level
    q2 = q[:, :2]
    assert np.abs(oracle.lrf_eval(H, q2, mutant) - oracle.lrf_eval(ax, q2, mutant)).max() < 1e-8
    assert np.abs(H.coef[:, 10:]).max() < 1e-7


def pin_lrf_schemes_search(mutant=0):
    """Noise-free signals of a source on grid nodes are recovered exactly by
    the contracting grids with each scheme (Gibbs' inequality), in 2D for
    composite and in 3D for axial+z and sliced."""
    sxy, comp, az, sl = _scheme_lrfs(mutant)
    P2 = oracle.CgsParams(n_xy=7, iters=5, step_xy=1.0)
    xt = np.array([[2.0, -1.0, 0.0]])
    s = 3000.0 * oracle.lrf_eval(comp, xt[:, :2], mutant)
    r = oracle.cgs(comp, P2, s, start_xyz=xt - np.array([[2.0, -1.0, 0.0]]), mutant=mutant)
    assert np.abs(r["xyz"] - xt).max() < 1e-12, r["xyz"]
    P3 = oracle.CgsParams(n_xy=7, iters=5, step_xy=1.0, n_z=5, step_z=2.0, z0=10.0)
    for L in (az, sl):
        xt = np.array([[1.0, 2.0, 12.0]])
        s = 3000.0 * oracle.lrf_eval(L, xt, mutant)
        r = oracle.cgs(L, P3, s, start_xyz=xt - np.array([[1.0, -1.0, 2.0]]), mutant=mutant)
        assert np.abs(r["xyz"] - xt).max() < 1e-12, (L.type, r["xyz"])


ALL_PINS = [
    pin_bspline_golden, pin_partition_of_unity, pin_fit_reproduces_cubics, pin_fit_h4_convergence,
    pin_lrf_matches_closed_form, pin_cog, pin_energy_is_ml, pin_logl_is_poisson, pin_profile_identity,
    pin_noise_free_recovery, pin_noise_free_recovery_3d, pin_cg_matches_brute_force, pin_ties_go_to_lowest_index, pin_domain,
    pin_event_status, pin_replay, pin_gelu, pin_mlp_forward, pin_mlp_gradient, pin_adam, pin_deviance,
    pin_poisson_sampler, pin_uniform_stream, pin_simulator, pin_logtable_ranks_like_likelihood,
    pin_chi2, pin_event_filter, pin_shift, pin_lrf_refit_exact, pin_iterative_lrf_converges,
    pin_variant_defaults_and_passive, pin_variant_start_and_cuts, pin_least_squares,
    pin_lrf_schemes_eval, pin_lrf_schemes_fit, pin_lrf_schemes_search,
]


# --------------------------------------------------------------------------
# Continuous minimisation (Sec. 5.1.2.1)
# --------------------------------------------------------------------------


def _all_type_lrfs(mutant=0, seed=6):
    """One LRF set of each type: radial (per sensor, with gains), XY, XYZ,
    axial+z and sliced (smooth responses sampled on the knot grids, random
    factors) on a 3 x 3 array of pitch 8 mm, and the composite set of the
    scheme pins (2 x 2 array)."""
    sxy2, comp, az, sl = _scheme_lrfs(mutant)
    sxy = synth.square_array(3, 8.0)
    rng = np.random.default_rng(seed)
    prof = 0.04 / (1 + (np.linspace(-5.0, 40.0, 10) / 20.0) ** 2) ** 1.5
    rad = oracle.Lrf(oracle.RADIAL, sxy, (7, 0, 0), (0.0, 0.0, 0.0), (35.0, 0.0, 0.0),
                     prof[None, :] * rng.uniform(0.95, 1.05, (9, 10)), gain=rng.uniform(0.9, 1.1, 9))
    kx = np.linspace(-12.0 - 6.0, 12.0 + 6.0, 9)
    X, Y = np.meshgrid(kx, kx)

    def bump(w):
        return np.stack([0.04 / (1 + ((X - sx) ** 2 + (Y - sy) ** 2) / w ** 2) ** 1.5 for sx, sy in sxy]).reshape(9, -1)

    xy = oracle.Lrf(oracle.XY, sxy, (6, 6, 0), (-12.0, -12.0, 0.0), (12.0, 12.0, 0.0),
                    bump(20.0) * rng.uniform(0.95, 1.05, (9, 81)))
    # XYZ: the bump widens with z (a z that only scaled every sensor alike
    # would be confounded with the energy)
    kz = np.linspace(-5.0, 25.0, 7)
    cxyz = np.stack([bump(15.0 + z) for z in kz], 1)  # [9][z][y*x]
    xyz = oracle.Lrf(oracle.XYZ, sxy, (6, 6, 4), (-12.0, -12.0, 0.0), (12.0, 12.0, 20.0),
                     cxyz.reshape(9, -1) * rng.uniform(0.95, 1.05, (9, 7 * 81)))
    # axial+z: the closed-form 3D response on the (r, z) grid; sliced: the
    # widening bump on the planes z = 0, 10, 20
    rz = synth.grid_samples((6, 5), (0.0, 0.0), (30.0, 20.0), 4)
    c1, _, _ = oracle.lrf_fit((6, 5), (0.0, 0.0), (30.0, 20.0), rz, synth.eta_3d(rz[:, 0], rz[:, 1], r0=15.0),
                              mutant=mutant)
    az3 = oracle.Lrf(oracle.AXIAL_Z, sxy, (6, 5, 0), (0.0, 0.0, 0.0), (30.0, 20.0, 0.0),
                     c1 * rng.uniform(0.95, 1.05, (9, 1)))
    csl = np.concatenate([bump(15.0 + z) for z in (0.0, 10.0, 20.0)], 1) * rng.uniform(0.95, 1.05, (9, 3 * 81))
    sl3 = oracle.Lrf(oracle.SLICED, sxy, (6, 6, 0), (-12.0, -12.0, 0.0), (12.0, 12.0, 20.0), csl, n_planes=3)
    return sxy, {"radial": rad, "xy": xy, "xyz": xyz, "composite": comp, "axial_z": az3, "sliced": sl3}


def pin_lrf_grad(mutant=0):
    """The analytic gradient of every LRF type equals central differences of
    the LRF values (h = 1e-5 mm) at interior points away from the sliced
    planes (where d/dz jumps) and from the sensors (where an axial LRF's
    direction is undefined)."""
    sxy, Ls = _all_type_lrfs(mutant)
    rng = np.random.default_rng(12)
    n = 60
    p = np.stack([rng.uniform(-10.0, 10.0, n), rng.uniform(-10.0, 10.0, n), rng.uniform(1.0, 19.0, n)], 1)
    p = p[np.abs(p[:, 2] - 10.0) > 0.5]
    h = 1e-5
    for name, L in Ls.items():
        d = 3 if L.type in (oracle.XYZ, oracle.AXIAL_Z, oracle.SLICED) else 2
        sx = L.sensor_xy
        q = p[np.all(np.hypot(p[:, None, 0] - sx[None, :, 0], p[:, None, 1] - sx[None, :, 1]) > 0.5, axis=1), :d]
        g = oracle.lrf_grad(L, q, mutant)
        scale = np.abs(oracle.lrf_eval(L, q, mutant)).max()
        for k in range(d):
            e = np.zeros(d)
            e[k] = h
            fd = (oracle.lrf_eval(L, q + e, mutant) - oracle.lrf_eval(L, q - e, mutant)) / (2 * h)
            err = np.abs(g[:, :, k] - fd).max()
            assert err < 1e-7 * scale, (name, k, err, scale)
        if d == 2:
            assert np.all(g[:, :, 2] == 0.0)


def _min_value(L, crit, s, p):
    """The match at p from plain LRF values (all sensors): F = sum s ln eta -
    S ln H, or minus Pearson's chi^2 with E = S / H."""
    eta = oracle.lrf_eval(L, p[None, :L_dim(L)])[0]
    S, H = s.sum(), eta.sum()
    if crit == 0:
        return float((s * np.log(eta)).sum() - S * np.log(H))
    mu = S / H * eta
    return float(-((s - mu) ** 2 / mu).sum())


def L_dim(L):
    return 3 if L.type in (oracle.XYZ, oracle.AXIAL_Z, oracle.SLICED) else 2


def pin_minimize_noise_free(mutant=0):
    """Noise-free signals s = E0 eta(p0) are matched exactly at p0 (Gibbs'
    inequality for maximum likelihood, a zero chi^2 for least squares): the
    minimisation from a start 1.8-2.7 mm away ends at p0 for every LRF type
    and both criteria, and E = E0."""
    sxy, Ls = _all_type_lrfs(mutant)
    M = oracle.Minimize(max_iter=100, tol=1e-10, lambda0=1e-3)
    for name, L in Ls.items():
        d = L_dim(L)
        p0 = np.array([[1.5, -2.0, 11.0]])[:, :d]
        s = 3000.0 * oracle.lrf_eval(L, p0, mutant)
        start = np.array([[0.0, -1.0, 13.0]]) if d == 3 else np.array([[0.0, -1.0, 0.0]])
        for crit in (0, 1):
            r = oracle.minimize(L, s, oracle.Variant(criterion=crit), M, start_xyz=start, mutant=mutant)
            assert r["status"][0] == 0 and r["n_iter"][0] > 0, (name, crit, r["n_iter"])
            err = np.abs(r["xyz"][0, :d] - p0[0]).max()
            assert err < 1e-7, (name, crit, err, r["xyz"][0], r["n_iter"])
            assert abs(r["E"][0] / 3000.0 - 1.0) < 1e-8, (name, crit, r["E"][0])


def pin_minimize_stationary(mutant=0):
    """On Poisson events the result is a local optimum of the match as
    computed from plain LRF values: no probe 0.01 mm away along any axis
    (inside the domain) is better, for the events that converged (at least
    90 %; an optimum beyond the domain's edge is approached step by step;
    sliced results on a plane, where the match has a kink, are left out),
    and it is at least as good as the contracting grids' result it started
    from (their last spacing is 0.0625 mm)."""
    sxy, Ls = _all_type_lrfs(mutant)
    rng = np.random.default_rng(21)
    M = oracle.Minimize(max_iter=200, tol=1e-6)
    for name in ("xy", "radial", "xyz", "sliced"):
        L = Ls[name]
        d = L_dim(L)
        n = 12
        p0 = np.stack([rng.uniform(-6, 6, n), rng.uniform(-6, 6, n), rng.uniform(6, 14, n)], 1)[:, :d]
        sig = rng.poisson(5000.0 * oracle.lrf_eval(L, p0, mutant)).astype(np.float64)
        P = oracle.CgsParams(n_xy=9, iters=7, step_xy=4.0, n_z=5 if d == 3 else 1, step_z=4.0 if d == 3 else 0.0,
                             z0=10.0)
        cg = oracle.cgs(L, P, sig, mutant=mutant)
        for crit in (0, 1):
            start = cg["xyz"] if crit == 0 else None
            r = oracle.minimize(L, sig, oracle.Variant(criterion=crit), M, z0=10.0, start_xyz=start, mutant=mutant)
            assert np.all(r["status"] == 0)
            assert (r["n_iter"] > 0).mean() >= 0.9, (name, crit, r["n_iter"])
            for e in np.nonzero(r["n_iter"] > 0)[0]:
                p = r["xyz"][e]
                if name == "sliced" and np.abs(p[2] - np.array([0.0, 10.0, 20.0])).min() < 0.05:
                    continue  # on a plane the match has a kink along z: a gradient method stops at its edge
                C0 = _min_value(L, crit, sig[e], p)
                for k in range(d):
                    for sgn in (-1.0, 1.0):
                        q = p.copy()
                        q[k] += sgn * 0.01
                        Cq = _min_value(L, crit, sig[e], q)  # NaN outside the domain: no probe
                        assert not (Cq > C0 + 1e-9), (name, crit, e, k, Cq - C0)
                if crit == 0:
                    assert C0 >= _min_value(L, 0, sig[e], cg["xyz"][e]) - 1e-9, (name, e)


def pin_minimize_status(mutant=0):
    """Status as for the search variants (bad or zero signals, a start
    outside the domain) with NaN outputs; n_iter < 0 when max_iter runs out."""
    sxy, Ls = _all_type_lrfs(mutant)
    L = Ls["xy"]
    s = 3000.0 * oracle.lrf_eval(L, np.array([[1.0, 1.0], [0.0, 0.0], [0.0, 0.0], [2.0, 2.0]]), mutant)
    s[1] = 0.0
    s[2, 1] = -1.0
    start = np.array([[-5.0, -5.0, 0.0], [0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [40.0, 0.0, 0.0]])
    r = oracle.minimize(L, s, oracle.Variant(), oracle.Minimize(max_iter=1), start_xyz=start, mutant=mutant)
    assert list(r["status"]) == [0, 2, 3, 4]
    assert r["n_iter"][0] == -1 and np.all(np.isnan(r["xyz"][1:]))


ALL_PINS += [pin_lrf_grad, pin_minimize_noise_free, pin_minimize_stationary, pin_minimize_status]


# --------------------------------------------------------------------------
# Optical photon transport (Sec. 4.2.3, 4.2.4, 4.2.6, 3.5)
# --------------------------------------------------------------------------


def _corner_solid_angle(x, y, d):
    """Solid angle of the rectangle [0, x] x [0, y] seen from height d above
    its corner (x, y >= 0)."""
    return np.arctan(x * y / (d * np.sqrt(x * x + y * y + d * d)))


def _rect_solid_angle(x0, x1, y0, y1, d):
    """Solid angle of [x0, x1] x [y0, y1] seen from (0, 0, d): signed sums of
    corner rectangles."""
    def c(x, y):
        return np.sign(x) * np.sign(y) * _corner_solid_angle(abs(x), abs(y), d)
    return c(x1, y1) - c(x0, y1) - c(x1, y0) + c(x0, y0)


def _bare_optics(**kw):
    """One vacuum-like layer (n = 1 everywhere, no reflection) over a 2 x 2
    array of 6 mm windows, pitch 8 mm, QE 1."""
    sxy = np.array([[-4.0, -4.0], [4.0, -4.0], [-4.0, 4.0], [4.0, 4.0]])
    args = dict(z=(0.0, 30.0), n=(1.0,), abs_len=(0.0,), ray_len=(0.0,), sensor_xy=sxy, sensor_size=6.0,
                qe=np.ones(4), n_sensor=1.0)
    args.update(kw)
    return oracle.Optics(**args)


def _binomial_ok(k, n, p, sig=5.0):
    return abs(k - n * p) <= sig * np.sqrt(n * p * (1 - p)) + 1.0


def pin_optics_solid_angle(mutant=0):
    """Without refraction, reflection or attenuation a window detects the
    fraction Omega / 4 pi of the photons, Omega the closed-form solid angle of
    the rectangle (sums of corner terms arctan(x y / (d sqrt(x^2 + y^2 +
    d^2)))); within 5 binomial sigmas for two source positions."""
    O = _bare_optics()
    n = 200_000
    for src in ((1.5, -0.5, 7.0), (-6.0, 3.0, 12.0)):
        c = oracle.trace_photons(O, [src], n, seed=11, mutant=mutant)[0]
        for i, (sx, sy) in enumerate(O.sensor_xy):
            om = _rect_solid_angle(sx - 3.0 - src[0], sx + 3.0 - src[0], sy - 3.0 - src[1], sy + 3.0 - src[1],
                                   src[2])
            assert _binomial_ok(c[i], n, om / (4 * np.pi)), (src, i, c[i], n * om / (4 * np.pi))


def pin_optics_absorption(mutant=0):
    """With an absorption length L the detected fraction is (1 / 4 pi) times
    the integral over the window of d exp(-r / L) / r^3 (midpoint rule on a
    400 x 400 grid); within 5 binomial sigmas."""
    L = 15.0
    O = _bare_optics(abs_len=(L,))
    n = 200_000
    src = (2.0, 1.0, 10.0)
    c = oracle.trace_photons(O, [src], n, seed=12, mutant=mutant)[0]
    m = 400
    for i, (sx, sy) in enumerate(O.sensor_xy):
        u = (np.arange(m) + 0.5) / m * 6.0 - 3.0
        X, Y = np.meshgrid(sx + u - src[0], sy + u - src[1])
        r = np.sqrt(X ** 2 + Y ** 2 + src[2] ** 2)
        frac = (src[2] * np.exp(-r / L) / r ** 3).sum() * (6.0 / m) ** 2 / (4 * np.pi)
        assert _binomial_ok(c[i], n, frac), (i, c[i], n * frac)
    # every photon ends in exactly one class
    _, o = oracle.trace_photons(O, [src], 5000, seed=12, want_outcome=True, mutant=mutant)
    assert np.all((o >= -2) & (o < 4))


def pin_fresnel(mutant=0):
    """The unpolarised Fresnel coefficient: ((n1 - n2) / (n1 + n2))^2 at normal
    incidence, 0 between equal media, 1 beyond the critical angle, half the s
    term sin^2(ti - tt) at Brewster's angle (p term 0), the same for the
    reversed ray (n2 into n1 at the refracted angle), 1 at grazing incidence."""
    f = lambda a, b, c: oracle.fresnel(a, b, c, mutant)
    for n1, n2 in ((1.0, 1.5), (1.5, 1.0), (1.33, 1.8)):
        assert abs(f(n1, n2, 1.0) - ((n1 - n2) / (n1 + n2)) ** 2) < 1e-15
        assert abs(f(n1, n1, 0.3)) < 1e-15
        tb = np.arctan(n2 / n1)
        tt = np.arcsin(n1 / n2 * np.sin(tb))
        assert abs(f(n1, n2, np.cos(tb)) - 0.5 * np.sin(tb - tt) ** 2) < 1e-12
        for ti in (0.2, 0.5, 0.7):
            st = n1 / n2 * np.sin(ti)
            if st < 1:
                assert abs(f(n1, n2, np.cos(ti)) - f(n2, n1, np.sqrt(1 - st * st))) < 1e-12
        assert abs(f(n1, n2, 1e-9) - 1.0) < 1e-6
    assert f(1.5, 1.0, np.cos(0.75)) == 1.0  # beyond asin(1 / 1.5) = 0.7297


def pin_rayleigh_and_turn(mutant=0):
    """The Rayleigh sampler inverts the CDF (mu^3 + 3 mu + 4) / 8 and has the
    moments E[mu] = 0, E[mu^2] = 2/5 (midpoint grid of 20001 u values); a
    turned direction is a unit vector at cosine mu from the old one."""
    u = (np.arange(20001) + 0.5) / 20001
    mu = np.array([oracle.rayleigh_mu(x, mutant) for x in u])
    assert np.abs((mu ** 3 + 3 * mu + 4) / 8 - u).max() < 1e-12
    assert abs(mu.mean()) < 1e-6 and abs((mu ** 2).mean() - 0.4) < 1e-6
    rng = np.random.default_rng(3)
    for _ in range(50):
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        m, ph = rng.uniform(-1, 1), rng.uniform(0, 2 * np.pi)
        t = oracle.turn_dir(d, m, ph, mutant)
        assert abs(np.linalg.norm(t) - 1) < 1e-12 and abs(t @ d - m) < 1e-12
    t = oracle.turn_dir(np.array([0.0, 0.0, 1.0]), 0.3, 0.0, mutant)
    assert abs(t[2] - 0.3) < 1e-12


def pin_optics_fresnel_mc(mutant=0):
    """A source in a layer of index 1.5 over one window of index 1 that
    covers the whole floor, an absorbing ceiling: photons going down enter
    the window with probability 1 - R(mu) (none beyond the critical angle),
    reflected ones are absorbed above, so the detected fraction is (1/2)
    int_0^1 (1 - R(mu)) d mu (Simpson, 4001 points); within 5 sigmas."""
    O = oracle.Optics(z=(0.0, 10.0), n=(1.5,), abs_len=(0.0,), ray_len=(0.0,), sensor_xy=np.array([[0.0, 0.0]]),
                      sensor_size=1e7, qe=np.ones(1), n_sensor=1.0, p_abs=(0.0, 1.0))
    n = 200_000
    c = oracle.trace_photons(O, [(0.0, 0.0, 5.0)], n, seed=13, mutant=mutant)[0, 0]
    mu = np.linspace(0.0, 1.0, 4001)
    T = np.array([1.0 - oracle.fresnel(1.5, 1.0, m) for m in mu])
    w = np.ones(4001)
    w[1:-1:2], w[2:-1:2] = 4, 2
    frac = 0.5 * (w * T).sum() / (3 * 4000)
    assert _binomial_ok(c, n, frac), (c, n * frac)


def pin_optics_diffuse_and_prereject(mutant=0):
    """A Lambertian ceiling that reflects half of the photons and absorbs the
    rest over a floor-wide window (n = 1 everywhere): 3/4 are detected. With
    QE 0.25 the pre-rejection mode detects as many as plain tracing (5
    sigmas), and rejects 3/4 of the photons before tracing."""
    sxy = np.array([[0.0, 0.0]])
    O = oracle.Optics(z=(0.0, 10.0), n=(1.0,), abs_len=(0.0,), ray_len=(0.0,), sensor_xy=sxy, sensor_size=1e7,
                      qe=np.ones(1), n_sensor=1.0, p_abs=(0.0, 0.5), p_diff=(0.0, 0.5))
    n = 100_000
    c = oracle.trace_photons(O, [(0.0, 0.0, 5.0)], n, seed=14, mutant=mutant)[0, 0]
    assert _binomial_ok(c, n, 0.75), c
    O2 = _bare_optics(qe=np.full(4, 0.25))
    O3 = _bare_optics(qe=np.full(4, 0.25), pre_reject=1)
    src = [(1.0, 2.0, 6.0)]
    a = oracle.trace_photons(O2, src, n, seed=15, mutant=mutant)[0].sum()
    b, o = oracle.trace_photons(O3, src, n, seed=16, want_outcome=True, mutant=mutant)
    p = a / n
    assert abs(b[0].sum() - a) <= 5 * np.sqrt(2 * n * p * (1 - p)), (a, b[0].sum())
    assert _binomial_ok((o == oracle.PH_REJECTED).sum(), n, 0.75)


ALL_PINS += [pin_optics_solid_angle, pin_optics_absorption, pin_fresnel, pin_rayleigh_and_turn, pin_optics_fresnel_mc,
             pin_optics_diffuse_and_prereject]


# --------------------------------------------------------------------------
# Sensor groups (Sec. 6.2)
# --------------------------------------------------------------------------


def pin_sensor_groups(mutant=0):
    """A grouped radial LRF evaluates sensor i with its group's profile times
    its gain: equal to the per-sensor LRF whose rows are the groups' rows,
    to the shared LRF when there is one group. Grouping by distance from
    the centre: the 19-PMT hexagon has rings of 1, 6, 6 and 6 sensors at 0,
    p, sqrt(3) p and 2 p; an 8 x 8 square array has one group per distinct
    distance |(a, b)|, a, b in {3, 9, 15, 21} mm, whose sizes count the
    sensors at that distance."""
    w = synth.workloads.get("hex19_radial")
    g, k = oracle.sensor_rings(w.sensor_xy, 1.0, mutant)
    assert k == 4 and list(np.bincount(g)) == [1, 6, 6, 6], (k, np.bincount(g))
    d = np.hypot(*(w.sensor_xy - w.sensor_xy.mean(0)).T)
    for j, r in enumerate((0.0, 30.0, 30.0 * np.sqrt(3.0), 60.0)):
        assert np.allclose(d[g == j], r, atol=1e-9)
    sq = synth.square_array(8, 6.0)
    g8, k8 = oracle.sensor_rings(sq, 0.01, mutant)
    a = np.array([3.0, 9.0, 15.0, 21.0])
    dist = sorted({round(float(np.hypot(x, y)), 6) for x in a for y in a})
    assert k8 == len(dist)
    dd = np.hypot(*(sq - sq.mean(0)).T)
    for j, r in enumerate(dist):
        assert np.all(np.abs(dd[g8 == j] - r) < 1e-6)
    # evaluation with groups
    rng = np.random.default_rng(8)
    prof = 0.04 / (1 + (np.linspace(-7.5, 157.5, 23) / 40.0) ** 2) ** 1.5
    rows = prof[None, :] * rng.uniform(0.9, 1.1, (k, 23))
    gains = rng.uniform(0.9, 1.1, 19)
    G = oracle.Lrf(oracle.RADIAL, w.sensor_xy, (20, 0, 0), (0.0, 0.0, 0.0), (150.0, 0.0, 0.0), rows, gain=gains,
                   group=g)
    P = oracle.Lrf(oracle.RADIAL, w.sensor_xy, (20, 0, 0), (0.0, 0.0, 0.0), (150.0, 0.0, 0.0), rows[g], gain=gains)
    pts = rng.uniform(-50.0, 50.0, (200, 2))
    assert np.array_equal(oracle.lrf_eval(G, pts, mutant), oracle.lrf_eval(P, pts, mutant))
    one = oracle.Lrf(oracle.RADIAL, w.sensor_xy, (20, 0, 0), (0.0, 0.0, 0.0), (150.0, 0.0, 0.0), rows[:1],
                     gain=gains, group=np.zeros(19, dtype=np.int32))
    sh = oracle.Lrf(oracle.RADIAL, w.sensor_xy, (20, 0, 0), (0.0, 0.0, 0.0), (150.0, 0.0, 0.0), rows[:1],
                    gain=gains, shared=True)
    assert np.array_equal(oracle.lrf_eval(one, pts, mutant), oracle.lrf_eval(sh, pts, mutant))


ALL_PINS += [pin_sensor_groups]


def pin_grouped_refit_exact(mutant=0):
    """Noise-free signals E g_i f_{group(i)}(r) of the hexagon's four rings:
    the grouped refit recovers each ring's profile where it is sampled, and
    with the gain refit the planted gains scaled to mean 1 within each ring
    (the ring's profile taking the mean), eta = g f unchanged."""
    rng = np.random.default_rng(14)
    w = synth.workloads.get("hex19_radial")
    g, k = oracle.sensor_rings(w.sensor_xy, 1.0, mutant)
    pts, vals = w.fit_samples()
    base, _, _ = oracle.lrf_fit(w.n_int, w.lo, w.hi, pts, vals, mutant=mutant)
    rows = base[0][None, :] * rng.uniform(0.8, 1.2, (k, 1))
    gains = rng.uniform(0.85, 1.15, 19)
    Lt = oracle.Lrf(oracle.RADIAL, w.sensor_xy, w.n_int + (0, 0), w.lo + (0, 0), w.hi + (0, 0), rows, gain=gains,
                    group=g)
    xy = rng.uniform(-60, 60, (3000, 2))
    xyz = np.concatenate([xy, np.zeros((3000, 1))], axis=1)
    E = rng.uniform(5000, 15000, 3000)
    s = E[:, None] * np.nan_to_num(oracle.lrf_eval(Lt, xy, mutant))
    # each ring's profile is compared where its sensors have samples (the
    # unsampled tail is set by the ridge fallback)
    dist = np.hypot(xy[:, None, 0] - w.sensor_xy[None, :, 0], xy[:, None, 1] - w.sensor_xy[None, :, 1])
    reach = [0.95 * dist[:, g == j].max() for j in range(k)]
    prof = lambda c, j: oracle.spline_eval(w.n_int, w.lo, w.hi, c, np.linspace(0.0, reach[j], 60)[:, None], mutant)
    R = oracle.lrf_refit(Lt, s, xyz, E, mutant=mutant)
    for j in range(k):
        # 1e-6: the innermost ring is one sensor with few samples near r = 0
        assert np.abs(prof(R.coef[j], j) - prof(rows[j], j)).max() < 1e-6 * prof(rows[j], j).max(), j
    # from unit gains: the gain refit recovers the planted ones up to each ring's scale
    L1 = oracle.Lrf(oracle.RADIAL, w.sensor_xy, w.n_int + (0, 0), w.lo + (0, 0), w.hi + (0, 0), rows, gain=gains,
                    group=g)
    R2 = oracle.lrf_refit(L1, s, xyz, E, refit_gains=True, mutant=mutant)
    for j in range(k):
        m = g == j
        want = gains[m] / gains[m].mean()
        assert np.abs(R2.gain[m] - want).max() < 1e-7, j
        want_p = prof(rows[j], j) * gains[m].mean()
        assert np.abs(prof(R2.coef[j], j) - want_p).max() < 1e-6 * want_p.max(), j


ALL_PINS += [pin_grouped_refit_exact]


def pin_symmetry_groups(mutant=0):
    """Sec. 6.2 classes by the array's symmetry: the 8 x 8 square has the 8
    operations of the square's group and 10 classes (4 of 4 sensors on the
    diagonals, 6 of 8); the 19-PMT hexagon 4 classes (1, 6, 6, 6); a 4 x 2
    rectangle 2 classes of 4. A class LRF evaluated at the mapped point
    M^T (p - c) + c equals, on a knot grid symmetric about the centre, the
    per-sensor LRF whose coefficient grid is the class's with its indices
    transformed by M (B_j(-x) = B_{N-j}(x) on symmetric knots), and its
    analytic gradient equals central differences."""
    sq = synth.square_array(8, 6.0)
    g, op, k, c = oracle.sensor_symmetry(sq, 1e-6, mutant)
    assert k == 10 and sorted(np.bincount(g)) == [4] * 4 + [8] * 6
    assert sorted(set(op.tolist())) == [0, 3, 6, 9, 12, 15, 18, 21]
    gh, _, kh, _ = oracle.sensor_symmetry(synth.workloads.get("hex19_radial").sensor_xy, 1e-6, mutant)
    assert kh == 4 and sorted(np.bincount(gh)) == [1, 6, 6, 6]
    rect = np.array([[x, y] for y in (-2.0, 2.0) for x in (-6.0, -2.0, 2.0, 6.0)])
    gr, _, kr, _ = oracle.sensor_symmetry(rect, 1e-6, mutant)
    assert kr == 2 and list(np.bincount(gr)) == [4, 4]
    # class LRFs with random coefficients on a symmetric 6 x 6 grid over [-24, 24]^2
    rng = np.random.default_rng(30)
    n = 6
    N = n + 2
    cls = rng.uniform(0.5, 1.5, (k, (n + 3) * (n + 3)))
    gains = rng.uniform(0.9, 1.1, 64)
    G = oracle.Lrf(oracle.XY, sq, (n, n, 0), (-24.0, -24.0, 0.0), (24.0, 24.0, 0.0), cls, gain=gains, group=g, op=op,
                   sym_c=c)
    per = np.empty((64, (n + 3) * (n + 3)))
    for i in range(64):
        M = np.rint(oracle.sym_matrix(int(op[i]))).astype(int)
        F = cls[g[i]].reshape(n + 3, n + 3)  # [jy][jx]
        P = np.empty_like(F)
        for jy in range(n + 3):
            for jx in range(n + 3):
                u = np.array([2 * jx - N, 2 * jy - N])  # twice the centred index
                w = M.T @ u
                P[jy, jx] = F[(w[1] + N) // 2, (w[0] + N) // 2]
        per[i] = P.ravel() * gains[i]
    Lp = oracle.Lrf(oracle.XY, sq, (n, n, 0), (-24.0, -24.0, 0.0), (24.0, 24.0, 0.0), per)
    pts = rng.uniform(-23.0, 23.0, (300, 2))
    a, b = oracle.lrf_eval(G, pts, mutant), oracle.lrf_eval(Lp, pts, mutant)
    assert np.abs(a - b).max() < 1e-12 * np.abs(b).max()
    gr_ = oracle.lrf_grad(G, pts, mutant)
    h = 1e-5
    for kk in range(2):
        e = np.zeros(2)
        e[kk] = h
        fd = (oracle.lrf_eval(G, pts + e, mutant) - oracle.lrf_eval(G, pts - e, mutant)) / (2 * h)
        assert np.abs(gr_[:, :, kk] - fd).max() < 1e-7 * np.abs(a).max()


ALL_PINS += [pin_symmetry_groups]


def pin_symmetric_fit_exact(mutant=0):
    """Noise-free samples of a symmetry-class XY LRF set on the 8 x 8 array
    (random class coefficients, gains): the class fit from the members'
    mapped samples recovers every class's coefficients."""
    sq = synth.square_array(8, 6.0)
    g, op, k, c = oracle.sensor_symmetry(sq, 1e-6, mutant)
    rng = np.random.default_rng(31)
    n = 6
    cls = rng.uniform(0.5, 1.5, (k, (n + 3) * (n + 3)))
    gains = rng.uniform(0.9, 1.1, 64)
    G = oracle.Lrf(oracle.XY, sq, (n, n, 0), (-24.0, -24.0, 0.0), (24.0, 24.0, 0.0), cls, gain=gains, group=g, op=op,
                   sym_c=c)
    pts = rng.uniform(-24.0, 24.0, (1500, 2))
    vals = oracle.lrf_eval(G, pts, mutant)
    F = oracle.lrf_fit_symmetric(sq, g, op, c, (n, n), (-24.0, -24.0), (24.0, 24.0), pts, vals, gain=gains,
                                 mutant=mutant)
    assert np.abs(F.coef - cls).max() < 1e-8 * np.abs(cls).max()


ALL_PINS += [pin_symmetric_fit_exact]
