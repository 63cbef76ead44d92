"""Shared helpers of the GPU parity tests: build the same LRF for the oracle
and for libants, run both, and compare with the tie-certification rule.

The LRF coefficients come from the oracle's FP64 fit (an input to both
sides); the library's own fit is compared with the oracle's separately."""
from __future__ import annotations

import numpy as np

import oracle
import synth.workloads

TYPES = {"radial": oracle.RADIAL, "xy": oracle.XY, "xyz": oracle.XYZ}


def oracle_lrf(w, coef=None):
    dims = {"radial": 1, "xy": 2, "xyz": 3}[w.lrf_type]
    if coef is None:
        pts, vals = w.fit_samples()
        coef, _, _ = oracle.lrf_fit(w.n_int, w.lo, w.hi, pts, vals)
    pad = lambda t, v: tuple(list(t[:dims]) + [v] * (3 - dims))
    return oracle.Lrf(TYPES[w.lrf_type], w.sensor_xy, pad(w.n_int, 0), pad(w.lo, 0.0), pad(w.hi, 0.0), coef,
                      shared=w.shared)


def oracle_params(w):
    return oracle.CgsParams(n_xy=w.n_xy, iters=w.iters, step_xy=w.step_xy, shrink=w.shrink, n_z=w.n_z,
                            step_z=w.step_z, z0=w.z0)


def gpu_objects(w, L_or, ctx=None):
    import paper_1602_07247_gb300 as ants
    ctx = ctx or ants.Context(0)
    det = ants.Detector(w.sensor_xy, w.gains)
    lrf = ants.Lrf.from_coefficients(ctx, det, L_or.type, w.n_int, w.lo, w.hi, L_or.coef, shared=w.shared)
    p = ants.CgsParams(n_xy=w.n_xy, iters=w.iters, step_xy=w.step_xy, shrink=w.shrink, n_z=w.n_z,
                       step_z=w.step_z, z0=w.z0)
    return ctx, det, lrf, p


def compare(w, L_or, sig, gpu, start=None, tol_xy=1e-3, tol_logl=1e-5, tol_E=1e-5):
    """Check a GPU result (numpy dict with xyz, E, logL, status, trace) against
    the oracle.  Returns a dict of statistics; raises AssertionError."""
    P = oracle_params(w)
    sig64 = np.asarray(sig, dtype=np.float64)
    trace = np.asarray(gpu["trace"], dtype=np.int32)
    rp = oracle.cgs_replay(L_or, P, sig64, trace, gain_cog=w.gains, start_xyz=start)
    own = oracle.cgs(L_or, P, sig64, gain_cog=w.gains, start_xyz=start)
    assert np.array_equal(gpu["status"], own["status"]), "event status differs"
    ok = own["status"] == 0
    assert np.all(rp["n_bad"][ok] == 0), f"{int((rp['n_bad'][ok] > 0).sum())} events chose a node outside tau"
    dxy = np.abs(gpu["xyz"][ok] - rp["xyz"][ok]).max(initial=0.0)
    assert dxy <= tol_xy, f"max |dxyz| {dxy}"
    rel_l = np.abs(gpu["logL"][ok] / rp["logL"][ok] - 1.0).max(initial=0.0)
    assert rel_l <= tol_logl, f"max rel dlogL {rel_l}"
    rel_e = np.abs(gpu["E"][ok] / rp["E"][ok] - 1.0).max(initial=0.0)
    assert rel_e <= tol_E, f"max rel dE {rel_e}"
    tie = rp["n_tie"][ok] > 0
    same = np.all(trace[ok] == own["trace"][ok], axis=1)
    # events without a certified tie followed exactly the oracle's own path
    assert np.all(same[~tie]), "an event without ties left the oracle's path"
    d_own = np.abs(gpu["xyz"][ok][~tie] - own["xyz"][ok][~tie]).max(initial=0.0)
    assert d_own <= tol_xy
    assert np.all(np.isnan(gpu["xyz"][~ok])) and np.all(np.isnan(gpu["E"][~ok]))
    return dict(n=int(ok.sum()), tie_frac=float(tie.mean()) if tie.size else 0.0, max_dxy=float(dxy),
                max_rel_logl=float(rel_l), max_rel_E=float(rel_e))


def to_numpy(res):
    return dict(xyz=res.xyz.cpu().numpy().astype(np.float64), E=res.E.cpu().numpy().astype(np.float64),
                logL=res.logL.cpu().numpy().astype(np.float64), status=res.status.cpu().numpy(),
                trace=None if res.trace is None else res.trace.cpu().numpy())
