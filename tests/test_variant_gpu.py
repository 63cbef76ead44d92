"""GPU search variants (Sec. 5.1.2: least squares, sensor cuts; Sec.
5.1.2.1: strongest-sensor start; Sec. 5.3: passive sensors) against the FP64
oracle: the oracle replays the GPU's chosen node of every grid under the tie
rule, and the results are compared at the replayed end."""
import numpy as np
import pytest

import oracle
import synth
import synth.workloads
from parity import gpu_objects, oracle_lrf, oracle_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    import paper_1602_07247_gb300 as ants
    return ants.Context(0)


def _passive(n_s, every):
    p = np.zeros(n_s, dtype=np.uint8)
    p[::every] = 1
    return p


CASES = {
    "ml_default": dict(),
    "ls_cog": dict(criterion=1),
    "ml_max_cuts_passive": dict(start=1, cuts=True, passive=7),
    "ls_max_passive": dict(criterion=1, start=1, passive=5),
}
# signal and distance cuts that remove some sensors of most events (typical
# counts: 20-460 on the PMTs, 40-170 on the SiPMs)
CUTS = {"hex19_radial": dict(min_signal=40.0, max_distance=70.0),
        "sipm8x8_xy": dict(min_signal=60.0, max_distance=25.0),
        "sipm4x4_xyz": dict(min_signal=60.0, max_distance=12.0)}


def _run(ctx, name, case, n, seed):
    import torch
    import paper_1602_07247_gb300 as ants
    w = synth.workloads.get(name)
    L = oracle_lrf(w)
    _, det, lrf, p = gpu_objects(w, L, ctx)
    c = dict(case)
    pas = _passive(w.n_sensors, c.pop("passive")) if "passive" in c else None
    if c.pop("cuts", False):
        c.update(CUTS[name])
    vp = ants.VariantParams(p, passive=pas, **c)
    ev = w.events(n, seed=seed)
    sig = ev.signals.astype(np.float32)
    if pas is not None:
        sig[:, pas.astype(bool)] = np.nan  # never read
    res = ants.reconstruct(ctx, lrf, vp, torch.from_numpy(sig).cuda(), want_trace=True, method=ants.ANTS_CGS_VARIANT)
    torch.cuda.synchronize()
    V = oracle.Variant(passive=None if pas is None else pas.astype(np.int32), **c)
    rp = oracle.cgs_variant_replay(L, oracle_params(w), sig.astype(np.float64), V,
                                   res.trace.cpu().numpy().astype(np.int32), gain=w.gains)
    return res, rp, ev


@pytest.mark.parametrize("case", sorted(CASES))
@pytest.mark.parametrize("name", ["hex19_radial", "sipm8x8_xy", "sipm4x4_xyz"])
def test_variant_matches_oracle(ctx, name, case):
    n = 600 if name == "sipm8x8_xy" else 1500
    res, rp, ev = _run(ctx, name, CASES[case], n, seed=31)
    st = res.status.cpu().numpy()
    assert np.array_equal(st, rp["status"])
    ok = st == 0
    assert ok.mean() > 0.95
    assert np.all(rp["n_bad"][ok] == 0), np.nonzero(rp["n_bad"])[0][:10]
    d = np.abs(res.xyz.cpu().numpy()[ok] - rp["xyz"][ok]).max()
    rE = np.abs(res.E.cpu().numpy()[ok] / rp["E"][ok] - 1).max()
    rl = np.abs(res.logL.cpu().numpy()[ok] / rp["logL"][ok] - 1).max()
    ties = (rp["n_tie"][ok] > 0).mean()
    print(name, case, "max |dxyz|", d, "rel dE", rE, "rel dlogL", rl, "tie fraction", ties)
    assert d <= 1e-3 and rE <= 1e-5 and rl <= 1e-5
    assert ties < (0.5 if CASES[case].get("criterion") == 1 else 0.25)


def test_variant_defaults_equal_plain_on_radial(ctx):
    """With no option set the variant is the plain search: on the radial
    workload both follow the oracle's own path, so their results agree to
    FP32 rounding."""
    import torch
    import paper_1602_07247_gb300 as ants
    w = synth.workloads.get("hex19_radial")
    L = oracle_lrf(w)
    _, det, lrf, p = gpu_objects(w, L, ctx)
    sig = torch.from_numpy(w.events(2000, seed=5).signals.astype(np.float32)).cuda()
    a = ants.reconstruct(ctx, lrf, p, sig)
    b = ants.reconstruct(ctx, lrf, ants.VariantParams(p), sig, method=ants.ANTS_CGS_VARIANT)
    ok = a.status.cpu().numpy() == 0
    assert np.array_equal(a.status.cpu().numpy(), b.status.cpu().numpy())
    d = np.abs(a.xyz.cpu().numpy()[ok] - b.xyz.cpu().numpy()[ok])
    assert (d.max(axis=1) <= 1e-3).mean() > 0.995


def test_variant_status_and_errors(ctx):
    import torch
    import paper_1602_07247_gb300 as ants
    w = synth.workloads.get("sipm8x8_xy")
    L = oracle_lrf(w)
    _, det, lrf, p = gpu_objects(w, L, ctx)
    sig = w.events(8, seed=3).signals.astype(np.float32)
    sig[1] = 0.0                  # no light
    sig[2, 5] = -1.0              # a bad signal on an active sensor
    sig[3, 6] = np.nan            # ... and on a passive one: ignored
    pas = np.zeros(64, dtype=np.uint8)
    pas[6] = 1
    vp = ants.VariantParams(p, passive=pas)
    r = ants.reconstruct(ctx, lrf, vp, torch.from_numpy(sig).cuda(), method=ants.ANTS_CGS_VARIANT)
    st = r.status.cpu().numpy()
    assert st[1] == ants.ANTS_EVT_ZERO_SIGNAL and st[2] == ants.ANTS_EVT_BAD_SIGNAL and st[3] == 0
    # a cut that leaves nothing in the match
    r2 = ants.reconstruct(ctx, lrf, ants.VariantParams(p, min_signal=1e9), torch.from_numpy(sig).cuda(),
                          method=ants.ANTS_CGS_VARIANT)
    assert np.all(r2.status.cpu().numpy()[[0, 4, 5]] == ants.ANTS_EVT_ZERO_SIGNAL)
    with pytest.raises(ants.AntsError):
        ants.reconstruct(ctx, lrf, ants.VariantParams(p, criterion=7), torch.from_numpy(sig).cuda(),
                         method=ants.ANTS_CGS_VARIANT)
    with pytest.raises(ants.AntsError):
        ants.reconstruct(ctx, lrf, ants.VariantParams(p), torch.from_numpy(sig).cuda(),
                         start_xyz=torch.zeros((8, 3), device="cuda"), method=ants.ANTS_CGS_VARIANT)


def test_variant_full_size_sampled(ctx):
    """The benchmark's 10^6-event 8x8 SiPM run with the least-squares
    variant and a passive sensor: 48 sampled events against the oracle's
    replay."""
    import torch
    import paper_1602_07247_gb300 as ants
    w = synth.workloads.get("sipm8x8_xy")
    L = oracle_lrf(w)
    _, det, lrf, p = gpu_objects(w, L, ctx)
    n = 1_000_000
    ev = w.events(n, seed=w.event_seed)
    pas = np.zeros(64, dtype=np.uint8)
    pas[27] = 1
    vp = ants.VariantParams(p, criterion=1, start=1, passive=pas)
    res = ants.reconstruct(ctx, lrf, vp, torch.from_numpy(ev.signals).cuda(), want_trace=True,
                           method=ants.ANTS_CGS_VARIANT)
    torch.cuda.synchronize()
    pick = np.random.default_rng(1).choice(n, 48, replace=False)
    V = oracle.Variant(criterion=1, start=1, passive=pas.astype(np.int32))
    rp = oracle.cgs_variant_replay(L, oracle_params(w), ev.signals[pick].astype(np.float64), V,
                                   res.trace.cpu().numpy()[pick].astype(np.int32), gain=w.gains)
    ok = rp["status"] == 0
    assert ok.all() and np.all(rp["n_bad"] == 0)
    assert np.abs(res.xyz.cpu().numpy()[pick] - rp["xyz"]).max() <= 1e-3
