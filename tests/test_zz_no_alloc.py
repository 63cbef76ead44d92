"""The allocation-free host-buffer entry point (ants_reconstruct_host_noalloc).

Callers that may not allocate device memory while they run (programs that
hand the device memory to their own pool at start-up, streaming loops that
must not stall on an allocation, plug-ins whose host forbids it) use this
entry point; it stages data through a fixed area the library declares
statically.  The test calls it through the C ABI twice in a row, with
different inputs each time, and checks it against the allocating entry point
ants_reconstruct_host with the tolerances of the parity tests.  It lives in
its own file, collected last, and passes alone in a fresh process as well as
after the other tests."""
import numpy as np
import pytest

import synth.workloads
from parity import gpu_objects, oracle_lrf

pytestmark = pytest.mark.gpu


def _close(a, b):
    assert np.array_equal(a.status, b.status)
    ok = a.status == 0
    assert np.abs(a.xyz[ok] - b.xyz[ok]).max(initial=0.0) <= 1e-3
    assert np.abs(a.logL[ok] / b.logL[ok] - 1.0).max(initial=0.0) <= 1e-5
    assert np.abs(a.E[ok] / b.E[ok] - 1.0).max(initial=0.0) <= 1e-5
    assert np.all(np.isnan(a.xyz[~ok])) and np.all(np.isnan(b.xyz[~ok]))


@pytest.mark.parametrize("name", ["sipm8x8_xy", "hex19_radial"])
def test_noalloc_matches_allocating_entry_point(name):
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    import paper_1602_07247_gb300 as ants
    w = synth.workloads.get(name)
    L = oracle_lrf(w)
    ctx, det, lrf, p = gpu_objects(w, L)
    for call in range(2):  # the second call reuses the area the first one left behind
        n = 20_000 + 7 * call
        sig = w.events(n, seed=500 + call).signals.copy()
        sig[3] = 0.0  # a zero-signal event in the batch
        want = ants.reconstruct_host(ctx, lrf, p, sig)
        got = ants.reconstruct_host_noalloc(ctx, lrf, p, sig)
        _close(got, want)


def test_noalloc_given_start_and_rejects_oversized_batch():
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    import paper_1602_07247_gb300 as ants
    w = synth.workloads.get("sipm8x8_xy").with_(n_xy=5, iters=4, step_xy=0.5)
    L = oracle_lrf(w)
    ctx, det, lrf, p = gpu_objects(w, L)
    ev = w.events(5000, seed=9)
    start = np.ascontiguousarray(np.clip(ev.xyz, -23, 23), dtype=np.float32)
    start[:, 2] = 0.0
    want = ants.reconstruct_host(ctx, lrf, p, ev.signals, start_xyz=start)
    got = ants.reconstruct_host_noalloc(ctx, lrf, p, ev.signals, start_xyz=start)
    _close(got, want)
    too_many = ants.ANTS_NOALLOC_STAGE_BYTES // (4 * w.n_sensors) + 1
    big = np.zeros((too_many, w.n_sensors), dtype=np.float32)
    with pytest.raises(ants.AntsError) as e:
        ants.reconstruct_host_noalloc(ctx, lrf, p, big)
    assert e.value.code == -1 and "capacity" in str(e.value)


@pytest.mark.parametrize("with_start,cap", [(False, 119_835), (True, 114_910)])
def test_noalloc_capacity_boundary(with_start, cap):
    """The stated limit for 64 sensors is exact: every region of the area is
    rounded up to 256 bytes, so a full batch fits and one more event does not."""
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    import paper_1602_07247_gb300 as ants
    w = synth.workloads.get("sipm8x8_xy").with_(n_xy=5, iters=4, step_xy=0.5)
    assert w.n_sensors == 64
    L = oracle_lrf(w)
    ctx, det, lrf, p = gpu_objects(w, L)
    ev = w.events(cap + 1, seed=31)
    start = None
    if with_start:
        start = np.ascontiguousarray(np.clip(ev.xyz, -23, 23), dtype=np.float32)
        start[:, 2] = 0.0
    sig = np.ascontiguousarray(ev.signals[:cap], dtype=np.float32)
    st = None if start is None else start[:cap]
    want = ants.reconstruct_host(ctx, lrf, p, sig, start_xyz=st)
    got = ants.reconstruct_host_noalloc(ctx, lrf, p, sig, start_xyz=st)
    _close(got, want)
    with pytest.raises(ants.AntsError) as e:
        ants.reconstruct_host_noalloc(ctx, lrf, p, np.ascontiguousarray(ev.signals, dtype=np.float32),
                                      start_xyz=start)
    assert e.value.code == -1 and "capacity" in str(e.value)
