"""The allocation-free host-buffer entry point (ants_reconstruct_host_noalloc).

Callers that may not allocate device memory while they run (programs that
hand the device memory to their own pool at start-up, streaming loops that
must not stall on an allocation, plug-ins whose host forbids it) use this
entry point; it stages data through a fixed area the library declares
statically.  The tests call it through the C ABI twice in a row, with
different inputs each time, and check it against the allocating entry point
ants_reconstruct_host: both run the same search kernel on the same inputs,
so the results must be equal bit for bit.  A warm call must not change the
device's free memory, and a call with no events sets the area up (reserves
it) in a fresh process.  The file is collected last, and passes alone in a
fresh process as well as after the other tests."""
import os
import subprocess
import sys

import numpy as np
import pytest

import synth.workloads
from parity import gpu_objects, oracle_lrf

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _same(a, b):
    """Bitwise equality of two results (NaN outputs of failed events included)."""
    assert np.array_equal(a.status, b.status)
    for k in ("xyz", "E", "logL"):
        x, y = getattr(a, k), getattr(b, k)
        assert np.array_equal(x.view(np.uint32), y.view(np.uint32)), k
    bad = a.status != 0
    assert np.all(np.isnan(a.xyz[bad]))


@pytest.mark.parametrize("name", ["sipm8x8_xy", "hex19_radial"])
def test_noalloc_matches_allocating_entry_point(name):
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    import paper_1602_07247_gb300 as ants
    w = synth.workloads.get(name)
    L = oracle_lrf(w)
    ctx, det, lrf, p = gpu_objects(w, L)
    free = []
    for call in range(2):  # the second call reuses the area the first one left behind
        n = 20_000 + 7 * call
        sig = w.events(n, seed=500 + call).signals.copy()
        sig[3] = 0.0  # a zero-signal event in the batch
        want = ants.reconstruct_host(ctx, lrf, p, sig)
        torch.cuda.synchronize()
        free.append(torch.cuda.mem_get_info()[0])
        got = ants.reconstruct_host_noalloc(ctx, lrf, p, sig)
        free.append(torch.cuda.mem_get_info()[0])
        _same(got, want)
    # the warm (second) call leaves the device's free memory as it was
    assert free[3] == free[2], free


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
    _same(got, want)
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
    _same(got, want)
    with pytest.raises(ants.AntsError) as e:
        ants.reconstruct_host_noalloc(ctx, lrf, p, np.ascontiguousarray(ev.signals, dtype=np.float32),
                                      start_xyz=start)
    assert e.value.code == -1 and "capacity" in str(e.value)


def test_noalloc_refuses_other_types_and_methods():
    """FP16 signals and the forms that need scratch growing with the batch are
    refused by the library (ANTS_E_UNIMPLEMENTED); buffers whose element type
    does not match the declared one are refused by the binding before the call."""
    import torch
    assert torch.cuda.is_available(), "needs a CUDA device"
    import paper_1602_07247_gb300 as ants
    w = synth.workloads.get("sipm8x8_xy").with_(n_xy=5, iters=4, step_xy=0.5)
    L = oracle_lrf(w)
    ctx, det, lrf, p = gpu_objects(w, L)
    ev = w.events(64, seed=3)
    n = ev.signals.shape[0]
    outs = (np.empty((n, 3), np.float32), np.empty(n, np.float32), np.empty(n, np.float32), np.empty(n, np.int32))
    with pytest.raises(ants.AntsError) as e:
        ants.ants_reconstruct_host_noalloc(ctx.handle, lrf.handle, ants.ANTS_CGS_PLAIN, p,
                                           ev.signals.astype(np.float16), w.n_sensors, *outs,
                                           signal_dtype=ants.ANTS_F16)
    assert e.value.code == ants.ANTS_E_UNIMPLEMENTED
    gp = ants.GemmParams()
    with pytest.raises(ants.AntsError) as e:
        ants.ants_reconstruct_host_noalloc(ctx.handle, lrf.handle, ants.ANTS_GEMM_TOPK, gp, ev.signals, w.n_sensors,
                                           *outs)
    assert e.value.code == ants.ANTS_E_UNIMPLEMENTED
    for bad in (ev.signals.astype(np.float16), ev.signals.astype(np.float64)):
        with pytest.raises(TypeError):
            ants.reconstruct_host_noalloc(ctx, lrf, p, bad)
    with pytest.raises(TypeError):
        ants.reconstruct_host_noalloc(ctx, lrf, p, ev.signals, start_xyz=np.zeros((n, 3)))


_FRESH = r"""
import sys
sys.path.insert(0, sys.argv[1])
import numpy as np, torch
import paper_1602_07247_gb300 as ants
import synth.workloads
torch.cuda.set_device(0)
free0 = torch.cuda.mem_get_info()[0]
w = synth.workloads.get("hex19_radial")
ctx = ants.Context(0)
det = ants.Detector(w.sensor_xy, w.gains)
coef = np.ones((1, w.n_int[0] + 3))
lrf = ants.Lrf.from_coefficients(ctx, det, ants.ANTS_LRF_RADIAL, w.n_int, w.lo, w.hi, coef, shared=True)
p = ants.CgsParams(n_xy=w.n_xy, iters=w.iters, step_xy=w.step_xy, shrink=w.shrink)
r = ants.reconstruct_host_noalloc(ctx, lrf, p, np.zeros((0, w.n_sensors), np.float32))
free1 = torch.cuda.mem_get_info()[0]
print(free0 - free1)
"""


def test_noalloc_empty_call_reserves_the_area():
    """In a fresh process, by the end of a call with no events the static area
    is held on the device (the set-up step a caller makes before handing the
    rest of device memory to its own pool)."""
    import paper_1602_07247_gb300 as ants
    out = subprocess.run([sys.executable, "-c", _FRESH, ROOT], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stderr[-2000:]
    used = int(out.stdout.strip().splitlines()[-1])
    assert used >= ants.ANTS_NOALLOC_STAGE_BYTES, used
