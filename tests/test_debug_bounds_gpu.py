"""The index-checking build (ANTS_DEBUG_BOUNDS).

A memory checker is not available here, so the library can be compiled with
index checks in its main kernels instead: the separable XY team kernel (table
in shared and in global memory), the small-grid patch kernel and the tcgen05
product (top-K, inference and training epilogues).  In that build an index
outside its buffer is not accessed and the site of the first one is recorded;
the calls then return ANTS_E_INTERNAL.  The test builds that library, runs the
checked paths on small cases in a separate process that loads it, and
requires (a) the self-test's deliberate check (index 7 against an extent of 5,
no access) to be recorded, (b) no other check to fire, and (c) the searches to
pass the same parity with the FP64 oracle as the normal build."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

_SCRIPT = r"""
import sys
root = sys.argv[1]
sys.path.insert(0, root)
sys.path.insert(0, root + "/tests")
import numpy as np, torch
import oracle, synth, synth.workloads
import paper_1602_07247_gb300 as ants
from parity import compare, gpu_objects, oracle_lrf, to_numpy

assert ants.ants_build_flags() == ants.ANTS_BUILD_DEBUG_BOUNDS
ctx = ants.Context(0)
ants.ants_selftest_bounds(ctx.handle)
assert ants.ants_debug_bounds_site(ctx.handle) == 9999
assert ants.ants_debug_bounds_site(ctx.handle) == 0  # read and cleared

def clean(what):
    site = ants.ants_debug_bounds_site(ctx.handle)
    assert site == 0, (what, site)
    print("checked:", what)

# separable XY team kernel, table in shared memory (8 x 8 SiPMs, 11 x 11 x 8)
w = synth.workloads.get("sipm8x8_xy")
L = oracle_lrf(w)
_, det, lrf, p = gpu_objects(w, L, ctx)
ev = w.events(300, seed=3)
res = ants.reconstruct(ctx, lrf, p, torch.from_numpy(ev.signals).cuda(), want_trace=True)
compare(w, L, ev.signals, to_numpy(res))
clean("team kernel, shared-memory table")

# team kernel with the table in global memory, and the patch kernel (16 x 16)
w16 = synth.workloads.get("sipm16x16_xy")
L16 = oracle_lrf(w16)
_, det16, lrf16, p16 = gpu_objects(w16, L16, ctx)
ev16 = w16.events(200, seed=4)
sig16 = torch.from_numpy(ev16.signals).cuda()
res = ants.reconstruct(ctx, lrf16, p16, sig16, want_trace=True)
compare(w16, L16, ev16.signals, to_numpy(res))
clean("team kernel, global-memory table")
wr = w16.with_(n_xy=5, iters=4, step_xy=0.5)
start = np.clip(ev16.xyz + np.random.default_rng(1).normal(0.0, 0.3, ev16.xyz.shape), -25.0, 25.0)
start[:, 2] = 0.0
start = start.astype(np.float32)
pr = ants.CgsParams(n_xy=5, iters=4, step_xy=0.5)
res = ants.reconstruct(ctx, lrf16, pr, sig16, start_xyz=torch.from_numpy(start).cuda(), want_trace=True)
compare(wr, L16, ev16.signals, to_numpy(res), start=start.astype(np.float64))
clean("patch kernel")

# tcgen05 top-K product and the precision form
table = ants.LogTable(ctx, lrf16, 64, 64)
sc, ix = table.topk(sig16, 8)
gp = table.params(ants.CgsParams(n_xy=7, iters=5, step_xy=0.8 / 3), top_k=8, nms_cells=1.5)
ants.reconstruct(ctx, lrf16, gp, sig16.half(), method=ants.ANTS_GEMM_TOPK)
clean("tcgen05 top-K product")

# tcgen05 network: inference (bias + GELU) and training (forward with z,
# GELU backward, weight gradients)
M = ants.Mlp.create(ctx, 64, 96, 24.0, float(np.log(3000.0)), 0.05, seed=3)
out = torch.empty((300, 3), device="cuda")
ants.ants_mlp_forward(ctx.handle, M.handle, torch.from_numpy(ev.signals).cuda(), out, bf16=1)
truth = np.concatenate([ev.xyz, ev.energy[:, None]], 1).astype(np.float32)
ants.ants_mlp_loss_grad(ctx.handle, M.handle, torch.from_numpy(ev.signals).cuda(), torch.from_numpy(truth).cuda(),
                        bf16=1)
ev2 = w.events(6000, seed=5)
t2 = np.concatenate([ev2.xyz, ev2.energy[:, None]], 1).astype(np.float32)
M.train(torch.from_numpy(ev2.signals).cuda(), torch.from_numpy(t2).cuda(), ants.TrainParams(epochs=2, batch=512))
clean("tcgen05 network products")
print("DEBUG_BOUNDS_OK")
"""


def test_debug_bounds_build_runs_clean():
    from paper_1602_07247_gb300 import _build
    lib = _build.build_debug()
    env = dict(os.environ, ANTS_LIBRARY=lib)
    out = subprocess.run([sys.executable, "-c", _SCRIPT, ROOT], capture_output=True, text=True, timeout=900, env=env)
    print(out.stdout[-3000:])
    assert out.returncode == 0, out.stderr[-3000:]
    assert "DEBUG_BOUNDS_OK" in out.stdout
