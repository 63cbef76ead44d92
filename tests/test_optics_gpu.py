"""Optical photon transport (Sec. 4.2.3, 4.2.4, 4.2.6, 3.5) on the GPU
against the FP64 oracle, photon by photon: both draw every photon's
uniforms from the same counter-based stream, so the FP64 kernel reproduces
the oracle's outcome of each photon; the FP32 kernel differs only where a
single-precision decision falls on the other side of a boundary."""
import numpy as np
import pytest

import oracle
import pins

pytestmark = pytest.mark.gpu


def _stack(pre_reject=0):
    """Three layers over a 4 x 4 array: light guide (n 1.5), scintillator
    (n 1.8, absorption and Rayleigh scattering), window (n 1.5); a diffuse
    reflector on top, a partly absorbing, partly specular floor between the
    sensor windows, lateral walls at 20 mm."""
    g = np.arange(4) * 8.0 - 12.0
    sxy = np.array([(x, y) for y in g for x in g])
    qe = 0.2 + 0.1 * np.random.default_rng(4).uniform(size=16)
    return dict(z=(0.0, 2.0, 12.0, 14.0), n=(1.5, 1.8, 1.5), abs_len=(200.0, 100.0, 0.0), ray_len=(0.0, 40.0, 0.0),
                sensor_xy=sxy, sensor_size=6.0, qe=qe, n_below=1.0, n_above=1.0, half_x=20.0, half_y=20.0,
                p_abs=(0.3, 0.0, 0.0, 0.1), p_spec=(0.2, 0.0, 0.0, 0.0), p_diff=(0.0, 0.0, 0.0, 0.9),
                n_sensor=1.5, ang=np.array([1.0, 0.98, 0.9, 0.7, 0.3]), max_cycles=200, pre_reject=pre_reject)


def _bare():
    sxy = np.array([[-4.0, -4.0], [4.0, -4.0], [-4.0, 4.0], [4.0, 4.0]])
    return dict(z=(0.0, 30.0), n=(1.0,), abs_len=(0.0,), ray_len=(0.0,), sensor_xy=sxy, sensor_size=6.0,
                qe=np.ones(4), n_sensor=1.0)


CONFIGS = {"bare": (_bare, [(1.5, -0.5, 7.0), (-6.0, 3.0, 12.0)]),
           "stack": (lambda: _stack(0), [(0.0, 0.0, 7.0), (5.0, -3.0, 3.0), (-11.0, 9.0, 11.5), (18.0, 1.0, 6.0)]),
           "stack_prereject": (lambda: _stack(1), [(0.0, 0.0, 7.0), (-7.0, 2.0, 9.0)])}


@pytest.fixture(scope="module")
def ctx():
    import torch
    assert torch.cuda.is_available()
    import paper_1602_07247_gb300 as ants
    return ants.Context(0)


def _run(ctx, cfg, src, n, seed, fp64):
    import torch
    import paper_1602_07247_gb300 as ants
    P = ants.OpticsParams(**cfg)
    s = torch.tensor(np.asarray(src, dtype=np.float32)).cuda()
    c, o, eta = ants.trace_photons(ctx, P, s, n, seed, fp64=fp64, want_outcome=True, want_eta=True)
    torch.cuda.synchronize()
    return c.cpu().numpy(), o.cpu().numpy().astype(np.int32), eta.cpu().numpy()


def _oracle(cfg, src, n, seed):
    src64 = np.asarray(src, dtype=np.float32).astype(np.float64)
    return oracle.trace_photons(oracle.Optics(**cfg), src64, n, seed, want_outcome=True)


@pytest.mark.parametrize("name", sorted(CONFIGS))
def test_fp64_matches_oracle_photon_by_photon(ctx, name):
    make, src = CONFIGS[name]
    cfg = make()
    n = 20000
    c, o, eta = _run(ctx, cfg, src, n, seed=99, fp64=True)
    oc, oo = _oracle(cfg, src, n, seed=99)
    same = (o == oo).mean()
    print(name, "fp64 photon agreement", same, "detected", c.sum(), "outcome mix",
          {k: int((oo == k).sum()) for k in range(-5, 0)})
    assert same >= 1.0 - 1e-5
    assert np.abs(c - oc).sum() <= int((o != oo).sum())
    assert np.array_equal(eta, (c / np.float32(n)).astype(np.float32)) or np.allclose(eta, c / n, rtol=1e-7)


@pytest.mark.parametrize("name", sorted(CONFIGS))
def test_fp32_close_to_oracle(ctx, name):
    make, src = CONFIGS[name]
    cfg = make()
    n = 20000
    c, o, _ = _run(ctx, cfg, src, n, seed=7, fp64=False)
    oc, oo = _oracle(cfg, src, n, seed=7)
    same = (o == oo).mean()
    print(name, "fp32 photon agreement", same)
    # a photon's outcome changes only when an FP32 comparison lands on the
    # other side of a boundary; a few per 10^4 photons over ~10 decisions each
    assert same >= 0.998
    assert np.abs(c - oc).sum() <= int((o != oo).sum())


def test_deterministic_and_shape_free(ctx):
    cfg = _stack(0)
    src = [(0.0, 0.0, 7.0), (3.0, 3.0, 5.0)]
    a = _run(ctx, cfg, src, 5000, seed=3, fp64=False)
    b = _run(ctx, cfg, src, 5000, seed=3, fp64=False)
    assert all(np.array_equal(x, y) for x, y in zip(a, b))
    # the first 3000 photons of a longer run are the same photons
    c = _run(ctx, cfg, src, 3000, seed=3, fp64=False)
    assert np.array_equal(c[1], a[1][:, :3000])


def test_full_size_one_source(ctx):
    """10^6 photons of one source in the stack (FP64 kernel): every photon's
    outcome against the oracle."""
    cfg = _stack(0)
    src = [(2.0, -1.0, 6.0)]
    n = 1_000_000
    c, o, _ = _run(ctx, cfg, src, n, seed=2024, fp64=True)
    oc, oo = _oracle(cfg, src, n, seed=2024)
    same = (o == oo).mean()
    print("full size fp64 agreement", same, "detected", c.sum())
    assert same >= 1.0 - 1e-5


def test_errors(ctx):
    import torch
    import paper_1602_07247_gb300 as ants
    s = torch.zeros((1, 3), device="cuda")
    for bad in (dict(z=(0.0, 0.0), n=(1.0,)), dict(p_abs=(0.6, 0.0), p_spec=(0.6, 0.0)), dict(qe=np.array([1.5] * 4)),
                dict(max_cycles=0), dict(ang=np.array([1.0]))):
        cfg = _bare()
        cfg.update(bad)
        with pytest.raises(ants.AntsError):
            ants.trace_photons(ctx, ants.OpticsParams(**cfg), s, 10, 1)
    with pytest.raises(ants.AntsError):
        c = torch.empty((1, 4), dtype=torch.int32, device="cuda")
        ants.ants_trace_photons(ctx.handle, ants.OpticsParams(**_bare()), s, 10, 1, 7, c)


def test_empty_calls(ctx):
    """No photons: zero counts (the buffer is cleared) and zero light
    response; no sources: nothing to do."""
    import torch
    import paper_1602_07247_gb300 as ants
    P = ants.OpticsParams(**_bare())
    s = torch.zeros((2, 3), device="cuda")
    s[:, 2] = 5.0
    counts = torch.full((2, 4), 7, dtype=torch.int32, device="cuda")
    eta = torch.full((2, 4), 7.0, device="cuda")
    ants.ants_trace_photons(ctx.handle, P, s, 0, 1, ants.ANTS_F32, counts, eta=eta)
    torch.cuda.synchronize()
    assert int(counts.abs().sum()) == 0 and float(eta.abs().sum()) == 0.0
    c, _, _ = ants.trace_photons(ctx, P, torch.zeros((0, 3), device="cuda"), 100, 1)
    assert c.shape == (0, 4)
