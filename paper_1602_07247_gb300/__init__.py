"""Python binding of libants (include/ants.h): argument marshalling only.

Every step of the reconstruction runs in the CUDA kernels of libants.so; this
module converts torch tensors / numpy arrays to pointers and sizes and turns
non-OK return codes into exceptions.  There is no CPU path: if the library is
missing or cannot load, every call raises.

The functions keep the C names (ants_ctx_create, ants_lrf_create,
ants_reconstruct, ...).  Small wrapper classes (Context, Detector, Lrf) own
the handles and free them when collected.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from . import _build

# the library to load: the in-tree build, or another build of the same sources
# named by ANTS_LIBRARY (the index-checking ANTS_DEBUG_BOUNDS build, _build.DEBUG_LIB)
LIB_PATH = os.environ.get("ANTS_LIBRARY") or _build.LIB

# enums of include/ants.h
ANTS_OK = 0
ANTS_E_ARG, ANTS_E_CUDA, ANTS_E_OOM, ANTS_E_LRF, ANTS_E_SHAPE = -1, -2, -3, -4, -5
ANTS_E_TIMEOUT, ANTS_E_INTERNAL, ANTS_E_UNIMPLEMENTED, ANTS_E_IO = -6, -7, -8, -9
ANTS_LRF_RADIAL, ANTS_LRF_XY, ANTS_LRF_XYZ = 1, 2, 3
ANTS_LRF_COMPOSITE, ANTS_LRF_AXIAL_Z, ANTS_LRF_SLICED = 4, 5, 6
ANTS_EVT_OK, ANTS_EVT_FALLBACK, ANTS_EVT_ZERO_SIGNAL = 0, 1, 2
ANTS_EVT_BAD_SIGNAL, ANTS_EVT_OUT_OF_DOMAIN, ANTS_EVT_LOW_LOGL = 3, 4, 5
ANTS_CGS_PLAIN = 0
ANTS_GEMM_TOPK = 1
ANTS_MLP_SEEDED = 2
ANTS_CGS_VARIANT = 3
ANTS_MINIMIZE = 4
ANTS_F64 = 2
ANTS_PH_ABSORBED, ANTS_PH_ESCAPED, ANTS_PH_MAX_CYCLES, ANTS_PH_UNDETECTED, ANTS_PH_REJECTED = -1, -2, -3, -4, -5
ANTS_CRIT_ML, ANTS_CRIT_LS = 0, 1
ANTS_START_COG, ANTS_START_MAX_SENSOR = 0, 1
ANTS_F32 = 0
ANTS_F16 = 1
ANTS_NOALLOC_STAGE_BYTES = 33554432
ANTS_BUILD_DEBUG_BOUNDS = 1

_STATUS_NAMES = {0: "ANTS_OK", -1: "ANTS_E_ARG", -2: "ANTS_E_CUDA", -3: "ANTS_E_OOM", -4: "ANTS_E_LRF",
                 -5: "ANTS_E_SHAPE", -6: "ANTS_E_TIMEOUT", -7: "ANTS_E_INTERNAL", -8: "ANTS_E_UNIMPLEMENTED",
                 -9: "ANTS_E_IO"}


class AntsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


class CgsParams(C.Structure):
    """ants_cgs_params: contracting-grid search settings."""
    _fields_ = [("n_xy", C.c_int), ("n_z", C.c_int), ("iters", C.c_int), ("shrink", C.c_float),
                ("step_xy", C.c_float), ("step_z", C.c_float), ("z0", C.c_float)]

    def __init__(self, n_xy=9, iters=6, step_xy=1.0, shrink=0.5, n_z=1, step_z=0.0, z0=0.0):
        super().__init__(n_xy, n_z, iters, shrink, step_xy, step_z, z0)


class MlpConfig(C.Structure):
    """ants_mlp_config: hidden width and output scaling of the proposal network."""
    _fields_ = [("n_hidden", C.c_int), ("xy_scale", C.c_float), ("loge_mean", C.c_float), ("loge_std", C.c_float)]


class TrainParams(C.Structure):
    """ants_train_params."""
    _fields_ = [("epochs", C.c_int), ("batch", C.c_int), ("lr", C.c_float), ("beta1", C.c_float),
                ("beta2", C.c_float), ("eps", C.c_float), ("monitor_frac", C.c_float), ("patience", C.c_int),
                ("bf16", C.c_int), ("seed", C.c_uint64)]

    def __init__(self, epochs=20, batch=1024, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, monitor_frac=0.1,
                 patience=3, bf16=1, seed=2001):
        super().__init__(epochs, batch, lr, beta1, beta2, eps, monitor_frac, patience, bf16, seed)


class TrainReport(C.Structure):
    _fields_ = [("epochs_run", C.c_int), ("best_epoch", C.c_int), ("best_monitor_mse", C.c_float),
                ("last_train_mse", C.c_float)]


class SimParams(C.Structure):
    """ants_sim_params: source region, energy and single photo-electron response."""
    _fields_ = [("region", C.c_int), ("extent", C.c_float), ("cx", C.c_float), ("cy", C.c_float),
                ("z_lo", C.c_float), ("z_hi", C.c_float), ("e0", C.c_float), ("e_spread", C.c_float),
                ("spe_sigma", C.c_float)]

    def __init__(self, region="square", extent=10.0, cx=0.0, cy=0.0, z_lo=0.0, z_hi=0.0, e0=1000.0, e_spread=0.05,
                 spe_sigma=0.0):
        codes = {"disk": 0, "square": 1, 0: 0, 1: 1}
        if region not in codes:
            raise ValueError(f"region must be 'disk' (0) or 'square' (1), not {region!r}")
        super().__init__(codes[region], extent, cx, cy, z_lo, z_hi, e0, e_spread, spe_sigma)


class BatchItem(C.Structure):
    """ants_batch_item: one detector's share of a batched run."""
    _fields_ = [("lrf", C.c_void_p), ("params", CgsParams), ("signals_dev", C.c_void_p), ("n_events", C.c_long),
                ("start_xyz_dev", C.c_void_p), ("xyz_dev", C.c_void_p), ("E_dev", C.c_void_p),
                ("logL_dev", C.c_void_p), ("status_dev", C.c_void_p), ("trace_dev", C.c_void_p)]


class BatchConfig(C.Structure):
    """ants_batch_config: events per work unit, warps per block, blocks per SM."""
    _fields_ = [("unit_events", C.c_int), ("warps_per_block", C.c_int), ("blocks_per_sm", C.c_int)]


class GemmParams(C.Structure):
    """ants_gemm_params: log-response table, top-K, suppression radius, refine."""
    _fields_ = [("table", C.c_void_p), ("top_k", C.c_int), ("nms_cells", C.c_float), ("refine", CgsParams)]


class SeededParams(C.Structure):
    """ants_mlp_seeded_params: network start, local refine, plain fallback."""
    _fields_ = [("mlp", C.c_void_p), ("bf16", C.c_int), ("refine", CgsParams), ("fallback", CgsParams),
                ("deviance_max", C.c_float), ("border_fallback", C.c_int)]


class VariantParams(C.Structure):
    """ants_cgs_variant_params: grid, criterion, start, sensor cuts, passive mask."""
    _fields_ = [("grid", CgsParams), ("criterion", C.c_int), ("start", C.c_int), ("min_signal", C.c_float),
                ("max_distance", C.c_float), ("passive_host", C.c_void_p)]

    def __init__(self, grid, criterion=0, start=0, min_signal=0.0, max_distance=0.0, passive=None):
        self._passive = None if passive is None else np.ascontiguousarray(np.asarray(passive, dtype=np.uint8))
        super().__init__(grid, int(criterion), int(start), float(min_signal), float(max_distance),
                         None if self._passive is None else self._passive.ctypes.data)


class MinimizeParams(C.Structure):
    """ants_minimize_params (Sec. 5.1.2.1): continuous minimisation of the
    match (damped Fisher scoring, E profiled) from the centroid, the strongest
    sensor or given starts."""
    _fields_ = [("criterion", C.c_int), ("start", C.c_int), ("z0", C.c_float), ("fit_z", C.c_int),
                ("max_iter", C.c_int), ("tol", C.c_float), ("lambda0", C.c_float), ("min_signal", C.c_float),
                ("max_distance", C.c_float), ("passive_host", C.c_void_p)]

    def __init__(self, criterion=0, start=0, z0=0.0, fit_z=1, max_iter=30, tol=1e-3, lambda0=1e-3, min_signal=0.0,
                 max_distance=0.0, passive=None):
        self._passive = None if passive is None else np.ascontiguousarray(np.asarray(passive, dtype=np.uint8))
        super().__init__(int(criterion), int(start), float(z0), int(fit_z), int(max_iter), float(tol),
                         float(lambda0), float(min_signal), float(max_distance),
                         None if self._passive is None else self._passive.ctypes.data)


_OML = 8  # ANTS_OPT_MAX_LAYERS


class OpticsParams(C.Structure):
    """ants_optics_params (Sec. 4.2.3, 4.2.4, 4.2.6, 3.5): a slab stack over
    square sensor windows on its bottom boundary."""
    _fields_ = [("n_layers", C.c_int), ("z", C.c_double * (_OML + 1)), ("n", C.c_double * _OML),
                ("abs_len", C.c_double * _OML), ("ray_len", C.c_double * _OML), ("n_below", C.c_double),
                ("n_above", C.c_double), ("half_x", C.c_double), ("half_y", C.c_double),
                ("p_abs", C.c_double * (_OML + 1)), ("p_spec", C.c_double * (_OML + 1)),
                ("p_diff", C.c_double * (_OML + 1)), ("n_sensors", C.c_int), ("sensor_xy_host", C.c_void_p),
                ("sensor_size", C.c_double), ("n_sensor", C.c_double), ("qe_host", C.c_void_p), ("n_ang", C.c_int),
                ("ang_host", C.c_void_p), ("max_cycles", C.c_int), ("pre_reject", C.c_int)]

    def __init__(self, z, n, abs_len, ray_len, sensor_xy, sensor_size, qe, n_below=1.0, n_above=1.0, half_x=1e9,
                 half_y=1e9, p_abs=(), p_spec=(), p_diff=(), n_sensor=1.5, ang=None, max_cycles=1000, pre_reject=0):
        pad = lambda v, m: [float(x) for x in v] + [0.0] * (m - len(v))
        self._sxy = np.ascontiguousarray(np.asarray(sensor_xy, dtype=np.float64))
        self._qe = np.ascontiguousarray(np.asarray(qe, dtype=np.float64))
        self._ang = None if ang is None else np.ascontiguousarray(np.asarray(ang, dtype=np.float64))
        super().__init__(len(n), (C.c_double * (_OML + 1))(*pad(z, _OML + 1)), (C.c_double * _OML)(*pad(n, _OML)),
                         (C.c_double * _OML)(*pad(abs_len, _OML)), (C.c_double * _OML)(*pad(ray_len, _OML)),
                         float(n_below), float(n_above), float(half_x), float(half_y),
                         (C.c_double * (_OML + 1))(*pad(p_abs, _OML + 1)),
                         (C.c_double * (_OML + 1))(*pad(p_spec, _OML + 1)),
                         (C.c_double * (_OML + 1))(*pad(p_diff, _OML + 1)), self._sxy.shape[0],
                         self._sxy.ctypes.data, float(sensor_size), float(n_sensor), self._qe.ctypes.data,
                         0 if self._ang is None else self._ang.shape[0],
                         None if self._ang is None else self._ang.ctypes.data, int(max_cycles), int(pre_reject))


class EventCuts(C.Structure):
    """ants_event_cuts (Sec. 5.2): a cut is off when chi2_max <= 0, r_max <= 0
    or its window's upper bound is not above its lower bound."""
    _fields_ = [(n, C.c_double) for n in ("chi2_max", "e_lo", "e_hi", "sum_lo", "sum_hi", "r_max", "cx", "cy")]


class RefitParams(C.Structure):
    """ants_refit_params: grouping, gain refit, seeded shift, ridge."""
    _fields_ = [("shared", C.c_int), ("refit_gains", C.c_int), ("shift_sigma", C.c_double), ("seed", C.c_uint64),
                ("cycle", C.c_int), ("ridge", C.c_double)]


class IterParams(C.Structure):
    """ants_iter_params: the cycles of Sec. 8."""
    _fields_ = [("cgs", CgsParams), ("cycles", C.c_int), ("cuts", EventCuts), ("refit_gains", C.c_int),
                ("shift_sigma", C.c_double), ("shift_cycles", C.c_int), ("seed", C.c_uint64), ("ridge", C.c_double),
                ("method", C.c_int), ("minimize", MinimizeParams)]


class IterStats(C.Structure):
    _fields_ = [("n_kept", C.c_long), ("mean_chi2", C.c_double), ("mean_E", C.c_double),
                ("rel_change", C.c_double)]


_lib: C.CDLL | None = None
_VP = C.c_void_p
_DP = C.POINTER(C.c_double)
_IP = C.POINTER(C.c_int)


def lib() -> C.CDLL:
    """Load libants.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"libants.so not built ({LIB_PATH}); run __graft_entry__.build()")
        L = C.CDLL(LIB_PATH)
        L.ants_last_error.restype = C.c_char_p
        L.ants_version.restype = C.c_int
        L.ants_last_launch_count.restype = C.c_long
        L.ants_ctx_create.argtypes = [C.c_int, C.POINTER(_VP)]
        L.ants_ctx_destroy.argtypes = [_VP]
        L.ants_ctx_destroy.restype = None
        L.ants_ctx_fault.argtypes = [_VP, C.POINTER(C.c_int)]
        L.ants_selftest_stalled_product.argtypes = [_VP]
        L.ants_build_flags.restype = C.c_int
        L.ants_debug_bounds_site.argtypes = [_VP, C.POINTER(C.c_int)]
        L.ants_selftest_bounds.argtypes = [_VP]
        L.ants_detector_create.argtypes = [C.c_int, _DP, _DP, C.POINTER(_VP)]
        L.ants_detector_free.argtypes = [_VP]
        L.ants_detector_free.restype = None
        L.ants_lrf_create.argtypes = [_VP, _VP, C.c_int, _IP, _DP, _DP, C.c_int, _DP, _DP, C.POINTER(_VP)]
        L.ants_lrf_fit.argtypes = [_VP, _VP, C.c_int, _IP, _DP, _DP, C.c_int, C.c_long, _DP, _DP, C.c_double, _DP,
                                   C.POINTER(_VP)]
        L.ants_lrf_coefficients.argtypes = [_VP, _DP, C.c_size_t, _IP, _IP]
        L.ants_lrf_eval.argtypes = [_VP, _VP, C.c_long, C.c_int, _VP, _VP]
        L.ants_lrf_save.argtypes = [_VP, C.c_char_p]
        L.ants_lrf_load.argtypes = [_VP, _VP, C.c_char_p, C.POINTER(_VP)]
        L.ants_lrf_free.argtypes = [_VP]
        L.ants_lrf_free.restype = None
        L.ants_reconstruct.argtypes = [_VP, _VP, C.c_int, _VP, _VP, C.c_int, C.c_long, C.c_int, _VP, _VP, _VP,
                                       _VP, _VP, _VP, _VP]
        L.ants_reconstruct_host.argtypes = [_VP, _VP, C.c_int, _VP, _VP, C.c_int, C.c_long, C.c_int, _VP, _VP,
                                            _VP, _VP, _VP]
        L.ants_reconstruct_host_noalloc.argtypes = [_VP, _VP, C.c_int, _VP, _VP, C.c_int, C.c_long, C.c_int, _VP,
                                                    _VP, _VP, _VP, _VP]
        L.ants_reconstruct_host_noalloc.restype = C.c_int
        L.ants_logtable_create.argtypes = [_VP, _VP, C.c_int, C.c_int, C.POINTER(_VP)]
        L.ants_logtable_values.argtypes = [_VP, _VP, _VP]
        L.ants_logtable_topk.argtypes = [_VP, _VP, _VP, C.c_long, C.c_int, C.c_int, _VP, _VP, _VP]
        L.ants_logtable_free.argtypes = [_VP]
        L.ants_logtable_free.restype = None
        L.ants_batch_plan_create.argtypes = [_VP, C.c_int, C.POINTER(BatchItem), C.POINTER(BatchConfig),
                                             C.POINTER(_VP)]
        L.ants_batch_run.argtypes = [_VP, _VP]
        L.ants_batch_autotune.argtypes = [_VP, C.c_char_p, C.c_long, C.POINTER(BatchConfig)]
        L.ants_batch_get_config.argtypes = [_VP, C.POINTER(BatchConfig)]
        L.ants_batch_plan_free.argtypes = [_VP]
        L.ants_batch_plan_free.restype = None
        L.ants_simulate_events.argtypes = [_VP, _VP, C.POINTER(SimParams), C.c_uint64, C.c_long, C.c_long, _VP, _VP,
                                           _VP]
        L.ants_deviance.argtypes = [_VP, _VP, _VP, C.c_long, C.c_int, _VP, _VP, _VP]
        L.ants_mlp_create.argtypes = [_VP, C.c_int, C.POINTER(MlpConfig), C.c_uint64, C.POINTER(_VP)]
        L.ants_mlp_free.argtypes = [_VP]
        L.ants_mlp_free.restype = None
        L.ants_mlp_shape.argtypes = [_VP, C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_long)]
        L.ants_mlp_set_params.argtypes = [_VP, _VP, C.c_long]
        L.ants_mlp_get_params.argtypes = [_VP, _VP, C.c_long]
        L.ants_mlp_forward.argtypes = [_VP, _VP, _VP, C.c_long, C.c_int, C.c_int, _VP, _VP, _VP, _VP]
        L.ants_mlp_loss_grad.argtypes = [_VP, _VP, _VP, _VP, C.c_long, C.c_int, C.c_int, C.POINTER(C.c_float), _VP]
        L.ants_mlp_train.argtypes = [_VP, _VP, _VP, _VP, C.c_long, C.c_int, C.POINTER(TrainParams),
                                     C.POINTER(TrainReport)]
        L.ants_mlp_save.argtypes = [_VP, C.c_char_p]
        L.ants_mlp_load.argtypes = [_VP, C.c_char_p, C.POINTER(_VP)]
        L.ants_lrf_gains.argtypes = [_VP, _DP, C.c_size_t]
        L.ants_lrf_create_scheme.argtypes = [_VP, _VP, C.c_int, _IP, _DP, _DP, C.c_int, C.c_double, C.c_int, _DP,
                                             C.POINTER(_VP)]
        L.ants_lrf_fit_scheme.argtypes = [_VP, _VP, C.c_int, _IP, _DP, _DP, C.c_int, C.c_double, C.c_int, C.c_long,
                                          _DP, _DP, C.c_double, C.POINTER(_VP)]
        L.ants_event_centroid.argtypes = [_VP, _VP, _VP, C.c_long, _VP, _VP, _VP]
        L.ants_trace_photons.argtypes = [_VP, _VP, _VP, C.c_long, C.c_long, C.c_uint64, C.c_int, _VP, _VP, _VP, _VP]
        L.ants_lrf_create_grouped.argtypes = [_VP, _VP, _IP, _DP, _DP, C.c_int, _IP, _DP, _DP, C.POINTER(_VP)]
        L.ants_sensor_rings.argtypes = [_VP, C.c_double, _IP, _IP]
        L.ants_lrf_create_symmetric.argtypes = [_VP, _VP, _IP, _DP, _DP, C.c_int, _IP, _IP, _DP, _DP, _DP,
                                                C.POINTER(_VP)]
        L.ants_sensor_symmetry.argtypes = [_VP, C.c_double, _IP, _IP, _DP, _IP]
        L.ants_lrf_fit_symmetric.argtypes = [_VP, _VP, _IP, _DP, _DP, C.c_int, _IP, _IP, _DP, C.c_long, _DP, _DP,
                                             _DP, C.c_double, C.POINTER(_VP)]
        L.ants_event_chi2.argtypes = [_VP, _VP, _VP, C.c_long, _VP, _VP, _VP, _VP, _VP]
        L.ants_event_filter.argtypes = [_VP, C.c_long, _VP, _VP, _VP, _VP, _VP, C.POINTER(EventCuts), _VP,
                                        C.POINTER(C.c_long), _VP]
        L.ants_lrf_refit.argtypes = [_VP, _VP, _VP, C.c_long, _VP, _VP, _VP, C.c_long, C.POINTER(RefitParams),
                                     C.POINTER(_VP)]
        L.ants_lrf_iterate.argtypes = [_VP, _VP, _VP, C.c_long, C.POINTER(IterParams), C.POINTER(IterStats),
                                       C.POINTER(_VP)]
        _lib = L
    return _lib


def _check(rc: int) -> None:
    if rc != ANTS_OK:
        raise AntsError(rc, lib().ants_last_error().decode())


def _dptr(a):
    return a.ctypes.data_as(_DP) if a is not None else C.cast(None, _DP)


def _f64(a):
    return None if a is None else np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def _tptr(t) -> int | None:
    """Device (or host) address of a torch tensor / numpy array; None -> NULL."""
    if t is None:
        return None
    if isinstance(t, np.ndarray):
        if not t.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return t.ctypes.data
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return t.data_ptr()


def _dtype_name(a) -> str:
    return str(a.dtype).replace("torch.", "")


def _check_signals(signals, signal_dtype: int) -> None:
    """The signal buffer's element type must be the one signal_dtype names
    (float32 for ANTS_F32, float16 for ANTS_F16): the library reads
    n_events x n_sensors elements of that size from it."""
    want = {ANTS_F32: "float32", ANTS_F16: "float16"}.get(signal_dtype)
    if want is not None and _dtype_name(signals) != want:
        raise TypeError(f"signals are {_dtype_name(signals)}, signal_dtype {signal_dtype} needs {want}")


def _check_start(start_xyz, n: int) -> None:
    """Start positions, when given: float32 [n_events, 3]."""
    if start_xyz is None:
        return
    if _dtype_name(start_xyz) != "float32":
        raise TypeError(f"start_xyz is {_dtype_name(start_xyz)}, needs float32")
    if tuple(start_xyz.shape) != (n, 3):
        raise ValueError(f"start_xyz has shape {tuple(start_xyz.shape)}, needs ({n}, 3)")


def _signal_dtype_of(signals) -> int:
    """ANTS_F16 for float16 signals, ANTS_F32 for float32; anything else is refused."""
    name = _dtype_name(signals)
    if name == "float16":
        return ANTS_F16
    if name == "float32":
        return ANTS_F32
    raise TypeError(f"signals must be float32 or float16, not {name}")


def _stream_handle(stream) -> int | None:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return stream if isinstance(stream, int) else stream.cuda_stream


def last_launch_count() -> int:
    return int(lib().ants_last_launch_count())


# --------------------------------------------------------------------------
# C-named calls
# --------------------------------------------------------------------------


def ants_version() -> int:
    return int(lib().ants_version())


def ants_ctx_create(device: int = 0) -> int:
    h = _VP()
    _check(lib().ants_ctx_create(device, C.byref(h)))
    return h.value


def ants_ctx_destroy(ctx: int) -> None:
    lib().ants_ctx_destroy(ctx)


def ants_ctx_fault(ctx: int) -> int:
    """Synchronise, read and clear the device fault word (0: no kernel gave up a
    bounded wait); raises AntsError(ANTS_E_TIMEOUT) when it was set."""
    f = C.c_int(0)
    _check(lib().ants_ctx_fault(ctx, C.byref(f)))
    return f.value


def ants_build_flags() -> int:
    return int(lib().ants_build_flags())


def ants_debug_bounds_site(ctx: int) -> int:
    """Site of the first out-of-range index a checked kernel recorded (0: none),
    then cleared; always 0 in the normal build."""
    site = C.c_int(0)
    _check(lib().ants_debug_bounds_site(ctx, C.byref(site)))
    return site.value


def ants_selftest_bounds(ctx: int) -> None:
    _check(lib().ants_selftest_bounds(ctx))


def ants_selftest_stalled_product(ctx: int) -> None:
    """Run the bounded-wait self-test of the tensor-core kernels (raises on failure)."""
    _check(lib().ants_selftest_stalled_product(ctx))


def ants_detector_create(sensor_xy, rel_gain=None) -> int:
    xy = _f64(sensor_xy)
    g = _f64(rel_gain)
    h = _VP()
    _check(lib().ants_detector_create(int(xy.shape[0]), _dptr(xy), _dptr(g), C.byref(h)))
    return h.value


def ants_detector_free(det: int) -> None:
    lib().ants_detector_free(det)


def ants_lrf_create(ctx: int, det: int, type: int, n_int, lo, hi, shared: bool, coef, gain=None) -> int:
    ni = (C.c_int * 3)(*[int(v) for v in (list(n_int) + [0, 0, 0])[:3]])
    lo_ = _f64((list(lo) + [0.0, 0.0, 0.0])[:3])
    hi_ = _f64((list(hi) + [0.0, 0.0, 0.0])[:3])
    cf = _f64(coef)
    g = _f64(gain)
    h = _VP()
    _check(lib().ants_lrf_create(ctx, det, int(type), ni, _dptr(lo_), _dptr(hi_), 1 if shared else 0, _dptr(cf),
                                 _dptr(g), C.byref(h)))
    return h.value


def ants_lrf_fit(ctx: int, det: int, type: int, n_int, lo, hi, shared: bool, pts, vals, ridge: float = 0.0):
    """Returns (handle, ridge_used)."""
    ni = (C.c_int * 3)(*[int(v) for v in (list(n_int) + [0, 0, 0])[:3]])
    lo_ = _f64((list(lo) + [0.0, 0.0, 0.0])[:3])
    hi_ = _f64((list(hi) + [0.0, 0.0, 0.0])[:3])
    p = _f64(pts)
    v = _f64(vals)
    if v.ndim == 1:
        v = v[:, None]
    lam = C.c_double()
    h = _VP()
    _check(lib().ants_lrf_fit(ctx, det, int(type), ni, _dptr(lo_), _dptr(hi_), 1 if shared else 0,
                              int(p.shape[0]), _dptr(p), _dptr(v), float(ridge), C.byref(lam), C.byref(h)))
    return h.value, lam.value


def ants_lrf_coefficients(lrf: int) -> np.ndarray:
    ns, nc = C.c_int(), C.c_int()
    _check(lib().ants_lrf_coefficients(lrf, None, 0, C.byref(ns), C.byref(nc)))
    out = np.empty((ns.value, nc.value))
    _check(lib().ants_lrf_coefficients(lrf, _dptr(out), out.size, None, None))
    return out


def _grid3(n_int, lo, hi):
    ni = np.zeros(3, dtype=np.int32)
    l3, h3 = np.zeros(3), np.zeros(3)
    ni[:len(n_int)] = n_int
    l3[:len(lo)] = lo
    h3[:len(hi)] = hi
    return ni, l3, h3


def ants_lrf_create_scheme(ctx: int, det: int, type: int, n_int, lo, hi, coef, n_int_r: int = 0, hi_r: float = 0.0,
                           n_planes: int = 0) -> int:
    ni, l3, h3 = _grid3(n_int, lo, hi)
    c = _f64(coef).ravel()
    h = _VP()
    _check(lib().ants_lrf_create_scheme(ctx, det, type, ni.ctypes.data_as(_IP), _dptr(l3), _dptr(h3), int(n_int_r),
                                        float(hi_r), int(n_planes), _dptr(c), C.byref(h)))
    return h.value


def ants_lrf_fit_scheme(ctx: int, det: int, type: int, n_int, lo, hi, pts, vals, n_int_r: int = 0,
                        hi_r: float = 0.0, n_planes: int = 0, ridge: float = 0.0) -> int:
    ni, l3, h3 = _grid3(n_int, lo, hi)
    p, v = _f64(pts), _f64(vals)
    h = _VP()
    _check(lib().ants_lrf_fit_scheme(ctx, det, type, ni.ctypes.data_as(_IP), _dptr(l3), _dptr(h3), int(n_int_r),
                                     float(hi_r), int(n_planes), int(p.shape[0]), _dptr(p), _dptr(v), float(ridge),
                                     C.byref(h)))
    return h.value


def ants_lrf_gains(lrf: int, n_sensors: int) -> np.ndarray:
    g = np.empty(n_sensors)
    _check(lib().ants_lrf_gains(lrf, _dptr(g), n_sensors))
    return g


def ants_event_centroid(ctx: int, lrf: int, signals, xyz, ssum=None, stream=None) -> None:
    _check(lib().ants_event_centroid(ctx, lrf, _tptr(signals), signals.shape[0], _tptr(xyz), _tptr(ssum),
                                     _stream_handle(stream)))


def ants_event_chi2(ctx: int, lrf: int, signals, xyz, E, chi2, ssum=None, stream=None) -> None:
    _check(lib().ants_event_chi2(ctx, lrf, _tptr(signals), signals.shape[0], _tptr(xyz), _tptr(E), _tptr(chi2),
                                 _tptr(ssum), _stream_handle(stream)))


def ants_event_filter(ctx: int, status, xyz, E, chi2, ssum, cuts: EventCuts, index, stream=None) -> int:
    n = C.c_long(0)
    _check(lib().ants_event_filter(ctx, status.shape[0], _tptr(status), _tptr(xyz), _tptr(E), _tptr(chi2),
                                   _tptr(ssum), C.byref(cuts), _tptr(index), C.byref(n), _stream_handle(stream)))
    return int(n.value)


def ants_lrf_refit(ctx: int, lrf: int, signals, xyz, E, index, n_kept: int, params: RefitParams) -> int:
    h = _VP()
    _check(lib().ants_lrf_refit(ctx, lrf, _tptr(signals), signals.shape[0], _tptr(xyz), _tptr(E), _tptr(index),
                                n_kept, C.byref(params), C.byref(h)))
    return h.value


def ants_lrf_iterate(ctx: int, lrf: int, signals, params: IterParams):
    stats = (IterStats * params.cycles)()
    h = _VP()
    _check(lib().ants_lrf_iterate(ctx, lrf, _tptr(signals), signals.shape[0], C.byref(params), stats, C.byref(h)))
    return h.value, [dict(n_kept=s.n_kept, mean_chi2=s.mean_chi2, mean_E=s.mean_E, rel_change=s.rel_change)
                     for s in stats]


def ants_lrf_eval(lrf: int, pts, out, stream=None) -> None:
    _check(lib().ants_lrf_eval(lrf, _tptr(pts), int(pts.shape[0]), int(pts.shape[1]), _tptr(out),
                               _stream_handle(stream)))


def ants_lrf_save(lrf: int, path: str) -> None:
    _check(lib().ants_lrf_save(lrf, path.encode()))


def ants_lrf_load(ctx: int, det: int, path: str) -> int:
    h = _VP()
    _check(lib().ants_lrf_load(ctx, det, path.encode(), C.byref(h)))
    return h.value


def ants_lrf_free(lrf: int) -> None:
    lib().ants_lrf_free(lrf)


def ants_reconstruct(ctx: int, lrf: int, method: int, params, signals, n_sensors: int, xyz, E, logL, status,
                     start_xyz=None, trace=None, stream=None, signal_dtype: int = ANTS_F32) -> None:
    _check_signals(signals, signal_dtype)
    _check_start(start_xyz, int(signals.shape[0]))
    _check(lib().ants_reconstruct(ctx, lrf, method, C.addressof(params), _tptr(signals), signal_dtype,
                                  int(signals.shape[0]), int(n_sensors), _tptr(start_xyz), _tptr(xyz), _tptr(E),
                                  _tptr(logL), _tptr(status), _tptr(trace), _stream_handle(stream)))


def ants_reconstruct_host(ctx: int, lrf: int, method: int, params, signals, n_sensors: int, xyz, E, logL,
                          status, start_xyz=None, signal_dtype: int = ANTS_F32) -> None:
    _check_signals(signals, signal_dtype)
    _check_start(start_xyz, int(signals.shape[0]))
    _check(lib().ants_reconstruct_host(ctx, lrf, method, C.addressof(params), _tptr(signals), signal_dtype,
                                       int(signals.shape[0]), int(n_sensors), _tptr(start_xyz), _tptr(xyz),
                                       _tptr(E), _tptr(logL), _tptr(status)))


def ants_reconstruct_host_noalloc(ctx: int, lrf: int, method: int, params, signals, n_sensors: int, xyz, E, logL,
                                  status, start_xyz=None, signal_dtype: int = ANTS_F32) -> None:
    """Host-buffer reconstruction through the library's static staging area
    (no device allocation; batch limited by ANTS_NOALLOC_STAGE_BYTES)."""
    _check_signals(signals, signal_dtype)
    _check_start(start_xyz, int(signals.shape[0]))
    _check(lib().ants_reconstruct_host_noalloc(ctx, lrf, method, C.addressof(params), _tptr(signals), signal_dtype,
                                               int(signals.shape[0]), int(n_sensors), _tptr(start_xyz), _tptr(xyz),
                                               _tptr(E), _tptr(logL), _tptr(status)))


def ants_logtable_create(ctx: int, lrf: int, nx: int, ny: int) -> int:
    h = _VP()
    _check(lib().ants_logtable_create(ctx, lrf, int(nx), int(ny), C.byref(h)))
    return h.value


def ants_logtable_values(table: int, n_points: int, n_sensors: int):
    T = np.empty((n_points, n_sensors), dtype=np.float32)
    m = np.empty(n_sensors, dtype=np.float32)
    _check(lib().ants_logtable_values(table, T.ctypes.data, m.ctypes.data))
    return T, m


def ants_logtable_topk(ctx: int, table: int, signals, top_k: int, score, index, stream=None) -> None:
    _check(lib().ants_logtable_topk(ctx, table, _tptr(signals), int(signals.shape[0]), int(signals.shape[1]),
                                    int(top_k), _tptr(score), _tptr(index), _stream_handle(stream)))


def ants_logtable_free(table: int) -> None:
    lib().ants_logtable_free(table)


class LogTable:
    """Global-grid log-response table of an XY LRF set (owning wrapper)."""

    def __init__(self, ctx: Context, lrf: "Lrf", nx: int, ny: int):
        self.ctx, self.lrf, self.nx, self.ny = ctx, lrf, nx, ny
        self.handle = ants_logtable_create(ctx.handle, lrf.handle, nx, ny)

    def values(self):
        return ants_logtable_values(self.handle, self.nx * self.ny, self.lrf.n_sensors)

    def topk(self, signals, k: int, stream=None):
        import torch
        n = signals.shape[0]
        sc = torch.empty((n, k), dtype=torch.float32, device=signals.device)
        ix = torch.empty((n, k), dtype=torch.int32, device=signals.device)
        ants_logtable_topk(self.ctx.handle, self.handle, signals, k, sc, ix, stream)
        return sc, ix

    def params(self, refine: CgsParams, top_k: int = 8, nms_cells: float = 1.5) -> GemmParams:
        return GemmParams(self.handle, int(top_k), float(nms_cells), refine)

    def __del__(self):
        if getattr(self, "handle", None):
            ants_logtable_free(self.handle)
            self.handle = None


def ants_batch_plan_create(ctx: int, items, cfg: BatchConfig | None = None) -> int:
    arr = (BatchItem * len(items))(*items)
    h = _VP()
    _check(lib().ants_batch_plan_create(ctx, len(items), arr, C.byref(cfg) if cfg is not None else None, C.byref(h)))
    return h.value


def ants_batch_run(plan: int, stream=None) -> None:
    _check(lib().ants_batch_run(plan, _stream_handle(stream)))


def ants_batch_autotune(plan: int, cache_path: str | None = None, events_per_item: int = 2048) -> BatchConfig:
    c = BatchConfig()
    _check(lib().ants_batch_autotune(plan, cache_path.encode() if cache_path else None, int(events_per_item),
                                     C.byref(c)))
    return c


def ants_batch_get_config(plan: int) -> BatchConfig:
    c = BatchConfig()
    _check(lib().ants_batch_get_config(plan, C.byref(c)))
    return c


def ants_batch_plan_free(plan: int) -> None:
    lib().ants_batch_plan_free(plan)


class BatchPlan:
    """A batched persistent run over several detectors (owning wrapper).

    items: list of (lrf, params, signals, start_xyz or None); outputs are
    allocated here (xyz, E, logL, status, trace per item)."""

    def __init__(self, ctx: Context, items, cfg: BatchConfig | None = None, want_trace=False):
        import torch
        self.ctx, self.outs, self._keep = ctx, [], []
        c_items = []
        for lrf, params, sig, start in items:
            n = int(sig.shape[0])
            o = Result(torch.empty((n, 3), device=sig.device), torch.empty(n, device=sig.device),
                       torch.empty(n, device=sig.device), torch.empty(n, dtype=torch.int32, device=sig.device),
                       torch.empty((n, params.iters), dtype=torch.int16, device=sig.device) if want_trace else None)
            self.outs.append(o)
            self._keep.append((lrf, sig, start))
            c_items.append(BatchItem(lrf.handle, params, sig.data_ptr(), n, _tptr(start), o.xyz.data_ptr(),
                                     o.E.data_ptr(), o.logL.data_ptr(), o.status.data_ptr(), _tptr(o.trace)))
        self.handle = ants_batch_plan_create(ctx.handle, c_items, cfg)

    def run(self, stream=None):
        ants_batch_run(self.handle, stream)

    def autotune(self, cache_path=None, events_per_item=2048) -> BatchConfig:
        return ants_batch_autotune(self.handle, cache_path, events_per_item)

    def config(self) -> BatchConfig:
        return ants_batch_get_config(self.handle)

    def __del__(self):
        if getattr(self, "handle", None):
            ants_batch_plan_free(self.handle)
            self.handle = None


def ants_simulate_events(ctx: int, lrf: int, params: SimParams, seed: int, first_event: int, signals, truth=None,
                         stream=None) -> None:
    _check(lib().ants_simulate_events(ctx, lrf, C.byref(params), int(seed), int(first_event), int(signals.shape[0]),
                                      _tptr(signals), _tptr(truth), _stream_handle(stream)))


def simulate(ctx: Context, lrf: "Lrf", params: SimParams, n: int, seed: int, first_event: int = 0, stream=None):
    """Device signals [n, n_sensors] and truth [n, 4] (x, y, z, E)."""
    import torch
    sig = torch.empty((n, lrf.n_sensors), dtype=torch.float32, device="cuda")
    truth = torch.empty((n, 4), dtype=torch.float32, device="cuda")
    ants_simulate_events(ctx.handle, lrf.handle, params, seed, first_event, sig, truth, stream)
    return sig, truth


def ants_deviance(ctx: int, lrf: int, signals, xyz, D, stream=None) -> None:
    _check(lib().ants_deviance(ctx, lrf, _tptr(signals), int(signals.shape[0]), int(signals.shape[1]), _tptr(xyz),
                               _tptr(D), _stream_handle(stream)))


def ants_mlp_create(ctx: int, n_in: int, cfg: MlpConfig, seed: int = 0) -> int:
    h = _VP()
    _check(lib().ants_mlp_create(ctx, int(n_in), C.byref(cfg), int(seed), C.byref(h)))
    return h.value


def ants_mlp_free(mlp: int) -> None:
    lib().ants_mlp_free(mlp)


def ants_mlp_shape(mlp: int):
    a, b, c = C.c_int(), C.c_int(), C.c_long()
    _check(lib().ants_mlp_shape(mlp, C.byref(a), C.byref(b), C.byref(c)))
    return a.value, b.value, c.value


def ants_mlp_set_params(mlp: int, params) -> None:
    p = np.ascontiguousarray(np.asarray(params, dtype=np.float32))
    _check(lib().ants_mlp_set_params(mlp, p.ctypes.data, int(p.size)))


def ants_mlp_get_params(mlp: int) -> np.ndarray:
    n = ants_mlp_shape(mlp)[2]
    out = np.empty(n, dtype=np.float32)
    _check(lib().ants_mlp_get_params(mlp, out.ctypes.data, n))
    return out


def ants_mlp_forward(ctx: int, mlp: int, signals, out, start_xyz=None, E=None, bf16: int = 1, stream=None) -> None:
    _check(lib().ants_mlp_forward(ctx, mlp, _tptr(signals), int(signals.shape[0]), int(signals.shape[1]), int(bf16),
                                  _tptr(out), _tptr(start_xyz), _tptr(E), _stream_handle(stream)))


def ants_mlp_loss_grad(ctx: int, mlp: int, signals, truth, bf16: int = 0):
    """Returns (loss, grads as one float32 vector in parameter order)."""
    n = ants_mlp_shape(mlp)[2]
    g = np.empty(n, dtype=np.float32)
    loss = C.c_float()
    _check(lib().ants_mlp_loss_grad(ctx, mlp, _tptr(signals), _tptr(truth), int(signals.shape[0]),
                                    int(signals.shape[1]), int(bf16), C.byref(loss), g.ctypes.data))
    return float(loss.value), g


def ants_mlp_train(ctx: int, mlp: int, signals, truth, params: TrainParams) -> TrainReport:
    rep = TrainReport()
    _check(lib().ants_mlp_train(ctx, mlp, _tptr(signals), _tptr(truth), int(signals.shape[0]), int(signals.shape[1]),
                                C.byref(params), C.byref(rep)))
    return rep


def ants_mlp_save(mlp: int, path: str) -> None:
    _check(lib().ants_mlp_save(mlp, path.encode()))


def ants_mlp_load(ctx: int, path: str) -> int:
    h = _VP()
    _check(lib().ants_mlp_load(ctx, path.encode(), C.byref(h)))
    return h.value


# --------------------------------------------------------------------------
# owning wrappers
# --------------------------------------------------------------------------


class Context:
    def __init__(self, device: int = 0):
        self.handle = ants_ctx_create(device)
        self.device = device

    def __del__(self):
        if getattr(self, "handle", None):
            ants_ctx_destroy(self.handle)
            self.handle = None


class Detector:
    def __init__(self, sensor_xy, rel_gain=None):
        self.sensor_xy = np.asarray(sensor_xy, dtype=np.float64)
        self.n_sensors = int(self.sensor_xy.shape[0])
        self.handle = ants_detector_create(self.sensor_xy, rel_gain)

    def symmetry(self, tol: float = 1e-3):
        """Sec. 6.2 classes by rotation and reflection symmetry: (class, operation, n_classes, centre)."""
        return ants_sensor_symmetry(self.handle, self.n_sensors, tol)

    def rings(self, tol: float = 1e-3):
        """Sec. 6.2 grouping by distance from the array's centre: (group of each sensor, number of groups)."""
        return ants_sensor_rings(self.handle, self.n_sensors, tol)

    def __del__(self):
        if getattr(self, "handle", None):
            ants_detector_free(self.handle)
            self.handle = None


class Lrf:
    """An LRF set living on the context's device."""

    def __init__(self, ctx: Context, det: Detector, handle: int, type: int):
        self.ctx, self.det, self.handle, self.type = ctx, det, handle, type
        self.n_sensors = det.n_sensors
        self.shared = False

    @classmethod
    def from_coefficients(cls, ctx, det, type, n_int, lo, hi, coef, shared=False, gain=None):
        L = cls(ctx, det, ants_lrf_create(ctx.handle, det.handle, type, n_int, lo, hi, shared, coef, gain), type)
        L.shared = bool(shared)
        return L

    @classmethod
    def from_groups(cls, ctx, det, n_int, lo, hi, group, coef, gain=None):
        """A grouped RADIAL set (ants_lrf_create_grouped): one profile per group, per-sensor gains."""
        return cls(ctx, det, ants_lrf_create_grouped(ctx.handle, det.handle, n_int, lo, hi, group, coef, gain),
                   ANTS_LRF_RADIAL)

    @classmethod
    def from_symmetry(cls, ctx, det, n_int, lo, hi, classes, ops, centre, coef, gain=None):
        """An XY set with symmetry classes (ants_lrf_create_symmetric)."""
        return cls(ctx, det, ants_lrf_create_symmetric(ctx.handle, det.handle, n_int, lo, hi, classes, ops, centre,
                                                       coef, gain), ANTS_LRF_XY)

    @classmethod
    def fit_symmetric(cls, ctx, det, n_int, lo, hi, classes, ops, centre, pts, vals, gain=None, ridge=0.0):
        """XY symmetry-class LRFs fitted on the device (ants_lrf_fit_symmetric)."""
        return cls(ctx, det, ants_lrf_fit_symmetric(ctx.handle, det.handle, n_int, lo, hi, classes, ops, centre, pts,
                                                    vals, gain, ridge), ANTS_LRF_XY)

    @classmethod
    def fit(cls, ctx, det, type, n_int, lo, hi, pts, vals, shared=False, ridge=0.0):
        h, lam = ants_lrf_fit(ctx.handle, det.handle, type, n_int, lo, hi, shared, pts, vals, ridge)
        L = cls(ctx, det, h, type)
        L.ridge_used = lam
        L.shared = bool(shared)
        return L

    @classmethod
    def from_scheme(cls, ctx, det, type, n_int, lo, hi, coef, n_int_r=0, hi_r=0.0, n_planes=0):
        """A composite, axial+z or sliced set from coefficients (ants_lrf_create_scheme)."""
        return cls(ctx, det, ants_lrf_create_scheme(ctx.handle, det.handle, type, n_int, lo, hi, coef, n_int_r, hi_r,
                                                    n_planes), type)

    @classmethod
    def fit_scheme(cls, ctx, det, type, n_int, lo, hi, pts, vals, n_int_r=0, hi_r=0.0, n_planes=0, ridge=0.0):
        """A composite, axial+z or sliced set fitted on the device (ants_lrf_fit_scheme)."""
        return cls(ctx, det, ants_lrf_fit_scheme(ctx.handle, det.handle, type, n_int, lo, hi, pts, vals, n_int_r, hi_r,
                                                 n_planes, ridge), type)

    @classmethod
    def load(cls, ctx, det, path):
        h = ants_lrf_load(ctx.handle, det.handle, path)
        L = cls(ctx, det, h, 0)
        return L

    def save(self, path):
        ants_lrf_save(self.handle, path)

    def coefficients(self) -> np.ndarray:
        return ants_lrf_coefficients(self.handle)

    def gains(self) -> np.ndarray:
        return ants_lrf_gains(self.handle, self.n_sensors)

    def refit(self, signals, xyz, E, index=None, n_kept=None, shared=None, refit_gains=False, shift_sigma=0.0,
              seed=0, cycle=0, ridge=0.0) -> "Lrf":
        """A new LRF set fitted to reconstructed events (ants_lrf_refit);
        shared=None keeps this set's grouping."""
        sh = self.shared if shared is None else bool(shared)
        p = RefitParams(int(sh), int(refit_gains), float(shift_sigma), int(seed), int(cycle), float(ridge))
        n = signals.shape[0] if index is None else (index.shape[0] if n_kept is None else n_kept)
        L = Lrf(self.ctx, self.det, ants_lrf_refit(self.ctx.handle, self.handle, signals, xyz, E, index, n, p),
                self.type)
        L.shared = sh
        return L

    def iterate(self, signals, cgs, cycles: int, cuts: EventCuts | None = None, refit_gains=False,
                shift_sigma=0.0, shift_cycles=0, seed=0, ridge=0.0):
        """Iterative LRF reconstruction (ants_lrf_iterate): (new Lrf, per-cycle stats).  cgs: CgsParams
        (contracting grids every cycle) or MinimizeParams (the continuous minimisation)."""
        mini = isinstance(cgs, MinimizeParams)
        p = IterParams(CgsParams() if mini else cgs, int(cycles), cuts if cuts is not None else EventCuts(),
                       int(refit_gains), float(shift_sigma), int(shift_cycles), int(seed), float(ridge),
                       ANTS_MINIMIZE if mini else ANTS_CGS_PLAIN, cgs if mini else MinimizeParams())
        p._keep = cgs
        h, stats = ants_lrf_iterate(self.ctx.handle, self.handle, signals, p)
        L = Lrf(self.ctx, self.det, h, self.type)
        L.shared = self.shared
        return L, stats

    def eval(self, pts, stream=None):
        import torch
        out = torch.empty((pts.shape[0], self.n_sensors), dtype=torch.float32, device=pts.device)
        ants_lrf_eval(self.handle, pts, out, stream)
        return out

    def __del__(self):
        if getattr(self, "handle", None):
            ants_lrf_free(self.handle)
            self.handle = None


class Mlp:
    """The learned proposal network (owning wrapper)."""

    def __init__(self, ctx: Context, handle: int):
        self.ctx, self.handle = ctx, handle
        self.n_in, self.n_hidden, self.n_params = ants_mlp_shape(handle)

    @classmethod
    def create(cls, ctx: Context, n_in: int, n_hidden: int, xy_scale: float, loge_mean: float, loge_std: float,
               seed: int = 2001):
        cfg = MlpConfig(n_hidden, xy_scale, loge_mean, loge_std)
        return cls(ctx, ants_mlp_create(ctx.handle, n_in, cfg, seed))

    @classmethod
    def load(cls, ctx: Context, path: str):
        return cls(ctx, ants_mlp_load(ctx.handle, path))

    def save(self, path: str):
        ants_mlp_save(self.handle, path)

    def params(self) -> np.ndarray:
        return ants_mlp_get_params(self.handle)

    def set_params(self, p):
        ants_mlp_set_params(self.handle, p)

    def train(self, signals, truth, params: TrainParams | None = None) -> TrainReport:
        return ants_mlp_train(self.ctx.handle, self.handle, signals, truth, params or TrainParams())

    def forward(self, signals, bf16: int = 1, stream=None):
        import torch
        n = signals.shape[0]
        out = torch.empty((n, 3), dtype=torch.float32, device=signals.device)
        xyz = torch.empty((n, 3), dtype=torch.float32, device=signals.device)
        E = torch.empty(n, dtype=torch.float32, device=signals.device)
        ants_mlp_forward(self.ctx.handle, self.handle, signals, out, xyz, E, bf16=bf16, stream=stream)
        return out, xyz, E

    def __del__(self):
        if getattr(self, "handle", None):
            ants_mlp_free(self.handle)
            self.handle = None


def seeded_params(mlp: Mlp, refine: CgsParams, fallback: CgsParams, deviance_max: float = 0.0,
                  border_fallback: bool = True, bf16: int = 1) -> SeededParams:
    return SeededParams(mlp.handle, int(bf16), refine, fallback, float(deviance_max), 1 if border_fallback else 0)


@dataclass
class Result:
    xyz: object
    E: object
    logL: object
    status: object
    trace: object = None


def ants_lrf_create_grouped(ctx: int, det: int, n_int, lo, hi, group, coef, gain=None) -> int:
    g = np.ascontiguousarray(np.asarray(group, dtype=np.int32))
    c = np.ascontiguousarray(np.asarray(coef, dtype=np.float64))
    gn = None if gain is None else np.ascontiguousarray(np.asarray(gain, dtype=np.float64))
    ni = (C.c_int * 1)(int(n_int[0]))
    lo_ = (C.c_double * 1)(float(lo[0]))
    hi_ = (C.c_double * 1)(float(hi[0]))
    h = _VP()
    _check(lib().ants_lrf_create_grouped(ctx, det, ni, lo_, hi_, int(c.shape[0]), g.ctypes.data_as(_IP),
                                         c.ctypes.data_as(_DP), None if gn is None else gn.ctypes.data_as(_DP),
                                         C.byref(h)))
    return h.value


def ants_lrf_create_symmetric(ctx: int, det: int, n_int, lo, hi, classes, ops, centre, coef, gain=None) -> int:
    cl = np.ascontiguousarray(np.asarray(classes, dtype=np.int32))
    op = np.ascontiguousarray(np.asarray(ops, dtype=np.int32))
    c = np.ascontiguousarray(np.asarray(coef, dtype=np.float64))
    ce = np.ascontiguousarray(np.asarray(centre, dtype=np.float64))
    gn = None if gain is None else np.ascontiguousarray(np.asarray(gain, dtype=np.float64))
    ni = (C.c_int * 2)(int(n_int[0]), int(n_int[1]))
    lo_ = (C.c_double * 2)(float(lo[0]), float(lo[1]))
    hi_ = (C.c_double * 2)(float(hi[0]), float(hi[1]))
    h = _VP()
    _check(lib().ants_lrf_create_symmetric(ctx, det, ni, lo_, hi_, int(c.shape[0]), cl.ctypes.data_as(_IP),
                                           op.ctypes.data_as(_IP), ce.ctypes.data_as(_DP), c.ctypes.data_as(_DP),
                                           None if gn is None else gn.ctypes.data_as(_DP), C.byref(h)))
    return h.value


def ants_lrf_fit_symmetric(ctx: int, det: int, n_int, lo, hi, classes, ops, centre, pts, vals, gain=None,
                           ridge=0.0) -> int:
    cl = np.ascontiguousarray(np.asarray(classes, dtype=np.int32))
    op = np.ascontiguousarray(np.asarray(ops, dtype=np.int32))
    ce = np.ascontiguousarray(np.asarray(centre, dtype=np.float64))
    p = np.ascontiguousarray(np.asarray(pts, dtype=np.float64))
    v = np.ascontiguousarray(np.asarray(vals, dtype=np.float64))
    gn = None if gain is None else np.ascontiguousarray(np.asarray(gain, dtype=np.float64))
    ni = (C.c_int * 2)(int(n_int[0]), int(n_int[1]))
    lo_ = (C.c_double * 2)(float(lo[0]), float(lo[1]))
    hi_ = (C.c_double * 2)(float(hi[0]), float(hi[1]))
    h = _VP()
    _check(lib().ants_lrf_fit_symmetric(ctx, det, ni, lo_, hi_, int(cl.max()) + 1, cl.ctypes.data_as(_IP),
                                        op.ctypes.data_as(_IP), ce.ctypes.data_as(_DP), p.shape[0],
                                        p.ctypes.data_as(_DP), v.ctypes.data_as(_DP),
                                        None if gn is None else gn.ctypes.data_as(_DP), float(ridge), C.byref(h)))
    return h.value


def ants_sensor_symmetry(det: int, n_sensors: int, tol: float):
    """(class of each sensor, its operation, number of classes, centre)."""
    cl = np.empty(n_sensors, dtype=np.int32)
    op = np.empty(n_sensors, dtype=np.int32)
    ce = np.empty(2)
    k = C.c_int()
    _check(lib().ants_sensor_symmetry(det, float(tol), cl.ctypes.data_as(_IP), op.ctypes.data_as(_IP),
                                      ce.ctypes.data_as(_DP), C.byref(k)))
    return cl, op, k.value, (float(ce[0]), float(ce[1]))


def ants_sensor_rings(det: int, n_sensors: int, tol: float):
    """(group of each sensor, number of groups) by distance from the array's centre."""
    g = np.empty(n_sensors, dtype=np.int32)
    k = C.c_int()
    _check(lib().ants_sensor_rings(det, float(tol), g.ctypes.data_as(_IP), C.byref(k)))
    return g, k.value


def ants_trace_photons(ctx: int, params: OpticsParams, src_xyz, n_photons: int, seed: int, precision: int, counts,
                       outcome=None, eta=None, stream=None) -> None:
    _check(lib().ants_trace_photons(ctx, C.addressof(params), _tptr(src_xyz), int(src_xyz.shape[0]), int(n_photons),
                                    int(seed), int(precision), _tptr(counts), _tptr(outcome), _tptr(eta),
                                    _stream_handle(stream)))


def trace_photons(ctx: Context, params: OpticsParams, src_xyz, n_photons: int, seed: int, fp64: bool = False,
                  want_outcome: bool = False, want_eta: bool = False, stream=None):
    """ants_trace_photons: photons from every source of src_xyz (torch [n_src, 3]
    float32 on the device); returns counts [n_src, n_sensors] int32 and, on
    request, the outcomes [n_src, n_photons] int16 and eta = counts / n_photons."""
    import torch
    n_src = int(src_xyz.shape[0])
    dev = src_xyz.device
    counts = torch.empty((n_src, params.n_sensors), dtype=torch.int32, device=dev)
    outcome = torch.empty((n_src, n_photons), dtype=torch.int16, device=dev) if want_outcome else None
    eta = torch.empty((n_src, params.n_sensors), dtype=torch.float32, device=dev) if want_eta else None
    ants_trace_photons(ctx.handle, params, src_xyz, n_photons, seed, ANTS_F64 if fp64 else ANTS_F32, counts, outcome,
                       eta, stream)
    return counts, outcome, eta


def reconstruct(ctx: Context, lrf: Lrf, params: CgsParams, signals, start_xyz=None, want_trace=False,
                stream=None, method: int = ANTS_CGS_PLAIN) -> Result:
    """Reconstruct device-resident signals [n, n_sensors] (torch float32 or float16)."""
    import torch
    n = int(signals.shape[0])
    dev = signals.device
    xyz = torch.empty((n, 3), dtype=torch.float32, device=dev)
    E = torch.empty(n, dtype=torch.float32, device=dev)
    logL = torch.empty(n, dtype=torch.float32, device=dev)
    status = torch.empty(n, dtype=torch.int32, device=dev)
    iters = (params.refine.iters if isinstance(params, (SeededParams, GemmParams))
             else params.grid.iters if isinstance(params, VariantParams)
             else 1 if isinstance(params, MinimizeParams) else params.iters)
    trace = torch.empty((n, iters), dtype=torch.int16, device=dev) if want_trace else None
    n_s = int(signals.shape[1]) if signals.dim() == 2 else -1
    dtype = _signal_dtype_of(signals)
    ants_reconstruct(ctx.handle, lrf.handle, method, params, signals, n_s, xyz, E, logL, status,
                     start_xyz=start_xyz, trace=trace, stream=stream, signal_dtype=dtype)
    return Result(xyz, E, logL, status, trace)


def reconstruct_host_noalloc(ctx: Context, lrf: Lrf, params: CgsParams, signals: np.ndarray, start_xyz=None,
                             method: int = ANTS_CGS_PLAIN) -> Result:
    """The plain search of reconstruct_host (FP32 signals) without any device
    allocation: signals and results pass through the library's static staging
    area, so the batch must fit it (ANTS_NOALLOC_STAGE_BYTES)."""
    n = int(signals.shape[0])
    xyz = np.empty((n, 3), dtype=np.float32)
    E = np.empty(n, dtype=np.float32)
    logL = np.empty(n, dtype=np.float32)
    status = np.empty(n, dtype=np.int32)
    n_s = int(signals.shape[1]) if signals.ndim == 2 else -1
    if _signal_dtype_of(signals) != ANTS_F32:
        raise TypeError("reconstruct_host_noalloc reads float32 signals only")
    ants_reconstruct_host_noalloc(ctx.handle, lrf.handle, method, params, signals, n_s, xyz, E, logL, status,
                                  start_xyz=start_xyz)
    return Result(xyz, E, logL, status)


def reconstruct_host(ctx: Context, lrf: Lrf, params: CgsParams, signals: np.ndarray, start_xyz=None,
                     method: int = ANTS_CGS_PLAIN) -> Result:
    """Reconstruct host-resident signals (numpy float32/float16 or pinned torch CPU tensor); synchronous."""
    n = int(signals.shape[0])
    xyz = np.empty((n, 3), dtype=np.float32)
    E = np.empty(n, dtype=np.float32)
    logL = np.empty(n, dtype=np.float32)
    status = np.empty(n, dtype=np.int32)
    n_s = int(signals.shape[1]) if signals.ndim == 2 else -1
    dtype = _signal_dtype_of(signals)
    ants_reconstruct_host(ctx.handle, lrf.handle, method, params, signals, n_s, xyz, E, logL, status,
                          start_xyz=start_xyz, signal_dtype=dtype)
    return Result(xyz, E, logL, status)
