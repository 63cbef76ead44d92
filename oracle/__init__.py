"""FP64 CPU oracle for ANTS2 maximum-likelihood reconstruction.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the CPU
baseline leg of ``bench.py`` are the only users.  The product library never
imports, links or runs anything here, and this package imports nothing from
the product.  The arithmetic lives in ``ants_oracle.c`` (plain C, FP64, built
with gcc without fast-math); this module only marshals numpy arrays.

Functions follow the paper (Morozov et al., arXiv:1602.07247):
  cog            Sec. 5.1.1 centroid equation
  cgs            Sec. 5.1.2 / 5.1.2.2 ML contracting grids, E = sum s / sum eta
  cgs_replay     the same search replayed along another implementation's
                 chosen nodes, with the tie-certification rule
  lrf_fit        Sec. 6 B-spline LRFs fitted to (position, value) data
  lrf_eval       Sec. 6.1.1 / 6.1.2 axial, XY and XYZ LRFs, Sec. 6.2 grouping
  bspline_*      uniform cubic B-spline basis (Cox-de Boor)
  cgs_variant(_replay)
                 Sec. 5.1.2 / 5.3 search variants: least squares, strongest-
                 sensor start, sensor cuts, passive sensors
  chi2_at, event_filter
                 Sec. 5.2 reconstruction chi-squared and event cuts
  shift_xy, lrf_refit, gain_refit, centroid_lrf, lrf_iterate
                 Sec. 8 iterative LRF reconstruction, Sec. 6.2 / 6.3 groups
                 and their relative gains
Parity pins live in tests/test_oracle_*.py.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ants_oracle.c")

RADIAL, XY, XYZ = 1, 2, 3
COMPOSITE, AXIAL_Z, SLICED = 4, 5, 6   # Sec. 6.1.1, 6.1.2 parameterisation schemes
EVT_OK, EVT_ZERO_SIGNAL, EVT_BAD_SIGNAL, EVT_OUT_OF_DOMAIN = 0, 2, 3, 4
TAU_REL = 8.0 * 2.0 ** -24


def _so_path(mutant: int = 0) -> str:
    name = "liboracle.so" if mutant == 0 else f"liboracle_m{mutant}.so"
    return os.path.join(_HERE, "_build", name)


def build(mutant: int = 0, force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math, OpenMP when present)."""
    out = _so_path(mutant)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(_SRC):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    base = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", f"-DOR_MUTANT={mutant}"]
    tmp = out + f".tmp{os.getpid()}"
    cmd = base + ["-fopenmp", _SRC, "-o", tmp, "-lm"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:  # no OpenMP runtime: build single-threaded
        r = subprocess.run(base + [_SRC, "-o", tmp, "-lm"], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + r.stderr)
    os.replace(tmp, out)
    return out


_libs: dict[int, C.CDLL] = {}


def lib(mutant: int = 0) -> C.CDLL:
    if mutant not in _libs:
        L = C.CDLL(build(mutant))
        _declare(L)
        _libs[mutant] = L
    return _libs[mutant]


class _Lrf(C.Structure):
    _fields_ = [
        ("type", C.c_int),
        ("n_sensors", C.c_int),
        ("n_int", C.c_int * 3),
        ("lo", C.c_double * 3),
        ("hi", C.c_double * 3),
        ("shared", C.c_int),
        ("coef", C.POINTER(C.c_double)),
        ("gain", C.POINTER(C.c_double)),
        ("sensor_xy", C.POINTER(C.c_double)),
        ("n_int_r", C.c_int),
        ("hi_r", C.c_double),
        ("n_planes", C.c_int),
        ("group", C.POINTER(C.c_int)),
        ("op", C.POINTER(C.c_int)),
        ("sym_c", C.c_double * 2),
    ]


class _Cgs(C.Structure):
    _fields_ = [
        ("n_xy", C.c_int),
        ("n_z", C.c_int),
        ("iters", C.c_int),
        ("shrink", C.c_double),
        ("step_xy", C.c_double),
        ("step_z", C.c_double),
        ("z0", C.c_double),
    ]


_D = C.POINTER(C.c_double)
_I = C.POINTER(C.c_int)


def _declare(L: C.CDLL) -> None:
    L.or_bspline_basis_all.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, _D]
    L.or_bspline_basis_all.restype = C.c_int
    L.or_bspline_basis4.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, _D]
    L.or_bspline_basis4.restype = C.c_int
    L.or_lrf_eval.argtypes = [C.POINTER(_Lrf), C.c_long, _D, C.c_int, _D]
    L.or_spline_eval.argtypes = [C.c_int, _I, _D, _D, _D, C.c_long, _D, _D]
    L.or_lrf_fit.argtypes = [C.c_int, _I, _D, _D, C.c_long, _D, C.c_int, _D, C.c_double, _D, _D]
    L.or_lrf_fit.restype = C.c_int
    L.or_cog.argtypes = [C.c_long, C.c_int, _D, _D, _D, _D]
    L.or_objective_at.argtypes = [C.POINTER(_Lrf), C.c_long, _D, _D, _D]
    L.or_energy_logl_at.argtypes = [C.POINTER(_Lrf), C.c_long, _D, _D, _D, _D]
    L.or_logl_at_energy.argtypes = [C.POINTER(_Lrf), _D, C.c_double, C.c_double, C.c_double, C.c_double]
    L.or_logl_at_energy.restype = C.c_double
    L.or_cgs.argtypes = [C.POINTER(_Lrf), C.POINTER(_Cgs), _D, _D, C.c_long, _D, _D, _D, _D, _I, _I]
    L.or_cgs_replay.argtypes = [C.POINTER(_Lrf), C.POINTER(_Cgs), _D, _D, C.c_long, _D, _I, C.c_double,
                                _D, _D, _D, _I, _I, _I]
    L.or_brute_force.argtypes = [C.POINTER(_Lrf), C.c_long, _D, C.c_double, C.c_double, C.c_int,
                                 C.c_double, C.c_double, C.c_int, C.c_double, _D, _D]
    L.or_num_threads.restype = C.c_int


def _d(a: np.ndarray) -> C.POINTER(C.c_double):
    return a.ctypes.data_as(_D)


def _i(a: np.ndarray) -> C.POINTER(C.c_int):
    return a.ctypes.data_as(_I)


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


# --------------------------------------------------------------------------
# data model
# --------------------------------------------------------------------------


@dataclass
class Lrf:
    """A set of LRFs: type, per-axis knot grid and FP64 coefficients.

    coef has shape [n_sets, n_coef]; n_sets is 1 for a shared radial LRF
    (Sec. 6.2 "one group"), else n_sensors.  Coefficients are stored x
    fastest, then y, then z.  gain multiplies a radial LRF per sensor.
    COMPOSITE (Sec. 6.1.1): per sensor the n_int_r + 3 coefficients of the
    axial part on [0, hi_r], then those of the XY part on the n_int / lo / hi
    box.  AXIAL_Z (Sec. 6.1.2): one spline of (r, z), axis 0 = r on [0,
    hi[0]], axis 1 = z.  SLICED (Sec. 6.1.2): per sensor n_planes XY LRFs on
    the box, planes evenly spaced from lo[2] to hi[2].
    """

    type: int
    sensor_xy: np.ndarray
    n_int: tuple
    lo: tuple
    hi: tuple
    coef: np.ndarray
    shared: bool = False
    gain: np.ndarray | None = None
    n_int_r: int = 0
    hi_r: float = 0.0
    n_planes: int = 0
    group: np.ndarray | None = None
    op: np.ndarray | None = None
    sym_c: tuple = (0.0, 0.0)
    _keep: list = field(default_factory=list, repr=False)

    @property
    def n_sensors(self) -> int:
        return int(self.sensor_xy.shape[0])

    def _struct(self) -> _Lrf:
        s = _Lrf()
        s.type = self.type
        s.n_sensors = self.n_sensors
        dims = {RADIAL: 1, XY: 2, XYZ: 3, COMPOSITE: 2, AXIAL_Z: 2, SLICED: 3}[self.type]
        s.n_int_r, s.hi_r, s.n_planes = int(self.n_int_r), float(self.hi_r), int(self.n_planes)
        for a in range(3):
            s.n_int[a] = int(self.n_int[a]) if a < dims and not (self.type == SLICED and a == 2) else 0
            s.lo[a] = float(self.lo[a]) if a < dims else 0.0
            s.hi[a] = float(self.hi[a]) if a < dims else 0.0
        s.shared = 1 if self.shared else 0
        coef = _f64(self.coef)
        sxy = _f64(self.sensor_xy)
        gain = _f64(self.gain) if self.gain is not None else None
        grp = np.ascontiguousarray(np.asarray(self.group, dtype=np.int32)) if self.group is not None else None
        op = np.ascontiguousarray(np.asarray(self.op, dtype=np.int32)) if self.op is not None else None
        self._keep[:] = [coef, sxy, gain, grp, op]
        s.coef = _d(coef)
        s.sensor_xy = _d(sxy)
        s.gain = _d(gain) if gain is not None else C.cast(None, _D)
        s.group = _i(grp) if grp is not None else C.cast(None, _I)
        s.op = _i(op) if op is not None else C.cast(None, _I)
        s.sym_c[0], s.sym_c[1] = float(self.sym_c[0]), float(self.sym_c[1])
        return s


@dataclass
class CgsParams:
    n_xy: int
    iters: int
    step_xy: float
    shrink: float = 0.5
    n_z: int = 1
    step_z: float = 0.0
    z0: float = 0.0

    def _struct(self) -> _Cgs:
        p = _Cgs()
        p.n_xy, p.n_z, p.iters = self.n_xy, self.n_z, self.iters
        p.shrink, p.step_xy, p.step_z, p.z0 = self.shrink, self.step_xy, self.step_z, self.z0
        return p


# --------------------------------------------------------------------------
# wrappers
# --------------------------------------------------------------------------


def bspline_basis_all(n_int: int, lo: float, hi: float, x: float, mutant: int = 0):
    B = np.zeros(n_int + 3)
    m = lib(mutant).or_bspline_basis_all(n_int, lo, hi, x, _d(B))
    return m, B


def bspline_basis4(n_int: int, lo: float, hi: float, x: float, mutant: int = 0):
    B = np.zeros(4)
    j0 = lib(mutant).or_bspline_basis4(n_int, lo, hi, x, _d(B))
    return j0, B


def spline_eval(n_int, lo, hi, coef, pts, mutant: int = 0) -> np.ndarray:
    pts = _f64(pts)
    dim = pts.shape[1]
    ni = np.ascontiguousarray(np.asarray(n_int, dtype=np.int32))
    out = np.empty(pts.shape[0])
    lib(mutant).or_spline_eval(dim, _i(ni), _d(_f64(lo)), _d(_f64(hi)), _d(_f64(coef)), pts.shape[0],
                               _d(pts), _d(out))
    return out


def lrf_fit(n_int, lo, hi, pts, vals, ridge: float = 0.0, mutant: int = 0):
    """Least-squares B-spline fit; returns (coef[n_out, n_coef], rc, lambda)."""
    pts = _f64(pts)
    if pts.ndim == 1:
        pts = pts[:, None]
    vals = _f64(vals)
    if vals.ndim == 1:
        vals = vals[:, None]
    dim = pts.shape[1]
    ni = np.ascontiguousarray(np.asarray(n_int[:dim], dtype=np.int32))
    nc = int(np.prod([n + 3 for n in ni]))
    coef = np.zeros((vals.shape[1], nc))
    lam = np.zeros(1)
    rc = lib(mutant).or_lrf_fit(dim, _i(ni), _d(_f64(lo[:dim])), _d(_f64(hi[:dim])), pts.shape[0],
                                _d(pts), vals.shape[1], _d(vals), float(ridge), _d(coef), _d(lam))
    if rc < 0:
        raise RuntimeError("oracle LRF fit failed")
    return coef, rc, float(lam[0])


def lrf_eval(lrf: Lrf, pts, mutant: int = 0) -> np.ndarray:
    pts = _f64(pts)
    s = lrf._struct()
    out = np.empty((pts.shape[0], lrf.n_sensors))
    lib(mutant).or_lrf_eval(C.byref(s), pts.shape[0], _d(pts), pts.shape[1], _d(out))
    return out


def sensor_symmetry(sensor_xy, tol: float, mutant: int = 0):
    """Sec. 6.2 grouping by the rotation and reflection symmetry of the array:
    (class of each sensor, its symmetry operation, number of classes,
    centre)."""
    sxy = _f64(sensor_xy)
    g = np.empty(sxy.shape[0], dtype=np.int32)
    op = np.empty(sxy.shape[0], dtype=np.int32)
    c = np.empty(2)
    L = lib(mutant)
    L.or_sensor_symmetry.argtypes = [C.c_int, _D, C.c_double, _I, _I, _D]
    L.or_sensor_symmetry.restype = C.c_int
    k = L.or_sensor_symmetry(sxy.shape[0], _d(sxy), float(tol), _i(g), _i(op), _d(c))
    return g, op, k, (float(c[0]), float(c[1]))


def sym_matrix(k: int) -> np.ndarray:
    """The 2 x 2 matrix of symmetry operation k (rotation by (k mod 12) x 30
    degrees, after the reflection y -> -y for k >= 12)."""
    t = (k % 12) * np.pi / 6
    c, s = np.cos(t), np.sin(t)
    if k % 3 == 0:  # exact at multiples of 90 degrees
        q = (k % 12) // 3
        c, s = (1.0, 0.0, -1.0, 0.0)[q], (0.0, 1.0, 0.0, -1.0)[q]
    f = -1.0 if k >= 12 else 1.0
    return np.array([[c, -s * f], [s, c * f]])


def lrf_fit_symmetric(sensor_xy, classes, ops, centre, n_int, lo, hi, pts, vals, gain=None, ridge: float = 0.0,
                      mutant: int = 0) -> Lrf:
    """XY LRFs of symmetry classes (Sec. 6.2) from samples: each class's LRF
    is fitted to its members' samples mapped into the representative's frame,
    M_i^T (p - c) + c, with values v_i / g_i; mapped points outside the box
    are left out.  pts [n, 2], vals [n, n_s]."""
    pts, vals = _f64(pts), _f64(vals)
    cl, op = np.asarray(classes), np.asarray(ops)
    g = np.ones(len(cl)) if gain is None else _f64(gain)
    k = int(cl.max()) + 1
    c = np.asarray(centre, dtype=np.float64)
    rows = []
    for j in range(k):
        P, V = [], []
        for i in np.nonzero(cl == j)[0]:
            M = sym_matrix(int(op[i]))
            q = (pts - c) @ M + c  # rows: M^T (p - c) + c
            inside = (q[:, 0] >= lo[0]) & (q[:, 0] <= hi[0]) & (q[:, 1] >= lo[1]) & (q[:, 1] <= hi[1])
            P.append(q[inside])
            V.append(vals[inside, i] / g[i])
        coef, _, _ = lrf_fit(tuple(n_int[:2]), tuple(lo[:2]), tuple(hi[:2]), np.concatenate(P),
                             np.concatenate(V)[:, None], ridge, mutant)
        rows.append(coef[0])
    return Lrf(XY, _f64(sensor_xy), (n_int[0], n_int[1], 0), (lo[0], lo[1], 0.0), (hi[0], hi[1], 0.0),
               np.stack(rows), gain=None if gain is None else g, group=cl.astype(np.int32), op=op.astype(np.int32),
               sym_c=(float(c[0]), float(c[1])))


def sensor_rings(sensor_xy, tol: float, mutant: int = 0):
    """Sec. 6.2 grouping by distance from the array's centre: (group of each
    sensor, number of groups); groups ordered outwards."""
    sxy = _f64(sensor_xy)
    g = np.empty(sxy.shape[0], dtype=np.int32)
    L = lib(mutant)
    L.or_sensor_rings.argtypes = [C.c_int, _D, C.c_double, _I]
    L.or_sensor_rings.restype = C.c_int
    k = L.or_sensor_rings(sxy.shape[0], _d(sxy), float(tol), _i(g))
    return g, k


def cog(sig, sensor_xy, gain=None, mutant: int = 0) -> np.ndarray:
    sig = _f64(sig)
    out = np.empty((sig.shape[0], 2))
    g = _f64(gain) if gain is not None else None
    lib(mutant).or_cog(sig.shape[0], sig.shape[1], _d(sig), _d(_f64(sensor_xy)),
                       _d(g) if g is not None else C.cast(None, _D), _d(out))
    return out


def objective_at(lrf: Lrf, sig, xyz, mutant: int = 0) -> np.ndarray:
    sig, xyz = _f64(sig), _f64(xyz)
    s = lrf._struct()
    out = np.empty(sig.shape[0])
    lib(mutant).or_objective_at(C.byref(s), sig.shape[0], _d(sig), _d(xyz), _d(out))
    return out


def energy_logl_at(lrf: Lrf, sig, xyz, mutant: int = 0):
    sig, xyz = _f64(sig), _f64(xyz)
    s = lrf._struct()
    E = np.empty(sig.shape[0])
    L = np.empty(sig.shape[0])
    lib(mutant).or_energy_logl_at(C.byref(s), sig.shape[0], _d(sig), _d(xyz), _d(E), _d(L))
    return E, L


def logl_at_energy(lrf: Lrf, s, xyz, E: float, mutant: int = 0) -> float:
    s = _f64(s)
    st = lrf._struct()
    return float(lib(mutant).or_logl_at_energy(C.byref(st), _d(s), float(xyz[0]), float(xyz[1]),
                                               float(xyz[2]), float(E)))


def _opt(a):
    return _f64(a) if a is not None else None


def _p(a):
    return _d(a) if a is not None else C.cast(None, _D)


def cgs(lrf: Lrf, params: CgsParams, sig, gain_cog=None, start_xyz=None, mutant: int = 0):
    """Plain contracting-grid ML search.  Returns dict of xyz, E, logL,
    status and trace (chosen flat node index per grid).  start_xyz [n, 3]
    replaces the COG start when given."""
    sig = _f64(sig)
    n = sig.shape[0]
    s, p = lrf._struct(), params._struct()
    xyz = np.empty((n, 3))
    E = np.empty(n)
    logL = np.empty(n)
    status = np.empty(n, dtype=np.int32)
    trace = np.empty((n, params.iters), dtype=np.int32)
    g, st = _opt(gain_cog), _opt(start_xyz)
    lib(mutant).or_cgs(C.byref(s), C.byref(p), _p(g), _p(st), n, _d(sig), _d(xyz), _d(E), _d(logL),
                       _i(status), _i(trace))
    return dict(xyz=xyz, E=E, logL=logL, status=status, trace=trace)


def cgs_replay(lrf: Lrf, params: CgsParams, sig, trace, gain_cog=None, start_xyz=None,
               tau_rel: float = TAU_REL, mutant: int = 0):
    sig = _f64(sig)
    n = sig.shape[0]
    tr = np.ascontiguousarray(np.asarray(trace, dtype=np.int32))
    s, p = lrf._struct(), params._struct()
    xyz = np.empty((n, 3))
    E = np.empty(n)
    logL = np.empty(n)
    status = np.empty(n, dtype=np.int32)
    n_tie = np.empty(n, dtype=np.int32)
    n_bad = np.empty(n, dtype=np.int32)
    g, st = _opt(gain_cog), _opt(start_xyz)
    lib(mutant).or_cgs_replay(C.byref(s), C.byref(p), _p(g), _p(st), n, _d(sig), _i(tr), float(tau_rel), _d(xyz), _d(E), _d(logL), _i(status),
                              _i(n_tie), _i(n_bad))
    return dict(xyz=xyz, E=E, logL=logL, status=status, n_tie=n_tie, n_bad=n_bad)


class _Variant(C.Structure):
    _fields_ = [("criterion", C.c_int), ("start", C.c_int), ("min_signal", C.c_double),
                ("max_distance", C.c_double), ("passive", _I)]


@dataclass
class Variant:
    """Search variant (Sec. 5.1.2, 5.3): criterion 0 maximum likelihood / 1
    least squares; start 0 centroid / 1 strongest sensor; sensors below
    min_signal or farther than max_distance from the start (when > 0) and
    passive ones are left out of the match."""

    criterion: int = 0
    start: int = 0
    min_signal: float = 0.0
    max_distance: float = 0.0
    passive: np.ndarray | None = None
    _keep: list = field(default_factory=list, repr=False)

    def _struct(self) -> _Variant:
        pas = None if self.passive is None else np.ascontiguousarray(np.asarray(self.passive, dtype=np.int32))
        self._keep[:] = [pas]
        return _Variant(int(self.criterion), int(self.start), float(self.min_signal), float(self.max_distance),
                        _i(pas) if pas is not None else C.cast(None, _I))


def _vlib(mutant=0):
    L = lib(mutant)
    if not getattr(L, "_var_declared", False):
        L.or_cgs_variant.argtypes = [C.POINTER(_Lrf), C.POINTER(_Cgs), C.POINTER(_Variant), _D, C.c_long, _D, _D,
                                     _D, _D, _I, _I]
        L.or_cgs_variant_replay.argtypes = [C.POINTER(_Lrf), C.POINTER(_Cgs), C.POINTER(_Variant), _D, C.c_long,
                                            _D, _I, C.c_double, _D, _D, _D, _I, _I, _I]
        L._var_declared = True
    return L


def cgs_variant(lrf: Lrf, params: CgsParams, sig, variant: Variant, gain=None, mutant: int = 0):
    """Contracting grids with a search variant; gain: the relative gains used
    by the start (centroid weights, strongest-sensor comparison)."""
    sig = _f64(sig)
    n = sig.shape[0]
    s, p, v = lrf._struct(), params._struct(), variant._struct()
    xyz, E, logL = np.empty((n, 3)), np.empty(n), np.empty(n)
    status = np.empty(n, dtype=np.int32)
    trace = np.empty((n, params.iters), dtype=np.int32)
    g = _opt(gain)
    _vlib(mutant).or_cgs_variant(C.byref(s), C.byref(p), C.byref(v), _p(g), n, _d(sig), _d(xyz), _d(E), _d(logL),
                                 _i(status), _i(trace))
    return dict(xyz=xyz, E=E, logL=logL, status=status, trace=trace)


def cgs_variant_replay(lrf: Lrf, params: CgsParams, sig, variant: Variant, trace, gain=None,
                       tau_rel: float = TAU_REL, mutant: int = 0):
    sig = _f64(sig)
    n = sig.shape[0]
    tr = np.ascontiguousarray(np.asarray(trace, dtype=np.int32))
    s, p, v = lrf._struct(), params._struct(), variant._struct()
    xyz, E, logL = np.empty((n, 3)), np.empty(n), np.empty(n)
    status = np.empty(n, dtype=np.int32)
    n_tie = np.empty(n, dtype=np.int32)
    n_bad = np.empty(n, dtype=np.int32)
    g = _opt(gain)
    _vlib(mutant).or_cgs_variant_replay(C.byref(s), C.byref(p), C.byref(v), _p(g), n, _d(sig), _i(tr),
                                        float(tau_rel), _d(xyz), _d(E), _d(logL), _i(status), _i(n_tie), _i(n_bad))
    return dict(xyz=xyz, E=E, logL=logL, status=status, n_tie=n_tie, n_bad=n_bad)


class _MinParams(C.Structure):
    _fields_ = [("max_iter", C.c_int), ("tol", C.c_double), ("lambda0", C.c_double), ("fit_z", C.c_int)]


@dataclass
class Minimize:
    """Continuous minimisation (Sec. 5.1.2.1): damped Fisher scoring
    (Levenberg-Marquardt) of the variant's criterion over x, y (and z for a
    3D LRF with fit_z), E profiled; at most max_iter trial steps, converged
    when an accepted step is shorter than tol (mm)."""

    max_iter: int = 30
    tol: float = 1e-3
    lambda0: float = 1e-3
    fit_z: int = 1

    def _struct(self) -> _MinParams:
        return _MinParams(int(self.max_iter), float(self.tol), float(self.lambda0), int(self.fit_z))


def _minlib(mutant=0):
    L = _vlib(mutant)
    if not getattr(L, "_min_declared", False):
        L.or_lrf_grad.argtypes = [C.POINTER(_Lrf), C.c_long, _D, C.c_int, _D]
        L.or_bspline_dbasis4.argtypes = [C.c_int, C.c_double, C.c_double, C.c_double, _D, _D]
        L.or_bspline_dbasis4.restype = C.c_int
        L.or_minimize.argtypes = [C.POINTER(_Lrf), C.POINTER(_Cgs), C.POINTER(_Variant), C.POINTER(_MinParams), _D,
                                  C.c_long, _D, _D, _D, _D, _D, _I, _I]
        L._min_declared = True
    return L


def bspline_dbasis4(n_int: int, lo: float, hi: float, x: float, mutant: int = 0):
    """(first index, B[4], dB/dx[4]) of the cubic basis at x; index -1 outside."""
    B, D = np.empty(4), np.empty(4)
    j = _minlib(mutant).or_bspline_dbasis4(int(n_int), float(lo), float(hi), float(x), _d(B), _d(D))
    return j, B, D


def lrf_grad(lrf: Lrf, pts, mutant: int = 0) -> np.ndarray:
    """Gradients (d/dx, d/dy, d/dz) of every sensor's LRF at the points:
    [n_pts, n_sensors, 3], NaN where undefined."""
    pts = _f64(pts)
    s = lrf._struct()
    out = np.empty((pts.shape[0], lrf.n_sensors, 3))
    _minlib(mutant).or_lrf_grad(C.byref(s), pts.shape[0], _d(pts), pts.shape[1], _d(out))
    return out


def minimize(lrf: Lrf, sig, variant: Variant, params: Minimize, z0: float = 0.0, start_xyz=None, gain=None,
             mutant: int = 0):
    """The continuous minimisation of every event from the variant's start
    (or start_xyz [n, 3]); returns xyz, E, logL, status and n_iter (trials
    used, negative when max_iter ran out)."""
    sig = _f64(sig)
    n = sig.shape[0]
    s, v, m = lrf._struct(), variant._struct(), params._struct()
    p = CgsParams(n_xy=1, iters=0, step_xy=0.0, z0=z0)._struct()
    xyz, E, logL = np.empty((n, 3)), np.empty(n), np.empty(n)
    status = np.empty(n, dtype=np.int32)
    n_iter = np.empty(n, dtype=np.int32)
    st = _f64(start_xyz) if start_xyz is not None else None
    g = _opt(gain)
    _minlib(mutant).or_minimize(C.byref(s), C.byref(p), C.byref(v), C.byref(m), _p(g), n, _d(sig),
                              _d(st) if st is not None else C.cast(None, _D), _d(xyz), _d(E), _d(logL), _i(status),
                              _i(n_iter))
    return dict(xyz=xyz, E=E, logL=logL, status=status, n_iter=n_iter)


_ML = 8  # layers of an optical stack, at most


class _Optics(C.Structure):
    _fields_ = [("n_layers", C.c_int), ("z", C.c_double * (_ML + 1)), ("n", C.c_double * _ML),
                ("abs_len", C.c_double * _ML), ("ray_len", C.c_double * _ML), ("n_below", C.c_double),
                ("n_above", C.c_double), ("half_x", C.c_double), ("half_y", C.c_double),
                ("p_abs", C.c_double * (_ML + 1)), ("p_spec", C.c_double * (_ML + 1)),
                ("p_diff", C.c_double * (_ML + 1)), ("n_sensors", C.c_int), ("sensor_xy", _D),
                ("sensor_size", C.c_double), ("n_sensor", C.c_double), ("qe", _D), ("n_ang", C.c_int), ("ang", _D),
                ("max_cycles", C.c_int), ("pre_reject", C.c_int)]


# photon outcomes (>= 0: the detecting sensor)
PH_ABSORBED, PH_ESCAPED, PH_MAX_CYCLES, PH_UNDETECTED, PH_REJECTED = -1, -2, -3, -4, -5


@dataclass
class Optics:
    """A stack of horizontal slabs (Sec. 4.2.3, 4.2.4, 4.2.6, 3.5): boundaries
    z[0] < ... < z[K], per layer the refractive index and the absorption and
    Rayleigh lengths (0 = none), the media below and above, the lateral
    extent, custom interface probabilities per boundary (absorb, specular,
    diffuse), square sensor windows of side sensor_size on z[0] with their
    index, QE and a relative angular response, the cycle limit and the
    pre-rejection switch."""

    z: tuple
    n: tuple
    abs_len: tuple
    ray_len: tuple
    sensor_xy: np.ndarray
    sensor_size: float
    qe: np.ndarray
    n_below: float = 1.0
    n_above: float = 1.0
    half_x: float = 1e9
    half_y: float = 1e9
    p_abs: tuple = ()
    p_spec: tuple = ()
    p_diff: tuple = ()
    n_sensor: float = 1.5
    ang: np.ndarray | None = None
    max_cycles: int = 1000
    pre_reject: int = 0
    _keep: list = field(default_factory=list, repr=False)

    def _struct(self) -> _Optics:
        K = len(self.n)
        o = _Optics()
        o.n_layers = K
        pad = lambda v, m: list(v) + [0.0] * (m - len(v))
        o.z[:] = pad(self.z, _ML + 1)
        o.n[:] = pad(self.n, _ML)
        o.abs_len[:] = pad(self.abs_len, _ML)
        o.ray_len[:] = pad(self.ray_len, _ML)
        o.n_below, o.n_above, o.half_x, o.half_y = self.n_below, self.n_above, self.half_x, self.half_y
        o.p_abs[:] = pad(self.p_abs, _ML + 1)
        o.p_spec[:] = pad(self.p_spec, _ML + 1)
        o.p_diff[:] = pad(self.p_diff, _ML + 1)
        sxy = _f64(self.sensor_xy)
        qe = _f64(self.qe)
        ang = _f64(self.ang) if self.ang is not None else None
        self._keep[:] = [sxy, qe, ang]
        o.n_sensors = sxy.shape[0]
        o.sensor_xy, o.qe = _d(sxy), _d(qe)
        o.sensor_size, o.n_sensor = self.sensor_size, self.n_sensor
        o.n_ang = 0 if ang is None else ang.shape[0]
        o.ang = _d(ang) if ang is not None else C.cast(None, _D)
        o.max_cycles, o.pre_reject = int(self.max_cycles), int(self.pre_reject)
        return o


def _olib(mutant=0):
    L = lib(mutant)
    if not getattr(L, "_opt_declared", False):
        L.or_fresnel.argtypes = [C.c_double, C.c_double, C.c_double]
        L.or_fresnel.restype = C.c_double
        L.or_rayleigh_mu.argtypes = [C.c_double]
        L.or_rayleigh_mu.restype = C.c_double
        L.or_trace_photons.argtypes = [C.POINTER(_Optics), C.c_long, _D, C.c_long, C.c_uint64, _I, _I]
        L.or_turn_dir.argtypes = [_D, C.c_double, C.c_double, _D]
        L._opt_declared = True
    return L


def fresnel(n1: float, n2: float, ci: float, mutant: int = 0) -> float:
    """Unpolarised Fresnel reflection coefficient from n1 into n2 at incidence cosine ci."""
    return _olib(mutant).or_fresnel(float(n1), float(n2), float(ci))


def rayleigh_mu(u: float, mutant: int = 0) -> float:
    """cos(theta) of the Rayleigh phase function at the CDF value u."""
    return _olib(mutant).or_rayleigh_mu(float(u))


def turn_dir(d, mu: float, phi: float, mutant: int = 0) -> np.ndarray:
    """The unit direction at angle acos(mu) from d and azimuth phi about it."""
    d = _f64(d)
    out = np.empty(3)
    _olib(mutant).or_turn_dir(_d(d), float(mu), float(phi), _d(out))
    return out


def trace_photons(optics: Optics, src_xyz, n_photons: int, seed: int, want_outcome: bool = False, mutant: int = 0):
    """n_photons photons from each source [n_src, 3]: counts [n_src, n_sensors]
    and, with want_outcome, every photon's outcome [n_src, n_photons]."""
    src = _f64(np.atleast_2d(src_xyz))
    o = optics._struct()
    counts = np.empty((src.shape[0], o.n_sensors), dtype=np.int32)
    out = np.empty((src.shape[0], n_photons), dtype=np.int32) if want_outcome else None
    _olib(mutant).or_trace_photons(C.byref(o), src.shape[0], _d(src), int(n_photons), int(seed), _i(counts),
                                   _i(out) if out is not None else C.cast(None, _I))
    return (counts, out) if want_outcome else counts


def brute_force(lrf: Lrf, sig, x_rng, nx, y_rng, ny, z=0.0, mutant: int = 0):
    sig = _f64(sig)
    n = sig.shape[0]
    s = lrf._struct()
    xy = np.empty((n, 2))
    F = np.empty(n)
    lib(mutant).or_brute_force(C.byref(s), n, _d(sig), float(x_rng[0]), float(x_rng[1]), int(nx),
                               float(y_rng[0]), float(y_rng[1]), int(ny), float(z), _d(xy), _d(F))
    return xy, F


def num_threads() -> int:
    return int(lib().or_num_threads())


def set_num_threads(n: int) -> None:
    """Threads of the following oracle calls (for timing it single-threaded)."""
    L = lib()
    L.or_set_num_threads.argtypes = [C.c_int]
    L.or_set_num_threads(int(n))


# --------------------------------------------------------------------------
# learned proposal (multilayer perceptron) and deviance
# --------------------------------------------------------------------------


class _Mlp(C.Structure):
    _fields_ = [("n_in", C.c_int), ("n_hid", C.c_int), ("n_out", C.c_int), ("W1", _D), ("b1", _D), ("W2", _D),
                ("b2", _D), ("W3", _D), ("b3", _D)]


@dataclass
class Mlp:
    """Weights of u -> GELU(W1 u + b1) -> GELU(W2 . + b2) -> W3 . + b3 (row-major [out][in])."""
    W1: np.ndarray
    b1: np.ndarray
    W2: np.ndarray
    b2: np.ndarray
    W3: np.ndarray
    b3: np.ndarray
    _keep: list = field(default_factory=list, repr=False)

    @property
    def shape(self):
        return self.W1.shape[1], self.W1.shape[0], self.W3.shape[0]

    def _struct(self) -> _Mlp:
        arrs = [_f64(a) for a in (self.W1, self.b1, self.W2, self.b2, self.W3, self.b3)]
        self._keep[:] = arrs
        s = _Mlp()
        s.n_in, s.n_hid, s.n_out = self.shape
        s.W1, s.b1, s.W2, s.b2, s.W3, s.b3 = [_d(a) for a in arrs]
        return s

    def params(self):
        return [self.W1, self.b1, self.W2, self.b2, self.W3, self.b3]


def _declare_mlp(L):
    L.or_gelu_value.argtypes = [C.c_double]
    L.or_gelu_value.restype = C.c_double
    L.or_mlp_forward.argtypes = [C.POINTER(_Mlp), C.c_long, _D, _D]
    L.or_mlp_loss_grad.argtypes = [C.POINTER(_Mlp), C.c_long, _D, _D, _D, _D, _D, _D, _D, _D]
    L.or_mlp_loss_grad.restype = C.c_double
    L.or_adam_step.argtypes = [C.c_long, _D, _D, _D, _D, C.c_int, C.c_double, C.c_double, C.c_double, C.c_double]
    L.or_deviance_at.argtypes = [C.POINTER(_Lrf), C.c_long, _D, _D, _D]


def _mlib(mutant=0):
    L = lib(mutant)
    if not getattr(L, "_mlp_declared", False):
        _declare_mlp(L)
        L._mlp_declared = True
    return L


def gelu(x: float, mutant: int = 0) -> float:
    return float(_mlib(mutant).or_gelu_value(float(x)))


def mlp_forward(mlp: Mlp, sig, mutant: int = 0) -> np.ndarray:
    """Normalise signals by their sum and run the network: [n, n_out]."""
    sig = _f64(sig)
    s = mlp._struct()
    out = np.empty((sig.shape[0], s.n_out))
    _mlib(mutant).or_mlp_forward(C.byref(s), sig.shape[0], _d(sig), _d(out))
    return out


def mlp_loss_grad(mlp: Mlp, sig, target, mutant: int = 0):
    """Mean squared error and its gradient [gW1, gb1, gW2, gb2, gW3, gb3]."""
    sig, target = _f64(sig), _f64(target)
    s = mlp._struct()
    grads = [np.zeros_like(_f64(a)) for a in mlp.params()]
    loss = _mlib(mutant).or_mlp_loss_grad(C.byref(s), sig.shape[0], _d(sig), _d(target), *[_d(g) for g in grads])
    return float(loss), grads


def adam_step(p: np.ndarray, g, m: np.ndarray, v: np.ndarray, t: int, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8,
              mutant: int = 0) -> None:
    """In-place Adam update of float64 arrays p, m, v."""
    g = _f64(g)
    for a in (p, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    _mlib(mutant).or_adam_step(p.size, _d(p), _d(g), _d(m), _d(v), int(t), lr, b1, b2, eps)


def deviance_at(lrf: Lrf, sig, xyz, mutant: int = 0) -> np.ndarray:
    """Poisson deviance 2 sum[s ln(s/mu) - (s - mu)] at the given positions (E = S/H)."""
    sig, xyz = _f64(sig), _f64(xyz)
    s = lrf._struct()
    D = np.empty(sig.shape[0])
    _mlib(mutant).or_deviance_at(C.byref(s), sig.shape[0], _d(sig), _d(xyz), _d(D))
    return D


# --------------------------------------------------------------------------
# event simulation (Philox4x32-10 + Poisson)
# --------------------------------------------------------------------------


class _Sim(C.Structure):
    _fields_ = [("region", C.c_int), ("extent", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("z_lo", C.c_double), ("z_hi", C.c_double), ("e0", C.c_double), ("e_spread", C.c_double),
                ("spe_sigma", C.c_double)]


def _slib(mutant=0):
    L = _mlib(mutant)
    if not getattr(L, "_sim_declared", False):
        L.or_philox_block.argtypes = [C.c_uint64, C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint32,
                                      C.POINTER(C.c_uint32)]
        L.or_simulate.argtypes = [C.POINTER(_Lrf), C.POINTER(_Sim), C.c_uint64, C.c_long, C.c_long, _D, _D]
        L.or_poisson_draws.argtypes = [C.c_double, C.c_uint64, C.c_long, _D]
        L._sim_declared = True
    return L


def philox(seed: int, ctr, mutant: int = 0) -> np.ndarray:
    out = (C.c_uint32 * 4)()
    _slib(mutant).or_philox_block(int(seed), *[int(c) & 0xFFFFFFFF for c in ctr], out)
    return np.array(list(out), dtype=np.uint64)


def simulate(lrf: Lrf, seed: int, first_event: int, n: int, region="square", extent=10.0, cx=0.0, cy=0.0,
             z_lo=0.0, z_hi=0.0, e0=1000.0, e_spread=0.05, spe_sigma=0.0, mutant: int = 0):
    """Signals [n, n_s] and truth [n, 4] (x, y, z, E) of events first_event.."""
    p = _Sim(0 if region == "disk" else 1, extent, cx, cy, z_lo, z_hi, e0, e_spread, spe_sigma)
    s = lrf._struct()
    sig = np.empty((n, lrf.n_sensors))
    truth = np.empty((n, 4))
    _slib(mutant).or_simulate(C.byref(s), C.byref(p), int(seed), int(first_event), int(n), _d(sig), _d(truth))
    return sig, truth


def poisson_draws(lam: float, seed: int, n: int, mutant: int = 0) -> np.ndarray:
    out = np.empty(n)
    _slib(mutant).or_poisson_draws(float(lam), int(seed), int(n), _d(out))
    return out


def logtable(lrf: Lrf, nx: int, ny: int, mutant: int = 0):
    """T [nx*ny, n_s] = ln p_i(g) - m_i and m [n_s] (FP64)."""
    L = _mlib(mutant)
    if not getattr(L, "_lt_declared", False):
        L.or_logtable.argtypes = [C.POINTER(_Lrf), C.c_int, C.c_int, _D, _D]
        L._lt_declared = True
    s = lrf._struct()
    T = np.empty((nx * ny, lrf.n_sensors))
    m = np.empty(lrf.n_sensors)
    L.or_logtable(C.byref(s), int(nx), int(ny), _d(T), _d(m))
    return T, m


# --------------------------------------------------------------------------
# Sec. 5.2 event filters and Sec. 8 iterative LRF reconstruction
# --------------------------------------------------------------------------


class _Filter(C.Structure):
    _fields_ = [(n, C.c_double) for n in ("chi2_max", "e_lo", "e_hi", "sum_lo", "sum_hi", "r_max", "cx", "cy")]


@dataclass
class EventCuts:
    """The cuts of Sec. 5.2 used between cycles.  chi2_max and r_max are off
    when <= 0; an energy or signal-sum window is off when its upper bound is
    not above its lower bound."""

    chi2_max: float = 0.0
    e_lo: float = 0.0
    e_hi: float = 0.0
    sum_lo: float = 0.0
    sum_hi: float = 0.0
    r_max: float = 0.0
    cx: float = 0.0
    cy: float = 0.0

    def _struct(self) -> _Filter:
        return _Filter(self.chi2_max, self.e_lo, self.e_hi, self.sum_lo, self.sum_hi, self.r_max, self.cx, self.cy)


def _ilib(mutant=0):
    L = _slib(mutant)
    if not getattr(L, "_it_declared", False):
        L.or_chi2_at.argtypes = [C.POINTER(_Lrf), C.c_long, _D, _D, _D, _D]
        L.or_event_filter.argtypes = [C.c_long, _I, _D, _D, _D, _D, C.POINTER(_Filter), _I]
        L.or_shift_xy.argtypes = [C.c_uint64, C.c_int, C.c_long, C.POINTER(C.c_long), C.c_double, _D]
        L.or_gain_refit.argtypes = [C.c_int, C.c_double, C.c_double, _D, C.c_long, C.c_int, _D, _D, _D]
        L._it_declared = True
    return L


def chi2_at(lrf: Lrf, sig, xyz, E, mutant: int = 0) -> np.ndarray:
    """Reduced Pearson chi-squared of each event at (xyz, E) (Sec. 5.2)."""
    sig, xyz, E = _f64(sig), _f64(xyz), _f64(E)
    s = lrf._struct()
    out = np.empty(sig.shape[0])
    _ilib(mutant).or_chi2_at(C.byref(s), sig.shape[0], _d(sig), _d(xyz), _d(E), _d(out))
    return out


def event_filter(status, xyz, E, chi2, ssum, cuts: EventCuts, mutant: int = 0) -> np.ndarray:
    """Boolean keep mask of the Sec. 5.2 cuts."""
    st = np.ascontiguousarray(np.asarray(status, dtype=np.int32))
    xyz, E, chi2, ssum = _f64(xyz), _f64(E), _f64(chi2), _f64(ssum)
    keep = np.empty(st.shape[0], dtype=np.int32)
    f = cuts._struct()
    _ilib(mutant).or_event_filter(st.shape[0], _i(st), _d(xyz), _d(E), _d(chi2), _d(ssum), C.byref(f), _i(keep))
    return keep.astype(bool)


def shift_xy(seed: int, cycle: int, events, sigma: float, mutant: int = 0) -> np.ndarray:
    """Seeded normal offsets [k, 2] of standard deviation sigma for the given
    event indices (Sec. 8 random shift)."""
    ev = np.ascontiguousarray(np.asarray(events, dtype=np.int64))
    out = np.empty((ev.shape[0], 2))
    _ilib(mutant).or_shift_xy(int(seed), int(cycle), ev.shape[0], ev.ctypes.data_as(C.POINTER(C.c_long)),
                              float(sigma), _d(out))
    return out


def gain_refit(n_int: int, lo: float, hi: float, coef, r, v, mutant: int = 0) -> np.ndarray:
    """Least-squares relative gains with a fixed radial profile (Sec. 6.3);
    r, v: [n_e, n_s]."""
    r, v, coef = _f64(r), _f64(v), _f64(coef).ravel()
    g = np.empty(r.shape[1])
    _ilib(mutant).or_gain_refit(int(n_int), float(lo), float(hi), _d(coef), r.shape[0], r.shape[1], _d(r), _d(v),
                                _d(g))
    return g


def lrf_refit(lrf: Lrf, sig, xyz, E, shared=None, refit_gains: bool = False, ridge: float = 0.0,
              mutant: int = 0) -> Lrf:
    """LRFs refitted to the signals of reconstructed events (Sec. 6: LRFs
    from (position, signal) data; Sec. 8: the positions are reconstructed).
    Each event e gives, for every sensor i, the value v_ei = s_ei / E_e at its
    position.  XY / XYZ: one least-squares fit with the points (x, y[, z]) and
    one value column per sensor.  RADIAL grouped (Sec. 6.2): one fit of the
    profile to every (r_ei, v_ei / g_i), g_i the group's current gains; with
    refit_gains the gains are then refitted with the new profile fixed
    (Sec. 6.3) and scaled to mean 1, the profile taking the inverse factor so
    that g_i f is unchanged.  RADIAL per sensor: one fit of (r_ei, v_ei) per
    sensor, gains 1.  RADIAL with sensor groups (lrf.group): one profile per
    group, gains refitted within each group.  The knot grid is the input's;
    `shared` (default: the input's) selects grouped or per-sensor output for
    RADIAL without groups."""
    sig, xyz, E = _f64(sig), _f64(xyz), _f64(E)
    shared = lrf.shared if shared is None else bool(shared)
    v = sig / E[:, None]
    n_s = lrf.n_sensors
    if lrf.type == XY and lrf.op is not None:
        # symmetry classes: each class refitted to its members' mapped samples, gains kept
        return lrf_fit_symmetric(lrf.sensor_xy, lrf.group, lrf.op, lrf.sym_c, lrf.n_int[:2], lrf.lo[:2], lrf.hi[:2],
                                 xyz[:, :2], v, gain=lrf.gain, ridge=ridge, mutant=mutant)
    if lrf.type != RADIAL:
        dims = 2 if lrf.type == XY else 3
        coef, _, _ = lrf_fit(lrf.n_int, lrf.lo, lrf.hi, xyz[:, :dims], v, ridge, mutant)
        return Lrf(lrf.type, lrf.sensor_xy, lrf.n_int, lrf.lo, lrf.hi, coef)
    d = xyz[:, None, :2] - lrf.sensor_xy[None, :, :]
    r = np.sqrt(d[..., 0] ** 2 + d[..., 1] ** 2)
    if lrf.group is not None:
        # groups (Sec. 6.2): one profile per group from its sensors' samples
        # divided by their gains; with refit_gains each sensor's gain against
        # its group's new profile, scaled to mean 1 within the group
        grp = np.asarray(lrf.group)
        k = int(grp.max()) + 1
        g = np.ones(n_s) if lrf.gain is None else _f64(lrf.gain).copy()
        coef = np.zeros((k, lrf.n_int[0] + 3))
        for j in range(k):
            m = np.nonzero(grp == j)[0]
            coef[j], _, _ = lrf_fit(lrf.n_int, lrf.lo, lrf.hi, r[:, m].reshape(-1), (v[:, m] / g[None, m]).reshape(-1),
                                    ridge, mutant)
            if refit_gains:
                gj = gain_refit(lrf.n_int[0], lrf.lo[0], lrf.hi[0], coef[j], r[:, m], v[:, m], mutant)
                gm = gj.mean()
                g[m] = gj / gm
                coef[j] = coef[j] * gm
        return Lrf(RADIAL, lrf.sensor_xy, lrf.n_int, lrf.lo, lrf.hi, coef, gain=g, group=grp.copy())
    if not shared:
        coef = np.concatenate([lrf_fit(lrf.n_int, lrf.lo, lrf.hi, r[:, i], v[:, i], ridge, mutant)[0]
                               for i in range(n_s)])
        return Lrf(RADIAL, lrf.sensor_xy, lrf.n_int, lrf.lo, lrf.hi, coef, shared=False)
    g = np.ones(n_s) if lrf.gain is None or not lrf.shared else _f64(lrf.gain)
    coef, _, _ = lrf_fit(lrf.n_int, lrf.lo, lrf.hi, r.reshape(-1), (v / g[None, :]).reshape(-1), ridge, mutant)
    if refit_gains:
        g = gain_refit(lrf.n_int[0], lrf.lo[0], lrf.hi[0], coef, r, v, mutant)
        gm = g.mean()
        g = g / gm
        coef = coef * gm
    return Lrf(RADIAL, lrf.sensor_xy, lrf.n_int, lrf.lo, lrf.hi, coef, shared=True, gain=g.copy())


def centroid_lrf(lrf: Lrf, sig, gain_cog=None, shared=None, ridge: float = 0.0, mutant: int = 0) -> Lrf:
    """Initial LRFs without a known response (Sec. 8): every event at its
    centroid position (Sec. 5.1.1) with E = the sum of its signals, refitted
    on `lrf`'s knot grid (gains of a radial group start at 1)."""
    sig = _f64(sig)
    xy = cog(sig, lrf.sensor_xy, gain_cog, mutant)
    S = sig.sum(axis=1)
    ok = np.isfinite(xy).all(axis=1) & (S > 0)
    xyz = np.concatenate([xy, np.zeros((xy.shape[0], 1))], axis=1)
    base = Lrf(lrf.type, lrf.sensor_xy, lrf.n_int, lrf.lo, lrf.hi, lrf.coef, shared=lrf.shared,
               gain=np.ones(lrf.n_sensors) if lrf.type == RADIAL else None)
    return lrf_refit(base, sig[ok], xyz[ok], S[ok], shared, False, ridge, mutant)


def lrf_iterate(lrf0: Lrf, params, sig, cycles: int, cuts: EventCuts, shift_sigma: float = 0.0,
                shift_cycles: int = 0, seed: int = 0, refit_gains: bool = False, gain_cog=None,
                ridge: float = 0.0, mutant: int = 0):
    """Iterative LRF reconstruction from flood data (Sec. 8).  Each cycle:
    reconstruct every event with the current LRFs (params: CgsParams for the
    contracting grids, Sec. 5.1.2.2, or Minimize for the continuous
    minimisation from the centroid, Sec. 5.1.2.1), keep the events that pass
    the cuts (Sec. 5.2), offset the
    kept positions by seeded normal shifts during the first shift_cycles
    cycles, and refit the LRFs from the kept events (lrf_refit).  Returns the
    final LRFs and per-cycle statistics (events kept, their mean chi2 and
    mean energy)."""
    sig = _f64(sig)
    L = lrf0
    stats = []
    ssum = sig.sum(axis=1)
    for c in range(cycles):
        if isinstance(params, Minimize):
            r = minimize(L, sig, Variant(), params, gain=gain_cog, mutant=mutant)
        else:
            r = cgs(L, params, sig, gain_cog=gain_cog, mutant=mutant)
        chi2 = chi2_at(L, sig, r["xyz"], r["E"], mutant)
        keep = event_filter(r["status"], r["xyz"], r["E"], chi2, ssum, cuts, mutant)
        idx = np.nonzero(keep)[0]
        xyz = r["xyz"][idx].copy()
        if c < shift_cycles and shift_sigma > 0.0:
            xyz[:, :2] += shift_xy(seed, c, idx, shift_sigma, mutant)
        stats.append(dict(n_kept=int(idx.size), mean_chi2=float(chi2[idx].mean()) if idx.size else float("nan"),
                          mean_E=float(r["E"][idx].mean()) if idx.size else float("nan")))
        L = lrf_refit(L, sig[idx], xyz, r["E"][idx], None, refit_gains, ridge, mutant)
    return L, stats



# --------------------------------------------------------------------------
# Sec. 6.1.1 / 6.1.2 parameterisation schemes: fits
# --------------------------------------------------------------------------


def _dist(sensor_xy, pts):
    d = pts[:, None, :2] - sensor_xy[None, :, :]
    return np.sqrt(d[..., 0] ** 2 + d[..., 1] ** 2)


def lrf_fit_composite(sensor_xy, pts, vals, n_int_r, hi_r, n_int, lo, hi, ridge=0.0, mutant: int = 0) -> Lrf:
    """Composite LRFs (Sec. 6.1.1): per sensor the axial part is fitted first
    to (r_i, v_i); the XY part is then fitted to the residual v_i - A_i(r_i)
    on the n_int / lo / hi box (one value column per sensor; a sample beyond
    the axial part's reach, r_i > hi_r, gives a zero residual).  pts [n, 2],
    vals [n, n_s]."""
    pts, vals = _f64(pts), _f64(vals)
    r = _dist(_f64(sensor_xy), pts)
    n_s = vals.shape[1]
    ca = np.concatenate([lrf_fit((n_int_r,), (0.0,), (hi_r,), r[:, i], vals[:, i], ridge, mutant)[0]
                         for i in range(n_s)])
    res = np.stack([vals[:, i] - spline_eval((n_int_r,), (0.0,), (hi_r,), ca[i], r[:, i:i + 1], mutant)
                    for i in range(n_s)], axis=1)
    res[~np.isfinite(res)] = 0.0
    cxy, _, _ = lrf_fit(n_int[:2], lo[:2], hi[:2], pts[:, :2], res, ridge, mutant)
    coef = np.concatenate([ca, cxy], axis=1)
    return Lrf(COMPOSITE, _f64(sensor_xy), tuple(n_int[:2]) + (0,), tuple(lo[:2]) + (0.0,), tuple(hi[:2]) + (0.0,),
               coef, n_int_r=n_int_r, hi_r=hi_r)


def lrf_fit_axial_z(sensor_xy, pts, vals, n_int_rz, hi_r, z_lo, z_hi, ridge=0.0, mutant: int = 0) -> Lrf:
    """Axial+Z LRFs (Sec. 6.1.2): per sensor one spline of (r_i, z) fitted to
    its values.  pts [n, 3], vals [n, n_s]."""
    pts, vals = _f64(pts), _f64(vals)
    r = _dist(_f64(sensor_xy), pts)
    coef = np.concatenate([lrf_fit(n_int_rz, (0.0, z_lo), (hi_r, z_hi), np.stack([r[:, i], pts[:, 2]], axis=1),
                                   vals[:, i], ridge, mutant)[0] for i in range(vals.shape[1])])
    return Lrf(AXIAL_Z, _f64(sensor_xy), tuple(n_int_rz) + (0,), (0.0, z_lo, 0.0), (hi_r, z_hi, 0.0), coef)


def lrf_fit_sliced(sensor_xy, pts, vals, n_int, lo, hi, n_planes, z_lo, z_hi, ridge=0.0, mutant: int = 0) -> Lrf:
    """Sliced LRFs (Sec. 6.1.2): the XY LRFs of plane j (z_j = z_lo + j dz)
    are fitted to the samples whose nearest plane is j (reading: the paper
    names the planes, not how their samples are chosen).  pts [n, 3]."""
    pts, vals = _f64(pts), _f64(vals)
    dz = (z_hi - z_lo) / (n_planes - 1)
    plane = np.clip(np.floor((pts[:, 2] - z_lo) / dz + 0.5), 0, n_planes - 1).astype(int)
    parts = []
    for j in range(n_planes):
        sel = plane == j
        parts.append(lrf_fit(n_int[:2], lo[:2], hi[:2], pts[sel, :2], vals[sel], ridge, mutant)[0])
    coef = np.concatenate(parts, axis=1)  # [n_s, n_planes * n_coef_xy]
    return Lrf(SLICED, _f64(sensor_xy), tuple(n_int[:2]) + (0,), tuple(lo[:2]) + (z_lo,), tuple(hi[:2]) + (z_hi,),
               coef, n_planes=n_planes)
