"""The synthetic workloads: detector, LRF knot grid, search grid, event recipe.

Numbers only; no reconstruction arithmetic.  Each workload stands in for a
detector class the paper discusses (Sec. 1, 3.3: PMT Anger cameras with
hexagonal arrays, SiPM cameras with square arrays); none of the paper's
datasets exists here.
"""
from __future__ import annotations

from dataclasses import dataclass, field, replace

import numpy as np

from . import (draw_events, eta_axial, grid_samples, hex_array, sensor_gains, square_array,
               truth_eta)


@dataclass
class Workload:
    name: str
    sensor_xy: np.ndarray
    gains: np.ndarray          # true relative gains (COG weights; baked into XY LRFs)
    lrf_type: str              # 'radial' | 'xy' | 'xyz'
    n_int: tuple
    lo: tuple
    hi: tuple
    shared: bool               # radial: one LRF for all sensors ("one group")
    n_xy: int                  # contracting grid: nodes per axis
    iters: int
    step_xy: float             # first grid's node spacing (mm)
    shrink: float = 0.5
    n_z: int = 1
    step_z: float = 0.0
    z0: float = 0.0
    n_events: int = 10_000
    event_seed: int = 1001
    event: dict = field(default_factory=dict)

    @property
    def n_sensors(self) -> int:
        return int(self.sensor_xy.shape[0])

    def fit_samples(self, per_interval: int = 4):
        """Noise-free samples of the truth LRF on a dense tensor grid:
        (points [n_pts, d], values [n_pts, n_sets])."""
        dims = {"radial": 1, "xy": 2, "xyz": 3}[self.lrf_type]
        pts = grid_samples(self.n_int[:dims], self.lo[:dims], self.hi[:dims], per_interval)
        if self.lrf_type == "radial":
            vals = eta_axial(pts[:, 0])[:, None]
            if not self.shared:
                vals = vals * self.gains[None, :]
            return pts, vals
        return pts, truth_eta(self.sensor_xy, self.gains, pts)

    def events(self, n: int | None = None, seed: int | None = None):
        n = self.n_events if n is None else n
        seed = self.event_seed if seed is None else seed
        return draw_events(self.sensor_xy, self.gains, n, seed, **self.event)

    def with_(self, **kw) -> "Workload":
        return replace(self, **kw)


def hex19_radial() -> Workload:
    """19 PMTs, hexagonal, pitch 30 mm; one axial LRF (20 intervals on
    [0, 150] mm); 10^4 events in a 60 mm disk, E = 1e4 +- 5 %, Poisson
    photo-electrons with a normal single-p.e. response (sigma 10 %);
    contracting grid 9 x 9, 6 grids, shrink 0.5, first spacing 7.5 mm."""
    sxy = hex_array(2, 30.0)
    return Workload(
        name="hex19_radial", sensor_xy=sxy, gains=np.ones(sxy.shape[0]), lrf_type="radial",
        n_int=(20,), lo=(0.0,), hi=(150.0,), shared=True, n_xy=9, iters=6, step_xy=7.5,
        n_events=10_000, event_seed=1000,
        event=dict(region="disk", extent=60.0, e0=1.0e4, spe_sigma=0.1))


def sipm8x8_xy() -> Workload:
    """8 x 8 SiPMs, pitch 6 mm; per-sensor XY LRFs (24 x 24 intervals over
    48 x 48 mm) of the truth LRF times a gain jitter N(1, 0.05^2);
    10^6 events uniform over the sensor area, E = 3000 +- 5 %, Poisson;
    contracting grid 11 x 11, 8 grids, first spacing 4.8 mm (the first grid
    spans the whole field of view: the COG of so broad an LRF sits far from
    the source, 13 mm RMS)."""
    sxy = square_array(8, 6.0)
    return Workload(
        name="sipm8x8_xy", sensor_xy=sxy, gains=sensor_gains(64, 0.05, 102), lrf_type="xy",
        n_int=(24, 24), lo=(-24.0, -24.0), hi=(24.0, 24.0), shared=False, n_xy=11, iters=8,
        step_xy=4.8, n_events=1_000_000, event_seed=1001,
        event=dict(region="square", extent=21.0, e0=3000.0))


def sipm16x16_xy() -> Workload:
    """16 x 16 SiPMs, pitch 3.2 mm; per-sensor XY LRFs (32 x 32 intervals
    over 51.2 x 51.2 mm); 4 x 10^6 events, E = 2000 +- 5 %, Poisson; plain
    contracting grid 11 x 11, 8 grids, first spacing 5.12 mm (first grid spans
    the field of view)."""
    sxy = square_array(16, 3.2)
    return Workload(
        name="sipm16x16_xy", sensor_xy=sxy, gains=sensor_gains(256, 0.05, 103), lrf_type="xy",
        n_int=(32, 32), lo=(-25.6, -25.6), hi=(25.6, 25.6), shared=False, n_xy=11, iters=8,
        step_xy=5.12, n_events=4_000_000, event_seed=1002,
        event=dict(region="square", extent=24.0, e0=2000.0))


def sipm4x4_xyz() -> Workload:
    """Small 3D case: 4 x 4 SiPMs, pitch 6 mm; per-sensor XYZ LRFs of the
    depth-dependent truth (8 x 8 x 4 intervals over 24 x 24 x 20 mm); sources
    uniform in x, y and z; contracting grid 7 x 7 x 5, 5 grids."""
    sxy = square_array(4, 6.0)
    return Workload(
        name="sipm4x4_xyz", sensor_xy=sxy, gains=sensor_gains(16, 0.05, 104), lrf_type="xyz",
        n_int=(8, 8, 4), lo=(-12.0, -12.0, 0.0), hi=(12.0, 12.0, 20.0), shared=False, n_xy=7, iters=5,
        step_xy=4.0, n_z=5, step_z=5.0, z0=10.0, n_events=10_000, event_seed=1004,
        event=dict(region="square", extent=9.0, e0=3000.0, z_range=(0.0, 20.0)))


WORKLOADS = {w().name: w for w in (hex19_radial, sipm8x8_xy, sipm16x16_xy, sipm4x4_xyz)}


def batch8_xyz() -> list:
    """Eight detectors with depth-dependent (XYZ) LRFs for one batched run:
    hexagonal PMT arrays of 19/37/61/91/127 at pitch 30 mm and square SiPM
    arrays 8 x 8 at 6 mm and 2 x (16 x 16) at 3.2 mm.  LRFs: 16 x 16 x 8
    intervals over the field of view x z in [0, 20] mm; sources uniform over
    the sensor area and in z; contracting grid 7 x 7 x 5, 7 grids.  Event
    counts 2e5, 1e4, 6e4, 3.5e5, 3e4, 1e5, 2e6, 2.5e5 (3.0e6 in total)."""
    out = []
    hexes = ((2, 200_000), (3, 10_000), (4, 60_000), (5, 30_000), (6, 100_000))
    for k, (rings, n) in enumerate(hexes):
        sxy = hex_array(rings, 30.0)
        half = rings * 30.0 + 30.0
        out.append(Workload(
            name=f"hex{sxy.shape[0]}_xyz", sensor_xy=sxy, gains=sensor_gains(sxy.shape[0], 0.05, 110 + k),
            lrf_type="xyz", n_int=(16, 16, 8), lo=(-half, -half, 0.0), hi=(half, half, 20.0), shared=False,
            n_xy=7, iters=7, step_xy=10.0, n_z=5, step_z=5.0, z0=10.0, n_events=n, event_seed=1010 + k,
            event=dict(region="disk", extent=rings * 30.0, e0=1.0e4, z_range=(0.0, 20.0))))
    squares = ((8, 6.0, 350_000, 3000.0), (16, 3.2, 2_000_000, 2000.0), (16, 3.2, 250_000, 2000.0))
    for k, (m, pitch, n, e0) in enumerate(squares):
        sxy = square_array(m, pitch)
        half = m * pitch / 2.0
        out.append(Workload(
            name=f"sipm{m}x{m}{'ab'[k - 1] if m == 16 else ''}_xyz", sensor_xy=sxy,
            gains=sensor_gains(m * m, 0.05, 120 + k), lrf_type="xyz", n_int=(16, 16, 8), lo=(-half, -half, 0.0),
            hi=(half, half, 20.0), shared=False, n_xy=7, iters=7, step_xy=half / 3.0, n_z=5, step_z=5.0, z0=10.0,
            n_events=n, event_seed=1020 + k,
            event=dict(region="square", extent=half - pitch / 2.0, e0=e0, z_range=(0.0, 20.0))))
    order = [0, 1, 2, 5, 3, 4, 6, 7]  # sensor counts 19, 37, 61, 64, 91, 127, 256, 256
    return [out[i] for i in order]


def get(name: str) -> Workload:
    return WORKLOADS[name]()
