"""Sensor grouping by distance from the array's centre (Sec. 6.2): the C ABI's
host routine against the oracle's (no GPU needed)."""
import numpy as np

import oracle
import synth
import synth.workloads


def test_rings_match_oracle():
    import paper_1602_07247_gb300 as ants
    rng = np.random.default_rng(3)
    arrays = [synth.workloads.get("hex19_radial").sensor_xy, synth.square_array(8, 6.0), synth.square_array(16, 3.2),
              rng.uniform(-30, 30, (40, 2))]
    for sxy in arrays:
        for tol in (1e-6, 0.5, 5.0):
            det = ants.Detector(sxy)
            g, k = det.rings(tol)
            go, ko = oracle.sensor_rings(sxy, tol)
            assert k == ko and np.array_equal(g, go), (sxy.shape, tol)
