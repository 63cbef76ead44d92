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


def test_symmetry_matches_oracle():
    import paper_1602_07247_gb300 as ants
    rect = np.array([[x, y] for y in (-2.0, 2.0) for x in (-6.0, -2.0, 2.0, 6.0)])
    arrays = [synth.workloads.get("hex19_radial").sensor_xy, synth.square_array(8, 6.0), rect,
              np.random.default_rng(4).uniform(-20, 20, (12, 2))]
    for sxy in arrays:
        det = ants.Detector(sxy)
        cl, op, k, c = det.symmetry(1e-6)
        clo, opo, ko, co = oracle.sensor_symmetry(sxy, 1e-6)
        assert k == ko and np.array_equal(cl, clo) and np.array_equal(op, opo)
        assert np.allclose(c, co, atol=1e-12)
