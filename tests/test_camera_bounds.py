"""Every camera of the five workloads keeps its pixel centres in [-1, 2]^3, the
range that bounds every exact traversal product below 2^62 (|X0 - F| < 2^38,
|D| <= 2^23, and a cross-product sums two such terms), and its direction
quantises to a largest component of exactly 2^23."""
import math

import numpy as np

from oracle import bruteforce as bf
from paper_1210_8014_gb300 import inputs


def _fake_tree(normal=(0.0, 0.0, 1.0)):
    t = inputs.complete_tree(1, 1.0)
    t.info["normal"] = list(normal)
    return t


def corners_ok(cam):
    for i in (0, cam.nx - 1):
        for j in (0, cam.ny - 1):
            X0 = bf.origin(cam, i, j)
            if not all(-(1 << 36) <= x <= 2 * (1 << 36) for x in X0):
                return False
    D = bf.quantised_direction(cam)
    return int(np.abs(D).max()) == 1 << 23


def test_all_workload_cameras_within_the_product_bound():
    rng = np.random.default_rng(0)
    normal = inputs.random_direction(rng)
    t = _fake_tree(normal)
    cams = inputs.tiny_workload()[1]
    cams += inputs.galaxy_precision_cameras(t)
    cams += inputs.batch_cameras(t)
    cams += inputs.zoom_cameras(t)
    cams += [c for _, c in inputs.request_stream(t, duration_s=60.0)]
    cams.append(inputs.deep_centre_camera(t))
    assert len(cams) > 3000
    bad = [k for k, c in enumerate(cams) if not corners_ok(c)]
    assert not bad, bad[:5]
    # the bound itself: worst |X0 - F| times worst |D|, twice
    assert 2 * ((1 << 38) * (1 << 23)) <= 1 << 62
    assert math.log2(3 * (1 << 36) * (1 << 23) * 2) < 62
