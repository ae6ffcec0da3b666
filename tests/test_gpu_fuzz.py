"""Seeded fuzzing of the CUDA path against the oracle: random octrees of depth
5-8 and cameras drawn to hit the special cases of the exact traversal — rays
along an axis (two direction components zero), along face and space diagonals
(ties on two and three axes), dyadic slopes, views partly outside the box, cut
levels above the finest leaves — in every mode, FP64 and FP32 compensated.
Counts must match exactly; maps within the parity tolerances."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from parity import assert_parity
from paper_1210_8014_gb300 import amr, inputs

pytestmark = pytest.mark.gpu

N_CASES = 36
SPECIAL = [(0.0, 0.0, 1.0), (0.0, -1.0, 0.0), (1.0, 0.0, 0.0), (1.0, 1.0, 0.0), (0.0, 1.0, -1.0),
           (1.0, -1.0, 1.0), (-1.0, -1.0, -1.0), (0.5, 0.25, -1.0), (1.0, 0.125, 0.0), (0.75, -1.0, 0.375)]


def fuzz_case(k):
    rng = np.random.default_rng(9000 + k)
    depth = int(rng.integers(5, 9))
    tree = inputs.random_tree(rng, depth=depth, p_refine=float(rng.uniform(0.2, 0.4)))
    w = SPECIAL[k % len(SPECIAL)] if k < 2 * len(SPECIAL) else tuple(inputs.random_direction(rng))
    fov = float(2.0 ** rng.uniform(-6, 0.5))
    centre = tuple(rng.uniform(-0.2, 1.2, 3)) if k % 3 == 0 else tuple(rng.uniform(0.3, 0.7, 3))
    n = (int(rng.integers(17, 60)), int(rng.integers(9, 45)))
    L = -1 if k % 4 == 0 else int(rng.integers(2, depth + 1))
    cams = []
    for mode in (0, 1, 2, 3):
        cams.append(inputs.camera_along(w, centre=centre, fov=fov, n=n, max_level=L, mode=mode))
    return tree, cams


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return 0


@pytest.mark.parametrize("k", range(N_CASES))
def test_fuzz_against_oracle(gpu, k):
    tree, cams = fuzz_case(k)
    with amr.Renderer(tree) as r:
        for cam in cams:
            # centres in [-0.2, 1.2] and fov <= 2^0.5 keep every pixel centre in [-1, 2]^3
            ref, rc = oracle.render(tree, cam)
            for p in (amr.AMR_PREC_FP64, amr.AMR_PREC_FP32_KAHAN):
                m, c = r.render(cam.with_(precision=p))
                torch.cuda.synchronize()
                assert_parity(cam.mode, p, m.cpu().numpy(), c.cpu().numpy(), ref, rc, field_is_f32=False,
                              ctx=f"fuzz case {k} mode {cam.mode} prec {p}")
