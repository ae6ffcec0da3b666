"""Full-size workloads in the launch configuration bench.py times, checked on
sampled pixels against the oracle (pytest -m gpu).

- the 64-camera batch on the 16M-leaf galaxy octree (one persistent launch per
  precision, as bench.py launches it): FP32 compensated and FP64;
- the 8-frame 4096^2 zoom on the 193M-leaf level-22 octree, FP32 compensated;
- a full-depth level-22 view of the centre (512^2, fov 2^-13).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from parity import assert_parity
from paper_1210_8014_gb300 import amr, inputs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")


def sample(cam, k, rng):
    return rng.integers(0, cam.nx, k), rng.integers(0, cam.ny, k)


def check_batch(r, tree, cams, per_cam, seed):
    outs = r.render_batch(cams)
    torch.cuda.synchronize()
    prepared = oracle.prepare(tree)
    rng = np.random.default_rng(seed)
    for q, (cam, (m, c)) in enumerate(zip(cams, outs)):
        pi, pj = sample(cam, per_cam, rng)
        ref, rc = oracle.render(prepared, cam, pixels=(pi, pj))
        mh = m.cpu().numpy()[pj, pi]
        ch = c.cpu().numpy()[pj, pi]
        assert_parity(cam.mode, cam.precision, mh, ch, ref, rc, ctx=f"camera {q} ({cam.nx}^2 mode {cam.mode})")
    return outs


def test_batch_64_cameras_full_size(gpu):
    tree = inputs.batch_tree()
    cams = inputs.batch_cameras(tree)
    with amr.Renderer(tree) as r:
        check_batch(r, tree, cams, 48, seed=1)
        check_batch(r, tree, [c.with_(precision=amr.AMR_PREC_FP64) for c in cams], 24, seed=2)
        st = r.stats()
        assert st["device_errors"] == 0


def test_zoom_level22_full_size(gpu, zoom_tree):
    tree = zoom_tree
    assert tree.depth == 22 and 190e6 <= tree.n_leaves <= 210e6
    cams = inputs.zoom_cameras(tree)
    with amr.Renderer(tree) as r:
        levels = [amr.amr_camera_check(r.ctx, c) for c in cams]
        assert levels == list(range(12, 20))
        check_batch(r, tree, cams, 96, seed=3)
        deep = [inputs.deep_centre_camera(tree, mode=m) for m in (0, 2)]
        assert amr.amr_camera_check(r.ctx, deep[0]) == 22
        check_batch(r, tree, deep, 2000, seed=4)
        assert r.stats()["device_errors"] == 0


def test_serving_stream_alone_vs_mix(gpu):
    """The Poisson request stream on the 16.0M-leaf batch tree (sizes 256^2 ..
    2048^2, fov 2^-12 .. 1, mixed modes) submitted at once, so that requests
    overlap on the device, share tile-granular launches and overtake each
    other: every result equals the same camera rendered alone, bit for bit,
    and a sample of pixels matches the oracle."""
    tree = inputs.batch_tree()
    reqs = [cam for _, cam in inputs.request_stream(tree, duration_s=1.2)]
    assert len(reqs) >= 40
    with amr.Renderer(tree) as r:
        amr.amr_server_config(r.ctx, slots=3, map_budget_bytes=1 << 30, max_batch=16)
        bufs, tickets = [], []
        for k, cam in enumerate(reqs):
            if k % 3:
                m = torch.zeros((cam.ny, cam.nx), dtype=torch.float32, pin_memory=True).numpy()
                c = torch.zeros((cam.ny, cam.nx), dtype=torch.int32, pin_memory=True).numpy()
            else:                                        # pageable: staged in the server arena
                m = np.zeros((cam.ny, cam.nx), np.float32)
                c = np.zeros((cam.ny, cam.nx), np.int32)
            bufs.append((m, c))
            tickets.append(amr.amr_submit(r.ctx, cam, m, c))
        for t in tickets:
            amr.amr_wait(r.ctx, t, 120_000_000)
        st = r.stats()["server"]
        assert st["done"] == len(reqs) and st["failed"] == 0
        assert st["batches"] > len(reqs) // 2             # large requests were split across launches
        prepared = oracle.prepare(tree)
        rng = np.random.default_rng(55)
        for k, (cam, (m, c)) in enumerate(zip(reqs, bufs)):
            m1, c1 = r.render(cam)
            torch.cuda.synchronize()
            assert (m == m1.cpu().numpy()).all() and (c == c1.cpu().numpy()).all(), k
            if k % 8 == 0:
                pi, pj = sample(cam, 24, rng)
                ref, rc = oracle.render(prepared, cam, pixels=(pi, pj))
                assert_parity(cam.mode, cam.precision, m[pj, pi], c[pj, pi], ref, rc, ctx=f"request {k}")
