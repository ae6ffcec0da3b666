"""CUDA path vs the CPU oracle, through the C ABI (pytest -m gpu).

Counts are compared bit-exactly; maps within the tolerances of tests/parity.py
(FP64 kernel 1e-12, FP32 compensated 1e-5, max mode bit-exact).
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import oracle_pins
from parity import TOL, assert_parity, errors
from paper_1210_8014_gb300 import amr, inputs

pytestmark = pytest.mark.gpu

PRECS = (amr.AMR_PREC_FP64, amr.AMR_PREC_FP32_KAHAN, amr.AMR_PREC_FP32_PLAIN)


@pytest.fixture(scope="module")
def gpu():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return 0


_trees = {}


def tree_of(name):
    if name not in _trees:
        if name == "tiny":
            _trees[name] = inputs.plain_tree(np.float64)
        elif name == "galaxy":
            _trees[name] = inputs.galaxy_precision_tree(np.float32)
        elif name == "batch":
            _trees[name] = inputs.batch_tree(np.float32)
    return _trees[name]


def host(t):
    return t.detach().cpu().numpy()


def test_golden_cases_on_gpu(gpu):
    tree, cases = oracle_pins.golden_tree()
    with amr.Renderer(tree) as r:
        for case in cases:
            for p in PRECS:
                cam = oracle_pins.golden_camera(case).with_(precision=p)
                m, c = r.render(cam)
                torch.cuda.synchronize()
                assert int(host(c)[0, 0]) == case["count"], (case["name"], p)
                tol = 1e-15 if p == 0 else 1e-6
                got = float(host(m)[0, 0])
                assert abs(got - case["expected"]) <= tol * max(1.0, abs(case["expected"])), (case["name"], p, got)


def test_tiny_plain_method_fp64_and_fp32(gpu):
    tree = tree_of("tiny")
    cam = inputs.tiny_workload()[1][0]
    ref, rc = oracle.render(tree, cam)
    with amr.Renderer(tree) as r:
        for p in PRECS:
            m, c = r.render(cam.with_(precision=p))
            e = assert_parity(0, p, host(m), host(c), ref, rc, field_is_f32=False, ctx=f"tiny prec {p}")
            if p == 0:
                assert e["max"] <= 1e-12


@pytest.mark.parametrize("k", range(len(oracle_pins._bruteforce_cases())))
def test_random_small_trees_all_modes(gpu, k):
    tree, cam = oracle_pins._bruteforce_cases()[k]
    ref, rc = oracle.render(tree, cam)
    with amr.Renderer(tree) as r:
        for p in PRECS:
            m, c = r.render(cam.with_(precision=p))
            assert_parity(cam.mode, p, host(m), host(c), ref, rc, field_is_f32=False, ctx=f"case {k} prec {p}")


def ragged_cameras(tree, n=(203, 157)):
    rng = np.random.default_rng(2)
    w = inputs.random_direction(rng)
    return [inputs.camera_along(w, fov=1.0, n=n, max_level=tree.depth, mode=m) for m in (0, 1, 2)]


def test_galaxy_full_map_every_mode_and_precision(gpu):
    tree = tree_of("galaxy")
    with amr.Renderer(tree) as r:
        for cam in ragged_cameras(tree):
            ref, rc = oracle.render(tree, cam)
            for p in PRECS:
                m, c = r.render(cam.with_(precision=p))
                assert_parity(cam.mode, p, host(m), host(c), ref, rc, ctx=f"galaxy mode {cam.mode} prec {p}")


def test_galaxy_1024_sampled_pixels(gpu):
    """The 1024^2 precision workload at full size, checked on sampled pixels."""
    tree = tree_of("galaxy")
    cams = inputs.galaxy_precision_cameras(tree)
    rng = np.random.default_rng(0)
    pi = rng.integers(0, 1024, 3000)
    pj = rng.integers(0, 1024, 3000)
    with amr.Renderer(tree) as r:
        refs = {}
        for cam in cams:
            if cam.mode not in refs:
                refs[cam.mode] = oracle.render(tree, cam, pixels=(pi, pj))
            ref, rc = refs[cam.mode]
            m, c = r.render(cam)
            assert_parity(cam.mode, cam.precision, host(m)[pj, pi], host(c)[pj, pi], ref, rc,
                          ctx=f"1024 mode {cam.mode} prec {cam.precision}")


def test_kahan_beats_plain_fp32(gpu):
    tree = tree_of("galaxy")
    cam = inputs.galaxy_precision_cameras(tree, n=256)[0]
    ref, _ = oracle.render(tree, cam)
    with amr.Renderer(tree) as r:
        mk, _ = r.render(cam.with_(precision=amr.AMR_PREC_FP32_KAHAN))
        mp, _ = r.render(cam.with_(precision=amr.AMR_PREC_FP32_PLAIN))
        ek = errors(0, host(mk), ref)
        ep = errors(0, host(mp), ref)
    assert ek["max"] <= 1e-5
    assert ek["p99"] <= ep["p99"], (ek, ep)


def mixed_batch(tree, n_cams, seed, sizes=((128, 128), (130, 77), (256, 256), (33, 5), (512, 300))):
    rng = np.random.default_rng(seed)
    normal = tree.info.get("normal", (0, 0, 1))
    cams = []
    for q in range(n_cams):
        nx, ny = sizes[q % len(sizes)]
        cams.append(inputs.camera_along(inputs.random_direction(rng), centre=inputs.disk_point(rng, normal),
                                        fov=float(2.0 ** rng.uniform(-6, 0)), n=(nx, ny), max_level=-1,
                                        mode=int(rng.integers(0, 3)), precision=int(rng.integers(0, 3))))
    return cams


def test_batch_equals_alone_and_oracle(gpu):
    tree = tree_of("galaxy")
    cams = mixed_batch(tree, 20, seed=7)
    with amr.Renderer(tree) as r:
        outs = r.render_batch(cams)
        torch.cuda.synchronize()
        rng = np.random.default_rng(1)
        for q, cam in enumerate(cams):
            m1, c1 = r.render(cam)
            assert torch.equal(outs[q][0], m1) and torch.equal(outs[q][1], c1), f"camera {q}: batch != alone"
            pi = rng.integers(0, cam.nx, 64)
            pj = rng.integers(0, cam.ny, 64)
            ref, rc = oracle.render(tree, cam, pixels=(pi, pj))
            assert_parity(cam.mode, cam.precision, host(m1)[pj, pi], host(c1)[pj, pi], ref, rc, ctx=f"cam {q}")


@pytest.mark.parametrize("dtype", [np.float32, np.float64])
def test_wmean_packed_fields_per_choice(gpu, dtype):
    """Weighted means read (weight, v_x, v_y, v_z) from a packed copy built once
    per choice of fields: each choice matches the oracle, a repeated choice
    reuses its copy, and loading a tree frees them."""
    tree = inputs.random_tree(np.random.default_rng(11), depth=6, n_fields=5, dtype=dtype)
    rng = np.random.default_rng(4)
    base = inputs.camera_along(inputs.random_direction(rng), fov=1.0, n=(97, 61), max_level=-1,
                               mode=amr.AMR_MODE_WMEAN)
    choices = [(0, (1, 2, 3)), (0, (3, 1, 4)), (0, (1, 2, 3)), (0, (2, 2, 4))]
    cell_bytes = 16 if dtype == np.float32 else 32
    with amr.Renderer(tree) as r:
        for k, (wf, vel) in enumerate(choices):
            cam = base.with_(field_weight=wf, field_vel=vel)
            ref, rc = oracle.render(tree, cam)
            for p in PRECS:
                m, c = r.render(cam.with_(precision=p))
                assert_parity(1, p, host(m), host(c), ref, rc, field_is_f32=dtype == np.float32,
                              ctx=f"choice {k} prec {p}")
        st = r.stats()["tree"]
        assert st["packed_fields"] == 3, st
        assert st["packed_bytes"] == 3 * tree.n_oct * 8 * cell_bytes, st
        amr.amr_load_octree(r.ctx, tree.n_oct, np.ascontiguousarray(tree.level, np.uint8),
                            np.ascontiguousarray(tree.coord, np.int32), np.ascontiguousarray(tree.child, np.int32),
                            [np.ascontiguousarray(f) for f in tree.fields], r.field_dtype)
        assert r.stats()["tree"]["packed_fields"] == 0


def test_segments_counter_matches_counts(gpu):
    tree = tree_of("galaxy")
    cams = mixed_batch(tree, 8, seed=3)
    with amr.Renderer(tree) as r:
        before = r.stats()["segments"]
        outs = r.render_batch(cams)
        torch.cuda.synchronize()
        total = sum(int(o[1].sum()) for o in outs)
        # stats harvest completed launches
        after = r.stats()["segments"]
        assert after - before == total


def test_host_output_path(gpu):
    tree = tree_of("galaxy")
    cam = ragged_cameras(tree, n=(64, 48))[0].with_(precision=amr.AMR_PREC_FP32_KAHAN)
    with amr.Renderer(tree) as r:
        md, cd = r.render(cam)
        mh = np.zeros((48, 64), np.float32)
        ch = np.zeros((48, 64), np.int32)
        amr.amr_render(r.ctx, cam, mh, ch, 0)
        assert (mh == host(md)).all() and (ch == host(cd)).all()
        mb = [np.zeros((48, 64), np.float32), np.zeros((48, 64), np.float64)]
        cams = [cam, cam.with_(precision=0, mode=1)]
        amr.amr_render_batch(r.ctx, cams, mb, None, 0)
        m2, _ = r.render(cams[1])
        assert (mb[0] == host(md)).all() and (mb[1] == host(m2)).all()


def test_host_output_page_locked_written_in_place(gpu):
    """Page-locked host maps are written by the kernel directly (no staging);
    a batch that mixes them with pageable buffers gives the same results as
    device outputs, for every camera, and stale values never survive."""
    tree = tree_of("galaxy")
    cams = mixed_batch(tree, 6, seed=23)
    with amr.Renderer(tree) as r:
        ref = [(host(m), host(c)) for m, c in r.render_batch(cams)]
        torch.cuda.synchronize()
        pinned = [k % 2 == 0 for k in range(len(cams))]
        maps, cnts = [], []
        for k, c in enumerate(cams):
            dt = torch.float64 if c.precision == 0 else torch.float32
            if pinned[k]:
                maps.append(torch.full((c.ny, c.nx), float("nan"), dtype=dt, pin_memory=True).numpy())
                cnts.append(torch.full((c.ny, c.nx), -7, dtype=torch.int32, pin_memory=True).numpy())
            else:
                maps.append(np.full((c.ny, c.nx), np.nan, np.float64 if c.precision == 0 else np.float32))
                cnts.append(np.full((c.ny, c.nx), -7, np.int32))
        amr.amr_render_batch(r.ctx, cams, maps, cnts, 0)
        for k in range(len(cams)):
            assert np.array_equal(cnts[k], ref[k][1]), k
            assert np.array_equal(maps[k], ref[k][0]), k
        # maps only (counts NULL), all page-locked
        maps2 = [torch.zeros((c.ny, c.nx), dtype=torch.float64 if c.precision == 0 else torch.float32,
                             pin_memory=True).numpy() for c in cams]
        amr.amr_render_batch(r.ctx, cams, maps2, None, 0)
        for k in range(len(cams)):
            assert np.array_equal(maps2[k], ref[k][0]), k


def test_deterministic(gpu):
    tree = tree_of("galaxy")
    cams = mixed_batch(tree, 6, seed=11)
    with amr.Renderer(tree) as r:
        a = r.render_batch(cams)
        b = r.render_batch(cams)
        torch.cuda.synchronize()
        for x, y in zip(a, b):
            assert torch.equal(x[0], y[0]) and torch.equal(x[1], y[1])


def test_edge_cases(gpu):
    tree = oracle_pins.golden_tree()[0]
    outside = inputs.Camera((-0.5, 0.5, 0.5), (0, 0, 1), (1, 0, 0), (0, 1, 0), (0.2, 0.2), 7, 3, max_level=2)
    cams = [
        inputs.camera_along((0.2, 0.3, 0.9), n=1, max_level=2),             # single pixel
        inputs.camera_along((0.2, 0.3, 0.9), n=(33, 5), max_level=9),       # ragged, level clamped to depth
        inputs.camera_along((0.0, -1.0, 0.0), n=(17, 31), max_level=1),     # level 1, axis-aligned
        outside,                                                             # misses the box: zeros
        inputs.camera_along((1.0, 1.0, 1.0), fov=1.8, n=(40, 40), max_level=2),
    ]
    with amr.Renderer(tree) as r:
        for k, cam in enumerate(cams):
            for mode in (0, 1, 2):
                for p in PRECS:
                    c2 = cam.with_(mode=mode, precision=p)
                    ref, rc = oracle.render(tree, c2)
                    m, c = r.render(c2)
                    assert_parity(mode, p, host(m), host(c), ref, rc, field_is_f32=False, ctx=f"edge {k}")
        m, c = r.render(outside)
        assert int(c.sum()) == 0 and float(m.abs().sum()) == 0.0
        assert amr.amr_camera_check(r.ctx, cams[1]) == 2


def test_invalid_cameras_rejected(gpu):
    tree = oracle_pins.golden_tree()[0]
    base = inputs.camera_along((0, 0, 1), n=8, max_level=2)
    bad = [base.with_(nx=0), base.with_(mode=5), base.with_(precision=9), base.with_(u=(1.0, 0.1, 0.0)),
           base.with_(fov=(0.0, 1.0)), base.with_(centre=(5.0, 0.5, 0.5)), base.with_(field_value=7),
           base.with_(mode=1, field_vel=(1, 2, 9)), base.with_(max_level=0), base.with_(centre=(float("nan"), 0.5, 0.5))]
    with amr.Renderer(tree) as r:
        for k, cam in enumerate(bad):
            with pytest.raises(amr.AmrError) as e:
                r.render(cam)
            assert e.value.status == amr.AMR_E_INVALID, k


def test_bad_trees_rejected(gpu):
    tree, _ = oracle_pins.golden_tree()
    ctx = amr.amr_create(0)
    try:
        def load(level, coord, child):
            f = [np.zeros((len(level), 8))]
            amr.amr_load_octree(ctx, len(level), np.array(level, np.uint8), np.array(coord, np.int32),
                                np.array(child, np.int32), f, amr.AMR_F64)

        ok = (tree.level, tree.coord, tree.child)
        load(*ok)
        cases = {
            "root level": ([2, 2], tree.coord, tree.child),
            "child level": ([1, 3], tree.coord, tree.child),
            "child coord": (tree.level, [[0, 0, 0], [2, 0, 0]], tree.child),
            "shared child": ([1, 2], tree.coord, [[1, 1, -1, -1, -1, -1, -1, -1], [-1] * 8]),
            "cycle": ([1, 2], tree.coord, [[1] + [-1] * 7, [1] + [-1] * 7]),
            "unreachable": ([1, 2], tree.coord, [[-1] * 8, [-1] * 8]),
            "index range": ([1, 2], tree.coord, [[5] + [-1] * 7, [-1] * 8]),
            "odd coord": ([1, 2], [[0, 0, 0], [1, 0, 0]], tree.child),
        }
        for name, (lv, co, ch) in cases.items():
            with pytest.raises(amr.AmrError) as e:
                load(lv, co, ch)
            assert e.value.status == amr.AMR_E_BADTREE, name
            assert "oct" in str(e.value), name
    finally:
        amr.amr_destroy(ctx)


def test_autotune_keeps_results(gpu):
    tree = tree_of("galaxy")
    cams = mixed_batch(tree, 10, seed=5)
    with amr.Renderer(tree) as r:
        a = r.render_batch(cams)
        best, ms = amr.amr_autotune(r.ctx, cams, reps=1)
        assert best["tile_w"] * best["tile_h"] == 32 and ms > 0
        assert best["max_regs"] in (0, 56, 64, 72)
        assert amr.amr_get_options(r.ctx).as_dict() == best
        b = r.render_batch(cams)
        torch.cuda.synchronize()
        for x, y in zip(a, b):
            assert torch.equal(x[0], y[0]) and torch.equal(x[1], y[1])


def test_register_caps_give_identical_maps(gpu):
    """The register cap (56, 64, 72 per thread) changes occupancy and spills,
    not arithmetic: every cap renders the mixed batch bit for bit alike, the
    FP64 kernel included; other caps are rejected."""
    tree = tree_of("galaxy")
    cams = mixed_batch(tree, 12, seed=9)
    with amr.Renderer(tree) as r:
        ref = r.render_batch(cams)
        torch.cuda.synchronize()
        for regs in (56, 72, 64, 0):
            amr.amr_set_options(r.ctx, max_regs=regs)
            out = r.render_batch(cams)
            torch.cuda.synchronize()
            st = r.stats()
            assert st["options"]["max_regs"] == regs
            assert all(0 < v <= (regs or 64) for v in st["regs"].values()), st["regs"]
            for q, (x, y) in enumerate(zip(ref, out)):
                assert torch.equal(x[1], y[1]), f"cap {regs} camera {q}: counts differ"
                assert torch.equal(x[0], y[0]), f"cap {regs} camera {q}: maps differ"
        for bad in (48, 60, 80, -1):
            with pytest.raises(amr.AmrError):
                amr.amr_set_options(r.ctx, max_regs=bad)


def test_server_alone_vs_mix(gpu):
    """Requests submitted together overlap on the device; each result equals
    the same camera rendered alone.  Every other request brings page-locked
    buffers (written in place by the kernel), the rest pageable ones (slot
    buffer and copy), so batches mix both deliveries."""
    tree = tree_of("galaxy")
    cams = mixed_batch(tree, 24, seed=9)
    with amr.Renderer(tree) as r:
        amr.amr_server_config(r.ctx, slots=3, map_budget_bytes=8 << 20, max_batch=6)
        bufs, tickets = [], []
        for k, cam in enumerate(cams):
            if k % 2:
                dt = torch.float64 if cam.precision == 0 else torch.float32
                mh = torch.zeros((cam.ny, cam.nx), dtype=dt, pin_memory=True).numpy()
                ch = torch.zeros((cam.ny, cam.nx), dtype=torch.int32, pin_memory=True).numpy()
            else:
                mh = np.zeros((cam.ny, cam.nx), np.float64 if cam.precision == 0 else np.float32)
                ch = np.zeros((cam.ny, cam.nx), np.int32)
            bufs.append((mh, ch))
            tickets.append(amr.amr_submit(r.ctx, cam, mh, ch))
        for t in tickets:
            amr.amr_wait(r.ctx, t, 60_000_000)
        for cam, (mh, ch) in zip(cams, bufs):
            m1, c1 = r.render(cam)
            assert (mh == host(m1)).all() and (ch == host(c1)).all()
        st = r.stats()["server"]
        assert st["done"] == len(cams) and st["failed"] == 0
        assert st["p99_ms"] >= st["p50_ms"] > 0
        with pytest.raises(amr.AmrError) as e:
            amr.amr_wait(r.ctx, 10 ** 9, 0)
        assert e.value.status == amr.AMR_E_INVALID


def test_graph_replay_matches_direct_launches(gpu):
    """With use_graph, a launch slot captures its sequence once per batch shape
    and replays it; new camera contents of the same shape must reach the kernel."""
    tree = tree_of("galaxy")
    a = mixed_batch(tree, 6, seed=21)
    rng = np.random.default_rng(5)
    b = [c.with_(w=tuple(inputs.basis_from_direction(inputs.random_direction(rng))[2]),
                 u=None, v=None) for c in a]
    b = [inputs.camera_along(c.w, centre=c.centre, fov=c.fov[0], n=(c.nx, c.ny), max_level=-1, mode=c.mode,
                             precision=c.precision) for c in b]
    with amr.Renderer(tree) as r:
        ref_a = r.render_batch(a)
        ref_b = r.render_batch(b)
        amr.amr_set_options(r.ctx, use_graph=1)
        for _ in range(10):                      # more than the 8 launch slots: every slot replays
            for cams, ref in ((a, ref_a), (b, ref_b)):
                got = r.render_batch(cams)
                torch.cuda.synchronize()
                for x, y in zip(got, ref):
                    assert torch.equal(x[0], y[0]) and torch.equal(x[1], y[1])
        shorter = r.render_batch(a[:3])          # a new shape: captured anew
        torch.cuda.synchronize()
        for x, y in zip(shorter, ref_a[:3]):
            assert torch.equal(x[0], y[0]) and torch.equal(x[1], y[1])
        st = r.stats()
        assert st["graph_launches"] >= 21 and 1 <= st["graph_captures"] <= 10


def test_slice_map_matches_oracle(gpu):
    """Slice maps (Sec. 3.3 Slicemap): values and leaf levels bit-exact."""
    tree = tree_of("galaxy")
    rng = np.random.default_rng(12)
    normal = tree.info["normal"]
    cams = [inputs.camera_along(inputs.random_direction(rng), centre=inputs.disk_point(rng, normal),
                                fov=float(2.0 ** rng.uniform(-8, 0.5)), n=(97, 61), max_level=-1,
                                field_value=int(rng.integers(0, 4))) for _ in range(6)]
    cams.append(inputs.camera_along((0.0, 0.0, 1.0), fov=2.5, n=64, max_level=11))  # partly outside the box
    with amr.Renderer(tree) as r:
        for k, cam in enumerate(cams):
            ref, rl = oracle.slice_map(tree, cam)
            m, lv = r.slice(cam.with_(precision=amr.AMR_PREC_FP32_KAHAN))
            assert (host(lv) == rl).all(), k
            assert (host(m).astype(np.float64) == ref).all(), k
            m64 = np.zeros((cam.ny, cam.nx), np.float64)
            amr.amr_slice(r.ctx, cam.with_(precision=amr.AMR_PREC_FP64), m64, None, 0)
            assert (m64 == ref).all(), k
            # page-locked host outputs are written in place
            mp = torch.full((cam.ny, cam.nx), float("nan"), dtype=torch.float32, pin_memory=True).numpy()
            lp = torch.full((cam.ny, cam.nx), -1, dtype=torch.int32, pin_memory=True).numpy()
            amr.amr_slice(r.ctx, cam.with_(precision=amr.AMR_PREC_FP32_KAHAN), mp, lp, 0)
            assert (lp == rl).all() and (mp.astype(np.float64) == ref).all(), k


def test_mean_level_and_adaptive_blur(gpu):
    """Sec. 2.2 adaptive blur: the mean-level map against the oracle, then the
    blur of the GPU column map against the oracle blur of the same inputs."""
    from oracle import blur as oblur
    tree = tree_of("galaxy")
    rng = np.random.default_rng(8)
    # level 11 cells are a third of a pixel (left sharp), level-7 cells ~5 pixels (blurred)
    cam = inputs.camera_along(inputs.random_direction(rng), centre=(0.5, 0.5, 0.5), fov=0.15, n=(96, 72),
                              max_level=11, precision=amr.AMR_PREC_FP32_KAHAN)
    lvl_cam = cam.with_(mode=amr.AMR_MODE_LEVEL)
    ref_lv, rc = oracle.render(tree, lvl_cam)
    with amr.Renderer(tree) as r:
        col, _ = r.render(cam)
        lv, c = r.render(lvl_cam)
        assert_parity(3, 1, host(lv), host(c), ref_lv, rc, ctx="mean level")
        out = torch.empty_like(col)
        pixel = cam.fov[0] / cam.nx
        amr.amr_blur(r.ctx, cam.nx, cam.ny, col, lv, pixel, out, torch.cuda.current_stream().cuda_stream)
        torch.cuda.synchronize()
    ref = oblur.adaptive_blur(host(col).astype(np.float64), host(lv).astype(np.float64), pixel)
    sig = oblur.sigma_map(host(lv), pixel)
    assert (sig >= 0.5).any() and (sig < 0.5).any()     # the view mixes blurred and sharp pixels
    assert np.abs(host(out) - ref).max() <= 1e-5 * np.abs(ref).max()


def test_server_timeout_cancel_budget_and_shutdown(gpu):
    """Failure paths of the request server, all made on the host: a wait that
    runs out of time, a queued request cancelled, a request over the memory
    budget, and a context destroyed with work still queued."""
    tree = tree_of("galaxy")
    big = inputs.camera_along((0.3, 0.5, 0.8), fov=1.0, n=2048, max_level=tree.depth,
                              precision=amr.AMR_PREC_FP32_KAHAN)
    bufs = [(np.zeros((2048, 2048), np.float32), np.zeros((2048, 2048), np.int32)) for _ in range(4)]
    with amr.Renderer(tree) as r:
        amr.amr_server_config(r.ctx, slots=1, map_budget_bytes=40 << 20, max_batch=1)
        tickets = [amr.amr_submit(r.ctx, big, m, c) for m, c in bufs]
        with pytest.raises(amr.AmrError) as e:
            amr.amr_wait(r.ctx, tickets[0], 0)           # the first render takes milliseconds
        assert e.value.status == amr.AMR_E_TIMEOUT
        amr.amr_cancel(r.ctx, tickets[3])                # still queued behind the others
        with pytest.raises(amr.AmrError) as e:
            amr.amr_wait(r.ctx, tickets[3], -1)
        assert e.value.status == amr.AMR_E_CANCELLED
        for t in tickets[:3]:
            amr.amr_wait(r.ctx, t, 60_000_000)
        with pytest.raises(amr.AmrError) as e:
            amr.amr_cancel(r.ctx, tickets[0])            # finished and collected
        assert e.value.status == amr.AMR_E_INVALID
        ref, rc = r.render(big)
        assert (bufs[0][0] == host(ref)).all() and (bufs[2][1] == host(rc)).all()
        huge = big.with_(nx=8192, ny=8192)                # 512 MiB of map: over the 40 MiB budget
        tiny_buf = np.zeros(1, np.float32)                # refused at submit, before anything is written;
        with pytest.raises(amr.AmrError) as e:             # a raw pointer skips the binding's size check
            amr.amr_submit(r.ctx, huge, tiny_buf.ctypes.data)
        assert e.value.status == amr.AMR_E_OOM
        st = r.stats()["server"]
        assert st["done"] == 3 and st["queued"] == 0
    # shutdown with requests still queued: they end cancelled, destroy returns
    ctx = amr.amr_create(0)
    amr.amr_load_octree(ctx, tree.n_oct, tree.level, tree.coord, tree.child, tree.fields, amr.AMR_F32)
    amr.amr_server_config(ctx, slots=1, map_budget_bytes=40 << 20, max_batch=1)
    for m, c in bufs:
        amr.amr_submit(ctx, big, m, c)
    amr.amr_destroy(ctx)


def test_server_destroy_with_every_slot_busy(gpu):
    """amr_destroy while three launch slots are rendering and more requests
    wait (admitted with tiles outstanding, and queued): it returns, and the
    device is healthy afterwards (a new context renders correctly)."""
    tree = tree_of("galaxy")
    big = inputs.camera_along((0.3, 0.5, 0.8), fov=1.0, n=2048, max_level=tree.depth,
                              precision=amr.AMR_PREC_FP32_KAHAN)
    bufs = [(torch.zeros((2048, 2048), dtype=torch.float32, pin_memory=True).numpy(),
             torch.zeros((2048, 2048), dtype=torch.int32, pin_memory=True).numpy()) for _ in range(8)]
    ctx = amr.amr_create(0)
    amr.amr_load_octree(ctx, tree.n_oct, tree.level, tree.coord, tree.child, tree.fields, amr.AMR_F32)
    amr.amr_server_config(ctx, slots=3, map_budget_bytes=1 << 30, max_batch=4)
    tickets = [amr.amr_submit(ctx, big, m, c) for m, c in bufs]
    amr.amr_wait(ctx, tickets[0], 60_000_000)             # work is flowing
    st = amr.amr_stats(ctx)["server"]
    assert st["done"] >= 1
    amr.amr_destroy(ctx)                                  # remaining requests end cancelled
    with amr.Renderer(tree) as r:
        m, c = r.render(big)
        torch.cuda.synchronize()
        assert (host(m) == bufs[0][0]).all() and (host(c) == bufs[0][1]).all()


def test_large_batch_grows_launch_scratch(gpu):
    """150 cameras in one batch (beyond the initial scratch of 64): every map
    equals its camera rendered alone."""
    tree = tree_of("galaxy")
    cams = mixed_batch(tree, 150, seed=41, sizes=((32, 32), (17, 9), (40, 24)))
    with amr.Renderer(tree) as r:
        outs = r.render_batch(cams)
        torch.cuda.synchronize()
        for q in range(0, 150, 7):
            m1, c1 = r.render(cams[q])
            assert torch.equal(outs[q][0], m1) and torch.equal(outs[q][1], c1), q
