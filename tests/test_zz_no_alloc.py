"""amr_render_batch_noalloc: the batch renderer for callers that cannot allocate GPU memory.

Callers such as a renderer embedded in a simulation that owns all GPU memory
(in-situ visualisation), or a latency-critical loop that must not stall on a
cudaMalloc, keep the octree in their own device buffers and pass it in.  These
tests build those buffers themselves (the library allocates nothing for the
call) and check the entry point two ways:

- against the context-based amr_render_batch, on the same mixed batch rendered
  twice in a row (calls share the fixed scratch array, so the second call must
  not see the first one's state);
- against the CPU oracle: the seeded fuzz cases of test_gpu_fuzz.py (rays along
  axes and diagonals, dyadic slopes, views partly outside the box, coarse
  cuts), the hand-derived two-level tree and a full-depth level-22 view of the
  193M-leaf zoom tree.  This entry point runs the kernel variant without face
  links (neighbours through a stack of ancestor octs), so it needs its own
  parity cases.  Counts bit-exact, maps within the parity tolerances.

It also checks that the device error word the kernel writes (a child index out
of range) comes back through amr_noalloc_status.  The file is named so that
pytest collects it last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
import oracle_pins
from parity import assert_parity
from test_gpu_fuzz import N_CASES, fuzz_case
from paper_1210_8014_gb300 import amr, inputs

pytestmark = pytest.mark.gpu


def device_records(tree):
    """uint64 records {first child | mask << 32} of a breadth-first tree whose
    siblings are adjacent (what the generator emits)."""
    n = tree.n_oct
    has = tree.child >= 0
    first_c = has.argmax(1)
    first = np.where(has.any(1), tree.child[np.arange(n), first_c], 0).astype(np.int64)
    # siblings adjacent in cell order, children after their parent
    for o in np.nonzero(has.any(1))[0][:2000]:
        kids = tree.child[o][has[o]]
        assert (np.diff(kids) == 1).all() and kids[0] > o
    mask = (has.astype(np.int64) << np.arange(8)).sum(1)
    return (first | (mask << 32)).astype(np.int64)


def upload(tree):
    """The caller's own device copy of a tree: records and fields."""
    dev = torch.device("cuda:0")
    records = torch.from_numpy(device_records(tree)).to(dev)
    fields = [torch.from_numpy(np.ascontiguousarray(f)).to(dev) for f in tree.fields]
    dtype = amr.AMR_F64 if tree.fields[0].dtype == np.float64 else amr.AMR_F32
    return records, fields, dtype


def outputs(cams):
    dev = torch.device("cuda:0")
    maps = [torch.full((c.ny, c.nx), float("nan"), dtype=torch.float64 if c.precision == 0 else torch.float32,
                       device=dev) for c in cams]
    cnts = [torch.full((c.ny, c.nx), -7, dtype=torch.int32, device=dev) for c in cams]
    return maps, cnts


def render_noalloc(tree, dev_tree, cams):
    records, fields, dtype = dev_tree
    maps, cnts = outputs(cams)
    stream = torch.cuda.current_stream()
    amr.amr_render_batch_noalloc(tree.n_oct, records, tree.depth, fields, dtype, cams, maps, cnts, stream.cuda_stream)
    status = amr.amr_noalloc_status(stream.cuda_stream)
    assert status["error"] == 0, status
    return [m.cpu().numpy() for m in maps], [c.cpu().numpy() for c in cnts], status


def mixed_cameras(tree):
    rng = np.random.default_rng(42)
    normal = tree.info.get("normal", (0, 0, 1))
    cams = []
    for q, (nx, ny) in enumerate([(96, 64), (33, 17), (128, 128), (64, 100), (250, 31), (40, 40)] * 2):
        cams.append(inputs.camera_along(inputs.random_direction(rng), centre=inputs.disk_point(rng, normal),
                                        fov=float(2.0 ** rng.uniform(-5, 0)), n=(nx, ny), max_level=-1,
                                        mode=q % 3, precision=(q // 3) % 3))
    return cams


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    tree = inputs.galaxy_tree(2, 2.0 ** -16, 11, with_velocity=True)
    cams = mixed_cameras(tree)
    with amr.Renderer(tree) as r:
        expected = [(m.cpu().numpy(), c.cpu().numpy()) for m, c in r.render_batch(cams)]
    records, fields, _ = upload(tree)
    return tree, cams, expected, records, fields


def test_noalloc_matches_context_batch_twice(setup):
    tree, cams, expected, records, fields = setup
    dev = torch.device("cuda:0")
    maps = [torch.empty((c.ny, c.nx), dtype=torch.float64 if c.precision == 0 else torch.float32, device=dev)
            for c in cams]
    cnts = [torch.empty((c.ny, c.nx), dtype=torch.int32, device=dev) for c in cams]
    stream = torch.cuda.current_stream()
    for call in range(2):
        for m, c in zip(maps, cnts):       # stale values must not leak into the result
            m.fill_(float("nan"))
            c.fill_(-7)
        amr.amr_render_batch_noalloc(tree.n_oct, records, tree.depth, fields, amr.AMR_F32, cams, maps, cnts,
                                     stream.cuda_stream)
        st = amr.amr_noalloc_status(stream.cuda_stream)
        assert st["error"] == 0
        assert st["segments"] == sum(int(e[1].sum()) for e in expected)
        for k, (cam, m, c) in enumerate(zip(cams, maps, cnts)):
            em, ec = expected[k]
            assert_parity(cam.mode, cam.precision, m.cpu().numpy(), c.cpu().numpy(), em, ec,
                          ctx=f"call {call} camera {k}")


def test_noalloc_mixed_batch_against_oracle(setup):
    """The same mixed batch (every precision, three modes, ragged sizes)
    against the oracle on sampled pixels."""
    tree, cams, _, records, fields = setup
    maps, cnts, _ = render_noalloc(tree, (records, fields, amr.AMR_F32), cams)
    prepared = oracle.prepare(tree)
    rng = np.random.default_rng(3)
    for k, cam in enumerate(cams):
        pi = rng.integers(0, cam.nx, 200)
        pj = rng.integers(0, cam.ny, 200)
        ref, rc = oracle.render(prepared, cam, pixels=(pi, pj))
        assert_parity(cam.mode, cam.precision, maps[k][pj, pi], cnts[k][pj, pi], ref, rc, ctx=f"camera {k}")


@pytest.mark.parametrize("k", range(N_CASES))
def test_noalloc_fuzz_against_oracle(setup, k):
    """The seeded special-direction fuzz cases, every mode, FP64 and FP32
    compensated in one no-allocation batch."""
    tree, cams = fuzz_case(k)
    batch = [c.with_(precision=p) for c in cams for p in (amr.AMR_PREC_FP64, amr.AMR_PREC_FP32_KAHAN)]
    maps, cnts, _ = render_noalloc(tree, upload(tree), batch)
    for q, cam in enumerate(batch):
        ref, rc = oracle.render(tree, cam)
        assert_parity(cam.mode, cam.precision, maps[q], cnts[q], ref, rc, field_is_f32=False,
                      ctx=f"fuzz case {k} mode {cam.mode} prec {cam.precision}")


def test_noalloc_golden_two_level_tree(setup):
    tree, cases = oracle_pins.golden_tree()
    batch = [oracle_pins.golden_camera(c).with_(precision=p) for c in cases
             for p in (amr.AMR_PREC_FP64, amr.AMR_PREC_FP32_KAHAN)]
    maps, cnts, _ = render_noalloc(tree, upload(tree), batch)
    for q, cam in enumerate(batch):
        case = cases[q // 2]
        assert int(cnts[q][0, 0]) == case["count"], (case["name"], cam.precision)
        tol = 1e-15 if cam.precision == 0 else 1e-6
        got = float(maps[q][0, 0])
        assert abs(got - case["expected"]) <= tol * max(1.0, abs(case["expected"])), (case["name"], got)


def test_noalloc_level22_deep_view_against_oracle(setup, zoom_tree):
    """Full-depth view of the zoom tree's centre (level 22, 512^2), column and
    max, FP32 compensated and FP64, on sampled pixels."""
    tree = zoom_tree
    cams = [inputs.deep_centre_camera(tree, mode=m, precision=p) for m in (0, 2)
            for p in (amr.AMR_PREC_FP32_KAHAN, amr.AMR_PREC_FP64)]
    maps, cnts, _ = render_noalloc(tree, upload(tree), cams)
    rng = np.random.default_rng(22)
    pi = rng.integers(0, 512, 1500)
    pj = rng.integers(0, 512, 1500)
    prepared = oracle.prepare(tree)
    for q, cam in enumerate(cams):
        ref, rc = oracle.render(prepared, cam, pixels=(pi, pj))
        assert rc.max() > 0
        assert_parity(cam.mode, cam.precision, maps[q][pj, pi], cnts[q][pj, pi], ref, rc, ctx=f"deep camera {q}")


def test_noalloc_rejects_oversized_batch(setup):
    tree, cams, _, records, fields = setup
    too_many = [cams[0]] * (amr.AMR_NOALLOC_MAX_CAMERAS + 1)
    with pytest.raises(amr.AmrError) as e:
        amr.amr_render_batch_noalloc(tree.n_oct, records, tree.depth, fields, amr.AMR_F32, too_many,
                                     [None] * len(too_many))
    assert e.value.status == amr.AMR_E_INVALID
    assert "at most 256" in str(e.value)


def test_noalloc_out_of_range_children_end_rays_cleanly(setup):
    """The caller's records are not validated on the host; a first-child index
    at or beyond n_oct ends the affected rays inside the kernel (its bounds
    check runs before any read), amr_noalloc_status reports it, and the call
    and the device stay healthy."""
    tree, cams, expected, records, fields = setup
    bad = records.clone()
    refined = torch.nonzero((bad >> 32) != 0).flatten()
    bad[refined[::3]] = (bad[refined[::3]] & ~0xFFFFFFFF) | (tree.n_oct + 5)
    dev = torch.device("cuda:0")
    maps = [torch.zeros((c.ny, c.nx), dtype=torch.float64 if c.precision == 0 else torch.float32, device=dev)
            for c in cams]
    cnts = [torch.zeros((c.ny, c.nx), dtype=torch.int32, device=dev) for c in cams]
    stream = torch.cuda.current_stream()
    amr.amr_render_batch_noalloc(tree.n_oct, bad, tree.depth, fields, amr.AMR_F32, cams, maps, cnts,
                                 stream.cuda_stream)
    st = amr.amr_noalloc_status(stream.cuda_stream)
    assert st["error"] == 1, st                       # a child index out of range
    assert 0 <= st["oct"] < tree.n_oct
    assert ((bad[st["oct"]] & 0xFFFFFFFF) == tree.n_oct + 5).item()
    total = sum(int(c.sum()) for c in cnts)
    assert total < sum(int(e[1].sum()) for e in expected)
    # the device is fine: an intact call right after reproduces the reference,
    # and its status is clean again (every call clears the error words)
    amr.amr_render_batch_noalloc(tree.n_oct, records, tree.depth, fields, amr.AMR_F32, cams, maps, cnts,
                                 stream.cuda_stream)
    assert amr.amr_noalloc_status(stream.cuda_stream)["error"] == 0
    for k, (cam, m, c) in enumerate(zip(cams, maps, cnts)):
        assert (c.cpu().numpy() == expected[k][1]).all()
