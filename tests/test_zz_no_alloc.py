"""amr_render_batch_noalloc: the batch renderer for callers that cannot allocate GPU memory.

Callers such as a renderer embedded in a simulation that owns all GPU memory
(in-situ visualisation), or a latency-critical loop that must not stall on a
cudaMalloc, keep the octree in their own device buffers and pass it in.  This
test builds those buffers itself (the library allocates nothing for the call),
renders the same mixed batch twice in a row through the no-allocation entry
point, and checks both results against the context-based amr_render_batch
within the parity tolerances the other tests use.  The file is named so that
pytest collects it last.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from parity import assert_parity
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
    dev = torch.device("cuda:0")
    records = torch.from_numpy(device_records(tree)).to(dev)
    fields = [torch.from_numpy(np.ascontiguousarray(f)).to(dev) for f in tree.fields]
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
        torch.cuda.synchronize()
        for k, (cam, m, c) in enumerate(zip(cams, maps, cnts)):
            em, ec = expected[k]
            assert_parity(cam.mode, cam.precision, m.cpu().numpy(), c.cpu().numpy(), em, ec,
                          ctx=f"call {call} camera {k}")


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
    check runs before any read), and the call and the device stay healthy."""
    tree, cams, expected, records, fields = setup
    bad = records.clone()
    refined = torch.nonzero((bad >> 32) != 0).flatten()
    bad[refined[::3]] = (bad[refined[::3]] & ~0xFFFFFFFF) | (tree.n_oct + 5)
    dev = torch.device("cuda:0")
    maps = [torch.zeros((c.ny, c.nx), dtype=torch.float64 if c.precision == 0 else torch.float32, device=dev)
            for c in cams]
    cnts = [torch.zeros((c.ny, c.nx), dtype=torch.int32, device=dev) for c in cams]
    amr.amr_render_batch_noalloc(tree.n_oct, bad, tree.depth, fields, amr.AMR_F32, cams, maps, cnts,
                                 torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    total = sum(int(c.sum()) for c in cnts)
    assert total < sum(int(e[1].sum()) for e in expected)
    # the device is fine: an intact call right after reproduces the reference
    amr.amr_render_batch_noalloc(tree.n_oct, records, tree.depth, fields, amr.AMR_F32, cams, maps, cnts,
                                 torch.cuda.current_stream().cuda_stream)
    torch.cuda.synchronize()
    for k, (cam, m, c) in enumerate(zip(cams, maps, cnts)):
        assert (c.cpu().numpy() == expected[k][1]).all()
