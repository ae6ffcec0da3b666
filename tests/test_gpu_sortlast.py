"""Sort-last rendering on the GPU against the oracle (Sec. 3.1: the tree is
split among workers, each renders its part, the partial images are merged;
Sec. 2.2: contributions add in any order).

Each domain's tree is rendered on the GPU into partial accumulators
(amr_render_batch_partial), the domains are merged on the GPU
(amr_merge_partials) and the merged map is compared, pixel by pixel, with the
oracle's render of the WHOLE tree: columns per pixel, weighted means and mean
levels normwise, within the FP32-compensated or FP64 tolerance; maxima
bit-exact.  Pruned per-domain subtrees (2, 4 and 8 Morton domains) and
full-structure domain trees (where every domain crosses the same cells, so the
counts must equal the oracle's) are both covered.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle
from parity import TOL, errors
from paper_1210_8014_gb300 import amr, inputs, sortlast

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tree():
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    return inputs.galaxy_precision_tree(np.float32)


def cameras(tree, precision):
    """Ragged views of the disk in every mode, at the pixel-rule cut and at a
    coarser cut (where refined cells are read as leaves)."""
    rng = np.random.default_rng(61)
    normal = tree.info["normal"]
    out = []
    for q, (nx, ny) in enumerate([(131, 77), (96, 64), (64, 100), (57, 33)]):
        w = inputs.random_direction(rng)
        centre = inputs.disk_point(rng, normal)
        fov = float(2.0 ** rng.uniform(-4, 0))
        L = -1 if q % 2 == 0 else 8
        out.append(inputs.camera_along(w, centre=centre, fov=fov, n=(nx, ny), max_level=L, mode=q,
                                       precision=precision))
    return out


def check_merged(cam, merged, ref, ctx):
    got = merged.cpu().numpy().astype(np.float64)
    if cam.mode == amr.AMR_MODE_MAX:
        assert (got == ref).all(), f"{ctx}: max differs at {int((got != ref).sum())} pixels"
        return
    e = errors(cam.mode, got, ref)
    assert e["zero_ok"], f"{ctx}: nonzero where the oracle has an empty ray"
    assert e["max"] <= TOL[cam.precision], f"{ctx}: max error {e['max']:.3e}"


@pytest.mark.parametrize("n_domains", [2, 4, 8])
@pytest.mark.parametrize("precision", [amr.AMR_PREC_FP32_KAHAN, amr.AMR_PREC_FP64])
def test_pruned_subtrees_merged_on_gpu_equal_oracle(tree, n_domains, precision):
    own = sortlast.domain_owner(tree, n_domains)
    cams = cameras(tree, precision)
    parts = [[] for _ in cams]
    for d in range(n_domains):
        sub = sortlast.domain_subtree(tree, own, d)
        assert sub.n_oct < (1.5 / n_domains + 0.02) * tree.n_oct
        with amr.Renderer(sub) as r:
            for q, (p, _) in enumerate(r.render_partial(cams)):
                parts[q].append(p)
    prepared = oracle.prepare(tree)
    for q, cam in enumerate(cams):
        merged = sortlast.merge_device(cam, parts[q])
        torch.cuda.synchronize()
        ref, _ = oracle.render(prepared, cam)
        check_merged(cam, merged, ref, f"{n_domains} domains, camera {q} (mode {cam.mode})")


def test_domain_trees_merged_on_gpu_counts_equal_oracle(tree):
    """Full-structure domain trees: every domain crosses exactly the oracle's
    leaves (counts bit-exact), and the merged maps match the oracle."""
    own = sortlast.domain_owner(tree, 3)
    cams = cameras(tree, amr.AMR_PREC_FP32_KAHAN)
    prepared = oracle.prepare(tree)
    refs = [oracle.render(prepared, c) for c in cams]
    parts = [[] for _ in cams]
    for d in range(3):
        with amr.Renderer(sortlast.domain_tree(tree, own, d)) as r:
            for q, (p, c) in enumerate(r.render_partial(cams)):
                parts[q].append(p)
                assert (c.cpu().numpy() == refs[q][1]).all(), (d, q)
    for q, cam in enumerate(cams):
        check_merged(cam, sortlast.merge_device(cam, parts[q]), refs[q][0], f"domain trees, camera {q}")


def test_one_partial_merges_to_the_plain_render(tree):
    """A single domain holding everything: the merge of its one partial equals
    the ordinary render bit for bit (the finishing arithmetic is the same)."""
    cams = cameras(tree, amr.AMR_PREC_FP32_KAHAN) + cameras(tree, amr.AMR_PREC_FP64)
    with amr.Renderer(tree) as r:
        plain = r.render_batch(cams)
        parts = r.render_partial(cams)
        for cam, (m, c), (p, pc) in zip(cams, plain, parts):
            merged = sortlast.merge_device(cam, [p])
            torch.cuda.synchronize()
            assert torch.equal(c, pc)
            assert torch.equal(merged, m), cam.mode


def test_merge_rejects_bad_arguments(tree):
    cam = cameras(tree, amr.AMR_PREC_FP32_KAHAN)[0]
    p = torch.zeros((cam.ny, cam.nx, 2), dtype=torch.float32, device="cuda")
    out = torch.empty((cam.ny, cam.nx), dtype=torch.float32, device="cuda")
    L = amr.lib()
    import ctypes
    arr = (ctypes.c_void_p * 1)(p.data_ptr())
    assert L.amr_merge_partials(0, 0, 1, cam.nx * cam.ny, arr, out.data_ptr(), None) == amr.AMR_E_INVALID
    assert L.amr_merge_partials(amr.AMR_MERGE_MAX_PARTS + 1, 0, 1, 1, arr, out.data_ptr(), None) == amr.AMR_E_INVALID
    assert L.amr_merge_partials(1, 7, 1, 1, arr, out.data_ptr(), None) == amr.AMR_E_INVALID
    assert L.amr_merge_partials(1, 0, 1, 4, None, out.data_ptr(), None) == amr.AMR_E_INVALID
