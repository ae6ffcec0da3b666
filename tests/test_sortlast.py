"""Sort-last decomposition (Sec. 3.1): partial maps over disjoint leaf domains
merge into the whole map, in one process and across gloo ranks on CPU; and the
multi-rank benchmark helpers (max over ranks, replica throughput)."""
import os
import socket
import sys

import numpy as np
import pytest

import oracle
from paper_1210_8014_gb300 import inputs, sortlast

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def small_galaxy():
    return inputs.galaxy_tree(5, 2.0 ** -14, 10, with_velocity=True, dtype=np.float64)


def cams_for(tree):
    rng = np.random.default_rng(17)
    w = inputs.random_direction(rng)
    return [inputs.camera_along(w, centre=inputs.disk_point(rng, tree.info["normal"]), fov=0.3, n=(24, 20),
                                max_level=-1, mode=m) for m in (0, 1, 2)]


def test_domains_partition_the_leaves():
    tree = small_galaxy()
    for n in (1, 2, 3, 5):
        own = sortlast.domain_owner(tree, n)
        leaf = tree.child < 0
        sizes = np.bincount(own[leaf], minlength=n)
        assert sizes.sum() == leaf.sum() and len(sizes) == n
        assert sizes.max() - sizes.min() <= max(2, leaf.sum() // 1000)


@pytest.mark.parametrize("n_domains", [2, 3, 4])
def test_merged_partials_equal_whole_render(n_domains):
    tree = small_galaxy()
    own = sortlast.domain_owner(tree, n_domains)
    for cam in cams_for(tree):
        whole, wc = oracle.render(tree, cam)
        parts, counts = [], []
        for d in range(n_domains):
            dt = sortlast.domain_tree(tree, own, d, with_momentum=cam.mode == 1)
            maps = []
            for pc in sortlast.partial_cameras(cam):
                m, c = oracle.render(dt, pc)
                maps.append(m)
                counts.append(c)
            parts.append(maps)
        merged, mc = sortlast.merge(cam, parts, counts[::len(sortlast.partial_cameras(cam))])
        assert (mc == wc).all()
        if cam.mode == 2:
            assert (merged == whole).all()
        elif cam.mode == 0:
            assert np.abs(merged - whole).max() <= 1e-13 * np.abs(whole).max()
        else:
            assert np.abs(merged - whole).max() <= 1e-12 * np.abs(whole).max()


def _check_tree(t):
    """What amr_load_octree validates: root at index 0, level 1, coordinate 0;
    each child one level deeper at twice its parent cell's coordinates; every
    non-root oct referenced exactly once."""
    assert t.level[0] == 1 and (t.coord[0] == 0).all()
    refs = np.zeros(t.n_oct, np.int64)
    o, c = np.nonzero(t.child >= 0)
    ch = t.child[o, c]
    np.add.at(refs, ch, 1)
    assert refs[0] == 0 and (refs[1:] == 1).all()
    assert (t.level[ch] == t.level[o] + 1).all()
    off = np.stack([(c >> a) & 1 for a in range(3)], axis=1)
    assert (t.coord[ch] == 2 * (t.coord[o] + off)).all()


def test_subtrees_are_valid_and_split_the_tree():
    tree = small_galaxy()
    for n in (2, 4, 7):
        own = sortlast.domain_owner(tree, n)
        sizes = []
        for d in range(n):
            st = sortlast.domain_subtree(tree, own, d)
            _check_tree(st)
            sizes.append(st.n_oct)
            # every owned value survives; nothing else is nonzero
            assert np.isclose(float(st.fields[0].sum()), float(tree.fields[0][own == d].sum()), rtol=1e-12)
        # the domains together hold the tree once plus shared ancestors
        assert sum(sizes) < tree.n_oct * 1.25 and max(sizes) < tree.n_oct / n * 1.3


@pytest.mark.parametrize("n_domains", [2, 4])
def test_merged_subtree_partials_equal_whole_render(n_domains):
    """Pruned per-domain trees merge into the whole render at the pixel-rule
    cut and at cuts above the finest level (where owned refined cells read as
    leaves and foreign ones as zeros)."""
    tree = small_galaxy()
    own = sortlast.domain_owner(tree, n_domains)
    cams = cams_for(tree) + [c.with_(max_level=L) for c in cams_for(tree) for L in (5, 7)]
    subs = {(d, mom): sortlast.domain_subtree(tree, own, d, with_momentum=mom)
            for d in range(n_domains) for mom in (False, True)}
    for cam in cams:
        whole, _ = oracle.render(tree, cam)
        parts = []
        for d in range(n_domains):
            st = subs[(d, cam.mode == 1)]
            parts.append([oracle.render(st, pc)[0] for pc in sortlast.partial_cameras(cam)])
        merged, mc = sortlast.merge(cam, parts)
        assert mc is None
        if cam.mode == 2:
            assert (merged == whole).all()
        elif cam.mode == 0:
            assert np.abs(merged - whole).max() <= 1e-13 * np.abs(whole).max()
        else:
            assert np.abs(merged - whole).max() <= 1e-12 * np.abs(whole).max()


def test_subtree_owned_refined_cell_with_foreign_descendants():
    """Refined cells owned by another domain than their descendants (random
    owners for refined cells): the owner keeps one level of zero-valued children
    under each such cell, so cuts below it still read zeros there.  Without
    that level the merge is off by percents at cuts 7 and the pixel rule."""
    tree = small_galaxy()
    own = sortlast.domain_owner(tree, 3)
    refined = tree.child >= 0
    own[refined] = np.random.default_rng(3).integers(0, 3, int(refined.sum()))
    subs = [sortlast.domain_subtree(tree, own, d) for d in range(3)]
    for st in subs:
        _check_tree(st)
    for cam in [c for c in cams_for(tree) if c.mode != 1]:
        for L in (5, 7, -1):
            c = cam.with_(max_level=L)
            whole, _ = oracle.render(tree, c)
            merged, _ = sortlast.merge(c, [[oracle.render(st, c)[0]] for st in subs])
            if c.mode == 2:
                assert (merged == whole).all()
            else:
                assert np.abs(merged - whole).max() <= 1e-13 * np.abs(whole).max()


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        tree = small_galaxy()
        own = sortlast.domain_owner(tree, world)
        results = []
        for cam in cams_for(tree):
            dt = sortlast.domain_tree(tree, own, rank, with_momentum=cam.mode == 1)
            local = [oracle.render(dt, pc)[0] for pc in sortlast.partial_cameras(cam)]
            results.append(sortlast.merge_distributed(cam, local))
        mx = bench.max_over_ranks(10.0 + rank)
        sm = bench.sum_over_ranks(1000 + rank)
        np.savez(os.path.join(out_dir, f"rank{rank}.npz"), *results, mx=np.array([mx]), sm=np.array([sm]))
    finally:
        dist.destroy_process_group()


def test_sortlast_merge_across_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    tree = small_galaxy()
    cams = cams_for(tree)
    r0 = np.load(tmp_path / "rank0.npz")
    r1 = np.load(tmp_path / "rank1.npz")
    for k, cam in enumerate(cams):
        whole, _ = oracle.render(tree, cam)
        a, b = r0[f"arr_{k}"], r1[f"arr_{k}"]
        assert (a == b).all()                         # every rank holds the merged map
        tol = 0 if cam.mode == 2 else 1e-12 * np.abs(whole).max()
        assert np.abs(a - whole).max() <= tol
    assert float(r0["mx"][0]) == float(r1["mx"][0]) == 11.0
    assert int(r0["sm"][0]) == int(r1["sm"][0]) == 2001


def test_replica_throughput():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_throughput(2 * 10 ** 9, 100.0) == pytest.approx(20.0)
    assert bench.replica_throughput(8 * 10 ** 9, 100.0) == pytest.approx(80.0)
