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
