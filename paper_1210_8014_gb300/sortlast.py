"""Sort-last domain decomposition of the ray-casting pass (Sec. 3.1, 3.2).

The paper distributes the octree among processes, each rendering its own part
(sort-last compositing), and merges the partial images.  Because every leaf's contribution is added without ordering
(Sec. 2.2), partial maps rendered over disjoint leaf domains combine exactly:

  column : sum of the partial column maps
  max    : maximum of the partial maps (densities are positive)
  wmean  : sum_a w_a * sum_d column_d(rho v_a)  /  sum_d column_d(rho)
           (each domain renders column maps of rho and rho*v_x, rho*v_y,
           rho*v_z, so a weighted mean merges from sums alone)

Each domain keeps the whole tree structure and zeroes the values of leaves it
does not own, so every domain traverses the same cells: per-pixel counts are
identical across domains and are checked, not added.

The domain split is spatial: leaves sorted by the Morton key of their centre
(at level 22) and cut into contiguous key ranges of equal leaf count.
"""
from __future__ import annotations

from dataclasses import replace
from typing import Sequence

import numpy as np

from .inputs import MODE_COLUMN, MODE_MAX, MODE_WMEAN, Camera, Tree, cell_centres


def _spread3(v: np.ndarray) -> np.ndarray:
    """Interleave the low 21 bits of v with two zero bits between each."""
    v = v.astype(np.uint64) & np.uint64(0x1FFFFF)
    v = (v | (v << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    v = (v | (v << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    v = (v | (v << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    v = (v | (v << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    v = (v | (v << np.uint64(2))) & np.uint64(0x1249249249249249)
    return v


def morton_keys(tree: Tree) -> np.ndarray:
    """Morton key of every cell centre on the 2^21 grid, [n_oct, 8] uint64."""
    x, y, z, _ = cell_centres(tree)
    q = [np.minimum(np.floor(a * (1 << 21)), (1 << 21) - 1).astype(np.uint64) for a in (x, y, z)]
    return _spread3(q[0]) | (_spread3(q[1]) << np.uint64(1)) | (_spread3(q[2]) << np.uint64(2))


def domain_owner(tree: Tree, n_domains: int) -> np.ndarray:
    """Domain index of every cell, [n_oct, 8] int32: the Morton key range is cut
    so that each domain holds (nearly) the same number of leaves; every cell,
    refined or not, belongs to the range holding its centre (a refined cell is
    read only at a level cut, and then its owner alone adds it)."""
    keys = morton_keys(tree)
    leaf = tree.child < 0
    lk = np.sort(keys[leaf])
    if n_domains < 1:
        raise ValueError("need at least one domain")
    bounds = lk[np.linspace(0, lk.size, n_domains + 1).astype(np.int64)[1:-1]] if n_domains > 1 else np.array([], np.uint64)
    return np.searchsorted(bounds, keys, side="right").astype(np.int32)


def domain_tree(tree: Tree, owner: np.ndarray, d: int, with_momentum: bool = False) -> Tree:
    """The tree with the values of cells outside domain d set to zero.  With
    with_momentum, fields become [rho, rho*v_x, rho*v_y, rho*v_z] (the column
    fields a weighted-mean merge needs)."""
    mine = owner == d
    rho = np.where(mine, tree.fields[0], 0)
    fields = [rho.astype(tree.fields[0].dtype)]
    if with_momentum:
        for a in (1, 2, 3):
            fields.append(np.where(mine, tree.fields[0].astype(np.float64) * tree.fields[a], 0)
                          .astype(tree.fields[0].dtype))
    else:
        fields += [np.where(mine, f, 0).astype(f.dtype) for f in tree.fields[1:]]
    return replace(tree, fields=fields)


def partial_cameras(cam: Camera) -> list[Camera]:
    """The column/max renders whose maps make up one domain's partial state for cam."""
    if cam.mode == MODE_WMEAN:
        return [cam.with_(mode=MODE_COLUMN, field_value=f) for f in (0, 1, 2, 3)]
    return [cam]


def merge(cam: Camera, partials: Sequence[Sequence[np.ndarray]], counts: Sequence[np.ndarray] | None = None):
    """Merge per-domain partial maps for cam.

    partials[d] is the list of maps partial_cameras(cam) rendered for domain d.
    Returns (map, counts) with sums taken in float64."""
    if counts is not None:
        for c in counts[1:]:
            if not np.array_equal(c, counts[0]):
                raise ValueError("domains traversed different cells")
    if cam.mode == MODE_MAX:
        out = np.max(np.stack([np.asarray(p[0], np.float64) for p in partials]), axis=0)
    elif cam.mode == MODE_COLUMN:
        out = np.sum(np.stack([np.asarray(p[0], np.float64) for p in partials]), axis=0)
    else:
        tot = [np.sum(np.stack([np.asarray(p[k], np.float64) for p in partials]), axis=0) for k in range(4)]
        w = np.asarray(cam.w, np.float64)
        num = w[0] * tot[1] + w[1] * tot[2] + w[2] * tot[3]
        out = np.divide(num, tot[0], out=np.zeros_like(num), where=tot[0] != 0)
    return out, (counts[0] if counts is not None else None)


def merge_distributed(cam: Camera, local_partial: Sequence, group=None):
    """Merge this rank's partial maps with every other rank's through
    torch.distributed (sum for column-type maps, max for MIP) and return the
    final map on every rank.  The maps travel as host float64 tensors (gloo
    backend); a GPU rank copies its partial maps to the host first."""
    import torch
    import torch.distributed as dist
    if cam.mode == MODE_MAX:
        t = torch.as_tensor(np.asarray(local_partial[0], np.float64))
        dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
        return t.numpy()
    stacked = torch.as_tensor(np.stack([np.asarray(p, np.float64) for p in local_partial]))
    dist.all_reduce(stacked, op=dist.ReduceOp.SUM, group=group)
    tot = stacked.numpy()
    if cam.mode == MODE_COLUMN:
        return tot[0]
    w = np.asarray(cam.w, np.float64)
    num = w[0] * tot[1] + w[1] * tot[2] + w[2] * tot[3]
    return np.divide(num, tot[0], out=np.zeros_like(num), where=tot[0] != 0)
