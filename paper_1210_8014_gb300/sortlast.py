"""Sort-last domain decomposition of the ray-casting pass (Sec. 3.1, 3.2).

The paper distributes the octree among processes, each rendering its own part
(sort-last compositing), and merges the partial images.  Because every leaf's contribution is added without ordering
(Sec. 2.2), partial maps rendered over disjoint leaf domains combine exactly:

  column : sum of the partial column maps
  max    : maximum of the partial maps (densities are positive)
  wmean  : sum_a w_a * sum_d column_d(rho v_a)  /  sum_d column_d(rho)
           (each domain renders column maps of rho and rho*v_x, rho*v_y,
           rho*v_z, so a weighted mean merges from sums alone)

Two forms of a domain's tree:
  domain_tree     the whole structure with the values of cells it does not own
                  zeroed: every domain traverses the same cells, so per-pixel
                  counts are identical across domains and are checked, not added;
  domain_subtree  only what the domain needs, for trees too large for one
                  device: the octs above its own cells, foreign subtrees cut
                  back to zero-valued leaves (and one level of zero-valued
                  children under an owned refined cell whose descendants are all
                  foreign, so cuts below that cell still read zeros there).
                  Partial maps merge exactly as before; counts are per domain
                  (they include the zero-valued cells it crosses) and are not
                  merged.

The domain split is spatial: leaves sorted by the Morton key of their centre
(at level 22) and cut into contiguous key ranges of equal leaf count.

On the GPU a domain renders its partial state directly (libamr's
amr_render_batch_partial: each pixel's accumulators, FP32 sums as compensated
(high, low) pairs, with rho and v read from the domain tree, foreign cells
holding zero density) and merge_device combines the domains on the device
(amr_merge_partials: TwoSum sums, then N / S for weighted means, max for MIP).
merge() and merge_distributed() are the host forms over plain maps, used by
CPU ranks.
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
    return replace(tree, fields=_fields_for(tree, owner == d, with_momentum))


def _fields_for(tree: Tree, mine: np.ndarray, with_momentum: bool) -> list:
    rho = np.where(mine, tree.fields[0], 0).astype(tree.fields[0].dtype)
    out = [rho]
    if with_momentum:
        for a in (1, 2, 3):
            out.append(np.where(mine, tree.fields[0].astype(np.float64) * tree.fields[a], 0)
                       .astype(tree.fields[0].dtype))
    else:
        out += [np.where(mine, f, 0).astype(f.dtype) for f in tree.fields[1:]]
    return out


def domain_subtree(tree: Tree, owner: np.ndarray, d: int, with_momentum: bool = False) -> Tree:
    """The pruned tree of domain d (see the module docstring): keeps oct o when
    its subtree holds a cell owned by d, or when o refines a cell owned by d
    (then, if nothing below o is owned by d, o is kept as zero-valued leaves).
    Values of cells not owned by d are zero.  The root is always kept."""
    n = tree.n_oct
    owned = owner == d
    child = tree.child
    level = tree.level.astype(np.int64)
    # sub[o]: the subtree of oct o holds a cell owned by d (children are deeper,
    # so one sweep from the deepest level up settles every oct)
    sub = owned.any(axis=1)
    for lv in range(int(level.max()), 0, -1):
        octs = np.nonzero(level == lv)[0]
        ch = child[octs]
        has = ch >= 0
        if has.any():
            hit = np.zeros(ch.shape, bool)
            hit[has] = sub[ch[has]]
            sub[octs] |= hit.any(axis=1)
    keep = np.zeros(n, bool)
    leafify = np.zeros(n, bool)          # kept with every cell a zero leaf
    keep[0] = True
    for lv in range(1, int(level.max()) + 1):
        octs = np.nonzero((level == lv) & keep & ~leafify)[0]
        ch = child[octs]
        has = ch >= 0
        if not has.any():
            continue
        c_oct = ch[has]
        c_owned = owned[octs][has]
        into = sub[c_oct]
        keep[c_oct[into]] = True
        zero = ~into & c_owned
        keep[c_oct[zero]] = True
        leafify[c_oct[zero]] = True
    old = np.nonzero(keep)[0]
    new_index = np.full(n, -1, np.int64)
    new_index[old] = np.arange(old.size)
    ch = child[old]
    nc = np.where(ch >= 0, new_index[np.maximum(ch, 0)], -1)
    nc[leafify[old]] = -1
    mine = owned[old] & ~leafify[old][:, None]
    sub_tree = Tree(level=tree.level[old].copy(), coord=tree.coord[old].copy(), child=nc.astype(np.int32),
                    fields=[], info=dict(tree.info))
    base = Tree(level=sub_tree.level, coord=sub_tree.coord, child=sub_tree.child,
                fields=[np.asarray(f)[old] for f in tree.fields], info=sub_tree.info)
    return replace(sub_tree, fields=_fields_for(base, mine, with_momentum))


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


def merge_device(cam: Camera, partials: Sequence, stream=None):
    """Merge the domains' partial renders of cam on the GPU (libamr's
    amr_merge_partials: compensated TwoSum sums, max for MIP).  partials: the
    per-domain tensors from Renderer.render_partial.  Returns the map tensor."""
    import torch
    from . import amr
    dt = torch.float64 if cam.precision == amr.AMR_PREC_FP64 else torch.float32
    out = torch.empty((cam.ny, cam.nx), dtype=dt, device=partials[0].device)
    s = stream if stream is not None else torch.cuda.current_stream(partials[0].device)
    amr.amr_merge_partials(cam.mode, cam.precision, cam.nx * cam.ny, list(partials), out, s.cuda_stream)
    return out


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
