"""Seeded synthetic inputs: octrees and cameras.

This module only *generates* inputs.  It holds none of the ray-casting
arithmetic, and both the CUDA library and the CPU oracle consume what it makes.

Trees follow the RAMSES octree model of Sec. 1 (octs of 8 cells, root oct at
level 1, refinement to level 22) in the linearised layout of
``amr_load_octree``: ``level[n_oct]`` u8, ``coord[n_oct][3]`` i32 (corner of the
oct's cell 0 in level-l cell units), ``child[n_oct][8]`` i32 (-1 = leaf) and
per-cell fields ``[n_oct][8]``.

Camera recipes reproduce the workload shapes: the tiny plain-method tree, the
galaxy-disk precision case, the 64-camera batch, the 8-frame zoom toward the
galactic centre and the interactive-zoom request stream (Sec. 1: iterative
zooming; Fig. 3: level-22, ~200M-cell Milky-Way output).
"""
from __future__ import annotations

import ctypes
import json
import math
from dataclasses import dataclass, field, replace
from typing import Callable, Optional, Sequence

import numpy as np

from . import _build

MODE_COLUMN, MODE_WMEAN, MODE_MAX, MODE_LEVEL = 0, 1, 2, 3
PREC_FP64, PREC_FP32_KAHAN, PREC_FP32_PLAIN = 0, 1, 2
LEVEL_AUTO = -1
MODE_NAMES = {MODE_COLUMN: "column", MODE_WMEAN: "wmean", MODE_MAX: "max", MODE_LEVEL: "level"}
PREC_NAMES = {PREC_FP64: "fp64", PREC_FP32_KAHAN: "fp32_kahan", PREC_FP32_PLAIN: "fp32_plain"}


# --------------------------------------------------------------------------- trees
@dataclass
class Tree:
    level: np.ndarray            # [n] uint8
    coord: np.ndarray            # [n, 3] int32
    child: np.ndarray            # [n, 8] int32
    fields: list                 # list of [n, 8] float32 / float64
    info: dict = field(default_factory=dict)

    @property
    def n_oct(self) -> int:
        return int(self.level.shape[0])

    @property
    def depth(self) -> int:
        return int(self.level.max())

    @property
    def n_leaves(self) -> int:
        return int((self.child < 0).sum())

    def astype(self, dtype) -> "Tree":
        return replace(self, fields=[np.ascontiguousarray(f, dtype=dtype) for f in self.fields])


class _GenParams(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int32), ("base_level", ctypes.c_int32), ("max_level", ctypes.c_int32),
                ("with_velocity", ctypes.c_int32), ("threshold", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("n_modes", ctypes.c_int32), ("n_clumps", ctypes.c_int32), ("n_threads", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


_gen = None


def _genlib():
    global _gen
    if _gen is None:
        lib = ctypes.CDLL(str(_build.build_gen()))
        lib.amrgen_build.argtypes = [ctypes.POINTER(_GenParams), ctypes.POINTER(ctypes.c_void_p)]
        lib.amrgen_build.restype = ctypes.c_int
        lib.amrgen_n_oct.argtypes = [ctypes.c_void_p]
        lib.amrgen_n_oct.restype = ctypes.c_int64
        lib.amrgen_n_fields.argtypes = [ctypes.c_void_p]
        lib.amrgen_n_fields.restype = ctypes.c_int32
        lib.amrgen_copy.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.POINTER(ctypes.c_void_p), ctypes.c_int32]
        lib.amrgen_copy.restype = ctypes.c_int
        lib.amrgen_info.argtypes = [ctypes.c_void_p, ctypes.c_char_p, ctypes.c_int64]
        lib.amrgen_info.restype = ctypes.c_int64
        lib.amrgen_free.argtypes = [ctypes.c_void_p]
        lib.amrgen_free.restype = None
        lib.amrgen_sample.argtypes = [ctypes.POINTER(_GenParams), ctypes.c_int32, ctypes.c_int64,
                                      ctypes.c_void_p, ctypes.c_void_p]
        lib.amrgen_sample.restype = ctypes.c_int
        _gen = lib
    return _gen


GEN_PLAIN, GEN_GALAXY = 0, 1


def _params(kind, base_level, max_level, threshold, seed=0, with_velocity=False, n_modes=256,
            n_clumps=0, n_threads=0) -> _GenParams:
    return _GenParams(kind, base_level, max_level, int(bool(with_velocity)), float(threshold),
                      int(seed) & 0xFFFFFFFFFFFFFFFF, n_modes, n_clumps, n_threads, 0)


def generate(kind, base_level, max_level, threshold, seed=0, with_velocity=False, n_modes=256,
             n_clumps=0, dtype=np.float32, n_threads=0) -> Tree:
    """Run the C++ generator and copy its arrays into numpy."""
    lib = _genlib()
    p = _params(kind, base_level, max_level, threshold, seed, with_velocity, n_modes, n_clumps, n_threads)
    h = ctypes.c_void_p()
    st = lib.amrgen_build(ctypes.byref(p), ctypes.byref(h))
    if st != 0:
        raise RuntimeError(f"amrgen_build failed ({st})")
    try:
        n = lib.amrgen_n_oct(h)
        nf = lib.amrgen_n_fields(h)
        level = np.empty(n, np.uint8)
        coord = np.empty((n, 3), np.int32)
        child = np.empty((n, 8), np.int32)
        fields = [np.empty((n, 8), dtype) for _ in range(nf)]
        ptrs = (ctypes.c_void_p * nf)(*[f.ctypes.data for f in fields])
        st = lib.amrgen_copy(h, level.ctypes.data, coord.ctypes.data, child.ctypes.data, ptrs,
                             1 if np.dtype(dtype) == np.float64 else 0)
        if st != 0:
            raise RuntimeError(f"amrgen_copy failed ({st})")
        buf = ctypes.create_string_buffer(1 << 14)
        lib.amrgen_info(h, buf, len(buf))
        info = json.loads(buf.value.decode())
    finally:
        lib.amrgen_free(h)
    info.update(kind=kind, base_level=base_level, max_level=max_level, threshold=threshold, seed=seed,
                n_modes=n_modes, n_clumps=n_clumps)
    return Tree(level, coord, child, fields, info)


def sample_model(kind, which, xyz, threshold=0.0, seed=0, with_velocity=False, n_modes=256, n_clumps=0):
    """The generator's point functions at points xyz[n, 3] (0 density, 1 g, 2..4 velocity)."""
    lib = _genlib()
    p = _params(kind, 1, 1, threshold, seed, with_velocity, n_modes, n_clumps)
    xyz = np.ascontiguousarray(xyz, np.float64)
    out = np.empty(xyz.shape[0], np.float64)
    st = lib.amrgen_sample(ctypes.byref(p), which, xyz.shape[0], xyz.ctypes.data, out.ctypes.data)
    if st != 0:
        raise RuntimeError(f"amrgen_sample failed ({st})")
    return out


def plain_tree(dtype=np.float64) -> Tree:
    """Plain-method tiny tree: base level 3, refine while rho V > 1e-4, cap 7."""
    return generate(GEN_PLAIN, 3, 7, 1e-4, dtype=dtype)


def galaxy_tree(seed, rel_threshold, max_level, with_velocity=True, n_clumps=0, dtype=np.float32,
                base_level=7, n_modes=256) -> Tree:
    return generate(GEN_GALAXY, base_level, max_level, rel_threshold, seed=seed, with_velocity=with_velocity,
                    n_modes=n_modes, n_clumps=n_clumps, dtype=dtype)


def complete_tree(depth: int, value: Callable[[np.ndarray, np.ndarray, np.ndarray, int], np.ndarray] | float = 1.0,
                  n_fields: int = 1, dtype=np.float64) -> Tree:
    """Every cell refined down to cells of level ``depth``; breadth-first order.

    ``value(x, y, z, level)`` gives field 0 at cell centres (arrays); the other
    fields are zero.  Refined cells hold the mean of their children.
    """
    levels, coords, childs = [], [], []
    offs = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], np.int32)
    cur = np.zeros((1, 3), np.int32)
    base = 0
    for lvl in range(1, depth + 1):
        n = cur.shape[0]
        levels.append(np.full(n, lvl, np.uint8))
        coords.append(cur)
        ch = np.full((n, 8), -1, np.int32)
        if lvl < depth:
            ch[:] = base + n + np.arange(n * 8, dtype=np.int64).reshape(n, 8)
        childs.append(ch)
        base += n
        cur = (2 * (cur[:, None, :] + offs[None, :, :])).reshape(-1, 3).astype(np.int32)
    level = np.concatenate(levels)
    coord = np.concatenate(coords)
    child = np.concatenate(childs)
    t = Tree(level, coord, child, [], {"kind": "complete", "depth": depth})
    rho = cell_values(t, value) if callable(value) else np.full((t.n_oct, 8), float(value))
    t.fields = [rho.astype(dtype)] + [np.zeros((t.n_oct, 8), dtype) for _ in range(n_fields - 1)]
    restrict(t)
    return t


def cell_centres(tree: Tree):
    """Centres (x, y, z) and levels of every cell, each [n_oct, 8]."""
    offs = np.array([[c & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], np.float64)
    h = np.ldexp(1.0, -tree.level.astype(np.int64))[:, None]
    ctr = (tree.coord[:, None, :].astype(np.float64) + offs[None] + 0.5) * h[..., None]
    lv = np.broadcast_to(tree.level[:, None], (tree.n_oct, 8))
    return ctr[..., 0], ctr[..., 1], ctr[..., 2], lv


def cell_values(tree: Tree, fn) -> np.ndarray:
    x, y, z, lv = cell_centres(tree)
    return np.asarray(fn(x, y, z, lv), np.float64) * np.ones_like(x)


def restrict(tree: Tree) -> None:
    """Refined cells take the mean of their children (deepest octs first)."""
    for lvl in range(int(tree.level.max()) - 1, 0, -1):
        o_idx, c_idx = np.nonzero((tree.child >= 0) & (tree.level[:, None] == lvl))
        if o_idx.size == 0:
            continue
        kids = tree.child[o_idx, c_idx]
        for f in tree.fields:
            f[o_idx, c_idx] = f[kids].mean(axis=1)


def split_leaf(tree: Tree, oct_index: int, cell: int) -> Tree:
    """Refine leaf (oct_index, cell) into 8 children holding its values."""
    assert tree.child[oct_index, cell] < 0
    n = tree.n_oct
    offs = np.array([cell & 1, (cell >> 1) & 1, (cell >> 2) & 1], np.int32)
    level = np.concatenate([tree.level, [tree.level[oct_index] + 1]]).astype(np.uint8)
    coord = np.concatenate([tree.coord, (2 * (tree.coord[oct_index] + offs))[None]]).astype(np.int32)
    child = np.concatenate([tree.child, np.full((1, 8), -1, np.int32)])
    child[oct_index, cell] = n
    fields = [np.concatenate([f, np.full((1, 8), f[oct_index, cell], f.dtype)]) for f in tree.fields]
    return Tree(level, coord, child, fields, dict(tree.info))


# --------------------------------------------------------------------------- cameras
@dataclass
class Camera:
    """Orthographic camera in box units (the box is [0,1)^3)."""
    centre: Sequence[float]
    u: Sequence[float]
    v: Sequence[float]
    w: Sequence[float]
    fov: Sequence[float]
    nx: int
    ny: int
    max_level: int = LEVEL_AUTO
    mode: int = MODE_COLUMN
    precision: int = PREC_FP64
    field_value: int = 0
    field_weight: int = 0
    field_vel: Sequence[int] = (1, 2, 3)

    def with_(self, **kw) -> "Camera":
        return replace(self, **kw)


def basis_from_direction(w) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """u = normalise(e x w) with e = e_z unless |w.e_z| > 0.9 (then e_x); v = w x u."""
    w = np.asarray(w, np.float64)
    w = w / np.linalg.norm(w)
    e = np.array([0.0, 0.0, 1.0]) if abs(w[2]) <= 0.9 else np.array([1.0, 0.0, 0.0])
    u = np.cross(e, w)
    u /= np.linalg.norm(u)
    v = np.cross(w, u)
    v /= np.linalg.norm(v)
    return u, v, w


def random_direction(rng: np.random.Generator) -> np.ndarray:
    z = rng.uniform(-1.0, 1.0)
    phi = rng.uniform(0.0, 2.0 * math.pi)
    r = math.sqrt(max(0.0, 1.0 - z * z))
    return np.array([r * math.cos(phi), r * math.sin(phi), z])


def camera_along(w, centre=(0.5, 0.5, 0.5), fov=1.0, n=256, **kw) -> Camera:
    u, v, w = basis_from_direction(w)
    fov2 = (float(fov), float(fov)) if np.isscalar(fov) else tuple(map(float, fov))
    nx, ny = (n, n) if np.isscalar(n) else n
    return Camera(tuple(map(float, centre)), tuple(u), tuple(v), tuple(w), fov2, int(nx), int(ny), **kw)


def axis_camera(n=256, fov=1.0, centre=(0.5, 0.5, 0.5), max_level=7, **kw) -> Camera:
    """+z view with u = +x, v = +y (pixel grid aligned with the octree)."""
    return Camera(tuple(map(float, centre)), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0),
                  (float(fov), float(fov)), n, n, max_level=max_level, **kw)


def disk_point(rng: np.random.Generator, normal) -> np.ndarray:
    """A point drawn from the disk: R ~ Gamma(2, 0.05), z ~ Laplace(0.005)."""
    n = np.asarray(normal, np.float64)
    ref = np.array([1.0, 0.0, 0.0]) if abs(n[0]) <= 0.9 else np.array([0.0, 1.0, 0.0])
    e1 = np.cross(n, ref)
    e1 /= np.linalg.norm(e1)
    e2 = np.cross(n, e1)
    R = min(rng.gamma(2.0, 0.05), 0.4)
    ang = rng.uniform(0.0, 2.0 * math.pi)
    z = rng.laplace(0.0, 0.005)
    return 0.5 + R * (math.cos(ang) * e1 + math.sin(ang) * e2) + z * n


# --------------------------------------------------------------------------- workloads
SIZES_BATCH = (128, 256, 512, 1024, 2048)
SIZES_SERVE = (256, 512, 1024, 2048)


def tiny_workload():
    """Plain method, tiny: ~30-40k leaves, f64, +z view, 256^2, level 7, column, FP64."""
    return plain_tree(np.float64), [axis_camera(256, max_level=7, mode=MODE_COLUMN, precision=PREC_FP64)]


def galaxy_precision_tree(dtype=np.float32) -> Tree:
    return galaxy_tree(2, 2.0 ** -20, 14, with_velocity=True, dtype=dtype)


def galaxy_precision_cameras(tree: Tree, n=1024, precisions=(PREC_FP64, PREC_FP32_KAHAN, PREC_FP32_PLAIN)):
    """Seeded random direction, whole-disk view, every mode x precision, full tree depth."""
    rng = np.random.default_rng(2)
    w = random_direction(rng)
    cams = []
    for p in precisions:
        for m in (MODE_COLUMN, MODE_WMEAN, MODE_MAX):
            cams.append(camera_along(w, fov=1.0, n=n, max_level=tree.depth, mode=m, precision=p))
    return cams


def batch_tree(dtype=np.float32) -> Tree:
    """~20M-leaf galaxy (levels 7-16, mass threshold 2^-22), density + velocity."""
    return galaxy_tree(3, 2.0 ** -22, 16, with_velocity=True, dtype=dtype)


def batch_cameras(tree: Tree, n_cams=64, precision=PREC_FP32_KAHAN, seed=3):
    """64 cameras: sizes uniform over 128^2..2048^2, fov log-uniform [1/64, 1],
    centred on seeded disk points, random directions, level by the pixel rule,
    modes uniform."""
    rng = np.random.default_rng(seed)
    normal = tree.info.get("normal", (0.0, 0.0, 1.0))
    cams = []
    for _ in range(n_cams):
        n = int(rng.choice(SIZES_BATCH))
        fov = float(2.0 ** rng.uniform(-6.0, 0.0))
        centre = disk_point(rng, normal)
        w = random_direction(rng)
        mode = int(rng.integers(0, 3))
        cams.append(camera_along(w, centre=centre, fov=fov, n=n, max_level=LEVEL_AUTO, mode=mode,
                                 precision=precision))
    return cams


# Relative mass threshold of the level-22 zoom tree, picked once by bisection on
# the generator's leaf count (target ~200M leaves): 2^-24 gives 57.7M leaves,
# 2^-25 116.8M, 2^-25.75 193.2M (27.6M octs, leaves at levels 7-22).
ZOOM_THRESHOLD = 2.0 ** -25.75


def zoom_tree(dtype=np.float32, threshold=ZOOM_THRESHOLD) -> Tree:
    """Milky-Way scale: levels 7-22, 64 Plummer clumps + 1 central, density only."""
    return galaxy_tree(4, threshold, 22, with_velocity=False, n_clumps=64, dtype=dtype)


def zoom_cameras(tree: Tree, n_frames=8, n=4096, precision=PREC_FP32_KAHAN):
    """8 frames of n^2, fov 1 -> 1/128 (halving) toward the galactic centre."""
    rng = np.random.default_rng(4)
    w = random_direction(rng)
    return [camera_along(w, centre=(0.5, 0.5, 0.5), fov=2.0 ** -f, n=n, max_level=LEVEL_AUTO,
                         mode=MODE_COLUMN, precision=precision) for f in range(n_frames)]


def deep_centre_camera(tree: Tree, n=512, precision=PREC_FP32_KAHAN, mode=MODE_COLUMN):
    """Full-depth view of the galactic centre: fov 2^-13 at 512^2 puts the pixel
    rule at level 22."""
    rng = np.random.default_rng(44)
    return camera_along(random_direction(rng), centre=(0.5, 0.5, 0.5), fov=2.0 ** -13, n=n, max_level=LEVEL_AUTO,
                        mode=mode, precision=precision)


def request_stream(tree: Tree, duration_s=60.0, rate=50.0, seed=5, precision=PREC_FP32_KAHAN):
    """Poisson arrivals; each request a random-direction camera around a disk point,
    size uniform over 256^2..2048^2, fov log-uniform [2^-12, 1], mode uniform."""
    rng = np.random.default_rng(seed)
    normal = tree.info.get("normal", (0.0, 0.0, 1.0))
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= duration_s:
            break
        n = int(rng.choice(SIZES_SERVE))
        fov = float(2.0 ** rng.uniform(-12.0, 0.0))
        centre = disk_point(rng, normal)
        w = random_direction(rng)
        mode = int(rng.integers(0, 3))
        out.append((t, camera_along(w, centre=centre, fov=fov, n=n, max_level=LEVEL_AUTO, mode=mode,
                                    precision=precision)))
    return out


def random_tree(rng: np.random.Generator, depth: int, p_refine: float = 0.4, n_fields: int = 4,
                dtype=np.float64, positive: bool = True) -> Tree:
    """Small random octree: every cell of level < depth refined with probability
    p_refine (the root's cells always); seeded uniform values in [0.5, 2) for
    field 0 (density) and [-1, 1) for the others."""
    level, coord, child = [1], [[0, 0, 0]], [[-1] * 8]
    frontier = [0]
    while frontier:
        nxt = []
        for o in frontier:
            lvl = level[o]
            if lvl >= depth:
                continue
            for c in range(8):
                if lvl == 1 or rng.random() < p_refine:
                    child[o][c] = len(level)
                    level.append(lvl + 1)
                    coord.append([2 * (coord[o][a] + ((c >> a) & 1)) for a in range(3)])
                    child.append([-1] * 8)
                    nxt.append(len(level) - 1)
        frontier = nxt
    n = len(level)
    lo = 0.5 if positive else -1.0
    fields = [rng.uniform(lo, 2.0, (n, 8))] + [rng.uniform(-1.0, 1.0, (n, 8)) for _ in range(n_fields - 1)]
    t = Tree(np.array(level, np.uint8), np.array(coord, np.int32), np.array(child, np.int32),
             [f.astype(dtype) for f in fields], {"kind": "random", "depth": depth})
    return t


# --------------------------------------------------------------------------- tree files
TREE_MAGIC = b"AMRTREE1"


def save_tree(tree: Tree, path) -> None:
    """Write a tree as one file: magic, a JSON header (sizes, dtypes, level
    histogram, generator parameters, a CRC-32 of the payload) and the raw
    little-endian arrays level, coord, child, fields in that order."""
    import json
    import zlib
    arrays = [np.ascontiguousarray(tree.level, "<u1"), np.ascontiguousarray(tree.coord, "<i4"),
              np.ascontiguousarray(tree.child, "<i4")]
    fdt = "<f8" if tree.fields and tree.fields[0].dtype == np.float64 else "<f4"
    arrays += [np.ascontiguousarray(f, fdt) for f in tree.fields]
    crc = 0
    for a in arrays:
        crc = zlib.crc32(memoryview(a).cast("B"), crc)
    lv = tree.level.astype(np.int64)
    leaf_hist = np.bincount(np.repeat(lv, (tree.child < 0).sum(axis=1)), minlength=23)
    header = {"n_oct": tree.n_oct, "n_fields": len(tree.fields), "field_dtype": fdt, "crc32": crc,
              "leaf_hist": {str(l): int(n) for l, n in enumerate(leaf_hist) if n},
              "info": {k: v for k, v in tree.info.items() if isinstance(v, (int, float, str, list, dict))}}
    hb = json.dumps(header).encode()
    with open(path, "wb") as f:
        f.write(TREE_MAGIC)
        f.write(len(hb).to_bytes(8, "little"))
        f.write(hb)
        for a in arrays:
            f.write(memoryview(a).cast("B"))


def load_tree(path) -> Tree:
    """Read a file written by save_tree; raises ValueError on a bad magic,
    truncation or a checksum mismatch."""
    import json
    import zlib
    with open(path, "rb") as f:
        if f.read(8) != TREE_MAGIC:
            raise ValueError(f"{path}: not a tree file")
        hlen = int.from_bytes(f.read(8), "little")
        header = json.loads(f.read(hlen).decode())
        n, nf, fdt = header["n_oct"], header["n_fields"], header["field_dtype"]
        specs = [("<u1", (n,)), ("<i4", (n, 3)), ("<i4", (n, 8))] + [(fdt, (n, 8))] * nf
        arrays, crc = [], 0
        for dt, shape in specs:
            count = int(np.prod(shape))
            a = np.fromfile(f, dtype=dt, count=count)
            if a.size != count:
                raise ValueError(f"{path}: truncated")
            crc = zlib.crc32(memoryview(a).cast("B"), crc)
            arrays.append(a.reshape(shape))
    if crc != header["crc32"]:
        raise ValueError(f"{path}: checksum mismatch")
    native = np.float64 if fdt == "<f8" else np.float32
    return Tree(arrays[0].astype(np.uint8), arrays[1].astype(np.int32), arrays[2].astype(np.int32),
                [a.astype(native) for a in arrays[3:]], dict(header.get("info", {})))


def cached(name: str, make, cache_dir=None) -> Tree:
    """make() once per name and keep the tree in cache_dir (env AMR_TREE_CACHE;
    no caching when neither is set)."""
    import os
    from pathlib import Path
    d = cache_dir or os.environ.get("AMR_TREE_CACHE")
    if not d:
        return make()
    p = Path(d) / f"{name}.amrtree"
    if p.exists():
        try:
            return load_tree(p)
        except ValueError:
            p.unlink()
    t = make()
    Path(d).mkdir(parents=True, exist_ok=True)
    tmp = p.with_suffix(".tmp")
    save_tree(t, tmp)
    tmp.replace(p)
    return t
