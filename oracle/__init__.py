"""CPU oracle for the octree ray-casting pass — TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline /
reference leg may import this package.  The product library never calls it and
has no fallback to it.  It shares no code with the CUDA path: it is compiled
from ``amr_oracle.c`` alone, and its camera record is declared here, not taken
from the product's headers.

``render()``     plain FP64 walk of Sec. 2.2 (C, OpenMP, exact __int128 tests).
``touched()``    the same walk, instrumented: which leaves and refined cells a
                 camera's rays touch (the data a frame must read at least once).
``bruteforce``   O(pixels x leaves) slab tests in exact integers (numpy), the
                 independent check that pins the walk on tiny trees.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from pathlib import Path

import numpy as np

HERE = Path(__file__).resolve().parent
SRC = HERE / "amr_oracle.c"
LIB = HERE / "liboracle.so"

OR_OK, OR_E_INVALID, OR_E_BADTREE = 0, -1, -2


class OracleCamera(ctypes.Structure):
    _fields_ = [("centre", ctypes.c_double * 3), ("u", ctypes.c_double * 3), ("v", ctypes.c_double * 3),
                ("w", ctypes.c_double * 3), ("fov", ctypes.c_double * 2), ("nx", ctypes.c_int32),
                ("ny", ctypes.c_int32), ("max_level", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("field_value", ctypes.c_int32), ("field_weight", ctypes.c_int32),
                ("field_vel", ctypes.c_int32 * 3), ("reserved", ctypes.c_int32)]


def compile_command(out: Path = LIB) -> list[str]:
    return ["gcc", "-O2", "-std=gnu11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
            "-shared", "-Wall", str(SRC), "-o", str(out), "-lm"]


def build(force: bool = False) -> Path:
    if force or not LIB.exists() or LIB.stat().st_mtime < SRC.stat().st_mtime:
        tmp = LIB.with_suffix(".so.tmp%d" % os.getpid())
        res = subprocess.run(compile_command(tmp), stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
        if res.returncode != 0:
            raise RuntimeError("oracle build failed:\n" + res.stdout)
        tmp.replace(LIB)
    return LIB


_lib = None


def load(path: Path | None = None):
    """Load liboracle (building it first if needed)."""
    global _lib
    if path is not None:
        lib = ctypes.CDLL(str(path))
    else:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(str(build()))
    P = ctypes.c_void_p
    lib.oracle_render.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_int32, ctypes.POINTER(P),
                                  ctypes.POINTER(OracleCamera), ctypes.c_int64, P, P, P, P, ctypes.c_int32]
    lib.oracle_render.restype = ctypes.c_int
    lib.oracle_view_info.argtypes = [ctypes.c_int64, P, ctypes.POINTER(OracleCamera), P, P, P]
    lib.oracle_view_info.restype = ctypes.c_int
    lib.oracle_ray_origin.argtypes = [ctypes.POINTER(OracleCamera), ctypes.c_int32, ctypes.c_int32, P]
    lib.oracle_ray_origin.restype = ctypes.c_int
    lib.oracle_slice.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_int32, ctypes.POINTER(P),
                                 ctypes.POINTER(OracleCamera), P, P, ctypes.c_int32]
    lib.oracle_slice.restype = ctypes.c_int
    lib.oracle_touched.argtypes = [ctypes.c_int64, P, P, P, ctypes.c_int32, ctypes.POINTER(P),
                                   ctypes.POINTER(OracleCamera), P, P, ctypes.c_int32]
    lib.oracle_touched.restype = ctypes.c_int
    if path is None:
        _lib = lib
    return lib


def to_camera(cam) -> OracleCamera:
    """Marshal any object with the camera attributes into the oracle's record."""
    c = OracleCamera()
    for name in ("centre", "u", "v", "w"):
        getattr(c, name)[:] = [float(x) for x in getattr(cam, name)]
    c.fov[:] = [float(x) for x in cam.fov]
    c.nx, c.ny, c.max_level, c.mode = int(cam.nx), int(cam.ny), int(cam.max_level), int(cam.mode)
    c.field_value, c.field_weight = int(cam.field_value), int(cam.field_weight)
    c.field_vel[:] = [int(x) for x in cam.field_vel]
    return c


class Prepared:
    """The oracle's view of a tree: contiguous arrays, fields widened to float64
    once (exact for float32 input), so repeated renders pay no conversion."""

    def __init__(self, tree):
        self.level = np.ascontiguousarray(tree.level, np.uint8)
        self.coord = np.ascontiguousarray(tree.coord, np.int32)
        self.child = np.ascontiguousarray(tree.child, np.int32)
        self.fields = [np.ascontiguousarray(f, np.float64) for f in tree.fields]
        self.ptrs = (ctypes.c_void_p * len(self.fields))(*[f.ctypes.data for f in self.fields])


def prepare(tree) -> Prepared:
    return tree if isinstance(tree, Prepared) else Prepared(tree)


def render(tree, cam, pixels=None, threads: int = 0, lib=None):
    """FP64 map and per-pixel leaf counts.

    tree: an input tree or a Prepared one.  pixels: None for the whole [ny, nx]
    map, else (i_array, j_array) and the results are 1-D in that order.
    """
    lib = lib or load()
    t = prepare(tree)
    level, coord, child, f64, ptrs = t.level, t.coord, t.child, t.fields, t.ptrs
    c = to_camera(cam)
    if pixels is None:
        n_pix, pi, pj = -1, None, None
        shape = (int(cam.ny), int(cam.nx))
    else:
        pi = np.ascontiguousarray(pixels[0], np.int32)
        pj = np.ascontiguousarray(pixels[1], np.int32)
        n_pix, shape = pi.shape[0], (pi.shape[0],)
    out = np.zeros(shape, np.float64)
    cnt = np.zeros(shape, np.int32)
    st = lib.oracle_render(level.shape[0], level.ctypes.data, coord.ctypes.data, child.ctypes.data, len(f64),
                           ptrs, ctypes.byref(c), n_pix, None if pi is None else pi.ctypes.data,
                           None if pj is None else pj.ctypes.data, out.ctypes.data, cnt.ctypes.data, threads)
    if st != OR_OK:
        raise ValueError(f"oracle_render failed ({st})")
    return out, cnt


def view_info(tree, cam, lib=None):
    """(L, D[3], lambda) of the camera's quantised ray family."""
    lib = lib or load()
    level = np.ascontiguousarray(tree.level, np.uint8)
    L = np.zeros(1, np.int32)
    D = np.zeros(3, np.int64)
    lam = np.zeros(1, np.float64)
    st = lib.oracle_view_info(level.shape[0], level.ctypes.data, ctypes.byref(to_camera(cam)), L.ctypes.data,
                              D.ctypes.data, lam.ctypes.data)
    if st != OR_OK:
        raise ValueError(f"oracle_view_info failed ({st})")
    return int(L[0]), D, float(lam[0])


def ray_origin(cam, i, j, lib=None):
    lib = lib or load()
    X0 = np.zeros(3, np.int64)
    st = lib.oracle_ray_origin(ctypes.byref(to_camera(cam)), int(i), int(j), X0.ctypes.data)
    if st != OR_OK:
        raise ValueError(f"oracle_ray_origin failed ({st})")
    return X0


def slice_map(tree, cam, threads: int = 0, lib=None):
    """Slice map: (values float64 [ny, nx], leaf levels int32 [ny, nx])."""
    lib = lib or load()
    t = prepare(tree)
    c = to_camera(cam)
    out = np.zeros((int(cam.ny), int(cam.nx)), np.float64)
    lv = np.zeros((int(cam.ny), int(cam.nx)), np.int32)
    st = lib.oracle_slice(t.level.shape[0], t.level.ctypes.data, t.coord.ctypes.data, t.child.ctypes.data,
                          len(t.fields), t.ptrs, ctypes.byref(c), out.ctypes.data, lv.ctypes.data, threads)
    if st != OR_OK:
        raise ValueError(f"oracle_slice failed ({st})")
    return out, lv


def touched(tree, cam, leaf=None, inner=None, threads: int = 0, lib=None):
    """Instrumented pass over every pixel ray of cam: boolean [n_oct, 8] masks
    of the leaves crossed and of the refined cells descended through.  Pass
    masks (uint8 [n_oct, 8]) to accumulate over several cameras."""
    lib = lib or load()
    t = prepare(tree)
    n = t.level.shape[0]
    leaf = np.zeros((n, 8), np.uint8) if leaf is None else leaf
    inner = np.zeros((n, 8), np.uint8) if inner is None else inner
    assert leaf.dtype == np.uint8 and inner.dtype == np.uint8 and leaf.flags.c_contiguous and inner.flags.c_contiguous
    st = lib.oracle_touched(n, t.level.ctypes.data, t.coord.ctypes.data, t.child.ctypes.data, len(t.fields), t.ptrs,
                            ctypes.byref(to_camera(cam)), leaf.ctypes.data, inner.ctypes.data, threads)
    if st != OR_OK:
        raise ValueError(f"oracle_touched failed ({st})")
    return leaf, inner
