"""ctypes binding of libamr (include/amr.h), same names as the C entry points.

Argument marshalling only: every step of the ray-casting pass runs in the CUDA
kernels of libamr.  There is no host fallback; importing this module fails
loudly when the library cannot be built or loaded.

Arrays may be numpy arrays (host) or torch tensors (host or device); device
buffers and streams come from PyTorch.
"""
from __future__ import annotations

import ctypes
import json
from typing import Optional, Sequence

import numpy as np

from . import _build
from .inputs import Camera, Tree

AMR_OK, AMR_E_INVALID, AMR_E_BADTREE, AMR_E_OOM, AMR_E_CUDA = 0, -1, -2, -3, -4
AMR_E_TIMEOUT, AMR_E_BUSY, AMR_E_CANCELLED = -5, -6, -7
AMR_F32, AMR_F64 = 0, 1
AMR_MODE_COLUMN, AMR_MODE_WMEAN, AMR_MODE_MAX, AMR_MODE_LEVEL = 0, 1, 2, 3
AMR_PREC_FP64, AMR_PREC_FP32_KAHAN, AMR_PREC_FP32_PLAIN = 0, 1, 2
AMR_LEVEL_AUTO = -1

STATUS_NAMES = {0: "AMR_OK", -1: "AMR_E_INVALID", -2: "AMR_E_BADTREE", -3: "AMR_E_OOM", -4: "AMR_E_CUDA",
                -5: "AMR_E_TIMEOUT", -6: "AMR_E_BUSY", -7: "AMR_E_CANCELLED"}


class AmrError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class amr_camera(ctypes.Structure):
    _fields_ = [("centre", ctypes.c_double * 3), ("u", ctypes.c_double * 3), ("v", ctypes.c_double * 3),
                ("w", ctypes.c_double * 3), ("fov", ctypes.c_double * 2), ("nx", ctypes.c_int32),
                ("ny", ctypes.c_int32), ("max_level", ctypes.c_int32), ("mode", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("field_value", ctypes.c_int32), ("field_weight", ctypes.c_int32),
                ("field_vel", ctypes.c_int32 * 3)]


class amr_options(ctypes.Structure):
    _fields_ = [("tile_w", ctypes.c_int32), ("tile_h", ctypes.c_int32), ("block_threads", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("tiles_per_grab", ctypes.c_int32), ("use_graph", ctypes.c_int32),
                ("max_regs", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: int(getattr(self, k)) for k, _ in self._fields_}


_lib = None


def lib():
    """Load libamr (compiling it in-tree first if its sources changed)."""
    global _lib
    if _lib is None:
        path = _build.build_amr()
        L = ctypes.CDLL(str(path))
        P, I32, I64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64
        sigs = {
            "amr_create": [ctypes.POINTER(P), ctypes.c_int],
            "amr_destroy": [P],
            "amr_load_octree": [P, I64, P, P, P, I32, ctypes.POINTER(P), I32],
            "amr_render": [P, ctypes.POINTER(amr_camera), P, P, ctypes.c_int, P],
            "amr_render_batch": [P, I32, ctypes.POINTER(amr_camera), ctypes.POINTER(P), ctypes.POINTER(P),
                                 ctypes.c_int, P],
            "amr_camera_check": [P, ctypes.POINTER(amr_camera), ctypes.POINTER(I32)],
            "amr_slice": [P, ctypes.POINTER(amr_camera), P, P, ctypes.c_int, P],
            "amr_blur": [P, I32, I32, P, P, ctypes.c_double, P, P],
            "amr_set_options": [P, ctypes.POINTER(amr_options)],
            "amr_get_options": [P, ctypes.POINTER(amr_options)],
            "amr_autotune": [P, I32, ctypes.POINTER(amr_camera), I32, ctypes.POINTER(amr_options),
                             ctypes.POINTER(ctypes.c_double)],
            "amr_server_config": [P, I32, I64, I32],
            "amr_submit": [P, ctypes.POINTER(amr_camera), P, P, ctypes.POINTER(ctypes.c_uint64)],
            "amr_wait": [P, ctypes.c_uint64, I64],
            "amr_cancel": [P, ctypes.c_uint64],
            "amr_stats": [P, ctypes.c_char_p, I64],
            "amr_tree_info": [P, ctypes.POINTER(I64), ctypes.POINTER(I32), ctypes.POINTER(I64)],
            "amr_render_batch_noalloc": [I64, P, I32, I32, ctypes.POINTER(P), I32, I32, ctypes.POINTER(amr_camera),
                                         ctypes.POINTER(P), ctypes.POINTER(P), P],
            "amr_noalloc_status": [P, ctypes.POINTER(I32), ctypes.POINTER(I32), ctypes.POINTER(ctypes.c_uint64)],
            "amr_render_batch_partial": [P, I32, ctypes.POINTER(amr_camera), ctypes.POINTER(P), ctypes.POINTER(P), P],
            "amr_merge_partials": [I32, I32, I32, I64, ctypes.POINTER(P), P, P],
        }
        for name, args in sigs.items():
            fn = getattr(L, name)
            fn.argtypes = args
            fn.restype = ctypes.c_int32
        L.amr_last_error.argtypes = [P]
        L.amr_last_error.restype = ctypes.c_char_p
        _lib = L
    return _lib


def amr_last_error(ctx=None) -> str:
    return lib().amr_last_error(ctx).decode(errors="replace")


def _check(st: int) -> None:
    if st != AMR_OK:
        raise AmrError(st, amr_last_error())


def _ptr(x) -> Optional[int]:
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    if isinstance(x, np.ndarray):
        return x.ctypes.data
    raise TypeError(f"cannot take a pointer of {type(x)}")


def _buf(x, n: int, itemsize: int, kind: str, where: Optional[str], name: str) -> Optional[int]:
    """Pointer of a buffer a call reads or writes, after checking what the C
    call will touch (the library cannot): at least n elements of itemsize
    bytes of the right kind ('f' float, 'i' integer), contiguous, on the
    expected side ('device', 'host', or None for either).  Raw integer
    pointers pass unchecked."""
    if x is None or isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        is_float, count, size, dev = x.is_floating_point(), x.numel(), x.element_size(), x.is_cuda
        contiguous = x.is_contiguous()
        ptr = x.data_ptr
    elif isinstance(x, np.ndarray):
        is_float, count, size, dev = x.dtype.kind == "f", x.size, x.itemsize, False
        contiguous = x.flags.c_contiguous
        ptr = lambda: x.ctypes.data
    else:
        raise TypeError(f"{name}: cannot take a pointer of {type(x)}")
    if not contiguous:
        raise ValueError(f"{name}: buffer is not contiguous")
    if is_float != (kind == "f") or size != itemsize:
        want = ("float" if kind == "f" else "int") + str(8 * itemsize)
        raise ValueError(f"{name}: need {want} elements")
    if count < n:
        raise ValueError(f"{name}: {count} elements, need {n}")
    if where == "device" and not dev:
        raise ValueError(f"{name}: a host buffer where a device buffer is needed")
    if where == "current-device":
        import torch
        if not dev:
            raise ValueError(f"{name}: a host buffer where a device buffer is needed")
        if x.device.index != torch.cuda.current_device():
            raise ValueError(f"{name}: on cuda:{x.device.index}, but the call runs on the current device "
                             f"cuda:{torch.cuda.current_device()}")
    if where == "host" and dev:
        raise ValueError(f"{name}: a device buffer where a host buffer is needed")
    return ptr()


def _map_size(cam: Camera) -> int:
    return 8 if int(cam.precision) == AMR_PREC_FP64 else 4


def _side(out_on_device) -> str:
    return "device" if out_on_device else "host"


def to_camera(cam: Camera) -> amr_camera:
    c = amr_camera()
    for name in ("centre", "u", "v", "w"):
        getattr(c, name)[:] = [float(x) for x in getattr(cam, name)]
    c.fov[:] = [float(x) for x in cam.fov]
    c.nx, c.ny, c.max_level = int(cam.nx), int(cam.ny), int(cam.max_level)
    c.mode, c.precision = int(cam.mode), int(cam.precision)
    c.field_value, c.field_weight = int(cam.field_value), int(cam.field_weight)
    c.field_vel[:] = [int(x) for x in cam.field_vel]
    return c


# ---------------------------------------------------------------- entry points
def amr_create(device: int = 0) -> int:
    h = ctypes.c_void_p()
    _check(lib().amr_create(ctypes.byref(h), device))
    return h.value


def amr_destroy(ctx) -> None:
    _check(lib().amr_destroy(ctx))


def amr_load_octree(ctx, n_oct, level, coord, child, fields: Sequence, field_dtype: int) -> None:
    n = int(n_oct)
    fsize = 8 if int(field_dtype) == AMR_F64 else 4
    ptrs = (ctypes.c_void_p * len(fields))(*[_buf(f, n * 8, fsize, "f", "host", f"fields[{i}]")
                                             for i, f in enumerate(fields)])
    _check(lib().amr_load_octree(ctx, n, _buf(level, n, 1, "i", "host", "level"),
                                 _buf(coord, n * 3, 4, "i", "host", "coord"), _buf(child, n * 8, 4, "i", "host", "child"),
                                 len(fields), ptrs, int(field_dtype)))


def amr_render(ctx, cam: Camera, map_out, count_out=None, out_on_device: int = 1, cuda_stream=None) -> None:
    c = to_camera(cam)
    px, side = int(cam.nx) * int(cam.ny), _side(out_on_device)
    m = _buf(map_out, px, _map_size(cam), "f", side, "map_out")
    k = _buf(count_out, px, 4, "i", side, "count_out")
    _check(lib().amr_render(ctx, ctypes.byref(c), m, k, int(out_on_device),
                            _ptr(cuda_stream) if cuda_stream is not None else None))


def amr_render_batch(ctx, cams: Sequence[Camera], maps: Sequence, counts: Optional[Sequence] = None,
                     out_on_device: int = 1, cuda_stream=None) -> None:
    n = len(cams)
    if len(maps) != n or (counts is not None and len(counts) != n):
        raise ValueError("one map (and one counts entry, if counts are given) per camera")
    carr = (amr_camera * n)(*[to_camera(c) for c in cams])
    side = _side(out_on_device)
    marr = (ctypes.c_void_p * n)(*[_buf(m, int(c.nx) * int(c.ny), _map_size(c), "f", side, f"maps[{i}]")
                                   for i, (m, c) in enumerate(zip(maps, cams))])
    karr = (ctypes.c_void_p * n)(*[_buf(k, int(c.nx) * int(c.ny), 4, "i", side, f"counts[{i}]")
                                   for i, (k, c) in enumerate(zip(counts, cams))]) if counts is not None else None
    _check(lib().amr_render_batch(ctx, n, carr, marr, karr, int(out_on_device),
                                  _ptr(cuda_stream) if cuda_stream is not None else None))


def amr_slice(ctx, cam: Camera, map_out, level_out=None, out_on_device: int = 1, cuda_stream=None) -> None:
    c = to_camera(cam)
    px, side = int(cam.nx) * int(cam.ny), _side(out_on_device)
    m = _buf(map_out, px, _map_size(cam), "f", side, "map_out")
    lv = _buf(level_out, px, 4, "i", side, "level_out")
    _check(lib().amr_slice(ctx, ctypes.byref(c), m, lv, int(out_on_device),
                           _ptr(cuda_stream) if cuda_stream is not None else None))


def amr_blur(ctx, nx: int, ny: int, map_in, level, pixel: float, map_out, cuda_stream=None) -> None:
    px = int(nx) * int(ny)
    a = _buf(map_in, px, 4, "f", "device", "map_in")
    lv = _buf(level, px, 4, "f", "device", "level")
    b = _buf(map_out, px, 4, "f", "device", "map_out")
    _check(lib().amr_blur(ctx, int(nx), int(ny), a, lv, float(pixel), b,
                          _ptr(cuda_stream) if cuda_stream is not None else None))


def amr_camera_check(ctx, cam: Camera) -> int:
    L = ctypes.c_int32()
    _check(lib().amr_camera_check(ctx, ctypes.byref(to_camera(cam)), ctypes.byref(L)))
    return int(L.value)


def amr_set_options(ctx, **kw) -> None:
    o = amr_get_options(ctx)
    for k, v in kw.items():
        setattr(o, k, int(v))
    _check(lib().amr_set_options(ctx, ctypes.byref(o)))


def amr_get_options(ctx) -> amr_options:
    o = amr_options()
    _check(lib().amr_get_options(ctx, ctypes.byref(o)))
    return o


def amr_autotune(ctx, cams: Sequence[Camera], reps: int = 3):
    n = len(cams)
    carr = (amr_camera * n)(*[to_camera(c) for c in cams])
    best = amr_options()
    ms = ctypes.c_double()
    _check(lib().amr_autotune(ctx, n, carr, reps, ctypes.byref(best), ctypes.byref(ms)))
    return best.as_dict(), float(ms.value)


def amr_server_config(ctx, slots: int = 2, map_budget_bytes: int = 0, max_batch: int = 64) -> None:
    _check(lib().amr_server_config(ctx, slots, map_budget_bytes, max_batch))


def amr_submit(ctx, cam: Camera, map_host, counts_host=None) -> int:
    t = ctypes.c_uint64()
    px = int(cam.nx) * int(cam.ny)
    m = _buf(map_host, px, _map_size(cam), "f", "host", "map_host")
    k = _buf(counts_host, px, 4, "i", "host", "counts_host")
    _check(lib().amr_submit(ctx, ctypes.byref(to_camera(cam)), m, k, ctypes.byref(t)))
    return int(t.value)


def amr_wait(ctx, ticket: int, timeout_us: int = -1) -> None:
    _check(lib().amr_wait(ctx, ticket, timeout_us))


def amr_cancel(ctx, ticket: int) -> None:
    _check(lib().amr_cancel(ctx, ticket))


def amr_stats(ctx) -> dict:
    buf = ctypes.create_string_buffer(4096)
    _check(lib().amr_stats(ctx, buf, len(buf)))
    return json.loads(buf.value.decode())


def amr_tree_info(ctx):
    n, d, b = ctypes.c_int64(), ctypes.c_int32(), ctypes.c_int64()
    _check(lib().amr_tree_info(ctx, ctypes.byref(n), ctypes.byref(d), ctypes.byref(b)))
    return int(n.value), int(d.value), int(b.value)


AMR_NOALLOC_MAX_CAMERAS = 256


def amr_render_batch_noalloc(n_oct: int, records, depth: int, fields: Sequence, field_dtype: int,
                             cams: Sequence[Camera], maps: Sequence, counts: Optional[Sequence] = None,
                             cuda_stream=None) -> None:
    """Batch render with no GPU allocation: tree, maps and counts are the caller's device buffers."""
    n = len(cams)
    fsize = 8 if int(field_dtype) == AMR_F64 else 4
    farr = (ctypes.c_void_p * len(fields))(*[_buf(f, int(n_oct) * 8, fsize, "f", "current-device", f"fields[{i}]")
                                             for i, f in enumerate(fields)])
    carr = (amr_camera * max(n, 1))(*[to_camera(c) for c in cams])
    marr = (ctypes.c_void_p * max(n, 1))(*[_buf(m, int(c.nx) * int(c.ny), _map_size(c), "f", "current-device", f"maps[{i}]")
                                           for i, (m, c) in enumerate(zip(maps, cams))])
    karr = (ctypes.c_void_p * max(n, 1))(*[_buf(k, int(c.nx) * int(c.ny), 4, "i", "current-device", f"counts[{i}]")
                                           for i, (k, c) in enumerate(zip(counts, cams))]) if counts is not None else None
    recs = _buf(records, int(n_oct), 8, "i", "current-device", "records")
    _check(lib().amr_render_batch_noalloc(int(n_oct), recs, int(depth), len(fields), farr, int(field_dtype),
                                          n, carr, marr, karr, _ptr(cuda_stream) if cuda_stream is not None else None))


def amr_noalloc_status(cuda_stream=None) -> dict:
    """Device status of the last no-allocation batch on the current device
    (synchronises the stream): error 0 ok, 1 bad child index (oct), 2 step cap."""
    err, oct_, segs = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_uint64()
    _check(lib().amr_noalloc_status(_ptr(cuda_stream) if cuda_stream is not None else None, ctypes.byref(err),
                                    ctypes.byref(oct_), ctypes.byref(segs)))
    return {"error": int(err.value), "oct": int(oct_.value), "segments": int(segs.value)}


AMR_MERGE_MAX_PARTS = 64


def partial_components(mode: int, precision: int) -> int:
    """Values per pixel of a partial render: FP32 column (high, low) 2, weighted
    (S high, S low, N high, N low) 4, max 1; FP64 column 1, weighted (S, N) 2,
    max 1 (float32 or float64 elements)."""
    weighted = int(mode) in (AMR_MODE_WMEAN, AMR_MODE_LEVEL)
    if int(precision) == AMR_PREC_FP64:
        return 2 if weighted else 1
    return 4 if weighted else (1 if int(mode) == AMR_MODE_MAX else 2)


def amr_render_batch_partial(ctx, cams: Sequence[Camera], partials: Sequence, counts: Optional[Sequence] = None,
                             cuda_stream=None) -> None:
    """Sort-last partial renders (device buffers): each pixel's accumulators."""
    n = len(cams)
    if len(partials) != n or (counts is not None and len(counts) != n):
        raise ValueError("one partial (and one counts entry, if counts are given) per camera")
    carr = (amr_camera * n)(*[to_camera(c) for c in cams])
    parr = (ctypes.c_void_p * n)(*[_buf(m, int(c.nx) * int(c.ny) * partial_components(c.mode, c.precision),
                                        _map_size(c), "f", "device", f"partials[{i}]")
                                   for i, (m, c) in enumerate(zip(partials, cams))])
    karr = (ctypes.c_void_p * n)(*[_buf(k, int(c.nx) * int(c.ny), 4, "i", "device", f"counts[{i}]")
                                   for i, (k, c) in enumerate(zip(counts, cams))]) if counts is not None else None
    _check(lib().amr_render_batch_partial(ctx, n, carr, parr, karr,
                                          _ptr(cuda_stream) if cuda_stream is not None else None))


def amr_merge_partials(mode: int, precision: int, n_px: int, partials: Sequence, map_out, cuda_stream=None) -> None:
    """Merge partial renders of one camera into its map (device buffers)."""
    size = 8 if int(precision) == AMR_PREC_FP64 else 4
    comps = partial_components(mode, precision)
    parr = (ctypes.c_void_p * max(len(partials), 1))(*[_buf(q, int(n_px) * comps, size, "f", "current-device",
                                                            f"partials[{i}]") for i, q in enumerate(partials)])
    m = _buf(map_out, int(n_px), size, "f", "current-device", "map_out")
    _check(lib().amr_merge_partials(len(partials), int(mode), int(precision), int(n_px), parr, m,
                                    _ptr(cuda_stream) if cuda_stream is not None else None))


# ---------------------------------------------------------------- convenience
class Renderer:
    """A context with a loaded tree; maps and streams are torch CUDA tensors/streams."""

    def __init__(self, tree: Tree, device: int = 0):
        import torch
        self.torch = torch
        self.device = device
        self.ctx = amr_create(device)
        f64 = tree.fields[0].dtype == np.float64
        self.field_dtype = AMR_F64 if f64 else AMR_F32
        fields = [np.ascontiguousarray(f) for f in tree.fields]
        amr_load_octree(self.ctx, tree.n_oct, np.ascontiguousarray(tree.level, np.uint8),
                        np.ascontiguousarray(tree.coord, np.int32), np.ascontiguousarray(tree.child, np.int32),
                        fields, self.field_dtype)

    def close(self) -> None:
        if self.ctx:
            amr_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def alloc(self, cam: Camera):
        t = self.torch
        dt = t.float64 if cam.precision == AMR_PREC_FP64 else t.float32
        dev = f"cuda:{self.device}"
        return t.empty((cam.ny, cam.nx), dtype=dt, device=dev), t.empty((cam.ny, cam.nx), dtype=t.int32, device=dev)

    def render(self, cam: Camera, stream=None):
        m, c = self.alloc(cam)
        s = stream if stream is not None else self.torch.cuda.current_stream(self.device)
        amr_render(self.ctx, cam, m, c, 1, s.cuda_stream)
        return m, c

    def render_batch(self, cams: Sequence[Camera], stream=None, with_counts: bool = True):
        outs = [self.alloc(c) for c in cams]
        s = stream if stream is not None else self.torch.cuda.current_stream(self.device)
        amr_render_batch(self.ctx, cams, [o[0] for o in outs], [o[1] for o in outs] if with_counts else None, 1,
                         s.cuda_stream)
        return outs

    def alloc_partial(self, cam: Camera):
        t = self.torch
        dt = t.float64 if cam.precision == AMR_PREC_FP64 else t.float32
        dev = f"cuda:{self.device}"
        k = partial_components(cam.mode, cam.precision)
        return t.empty((cam.ny, cam.nx, k), dtype=dt, device=dev), t.empty((cam.ny, cam.nx), dtype=t.int32, device=dev)

    def render_partial(self, cams: Sequence[Camera], stream=None):
        """Partial renders (sort-last domain shares) of cams: [(partial, counts)]."""
        outs = [self.alloc_partial(c) for c in cams]
        s = stream if stream is not None else self.torch.cuda.current_stream(self.device)
        amr_render_batch_partial(self.ctx, cams, [o[0] for o in outs], [o[1] for o in outs], s.cuda_stream)
        return outs

    def slice(self, cam: Camera, stream=None):
        m, c = self.alloc(cam)
        s = stream if stream is not None else self.torch.cuda.current_stream(self.device)
        amr_slice(self.ctx, cam, m, c, 1, s.cuda_stream)
        return m, c

    def stats(self) -> dict:
        return amr_stats(self.ctx)
