"""The C ABI: every declared symbol is exported, and calls fail cleanly without a GPU."""
import ctypes
import re
from pathlib import Path

import pytest

from paper_1210_8014_gb300 import _build

ROOT = Path(__file__).resolve().parents[1]
DECL = re.compile(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*\**\s*([a-z_][a-z0-9_]*)\s*\(", re.M)


def declared(header: Path):
    text = re.sub(r"/\*.*?\*/", "", header.read_text(), flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    names = set(DECL.findall(text))
    return sorted(n for n in names if not n.startswith("defined"))


LIBS = {"amr.h": _build.build_amr, "amr_gen.h": _build.build_gen}


@pytest.mark.parametrize("header", sorted(LIBS))
def test_every_declared_symbol_is_exported(header):
    names = declared(ROOT / "include" / header)
    assert len(names) >= 5
    lib = ctypes.CDLL(str(LIBS[header]()))
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_amr_h_declares_the_boundary():
    names = set(declared(ROOT / "include" / "amr.h"))
    for n in ("amr_create", "amr_destroy", "amr_load_octree", "amr_render", "amr_render_batch", "amr_submit",
              "amr_wait", "amr_stats", "amr_last_error", "amr_autotune"):
        assert n in names


def test_camera_struct_layout_matches_header():
    from paper_1210_8014_gb300 import amr
    assert ctypes.sizeof(amr.amr_camera) == 14 * 8 + 10 * 4
    assert ctypes.sizeof(amr.amr_options) == 7 * 4


def test_calls_fail_cleanly_without_a_device():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1210_8014_gb300 import amr
    with pytest.raises(amr.AmrError) as e:
        amr.amr_create(0)
    assert e.value.status in (amr.AMR_E_CUDA, amr.AMR_E_INVALID)
    assert amr.amr_last_error()
    # null context / null arguments are rejected before any device work
    L = amr.lib()
    assert L.amr_render(None, None, None, None, 1, None) == amr.AMR_E_INVALID
    assert L.amr_render_batch(None, 1, None, None, None, 1, None) == amr.AMR_E_INVALID
    assert L.amr_destroy(None) == amr.AMR_OK
    assert L.amr_stats(None, None, 0) == amr.AMR_E_INVALID


def test_binding_checks_buffers_before_the_call():
    """The library cannot see buffer sizes; the binding checks what a call will
    touch (length, element type, contiguity, host or device side) and raises
    before any native call (ctx None: nothing reaches the library)."""
    import numpy as np
    import torch
    from paper_1210_8014_gb300 import amr, inputs
    cam = inputs.axis_camera(16, max_level=3, precision=amr.AMR_PREC_FP32_KAHAN)
    ok_map, ok_cnt = np.zeros((16, 16), np.float32), np.zeros((16, 16), np.int32)
    bad = [
        ((np.zeros(100, np.float32), ok_cnt), "elements, need 256"),        # too short
        ((np.zeros((16, 16), np.float64), ok_cnt), "need float32"),         # FP32 map given doubles
        ((np.zeros((16, 16), np.int32), ok_cnt), "need float32"),           # integers for a map
        ((ok_map, np.zeros((16, 16), np.float32)), "need int32"),           # floats for counts
        ((np.zeros((16, 32), np.float32)[:, ::2], ok_cnt), "not contiguous"),
    ]
    for (m, c), msg in bad:
        with pytest.raises(ValueError, match=msg):
            amr.amr_render(None, cam, m, c, 0)
    with pytest.raises(ValueError, match="device buffer is needed"):
        amr.amr_render(None, cam, ok_map, ok_cnt, 1)                        # host arrays, device outputs
    with pytest.raises(ValueError, match="need float64"):
        amr.amr_render(None, cam.with_(precision=amr.AMR_PREC_FP64), ok_map, None, 0)
    with pytest.raises(ValueError, match="one map"):
        amr.amr_render_batch(None, [cam, cam], [ok_map], None, 0)
    with pytest.raises(ValueError, match=r"maps\[1\]"):
        amr.amr_render_batch(None, [cam, cam.with_(nx=32)], [ok_map, ok_map], None, 0)
    with pytest.raises(ValueError, match="need int32"):
        amr.amr_slice(None, cam, ok_map, np.zeros((16, 16), np.float32), 0)
    with pytest.raises(ValueError, match="device buffer is needed"):
        amr.amr_blur(None, 16, 16, ok_map, ok_map, 0.1, ok_map)
    with pytest.raises(ValueError, match="elements, need 256"):
        amr.amr_submit(None, cam, torch.zeros(10), None)
    tree = inputs.plain_tree(np.float64)
    with pytest.raises(ValueError, match=r"child: .*elements, need"):
        amr.amr_load_octree(None, tree.n_oct, tree.level, tree.coord, tree.child[:-1], tree.fields, amr.AMR_F64)
    with pytest.raises(ValueError, match="need float32"):
        amr.amr_load_octree(None, tree.n_oct, tree.level, tree.coord, tree.child, tree.fields, amr.AMR_F32)
    with pytest.raises(ValueError, match="need int8"):
        amr.amr_load_octree(None, tree.n_oct, tree.level.astype(np.int32), tree.coord, tree.child, tree.fields,
                            amr.AMR_F64)
