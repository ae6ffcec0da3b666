"""Tree files: round trip, header, corruption detection, caching."""
import numpy as np
import pytest

from paper_1210_8014_gb300 import inputs


def test_round_trip(tmp_path):
    t = inputs.galaxy_tree(2, 2.0 ** -12, 9, with_velocity=True)
    p = tmp_path / "g.amrtree"
    inputs.save_tree(t, p)
    u = inputs.load_tree(p)
    assert u.n_oct == t.n_oct and (u.level == t.level).all() and (u.coord == t.coord).all()
    assert (u.child == t.child).all() and len(u.fields) == 4
    assert all((a == b).all() and a.dtype == b.dtype for a, b in zip(u.fields, t.fields))
    assert u.info["normal"] == t.info["normal"]
    d = inputs.plain_tree()
    inputs.save_tree(d, tmp_path / "p.amrtree")
    assert inputs.load_tree(tmp_path / "p.amrtree").fields[0].dtype == np.float64


def test_corruption_is_detected(tmp_path):
    t = inputs.complete_tree(3, 1.0)
    p = tmp_path / "c.amrtree"
    inputs.save_tree(t, p)
    raw = bytearray(p.read_bytes())
    raw[-5] ^= 0x40
    p.write_bytes(bytes(raw))
    with pytest.raises(ValueError, match="checksum"):
        inputs.load_tree(p)
    p.write_bytes(bytes(raw[:-100]))
    with pytest.raises(ValueError, match="truncated"):
        inputs.load_tree(p)
    p.write_bytes(b"NOTATREE" + bytes(raw[8:]))
    with pytest.raises(ValueError, match="not a tree file"):
        inputs.load_tree(p)


def test_cache(tmp_path):
    calls = []

    def make():
        calls.append(1)
        return inputs.complete_tree(2, 3.0)

    a = inputs.cached("uniform", make, cache_dir=tmp_path)
    b = inputs.cached("uniform", make, cache_dir=tmp_path)
    assert len(calls) == 1 and (a.fields[0] == b.fields[0]).all()
