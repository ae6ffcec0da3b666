"""Pins of the CPU oracle: checks against what the paper and the mathematics fix.

Each ``pin_*`` takes a loaded oracle library handle and raises AssertionError on
a mismatch, so the same pins run against the real oracle (tests/test_oracle_pins.py)
and against copies of it with planted mistakes (tests/test_oracle_mutants.py).

Sources of truth (none of them is the oracle itself):
  - hand-derived values for a two-level tree (tests/golden/two_level_tree.json),
  - closed forms: a uniform box gives value x exact slab chord; a single
    non-zero leaf gives its own exact chord (exact rationals via fractions),
  - brute force: O(pixels x leaves) exact slab tests (oracle/bruteforce.py),
  - invariants: mass (column map x pixel area = mass in view) at every cut
    level, splitting a leaf, reversing the ray, sort-last additivity, constant
    velocity in wmean, the camera level rule.
"""
from __future__ import annotations

import json
import math
from fractions import Fraction
from pathlib import Path

import numpy as np

import oracle
from oracle import bruteforce as bf
from paper_1210_8014_gb300 import inputs

GOLDEN = Path(__file__).resolve().parent / "golden"


def golden_tree():
    g = json.loads((GOLDEN / "two_level_tree.json").read_text())
    t = g["tree"]
    tree = inputs.Tree(np.array(t["level"], np.uint8), np.array(t["coord"], np.int32),
                       np.array(t["child"], np.int32), [np.array(f, np.float64) for f in t["fields"]])
    return tree, g["cases"]


def golden_camera(case):
    return inputs.Camera(case["centre"], case["u"], case["v"], case["w"], (1.0, 1.0), 1, 1,
                         max_level=case["max_level"], mode=case["mode"])


def exact_box_chord(cam, i, j, lo, hi):
    """Chord of pixel (i, j)'s quantised ray through the box [lo, hi)^3 (2^-36 units)."""
    X0 = bf.origin(cam, i, j)
    D = bf.quantised_direction(cam)
    tin, tout = None, None
    for a in range(3):
        if D[a] == 0:
            if not (lo[a] <= X0[a] < hi[a]):
                return 0.0
            continue
        t0 = Fraction(int(lo[a]) - int(X0[a]), int(D[a]))
        t1 = Fraction(int(hi[a]) - int(X0[a]), int(D[a]))
        t0, t1 = min(t0, t1), max(t0, t1)
        tin = t0 if tin is None else max(tin, t0)
        tout = t1 if tout is None else min(tout, t1)
    if tout <= tin:
        return 0.0
    return float(tout - tin) * math.sqrt(int((D * D).sum())) * 2.0 ** -36


def pin_golden(lib):
    tree, cases = golden_tree()
    for case in cases:
        m, c = oracle.render(tree, golden_camera(case), lib=lib)
        assert int(c[0, 0]) == case["count"], (case["name"], int(c[0, 0]))
        exp = case["expected"]
        assert abs(m[0, 0] - exp) <= 1e-15 * max(1.0, abs(exp)), (case["name"], m[0, 0], exp)


def pin_uniform_axis(lib):
    tree = inputs.complete_tree(4, 1.0)
    for L in range(1, 5):
        cam = inputs.axis_camera(32, max_level=L)
        m, c = oracle.render(tree, cam, lib=lib)
        assert (c == 2 ** L).all(), ("counts", L)
        assert (m == 1.0).all(), ("column", L, m.min(), m.max())


def pin_uniform_oblique(lib):
    tree = inputs.complete_tree(4, 2.5)
    rng = np.random.default_rng(11)
    full = 1 << 36
    for _ in range(4):
        cam = inputs.camera_along(inputs.random_direction(rng), centre=rng.uniform(0.3, 0.7, 3), fov=1.2, n=12,
                                  max_level=4)
        m, c = oracle.render(tree, cam, lib=lib)
        for j in range(cam.ny):
            for i in range(cam.nx):
                ch = exact_box_chord(cam, i, j, (0, 0, 0), (full, full, full))
                assert abs(m[j, i] - 2.5 * ch) <= 1e-14 * max(1.0, 2.5 * ch), (i, j, m[j, i], 2.5 * ch)
                assert (c[j, i] > 0) == (ch > 0)


def pin_single_leaf(lib):
    target = (3, 5, 2)      # level-3 cell with this integer corner
    lvl = 3

    def val(x, y, z, lv):
        k = np.floor(np.stack([x, y, z]) * 2.0 ** lvl).astype(int)
        return ((k[0] == target[0]) & (k[1] == target[1]) & (k[2] == target[2]) & (lv == lvl)).astype(float)

    tree = inputs.complete_tree(lvl, val)
    size = 1 << (36 - lvl)
    lo = tuple(t * size for t in target)
    hi = tuple((t + 1) * size for t in target)
    rng = np.random.default_rng(5)
    for _ in range(3):
        cam = inputs.camera_along(inputs.random_direction(rng), centre=(0.45, 0.65, 0.3), fov=0.4, n=10,
                                  max_level=lvl)
        m, _ = oracle.render(tree, cam, lib=lib)
        for j in range(cam.ny):
            for i in range(cam.nx):
                ch = exact_box_chord(cam, i, j, lo, hi)
                assert abs(m[j, i] - ch) <= 1e-14, (i, j, m[j, i], ch)


def _bruteforce_cases():
    rng = np.random.default_rng(1234)
    cases = []
    for k in range(6):
        tree = inputs.random_tree(rng, depth=4 if k % 2 else 5, p_refine=0.35)
        if k == 0:
            w = (0.0, 0.0, 1.0)                      # axis-aligned: rays on faces and edges
            cam = inputs.axis_camera(16, max_level=5)
        else:
            if k == 1:
                w = (1.0, 1.0, 0.0)                  # edges: simultaneous crossings on 2 axes
            elif k == 2:
                w = (1.0, -1.0, 1.0)                 # corners on 3 axes
            elif k == 3:
                w = (0.5, 0.25, -1.0)                # dyadic slopes: many exact ties
            else:
                w = inputs.random_direction(rng)
            L = int(rng.integers(2, 6)) if k > 3 else -1
            cam = inputs.camera_along(w, centre=(0.5, 0.5, 0.5), fov=(1.0, 0.75), n=(16, 12), max_level=L)
        for mode in (0, 1, 2, 3):
            cases.append((tree, cam.with_(mode=mode)))
    return cases


def pin_bruteforce(lib):
    for tree, cam in _bruteforce_cases():
        m, c = oracle.render(tree, cam, lib=lib)
        bm, bc = bf.bruteforce(tree, cam)
        assert (c == bc).all(), ("counts", cam.mode, int(np.abs(c - bc).max()))
        if cam.mode == 0:
            err = np.abs(m - bm) / np.maximum(np.abs(bm), 1e-300)
            err[bm == 0] = np.abs(m[bm == 0])
            assert err.max() <= 1e-14, ("column", err.max())
        elif cam.mode in (1, 3):
            assert np.abs(m - bm).max() <= 1e-13 * max(1e-300, np.abs(bm).max()), ("wmean", np.abs(m - bm).max())
        else:
            assert (m == bm).all(), "max"


def pin_mass(lib):
    tree = inputs.plain_tree()
    for L in range(1, 8):
        cam = inputs.axis_camera(256, max_level=L)
        m, c = oracle.render(tree, cam, lib=lib)
        lv = tree.level.astype(np.int64)
        leaf = ((tree.child < 0) & (lv[:, None] <= L)) | (lv[:, None] == L)
        mass = float((tree.fields[0] * np.ldexp(1.0, -3 * lv)[:, None])[leaf].sum())
        assert abs(m.sum() / 256 ** 2 - mass) <= 1e-13 * mass, (L, m.sum() / 256 ** 2, mass)
        assert (c >= 2 ** min(L, 3)).all()


def pin_split(lib):
    rng = np.random.default_rng(77)
    tree = inputs.random_tree(rng, depth=4, p_refine=0.3)
    o, c = [(o, c) for o in range(tree.n_oct) for c in range(8) if tree.child[o, c] < 0 and tree.level[o] == 2][3]
    split = inputs.split_leaf(tree, o, c)
    lvl = int(tree.level[o])
    for w in ((0.0, 0.0, 1.0), (0.3, -0.6, 0.74)):
        for mode in (0, 1, 2):
            cam = inputs.camera_along(w, fov=1.1, n=20, max_level=4, mode=mode)
            m0, c0 = oracle.render(tree, cam, lib=lib)
            m1, c1 = oracle.render(split, cam, lib=lib)
            if mode == 2:
                assert (m0 == m1).all()
            else:
                assert np.abs(m0 - m1).max() <= 1e-13 * np.abs(m0).max()
            d = c1 - c0
            assert d.min() >= 0 and d.max() <= 3
            if w == (0.0, 0.0, 1.0):
                # each ray through the split cell's footprint crosses one more cell
                k = tree.coord[o] + np.array([(c >> a) & 1 for a in range(3)])
                shift = 36 - lvl
                inside = np.zeros((cam.ny, cam.nx), int)
                for j in range(cam.ny):
                    for i in range(cam.nx):
                        X0 = bf.origin(cam, i, j)
                        inside[j, i] = int((X0[0] >> shift) == k[0] and (X0[1] >> shift) == k[1])
                assert (d == inside).all()


def pin_symmetry(lib):
    tree = inputs.random_tree(np.random.default_rng(3), depth=5, p_refine=0.3)
    rng = np.random.default_rng(8)
    for _ in range(3):
        u, v, w = inputs.basis_from_direction(inputs.random_direction(rng))
        cam = inputs.Camera((0.5, 0.45, 0.55), tuple(u), tuple(v), tuple(w), (1.25, 1.25), 16, 16, max_level=5)
        rev = cam.with_(u=tuple(-u), w=tuple(-w))
        m0, c0 = oracle.render(tree, cam, lib=lib)
        m1, c1 = oracle.render(tree, rev, lib=lib)
        assert (c0 == c1[:, ::-1]).all()
        assert np.abs(m0 - m1[:, ::-1]).max() <= 1e-14 * np.abs(m0).max()


def pin_sortlast(lib):
    """Sec. 2.2 order-independence / Sec. 3.1 sort-last: partial maps over
    disjoint leaf domains add up to the whole map."""
    rng = np.random.default_rng(21)
    tree = inputs.random_tree(rng, depth=5, p_refine=0.3)
    cam = inputs.camera_along(inputs.random_direction(rng), fov=1.3, n=24, max_level=5)
    m, c = oracle.render(tree, cam, lib=lib)
    x, y, z, _ = inputs.cell_centres(tree)
    dom = (np.floor(x * 2).astype(int) + 2 * np.floor(y * 2).astype(int)) % 3   # 3 spatial domains
    total = np.zeros_like(m)
    for d in range(3):
        part = inputs.Tree(tree.level, tree.coord, tree.child, [np.where(dom == d, tree.fields[0], 0.0)])
        pm, pc = oracle.render(part, cam, lib=lib)
        assert (pc == c).all()
        total += pm
    assert np.abs(total - m).max() <= 1e-13 * np.abs(m).max()


def pin_wmean_constant(lib):
    tree = inputs.random_tree(np.random.default_rng(9), depth=4, p_refine=0.4)
    vel = np.array([0.3, -1.7, 0.9])
    for a in range(3):
        tree.fields[1 + a][:] = vel[a]
    rng = np.random.default_rng(10)
    for _ in range(3):
        cam = inputs.camera_along(inputs.random_direction(rng), fov=1.6, n=16, max_level=4, mode=1)
        m, c = oracle.render(tree, cam, lib=lib)
        exp = float(vel @ np.asarray(cam.w))
        assert np.abs(m[c > 0] - exp).max() <= 1e-14, np.abs(m[c > 0] - exp).max()
        assert (m[c == 0] == 0).all()


def pin_mean_level_uniform(lib):
    """A complete tree gives mean level = the cut level exactly, at every cut."""
    tree = inputs.complete_tree(4, 1.7)
    rng = np.random.default_rng(4)
    for L in range(1, 5):
        cam = inputs.camera_along(inputs.random_direction(rng), fov=1.2, n=10, max_level=L, mode=3)
        m, c = oracle.render(tree, cam, lib=lib)
        assert (np.abs(m[c > 0] - L) <= 1e-13).all(), (L, m[c > 0].min(), m[c > 0].max())


def pin_level_rule(lib):
    deep = inputs.Tree(np.array([1, 22], np.uint8), np.zeros((2, 3), np.int32),
                       np.array([[1] + [-1] * 7, [-1] * 8], np.int32), [np.ones((2, 8))])
    cases = [(1.0, 256, 8), (1.0, 4096, 12), (2.0 ** -7, 4096, 19), (0.3, 100, 8), (1.0, 1, 1),
             (2.0 ** -12, 2048, 22), (0.75, 1024, 10), (1.0, 1023, 9)]
    for fov, n, L in cases:
        got = oracle.view_info(deep, inputs.camera_along((0, 0, 1), fov=fov, n=n, max_level=-1), lib=lib)[0]
        assert got == L, (fov, n, got, L)
    shallow = inputs.complete_tree(3, 1.0)
    assert oracle.view_info(shallow, inputs.camera_along((0, 0, 1), fov=1.0, n=4096, max_level=-1), lib=lib)[0] == 3
    assert oracle.view_info(shallow, inputs.camera_along((0, 0, 1), fov=1.0, n=64, max_level=2), lib=lib)[0] == 2


def pin_quantisation(lib):
    """Ray origin and direction: round-half-even of x 2^36 and w/max|w| 2^23."""
    cam = inputs.Camera((0.5, 0.5, 0.5), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0), (2.0 ** -30, 1.0),
                        4, 2, max_level=3)
    # s = ((i+0.5)/4 - 0.5) 2^-30 -> x = 0.5 + {-3/8,-1/8,1/8,3/8} 2^-30 ; x 2^36 = 2^35 + {-24,-8,8,24}
    for i, dx in enumerate((-24, -8, 8, 24)):
        X0 = oracle.ray_origin(cam, i, 0, lib=lib)
        assert int(X0[0]) == 2 ** 35 + dx and int(X0[1]) == 2 ** 35 - 2 ** 34, (i, X0)
    half = inputs.Camera((2.0 ** -37, 0.5, 0.5), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0), (1.0, 1.0), 1, 1)
    assert int(oracle.ray_origin(half, 0, 0, lib=lib)[0]) == 0        # 0.5 ulp of the lattice rounds to even 0
    half3 = half.with_(centre=(3 * 2.0 ** -37, 0.5, 0.5))
    assert int(oracle.ray_origin(half3, 0, 0, lib=lib)[0]) == 2       # 1.5 rounds to even 2
    tree = inputs.complete_tree(2, 1.0)
    for frac, dy in ((1, 0), (3, 1)):   # 2^22 + 0.25 rounds down, 2^22 + 0.75 rounds up
        w = np.array([1.0, 0.5 + frac * 2.0 ** -25, -0.25])
        w /= np.linalg.norm(w)
        _, D, lam = oracle.view_info(tree, inputs.camera_along(w, max_level=2), lib=lib)
        assert list(D) == [2 ** 23, 2 ** 22 + dy, -(2 ** 21)], D
        assert lam == math.sqrt(2 ** 46 + (2 ** 22 + dy) ** 2 + 2 ** 42) * 2.0 ** -36


ALL_PINS = [pin_golden, pin_quantisation, pin_uniform_axis, pin_uniform_oblique, pin_single_leaf,
            pin_bruteforce, pin_mass, pin_split, pin_symmetry, pin_sortlast, pin_wmean_constant, pin_level_rule,
            pin_mean_level_uniform]


def pin_slice(lib):
    """Slice map: golden points of the two-level tree, and brute-force containment."""
    tree, _ = golden_tree()
    # pixel centres x, y in {0.125, 0.375} on the plane z = 0.25, the low face of
    # level-2 z-index 1: the cells with z-bit 1 of the refined oct in root cell 0
    cam = inputs.Camera((0.25, 0.25, 0.25), (1.0, 0.0, 0.0), (0.0, 1.0, 0.0), (0.0, 0.0, 1.0), (0.5, 0.5), 2, 2,
                        max_level=2)
    m, lv = oracle.slice_map(tree, cam, lib=lib)
    assert m.tolist() == [[14.0, 15.0], [16.0, 17.0]] and (lv == 2).all(), (m, lv)
    m1, lv1 = oracle.slice_map(tree, cam.with_(max_level=1), lib=lib)
    assert (m1 == 13.5).all() and (lv1 == 1).all()
    rng = np.random.default_rng(99)
    for k in range(3):
        t = inputs.random_tree(rng, depth=4, p_refine=0.4)
        c = inputs.camera_along(inputs.random_direction(rng), centre=rng.uniform(0.2, 0.8, 3), fov=1.4, n=9,
                                max_level=int(rng.integers(1, 5)))
        m, lv = oracle.slice_map(t, c, lib=lib)
        bm, blv = bf.bruteforce_slice(t, c)
        assert (m == bm).all() and (lv == blv).all(), k


ALL_PINS.append(pin_slice)


def pin_touched(lib):
    """Instrumented pass (compulsory bytes): the leaves it marks are exactly
    those some pixel's ray crosses by brute-force slab tests, and the refined
    cells it marks are exactly the proper ancestors of those leaves."""
    for tree, cam in _bruteforce_cases()[::4]:
        leaf, inner = oracle.touched(tree, cam, lib=lib)
        hits = np.zeros((tree.n_oct, 8), bool)
        bf.bruteforce(tree, cam, hits_out=hits)
        assert hits.any() and (leaf.astype(bool) == hits).all(), ("leaves", int((leaf.astype(bool) != hits).sum()))
        parent = {}
        for p_, c_ in zip(*np.nonzero(tree.child >= 0)):
            parent[int(tree.child[p_, c_])] = (int(p_), int(c_))
        anc = np.zeros((tree.n_oct, 8), bool)
        for o, _ in zip(*np.nonzero(hits)):
            o = int(o)
            while o in parent:
                o, c = parent[o]
                anc[o, c] = True
        assert (inner.astype(bool) == anc).all(), ("refined cells", int((inner.astype(bool) != anc).sum()))


ALL_PINS.append(pin_touched)
