"""Brute-force slab checker — TEST INFRASTRUCTURE ONLY.

An independent second statement of the ray-casting result of Sec. 2.2 for tiny
trees: for every pixel ray, test every render leaf with the textbook slab
method in exact integers on the quantised ray, and sum value x chord in
extended precision.  It shares nothing with ``amr_oracle.c`` (camera set-up
included: it is re-derived here from the same written definitions), so the
two pin each other.

Definitions used (the readings the oracle states):
  - render leaves at cut L: cells of level l <= L with no child, or l == L.
  - pixel centre = centre + ((i+0.5)/nx - 0.5) fov0 u + ((j+0.5)/ny - 0.5) fov1 v
    in IEEE double; X0 = round-half-even(x 2^36); D = round-half-even(w/max|w| 2^23).
  - a cell is crossed iff the exact parameter interval inside it has positive
    length; chord = length x sqrt(sum D^2) 2^-36.
"""
from __future__ import annotations

import numpy as np

K = 36
DBITS = 23


def cut_level(cam, depth: int) -> int:
    if cam.max_level > 0:
        L = int(cam.max_level)
    else:
        L = 1
        for lvl in range(1, 23):
            if np.ldexp(float(cam.fov[0]), lvl) <= cam.nx and np.ldexp(float(cam.fov[1]), lvl) <= cam.ny:
                L = lvl
    return max(1, min(L, depth))


def quantised_direction(cam) -> np.ndarray:
    w = np.asarray(cam.w, np.float64)
    return np.rint(np.ldexp(w / np.max(np.abs(w)), DBITS)).astype(np.int64)


def origin(cam, i: int, j: int) -> np.ndarray:
    s = ((np.float64(i) + 0.5) / np.float64(cam.nx) - 0.5) * np.float64(cam.fov[0])
    t = ((np.float64(j) + 0.5) / np.float64(cam.ny) - 0.5) * np.float64(cam.fov[1])
    c = np.asarray(cam.centre, np.float64)
    x = (c + s * np.asarray(cam.u, np.float64)) + t * np.asarray(cam.v, np.float64)
    return np.rint(np.ldexp(x, K)).astype(np.int64)


def render_leaves(tree, L: int):
    """(oct, cell, level, lo[3], hi[3]) of the render leaves, integers in 2^-36 units."""
    lv = tree.level.astype(np.int64)
    o, c = np.nonzero(((tree.child < 0) & (lv[:, None] <= L)) | (lv[:, None] == L))
    lvl = lv[o]
    k = tree.coord[o].astype(np.int64) + np.stack([(c >> a) & 1 for a in range(3)], axis=1)
    size = np.left_shift(np.int64(1), K - lvl)[:, None]
    lo = k * size
    return o, c, lvl, lo, lo + size


def bruteforce(tree, cam, pixels=None, hits_out=None):
    """(map, counts) by slab tests; map as float64 rounded from long double sums.
    hits_out (optional bool [n_oct, 8]): set where some pixel's ray crosses that leaf."""
    L = cut_level(cam, int(tree.level.max()))
    D = quantised_direction(cam)
    aD = np.abs(D)
    lam = np.sqrt(np.longdouble(int((D * D).sum()))) / np.longdouble(2.0 ** K)
    o, c, lvls, lo, hi = render_leaves(tree, L)
    fld = [np.asarray(f, np.float64)[o, c].astype(np.longdouble) for f in tree.fields]
    w = np.asarray(cam.w, np.float64)
    if pixels is None:
        jj, ii = np.meshgrid(np.arange(cam.ny), np.arange(cam.nx), indexing="ij")
        pix = list(zip(ii.ravel(), jj.ravel()))
        shape = (cam.ny, cam.nx)
    else:
        pix = list(zip(pixels[0], pixels[1]))
        shape = (len(pix),)
    out = np.zeros(len(pix), np.float64)
    cnt = np.zeros(len(pix), np.int32)
    n = lo.shape[0]
    for q, (i, j) in enumerate(pix):
        X0 = origin(cam, i, j)
        inside = np.ones(n, bool)
        # running max of entry times and min of exit times: num / den, den > 0
        en_n = en_d = ex_n = ex_d = None
        for a in range(3):
            if D[a] == 0:
                inside &= (lo[:, a] <= X0[a]) & (X0[a] < hi[:, a])
                continue
            if D[a] > 0:
                a_en, a_ex = lo[:, a] - X0[a], hi[:, a] - X0[a]
            else:
                a_en, a_ex = X0[a] - hi[:, a], X0[a] - lo[:, a]
            d = np.full(n, aD[a], np.int64)
            if en_n is None:
                en_n, en_d, ex_n, ex_d = a_en, d, a_ex, d
            else:
                later = a_en * en_d > en_n * d
                en_n, en_d = np.where(later, a_en, en_n), np.where(later, d, en_d)
                earlier = a_ex * ex_d < ex_n * d
                ex_n, ex_d = np.where(earlier, a_ex, ex_n), np.where(earlier, d, ex_d)
        num = ex_n * en_d - en_n * ex_d          # (t_exit - t_entry) * ex_d * en_d
        hit = inside & (num > 0)
        if hits_out is not None:
            hits_out[o[hit], c[hit]] = True
        ln = num[hit].astype(np.longdouble) / (ex_d[hit].astype(np.longdouble) * en_d[hit]) * lam
        cnt[q] = int(hit.sum())
        if cam.mode == 0:
            out[q] = float(np.sum(fld[cam.field_value][hit] * ln))
        elif cam.mode == 1:
            rho = fld[cam.field_weight][hit]
            vlos = (fld[cam.field_vel[0]][hit] * np.longdouble(w[0]) + fld[cam.field_vel[1]][hit] * np.longdouble(w[1])
                    + fld[cam.field_vel[2]][hit] * np.longdouble(w[2]))
            S = np.sum(rho * ln)
            out[q] = float(np.sum(rho * vlos * ln) / S) if S != 0 else 0.0
        elif cam.mode == 3:
            rho = fld[cam.field_weight][hit]
            S = np.sum(rho * ln)
            out[q] = float(np.sum(rho * ln * lvls[hit].astype(np.longdouble)) / S) if S != 0 else 0.0
        else:
            out[q] = float(np.max(fld[cam.field_value][hit])) if cnt[q] else 0.0
    return out.reshape(shape), cnt.reshape(shape)


def bruteforce_slice(tree, cam):
    """Slice map by scanning every render leaf for the one containing each
    quantised pixel centre (half-open cells)."""
    L = cut_level(cam, int(tree.level.max()))
    o, c, lvl, lo, hi = render_leaves(tree, L)
    vals = np.asarray(tree.fields[cam.field_value], np.float64)[o, c]
    out = np.zeros((cam.ny, cam.nx), np.float64)
    lv = np.zeros((cam.ny, cam.nx), np.int32)
    for j in range(cam.ny):
        for i in range(cam.nx):
            X0 = origin(cam, i, j)
            hit = np.nonzero(((lo <= X0) & (X0 < hi)).all(axis=1))[0]
            if hit.size:
                assert hit.size == 1
                out[j, i] = vals[hit[0]]
                lv[j, i] = lvl[hit[0]]
    return out, lv
