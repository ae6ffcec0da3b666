"""Parity metrics between the CUDA path and the oracle.

counts : bit-exact, every pixel.
column : per-pixel |a - b| / b where b > 0, and a == 0 exactly where b == 0.
wmean  : normwise |a - b| / max|b| (the line-of-sight velocity changes sign);
         the mean-level mode likewise.
max    : bit-exact (a maximum over the same float32 values), compared in the
         kernel's output precision.
Tolerances: FP64 kernel 1e-12; FP32 compensated 1e-5.  The FP32 plain kernel is
reported, with a looser bound that only guards against gross errors.
"""
import numpy as np

TOL = {0: 1e-12, 1: 1e-5, 2: 1e-4}


def errors(mode, gpu_map, ref_map):
    a = np.asarray(gpu_map, np.float64)
    b = np.asarray(ref_map, np.float64)
    if mode == 0:
        pos = b > 0
        rel = np.zeros_like(b)
        rel[pos] = np.abs(a[pos] - b[pos]) / b[pos]
        zero_ok = bool((a[~pos] == 0).all())
        return {"max": float(rel.max(initial=0.0)), "p99": float(np.percentile(rel, 99)) if rel.size else 0.0,
                "zero_ok": zero_ok}
    if mode in (1, 3):
        scale = float(np.abs(b).max(initial=0.0))
        e = np.abs(a - b) / scale if scale > 0 else np.abs(a - b)
        return {"max": float(e.max(initial=0.0)), "p99": float(np.percentile(e, 99)) if e.size else 0.0,
                "zero_ok": True}
    return {"max": float(np.abs(a - b).max(initial=0.0)), "p99": 0.0, "zero_ok": True}


def assert_parity(mode, prec, gpu_map, gpu_counts, ref_map, ref_counts, field_is_f32=True, tol=None, ctx=""):
    gc = np.asarray(gpu_counts)
    rc = np.asarray(ref_counts)
    assert (gc == rc).all(), f"{ctx}: counts differ at {int((gc != rc).sum())} pixels (max |d| {int(np.abs(gc - rc).max())})"
    if mode == 2:
        a = np.asarray(gpu_map, np.float64)
        b = np.asarray(ref_map, np.float64)
        if prec != 0 and not field_is_f32:
            b = b.astype(np.float32).astype(np.float64)
        assert (a == b).all(), f"{ctx}: max map differs at {int((a != b).sum())} pixels"
        return {"max": 0.0, "p99": 0.0}
    e = errors(mode, gpu_map, ref_map)
    t = TOL[prec] if tol is None else tol
    assert e["zero_ok"], f"{ctx}: nonzero value where the oracle has an empty ray"
    assert e["max"] <= t, f"{ctx}: max error {e['max']:.3e} > {t:.0e} (p99 {e['p99']:.3e})"
    return e
