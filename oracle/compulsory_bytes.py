"""Compulsory bytes of a workload, counted by the oracle's instrumented pass.

TEST INFRASTRUCTURE: this script calls only the oracle (and the seeded input
generators); it writes profiles/compulsory_bytes_<workload>.txt, which the
benchmark reads beside its measured DRAM traffic.

Sec. 2.2 reads, for every leaf a ray crosses, the leaf's value, and reaches the
leaf through its ancestors' child indices.  A frame therefore has to read at
least once (its compulsory bytes, whatever the caching):
  - for each leaf crossed by any of its rays: the child word that says it is a
    leaf at this cut (4 B) and its scalars (4 B density for column and max,
    16 B density and velocity for the weighted mean, float32 fields);
  - for each refined cell its descents pass through: that cell's child word (4 B).
This is the no-reuse-within-a-frame floor in the units of the per-segment
algorithmic bytes (4 B child word + scalars per segment).  The same unique
cells in the GPU layout (an 8-byte oct record and a 64-byte link block per oct
touched, plus the scalars) are reported beside it.  Per launch the per-frame
figures are summed (frames of one launch read their data independently), and
the union over the launch's frames (data shared by several frames counted
once) is given too.

  python oracle/compulsory_bytes.py batch   # the 64-camera batch on the 16.0M-leaf tree
  python oracle/compulsory_bytes.py zoom    # the 8-frame 4096^2 zoom on the 193M-leaf tree
"""
from __future__ import annotations

import sys
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parents[1]
if str(ROOT) not in sys.path:
    sys.path.insert(0, str(ROOT))

import oracle  # noqa: E402
from paper_1210_8014_gb300 import inputs  # noqa: E402

VALUE_BYTES = {0: 4, 1: 16, 2: 4}     # float32 scalars a leaf needs, by mode


def frame_figures(leaf, inner, mode):
    n_leaf = int(leaf.sum())
    n_inner = int(inner.sum())
    n_octs = int((leaf.any(axis=1) | inner.any(axis=1)).sum())
    algo = n_leaf * (4 + VALUE_BYTES[mode]) + n_inner * 4
    layout = n_octs * (8 + 64) + n_leaf * VALUE_BYTES[mode]
    return n_leaf, n_inner, n_octs, algo, layout


def count(workload: str):
    if workload == "batch":
        tree = inputs.batch_tree()
        cams = inputs.batch_cameras(tree)
        what = (f"64-camera batch (sizes 128^2..2048^2, fov 1..1/64, pixel-rule cuts, mixed modes) on the "
                f"{tree.n_leaves}-leaf galaxy octree")
    elif workload == "zoom":
        tree = inputs.zoom_tree()
        cams = inputs.zoom_cameras(tree)
        what = f"8-frame 4096^2 zoom (fov 1 -> 1/128, column) on the {tree.n_leaves}-leaf level-22 octree"
    else:
        raise SystemExit(f"unknown workload {workload!r}: batch or zoom")
    prepared = oracle.prepare(tree)
    n = tree.n_oct
    union_leaf = np.zeros((n, 8), bool)
    union_vel = np.zeros((n, 8), bool)
    union_inner = np.zeros((n, 8), bool)
    tot = np.zeros(5, np.int64)
    t0 = time.time()
    frames = []
    for k, cam in enumerate(cams):
        leaf, inner = oracle.touched(prepared, cam)
        fig = frame_figures(leaf, inner, cam.mode)
        tot += np.array(fig, np.int64)
        lb = leaf.astype(bool)
        union_leaf |= lb
        if cam.mode == 1:
            union_vel |= lb
        union_inner |= inner.astype(bool)
        frames.append((k, cam.nx, cam.mode) + fig)
        print(f"camera {k}: {cam.nx}^2 mode {cam.mode}: {fig[0]} leaves, {fig[1]} refined cells, "
              f"{fig[3]} B ({time.time() - t0:.0f} s)", flush=True)
    u_leaf = int(union_leaf.sum())
    u_algo = u_leaf * 8 + int(union_vel.sum()) * 12 + int(union_inner.sum()) * 4
    u_octs = int((union_leaf.any(axis=1) | union_inner.any(axis=1)).sum())
    lines = [
        f"# Compulsory bytes of the {what}:",
        "# unique leaves crossed (child word 4 B + float32 scalars) and refined cells descended through",
        "# (child word 4 B), per frame, from the oracle's instrumented pass (oracle.touched).",
        "#",
        "# command:",
        f"#   python oracle/compulsory_bytes.py {workload}",
        "#",
        "# per frame: camera, size, mode, leaves, refined cells, octs, compulsory bytes, bytes in the GPU layout",
    ]
    lines += [f"# frame {f[0]}: {f[1]}^2 mode {f[2]}: {f[3]} {f[4]} {f[5]} {f[6]} {f[7]}" for f in frames]
    lines += [
        f"frames: {len(cams)}",
        f"unique_leaves_summed_over_frames: {int(tot[0])}",
        f"unique_refined_cells_summed_over_frames: {int(tot[1])}",
        f"compulsory_bytes_per_launch: {int(tot[3])}",
        f"compulsory_bytes_per_launch_gpu_layout: {int(tot[4])}",
        f"compulsory_bytes_union_over_launch: {u_algo}",
        f"octs_touched_union_over_launch: {u_octs}",
        f"tree_octs: {n}",
    ]
    out = ROOT / "profiles" / f"compulsory_bytes_{workload}.txt"
    out.write_text("\n".join(lines) + "\n")
    print(out.read_text())


if __name__ == "__main__":
    count(sys.argv[1] if len(sys.argv) > 1 else "batch")
