"""The launch tables give a ray's lattice origin as rint(A_i + B_j), with the
column term A_i = (centre + s_i u) 2^36 and the row term B_j = (t_j v) 2^36
rounded on the host.  The same arithmetic restated here in float64 (numpy,
no contraction) must give, bit for bit, the oracle's origin
rint(((centre + s_i u) + t_j v) 2^36) — scaling by a power of two commutes
with the rounding of the sum — over random cameras, including tiny fields of
view, centres near 0 and axes with tiny components."""
import numpy as np

import oracle
from paper_1210_8014_gb300 import inputs

SCALE = np.float64(68719476736.0)   # 2^36


def table_origin(cam, i, j):
    s = ((np.float64(i) + 0.5) / np.float64(cam.nx) - 0.5) * np.float64(cam.fov[0])
    t = ((np.float64(j) + 0.5) / np.float64(cam.ny) - 0.5) * np.float64(cam.fov[1])
    c = np.asarray(cam.centre, np.float64)
    A = (c + s * np.asarray(cam.u, np.float64)) * SCALE
    B = (t * np.asarray(cam.v, np.float64)) * SCALE
    return np.rint(A + B).astype(np.int64)


def test_column_and_row_terms_reproduce_the_oracle_origin():
    lib = oracle.load()
    rng = np.random.default_rng(77)
    cams = []
    for k in range(60):
        w = inputs.random_direction(rng) if k % 4 else (1e-9, 2e-12, 1.0)   # near-axis: tiny components
        centre = rng.uniform(-0.4, 1.4, 3) if k % 3 else rng.uniform(-1e-6, 1e-6, 3)
        fov = float(2.0 ** rng.uniform(-30, 0.4))
        n = (int(rng.integers(1, 40)), int(rng.integers(1, 40)))
        cams.append(inputs.camera_along(w, centre=tuple(centre), fov=fov, n=n))
    checked = 0
    for cam in cams:
        for j in range(cam.ny):
            for i in range(cam.nx):
                assert (table_origin(cam, i, j) == oracle.ray_origin(cam, i, j, lib=lib)).all(), (cam, i, j)
                checked += 1
    assert checked > 10000
