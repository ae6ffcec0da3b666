"""The seeded input generator: determinism, tree validity, restriction, random field."""
import numpy as np
import pytest

from paper_1210_8014_gb300 import inputs


def check_tree(t):
    n = t.n_oct
    assert t.level[0] == 1 and (t.coord[0] == 0).all()
    refs = t.child[t.child >= 0]
    assert len(np.unique(refs)) == refs.size == n - 1          # every non-root oct referenced once
    o, c = np.nonzero(t.child >= 0)
    ch = t.child[o, c]
    assert (t.level[ch] == t.level[o] + 1).all()
    off = np.stack([(c >> a) & 1 for a in range(3)], 1)
    assert (t.coord[ch] == 2 * (t.coord[o] + off)).all()
    assert (ch > o).all()                                       # breadth-first: children after parents


def test_plain_tree_shape():
    t = inputs.plain_tree()
    check_tree(t)
    assert 30_000 <= t.n_leaves <= 45_000
    assert set(int(k) for k in t.info["leaf_hist"]) <= {5, 6, 7}
    assert t.depth == 7


def test_restriction_conserves_mass_and_momentum():
    t = inputs.galaxy_tree(2, 2.0 ** -14, 10, with_velocity=True, dtype=np.float64)
    check_tree(t)
    lv = t.level.astype(np.int64)
    vol = np.ldexp(1.0, -3 * lv)[:, None]
    leaf = t.child < 0
    m_leaf = (t.fields[0] * vol)[leaf].sum()
    m_root = (t.fields[0][0] * vol[0]).sum()
    assert abs(m_leaf - m_root) <= 1e-12 * m_root
    for a in range(1, 4):
        p_leaf = (t.fields[0] * t.fields[a] * vol)[leaf].sum()
        p_root = (t.fields[0][0] * t.fields[a][0] * vol[0]).sum()
        assert abs(p_leaf - p_root) <= 1e-10 * np.abs(t.fields[0] * vol)[leaf].sum()


def test_deterministic():
    a = inputs.galaxy_tree(5, 2.0 ** -12, 9, with_velocity=False)
    b = inputs.galaxy_tree(5, 2.0 ** -12, 9, with_velocity=False, )
    assert a.n_oct == b.n_oct
    assert (a.child == b.child).all() and (a.fields[0] == b.fields[0]).all()
    c = inputs.galaxy_tree(6, 2.0 ** -12, 9, with_velocity=False)
    assert c.n_oct != a.n_oct or not (c.fields[0] == a.fields[0]).all()


def test_grf_unit_variance_and_kolmogorov_slope():
    rng = np.random.default_rng(0)
    for seed in (2, 3, 4):
        g = inputs.sample_model(inputs.GEN_GALAXY, 1, rng.uniform(0, 1, (100_000, 3)), seed=seed)
        assert abs(g.mean()) < 0.25 and 0.7 < g.var() < 1.4
    n = 64
    ax = (np.arange(n) + 0.5) / n
    X, Y, Z = np.meshgrid(ax, ax, ax, indexing="ij")
    g = inputs.sample_model(inputs.GEN_GALAXY, 1, np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1),
                            seed=3).reshape(n, n, n)
    P = np.abs(np.fft.fftn(g)) ** 2
    k = np.fft.fftfreq(n, 1.0 / n)
    K = np.sqrt(sum(q ** 2 for q in np.meshgrid(k, k, k, indexing="ij")))
    edges = 2.0 ** np.arange(0, 5.01, 0.5)
    kc, pk = [], []
    for lo, hi in zip(edges[:-1], edges[1:]):
        m = (K >= lo) & (K < hi)
        kc.append(np.sqrt(lo * hi))
        pk.append(P[m].mean())
    slope = np.polyfit(np.log(kc), np.log(pk), 1)[0]
    assert abs(slope - (-11.0 / 3.0)) < 0.3, slope


def test_generator_rejects_bad_params():
    with pytest.raises(RuntimeError):
        inputs.generate(inputs.GEN_GALAXY, 7, 23, 1e-3)
    with pytest.raises(RuntimeError):
        inputs.generate(7, 3, 7, 1e-3)
