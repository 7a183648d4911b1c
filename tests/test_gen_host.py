"""The seeded input generators: the large-graph path that runs its searches and sorts in torch
builds the same graph as the numpy path."""
import numpy as np
import pytest

import gen


def test_chung_lu_same_graph_with_torch_sorts():
    a = gen.chung_lu_clusters(200_000, n_clusters=16, seed=5)
    b = gen.chung_lu_clusters(200_000, n_clusters=16, seed=5, device="cpu")
    assert a.nnz > 1_000_000
    assert np.array_equal(a.row_ptr, b.row_ptr)
    assert np.array_equal(a.col_idx, b.col_idx)
    assert np.array_equal(a.w, b.w)
    assert np.array_equal(a.labels, b.labels)


def test_from_edges_merges_duplicates_keeping_first_weight_with_torch_sorts():
    rng = np.random.default_rng(3)
    ea, eb = rng.integers(0, 500, 20_000), rng.integers(0, 500, 20_000)
    w = rng.uniform(0.5, 1.5, 20_000).astype(np.float32)
    x = gen.from_edges(500, ea, eb, w=w)
    y = gen.from_edges(500, ea, eb, w=w, device="cpu")
    assert np.array_equal(x.row_ptr, y.row_ptr) and np.array_equal(x.col_idx, y.col_idx)
    assert np.array_equal(x.w, y.w)


def test_common_neighbour_scores_brute_force():
    # shared neighbours counted pair by pair with Python sets on a small random graph
    rng = np.random.default_rng(5)
    n = 40
    pairs = {tuple(sorted(p)) for p in rng.integers(0, n, size=(150, 2)) if p[0] != p[1]}
    pairs = np.array(sorted(pairs))
    oa, ob = pairs[:, 0], pairs[:, 1]
    nb = {i: set() for i in range(n)}
    for x, y in zip(oa, ob):
        nb[x].add(y)
        nb[y].add(x)
    ra = rng.integers(0, n, size=60)
    rb = (ra + 1 + rng.integers(0, n - 1, size=60)) % n
    got = gen.common_neighbour_scores(n, oa, ob, ra, rb)
    want = [len(nb[x] & nb[y]) for x, y in zip(ra, rb)]
    assert got.tolist() == want


def test_link_completed_cliques_structure():
    sizes = [30, 25, 35]
    g, removed = gen.link_completed_cliques(sizes, short_circuit=4, p_remove=0.2, seed=9)
    base = gen.cliques(sizes, 4, seed=9)

    def edge_set(h):
        r = np.repeat(np.arange(h.n), np.diff(h.row_ptr))
        w = np.ones(h.nnz, np.float32) if h.w is None else h.w
        return {(int(i), int(j)): float(x) for i, j, x in zip(r, h.col_idx, w) if i < j}

    E, B = edge_set(g), edge_set(base)
    rem = {(int(i), int(j)) for i, j in removed.T}
    assert rem <= set(B) and all(i < j for i, j in rem)
    obs = set(B) - rem
    # every observed edge keeps weight 1; removed ones come back only with a positive score
    assert all(E.get(e) == 1.0 for e in obs)
    assert set(E) <= set(B)
    nb = {i: set() for i in range(g.n)}
    for i, j in obs:
        nb[i].add(j)
        nb[j].add(i)
    cn = {e: len(nb[e[0]] & nb[e[1]]) for e in rem}
    top = max(cn.values())
    for e in rem:
        if cn[e] == 0:
            assert e not in E
        else:
            assert E[e] == pytest.approx(cn[e] / top, rel=1e-6)
    # removal rate: binomial with p = 0.2 over the base edges, within 5 standard deviations
    m = len(B)
    assert abs(len(rem) - 0.2 * m) <= 5 * np.sqrt(m * 0.2 * 0.8)
    # symmetric storage, weights in (0, 1]
    assert g.w.min() > 0 and g.w.max() == 1.0
    assert np.array_equal(g.labels, base.labels)
