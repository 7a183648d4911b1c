"""The seeded input generators: the large-graph path that runs its searches and sorts in torch
builds the same graph as the numpy path."""
import numpy as np

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
