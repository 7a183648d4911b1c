"""Pins for the oracle's minibatch estimates (the stochastic optimisation model of Sections 2
and 6: edges fed in minibatches; L as the sum of the edges' outer products, Section 4.3).

The exact chains they are checked against (poly_limit, poly_horner, poly_chebyshev,
laplacian_apply) are pinned on their own in test_oracle_laplacian.py / test_oracle_poly.py."""
import itertools

import numpy as np
import pytest

import gen
import oracle


def _tiny_weighted():
    # 5 nodes, 4 edges (a path with one chord), distinct weights
    g = gen.from_edges(5, np.array([0, 1, 2, 1]), np.array([1, 2, 3, 4]),
                       w=np.array([1.0, 0.5, 2.0, 1.5], dtype=np.float32))
    return g


def _fixed_operator(m, edges_per_step):
    """L_hat_t from a given list of per-step edge samples (a, b, w arrays)."""
    def apply(t, X):
        a, b, w = edges_per_step[t]
        return oracle.minibatch_laplacian_apply(m, X, a, b, w)
    return apply


def test_edge_ids_uniform_and_in_range():
    m, B = 37, 74000
    ids = oracle.minibatch_edge_ids(m, seed=5, step=3, batch=B)
    assert ids.min() >= 0 and ids.max() < m
    counts = np.bincount(ids, minlength=m)
    e = B / m
    chi2 = float(np.sum((counts - e) ** 2 / e))
    assert chi2 < 90.0  # 36 dof: p ~ 3e-6
    # the draws of different steps are different streams
    other = oracle.minibatch_edge_ids(m, seed=5, step=4, batch=B)
    assert np.mean(ids == other) < 2.0 / m
    # a draw does not depend on the batch size (one stream per draw)
    assert np.array_equal(oracle.minibatch_edge_ids(m, 5, 3, 100), ids[:100])


def test_sampled_edges_are_edges_of_the_graph():
    g = gen.uniform_edge_weights(gen.random_graph(60, 150, seed=3), seed=4)
    A = np.zeros((g.n, g.n))
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr))
    A[rows, g.col_idx] = g.w
    a, b, w = oracle.minibatch_edges(g, seed=9, step=0, batch=500)
    assert np.all(a < b)
    assert np.all(A[a, b] > 0)
    assert np.allclose(w, A[a, b])


def test_one_minibatch_is_unbiased_exactly():
    # E over every equally likely pair of draws (B = 2) of L_hat X equals L X
    g = _tiny_weighted()
    a, b, w = oracle.edge_list(g)
    m = len(a)
    X = gen.gaussian_block(g.n, 3, seed=1)
    acc = np.zeros_like(X)
    for i, j in itertools.product(range(m), repeat=2):
        idx = np.array([i, j])
        acc += oracle.minibatch_laplacian_apply(m, X, a[idx], b[idx], w[idx])
    assert np.allclose(acc / m ** 2, oracle.laplacian_apply(g, X), rtol=0, atol=1e-13)


@pytest.mark.parametrize("family", ["limit", "horner", "clenshaw"])
def test_chain_is_unbiased_by_exhaustive_enumeration(family):
    # one edge per multiplication, every sequence of edges over the l multiplications
    g = _tiny_weighted()
    a, b, w = oracle.edge_list(g)
    m, ell = len(a), 3
    V = gen.gaussian_block(g.n, 2, seed=2)
    coeffs = oracle.taylor_exp_coeffs(ell)
    if family == "limit":
        exact = oracle.poly_limit(g, V, 0.2, ell)
    elif family == "horner":
        exact = oracle.poly_horner(g, V, coeffs, shift=-0.3)
    else:
        exact = oracle.poly_chebyshev(g, V, [0.3, -0.2, 0.7, 0.4], 0.1, 5.0)
    acc = np.zeros_like(V)
    for seq in itertools.product(range(m), repeat=ell):
        op = _fixed_operator(m, [(a[[e]], b[[e]], w[[e]]) for e in seq])
        if family == "limit":
            acc += oracle.stochastic_limit(V, 0.2, ell, op)
        elif family == "horner":
            acc += oracle.stochastic_horner(V, coeffs, -0.3, op)
        else:
            acc += oracle.stochastic_clenshaw(V, [0.3, -0.2, 0.7, 0.4], 0.1, 5.0, op)
    assert np.allclose(acc / m ** ell, exact, rtol=0, atol=1e-12 * np.abs(exact).max())


def test_reusing_one_sample_for_every_factor_would_be_biased():
    # the same enumeration with one shared edge per chain: E[(I - s m w x x^T)^l] != (I - sL)^l
    g = _tiny_weighted()
    a, b, w = oracle.edge_list(g)
    m, ell, s = len(a), 3, 0.2
    V = gen.gaussian_block(g.n, 2, seed=2)
    acc = np.zeros_like(V)
    for e in range(m):
        op = _fixed_operator(m, [(a[[e]], b[[e]], w[[e]])] * ell)
        acc += oracle.stochastic_limit(V, s, ell, op)
    assert np.abs(acc / m - oracle.poly_limit(g, V, s, ell)).max() > 1e-2


def test_single_edge_graph_is_exact_for_any_sample():
    # with one edge every draw is that edge and L_hat = L, whatever the batch size
    g = gen.from_edges(6, np.array([2]), np.array([4]), w=np.array([1.7], dtype=np.float32))
    V = gen.gaussian_block(g.n, 3, seed=4)
    for B in (1, 3, 8):
        op = oracle.minibatch_operator(g, seed=11, batch=B)
        assert np.allclose(oracle.stochastic_limit(V, 0.25, 5, op),
                           oracle.poly_limit(g, V, 0.25, 5), atol=1e-13)
        c = oracle.taylor_log_coeffs(4)
        assert np.allclose(oracle.stochastic_horner(V, c, -0.999, op),
                           oracle.poly_horner(g, V, c, shift=-0.999), atol=1e-13)
        cc = [0.1, 0.2, -0.3, 0.4, 0.5]
        assert np.allclose(oracle.stochastic_clenshaw(V, cc, 0.2, 3.0, op),
                           oracle.poly_chebyshev(g, V, cc, 0.2, 3.0), atol=1e-12)


def test_sampler_and_chain_mean_converges():
    # the real sampler (streams keyed by step) over many seeds: the sample mean of the chain
    # lies within a few standard errors of (I - sL)^l V
    g = _tiny_weighted()
    V = gen.gaussian_block(g.n, 2, seed=7)
    ell, s, R = 3, 0.15, 3000
    outs = np.stack([oracle.stochastic_limit(V, s, ell, oracle.minibatch_operator(g, r, 2))
                     for r in range(R)])
    mean, se = outs.mean(0), outs.std(0, ddof=1) / np.sqrt(R)
    exact = oracle.poly_limit(g, V, s, ell)
    assert np.all(np.abs(mean - exact) <= 5.0 * se + 1e-12)


# ---- stratified minibatches (variance reduction) ----------------------------------------
def test_strata_partition_the_edges():
    for m, B in [(37, 5), (37, 37), (10, 16), (1000, 7)]:
        ids, sizes = oracle.stratified_edge_ids(m, seed=3, step=2, batch=B)
        assert sizes.sum() == m
        lo = np.array([j * m // B for j in range(B)])
        assert np.all((sizes == 0) == (ids < 0))
        nz = sizes > 0
        assert np.all(ids[nz] >= lo[nz]) and np.all(ids[nz] < lo[nz] + sizes[nz])
    # within one stratum the draw is uniform
    m, B = 50, 5
    hits = np.stack([oracle.stratified_edge_ids(m, s, 0, B)[0] for s in range(20000)])
    counts = np.bincount(hits[:, 2], minlength=m)[20:30]
    chi2 = float(np.sum((counts - 2000.0) ** 2 / 2000.0))
    assert chi2 < 40.0  # 9 dof


def test_stratified_sample_is_unbiased_exactly():
    # every combination of one edge per stratum, each with probability prod 1/|S_j|
    g = _tiny_weighted()
    a, b, w = oracle.edge_list(g)
    m, B = len(a), 3
    X = gen.gaussian_block(g.n, 2, seed=5)
    lo = [j * m // B for j in range(B)]
    hi = [(j + 1) * m // B for j in range(B)]
    sizes = np.array([h - l for l, h in zip(lo, hi)], dtype=np.float64)
    acc, count = np.zeros_like(X), 0
    for combo in itertools.product(*[range(l, h) for l, h in zip(lo, hi)]):
        idx = np.array(combo)
        acc += oracle.stratified_laplacian_apply(X, a[idx], b[idx], w[idx], sizes)
        count += 1
    assert count == int(np.prod(sizes))
    assert np.allclose(acc / count, oracle.laplacian_apply(g, X), rtol=0, atol=1e-13)


def test_one_stratum_per_edge_is_exact():
    g = gen.uniform_edge_weights(gen.random_graph(40, 90, seed=6), seed=7)
    m = len(oracle.edge_list(g)[0])
    V = gen.gaussian_block(g.n, 3, seed=8)
    for B in (m, m + 13):  # |S_j| = 1, or empty strata
        op = oracle.minibatch_operator(g, seed=4, batch=B, stratified=True)
        assert np.allclose(oracle.stochastic_limit(V, 0.1, 5, op), oracle.poly_limit(g, V, 0.1, 5),
                           atol=1e-12)


def test_stratified_chain_mean_converges():
    g = _tiny_weighted()
    V = gen.gaussian_block(g.n, 2, seed=7)
    ell, s, R = 3, 0.15, 3000
    outs = np.stack([oracle.stochastic_limit(V, s, ell,
                                             oracle.minibatch_operator(g, r, 2, stratified=True))
                     for r in range(R)])
    mean, se = outs.mean(0), outs.std(0, ddof=1) / np.sqrt(R)
    assert np.all(np.abs(mean - oracle.poly_limit(g, V, s, ell)) <= 5.0 * se + 1e-12)
