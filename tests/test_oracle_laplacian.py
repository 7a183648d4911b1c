"""Pins for the oracle's Laplacian application (Section 2) against closed forms and identities
that do not go through the oracle's own code path."""
import math

import numpy as np
import pytest

import gen
import oracle


def _dense_via_oracle(g):
    return oracle.laplacian_apply(g, np.eye(g.n))


def test_ones_in_kernel_unweighted_and_weighted():
    # Section 2: L 1 = 0
    for g in [gen.sbm(300, 3, 0.1, 0.01, seed=1),
              gen.uniform_edge_weights(gen.random_graph(200, 900, seed=2), seed=3),
              gen.chung_lu_clusters(500, n_clusters=4, seed=4)]:
        y = oracle.laplacian_apply(g, np.ones(g.n))
        assert np.max(np.abs(y)) < 1e-10


def test_cut_quadratic_form_eq1():
    # Eq. 1: v^T L v = sum_e w_e (v_i - v_j)^2, summed over the edge list directly
    g = gen.uniform_edge_weights(gen.random_graph(150, 700, seed=5), seed=6)
    rng = np.random.default_rng(0)
    for _ in range(3):
        v = rng.standard_normal(g.n)
        lhs = float(v @ oracle.laplacian_apply(g, v))
        assert lhs == pytest.approx(oracle.cut_value(g, v), rel=1e-12)
    # the +-1 cut indicator counts 4x the crossing edges (Section 2.1)
    gu = gen.random_graph(120, 400, seed=7)
    s = np.where(np.arange(gu.n) < 60, 1.0, -1.0)
    a, b, _ = oracle.edge_list(gu)
    crossing = int(np.sum((a < 60) != (b < 60)))
    assert float(s @ oracle.laplacian_apply(gu, s)) == pytest.approx(4 * crossing)


def test_incidence_gram_equals_laplacian():
    # Section 2: L = X^T W X = sum_e w_e x_e x_e^T (weighted incidence rows)
    g = gen.uniform_edge_weights(gen.random_graph(60, 200, seed=8), seed=9)
    X = oracle.incidence_matrix(g)
    assert np.allclose(X.T @ X, _dense_via_oracle(g), atol=1e-12)


def test_dense_brute_force():
    g = gen.uniform_edge_weights(gen.random_graph(64, 300, seed=10, hub=3, hub_degree=40,
                                                  isolated=5), seed=11)
    V = np.random.default_rng(1).standard_normal((g.n, 5))
    assert np.allclose(oracle.dense_laplacian(g) @ V, oracle.laplacian_apply(g, V),
                       rtol=1e-13, atol=1e-12)


def test_path_closed_form_eigenpairs():
    # path P_n: lambda_j = 2 - 2 cos(pi j / n), eigenvector cos(pi j (i + 1/2) / n)
    n = 37
    g = gen.path(n)
    i = np.arange(n)
    for j in range(n):
        u = np.cos(math.pi * j * (i + 0.5) / n)
        lam = 2 - 2 * math.cos(math.pi * j / n)
        assert np.allclose(oracle.laplacian_apply(g, u), lam * u, atol=1e-12)


@pytest.mark.parametrize("kind", ["cycle", "complete", "star", "grid", "cliques"])
def test_closed_form_spectra(kind):
    if kind == "cycle":
        n = 24
        g = gen.cycle(n)
        want = np.sort([2 - 2 * math.cos(2 * math.pi * j / n) for j in range(n)])
    elif kind == "complete":
        n = 15
        g = gen.complete(n)
        want = np.array([0.0] + [float(n)] * (n - 1))
    elif kind == "star":
        n = 13
        g = gen.star(n)
        want = np.array([0.0] + [1.0] * (n - 2) + [float(n)])
    elif kind == "grid":
        r, c = 5, 7
        g = gen.grid(r, c)
        pr = [2 - 2 * math.cos(math.pi * j / r) for j in range(r)]
        pc = [2 - 2 * math.cos(math.pi * j / c) for j in range(c)]
        want = np.sort([x + y for x in pr for y in pc])
    else:
        sizes = [5, 7, 4, 9]
        g = gen.cliques(sizes)
        want = np.sort([0.0] * len(sizes) + sum([[float(s)] * (s - 1) for s in sizes], []))
    lam = np.linalg.eigvalsh(_dense_via_oracle(g))
    assert np.allclose(lam, want, atol=1e-10)
    if kind == "cliques":
        # zero-eigenvalue multiplicity = number of connected components
        assert int(np.sum(np.abs(lam) < 1e-9)) == 4


def test_gershgorin_bound():
    # Section 5.4: the spectral radius is at most twice the maximum degree
    for g in [gen.star(30), gen.complete(12), gen.sbm(400, 4, 0.08, 0.01, seed=3),
              gen.uniform_edge_weights(gen.random_graph(80, 300, seed=4), seed=5)]:
        lam = np.linalg.eigvalsh(_dense_via_oracle(g))
        assert lam[-1] <= oracle.gershgorin_bound(g) + 1e-9


def test_degrees_are_row_sums():
    g = gen.uniform_edge_weights(gen.random_graph(90, 400, seed=12), seed=13)
    d = oracle.degrees(g)
    L = oracle.dense_laplacian(g)
    assert np.allclose(d, np.diag(L), rtol=1e-13)


def test_planted_mistake_is_caught(monkeypatch):
    # A dropped diagonal term or a flipped off-diagonal sign must fail the pins above.
    g = gen.path(9)
    true = oracle.laplacian_apply

    def wrong_sign(gg, X):
        return true(gg, X) - 2 * (oracle.degrees(gg)[:, None] * np.atleast_2d(X.T).T
                                  - true(gg, X)) if X.ndim == 2 else None

    def no_diag(gg, X):
        X2 = X if X.ndim == 2 else X[:, None]
        out = true(gg, X2) - oracle.degrees(gg)[:, None] * X2
        return out if X.ndim == 2 else out[:, 0]

    y = no_diag(g, np.ones(g.n))
    assert np.max(np.abs(y)) > 0.5  # L 1 = 0 fails
    i = np.arange(g.n)
    u = np.cos(math.pi * 1 * (i + 0.5) / g.n)
    lam = 2 - 2 * math.cos(math.pi / g.n)
    bad = wrong_sign(g, u[:, None])[:, 0]
    assert not np.allclose(bad, lam * u, atol=1e-6)


def test_linear_time_cycle_builder_matches_the_edge_list_builder():
    for n in (3, 4, 5, 17):
        a, b = gen.cycle_csr(n), gen.cycle(n)
        assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col_idx, b.col_idx)
    # the hashed block is the same on the host and in torch, and exact in BF16
    torch = pytest.importorskip("torch")
    rows = np.array([0, 1, 7, 2 ** 27 + 3])
    h = gen.hash_block(rows, 6)
    assert np.array_equal(h, gen.hash_block(torch.from_numpy(rows), 6, xp=torch).numpy())
    assert np.array_equal(h, torch.from_numpy(h).to(torch.bfloat16).double().numpy())
