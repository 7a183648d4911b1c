"""Pins for the oracle's solvers, metrics, clustering and utility gradients (Sections 3, 5.1,
5.2; the EigenGame updates cited in Section 5.1)."""
import itertools
import math

import numpy as np
import pytest

import gen
import oracle


def _path_pairs(n):
    i = np.arange(n)
    U = np.stack([np.cos(math.pi * j * (i + 0.5) / n) for j in range(n)], axis=1)
    U /= np.linalg.norm(U, axis=0)
    lam = np.array([2 - 2 * math.cos(math.pi * j / n) for j in range(n)])
    return lam, U


def test_mu_eg_fixed_point():
    # true eigenvectors of M (ordered by decreasing eigenvalue) are a fixed point: r_i = 0
    n, k = 20, 5
    g = gen.path(n)
    lam, U = _path_pairs(n)
    lam_star = oracle.gershgorin_bound(g) * 1.01
    Uk = U[:, :k]
    Y = lam_star * Uk - oracle.laplacian_apply(g, Uk)  # Eq. reveig: L^- = lambda* I - L
    assert np.allclose(oracle.mu_eg_step(Uk, Y, 0.3), Uk, atol=1e-12)
    Y = oracle.poly_limit(g, Uk, 1 / 9, 9)
    assert np.allclose(oracle.mu_eg_step(Uk, Y, 0.7), Uk, atol=1e-12)


def test_mu_eg_and_oja_converge_to_bottom_k():
    g = gen.sbm(240, 4, 0.25, 0.01, seed=2)
    k = 4
    lam, Ustar = oracle.bottom_k(g, k)
    s = oracle.scale_rule(oracle.gershgorin_bound(g), 21)
    V = gen.gaussian_block(g.n, k, seed=3)
    V /= np.linalg.norm(V, axis=0)
    W = V.copy()
    for _ in range(170):
        V = oracle.mu_eg_step(V, oracle.poly_limit(g, V, s, 21), 1.0)
    for _ in range(40):
        W = oracle.oja_step(W, oracle.poly_limit(g, W, s, 21), 10.0)
    assert oracle.principal_angle_max(Ustar, V) < 1e-7
    assert oracle.principal_angle_max(Ustar, W) < 1e-7
    # Rayleigh-Ritz on the converged subspace recovers the bottom eigenvalues; individual
    # vectors of the close pair lambda_2 ~ lambda_3 converge more slowly than the span
    Q = oracle.orthonormal_basis(V)
    assert np.allclose(np.linalg.eigvalsh(Q.T @ oracle.laplacian_apply(g, Q)), lam, atol=1e-9)
    rho = oracle.ritz_values(V, oracle.laplacian_apply(g, V))
    assert abs(rho[0]) < 1e-9 and abs(rho[3] - lam[3]) < 1e-6


def _rotated_pair(n, k, thetas, seed=0):
    Q, _ = np.linalg.qr(np.random.default_rng(seed).standard_normal((n, 2 * k)))
    A = Q[:, :k]
    B = np.stack([math.cos(t) * Q[:, i] + math.sin(t) * Q[:, k + i]
                  for i, t in enumerate(thetas)], axis=1)
    return A, B


def test_principal_angle_and_subspace_error_closed_form():
    thetas = [1e-6, 3e-4, 0.2, 0.05]
    A, B = _rotated_pair(50, 4, thetas)
    assert oracle.principal_angle_max(A, B) == pytest.approx(max(thetas), rel=1e-9)
    # Section 5.2: delta = 1 - tr(U* P)/k = mean of sin^2 of the principal angles
    want = float(np.mean(np.sin(thetas) ** 2))
    assert oracle.subspace_error(A, B @ np.diag([2.0, -1.0, 0.5, 3.0])) == pytest.approx(
        want, rel=1e-9)
    A2, B2 = _rotated_pair(50, 3, [1e-9, 2e-9, 5e-10], seed=3)
    assert oracle.principal_angle_max(A2, B2) == pytest.approx(2e-9, rel=1e-4)


def test_streak():
    A, B = _rotated_pair(40, 4, [0.01, 0.02, 0.5, 0.001], seed=1)
    assert oracle.eigenvector_streak(B, A, math.pi / 8) == 2
    assert oracle.eigenvector_streak(B, A, 0.015) == 1
    assert oracle.eigenvector_streak(-B, A, 0.6) == 4


def test_kmeans_disjoint_cliques_exact_labels():
    sizes = [30, 20, 40, 25]
    g = gen.cliques(sizes)
    lam, U = oracle.bottom_k(g, len(sizes))
    labels = oracle.kmeans(U, len(sizes), seed=7)
    assert np.array_equal(labels, g.labels)  # components in node order, canonical relabel


def test_kmeans_brute_force_tiny():
    rng = np.random.default_rng(4)
    X = np.concatenate([rng.normal(0, 0.1, (4, 2)), rng.normal(5, 0.1, (3, 2)),
                        rng.normal([0, 9], 0.1, (2, 2))])
    K = 3
    best = None
    for assign in itertools.product(range(K), repeat=len(X)):
        a = np.array(assign)
        if len(set(assign)) < K:
            continue
        sse = sum(np.sum((X[a == c] - X[a == c].mean(0)) ** 2) for c in range(K))
        if best is None or sse < best[0] - 1e-12:
            best = (sse, a)
    lab = oracle.kmeans(X, K, seed=3)
    sse = sum(np.sum((X[lab == c] - X[lab == c].mean(0)) ** 2) for c in range(K))
    assert sse == pytest.approx(best[0], rel=1e-12)


def test_kmeanspp_seeding_distribution():
    # k-means++ (Arthur and Vassilvitskii, 2007): the first centre is uniform over the rows and
    # the second is drawn with probability D^2(x) / sum D^2 given the first
    X = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 2.0], [3.0, 1.0], [-1.0, -1.0], [2.0, 2.0]])
    n, trials = len(X), 6000
    first = np.zeros(n)
    pair = np.zeros((n, n))
    for s in range(trials):
        p = oracle.kmeanspp_seeds(X, 2, seed=s)
        first[p[0]] += 1
        pair[p[0], p[1]] += 1
    chi2 = float(np.sum((first - trials / n) ** 2 / (trials / n)))
    assert chi2 < 5 + 6 * np.sqrt(10)  # 5 dof
    D2 = np.sum((X[:, None, :] - X[None, :, :]) ** 2, axis=2)
    for f0 in range(n):
        m = pair[f0].sum()
        want = m * D2[f0] / D2[f0].sum()
        assert pair[f0, f0] == 0  # the first centre has D^2 = 0
        ok = want > 0
        chi2 = float(np.sum((pair[f0, ok] - want[ok]) ** 2 / want[ok]))
        assert chi2 < 4 + 6 * np.sqrt(8), (f0, pair[f0], want)


def test_kmeanspp_forced_choices():
    # rows at the first centre have D^2 = 0 and are never drawn again: with only one row away
    # from it, the second centre is that row whatever the draw; then a third centre can only
    # be the remaining distinct row
    X = np.array([[1.0, 1.0]] * 5 + [[4.0, 5.0]] + [[1.0, 1.0]] * 3 + [[-2.0, 0.5]])
    for s in range(50):
        p = oracle.kmeanspp_seeds(X, 3, seed=s)
        if p[0] not in (5, 9):
            assert {p[1], p[2]} == {5, 9}
        assert len({tuple(X[i]) for i in p}) == 3


def _fd_grad_V(f, V, h=1e-4):
    G = np.empty_like(V)
    for idx in np.ndindex(V.shape):
        Vp, Vm = V.copy(), V.copy()
        Vp[idx] += h
        Vm[idx] -= h
        G[idx] = (f(Vp) - f(Vm)) / (2 * h)
    return G


def test_utility_gradients_against_finite_differences():
    g = gen.uniform_edge_weights(gen.sbm(40, 2, 0.3, 0.05, seed=6), seed=7)
    s, ell, k = 0.02, 5, 3
    V = gen.gaussian_block(g.n, k, seed=8)
    g_u = np.array([1.0, 0.5, 2.0])

    def f(Vx):
        return float(g_u @ oracle.eg_utilities(Vx, oracle.poly_limit(g, Vx, s, ell)))

    Y = oracle.poly_limit(g, V, s, ell)
    assert np.allclose(_fd_grad_V(f, V), oracle.eg_grad_full(V, Y, g_u), rtol=1e-6, atol=1e-7)
    # detached parents: d u_i / d v_i with v_j (j < i) frozen -- the EigenGame direction
    Gd = oracle.eg_grad_detached(V, Y)
    for i in range(k):
        def fi(col):
            Vx = V.copy()
            Vx[:, i] = col
            return float(oracle.eg_utilities(Vx, oracle.poly_limit(g, Vx, s, ell))[i])
        fd = _fd_grad_V(lambda c: fi(c[:, 0]), V[:, i:i + 1])[:, 0]
        assert np.allclose(fd, Gd[:, i], rtol=1e-6, atol=1e-7)


def test_edge_gradient_against_finite_differences():
    g = gen.uniform_edge_weights(gen.sbm(30, 2, 0.3, 0.08, seed=9), seed=10)
    s, ell, k = 0.03, 6, 3
    V = gen.gaussian_block(g.n, k, seed=11)
    g_u = np.array([1.0, -0.7, 0.4])
    a, b, w = oracle.edge_list(g)

    def f(wv):
        gg = oracle.with_edge_weights(g, wv)
        return float(g_u @ oracle.eg_utilities(V, oracle.poly_limit(gg, V, s, ell)))

    Y = oracle.poly_limit(g, V, s, ell)
    Hb = oracle.eg_utility_hbar(V.T @ Y, g_u)
    grad = oracle.limit_edge_grad(g, V, s, ell, Hb)
    h = 1e-4
    # weights pass through float32 storage: perturb in float64 by building the graph from an
    # exactly representable base
    w0 = w.astype(np.float32).astype(np.float64)
    rng = np.random.default_rng(0)
    for e in rng.choice(len(w0), size=min(12, len(w0)), replace=False):
        hp = np.float32(w0[e] + h) - w0[e]
        hm = w0[e] - np.float32(w0[e] - h)
        wp, wm = w0.copy(), w0.copy()
        wp[e] += hp
        wm[e] -= hm
        fd = (f(wp) - f(wm)) / (hp + hm)
        assert fd == pytest.approx(grad[e], rel=2e-5, abs=1e-8)


def test_rayleigh_ritz_invariant_subspace_gives_exact_eigenpairs():
    # path graph P_n: lambda_j = 2 - 2 cos(pi j / n), u_j(x) = cos(pi j (x + 1/2) / n)
    n, k = 40, 5
    g = gen.path(n)
    x = np.arange(n) + 0.5
    U = np.stack([np.cos(np.pi * j * x / n) for j in range(k)], axis=1)
    lam = 2.0 - 2.0 * np.cos(np.pi * np.arange(k) / n)
    G = np.random.default_rng(1).standard_normal((k, k))  # any basis of the same span
    theta, W = oracle.rayleigh_ritz(g, U @ G)
    assert np.allclose(theta, lam, atol=1e-12)
    X = U @ G @ W  # Ritz vectors: orthonormal eigenvectors, up to sign
    assert np.allclose(X.T @ X, np.eye(k), atol=1e-12)
    for i in range(k):
        u = U[:, i] / np.linalg.norm(U[:, i])
        assert abs(abs(u @ X[:, i]) - 1.0) <= 1e-12


def test_rayleigh_ritz_interlacing_and_galerkin_condition():
    # cycle C_n: lambda = 2 - 2 cos(2 pi j / n); for any k-dimensional span the i-th Ritz
    # value lies between the i-th smallest and the i-th of the top k eigenvalues (Cauchy)
    n, k = 31, 6
    g = gen.cycle(n)
    lam = np.sort(2.0 - 2.0 * np.cos(2.0 * np.pi * np.arange(n) / n))
    V = np.random.default_rng(2).standard_normal((n, k))
    theta, W = oracle.rayleigh_ritz(g, V)
    assert np.all(np.diff(theta) >= -1e-12)
    assert np.all(theta >= lam[:k] - 1e-12) and np.all(theta <= lam[n - k:] + 1e-12)
    X = V @ W
    R = oracle.laplacian_apply(g, X) - X * theta  # residuals orthogonal to span(V)
    assert np.abs(V.T @ R).max() <= 1e-10 * np.abs(V).max() * np.abs(X).max() * n
    theta2, _ = oracle.rayleigh_ritz(g, V @ np.random.default_rng(3).standard_normal((k, k)))
    assert np.allclose(theta2, theta, atol=1e-12)
