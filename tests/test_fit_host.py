"""Host-side algebra of the coefficient fit used by the benchmark's fitted-polynomial
measurement: the quadratic forms built from the block moments equal Y^T Y and Y^T L Y computed
directly from Y = M V (oracle chains), and the fit does not increase the Ritz-value sum."""
import numpy as np
import pytest

import bench
import gen
import oracle


def test_quadratic_forms_from_moments_match_direct_products():
    pytest.importorskip("scipy")
    g = gen.uniform_edge_weights(gen.random_graph(120, 400, seed=81), seed=82)
    k, d = 3, 6
    V = gen.gaussian_block(g.n, k, seed=83)
    a, b = 0.0, oracle.gershgorin_bound(g)
    mu = oracle.poly_moments(g, V, 2 * d + 2, basis="chebyshev", a=a, b=b)
    A, Bm = bench._cheb_quadratic_forms(mu, d, k, a, b)
    c = np.random.default_rng(84).standard_normal(d + 1)
    Y = oracle.poly_chebyshev(g, V, c, a, b)
    S = np.einsum("l,m,lmij->ij", c, c, A)
    Q = np.einsum("l,m,lmij->ij", c, c, Bm)
    assert np.allclose(S, Y.T @ Y, rtol=1e-9, atol=1e-9 * np.abs(S).max())
    LY = oracle.laplacian_apply(g, Y)
    assert np.allclose(Q, Y.T @ LY, rtol=1e-9, atol=1e-9 * np.abs(Q).max())


def test_fit_lowers_the_ritz_value_sum():
    pytest.importorskip("scipy")
    g = gen.sbm(300, 3, 0.1, 0.005, seed=85)
    k, d = 3, 8
    V = gen.gaussian_block(g.n, k, seed=86)
    a, b = 0.0, oracle.gershgorin_bound(g)
    mu = oracle.poly_moments(g, V, 2 * d + 2, basis="chebyshev", a=a, b=b)
    c0 = np.zeros(d + 1)
    c0[0] = 1.0  # M = I: the Ritz values of L on span(V) itself
    c, fval = bench._fit_chebyshev(mu, d, k, a, b, c0)
    Q, _ = np.linalg.qr(V)
    start = float(np.trace(Q.T @ oracle.laplacian_apply(g, Q)))
    assert fval < start
    Y = oracle.poly_chebyshev(g, V, c, a, b)
    Qy, _ = np.linalg.qr(Y)
    assert float(np.trace(Qy.T @ oracle.laplacian_apply(g, Qy))) == pytest.approx(fval, rel=1e-6)
    lam = np.linalg.eigvalsh(oracle.dense_laplacian(g))
    assert fval >= lam[:k].sum() - 1e-9
