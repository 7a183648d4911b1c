"""Pins for the oracle's eigenvector-preserving polynomials (Sections 4.1-4.2, Table 2)."""
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


@pytest.mark.parametrize("ell", [1, 5, 11, 51])
def test_limit_preserves_eigenvectors(ell):
    # Section 4.1: p(L) v_i = p(lambda_i) v_i, p(lambda) = (1 - s lambda)^ell
    n = 31
    g = gen.path(n)
    lam, U = _path_pairs(n)
    s = 1.0 / ell if ell >= 2 else 0.2
    Y = oracle.poly_limit(g, U, s, ell)
    assert np.allclose(Y, U * oracle.limit_scalar(lam, s, ell), atol=1e-12)


def test_limit_is_monotone_for_odd_ell():
    # Table 2 note: ell odd, so (1 - s lambda)^ell is monotone on the whole real line
    lam = np.linspace(-3, 300, 2001)
    for ell in [1, 3, 11, 251]:
        p = oracle.limit_scalar(lam, 1.0 / ell, ell)
        assert np.all(np.diff(p) <= 0)


def test_limit_approaches_decaying_exponential():
    # e^{-x} (1 - x^2/ell) <= (1 - x/ell)^ell <= e^{-x} for 0 <= x <= ell (textbook bound)
    n = 25
    g = gen.path(n)
    lam, U = _path_pairs(n)
    for ell in [11, 51, 151, 251]:
        Y = oracle.poly_limit(g, U, 1.0 / ell, ell)
        got = np.einsum("ni,ni->i", U, Y)
        hi = np.exp(-lam)
        lo = np.exp(-lam) * (1 - lam ** 2 / ell)
        assert np.all(got <= hi + 1e-12) and np.all(got >= lo - 1e-12)


def test_brute_force_spectral_calculus():
    # U p(Lambda) U^T V by dense eigendecomposition on a random weighted graph
    g = gen.uniform_edge_weights(gen.random_graph(120, 500, seed=21, isolated=3), seed=22)
    V = np.random.default_rng(2).standard_normal((g.n, 4))
    lam, U = np.linalg.eigh(oracle.dense_laplacian(g))
    s, ell = 1.0 / oracle.gershgorin_bound(g), 9
    want = U @ (oracle.limit_scalar(lam, s, ell)[:, None] * (U.T @ V))
    assert np.allclose(oracle.poly_limit(g, V, s, ell), want, atol=1e-11)
    c = oracle.taylor_exp_coeffs(12)
    Ls = lam * 0.1  # scale the graph so the Taylor series is accurate
    gs = gen.CSRGraph(g.n, g.row_ptr, g.col_idx, (g.w * 0.1).astype(np.float32))
    want = U @ (np.polyval(c[::-1], np.linalg.eigvalsh(oracle.dense_laplacian(gs)))[:, None]
                * (U.T @ V))
    assert np.allclose(oracle.poly_horner(gs, V, c), want, atol=1e-10)


def test_horner_taylor_exp_on_eigenpairs():
    # Table 2: Taylor -e^{-L}, reversed (lambda* = 0): M = sum_i (-L)^i / i!
    n = 21
    g = gen.path(n)
    lam, U = _path_pairs(n)
    ell = 31
    Y = oracle.poly_horner(g, U, oracle.taylor_exp_coeffs(ell))
    want = np.array([sum((-x) ** i / math.factorial(i) for i in range(ell + 1)) for x in lam])
    assert np.allclose(Y, U * want, atol=1e-12)
    # and it approximates e^{-lambda} there (spectrum of the path lies in [0, 4])
    assert np.allclose(want, np.exp(-lam), atol=1e-12)


def test_horner_taylor_log_small_radius():
    # Table 2: Taylor series of log(L + eps I) converges only for spectral radius < 2 (Sec 5.3)
    n = 15
    lam, U = _path_pairs(n)
    scale = 0.45  # weights 0.45 -> spectrum in [0, 1.8]
    base = gen.path(n)
    g = gen.CSRGraph(n, base.row_ptr, base.col_idx,
                     np.full(base.nnz, scale, dtype=np.float32))
    eps, ell = 1e-3, 400
    c = oracle.taylor_log_coeffs(ell)
    Y = oracle.poly_horner(g, U, c, shift=eps - 1.0)
    mu = lam * scale
    got = np.einsum("ni,ni->i", U, Y)
    # exact truncated series on each eigenvalue
    trunc = np.array([sum((-1) ** (i + 1) * (m + eps - 1) ** i / i for i in range(1, ell + 1))
                      for m in mu])
    assert np.allclose(got, trunc, atol=1e-11)
    # away from the eps pole the truncation error is small
    far = mu > 0.05
    assert np.allclose(got[far], np.log(mu[far] + eps), atol=1e-6)


def test_power_coefficients_match_limit():
    g = gen.sbm(60, 3, 0.3, 0.05, seed=5)
    V = np.random.default_rng(3).standard_normal((g.n, 3))
    s, ell = 0.02, 7
    assert np.allclose(oracle.walk_exact_terms(g, V, oracle.limit_power_coeffs(s, ell)),
                       oracle.poly_limit(g, V, s, ell), atol=1e-11)


def test_scale_rule():
    assert oracle.scale_rule(80.0, 41) == pytest.approx(1 / 41)
    assert oracle.scale_rule(300.0, 41) == pytest.approx(2 / 300)


def test_chebyshev_on_closed_form_eigenpairs():
    # path graph eigenpairs; the interval covers part of the spectrum so both the cos and the
    # cosh branches of T_j occur
    n = 30
    g = gen.path(n)
    x = np.arange(n) + 0.5
    j = np.arange(n)
    U = np.cos(np.pi * np.outer(x, j) / n)
    lam = 2.0 - 2.0 * np.cos(np.pi * j / n)
    c = np.array([0.3, -0.7, 0.25, 0.0, 1.1, -0.05, 0.4])
    a, b = 0.6, 3.2
    Y = oracle.poly_chebyshev(g, U, c, a, b)
    want = U * oracle.chebyshev_scalar(c, (2.0 * lam - (a + b)) / (b - a))
    assert np.allclose(Y, want, rtol=1e-10, atol=1e-9 * np.abs(want).max())


def test_chebyshev_product_identity():
    # T_m T_n = (T_{m+n} + T_{|m-n|}) / 2 as operators on a random block
    g = gen.random_graph(80, 300, seed=9)
    V = np.random.default_rng(3).standard_normal((g.n, 3))
    a, b = 0.0, float(2 * np.diff(g.row_ptr).max())
    def e(j):
        c = np.zeros(j + 1)
        c[j] = 1.0
        return c
    for m, k in [(2, 3), (4, 1), (3, 3)]:
        lhs = oracle.poly_chebyshev(g, oracle.poly_chebyshev(g, V, e(k), a, b), e(m), a, b)
        rhs = 0.5 * (oracle.poly_chebyshev(g, V, e(m + k), a, b) +
                     oracle.poly_chebyshev(g, V, e(abs(m - k)), a, b))
        assert np.allclose(lhs, rhs, rtol=1e-10, atol=1e-10 * np.abs(rhs).max())


# ---- block moments of the polynomial bases (for fitting coefficients) --------------------
def test_moments_on_closed_form_eigenpairs():
    # V = eigenvectors: Omega_l = diag(lambda^l) (power) and diag(T_l(x(lambda))) (Chebyshev)
    n = 24
    g = gen.path(n)
    lam, U = _path_pairs(n)
    idx = [0, 3, 7, 20]
    V = U[:, idx]
    P = oracle.poly_moments(g, V, 6, basis="power")
    for l in range(6):
        assert np.allclose(P[l], np.diag(lam[idx] ** l), atol=1e-11 * max(1, 4.0 ** l))
    a, b = 0.1, 4.0
    C = oracle.poly_moments(g, V, 9, basis="chebyshev", a=a, b=b)
    x = (2 * lam[idx] - (a + b)) / (b - a)
    for l in range(9):
        e = np.zeros(l + 1)
        e[l] = 1.0
        assert np.allclose(C[l], np.diag(oracle.chebyshev_scalar(e, x)), atol=1e-11)


def test_moments_product_identity_and_linearity():
    # (T_l V)^T (T_m V) = (Omega_{l+m} + Omega_{|l-m|}) / 2, and sum_l c_l Omega_l = V^T M V
    g = gen.uniform_edge_weights(gen.random_graph(80, 300, seed=3), seed=4)
    V = gen.gaussian_block(g.n, 3, seed=5)
    a, b = 0.0, oracle.gershgorin_bound(g)
    C = oracle.poly_moments(g, V, 12, a=a, b=b)
    for l, m in [(0, 0), (1, 4), (5, 5), (2, 7)]:
        el, em = np.zeros(l + 1), np.zeros(m + 1)
        el[l], em[m] = 1.0, 1.0
        TlV = oracle.poly_chebyshev(g, V, el, a, b)
        TmV = oracle.poly_chebyshev(g, V, em, a, b)
        assert np.allclose(TlV.T @ TmV, 0.5 * (C[l + m] + C[abs(l - m)]), rtol=1e-10,
                           atol=1e-10)
    c = np.random.default_rng(6).standard_normal(8)
    assert np.allclose(np.tensordot(c, C[:8], axes=1), V.T @ oracle.poly_chebyshev(g, V, c, a, b),
                       rtol=1e-10, atol=1e-10)
    P = oracle.poly_moments(g, V, 5, basis="power")
    assert np.allclose(P[3], V.T @ oracle.walk_exact_terms(g, V, [0, 0, 0, 1.0]), rtol=1e-12)
