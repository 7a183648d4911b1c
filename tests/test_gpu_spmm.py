"""Parity of the fused chain step Y = alpha V + gamma X + beta L X (Section 2) and of p(L) V
(Table 2) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2207_14589_gb300 as sped
from util_gpu import assert_close, DEV, TOL, host, rel, stored, to_block

pytestmark = pytest.mark.gpu

GRAPHS = {
    # ragged rows, empty rows (isolated nodes) and a long hub row
    "ragged": lambda: gen.random_graph(3001, 12000, seed=1, hub=7, hub_degree=900, isolated=40),
    "ragged_w": lambda: gen.uniform_edge_weights(
        gen.random_graph(2503, 9000, seed=2, hub=0, hub_degree=600, isolated=17), seed=3),
    "sbm": lambda: gen.sbm(4000, 4, 0.01, 0.0005, seed=4),
    "powerlaw_w": lambda: gen.chung_lu_clusters(6000, n_clusters=8, d_max=2000, seed=5),
}

PAIRS = [(torch.float64, torch.float64), (torch.float32, torch.float32),
         (torch.bfloat16, torch.bfloat16), (torch.float32, torch.bfloat16),
         (torch.bfloat16, torch.float32), (torch.float32, torch.float64)]


@pytest.mark.parametrize("gname", list(GRAPHS))
@pytest.mark.parametrize("xt,yt", PAIRS)
@pytest.mark.parametrize("k", [3, 8, 20])
@pytest.mark.parametrize("split", [1, 2])
def test_laplacian_step(gname, xt, yt, k, split):
    g = GRAPHS[gname]()
    G = sped.Graph.from_csr(g)
    X0 = gen.gaussian_block(g.n, k, seed=k)
    X = to_block(X0, xt)
    Y = sped.alloc_block(g.n, k, yt, DEV, fill=float("nan"))
    a, b, c = 0.0, -0.03, 1.0
    sped.poly_step(G, X, Y, k, alpha=a, beta=b, gamma=c, split=split)
    torch.cuda.synchronize()
    Xs = stored(X0, xt)
    want = c * Xs + b * oracle.laplacian_apply(g, Xs)
    # the output storage decides the bound: inputs are compared as stored, F64 output means
    # F64 accumulation, otherwise F32 accumulation and rounding to the output type
    assert_close(host(Y, k), want, TOL[yt])
    # padding columns were never written
    if Y.shape[1] > k:
        assert torch.isnan(Y[:, k:]).all()


@pytest.mark.parametrize("split", [1, 2])
def test_step_with_v_term(split):
    g = GRAPHS["ragged_w"]()
    G = sped.Graph.from_csr(g)
    k = 6
    X0, V0 = gen.gaussian_block(g.n, k, seed=1), gen.gaussian_block(g.n, k, seed=2)
    X, V = to_block(X0, torch.float64), to_block(V0, torch.float64)
    Y = sped.alloc_block(g.n, k, torch.float64, DEV)
    sped.poly_step(G, X, Y, k, alpha=0.7, beta=1.0, gamma=-0.2, V=V, split=split)
    torch.cuda.synchronize()
    want = 0.7 * V0 - 0.2 * X0 + oracle.laplacian_apply(g, X0)
    assert_close(host(Y, k), want, 1e-12)


def test_merge_equals_rowgroup_fp64():
    g = GRAPHS["powerlaw_w"]()
    G = sped.Graph.from_csr(g)
    k = 5
    X = to_block(gen.gaussian_block(g.n, k, seed=9), torch.float64)
    Y1 = sped.alloc_block(g.n, k, torch.float64, DEV)
    Y2 = sped.alloc_block(g.n, k, torch.float64, DEV)
    sped.poly_step(G, X, Y1, k, split=1)
    sped.poly_step(G, X, Y2, k, split=2)
    torch.cuda.synchronize()
    assert_close(host(Y2, k), host(Y1, k), 1e-14)


@pytest.mark.parametrize("ell", [1, 3, 9, 41])
@pytest.mark.parametrize("chain,yt,tol", [(torch.float64, torch.float64, 1e-12),
                                          (torch.float32, torch.float32, 1e-5),
                                          (torch.bfloat16, torch.float32, 1e-2)])
def test_apply_poly_limit(ell, chain, yt, tol):
    g = gen.sbm(3000, 3, 0.012, 0.0008, seed=7)
    G = sped.Graph.from_csr(g)
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
    k = 4
    vt = torch.float64 if chain == torch.float64 else torch.float32
    V0 = gen.gaussian_block(g.n, k, seed=8)
    V = to_block(V0, vt)
    Y = sped.alloc_block(g.n, k, yt, DEV)
    sped.apply_poly(G, V, Y, k, chain_dtype=chain)
    torch.cuda.synchronize()
    want = oracle.poly_limit(g, stored(V0, vt), info.scale_s, ell)
    assert_close(host(Y, k), want, tol)


@pytest.mark.parametrize("chain", [torch.float64, torch.bfloat16])
def test_apply_poly_two_step_chain(chain):
    # degree 2: one intermediate buffer (the other chain lengths use two, or none)
    g = gen.sbm(2500, 5, 0.01, 0.001, seed=3)
    G = sped.Graph.from_csr(g)
    coeffs = [0.25, -0.05, 0.001]
    G.set_polynomial(sped.POLY_MONOMIAL, 2, coeffs=coeffs)
    k = 9
    vt = torch.float64 if chain == torch.float64 else torch.float32
    V0 = gen.gaussian_block(g.n, k, seed=1)
    V = to_block(V0, vt)
    Y = sped.alloc_block(g.n, k, vt, DEV)
    sped.apply_poly(G, V, Y, k, chain_dtype=chain)
    torch.cuda.synchronize()
    want = oracle.poly_horner(g, stored(V0, vt), np.array(coeffs))
    assert_close(host(Y, k), want, (1e-12 if chain == torch.float64 else 1e-2))


def test_apply_poly_scale_rule_and_oddness():
    g = gen.sbm(500, 2, 0.1, 0.01, seed=3)
    G = sped.Graph.from_csr(g)
    lb = G.info().lambda_bound
    assert lb == pytest.approx(oracle.gershgorin_bound(g))
    assert G.set_polynomial(sped.POLY_LIMIT_EXP, 251).scale_s == pytest.approx(
        oracle.scale_rule(lb, 251))
    assert G.set_polynomial(sped.POLY_LIMIT_EXP, 5).scale_s == pytest.approx(
        oracle.scale_rule(lb, 5))
    with pytest.raises(sped.SpedError):
        G.set_polynomial(sped.POLY_LIMIT_EXP, 10)  # even degree is not monotone


def test_apply_poly_horner_taylor_exp_and_shift():
    g = gen.uniform_edge_weights(gen.random_graph(1500, 4000, seed=5), lo=0.05, hi=0.2, seed=6)
    G = sped.Graph.from_csr(g)
    k = 3
    V0 = gen.gaussian_block(g.n, k, seed=2)
    V = to_block(V0, torch.float64)
    Y = sped.alloc_block(g.n, k, torch.float64, DEV)
    G.set_polynomial(sped.POLY_TAYLOR_EXP, 12)
    sped.apply_poly(G, V, Y, k)
    torch.cuda.synchronize()
    assert_close(host(Y, k), oracle.poly_horner(g, V0, oracle.taylor_exp_coeffs(12)), 1e-12)
    info = G.set_polynomial(sped.POLY_SHIFT, 1)
    sped.apply_poly(G, V, Y, k)
    torch.cuda.synchronize()
    want = info.lambda_star * V0 - oracle.laplacian_apply(g, V0)
    assert_close(host(Y, k), want, 1e-12)
    coeffs = [0.5, -0.25, 0.125, 0.3]
    G.set_polynomial(sped.POLY_MONOMIAL, 3, coeffs=coeffs)
    sped.apply_poly(G, V, Y, k)
    torch.cuda.synchronize()
    assert_close(host(Y, k), oracle.poly_horner(g, V0, np.array(coeffs)), 1e-12)


def test_apply_poly_taylor_log_small_radius():
    base = gen.path(400)
    g = gen.CSRGraph(base.n, base.row_ptr, base.col_idx,
                     np.full(base.nnz, 0.45, dtype=np.float32))
    G = sped.Graph.from_csr(g)
    info = G.set_polynomial(sped.POLY_TAYLOR_LOG, 60, eps=1e-3)
    k = 2
    V0 = gen.gaussian_block(g.n, k, seed=4)
    V = to_block(V0, torch.float64)
    Y = sped.alloc_block(g.n, k, torch.float64, DEV)
    sped.apply_poly(G, V, Y, k)
    torch.cuda.synchronize()
    c = -oracle.taylor_log_coeffs(60)
    c[0] += info.lambda_star
    assert_close(host(Y, k), oracle.poly_horner(g, V0, c, shift=1e-3 - 1.0), 1e-12)


def test_ones_fixed_by_limit_form():
    # L 1 = 0 (Section 2), so (I - sL)^l 1 = 1 at any size
    g = gen.chung_lu_clusters(20000, n_clusters=16, d_max=3000, seed=9)
    G = sped.Graph.from_csr(g)
    G.set_polynomial(sped.POLY_LIMIT_EXP, 21)
    k = 2
    V = to_block(np.ones((g.n, k)), torch.float32)
    Y = sped.alloc_block(g.n, k, torch.float32, DEV)
    sped.apply_poly(G, V, Y, k, chain_dtype=torch.float32)
    torch.cuda.synchronize()
    assert np.abs(host(Y, k) - 1.0).max() < 1e-4


def test_invalid_csr_rejected():
    g = gen.random_graph(200, 600, seed=1)
    rp = torch.from_numpy(g.row_ptr).to(DEV)
    ci = torch.from_numpy(g.col_idx.copy()).to(DEV)
    bad = ci.clone()
    bad[5] = g.n + 3  # column out of range
    with pytest.raises(sped.SpedError) as e:
        sped.Graph(rp, bad)
    assert e.value.status == sped.ERR_BAD_CSR
    asym = gen.from_edges(10, [0, 1], [1, 2])
    ci2 = torch.from_numpy(asym.col_idx.copy()).to(DEV)
    ci2[-1] = 3  # breaks symmetry, stays sorted and in range
    with pytest.raises(sped.SpedError):
        sped.Graph(torch.from_numpy(asym.row_ptr).to(DEV), ci2)
    rp_bad = rp.clone()
    rp_bad[10] = rp_bad[11] + 5  # not monotone
    with pytest.raises(sped.SpedError):
        sped.Graph(rp_bad, ci)


@pytest.mark.parametrize("ell", [1, 2, 3, 4, 9, 24])
@pytest.mark.parametrize("ct,tol", [(torch.float64, 1e-12), (torch.float32, 1e-5)])
@pytest.mark.parametrize("gname", ["ragged_w", "sbm"])
def test_chebyshev_series_matches_oracle(ell, ct, tol, gname):
    # Clenshaw chain (three buffers, the step before last added back) against the oracle's
    # three-term recurrence; the interval covers only part of the spectrum, so the cosh
    # branch of T_j occurs too
    g = GRAPHS[gname]()
    G = sped.Graph.from_csr(g)
    lam_b = G.info().lambda_bound
    c = np.random.default_rng(ell).standard_normal(ell + 1) / (1.0 + np.arange(ell + 1)) ** 2
    a, b = 0.05 * lam_b, 0.6 * lam_b
    G.set_polynomial(sped.POLY_CHEBYSHEV, ell, eps=a, coeffs=c, lambda_star=b)
    k = 5
    V0 = gen.gaussian_block(g.n, k, seed=ell + 40)
    V = to_block(V0, torch.float64 if ct == torch.float64 else torch.float32)
    Y = sped.alloc_block(g.n, k, torch.float64, DEV)
    sped.apply_poly(G, V, Y, k, chain_dtype=ct)
    torch.cuda.synchronize()
    Vs = stored(V0, V.dtype)
    want = oracle.poly_chebyshev(g, Vs, c, a, b)
    assert_close(host(Y, k), want, tol)


def test_chebyshev_power_coefficients():
    g = GRAPHS["sbm"]()
    G = sped.Graph.from_csr(g)
    c = np.array([0.5, -0.25, 0.125, 0.7, -0.3])
    a, b = 1.0, 9.0
    G.set_polynomial(sped.POLY_CHEBYSHEV, 4, eps=a, coeffs=c, lambda_star=b)
    # sum_j c_j T_j(al x + be) in powers of x, by evaluating at 5 points and solving
    xs = np.linspace(0.0, 10.0, 5)
    vals = oracle.chebyshev_scalar(c, (2.0 * xs - (a + b)) / (b - a))
    want = np.linalg.solve(np.vander(xs, 5, increasing=True), vals)
    assert np.allclose(G.power_coeffs(), want, rtol=1e-9, atol=1e-12)


def test_chebyshev_rejects_empty_interval():
    G = sped.Graph.from_csr(GRAPHS["sbm"]())
    with pytest.raises(sped.SpedError):
        G.set_polynomial(sped.POLY_CHEBYSHEV, 3, eps=5.0, coeffs=[1.0, 0.0, 0.0, 1.0],
                         lambda_star=2.0)
