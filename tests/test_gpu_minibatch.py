"""GPU parity of the edge-minibatch path (the stochastic optimisation model of Sections 2 and 6:
the solver sees edges in minibatches; L = sum_e w_e x_e x_e^T, Section 4.3) against the FP64
oracle on the same Philox draws: the sampled edges bit for bit, one step on caller edges, the
chains of every polynomial family, a solver step, and the estimator's mean."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2207_14589_gb300 as sped
from util_gpu import assert_close, DEV, TOL, host, rel, stored, to_block

pytestmark = pytest.mark.gpu


def _weighted():
    return gen.uniform_edge_weights(gen.random_graph(700, 2600, seed=31, hub=2, hub_degree=150,
                                                     isolated=5), seed=32)


@pytest.mark.parametrize("count", [1, 1000, 4097])
@pytest.mark.parametrize("step", [0, 7])
def test_sampled_edges_match_oracle(count, step):
    g = _weighted()
    G = sped.Graph.from_csr(g)
    a, b, w = sped.sample_edges(G, seed=2718281828, step=step, count=count)
    torch.cuda.synchronize()
    oa, ob, ow = oracle.minibatch_edges(g, 2718281828, step, count)
    assert np.array_equal(a.cpu().numpy(), oa)
    assert np.array_equal(b.cpu().numpy(), ob)
    assert np.array_equal(w.cpu().numpy().astype(np.float64), ow)


def test_sampled_edges_unweighted_and_empty():
    g = gen.random_graph(200, 500, seed=33)
    G = sped.Graph.from_csr(g)
    a, b, w = sped.sample_edges(G, 5, 1, 300)
    oa, ob, _ = oracle.minibatch_edges(g, 5, 1, 300)
    assert np.array_equal(a.cpu().numpy(), oa) and np.array_equal(b.cpu().numpy(), ob)
    assert torch.all(w == 1.0)
    a, b, w = sped.sample_edges(G, 5, 1, 0)
    assert a.numel() == 0


@pytest.mark.parametrize("xt,yt", [(torch.float64, torch.float64), (torch.float32, torch.float32),
                                   (torch.float32, torch.float64), (torch.float64, torch.float32)])
@pytest.mark.parametrize("k", [1, 3, 5, 8, 20, 33, 130])
def test_edge_step_on_caller_edges(xt, yt, k):
    # arbitrary caller edges: duplicates, both orientations, self loops, four out of range
    n, B = 500, 3001
    rng = np.random.default_rng(k)
    a = rng.integers(0, n, B).astype(np.int32)
    b = rng.integers(0, n, B).astype(np.int32)
    b[:40] = a[:40]
    bad = np.array([5, 17, 2000, 3000])
    a[bad[:2]] = n
    b[bad[2:]] = -1
    w = rng.uniform(0.1, 2.0, B).astype(np.float32)
    X0 = gen.gaussian_block(n, k, seed=34)
    V0 = gen.gaussian_block(n, k, seed=35)
    X, V = to_block(X0, xt), to_block(V0, torch.float64 if yt == torch.float64 else torch.float32)
    Y = sped.alloc_block(n, k, yt, DEV, fill=float("nan"))
    skipped = torch.zeros(1, dtype=torch.int32, device=DEV)
    da, db, dw = (torch.from_numpy(x).to(DEV) for x in (a, b, w))
    scale, al, be, ga = 0.37, 0.5, -0.8, 1.25
    sped.edge_step(n, X, Y, k, da, db, dw, edge_scale=scale, alpha=al, beta=be, gamma=ga, V=V,
                   skipped=skipped)
    torch.cuda.synchronize()
    assert int(skipped.item()) == 4
    keep = np.ones(B, bool)
    keep[bad] = False
    Xs, Vs = stored(X0, xt), stored(V0, V.dtype)
    # minibatch_laplacian_apply scales by n_edges / B: pass n_edges = scale * B
    LX = oracle.minibatch_laplacian_apply(scale * keep.sum(), Xs, a[keep], b[keep],
                                          w[keep].astype(np.float64))
    want = al * Vs + ga * Xs + be * LX
    tol = TOL[torch.float64] if (xt, yt) == (torch.float64, torch.float64) else 4 * TOL[torch.float32]
    assert_close(host(Y, k), want, tol)
    assert torch.isnan(Y[:, k:]).all()  # row padding untouched


def _family(G, g, fam, ell):
    """Set the graph's polynomial; return the oracle's chain with the same coefficients."""
    if fam == "limit":
        info = G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
        return lambda V, op: oracle.stochastic_limit(V, info.scale_s, ell, op)
    if fam == "taylor_exp":
        G.set_polynomial(sped.POLY_TAYLOR_EXP, ell)
        return lambda V, op: oracle.stochastic_horner(V, oracle.taylor_exp_coeffs(ell), 0.0, op)
    if fam == "taylor_log":
        info = G.set_polynomial(sped.POLY_TAYLOR_LOG, ell, eps=0.01)
        h = -oracle.taylor_log_coeffs(ell)
        h[0] = info.lambda_star
        return lambda V, op: oracle.stochastic_horner(V, h, 0.01 - 1.0, op)
    if fam == "monomial":
        c = np.array([0.5, -0.3, 0.02, 0.001, -0.0002][:ell + 1])
        G.set_polynomial(sped.POLY_MONOMIAL, ell, coeffs=c)
        return lambda V, op: oracle.stochastic_horner(V, c, 0.0, op)
    if fam == "shift":
        info = G.set_polynomial(sped.POLY_SHIFT, 1)
        return lambda V, op: oracle.stochastic_horner(V, [info.lambda_star, -1.0], 0.0, op)
    c = np.linspace(1.0, -0.5, ell + 1)
    hi = oracle.gershgorin_bound(g)
    G.set_polynomial(sped.POLY_CHEBYSHEV, ell, eps=0.05, coeffs=c, lambda_star=hi)
    return lambda V, op: oracle.stochastic_clenshaw(V, c, 0.05, hi, op)


@pytest.mark.parametrize("fam,ell", [("limit", 1), ("limit", 3), ("limit", 9),
                                     ("taylor_exp", 4), ("taylor_log", 3), ("monomial", 4),
                                     ("shift", 1), ("chebyshev", 1), ("chebyshev", 2),
                                     ("chebyshev", 5)])
@pytest.mark.parametrize("ct", [torch.float64, torch.float32])
@pytest.mark.parametrize("B", [1, 97, 5000])
def test_chain_same_draws_as_oracle(fam, ell, ct, B):
    g = _weighted()
    G = sped.Graph.from_csr(g)
    chain = _family(G, g, fam, ell)
    k = 6
    V0 = gen.gaussian_block(g.n, k, seed=36)
    V = to_block(V0, ct)
    Y = sped.alloc_block(g.n, k, ct, DEV)
    seed = 1234567 + B
    sped.apply_poly(G, V, Y, k, chain_dtype=ct, mode=sped.STOCHASTIC_MINIBATCH, walkers=B,
                    seed=seed)
    torch.cuda.synchronize()
    want = chain(stored(V0, ct), oracle.minibatch_operator(g, seed, B))
    # the same draws; only the order of the atomic additions (and F32 rounding) differs
    tol = 1e-11 if ct == torch.float64 else 2e-5 * max(1, ell)
    assert_close(host(Y, k), want, tol)


def test_minibatch_mean_converges_to_the_exact_operator():
    # unbiasedness on the device: the mean over independent seeds of (I - sL_hat)...(I - sL_hat) V
    # lies within a few standard errors of (I - sL)^l V
    g = gen.sbm(600, 3, 0.05, 0.004, seed=37)
    G = sped.Graph.from_csr(g)
    ell, k, R = 5, 2, 400
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
    V0 = gen.gaussian_block(g.n, k, seed=38)
    V = to_block(V0, torch.float64)
    Y = sped.alloc_block(g.n, k, torch.float64, DEV)
    outs = []
    for r in range(R):
        sped.apply_poly(G, V, Y, k, chain_dtype=torch.float64, mode=sped.STOCHASTIC_MINIBATCH,
                        walkers=2000, seed=r)
        outs.append(host(Y, k))
    outs = np.stack(outs)
    mean, se = outs.mean(0), outs.std(0, ddof=1) / np.sqrt(R)
    z = (mean - oracle.poly_limit(g, V0, info.scale_s, ell)) / np.maximum(se, 1e-300)
    assert float(np.mean(z ** 2)) < 1.3
    assert float(np.abs(z).max()) < 6.0


def test_graph_without_edges_gives_the_exact_result():
    g = gen.from_edges(40, np.array([], dtype=np.int64), np.array([], dtype=np.int64))
    G = sped.Graph.from_csr(g)
    G.set_polynomial(sped.POLY_SHIFT, 1, lambda_star=2.5)
    V0 = gen.gaussian_block(g.n, 3, seed=39)
    V = to_block(V0, torch.float64)
    Y = sped.alloc_block(g.n, 3, torch.float64, DEV)
    sped.apply_poly(G, V, Y, 3, chain_dtype=torch.float64, mode=sped.STOCHASTIC_MINIBATCH,
                    walkers=10, seed=1)
    torch.cuda.synchronize()
    assert np.array_equal(host(Y, 3), 2.5 * V0)


def test_eig_step_on_a_minibatch_estimate():
    g = gen.sbm(1500, 3, 0.02, 0.001, seed=40)
    G = sped.Graph.from_csr(g)
    ell, k, B, seed = 9, 5, 4000, 99
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
    V0 = gen.gaussian_block(g.n, k, seed=41)
    V0 /= np.linalg.norm(V0, axis=0)
    V = to_block(V0, torch.float64)
    opts = sped.step_opts(sped.MU_EG, 0.5, torch.float64, torch.float64,
                          mode=sped.STOCHASTIC_MINIBATCH, walkers=B, seed=seed)
    stats = torch.zeros(3 * k, dtype=torch.float64, device=DEV)
    sped.eig_step(G, V, k, opts, stats=stats)
    torch.cuda.synchronize()
    Y0 = oracle.stochastic_limit(V0, info.scale_s, ell, oracle.minibatch_operator(g, seed, B))
    assert np.abs(host(V, k) - oracle.mu_eg_step(V0, Y0, 0.5)).max() <= 1e-10
    assert np.allclose(stats.cpu().numpy()[:k], oracle.ritz_values(V0, Y0), rtol=1e-11)


def test_minibatch_rejects_what_it_cannot_do():
    g = gen.random_graph(100, 300, seed=42)
    G = sped.Graph.from_csr(g)
    G.set_polynomial(sped.POLY_LIMIT_EXP, 3)
    V = to_block(gen.gaussian_block(g.n, 4, seed=43), torch.float32)
    Y = sped.alloc_block(g.n, 4, torch.float32, DEV)
    with pytest.raises(sped.SpedError):  # BF16 chain: atomic accumulation needs F32 or F64
        sped.apply_poly(G, V, Y, 4, chain_dtype=torch.bfloat16,
                        mode=sped.STOCHASTIC_MINIBATCH, walkers=10)
    with pytest.raises(sped.SpedError):  # an empty minibatch estimates nothing
        sped.apply_poly(G, V, Y, 4, chain_dtype=torch.float32,
                        mode=sped.STOCHASTIC_MINIBATCH, walkers=0)
    with pytest.raises(sped.SpedError):
        sped.edge_step(g.n, V, V, 4, torch.zeros(1, dtype=torch.int32, device=DEV),
                       torch.zeros(1, dtype=torch.int32, device=DEV))


# ---- stratified minibatches ------------------------------------------------------------
@pytest.mark.parametrize("count", [1, 1000, 4097, 20000])
def test_stratified_edges_match_oracle(count):
    g = _weighted()
    G = sped.Graph.from_csr(g)
    a, b, w, size = sped.sample_edges(G, seed=77, step=3, count=count, stratified=True)
    torch.cuda.synchronize()
    ea, eb, ew = oracle.edge_list(g)
    ids, sizes = oracle.stratified_edge_ids(len(ea), 77, 3, count)
    assert np.array_equal(size.cpu().numpy(), sizes)
    keep = sizes > 0  # count > |E| leaves empty strata: a = b = -1, w = 0
    assert np.array_equal(a.cpu().numpy()[keep], ea[ids[keep]])
    assert np.array_equal(b.cpu().numpy()[keep], eb[ids[keep]])
    assert np.array_equal(w.cpu().numpy()[keep].astype(np.float64), ew[ids[keep]])
    assert np.all(a.cpu().numpy()[~keep] == -1) and np.all(w.cpu().numpy()[~keep] == 0)


@pytest.mark.parametrize("fam,ell", [("limit", 3), ("limit", 9), ("taylor_exp", 4),
                                     ("chebyshev", 5)])
@pytest.mark.parametrize("ct", [torch.float64, torch.float32])
@pytest.mark.parametrize("B", [1, 97, 5000])
def test_stratified_chain_same_draws_as_oracle(fam, ell, ct, B):
    g = _weighted()
    G = sped.Graph.from_csr(g)
    chain = _family(G, g, fam, ell)
    k = 6
    V0 = gen.gaussian_block(g.n, k, seed=46)
    V = to_block(V0, ct)
    Y = sped.alloc_block(g.n, k, ct, DEV)
    seed = 7654321 + B
    sped.apply_poly(G, V, Y, k, chain_dtype=ct, mode=sped.STOCHASTIC_MINIBATCH_STRATIFIED,
                    walkers=B, seed=seed)
    torch.cuda.synchronize()
    want = chain(stored(V0, ct), oracle.minibatch_operator(g, seed, B, stratified=True))
    tol = 1e-11 if ct == torch.float64 else 2e-5 * max(1, ell)
    assert_close(host(Y, k), want, tol)


def test_stratified_with_one_edge_per_stratum_is_exact():
    g = _weighted()
    G = sped.Graph.from_csr(g)
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, 5)
    k = 4
    V0 = gen.gaussian_block(g.n, k, seed=47)
    V = to_block(V0, torch.float64)
    Y = sped.alloc_block(g.n, k, torch.float64, DEV)
    for B in (info.n_edges, info.n_edges + 31):
        sped.apply_poly(G, V, Y, k, chain_dtype=torch.float64,
                        mode=sped.STOCHASTIC_MINIBATCH_STRATIFIED, walkers=B, seed=5)
        torch.cuda.synchronize()
        assert_close(host(Y, k), oracle.poly_limit(g, V0, info.scale_s, 5), 1e-12)


def test_stratified_mean_converges_and_beats_uniform():
    g = gen.sbm(600, 3, 0.05, 0.004, seed=37)
    G = sped.Graph.from_csr(g)
    ell, k, R = 5, 2, 300
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
    V0 = gen.gaussian_block(g.n, k, seed=38)
    V = to_block(V0, torch.float64)
    Y = sped.alloc_block(g.n, k, torch.float64, DEV)
    exact = oracle.poly_limit(g, V0, info.scale_s, ell)
    spread = {}
    for mode in (sped.STOCHASTIC_MINIBATCH, sped.STOCHASTIC_MINIBATCH_STRATIFIED):
        outs = []
        for r in range(R):
            sped.apply_poly(G, V, Y, k, chain_dtype=torch.float64, mode=mode, walkers=2000,
                            seed=r)
            outs.append(host(Y, k))
        outs = np.stack(outs)
        mean, se = outs.mean(0), outs.std(0, ddof=1) / np.sqrt(R)
        z = (mean - exact) / np.maximum(se, 1e-300)
        assert float(np.mean(z ** 2)) < 1.4
        assert float(np.abs(z).max()) < 6.0
        spread[mode] = float(np.mean(np.linalg.norm(outs - exact, axis=(1, 2))))
    assert spread[sped.STOCHASTIC_MINIBATCH_STRATIFIED] < spread[sped.STOCHASTIC_MINIBATCH]


@pytest.mark.parametrize("mode", [sped.STOCHASTIC_MINIBATCH, sped.STOCHASTIC_MINIBATCH_STRATIFIED])
def test_solve_on_minibatches_reaches_the_noise_floor(mode):
    # mu-EG with every step's p(L) V estimated from edge minibatches (fresh draws each step):
    # a fixed step size stops at a noise floor set by the minibatch variance; the subspace gets
    # there from a random start
    g = gen.sbm(2000, 4, 0.05, 0.001, seed=gen.DEFAULT_SEED)
    G = sped.Graph.from_csr(g)
    k = 4
    G.set_polynomial(sped.POLY_LIMIT_EXP, 7)
    _, Ustar = oracle.bottom_k(g, k)
    V0 = gen.gaussian_block(g.n, k, seed=87)
    start = oracle.principal_angle_max(Ustar, V0)
    V = to_block(V0, torch.float64)
    opts = sped.solve_opts(sped.MU_EG, 0.5, torch.float64, torch.float64, max_steps=80,
                           check_every=10, tol=1e-12, refine_dtype=torch.float64, mode=mode,
                           walkers=g.nnz // 8, seed=3)
    _, rep = sped.solve_bottom_k(G, V, k, opts)
    assert rep["steps"] == 80 and not rep["converged"]  # the residual never reaches 1e-12
    ang = oracle.principal_angle_max(Ustar, host(V, k))
    assert start > 1.0 and ang < 0.15, (start, ang)
