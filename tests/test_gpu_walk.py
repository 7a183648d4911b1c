"""Parity of the stochastic p(L) V estimator (Section 4.3) with the oracle: the same Philox
draws give the same walks, so the two agree sample by sample; and its mean converges to the
exact polynomial."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2207_14589_gb300 as sped
from util_gpu import assert_close, DEV, host, rel, to_block

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("mode", [sped.STOCHASTIC_IS, sped.STOCHASTIC_REJECT])
@pytest.mark.parametrize("gname", ["rand", "rand_w", "star"])
@pytest.mark.parametrize("ell,k", [(1, 3), (3, 5), (7, 20)])
def test_walk_same_draws_as_oracle(mode, gname, ell, k):
    if gname == "rand":
        g = gen.random_graph(300, 900, seed=4, isolated=3)
    elif gname == "rand_w":
        g = gen.uniform_edge_weights(gen.random_graph(250, 800, seed=5, hub=1, hub_degree=60),
                                     seed=6)
    else:
        g = gen.star(40)
    G = sped.Graph.from_csr(g)
    G.set_polynomial(sped.POLY_LIMIT_EXP, ell, scale=0.01)
    c = np.array(G.power_coeffs())
    assert np.allclose(c, oracle.limit_power_coeffs(0.01, ell), rtol=1e-14)
    V0 = gen.gaussian_block(g.n, k, seed=7)
    V = to_block(V0, torch.float64)
    Y = sped.alloc_block(g.n, k, torch.float64, DEV)
    walkers, seed = 20000, 123456789
    sped.apply_poly(G, V, Y, k, mode=mode, walkers=walkers, seed=seed)
    torch.cuda.synchronize()
    want = oracle.walk_estimate(g, V0, c, walkers, seed, mode=mode)
    # identical walks; only the order of the final atomic additions differs
    assert_close(host(Y, k), want, 1e-11)


@pytest.mark.parametrize("mode", [sped.STOCHASTIC_IS, sped.STOCHASTIC_REJECT])
@pytest.mark.parametrize("ell,k", [(3, 5), (7, 20), (5, 13)])
def test_walk_fp32_same_draws_as_oracle(mode, ell, k):
    # F32 blocks: the walk's draws and weights stay FP64 (same decisions as the oracle); the
    # per-walker sums are F32, so agreement is to F32 rounding of each term
    g = gen.uniform_edge_weights(gen.random_graph(250, 800, seed=5, hub=1, hub_degree=60), seed=6)
    G = sped.Graph.from_csr(g)
    G.set_polynomial(sped.POLY_LIMIT_EXP, ell, scale=0.01)
    c = np.array(G.power_coeffs())
    V0 = gen.gaussian_block(g.n, k, seed=8)
    V = to_block(V0, torch.float32)
    Y = sped.alloc_block(g.n, k, torch.float32, DEV)
    walkers, seed = 20000, 987654321
    sped.apply_poly(G, V, Y, k, mode=mode, walkers=walkers, seed=seed)
    torch.cuda.synchronize()
    want = oracle.walk_estimate(g, V0.astype(np.float32).astype(np.float64), c, walkers, seed,
                                mode=mode)
    assert_close(host(Y, k), want, 2e-5)


def test_walk_fp32_output_and_mean():
    g = gen.from_edges(6, [0, 1, 2, 3, 0, 1], [1, 2, 3, 4, 2, 5])
    G = sped.Graph.from_csr(g)
    G.set_polynomial(sped.POLY_LIMIT_EXP, 3, scale=0.15)
    c = np.array(G.power_coeffs())
    k = 2
    V0 = gen.gaussian_block(g.n, k, seed=5)
    V = to_block(V0, torch.float32)
    Y = sped.alloc_block(g.n, k, torch.float32, DEV)
    exact = oracle.walk_exact_terms(g, V0.astype(np.float32).astype(np.float64), c)
    ests = []
    for b in range(16):
        sped.apply_poly(G, V, Y, k, mode=sped.STOCHASTIC_IS, walkers=200000, seed=1000 + b)
        torch.cuda.synchronize()
        ests.append(host(Y, k))
    ests = np.stack(ests)
    mean = ests.mean(0)
    se = ests.std(0, ddof=1) / np.sqrt(len(ests))
    assert np.all(np.abs(mean - exact) <= 5 * se + 1e-5)


def test_single_edge_walk_exact_on_gpu():
    g = gen.uniform_edge_weights(gen.from_edges(3, [0], [2]), seed=1)
    G = sped.Graph.from_csr(g)
    G.set_polynomial(sped.POLY_MONOMIAL, 4, coeffs=[0.3, -1.0, 0.5, -0.25, 0.125])
    k = 4
    V0 = np.random.default_rng(0).standard_normal((3, k))
    V = to_block(V0, torch.float64)
    Y = sped.alloc_block(3, k, torch.float64, DEV)
    for mode in (sped.STOCHASTIC_IS, sped.STOCHASTIC_REJECT):
        sped.apply_poly(G, V, Y, k, mode=mode, walkers=7, seed=3)
        torch.cuda.synchronize()
        want = oracle.walk_exact_terms(g, V0, np.array([0.3, -1.0, 0.5, -0.25, 0.125]))
        assert_close(host(Y, k), want, 1e-12)


@pytest.mark.parametrize("mode", [sped.STOCHASTIC_IS, sped.STOCHASTIC_REJECT])
@pytest.mark.parametrize("vt,yt,k,tol", [(torch.float64, torch.float64, 16, 1e-11),
                                         (torch.float32, torch.float64, 20, 1e-11),
                                         (torch.float32, torch.float64, 32, 1e-11)])
def test_walk_several_walkers_per_thread(mode, vt, yt, k, tol):
    # more walkers than one wave of resident threads (at most 152 SMs x 7 blocks x 128), so every
    # thread takes several walkers through the grid-stride loop; still walk for walk the oracle's.
    # FP64 outputs, whose per-walker sums and atomics are FP64: with F32 outputs each row here
    # takes about 2,400 F32 atomic adds in arbitrary order, a rounding of order 1e-4 per entry
    # (the F32 tests above bound it at their 20,000 walkers)
    g = gen.uniform_edge_weights(gen.random_graph(250, 800, seed=5, hub=1, hub_degree=60), seed=6)
    G = sped.Graph.from_csr(g)
    G.set_polynomial(sped.POLY_LIMIT_EXP, 5, scale=0.01)
    c = np.array(G.power_coeffs())
    V0 = gen.gaussian_block(g.n, k, seed=9)
    V = to_block(V0, vt)
    Y = sped.alloc_block(g.n, k, yt, DEV)
    walkers, seed = 300_001, 24681357
    sped.apply_poly(G, V, Y, k, mode=mode, walkers=walkers, seed=seed)
    torch.cuda.synchronize()
    Vs = torch.from_numpy(V0).to(vt).double().numpy()
    want = oracle.walk_estimate(g, Vs, c, walkers, seed, mode=mode)
    assert_close(host(Y, k), want, tol)
