"""Parity at the benchmark's full size and launch configuration: the stochastic block model with
N = 1,000,000 nodes in 20 blocks, mean degree 16, k = 20, limit form of degree 41, BF16 chain with
F32 master. Sampled output rows are recomputed one by one by the oracle; whole-size results
are checked against the oracle where it finishes in tens of seconds, or against properties that
hold at any size."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2207_14589_gb300 as sped
from util_gpu import DEV, assert_close, assert_gram_close, assert_step_close, host, stored, to_block

pytestmark = pytest.mark.gpu

N, BLOCKS, K, ELL = 1_000_000, 20, 20, 41


@pytest.fixture(scope="module")
def sbm_n1e6():
    g = gen.sbm(N, BLOCKS, 14 / 49_999, 2 / 950_000, seed=gen.DEFAULT_SEED)
    G = sped.Graph.from_csr(g)
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, ELL)
    return g, G, info


def test_chain_step_sampled_rows(sbm_n1e6):
    g, G, info = sbm_n1e6
    s = info.scale_s
    X0 = gen.gaussian_block(N, K, seed=3)
    X = to_block(X0, torch.bfloat16)
    Y = sped.alloc_block(N, K, torch.float32, DEV)
    sped.poly_step(G, X, Y, K, alpha=0.0, beta=-s, gamma=1.0)
    torch.cuda.synchronize()
    Xs = stored(X0, torch.bfloat16)
    rows = np.random.default_rng(0).choice(N, size=3000, replace=False)
    got = Y[torch.from_numpy(rows).to(DEV), :K].double().cpu().numpy()
    want = np.empty((len(rows), K))
    for t, r in enumerate(rows):  # one row at a time: x_r - s (d_r x_r - sum_j x_j)
        nb = g.col_idx[g.row_ptr[r]:g.row_ptr[r + 1]]
        want[t] = Xs[r] - s * (len(nb) * Xs[r] - Xs[nb].sum(axis=0))
    assert_close(got, want, 1e-5)


def test_chain_keeps_constant_vector(sbm_n1e6):
    # L 1 = 0, so every step maps 1 to 1 exactly (BF16 storage, F32 accumulation)
    g, G, info = sbm_n1e6
    V = to_block(np.ones((N, K)), torch.float32)
    Y = sped.alloc_block(N, K, torch.float32, DEV)
    sped.apply_poly(G, V, Y, K, chain_dtype=torch.bfloat16)
    torch.cuda.synchronize()
    assert torch.all(Y[:, :K] == 1.0)


def test_tensor_gram_full_size():
    A0 = gen.gaussian_block(N, K, seed=5)
    B0 = gen.gaussian_block(N, K, seed=6) * 0.01
    A, B = to_block(A0, torch.float32), to_block(B0, torch.float32)
    Gm = sped.gram(A, K, B, K).cpu().numpy()
    M = np.concatenate([stored(A0, torch.float32), stored(B0, torch.float32)], axis=1)
    assert_gram_close(Gm, M.T @ M, 2e-6)


def test_mixed_eig_step_full_size(sbm_n1e6):
    # one benchmark step (BF16 chain, F32 master, mu-EG eta = 1) against the oracle's FP64 step
    g, G, info = sbm_n1e6
    V0 = gen.gaussian_block(N, K, seed=7)
    V0 /= np.linalg.norm(V0, axis=0)
    V = to_block(V0, torch.float32)
    opts = sped.step_opts(sped.MU_EG, 1.0, torch.bfloat16, torch.float32)
    sped.eig_step(G, V, K, opts)
    torch.cuda.synchronize()
    Vs = stored(V0, torch.float32)
    Y = oracle.poly_limit(g, Vs, info.scale_s, ELL)
    want = oracle.mu_eg_step(Vs, Y, 1.0)
    # the BF16 storage bound on p(L) V, carried through the step (gain measured on the oracle)
    assert_step_close(host(V, K), want, lambda Yp: oracle.mu_eg_step(Vs, Yp, 1.0), Y, 1e-2,
                      seed=1)


def test_minibatch_chain_full_size(sbm_n1e6):
    # the edge-minibatch chain at full size, 2^20 edges per multiplication (the benchmark's
    # minibatch), F32 chain: three factors of (I - s L_hat_t) against the oracle's draws
    g, G, _ = sbm_n1e6
    Gm = sped.Graph.from_csr(g)
    s, ell, B, seed = 1.0 / 41, 3, 1 << 20, 20220729
    Gm.set_polynomial(sped.POLY_LIMIT_EXP, ell, scale=s)
    V0 = gen.gaussian_block(N, K, seed=8)
    V = to_block(V0, torch.float32)
    Y = sped.alloc_block(N, K, torch.float32, DEV)
    sped.apply_poly(Gm, V, Y, K, chain_dtype=torch.float32, mode=sped.STOCHASTIC_MINIBATCH,
                    walkers=B, seed=seed)
    torch.cuda.synchronize()
    want = oracle.stochastic_limit(stored(V0, torch.float32), s, ell,
                                   oracle.minibatch_operator(g, seed, B))
    assert_close(host(Y, K), want, 1e-5)
