"""Sizes past 32-bit element offsets: a cycle of N = 2^27 + 12,345 nodes, so that every block of
k = 20 columns holds more than 2^31 elements (and more than 4 GB of F32). Inputs are dyadic
values with at most 8 significant bits (gen.hash_block), exact in BF16, so the chain step and
the Gram of structured blocks are checked for exact results; the solver step is checked on
exact eigenvectors of the cycle (Section 2: L = D - A), which mu-EG leaves in place."""
import math

import numpy as np
import pytest
import torch

import gen
import paper_2207_14589_gb300 as sped
from util_gpu import DEV

pytestmark = pytest.mark.gpu

N = (1 << 27) + 12_345
K = 20
CHUNK = 1 << 24


@pytest.fixture(scope="module")
def cycle():
    g = gen.cycle_csr(N)
    return g, sped.Graph.from_csr(g)


def _fill_hash(T, k):
    for r0 in range(0, N, CHUNK):
        rows = torch.arange(r0, min(N, r0 + CHUNK), device=DEV)
        T[r0:r0 + len(rows), :k] = gen.hash_block(rows, k, xp=torch).to(T.dtype)


def test_chain_step_past_32_bit_offsets(cycle):
    g, G = cycle
    assert N * sped.padded_ld(K, torch.bfloat16) > 2 ** 31
    X = sped.alloc_block(N, K, torch.bfloat16, DEV)
    _fill_hash(X, K)
    Y = sped.alloc_block(N, K, torch.float32, DEV)
    s = 0.25
    sped.poly_step(G, X, Y, K, alpha=0.0, beta=-s, gamma=1.0)
    torch.cuda.synchronize()
    rng = np.random.default_rng(1)
    rows = np.unique(np.concatenate([[0, 1, N - 2, N - 1, (1 << 27) - 1, 1 << 27, (1 << 27) + 1],
                                     rng.integers(0, N, 2000)]))
    x = lambda r: gen.hash_block(np.asarray(r) % N, K)
    want = x(rows) - s * (2 * x(rows) - x(rows - 1) - x(rows + 1))
    got = Y[torch.from_numpy(rows).to(DEV), :K].double().cpu().numpy()
    assert np.array_equal(got, want)  # dyadic inputs: every operation is exact
    del X, Y
    torch.cuda.empty_cache()


def test_gram_past_32_bit_offsets():
    # columns: even c all ones, odd c alternating (-1)^r; B = A / 2. Every Gram entry is an
    # exact integer (or a quarter / half of one): N, or sum_r (-1)^r = 1 for odd N
    A = sped.alloc_block(N, K, torch.float32, DEV)
    sign = torch.ones(N, device=DEV)
    sign[1::2] = -1.0
    for c in range(K):
        A[:, c] = 1.0 if c % 2 == 0 else sign
    B = sped.alloc_block(N, K, torch.float32, DEV)
    B[:, :K] = 0.5 * A[:, :K]
    Gm = sped.gram(A, K, B, K).cpu().numpy()
    par = np.arange(2 * K) % 2
    base = np.where(par[:, None] == par[None, :], float(N), 1.0)
    scale = np.where(np.arange(2 * K) < K, 1.0, 0.5)
    assert np.array_equal(Gm, base * scale[:, None] * scale[None, :])
    del A, B
    torch.cuda.empty_cache()


def test_eig_step_keeps_exact_eigenvectors(cycle):
    # cos and sin of frequencies 1 and 2 are eigenvectors of the cycle's L (eigenvalues
    # 2 - 2 cos(2 pi j / N)) and mutually orthogonal, so the mu-EG residuals vanish and the
    # step leaves the unit columns in place
    g, G = cycle
    k = 4
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, 1, scale=0.25)
    V = sped.alloc_block(N, k, torch.float32, DEV)
    for r0 in range(0, N, CHUNK):
        r = torch.arange(r0, min(N, r0 + CHUNK), device=DEV, dtype=torch.float64)
        for j, (f, freq) in enumerate([(torch.cos, 1), (torch.sin, 1), (torch.cos, 2),
                                       (torch.sin, 2)]):
            V[r0:r0 + len(r), j] = f(2 * math.pi * freq * r / N).float()
    # unit columns (the mu-EG players are unit vectors)
    V[:, :k] /= torch.linalg.vector_norm(V[:, :k].double(), dim=0).float()
    V0 = V[:, :k].clone()
    opts = sped.step_opts(sped.MU_EG, 0.5, torch.float32, torch.float32)
    stats = torch.zeros(3 * k, dtype=torch.float64, device=DEV)
    sped.eig_step(G, V, k, opts, stats=stats)
    torch.cuda.synchronize()
    unit = V0 / torch.linalg.vector_norm(V0.double(), dim=0).float()
    err = float((V[:, :k] - unit).abs().max() / unit.abs().max())
    assert err <= 1e-5
    mu = 1.0 - info.scale_s * (2.0 - 2.0 * np.cos(2 * np.pi * np.array([1, 1, 2, 2]) / N))
    assert np.allclose(stats.cpu().numpy()[:k], mu, rtol=0, atol=1e-6)
