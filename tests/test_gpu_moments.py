"""Block moments V^T B_l V of the power and Chebyshev bases (the data for fitting polynomial
coefficients) against the FP64 oracle."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2207_14589_gb300 as sped
from util_gpu import DEV, host, stored, to_block

pytestmark = pytest.mark.gpu


def _graph():
    return gen.uniform_edge_weights(gen.random_graph(900, 3500, seed=51, hub=2, hub_degree=120),
                                    seed=52)


@pytest.mark.parametrize("vt", [torch.float64, torch.float32])
@pytest.mark.parametrize("k,m", [(1, 1), (4, 2), (4, 3), (13, 17), (32, 9)])
def test_chebyshev_moments_match_oracle(vt, k, m):
    g = _graph()
    G = sped.Graph.from_csr(g)
    V0 = gen.gaussian_block(g.n, k, seed=53)
    V = to_block(V0, vt)
    a = 0.05
    out = sped.poly_moments(G, V, k, m, basis="chebyshev", a=a).cpu().numpy()
    want = oracle.poly_moments(g, stored(V0, vt), m, basis="chebyshev", a=a,
                               b=oracle.gershgorin_bound(g))
    tol = 1e-10 if vt == torch.float64 else 2e-5 * max(1, m)
    scale = np.abs(want[0]).max()
    assert np.abs(out - want).max() <= tol * scale


@pytest.mark.parametrize("vt", [torch.float64, torch.float32])
def test_power_moments_match_oracle(vt):
    g = _graph()
    G = sped.Graph.from_csr(g)
    k, m = 5, 7
    V0 = gen.gaussian_block(g.n, k, seed=54)
    V = to_block(V0, vt)
    out = sped.poly_moments(G, V, k, m, basis="power").cpu().numpy()
    want = oracle.poly_moments(g, stored(V0, vt), m, basis="power")
    tol = 1e-10 if vt == torch.float64 else 2e-5 * m
    for l in range(m):  # the moments grow like lambda_max^l: compare each at its own scale
        assert np.abs(out[l] - want[l]).max() <= tol * np.abs(want[l]).max()


def test_moments_reject_what_they_cannot_do():
    g = _graph()
    G = sped.Graph.from_csr(g)
    V = to_block(gen.gaussian_block(g.n, 4, seed=55), torch.bfloat16)
    with pytest.raises(sped.SpedError):
        sped.poly_moments(G, V, 4, 3)
    V = to_block(gen.gaussian_block(g.n, 4, seed=55), torch.float64)
    with pytest.raises(sped.SpedError):
        sped.poly_moments(G, V, 4, 3, a=5.0, b=2.0)
