"""Degenerate and boundary cases of the chain step, the polynomial (Section 2, Table 2) and the
solver (Section 5.1): graphs without edges, a single node, graphs smaller than one warp's rows,
every block width from one column to the widest the solver takes, a zero eigenvalue of
multiplicity equal to the number of components, and the rejected empty graph."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2207_14589_gb300 as sped
from util_gpu import DEV, TOL, assert_close, host, stored, to_block

pytestmark = pytest.mark.gpu

DTYPES = [torch.float64, torch.float32, torch.bfloat16]


def _graph(n, edges):
    a = np.array([e[0] for e in edges], dtype=np.int64)
    b = np.array([e[1] for e in edges], dtype=np.int64)
    return gen.from_edges(n, a, b, name=f"g{n}")


@pytest.mark.parametrize("n", [1, 7, 1000])
@pytest.mark.parametrize("chain", DTYPES)
@pytest.mark.parametrize("split", [1, 2])
def test_edgeless_graph_maps_every_block_to_itself(n, chain, split):
    # L = 0: every factor (I - sL) is the identity, so p(L) V = V exactly; only the chain's
    # storage rounds it (a BF16 chain carries the BF16 value of each entry to the end)
    g = _graph(n, [])
    G = sped.Graph.from_csr(g)
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, 41)
    assert info.nnz == 0 and info.lambda_bound == 0.0
    assert info.scale_s == pytest.approx(1.0 / 41)
    G.set_schedule(split=split)
    k = 5
    vt = torch.float64 if chain == torch.float64 else torch.float32
    V0 = gen.gaussian_block(n, k, seed=n)
    V = to_block(V0, vt)
    Y = sped.alloc_block(n, k, vt, DEV, fill=float("nan"))
    sped.apply_poly(G, V, Y, k, chain_dtype=chain)
    torch.cuda.synchronize()
    assert np.array_equal(host(Y, k), stored(stored(V0, vt), chain))
    assert np.array_equal(oracle.poly_limit(g, stored(V0, vt), info.scale_s, 41),
                          stored(V0, vt))


TINY = {
    "single_edge": (2, [(0, 1)]),
    "path3": (3, [(0, 1), (1, 2)]),
    "triangle_and_isolated": (4, [(0, 1), (1, 2), (0, 2)]),
    "k4": (4, [(i, j) for i in range(4) for j in range(i + 1, 4)]),
    "star6": (6, [(0, j) for j in range(1, 6)]),
}


@pytest.mark.parametrize("name", list(TINY))
@pytest.mark.parametrize("chain", DTYPES)
@pytest.mark.parametrize("split", [1, 2])
def test_graphs_smaller_than_one_warp(name, chain, split):
    # fewer rows than one warp's row groups: most lanes of the only warp have no row
    n, edges = TINY[name]
    g = _graph(n, edges)
    G = sped.Graph.from_csr(g)
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, 9)
    G.set_schedule(split=split)
    k = 3
    vt = torch.float64 if chain == torch.float64 else torch.float32
    V0 = gen.gaussian_block(n, k, seed=3)
    V = to_block(V0, vt)
    Y = sped.alloc_block(n, k, vt, DEV, fill=float("nan"))
    sped.apply_poly(G, V, Y, k, chain_dtype=chain)
    torch.cuda.synchronize()
    want = oracle.poly_limit(g, stored(V0, vt), info.scale_s, 9)
    assert_close(host(Y, k), want, TOL[chain])
    assert torch.isnan(Y[:, k:]).all()


@pytest.mark.parametrize("k", [1, 2, 7, 16, 17, 32, 33, 40])
@pytest.mark.parametrize("xt", DTYPES)
@pytest.mark.parametrize("split", [1, 2])
def test_step_every_block_width(k, xt, split):
    # one to several 16-byte lanes per row (1 .. 20 lanes for F64), ragged and empty rows
    g = gen.random_graph(1531, 6000, seed=k, hub=3, hub_degree=400, isolated=9)
    G = sped.Graph.from_csr(g)
    X0 = gen.gaussian_block(g.n, k, seed=100 + k)
    X = to_block(X0, xt)
    Y = sped.alloc_block(g.n, k, xt, DEV, fill=float("nan"))
    sped.poly_step(G, X, Y, k, alpha=0.0, beta=-0.03, gamma=1.0, split=split)
    torch.cuda.synchronize()
    Xs = stored(X0, xt)
    assert_close(host(Y, k), Xs - 0.03 * oracle.laplacian_apply(g, Xs), TOL[xt])
    if Y.shape[1] > k:
        assert torch.isnan(Y[:, k:]).all()


def test_empty_graph_rejected():
    rp = torch.zeros(1, dtype=torch.int32, device=DEV)
    ci = torch.zeros(0, dtype=torch.int32, device=DEV)
    with pytest.raises(sped.SpedError):
        sped.Graph(rp, ci)


@pytest.mark.parametrize("solver", [sped.OJA, sped.MU_EG])
def test_zero_eigenvalue_of_multiplicity_five(solver):
    # five disjoint cliques: eigenvalue 0 with multiplicity 5 (one per component), then the
    # clique sizes; the bottom-5 subspace is the span of the component indicators even though
    # no single eigenvector in it is unique
    sizes = [40, 25, 60, 10, 30]
    g = gen.cliques(sizes)
    G = sped.Graph.from_csr(g)
    k = len(sizes)
    G.set_polynomial(sped.POLY_LIMIT_EXP, 7)
    eta = 0.0 if solver == sped.OJA else 1.5
    opts = sped.solve_opts(solver, eta, torch.float64, torch.float64, max_steps=2000, tol=1e-8,
                           refine_dtype=torch.float64)
    V = to_block(gen.gaussian_block(g.n, k, seed=4), torch.float64)
    lam, rep = sped.solve_bottom_k(G, V, k, opts)
    assert rep["converged"], rep
    ind = np.zeros((g.n, k))
    ind[np.arange(g.n), g.labels] = 1.0
    got = host(V, k)
    assert oracle.principal_angle_max(ind, got) <= 1e-6
    assert np.abs(np.array(lam)).max() <= 1e-9
    # k-means on the solver's rows recovers the components (canonical labels follow node order)
    labels, _ = sped.cluster_assign(V, k, k, seed=2)
    assert np.array_equal(labels.cpu().numpy(), g.labels)
