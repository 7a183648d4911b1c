"""Parity at the full sizes of the other benchmark workloads, in the launch configurations the
benchmark times: the merge-path chain step on the planted-cluster power-law graph (N = 16,000,000,
3.2e8 stored entries, weights U(0.5, 1.5), k = 32, BF16 storage) with sampled output rows
recomputed one by one by the oracle's definition, and one batched solver step over all 4,096
graphs of the batched workload (k = 8, degree 31, BF16 chain) with sampled graphs stepped by the
oracle."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2207_14589_gb300 as sped
from util_gpu import DEV, assert_close, assert_step_close, host, stored, to_block

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def chung_lu_full():
    g = gen.chung_lu_clusters(16_000_000, target_nnz=3.2e8, seed=gen.DEFAULT_SEED, device=DEV)
    G = sped.Graph.from_csr(g)
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, 251)
    return g, G, info


def _rows_one_by_one(g, X, rows, s):
    """x_r - s (d_r x_r - sum_j w_rj x_j) for each sampled row r (weighted L = D - A), from the
    stored BF16 rows of X (only the rows these outputs read are copied to the host)."""
    nbrs = [g.col_idx[g.row_ptr[r]:g.row_ptr[r + 1]] for r in rows]
    need = np.unique(np.concatenate([rows] + nbrs))
    Xn = X[torch.from_numpy(need).to(X.device)].double().cpu().numpy()
    pos = {int(j): t for t, j in enumerate(need)}
    want = np.empty((len(rows), X.shape[1]))
    for t, r in enumerate(rows):
        p0, p1 = g.row_ptr[r], g.row_ptr[r + 1]
        w = g.w[p0:p1].astype(np.float64)
        xn = Xn[[pos[int(j)] for j in nbrs[t]]]
        xr = Xn[pos[int(r)]]
        want[t] = xr - s * (w.sum() * xr - w @ xn)
    return want


@pytest.mark.parametrize("split", [2, 1])  # merge path (the tuned schedule), row groups
@pytest.mark.parametrize("yt,tol", [(torch.bfloat16, 1e-2), (torch.float32, 1e-5)])
def test_chung_lu_chain_step_sampled_rows(chung_lu_full, split, yt, tol):
    g, G, info = chung_lu_full
    assert g.nnz > 3.0e8 and int(np.diff(g.row_ptr).max()) > 10_000
    k, s = 32, info.scale_s
    X = sped.alloc_block(g.n, k, torch.bfloat16, DEV)
    gen_t = torch.Generator(device=DEV).manual_seed(3)
    X[:, :k] = torch.randn(g.n, k, generator=gen_t, device=DEV).to(torch.bfloat16)
    Y = sped.alloc_block(g.n, k, yt, DEV)
    sped.poly_step(G, X, Y, k, alpha=0.0, beta=-s, gamma=1.0, split=split)
    torch.cuda.synchronize()
    deg = np.diff(g.row_ptr)
    rng = np.random.default_rng(4)
    # uniform rows plus the heaviest rows (hubs cut across many merge-path shares)
    rows = np.unique(np.concatenate([rng.choice(g.n, size=2000, replace=False),
                                     np.argsort(deg)[-50:]]))
    got = Y[torch.from_numpy(rows).to(DEV), :k].double().cpu().numpy()
    want = _rows_one_by_one(g, X[:, :k], rows, s)
    assert_close(got, want, tol)


def test_batched_full_workload_sampled_graphs():
    graphs = gen.batched_sbm(4096)
    k, ell, eta = 8, 31, 1.0
    B = sped.Batch.from_graphs(graphs, degree=ell)
    scales = B.scales()
    V = sped.batch_block(B.n_total, k)
    V[:, :k] = torch.from_numpy(gen.gaussian_block(B.n_total, k, seed=13)).float().cuda()
    off = np.concatenate([[0], np.cumsum([g.n for g in graphs])])
    sizes = np.array([g.n for g in graphs])
    pick = np.unique(np.concatenate([[int(np.argmax(sizes)), int(np.argmin(sizes))],
                                     np.random.default_rng(5).choice(len(graphs), 10,
                                                                     replace=False)]))
    V0 = {int(i): V[off[i]:off[i + 1], :k].double().cpu().numpy() for i in pick}
    B.eig_steps(V, k, steps=1, eta=eta, chain_dtype=torch.bfloat16)
    torch.cuda.synchronize()
    for i in pick:
        i = int(i)
        g, Vi = graphs[i], V0[i]
        Yi = oracle.poly_limit(g, Vi, scales[i], ell)
        want = oracle.mu_eg_step(Vi, Yi, eta)
        got = V[off[i]:off[i + 1], :k].double().cpu().numpy()
        assert_step_close(got, want, lambda Yp: oracle.mu_eg_step(Vi, Yp, eta), Yi, 1e-2, seed=i)


@pytest.mark.parametrize("dt,tol_v,tol_w", [(torch.float64, 1e-10, 1e-9),
                                            (torch.float32, 1e-4, 1e-4)])
def test_differentiable_full_size(dt, tol_v, tol_w):
    # the differentiable workload at its full size: SBM N = 200,000, 10 blocks, mean degree 20,
    # 87.5 % intra-block edge ends, weights U(0.5, 1.5), k = 10, degree 11; the gradients of
    # sum_i g_i u_i w.r.t. V (adjoint chain) and w.r.t. every edge weight (checkpointed SDDMM)
    # against the oracle's analytic gradients
    g = gen.uniform_edge_weights(gen.sbm_by_degree(200_000, 10, 20.0, 0.875, seed=5), seed=6)
    G = sped.Graph.from_csr(g)
    ell, k = 11, 10
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
    a, b, w = oracle.edge_list(g)
    V0 = gen.gaussian_block(g.n, k, seed=19)
    V = to_block(V0, dt).requires_grad_(True)
    wt = torch.tensor(w, dtype=dt, device=DEV, requires_grad=True)
    gu = torch.linspace(1.0, 0.1, k, dtype=torch.float64, device=DEV)
    u = sped.eigengame_utilities(V, wt, G, k)
    (u * gu).sum().backward()
    Vs = stored(V0, dt)
    Y0 = oracle.poly_limit(g, Vs, info.scale_s, ell)
    gn = gu.cpu().numpy()
    assert np.allclose(u.detach().cpu().numpy(), oracle.eg_utilities(Vs, Y0), rtol=tol_v)
    assert_close(V.grad[:, :k].double().cpu().numpy(), oracle.eg_grad_full(Vs, Y0, gn), tol_v)
    Hb = oracle.eg_utility_hbar(Vs.T @ Y0, gn)
    assert_close(wt.grad.double().cpu().numpy(),
                 oracle.limit_edge_grad(g, Vs, info.scale_s, ell, Hb), tol_w)
