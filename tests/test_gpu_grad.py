"""Parity of the differentiable utilities with the oracle: utilities, Hbar and the EigenGame
(detached) direction; the full gradients w.r.t. V (adjoint polynomial chain) and w.r.t. the
edge weights (checkpointed SDDMM), against the oracle's analytic gradients (themselves pinned
to finite differences) and against central finite differences of the GPU forward."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2207_14589_gb300 as sped
from util_gpu import assert_close, DEV, host, rel, to_block

pytestmark = pytest.mark.gpu


def _setup(n=400, blocks=4, k=4, ell=7, seed=3):
    g = gen.uniform_edge_weights(gen.sbm_by_degree(n, blocks, 12.0, 0.85, seed=seed), seed=seed + 1)
    G = sped.Graph.from_csr(g)
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
    a, b, w = oracle.edge_list(g)
    V0 = gen.gaussian_block(g.n, k, seed=seed + 2)
    return g, G, info, w, V0


def test_utilities_hbar_and_detached_direction():
    g, G, info, w, V0 = _setup()
    k = V0.shape[1]
    V = to_block(V0, torch.float64)
    Y = sped.alloc_block(g.n, k, torch.float64, DEV)
    sped.apply_poly(G, V, Y, k)
    Gm = sped.gram(V, k, Y, k)
    gu = torch.tensor([1.0, -0.5, 2.0, 0.25], dtype=torch.float64)
    u, Hbar, S = sped.eg_utilities(Gm, k, gu)
    Y0 = oracle.poly_limit(g, V0, info.scale_s, 7)
    assert np.allclose(u.cpu().numpy(), oracle.eg_utilities(V0, Y0), rtol=1e-11)
    Hb = oracle.eg_utility_hbar(V0.T @ Y0, gu.numpy())
    assert np.allclose(Hbar.cpu().numpy(), Hb, rtol=1e-10, atol=1e-12)
    D = sped.block_combine(Y, k, S)
    assert_close(D[:, :k].cpu().numpy(), oracle.eg_grad_detached(V0, Y0), 1e-11)


@pytest.mark.parametrize("ell", [1, 5, 9])
def test_autograd_matches_oracle_gradients(ell):
    g, G, info, w, V0 = _setup(ell=ell)
    k = V0.shape[1]
    V = to_block(V0, torch.float64).requires_grad_(True)
    wt = torch.tensor(w, dtype=torch.float64, device=DEV, requires_grad=True)
    gu = torch.tensor([1.0, 0.5, -0.7, 2.0], dtype=torch.float64, device=DEV)
    u = sped.eigengame_utilities(V, wt, G, k)
    (u * gu).sum().backward()
    Y0 = oracle.poly_limit(g, V0, info.scale_s, ell)
    gn = gu.cpu().numpy()
    assert_close(V.grad[:, :k].cpu().numpy(), oracle.eg_grad_full(V0, Y0, gn), 1e-10)
    assert torch.all(V.grad[:, k:] == 0)
    Hb = oracle.eg_utility_hbar(V0.T @ Y0, gn)
    want = oracle.limit_edge_grad(g, V0, info.scale_s, ell, Hb)
    assert_close(wt.grad.cpu().numpy(), want, 1e-9)


def test_autograd_against_finite_differences():
    g, G, info, w, V0 = _setup(n=300, k=3, ell=5, seed=11)
    k = 3
    gu = torch.tensor([1.0, -0.7, 0.4], dtype=torch.float64, device=DEV)
    V = to_block(V0, torch.float64).requires_grad_(True)
    w32 = w.astype(np.float32).astype(np.float64)
    wt = torch.tensor(w32, dtype=torch.float64, device=DEV, requires_grad=True)
    (sped.eigengame_utilities(V, wt, G, k) * gu).sum().backward()

    def f(Vx, wx):
        with torch.no_grad():
            return float((sped.eigengame_utilities(Vx, wx, G, k) * gu).sum())

    h = 1e-4
    rng = np.random.default_rng(0)
    for e in rng.choice(len(w32), size=6, replace=False):
        hp = float(np.float32(w32[e] + h) - w32[e])
        hm = float(w32[e] - np.float32(w32[e] - h))
        wp, wm = wt.detach().clone(), wt.detach().clone()
        wp[e] += hp
        wm[e] -= hm
        fd = (f(V.detach(), wp) - f(V.detach(), wm)) / (hp + hm)
        assert fd == pytest.approx(float(wt.grad[e]), rel=2e-5, abs=1e-8)
    for (r, c) in [(0, 0), (17, 2), (151, 1)]:
        Vp, Vm = V.detach().clone(), V.detach().clone()
        Vp[r, c] += h
        Vm[r, c] -= h
        fd = (f(Vp, wt.detach()) - f(Vm, wt.detach())) / (2 * h)
        assert fd == pytest.approx(float(V.grad[r, c]), rel=1e-6, abs=1e-9)


def test_edge_grad_full_size_spot_check():
    # differentiable workload at full size: SBM N=200,000, 10 blocks, mean degree 20, weights
    # U(0.5, 1.5), k=10; sampled edges and rows against the oracle's analytic gradients
    g = gen.uniform_edge_weights(gen.sbm_by_degree(200_000, 10, 20.0, 0.875, seed=5), seed=6)
    G = sped.Graph.from_csr(g)
    ell, k = 11, 10
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
    V0 = gen.gaussian_block(g.n, k, seed=7)
    V = to_block(V0, torch.float64)
    gu = np.linspace(1.0, 0.1, k)
    Y0 = oracle.poly_limit(g, V0, info.scale_s, ell)
    Hb = oracle.eg_utility_hbar(V0.T @ Y0, gu)
    got = sped.edge_grad(G, V, k, torch.tensor(Hb.T.copy(), device=DEV)).cpu().numpy()
    want = oracle.limit_edge_grad(g, V0, info.scale_s, ell, Hb)
    assert_close(got, want, 1e-9)


@pytest.mark.parametrize("kind", ["limit", "chebyshev"])
def test_apply_poly_backward_is_the_adjoint(kind):
    # <dY, M V> = <M^T dY, V> with M = p(L) symmetric, and dV matches the oracle's M dY
    g = gen.uniform_edge_weights(gen.random_graph(800, 3000, seed=71), seed=72)
    G = sped.Graph.from_csr(g)
    k = 5
    if kind == "limit":
        info = G.set_polynomial(sped.POLY_LIMIT_EXP, 9)
        apply = lambda X: oracle.poly_limit(g, X, info.scale_s, 9)
    else:
        c = [0.4, -0.3, 0.2, 0.1]
        hi = oracle.gershgorin_bound(g)
        G.set_polynomial(sped.POLY_CHEBYSHEV, 3, eps=0.1, coeffs=c, lambda_star=hi)
        apply = lambda X: oracle.poly_chebyshev(g, X, c, 0.1, hi)
    V0 = gen.gaussian_block(g.n, k, seed=73)
    dY0 = gen.gaussian_block(g.n, k, seed=74)
    dY = to_block(dY0, torch.float64)
    dV = sped.alloc_block(g.n, k, torch.float64, DEV)
    sped.apply_poly_backward(G, dY, dV, k)
    torch.cuda.synchronize()
    got = host(dV, k)
    assert np.linalg.norm(got - apply(dY0)) <= 1e-12 * np.linalg.norm(got)
    lhs = float(np.sum(dY0 * apply(V0)))
    assert abs(lhs - float(np.sum(got * V0))) <= 1e-10 * abs(lhs)


@pytest.mark.parametrize("k", [1, 2, 5, 9, 16, 17, 32])
@pytest.mark.parametrize("dt,tol", [(torch.float64, 1e-10), (torch.float32, 1e-4)])
def test_edge_grad_block_widths(k, dt, tol):
    # the checkpointed SDDMM at every row layout it takes: one to eight 16-byte chunks per row,
    # partial last chunks, both accumulator widths (k <= 16, k <= 32); every edge against the
    # oracle's analytic edge gradient of sum_a g_a u_a
    g, G, info, w, V0 = _setup(n=300, blocks=3, k=k, ell=5, seed=21)
    Vs = V0.astype(np.float32).astype(np.float64) if dt == torch.float32 else V0
    V = to_block(Vs, dt)
    gu = np.linspace(1.0, 0.2, k)
    Y0 = oracle.poly_limit(g, Vs, info.scale_s, 5)
    Hb = oracle.eg_utility_hbar(Vs.T @ Y0, gu)
    got = sped.edge_grad(G, V, k, torch.tensor(Hb.T.copy(), device=DEV)).cpu().numpy()
    want = oracle.limit_edge_grad(g, Vs, info.scale_s, 5, Hb)
    assert_close(got, want, tol)
