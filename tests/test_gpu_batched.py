"""Parity of the batched persistent solver (many graphs in one launch) with per-graph oracle
steps: the limit-form chain (Table 2) and the mu-EG update (Section 5.1) for every graph."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2207_14589_gb300 as sped
from util_gpu import assert_close, assert_step_close

pytestmark = pytest.mark.gpu


def _graphs(count, seed, n_lo=150, n_hi=1500, sep=False):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        n = int(rng.integers(n_lo, n_hi))
        b = int(rng.integers(2, 7))
        if sep:
            out.append(gen.sbm(n, b, min(1.0, 16.0 / (n / b)), 0.3 / n, seed=seed + i))
        else:
            out.append(gen.sbm_by_degree(n, b, 10.0, 0.85, seed=seed + i))
    return out


def _split(V, graphs, k):
    off = np.concatenate([[0], np.cumsum([g.n for g in graphs])])
    return [V[off[i]:off[i + 1], :k] for i in range(len(graphs))]


@pytest.mark.parametrize("k,chain,tol", [(8, torch.float32, 1e-5), (5, torch.float32, 1e-5),
                                         (8, torch.bfloat16, 1e-2), (13, torch.float32, 1e-5)])
def test_batched_one_step_matches_oracle(k, chain, tol):
    graphs = _graphs(24, 100 + k)
    ell = 9
    B = sped.Batch.from_graphs(graphs, degree=ell)
    scales = B.scales()
    V0 = gen.gaussian_block(B.n_total, k, seed=5)
    V = sped.batch_block(B.n_total, k)
    V[:, :k] = torch.from_numpy(V0).float().cuda()
    Vs = V[:, :k].double().cpu().numpy()
    _, ritz = B.eig_steps(V, k, steps=1, eta=0.8, chain_dtype=chain)
    torch.cuda.synchronize()
    got = _split(V.double().cpu().numpy(), graphs, k)
    ritz = ritz.cpu().numpy()
    eta = 0.8
    for i, (g, Vi) in enumerate(zip(graphs, _split(Vs, graphs, k))):
        assert scales[i] == pytest.approx(oracle.scale_rule(oracle.gershgorin_bound(g), ell))
        Yi = oracle.poly_limit(g, Vi, scales[i], ell)
        want = oracle.mu_eg_step(Vi, Yi, eta)
        # the chain bound (tol on Y = p(L) V) reaches the step output through the eta Y term and
        # through the Gram-derived coefficients; the gain is measured on the oracle
        assert_step_close(got[i], want, lambda Yp: oracle.mu_eg_step(Vi, Yp, eta), Yi, tol,
                          seed=i)
        assert np.allclose(ritz[i], oracle.ritz_values(Vi, Yi), rtol=max(tol, 1e-5))


@pytest.mark.parametrize("chain,tol", [(torch.bfloat16, 1e-2), (torch.float32, 1e-5)])
def test_batched_config4_sizes_match_oracle(chain, tol):
    # the batched workload's largest graphs (20,000 nodes, 8 blocks, mean degree 12, 87.5 %
    # intra-block edge ends) beside small ones, k = 8 and the benchmark's degree 31: a 512-thread
    # CTA walks a large graph's rows in many passes per chain step and Gram
    rng = np.random.default_rng(44)
    graphs = [gen.sbm_by_degree(20000, 8, 12.0, 0.875, seed=401),
              gen.sbm_by_degree(200, 2, 12.0, 0.875, seed=402),
              gen.sbm_by_degree(13001, 5, 12.0, 0.875, seed=403),
              gen.sbm_by_degree(20000, 3, 12.0, 0.875, seed=404)]
    graphs += [gen.sbm_by_degree(int(rng.integers(200, 4000)), int(rng.integers(2, 9)), 12.0,
                                 0.875, seed=410 + i) for i in range(8)]
    k, ell, eta = 8, 31, 1.0
    B = sped.Batch.from_graphs(graphs, degree=ell)
    scales = B.scales()
    V = sped.batch_block(B.n_total, k)
    V[:, :k] = torch.from_numpy(gen.gaussian_block(B.n_total, k, seed=45)).float().cuda()
    Vs = _split(V[:, :k].double().cpu().numpy(), graphs, k)
    _, ritz = B.eig_steps(V, k, steps=1, eta=eta, chain_dtype=chain)
    torch.cuda.synchronize()
    got = _split(V.double().cpu().numpy(), graphs, k)
    ritz = ritz.cpu().numpy()
    for i, (g, Vi) in enumerate(zip(graphs, Vs)):
        Yi = oracle.poly_limit(g, Vi, scales[i], ell)
        want = oracle.mu_eg_step(Vi, Yi, eta)
        assert_step_close(got[i], want, lambda Yp: oracle.mu_eg_step(Vi, Yp, eta), Yi, tol,
                          seed=i)
        assert np.allclose(ritz[i], oracle.ritz_values(Vi, Yi), rtol=max(tol, 1e-5))


def test_batched_trajectory_matches_oracle():
    graphs = _graphs(12, 31)
    k, ell, eta, steps = 6, 7, 1.0, 8
    B = sped.Batch.from_graphs(graphs, degree=ell)
    scales = B.scales()
    V = sped.batch_block(B.n_total, k)
    V[:, :k] = torch.from_numpy(gen.gaussian_block(B.n_total, k, seed=8)).float().cuda()
    V0 = _split(V[:, :k].double().cpu().numpy(), graphs, k)
    B.eig_steps(V, k, steps=steps, eta=eta, chain_dtype=torch.float32)
    torch.cuda.synchronize()
    got = _split(V.double().cpu().numpy(), graphs, k)
    for i, g in enumerate(graphs):
        W = V0[i]
        for _ in range(steps):
            W = oracle.mu_eg_step(W, oracle.poly_limit(g, W, scales[i], ell), eta)
        assert_close(got[i], W, 1e-4)


def test_batched_converges_to_every_bottom_k():
    # 4-block graphs with a clear gap after lambda_4 (lambda_4 ~ 0.3, lambda_5 ~ 4.5); the oracle
    # reaches machine precision with these settings in fewer than 60 steps
    rng = np.random.default_rng(7)
    graphs = []
    for i in range(24):
        n = int(rng.integers(200, 900))
        graphs.append(gen.sbm(n, 4, min(1.0, 16.0 / (n / 4)), 0.3 / n, seed=700 + i))
    k = 4
    B = sped.Batch.from_graphs(graphs, degree=5)
    V = sped.batch_block(B.n_total, k)
    V[:, :k] = torch.from_numpy(gen.gaussian_block(B.n_total, k, seed=3)).float().cuda()
    B.eig_steps(V, k, steps=60, eta=1.5, chain_dtype=torch.float32)
    torch.cuda.synchronize()
    got = _split(V.double().cpu().numpy(), graphs, k)
    for g, Vi in zip(graphs, got):
        lam, U = oracle.bottom_k(g, k)
        assert oracle.principal_angle_max(U, Vi) <= 1e-3


def test_batched_graph_capture_replay():
    graphs = _graphs(40, 11)
    k = 8
    B = sped.Batch.from_graphs(graphs, degree=7)
    V0 = torch.from_numpy(gen.gaussian_block(B.n_total, k, seed=9)).float().cuda()
    scr = torch.empty(B.scratch_bytes(k), dtype=torch.uint8, device="cuda")
    ritz = torch.empty((B.n_graphs, k), dtype=torch.float64, device="cuda")
    Va = sped.batch_block(B.n_total, k)
    Va[:, :k] = V0
    for _ in range(2):
        B.eig_steps(Va, k, steps=2, eta=1.0, ritz=ritz, scratch=scr)
    Vb = sped.batch_block(B.n_total, k)
    Vb[:, :k] = V0
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        B.eig_steps(Vb, k, steps=2, eta=1.0, ritz=ritz, scratch=scr, stream=s)  # warm-up
    torch.cuda.current_stream().wait_stream(s)
    Vb[:, :k] = V0
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        B.eig_steps(Vb, k, steps=2, eta=1.0, ritz=ritz, scratch=scr)
    graph.replay()
    graph.replay()
    torch.cuda.synchronize()
    a, b = Va[:, :k].double().cpu().numpy(), Vb[:, :k].double().cpu().numpy()
    assert np.linalg.norm(a - b) / np.linalg.norm(a) <= 1e-5


def test_batched_rejects_columns_outside_their_graph():
    graphs = _graphs(3, 2)
    big, node_off, _ = gen.concat_graphs(graphs)
    ci = big.col_idx.copy()
    ci[big.row_ptr[node_off[1]]] = node_off[2] + 1  # first row of graph 1 points into graph 2
    with pytest.raises(sped.SpedError) as e:
        sped.Batch(node_off, torch.from_numpy(big.row_ptr).cuda(), torch.from_numpy(ci).cuda())
    assert e.value.status == sped.ERR_BAD_CSR


SCHEDULES = [(512, 2), (512, 4), (256, 4), (256, 8), (128, 8), (128, 16)]


@pytest.mark.parametrize("threads,cps", SCHEDULES)
@pytest.mark.parametrize("k", [6, 12])
def test_batched_every_schedule_matches_oracle(threads, cps, k):
    graphs = _graphs(20, 200 + k)
    ell, eta = 7, 0.8
    B = sped.Batch.from_graphs(graphs, degree=ell)
    B.set_schedule(threads, cps)
    scales = B.scales()
    V = sped.batch_block(B.n_total, k)
    V[:, :k] = torch.from_numpy(gen.gaussian_block(B.n_total, k, seed=9)).float().cuda()
    Vs = _split(V[:, :k].double().cpu().numpy(), graphs, k)
    B.eig_steps(V, k, steps=1, eta=eta, chain_dtype=torch.float32)
    torch.cuda.synchronize()
    got = _split(V.double().cpu().numpy(), graphs, k)
    for i, (g, Vi) in enumerate(zip(graphs, Vs)):
        want = oracle.mu_eg_step(Vi, oracle.poly_limit(g, Vi, scales[i], ell), eta)
        assert_close(got[i], want, 1e-4)


def test_batched_autotune_keeps_v_and_a_valid_schedule():
    graphs = _graphs(40, 77)
    k = 8
    B = sped.Batch.from_graphs(graphs, degree=9)
    V = sped.batch_block(B.n_total, k)
    V[:, :k] = torch.from_numpy(gen.gaussian_block(B.n_total, k, seed=10)).float().cuda()
    before = V.clone()
    rep = B.autotune(V, k)
    torch.cuda.synchronize()
    assert torch.equal(V, before)  # timed on a copy
    assert (rep["threads"], rep["ctas_per_sm"]) in SCHEDULES
    if not rep["cached"]:
        assert len(rep["ms"]) == len(SCHEDULES) and all(t > 0 for t in rep["ms"])
        assert SCHEDULES[int(np.argmin(rep["ms"]))] == (rep["threads"], rep["ctas_per_sm"])
    again = sped.Batch.from_graphs(graphs, degree=9).autotune(V, k)
    assert again["cached"] and (again["threads"], again["ctas_per_sm"]) == \
        (rep["threads"], rep["ctas_per_sm"])


def test_batched_set_schedule_rejects_bad_arguments():
    B = sped.Batch.from_graphs(_graphs(2, 3), degree=3)
    for th, cps in [(64, 2), (1024, 1), (512, 0), (256, 17)]:
        with pytest.raises(sped.SpedError):
            B.set_schedule(th, cps)
