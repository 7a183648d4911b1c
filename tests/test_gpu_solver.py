"""Parity of the Gram, the solver step (mu-EG / Oja, Section 5.1), the bottom-k solve and the
hard clustering (Sections 1, 2.1) against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2207_14589_gb300 as sped
from util_gpu import DEV, assert_close, assert_gram_close, assert_step_close, host, stored, to_block

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("at,bt,tol", [(torch.float64, torch.float64, 1e-13),
                                       (torch.float32, torch.float32, 2e-6),
                                       (torch.bfloat16, torch.bfloat16, 1e-6),
                                       (torch.float32, torch.float64, 1e-13)])
@pytest.mark.parametrize("n,ka,kb", [(1, 1, 0), (1000, 4, 4), (33333, 20, 20), (5000, 32, 32),
                                     (777, 7, 3), (4099, 40, 40), (3001, 37, 36)])
def test_gram(at, bt, tol, n, ka, kb):
    A0 = gen.gaussian_block(n, ka, seed=1)
    B0 = gen.gaussian_block(n, kb, seed=2) if kb else None
    A = to_block(A0, at)
    B = to_block(B0, bt) if kb else None
    G = sped.gram(A, ka, B, kb)
    torch.cuda.synchronize()
    M = stored(A0, at) if not kb else np.concatenate([stored(A0, at), stored(B0, bt)], axis=1)
    want = M.T @ M
    if not kb and at != torch.float64:
        tol = max(tol, 2e-6)  # A alone: products in F32
    assert_gram_close(G.cpu().numpy(), want, tol)


@pytest.mark.parametrize("solver", [sped.MU_EG, sped.OJA])
@pytest.mark.parametrize("poly", ["limit", "shift"])
def test_eig_step_fp64(solver, poly):
    g = gen.sbm(1500, 3, 0.02, 0.001, seed=3)
    G = sped.Graph.from_csr(g)
    k = 5
    if poly == "limit":
        info = G.set_polynomial(sped.POLY_LIMIT_EXP, 9)
    else:
        info = G.set_polynomial(sped.POLY_SHIFT, 1)
    V0 = gen.gaussian_block(g.n, k, seed=4)
    V0 /= np.linalg.norm(V0, axis=0)
    V = to_block(V0, torch.float64)
    eta = 0.5 if solver == sped.MU_EG else 2.0
    if poly == "shift":
        eta /= info.lambda_star
    opts = sped.step_opts(solver, eta, torch.float64, torch.float64)
    stats = torch.zeros(3 * k, dtype=torch.float64, device=DEV)
    sped.eig_step(G, V, k, opts, stats=stats)
    torch.cuda.synchronize()
    if poly == "limit":
        Y0 = oracle.poly_limit(g, V0, info.scale_s, 9)
    else:
        Y0 = info.lambda_star * V0 - oracle.laplacian_apply(g, V0)
    want = oracle.mu_eg_step(V0, Y0, eta) if solver == sped.MU_EG else oracle.oja_step(V0, Y0, eta)
    assert np.abs(host(V, k) - want).max() <= 1e-10
    st = stats.cpu().numpy()
    assert np.allclose(st[:k], oracle.ritz_values(V0, Y0), rtol=1e-12)
    # invariant-subspace residual ||(I - P_V) y_i|| / ||y_i|| and the step sizes
    Q = oracle.orthonormal_basis(V0)
    res = np.linalg.norm(Y0 - Q @ (Q.T @ Y0), axis=0) / np.linalg.norm(Y0, axis=0)
    assert np.allclose(st[k:2 * k], res, rtol=1e-6, atol=1e-12)
    assert np.allclose(st[2 * k:], np.linalg.norm(want - V0, axis=0), rtol=1e-7, atol=1e-12)


def test_eig_step_mixed_precision_close_to_fp64():
    g = gen.sbm(5000, 5, 0.01, 0.0004, seed=5)
    G = sped.Graph.from_csr(g)
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, 21)
    k = 5
    V0 = gen.gaussian_block(g.n, k, seed=6)
    V0 /= np.linalg.norm(V0, axis=0)
    V = to_block(V0, torch.float32)
    opts = sped.step_opts(sped.MU_EG, 1.0, torch.bfloat16, torch.float32)
    sped.eig_step(G, V, k, opts)
    torch.cuda.synchronize()
    Vs = stored(V0, torch.float32)
    Y = oracle.poly_limit(g, Vs, info.scale_s, 21)
    want = oracle.mu_eg_step(Vs, Y, 1.0)
    assert_step_close(host(V, k), want, lambda Yp: oracle.mu_eg_step(Vs, Yp, 1.0), Y, 1e-2)


def _sbm_n2000_k4():
    return gen.sbm(2000, 4, 0.05, 0.001, seed=gen.DEFAULT_SEED)


def test_bf16_shadow_tracks_master_and_feeds_the_chain():
    # the update writes bf16(V_new) into the shadow (bit for bit, padding untouched); a step
    # that starts its BF16 chain from the shadow stays within the BF16 storage bound
    g = gen.sbm(5000, 5, 0.01, 0.0004, seed=25)
    G = sped.Graph.from_csr(g)
    ell = 21
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, ell)
    k = 6
    V0 = gen.gaussian_block(g.n, k, seed=26)
    V0 /= np.linalg.norm(V0, axis=0)
    V = to_block(V0, torch.float32)
    Vb = sped.alloc_block(g.n, k, torch.bfloat16, DEV, fill=float("nan"))
    opts = sped.step_opts(sped.MU_EG, 1.0, torch.bfloat16, torch.float32, v_shadow=Vb)
    sped.eig_step(G, V, k, opts)
    torch.cuda.synchronize()
    assert torch.equal(Vb[:, :k], V[:, :k].to(torch.bfloat16))
    if Vb.shape[1] > k:
        assert torch.isnan(Vb[:, k:]).all()
    V1 = host(V, k)
    opts = sped.step_opts(sped.MU_EG, 1.0, torch.bfloat16, torch.float32, v_shadow=Vb,
                          shadow_valid=True)
    sped.eig_step(G, V, k, opts)
    torch.cuda.synchronize()
    assert torch.equal(Vb[:, :k], V[:, :k].to(torch.bfloat16))
    Y1 = oracle.poly_limit(g, V1, info.scale_s, ell)
    want = oracle.mu_eg_step(V1, Y1, 1.0)
    assert_step_close(host(V, k), want, lambda Yp: oracle.mu_eg_step(V1, Yp, 1.0), Y1, 1e-2)
    # the shadow needs an F32 master
    V64 = to_block(V0, torch.float64)
    with pytest.raises(sped.SpedError):
        sped.eig_step(G, V64, k, sped.step_opts(sped.MU_EG, 1.0, torch.bfloat16, torch.float64,
                                                v_shadow=Vb))


@pytest.mark.parametrize("arm", ["plain_fp64", "dilated_fp64", "dilated_mixed", "dilated_oja"])
def test_solve_bottom_k_sbm_n2000_k4(arm):
    g = _sbm_n2000_k4()
    G = sped.Graph.from_csr(g)
    k = 4
    lam, Ustar = oracle.bottom_k(g, k)
    V0 = gen.gaussian_block(g.n, k, seed=gen.DEFAULT_SEED)
    if arm == "plain_fp64":
        info = G.set_polynomial(sped.POLY_SHIFT, 1)
        opts = sped.solve_opts(sped.MU_EG, 2.0 / info.lambda_star, torch.float64, torch.float64,
                               max_steps=5000, check_every=10, tol=1e-5,
                               refine_dtype=torch.float64)
        vt = torch.float64
    else:
        G.set_polynomial(sped.POLY_LIMIT_EXP, 7)
        if arm == "dilated_fp64":
            opts = sped.solve_opts(sped.MU_EG, 1.5, torch.float64, torch.float64, max_steps=400,
                                   tol=1e-5, refine_dtype=torch.float64)
            vt = torch.float64
        elif arm == "dilated_oja":
            opts = sped.solve_opts(sped.OJA, 0.0, torch.float64, torch.float64, max_steps=200,
                                   tol=1e-5, refine_dtype=torch.float64)
            vt = torch.float64
        else:
            opts = sped.solve_opts(sped.MU_EG, 1.5, torch.bfloat16, torch.float32, max_steps=400,
                                   tol=1e-5, switch_tol=3e-3, phase1_steps=100,
                                   refine_dtype=torch.float32)
            vt = torch.float32
    V = to_block(V0, vt)
    lam_gpu, rep = sped.solve_bottom_k(G, V, k, opts)
    assert rep["converged"], rep
    got = host(V, k)
    ang = oracle.principal_angle_max(Ustar, got)
    assert ang <= 1e-3, (arm, ang, rep)
    # Rayleigh quotients of L on the converged subspace match the true bottom eigenvalues
    Q = oracle.orthonormal_basis(got)
    ritz = np.linalg.eigvalsh(Q.T @ oracle.laplacian_apply(g, Q))
    assert np.allclose(ritz, lam, atol=1e-4, rtol=1e-5)
    # the reported per-vector quotients equal the oracle's on the returned V
    assert np.allclose(lam_gpu, oracle.ritz_values(got, oracle.laplacian_apply(g, got)),
                       rtol=1e-9, atol=1e-12)


def test_cluster_assign_sbm_n2000_k4_labels_bit_exact():
    g = _sbm_n2000_k4()
    k = 4
    lam, U = oracle.bottom_k(g, k)
    for dtype in (torch.float64, torch.float32):
        V = to_block(U, dtype)
        labels, iters = sped.cluster_assign(V, k, 4, seed=5)
        want = oracle.kmeans(stored(U, dtype), 4, seed=5)
        assert np.array_equal(labels.cpu().numpy(), want)
    # well-separated nodes (majority of neighbours inside the block) carry the planted labels
    deg = np.diff(g.row_ptr)
    rows = np.repeat(np.arange(g.n), deg)
    same = np.bincount(rows, weights=(g.labels[rows] == g.labels[g.col_idx]), minlength=g.n)
    sep = same > deg / 2
    lab = labels.cpu().numpy()
    planted = g.labels
    # labels are canonical by first occurrence, planted blocks are in node order too
    assert np.array_equal(lab[sep], planted[sep])


def test_cluster_assign_cliques_and_empty_restart():
    g = gen.cliques([40, 25, 60, 10, 30])
    lam, U = oracle.bottom_k(g, 5)
    V = to_block(U, torch.float64)
    labels, _ = sped.cluster_assign(V, 5, 5, seed=1)
    assert np.array_equal(labels.cpu().numpy(), g.labels)
    X = np.repeat(np.eye(3), [5, 1, 4], axis=0) * 10.0
    V = to_block(X, torch.float64)
    for seed in range(6):
        labels, _ = sped.cluster_assign(V, 3, 4, seed=seed)
        assert np.array_equal(labels.cpu().numpy(), oracle.kmeans(X, 4, seed=seed))


def test_rayleigh_on_closed_form_eigenvectors():
    n = 300
    g = gen.path(n)
    G = sped.Graph.from_csr(g)
    i = np.arange(n)
    js = [1, 2, 5, 17]
    U = np.stack([np.cos(np.pi * j * (i + 0.5) / n) for j in js], axis=1)
    V = to_block(U, torch.float64)
    lam = sped.rayleigh(G, V, len(js)).cpu().numpy()
    assert np.allclose(lam, [2 - 2 * np.cos(np.pi * j / n) for j in js], rtol=1e-12)


@pytest.mark.parametrize("k", [1, 5, 8, 13, 32, 33, 40])
@pytest.mark.parametrize("vt", [torch.float64, torch.float32])
def test_rayleigh_ritz_matches_oracle(k, vt):
    g = gen.sbm(1200, 4, 0.03, 0.002, seed=30 + k)
    G = sped.Graph.from_csr(g)
    V0 = gen.gaussian_block(g.n, k, seed=31)
    V = to_block(V0, vt)
    theta, W = sped.rayleigh_ritz(G, V, k)
    Vs = stored(V0, vt)
    want_t, want_W = oracle.rayleigh_ritz(g, Vs)
    tol = 1e-10 if vt == torch.float64 else 1e-5
    assert np.allclose(theta.cpu().numpy(), want_t, rtol=tol, atol=tol * abs(want_t).max())
    # Ritz vectors agree up to the sign of each column
    X, Xw = Vs @ W.cpu().numpy(), Vs @ want_W
    for i in range(k):
        assert abs(abs(X[:, i] @ Xw[:, i]) - 1.0) <= (1e-8 if vt == torch.float64 else 1e-4)
    # rotate=True: V becomes the orthonormal Ritz vectors, with the same Ritz values
    sped.rayleigh_ritz(G, V, k, rotate=True)
    torch.cuda.synchronize()
    R = host(V, k)
    assert np.allclose(R.T @ R, np.eye(k), atol=1e-10 if vt == torch.float64 else 1e-4)
    theta2, _ = sped.rayleigh_ritz(G, V, k)
    assert np.allclose(theta2.cpu().numpy(), want_t, rtol=10 * tol, atol=10 * tol * abs(want_t).max())


def test_rayleigh_ritz_on_an_invariant_subspace_is_exact():
    # path graph: the span of the first k closed-form eigenvectors (in a random basis)
    n, k = 64, 6
    g = gen.path(n)
    G = sped.Graph.from_csr(g)
    x = np.arange(n) + 0.5
    U = np.stack([np.cos(np.pi * j * x / n) for j in range(k)], axis=1)
    B = U @ np.random.default_rng(5).standard_normal((k, k))
    theta, _ = sped.rayleigh_ritz(G, to_block(B, torch.float64), k)
    assert np.allclose(theta.cpu().numpy(), 2.0 - 2.0 * np.cos(np.pi * np.arange(k) / n),
                       atol=1e-12)


@pytest.mark.parametrize("dtype,ld", [(torch.bfloat16, 7), (torch.float32, 67),
                                      (torch.float64, 5)])
def test_gram_rejects_rows_that_are_not_16_byte_multiples(dtype, ld):
    # rows of ld * sizeof bytes that are not whole 16-byte chunks are rejected before any launch
    # (the tensor path moves whole tiles with bulk copies)
    import ctypes
    n, ka = 300, min(ld, 4)
    T = torch.zeros((n, ld), dtype=dtype, device=DEV)
    G = torch.full((2 * ka, 2 * ka), float("nan"), dtype=torch.float64, device=DEV)
    scr = torch.empty(1 << 20, dtype=torch.uint8, device=DEV)
    dt = {torch.bfloat16: sped.BF16, torch.float32: sped.F32, torch.float64: sped.F64}[dtype]
    st = sped.lib().sped_gram(n, ctypes.c_void_p(T.data_ptr()), dt, ld, ka,
                              ctypes.c_void_p(T.data_ptr()), dt, ld, ka,
                              ctypes.c_void_p(G.data_ptr()), ctypes.c_void_p(scr.data_ptr()),
                              scr.numel(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    assert st == sped.ERR_INVALID_ARG
    assert b"multiple of 16" in sped.lib().sped_last_error()
    assert torch.isnan(G).all()  # nothing launched


def test_gram_wait_timeout_surfaces_as_status():
    # the tensor Gram's bounded waits: with its bulk copies skipped (nothing in flight) and a
    # short poll limit, the first wait runs out; the CTAs free their tensor memory and return,
    # the Gram is NaN and the next status read reports SPED_ERR_TIMEOUT. The context stays
    # usable: the same call afterwards is exact again and the status is clear.
    n, k = 5000, 20
    A0 = gen.gaussian_block(n, k, seed=61)
    A = to_block(A0, torch.float32)
    want = stored(A0, torch.float32).T @ stored(A0, torch.float32)
    sped.device_status()  # start from a clear word
    try:
        sped.test_gram_waits(wait_limit=2000, skip_fills=True)
        G = sped.gram(A, k)
        with pytest.raises(sped.SpedError) as e:
            sped.device_status()
        assert e.value.status == sped.ERR_TIMEOUT
        assert torch.isnan(G).all()
    finally:
        sped.test_gram_waits(0, False)
    sped.device_status()  # cleared by the read above
    G = sped.gram(A, k)
    sped.device_status()
    assert_gram_close(G.cpu().numpy(), want, 2e-6)


def test_solve_reports_a_timed_out_wait():
    g = gen.sbm(3000, 3, 0.02, 0.001, seed=62)
    G = sped.Graph.from_csr(g)
    G.set_polynomial(sped.POLY_LIMIT_EXP, 9)
    k = 4
    V = to_block(gen.gaussian_block(g.n, k, seed=63), torch.float32)
    opts = sped.solve_opts(sped.OJA, 0.0, torch.bfloat16, torch.float32, max_steps=3,
                           check_every=1)
    try:
        sped.test_gram_waits(wait_limit=2000, skip_fills=True)
        with pytest.raises(sped.SpedError) as e:
            sped.solve_bottom_k(G, V, k, opts)
        assert e.value.status == sped.ERR_TIMEOUT
    finally:
        sped.test_gram_waits(0, False)
    sped.device_status()


@pytest.mark.parametrize("solver", [sped.MU_EG, sped.OJA])
@pytest.mark.parametrize("k", [33, 40])
def test_eig_step_fp64_wide_blocks(solver, k):
    # k in (32, 40]: the widest update kernel, the k x k stage in dynamic shared memory and the
    # 2k-column Gram on the CUDA cores
    g = gen.sbm(2500, 5, 0.02, 0.001, seed=70 + k)
    G = sped.Graph.from_csr(g)
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, 7)
    V0 = gen.gaussian_block(g.n, k, seed=71)
    V0 /= np.linalg.norm(V0, axis=0)
    V = to_block(V0, torch.float64)
    eta = 0.5 if solver == sped.MU_EG else 2.0
    opts = sped.step_opts(solver, eta, torch.float64, torch.float64)
    stats = torch.zeros(3 * k, dtype=torch.float64, device=DEV)
    sped.eig_step(G, V, k, opts, stats=stats)
    torch.cuda.synchronize()
    Y0 = oracle.poly_limit(g, V0, info.scale_s, 7)
    want = oracle.mu_eg_step(V0, Y0, eta) if solver == sped.MU_EG else oracle.oja_step(V0, Y0, eta)
    assert_close(host(V, k), want, 1e-10)
    assert np.allclose(stats.cpu().numpy()[:k], oracle.ritz_values(V0, Y0), rtol=1e-11)


def test_mixed_eig_step_k36():
    g = gen.sbm(6000, 6, 0.01, 0.0004, seed=75)
    G = sped.Graph.from_csr(g)
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, 21)
    k = 36
    V0 = gen.gaussian_block(g.n, k, seed=76)
    V0 /= np.linalg.norm(V0, axis=0)
    V = to_block(V0, torch.float32)
    Vb = sped.alloc_block(g.n, k, torch.bfloat16, DEV)
    opts = sped.step_opts(sped.OJA, 0.0, torch.bfloat16, torch.float32, v_shadow=Vb)
    sped.eig_step(G, V, k, opts)
    torch.cuda.synchronize()
    assert torch.equal(Vb[:, :k], V[:, :k].to(torch.bfloat16))
    Vs = stored(V0, torch.float32)
    Y = oracle.poly_limit(g, Vs, info.scale_s, 21)
    orth = lambda Yp: oracle.oja_step(np.zeros_like(Vs), Yp, 1.0)
    assert_step_close(host(V, k), orth(Y), orth, Y, 1e-2)


def test_eig_step_rejects_more_than_40_columns():
    g = gen.sbm(500, 2, 0.05, 0.01, seed=3)
    G = sped.Graph.from_csr(g)
    V = to_block(gen.gaussian_block(g.n, 41, seed=4), torch.float64)
    with pytest.raises(sped.SpedError):
        sped.eig_step(G, V, 41, sped.step_opts(sped.OJA, 0.0, torch.float64, torch.float64))
