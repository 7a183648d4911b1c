"""The paper's own workloads solved on the GPU and compared with the FP64 oracle: the 3-room
grid world of Section 5.3 (s = 2, h = 10) and the cliques graphs with short-circuit edges of
Section 5.4 / App. A.2, with the degree threshold of the limit form under the table's scale
s = 1/l. Steps run through the C ABI (FP64 Oja, V <- orth(M V)); the oracle runs the same
iteration from the same V0, and both are graded against the oracle's dense
eigendecomposition of L."""
import numpy as np
import pytest
import torch

import gen
import oracle
import paper_2207_14589_gb300 as sped
from util_gpu import DEV, assert_close, host, to_block

pytestmark = pytest.mark.gpu


def _gpu_steps_to_angle(G, V0, k, Ustar, cap, tol=1e-3):
    """FP64 Oja steps (eta = 0: V <- orth(M V)) on the GPU until the largest principal angle to
    span(Ustar) is <= tol; returns (first such step or None, last angle, V after step 1)."""
    opts = sped.step_opts(sped.OJA, 0.0, torch.float64, torch.float64)
    V = to_block(V0, torch.float64)
    scr = torch.empty(sped.eig_step_scratch_bytes(G, opts, k), dtype=torch.uint8, device=DEV)
    ang, first = None, None
    for t in range(1, cap + 1):
        sped.eig_step(G, V, k, opts, scratch=scr)
        Vh = host(V, k)
        if t == 1:
            first = Vh
        ang = oracle.principal_angle_max(Ustar, Vh)
        if ang <= tol:
            return t, ang, first
    return None, ang, first


def _oracle_steps_to_angle(apply_m, V0, Ustar, cap, tol=1e-3):
    V = np.array(V0, dtype=np.float64)
    ang = None
    for t in range(1, cap + 1):
        V = oracle.oja_step(np.zeros_like(V), apply_m(V), 1.0)  # orth(M V)
        ang = oracle.principal_angle_max(Ustar, V)
        if ang <= tol:
            return t, ang
    return None, ang


@pytest.mark.parametrize("arm", ["dilated251", "plain"])
def test_three_room_steps_to_bottom_k_match_oracle(arm):
    g = gen.three_room_grid(2, 10)
    k = 3  # one mode per room
    lam, U = oracle.bottom_k(g, k)
    G = sped.Graph.from_csr(g)
    V0 = gen.gaussian_block(g.n, k, seed=29)
    if arm == "dilated251":
        info = G.set_polynomial(sped.POLY_LIMIT_EXP, 251)
        s = info.scale_s
        assert s == pytest.approx(oracle.scale_rule(oracle.gershgorin_bound(g), 251))
        apply_m = lambda X: oracle.poly_limit(g, X, s, 251)
        cap = 1000
    else:
        info = G.set_polynomial(sped.POLY_SHIFT, 1)
        ls = info.lambda_star
        apply_m = lambda X: ls * X - oracle.laplacian_apply(g, X)
        cap = 8000
    t_gpu, a_gpu, V1 = _gpu_steps_to_angle(G, V0, k, U, cap)
    t_orc, a_orc = _oracle_steps_to_angle(apply_m, V0, U, cap)
    assert t_gpu is not None and t_orc is not None, (a_gpu, a_orc)
    assert abs(t_gpu - t_orc) <= 1, (t_gpu, t_orc)
    # the first step itself agrees element by element
    assert_close(V1, oracle.oja_step(np.zeros_like(V0), apply_m(V0), 1.0), 1e-10)
    if arm == "dilated251":
        test_three_room_steps_to_bottom_k_match_oracle.dilated = t_gpu
    else:
        # Section 5.3: the dilated operator needs several times fewer solver steps (the paper
        # reports about 10x for its degree-251 transform)
        d = getattr(test_three_room_steps_to_bottom_k_match_oracle, "dilated", None)
        if d is not None:
            assert t_gpu >= 5 * d, (t_gpu, d)


@pytest.fixture(scope="module")
def cliques_sc25():
    g = gen.cliques([450] * 4, short_circuit=25, seed=gen.DEFAULT_SEED)
    lam, U = np.linalg.eigh(oracle.dense_laplacian(g))
    return g, lam, U


@pytest.mark.parametrize("ell", [11, 51, 151, 251])
def test_cliques_degree_threshold_pattern(cliques_sc25, ell):
    # App. A.2: with the table's scale s = 1/l the limit form fails at l = 11, 51, 151 and
    # succeeds at l = 251 on the cliques graphs (lambda_max ~ 450): |1 - lambda/l| > 1 on the
    # clique modes below l ~ lambda_max / 2 makes them the dominant modes of M. The oracle
    # predicts success from the dense spectrum (the k largest |p(lambda_i)| are the bottom k of
    # L); the GPU's iteration must succeed exactly when predicted, within a few steps.
    g, lam, U = cliques_sc25
    k = 4
    s = 1.0 / ell
    p = np.abs(oracle.limit_scalar(lam, s, ell))
    top = np.argsort(-p, kind="stable")[:k]
    predicted = set(top.tolist()) == set(range(k)) and p[k - 1] > p[k:].max()
    assert predicted == (ell == 251)  # the paper's pattern, from the spectrum alone
    G = sped.Graph.from_csr(g)
    G.set_polynomial(sped.POLY_LIMIT_EXP, ell, scale=s)
    V0 = gen.gaussian_block(g.n, k, seed=23)
    t_gpu, a_gpu, V1 = _gpu_steps_to_angle(G, V0, k, U[:, :k], cap=12)
    assert (t_gpu is not None) == predicted, (ell, t_gpu, a_gpu)
    if predicted:
        t_orc, _ = _oracle_steps_to_angle(lambda X: oracle.poly_limit(g, X, s, ell), V0,
                                          U[:, :k], cap=12)
        assert t_orc is not None and abs(t_gpu - t_orc) <= 1, (t_gpu, t_orc)
        assert_close(V1, oracle.oja_step(np.zeros_like(V0),
                                         oracle.poly_limit(g, V0, s, ell), 1.0), 1e-10)
    else:
        assert a_gpu > 0.5  # the clique modes took over: far from the bottom-k subspace


@pytest.fixture(scope="module")
def link_completed():
    # App. A.1: four 100-cliques joined by 25 short-circuit edges, 20 % of the edges removed and
    # put back with common-neighbours scores as weights in (0, 1]
    g, _ = gen.link_completed_cliques([100] * 4, short_circuit=25, p_remove=0.2,
                                      seed=gen.DEFAULT_SEED)
    lam, U = np.linalg.eigh(oracle.dense_laplacian(g))
    return g, lam, U


def _gpu_oja_run(G, V0, k, steps):
    """FP64 Oja steps on the GPU; returns the host copy of V after every step."""
    opts = sped.step_opts(sped.OJA, 0.0, torch.float64, torch.float64)
    V = to_block(V0, torch.float64)
    scr = torch.empty(sped.eig_step_scratch_bytes(G, opts, k), dtype=torch.uint8, device=DEV)
    out = []
    for _ in range(steps):
        sped.eig_step(G, V, k, opts, scratch=scr)
        out.append(host(V, k))
    return out


def test_link_completed_cliques_streak_matches_oracle(link_completed):
    # the dilated operator (limit form, degree 251) resolves the individual bottom-4
    # eigenvectors of the weighted, link-completed graph: the GPU's FP64 Oja reaches a streak
    # of 4 (Section 5.2: every vector within pi/8 of its eigenvector) within one step of the
    # oracle's iteration from the same V0, and its first step agrees entry by entry
    g, lam, U = link_completed
    k = 4
    assert lam[k] - lam[k - 1] > 50 and lam[k - 1] < 1  # four slow modes, then the cliques
    G = sped.Graph.from_csr(g)
    info = G.set_polynomial(sped.POLY_LIMIT_EXP, 251)
    s = info.scale_s
    assert s == pytest.approx(oracle.scale_rule(oracle.gershgorin_bound(g), 251))
    V0 = gen.gaussian_block(g.n, k, seed=31)
    cap = 160
    gpu = _gpu_oja_run(G, V0, k, cap)
    t_gpu = next((t + 1 for t, V in enumerate(gpu)
                  if oracle.eigenvector_streak(V, U[:, :k], np.pi / 8) == k), None)
    V, t_orc = V0.copy(), None
    for t in range(1, cap + 1):
        V = oracle.oja_step(np.zeros_like(V), oracle.poly_limit(g, V, s, 251), 1.0)
        if t == 1:
            assert_close(gpu[0], V, 1e-10)
        if oracle.eigenvector_streak(V, U[:, :k], np.pi / 8) == k:
            t_orc = t
            break
    assert t_gpu is not None and t_orc is not None, (t_gpu, t_orc)
    assert abs(t_gpu - t_orc) <= 1, (t_gpu, t_orc)


def test_link_completed_cliques_plain_operator_leaves_them_unresolved(link_completed):
    # the plain reversed Laplacian lambda* I - L separates the four bottom eigenvalues (0 to
    # 0.15 against lambda* near 200) by factors within 1e-3 of 1 per step: after 300 steps the
    # streak is still 0, on the GPU as in the oracle's iteration, and the two iterations agree
    # entry by entry
    g, lam, U = link_completed
    k = 4
    G = sped.Graph.from_csr(g)
    ls = G.set_polynomial(sped.POLY_SHIFT, 1).lambda_star
    V0 = gen.gaussian_block(g.n, k, seed=31)
    steps = 300
    Vg = _gpu_oja_run(G, V0, k, steps)[-1]
    V = V0.copy()
    for _ in range(steps):
        V = oracle.oja_step(np.zeros_like(V), ls * V - oracle.laplacian_apply(g, V), 1.0)
    assert oracle.eigenvector_streak(V, U[:, :k], np.pi / 8) == 0
    assert oracle.eigenvector_streak(Vg, U[:, :k], np.pi / 8) == 0
    assert_close(Vg, V, 1e-8)
