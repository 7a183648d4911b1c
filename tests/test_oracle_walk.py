"""Pins for the oracle's stochastic estimator (Section 4.3, Eq. walk_summand, Table 1) and its
random-number specification."""
import os

import numpy as np
import pytest

import gen
import oracle

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    for line in open(os.path.join(GOLD, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        x = [int(t, 16) for t in line.split()]
        assert oracle.philox4x32_10(x[:4], x[4:6]) == x[6:]


def test_lemire_bounded_draws():
    d = oracle.bounded_draws(123, 7, 0, 5, 1, 100)
    assert np.all(d == 0)
    d = oracle.bounded_draws(123, 7, 0, 5, 7, 70000)
    assert d.max() < 7
    counts = np.bincount(d, minlength=7)
    chi2 = float(np.sum((counts - 10000.0) ** 2 / 10000.0))
    assert chi2 < 30.0  # 6 dof, p ~ 4e-5
    # without a rejection the draw is floor(x * r / 2^32) of the stream's first word
    w = oracle.philox4x32_10([9, 0, 3, 0], [42, 0])[0]
    r = 1000
    if (w * r) & 0xFFFFFFFF >= (2 ** 32 - r) % r:
        assert oracle.bounded_draws(42, 9, 0, 3, r, 1)[0] == (w * r) >> 32


def test_table1_inner_products():
    for line in open(os.path.join(GOLD, "table1_incidence.txt")):
        if line.startswith("#") or not line.strip():
            continue
        name, a1, b1, a2, b2, val = line.split()
        got = oracle.incidence_dot((int(a1), int(b1)), (int(a2), int(b2)))
        assert got == float(val), name
        # edge direction is set by node numbers, not by argument order
        assert oracle.incidence_dot((int(b1), int(a1)), (int(b2), int(a2))) == float(val)
    # weighted rows scale by sqrt(w_e w_f)
    assert oracle.incidence_dot((0, 1), (1, 2), 4.0, 9.0) == pytest.approx(-6.0)


def test_incidence_degree():
    # footnote of Section 4.3: every node of the edge-incidence graph has a self loop, so
    # deg_inc(e) = deg(i) + deg(j) - 1 <= 2 deg* - 1
    g = gen.random_graph(40, 120, seed=3, hub=0, hub_degree=20)
    X = oracle.incidence_matrix(g)
    Gm = X @ X.T
    a, b, _ = oracle.edge_list(g)
    deg = np.diff(g.row_ptr)
    counts = np.sum(np.abs(Gm) > 1e-12, axis=1)
    assert np.array_equal(counts, deg[a] + deg[b] - 1)
    assert counts.max() <= 2 * deg.max() - 1


TINY = [
    ("path4", lambda: gen.path(4)),
    ("star4", lambda: gen.star(4)),
    ("tri_tail", lambda: gen.from_edges(5, [0, 1, 0, 2, 3], [1, 2, 2, 3, 4])),
    ("w_path5", lambda: gen.uniform_edge_weights(gen.path(5), seed=3)),
    ("w_tri_tail", lambda: gen.uniform_edge_weights(
        gen.from_edges(5, [0, 1, 0, 2, 3, 1], [1, 2, 2, 3, 4, 4]), seed=4)),
]


@pytest.mark.parametrize("name,make", TINY)
@pytest.mark.parametrize("ell", [1, 2, 3, 4])
def test_exhaustive_expectation_equals_exact(name, make, ell):
    # Eq. walk_summand: summing alpha_c x_e1 x_el^T over all chains of the walk gives L^l
    g = make()
    assert g.n_edges <= 6
    V = np.random.default_rng(ell).standard_normal((g.n, 3))
    c = np.array([0.7, -0.5, 0.3, -0.2, 0.1][: ell + 1])
    assert np.allclose(oracle.walk_expectation_exhaustive(g, V, c),
                       oracle.walk_exact_terms(g, V, c), atol=1e-12)


def test_single_edge_walk_is_exact():
    # one edge: the incidence graph is one node with a self loop, every walk is the same,
    # so any single walker returns p(L) V exactly
    g = gen.uniform_edge_weights(gen.from_edges(3, [0], [2]), seed=1)
    V = np.random.default_rng(0).standard_normal((3, 4))
    c = np.array([0.3, -1.0, 0.5, -0.25, 0.125])
    for mode in (1, 2):
        got = oracle.walk_estimate(g, V, c, walkers=1, seed=99, mode=mode)
        assert np.allclose(got, oracle.walk_exact_terms(g, V, c), atol=1e-13)


@pytest.mark.parametrize("mode", [1, 2])
def test_sample_mean_converges(mode):
    # unbiasedness (Section 4.3): batch means of independent seeds agree with the exact
    # value within 5 standard errors per entry
    g = gen.from_edges(6, [0, 1, 2, 3, 0, 1], [1, 2, 3, 4, 2, 5])
    V = np.random.default_rng(5).standard_normal((g.n, 2))
    c = oracle.limit_power_coeffs(0.15, 3)
    exact = oracle.walk_exact_terms(g, V, c)
    B, M = 24, 4000
    est = np.stack([oracle.walk_estimate(g, V, c, M, seed=1000 + b, mode=mode) for b in range(B)])
    mean = est.mean(axis=0)
    se = est.std(axis=0, ddof=1) / np.sqrt(B)
    assert np.all(np.abs(mean - exact) <= 5 * se + 1e-9)
    # and the error shrinks like 1/sqrt(M): one big run is closer than one small run on average
    big = oracle.walk_estimate(g, V, c, 200000, seed=7, mode=mode)
    assert np.linalg.norm(big - exact) < 0.5 * np.mean(
        [np.linalg.norm(e - exact) for e in est])


def test_walk_deterministic_in_seed():
    g = gen.random_graph(30, 80, seed=2)
    V = np.random.default_rng(1).standard_normal((g.n, 3))
    c = oracle.limit_power_coeffs(0.05, 5)
    a = oracle.walk_estimate(g, V, c, 500, seed=11)
    b = oracle.walk_estimate(g, V, c, 500, seed=11)
    d = oracle.walk_estimate(g, V, c, 500, seed=12)
    assert np.array_equal(a, b) and not np.array_equal(a, d)


def _enumerate_chains(g, V, coeffs):
    """Every chain (e_1, ..., e_l) of the edge-incidence walk of Section 4.3 (e_1 uniform over
    the edges, each next edge uniform over the deg(a) + deg(b) - 1 edges incident to the
    current one, itself included), with, per prefix i: its probability q_i, the product alpha_i
    of Table 1 inner products along it, and the summand c_i alpha_i x_e1 (x_ei^T V) of Eq.
    walk_summand (n x k)."""
    a, b, w = oracle.edge_list(g)
    E = len(a)
    ell = len(coeffs) - 1
    nb = [list(g.col_idx[g.row_ptr[r]:g.row_ptr[r + 1]]) for r in range(g.n)]
    eid = {(int(a[e]), int(b[e])): e for e in range(E)}

    def incident(e):
        x, y = int(a[e]), int(b[e])
        return sorted({eid[(min(x, z), max(x, z))] for z in nb[x]} |
                      {eid[(min(y, z), max(y, z))] for z in nb[y]})

    def xvec(e):
        v = np.zeros(g.n)
        v[a[e]], v[b[e]] = np.sqrt(w[e]), -np.sqrt(w[e])
        return v

    out = []

    def rec(chain, q, alpha, terms, qs):
        e1, ei = chain[0], chain[-1]
        i = len(chain)
        terms = terms + [coeffs[i] * alpha * np.outer(xvec(e1), xvec(ei) @ V)]
        qs = qs + [q]
        if i == ell:
            out.append((tuple(chain), q, terms, qs))
            return
        nxt = incident(ei)
        for f in nxt:
            rec(chain + [f], q / len(nxt), alpha * float(xvec(ei) @ xvec(f)), terms, qs)

    for e in range(E):
        rec([e], 1.0 / E, 1.0, [], [])
    return out


WALK_GRAPHS = [
    ("w_tri_tail", lambda: gen.uniform_edge_weights(
        gen.from_edges(5, [0, 1, 0, 2, 3, 1], [1, 2, 2, 3, 4, 4]), seed=4)),
    ("w_star_path", lambda: gen.uniform_edge_weights(
        gen.from_edges(6, [0, 0, 0, 3, 4], [1, 2, 3, 4, 5]), seed=8)),
]


@pytest.mark.parametrize("name,make", WALK_GRAPHS)
def test_each_importance_weighted_walk_is_one_chains_estimate(name, make):
    # one walker per seed: the estimator's output minus c_0 V must be, to rounding, the
    # Horvitz-Thompson estimate sum_i c_i alpha_i / q_i x_e1 (x_ei^T V) of one chain of the walk
    # (Eq. walk_summand with the prefix probabilities q_i of the enumeration); a wrong 1/q_i,
    # alpha or edge weight on any branch gives an output that matches no chain. The chains the
    # walkers took are recovered this way, and their frequencies follow the enumeration's
    # probabilities (chi-square).
    g = make()
    ell = 4
    c = np.array([0.4, -0.9, 0.7, -0.45, 0.3])
    V = np.random.default_rng(21).standard_normal((g.n, 3))
    chains = _enumerate_chains(g, V, c)
    est = np.stack([sum(t / q for t, q in zip(terms, qs)).ravel()
                    for _, _, terms, qs in chains])
    scale = np.abs(est).max()
    seeds = 6000
    counts = np.zeros(len(chains))
    for s in range(seeds):
        D = (oracle.walk_estimate(g, V, c, walkers=1, seed=s, mode=1) - c[0] * V).ravel()
        dist = np.abs(est - D).max(axis=1)
        j = int(np.argmin(dist))
        assert dist[j] <= 1e-12 * scale, (s, dist[j])
        counts[j] += 1
    p = np.array([q for _, q, _, _ in chains])
    assert p.sum() == pytest.approx(1.0)
    # pool chains with small expected counts into one cell
    expect = seeds * p
    big = expect >= 5
    obs = np.append(counts[big], counts[~big].sum())
    exp = np.append(expect[big], expect[~big].sum())
    keep = exp > 0
    chi2 = float(np.sum((obs[keep] - exp[keep]) ** 2 / exp[keep]))
    dof = int(keep.sum()) - 1
    assert chi2 <= dof + 6.0 * np.sqrt(2.0 * dof), (chi2, dof)


@pytest.mark.parametrize("name,make", WALK_GRAPHS)
def test_each_rejection_walk_is_one_chains_accepted_prefixes(name, make):
    # the rejection variant: prefix i of the walk is kept with probability p_min,i / q_i,
    # p_min,i = |E|^-1 (2 deg* - 1)^-(i-1) (accepted, not rejected, with that probability: the
    # reading under which the kept prefixes are uniform), and a kept prefix contributes
    # c_i alpha_i / p_min,i x_e1 (x_ei^T V). Every single walk's output must equal that sum over
    # the kept prefixes of one chain; the first prefix is always kept (p_min,1 = q_1).
    g = make()
    ell = 3
    c = np.array([0.4, -0.9, 0.7, -0.45])
    V = np.random.default_rng(22).standard_normal((g.n, 3))
    deg = np.diff(g.row_ptr)
    dstar = int(deg.max())
    E = g.n_edges
    pmin = [1.0 / E * (2 * dstar - 1) ** -(i - 1) for i in range(1, ell + 1)]
    chains = _enumerate_chains(g, V, c)
    masks = [m for m in range(1 << ell) if m & 1]  # prefix 1 is always kept
    cand = []
    for ch, _, terms, qs in chains:
        for mask in masks:
            cand.append(sum(terms[i] / pmin[i] for i in range(ell) if mask >> i & 1).ravel())
        assert all(pm <= q * (1 + 1e-12) for pm, q in zip(pmin, qs))  # probabilities <= 1
    cand = np.stack(cand)
    scale = np.abs(cand).max()
    kept = np.zeros(ell)
    expect = np.zeros(ell)
    var = np.zeros(ell)
    for s in range(4000):
        D = (oracle.walk_estimate(g, V, c, walkers=1, seed=s, mode=2, deg_star=dstar)
             - c[0] * V).ravel()
        dist = np.abs(cand - D).max(axis=1)
        j = int(np.argmin(dist))
        assert dist[j] <= 1e-12 * scale, (s, dist[j])
        ch, mask = chains[j // len(masks)], masks[j % len(masks)]
        for i in range(ell):
            acc = pmin[i] / ch[3][i]
            kept[i] += mask >> i & 1
            expect[i] += acc
            var[i] += acc * (1.0 - acc)
    # prefix i of the recovered chains is kept as often as its acceptance probability says
    assert kept[0] == 4000
    assert np.all(np.abs(kept[1:] - expect[1:]) <= 5.0 * np.sqrt(var[1:])), (kept, expect)
    assert np.all(kept[1:] > 0)
