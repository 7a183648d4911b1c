"""FP64 CPU oracle for the SPED hot path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline / reference leg
may import this package. It never imports the CUDA package, and the CUDA package never
imports it; the two share only the seeded input generators in ``gen``.

Each function is the plain definition, or the paper's algorithm taken step by step, in FP64
(numpy / the C loops in ``sped_oracle.c``); library primitives (dense matmul, symmetric
eigendecomposition, QR, SVD) serve as single steps. Paper: van der Pol, Gemp, Bachrach,
Everett, "Stochastic Parallelizable Eigengap Dilation for Large Graph Clustering",
arXiv 2207.14589. Section, equation and table numbers below refer to it.

Pinned against the paper and the mathematics by ``tests/test_oracle_*.py`` (closed-form
spectra, L 1 = 0, the cut identity of Eq. 1, Table 1, exhaustive walk enumeration,
eigenvector preservation, finite differences, Philox known-answer vectors, exhaustive
enumeration of edge minibatches). Functions with
no such pin say "parity unpinned" in their docstring.
"""
from __future__ import annotations

import ctypes
import math
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    """Load (building first if needed) the C part of the oracle."""
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        i64, i32p, f32p, f64p = (ctypes.c_int64, ctypes.POINTER(ctypes.c_int32),
                                 ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_double))
        L.orc_laplacian_apply.argtypes = [i64, i32p, i32p, f32p, f64p, ctypes.c_int, f64p]
        L.orc_laplacian_apply.restype = None
        L.orc_degrees.argtypes = [i64, i32p, f32p, f64p]
        L.orc_degrees.restype = None
        L.orc_poly_limit.argtypes = [i64, i32p, i32p, f32p, f64p, ctypes.c_int, ctypes.c_double,
                                     ctypes.c_int, f64p]
        L.orc_poly_limit.restype = None
        L.orc_poly_horner.argtypes = [i64, i32p, i32p, f32p, f64p, ctypes.c_int, f64p,
                                      ctypes.c_int, ctypes.c_double, f64p]
        L.orc_poly_horner.restype = None
        L.orc_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32),
                                        ctypes.POINTER(ctypes.c_uint32),
                                        ctypes.POINTER(ctypes.c_uint32)]
        L.orc_philox4x32_10.restype = None
        L.orc_bounded_draws.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.c_uint32, i64,
                                        ctypes.POINTER(ctypes.c_uint32)]
        L.orc_bounded_draws.restype = None
        L.orc_first_draws.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                      ctypes.c_uint32, i64, ctypes.POINTER(ctypes.c_uint32)]
        L.orc_first_draws.restype = None
        i64p = ctypes.POINTER(ctypes.c_int64)
        L.orc_stratified_draws.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32,
                                           i64, i64, i64p, i64p]
        L.orc_stratified_draws.restype = None
        L.orc_incidence_dot.argtypes = [i64, i64, ctypes.c_double, i64, i64, ctypes.c_double]
        L.orc_incidence_dot.restype = ctypes.c_double
        L.orc_walk_estimate.argtypes = [i64, i32p, i32p, f32p, f64p, ctypes.c_int, f64p,
                                        ctypes.c_int, i64, ctypes.c_uint64, ctypes.c_int, i64,
                                        f64p]
        L.orc_walk_estimate.restype = ctypes.c_int
        _lib = L
    return _lib


def _p(a, ct):
    return a.ctypes.data_as(ctypes.POINTER(ct))


def _graph_args(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int32)
    ci = np.ascontiguousarray(g.col_idx, dtype=np.int32)
    w = None if g.w is None else np.ascontiguousarray(g.w, dtype=np.float32)
    wp = None if w is None else _p(w, ctypes.c_float)
    return rp, ci, w, wp


# ----------------------------------------------------------------------------------------
# Section 2: Laplacian, incidence matrix, degrees
# ----------------------------------------------------------------------------------------
def laplacian_apply(g, X):
    """Y = L X with L = D - A (Section 2), weighted L = X^T W X (end of Section 2.1)."""
    X = np.ascontiguousarray(X, dtype=np.float64)
    squeeze = X.ndim == 1
    if squeeze:
        X = X[:, None]
    k = X.shape[1]
    Y = np.empty_like(X)
    rp, ci, w, wp = _graph_args(g)
    lib().orc_laplacian_apply(g.n, _p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32), wp,
                              _p(X, ctypes.c_double), k, _p(Y, ctypes.c_double))
    return Y[:, 0] if squeeze else Y


def degrees(g):
    """Weighted degrees d_i = sum_j w_ij (Section 2.1)."""
    d = np.empty(g.n, dtype=np.float64)
    rp, ci, w, wp = _graph_args(g)
    lib().orc_degrees(g.n, _p(rp, ctypes.c_int32), wp, _p(d, ctypes.c_double))
    return d


def edge_list(g):
    """Undirected edges (a < b) in CSR order of row a, with weights (1 if unweighted)."""
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr.astype(np.int64)))
    cols = g.col_idx.astype(np.int64)
    up = rows < cols
    w = np.ones(int(up.sum())) if g.w is None else g.w[up].astype(np.float64)
    return rows[up], cols[up], w


def incidence_matrix(g):
    """Weighted incidence rows sqrt(w_e) x_e, x_e = +1 at min(i,j), -1 at max(i,j) (Section 2)."""
    a, b, w = edge_list(g)
    X = np.zeros((len(a), g.n))
    X[np.arange(len(a)), a] = np.sqrt(w)
    X[np.arange(len(a)), b] = -np.sqrt(w)
    return X


def dense_laplacian(g):
    """Dense D - A written out from the edge list (Section 2), for brute-force checks."""
    a, b, w = edge_list(g)
    L = np.zeros((g.n, g.n))
    for i, j, x in zip(a, b, w):
        L[i, j] -= x
        L[j, i] -= x
        L[i, i] += x
        L[j, j] += x
    return L


def cut_value(g, v):
    """Eq. 1: sum over undirected edges of w_e (v_i - v_j)^2."""
    a, b, w = edge_list(g)
    return float(np.sum(w * (v[a] - v[b]) ** 2))


def incidence_dot(e1, e2, w1=1.0, w2=1.0):
    """<sqrt(w1) x_e1, sqrt(w2) x_e2> following Table 1."""
    return lib().orc_incidence_dot(e1[0], e1[1], w1, e2[0], e2[1], w2)


def gershgorin_bound(g):
    """lambda_max <= 2 max_i d_i (the spectral-radius bound quoted in Section 5.4)."""
    return 2.0 * float(degrees(g).max()) if g.n else 0.0


# ----------------------------------------------------------------------------------------
# Sections 4.1-4.2, Table 2: eigenvector-preserving polynomials
# ----------------------------------------------------------------------------------------
def poly_limit(g, V, s, ell):
    """(I - sL)^ell V by ell explicit steps (Table 2 limit row; s = 1/ell is the table's)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    squeeze = V.ndim == 1
    if squeeze:
        V = V[:, None]
    Y = np.empty_like(V)
    rp, ci, w, wp = _graph_args(g)
    lib().orc_poly_limit(g.n, _p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32), wp,
                         _p(V, ctypes.c_double), V.shape[1], float(s), int(ell),
                         _p(Y, ctypes.c_double))
    return Y[:, 0] if squeeze else Y


def poly_horner(g, V, coeffs, shift=0.0):
    """sum_j c_j (L + shift I)^j V by Horner's rule (Table 2 Taylor rows)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    squeeze = V.ndim == 1
    if squeeze:
        V = V[:, None]
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    Y = np.empty_like(V)
    rp, ci, w, wp = _graph_args(g)
    lib().orc_poly_horner(g.n, _p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32), wp,
                          _p(V, ctypes.c_double), V.shape[1], _p(c, ctypes.c_double),
                          len(c) - 1, float(shift), _p(Y, ctypes.c_double))
    return Y[:, 0] if squeeze else Y


def limit_scalar(lam, s, ell):
    """Scalar transform of the limit form: p(lambda) = (1 - s lambda)^ell."""
    return (1.0 - s * np.asarray(lam, dtype=np.float64)) ** ell


def poly_chebyshev(g, V, coeffs, a, b):
    """sum_j c_j T_j(x) V with x = (2 L - (a + b) I) / (b - a), the Chebyshev polynomials of
    the first kind by their three-term recurrence (T_0 = 1, T_1 = x, T_{j+1} = 2 x T_j -
    T_{j-1}); [a, b] is the interval mapped onto [-1, 1]."""
    V = np.asarray(V, dtype=np.float64)
    c = np.asarray(coeffs, dtype=np.float64)
    al, be = 2.0 / (b - a), -(a + b) / (b - a)

    def X(Z):
        return al * laplacian_apply(g, Z) + be * Z
    T0 = V
    Y = c[0] * T0
    if len(c) > 1:
        T1 = X(V)
        Y = Y + c[1] * T1
        for j in range(1, len(c) - 1):
            T2 = 2.0 * X(T1) - T0
            Y = Y + c[j + 1] * T2
            T0, T1 = T1, T2
    return Y


def chebyshev_scalar(coeffs, x):
    """sum_j c_j T_j(x) for real x by the closed forms T_j = cos(j arccos x) on [-1, 1] and
    cosh(j arccosh |x|) (times (-1)^j for x < -1) outside."""
    x = np.asarray(x, dtype=np.float64)
    out = np.zeros_like(x)
    for j, cj in enumerate(coeffs):
        inside = np.abs(x) <= 1.0
        t = np.empty_like(x)
        t[inside] = np.cos(j * np.arccos(x[inside]))
        ax = np.abs(x[~inside])
        t[~inside] = np.cosh(j * np.arccosh(ax)) * np.where(x[~inside] < 0, (-1.0) ** j, 1.0)
        out += cj * t
    return out


def taylor_exp_coeffs(ell):
    """Reversed Taylor -e^{-L} of Table 2 (lambda* = 0, Section 4.2): M = sum_i (-L)^i / i!."""
    return np.array([(-1.0) ** i / math.factorial(i) for i in range(ell + 1)])


def taylor_log_coeffs(ell):
    """Taylor log(L + eps I) of Table 2 in powers of T = L + (eps - 1) I:
    c_0 = 0, c_i = (-1)^{i+1} / i."""
    return np.array([0.0] + [(-1.0) ** (i + 1) / i for i in range(1, ell + 1)])


def limit_power_coeffs(s, ell):
    """Power-basis coefficients of (1 - s L)^ell: c_i = C(ell, i) (-s)^i."""
    return np.array([math.comb(ell, i) * (-s) ** i for i in range(ell + 1)])


def scale_rule(lam_bound, ell):
    """Step scale for the limit form when the caller gives none: s = 1/ell when
    ell >= lam_bound / 2 (so |1 - s lambda| <= 1 on [0, lam_bound]), else s = 2 / lam_bound.
    The paper fixes s = 1/ell (Table 2) and explains the failures at small ell by the
    spectral radius (Section 5.4, Appendix A.2); this reading keeps the map contractive."""
    if lam_bound <= 0:
        return 1.0 / ell
    return 1.0 / ell if ell >= lam_bound / 2.0 else 2.0 / lam_bound


def poly_moments(g, V, n_moments, basis="chebyshev", a=0.0, b=1.0):
    """Block moments Omega_l = V^T B_l V (k x k), l = 0..n_moments-1, of the power basis
    B_l = L^l or the Chebyshev basis B_l = T_l(x), x = (2L - (a + b) I) / (b - a) (three-term
    recurrence). For M = sum_l c_l B_l they give V^T M V = sum_l c_l Omega_l, the quantity a fit
    of the coefficients (the meta-learning the paper leaves to future work, Section 6) works
    on."""
    V = np.asarray(V, dtype=np.float64)
    out = []
    if basis == "power":
        X = V
        for _ in range(n_moments):
            out.append(V.T @ X)
            X = laplacian_apply(g, X)
        return np.stack(out)
    al, be = 2.0 / (b - a), -(a + b) / (b - a)
    T0, T1 = V, None
    for l in range(n_moments):
        if l == 0:
            T = V
        elif l == 1:
            T1 = al * laplacian_apply(g, V) + be * V
            T = T1
        else:
            T2 = 2.0 * (al * laplacian_apply(g, T1) + be * T1) - T0
            T0, T1 = T1, T2
            T = T2
        out.append(V.T @ T)
    return np.stack(out)


# ----------------------------------------------------------------------------------------
# Section 4.3: stochastic estimate over sampled walks
# ----------------------------------------------------------------------------------------
def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(x) & 0xFFFFFFFF for x in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(x) & 0xFFFFFFFF for x in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return [int(x) for x in o]


def bounded_draws(seed, a, b, tag, rng_range, count):
    out = np.empty(count, dtype=np.uint32)
    lib().orc_bounded_draws(seed, a, b, tag, rng_range, count, _p(out, ctypes.c_uint32))
    return out


def walk_estimate(g, V, coeffs, walkers, seed, mode=1, deg_star=None):
    """Unbiased estimate of sum_i c_i L^i V from ``walkers`` walks (Section 4.3).

    mode 1: importance weights 1/q_i; mode 2: the text's rejection step with
    deg*_inc = 2 deg* - 1 (deg* defaults to the maximum count degree)."""
    V = np.ascontiguousarray(V, dtype=np.float64)
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    if deg_star is None:
        deg_star = int(np.diff(g.row_ptr).max()) if g.n else 1
    Y = np.empty_like(V)
    rp, ci, w, wp = _graph_args(g)
    rc = lib().orc_walk_estimate(g.n, _p(rp, ctypes.c_int32), _p(ci, ctypes.c_int32), wp,
                                 _p(V, ctypes.c_double), V.shape[1], _p(c, ctypes.c_double),
                                 len(c) - 1, int(walkers), int(seed), int(mode), int(deg_star),
                                 _p(Y, ctypes.c_double))
    if rc:
        raise ValueError("walk_estimate: bad arguments")
    return Y


def walk_expectation_exhaustive(g, V, coeffs):
    """E[walk estimate] by enumerating every chain of the edge-incidence walk with its
    probability (tiny graphs only): sum over chains of q(chain) * estimate(chain).

    Independent of the C estimator: it follows Eq. walk_summand and the walk's transition
    rule (uniform over the deg(a)+deg(b)-1 incident edges, self loop included) directly."""
    a, b, w = edge_list(g)
    E = len(a)
    ell = len(coeffs) - 1
    V = np.asarray(V, dtype=np.float64)
    nb = [list(g.col_idx[g.row_ptr[r]:g.row_ptr[r + 1]]) for r in range(g.n)]
    eid = {(int(a[e]), int(b[e])): e for e in range(E)}
    Y = coeffs[0] * V.copy()
    if ell == 0 or E == 0:
        return Y

    def incident(e):
        x, y = int(a[e]), int(b[e])
        out = [eid[(min(x, z), max(x, z))] for z in nb[x]]
        out += [eid[(min(y, z), max(y, z))] for z in nb[y] if z != x]
        return out

    def xvec(e):
        v = np.zeros(g.n)
        v[a[e]] = math.sqrt(w[e])
        v[b[e]] = -math.sqrt(w[e])
        return v

    deg = np.diff(g.row_ptr.astype(np.int64))

    def rec(chain, prob, inv_q, alpha):
        # prob: probability of this prefix under the walk (from the enumeration itself);
        # inv_q: the estimator's importance weight |E| prod deg_inc(e_t), deg_inc = deg a +
        # deg b - 1 (Section 4.3); a wrong degree formula breaks prob * inv_q = 1.
        i = len(chain)
        e1, ei = chain[0], chain[-1]
        term = coeffs[i] * alpha * inv_q * np.outer(xvec(e1), xvec(ei) @ V)
        Y[:] += prob * term
        if i == ell:
            return
        nxt = incident(ei)
        deg_inc = int(deg[a[ei]] + deg[b[ei]] - 1)
        for f in nxt:
            dot = float(xvec(ei) @ xvec(f))
            rec(chain + [f], prob / len(nxt), inv_q * deg_inc, alpha * dot)

    for e in range(E):
        rec([e], 1.0 / E, float(E), 1.0)
    return Y


def walk_exact_terms(g, V, coeffs):
    """sum_i c_i L^i V by repeated Laplacian application (the target of the estimator)."""
    out = coeffs[0] * np.asarray(V, dtype=np.float64)
    X = np.asarray(V, dtype=np.float64)
    for i in range(1, len(coeffs)):
        X = laplacian_apply(g, X)
        out = out + coeffs[i] * X
    return out


# ----------------------------------------------------------------------------------------
# Sections 2, 4.3 and 6: edges fed in minibatches (the stochastic optimisation model)
# ----------------------------------------------------------------------------------------
MINIBATCH_TAG = 0x4D42


def minibatch_edge_ids(n_edges, seed, step, batch):
    """Edge ids of the minibatch of chain multiplication ``step``: ``batch`` independent
    uniform draws from [0, |E|) (with replacement); draw j is the first bounded draw of the
    word stream keyed by ``seed`` with counter words (j, step, MINIBATCH_TAG)."""
    out = np.empty(int(batch), dtype=np.uint32)
    if batch > 0:
        lib().orc_first_draws(int(seed), int(step), MINIBATCH_TAG, int(n_edges), int(batch),
                              _p(out, ctypes.c_uint32))
    return out.astype(np.int64)


def stratified_edge_ids(n_edges, seed, step, batch):
    """Variance-reduced minibatch (the paper leaves variance reduction to future work, Section
    6): the edge ids are cut into ``batch`` contiguous strata S_j = [floor(j|E|/B),
    floor((j+1)|E|/B)) and draw j is uniform in S_j (first bounded draw over |S_j| of the
    stream (seed; j, step, MINIBATCH_TAG)). Returns (ids, |S_j|); an empty stratum (B > |E|)
    gives id -1 and size 0."""
    ids = np.empty(int(batch), dtype=np.int64)
    sizes = np.empty(int(batch), dtype=np.int64)
    if batch > 0:
        lib().orc_stratified_draws(int(seed), int(step), MINIBATCH_TAG, int(n_edges), int(batch),
                                   _p(ids, ctypes.c_int64), _p(sizes, ctypes.c_int64))
    return ids, sizes


def minibatch_edges(g, seed, step, batch):
    """The sampled edges (a_j < b_j, weight w_j) of that minibatch, edges numbered as in
    ``edge_list`` (the CSR order of their upper entries)."""
    a, b, w = edge_list(g)
    ids = minibatch_edge_ids(len(a), seed, step, batch)
    return a[ids], b[ids], w[ids]


def minibatch_laplacian_apply(n_edges, X, a, b, w):
    """L_hat X for one edge sample: L_hat = (|E| / B) sum_j w_j x_j x_j^T with x_j = e_{a_j} -
    e_{b_j}. The Laplacian is the sum of the edges' outer products (Section 4.3, weighted as
    at the end of Section 2.1), and each draw picks an edge with probability 1/|E|, so
    E[L_hat] = L."""
    X = np.asarray(X, dtype=np.float64)
    B = len(a)
    if B < 1:
        raise ValueError("minibatch of no edges")
    d = (X[a] - X[b]) * (np.asarray(w, dtype=np.float64) * (n_edges / B))[:, None]
    Y = np.zeros_like(X)
    np.add.at(Y, a, d)
    np.add.at(Y, b, -d)
    return Y


def stratified_laplacian_apply(X, a, b, w, sizes):
    """L_hat X for a stratified sample: L_hat = sum_j |S_j| w_j x_j x_j^T (draw j stands for its
    stratum: each edge of S_j is drawn with probability 1/|S_j|, so E[L_hat] = L)."""
    X = np.asarray(X, dtype=np.float64)
    d = (X[a] - X[b]) * (np.asarray(w, dtype=np.float64) * sizes)[:, None]
    Y = np.zeros_like(X)
    np.add.at(Y, a, d)
    np.add.at(Y, b, -d)
    return Y


def minibatch_operator(g, seed, batch, stratified=False):
    """(t, X) -> L_hat_t X, each multiplication t with the minibatch drawn for it (uniform
    draws, or one draw per stratum of the edge order)."""
    a, b, w = edge_list(g)
    m = len(a)

    def apply(t, X):
        if stratified:
            ids, sizes = stratified_edge_ids(m, seed, t, batch)
            keep = sizes > 0
            ids, sizes = ids[keep], sizes[keep]
            return stratified_laplacian_apply(X, a[ids], b[ids], w[ids], sizes.astype(np.float64))
        ids = minibatch_edge_ids(m, seed, t, batch)
        return minibatch_laplacian_apply(m, X, a[ids], b[ids], w[ids])
    return apply


def stochastic_limit(V, s, ell, Lhat):
    """(I - sL)^ell V with factor t (t = 0 applied first) replaced by I - s L_hat_t. With the
    factors' samples independent, the expectation of the product is the product of the
    expectations: (I - sL)^ell V (Table 2 limit row)."""
    Z = np.array(V, dtype=np.float64)
    for t in range(ell):
        Z = Z - s * Lhat(t, Z)
    return Z


def stochastic_horner(V, h, shift, Lhat):
    """sum_j h_j (L + shift I)^j V by Horner's rule (Z = h_l V; Z <- h_j V + (L + shift I) Z for
    j = l-1..0), the t-th multiplication (evaluation order) by L_hat_t + shift I. Each
    multiplication is independent of the Z it multiplies, so the result is unbiased."""
    V = np.asarray(V, dtype=np.float64)
    ell = len(h) - 1
    Z = h[ell] * V
    for t, j in enumerate(range(ell - 1, -1, -1)):
        Z = h[j] * V + Lhat(t, Z) + shift * Z
    return Z


def stochastic_clenshaw(V, c, a, b, Lhat):
    """sum_j c_j T_j(x) V, x = (2 L - (a + b) I) / (b - a), by Clenshaw's recurrence
    (b_{l+1} = b_{l+2} = 0, b_j = c_j V + 2 x b_{j+1} - b_{j+2}, result c_0 V + x b_1 - b_2),
    the t-th multiplication by x (evaluation order) using L_hat_t."""
    V = np.asarray(V, dtype=np.float64)
    ell = len(c) - 1
    al, be = 2.0 / (b - a), -(a + b) / (b - a)
    t = 0

    def x(Z):
        nonlocal t
        out = al * Lhat(t, Z) + be * Z
        t += 1
        return out
    b1, b2 = c[ell] * V, np.zeros_like(V)
    for j in range(ell - 1, 0, -1):
        b1, b2 = c[j] * V + 2.0 * x(b1) - b2, b1
    return c[0] * V + x(b1) - b2


# ----------------------------------------------------------------------------------------
# Section 3 / Section 5.1: solvers (mu-EG and Oja), Section 5.2: metrics
# ----------------------------------------------------------------------------------------
def mu_eg_step(V, Y, eta):
    """One parallel mu-EG step (EigenGame Unloaded, the solver of Section 5.1; the update is
    cited there, not restated). For every player i, with y = M v:
      delta_i = y_i - sum_{j<i} <v_i, y_j> v_j      (unloaded penalty)
      r_i     = delta_i - <v_i, delta_i> v_i         (Riemannian projection)
      v_i    <- (v_i + eta r_i) / ||v_i + eta r_i||
    All players read the same V and Y."""
    V = np.asarray(V, dtype=np.float64)
    Y = np.asarray(Y, dtype=np.float64)
    k = V.shape[1]
    out = np.empty_like(V)
    for i in range(k):
        delta = Y[:, i].copy()
        for j in range(i):
            delta -= float(V[:, i] @ Y[:, j]) * V[:, j]
        r = delta - float(V[:, i] @ delta) * V[:, i]
        u = V[:, i] + eta * r
        out[:, i] = u / np.linalg.norm(u)
    return out


def oja_step(V, Y, eta):
    """Oja / subspace step: V <- orth(V + eta M V), orthonormalised by QR with a positive
    diagonal of R (Section 5.1 names Oja's algorithm; this is its block form)."""
    W = np.asarray(V, dtype=np.float64) + eta * np.asarray(Y, dtype=np.float64)
    Q, R = np.linalg.qr(W)
    sgn = np.sign(np.diag(R))
    sgn[sgn == 0] = 1.0
    return Q * sgn


def ritz_values(V, Y):
    """Rayleigh quotients <v_i, M v_i> / <v_i, v_i>."""
    return np.einsum("ni,ni->i", V, Y) / np.einsum("ni,ni->i", V, V)


def rayleigh_ritz(g, V):
    """Ritz pairs of L on span(V) (the Rayleigh-Ritz procedure): with R the upper Cholesky
    factor of V^T V (so Q = V R^{-1} is an orthonormal basis of span(V)), the eigenpairs
    (theta_i, z_i) of the symmetric k x k matrix Q^T L Q = R^{-T} (V^T L V) R^{-1}, theta
    ascending. Returns theta and W = R^{-1} Z, so that the Ritz vectors are the columns of V W
    (orthonormal)."""
    V = np.asarray(V, dtype=np.float64)
    P = V.T @ V
    H = V.T @ laplacian_apply(g, V)
    R = np.linalg.cholesky(P).T
    Ri = np.linalg.solve(R, np.eye(R.shape[0]))
    Hs = Ri.T @ H @ Ri
    theta, Z = np.linalg.eigh(0.5 * (Hs + Hs.T))
    return theta, Ri @ Z


def bottom_k(g, k):
    """Ground truth by dense symmetric eigendecomposition of D - A (small graphs)."""
    lam, U = np.linalg.eigh(dense_laplacian(g))
    return lam[:k], U[:, :k]


def orthonormal_basis(V):
    Q, _ = np.linalg.qr(np.asarray(V, dtype=np.float64))
    return Q


def principal_angle_max(A, B):
    """Largest principal angle between span(A) and span(B), in sine form
    arcsin ||(I - Q_A Q_A^T) Q_B||_2 (accurate near zero)."""
    Qa, Qb = orthonormal_basis(A), orthonormal_basis(B)
    R = Qb - Qa @ (Qa.T @ Qb)
    s = np.linalg.norm(R, 2)
    return float(np.arcsin(min(1.0, s)))


def subspace_error(Ustar, V):
    """Section 5.2: delta = 1 - tr(U* P)/k, U* and P the orthogonal projectors onto the
    true and the estimated subspace (P = V V^dagger)."""
    Qs, Qv = orthonormal_basis(Ustar), orthonormal_basis(V)
    k = Qs.shape[1]
    return float(1.0 - np.linalg.norm(Qs.T @ Qv, "fro") ** 2 / k)


def eigenvector_streak(V, Vstar, eps):
    """Section 5.2: length of the leading run of columns whose angle to the matching true
    eigenvector is at most eps (sign ignored)."""
    n = 0
    for i in range(V.shape[1]):
        v = V[:, i] / np.linalg.norm(V[:, i])
        u = Vstar[:, i] / np.linalg.norm(Vstar[:, i])
        s = np.linalg.norm(v - (v @ u) * u)
        if np.arcsin(min(1.0, s)) <= eps:
            n += 1
        else:
            break
    return n


# ----------------------------------------------------------------------------------------
# differentiable utilities (EigenGame alpha-utilities under M = p(L))
# ----------------------------------------------------------------------------------------
def eg_utilities(V, Y):
    """u_i = <v_i, M v_i> - sum_{j<i} <v_i, M v_j>^2 / <v_j, M v_j>, with Y = M V."""
    H = V.T @ Y
    k = H.shape[0]
    return np.array([H[i, i] - sum(H[i, j] ** 2 / H[j, j] for j in range(i))
                     for i in range(k)])


def eg_utility_hbar(H, g_u):
    """d(sum_i g_i u_i)/dH_ij, treating every entry H_ij = <v_i, M v_j> as independent."""
    k = H.shape[0]
    Hb = np.zeros((k, k))
    for i in range(k):
        Hb[i, i] += g_u[i]
        for j in range(i):
            Hb[i, j] += -2.0 * g_u[i] * H[i, j] / H[j, j]
            Hb[j, j] += g_u[i] * H[i, j] ** 2 / H[j, j] ** 2
    return Hb


def eg_grad_full(V, Y, g_u):
    """Full gradient of sum_i g_i u_i w.r.t. V: Y Hbar^T + M (V Hbar) = Y (Hbar + Hbar^T)."""
    Hb = eg_utility_hbar(V.T @ Y, g_u)
    return Y @ (Hb + Hb.T)


def eg_grad_detached(V, Y):
    """Per-player gradient with parents held fixed (the EigenGame update direction):
    du_i/dv_i = 2 M v_i - 2 sum_{j<i} (<v_i, M v_j> / <v_j, M v_j>) M v_j."""
    H = V.T @ Y
    k = H.shape[0]
    G = np.empty_like(V)
    for i in range(k):
        gi = 2.0 * Y[:, i]
        for j in range(i):
            gi -= 2.0 * H[i, j] / H[j, j] * Y[:, j]
        G[:, i] = gi
    return G


def limit_edge_grad(g, V, s, ell, Hbar):
    """d f / d w_e for f(H), H = V^T B^ell V, B = I - sL (limit form), with V fixed:
    dB/dw_e = -s x_e x_e^T (L = sum_e w_e x_e x_e^T, Section 2.1), hence
    df/dw_e = -s sum_{t=0}^{ell-1} (x_e^T B^t V) Hbar (x_e^T B^{ell-1-t} V)^T.
    All B^t V are stored (tiny graphs only)."""
    a, b, _ = edge_list(g)
    A = [np.asarray(V, dtype=np.float64)]
    for _ in range(ell - 1):
        A.append(poly_limit(g, A[-1], s, 1))
    grad = np.zeros(len(a))
    for t in range(ell):
        P = A[t][a] - A[t][b]
        Q = A[ell - 1 - t][a] - A[ell - 1 - t][b]
        grad += -s * np.einsum("ei,ij,ej->e", P, Hbar, Q)
    return grad


def with_edge_weights(g, w_edge):
    """Same graph with the undirected-edge weights w_edge (CSR order of upper entries)."""
    import copy
    a, b, _ = edge_list(g)
    rows = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(g.row_ptr.astype(np.int64)))
    cols = g.col_idx.astype(np.int64)
    lookup = {(int(x), int(y)): float(z) for x, y, z in zip(a, b, w_edge)}
    w = np.array([lookup[(min(r, c), max(r, c))] for r, c in zip(rows, cols)], dtype=np.float32)
    h = copy.copy(g)
    h.w = w
    return h


# ----------------------------------------------------------------------------------------
# Sections 1 and 2.1: hard clustering by k-means on the rows of the eigenvector block
# ----------------------------------------------------------------------------------------
def _sqdist(P, C):
    """Squared distances sum_d (p_d - c_d)^2, accumulated in dimension order."""
    out = np.zeros((P.shape[0], C.shape[0]))
    for t in range(P.shape[1]):
        out += (P[:, t][:, None] - C[None, :, t]) ** 2
    return out


def kmeanspp_seeds(X, n_clusters, seed):
    """k-means++ seeding (Arthur and Vassilvitskii, 2007): the first centre uniform over the
    rows, every further centre drawn with probability proportional to the squared distance
    D^2(x) to the nearest centre chosen so far. Draws from Philox4x32-10 with key (seed) and
    counter (c, 0, 0, 0x6B6D) for the c-th centre: centre 0 is a bounded draw in [0, n);
    centre c >= 1 is the first row whose running sum of D^2 exceeds u * total,
    u = (word + 0.5) 2^-32. Returns the row indices of the centres."""
    X = np.asarray(X, dtype=np.float64)
    n = X.shape[0]
    picks = [int(bounded_draws(seed, 0, 0, 0x6B6D, n, 1)[0])]
    D2 = _sqdist(X, X[picks[0]][None, :])[:, 0]
    for c in range(1, n_clusters):
        word = philox4x32_10([c, 0, 0, 0x6B6D], [seed & 0xFFFFFFFF, seed >> 32])[0]
        u = (word + 0.5) * 2.0 ** -32
        cum = 0.0
        total = float(np.sum(D2))
        pick = n - 1
        target = u * total
        for i in range(n):
            cum += D2[i]
            if cum > target:
                pick = i
                break
        picks.append(pick)
        D2 = np.minimum(D2, _sqdist(X, X[pick][None, :])[:, 0])
    return picks


def kmeans(X, n_clusters, seed, max_iter=100):
    """k-means++ seeding (kmeanspp_seeds) then Lloyd iterations until the labels stop changing.

    The paper only says k-means on the embedding (Section 1, Section 2.1). Readings:
    distances are sum_d (x_d - m_d)^2 in dimension order; ties go to the lowest centroid;
    an empty cluster is re-seeded with the point farthest from its centroid (lowest index);
    labels are renumbered by first occurrence in row order. Pinned by separated clusters
    (exact labels), brute force over all partitions of tiny sets, and the seeding's
    distribution and forced choices (tests/test_oracle_solver.py)."""
    X = np.asarray(X, dtype=np.float64)
    n, d = X.shape
    K = n_clusters
    sqdist = _sqdist
    centers = X[kmeanspp_seeds(X, K, seed)].copy()
    labels = None
    for _ in range(max_iter):
        dist = sqdist(X, centers)
        new = np.argmin(dist, axis=1)
        if labels is not None and np.array_equal(new, labels):
            break
        labels = new
        for c in range(K):
            m = labels == c
            if m.any():
                centers[c] = X[m].mean(axis=0)
            else:
                far = dist[np.arange(n), labels]
                centers[c] = X[int(np.argmax(far))]
    # canonical relabel by first occurrence
    remap = {}
    out = np.empty(n, dtype=np.int32)
    for i in range(n):
        lab = int(labels[i])
        if lab not in remap:
            remap[lab] = len(remap)
        out[i] = remap[lab]
    return out
