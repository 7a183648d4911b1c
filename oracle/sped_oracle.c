/*
 * FP64 CPU oracle for the SPED hot path -- TEST INFRASTRUCTURE ONLY.
 *
 * Only the test suite, the package smoke check and the benchmark's CPU-baseline leg may load
 * this library. It shares no code, header, table or constant with the CUDA path; the two
 * meet only at the seeded input generators. Every routine is the plain definition (or the
 * paper's algorithm, step by step) in FP64 with straight loops, so it can be read against
 * the paper by eye. Nothing here is tuned.
 *
 * Paper: van der Pol, Gemp, Bachrach, Everett, "Stochastic Parallelizable Eigengap Dilation
 * for Large Graph Clustering" (arXiv 2207.14589).
 *
 * Graph input: symmetric CSR (row_ptr[n+1], col_idx[nnz], sorted columns, no self loops),
 * w = per-entry weight (NULL means every weight is 1).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------------------
 * Laplacian application, Section 2: L = D - A with D the (weighted) degree matrix.
 * Weighted graphs (end of Section 2.1): L = X^T W X, i.e. d_i = sum_j w_ij.
 * Y[r,:] = d_r * X[r,:] - sum_j w_rj X[j,:].
 * ------------------------------------------------------------------------------------ */
static double edge_w(const float *w, int64_t p) { return w ? (double)w[p] : 1.0; }

void orc_laplacian_apply(int64_t n, const int32_t *row_ptr, const int32_t *col_idx,
                         const float *w, const double *X, int k, double *Y) {
    for (int64_t r = 0; r < n; ++r) {
        double d = 0.0;
        for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p) d += edge_w(w, p);
        for (int c = 0; c < k; ++c) {
            double a = 0.0;
            for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p)
                a += edge_w(w, p) * X[(int64_t)col_idx[p] * k + c];
            Y[r * k + c] = d * X[r * k + c] - a;
        }
    }
}

/* Weighted degree vector d_i = sum_j w_ij (Section 2.1, weighted case). */
void orc_degrees(int64_t n, const int32_t *row_ptr, const float *w, double *d) {
    for (int64_t r = 0; r < n; ++r) {
        double s = 0.0;
        for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p) s += edge_w(w, p);
        d[r] = s;
    }
}

/* ------------------------------------------------------------------------------------
 * Limit approximation of the decaying exponential (Table 2, last row), with the step
 * scale s made explicit: X_0 = V, X_{t+1} = X_t - s * L X_t, ell times, so that
 * Y = (I - sL)^ell V. With s = 1/ell this is -(-(I - L/ell)^ell) V, i.e. the Table 2
 * transform reversed with lambda* = 0 (Section 4.2).
 * ------------------------------------------------------------------------------------ */
void orc_poly_limit(int64_t n, const int32_t *row_ptr, const int32_t *col_idx, const float *w,
                    const double *V, int k, double s, int ell, double *Y) {
    size_t sz = (size_t)n * k;
    double *X = (double *)malloc(sz * sizeof(double));
    double *LX = (double *)malloc(sz * sizeof(double));
    memcpy(X, V, sz * sizeof(double));
    for (int t = 0; t < ell; ++t) {
        orc_laplacian_apply(n, row_ptr, col_idx, w, X, k, LX);
        for (size_t i = 0; i < sz; ++i) X[i] = X[i] - s * LX[i];
    }
    memcpy(Y, X, sz * sizeof(double));
    free(X);
    free(LX);
}

/* ------------------------------------------------------------------------------------
 * General polynomial p(T) V = sum_{j=0}^{ell} c_j T^j V with T = L + shift * I, by Horner's
 * rule: Z = c_ell V; for j = ell-1 .. 0: Z = c_j V + T Z. Covers the Taylor rows of
 * Table 2 (Taylor -e^{-L}: shift 0; Taylor log(L + eps I): shift = eps - 1).
 * ------------------------------------------------------------------------------------ */
void orc_poly_horner(int64_t n, const int32_t *row_ptr, const int32_t *col_idx, const float *w,
                     const double *V, int k, const double *c, int ell, double shift, double *Y) {
    size_t sz = (size_t)n * k;
    double *Z = (double *)malloc(sz * sizeof(double));
    double *LZ = (double *)malloc(sz * sizeof(double));
    for (size_t i = 0; i < sz; ++i) Z[i] = c[ell] * V[i];
    for (int j = ell - 1; j >= 0; --j) {
        orc_laplacian_apply(n, row_ptr, col_idx, w, Z, k, LZ);
        for (size_t i = 0; i < sz; ++i) Z[i] = c[j] * V[i] + (LZ[i] + shift * Z[i]);
    }
    memcpy(Y, Z, sz * sizeof(double));
    free(Z);
    free(LZ);
}

/* ------------------------------------------------------------------------------------
 * Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw, SC'11), written from
 * its published definition: ten rounds of two 32x32->64 multiplies with a Weyl key
 * schedule.
 * ------------------------------------------------------------------------------------ */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += W0;
            k1 += W1;
        }
        uint64_t p0 = (uint64_t)M0 * c0;
        uint64_t p1 = (uint64_t)M1 * c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* A word stream: the words of philox(key, {a, b, tag, j}) for j = 0, 1, 2, ... in order. */
typedef struct {
    uint32_t key[2];
    uint32_t a, b, tag, j;
    uint32_t buf[4];
    int used;
} word_stream;

static void ws_init(word_stream *s, uint64_t seed, uint32_t a, uint32_t b, uint32_t tag) {
    s->key[0] = (uint32_t)seed;
    s->key[1] = (uint32_t)(seed >> 32);
    s->a = a; s->b = b; s->tag = tag; s->j = 0;
    s->used = 4;
}

static uint32_t ws_next(word_stream *s) {
    if (s->used == 4) {
        uint32_t ctr[4] = {s->a, s->b, s->tag, s->j};
        orc_philox4x32_10(ctr, s->key, s->buf);
        s->j += 1;
        s->used = 0;
    }
    return s->buf[s->used++];
}

/* Unbiased integer in [0, range) by Lemire's multiply-and-reject method (Lemire 2019,
 * "Fast random integer generation in an interval"). range >= 1. */
static uint32_t ws_bounded(word_stream *s, uint32_t range) {
    uint32_t x = ws_next(s);
    uint64_t m = (uint64_t)x * range;
    uint32_t l = (uint32_t)m;
    if (l < range) {
        uint32_t t = (uint32_t)(-range) % range;
        while (l < t) {
            x = ws_next(s);
            m = (uint64_t)x * range;
            l = (uint32_t)m;
        }
    }
    return (uint32_t)(m >> 32);
}

/* Exposed for the generator pins: n bounded draws from the stream (seed, a, b, tag). */
void orc_bounded_draws(uint64_t seed, uint32_t a, uint32_t b, uint32_t tag, uint32_t range,
                       int64_t count, uint32_t *out) {
    word_stream s;
    ws_init(&s, seed, a, b, tag);
    for (int64_t i = 0; i < count; ++i) out[i] = ws_bounded(&s, range);
}

/* One stream per draw: out[j] = the first bounded draw of the stream (seed, j, b, tag),
 * j < count. The edge minibatches use this form, so every draw is independent of the others
 * and of how many there are. */
void orc_first_draws(uint64_t seed, uint32_t b, uint32_t tag, uint32_t range, int64_t count,
                     uint32_t *out) {
    for (int64_t j = 0; j < count; ++j) {
        word_stream s;
        ws_init(&s, seed, (uint32_t)j, b, tag);
        out[j] = ws_bounded(&s, range);
    }
}

/* Stratified draws: the ids 0..range-1 are cut into `count` strata S_j = [floor(j range /
 * count), floor((j+1) range / count)); draw j is uniform in S_j (the first bounded draw of the
 * stream (seed, j, b, tag) over |S_j|). out_id[j] = -1 and out_size[j] = 0 for an empty
 * stratum. */
void orc_stratified_draws(uint64_t seed, uint32_t b, uint32_t tag, int64_t range, int64_t count,
                          int64_t *out_id, int64_t *out_size) {
    for (int64_t j = 0; j < count; ++j) {
        int64_t lo = (j * range) / count, hi = ((j + 1) * range) / count;
        out_size[j] = hi - lo;
        out_id[j] = -1;
        if (hi > lo) {
            word_stream s;
            ws_init(&s, seed, (uint32_t)j, b, tag);
            out_id[j] = lo + (int64_t)ws_bounded(&s, (uint32_t)(hi - lo));
        }
    }
}

/* ------------------------------------------------------------------------------------
 * Incidence algebra (Section 2, Section 4.3 Table 1). x_e has +1 at min(i,j) and -1 at
 * max(i,j); the weighted row is sqrt(w_e) x_e. The inner product of two edge rows is the
 * sum over their shared nodes of the product of the signs there; Table 1 lists the cases:
 * disjoint 0, serial -1, converging +1, diverging +1, repeated 2.
 * ------------------------------------------------------------------------------------ */
double orc_incidence_dot(int64_t a1, int64_t b1, double w1, int64_t a2, int64_t b2, double w2) {
    int64_t e1[2] = {a1 < b1 ? a1 : b1, a1 < b1 ? b1 : a1};
    int64_t e2[2] = {a2 < b2 ? a2 : b2, a2 < b2 ? b2 : a2};
    double sgn[2] = {1.0, -1.0};
    double dot = 0.0;
    for (int u = 0; u < 2; ++u)
        for (int v = 0; v < 2; ++v)
            if (e1[u] == e2[v]) dot += sgn[u] * sgn[v];
    return sqrt(w1) * sqrt(w2) * dot;
}

/* ------------------------------------------------------------------------------------
 * Stochastic estimate of p(L) V = sum_{i=0}^{ell} c_i L^i V (Section 4.3).
 *
 * Equation walk_summand writes L^i as a sum over chains e_1..e_i of the edge-incidence graph
 * (every node with a self loop, footnote of Section 4.3) of alpha_c x_{e_1} x_{e_i}^T. Each
 * of M walkers draws e_1 uniformly from the |E| undirected edges and then walks ell-1 steps,
 * each step uniform over the deg(a)+deg(b)-1 edges incident to the current edge {a, b}
 * (the edge itself included). Linearity lets one walk serve every term i <= ell.
 *
 * mode 1 (importance weights): term i contributes c_i alpha_i / q_i x~_{e1} x~_{ei}^T V with
 *   q_i = |E|^{-1} prod_{t<i} deg_inc(e_t)^{-1}, the probability of the prefix.
 * mode 2 (rejection, as in the text): prefix i is accepted with probability p_min,i / q_i,
 *   p_min,i = |E|^{-1} (deg*_inc)^{-(i-1)}, deg*_inc = 2 deg* - 1, and an accepted prefix
 *   contributes c_i alpha_i / p_min,i x~ x~^T V (a rejected one contributes nothing).
 *
 * Random draws (shared specification, not shared code): key = (seed_lo, seed_hi); for
 * walker w the edge choice at step t uses the words of philox(key, {w_lo, w_hi, t, j}),
 * j = 0, 1, ..., through Lemire's bounded draw (t = 0 draws e_1 in [0, |E|)); the
 * acceptance uniform of prefix i is u = (word + 0.5) 2^-32 with word the first word of
 * philox(key, {w_lo, w_hi, 0x80000000 | i, 0}).
 *
 * Edge order: undirected edge ids enumerate the upper-triangle CSR entries (a < b) in CSR
 * order. The step rule: with the current edge {a, b}, a < b, draw r in [0, deg(a)+deg(b)-1);
 * r < deg(a) selects a's r-th neighbour (edge {a, that}); otherwise r - deg(a) indexes b's
 * neighbour list with a skipped.
 *
 * Y (n x k) receives c_0 V plus the mean over walkers. Returns 0 on success.
 * ------------------------------------------------------------------------------------ */
int orc_walk_estimate(int64_t n, const int32_t *row_ptr, const int32_t *col_idx, const float *w,
                      const double *V, int k, const double *c, int ell, int64_t walkers,
                      uint64_t seed, int mode, int64_t deg_star, double *Y) {
    if (ell < 0 || walkers <= 0) return 1;
    /* enumerate undirected edges (upper entries, CSR order) */
    int64_t n_edges = 0;
    for (int64_t r = 0; r < n; ++r)
        for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p)
            if (col_idx[p] > r) n_edges++;
    for (int64_t i = 0; i < n * k; ++i) Y[i] = c[0] * V[i];
    if (ell == 0 || n_edges == 0) return 0;
    int64_t *ea = (int64_t *)malloc(n_edges * sizeof(int64_t));
    int64_t *eb = (int64_t *)malloc(n_edges * sizeof(int64_t));
    double *ew = (double *)malloc(n_edges * sizeof(double));
    int64_t e = 0;
    for (int64_t r = 0; r < n; ++r)
        for (int64_t p = row_ptr[r]; p < row_ptr[r + 1]; ++p)
            if (col_idx[p] > r) {
                ea[e] = r;
                eb[e] = col_idx[p];
                ew[e] = edge_w(w, p);
                e++;
            }
    double dstar_inc = (double)(2 * deg_star - 1);
    double *acc = (double *)malloc(k * sizeof(double));
    for (int64_t wk = 0; wk < walkers; ++wk) {
        uint32_t wlo = (uint32_t)wk, whi = (uint32_t)((uint64_t)wk >> 32);
        word_stream s;
        ws_init(&s, seed, wlo, whi, 0u);
        int64_t id = ws_bounded(&s, (uint32_t)n_edges);
        int64_t a1 = ea[id], b1 = eb[id];
        double w1 = ew[id];
        int64_t a = a1, b = b1;
        double wc = w1;
        double alpha = 1.0;             /* alpha_1 = empty product */
        double inv_q = (double)n_edges; /* 1/q_1 = |E| */
        double accept = 1.0;            /* prod_{t<i} deg_inc(e_t) / deg*_inc */
        for (int j = 0; j < k; ++j) acc[j] = 0.0;
        for (int i = 1; i <= ell; ++i) {
            double scale;
            if (mode == 1) {
                scale = c[i] * alpha * inv_q * sqrt(w1) * sqrt(wc);
            } else {
                word_stream su;
                ws_init(&su, seed, wlo, whi, 0x80000000u | (uint32_t)i);
                double u = ((double)ws_next(&su) + 0.5) * (1.0 / 4294967296.0);
                double inv_pmin = (double)n_edges * pow(dstar_inc, (double)(i - 1));
                scale = (u < accept) ? c[i] * alpha * inv_pmin * sqrt(w1) * sqrt(wc) : 0.0;
            }
            for (int j = 0; j < k; ++j) acc[j] += scale * (V[a * k + j] - V[b * k + j]);
            if (i == ell) break;
            /* step to the next edge of the chain */
            int64_t da = row_ptr[a + 1] - row_ptr[a];
            int64_t db = row_ptr[b + 1] - row_ptr[b];
            int64_t deg_inc = da + db - 1;
            word_stream st;
            ws_init(&st, seed, wlo, whi, (uint32_t)i);
            int64_t r = ws_bounded(&st, (uint32_t)deg_inc);
            int64_t na, nb;
            if (r < da) {
                na = a;
                nb = col_idx[row_ptr[a] + r];
            } else {
                int64_t rr = r - da, q = -1, seen = 0;
                for (int64_t p = row_ptr[b]; p < row_ptr[b + 1]; ++p) {
                    if (col_idx[p] == a) continue;
                    if (seen == rr) { q = col_idx[p]; break; }
                    seen++;
                }
                na = b;
                nb = q;
            }
            int64_t lo = na < nb ? na : nb, hi = na < nb ? nb : na;
            /* weight of the new edge: look it up in row lo */
            double wn = 1.0;
            for (int64_t p = row_ptr[lo]; p < row_ptr[lo + 1]; ++p)
                if (col_idx[p] == hi) { wn = edge_w(w, p); break; }
            alpha *= orc_incidence_dot(a, b, wc, lo, hi, wn);
            inv_q *= (double)deg_inc;
            accept *= (double)deg_inc / dstar_inc;
            a = lo; b = hi; wc = wn;
        }
        double inv_m = 1.0 / (double)walkers;
        for (int j = 0; j < k; ++j) {
            Y[a1 * k + j] += acc[j] * inv_m;
            Y[b1 * k + j] -= acc[j] * inv_m;
        }
    }
    free(acc);
    free(ea);
    free(eb);
    free(ew);
    return 0;
}
