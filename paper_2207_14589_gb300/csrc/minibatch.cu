// Edge minibatches: the stochastic optimisation model in which the solver sees the graph only
// through minibatches of edges (Sections 2 and 6). The Laplacian is the sum of the edges' outer
// products, L = sum_e w_e x_e x_e^T with x_e = e_a - e_b (Section 4.3; weighted as at the end
// of Section 2.1), so B edges drawn uniformly with replacement give the unbiased estimate
//   L_hat = (|E| / B) sum_{j<B} w_j x_j x_j^T,
//   (L_hat X)[a_j] += c_j (X[a_j] - X[b_j]),  (L_hat X)[b_j] -= c_j (X[a_j] - X[b_j]),  c_j = w_j |E| / B.
// One chain step Y = alpha V + gamma X + delta W2 + beta L_hat X runs as two launches: a dense
// pass writes the first three terms (one thread per 16-byte piece of a row), then one group of
// C lanes per draw adds the edge terms with 16-byte atomic adds (float4 / two doubles), C = the
// power of two covering a row's 16-byte pieces. A group draws C edges at once, one per lane
// (Philox once per draw, then one 8-byte load of the edge's endpoints), and hands each to the
// whole group by shuffles.
//
// Draws: draw j of multiplication t is the first Lemire bounded draw in [0, |E|) of the word
// stream (seed; counter words j, t, 0x4D42), so every draw is independent of the others and of
// the batch size; edges are numbered by the CSR order of their upper entries.
//
// Stratified minibatches (variance reduction, left to future work in Section 6): the edge ids
// are cut into B contiguous strata S_j = [floor(j|E|/B), floor((j+1)|E|/B)), draw j is uniform
// in S_j (the same stream, range |S_j|) and stands for its stratum with weight |S_j|, so
// L_hat = sum_j |S_j| w_j x_j x_j^T is unbiased. The strata follow the CSR order, so a
// minibatch covers every part of the graph in proportion, and consecutive draws touch nearby
// rows.
#include "sped_internal.cuh"

namespace sped {

constexpr uint32_t MB_TAG = 0x4D42u;
constexpr int MB_THREADS = 256;

// Draw j of a minibatch of `count`: uniform over the edges, or (STRAT) uniform in stratum j
// with size = |S_j|; an empty stratum gives a = b = -1, size 0.
template <bool STRAT>
__device__ __forceinline__ void draw_edge(uint64_t seed, uint32_t step, uint32_t j,
                                          uint32_t n_edges, uint64_t count,
                                          const int2 *__restrict__ edge_ab,
                                          const int32_t *__restrict__ edge_p,
                                          const float *__restrict__ w, int32_t &a, int32_t &b,
                                          float &wv, int32_t &size) {
    WordStream s(seed, j, step, MB_TAG);
    uint32_t e;
    if constexpr (STRAT) {
        const uint64_t lo = (uint64_t)j * n_edges / count;
        const uint64_t hi = ((uint64_t)j + 1) * n_edges / count;
        size = (int32_t)(hi - lo);
        if (size == 0) {
            a = b = -1;
            wv = 0.f;
            return;
        }
        e = (uint32_t)lo + s.bounded((uint32_t)size);
    } else {
        size = 1;
        e = s.bounded(n_edges);
    }
    const int2 ab = __ldg(edge_ab + e);
    a = ab.x;
    b = ab.y;
    wv = w ? __ldg(w + __ldg(edge_p + e)) : 1.0f;
}

// ---------------------------------------------------------------------------------------
// the sampled edges themselves
// ---------------------------------------------------------------------------------------
template <bool STRAT>
__global__ void __launch_bounds__(MB_THREADS)
    k_sample_edges(int64_t count, uint64_t seed, uint32_t step, uint32_t n_edges,
                   const int2 *__restrict__ edge_ab, const int32_t *__restrict__ edge_p,
                   const float *__restrict__ w, int32_t *__restrict__ out_a,
                   int32_t *__restrict__ out_b, float *__restrict__ out_w,
                   int32_t *__restrict__ out_size) {
    for (int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; j < count;
         j += (int64_t)gridDim.x * blockDim.x) {
        int32_t a, b, size;
        float wv;
        draw_edge<STRAT>(seed, step, (uint32_t)j, n_edges, (uint64_t)count, edge_ab, edge_p, w,
                         a, b, wv, size);
        if (out_a) out_a[j] = a;
        if (out_b) out_b[j] = b;
        if (out_w) out_w[j] = wv;
        if (STRAT && out_size) out_size[j] = size;
    }
}

// ---------------------------------------------------------------------------------------
// 16-byte pieces of a row (E elements of the output type) loaded into the accumulator type
// ---------------------------------------------------------------------------------------
template <typename TX, int E, typename A> struct ChunkLoad;
template <typename A> struct ChunkLoad<float, 4, A> {
    static __device__ __forceinline__ void run(const float *p, A *o) {
        const float4 v = __ldg(reinterpret_cast<const float4 *>(p));
        o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
    }
};
template <typename A> struct ChunkLoad<float, 2, A> {
    static __device__ __forceinline__ void run(const float *p, A *o) {
        const float2 v = __ldg(reinterpret_cast<const float2 *>(p));
        o[0] = v.x; o[1] = v.y;
    }
};
template <typename A> struct ChunkLoad<double, 2, A> {
    static __device__ __forceinline__ void run(const double *p, A *o) {
        const double2 v = __ldg(reinterpret_cast<const double2 *>(p));
        o[0] = (A)v.x; o[1] = (A)v.y;
    }
};
template <typename A> struct ChunkLoad<double, 4, A> {
    static __device__ __forceinline__ void run(const double *p, A *o) {
        const double2 u = __ldg(reinterpret_cast<const double2 *>(p));
        const double2 v = __ldg(reinterpret_cast<const double2 *>(p) + 1);
        o[0] = (A)u.x; o[1] = (A)u.y; o[2] = (A)v.x; o[3] = (A)v.y;
    }
};

template <typename T, int E, typename A> struct ChunkStore;
template <typename A> struct ChunkStore<float, 4, A> {
    static __device__ __forceinline__ void run(float *p, const A *v) {
        *reinterpret_cast<float4 *>(p) = make_float4((float)v[0], (float)v[1], (float)v[2],
                                                     (float)v[3]);
    }
};
template <typename A> struct ChunkStore<double, 2, A> {
    static __device__ __forceinline__ void run(double *p, const A *v) {
        *reinterpret_cast<double2 *>(p) = make_double2((double)v[0], (double)v[1]);
    }
};

// ---------------------------------------------------------------------------------------
// dense part: Y = alpha V + gamma X + delta W2, one thread per 16-byte piece of a Y row
// (flat over rows x pieces, so every lane works and a warp's accesses are contiguous)
// ---------------------------------------------------------------------------------------
template <typename TX, typename TV, typename TY, typename IDX>
__global__ void __launch_bounds__(MB_THREADS)
    k_mb_dense(int64_t n, int k, int chunks, const TX *__restrict__ X, int ldx,
               const TV *__restrict__ V, int ldv, const TX *__restrict__ W2, int ldw2,
               TY *__restrict__ Y, int ldy, double alpha, double gamma, double delta) {
    using A = typename AccOf<TY>::type;
    constexpr int E = 16 / (int)sizeof(TY);
    const A al = (A)alpha, ga = (A)gamma, de = (A)delta;
    const IDX total = (IDX)n * (IDX)chunks;
    const IDX stride = (IDX)gridDim.x * blockDim.x;
    for (IDX i = (IDX)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += stride) {
        const IDX r = i / (IDX)chunks;
        const int c0 = (int)(i - r * (IDX)chunks) * E;
        const TX *x = X + (int64_t)r * ldx + c0;
        TY *y = Y + (int64_t)r * ldy + c0;
        if (c0 + E <= k) {
            A acc[E], t[E];
            ChunkLoad<TX, E, A>::run(x, acc);
#pragma unroll
            for (int e = 0; e < E; ++e) acc[e] *= ga;
            if (V) {
                ChunkLoad<TV, E, A>::run(V + (int64_t)r * ldv + c0, t);
#pragma unroll
                for (int e = 0; e < E; ++e) acc[e] += al * t[e];
            }
            if (W2) {
                ChunkLoad<TX, E, A>::run(W2 + (int64_t)r * ldw2 + c0, t);
#pragma unroll
                for (int e = 0; e < E; ++e) acc[e] += de * t[e];
            }
            ChunkStore<TY, E, A>::run(y, acc);
        } else {
            for (int c = 0; c < k - c0; ++c) {
                A v = ga * cvt<A>(x[c]);
                if (V) v += al * cvt<A>(V[(int64_t)r * ldv + c0 + c]);
                if (W2) v += de * cvt<A>(W2[(int64_t)r * ldw2 + c0 + c]);
                y[c] = from_acc<TY>(v);
            }
        }
    }
}

// ---------------------------------------------------------------------------------------
// edge part: Y += coef * sum_j w_j x_j x_j^T X
// ---------------------------------------------------------------------------------------
__device__ __forceinline__ void chunk_atomic_add(float *p, const float *d, float sgn) {
    atomicAdd(reinterpret_cast<float4 *>(p), make_float4(sgn * d[0], sgn * d[1], sgn * d[2],
                                                         sgn * d[3]));
}
__device__ __forceinline__ void chunk_atomic_add(double *p, const double *d, double sgn) {
    atomicAdd(p, sgn * d[0]);
    atomicAdd(p + 1, sgn * d[1]);
}

// SRC: 0 = the caller's edge arrays, 1 = uniform draws, 2 = stratified draws
template <typename TX, typename TY, int SRC>
__global__ void __launch_bounds__(MB_THREADS)
    k_edge_scatter(int64_t n, int k, int lanes_log2, const TX *__restrict__ X, int ldx, TY *Y,
                   int ldy, int64_t count, double coef, uint64_t seed, uint32_t step,
                   uint32_t n_edges, const int2 *__restrict__ edge_ab,
                   const int32_t *__restrict__ edge_p, const int32_t *__restrict__ ea,
                   const int32_t *__restrict__ eb, const float *__restrict__ w,
                   int32_t *skipped) {
    using A = typename AccOf<TY>::type;
    constexpr int E = 16 / (int)sizeof(TY);  // elements in one 16-byte piece of a Y row
    const int C = 1 << lanes_log2;
    const int lane = threadIdx.x & 31;
    const int sub = lane & (C - 1);
    const int64_t gtid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t group = gtid >> lanes_log2;
    const int64_t warp_group0 = (gtid - lane) >> lanes_log2;  // first group of this warp
    const int64_t n_groups = ((int64_t)gridDim.x * blockDim.x) >> lanes_log2;
    const int chunks = (k + E - 1) / E;
    // the loop bound is the warp's first group, so all lanes of a warp take the same trips
    // through the shuffles below
    for (int64_t wbase = warp_group0 * C; wbase < count; wbase += n_groups * C) {
        const int64_t j = wbase + (group - warp_group0) * C + sub;
        int32_t a = -1, b = -1, size = 0;
        float wv = 0.f;
        if (j < count) {
            if constexpr (SRC != 0) {
                draw_edge<SRC == 2>(seed, step, (uint32_t)j, n_edges, (uint64_t)count, edge_ab,
                                    edge_p, w, a, b, wv, size);
            } else {
                a = __ldg(ea + j);
                b = __ldg(eb + j);
                wv = w ? __ldg(w + j) : 1.0f;
                if (a < 0 || b < 0 || (int64_t)a >= n || (int64_t)b >= n) {
                    if (skipped) atomicAdd(skipped, 1);
                    a = -1;
                }
            }
        }
        for (int q = 0; q < C; ++q) {
            const int32_t qa = __shfl_sync(0xffffffffu, a, q, C);
            const int32_t qb = __shfl_sync(0xffffffffu, b, q, C);
            const float qw = __shfl_sync(0xffffffffu, wv, q, C);
            if (qa < 0) continue;
            A cq;
            if constexpr (SRC == 2) {
                const int32_t qs = __shfl_sync(0xffffffffu, size, q, C);
                cq = (A)(coef * (double)qw * (double)qs);
            } else {
                cq = (A)(coef * (double)qw);
            }
            const TX *xa = X + (int64_t)qa * ldx;
            const TX *xb = X + (int64_t)qb * ldx;
            TY *ya = Y + (int64_t)qa * ldy;
            TY *yb = Y + (int64_t)qb * ldy;
            for (int ch = sub; ch < chunks; ch += C) {
                const int c0 = ch * E;
                if (c0 + E <= k) {
                    A va[E], vb[E], d[E];
                    ChunkLoad<TX, E, A>::run(xa + c0, va);
                    ChunkLoad<TX, E, A>::run(xb + c0, vb);
#pragma unroll
                    for (int i = 0; i < E; ++i) d[i] = cq * (va[i] - vb[i]);
                    chunk_atomic_add(ya + c0, d, (A)1);
                    chunk_atomic_add(yb + c0, d, (A)-1);
                } else {
                    for (int c = c0; c < k; ++c) {
                        const A d = cq * (cvt<A>(xa[c]) - cvt<A>(xb[c]));
                        atomicAdd(ya + c, d);
                        atomicAdd(yb + c, -d);
                    }
                }
            }
        }
    }
}

static int lanes_log2_for(int k, size_t elem_bytes) {
    const int chunks = (int)((k * elem_bytes + 15) / 16);
    int l = 0;
    while ((1 << l) < chunks && l < 5) ++l;
    return l;
}

static int grid_for(int64_t items, int lanes_log2) {
    const int64_t per_block = MB_THREADS >> lanes_log2;
    int64_t blocks = (items + per_block - 1) / per_block;
    const int64_t cap = (int64_t)device_sm_count() * 8;
    if (blocks > cap) blocks = cap;
    return (int)(blocks < 1 ? 1 : blocks);
}

template <typename TX, typename TV, typename TY>
static sped_status run_dense(int64_t n, int k, const void *X, int ldx, const void *V, int ldv,
                             const void *W2, int ldw2, void *Y, int ldy, double alpha,
                             double gamma, double delta, cudaStream_t st) {
    if (n == 0) return SPED_OK;
    const int chunks = (int)((k * sizeof(TY) + 15) / 16);
    const int64_t total = n * chunks;
    int64_t blocks = (total + MB_THREADS - 1) / MB_THREADS;
    const int64_t cap = (int64_t)device_sm_count() * 16;
    const int grid = (int)(blocks > cap ? cap : blocks);
    if (total < ((int64_t)1 << 31))
        k_mb_dense<TX, TV, TY, uint32_t><<<grid, MB_THREADS, 0, st>>>(
            n, k, chunks, (const TX *)X, ldx, (const TV *)V, ldv, (const TX *)W2, ldw2, (TY *)Y,
            ldy, alpha, gamma, delta);
    else
        k_mb_dense<TX, TV, TY, uint64_t><<<grid, MB_THREADS, 0, st>>>(
            n, k, chunks, (const TX *)X, ldx, (const TV *)V, ldv, (const TX *)W2, ldw2, (TY *)Y,
            ldy, alpha, gamma, delta);
    SPED_CHECK_LAUNCH("k_mb_dense");
    return SPED_OK;
}

template <typename TX, typename TY>
static sped_status run_scatter(int64_t n, int k, const void *X, int ldx, void *Y, int ldy,
                               const EdgeBatch &eb, double coef, cudaStream_t st) {
    if (eb.count == 0 || coef == 0.0) return SPED_OK;
    const int l2 = lanes_log2_for(k, sizeof(TY));
    const int64_t groups_needed = (eb.count + (1 << l2) - 1) >> l2;
    const int grid = grid_for(groups_needed, l2);
    if (eb.graph) {
        const sped_graph *g = eb.graph;
        if (eb.stratified)
            k_edge_scatter<TX, TY, 2><<<grid, MB_THREADS, 0, st>>>(
                n, k, l2, (const TX *)X, ldx, (TY *)Y, ldy, eb.count, coef, eb.seed, eb.step,
                (uint32_t)g->n_edges, g->edge_ab, g->edge_p, nullptr, nullptr, g->w, nullptr);
        else
            k_edge_scatter<TX, TY, 1><<<grid, MB_THREADS, 0, st>>>(
                n, k, l2, (const TX *)X, ldx, (TY *)Y, ldy, eb.count, coef, eb.seed, eb.step,
                (uint32_t)g->n_edges, g->edge_ab, g->edge_p, nullptr, nullptr, g->w, nullptr);
    } else {
        k_edge_scatter<TX, TY, 0><<<grid, MB_THREADS, 0, st>>>(
            n, k, l2, (const TX *)X, ldx, (TY *)Y, ldy, eb.count, coef, 0, 0, 0, nullptr, nullptr,
            eb.a, eb.b, eb.w, eb.skipped);
    }
    SPED_CHECK_LAUNCH("k_edge_scatter");
    return SPED_OK;
}

static bool f32_or_f64(sped_dtype t) { return t == SPED_F32 || t == SPED_F64; }

sped_status launch_edge_step(int64_t n, int k, const void *X, sped_dtype xt, int ldx,
                             const void *V, sped_dtype vt, int ldv, const void *W2, int ldw2,
                             double delta, void *Y, sped_dtype yt, int ldy, double alpha,
                             double beta, double gamma, const EdgeBatch &eb, cudaStream_t st) {
    if (!f32_or_f64(xt) || !f32_or_f64(yt) || (V && !f32_or_f64(vt)))
        return fail(SPED_ERR_UNSUPPORTED,
                    "minibatch step: X, Y and V must be F32 or F64 (x=%d y=%d v=%d)", (int)xt,
                    (int)yt, V ? (int)vt : -1);
    if (alpha == 0.0) V = nullptr;
    if (delta == 0.0) W2 = nullptr;
#define MB_DENSE(TXX, TVV, TYY)                                                             \
    SPED_TRY((run_dense<TXX, TVV, TYY>(n, k, X, ldx, V, ldv, W2, ldw2, Y, ldy, alpha, gamma, \
                                       delta, st)))
    const sped_dtype vv = V ? vt : xt;
    if (xt == SPED_F32) {
        if (vv == SPED_F32) {
            if (yt == SPED_F32) MB_DENSE(float, float, float); else MB_DENSE(float, float, double);
        } else {
            if (yt == SPED_F32) MB_DENSE(float, double, float); else MB_DENSE(float, double, double);
        }
    } else {
        if (vv == SPED_F32) {
            if (yt == SPED_F32) MB_DENSE(double, float, float); else MB_DENSE(double, float, double);
        } else {
            if (yt == SPED_F32) MB_DENSE(double, double, float); else MB_DENSE(double, double, double);
        }
    }
#undef MB_DENSE
    const double coef = beta * eb.scale;
    if (xt == SPED_F32 && yt == SPED_F32) return run_scatter<float, float>(n, k, X, ldx, Y, ldy, eb, coef, st);
    if (xt == SPED_F32 && yt == SPED_F64) return run_scatter<float, double>(n, k, X, ldx, Y, ldy, eb, coef, st);
    if (xt == SPED_F64 && yt == SPED_F32) return run_scatter<double, float>(n, k, X, ldx, Y, ldy, eb, coef, st);
    return run_scatter<double, double>(n, k, X, ldx, Y, ldy, eb, coef, st);
}

}  // namespace sped

using namespace sped;

extern "C" {

sped_status sped_sample_edges(const sped_graph *g, uint64_t seed, uint32_t step, int64_t count,
                              int stratified, int32_t *d_a, int32_t *d_b, float *d_w,
                              int32_t *d_size, void *stream) {
    if (!g) return fail(SPED_ERR_INVALID_ARG, "sample_edges: null graph");
    if (count < 0 || count > (int64_t)UINT32_MAX + 1)
        return fail(SPED_ERR_INVALID_ARG, "sample_edges: count %lld not in 0..2^32",
                    (long long)count);
    if (count > 0 && g->n_edges < 1)
        return fail(SPED_ERR_INVALID_ARG, "sample_edges: the graph has no edges");
    if (count == 0 || (!d_a && !d_b && !d_w && !d_size)) return SPED_OK;
    const int grid = grid_for(count, 0);
    if (stratified)
        k_sample_edges<true><<<grid, MB_THREADS, 0, as_stream(stream)>>>(
            count, seed, step, (uint32_t)g->n_edges, g->edge_ab, g->edge_p, g->w, d_a, d_b, d_w,
            d_size);
    else
        k_sample_edges<false><<<grid, MB_THREADS, 0, as_stream(stream)>>>(
            count, seed, step, (uint32_t)g->n_edges, g->edge_ab, g->edge_p, g->w, d_a, d_b, d_w,
            nullptr);
    SPED_CHECK_LAUNCH("k_sample_edges");
    return SPED_OK;
}

sped_status sped_edge_step(int64_t n, int k, const int32_t *d_a, const int32_t *d_b,
                           const float *d_w, int64_t count, double edge_scale, const void *d_X,
                           sped_dtype x_t, int ldx, const void *d_V, sped_dtype v_t, int ldv,
                           void *d_Y, sped_dtype y_t, int ldy, double alpha, double beta,
                           double gamma, int32_t *d_skipped, void *stream) {
    if (n < 0 || count < 0) return fail(SPED_ERR_INVALID_ARG, "edge_step: negative size");
    if (count > 0 && (!d_a || !d_b))
        return fail(SPED_ERR_INVALID_ARG, "edge_step: null edge endpoint array");
    if (n > 0) {
        SPED_TRY(check_layout(d_X, x_t, k, ldx, "edge_step X"));
        SPED_TRY(check_layout(d_Y, y_t, k, ldy, "edge_step Y"));
        if (d_V && alpha != 0.0) SPED_TRY(check_layout(d_V, v_t, k, ldv, "edge_step V"));
        if (d_X == d_Y) return fail(SPED_ERR_INVALID_ARG, "edge_step: X and Y must not alias");
    }
    if (alpha != 0.0 && !d_V) return fail(SPED_ERR_INVALID_ARG, "edge_step: alpha != 0 needs V");
    if (n == 0) return SPED_OK;
    EdgeBatch eb;
    eb.count = count;
    eb.scale = edge_scale;
    eb.a = d_a;
    eb.b = d_b;
    eb.w = d_w;
    eb.skipped = d_skipped;
    return launch_edge_step(n, k, d_X, x_t, ldx, d_V, v_t, ldv, nullptr, 0, 0.0, d_Y, y_t, ldy,
                            alpha, beta, gamma, eb, as_stream(stream));
}

}  // extern "C"
