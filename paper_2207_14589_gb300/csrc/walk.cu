// Stochastic estimate of p(L) V over sampled walks (Section 4.3), one thread per walker.
//
// Eq. walk_summand writes L^i as a sum over chains e_1..e_i of the edge-incidence graph (a self
// loop on every node, footnote of Section 4.3) of alpha_c x~_{e1} x~_{ei}^T, alpha_c the product
// of consecutive incidence inner products (Table 1, scaled by sqrt(w_e w_f) for weights).
// Each walker draws e_1 uniformly from the |E| undirected edges, then walks l-1 steps, each
// uniform over the deg(a)+deg(b)-1 edges incident to the current edge {a,b} (itself included).
// One walk serves every term i <= l (linearity of expectation, Section 4.3). The walker keeps
// sum_i c_i w_i alpha_i (V[a_i] - V[b_i]) in registers and scatters it once into rows a_1 and
// b_1 of Y (atomics), so a walk costs two row atomics instead of two per term.
//  * importance weights: w_i = 1/q_i = |E| prod_{t<i} deg_inc(e_t);
//  * rejection (as in the text): prefix i is kept with probability p_min,i / q_i,
//    p_min,i = |E|^{-1} (2 deg* - 1)^{-(i-1)}, and then weighted 1/p_min,i.
//
// Random draws (the same published specification the reference implements separately):
// Philox4x32-10 with key (seed_lo, seed_hi); walker w, step tag t: words of
// philox(key, {w_lo, w_hi, t, j}), j = 0, 1, ..., bounded draws by Lemire's multiply-and-reject;
// t = 0 draws e_1 in [0, |E|), t = i (1 <= i < l) draws the step after term i; the acceptance
// uniform of prefix i is (word + 0.5) 2^-32 of the first word of tag 0x80000000 | i.
// Edge ids follow the CSR order of the upper entries (a < b); the step rule takes a's r-th
// neighbour for r < deg(a), else b's (r - deg(a))-th neighbour with a skipped.
#include <algorithm>
#include <cmath>

#include "sped_internal.cuh"

namespace sped {

constexpr int WALK_MAX_ELL = 511;
constexpr int WALK_THREADS = 128;
// Resident blocks per SM the register budget is cut for, from the walker's accumulator size
// (k columns of the output's precision): 7 blocks (72 registers a thread) while it takes at most
// 96 bytes, fewer for wider or FP64 accumulators, which would spill under that budget. The walk
// is bound by the latency of its dependent loads, so resident warps are what it runs on.
template <typename A, int KM> constexpr int walk_blocks_per_sm() {
    return (int)sizeof(A) * KM <= 96 ? 7 : ((int)sizeof(A) * KM <= 160 ? 5 : 3);
}

struct WalkCoefs {
    double c[WALK_MAX_ELL + 1];
};

template <typename Ty, typename Tv>
__global__ void k_walk_init(int64_t n, int k, const Tv *__restrict__ V, int ldv, double c0,
                            Ty *__restrict__ Y, int ldy) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n * k) return;
    int64_t r = e / k;
    int j = (int)(e - r * k);
    Y[r * ldy + j] = from_acc<Ty>(c0 * cvt<double>(V[r * ldv + j]));
}

// scale * (V[a] - V[b]) added into the walker's accumulator one 16-byte chunk of each row at a
// time (when the layout allows 16-byte loads), so that only a chunk of each row is live instead
// of two whole rows: the registers saved buy resident warps, which hide the walk's dependent
// loads. Columns at or past k are not touched (their accumulator entries are never read).
template <int KM, typename Tv, typename A>
__device__ __forceinline__ void walk_add(const Tv *pa, const Tv *pb, int k, bool vec, A sc,
                                         A *acc) {
    constexpr int E = 16 / (int)sizeof(Tv);
    if (vec && KM % E == 0) {
#pragma unroll
        for (int q = 0; q < KM / E; ++q) {
            if (q * E < k) {
                const uint4 ca = __ldg(reinterpret_cast<const uint4 *>(pa) + q);
                const uint4 cb = __ldg(reinterpret_cast<const uint4 *>(pb) + q);
                const Tv *ea = reinterpret_cast<const Tv *>(&ca);
                const Tv *eb = reinterpret_cast<const Tv *>(&cb);
#pragma unroll
                for (int u = 0; u < E; ++u)
                    acc[q * E + u] += sc * (cvt<A>(ea[u]) - cvt<A>(eb[u]));
            }
        }
    } else {
#pragma unroll
        for (int j = 0; j < KM; ++j)
            if (j < k) acc[j] += sc * (cvt<A>(__ldg(pa + j)) - cvt<A>(__ldg(pb + j)));
    }
}

// The walk's bookkeeping (edge draws, alpha, 1/q, the acceptance product) runs in FP64 and in
// the oracle's order, so every sampled decision is the same; the k-column accumulation of
// scale_i (V[a_i] - V[b_i]) runs in the output's precision (F32 output: F32 products of the
// F32 difference with the FP64 scale rounded once per term).
template <typename Tv, typename Ty, bool W, int KM, int MODE>
__global__ void __launch_bounds__(WALK_THREADS,
                                  (walk_blocks_per_sm<typename AccOf<Ty>::type, KM>()))
k_walk(const int32_t *__restrict__ rp, const int32_t *__restrict__ ci, const float *__restrict__ w,
       const int32_t *__restrict__ rev, const int32_t *__restrict__ edge_p,
       const int32_t *__restrict__ edge_a, int64_t n_edges, const Tv *__restrict__ V, int ldv,
       int k, int ell, int64_t walkers, uint64_t seed, double dstar_inc, int vec, WalkCoefs cf,
       Ty *__restrict__ Y, int ldy) {
    using A = typename AccOf<Ty>::type;
    const double inv_m = 1.0 / (double)walkers;
    for (int64_t wk = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; wk < walkers;
         wk += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t wlo = (uint32_t)wk, whi = (uint32_t)((uint64_t)wk >> 32);
        WordStream s0(seed, wlo, whi, 0u);
        const int e1 = (int)s0.bounded((uint32_t)n_edges);
        int pc = __ldg(edge_p + e1);
        const int a1 = __ldg(edge_a + e1), b1 = __ldg(ci + pc);
        const double sw1 = W ? sqrt((double)__ldg(w + pc)) : 1.0;
        int a = a1, b = b1;
        double swc = sw1;
        double alpha = 1.0, inv_q = (double)n_edges, accept = 1.0, inv_pmin = (double)n_edges;
        A acc[KM];
#pragma unroll
        for (int j = 0; j < KM; ++j) acc[j] = A(0);
        for (int i = 1; i <= ell; ++i) {
            double scale;
            if (MODE == SPED_STOCHASTIC_IS) {
                scale = cf.c[i] * alpha * inv_q * sw1 * swc;
            } else {
                WordStream su(seed, wlo, whi, 0x80000000u | (uint32_t)i);
                const double u = ((double)su.next() + 0.5) * (1.0 / 4294967296.0);
                scale = (u < accept) ? cf.c[i] * alpha * inv_pmin * sw1 * swc : 0.0;
                inv_pmin *= dstar_inc;
            }
            if (scale != 0.0)
                walk_add<KM>(V + (int64_t)a * ldv, V + (int64_t)b * ldv, k, vec != 0, (A)scale,
                             acc);
            if (i == ell) break;
            const int ra = __ldg(rp + a), da = __ldg(rp + a + 1) - ra;
            const int rb = __ldg(rp + b), db = __ldg(rp + b + 1) - rb;
            const int deg_inc = da + db - 1;
            WordStream st(seed, wlo, whi, (uint32_t)i);
            const int r = (int)st.bounded((uint32_t)deg_inc);
            int q, na, nb;
            if (r < da) {
                q = ra + r;
                na = a;
            } else {
                const int rr = r - da;
                const int skip = __ldg(rev + pc) - rb;  // position of a in b's row
                q = rb + rr + (rr >= skip ? 1 : 0);
                na = b;
            }
            nb = __ldg(ci + q);
            const int lo = na < nb ? na : nb, hi = na < nb ? nb : na;
            const int pos = na < nb ? q : __ldg(rev + q);  // entry (lo, hi) in row lo
            const double swn = W ? sqrt((double)__ldg(w + pos)) : 1.0;
            // incidence inner product of {a, b} and {lo, hi} (+1 at the smaller node, -1 at the
            // larger), times sqrt(w_e w_f)
            double d = 0.0;
            if (a == lo) d += 1.0;
            if (a == hi) d -= 1.0;
            if (b == lo) d -= 1.0;
            if (b == hi) d += 1.0;
            alpha *= swc * swn * d;
            inv_q *= (double)deg_inc;
            if (MODE != SPED_STOCHASTIC_IS) accept *= (double)deg_inc / dstar_inc;
            a = lo;
            b = hi;
            pc = pos;
            swc = swn;
        }
        Ty *ya = Y + (int64_t)a1 * ldy, *yb = Y + (int64_t)b1 * ldy;
        const A im = (A)inv_m;
#pragma unroll
        for (int j = 0; j < KM; ++j) {
            if (j < k && acc[j] != A(0)) {
                atomicAdd(ya + j, (Ty)(acc[j] * im));
                atomicAdd(yb + j, (Ty)(-acc[j] * im));
            }
        }
    }
}

template <typename Tv, typename Ty>
static sped_status run_walk(const sped_graph *g, int k, const void *V, int ldv, void *Y, int ldy,
                            sped_mode mode, int64_t walkers, uint64_t seed, cudaStream_t st) {
    const Poly &P = g->poly;
    const int ell = P.ell;
    int64_t nk = g->n * (int64_t)k;
    k_walk_init<Ty, Tv><<<(unsigned)((nk + 255) / 256), 256, 0, st>>>(
        g->n, k, (const Tv *)V, ldv, P.power[0], (Ty *)Y, ldy);
    SPED_CHECK_LAUNCH("k_walk_init");
    if (g->n_edges == 0 || walkers == 0) return SPED_OK;
    WalkCoefs cf;
    for (int i = 0; i <= WALK_MAX_ELL; ++i) cf.c[i] = i <= ell ? P.power[i] : 0.0;
    double dstar_inc = 2.0 * g->max_deg - 1.0;
    const int vec = ((uintptr_t)V % 16 == 0) && ((size_t)ldv * (sizeof(Tv)) % 16 == 0);
    // one wave: as many blocks as are resident at once, the grid-stride loop spreads the walkers
    const int64_t want = (walkers + WALK_THREADS - 1) / WALK_THREADS;
    using Acc = typename AccOf<Ty>::type;
#define WALK3(KMV, WV, MV)                                                                     \
    k_walk<Tv, Ty, WV, KMV, MV><<<(unsigned)std::min<int64_t>(                                 \
        want, (int64_t)device_sm_count() * walk_blocks_per_sm<Acc, KMV>()), WALK_THREADS, 0, st>>>( \
        g->rp, g->ci, g->w, g->rev, g->edge_p, g->edge_a, g->n_edges, (const Tv *)V, ldv, k, ell, \
        walkers, seed, dstar_inc, vec, cf, (Ty *)Y, ldy)
#define WALK(KMV)                                                                              \
    do {                                                                                       \
        if (g->w) {                                                                            \
            if (mode == SPED_STOCHASTIC_IS) WALK3(KMV, true, SPED_STOCHASTIC_IS);              \
            else WALK3(KMV, true, SPED_STOCHASTIC_REJECT);                                     \
        } else {                                                                               \
            if (mode == SPED_STOCHASTIC_IS) WALK3(KMV, false, SPED_STOCHASTIC_IS);             \
            else WALK3(KMV, false, SPED_STOCHASTIC_REJECT);                                    \
        }                                                                                      \
    } while (0)
    if (k <= 8) WALK(8);
    else if (k <= 16) WALK(16);
    else if (k <= 20) WALK(20);
    else if (k <= 24) WALK(24);
    else WALK(32);
#undef WALK
#undef WALK3
    SPED_CHECK_LAUNCH("k_walk");
    return SPED_OK;
}

sped_status launch_walk(const sped_graph *g, int k, const void *V, sped_dtype vt, int ldv, void *Y,
                        sped_dtype yt, int ldy, sped_mode mode, int64_t walkers, uint64_t seed,
                        cudaStream_t st) {
    if (walkers < 0) return fail(SPED_ERR_INVALID_ARG, "walk: walkers < 0");
    if (k > 32) return fail(SPED_ERR_UNSUPPORTED, "walk: k=%d > 32", k);
    if (g->poly.ell > WALK_MAX_ELL)
        return fail(SPED_ERR_UNSUPPORTED, "walk: degree %d > %d", g->poly.ell, WALK_MAX_ELL);
    if (g->n_edges >= (int64_t)UINT32_MAX) return fail(SPED_ERR_UNSUPPORTED, "walk: too many edges");
    if (yt == SPED_F32 && vt == SPED_F32) return run_walk<float, float>(g, k, V, ldv, Y, ldy, mode, walkers, seed, st);
    if (yt == SPED_F64 && vt == SPED_F64) return run_walk<double, double>(g, k, V, ldv, Y, ldy, mode, walkers, seed, st);
    if (yt == SPED_F64 && vt == SPED_F32) return run_walk<float, double>(g, k, V, ldv, Y, ldy, mode, walkers, seed, st);
    if (yt == SPED_F32 && vt == SPED_BF16) return run_walk<__nv_bfloat16, float>(g, k, V, ldv, Y, ldy, mode, walkers, seed, st);
    return fail(SPED_ERR_UNSUPPORTED, "walk: V dtype %d / Y dtype %d (Y must be F32 or F64)",
                (int)vt, (int)yt);
}

}  // namespace sped
