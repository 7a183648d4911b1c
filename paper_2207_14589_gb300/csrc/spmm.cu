// The hot kernel: one fused step of the polynomial chain,
//     Y = alpha V + gamma X + beta L X,   L = D - A  (Section 2; weighted: end of Section 2.1)
// chained by apply_poly into the limit form (I - sL)^l (Table 2, last row; alpha=0, gamma=1,
// beta=-s), Horner's rule for the Taylor rows of Table 2 (alpha=c_j, beta=1, gamma=shift), or
// the plain reversed Laplacian lambda* I - L of Eq. reveig (gamma=lambda*, beta=-1).
//
// Two schedules, same arithmetic:
//  * row-group: C = ceil(k * sizeof(Tx) / 16) lanes share one row, each owning one 16-byte
//    chunk of the row vector across all neighbours (no cross-lane reduction); 32/C rows per
//    warp; four neighbours in flight per lane. Degree d_r is summed in the same loop.
//  * merge-path: equal shares of (rows + nonzeros) per lane group (Merrill & Garland's merge
//    path over row ends and nonzeros) for skewed degree distributions; rows cut by a share
//    boundary leave partial sums in scratch, finished by a fix-up kernel in fixed order.
#include "sped_internal.cuh"

namespace sped {

constexpr int STEP_THREADS = 256;
constexpr int UNROLL = 4;

template <typename Tx, typename Tv, typename Ty, typename A, bool W, int HV>
struct StepArgs {
    int n;
    const int32_t *__restrict__ rp;
    const int32_t *__restrict__ ci;
    const float *__restrict__ w;
    const Tx *__restrict__ X;
    int ldx;
    const Tv *__restrict__ V;
    int ldv;
    Ty *__restrict__ Y;
    int ldy;
    int k;
    int C;
    A alpha, beta, gamma;
    const Tx *__restrict__ W2;  // HV == 2: a second block added with weight delta
    int ldw2;
    A delta;
};

// epilogue of row r for the lane's chunk: out = alpha v + gamma x + beta (d x - acc)
// (+ delta w2 when HV == 2: the three-term recurrences)
template <typename Tx, typename Tv, typename Ty, typename A, bool W, int HV, int E>
__device__ __forceinline__ void finish_row(const StepArgs<Tx, Tv, Ty, A, W, HV> &a, int64_t r,
                                           int c, const A (&acc)[E], A dsum) {
    A xr[E];
    load_chunk<Tx, E, A>(a.X + r * a.ldx + c * E, xr);
    A out[E];
#pragma unroll
    for (int i = 0; i < E; ++i) out[i] = a.gamma * xr[i] + a.beta * (dsum * xr[i] - acc[i]);
    const int rem = a.k - c * E;
    if constexpr (HV) {
        A vr[E];
        if (rem >= E) load_chunk<Tv, E, A>(a.V + r * a.ldv + c * E, vr);
        else load_partial<Tv, E, A>(a.V + r * a.ldv + c * E, rem, vr);
#pragma unroll
        for (int i = 0; i < E; ++i) out[i] += a.alpha * vr[i];
    }
    if constexpr (HV == 2) {
        A wr[E];
        if (rem >= E) load_chunk<Tx, E, A>(a.W2 + r * a.ldw2 + c * E, wr);
        else load_partial<Tx, E, A>(a.W2 + r * a.ldw2 + c * E, rem, wr);
#pragma unroll
        for (int i = 0; i < E; ++i) out[i] += a.delta * wr[i];
    }
    if (rem >= E) store_chunk<Ty, E, A>(a.Y + r * a.ldy + c * E, out);
    else store_partial<Ty, E, A>(a.Y + r * a.ldy + c * E, rem, out);
}

// accumulate neighbours [p, p1) of the lane's chunk into acc / dsum
template <typename Tx, typename Tv, typename Ty, typename A, bool W, int HV, int E>
__device__ __forceinline__ void gather_range(const StepArgs<Tx, Tv, Ty, A, W, HV> &a, int c, int p,
                                             int p1, A (&acc)[E], A &dsum) {
    const Tx *Xc = a.X + c * E;
    for (; p + UNROLL <= p1; p += UNROLL) {
        int j[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) j[u] = __ldg(a.ci + p + u);
        A x[UNROLL][E];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) load_chunk<Tx, E, A>(Xc + (int64_t)j[u] * a.ldx, x[u]);
        if constexpr (W) {
            A wv[UNROLL];
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) wv[u] = (A)__ldg(a.w + p + u);
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) {
                dsum += wv[u];
#pragma unroll
                for (int i = 0; i < E; ++i) acc[i] += wv[u] * x[u][i];
            }
        } else {
#pragma unroll
            for (int u = 0; u < UNROLL; ++u)
#pragma unroll
                for (int i = 0; i < E; ++i) acc[i] += x[u][i];
        }
    }
    for (; p < p1; ++p) {
        const int j = __ldg(a.ci + p);
        A x[E];
        load_chunk<Tx, E, A>(Xc + (int64_t)j * a.ldx, x);
        if constexpr (W) {
            const A wv = (A)__ldg(a.w + p);
            dsum += wv;
#pragma unroll
            for (int i = 0; i < E; ++i) acc[i] += wv * x[i];
        } else {
#pragma unroll
            for (int i = 0; i < E; ++i) acc[i] += x[i];
        }
    }
}

// Row-group schedule: C = ceil(k * sizeof(Tx) / 16) lanes share a row, each owning one 16-byte
// chunk of the row vector across all neighbours; four neighbours' indices and rows are in
// flight per lane. Column indices come through the read-only path (consecutive neighbours of a
// row share their sectors in L1). 32 registers keep all 64 warps of an SM resident: the kernel
// is bound by the latency and sector throughput of the random row gathers, so occupancy is
// what keeps bytes in flight.
//
// Launched with programmatic dependent launch: a launch may be scheduled while the previous
// kernel in the stream is finishing, and waits (griddepcontrol.wait) for it to complete and its
// writes to be visible before touching any memory; each block signals its dependents once its
// own row is written, so the next chain step's blocks fill the SMs as this step's last wave
// drains instead of after a launch gap.
template <typename Tx, typename Tv, typename Ty, typename A, bool W, int HV>
__global__ void __launch_bounds__(STEP_THREADS)
k_step_rowgroup(StepArgs<Tx, Tv, Ty, A, W, HV> a, int rows_per_warp) {
    pdl_wait();
    constexpr int E = 16 / (int)sizeof(Tx);
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * STEP_THREADS + threadIdx.x) >> 5;
    const int rw = lane / a.C;
    const int c = lane - rw * a.C;
    if (rw >= rows_per_warp) return;
    const int64_t r = warp * rows_per_warp + rw;
    if (r >= a.n) return;
    const int p0 = __ldg(a.rp + r), p1 = __ldg(a.rp + r + 1);
    A acc[E];
#pragma unroll
    for (int i = 0; i < E; ++i) acc[i] = A(0);
    A dsum = A(0);
    gather_range<Tx, Tv, Ty, A, W, HV, E>(a, c, p0, p1, acc, dsum);
    if constexpr (!W) dsum = (A)(p1 - p0);
    finish_row<Tx, Tv, Ty, A, W, HV, E>(a, r, c, acc, dsum);
    pdl_trigger();
}

// ---------------------------------------------------------------------------------------
// merge path
// ---------------------------------------------------------------------------------------
// first (row, nonzero) coordinate of merge-path diagonal `diag`: the number of row ends i and
// nonzeros j consumed, i + j = diag, row end i consumed once j >= rp[i+1].
__device__ __forceinline__ void merge_search(int64_t diag, int n, int nnz,
                                             const int32_t *__restrict__ rp, int &i, int &j) {
    int64_t lo = diag > nnz ? diag - nnz : 0;
    int64_t hi = diag < n ? diag : n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if ((int64_t)__ldg(rp + mid + 1) <= diag - mid - 1) lo = mid + 1;
        else hi = mid;
    }
    i = (int)lo;
    j = (int)(diag - lo);
}

// merge-path coordinates of every share boundary g * ipg (g = 0 .. n_groups), once per step
__global__ void k_merge_coords(int64_t n_groups, int64_t ipg, int n, int nnz,
                               const int32_t *__restrict__ rp, int2 *__restrict__ coords) {
    const int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (g > n_groups) return;
    const int64_t total = (int64_t)n + nnz;
    const int64_t d = g * ipg < total ? g * ipg : total;
    int i, j;
    merge_search(d, n, nnz, rp, i, j);
    coords[g] = make_int2(i, j);
}

template <typename A> struct MergeParts {
    A *acc;        // [groups][2][KP]  (0 = head, 1 = tail)
    A *dsum;       // [groups][2]
    int32_t *row;  // [groups][2]      (-1 = none)
    const int2 *coords;  // [groups + 1] merge-path coordinates of the share boundaries
    int KP;
};

template <typename Tx, typename Tv, typename Ty, typename A, bool W, int HV>
__global__ void __launch_bounds__(STEP_THREADS)
k_step_merge(StepArgs<Tx, Tv, Ty, A, W, HV> a, int nnz, int groups_per_warp,
             int64_t n_groups, MergeParts<A> parts) {
    constexpr int E = 16 / (int)sizeof(Tx);
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * STEP_THREADS + threadIdx.x) >> 5;
    const int gw = lane / a.C;
    const int c = lane - gw * a.C;
    if (gw >= groups_per_warp) return;
    const int64_t g = warp * groups_per_warp + gw;
    if (g >= n_groups) return;
    const int2 cs = parts.coords[g], ce = parts.coords[g + 1];
    const int i0 = cs.x, j0 = cs.y, i1 = ce.x, j1 = ce.y;
    const Tx *Xc = a.X + c * E;
    A acc[E];
#pragma unroll
    for (int i = 0; i < E; ++i) acc[i] = A(0);
    A dsum = A(0);
    int i = i0;
    int rstart = (i0 < a.n) ? __ldg(a.rp + i0) : nnz;  // first nonzero of row i
    int rnext = (i0 < a.n) ? __ldg(a.rp + i0 + 1) : nnz;
    int64_t hslot = g * 2;
    if (c == 0) {
        parts.row[hslot] = -1;
        parts.row[hslot + 1] = -1;
    }
    auto end_row = [&]() {
        A ds = dsum;
        if constexpr (!W) ds = (A)(rnext - (rstart > j0 ? rstart : j0));
        if (i > i0 || rstart >= j0) {
            if constexpr (!W) ds = (A)(rnext - rstart);
            finish_row<Tx, Tv, Ty, A, W, HV, E>(a, i, c, acc, ds);
        } else {  // row began in an earlier share: leave the head piece for the fix-up
#pragma unroll
            for (int q = 0; q < E; ++q) parts.acc[hslot * parts.KP + c * E + q] = acc[q];
            if (c == 0) {
                parts.dsum[hslot] = ds;
                parts.row[hslot] = i;
            }
        }
#pragma unroll
        for (int q = 0; q < E; ++q) acc[q] = A(0);
        dsum = A(0);
        ++i;
        rstart = rnext;
        rnext = (i < a.n) ? __ldg(a.rp + i + 1) : nnz;
    };
    int p = j0;
    for (; p + UNROLL <= j1; p += UNROLL) {
        int jj[UNROLL];
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) jj[u] = __ldg(a.ci + p + u);
        uint4 x[UNROLL];  // raw 16-byte chunks (E elements of Tx) until they are added
#pragma unroll
        for (int u = 0; u < UNROLL; ++u)
            x[u] = __ldg(reinterpret_cast<const uint4 *>(Xc + (int64_t)jj[u] * a.ldx));
        float wv[UNROLL];
        if constexpr (W) {
#pragma unroll
            for (int u = 0; u < UNROLL; ++u) wv[u] = __ldg(a.w + p + u);
        }
#pragma unroll
        for (int u = 0; u < UNROLL; ++u) {
            while (p + u >= rnext && i < i1) end_row();
            const Tx *e = reinterpret_cast<const Tx *>(&x[u]);
            if constexpr (W) {
                dsum += (A)wv[u];
#pragma unroll
                for (int q = 0; q < E; ++q) acc[q] += (A)wv[u] * cvt<A>(e[q]);
            } else {
#pragma unroll
                for (int q = 0; q < E; ++q) acc[q] += cvt<A>(e[q]);
            }
        }
    }
    for (; p < j1; ++p) {
        while (p >= rnext && i < i1) end_row();
        int jx = __ldg(a.ci + p);
        A x[E];
        load_chunk<Tx, E, A>(Xc + (int64_t)jx * a.ldx, x);
        if constexpr (W) {
            A wv = (A)__ldg(a.w + p);
            dsum += wv;
#pragma unroll
            for (int q = 0; q < E; ++q) acc[q] += wv * x[q];
        } else {
#pragma unroll
            for (int q = 0; q < E; ++q) acc[q] += x[q];
        }
    }
    while (i < i1) end_row();
    if (i1 < a.n) {  // unfinished last row: tail piece
        A ds = dsum;
        if constexpr (!W) ds = (A)(j1 - (rstart > j0 ? rstart : j0));
#pragma unroll
        for (int q = 0; q < E; ++q) parts.acc[(hslot + 1) * parts.KP + c * E + q] = acc[q];
        if (c == 0) {
            parts.dsum[hslot + 1] = ds;
            parts.row[hslot + 1] = i1;
        }
    }
}

// Finish rows cut by share boundaries: the share holding a row's end sums its head piece and
// the tail pieces of the preceding shares (walking back while they belong to the row).
template <typename Tx, typename Tv, typename Ty, typename A, bool W, int HV>
__global__ void __launch_bounds__(STEP_THREADS)
k_merge_fixup(StepArgs<Tx, Tv, Ty, A, W, HV> a, int groups_per_warp, int64_t n_groups,
              MergeParts<A> parts) {
    constexpr int E = 16 / (int)sizeof(Tx);
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * STEP_THREADS + threadIdx.x) >> 5;
    const int gw = lane / a.C;
    const int c = lane - gw * a.C;
    if (gw >= groups_per_warp) return;
    const int64_t g = warp * groups_per_warp + gw;
    if (g >= n_groups) return;
    const int r = parts.row[g * 2];
    if (r < 0) return;
    A acc[E];
    A dsum = parts.dsum[g * 2];
#pragma unroll
    for (int q = 0; q < E; ++q) acc[q] = parts.acc[(g * 2) * parts.KP + c * E + q];
    for (int64_t h = g - 1; h >= 0 && parts.row[h * 2 + 1] == r; --h) {
        dsum += parts.dsum[h * 2 + 1];
#pragma unroll
        for (int q = 0; q < E; ++q) acc[q] += parts.acc[(h * 2 + 1) * parts.KP + c * E + q];
    }
    finish_row<Tx, Tv, Ty, A, W, HV, E>(a, r, c, acc, dsum);
}

// ---------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------
static bool use_merge(const sped_graph *g, int split) {
    if (split == 1) return false;
    if (split == 2) return true;
    if (g->tuned_split) return g->tuned_split == 2;
    double avg = g->n ? (double)g->nnz / (double)g->n : 0.0;
    return g->max_deg > 128 && g->max_deg > 8.0 * avg;
}

// Items (row ends + stored entries) per merge-path share, unless sped_autotune chose another.
// Shares are taken in order by consecutive lane groups and CTAs are dispatched in index order,
// so the rows being worked on at any moment form a window of about (resident groups x share)
// items; a short share keeps that window's gather source inside L2 on graphs whose nodes are
// ordered by cluster, at the price of more partial rows for the fix-up.
constexpr int MERGE_IPG_DEFAULT = 256;

struct MergePlan {
    int64_t ipg, n_groups;
    int KP;
    size_t acc_bytes, dsum_bytes, row_bytes, coord_bytes;
};

static MergePlan merge_plan(const sped_graph *g, int k, sped_dtype xt, size_t acc_size) {
    MergePlan m;
    int E = chunk_elems(xt);
    int C = (k + E - 1) / E;
    int64_t total = g->n + g->nnz;
    m.ipg = g->merge_ipg > 0 ? g->merge_ipg : MERGE_IPG_DEFAULT;
    m.n_groups = (total + m.ipg - 1) / m.ipg;
    m.KP = C * E;
    m.acc_bytes = (size_t)m.n_groups * 2 * m.KP * acc_size;
    m.dsum_bytes = (size_t)m.n_groups * 2 * acc_size;
    m.row_bytes = (size_t)m.n_groups * 2 * sizeof(int32_t);
    m.coord_bytes = (size_t)(m.n_groups + 1) * sizeof(int2);
    return m;
}

size_t merge_step_scratch(const sped_graph *g, int k, sped_dtype xt, int ipg) {
    sped_graph probe_shape;  // only n, nnz and the share size enter the plan
    probe_shape.n = g->n;
    probe_shape.nnz = g->nnz;
    probe_shape.merge_ipg = ipg;
    MergePlan m = merge_plan(&probe_shape, k, xt, 8);
    ScratchPlan p;
    p.add(m.acc_bytes);
    p.add(m.dsum_bytes);
    p.add(m.row_bytes);
    p.add(m.coord_bytes);
    return p.total();
}

size_t poly_step_scratch(const sped_graph *g, int k, sped_dtype xt, int split) {
    if (!use_merge(g, split)) return 0;
    MergePlan m = merge_plan(g, k, xt, 8);
    ScratchPlan p;
    p.add(m.acc_bytes);
    p.add(m.dsum_bytes);
    p.add(m.row_bytes);
    p.add(m.coord_bytes);
    return p.total();
}

template <typename Tx, typename Tv, typename Ty, typename A, bool W, int HV>
static sped_status run_step(const sped_graph *g, int k, const void *X, int ldx, const void *V,
                            int ldv, void *Y, int ldy, double alpha, double beta, double gamma,
                            const void *W2, int ldw2, double delta, int split, Scratch &scr,
                            cudaStream_t st) {
    constexpr int E = 16 / (int)sizeof(Tx);
    StepArgs<Tx, Tv, Ty, A, W, HV> a;
    a.n = (int)g->n;
    a.rp = g->rp;
    a.ci = g->ci;
    a.w = g->w;
    a.X = (const Tx *)X;
    a.ldx = ldx;
    a.V = (const Tv *)V;
    a.ldv = ldv;
    a.Y = (Ty *)Y;
    a.ldy = ldy;
    a.k = k;
    a.C = (k + E - 1) / E;
    a.alpha = (A)alpha;
    a.beta = (A)beta;
    a.gamma = (A)gamma;
    a.W2 = (const Tx *)W2;
    a.ldw2 = ldw2;
    a.delta = (A)delta;
    if (a.C > 32) return fail(SPED_ERR_UNSUPPORTED, "poly_step: row of %d chunks > 32", a.C);
    const int per_warp = 32 / a.C;
    if (!use_merge(g, split)) {
        int64_t warps = (g->n + per_warp - 1) / per_warp;
        int64_t blocks = (warps * 32 + STEP_THREADS - 1) / STEP_THREADS;
        if (blocks > 0)
            SPED_CUDA(launch_pdl(k_step_rowgroup<Tx, Tv, Ty, A, W, HV>, dim3((unsigned)blocks),
                                 dim3(STEP_THREADS), 0, st, a, per_warp));
        SPED_CHECK_LAUNCH("k_step_rowgroup");
        return SPED_OK;
    }
    MergePlan m = merge_plan(g, k, sizeof(Tx) == 2 ? SPED_BF16 : sizeof(Tx) == 4 ? SPED_F32 : SPED_F64,
                             sizeof(A));
    MergeParts<A> parts;
    parts.acc = (A *)scr.take(m.acc_bytes);
    parts.dsum = (A *)scr.take(m.dsum_bytes);
    parts.row = (int32_t *)scr.take(m.row_bytes);
    int2 *coords = (int2 *)scr.take(m.coord_bytes);
    parts.coords = coords;
    parts.KP = m.KP;
    if (!parts.acc || !parts.dsum || !parts.row || !coords)
        return fail(SPED_ERR_SCRATCH, "poly_step (merge path): scratch too small");
    if (m.n_groups == 0) return SPED_OK;
    k_merge_coords<<<(unsigned)((m.n_groups + 1 + 255) / 256), 256, 0, st>>>(
        m.n_groups, m.ipg, (int)g->n, (int)g->nnz, g->rp, coords);
    SPED_CHECK_LAUNCH("k_merge_coords");
    int64_t warps = (m.n_groups + per_warp - 1) / per_warp;
    int64_t blocks = (warps * 32 + STEP_THREADS - 1) / STEP_THREADS;
    k_step_merge<Tx, Tv, Ty, A, W, HV><<<(unsigned)blocks, STEP_THREADS, 0, st>>>(
        a, (int)g->nnz, per_warp, m.n_groups, parts);
    SPED_CHECK_LAUNCH("k_step_merge");
    k_merge_fixup<Tx, Tv, Ty, A, W, HV><<<(unsigned)blocks, STEP_THREADS, 0, st>>>(
        a, per_warp, m.n_groups, parts);
    SPED_CHECK_LAUNCH("k_merge_fixup");
    return SPED_OK;
}

template <typename Tx, typename Tv, typename Ty, typename A, int HV>
static sped_status run_step_w(const sped_graph *g, int k, const void *X, int ldx, const void *V,
                              int ldv, void *Y, int ldy, double al, double be, double ga,
                              const void *W2, int ldw2, double de, int split, Scratch &scr,
                              cudaStream_t st) {
    if (g->w)
        return run_step<Tx, Tv, Ty, A, true, HV>(g, k, X, ldx, V, ldv, Y, ldy, al, be, ga, W2,
                                                 ldw2, de, split, scr, st);
    return run_step<Tx, Tv, Ty, A, false, HV>(g, k, X, ldx, V, ldv, Y, ldy, al, be, ga, W2, ldw2,
                                              de, split, scr, st);
}

using bf16 = __nv_bfloat16;

sped_status launch_poly_step_w2(const sped_graph *g, int k, const void *X, sped_dtype xt,
                                int ldx, const void *V, sped_dtype vt, int ldv, void *Y,
                                sped_dtype yt, int ldy, double al, double be, double ga,
                                const void *W2, int ldw2, double de, int split, Scratch &scr,
                                cudaStream_t st) {
    const bool hw = W2 != nullptr && de != 0.0;
    const bool hv = hw || (V != nullptr && al != 0.0);
    if (hw && !V) return fail(SPED_ERR_INVALID_ARG, "poly_step: a second block needs V");
#define STEP(TX, TV, TY, ACC, HVV)                                                            \
    return run_step_w<TX, TV, TY, ACC, HVV>(g, k, X, ldx, V, ldv, Y, ldy, al, be, ga, W2,      \
                                            ldw2, de, split, scr, st)
#define STEP_V(TX, TV, TY, ACC)                                                                \
    do {                                                                                       \
        if (hw) STEP(TX, TV, TY, ACC, 2);                                                      \
        STEP(TX, TV, TY, ACC, 1);                                                              \
    } while (0)
    if (!hv) {
        if (xt == SPED_F64 && yt == SPED_F64) STEP(double, double, double, double, 0);
        if (xt == SPED_F32 && yt == SPED_F32) STEP(float, float, float, float, 0);
        if (xt == SPED_BF16 && yt == SPED_BF16) STEP(bf16, bf16, bf16, float, 0);
        if (xt == SPED_F32 && yt == SPED_BF16) STEP(float, float, bf16, float, 0);
        if (xt == SPED_BF16 && yt == SPED_F32) STEP(bf16, bf16, float, float, 0);
        if (xt == SPED_F32 && yt == SPED_F64) STEP(float, float, double, double, 0);
    } else {
        if (xt == SPED_F64 && yt == SPED_F64 && vt == SPED_F64) STEP_V(double, double, double, double);
        if (xt == SPED_F64 && yt == SPED_F64 && vt == SPED_F32) STEP_V(double, float, double, double);
        if (xt == SPED_F32 && yt == SPED_F32 && vt == SPED_F32) STEP_V(float, float, float, float);
        if (xt == SPED_BF16 && yt == SPED_BF16 && vt == SPED_F32) STEP_V(bf16, float, bf16, float);
        if (xt == SPED_F32 && yt == SPED_BF16 && vt == SPED_F32) STEP_V(float, float, bf16, float);
        if (xt == SPED_BF16 && yt == SPED_F32 && vt == SPED_F32) STEP_V(bf16, float, float, float);
        if (xt == SPED_F32 && yt == SPED_F64 && vt == SPED_F32) STEP_V(float, float, double, double);
        if (xt == SPED_F32 && yt == SPED_F64 && vt == SPED_F64) STEP_V(float, double, double, double);
    }
#undef STEP_V
#undef STEP
    return fail(SPED_ERR_UNSUPPORTED, "poly_step: unsupported dtype combination x=%d y=%d v=%d",
                (int)xt, (int)yt, hv ? (int)vt : -1);
}

sped_status launch_poly_step(const sped_graph *g, int k, const void *X, sped_dtype xt, int ldx,
                             const void *V, sped_dtype vt, int ldv, void *Y, sped_dtype yt,
                             int ldy, double al, double be, double ga, int split, Scratch &scr,
                             cudaStream_t st) {
    return launch_poly_step_w2(g, k, X, xt, ldx, V, vt, ldv, Y, yt, ldy, al, be, ga, nullptr, 0,
                               0.0, split, scr, st);
}

// ---------------------------------------------------------------------------------------
// exact p(L) V: the chain of steps for the graph's polynomial
// ---------------------------------------------------------------------------------------
struct StepCoef {
    double alpha, beta, gamma;
    bool uses_v;
    double delta = 0.0;   // weight of the output of the step before last (Clenshaw)
    bool uses_w2 = false;
};

static std::vector<StepCoef> chain_coefs(const Poly &P) {
    std::vector<StepCoef> out;
    if (P.kind == SPED_POLY_LIMIT_EXP) {
        for (int t = 0; t < P.ell; ++t) out.push_back({0.0, -P.s, 1.0, false});
    } else if (P.kind == SPED_POLY_SHIFT) {
        out.push_back({0.0, -1.0, P.lambda_star, false});
    } else if (P.kind == SPED_POLY_CHEBYSHEV) {
        // Clenshaw with x = al L + be I: b_j = c_j V + 2 x b_{j+1} - b_{j+2} (b_{l+1} = b_{l+2}
        // = 0, so b_l = c_l V is folded into the first two steps), then M V = c_0 V + x b_1 - b_2
        const auto &c = P.cheb;
        const int l = P.ell;
        const double al = 2.0 / (P.cheb_b - P.cheb_a), be = -(P.cheb_a + P.cheb_b) / (P.cheb_b - P.cheb_a);
        if (l == 1) {
            out.push_back({0.0, al * c[1], c[0] + be * c[1], false});
            return out;
        }
        out.push_back({0.0, 2.0 * al * c[l], c[l - 1] + 2.0 * be * c[l], false});  // b_{l-1}
        for (int j = l - 2; j >= 1; --j) {                                        // b_j
            if (j + 2 == l) out.push_back({c[j] - c[l], 2.0 * al, 2.0 * be, true});
            else out.push_back({c[j], 2.0 * al, 2.0 * be, true, -1.0, true});
        }
        if (l == 2) out.push_back({c[0] - c[2], al, be, true});                 // M V
        else out.push_back({c[0], al, be, true, -1.0, true});
    } else {
        const auto &h = P.horner;
        const int l = P.ell;
        // Z_{l-1} = h_{l-1} V + T (h_l V) = (h_{l-1} + h_l shift) V + h_l L V
        out.push_back({0.0, h[l], h[l - 1] + h[l] * P.shift, false});
        for (int j = l - 2; j >= 0; --j) out.push_back({h[j], 1.0, P.shift, true});
    }
    return out;
}

// chain buffers: two in turn, three when a step also reads the output of the step before last
static int chain_buffers(const std::vector<StepCoef> &cs) {
    const int steps = (int)cs.size();
    bool w2 = false;
    for (const auto &c : cs) w2 = w2 || c.uses_w2;
    return steps < 2 ? 0 : steps == 2 ? 1 : (w2 ? 3 : 2);
}

size_t apply_poly_scratch(const sped_graph *g, int k, sped_dtype ct, sped_mode mode) {
    if (mode != SPED_EXACT && mode != SPED_STOCHASTIC_MINIBATCH &&
        mode != SPED_STOCHASTIC_MINIBATCH_STRATIFIED)
        return 0;
    const int nbuf = chain_buffers(chain_coefs(g->poly));
    ScratchPlan p;
    size_t buf = (size_t)g->n * padded_ld(k, ct) * dtype_size(ct);
    for (int i = 0; i < nbuf; ++i) p.add(buf);
    if (mode != SPED_EXACT) return p.total();
    size_t ms = 0;
    for (sped_dtype t : {SPED_BF16, SPED_F32, SPED_F64}) {
        size_t x = poly_step_scratch(g, k, t, 0);
        if (x > ms) ms = x;
    }
    p.add(ms);
    return p.total();
}

sped_status apply_poly_impl(const sped_graph *g, int k, const void *V, sped_dtype vt, int ldv,
                            void *Y, sped_dtype yt, int ldy, sped_dtype ct, sped_mode mode,
                            int64_t walkers, uint64_t seed, Scratch &scr, cudaStream_t st,
                            const void *X0, sped_dtype x0t, int ldx0) {
    if (mode == SPED_STOCHASTIC_IS || mode == SPED_STOCHASTIC_REJECT)
        return launch_walk(g, k, V, vt, ldv, Y, yt, ldy, mode, walkers, seed, st);
    const bool stratified = mode == SPED_STOCHASTIC_MINIBATCH_STRATIFIED;
    const bool minibatch = mode == SPED_STOCHASTIC_MINIBATCH || stratified;
    if (mode != SPED_EXACT && !minibatch)
        return fail(SPED_ERR_INVALID_ARG, "apply_poly: mode %d", (int)mode);
    if (minibatch) {
        if (walkers < 1 || walkers > (int64_t)UINT32_MAX + 1)
            return fail(SPED_ERR_INVALID_ARG, "minibatch: %lld edges per batch not in 1..2^32",
                        (long long)walkers);
        if (ct == SPED_BF16)
            return fail(SPED_ERR_UNSUPPORTED, "minibatch: the chain accumulates by atomic adds, "
                                              "chain dtype must be F32 or F64");
        X0 = nullptr;  // the first multiplication reads V itself
    }
    std::vector<StepCoef> cs = chain_coefs(g->poly);
    const int steps = (int)cs.size();
    const int ldc = padded_ld(k, ct);
    const size_t buf = (size_t)g->n * ldc * dtype_size(ct);
    const int nbuf = chain_buffers(cs);
    void *b[3] = {nullptr, nullptr, nullptr};
    for (int i = 0; i < nbuf; ++i) {
        b[i] = scr.take(buf);
        if (!b[i]) return fail(SPED_ERR_SCRATCH, "apply_poly: scratch too small for the chain buffers");
    }
    const int nb = nbuf > 0 ? nbuf : 1;
    // what is left of the caller's scratch after the chain buffers serves each step in turn
    const size_t off = align_up(scr.used, 256);
    const size_t rest = (scr.base != nullptr && off < scr.cap) ? scr.cap - off : 0;
    Scratch step_scr(rest ? scr.base + off : nullptr, rest);
    // the first step reads X0 (a lower-precision copy of V) when the caller provides one
    const void *x_first = X0 ? X0 : V;
    const sped_dtype xt_first = X0 ? x0t : vt;
    const int ldx_first = X0 ? ldx0 : ldv;
    for (int t = 0; t < steps; ++t) {
        const void *x = t == 0 ? x_first : b[(t - 1) % nb];
        sped_dtype xt = t == 0 ? xt_first : ct;
        int ldx = t == 0 ? ldx_first : ldc;
        void *y = t == steps - 1 ? Y : b[t % nb];
        sped_dtype ytt = t == steps - 1 ? yt : ct;
        int ldyy = t == steps - 1 ? ldy : ldc;
        const void *w2 = cs[t].uses_w2 ? b[(t - 2) % nb] : nullptr;  // output of step t - 2
        if (minibatch) {
            EdgeBatch eb;
            eb.graph = g->n_edges > 0 ? g : nullptr;  // no edges: L = 0, nothing to add
            eb.seed = seed;
            eb.step = (uint32_t)t;
            eb.count = g->n_edges > 0 ? walkers : 0;
            eb.scale = stratified ? 1.0 : (double)g->n_edges / (double)walkers;
            eb.stratified = stratified;
            SPED_TRY(launch_edge_step(g->n, k, x, xt, ldx, cs[t].uses_v ? V : nullptr, vt, ldv,
                                      w2, ldc, cs[t].delta, y, ytt, ldyy, cs[t].alpha,
                                      cs[t].beta, cs[t].gamma, eb, st));
            continue;
        }
        step_scr.used = 0;
        SPED_TRY(launch_poly_step_w2(g, k, x, xt, ldx, cs[t].uses_v ? V : nullptr, vt, ldv, y,
                                     ytt, ldyy, cs[t].alpha, cs[t].beta, cs[t].gamma, w2, ldc,
                                     cs[t].delta, 0, step_scr, st));
    }
    return SPED_OK;
}

}  // namespace sped

using namespace sped;

extern "C" {

sped_status sped_poly_step_scratch_size(const sped_graph *g, int k, sped_dtype x_t, int split,
                                        size_t *bytes) {
    if (!g || !bytes || k < 1 || !dtype_valid(x_t))
        return fail(SPED_ERR_INVALID_ARG, "poly_step_scratch_size: bad args");
    *bytes = poly_step_scratch(g, k, x_t, split);
    return SPED_OK;
}

sped_status sped_poly_step(const sped_graph *g, int k, const void *d_X, sped_dtype x_t, int ldx,
                           const void *d_V, sped_dtype v_t, int ldv, void *d_Y, sped_dtype y_t,
                           int ldy, double alpha, double beta, double gamma, int split,
                           void *d_scratch, size_t scratch_bytes, void *stream) {
    if (!g) return fail(SPED_ERR_INVALID_ARG, "poly_step: null graph");
    if (split < 0 || split > 2) return fail(SPED_ERR_INVALID_ARG, "poly_step: split %d", split);
    SPED_TRY(check_layout(d_X, x_t, k, ldx, "poly_step X"));
    SPED_TRY(check_layout(d_Y, y_t, k, ldy, "poly_step Y"));
    if (d_V && alpha != 0.0) SPED_TRY(check_layout(d_V, v_t, k, ldv, "poly_step V"));
    if (d_X == d_Y) return fail(SPED_ERR_INVALID_ARG, "poly_step: X and Y must not alias");
    Scratch scr(d_scratch, scratch_bytes);
    return launch_poly_step(g, k, d_X, x_t, ldx, d_V, v_t, ldv, d_Y, y_t, ldy, alpha, beta, gamma,
                            split, scr, as_stream(stream));
}

sped_status sped_apply_poly_scratch_size(const sped_graph *g, int k, sped_dtype chain_t,
                                         sped_mode mode, size_t *bytes) {
    if (!g || !bytes || k < 1 || !dtype_valid(chain_t))
        return fail(SPED_ERR_INVALID_ARG, "apply_poly_scratch_size: bad args");
    *bytes = apply_poly_scratch(g, k, chain_t, mode);
    return SPED_OK;
}

sped_status sped_apply_poly(const sped_graph *g, int k, const void *d_V, sped_dtype v_t, int ldv,
                            void *d_Y, sped_dtype y_t, int ldy, sped_dtype chain_t, sped_mode mode,
                            int64_t walkers, uint64_t seed, void *d_scratch, size_t scratch_bytes,
                            void *stream) {
    if (!g) return fail(SPED_ERR_INVALID_ARG, "apply_poly: null graph");
    SPED_TRY(check_layout(d_V, v_t, k, ldv, "apply_poly V"));
    SPED_TRY(check_layout(d_Y, y_t, k, ldy, "apply_poly Y"));
    if (!dtype_valid(chain_t)) return fail(SPED_ERR_INVALID_ARG, "apply_poly: chain dtype");
    if (mode != SPED_EXACT && mode != SPED_STOCHASTIC_IS && mode != SPED_STOCHASTIC_REJECT &&
        mode != SPED_STOCHASTIC_MINIBATCH && mode != SPED_STOCHASTIC_MINIBATCH_STRATIFIED)
        return fail(SPED_ERR_INVALID_ARG, "apply_poly: mode %d", (int)mode);
    if (d_V == d_Y) return fail(SPED_ERR_INVALID_ARG, "apply_poly: V and Y must not alias");
    Scratch scr(d_scratch, scratch_bytes);
    return apply_poly_impl(g, k, d_V, v_t, ldv, d_Y, y_t, ldy, chain_t, mode, walkers, seed, scr,
                           as_stream(stream), nullptr, SPED_BF16, 0);
}

sped_status sped_apply_poly_backward(const sped_graph *g, int k, const void *d_dY, sped_dtype dy_t,
                                     int lddy, void *d_dV, sped_dtype dv_t, int lddv,
                                     sped_dtype chain_t, void *d_scratch, size_t scratch_bytes,
                                     void *stream) {
    if (!g) return fail(SPED_ERR_INVALID_ARG, "apply_poly_backward: null graph");
    SPED_TRY(check_layout(d_dY, dy_t, k, lddy, "apply_poly_backward dY"));
    SPED_TRY(check_layout(d_dV, dv_t, k, lddv, "apply_poly_backward dV"));
    if (!dtype_valid(chain_t)) return fail(SPED_ERR_INVALID_ARG, "apply_poly_backward: chain dtype");
    if (d_dY == d_dV) return fail(SPED_ERR_INVALID_ARG, "apply_poly_backward: dY and dV alias");
    // M = p(L) is symmetric (L is), so the adjoint of V -> M V is M itself: the same chain
    Scratch scr(d_scratch, scratch_bytes);
    return apply_poly_impl(g, k, d_dY, dy_t, lddy, d_dV, dv_t, lddv, chain_t, SPED_EXACT, 0, 0, scr,
                           as_stream(stream), nullptr, SPED_BF16, 0);
}

}  // extern "C"
