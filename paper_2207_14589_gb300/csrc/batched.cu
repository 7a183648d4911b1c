// Many independent graphs in one persistent launch: each CTA takes graphs from a work list
// ordered by decreasing size (longest-processing-time first; an atomic counter hands them
// out) and runs whole solver steps on its graph with CTA-local barriers only: the l chain steps
// of the limit form (I - s_g L_g)^l (Table 2), the Gram [V Y]^T [V Y], the FP64 k x k mu-EG
// algebra (Section 5.1) and the N_g x k update. No CTA ever waits for another, so the launch
// is safe to capture in a CUDA graph and replay.
//
// Schedule: threads per CTA (128, 256 or 512: a thread per row in the chain steps and the
// update, so small graphs waste fewer idle lanes with smaller CTAs) and CTAs per SM (the grid,
// and with it how many graphs are in flight). sped_batch_autotune times one solver step per
// candidate on the caller's batch and keeps the fastest in the handle; a per-process table
// keyed by the batch's shape serves later batches of the same shape.
#include <cstring>
#include <mutex>
#include <unordered_map>
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "sped_internal.cuh"

struct sped_batch {
    int device;
    int64_t n_graphs, n_total, nnz;
    const int32_t *rp, *ci;
    const float *w;
    int ell;
    int32_t *d_order;    // LPT order of graph ids
    int32_t *d_off;      // node offsets [G+1]
    double *d_scale;     // limit-form scale s_g per graph
    int32_t *d_counter;  // work-list counter
    std::vector<int64_t> h_off;
    std::vector<double> h_bound, h_scale;
    int threads = 512;     // schedule: threads per CTA
    int ctas_per_sm = 2;   // and CTAs per SM
};

namespace sped {

constexpr int BMAXK = 16;

struct BatchArgs {
    const int32_t *__restrict__ rp;
    const int32_t *__restrict__ ci;
    const float *__restrict__ w;
    const int32_t *__restrict__ order;
    const int32_t *__restrict__ off;
    const double *__restrict__ scale;
    int32_t *counter;
    int n_graphs;
    int ell, steps, k;
    double eta;
    float *V;       // master block, n_total x ldv (updated in place)
    int ldv;
    float *Y;       // scratch n_total x ldy
    int ldy;
    void *Xb0, *Xb1;  // chain scratch n_total x ldc
    int ldc;
    double *ritz;   // [G][k] Rayleigh quotients of M after the last step
    int *status;    // nonzero: a non-positive norm was met
};

// One chain step over rows [r0, r1): out = (1 - s d) x + s sum_j w_j x_j, thread per row.
template <typename Ti, typename To, bool W, int KP, int BT>
__device__ __forceinline__ void batch_chain_step(const BatchArgs &a, int r0, int r1, float s,
                                                 const Ti *X, int ldx, To *Yo, int ldo) {
    constexpr int E = 16 / (int)sizeof(Ti);
    constexpr int NC = KP / E;
    for (int r = r0 + threadIdx.x; r < r1; r += BT) {
        const int p0 = __ldg(a.rp + r), p1 = __ldg(a.rp + r + 1);
        float acc[KP];
#pragma unroll
        for (int i = 0; i < KP; ++i) acc[i] = 0.f;
        float d = 0.f;
        for (int p = p0; p < p1; ++p) {
            const int j = __ldg(a.ci + p);
            const float wv = W ? __ldg(a.w + p) : 1.f;
            d += wv;
#pragma unroll
            for (int q = 0; q < NC; ++q) {
                float x[E];
                load_chunk_coherent<Ti, E, float>(X + (int64_t)j * ldx + q * E, x);
#pragma unroll
                for (int i = 0; i < E; ++i) acc[q * E + i] += wv * x[i];
            }
        }
        const float a0 = 1.f - s * d;
#pragma unroll
        for (int q = 0; q < NC; ++q) {
            float x[E], y[E];
            load_chunk_coherent<Ti, E, float>(X + (int64_t)r * ldx + q * E, x);
#pragma unroll
            for (int i = 0; i < E; ++i) y[i] = a0 * x[i] + s * acc[q * E + i];
            // To chunks of E elements: E * sizeof(To) bytes, naturally aligned
            store_chunk<To, E, float>(Yo + (int64_t)r * ldo + q * E, y);
        }
    }
}

template <typename Tc, bool W, int KP, int BT>
__global__ void __launch_bounds__(BT) k_batch(BatchArgs a) {
    constexpr int K2 = 2 * KP;
    constexpr int NB = K2 / 4;
    constexpr int NP = NB * (NB + 1) / 2;
    __shared__ double sG[K2 * K2];
    __shared__ double sA[KP * KP];
    __shared__ double sS[KP];
    __shared__ int s_g;
    const int k = a.k;
    const int t = threadIdx.x;
    // Gram work split: worker = (pair of 4x4 blocks, slice of rows)
    const int pair = t % NP, slice = t / NP, nsl = BT / NP;
    int bi = 0, bj = 0;
    {
        int p = pair, row = 0, len = NB;
        while (p >= len) {
            p -= len;
            ++row;
            --len;
        }
        bi = row;
        bj = row + p;
    }
    const bool worker = slice < nsl;
    for (;;) {
        if (t == 0) s_g = atomicAdd(a.counter, 1);
        __syncthreads();
        const int gi = s_g;
        __syncthreads();
        if (gi >= a.n_graphs) break;
        const int g = a.order[gi];
        const int r0 = a.off[g], r1 = a.off[g + 1];
        const float s = (float)a.scale[g];
        for (int step = 0; step < a.steps; ++step) {
            // ---- chain: V (F32) -> Xb0 -> Xb1 -> ... -> Y (F32)
            for (int c = 0; c < a.ell; ++c) {
                const bool first = c == 0, last = c == a.ell - 1;
                Tc *xin = (Tc *)((c - 1) % 2 == 0 ? a.Xb0 : a.Xb1);
                Tc *xout = (Tc *)(c % 2 == 0 ? a.Xb0 : a.Xb1);
                if (first && last)
                    batch_chain_step<float, float, W, KP, BT>(a, r0, r1, s, a.V, a.ldv, a.Y,
                                                              a.ldy);
                else if (first)
                    batch_chain_step<float, Tc, W, KP, BT>(a, r0, r1, s, a.V, a.ldv, xout,
                                                           a.ldc);
                else if (last)
                    batch_chain_step<Tc, float, W, KP, BT>(a, r0, r1, s, xin, a.ldc, a.Y,
                                                           a.ldy);
                else
                    batch_chain_step<Tc, Tc, W, KP, BT>(a, r0, r1, s, xin, a.ldc, xout,
                                                        a.ldc);
                __syncthreads();
            }
            // ---- Gram of [V Y] over the graph's rows (F32 per worker, F64 in shared memory)
            for (int e = t; e < K2 * K2; e += BT) sG[e] = 0.0;
            __syncthreads();
            if (worker) {
                float acc[16];
#pragma unroll
                for (int q = 0; q < 16; ++q) acc[q] = 0.f;
                for (int r = r0 + slice; r < r1; r += nsl) {
                    float x[4], y[4];
#pragma unroll
                    for (int q = 0; q < 4; ++q) {
                        const int ci = bi * 4 + q, cj = bj * 4 + q;
                        x[q] = ci < KP ? a.V[(int64_t)r * a.ldv + ci] : a.Y[(int64_t)r * a.ldy + ci - KP];
                        y[q] = cj < KP ? a.V[(int64_t)r * a.ldv + cj] : a.Y[(int64_t)r * a.ldy + cj - KP];
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u)
#pragma unroll
                        for (int v = 0; v < 4; ++v) acc[u * 4 + v] += x[u] * y[v];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
#pragma unroll
                    for (int v = 0; v < 4; ++v) {
                        const int i = bi * 4 + u, j = bj * 4 + v;
                        atomicAdd(&sG[i * K2 + j], (double)acc[u * 4 + v]);
                        if (bi != bj) atomicAdd(&sG[j * K2 + i], (double)acc[u * 4 + v]);
                    }
            }
            __syncthreads();
            // ---- mu-EG coefficients in FP64 (P = V^T V, H = V^T Y, Q = Y^T Y)
            if (t < k) {
                const int i = t;
                auto P = [&](int x, int y) { return sG[x * K2 + y]; };
                auto H = [&](int x, int y) { return sG[x * K2 + KP + y]; };
                auto Q = [&](int x, int y) { return sG[(KP + x) * K2 + KP + y]; };
                const double eta = a.eta;
                double cc = H(i, i);
                for (int j = 0; j < i; ++j) cc -= H(i, j) * P(i, j);
                double av[BMAXK];
                for (int j = 0; j < KP; ++j) av[j] = 0.0;
                for (int j = 0; j < i; ++j) av[j] = -eta * H(i, j);
                av[i] = 1.0 - eta * cc;
                double nrm = eta * eta * Q(i, i);
                for (int j = 0; j <= i; ++j) {
                    double sm = 0.0;
                    for (int l = 0; l <= i; ++l) sm += av[l] * P(j, l);
                    nrm += av[j] * sm + 2.0 * eta * av[j] * H(j, i);
                }
                for (int j = 0; j < KP; ++j) sA[j * KP + i] = av[j];
                if (!(nrm > 0.0) || !isfinite(nrm)) {
                    atomicOr(a.status, 1);
                    sS[i] = 0.0;
                } else {
                    sS[i] = 1.0 / sqrt(nrm);
                }
                if (step == a.steps - 1) a.ritz[(int64_t)g * k + i] = H(i, i) / P(i, i);
            }
            __syncthreads();
            // ---- update V <- (V A + eta Y) diag(S), thread per row, in place
            for (int r = r0 + t; r < r1; r += BT) {
                float v[KP], y[KP];
#pragma unroll
                for (int j = 0; j < KP; ++j) {
                    v[j] = j < k ? a.V[(int64_t)r * a.ldv + j] : 0.f;
                    y[j] = j < k ? a.Y[(int64_t)r * a.ldy + j] : 0.f;
                }
#pragma unroll
                for (int i = 0; i < KP; ++i) {
                    if (i < k) {
                        float acc = (float)a.eta * y[i];
#pragma unroll
                        for (int j = 0; j <= i; ++j) acc += v[j] * (float)sA[j * KP + i];
                        a.V[(int64_t)r * a.ldv + i] = acc * (float)sS[i];
                    }
                }
            }
            __syncthreads();
        }
    }
}

__global__ void k_batch_bounds(const int32_t *rp, const float *w, const int32_t *off,
                               int n_graphs, double *bound, int *bad) {
    __shared__ double sm[256];
    const int g = blockIdx.x;
    if (g >= n_graphs) return;
    const int r0 = off[g], r1 = off[g + 1];
    double mx = 0.0;
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        double d = 0.0;
        for (int p = rp[r]; p < rp[r + 1]; ++p) d += w ? (double)w[p] : 1.0;
        mx = fmax(mx, d);
    }
    sm[threadIdx.x] = mx;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sm[threadIdx.x] = fmax(sm[threadIdx.x], sm[threadIdx.x + o]);
        __syncthreads();
    }
    if (threadIdx.x == 0) bound[g] = 2.0 * sm[0];
    (void)bad;
}

// block-diagonal check: every column of graph g lies in its node range, no self loops, sorted
__global__ void k_batch_check(const int32_t *rp, const int32_t *ci, const int32_t *off,
                              int n_graphs, int *bad) {
    const int g = blockIdx.x;
    if (g >= n_graphs) return;
    const int r0 = off[g], r1 = off[g + 1];
    for (int r = r0 + threadIdx.x; r < r1; r += blockDim.x) {
        int prev = -1;
        for (int p = rp[r]; p < rp[r + 1]; ++p) {
            const int c = ci[p];
            if (c < r0 || c >= r1 || c == r || c <= prev) atomicOr(bad, 1);
            prev = c;
        }
    }
}

struct BatchLayout {
    size_t order, off, scale, counter, bound, bad, total;
};

static BatchLayout batch_ws_layout(int64_t G) {
    BatchLayout L;
    ScratchPlan p;
    auto put = [&](size_t &o, size_t b) {
        p.used = align_up(p.used, 256);
        o = p.used;
        p.add(b);
    };
    put(L.order, sizeof(int32_t) * G);
    put(L.off, sizeof(int32_t) * (G + 1));
    put(L.scale, sizeof(double) * G);
    put(L.counter, sizeof(int32_t) * 4);
    put(L.bound, sizeof(double) * G);
    put(L.bad, sizeof(int32_t) * 4);
    L.total = p.total();
    return L;
}

static size_t batch_scratch_bytes(const sped_batch *b, int k, sped_dtype ct) {
    ScratchPlan p;
    const int KP = k <= 8 ? 8 : 16;
    p.add((size_t)b->n_total * KP * 4);                   // Y
    p.add((size_t)b->n_total * KP * dtype_size(ct));      // chain 0
    p.add((size_t)b->n_total * KP * dtype_size(ct));      // chain 1
    p.add(sizeof(int) * 4);                                // status
    return p.total();
}

// the solver steps with an explicit schedule (threads per CTA, CTAs per SM)
static sped_status batch_steps(const sped_batch *b, int steps, double eta, sped_dtype chain_t,
                               float *d_V, int k, int ld, double *d_ritz, void *d_scratch,
                               size_t scratch_bytes, cudaStream_t st, int threads, int cps) {
    if (steps < 1 || !(eta > 0.0) || !std::isfinite(eta))
        return fail(SPED_ERR_INVALID_ARG, "batch_eig_steps: steps >= 1 and eta > 0 required");
    if (k < 1 || k > BMAXK) return fail(SPED_ERR_UNSUPPORTED, "batch_eig_steps: k <= %d", BMAXK);
    if (chain_t != SPED_BF16 && chain_t != SPED_F32)
        return fail(SPED_ERR_INVALID_ARG, "batch_eig_steps: chain must be BF16 or F32");
    const int KP = k <= 8 ? 8 : 16;
    if (ld < KP || ((uintptr_t)d_V) % 16)
        return fail(SPED_ERR_INVALID_ARG, "batch_eig_steps: V needs ld >= %d and 16-byte "
                                          "alignment", KP);
    const size_t need = batch_scratch_bytes(b, k, chain_t);
    if (!d_scratch || scratch_bytes < need || ((uintptr_t)d_scratch) % 256)
        return fail(SPED_ERR_SCRATCH, "batch_eig_steps: scratch needs %zu bytes", need);
    Scratch scr(d_scratch, scratch_bytes);
    BatchArgs a;
    a.rp = b->rp;
    a.ci = b->ci;
    a.w = b->w;
    a.order = b->d_order;
    a.off = b->d_off;
    a.scale = b->d_scale;
    a.counter = b->d_counter;
    a.n_graphs = (int)b->n_graphs;
    a.ell = b->ell;
    a.steps = steps;
    a.k = k;
    a.eta = eta;
    a.V = d_V;
    a.ldv = ld;
    a.Y = (float *)scr.take((size_t)b->n_total * KP * 4);
    a.ldy = KP;
    a.Xb0 = scr.take((size_t)b->n_total * KP * dtype_size(chain_t));
    a.Xb1 = scr.take((size_t)b->n_total * KP * dtype_size(chain_t));
    a.ldc = KP;
    a.status = (int *)scr.take(sizeof(int) * 4);
    a.ritz = d_ritz;
    SPED_CUDA(cudaMemsetAsync(b->d_counter, 0, sizeof(int32_t), st));
    SPED_CUDA(cudaMemsetAsync(a.status, 0, sizeof(int), st));
    const int grid = device_sm_count() * cps;
    const bool W = b->w != nullptr;
#define LAUNCH(TC, WW, KK, NT) k_batch<TC, WW, KK, NT><<<grid, NT, 0, st>>>(a)
#define LAUNCH_T(TC, WW, KK)                            \
    do {                                                \
        if (threads == 128) LAUNCH(TC, WW, KK, 128);    \
        else if (threads == 256) LAUNCH(TC, WW, KK, 256); \
        else LAUNCH(TC, WW, KK, 512);                   \
    } while (0)
    if (chain_t == SPED_BF16) {
        if (KP == 8) { if (W) LAUNCH_T(__nv_bfloat16, true, 8); else LAUNCH_T(__nv_bfloat16, false, 8); }
        else { if (W) LAUNCH_T(__nv_bfloat16, true, 16); else LAUNCH_T(__nv_bfloat16, false, 16); }
    } else {
        if (KP == 8) { if (W) LAUNCH_T(float, true, 8); else LAUNCH_T(float, false, 8); }
        else { if (W) LAUNCH_T(float, true, 16); else LAUNCH_T(float, false, 16); }
    }
#undef LAUNCH_T
#undef LAUNCH
    SPED_CHECK_LAUNCH("k_batch");
    return SPED_OK;
}

// schedule candidates: {threads per CTA, CTAs per SM}
constexpr int BTUNE[][2] = {{512, 2}, {512, 4}, {256, 4}, {256, 8}, {128, 8}, {128, 16}};
constexpr int BTUNE_N = (int)(sizeof(BTUNE) / sizeof(BTUNE[0]));

static std::mutex g_btune_mu;
static std::unordered_map<uint64_t, std::pair<int, int>> g_btune;

static uint64_t batch_shape_key(const sped_batch *b, int k, sped_dtype ct) {
    uint64_t h = 0x42415443ull;
    auto mix = [&](uint64_t v) { h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2); };
    mix((uint64_t)b->n_graphs);
    mix((uint64_t)b->n_total);
    mix((uint64_t)b->nnz);
    mix((uint64_t)b->ell);
    mix(b->w != nullptr);
    mix((uint64_t)k);
    mix((uint64_t)ct);
    mix((uint64_t)b->device);
    mix((uint64_t)device_sm_count());
    return h;
}

struct BatchTuneLayout {
    size_t v, ritz, steps, total;
};

static BatchTuneLayout batch_tune_layout(const sped_batch *b, int k, sped_dtype ct) {
    BatchTuneLayout L;
    const int KP = k <= 8 ? 8 : 16;
    ScratchPlan p;
    L.v = 0;
    p.add((size_t)b->n_total * 16 * sizeof(float));  // copy of V (ld up to 16)
    p.used = align_up(p.used, 256);
    L.ritz = p.used;
    p.add(sizeof(double) * (size_t)b->n_graphs * BMAXK);
    p.used = align_up(p.used, 256);
    L.steps = p.used;
    p.add(batch_scratch_bytes(b, k, ct));
    L.total = p.total();
    (void)KP;
    return L;
}

}  // namespace sped

using namespace sped;

extern "C" {

sped_status sped_batch_workspace_size(int64_t n_graphs, size_t *bytes) {
    if (!bytes || n_graphs < 1) return fail(SPED_ERR_INVALID_ARG, "batch_workspace_size");
    *bytes = batch_ws_layout(n_graphs).total;
    return SPED_OK;
}

sped_status sped_batch_create(int64_t n_graphs, const int64_t *h_node_off,
                              const int32_t *d_row_ptr, const int32_t *d_col_idx,
                              const float *d_w, int degree, int check, void *d_workspace,
                              size_t ws_bytes, void *stream, sped_batch **out) {
    if (!out || !h_node_off || !d_row_ptr || !d_col_idx || n_graphs < 1)
        return fail(SPED_ERR_INVALID_ARG, "batch_create: null argument or no graphs");
    *out = nullptr;
    if (degree < 1 || degree % 2 == 0)
        return fail(SPED_ERR_INVALID_ARG, "batch_create: the limit form needs an odd degree");
    if (h_node_off[0] != 0) return fail(SPED_ERR_INVALID_ARG, "batch_create: offsets[0] != 0");
    for (int64_t g = 0; g < n_graphs; ++g)
        if (h_node_off[g + 1] <= h_node_off[g])
            return fail(SPED_ERR_INVALID_ARG, "batch_create: graph %lld is empty", (long long)g);
    const int64_t n_total = h_node_off[n_graphs];
    if (n_total >= INT32_MAX) return fail(SPED_ERR_UNSUPPORTED, "batch_create: too many nodes");
    BatchLayout L = batch_ws_layout(n_graphs);
    if (!d_workspace || ws_bytes < L.total || ((uintptr_t)d_workspace) % 256)
        return fail(SPED_ERR_SCRATCH, "batch_create: workspace needs %zu bytes", L.total);
    cudaStream_t st = as_stream(stream);
    char *ws = (char *)d_workspace;
    sped_batch *b = new sped_batch();
    cudaGetDevice(&b->device);
    b->n_graphs = n_graphs;
    b->n_total = n_total;
    b->rp = d_row_ptr;
    b->ci = d_col_idx;
    b->w = d_w;
    b->ell = degree;
    b->d_order = (int32_t *)(ws + L.order);
    b->d_off = (int32_t *)(ws + L.off);
    b->d_scale = (double *)(ws + L.scale);
    b->d_counter = (int32_t *)(ws + L.counter);
    b->h_off.assign(h_node_off, h_node_off + n_graphs + 1);
    std::vector<int32_t> off32(n_graphs + 1);
    for (int64_t g = 0; g <= n_graphs; ++g) off32[g] = (int32_t)h_node_off[g];
    int32_t nnz32 = 0;
    auto cleanup = [&](sped_status s) {
        delete b;
        return s;
    };
    cudaError_t e = cudaMemcpyAsync(b->d_off, off32.data(), sizeof(int32_t) * (n_graphs + 1),
                                    cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(&nnz32, d_row_ptr + n_total, sizeof(int32_t), cudaMemcpyDeviceToHost, st);
    int32_t *bad = (int32_t *)(ws + L.bad);
    if (e == cudaSuccess) e = cudaMemsetAsync(bad, 0, sizeof(int32_t), st);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "batch_create: copies"));
    if (check) k_batch_check<<<(unsigned)n_graphs, 256, 0, st>>>(d_row_ptr, d_col_idx, b->d_off,
                                                                 (int)n_graphs, bad);
    double *bound = (double *)(ws + L.bound);
    k_batch_bounds<<<(unsigned)n_graphs, 256, 0, st>>>(d_row_ptr, d_w, b->d_off, (int)n_graphs,
                                                       bound, bad);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "batch_create: kernels"));
    int hbad = 0;
    b->h_bound.resize(n_graphs);
    e = cudaMemcpyAsync(b->h_bound.data(), bound, sizeof(double) * n_graphs,
                        cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "batch_create: sync"));
    if (hbad)
        return cleanup(fail(SPED_ERR_BAD_CSR, "batch_create: a column leaves its graph's node "
                                              "range, or a row is unsorted / has a self loop"));
    b->nnz = nnz32;
    // per-graph scale (same automatic rule as sped_set_polynomial) and LPT order by nnz
    b->h_scale.resize(n_graphs);
    for (int64_t g = 0; g < n_graphs; ++g) {
        const double lb = b->h_bound[g];
        b->h_scale[g] = (lb <= 0.0 || degree >= lb / 2.0) ? 1.0 / degree : 2.0 / lb;
    }
    // graph sizes in nodes as the work estimate (edges per node are similar across the batch)
    std::vector<int32_t> order(n_graphs);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
        return (h_node_off[x + 1] - h_node_off[x]) > (h_node_off[y + 1] - h_node_off[y]);
    });
    e = cudaMemcpyAsync(b->d_order, order.data(), sizeof(int32_t) * n_graphs,
                        cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_scale, b->h_scale.data(), sizeof(double) * n_graphs,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cleanup(cuda_fail(e, "batch_create: upload"));
    *out = b;
    return SPED_OK;
}

void sped_batch_destroy(sped_batch *b) { delete b; }

sped_status sped_batch_scale(const sped_batch *b, double *h_scale, int capacity) {
    if (!b || !h_scale || capacity < b->n_graphs)
        return fail(SPED_ERR_INVALID_ARG, "batch_scale: bad arguments");
    for (int64_t g = 0; g < b->n_graphs; ++g) h_scale[g] = b->h_scale[g];
    return SPED_OK;
}

sped_status sped_batch_scratch_size(const sped_batch *b, int k, sped_dtype chain_t,
                                    size_t *bytes) {
    if (!b || !bytes || k < 1 || k > BMAXK || (chain_t != SPED_BF16 && chain_t != SPED_F32))
        return fail(SPED_ERR_INVALID_ARG, "batch_scratch_size: k in 1..%d, chain BF16 or F32",
                    BMAXK);
    *bytes = batch_scratch_bytes(b, k, chain_t);
    return SPED_OK;
}

sped_status sped_batch_eig_steps(const sped_batch *b, int steps, double eta, sped_dtype chain_t,
                                 float *d_V, int k, int ld, double *d_ritz, void *d_scratch,
                                 size_t scratch_bytes, void *stream) {
    if (!b || !d_V || !d_ritz) return fail(SPED_ERR_INVALID_ARG, "batch_eig_steps: null");
    return batch_steps(b, steps, eta, chain_t, d_V, k, ld, d_ritz, d_scratch, scratch_bytes,
                       as_stream(stream), b->threads, b->ctas_per_sm);
}

sped_status sped_batch_set_schedule(sped_batch *b, int threads, int ctas_per_sm) {
    if (!b) return fail(SPED_ERR_INVALID_ARG, "batch_set_schedule: null batch");
    if (threads != 128 && threads != 256 && threads != 512)
        return fail(SPED_ERR_INVALID_ARG, "batch_set_schedule: threads %d not 128, 256 or 512",
                    threads);
    if (ctas_per_sm < 1 || ctas_per_sm > 16)
        return fail(SPED_ERR_INVALID_ARG, "batch_set_schedule: %d CTAs per SM not in 1..16",
                    ctas_per_sm);
    b->threads = threads;
    b->ctas_per_sm = ctas_per_sm;
    return SPED_OK;
}

sped_status sped_batch_autotune_scratch_size(const sped_batch *b, int k, sped_dtype chain_t,
                                             size_t *bytes) {
    if (!b || !bytes || k < 1 || k > BMAXK || (chain_t != SPED_BF16 && chain_t != SPED_F32))
        return fail(SPED_ERR_INVALID_ARG, "batch_autotune_scratch_size: bad arguments");
    *bytes = batch_tune_layout(b, k, chain_t).total;
    return SPED_OK;
}

sped_status sped_batch_autotune(sped_batch *b, int k, sped_dtype chain_t, const float *d_V,
                                int ld, void *d_scratch, size_t scratch_bytes, void *stream,
                                sped_batch_tune_report *rep) {
    if (!b || !d_V || k < 1 || k > BMAXK || (chain_t != SPED_BF16 && chain_t != SPED_F32))
        return fail(SPED_ERR_INVALID_ARG, "batch_autotune: bad arguments");
    const int KP = k <= 8 ? 8 : 16;
    if (ld < KP || ((uintptr_t)d_V) % 16)
        return fail(SPED_ERR_INVALID_ARG, "batch_autotune: V needs ld >= %d, 16-byte aligned", KP);
    sped_batch_tune_report r;
    std::memset(&r, 0, sizeof(r));
    const uint64_t key = batch_shape_key(b, k, chain_t);
    {
        std::lock_guard<std::mutex> lk(g_btune_mu);
        auto it = g_btune.find(key);
        if (it != g_btune.end()) {
            b->threads = it->second.first;
            b->ctas_per_sm = it->second.second;
            r.threads = b->threads;
            r.ctas_per_sm = b->ctas_per_sm;
            r.cached = 1;
            if (rep) *rep = r;
            return SPED_OK;
        }
    }
    const BatchTuneLayout L = batch_tune_layout(b, k, chain_t);
    if (!d_scratch || scratch_bytes < L.total || ((uintptr_t)d_scratch) % 256)
        return fail(SPED_ERR_SCRATCH, "batch_autotune: scratch needs %zu bytes (256-aligned)",
                    L.total);
    cudaStream_t st = as_stream(stream);
    char *base = (char *)d_scratch;
    float *Vc = (float *)(base + L.v);
    double *ritz = (double *)(base + L.ritz);
    void *steps_scr = base + L.steps;
    const size_t steps_bytes = L.total - L.steps;
    // the copy of V is compact (ld = KP): only the KP columns the kernel reads
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&](sped_status s) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        return s;
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return cleanup(fail(SPED_ERR_CUDA, "batch_autotune: event creation failed"));
    int best = 0;
    double best_ms = 1e300;
    for (int c = 0; c < BTUNE_N; ++c) {
        const int th = BTUNE[c][0], cps = BTUNE[c][1];
        // every candidate starts from the caller's V, so all time the same work
        auto copy_v = [&]() {
            return cudaMemcpy2DAsync(Vc, sizeof(float) * KP, d_V, sizeof(float) * ld,
                                     sizeof(float) * KP, (size_t)b->n_total,
                                     cudaMemcpyDeviceToDevice, st);
        };
        if (copy_v() != cudaSuccess)
            return cleanup(fail(SPED_ERR_CUDA, "batch_autotune: copy of V failed"));
        sped_status s = batch_steps(b, 1, 1.0, chain_t, Vc, k, KP, ritz, steps_scr, steps_bytes,
                                    st, th, cps);  // warm-up
        if (s != SPED_OK) return cleanup(s);
        if (copy_v() != cudaSuccess || cudaEventRecord(e0, st) != cudaSuccess)
            return cleanup(fail(SPED_ERR_CUDA, "batch_autotune: timing set-up failed"));
        s = batch_steps(b, 1, 1.0, chain_t, Vc, k, KP, ritz, steps_scr, steps_bytes, st, th, cps);
        if (s != SPED_OK) return cleanup(s);
        float ms = 0.f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            return cleanup(fail(SPED_ERR_CUDA, "batch_autotune: timing failed"));
        r.ms[c] = ms;
        r.n_candidates = c + 1;
        if (ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    }
    b->threads = BTUNE[best][0];
    b->ctas_per_sm = BTUNE[best][1];
    {
        std::lock_guard<std::mutex> lk(g_btune_mu);
        g_btune[key] = {b->threads, b->ctas_per_sm};
    }
    r.threads = b->threads;
    r.ctas_per_sm = b->ctas_per_sm;
    if (rep) *rep = r;
    return cleanup(SPED_OK);
}

}  // extern "C"
