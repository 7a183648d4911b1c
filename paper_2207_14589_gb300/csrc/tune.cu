// Chain-step schedule selection (the paper gives no kernel design to follow here). The best
// schedule for one step X -> (I - sL) X depends on the graph: the row-group kernel is fastest
// when degrees are even, the merge path when a few rows hold a large share of the entries, and
// the merge path's share size trades the L2 locality of the rows in flight against the number
// of partial rows left for the fix-up. sped_autotune times the candidates on the caller's graph
// and keeps the fastest in the graph handle and in a per-process table keyed by the graph's
// shape (n, nnz, maximum degree, weights, k, chain dtype, device), so that a later graph of
// the same shape takes the choice without timing.
#include <cstring>
#include <mutex>
#include <unordered_map>

#include "sped_internal.cuh"

namespace sped {

constexpr int TUNE_IPG[] = {128, 256, 512, 1024};
constexpr int TUNE_NIPG = (int)(sizeof(TUNE_IPG) / sizeof(TUNE_IPG[0]));
constexpr int TUNE_REPS = 3;

struct TuneChoice {
    int split, ipg;
};

static std::mutex g_tune_mu;
static std::unordered_map<uint64_t, TuneChoice> g_tune_table;

static uint64_t mix(uint64_t h, uint64_t v) {
    h ^= v + 0x9E3779B97F4A7C15ull + (h << 6) + (h >> 2);
    return h;
}

static uint64_t shape_key(const sped_graph *g, int k, sped_dtype ct) {
    uint64_t h = 0x5BD1E995ull;
    h = mix(h, (uint64_t)g->n);
    h = mix(h, (uint64_t)g->nnz);
    h = mix(h, (uint64_t)g->max_deg);
    h = mix(h, g->w != nullptr);
    h = mix(h, (uint64_t)k);
    h = mix(h, (uint64_t)ct);
    h = mix(h, (uint64_t)g->device);
    h = mix(h, (uint64_t)device_sm_count());
    return h;
}

// scratch for tuning: the input and output blocks plus the merge-path partials at the
// smallest candidate share
static size_t tune_layout(const sped_graph *g, int k, sped_dtype ct, size_t *block) {
    *block = align_up((size_t)g->n * padded_ld(k, ct) * dtype_size(ct), 256);
    return 2 * *block + merge_step_scratch(g, k, ct, TUNE_IPG[0]) + 256;
}

}  // namespace sped

using namespace sped;

extern "C" {

sped_status sped_autotune_scratch_size(const sped_graph *g, int k, sped_dtype chain_t,
                                       size_t *bytes) {
    if (!g || !bytes || k < 1 || k > 256 || !dtype_valid(chain_t))
        return fail(SPED_ERR_INVALID_ARG, "autotune_scratch_size: bad arguments");
    size_t block;
    *bytes = tune_layout(g, k, chain_t, &block);
    return SPED_OK;
}

sped_status sped_set_schedule(sped_graph *g, int split, int merge_ipg) {
    if (!g) return fail(SPED_ERR_INVALID_ARG, "set_schedule: null graph");
    if (split < 0 || split > 2)
        return fail(SPED_ERR_INVALID_ARG, "set_schedule: split %d not in 0..2", split);
    if (merge_ipg != 0 && (merge_ipg < 32 || merge_ipg > (1 << 20)))
        return fail(SPED_ERR_INVALID_ARG, "set_schedule: merge share %d not in 32..2^20",
                    merge_ipg);
    g->tuned_split = split;
    g->merge_ipg = merge_ipg;
    return SPED_OK;
}

sped_status sped_autotune(sped_graph *g, int k, sped_dtype chain_t, void *d_scratch,
                          size_t scratch_bytes, void *stream, sped_tune_report *rep) {
    if (!g || k < 1 || !dtype_valid(chain_t))
        return fail(SPED_ERR_INVALID_ARG, "autotune: bad arguments");
    sped_tune_report r;
    std::memset(&r, 0, sizeof(r));
    const uint64_t key = shape_key(g, k, chain_t);
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto it = g_tune_table.find(key);
        if (it != g_tune_table.end()) {
            g->tuned_split = it->second.split;
            g->merge_ipg = it->second.ipg;
            r.split = it->second.split;
            r.merge_ipg = it->second.ipg;
            r.cached = 1;
            if (rep) *rep = r;
            return SPED_OK;
        }
    }
    size_t block;
    const size_t need = tune_layout(g, k, chain_t, &block);
    if (!d_scratch || scratch_bytes < need || ((uintptr_t)d_scratch) % 256)
        return fail(SPED_ERR_SCRATCH, "autotune: scratch needs %zu bytes (256-aligned)", need);
    cudaStream_t st = as_stream(stream);
    const int ld = padded_ld(k, chain_t);
    char *base = (char *)d_scratch;
    void *X = base, *Y = base + block;
    SPED_CUDA(cudaMemsetAsync(X, 0, block, st));
    const int saved_split = g->tuned_split, saved_ipg = g->merge_ipg;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    sped_status status = SPED_OK;
    auto cleanup = [&](sped_status s) {
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (s != SPED_OK) {
            g->tuned_split = saved_split;
            g->merge_ipg = saved_ipg;
        }
        return s;
    };
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return cleanup(fail(SPED_ERR_CUDA, "autotune: event creation failed"));
    TuneChoice best{1, 0};
    double best_ms = 1e300;
    for (int c = 0; c <= TUNE_NIPG; ++c) {
        g->tuned_split = c == 0 ? 1 : 2;
        g->merge_ipg = c == 0 ? saved_ipg : TUNE_IPG[c - 1];
        auto step = [&]() {
            Scratch scr(base + 2 * block, scratch_bytes - 2 * block);
            return launch_poly_step(g, k, X, chain_t, ld, nullptr, chain_t, ld, Y, chain_t, ld,
                                    0.0, -0.01, 1.0, 0, scr, st);
        };
        status = step();  // warm-up (and the first touch of the partial buffers)
        if (status != SPED_OK) return cleanup(status);
        if (cudaEventRecord(e0, st) != cudaSuccess)
            return cleanup(fail(SPED_ERR_CUDA, "autotune: event record failed"));
        for (int i = 0; i < TUNE_REPS && status == SPED_OK; ++i) status = step();
        if (status != SPED_OK) return cleanup(status);
        float ms = 0.f;
        if (cudaEventRecord(e1, st) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess ||
            cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess)
            return cleanup(fail(SPED_ERR_CUDA, "autotune: timing failed"));
        r.ms[c] = ms / TUNE_REPS;
        r.n_candidates = c + 1;
        if (r.ms[c] < best_ms) {
            best_ms = r.ms[c];
            best = TuneChoice{g->tuned_split, c == 0 ? 0 : TUNE_IPG[c - 1]};
        }
    }
    g->tuned_split = best.split;
    g->merge_ipg = best.ipg;
    {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        g_tune_table[key] = best;
    }
    r.split = best.split;
    r.merge_ipg = best.ipg;
    if (rep) *rep = r;
    return cleanup(SPED_OK);
}

}  // extern "C"
