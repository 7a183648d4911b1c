// Gather-rate probe (a measurement entry point, not on the solver path). The chain step's time
// is set by how fast the memory system serves its random row gathers, not by DRAM bandwidth:
// every stored entry pulls one k-column row of X from wherever it lies. This kernel reproduces
// the chain step's access stream without its arithmetic so that the step can be compared with
// what the GPU delivers for the same gathers:
//   mode 0: the CSR as given -- row r's lanes read col_idx[p] and gather those rows;
//   mode 1: the same number of gathers per row from uniformly hashed rows (no index stream);
//   mode 2: the same number of gathers per row from the consecutive rows r+1, r+2, ... (mod n):
//           the non-random case, where neighbouring lanes share cache lines.
// Same launch shape as the row-group chain step (a group of C lanes per row, one 16-byte chunk
// per lane, four gathers in flight per lane); each row writes the sum of its gathered chunks
// (BF16) so the loads stay live.
#include "sped_internal.cuh"

namespace sped {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_UNROLL = 4;

__device__ __forceinline__ uint32_t probe_hash(uint32_t x, uint32_t seed) {
    x ^= seed;
    x ^= x >> 16;
    x *= 0x7FEB352Du;
    x ^= x >> 15;
    x *= 0x846CA68Bu;
    x ^= x >> 16;
    return x;
}

template <int MODE>
__device__ __forceinline__ int64_t probe_col(const int32_t *__restrict__ ci, int64_t n, int64_t r,
                                             int p, int p0, uint32_t seed) {
    if constexpr (MODE == 0) return __ldg(ci + p);
    if constexpr (MODE == 1) return (int64_t)__umulhi(probe_hash((uint32_t)p, seed), (uint32_t)n);
    int64_t j = r + 1 + (p - p0);
    return j >= n ? j % n : j;
}

template <int MODE>
__global__ void __launch_bounds__(PROBE_THREADS)
    k_probe_gather(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                   const __nv_bfloat16 *__restrict__ X, int ldx, __nv_bfloat16 *__restrict__ Y,
                   int ldy, int C, int rows_per_warp, uint32_t seed) {
    constexpr int E = 8;
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * PROBE_THREADS + threadIdx.x) >> 5;
    const int rw = lane / C;
    const int c = lane - rw * C;
    if (rw >= rows_per_warp) return;
    const int64_t r = warp * rows_per_warp + rw;
    if (r >= n) return;
    const int p0 = __ldg(rp + r), p1 = __ldg(rp + r + 1);
    float acc[E];
#pragma unroll
    for (int i = 0; i < E; ++i) acc[i] = 0.f;
    const __nv_bfloat16 *Xc = X + c * E;
    int p = p0;
    for (; p + PROBE_UNROLL <= p1; p += PROBE_UNROLL) {
        int64_t j[PROBE_UNROLL];
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u) j[u] = probe_col<MODE>(ci, n, r, p + u, p0, seed);
        float x[PROBE_UNROLL][E];
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u) load_chunk<__nv_bfloat16, E, float>(Xc + j[u] * ldx, x[u]);
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u)
#pragma unroll
            for (int i = 0; i < E; ++i) acc[i] += x[u][i];
    }
    for (; p < p1; ++p) {
        const int64_t j = probe_col<MODE>(ci, n, r, p, p0, seed);
        float x[E];
        load_chunk<__nv_bfloat16, E, float>(Xc + j * ldx, x);
#pragma unroll
        for (int i = 0; i < E; ++i) acc[i] += x[i];
    }
    store_chunk<__nv_bfloat16, E, float>(Y + r * ldy + c * E, acc);
}

}  // namespace sped

using namespace sped;

extern "C" {

sped_status sped_probe_gather(const sped_graph *g, int k, const void *d_X, int ldx, void *d_Y,
                              int ldy, int mode, uint64_t seed, void *stream) {
    if (!g) return fail(SPED_ERR_INVALID_ARG, "probe_gather: null graph");
    SPED_TRY(check_layout(d_X, SPED_BF16, k, ldx, "probe_gather X"));
    SPED_TRY(check_layout(d_Y, SPED_BF16, k, ldy, "probe_gather Y"));
    if (mode < 0 || mode > 2) return fail(SPED_ERR_INVALID_ARG, "probe_gather: mode %d", mode);
    const int C = (k + 7) / 8;
    if (C > 32) return fail(SPED_ERR_UNSUPPORTED, "probe_gather: k = %d > 256", k);
    if (g->n == 0) return SPED_OK;
    const int rows_per_warp = 32 / C;
    const int64_t warps = (g->n + rows_per_warp - 1) / rows_per_warp;
    const int64_t blocks = (warps * 32 + PROBE_THREADS - 1) / PROBE_THREADS;
    cudaStream_t st = as_stream(stream);
    const auto *X = (const __nv_bfloat16 *)d_X;
    auto *Y = (__nv_bfloat16 *)d_Y;
    const uint32_t s32 = (uint32_t)(seed ^ (seed >> 32));
    if (mode == 0)
        k_probe_gather<0><<<(unsigned)blocks, PROBE_THREADS, 0, st>>>(g->n, g->rp, g->ci, X, ldx, Y,
                                                                     ldy, C, rows_per_warp, s32);
    else if (mode == 1)
        k_probe_gather<1><<<(unsigned)blocks, PROBE_THREADS, 0, st>>>(g->n, g->rp, g->ci, X, ldx, Y,
                                                                     ldy, C, rows_per_warp, s32);
    else
        k_probe_gather<2><<<(unsigned)blocks, PROBE_THREADS, 0, st>>>(g->n, g->rp, g->ci, X, ldx, Y,
                                                                     ldy, C, rows_per_warp, s32);
    SPED_CHECK_LAUNCH("k_probe_gather");
    return SPED_OK;
}

}  // extern "C"
