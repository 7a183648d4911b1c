// Gather-rate probe: a measurement library for the benchmark, not part of libsped and not on
// the solver path. The chain step's time is set by how fast the memory system serves its random
// row gathers, not by DRAM bandwidth: every stored entry pulls one k-column row of X from
// wherever it lies. These kernels reproduce the chain step's access stream without its
// arithmetic so that the step can be compared with what the GPU delivers for the same gathers:
//   mode 0: the CSR as given -- row r's lanes read col_idx[p] and gather those rows;
//   mode 1: the same number of gathers per row from uniformly hashed rows (no index stream);
//   mode 2: the same number of gathers per row from the consecutive rows r+1, r+2, ... (mod n):
//           the non-random case: the lane groups of a warp read neighbouring rows, so every
//           warp request is coalesced.
// Same launch shape as the row-group chain step (a group of C lanes per row, one 16-byte chunk
// per lane, four gathers in flight per lane); each row writes the sum of its gathered chunks
// (BF16) so the loads stay live.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "sped_probe.h"

namespace sped_probe {

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

// 16 bytes through the read-only path, as eight BF16 values summed into acc
__device__ __forceinline__ void add_chunk(const __nv_bfloat16 *p, float (&acc)[8]) {
    const uint4 u = __ldg(reinterpret_cast<const uint4 *>(p));
    const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        acc[2 * q] += __uint_as_float(w[q] << 16);
        acc[2 * q + 1] += __uint_as_float(w[q] & 0xffff0000u);
    }
}

template <int MODE>
__global__ void __launch_bounds__(PROBE_THREADS)
    k_probe_gather(int64_t n, const int32_t *__restrict__ rp, const int32_t *__restrict__ ci,
                   const __nv_bfloat16 *__restrict__ X, int ldx, __nv_bfloat16 *__restrict__ Y,
                   int ldy, int C, int rows_per_warp, uint32_t seed) {
    const int lane = threadIdx.x & 31;
    const int64_t warp = ((int64_t)blockIdx.x * PROBE_THREADS + threadIdx.x) >> 5;
    const int rw = lane / C;
    const int c = lane - rw * C;
    if (rw >= rows_per_warp) return;
    const int64_t r = warp * rows_per_warp + rw;
    if (r >= n) return;
    const int p0 = __ldg(rp + r), p1 = __ldg(rp + r + 1);
    float acc[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) acc[i] = 0.f;
    const __nv_bfloat16 *Xc = X + c * 8;
    int p = p0;
    for (; p + PROBE_UNROLL <= p1; p += PROBE_UNROLL) {
        int64_t j[PROBE_UNROLL];
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u)
            j[u] = probe_col<MODE>(ci, n, r, p + u, p0, seed);
#pragma unroll
        for (int u = 0; u < PROBE_UNROLL; ++u) add_chunk(Xc + j[u] * ldx, acc);
    }
    for (; p < p1; ++p) add_chunk(Xc + probe_col<MODE>(ci, n, r, p, p0, seed) * ldx, acc);
    uint32_t o[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const __nv_bfloat162 h = __floats2bfloat162_rn(acc[2 * q], acc[2 * q + 1]);
        o[q] = *reinterpret_cast<const uint32_t *>(&h);
    }
    *reinterpret_cast<uint4 *>(Y + r * ldy + c * 8) = make_uint4(o[0], o[1], o[2], o[3]);
}

}  // namespace sped_probe

using namespace sped_probe;

extern "C" {

int sped_probe_gather(int64_t n, const int32_t *d_row_ptr, const int32_t *d_col_idx, int k,
                      const void *d_X, int ldx, void *d_Y, int ldy, int mode, uint64_t seed,
                      void *stream) {
    if (n < 0 || k < 1 || !d_row_ptr || !d_col_idx || !d_X || !d_Y) return 1;
    if (ldx < k || ldy < k || (ldx * 2) % 16 || (ldy * 2) % 16) return 1;
    if (((uintptr_t)d_X) % 16 || ((uintptr_t)d_Y) % 16) return 1;
    if (mode < 0 || mode > 2) return 1;
    const int C = (k + 7) / 8;
    if (C > 32) return 2;
    if (n == 0) return 0;
    const int rows_per_warp = 32 / C;
    const int64_t warps = (n + rows_per_warp - 1) / rows_per_warp;
    const int64_t blocks = (warps * 32 + PROBE_THREADS - 1) / PROBE_THREADS;
    cudaStream_t st = (cudaStream_t)stream;
    const auto *X = (const __nv_bfloat16 *)d_X;
    auto *Y = (__nv_bfloat16 *)d_Y;
    const uint32_t s32 = (uint32_t)(seed ^ (seed >> 32));
    const dim3 grid((unsigned)blocks);
#define LAUNCH(M)                                                                              \
    k_probe_gather<M><<<grid, PROBE_THREADS, 0, st>>>(n, d_row_ptr, d_col_idx, X, ldx, Y, ldy, C, \
                                                      rows_per_warp, s32)
    if (mode == 0) LAUNCH(0);
    else if (mode == 1) LAUNCH(1);
    else LAUNCH(2);
#undef LAUNCH
    return cudaGetLastError() == cudaSuccess ? 0 : 3;
}

}  // extern "C"
