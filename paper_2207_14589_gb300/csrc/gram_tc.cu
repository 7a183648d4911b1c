// Tall-skinny Gram G = X^T X, X = [A B] (n x K2), on the 5th-generation tensor cores.
//
// Each F32 value x is split into BF16 pieces x = h + m + l (h = bf16(x), m = bf16(x - h),
// l = bf16(x - h - m)); products of BF16 pieces are exact in F32, so the nine piece products
// recover x_i x_j to F32 accuracy. The pieces are stacked as S*K2 <= 128 operand rows (S = 3
// for F32 inputs, 1 for BF16) and one tcgen05.mma (M = N = 128, K = 16 graph rows, kind::f16
// with BF16 operands, F32 accumulator in tensor memory) consumes 16 rows; the same
// shared-memory tile is both operands because G is a Gram matrix.
//
// Pipeline per CTA (one per SM, tiles of 128 graph rows taken round-robin):
//  * thread 0 keeps NRAW - 1 tiles of raw rows in flight: one bulk copy (cp.async.bulk) of the
//    tile's contiguous rows of A and one of B into a raw stage, completion counted in bytes on
//    the stage's mbarrier; a stage is refilled once every warp has arrived on its "empty"
//    barrier;
//  * all warps split the raw stage into the K-major core-matrix layout of an operand stage
//    (two operand stages, one per MMA batch in flight);
//  * thread 0 issues the tile's 8 MMAs and a tcgen05.commit to the operand stage's mbarrier;
//  * every 4 tiles the accumulator is read back and added to double-float (TwoSum) running
//    sums that live in spare tensor-memory columns (the accumulator uses 128 of 512), bounding
//    each F32 accumulation to 512 rows.
// At the end the running sums go to shared memory, the nine piece blocks are combined per
// (i, j) and the CTA writes an F64 partial; a second kernel sums the partials in a fixed order.
//
// Shared-memory operand layout (no swizzle, K-major): per 16-row slice a 128 x 16 BF16 block
// made of 8 x 8 core matrices (128 contiguous bytes each); core matrix (g = m/8, h = k/8) at
// byte (2g + h) * 128, so the K-adjacent core matrix is 128 bytes away (leading byte offset)
// and the next 8-row group 256 bytes away (stride byte offset).
//
// Every wait is bounded: if a completion is not observed within the limit the CTA stops issuing
// work, waits (bounded) for the copies and MMAs it issued, releases its tensor memory, writes
// NaN partials and sets bit 0 of the library's device status word, so the caller sees a
// non-finite Gram and SPED_ERR_TIMEOUT from sped_device_status instead of a hang.
#include <atomic>
#include <cmath>

#include "sped_internal.cuh"

namespace sped {

constexpr int TC_THREADS = 640;       // 20 warps: one split unit per thread at k = 20 (K2 = 40)
constexpr int TC_WARPS = TC_THREADS / 32;
constexpr int TC_RAW_CHUNKS = 2048;   // 16-byte chunks of one tile of A and B at most
constexpr int TC_RAW_BYTES = TC_RAW_CHUNKS * 16;
constexpr int TC_NRAW = 3;            // raw stages: two tiles' copies in flight during a split
constexpr int TC_FOLD_WARPS = 16;     // warps that read tensor memory (4 per TMEM lane quarter)
constexpr int TC_TILE = 128;          // graph rows per tile
constexpr int TC_SLICES = TC_TILE / 16;
constexpr int TC_SLICE_BYTES = 128 * 16 * 2;
constexpr int TC_STAGE_BYTES = TC_SLICES * TC_SLICE_BYTES;  // 32 KB
constexpr int TC_FLUSH = 4;           // tiles per F32 accumulation run
constexpr int TC_COLS = 128;          // accumulator columns (N)
constexpr int TC_HI = 128, TC_LO = 256;  // tensor-memory columns of the running sums
constexpr int TC_TMEM_COLS = 512;     // allocation (power of two >= 384)
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;

struct TcSmem {
    // the operand stages and the raw stages are contiguous: at the end they hold the running
    // sums read out of tensor memory (2 x 64 KB)
    alignas(1024) unsigned char stage[2][TC_STAGE_BYTES];
    alignas(128) unsigned char raw[TC_NRAW][TC_RAW_BYTES];
    alignas(8) uint64_t mma_bar[2];
    alignas(8) uint64_t full_bar[TC_NRAW];
    alignas(8) uint64_t empty_bar[TC_NRAW];
    uint32_t tmem_base;
    int timed_out;
    int wait_ok;
};
static_assert(sizeof(TcSmem::stage) + sizeof(TcSmem::raw) >= 2 * 128 * 128 * sizeof(float),
              "final staging of the running sums");

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t tc_desc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);          // start address
    d |= (uint64_t)(128u >> 4) << 16;                  // leading byte offset (K direction)
    d |= (uint64_t)(256u >> 4) << 32;                  // stride byte offset (M/N direction)
    d |= (uint64_t)1 << 46;                            // descriptor version
    return d;                                          // base offset 0, no swizzle
}

// kind::f16 instruction descriptor: F32 accumulator, BF16 A and B, both K-major, N = M = 128
__device__ __forceinline__ uint32_t tc_idesc() {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(TC_COLS >> 3) << 17) |
           ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t da, uint64_t db, uint32_t idesc,
                                       uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
        "l"(da), "l"(db), "r"(idesc), "r"(accumulate));
}

__device__ __forceinline__ void tc_commit(uint32_t mbar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
                 : "memory");
}

__device__ __forceinline__ bool mbar_test(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Device status word of this library on the current device: bit 0 is set when a bounded wait of
// the tensor Gram gave up. sped_device_status reads and clears it.
static __device__ unsigned int g_device_status;

// bounded wait for the given phase parity (at most `limit` polls); false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint32_t limit) {
    for (uint32_t it = 0; it < limit; ++it) {
        if (mbar_test(mbar, parity)) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count));
}

__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(mbar) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t mbar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes)
                 : "memory");
}

// bulk copy global -> shared (16-byte aligned ends, size a multiple of 16), completion counted
// in bytes on mbar
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes,
                                         uint32_t mbar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar)
        : "memory");
}

// 32 lanes x 16 columns of tensor memory, one 32-bit value per (lane, column)
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
          "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
          "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
        ::"r"(taddr), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]),
          "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]),
          "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}

__device__ __forceinline__ void two_sum(float &s, float &e, float x) {
    const float t = s + x;
    const float bp = t - s;
    e += (s - (t - bp)) + (x - bp);
    s = t;
}

template <typename Ta, typename Tb, int S>
__global__ void __launch_bounds__(TC_THREADS, 1)
k_gram_tc(int64_t n, const Ta *__restrict__ A, int lda, int ka, const Tb *__restrict__ B, int ldb,
          int kb, double *__restrict__ partial, uint32_t wait_limit, int skip_fills) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem &sm = *reinterpret_cast<TcSmem *>(
        smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023));
    const int t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31;
    const int K2 = ka + kb;
    const int c_first = t % K2, g_first = t / K2;                 // this thread's first split unit
    const int c_step = TC_THREADS % K2, g_step = TC_THREADS / K2;  // and the stride between units
    const int64_t ntiles = (n + TC_TILE - 1) / TC_TILE;
    const int64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    // ---- set-up: zero the operand stages (rows past S K2 stay zero), barriers, tensor memory
    for (int e = t; e < 2 * TC_STAGE_BYTES / 16; e += TC_THREADS)
        reinterpret_cast<uint4 *>(&sm.stage[0][0])[e] = make_uint4(0, 0, 0, 0);
    if (t == 0) {
        for (int i = 0; i < 2; ++i) mbar_init(smem_u32(&sm.mma_bar[i]), 1);
        for (int i = 0; i < TC_NRAW; ++i) {
            mbar_init(smem_u32(&sm.full_bar[i]), 1);
            mbar_init(smem_u32(&sm.empty_bar[i]), TC_WARPS);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sm.timed_out = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&sm.tmem_base)),
                     "r"(TC_TMEM_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = sm.tmem_base;
    // warp w < 16 owns TMEM lane quarter w % 4 and accumulator columns [32 (w / 4), +32)
    const bool folder = warp < TC_FOLD_WARPS;
    const uint32_t lane_q = (uint32_t)((warp & 3) * 32) << 16;
    const int col0 = (warp >> 2) * 32;
    if (folder) {  // running sums start at zero
        uint32_t z[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) z[q] = 0u;
#pragma unroll
        for (int h = 0; h < 32; h += 16) {
            tmem_st16(tmem + lane_q + (uint32_t)(TC_HI + col0 + h), z);
            tmem_st16(tmem + lane_q + (uint32_t)(TC_LO + col0 + h), z);
        }
        asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
    }
    const uint32_t idesc = tc_idesc();
    // raw tile loads (thread 0): fill number f of raw stage f % NRAW holds this CTA's tile f
    int64_t issued = 0;
    auto issue = [&]() {  // next fill, once its stage has been released by every warp
        const int64_t f = issued;
        if (f >= my_tiles) return true;
        if (skip_fills) return true;  // test of the timeout path: nothing is ever in flight
        const int rs = (int)(f % TC_NRAW);
        if (f >= TC_NRAW &&
            !mbar_wait(smem_u32(&sm.empty_bar[rs]), (uint32_t)(((f / TC_NRAW) - 1) & 1), wait_limit))
            return false;
        const int64_t r0 = (blockIdx.x + f * gridDim.x) * (int64_t)TC_TILE;
        const int rows = (int)(n - r0 < TC_TILE ? n - r0 : TC_TILE);
        const uint32_t ba = (uint32_t)((size_t)rows * lda * sizeof(Ta));
        const uint32_t bb = (uint32_t)((size_t)rows * ldb * sizeof(Tb));
        const uint32_t bar = smem_u32(&sm.full_bar[rs]);
        mbar_arrive_expect_tx(bar, ba + bb);
        bulk_g2s(smem_u32(sm.raw[rs]), A + r0 * lda, ba, bar);
        if (bb) bulk_g2s(smem_u32(sm.raw[rs]) + ba, B + r0 * ldb, bb, bar);
        ++issued;
        return true;
    };
    if (t == 0) {
        for (int f = 0; f < TC_NRAW - 1; ++f)
            if (!issue()) sm.timed_out = 1;
    }
    uint32_t mma_par[2] = {0, 0};
    bool pending[2] = {false, false};
    bool fresh = true;  // next MMA overwrites the accumulator
    bool ok = true;
    for (int64_t it = 0; it < my_tiles && ok; ++it) {
        const int64_t tile = blockIdx.x + it * gridDim.x;
        const int st = (int)(it & 1);
        const int rs = (int)(it % TC_NRAW);
        // ---- thread 0: keep NRAW - 1 fills ahead, then wait for this tile's rows and for the
        // MMAs that last read this operand stage; every thread gets the same answer
        if (t == 0) {
            bool good = sm.timed_out == 0;
            if (good && issued < my_tiles && !issue()) good = false;
            if (good && !mbar_wait(smem_u32(&sm.full_bar[rs]), (uint32_t)((it / TC_NRAW) & 1), wait_limit))
                good = false;
            if (good && pending[st] && !mbar_wait(smem_u32(&sm.mma_bar[st]), mma_par[st], wait_limit))
                good = false;
            if (!good) sm.timed_out = 1;
            sm.wait_ok = good ? 1 : 0;
        }
        __syncthreads();
        ok = sm.wait_ok != 0;
        if (!ok) break;
        if (pending[st]) {
            mma_par[st] ^= 1;
            pending[st] = false;
        }
        // ---- split: unit (c, g) is column c of [A B] over graph rows 8g .. 8g+7 (zero past the
        // end); each of its S BF16 pieces is 8 consecutive K elements, i.e. one 16-byte row of
        // a core matrix (operand row m = s K2 + c, K half g & 1 of slice g / 2)
        const int64_t r0 = tile * TC_TILE;
        const int rows = (int)(n - r0 < TC_TILE ? n - r0 : TC_TILE);
        {
            const Ta *ra = reinterpret_cast<const Ta *>(sm.raw[rs]);
            const Tb *rb = reinterpret_cast<const Tb *>(sm.raw[rs] + (size_t)rows * lda * sizeof(Ta));
            // unit uu = g K2 + c, advanced by TC_THREADS without a division per unit
            int c = c_first, g = g_first;
            for (; g < TC_TILE / 8; c += c_step, g += g_step) {
                if (c >= K2) {
                    c -= K2;
                    ++g;
                    if (g >= TC_TILE / 8) break;
                }
                float x[8];
#pragma unroll
                for (int rr = 0; rr < 8; ++rr) {
                    const int row = g * 8 + rr;
                    x[rr] = row >= rows ? 0.f
                            : c < ka    ? cvt<float>(ra[row * lda + c])
                                        : cvt<float>(rb[row * ldb + (c - ka)]);
                }
                unsigned char *slice = sm.stage[st] + (g >> 1) * TC_SLICE_BYTES + (g & 1) * 128;
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    uint32_t w[4];
#pragma unroll
                    for (int p2 = 0; p2 < 4; ++p2) {
                        const __nv_bfloat162 h2 = __floats2bfloat162_rn(x[2 * p2], x[2 * p2 + 1]);
                        w[p2] = *reinterpret_cast<const uint32_t *>(&h2);
                        if (s + 1 < S) {  // the rounding residual is exact in F32
                            x[2 * p2] -= __low2float(h2);
                            x[2 * p2 + 1] -= __high2float(h2);
                        }
                    }
                    const int m = s * K2 + c;
                    *reinterpret_cast<uint4 *>(slice + (m >> 3) * 256 + (m & 7) * 16) =
                        make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(smem_u32(&sm.empty_bar[rs]));  // raw stage may be refilled
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        __syncthreads();
        if (t == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sbase = smem_u32(sm.stage[st]);
#pragma unroll
            for (int s = 0; s < TC_SLICES; ++s) {
                const uint64_t d = tc_desc(sbase + s * TC_SLICE_BYTES);
                tc_mma(tmem, d, d, idesc, (fresh && s == 0) ? 0u : 1u);
            }
            tc_commit(smem_u32(&sm.mma_bar[st]));
        }
        fresh = false;
        pending[st] = true;
        if ((it + 1) % TC_FLUSH == 0 || it + 1 == my_tiles) {
            // ---- fold the accumulator into the double-float running sums in tensor memory
            if (t == 0) {
                const bool good = mbar_wait(smem_u32(&sm.mma_bar[st]), mma_par[st], wait_limit);
                if (!good) sm.timed_out = 1;
                sm.wait_ok = good ? 1 : 0;
            }
            __syncthreads();
            ok = sm.wait_ok != 0;
            if (!ok) break;
            mma_par[st] ^= 1;
            pending[st] = false;
            asm volatile("tcgen05.fence::after_thread_sync;");
            if (folder) {
#pragma unroll 1
                for (int h = 0; h < 32; h += 16) {
                    uint32_t v[16], hi[16], lo[16];
                    tmem_ld16(tmem + lane_q + (uint32_t)(col0 + h), v);
                    tmem_ld16(tmem + lane_q + (uint32_t)(TC_HI + col0 + h), hi);
                    tmem_ld16(tmem + lane_q + (uint32_t)(TC_LO + col0 + h), lo);
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        float sh = __uint_as_float(hi[q]), el = __uint_as_float(lo[q]);
                        two_sum(sh, el, __uint_as_float(v[q]));
                        hi[q] = __float_as_uint(sh);
                        lo[q] = __float_as_uint(el);
                    }
                    tmem_st16(tmem + lane_q + (uint32_t)(TC_HI + col0 + h), hi);
                    tmem_st16(tmem + lane_q + (uint32_t)(TC_LO + col0 + h), lo);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            fresh = true;
        }
    }
    // ---- on a timeout, wait (bounded) for whatever is still in flight: MMAs, raw copies
    if (t == 0) {
        if (!ok) sm.timed_out = 1;
        for (int s = 0; s < 2; ++s)
            if (pending[s] && !mbar_wait(smem_u32(&sm.mma_bar[s]), mma_par[s], wait_limit)) sm.timed_out = 2;
        // fills issued but not consumed by the loop (only after a timeout)
        if (!ok)
            for (int64_t f = 0; f < issued; ++f)
                if (!mbar_wait(smem_u32(&sm.full_bar[f % TC_NRAW]), (uint32_t)((f / TC_NRAW) & 1),
                               wait_limit))
                    sm.timed_out = 2;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    // the running sums to shared memory ([n][m] layout), unless copies may still be landing
    float *fin_hi = reinterpret_cast<float *>(&sm.stage[0][0]);
    float *fin_lo = fin_hi + 128 * 128;
    const int bad = sm.timed_out;
    if (bad && t == 0) atomicOr(&g_device_status, 1u);
    if (bad != 2 && folder) {
#pragma unroll 1
        for (int h = 0; h < 32; h += 16) {
            uint32_t hi[16], lo[16];
            tmem_ld16(tmem + lane_q + (uint32_t)(TC_HI + col0 + h), hi);
            tmem_ld16(tmem + lane_q + (uint32_t)(TC_LO + col0 + h), lo);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            const int m = (warp & 3) * 32 + lane;
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                fin_hi[(col0 + h + q) * 128 + m] = __uint_as_float(hi[q]);
                fin_lo[(col0 + h + q) * 128 + m] = __uint_as_float(lo[q]);
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TC_TMEM_COLS));
    // ---- combine the S x S piece blocks: G[i][j] = sum_{a,b} D[a K2 + i][b K2 + j], i <= j
    double *out = partial + (int64_t)blockIdx.x * K2 * K2;
    for (int e = t; e < K2 * K2; e += TC_THREADS) {
        const int i = e / K2, j = e % K2;
        if (i > j) continue;
        double v = NAN;
        if (!bad) {
            float s = 0.f, err = 0.f;
#pragma unroll
            for (int a = 0; a < S; ++a)
#pragma unroll
                for (int b = 0; b < S; ++b) {
                    const int idx = (b * K2 + j) * 128 + (a * K2 + i);
                    two_sum(s, err, fin_hi[idx]);
                    err += fin_lo[idx];
                }
            v = (double)s + (double)err;
        }
        out[i * K2 + j] = v;
        out[j * K2 + i] = v;
    }
}

// G[e] = sum over CTAs of partial[c][e]: a block per 32 outputs, 8 thread groups over the
// partials, then a fixed-order sum of the 8 group totals (deterministic)
constexpr int RED_OUT = 32, RED_GROUPS = 8;
__global__ void __launch_bounds__(RED_OUT *RED_GROUPS)
k_gram_tc_reduce(const double *__restrict__ partial, int nparts, int K2, double *__restrict__ G) {
    __shared__ double sm[RED_GROUPS][RED_OUT];
    const int o = threadIdx.x % RED_OUT, grp = threadIdx.x / RED_OUT;
    const int e = blockIdx.x * RED_OUT + o;
    const int tot = K2 * K2;
    double s = 0.0;
    if (e < tot)
        for (int c = grp; c < nparts; c += RED_GROUPS) s += partial[(int64_t)c * tot + e];
    sm[grp][o] = s;
    __syncthreads();
    if (grp == 0 && e < tot) {
        double r = 0.0;
#pragma unroll
        for (int q = 0; q < RED_GROUPS; ++q) r += sm[q][o];
        G[e] = r;
    }
}

static int tc_ctas(int64_t n) {
    int64_t tiles = (n + TC_TILE - 1) / TC_TILE;
    int64_t c = device_sm_count();
    if (tiles < c) c = tiles;
    return c < 1 ? 1 : (int)c;
}

// pieces per value for the tensor path, 0 when it does not apply
int gram_tc_pieces(sped_dtype at, sped_dtype bt, int ka, int kb, int lda, int ldb) {
    const bool a_ok = at == SPED_F32 || at == SPED_BF16;
    const bool b_ok = kb == 0 || bt == SPED_F32 || bt == SPED_BF16;
    if (!a_ok || !b_ok) return 0;
    // rows are whole 16-byte chunks (the bulk copies move rows * ld * size bytes)
    const size_t ra = (size_t)lda * dtype_size(at), rb = kb ? (size_t)ldb * dtype_size(bt) : 0;
    if (ra % 16 != 0 || rb % 16 != 0) return 0;
    // one tile of A and B fits the raw buffer (TC_RAW_CHUNKS 16-byte chunks)
    if ((size_t)TC_TILE * ((ra + 15) / 16 + (rb + 15) / 16) > (size_t)TC_RAW_CHUNKS) return 0;
    const int S = (at == SPED_F32 || (kb > 0 && bt == SPED_F32)) ? 3 : 1;
    return S * (ka + kb) <= 128 ? S : 0;
}

size_t gram_tc_scratch(int64_t n, int ka, int kb) {
    const int K2 = ka + kb;
    (void)n;
    return sizeof(double) * (size_t)K2 * K2 * 512;
}

// test controls of the bounded waits (sped_test_gram_waits): poll limit (0 = TC_WAIT_LIMIT) and
// whether the kernel skips issuing its bulk copies
static std::atomic<uint32_t> g_tc_wait_limit{0};
static std::atomic<int> g_tc_skip_fills{0};

template <typename Ta, typename Tb, int S>
static sped_status run_tc(int64_t n, const void *A, int lda, int ka, const void *B, int ldb, int kb,
                          double *G, double *partial, int ctas, cudaStream_t st) {
    const size_t smem = sizeof(TcSmem) + 1024;
    auto kern = k_gram_tc<Ta, Tb, S>;
    SPED_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    const uint32_t lim = g_tc_wait_limit.load();
    kern<<<ctas, TC_THREADS, smem, st>>>(n, (const Ta *)A, lda, ka, (const Tb *)B, ldb, kb,
                                         partial, lim ? lim : TC_WAIT_LIMIT,
                                         g_tc_skip_fills.load());
    SPED_CHECK_LAUNCH("k_gram_tc");
    const int K2 = ka + kb;
    k_gram_tc_reduce<<<(K2 * K2 + RED_OUT - 1) / RED_OUT, RED_OUT * RED_GROUPS, 0, st>>>(
        partial, ctas, K2, G);
    SPED_CHECK_LAUNCH("k_gram_tc_reduce");
    return SPED_OK;
}

using bf16 = __nv_bfloat16;

sped_status launch_gram_tc(int64_t n, const void *A, sped_dtype at, int lda, int ka, const void *B,
                           sped_dtype bt, int ldb, int kb, double *G, Scratch &scr,
                           cudaStream_t st) {
    const int S = gram_tc_pieces(at, bt, ka, kb, lda, kb ? ldb : 0);
    if (!S) return fail(SPED_ERR_UNSUPPORTED, "gram (tensor path): not applicable");
    const int ctas = tc_ctas(n);
    double *partial = (double *)scr.take(sizeof(double) * (size_t)(ka + kb) * (ka + kb) * ctas);
    if (!partial) return fail(SPED_ERR_SCRATCH, "gram (tensor path): scratch too small");
    if (kb == 0) {  // no B columns: no B chunks are read
        B = A;
        bt = at;
        ldb = 0;
    }
    if (S == 3) {
        if (at == SPED_F32 && bt == SPED_F32) return run_tc<float, float, 3>(n, A, lda, ka, B, ldb, kb, G, partial, ctas, st);
        if (at == SPED_F32 && bt == SPED_BF16) return run_tc<float, bf16, 3>(n, A, lda, ka, B, ldb, kb, G, partial, ctas, st);
        if (at == SPED_BF16 && bt == SPED_F32) return run_tc<bf16, float, 3>(n, A, lda, ka, B, ldb, kb, G, partial, ctas, st);
    } else {
        return run_tc<bf16, bf16, 1>(n, A, lda, ka, B, ldb, kb, G, partial, ctas, st);
    }
    return fail(SPED_ERR_UNSUPPORTED, "gram (tensor path): dtypes");
}

}  // namespace sped

using namespace sped;

extern "C" {

sped_status sped_device_status(void *stream) {
    SPED_CUDA(cudaStreamSynchronize(as_stream(stream)));
    unsigned int v = 0, zero = 0;
    SPED_CUDA(cudaMemcpyFromSymbol(&v, g_device_status, sizeof(v)));
    if (v) SPED_CUDA(cudaMemcpyToSymbol(g_device_status, &zero, sizeof(zero)));
    if (v & 1u)
        return fail(SPED_ERR_TIMEOUT, "a bounded wait of the tensor-core Gram gave up (its Gram "
                                      "is NaN)");
    return SPED_OK;
}

sped_status sped_test_gram_waits(uint32_t wait_limit, int skip_fills) {
    g_tc_wait_limit.store(wait_limit);
    g_tc_skip_fills.store(skip_fills ? 1 : 0);
    return SPED_OK;
}

}  // extern "C"
