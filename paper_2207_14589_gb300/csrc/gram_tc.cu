// Tall-skinny Gram G = X^T X, X = [A B] (n x K2), on the 5th-generation tensor cores.
//
// Each F32 value x is split into BF16 pieces x = h + m + l: h is the top 16 bits of x (a BF16
// value, truncated), m the top 16 bits of x - h, l = x - h - m (exactly a BF16 value: after two
// truncations at most 8 significant bits are left); every remainder is exact in F32, so the
// split is exact, and products of BF16 pieces are exact in F32, so the nine piece products
// recover x_i x_j to F32 accuracy. The pieces are stacked as S*K2 <= 128 operand rows (S = 3
// for F32 inputs, 1 for BF16) and one tcgen05.mma (M = N = 128, K = 16 graph rows, kind::f16
// with BF16 operands, F32 accumulator in tensor memory) consumes 16 rows; the same
// shared-memory tile is both operands because G is a Gram matrix.
//
// One persistent CTA per SM takes tiles of 128 graph rows round-robin through a warp-
// specialised pipeline (see k_gram_ws): a producer warp keeps a ring of raw tiles filled with
// bulk copies (cp.async.bulk, completion counted in bytes on each stage's mbarrier), splitter
// warps turn a raw tile into the K-major core-matrix layout of an operand stage, one thread
// issues the tile's 8 MMAs into one of two accumulators in tensor memory and commits them to
// the stage's mbarrier, and every 4 tiles (512 rows, bounding each F32 accumulation run) folder
// warps add the full accumulator to double-float (TwoSum) running sums kept in the other half
// of tensor memory while the MMAs fill the second accumulator. At the end the running sums go
// to shared memory, the nine piece blocks are combined per (i, j) and the CTA writes an F64
// partial; a second kernel sums the partials in a fixed order (deterministic).
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

constexpr int TC_RAW_CHUNKS = 2048;   // 16-byte chunks of one tile of A and B at most
constexpr int TC_TILE = 128;          // graph rows per tile
constexpr int TC_SLICES = TC_TILE / 16;
constexpr int TC_SLICE_BYTES = 128 * 16 * 2;
constexpr int TC_STAGE_BYTES = TC_SLICES * TC_SLICE_BYTES;  // 32 KB
constexpr int TC_FLUSH = 4;           // tiles per F32 accumulation run
constexpr int TC_COLS = 128;          // accumulator columns (N)
constexpr int TC_TMEM_COLS = 512;     // allocation (power of two >= 384)
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;

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

// ---------------------------------------------------------------------------------------
// Warp-specialised version: every stage of the pipeline has its own warps and mbarriers, so no
// warp waits for work it does not consume.
//   warp 0       producer: lane 0 keeps the raw ring full with bulk copies (nraw stages);
//   warps 1..NS  splitters: raw stage -> BF16 pieces in an operand stage;
//   warp NS+1    MMA: lane 0 issues the tile's 8 MMAs into one of two accumulators in tensor
//                memory and commits to the operand stage's "empty" barrier (and, every
//                TC_FLUSH tiles, to the accumulator's "full" barrier);
//   warps NS+2.. folders (one per tensor-memory lane quarter): add a full accumulator to the
//                double-float running sums while the MMA warp fills the other one.
// Tensor memory: accumulators in columns [0, 128) and [128, 256), running sums hi / lo in
// [256, 384) and [384, 512). Every wait is bounded and also gives up once another warp has
// given up; the CTA then waits (bounded) for its copies and MMAs in flight, frees its tensor
// memory, writes NaN partials and sets the device status word.
// ---------------------------------------------------------------------------------------
constexpr int WS_NS = 24;                         // splitter warps
constexpr int WS_MMA_WARP = 1 + WS_NS;
constexpr int WS_FOLD0 = WS_MMA_WARP + 1;         // first of the four folder warps
constexpr int WS_WARPS = WS_FOLD0 + 4;
constexpr int WS_THREADS = WS_WARPS * 32;
constexpr int WS_MAXRAW = 8;
constexpr int WS_NOP = 4;                         // operand stages
constexpr int WS_RAW_BYTES = 88 * 1024;
constexpr uint32_t WS_HI = 256, WS_LO = 384;

struct WsSmem {
    // operand stages and raw ring are contiguous: at the end they hold the running sums
    alignas(1024) unsigned char stage[WS_NOP][TC_STAGE_BYTES];
    alignas(1024) unsigned char raw[WS_RAW_BYTES];
    alignas(8) uint64_t raw_full[WS_MAXRAW];
    alignas(8) uint64_t raw_empty[WS_MAXRAW];
    alignas(8) uint64_t op_full[WS_NOP];
    alignas(8) uint64_t op_empty[WS_NOP];
    alignas(8) uint64_t acc_full[2];
    alignas(8) uint64_t acc_empty[2];
    uint32_t tmem_base;
    int abort;
    int timed_out;
};
static_assert(sizeof(WsSmem::stage) + sizeof(WsSmem::raw) >= 2 * 128 * 128 * sizeof(float),
              "final staging of the running sums");

// one potentially blocking probe of the phase: the hardware suspends the thread until the phase
// completes or a time limit of its own passes (no issue slots spent spinning)
__device__ __forceinline__ bool mbar_try(uint32_t mbar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(mbar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait (at most `limit` probes and about two seconds) that also gives up when another
// warp of the CTA has given up
__device__ __forceinline__ bool ws_wait(uint32_t mbar, uint32_t parity, uint32_t limit,
                                        volatile int *abort) {
    if (limit > 0 && mbar_try(mbar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 1; it < limit; ++it) {
        if (*abort) return false;
        if (mbar_try(mbar, parity)) return true;
        if (global_ns() - t0 > 2000000000ull) break;
    }
    *abort = 1;
    return false;
}

template <typename Ta, typename Tb, int S>
__global__ void __launch_bounds__(WS_THREADS, 1)
k_gram_ws(int64_t n, const Ta *__restrict__ A, int lda, int ka, const Tb *__restrict__ B, int ldb,
          int kb, double *__restrict__ partial, uint32_t wait_limit, int skip_fills) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    WsSmem &sm = *reinterpret_cast<WsSmem *>(
        smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023));
    const int t = threadIdx.x;
    const int warp = t >> 5, lane = t & 31;
    const int K2 = ka + kb;
    const int64_t ntiles = (n + TC_TILE - 1) / TC_TILE;
    const int64_t my_tiles = blockIdx.x < ntiles ? (ntiles - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t n_groups = (my_tiles + TC_FLUSH - 1) / TC_FLUSH;
    const uint32_t tile_max = (uint32_t)TC_TILE * ((uint32_t)lda * (uint32_t)sizeof(Ta) +
                                                   (kb ? (uint32_t)ldb * (uint32_t)sizeof(Tb) : 0u));
    const uint32_t stage_bytes = (tile_max + 127u) & ~127u;
    int nraw = (int)(WS_RAW_BYTES / stage_bytes);
    if (nraw > WS_MAXRAW) nraw = WS_MAXRAW;
    volatile int *abort = &sm.abort;
    // ---- set-up: zero the operand stages (rows past S K2 stay zero), barriers, tensor memory
    for (int e = t; e < WS_NOP * TC_STAGE_BYTES / 16; e += WS_THREADS)
        reinterpret_cast<uint4 *>(&sm.stage[0][0])[e] = make_uint4(0, 0, 0, 0);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // zeros seen by the MMAs
    if (t == 0) {
        for (int i = 0; i < WS_MAXRAW; ++i) {
            mbar_init(smem_u32(&sm.raw_full[i]), 1);
            mbar_init(smem_u32(&sm.raw_empty[i]), WS_NS);
        }
        for (int i = 0; i < WS_NOP; ++i) {
            mbar_init(smem_u32(&sm.op_full[i]), WS_NS);
            mbar_init(smem_u32(&sm.op_empty[i]), 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(smem_u32(&sm.acc_full[i]), 1);
            mbar_init(smem_u32(&sm.acc_empty[i]), 4);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sm.abort = 0;
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
    pdl_wait();  // the set-up above overlaps the previous kernel; its outputs are read below
    const uint32_t tmem = sm.tmem_base;
    int64_t issued = 0;      // producer (warp 0, lane 0): fills issued
    int64_t mma_issued = 0;  // MMA warp, lane 0: tiles whose MMAs were issued

    if (warp == 0) {
        // ---- producer
        if (lane == 0 && !skip_fills) {
            // stage rs of fill f = f % nraw and its use count u = f / nraw, kept incrementally
            int rs = 0;
            uint32_t u = 0;
            for (int64_t f = 0; f < my_tiles; ++f) {
                if (u > 0 && !ws_wait(smem_u32(&sm.raw_empty[rs]), (u - 1) & 1u, wait_limit, abort))
                    break;
                const int64_t r0 = (blockIdx.x + f * gridDim.x) * (int64_t)TC_TILE;
                const int rows = (int)(n - r0 < TC_TILE ? n - r0 : TC_TILE);
                const uint32_t ba = (uint32_t)((size_t)rows * lda * sizeof(Ta));
                const uint32_t bb = kb ? (uint32_t)((size_t)rows * ldb * sizeof(Tb)) : 0u;
                const uint32_t bar = smem_u32(&sm.raw_full[rs]);
                const uint32_t dst = smem_u32(sm.raw) + (uint32_t)rs * stage_bytes;
                mbar_arrive_expect_tx(bar, ba + bb);
                bulk_g2s(dst, A + r0 * lda, ba, bar);
                if (bb) bulk_g2s(dst + ba, B + r0 * ldb, bb, bar);
                issued = f + 1;
                if (++rs == nraw) {
                    rs = 0;
                    ++u;
                }
            }
        }
    } else if (warp <= WS_NS) {
        // ---- splitters: unit (c, g) is column c of [A B] over graph rows 8g .. 8g+7 of the
        // tile; each of its S BF16 pieces is one 16-byte row of a core matrix (operand row
        // m = s K2 + c, K half g & 1 of slice g / 2)
        const int st = t - 32;
        constexpr int NT = WS_NS * 32;
        const int c_first = st % K2, g_first = st / K2;
        const int c_step = NT % K2, g_step = NT / K2;
        int rs = 0;       // raw stage of tile it (it % nraw) and its use count (it / nraw)
        uint32_t ru = 0;
        for (int64_t it = 0; it < my_tiles; ++it) {
            const int o = (int)(it % WS_NOP);
            bool ok = ws_wait(smem_u32(&sm.raw_full[rs]), ru & 1u, wait_limit, abort);
            if (ok && it >= WS_NOP)
                ok = ws_wait(smem_u32(&sm.op_empty[o]), (uint32_t)(((it / WS_NOP) - 1) & 1),
                             wait_limit, abort);
            if (!__all_sync(0xffffffffu, ok)) break;
            const int64_t r0 = (blockIdx.x + it * gridDim.x) * (int64_t)TC_TILE;
            const int rows = (int)(n - r0 < TC_TILE ? n - r0 : TC_TILE);
            const unsigned char *raw = sm.raw + (size_t)rs * stage_bytes;
            const Ta *ra = reinterpret_cast<const Ta *>(raw);
            const Tb *rb = reinterpret_cast<const Tb *>(raw + (size_t)rows * lda * sizeof(Ta));
            int c = c_first, g = g_first;
            for (; g < TC_TILE / 8; c += c_step, g += g_step) {
                if (c >= K2) {
                    c -= K2;
                    ++g;
                    if (g >= TC_TILE / 8) break;
                }
                float x[8];
                const int r0 = g * 8;
                if (c < ka) {
#pragma unroll
                    for (int rr = 0; rr < 8; ++rr)
                        x[rr] = r0 + rr < rows ? cvt<float>(ra[(r0 + rr) * lda + c]) : 0.f;
                } else {
#pragma unroll
                    for (int rr = 0; rr < 8; ++rr)
                        x[rr] = r0 + rr < rows ? cvt<float>(rb[(r0 + rr) * ldb + (c - ka)]) : 0.f;
                }
                unsigned char *slice = sm.stage[o] + (g >> 1) * TC_SLICE_BYTES + (g & 1) * 128;
#pragma unroll
                for (int s = 0; s < S; ++s) {
                    // piece s: the top 16 bits (a BF16 value, truncated) of what is left; the
                    // remainder x - piece is exact in F32, and after three pieces nothing is
                    // left, so x = h + m + l exactly
                    uint32_t w[4];
#pragma unroll
                    for (int p2 = 0; p2 < 4; ++p2) {
                        const uint32_t a = __float_as_uint(x[2 * p2]) & 0xffff0000u;
                        const uint32_t b = __float_as_uint(x[2 * p2 + 1]) & 0xffff0000u;
                        w[p2] = __byte_perm(a, b, 0x7632);
                        if (s + 1 < S) {
                            x[2 * p2] -= __uint_as_float(a);
                            x[2 * p2 + 1] -= __uint_as_float(b);
                        }
                    }
                    const int m = s * K2 + c;
                    *reinterpret_cast<uint4 *>(slice + (m >> 3) * 256 + (m & 7) * 16) =
                        make_uint4(w[0], w[1], w[2], w[3]);
                }
            }
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            __syncwarp();
            if (lane == 0) {
                mbar_arrive(smem_u32(&sm.raw_empty[rs]));  // raw stage may be refilled
                mbar_arrive(smem_u32(&sm.op_full[o]));     // operand stage ready for the MMAs
            }
            if (++rs == nraw) {
                rs = 0;
                ++ru;
            }
        }
    } else if (warp == WS_MMA_WARP) {
        // ---- MMA issue
        if (lane == 0) {
            const uint32_t idesc = tc_idesc();
            int b = 0, in_group = 0;
            int64_t g = 0;
            for (int64_t it = 0; it < my_tiles; ++it) {
                const int o = (int)(it % WS_NOP);
                if (in_group == 0 && g >= 2 &&
                    !ws_wait(smem_u32(&sm.acc_empty[b]), (uint32_t)(((g >> 1) - 1) & 1),
                             wait_limit, abort))
                    break;
                if (!ws_wait(smem_u32(&sm.op_full[o]), (uint32_t)((it / WS_NOP) & 1), wait_limit,
                             abort))
                    break;
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t sbase = smem_u32(sm.stage[o]);
#pragma unroll
                for (int s = 0; s < TC_SLICES; ++s) {
                    const uint64_t d = tc_desc(sbase + s * TC_SLICE_BYTES);
                    tc_mma(tmem + (uint32_t)(b * TC_COLS), d, d, idesc,
                           (in_group == 0 && s == 0) ? 0u : 1u);
                }
                tc_commit(smem_u32(&sm.op_empty[o]));
                mma_issued = it + 1;
                if (++in_group == TC_FLUSH || it + 1 == my_tiles) {
                    tc_commit(smem_u32(&sm.acc_full[b]));
                    b ^= 1;
                    in_group = 0;
                    ++g;
                }
            }
        }
    } else {
        // ---- folders: warp w owns tensor-memory lanes 32 (w % 4) .. +32, all 128 columns
        const uint32_t lane_q = (uint32_t)((warp & 3) * 32) << 16;
        {
            uint32_t z[16];
#pragma unroll
            for (int q = 0; q < 16; ++q) z[q] = 0u;
#pragma unroll 1
            for (int h = 0; h < TC_COLS; h += 16) {
                tmem_st16(tmem + lane_q + WS_HI + (uint32_t)h, z);
                tmem_st16(tmem + lane_q + WS_LO + (uint32_t)h, z);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
        }
        for (int64_t g = 0; g < n_groups; ++g) {
            const int b = (int)(g & 1);
            const bool ok = ws_wait(smem_u32(&sm.acc_full[b]), (uint32_t)((g >> 1) & 1),
                                    wait_limit, abort);
            if (!__all_sync(0xffffffffu, ok)) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
#pragma unroll 1
            for (int h = 0; h < TC_COLS; h += 16) {
                uint32_t v[16], hi[16], lo[16];
                tmem_ld16(tmem + lane_q + (uint32_t)(b * TC_COLS + h), v);
                tmem_ld16(tmem + lane_q + WS_HI + (uint32_t)h, hi);
                tmem_ld16(tmem + lane_q + WS_LO + (uint32_t)h, lo);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int q = 0; q < 16; ++q) {
                    float sh = __uint_as_float(hi[q]), el = __uint_as_float(lo[q]);
                    two_sum(sh, el, __uint_as_float(v[q]));
                    hi[q] = __float_as_uint(sh);
                    lo[q] = __float_as_uint(el);
                }
                tmem_st16(tmem + lane_q + WS_HI + (uint32_t)h, hi);
                tmem_st16(tmem + lane_q + WS_LO + (uint32_t)h, lo);
            }
            asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_u32(&sm.acc_empty[b]));  // accumulator b free
        }
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    // ---- after a wait gave up: wait (bounded) for the copies and MMAs still in flight
    if (sm.abort) {
        if (warp == 0 && lane == 0) {
            int bad = 1;
            for (int64_t f = issued - nraw > 0 ? issued - nraw : 0; f < issued; ++f)
                if (!mbar_wait(smem_u32(&sm.raw_full[f % nraw]), (uint32_t)((f / nraw) & 1),
                               wait_limit))
                    bad = 2;
            if (bad == 2) sm.timed_out = 2;
        }
        if (warp == WS_MMA_WARP && lane == 0 && mma_issued > 0) {
            const int64_t it = mma_issued - 1;
            if (!mbar_wait(smem_u32(&sm.op_empty[it % WS_NOP]), (uint32_t)((it / WS_NOP) & 1),
                           wait_limit))
                sm.timed_out = 2;
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const int bad = sm.abort ? (sm.timed_out == 2 ? 2 : 1) : 0;
    if (bad && t == 0) atomicOr(&g_device_status, 1u);
    // the running sums to shared memory ([n][m] layout), unless copies may still be landing
    float *fin_hi = reinterpret_cast<float *>(&sm.stage[0][0]);
    float *fin_lo = fin_hi + 128 * 128;
    if (bad != 2 && warp >= WS_FOLD0) {
        const uint32_t lane_q = (uint32_t)((warp & 3) * 32) << 16;
        const int m = (warp & 3) * 32 + lane;
#pragma unroll 1
        for (int h = 0; h < TC_COLS; h += 16) {
            uint32_t hi[16], lo[16];
            tmem_ld16(tmem + lane_q + WS_HI + (uint32_t)h, hi);
            tmem_ld16(tmem + lane_q + WS_LO + (uint32_t)h, lo);
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
            for (int q = 0; q < 16; ++q) {
                fin_hi[(h + q) * 128 + m] = __uint_as_float(hi[q]);
                fin_lo[(h + q) * 128 + m] = __uint_as_float(lo[q]);
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
    for (int e = t; e < K2 * K2; e += WS_THREADS) {
        const int j = e / K2, i = e % K2;  // consecutive threads read consecutive m = a K2 + i
        if (i > j) continue;
        double v = NAN;
        if (!bad) {
            float s = 0.f, err = 0.f;
#pragma unroll
            for (int a = 0; a < S; ++a)
#pragma unroll
                for (int b2 = 0; b2 < S; ++b2) {
                    const int idx = (b2 * K2 + j) * 128 + (a * K2 + i);
                    two_sum(s, err, fin_hi[idx]);
                    err += fin_lo[idx];
                }
            v = (double)s + (double)err;
        }
        out[i * K2 + j] = v;
        out[j * K2 + i] = v;
    }
    pdl_trigger();
}

// G[e] = sum over CTAs of partial[c][e]: a block per 32 outputs, 32 thread groups over the
// partials, then a fixed-order sum of the 32 group totals (deterministic)
constexpr int RED_OUT = 32, RED_GROUPS = 32;
__global__ void __launch_bounds__(RED_OUT *RED_GROUPS)
k_gram_tc_reduce(const double *__restrict__ partial, int nparts, int K2, double *__restrict__ G) {
    __shared__ double sm[RED_GROUPS][RED_OUT];
    pdl_wait();
    const int o = threadIdx.x % RED_OUT, grp = threadIdx.x / RED_OUT;
    const int e = blockIdx.x * RED_OUT + o;
    const int tot = K2 * K2;
    double s = 0.0;
    if (e < tot) {
        // a group's partials (grp, grp + 32, ...) are loaded together, then added in order
        constexpr int B = 8;
        for (int c0 = grp; c0 < nparts; c0 += B * RED_GROUPS) {
            double v[B];
#pragma unroll
            for (int q = 0; q < B; ++q) {
                const int c = c0 + q * RED_GROUPS;
                v[q] = c < nparts ? partial[(int64_t)c * tot + e] : 0.0;
            }
#pragma unroll
            for (int q = 0; q < B; ++q) s += v[q];
        }
    }
    sm[grp][o] = s;
    __syncthreads();
    if (grp == 0 && e < tot) {
        double r = 0.0;
#pragma unroll
        for (int q = 0; q < RED_GROUPS; ++q) r += sm[q][o];
        G[e] = r;
    }
    pdl_trigger();
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
    const uint32_t lim = g_tc_wait_limit.load();
    const size_t smem = sizeof(WsSmem) + 1024;
    auto kern = k_gram_ws<Ta, Tb, S>;
    SPED_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    SPED_CUDA(launch_pdl(kern, dim3(ctas), dim3(WS_THREADS), smem, st, n, (const Ta *)A, lda, ka,
                         (const Tb *)B, ldb, kb, partial, lim ? lim : TC_WAIT_LIMIT,
                         g_tc_skip_fills.load()));
    SPED_CHECK_LAUNCH("k_gram_ws");
    const int K2 = ka + kb;
    SPED_CUDA(launch_pdl(k_gram_tc_reduce, dim3((K2 * K2 + RED_OUT - 1) / RED_OUT),
                         dim3(RED_OUT * RED_GROUPS), 0, st, (const double *)partial, ctas, K2, G));
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
