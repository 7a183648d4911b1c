// Tall-skinny Gram G = X^T X, X = [A B] (n x K2), on the 5th-generation tensor cores.
//
// Each F32 value x is split into BF16 pieces x = h + m + l (h = bf16(x), m = bf16(x - h),
// l = bf16(x - h - m)); products of BF16 pieces are exact in F32, so the nine piece products
// recover x_i x_j to F32 accuracy. The pieces are stacked as S*K2 <= 128 operand rows (S = 3
// for F32 inputs, 1 for BF16) and one tcgen05.mma (M = N = 128, K = 16 graph rows, kind::f16
// with BF16 operands, F32 accumulator in tensor memory) consumes 16 rows; the same
// shared-memory tile is both operands because G is a Gram matrix. 128 graph rows form a tile;
// two tiles are in flight (a tcgen05.commit per tile signals its mbarrier). Every few tiles
// the accumulator is read back with tcgen05.ld and added to double-float (two F32) sums in
// shared memory, bounding the F32 accumulation to a short run of rows. At the end the nine
// piece blocks are combined per (i, j) and the CTA writes an F64 partial; a second kernel
// sums the partials in a fixed order.
//
// Shared-memory operand layout (no swizzle, K-major): per 16-row slice a 128 x 16 BF16 block
// made of 8 x 8 core matrices (128 contiguous bytes each); core matrix (g = m/8, h = k/8) at
// byte (2g + h) * 128, so the K-adjacent core matrix is 128 bytes away (leading byte offset)
// and the next 8-row group 256 bytes away (stride byte offset).
//
// Every wait is bounded: if a tile's completion is not observed within the limit the CTA
// stops issuing work, waits (bounded) for what it issued, releases its tensor memory and
// writes NaN partials, so the caller sees a non-finite Gram instead of a hang.
#include <cmath>

#include "sped_internal.cuh"

namespace sped {

constexpr int TC_THREADS = 640;       // 20 warps: one split unit per thread at k = 20 (K2 = 40)
constexpr int TC_RAW_CHUNKS = 2048;   // 16-byte chunks of one tile of A and B at most
constexpr int TC_MAXQ = (TC_RAW_CHUNKS + TC_THREADS - 1) / TC_THREADS;  // per thread
constexpr int TC_FOLD_WARPS = 16;     // warps that read the accumulator (4 per TMEM lane quarter)
constexpr int TC_TILE = 128;          // graph rows per tile
constexpr int TC_SLICES = TC_TILE / 16;
constexpr int TC_SLICE_BYTES = 128 * 16 * 2;
constexpr int TC_STAGE_BYTES = TC_SLICES * TC_SLICE_BYTES;  // 32 KB
constexpr int TC_FLUSH = 4;           // tiles per F32 accumulation run
constexpr int TC_COLS = 128;          // tensor-memory columns (N)
constexpr uint32_t TC_WAIT_LIMIT = 1u << 22;

struct TcSmem {
    alignas(1024) unsigned char stage[2][TC_STAGE_BYTES];
    alignas(16) unsigned char raw[TC_RAW_CHUNKS * 16];  // one tile of A and B as read
    float acc_hi[128 * 128];  // [n][m]
    float acc_lo[128 * 128];
    alignas(8) uint64_t mbar[2];
    uint32_t tmem_base;
    int timed_out;
    int wait_ok;
};

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

// bounded wait for the given phase parity; false on timeout
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
    for (uint32_t it = 0; it < TC_WAIT_LIMIT; ++it) {
        if (mbar_test(mbar, parity)) return true;
        if (it > 64) __nanosleep(64);
    }
    return false;
}

// CTA-uniform bounded wait: thread 0 polls, every thread gets the same answer
__device__ __forceinline__ bool cta_wait(uint32_t mbar, uint32_t parity, int *flag) {
    if (threadIdx.x == 0) *flag = mbar_wait(mbar, parity) ? 1 : 0;
    __syncthreads();
    const bool r = *flag != 0;
    __syncthreads();
    return r;
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
          int kb, double *__restrict__ partial) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    TcSmem &sm = *reinterpret_cast<TcSmem *>(
        smem_raw + ((1024 - (smem_u32(smem_raw) & 1023)) & 1023));
    constexpr int EA = 16 / (int)sizeof(Ta), EB = 16 / (int)sizeof(Tb);
    const int t = threadIdx.x;
    const int warp = t >> 5;
    const int K2 = ka + kb;
    const int c_first = t % K2, g_first = t / K2;                 // this thread's first split unit
    const int c_step = TC_THREADS % K2, g_step = TC_THREADS / K2;  // and the stride between units
    // ---- set-up: zero operands and sums, barriers, tensor memory
    for (int e = t; e < 2 * TC_STAGE_BYTES / 16; e += TC_THREADS)
        reinterpret_cast<uint4 *>(&sm.stage[0][0])[e] = make_uint4(0, 0, 0, 0);
    for (int e = t; e < 128 * 128; e += TC_THREADS) {
        sm.acc_hi[e] = 0.f;
        sm.acc_lo[e] = 0.f;
    }
    if (t == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar[0])));
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&sm.mbar[1])));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        sm.timed_out = 0;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_u32(&sm.tmem_base)),
                     "r"(TC_COLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = sm.tmem_base;
    const uint32_t idesc = tc_idesc();
    uint32_t parity[2] = {0, 0};
    bool pending[2] = {false, false};
    bool fresh = true;  // next MMA overwrites the accumulator
    bool ok = true;
    const int64_t ntiles = (n + TC_TILE - 1) / TC_TILE;
    // the 16-byte chunks of the next two tiles held by this thread (two tiles in flight)
    uint4 buf[TC_MAXQ], buf2[TC_MAXQ];
    auto load_tile = [&](int64_t tl, uint4 (&dst)[TC_MAXQ]) {
        if (tl >= ntiles) return;
        const int64_t q0 = tl * TC_TILE;
        const int rws = (int)(n - q0 < TC_TILE ? n - q0 : TC_TILE);
        const int na = rws * lda / EA, nb = rws * ldb / EB;
#pragma unroll
        for (int u = 0; u < TC_MAXQ; ++u) {
            const int q = t + u * TC_THREADS;
            if (q < na) dst[u] = __ldg(reinterpret_cast<const uint4 *>(A + q0 * lda) + q);
            else if (q - na < nb) dst[u] = __ldg(reinterpret_cast<const uint4 *>(B + q0 * ldb) + (q - na));
        }
    };
    load_tile(blockIdx.x, buf);
    load_tile(blockIdx.x + gridDim.x, buf2);
    int it = 0;
    for (int64_t tile = blockIdx.x; tile < ntiles && ok; tile += gridDim.x, ++it) {
        const int st = it & 1;
        if (pending[st]) {  // MMAs of the tile that last used this stage have read it
            ok = cta_wait(smem_u32(&sm.mbar[st]), parity[st], &sm.wait_ok);
            parity[st] ^= 1;
            pending[st] = false;
            if (!ok) break;
        }
        // ---- stage: the tile's rows of A and B are contiguous (row stride lda / ldb); the CTA
        // read them as 16-byte chunks in address order two tiles ahead and now parks them in
        // shared memory as they are
        const int64_t r0 = tile * TC_TILE;
        const int rows = (int)(n - r0 < TC_TILE ? n - r0 : TC_TILE);
        const int qa = rows * lda / EA, qb = rows * ldb / EB;  // chunks of A and of B
#pragma unroll
        for (int u = 0; u < TC_MAXQ; ++u) {
            const int q = t + u * TC_THREADS;
            if (q < qa + qb) reinterpret_cast<uint4 *>(sm.raw)[q] = buf[u];
        }
        __syncthreads();
#pragma unroll
        for (int u = 0; u < TC_MAXQ; ++u) buf[u] = buf2[u];
        load_tile(tile + 2 * (int64_t)gridDim.x, buf2);  // flies during two splits and MMAs
        // ---- split: unit (c, g) is column c of [A B] over graph rows 8g .. 8g+7 (zero past the
        // end); each of its S BF16 pieces is 8 consecutive K elements, i.e. one 16-byte row of
        // a core matrix (operand row m = s K2 + c, K half g & 1 of slice g / 2)
        {
            const Ta *ra = reinterpret_cast<const Ta *>(sm.raw);
            const Tb *rb = reinterpret_cast<const Tb *>(sm.raw + (size_t)qa * 16);
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
            tc_commit(smem_u32(&sm.mbar[st]));
        }
        fresh = false;
        pending[st] = true;
        const bool last = tile + gridDim.x >= ntiles;
        if ((it + 1) % TC_FLUSH == 0 || last) {
            // ---- fold the accumulator into the double-float sums
            ok = cta_wait(smem_u32(&sm.mbar[st]), parity[st], &sm.wait_ok);
            parity[st] ^= 1;
            pending[st] = false;
            if (!ok) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            // warp w < 16 reads lane quarter w % 4 (its own TMEM lanes), column slice w / 4
            const int lane_m = (warp & 3) * 32 + (t & 31);
            constexpr int CW = TC_COLS / (TC_FOLD_WARPS / 4);  // columns per warp
#pragma unroll 1
            for (int c0 = (warp >> 2) * CW; warp < TC_FOLD_WARPS && c0 < ((warp >> 2) + 1) * CW; c0 += 32) {
                uint32_t v[32];
                const uint32_t taddr = tmem + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)c0;
                asm volatile(
                    "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                    "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                    "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                    : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]),
                      "=r"(v[6]), "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]),
                      "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]), "=r"(v[16]),
                      "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]),
                      "=r"(v[22]), "=r"(v[23]), "=r"(v[24]), "=r"(v[25]), "=r"(v[26]),
                      "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                    : "r"(taddr));
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int q = 0; q < 32; ++q) {
                    const int idx = (c0 + q) * 128 + lane_m;  // [n][m], m = this thread's lane
                    float s = sm.acc_hi[idx], e = sm.acc_lo[idx];
                    two_sum(s, e, __uint_as_float(v[q]));
                    sm.acc_hi[idx] = s;
                    sm.acc_lo[idx] = e;
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            fresh = true;
        }
        __syncthreads();
    }
    // ---- on a timeout, wait (bounded) for whatever is still in flight
    if (t == 0) {
        if (!ok) sm.timed_out = 1;
        for (int s = 0; s < 2; ++s)
            if (pending[s] && !mbar_wait(smem_u32(&sm.mbar[s]), parity[s])) sm.timed_out = 1;
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                     "r"(TC_COLS));
    // ---- combine the S x S piece blocks: G[i][j] = sum_{a,b} D[a K2 + i][b K2 + j], i <= j
    const bool bad = sm.timed_out != 0;
    double *out = partial + (int64_t)blockIdx.x * K2 * K2;
    for (int e = t; e < K2 * K2; e += TC_THREADS) {
        const int i = e / K2, j = e % K2;
        if (i > j) continue;
        float s = 0.f, err = 0.f;
#pragma unroll
        for (int a = 0; a < S; ++a)
#pragma unroll
            for (int b = 0; b < S; ++b) {
                const int idx = (b * K2 + j) * 128 + (a * K2 + i);
                two_sum(s, err, sm.acc_hi[idx]);
                err += sm.acc_lo[idx];
            }
        const double v = bad ? NAN : (double)s + (double)err;
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
    // one tile of A and B fits the raw buffer (TC_RAW_CHUNKS 16-byte chunks)
    const int ea = 16 / (int)dtype_size(at), eb = kb ? 16 / (int)dtype_size(bt) : 1;
    if (TC_TILE * (lda / ea + (kb ? ldb / eb : 0)) > TC_RAW_CHUNKS) return 0;
    const int S = (at == SPED_F32 || (kb > 0 && bt == SPED_F32)) ? 3 : 1;
    return S * (ka + kb) <= 128 ? S : 0;
}

size_t gram_tc_scratch(int64_t n, int ka, int kb) {
    const int K2 = ka + kb;
    (void)n;
    return sizeof(double) * (size_t)K2 * K2 * 512;
}

template <typename Ta, typename Tb, int S>
static sped_status run_tc(int64_t n, const void *A, int lda, int ka, const void *B, int ldb, int kb,
                          double *G, double *partial, int ctas, cudaStream_t st) {
    const size_t smem = sizeof(TcSmem) + 1024;
    auto kern = k_gram_tc<Ta, Tb, S>;
    SPED_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    kern<<<ctas, TC_THREADS, smem, st>>>(n, (const Ta *)A, lda, ka, (const Tb *)B, ldb, kb,
                                         partial);
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
