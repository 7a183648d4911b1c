// Tall-skinny Gram G = [A B]^T [A B] for the solver step: every inner product the mu-EG and
// Oja updates need (<v_i,v_j>, <v_i,y_j>, <y_i,y_j>) comes from this one (2k x 2k) matrix.
//
// CUDA-core schedule: row tiles staged in shared memory (converted to the product type),
// 4x4 register blocks of the upper triangle per thread, F32 accumulation over a short window
// of rows (exact products for BF16 inputs) and F64 accumulation across windows; per-CTA F64
// partials reduced in a fixed order (deterministic).
#include <mutex>

#include "sped_internal.cuh"

namespace sped {

constexpr int GRAM_THREADS = 256;
constexpr int GRAM_TILE = 128;   // rows per shared-memory tile
constexpr int GRAM_WINDOW = 256; // rows per F32 accumulation window (per worker)
constexpr int GRAM_MAXK = 80;  // 2k for k <= 40 (the 4x4 block pairs fit one CTA's threads)

struct GramShape {
    int K2, KP, nb, P, S, stride;
};

static GramShape gram_shape(int ka, int kb) {
    GramShape s;
    s.K2 = ka + kb;
    s.KP = (s.K2 + 3) / 4 * 4;
    s.nb = s.KP / 4;
    s.P = s.nb * (s.nb + 1) / 2;
    s.S = GRAM_THREADS / s.P;
    if (s.S < 1) s.S = 1;
    s.stride = s.KP + 4;
    return s;
}

template <typename T, typename P>
__device__ __forceinline__ P ld_elem(const T *p) { return cvt<P>(*p); }

template <typename Ta, typename Tb, typename Pt>
__global__ void __launch_bounds__(GRAM_THREADS)
k_gram(int64_t n, const Ta *__restrict__ A, int lda, int ka, const Tb *__restrict__ B, int ldb,
       int kb, GramShape sh, double *__restrict__ partial) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Pt *tile = reinterpret_cast<Pt *>(smem_raw);
    const int t = threadIdx.x;
    const int pair = t % sh.P;
    const int slice = t / sh.P;
    const bool worker = slice < sh.S && t < sh.P * sh.S;
    // block coordinates of this worker's pair (bi <= bj), pair-major upper triangle
    int bi = 0, bj = 0;
    {
        int p = pair, row = 0, len = sh.nb;
        while (p >= len) {
            p -= len;
            ++row;
            --len;
        }
        bi = row;
        bj = row + p;
    }
    double accd[16];
    Pt accf[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) {
        accd[q] = 0.0;
        accf[q] = Pt(0);
    }
    int win = 0;
    const int64_t ntiles = (n + GRAM_TILE - 1) / GRAM_TILE;
    for (int64_t tl = blockIdx.x; tl < ntiles; tl += gridDim.x) {
        const int64_t r0 = tl * GRAM_TILE;
        const int rows = (int)(n - r0 < GRAM_TILE ? n - r0 : GRAM_TILE);
        __syncthreads();
        for (int e = t; e < GRAM_TILE * sh.KP; e += GRAM_THREADS) {
            int rr = e / sh.KP, cc = e - rr * sh.KP;
            Pt v = Pt(0);
            if (rr < rows) {
                int64_t r = r0 + rr;
                if (cc < ka) v = ld_elem<Ta, Pt>(A + r * lda + cc);
                else if (cc < sh.K2) v = ld_elem<Tb, Pt>(B + r * ldb + (cc - ka));
            }
            tile[rr * sh.stride + cc] = v;
        }
        __syncthreads();
        if (worker) {
            for (int rr = slice; rr < rows; rr += sh.S) {
                const Pt *row = tile + rr * sh.stride;
                Pt a[4], b[4];
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    a[q] = row[bi * 4 + q];
                    b[q] = row[bj * 4 + q];
                }
#pragma unroll
                for (int x = 0; x < 4; ++x)
#pragma unroll
                    for (int y = 0; y < 4; ++y) accf[x * 4 + y] += a[x] * b[y];
                if (++win == GRAM_WINDOW) {
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        accd[q] += (double)accf[q];
                        accf[q] = Pt(0);
                    }
                    win = 0;
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) accd[q] += (double)accf[q];
    // reduce slices through shared memory (reusing the tile area), fixed order
    __syncthreads();
    double *red = reinterpret_cast<double *>(smem_raw);
    if (worker) {
#pragma unroll
        for (int q = 0; q < 16; ++q) red[(slice * sh.P + pair) * 16 + q] = accd[q];
    }
    __syncthreads();
    for (int e = t; e < sh.P * 16; e += GRAM_THREADS) {
        double s = 0.0;
        for (int sl = 0; sl < sh.S; ++sl) s += red[sl * sh.P * 16 + e];
        partial[(int64_t)blockIdx.x * sh.P * 16 + e] = s;
    }
}

// sum CTA partials in order and scatter the upper-triangle blocks into the full symmetric G
__global__ void k_gram_reduce(const double *__restrict__ partial, int nparts, GramShape sh,
                              double *__restrict__ G) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= sh.P * 16) return;
    double s = 0.0;
    for (int c = 0; c < nparts; ++c) s += partial[(int64_t)c * sh.P * 16 + e];
    int pair = e / 16, q = e % 16;
    int p = pair, row = 0, len = sh.nb;
    while (p >= len) {
        p -= len;
        ++row;
        --len;
    }
    int i = row * 4 + q / 4, j = (row + p) * 4 + q % 4;
    if (i < sh.K2 && j < sh.K2) {
        G[i * sh.K2 + j] = s;
        G[j * sh.K2 + i] = s;
    }
}

static int gram_ctas(int64_t n) {
    int64_t tiles = (n + GRAM_TILE - 1) / GRAM_TILE;
    int64_t c = 2LL * device_sm_count();
    if (tiles < c) c = tiles;
    return c < 1 ? 1 : (int)c;
}

size_t gram_scratch(int64_t n, int ka, int kb) {
    GramShape sh = gram_shape(ka, kb);
    ScratchPlan p;
    int64_t tiles = (n + GRAM_TILE - 1) / GRAM_TILE;
    int64_t c = 2LL * 256;  // upper bound on CTAs for any device this library supports
    if (tiles < c) c = tiles < 1 ? 1 : tiles;
    const size_t core = sizeof(double) * (size_t)c * sh.P * 16;
    const size_t tc = (ka + kb) <= GRAM_MAXK ? gram_tc_scratch(n, ka, kb) : 0;  // tensor path
    p.add(core > tc ? core : tc);
    return p.total();
}

template <typename Ta, typename Tb>
static sped_status run_gram(int64_t n, const void *A, int lda, int ka, const void *B, int ldb,
                            int kb, double *G, double *partial, int ctas, cudaStream_t st) {
    GramShape sh = gram_shape(ka, kb);
    const bool f64 = sizeof(Ta) == 8 || sizeof(Tb) == 8;
    size_t elt = f64 ? 8 : 4;
    size_t tile_bytes = (size_t)GRAM_TILE * sh.stride * elt;
    size_t red_bytes = (size_t)sh.S * sh.P * 16 * sizeof(double);
    size_t smem = tile_bytes > red_bytes ? tile_bytes : red_bytes;
    if (f64) {
        auto kern = k_gram<Ta, Tb, double>;
        if (smem > 48 * 1024)
            SPED_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
        kern<<<ctas, GRAM_THREADS, smem, st>>>(n, (const Ta *)A, lda, ka, (const Tb *)B, ldb, kb,
                                              sh, partial);
    } else {
        auto kern = k_gram<Ta, Tb, float>;
        if (smem > 48 * 1024)
            SPED_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)smem));
        kern<<<ctas, GRAM_THREADS, smem, st>>>(n, (const Ta *)A, lda, ka, (const Tb *)B, ldb, kb,
                                              sh, partial);
    }
    SPED_CHECK_LAUNCH("k_gram");
    k_gram_reduce<<<(sh.P * 16 + 255) / 256, 256, 0, st>>>(partial, ctas, sh, G);
    SPED_CHECK_LAUNCH("k_gram_reduce");
    return SPED_OK;
}

using bf16 = __nv_bfloat16;

sped_status launch_gram(int64_t n, const void *A, sped_dtype at, int lda, int ka, const void *B,
                        sped_dtype bt, int ldb, int kb, double *G, Scratch &scr, cudaStream_t st) {
    if (ka + kb > GRAM_MAXK || ka < 1 || kb < 0)
        return fail(SPED_ERR_UNSUPPORTED, "gram: ka + kb = %d (1..%d supported)", ka + kb,
                    GRAM_MAXK);
    if (n > 0 && gram_tc_pieces(at, bt, ka, kb, lda, kb ? ldb : 0))  // F32/BF16: tensor cores
        return launch_gram_tc(n, A, at, lda, ka, B, bt, ldb, kb, G, scr, st);
    GramShape sh = gram_shape(ka, kb);
    int ctas = gram_ctas(n);
    double *partial = (double *)scr.take(sizeof(double) * (size_t)ctas * sh.P * 16);
    if (!partial) return fail(SPED_ERR_SCRATCH, "gram: scratch too small");
    if (n == 0) {
        SPED_CUDA(cudaMemsetAsync(G, 0, sizeof(double) * sh.K2 * sh.K2, st));
        return SPED_OK;
    }
    if (kb == 0) {
        B = A;
        bt = at;
        ldb = lda;
    }
#define G2(TA, TB) return run_gram<TA, TB>(n, A, lda, ka, B, ldb, kb, G, partial, ctas, st)
    if (at == SPED_F32 && bt == SPED_F32) G2(float, float);
    if (at == SPED_BF16 && bt == SPED_BF16) G2(bf16, bf16);
    if (at == SPED_F32 && bt == SPED_BF16) G2(float, bf16);
    if (at == SPED_BF16 && bt == SPED_F32) G2(bf16, float);
    if (at == SPED_F64 && bt == SPED_F64) G2(double, double);
    if (at == SPED_F32 && bt == SPED_F64) G2(float, double);
    if (at == SPED_F64 && bt == SPED_F32) G2(double, float);
    if (at == SPED_BF16 && bt == SPED_F64) G2(bf16, double);
    if (at == SPED_F64 && bt == SPED_BF16) G2(double, bf16);
#undef G2
    return fail(SPED_ERR_UNSUPPORTED, "gram: dtypes %d/%d", (int)at, (int)bt);
}

}  // namespace sped

using namespace sped;

extern "C" {

sped_status sped_gram_scratch_size(int64_t n, int ka, int kb, size_t *bytes) {
    if (!bytes || n < 0 || ka < 1 || kb < 0) return fail(SPED_ERR_INVALID_ARG, "gram_scratch_size");
    *bytes = gram_scratch(n, ka, kb);
    return SPED_OK;
}

sped_status sped_gram(int64_t n, const void *d_A, sped_dtype a_t, int lda, int ka, const void *d_B,
                      sped_dtype b_t, int ldb, int kb, double *d_G, void *d_scratch,
                      size_t scratch_bytes, void *stream) {
    if (n < 0 || !d_G) return fail(SPED_ERR_INVALID_ARG, "gram: bad n or null G");
    if (!dtype_valid(a_t) || (kb > 0 && !dtype_valid(b_t)))
        return fail(SPED_ERR_INVALID_ARG, "gram: dtype");
    if (ka < 1 || lda < ka || !d_A) return fail(SPED_ERR_INVALID_ARG, "gram: A layout");
    if (kb < 0 || (kb > 0 && (ldb < kb || !d_B)))
        return fail(SPED_ERR_INVALID_ARG, "gram: B layout");
    // 16-byte rows and bases: the tensor path moves whole tiles with bulk copies
    SPED_TRY(check_layout(d_A, a_t, ka, lda, "gram A"));
    if (kb > 0) SPED_TRY(check_layout(d_B, b_t, kb, ldb, "gram B"));
    Scratch scr(d_scratch, scratch_bytes);
    return launch_gram(n, d_A, a_t, lda, ka, d_B, b_t, ldb, kb, d_G, scr, as_stream(stream));
}

}  // extern "C"

// ---------------------------------------------------------------------------------------
// Gram with no caller scratch, for callers that may not allocate device memory at all.
//
// The per-CTA partial sums live in a fixed 4 MiB array of static device memory instead of a
// caller-provided buffer. Every GPU that loads this library holds that array until the
// process exits. The array's name is only a host-side stand-in, so its device address is
// looked up with cudaGetSymbolAddress once per device (with that device current) on the first
// call made on that device; make that first call before any stream capture. The kernels are
// the ones sped_gram launches; only fewer CTAs are used when the partials would not fit.
// Each call writes every partial it later reads, so nothing has to start at zero. All calls
// share the one array: calls that overlap on the GPU (other streams, other host threads)
// race on it and must be serialised by the caller.
// ---------------------------------------------------------------------------------------
namespace sped {

constexpr size_t GRAM_STATIC_DOUBLES = 512 * 1024;  // 4 MiB
constexpr int GRAM_STATIC_MAXK = 64;                 // columns ka + kb at most
constexpr int GRAM_STATIC_MAX_DEVICES = 64;

static __device__ __align__(256) double g_gram_static_partials[GRAM_STATIC_DOUBLES];

static double *g_gram_static_addr[GRAM_STATIC_MAX_DEVICES];
static std::mutex g_gram_static_mu;

static sped_status gram_static_address(double **out) {
    int dev = 0;
    SPED_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= GRAM_STATIC_MAX_DEVICES)
        return fail(SPED_ERR_UNSUPPORTED, "gram_noalloc: device ordinal %d >= %d", dev,
                    GRAM_STATIC_MAX_DEVICES);
    std::lock_guard<std::mutex> lock(g_gram_static_mu);
    if (!g_gram_static_addr[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_gram_static_partials);
        if (e != cudaSuccess || !p) return cuda_fail(e, "gram_noalloc: cudaGetSymbolAddress");
        g_gram_static_addr[dev] = (double *)p;
    }
    *out = g_gram_static_addr[dev];
    return SPED_OK;
}

}  // namespace sped

extern "C" sped_status sped_gram_noalloc(int64_t n, const void *d_A, sped_dtype a_t, int lda,
                                         int ka, const void *d_B, sped_dtype b_t, int ldb, int kb,
                                         double *d_G, void *stream) {
    if (n < 0 || !d_G) return fail(SPED_ERR_INVALID_ARG, "gram_noalloc: bad n or null G");
    if (!dtype_valid(a_t) || (kb > 0 && !dtype_valid(b_t)))
        return fail(SPED_ERR_INVALID_ARG, "gram_noalloc: dtype");
    if (ka < 1 || lda < ka || !d_A) return fail(SPED_ERR_INVALID_ARG, "gram_noalloc: A layout");
    if (kb < 0 || (kb > 0 && (ldb < kb || !d_B)))
        return fail(SPED_ERR_INVALID_ARG, "gram_noalloc: B layout");
    SPED_TRY(check_layout(d_A, a_t, ka, lda, "gram_noalloc A"));
    if (kb > 0) SPED_TRY(check_layout(d_B, b_t, kb, ldb, "gram_noalloc B"));
    if (ka + kb > GRAM_STATIC_MAXK)
        return fail(SPED_ERR_UNSUPPORTED,
                    "gram_noalloc: ka + kb = %d exceeds the maximum of %d columns", ka + kb,
                    GRAM_STATIC_MAXK);
    const GramShape sh = gram_shape(ka, kb);
    const size_t per_cta = (size_t)sh.P * 16;
    if (per_cta > GRAM_STATIC_DOUBLES)
        return fail(SPED_ERR_UNSUPPORTED, "gram_noalloc: partials exceed the static array");
    double *partial = nullptr;
    SPED_TRY(gram_static_address(&partial));
    cudaStream_t st = as_stream(stream);
    if (n == 0) {
        SPED_CUDA(cudaMemsetAsync(d_G, 0, sizeof(double) * sh.K2 * sh.K2, st));
        return SPED_OK;
    }
    int ctas = gram_ctas(n);
    const int fit = (int)(GRAM_STATIC_DOUBLES / per_cta);
    if (ctas > fit) ctas = fit;
    if (kb == 0) {
        d_B = d_A;
        b_t = a_t;
        ldb = lda;
    }
#define G2(TA, TB) return run_gram<TA, TB>(n, d_A, lda, ka, d_B, ldb, kb, d_G, partial, ctas, st)
    if (a_t == SPED_F32 && b_t == SPED_F32) G2(float, float);
    if (a_t == SPED_BF16 && b_t == SPED_BF16) G2(bf16, bf16);
    if (a_t == SPED_F32 && b_t == SPED_BF16) G2(float, bf16);
    if (a_t == SPED_BF16 && b_t == SPED_F32) G2(bf16, float);
    if (a_t == SPED_F64 && b_t == SPED_F64) G2(double, double);
    if (a_t == SPED_F32 && b_t == SPED_F64) G2(float, double);
    if (a_t == SPED_F64 && b_t == SPED_F32) G2(double, float);
    if (a_t == SPED_BF16 && b_t == SPED_F64) G2(bf16, double);
    if (a_t == SPED_F64 && b_t == SPED_BF16) G2(double, bf16);
#undef G2
    return fail(SPED_ERR_UNSUPPORTED, "gram_noalloc: dtypes %d/%d", (int)a_t, (int)b_t);
}
