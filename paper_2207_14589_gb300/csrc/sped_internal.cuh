// Internal declarations shared by the CUDA translation units of libsped (not part of the ABI).
#pragma once

#include <cuda_bf16.h>
#include <type_traits>
#include <cuda_runtime.h>
#include <stdint.h>

#include <cstdarg>
#include <cstdio>
#include <vector>

#include "../../include/sped.h"

namespace sped {

// ---------------------------------------------------------------------------------------
// host-side error reporting
// ---------------------------------------------------------------------------------------
void set_error(const char *fmt, ...);
sped_status fail(sped_status st, const char *fmt, ...);
sped_status cuda_fail(cudaError_t e, const char *where);

#define SPED_CUDA(expr)                                                        \
    do {                                                                       \
        cudaError_t _e = (expr);                                               \
        if (_e != cudaSuccess) return ::sped::cuda_fail(_e, #expr);            \
    } while (0)

#define SPED_CHECK_LAUNCH(name)                                                \
    do {                                                                       \
        cudaError_t _e = cudaGetLastError();                                   \
        if (_e != cudaSuccess) return ::sped::cuda_fail(_e, name);             \
    } while (0)

#define SPED_TRY(expr)                                                         \
    do {                                                                       \
        sped_status _s = (expr);                                               \
        if (_s != SPED_OK) return _s;                                          \
    } while (0)

inline cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

// Launch with programmatic dependent launch: the kernel may be scheduled while the previous
// kernel in the stream is finishing. Every kernel launched this way executes pdl_wait() before
// its first access to memory another kernel writes, and pdl_trigger() once its own stores are
// issued.
template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t st, Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, static_cast<Args &&>(args)...);
}

inline size_t dtype_size(sped_dtype t) {
    return t == SPED_BF16 ? 2 : (t == SPED_F32 ? 4 : 8);
}
inline bool dtype_valid(int t) { return t == SPED_BF16 || t == SPED_F32 || t == SPED_F64; }

// elements per 16-byte chunk
inline int chunk_elems(sped_dtype t) { return (int)(16 / dtype_size(t)); }

// leading dimension rounded so that a row is a whole number of 16-byte chunks
inline int padded_ld(int k, sped_dtype t) {
    int e = chunk_elems(t);
    return (k + e - 1) / e * e;
}

inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

// Simple bump allocator over a caller-provided scratch buffer (256-byte aligned pieces).
struct Scratch {
    char *base;
    size_t cap, used;
    Scratch(void *p, size_t bytes) : base((char *)p), cap(bytes), used(0) {}
    void *take(size_t bytes) {
        size_t off = align_up(used, 256);
        if (off + bytes > cap || (base == nullptr && bytes > 0)) return nullptr;
        used = off + bytes;
        return base + off;
    }
};

// size accounting twin of Scratch
struct ScratchPlan {
    size_t used = 0;
    void add(size_t bytes) { used = align_up(used, 256) + bytes; }
    size_t total() const { return align_up(used, 256); }
};

int device_sm_count();

// ---------------------------------------------------------------------------------------
// graph
// ---------------------------------------------------------------------------------------
struct Poly {
    int kind = SPED_POLY_SHIFT;
    int ell = 1;
    double s = 0.0;            // limit form scale
    double shift = 0.0;        // Horner: T = L + shift I
    double lambda_star = 0.0;  // SHIFT / LOG reversal
    double eps = 0.0;
    std::vector<double> horner;  // c_0..c_l in powers of T (Horner kinds)
    std::vector<double> power;   // c_0..c_l in powers of L (stochastic mode)
    std::vector<double> cheb;    // c_0..c_l of the Chebyshev series (CHEBYSHEV)
    double cheb_a = 0.0, cheb_b = 0.0;  // interval mapped onto [-1, 1]
};

}  // namespace sped

struct sped_graph {
    int device;
    int64_t n, nnz, n_edges;
    const int32_t *rp, *ci;
    const float *w;       // active per-entry weights (caller array or ws_w) or nullptr
    int32_t *rev;         // rev[p]: position of the reverse entry of p
    int32_t *eid;         // undirected edge id of entry p
    int32_t *edge_p;      // entry position (row a, col b, a < b) of edge e
    int32_t *edge_a;      // row a of edge e
    int2 *edge_ab;        // (a, b) of edge e in one 8-byte word (one load per sampled edge)
    int32_t *eoff;        // first edge id of row r (n+1)
    float *ws_w;          // workspace copy for weights set per edge
    void *stats;          // small device statistics slot inside the workspace
    int32_t max_deg;
    double max_wdeg;
    double lambda_bound;
    sped::Poly poly;
    int32_t tuned_split;  // chain-step schedule chosen by sped_autotune: 0 none (degree rule),
                          // 1 row group, 2 merge path
    int32_t merge_ipg;    // merge-path share in items (rows + entries); 0 = default
};

namespace sped {

// ---------------------------------------------------------------------------------------
// device helpers
// ---------------------------------------------------------------------------------------
template <typename T> struct AccOf { using type = float; };
template <> struct AccOf<double> { using type = double; };

// Element conversion to an accumulator type A (float or double) and back.
template <typename A> __device__ __forceinline__ A cvt(__nv_bfloat16 x);
template <> __device__ __forceinline__ float cvt<float>(__nv_bfloat16 x) { return __bfloat162float(x); }
template <> __device__ __forceinline__ double cvt<double>(__nv_bfloat16 x) {
    return (double)__bfloat162float(x);
}
template <typename A> __device__ __forceinline__ A cvt(float x) { return (A)x; }
template <typename A> __device__ __forceinline__ A cvt(double x) { return (A)x; }

template <typename T> __device__ __forceinline__ T from_acc(float x);
template <typename T> __device__ __forceinline__ T from_acc(double x);
template <> __device__ __forceinline__ float from_acc<float>(float x) { return x; }
template <> __device__ __forceinline__ float from_acc<float>(double x) { return (float)x; }
template <> __device__ __forceinline__ double from_acc<double>(float x) { return (double)x; }
template <> __device__ __forceinline__ double from_acc<double>(double x) { return x; }
template <> __device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16>(float x) {
    return __float2bfloat16_rn(x);
}
template <> __device__ __forceinline__ __nv_bfloat16 from_acc<__nv_bfloat16>(double x) {
    return __float2bfloat16_rn((float)x);
}

template <int BYTES> struct VecOf;
template <> struct VecOf<4> { using type = uint32_t; };
template <> struct VecOf<8> { using type = uint2; };
template <> struct VecOf<16> { using type = uint4; };

// programmatic dependent launch: wait for the previous kernel of the stream (its writes
// visible), and let the next one be scheduled
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// BF16 -> F32 of the two halves of a 32-bit word: a BF16 value is the top half of the F32 with
// the same bits, so the conversion is a shift or a mask (exact)
__device__ __forceinline__ float bf16_lo(uint32_t w) { return __uint_as_float(w << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t w) { return __uint_as_float(w & 0xffff0000u); }

// Read E consecutive elements (E * sizeof(T) bytes, naturally aligned) through the read-only
// path, converting to the accumulator type.
template <typename T, int E, typename A>
__device__ __forceinline__ void load_chunk(const T *__restrict__ p, A (&out)[E]) {
    if constexpr (std::is_same<T, __nv_bfloat16>::value && std::is_same<A, float>::value &&
                  E == 8) {
        // one 16-byte load, converted word by word
        const uint4 u = __ldg(reinterpret_cast<const uint4 *>(p));
        const uint32_t w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            out[2 * q] = bf16_lo(w[q]);
            out[2 * q + 1] = bf16_hi(w[q]);
        }
        return;
    }
    constexpr int BYTES = E * (int)sizeof(T);
    static_assert(BYTES == 4 || BYTES == 8 || BYTES == 16 || BYTES == 32 || BYTES == 64, "chunk");
    constexpr int VB = BYTES < 16 ? BYTES : 16;
    constexpr int NV = BYTES / VB;
    constexpr int PER = VB / (int)sizeof(T);
    using V = typename VecOf<VB>::type;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        union { V v; T e[PER]; } u;
        u.v = __ldg(reinterpret_cast<const V *>(p) + q);
#pragma unroll
        for (int i = 0; i < PER; ++i) out[q * PER + i] = cvt<A>(u.e[i]);
    }
}

// Plain (coherent) load of a chunk, for data written earlier in the same kernel.
template <typename T, int E, typename A>
__device__ __forceinline__ void load_chunk_coherent(const T *p, A (&out)[E]) {
    constexpr int BYTES = E * (int)sizeof(T);
    constexpr int VB = BYTES < 16 ? BYTES : 16;
    constexpr int NV = BYTES / VB;
    constexpr int PER = VB / (int)sizeof(T);
    using V = typename VecOf<VB>::type;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        union { V v; T e[PER]; } u;
        u.v = reinterpret_cast<const V *>(p)[q];
#pragma unroll
        for (int i = 0; i < PER; ++i) out[q * PER + i] = cvt<A>(u.e[i]);
    }
}

template <typename T, int E, typename A>
__device__ __forceinline__ void store_chunk(T *p, const A (&in)[E]) {
    constexpr int BYTES = E * (int)sizeof(T);
    constexpr int VB = BYTES < 16 ? BYTES : 16;
    constexpr int NV = BYTES / VB;
    constexpr int PER = VB / (int)sizeof(T);
    using V = typename VecOf<VB>::type;
#pragma unroll
    for (int q = 0; q < NV; ++q) {
        union { V v; T e[PER]; } u;
#pragma unroll
        for (int i = 0; i < PER; ++i) u.e[i] = from_acc<T>(in[q * PER + i]);
        reinterpret_cast<V *>(p)[q] = u.v;
    }
}

// Tail-safe versions: only the first `cnt` (< E) elements are touched.
template <typename T, int E, typename A>
__device__ __forceinline__ void load_partial(const T *__restrict__ p, int cnt, A (&out)[E]) {
#pragma unroll
    for (int i = 0; i < E; ++i) out[i] = i < cnt ? cvt<A>(p[i]) : A(0);
}
// The partial store of a chunk writes the widest aligned pieces that fit (16, 8, then 4 bytes,
// then single elements), so a BF16 row of 20 columns ends with one 8-byte store, not four 2-byte
// ones. Chunks are 8, 16 or 32 bytes (E elements of T, naturally aligned at 16 bytes or more).
template <typename T, int E, typename A>
__device__ __forceinline__ void store_partial(T *p, int cnt, const A (&in)[E]) {
    constexpr int SZ = (int)sizeof(T);
    constexpr int NB = E * SZ;
    if constexpr (NB != 16 && NB != 32) {
#pragma unroll
        for (int i = 0; i < E; ++i)
            if (i < cnt) p[i] = from_acc<T>(in[i]);
    } else {
        union {
            uint32_t w[NB / 4];
            T e[E];
        } u;
#pragma unroll
        for (int i = 0; i < E; ++i) u.e[i] = from_acc<T>(in[i]);
        const int bytes = cnt * SZ;
        char *q = reinterpret_cast<char *>(p);
        int off = 0;
        if constexpr (NB == 32) {
            if (bytes >= 16) {
                *reinterpret_cast<uint4 *>(q) = make_uint4(u.w[0], u.w[1], u.w[2], u.w[3]);
                off = 16;
            }
        }
        if (bytes - off >= 8) {
            uint2 v = make_uint2(u.w[0], u.w[1]);
            if constexpr (NB == 32)
                if (off == 16) v = make_uint2(u.w[4], u.w[5]);
            *reinterpret_cast<uint2 *>(q + off) = v;
            off += 8;
        }
        if (bytes - off >= 4) {
            uint32_t v = off == 0 ? u.w[0] : u.w[2];
            if constexpr (NB == 32) {
                if (off == 16) v = u.w[4];
                if (off == 24) v = u.w[6];
            }
            *reinterpret_cast<uint32_t *>(q + off) = v;
            off += 4;
        }
#pragma unroll
        for (int i = 0; i < E; ++i)
            if (i * SZ >= off && i < cnt) p[i] = u.e[i];
    }
}

// Philox4x32-10 (Salmon et al., SC'11) -- device implementation of the published definition.
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
    const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r > 0) {
            k.x += W0;
            k.y += W1;
        }
        uint32_t hi0 = __umulhi(M0, c.x), lo0 = M0 * c.x;
        uint32_t hi1 = __umulhi(M1, c.z), lo1 = M1 * c.z;
        uint4 n;
        n.x = hi1 ^ c.y ^ k.x;
        n.y = lo1;
        n.z = hi0 ^ c.w ^ k.y;
        n.w = lo0;
        c = n;
    }
    return c;
}

// Word stream: words of philox(key, {a, b, tag, j}) for j = 0, 1, 2, ... in order.
struct WordStream {
    uint2 key;
    uint32_t a, b, tag, j;
    uint4 buf;
    int used;
    __device__ __forceinline__ WordStream(uint64_t seed, uint32_t a_, uint32_t b_, uint32_t tag_)
        : a(a_), b(b_), tag(tag_), j(0), used(4) {
        key.x = (uint32_t)seed;
        key.y = (uint32_t)(seed >> 32);
    }
    __device__ __forceinline__ uint32_t next() {
        if (used == 4) {
            buf = philox4x32_10(make_uint4(a, b, tag, j), key);
            ++j;
            used = 0;
        }
        uint32_t r = used == 0 ? buf.x : used == 1 ? buf.y : used == 2 ? buf.z : buf.w;
        ++used;
        return r;
    }
    // Lemire's multiply-and-reject bounded draw in [0, range), range >= 1.
    __device__ __forceinline__ uint32_t bounded(uint32_t range) {
        uint32_t x = next();
        uint64_t m = (uint64_t)x * range;
        uint32_t l = (uint32_t)m;
        if (l < range) {
            uint32_t t = (uint32_t)(0u - range) % range;
            while (l < t) {
                x = next();
                m = (uint64_t)x * range;
                l = (uint32_t)m;
            }
        }
        return (uint32_t)(m >> 32);
    }
};

// Internal launchers shared across translation units.
sped_status launch_poly_step(const sped_graph *g, int k, const void *X, sped_dtype xt, int ldx,
                             const void *V, sped_dtype vt, int ldv, void *Y, sped_dtype yt, int ldy,
                             double alpha, double beta, double gamma, int split, Scratch &scr,
                             cudaStream_t st);
// the same step plus delta * W2 (a block of X's type and layout ldw2; needs V)
sped_status launch_poly_step_w2(const sped_graph *g, int k, const void *X, sped_dtype xt,
                                int ldx, const void *V, sped_dtype vt, int ldv, void *Y,
                                sped_dtype yt, int ldy, double alpha, double beta, double gamma,
                                const void *W2, int ldw2, double delta, int split, Scratch &scr,
                                cudaStream_t st);
size_t poly_step_scratch(const sped_graph *g, int k, sped_dtype xt, int split);
size_t merge_step_scratch(const sped_graph *g, int k, sped_dtype xt, int ipg);
sped_status launch_gram(int64_t n, const void *A, sped_dtype at, int lda, int ka, const void *B,
                        sped_dtype bt, int ldb, int kb, double *G, Scratch &scr, cudaStream_t st);
size_t gram_scratch(int64_t n, int ka, int kb);
int gram_tc_pieces(sped_dtype at, sped_dtype bt, int ka, int kb, int lda, int ldb);
size_t gram_tc_scratch(int64_t n, int ka, int kb);
sped_status launch_gram_tc(int64_t n, const void *A, sped_dtype at, int lda, int ka, const void *B,
                           sped_dtype bt, int ldb, int kb, double *G, Scratch &scr,
                           cudaStream_t st);
// X0 (may be NULL): a copy of V in type x0t (leading dimension ldx0) read by the first chain
// step instead of V
sped_status apply_poly_impl(const sped_graph *g, int k, const void *V, sped_dtype vt, int ldv,
                            void *Y, sped_dtype yt, int ldy, sped_dtype ct, sped_mode mode,
                            int64_t walkers, uint64_t seed, Scratch &scr, cudaStream_t st,
                            const void *X0, sped_dtype x0t, int ldx0);
size_t apply_poly_scratch(const sped_graph *g, int k, sped_dtype ct, sped_mode mode);
sped_status launch_walk(const sped_graph *g, int k, const void *V, sped_dtype vt, int ldv, void *Y,
                        sped_dtype yt, int ldy, sped_mode mode, int64_t walkers, uint64_t seed,
                        cudaStream_t st);
sped_status check_layout(const void *p, sped_dtype t, int k, int ld, const char *name);

// One edge minibatch: drawn from a graph's edges (graph != NULL: draws j < count of
// multiplication `step`, seed as documented in minibatch.cu) or given by the caller's arrays.
struct EdgeBatch {
    const sped_graph *graph = nullptr;
    uint64_t seed = 0;
    uint32_t step = 0;
    int64_t count = 0;
    double scale = 1.0;  // |E| / count for uniform draws, 1 for stratified draws
    bool stratified = false;  // one draw per stratum of the edge order, weight |S_j|
    const int32_t *a = nullptr, *b = nullptr;
    const float *w = nullptr;
    int32_t *skipped = nullptr;
};
// Y = alpha V + gamma X + delta W2 + beta * scale * sum_j w_j x_j x_j^T X (X, V, W2, Y: F32 or
// F64; W2 of X's type; V and W2 may be NULL)
sped_status launch_edge_step(int64_t n, int k, const void *X, sped_dtype xt, int ldx,
                             const void *V, sped_dtype vt, int ldv, const void *W2, int ldw2,
                             double delta, void *Y, sped_dtype yt, int ldy, double alpha,
                             double beta, double gamma, const EdgeBatch &eb, cudaStream_t st);

}  // namespace sped
