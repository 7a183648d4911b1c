// The solver step's N x k update kernel (see solver.cu for the step it belongs to) and its
// launcher; each update_km*.cu includes this header and instantiates the launcher for its
// widths.
#pragma once

#include "solver_update.cuh"

namespace sped {

// One row of an N x k block into registers (zero past k): 16-byte loads when the row start and
// the leading dimension allow it (vec), else element loads. Loads stop at the 16-byte chunk that
// holds element k-1, which lies inside the row's leading dimension.
template <int KM, bool RO, typename T, typename Acc>
__device__ __forceinline__ void load_row(const T *p, int k, bool vec, Acc *out) {
    constexpr int E = 16 / (int)sizeof(T);
    static_assert(KM % E == 0, "row chunks");
    if (vec) {
#pragma unroll
        for (int q = 0; q < KM / E; ++q) {
            uint4 c = make_uint4(0, 0, 0, 0);
            if (q * E < k) c = RO ? __ldg(reinterpret_cast<const uint4 *>(p) + q)
                                  : reinterpret_cast<const uint4 *>(p)[q];
            const T *e = reinterpret_cast<const T *>(&c);
#pragma unroll
            for (int u = 0; u < E; ++u) out[q * E + u] = q * E + u < k ? cvt<Acc>(e[u]) : Acc(0);
        }
    } else {
#pragma unroll
        for (int j = 0; j < KM; ++j) out[j] = j < k ? cvt<Acc>(RO ? __ldg(p + j) : p[j]) : Acc(0);
    }
}

// V <- (V A + Y B) diag(scale), in place, one row per thread. The coefficient matrices sit in
// shared memory as [j][i] with i contiguous, so one 16-byte shared load feeds four outputs;
// B is diagonal for mu-EG (bdiag), which skips its k^2 products. The row is held in registers,
// so each group of four outputs is stored as soon as it is computed (and, with a shadow, its
// BF16 rounding into the shadow row, which the next step's BF16 chain starts from). With STATS
// it also accumulates, per column, ||v_new_i - v_i||^2 and the invariant-subspace residual
// ||y_i - V C_i||^2 (old V); without, it is the plain update (one read of V and Y, one write).
template <typename Tm, typename Ty, int KM, bool STATS>
__global__ void __launch_bounds__(256)
k_update(int64_t n, Tm *__restrict__ V, int ldv, const Ty *__restrict__ Y, int ldy, int k,
         Coefs *cf, int bdiag, int vec, __nv_bfloat16 *__restrict__ shadow, int lds) {
    using A = typename AccOf<Tm>::type;
    static_assert(KM % 4 == 0, "KM");
    __shared__ __align__(16) A sA[KM * KM];
    __shared__ __align__(16) A sB[KM * KM];
    __shared__ __align__(16) A sC[STATS ? KM * KM : 4];
    __shared__ A sS[KM];
    __shared__ double sdv[KM], sres[KM];
    pdl_wait();  // launched with programmatic dependent launch: the coefficients, V and Y
    for (int e = threadIdx.x; e < KM * KM; e += blockDim.x) {
        const int j = e / KM, i = e % KM;
        const bool in = i < k && j < k;
        sA[e] = in ? (A)cf->A[j * MAXK + i] : A(0);
        sB[e] = in ? (A)cf->B[j * MAXK + i] : A(0);
        if (STATS) sC[e] = in ? (A)cf->C[j * MAXK + i] : A(0);
    }
    for (int e = threadIdx.x; e < KM; e += blockDim.x) {
        sS[e] = e < k ? (A)cf->scale[e] : A(0);
        sdv[e] = 0.0;
        sres[e] = 0.0;
    }
    __syncthreads();
    A dv[STATS ? KM : 1], rs[STATS ? KM : 1];
#pragma unroll
    for (int i = 0; i < (STATS ? KM : 1); ++i) {
        dv[i] = A(0);
        rs[i] = A(0);
    }
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        Tm *vr = V + r * ldv;
        const Ty *yr = Y + r * ldy;
        A v[KM], y[KM];
        load_row<KM, false>(vr, k, vec != 0, v);
        load_row<KM, true>(yr, k, vec != 0, y);
        uint32_t sw0 = 0, sw1 = 0;  // first half of the shadow chunk being built (8 BF16 values)
#pragma unroll
        for (int i0 = 0; i0 < KM; i0 += 4) {
            if (i0 >= k) break;
            A s[4] = {A(0), A(0), A(0), A(0)}, pq[4] = {A(0), A(0), A(0), A(0)};
#pragma unroll
            for (int j = 0; j < KM; ++j) {
                const A *a4 = sA + j * KM + i0;
#pragma unroll
                for (int q = 0; q < 4; ++q) s[q] += v[j] * a4[q];
                if (STATS) {
                    const A *c4 = sC + j * KM + i0;
#pragma unroll
                    for (int q = 0; q < 4; ++q) pq[q] += v[j] * c4[q];
                }
                if (!bdiag) {
                    const A *b4 = sB + j * KM + i0;
#pragma unroll
                    for (int q = 0; q < 4; ++q) s[q] += y[j] * b4[q];
                }
            }
            alignas(16) Tm o[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + q;
                if (bdiag) s[q] += y[i] * sB[i * KM + i];
                s[q] *= sS[i];
                if (STATS) {
                    const A d = s[q] - v[i];
                    dv[STATS ? i : 0] += d * d;
                    const A e = y[i] - pq[q];
                    rs[STATS ? i : 0] += e * e;
                }
                o[q] = from_acc<Tm>(s[q]);
            }
            if (shadow) {  // BF16 copy of the new row in 16-byte chunks of eight values
                const __nv_bfloat162 lo2 = __floats2bfloat162_rn((float)o[0], (float)o[1]);
                const __nv_bfloat162 hi2 = __floats2bfloat162_rn((float)o[2], (float)o[3]);
                const uint32_t w0 = *reinterpret_cast<const uint32_t *>(&lo2);
                const uint32_t w1 = *reinterpret_cast<const uint32_t *>(&hi2);
                __nv_bfloat16 *sr = shadow + r * lds + (i0 & ~7);
                if ((i0 & 7) == 0) {
                    sw0 = w0;
                    sw1 = w1;
                    if (i0 + 4 >= k) {  // the row ends inside this half chunk
                        if (i0 + 4 == k) *reinterpret_cast<uint2 *>(sr) = make_uint2(w0, w1);
                        else
#pragma unroll
                            for (int q = 0; q < 3; ++q)
                                if (i0 + q < k) sr[q] = __float2bfloat16_rn((float)o[q]);
                    }
                } else if (i0 + 4 <= k) {
                    *reinterpret_cast<uint4 *>(sr) = make_uint4(sw0, sw1, w0, w1);
                } else {
                    *reinterpret_cast<uint2 *>(sr) = make_uint2(sw0, sw1);
#pragma unroll
                    for (int q = 0; q < 3; ++q)
                        if (i0 + q < k) sr[4 + q] = __float2bfloat16_rn((float)o[q]);
                }
            }
            if (vec && i0 + 4 <= k) {
                if (sizeof(Tm) == 4) {
                    *reinterpret_cast<uint4 *>(vr + i0) = *reinterpret_cast<const uint4 *>(o);
                } else {
                    reinterpret_cast<uint4 *>(vr + i0)[0] = reinterpret_cast<const uint4 *>(o)[0];
                    reinterpret_cast<uint4 *>(vr + i0)[1] = reinterpret_cast<const uint4 *>(o)[1];
                }
            } else {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (i0 + q < k) vr[i0 + q] = o[q];
            }
        }
    }
    if constexpr (STATS) {
        // column sums: warp shuffle, then shared, then one atomic per block and column
#pragma unroll
        for (int i = 0; i < (STATS ? KM : 1); ++i) {
            A x = dv[i], z = rs[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                x += __shfl_down_sync(0xffffffffu, x, o);
                z += __shfl_down_sync(0xffffffffu, z, o);
            }
            if ((threadIdx.x & 31) == 0 && i < k) {
                atomicAdd(&sdv[i], (double)x);
                atomicAdd(&sres[i], (double)z);
            }
        }
        __syncthreads();
        if (threadIdx.x < k) {
            atomicAdd(&cf->dv2[threadIdx.x], sdv[threadIdx.x]);
            atomicAdd(&cf->res2[threadIdx.x], sres[threadIdx.x]);
        }
    }
    pdl_trigger();
}

template <typename Tm, typename Ty, int KM>
sped_status launch_update(int blocks, int64_t n, void *V, int ldv, const void *Y, int ldy, int k,
                          Coefs *cf, int bdiag, int vec, bool stats, __nv_bfloat16 *shadow,
                          int lds, cudaStream_t st) {
    if (stats)
        SPED_CUDA(launch_pdl(k_update<Tm, Ty, KM, true>, dim3(blocks), dim3(256), 0, st, n,
                             (Tm *)V, ldv, (const Ty *)Y, ldy, k, cf, bdiag, vec, shadow, lds));
    else
        SPED_CUDA(launch_pdl(k_update<Tm, Ty, KM, false>, dim3(blocks), dim3(256), 0, st, n,
                             (Tm *)V, ldv, (const Ty *)Y, ldy, k, cf, bdiag, vec, shadow, lds));
    SPED_CHECK_LAUNCH("k_update");
    return SPED_OK;
}

}  // namespace sped

#define SPED_UPDATE_INSTANTIATE_PAIR(TM, TY, KM)                                               \
    namespace sped {                                                                           \
    template sped_status launch_update<TM, TY, KM>(int, int64_t, void *, int, const void *, int, \
                                                   int, Coefs *, int, int, bool,               \
                                                   __nv_bfloat16 *, int, cudaStream_t);        \
    }

#define SPED_UPDATE_INSTANTIATE(KM)                 \
    SPED_UPDATE_INSTANTIATE_PAIR(float, float, KM)  \
    SPED_UPDATE_INSTANTIATE_PAIR(float, double, KM) \
    SPED_UPDATE_INSTANTIATE_PAIR(double, double, KM) \
    SPED_UPDATE_INSTANTIATE_PAIR(double, float, KM)
