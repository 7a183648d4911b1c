// Differentiable utilities: EigenGame utilities under the dilated operator and their gradients
// with respect to the eigenvector block and to the edge weights.
//
//  u_i = H_ii - sum_{j<i} H_ij^2 / H_jj,  H = V^T M V, M = p(L)   (alpha-EigenGame utilities of
//  the solver family cited in Section 5.1).
//  dV  = Y Hbar^T + M^T (V Hbar),  Y = M V, Hbar = d(sum_i g_i u_i)/dH   (M^T = M: the adjoint of
//        the polynomial chain is the chain itself)
//  dw_e = -s sum_{t=0}^{l-1} (x_e^T A_t) . (x_e^T C_{l-1-t}),  A_t = B^t V, C_u = B^u (V Hbar^T),
//        B = I - sL, for the limit form M = B^l, since dL/dw_e = x_e x_e^T (Section 2, weighted L
//        of Section 2.1) and dB^l = sum_t B^t dB B^{l-1-t}.
// The C_u are needed in decreasing u while the A_t run forward, so C is stored only at every
// c-th step (c = ceil(sqrt(l))) and each segment is recomputed from its checkpoint when reached.
#include <cmath>
#include <vector>

#include "sped_internal.cuh"

namespace sped {

constexpr int BW_MAXK = 32;
constexpr int COMBINE_MAXK = 40;  // sped_block_combine (also applies Rayleigh-Ritz rotations)

// one CTA: utilities u, Hbar for weights g (may be NULL: no Hbar), and the detached-parents
// coefficients S with du_i/dv_i = sum_j y_j S[j][i] (parents v_j, j < i, held fixed)
__global__ void k_eg_util(int k, const double *__restrict__ H, int ldh,
                          const double *__restrict__ g, double *u, double *Hbar, double *S) {
    const int i = threadIdx.x;
    if (i < k) {
        double ui = H[i * ldh + i];
        for (int j = 0; j < i; ++j) ui -= H[i * ldh + j] * H[i * ldh + j] / H[j * ldh + j];
        if (u) u[i] = ui;
        if (S) {
            for (int j = 0; j < k; ++j) S[j * k + i] = 0.0;
            S[i * k + i] = 2.0;
            for (int j = 0; j < i; ++j) S[j * k + i] = -2.0 * H[i * ldh + j] / H[j * ldh + j];
        }
    }
    // Hbar: row a below the diagonal holds -2 g_a h_aj / h_jj (one term each); the diagonal
    // entry j is g_j plus the terms g_a h_aj^2 / h_jj^2 of the rows a > j, added in increasing a;
    // above the diagonal zeros. Thread i writes row i and diagonal entry i.
    if (i < k && Hbar && g) {
        for (int j = 0; j < k; ++j) {
            if (j < i) {
                const double hij = H[i * ldh + j], hjj = H[j * ldh + j];
                Hbar[i * k + j] = 0.0 + -2.0 * g[i] * hij / hjj;
            } else if (j > i) {
                Hbar[i * k + j] = 0.0;
            }
        }
        const double hii = H[i * ldh + i];
        double d = 0.0 + g[i];
        for (int a = i + 1; a < k; ++a) {
            const double hai = H[a * ldh + i];
            d += g[a] * hai * hai / (hii * hii);
        }
        Hbar[i * k + i] = d;
    }
}

// Out = A P (+ B Q), P, Q k x k row-major FP64 (Out[r][i] = sum_j A[r][j] P[j][i] + ...), one
// row per thread, in the block's own precision (FP64 blocks: FP64; F32 blocks: F32 with the
// coefficients rounded once), the row and the coefficients unrolled to KM >= k columns.
template <typename T, int KM>
__global__ void __launch_bounds__(256)
k_combine(int64_t n, int k, const T *__restrict__ A, int lda, const double *__restrict__ P,
          const T *__restrict__ B, int ldb, const double *__restrict__ Q, T *__restrict__ Out,
          int ldo) {
    using Acc = typename AccOf<T>::type;
    __shared__ Acc sP[KM * KM], sQ[KM * KM];
    for (int e = threadIdx.x; e < KM * KM; e += blockDim.x) {
        const int j = e / KM, i = e % KM;
        const bool in = i < k && j < k;
        sP[e] = in ? (Acc)P[j * k + i] : Acc(0);
        sQ[e] = in && Q ? (Acc)Q[j * k + i] : Acc(0);
    }
    __syncthreads();
    const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    Acc a[KM], b[KM];
#pragma unroll
    for (int j = 0; j < KM; ++j) {
        a[j] = j < k ? cvt<Acc>(A[r * lda + j]) : Acc(0);
        b[j] = (B && j < k) ? cvt<Acc>(B[r * ldb + j]) : Acc(0);
    }
#pragma unroll
    for (int i = 0; i < KM; ++i) {
        if (i >= k) break;
        Acc s = Acc(0);
#pragma unroll
        for (int j = 0; j < KM; ++j) s += a[j] * sP[j * KM + i] + b[j] * sQ[j * KM + i];
        Out[r * ldo + i] = from_acc<T>(s);
    }
}

// grad[e] += scale * (A[a] - A[b]) . (C[a] - C[b]) for every undirected edge e = (a, b); the
// k-term dot in the blocks' precision (terms added in column order), the accumulation into grad
// in FP64. The four rows arrive as 16-byte chunks (the blocks' rows are padded to 16 bytes), so
// an edge costs 4 ceil(k / E) loads rather than 4 k scalar ones.
template <typename T, int KM>
__global__ void __launch_bounds__(256)
k_sddmm(int64_t n_edges, const int32_t *__restrict__ edge_a, const int32_t *__restrict__ edge_p,
        const int32_t *__restrict__ ci, int k, const T *__restrict__ A, const T *__restrict__ C,
        int ld, double scale, double *__restrict__ grad) {
    using Acc = typename AccOf<T>::type;
    constexpr int E = 16 / (int)sizeof(T);
    const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n_edges) return;
    const int a = __ldg(edge_a + e), b = __ldg(ci + __ldg(edge_p + e));
    const uint4 *Aa = reinterpret_cast<const uint4 *>(A + (int64_t)a * ld);
    const uint4 *Ab = reinterpret_cast<const uint4 *>(A + (int64_t)b * ld);
    const uint4 *Ca = reinterpret_cast<const uint4 *>(C + (int64_t)a * ld);
    const uint4 *Cb = reinterpret_cast<const uint4 *>(C + (int64_t)b * ld);
    Acc s = Acc(0);
#pragma unroll
    for (int q = 0; q < KM / E; ++q) {
        if (q * E < k) {
            union { uint4 v; T x[E]; } aa, ab, ca, cb;
            aa.v = __ldg(Aa + q);
            ab.v = __ldg(Ab + q);
            ca.v = __ldg(Ca + q);
            cb.v = __ldg(Cb + q);
#pragma unroll
            for (int u = 0; u < E; ++u) {
                if (q * E + u < k) {
                    const Acc da = cvt<Acc>(aa.x[u]) - cvt<Acc>(ab.x[u]);
                    const Acc dc = cvt<Acc>(ca.x[u]) - cvt<Acc>(cb.x[u]);
                    s += da * dc;
                }
            }
        }
    }
    grad[e] += scale * (double)s;
}

template <typename T>
static void launch_combine(int64_t n, int k, const T *A, int lda, const double *P, const T *B,
                           int ldb, const double *Q, T *Out, int ldo, cudaStream_t st) {
    const unsigned nb = (unsigned)((n + 255) / 256);
    if (k <= 8) k_combine<T, 8><<<nb, 256, 0, st>>>(n, k, A, lda, P, B, ldb, Q, Out, ldo);
    else if (k <= 16) k_combine<T, 16><<<nb, 256, 0, st>>>(n, k, A, lda, P, B, ldb, Q, Out, ldo);
    else if (k <= 32) k_combine<T, 32><<<nb, 256, 0, st>>>(n, k, A, lda, P, B, ldb, Q, Out, ldo);
    else k_combine<T, 40><<<nb, 256, 0, st>>>(n, k, A, lda, P, B, ldb, Q, Out, ldo);
}

template <typename T>
static void launch_sddmm(const sped_graph *g, int k, const T *A, const T *C, int ld, double scale,
                         double *grad, cudaStream_t st) {
    const unsigned eb = (unsigned)((g->n_edges + 255) / 256);
    if (k <= 8) k_sddmm<T, 8><<<eb, 256, 0, st>>>(g->n_edges, g->edge_a, g->edge_p, g->ci, k, A, C, ld, scale, grad);
    else if (k <= 16) k_sddmm<T, 16><<<eb, 256, 0, st>>>(g->n_edges, g->edge_a, g->edge_p, g->ci, k, A, C, ld, scale, grad);
    else k_sddmm<T, 32><<<eb, 256, 0, st>>>(g->n_edges, g->edge_a, g->edge_p, g->ci, k, A, C, ld, scale, grad);
}

static int ckpt_stride(int ell) {
    int c = (int)std::ceil(std::sqrt((double)ell));
    return c < 1 ? 1 : c;
}

struct EdgeGradLayout {
    int c, nck, ld;
    size_t block, total;
};

static EdgeGradLayout eg_layout(const sped_graph *g, int k, sped_dtype t) {
    EdgeGradLayout L;
    const int ell = g->poly.ell;
    L.c = ckpt_stride(ell);
    L.nck = (ell + L.c - 1) / L.c;
    L.ld = padded_ld(k, t);
    L.block = align_up((size_t)g->n * L.ld * dtype_size(t), 256);
    ScratchPlan p;
    p.add(L.block * (size_t)(L.nck + L.c + 2));
    p.add(poly_step_scratch(g, k, t, 0));
    L.total = p.total();
    return L;
}

template <typename T>
static sped_status run_edge_grad(const sped_graph *g, const T *V, int ldv, int k,
                                 const double *Hbar_T, double *grad, char *base, size_t bytes,
                                 cudaStream_t st, sped_dtype t) {
    const EdgeGradLayout L = eg_layout(g, k, t);
    const int ell = g->poly.ell;
    const double s = g->poly.s;
    auto blk = [&](int i) { return (T *)(base + L.block * (size_t)i); };
    T *ck0 = blk(0);                      // checkpoints C_{j c}, j < nck
    T *seg0 = blk(L.nck);                 // segment buffers, c of them
    T *Aa = blk(L.nck + L.c), *Ab = blk(L.nck + L.c + 1);
    Scratch step_scr(base + L.block * (size_t)(L.nck + L.c + 2),
                     bytes - L.block * (size_t)(L.nck + L.c + 2));
    auto step = [&](const T *X, T *Y) {
        step_scr.used = 0;
        return launch_poly_step(g, k, X, t, L.ld, nullptr, t, L.ld, Y, t, L.ld, 0.0, -s, 1.0, 0,
                                step_scr, st);
    };
    // C_0 = V Hbar^T into checkpoint 0, then the forward C chain keeping every c-th block
    launch_combine<T>(g->n, k, V, ldv, Hbar_T, nullptr, 0, nullptr, ck0, L.ld, st);
    SPED_CHECK_LAUNCH("k_combine");
    for (int j = 1; j < L.nck; ++j) {
        const T *src = blk(j - 1);
        T *cur = seg0, *nxt = blk(L.nck + 1);
        for (int m = 1; m <= L.c; ++m) {
            T *dst = (m == L.c) ? blk(j) : (m % 2 ? cur : nxt);
            SPED_TRY(step(src, dst));
            src = dst;
        }
    }
    // A_0 = V (copied into the padded layout by a combine with the identity)
    std::vector<double> eye(k * k, 0.0);
    for (int i = 0; i < k; ++i) eye[i * k + i] = 1.0;
    double *d_eye = (double *)step_scr.take(sizeof(double) * k * k);
    if (!d_eye) return fail(SPED_ERR_SCRATCH, "edge_grad: scratch too small");
    SPED_CUDA(cudaMemcpyAsync(d_eye, eye.data(), sizeof(double) * k * k, cudaMemcpyHostToDevice, st));
    launch_combine<T>(g->n, k, V, ldv, d_eye, nullptr, 0, nullptr, Aa, L.ld, st);
    SPED_CHECK_LAUNCH("k_combine");
    const size_t keep = step_scr.used;
    auto step2 = [&](const T *X, T *Y) {
        step_scr.used = keep;
        return launch_poly_step(g, k, X, t, L.ld, nullptr, t, L.ld, Y, t, L.ld, 0.0, -s, 1.0, 0,
                                step_scr, st);
    };
    SPED_CUDA(cudaMemsetAsync(grad, 0, sizeof(double) * g->n_edges, st));
    int t_cur = 0;
    T *A = Aa, *Anext = Ab;
    for (int j = L.nck - 1; j >= 0; --j) {
        const int len = (ell - j * L.c) < L.c ? (ell - j * L.c) : L.c;
        // segment: seg[m] = C_{j c + m}, seg[0] = checkpoint j
        SPED_CUDA(cudaMemcpyAsync(seg0, blk(j), (size_t)g->n * L.ld * sizeof(T),
                                  cudaMemcpyDeviceToDevice, st));
        for (int m = 1; m < len; ++m) SPED_TRY(step2(blk(L.nck + m - 1), blk(L.nck + m)));
        for (int m = len - 1; m >= 0; --m) {
            // u = j c + m pairs with t = l - 1 - u (t runs forward)
            if (g->n_edges > 0) launch_sddmm<T>(g, k, A, blk(L.nck + m), L.ld, -s, grad, st);
            SPED_CHECK_LAUNCH("k_sddmm");
            if (t_cur + 1 < ell) {
                SPED_TRY(step2(A, Anext));
                T *tmp = A;
                A = Anext;
                Anext = tmp;
            }
            ++t_cur;
        }
    }
    return SPED_OK;
}

}  // namespace sped

using namespace sped;

extern "C" {

sped_status sped_eg_utilities(int k, const double *d_H, int ldh, const double *d_g, double *d_u,
                              double *d_Hbar, double *d_S, void *stream) {
    if (k < 1 || k > BW_MAXK || !d_H || ldh < k)
        return fail(SPED_ERR_INVALID_ARG, "eg_utilities: k in 1..%d and H (ldh >= k) required",
                    BW_MAXK);
    if (d_Hbar && !d_g) return fail(SPED_ERR_INVALID_ARG, "eg_utilities: Hbar needs g");
    k_eg_util<<<1, BW_MAXK, 0, as_stream(stream)>>>(k, d_H, ldh, d_g, d_u, d_Hbar, d_S);
    SPED_CHECK_LAUNCH("k_eg_util");
    return SPED_OK;
}

sped_status sped_block_combine(int64_t n, int k, const void *d_A, int lda, const double *d_P,
                               const void *d_B, int ldb, const double *d_Q, void *d_Out, int ldo,
                               sped_dtype t, void *stream) {
    if (n < 0 || k < 1 || k > COMBINE_MAXK || !d_A || !d_P || !d_Out || lda < k || ldo < k ||
        (d_B && (!d_Q || ldb < k)))
        return fail(SPED_ERR_INVALID_ARG, "block_combine: bad arguments");
    if (t != SPED_F32 && t != SPED_F64) return fail(SPED_ERR_UNSUPPORTED, "block_combine: F32/F64");
    if (n == 0) return SPED_OK;
    if (t == SPED_F64)
        launch_combine<double>(n, k, (const double *)d_A, lda, d_P, (const double *)d_B, ldb, d_Q,
                               (double *)d_Out, ldo, as_stream(stream));
    else
        launch_combine<float>(n, k, (const float *)d_A, lda, d_P, (const float *)d_B, ldb, d_Q,
                              (float *)d_Out, ldo, as_stream(stream));
    SPED_CHECK_LAUNCH("k_combine");
    return SPED_OK;
}

sped_status sped_edge_grad_scratch_size(const sped_graph *g, int k, sped_dtype v_t,
                                        size_t *bytes) {
    if (!g || !bytes || k < 1 || k > BW_MAXK || (v_t != SPED_F32 && v_t != SPED_F64))
        return fail(SPED_ERR_INVALID_ARG, "edge_grad_scratch_size: bad arguments");
    *bytes = eg_layout(g, k, v_t).total + 256 + sizeof(double) * k * k;
    return SPED_OK;
}

sped_status sped_edge_grad(const sped_graph *g, const void *d_V, sped_dtype v_t, int k, int ld,
                           const double *d_HbarT, double *d_grad, void *d_scratch,
                           size_t scratch_bytes, void *stream) {
    if (!g || !d_HbarT || !d_grad) return fail(SPED_ERR_INVALID_ARG, "edge_grad: null");
    if (g->poly.kind != SPED_POLY_LIMIT_EXP)
        return fail(SPED_ERR_UNSUPPORTED, "edge_grad: the limit form (I - sL)^l only");
    if (k < 1 || k > BW_MAXK || (v_t != SPED_F32 && v_t != SPED_F64))
        return fail(SPED_ERR_UNSUPPORTED, "edge_grad: k <= %d, V F32 or F64", BW_MAXK);
    SPED_TRY(check_layout(d_V, v_t, k, ld, "edge_grad V"));
    size_t need = 0;
    SPED_TRY(sped_edge_grad_scratch_size(g, k, v_t, &need));
    if (!d_scratch || scratch_bytes < need || ((uintptr_t)d_scratch) % 256)
        return fail(SPED_ERR_SCRATCH, "edge_grad: scratch needs %zu bytes", need);
    cudaStream_t st = as_stream(stream);
    if (v_t == SPED_F64)
        return run_edge_grad<double>(g, (const double *)d_V, ld, k, d_HbarT, d_grad,
                                     (char *)d_scratch, scratch_bytes, st, v_t);
    return run_edge_grad<float>(g, (const float *)d_V, ld, k, d_HbarT, d_grad, (char *)d_scratch,
                                scratch_bytes, st, v_t);
}

}  // extern "C"
