// Bottom-k solver step on the dilated operator M = p(L) (Section 4), reversed per Eq. reveig
// so that the wanted eigenvectors are the top-k of M, with the two solvers of Section 5.1:
//  * mu-EG (EigenGame Unloaded, cited there): per player i, with y = M v,
//      delta_i = y_i - sum_{j<i} <v_i, y_j> v_j,  r_i = delta_i - <v_i, delta_i> v_i,
//      v_i <- (v_i + eta r_i) / ||v_i + eta r_i||;
//  * Oja (block form): V <- (V + eta Y) R^{-1}, R the Cholesky factor of the Gram of V + eta Y.
// Every inner product comes from the Gram [V Y]^T [V Y], so the N x k work is one Gram pass and
// one update pass V <- (V A + Y B) diag(s); the k x k algebra runs in FP64 on one CTA.
#include <cmath>
#include <cstddef>
#include <cstring>

#include "sped_internal.cuh"

namespace sped {

constexpr int SMALL_THREADS = 128;
constexpr int MAXK = 32;

enum : int { SOLVE_ERR_NOT_PD = 1, SOLVE_ERR_NAN = 2 };

struct Coefs {
    double A[MAXK * MAXK];  // A[j*MAXK + i]: coefficient of v_j in the new v_i
    double B[MAXK * MAXK];  // B[j*MAXK + i]: coefficient of y_j in the new v_i
    double C[MAXK * MAXK];  // C = (V^T V)^{-1} V^T Y: projection of Y onto span(V)
    double scale[MAXK];
    double ynorm[MAXK];     // ||y_i||
    double dv2[MAXK];       // sum over rows of (v_new_i - v_i)^2 (filled by the update)
    double res2[MAXK];      // sum over rows of ((I - P_V) y_i)^2 (filled by the update)
    int err;
};

// Upper Cholesky factor R (R^T R = M) of a k x k matrix given by an accessor, in shared memory;
// sets *bad when a pivot is not positive. All threads of the block take part.
template <typename F>
__device__ void chol_upper(F Mf, double *R, int k, int *bad) {
    for (int j = 0; j < k; ++j) {
        if (threadIdx.x == 0) {
            double d = Mf(j, j);
            for (int p = 0; p < j; ++p) d -= R[p * MAXK + j] * R[p * MAXK + j];
            if (!(d > 0.0) || !isfinite(d)) {
                *bad = 1;
                d = 1.0;
            }
            R[j * MAXK + j] = sqrt(d);
        }
        __syncthreads();
        for (int i = j + 1 + threadIdx.x; i < k; i += blockDim.x) {
            double s = Mf(j, i);
            for (int p = 0; p < j; ++p) s -= R[p * MAXK + j] * R[p * MAXK + i];
            R[j * MAXK + i] = s / R[j * MAXK + j];
        }
        __syncthreads();
    }
}

// k x k stage. G is (2k x 2k): [P H; H^T Q] with P = V^T V, H = V^T Y, Q = Y^T Y.
__global__ void __launch_bounds__(SMALL_THREADS)
k_small(const double *__restrict__ G, int k, double eta, int solver, Coefs *cf, double *stats) {
    __shared__ double sG[2 * MAXK * 2 * MAXK];
    __shared__ double R[MAXK * MAXK];
    __shared__ int bad, badp;
    const int K2 = 2 * k;
    const int t = threadIdx.x;
    for (int e = t; e < K2 * K2; e += blockDim.x) sG[e] = G[e];
    if (t == 0) {
        bad = 0;
        badp = 0;
    }
    for (int e = t; e < MAXK * MAXK; e += blockDim.x) {
        cf->A[e] = 0.0;
        cf->B[e] = 0.0;
        cf->C[e] = 0.0;
        R[e] = 0.0;
    }
    if (t < MAXK) {
        cf->dv2[t] = 0.0;
        cf->res2[t] = 0.0;
        cf->scale[t] = 1.0;
        cf->ynorm[t] = 1.0;
    }
    __syncthreads();
    auto P = [&](int i, int j) { return sG[i * K2 + j]; };
    auto H = [&](int i, int j) { return sG[i * K2 + k + j]; };          // <v_i, y_j>
    auto Q = [&](int i, int j) { return sG[(k + i) * K2 + k + j]; };    // <y_i, y_j>
    if (t < k) {
        if (stats) stats[t] = H(t, t) / P(t, t);  // Rayleigh quotient of M
        cf->ynorm[t] = sqrt(Q(t, t));
    }
    // projection coefficients C = P^{-1} H (for the invariant-subspace residual)
    chol_upper(P, R, k, &badp);
    if (t < k && !badp) {
        double z[MAXK];
        for (int j = 0; j < k; ++j) {  // R^T z = H(:, t)
            double s = H(j, t);
            for (int p = 0; p < j; ++p) s -= R[p * MAXK + j] * z[p];
            z[j] = s / R[j * MAXK + j];
        }
        for (int j = k - 1; j >= 0; --j) {  // R c = z
            double s = z[j];
            for (int p = j + 1; p < k; ++p) s -= R[j * MAXK + p] * z[p];
            z[j] = s / R[j * MAXK + j];
        }
        for (int j = 0; j < k; ++j) cf->C[j * MAXK + t] = z[j];
    }
    __syncthreads();
    if (solver == SPED_SOLVER_MU_EG) {
        if (t < k) {
            const int i = t;
            double c = H(i, i);
            for (int j = 0; j < i; ++j) c -= H(i, j) * P(i, j);
            // u_i = sum_j a_j v_j + eta y_i with a_j = -eta H(i,j) (j<i), a_i = 1 - eta c
            double a[MAXK];
            for (int j = 0; j < k; ++j) a[j] = 0.0;
            for (int j = 0; j < i; ++j) a[j] = -eta * H(i, j);
            a[i] = 1.0 - eta * c;
            double nrm = eta * eta * Q(i, i);
            for (int j = 0; j <= i; ++j) {
                double s = 0.0;
                for (int l = 0; l <= i; ++l) s += a[l] * P(j, l);
                nrm += a[j] * s + 2.0 * eta * a[j] * H(j, i);
            }
            for (int j = 0; j <= i; ++j) cf->A[j * MAXK + i] = a[j];
            cf->B[i * MAXK + i] = eta;
            if (!(nrm > 0.0) || !isfinite(nrm)) {
                atomicOr(&cf->err, SOLVE_ERR_NAN);
                cf->scale[i] = 0.0;
            } else {
                cf->scale[i] = 1.0 / sqrt(nrm);
            }
        }
        return;
    }
    // Oja: W = V + eta Y (eta <= 0: W = Y), Cholesky R^T R = W^T W, V <- W R^{-1}
    const bool pure = !(eta > 0.0);
    auto Mw = [&](int i, int j) {
        return pure ? Q(i, j) : P(i, j) + eta * (H(i, j) + H(j, i)) + eta * eta * Q(i, j);
    };
    for (int e = t; e < MAXK * MAXK; e += blockDim.x) R[e] = 0.0;
    __syncthreads();
    chol_upper(Mw, R, k, &bad);
    if (t < k) {
        // column t of R^{-1} by back substitution
        const int i = t;
        double x[MAXK];
        for (int j = 0; j < k; ++j) x[j] = 0.0;
        x[i] = 1.0 / R[i * MAXK + i];
        for (int j = i - 1; j >= 0; --j) {
            double s = 0.0;
            for (int p = j + 1; p <= i; ++p) s += R[j * MAXK + p] * x[p];
            x[j] = -s / R[j * MAXK + j];
        }
        for (int j = 0; j <= i; ++j) {
            cf->A[j * MAXK + i] = pure ? 0.0 : x[j];
            cf->B[j * MAXK + i] = pure ? x[j] : eta * x[j];
        }
        cf->scale[i] = 1.0;
    }
    if (t == 0 && bad) atomicOr(&cf->err, SOLVE_ERR_NOT_PD);
}

// V <- (V A + Y B) diag(scale), in place, one row per thread. The coefficient matrices sit in
// shared memory as [j][i] with i contiguous, so one 16-byte shared load feeds four outputs;
// B is diagonal for mu-EG (bdiag), which skips its k^2 products. The row is held in registers,
// so each group of four outputs is stored as soon as it is computed. Accumulates, per column,
// ||v_new_i - v_i||^2 and the invariant-subspace residual ||y_i - V C_i||^2 (old V).
template <typename Tm, typename Ty, int KM>
__global__ void __launch_bounds__(256)
k_update(int64_t n, Tm *__restrict__ V, int ldv, const Ty *__restrict__ Y, int ldy, int k,
         Coefs *cf, int bdiag) {
    using A = typename AccOf<Tm>::type;
    static_assert(KM % 4 == 0, "KM");
    __shared__ __align__(16) A sA[KM * KM];
    __shared__ __align__(16) A sB[KM * KM];
    __shared__ __align__(16) A sC[KM * KM];
    __shared__ A sS[KM];
    __shared__ double sdv[KM], sres[KM];
    for (int e = threadIdx.x; e < KM * KM; e += blockDim.x) {
        const int j = e / KM, i = e % KM;
        const bool in = i < k && j < k;
        sA[e] = in ? (A)cf->A[j * MAXK + i] : A(0);
        sB[e] = in ? (A)cf->B[j * MAXK + i] : A(0);
        sC[e] = in ? (A)cf->C[j * MAXK + i] : A(0);
    }
    for (int e = threadIdx.x; e < KM; e += blockDim.x) {
        sS[e] = e < k ? (A)cf->scale[e] : A(0);
        sdv[e] = 0.0;
        sres[e] = 0.0;
    }
    __syncthreads();
    A dv[KM], rs[KM];
#pragma unroll
    for (int i = 0; i < KM; ++i) {
        dv[i] = A(0);
        rs[i] = A(0);
    }
    for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n;
         r += (int64_t)gridDim.x * blockDim.x) {
        Tm *vr = V + r * ldv;
        const Ty *yr = Y + r * ldy;
        A v[KM], y[KM];
#pragma unroll
        for (int j = 0; j < KM; ++j) {
            v[j] = j < k ? cvt<A>(vr[j]) : A(0);
            y[j] = j < k ? cvt<A>(__ldg(yr + j)) : A(0);
        }
#pragma unroll
        for (int i0 = 0; i0 < KM; i0 += 4) {
            if (i0 >= k) break;
            A s[4] = {A(0), A(0), A(0), A(0)}, pq[4] = {A(0), A(0), A(0), A(0)};
#pragma unroll
            for (int j = 0; j < KM; ++j) {
                const A *a4 = sA + j * KM + i0, *c4 = sC + j * KM + i0;
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    s[q] += v[j] * a4[q];
                    pq[q] += v[j] * c4[q];
                }
                if (!bdiag) {
                    const A *b4 = sB + j * KM + i0;
#pragma unroll
                    for (int q = 0; q < 4; ++q) s[q] += y[j] * b4[q];
                }
            }
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int i = i0 + q;
                if (bdiag) s[q] += y[i] * sB[i * KM + i];
                s[q] *= sS[i];
                const A d = s[q] - v[i];
                dv[i] += d * d;
                const A e = y[i] - pq[q];
                rs[i] += e * e;
                if (i < k) vr[i] = from_acc<Tm>(s[q]);
            }
        }
    }
    // column sums: warp shuffle, then shared, then one atomic per block and column
#pragma unroll
    for (int i = 0; i < KM; ++i) {
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

__global__ void k_finish_stats(int k, const Coefs *cf, double *stats) {
    int i = threadIdx.x;
    if (i < k && stats) {
        double yn = cf->ynorm[i];
        stats[k + i] = yn > 0.0 ? sqrt(cf->res2[i]) / yn : INFINITY;
        stats[2 * k + i] = sqrt(cf->dv2[i]);
    }
}

__global__ void k_rayleigh_out(const double *G, int k, double *out) {
    int i = threadIdx.x;
    if (i < k) out[i] = G[i * 2 * k + k + i] / G[i * 2 * k + i];
}

template <typename Tm, typename Ty>
static sped_status run_update(int64_t n, void *V, int ldv, const void *Y, int ldy, int k,
                              Coefs *cf, int bdiag, cudaStream_t st) {
    int blocks = device_sm_count() * 4;
    const int64_t need = (n + 255) / 256;
    if (need < blocks) blocks = (int)(need > 0 ? need : 1);
#define UPD(KMV) k_update<Tm, Ty, KMV><<<blocks, 256, 0, st>>>(n, (Tm *)V, ldv, (const Ty *)Y, ldy, k, cf, bdiag)
    if (k <= 8) UPD(8);
    else if (k <= 16) UPD(16);
    else if (k <= 20) UPD(20);
    else if (k <= 24) UPD(24);
    else UPD(32);
#undef UPD
    SPED_CHECK_LAUNCH("k_update");
    return SPED_OK;
}

struct StepLayout {
    size_t y, G, coefs, shared;
    int ldy;
    size_t total;
};

static StepLayout step_layout(const sped_graph *g, const sped_step_opts *o, int k) {
    StepLayout L;
    ScratchPlan p;
    L.ldy = padded_ld(k, o->y_t);
    L.y = p.used = align_up(p.used, 256);
    p.add((size_t)g->n * L.ldy * dtype_size(o->y_t));
    p.used = align_up(p.used, 256);
    L.G = p.used;
    p.add(sizeof(double) * 4 * k * k);
    p.used = align_up(p.used, 256);
    L.coefs = p.used;
    p.add(sizeof(Coefs));
    p.used = align_up(p.used, 256);
    L.shared = p.used;
    size_t a = apply_poly_scratch(g, k, o->chain_t, o->mode);
    size_t b = gram_scratch(g->n, k, k);
    p.add(a > b ? a : b);
    L.total = p.total();
    return L;
}

static sped_status check_opts(const sped_step_opts *o) {
    if (!o) return fail(SPED_ERR_INVALID_ARG, "step opts NULL");
    if (o->solver != SPED_SOLVER_MU_EG && o->solver != SPED_SOLVER_OJA)
        return fail(SPED_ERR_INVALID_ARG, "solver %d", (int)o->solver);
    if (o->y_t != SPED_F32 && o->y_t != SPED_F64)
        return fail(SPED_ERR_INVALID_ARG, "Y = M V must be stored as F32 or F64");
    if (!dtype_valid(o->chain_t)) return fail(SPED_ERR_INVALID_ARG, "chain dtype");
    if (!std::isfinite(o->eta)) return fail(SPED_ERR_INVALID_ARG, "eta not finite");
    if (o->solver == SPED_SOLVER_MU_EG && !(o->eta > 0.0))
        return fail(SPED_ERR_INVALID_ARG, "mu-EG needs eta > 0");
    return SPED_OK;
}

static sped_status eig_step_impl(const sped_graph *g, const sped_step_opts *o, void *V,
                                 sped_dtype vt, int k, int ld, double *d_stats, void *scr_p,
                                 size_t scr_bytes, cudaStream_t st, Coefs **cf_out) {
    StepLayout L = step_layout(g, o, k);
    if (!scr_p || scr_bytes < L.total || ((uintptr_t)scr_p) % 256)
        return fail(SPED_ERR_SCRATCH, "eig_step: scratch needs %zu bytes (256-aligned)", L.total);
    char *base = (char *)scr_p;
    void *Y = base + L.y;
    double *G = (double *)(base + L.G);
    Coefs *cf = (Coefs *)(base + L.coefs);
    Scratch shared(base + L.shared, scr_bytes - L.shared);
    if (o->ev_chain_begin) SPED_CUDA(cudaEventRecord((cudaEvent_t)o->ev_chain_begin, st));
    SPED_TRY(apply_poly_impl(g, k, V, vt, ld, Y, o->y_t, L.ldy, o->chain_t, o->mode, o->walkers,
                             o->seed, shared, st));
    if (o->ev_chain_end) SPED_CUDA(cudaEventRecord((cudaEvent_t)o->ev_chain_end, st));
    shared.used = 0;
    SPED_TRY(launch_gram(g->n, V, vt, ld, k, Y, o->y_t, L.ldy, k, G, shared, st));
    SPED_CUDA(cudaMemsetAsync(&cf->err, 0, sizeof(int), st));
    k_small<<<1, SMALL_THREADS, 0, st>>>(G, k, o->eta, (int)o->solver, cf, d_stats);
    SPED_CHECK_LAUNCH("k_small");
    const int bdiag = o->solver == SPED_SOLVER_MU_EG;  // mu-EG: Y enters through eta I
    if (vt == SPED_F32 && o->y_t == SPED_F32) SPED_TRY((run_update<float, float>(g->n, V, ld, Y, L.ldy, k, cf, bdiag, st)));
    else if (vt == SPED_F32 && o->y_t == SPED_F64) SPED_TRY((run_update<float, double>(g->n, V, ld, Y, L.ldy, k, cf, bdiag, st)));
    else if (vt == SPED_F64 && o->y_t == SPED_F64) SPED_TRY((run_update<double, double>(g->n, V, ld, Y, L.ldy, k, cf, bdiag, st)));
    else if (vt == SPED_F64 && o->y_t == SPED_F32) SPED_TRY((run_update<double, float>(g->n, V, ld, Y, L.ldy, k, cf, bdiag, st)));
    else return fail(SPED_ERR_UNSUPPORTED, "eig_step: master V must be F32 or F64");
    if (d_stats) {
        k_finish_stats<<<1, MAXK, 0, st>>>(k, cf, d_stats);
        SPED_CHECK_LAUNCH("k_finish_stats");
    }
    if (cf_out) *cf_out = cf;
    return SPED_OK;
}

static int poly_spmm_count(const sped_graph *g, sped_mode mode) {
    if (mode != SPED_EXACT) return 0;
    const Poly &P = g->poly;
    return P.kind == SPED_POLY_SHIFT ? 1 : P.ell;
}

}  // namespace sped

using namespace sped;

extern "C" {

sped_status sped_eig_step_scratch_size(const sped_graph *g, const sped_step_opts *opts, int k,
                                       size_t *bytes) {
    if (!g || !bytes || k < 1 || k > MAXK) return fail(SPED_ERR_INVALID_ARG, "eig_step_scratch_size");
    SPED_TRY(check_opts(opts));
    *bytes = step_layout(g, opts, k).total;
    return SPED_OK;
}

sped_status sped_eig_step(const sped_graph *g, const sped_step_opts *opts, void *d_V,
                          sped_dtype v_t, int k, int ld, double *d_stats, void *d_scratch,
                          size_t scratch_bytes, void *stream) {
    if (!g) return fail(SPED_ERR_INVALID_ARG, "eig_step: null graph");
    if (k < 1 || k > MAXK) return fail(SPED_ERR_UNSUPPORTED, "eig_step: k=%d (1..%d)", k, MAXK);
    SPED_TRY(check_opts(opts));
    if (v_t != SPED_F32 && v_t != SPED_F64)
        return fail(SPED_ERR_INVALID_ARG, "eig_step: master V must be F32 or F64");
    SPED_TRY(check_layout(d_V, v_t, k, ld, "eig_step V"));
    return eig_step_impl(g, opts, d_V, v_t, k, ld, d_stats, d_scratch, scratch_bytes,
                         as_stream(stream), nullptr);
}

sped_status sped_rayleigh_scratch_size(const sped_graph *g, int k, size_t *bytes) {
    if (!g || !bytes || k < 1 || 2 * k > 64) return fail(SPED_ERR_INVALID_ARG, "rayleigh_scratch_size");
    ScratchPlan p;
    p.add((size_t)g->n * padded_ld(k, SPED_F64) * 8);
    p.add(sizeof(double) * 4 * k * k);
    p.add(gram_scratch(g->n, k, k));
    p.add(poly_step_scratch(g, k, SPED_F64, 0));
    *bytes = p.total();
    return SPED_OK;
}

sped_status sped_rayleigh(const sped_graph *g, const void *d_V, sped_dtype v_t, int k, int ld,
                          double *d_out, void *d_scratch, size_t scratch_bytes, void *stream) {
    if (!g || !d_out) return fail(SPED_ERR_INVALID_ARG, "rayleigh: null");
    if (k < 1 || 2 * k > 64) return fail(SPED_ERR_UNSUPPORTED, "rayleigh: k=%d", k);
    if (v_t != SPED_F32 && v_t != SPED_F64)
        return fail(SPED_ERR_UNSUPPORTED, "rayleigh: V must be F32 or F64");
    SPED_TRY(check_layout(d_V, v_t, k, ld, "rayleigh V"));
    cudaStream_t st = as_stream(stream);
    Scratch scr(d_scratch, scratch_bytes);
    int ldl = padded_ld(k, SPED_F64);
    void *LV = scr.take((size_t)g->n * ldl * 8);
    double *G = (double *)scr.take(sizeof(double) * 4 * k * k);
    if (!LV || !G) return fail(SPED_ERR_SCRATCH, "rayleigh: scratch too small");
    SPED_TRY(launch_poly_step(g, k, d_V, v_t, ld, nullptr, v_t, ld, LV, SPED_F64, ldl, 0.0, 1.0,
                              0.0, 0, scr, st));
    SPED_TRY(launch_gram(g->n, d_V, v_t, ld, k, LV, SPED_F64, ldl, k, G, scr, st));
    k_rayleigh_out<<<1, 64, 0, st>>>(G, k, d_out);
    SPED_CHECK_LAUNCH("k_rayleigh_out");
    return SPED_OK;
}

static sped_step_opts phase_opts(const sped_solve_opts *o, int phase) {
    sped_step_opts s = o->step;
    if (phase == 2) s.chain_t = o->refine_chain_t;
    return s;
}

sped_status sped_solve_scratch_size(const sped_graph *g, const sped_solve_opts *opts, int k,
                                    size_t *bytes) {
    if (!g || !opts || !bytes) return fail(SPED_ERR_INVALID_ARG, "solve_scratch_size");
    size_t a = 0, b = 0, c = 0;
    sped_step_opts s1 = phase_opts(opts, 1), s2 = phase_opts(opts, 2);
    SPED_TRY(sped_eig_step_scratch_size(g, &s1, k, &a));
    SPED_TRY(sped_eig_step_scratch_size(g, &s2, k, &b));
    SPED_TRY(sped_rayleigh_scratch_size(g, k, &c));
    size_t m = a > b ? a : b;
    m = m > c ? m : c;
    *bytes = align_up(m, 256) + 1024;  // + stats slot (3k doubles)
    return SPED_OK;
}

sped_status sped_solve_bottom_k(const sped_graph *g, const sped_solve_opts *opts, void *d_V,
                                sped_dtype v_t, int k, int ld, double *h_lambda,
                                sped_solve_report *report, void *d_scratch, size_t scratch_bytes,
                                void *stream) {
    if (!g || !opts) return fail(SPED_ERR_INVALID_ARG, "solve_bottom_k: null");
    if (opts->max_steps < 1 || opts->check_every < 1)
        return fail(SPED_ERR_INVALID_ARG, "solve_bottom_k: max_steps/check_every < 1");
    size_t need = 0;
    SPED_TRY(sped_solve_scratch_size(g, opts, k, &need));
    if (!d_scratch || scratch_bytes < need)
        return fail(SPED_ERR_SCRATCH, "solve_bottom_k: scratch needs %zu bytes", need);
    cudaStream_t st = as_stream(stream);
    char *base = (char *)d_scratch;
    size_t body = need - 1024;
    const size_t coef_off = step_layout(g, &opts->step, k).coefs;  // same for both phases
    double *d_stats = (double *)(base + body);
    double h_stats[3 * MAXK];
    sped_solve_report rep;
    memset(&rep, 0, sizeof(rep));
    int phase = 1;
    double res = INFINITY;
    for (int step = 1; step <= opts->max_steps; ++step) {
        sped_step_opts so = phase_opts(opts, phase);
        SPED_TRY(sped_eig_step(g, &so, d_V, v_t, k, ld, d_stats, d_scratch, body, stream));
        rep.steps = step;
        rep.spmm_count += poly_spmm_count(g, so.mode);
        if (phase == 1) rep.phase1_steps = step;
        if (step % opts->check_every == 0 || step == opts->max_steps) {
            SPED_CUDA(cudaMemcpyAsync(h_stats, d_stats, sizeof(double) * 3 * k,
                                      cudaMemcpyDeviceToHost, st));
            int h_err = 0;
            SPED_CUDA(cudaMemcpyAsync(&h_err, base + coef_off + offsetof(Coefs, err), sizeof(int),
                                      cudaMemcpyDeviceToHost, st));
            SPED_CUDA(cudaStreamSynchronize(st));
            if (h_err & SOLVE_ERR_NOT_PD)
                return fail(SPED_ERR_NUMERIC, "solve: Gram of V + eta Y not positive definite");
            if (h_err & SOLVE_ERR_NAN) return fail(SPED_ERR_NUMERIC, "solve: non-finite norm");
            res = 0.0;
            for (int i = 0; i < k; ++i) {
                double x = h_stats[k + i];
                if (std::isnan(x)) return fail(SPED_ERR_NUMERIC, "solve: NaN residual");
                res = x > res ? x : res;
            }
            if (phase == 1 && (res <= opts->switch_tol || step >= opts->phase1_steps) &&
                opts->refine_chain_t != opts->step.chain_t) {
                phase = 2;
            } else if (res <= opts->tol && (phase == 2 || opts->refine_chain_t == opts->step.chain_t)) {
                rep.converged = 1;
                break;
            }
        }
    }
    rep.final_residual = res;
    if (h_lambda) {
        double *d_lam = d_stats;  // reuse the stats slot (2k doubles >= k)
        SPED_TRY(sped_rayleigh(g, d_V, v_t, k, ld, d_lam, d_scratch, body, stream));
        SPED_CUDA(cudaMemcpyAsync(h_lambda, d_lam, sizeof(double) * k, cudaMemcpyDeviceToHost, st));
    }
    SPED_CUDA(cudaStreamSynchronize(st));
    if (report) *report = rep;
    if (!rep.converged)
        return fail(SPED_ERR_NOT_CONVERGED, "solve_bottom_k: %d steps, residual %.3e > tol %.3e",
                    rep.steps, rep.final_residual, opts->tol);
    return SPED_OK;
}

}  // extern "C"
