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

#include "solver_update.cuh"

namespace sped {

constexpr int SMALL_THREADS = 256;
constexpr int SLD = MAXK + 1;  // row stride of the k x k work arrays (odd: conflict-free columns)
constexpr size_t SMALL_SMEM = 5 * sizeof(double) * MAXK * SLD;
constexpr size_t RR_SMEM = 4 * sizeof(double) * MAXK * SLD;

// The k x k stage is FP64 and latency-bound on one SM, so every kernel-level step below spreads
// its products over all threads and keeps the serial chain short: one rsqrt per Cholesky pivot,
// divisions replaced by that reciprocal, one barrier per elimination step.

// Right-looking Cholesky W = R^T R of a symmetric k x k array (upper triangle read, W
// overwritten), R upper in R[j*SLD + i] (i >= j), rinv[j] = 1 / R_jj. Sets *bad on a pivot
// that is not positive (that pivot is replaced by 1 so the rest stays finite).
__device__ void chol_rl(double *W, double *R, double *rinv, int k, int *bad) {
    const int t = threadIdx.x, nt = blockDim.x;
    for (int j = 0; j < k; ++j) {
        const double d = W[j * SLD + j];
        const bool ok = d > 0.0 && isfinite(d);
        const double ri = ok ? rsqrt(d) : 1.0;
        for (int i = j + t; i < k; i += nt) R[j * SLD + i] = i == j ? (ok ? d * ri : 1.0) : W[j * SLD + i] * ri;
        if (t == 0) {
            rinv[j] = ri;
            if (!ok) *bad = 1;
        }
        const int m = k - 1 - j;
        const double ri2 = ri * ri;
        for (int e = t; e < m * m; e += nt) {
            const int i = j + 1 + e / m, l = j + 1 + e % m;
            if (l >= i) W[i * SLD + l] -= W[j * SLD + i] * W[j * SLD + l] * ri2;
        }
        __syncthreads();
    }
}

// Forward substitution R^T Z = B for nrhs right-hand sides (B[j*SLD + c]); B is consumed.
__device__ void trsv_upper_t(const double *R, const double *rinv, double *B, double *Z, int k,
                             int nrhs) {
    const int t = threadIdx.x, nt = blockDim.x;
    for (int j = 0; j < k; ++j) {
        const double ri = rinv[j];
        for (int c = t; c < nrhs; c += nt) Z[j * SLD + c] = B[j * SLD + c] * ri;
        const int m = k - 1 - j;
        for (int e = t; e < m * nrhs; e += nt) {
            const int i = j + 1 + e / nrhs, c = e % nrhs;
            B[i * SLD + c] -= R[j * SLD + i] * (B[j * SLD + c] * ri);
        }
        __syncthreads();
    }
}

// Back substitution R X = Z (Z consumed), X[j*SLD + c].
__device__ void trsv_upper(const double *R, const double *rinv, double *Z, double *X, int k,
                           int nrhs) {
    const int t = threadIdx.x, nt = blockDim.x;
    for (int j = k - 1; j >= 0; --j) {
        const double ri = rinv[j];
        for (int c = t; c < nrhs; c += nt) X[j * SLD + c] = Z[j * SLD + c] * ri;
        for (int e = t; e < j * nrhs; e += nt) {
            const int i = e / nrhs, c = e % nrhs;
            Z[i * SLD + c] -= R[i * SLD + j] * (Z[j * SLD + c] * ri);
        }
        __syncthreads();
    }
}

// k x k stage. G is (2k x 2k): [P H; H^T Q] with P = V^T V, H = V^T Y, Q = Y^T Y.
__global__ void __launch_bounds__(SMALL_THREADS)
k_small(const double *__restrict__ G, int k, double eta, int solver, Coefs *cf, double *stats) {
    // five k x k work arrays (SMALL_SMEM bytes of dynamic shared memory)
    extern __shared__ __align__(16) double small_smem[];
    double *sP = small_smem, *sH = sP + MAXK * SLD, *sW = sH + MAXK * SLD, *sR = sW + MAXK * SLD,
           *sB = sR + MAXK * SLD;
    __shared__ double rinv[MAXK], cmu[MAXK];
    pdl_wait();  // launched with programmatic dependent launch: G comes from the kernel before
    __shared__ int bad, badp;
    const int K2 = 2 * k;
    const int t = threadIdx.x, nt = blockDim.x;
    for (int e = t; e < k * k; e += nt) {
        const int i = e / k, j = e % k;
        sP[i * SLD + j] = G[i * K2 + j];
        sH[i * SLD + j] = G[i * K2 + k + j];  // <v_i, y_j>
    }
    if (t == 0) {
        bad = 0;
        badp = 0;
    }
    for (int e = t; e < MAXK * MAXK; e += nt) {
        cf->A[e] = 0.0;
        cf->B[e] = 0.0;
        cf->C[e] = 0.0;
    }
    if (t < MAXK) {
        cf->dv2[t] = 0.0;
        cf->res2[t] = 0.0;
        cf->scale[t] = 1.0;
        cf->ynorm[t] = 1.0;
    }
    __syncthreads();
    if (t < k) {
        const double q = G[(k + t) * K2 + k + t];
        if (stats) stats[t] = sH[t * SLD + t] / sP[t * SLD + t];  // Rayleigh quotient of M
        cf->ynorm[t] = sqrt(q);
    }
    if (solver == SPED_SOLVER_MU_EG) {
        // player i: u_i = sum_{j<=i} a_ij v_j + eta y_i with a_ij = -eta H_ij (j < i) and
        // a_ii = 1 - eta c_i, c_i = H_ii - sum_{j<i} H_ij P_ij; ||u_i||^2 = a_i^T P a_i +
        // 2 eta a_i^T H_{:,i} + eta^2 Q_ii. The a_i sit in sW (row i), T = a P in sB.
        if (t < k) {
            double c = sH[t * SLD + t];
            for (int j = 0; j < t; ++j) c -= sH[t * SLD + j] * sP[t * SLD + j];
            cmu[t] = c;
        }
        __syncthreads();
        for (int e = t; e < k * k; e += nt) {
            const int i = e / k, j = e % k;
            sW[i * SLD + j] = j < i ? -eta * sH[i * SLD + j] : j == i ? 1.0 - eta * cmu[i] : 0.0;
        }
        __syncthreads();
        for (int e = t; e < k * k; e += nt) {
            const int i = e / k, j = e % k;
            if (j <= i) {
                double s = 0.0;
                for (int l = 0; l <= i; ++l) s += sW[i * SLD + l] * sP[j * SLD + l];
                sB[i * SLD + j] = s;
            }
        }
        __syncthreads();
        if (t < k) {
            const int i = t;
            double nrm = eta * eta * G[(k + i) * K2 + k + i];
            for (int j = 0; j <= i; ++j)
                nrm += sW[i * SLD + j] * (sB[i * SLD + j] + 2.0 * eta * sH[j * SLD + i]);
            for (int j = 0; j <= i; ++j) cf->A[j * MAXK + i] = sW[i * SLD + j];
            cf->B[i * MAXK + i] = eta;
            if (!(nrm > 0.0) || !isfinite(nrm)) {
                atomicOr(&cf->err, SOLVE_ERR_NAN);
                cf->scale[i] = 0.0;
            } else {
                cf->scale[i] = rsqrt(nrm);
            }
        }
        __syncthreads();
    }
    // projection coefficients C = P^{-1} H (for the invariant-subspace residual; only when the
    // caller asked for the step's statistics)
    if (stats) {
        for (int e = t; e < k * k; e += nt) {
            const int i = e / k, j = e % k;
            sW[i * SLD + j] = sP[i * SLD + j];
            sB[i * SLD + j] = sH[i * SLD + j];
        }
        __syncthreads();
        chol_rl(sW, sR, rinv, k, &badp);
    }
    if (stats && !badp) {
        trsv_upper_t(sR, rinv, sB, sW, k, k);
        trsv_upper(sR, rinv, sW, sB, k, k);
        for (int e = t; e < k * k; e += nt) {
            const int j = e / k, i = e % k;
            cf->C[j * MAXK + i] = sB[j * SLD + i];
        }
    }
    if (solver == SPED_SOLVER_MU_EG) return;
    // Oja: W = V + eta Y (eta <= 0: W = Y), Cholesky R^T R = W^T W, V <- W R^{-1}
    const bool pure = !(eta > 0.0);
    __syncthreads();
    for (int e = t; e < k * k; e += nt) {
        const int i = e / k, j = e % k;
        const double q = G[(k + i) * K2 + k + j];
        sW[i * SLD + j] = pure ? q : sP[i * SLD + j] + eta * (sH[i * SLD + j] + sH[j * SLD + i]) + eta * eta * q;
        sB[i * SLD + j] = i == j ? 1.0 : 0.0;
    }
    __syncthreads();
    chol_rl(sW, sR, rinv, k, &bad);
    trsv_upper(sR, rinv, sB, sW, k, k);  // sW = R^{-1}
    for (int e = t; e < k * k; e += nt) {
        const int j = e / k, i = e % k;
        const double x = j <= i ? sW[j * SLD + i] : 0.0;
        cf->A[j * MAXK + i] = pure ? 0.0 : x;
        cf->B[j * MAXK + i] = pure ? x : eta * x;
    }
    if (t < k) cf->scale[t] = 1.0;
    if (t == 0 && bad) atomicOr(&cf->err, SOLVE_ERR_NOT_PD);
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

// Rayleigh-Ritz on one CTA. G = [V LV]^T [V LV] (2k x 2k): P = V^T V = R^T R (Cholesky),
// Hs = R^{-T} H R^{-1} with H = V^T L V (the matrix of L in the orthonormal basis V R^{-1}),
// Hs = Z diag(theta) Z^T by cyclic Jacobi rotations, then W = R^{-1} Z so that V W are the Ritz
// vectors. Each round applies m/2 disjoint rotations at once (round-robin pairing of the m =
// k rounded up to even indices; an odd k gets an idle index whose rotations are the identity):
// the rotation angles from the 2 x 2 blocks, then all row pairs, then all column pairs (and Z).
// Sweeps stop when the off-diagonal mass is below 1e-30 of the diagonal's, or after RR_SWEEPS.
constexpr int RR_SWEEPS = 40;

__global__ void __launch_bounds__(SMALL_THREADS)
k_rayleigh_ritz(const double *__restrict__ G, int k, double *__restrict__ theta,
                double *__restrict__ W) {
    // four k x k work arrays (RR_SMEM bytes of dynamic shared memory)
    extern __shared__ __align__(16) double rr_smem[];
    double *sA = rr_smem, *sR = sA + MAXK * SLD, *sZ = sR + MAXK * SLD, *sT = sZ + MAXK * SLD;
    __shared__ double rinv[MAXK];
    __shared__ double rc[MAXK / 2], rs[MAXK / 2], red[SMALL_THREADS / 32][2];
    __shared__ int bad, perm[MAXK], done;
    const int t = threadIdx.x, nt = blockDim.x;
    const int K2 = 2 * k, m = (k + 1) & ~1;
    if (t == 0) {
        bad = 0;
        done = 0;
    }
    for (int e = t; e < MAXK * SLD; e += nt) {
        sA[e] = 0.0;
        sZ[e] = 0.0;
    }
    __syncthreads();
    for (int e = t; e < k * k; e += nt) {
        const int i = e / k, j = e % k;
        sA[i * SLD + j] = G[i * K2 + j];       // P, consumed by the factorisation
        sT[i * SLD + j] = G[i * K2 + k + j];   // H
    }
    __syncthreads();
    chol_rl(sA, sR, rinv, k, &bad);
    if (bad) {
        for (int i = t; i < k; i += nt) theta[i] = NAN;
        return;
    }
    // Hs = R^{-T} (R^{-T} H)^T, H symmetric
    trsv_upper_t(sR, rinv, sT, sA, k, k);  // sA = R^{-T} H
    for (int e = t; e < k * k; e += nt) {
        const int i = e / k, j = e % k;
        sT[j * SLD + i] = sA[i * SLD + j];
    }
    __syncthreads();
    trsv_upper_t(sR, rinv, sT, sA, k, k);  // sA = Hs
    for (int e = t; e < MAXK * SLD; e += nt) sT[e] = 0.0;
    __syncthreads();
    for (int e = t; e < k * k; e += nt) {
        const int i = e / k, j = e % k;
        if (i <= j) {
            const double v = 0.5 * (sA[i * SLD + j] + sA[j * SLD + i]);
            sT[i * SLD + j] = v;
            sT[j * SLD + i] = v;
        }
    }
    for (int i = t; i < m; i += nt) sZ[i * SLD + i] = 1.0;
    __syncthreads();
    // ---- Jacobi sweeps on sT (m x m, the idle index, if any, has zero off-diagonals)
    const int half = m / 2;
    for (int sweep = 0; sweep < RR_SWEEPS; ++sweep) {
        for (int r = 0; r < m - 1; ++r) {
            // pair i: positions i and m-1-i of the circle [0, (1..m-1 rotated by r)]
            auto player = [&](int pos) { return pos == 0 ? 0 : 1 + (pos - 1 + r) % (m - 1); };
            if (t < half) {
                int p = player(t), q = player(m - 1 - t);
                if (p > q) {
                    const int x = p;
                    p = q;
                    q = x;
                }
                const double apq = sT[p * SLD + q];
                double c = 1.0, sn = 0.0;
                if (apq != 0.0) {
                    const double tau = (sT[q * SLD + q] - sT[p * SLD + p]) / (2.0 * apq);
                    const double tt = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
                    c = rsqrt(1.0 + tt * tt);
                    sn = tt * c;
                }
                rc[t] = c;
                rs[t] = sn;
            }
            __syncthreads();
            for (int e = t; e < half * m; e += nt) {  // rows p, q <- J^T A
                const int i = e / m, j = e % m;
                int p = player(i), q = player(m - 1 - i);
                if (p > q) {
                    const int x = p;
                    p = q;
                    q = x;
                }
                const double c = rc[i], sn = rs[i];
                const double ap = sT[p * SLD + j], aq = sT[q * SLD + j];
                sT[p * SLD + j] = c * ap - sn * aq;
                sT[q * SLD + j] = sn * ap + c * aq;
            }
            __syncthreads();
            for (int e = t; e < half * m; e += nt) {  // columns p, q <- A J, and Z <- Z J
                const int i = e / m, j = e % m;
                int p = player(i), q = player(m - 1 - i);
                if (p > q) {
                    const int x = p;
                    p = q;
                    q = x;
                }
                const double c = rc[i], sn = rs[i];
                const double ap = sT[j * SLD + p], aq = sT[j * SLD + q];
                sT[j * SLD + p] = c * ap - sn * aq;
                sT[j * SLD + q] = sn * ap + c * aq;
                const double zp = sZ[j * SLD + p], zq = sZ[j * SLD + q];
                sZ[j * SLD + p] = c * zp - sn * zq;
                sZ[j * SLD + q] = sn * zp + c * zq;
            }
            __syncthreads();
        }
        // off-diagonal and diagonal mass
        double off = 0.0, dia = 0.0;
        for (int e = t; e < m * m; e += nt) {
            const int i = e / m, j = e % m;
            const double v = sT[i * SLD + j];
            if (i == j) dia += v * v;
            else off += v * v;
        }
        for (int o = 16; o > 0; o >>= 1) {
            off += __shfl_down_sync(0xffffffffu, off, o);
            dia += __shfl_down_sync(0xffffffffu, dia, o);
        }
        if ((t & 31) == 0) {
            red[t >> 5][0] = off;
            red[t >> 5][1] = dia;
        }
        __syncthreads();
        if (t == 0) {
            double o2 = 0.0, d2 = 0.0;
            for (int w = 0; w < nt / 32; ++w) {
                o2 += red[w][0];
                d2 += red[w][1];
            }
            done = !(o2 > 1e-30 * d2);
        }
        __syncthreads();
        if (done) break;
    }
    // ---- ascending order (ties by index), W = R^{-1} Z
    if (t < k) {
        const double v = sT[t * SLD + t];
        int rank = 0;
        for (int j = 0; j < k; ++j) {
            const double u = sT[j * SLD + j];
            rank += (u < v || (u == v && j < t)) ? 1 : 0;
        }
        perm[rank] = t;
    }
    __syncthreads();
    trsv_upper(sR, rinv, sZ, sA, k, k);  // sA = R^{-1} Z (first k rows and columns of Z)
    for (int i = t; i < k; i += nt) theta[i] = sT[perm[i] * SLD + perm[i]];
    if (W)
        for (int e = t; e < k * k; e += nt) {
            const int j = e / k, i = e % k;
            W[j * k + i] = sA[j * SLD + perm[i]];
        }
}

template <typename Tm, typename Ty>
static sped_status run_update(int64_t n, void *V, int ldv, const void *Y, int ldy, int k,
                              Coefs *cf, int bdiag, bool stats, __nv_bfloat16 *shadow, int lds,
                              cudaStream_t st) {
    int blocks = device_sm_count() * 4;
    const int64_t need = (n + 255) / 256;
    if (need < blocks) blocks = (int)(need > 0 ? need : 1);
    const int vec = ((uintptr_t)V % 16 == 0) && ((uintptr_t)Y % 16 == 0) &&
                    (ldv * (int)sizeof(Tm)) % 16 == 0 && (ldy * (int)sizeof(Ty)) % 16 == 0;
#define UPD(KMV)                                                                               \
    SPED_TRY((launch_update<Tm, Ty, KMV>(blocks, n, V, ldv, Y, ldy, k, cf, bdiag, vec, stats,   \
                                         shadow, lds, st)))
    if (k <= 8) UPD(8);
    else if (k <= 16) UPD(16);
    else if (k <= 20) UPD(20);
    else if (k <= 24) UPD(24);
    else if (k <= 32) UPD(32);
    else UPD(40);
#undef UPD
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

static sped_status check_shadow(const sped_step_opts *o, sped_dtype vt, int k) {
    if (!o->v_shadow) return SPED_OK;
    if (vt != SPED_F32) return fail(SPED_ERR_INVALID_ARG, "BF16 shadow needs an F32 master V");
    return check_layout(o->v_shadow, SPED_BF16, k, o->shadow_ld, "eig_step shadow");
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
    // a valid BF16 shadow of V feeds the first launch of a BF16 exact chain
    const bool read_shadow = o->v_shadow && o->shadow_valid && o->chain_t == SPED_BF16 &&
                             o->mode == SPED_EXACT;
    SPED_TRY(apply_poly_impl(g, k, V, vt, ld, Y, o->y_t, L.ldy, o->chain_t, o->mode, o->walkers,
                             o->seed, shared, st, read_shadow ? o->v_shadow : nullptr, SPED_BF16,
                             o->shadow_ld));
    if (o->ev_chain_end) SPED_CUDA(cudaEventRecord((cudaEvent_t)o->ev_chain_end, st));
    shared.used = 0;
    SPED_TRY(launch_gram(g->n, V, vt, ld, k, Y, o->y_t, L.ldy, k, G, shared, st));
    SPED_CUDA(cudaMemsetAsync(&cf->err, 0, sizeof(int), st));
    SPED_CUDA(cudaFuncSetAttribute(k_small, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)SMALL_SMEM));
    SPED_CUDA(launch_pdl(k_small, dim3(1), dim3(SMALL_THREADS), SMALL_SMEM, st,
                         (const double *)G, k, o->eta, (int)o->solver, cf, d_stats));
    SPED_CHECK_LAUNCH("k_small");
    const int bdiag = o->solver == SPED_SOLVER_MU_EG;  // mu-EG: Y enters through eta I
    __nv_bfloat16 *shadow = (__nv_bfloat16 *)o->v_shadow;
    if (vt == SPED_F32 && o->y_t == SPED_F32) SPED_TRY((run_update<float, float>(g->n, V, ld, Y, L.ldy, k, cf, bdiag, d_stats != nullptr, shadow, o->shadow_ld, st)));
    else if (vt == SPED_F32 && o->y_t == SPED_F64) SPED_TRY((run_update<float, double>(g->n, V, ld, Y, L.ldy, k, cf, bdiag, d_stats != nullptr, shadow, o->shadow_ld, st)));
    else if (vt == SPED_F64 && o->y_t == SPED_F64) SPED_TRY((run_update<double, double>(g->n, V, ld, Y, L.ldy, k, cf, bdiag, d_stats != nullptr, nullptr, 0, st)));
    else if (vt == SPED_F64 && o->y_t == SPED_F32) SPED_TRY((run_update<double, float>(g->n, V, ld, Y, L.ldy, k, cf, bdiag, d_stats != nullptr, nullptr, 0, st)));
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
    SPED_TRY(check_shadow(opts, v_t, k));
    return eig_step_impl(g, opts, d_V, v_t, k, ld, d_stats, d_scratch, scratch_bytes,
                         as_stream(stream), nullptr);
}

sped_status sped_rayleigh_scratch_size(const sped_graph *g, int k, size_t *bytes) {
    if (!g || !bytes || k < 1 || k > MAXK) return fail(SPED_ERR_INVALID_ARG, "rayleigh_scratch_size");
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
    if (k < 1 || k > MAXK) return fail(SPED_ERR_UNSUPPORTED, "rayleigh: k=%d (1..%d)", k, MAXK);
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

sped_status sped_rayleigh_ritz_scratch_size(const sped_graph *g, int k, size_t *bytes) {
    if (!g || !bytes || k < 1 || k > MAXK)
        return fail(SPED_ERR_INVALID_ARG, "rayleigh_ritz_scratch_size: k in 1..%d", MAXK);
    size_t b = 0;
    SPED_TRY(sped_rayleigh_scratch_size(g, k, &b));
    *bytes = b + align_up(sizeof(double) * k * k, 256) + 256;
    return SPED_OK;
}

sped_status sped_rayleigh_ritz(const sped_graph *g, void *d_V, sped_dtype v_t, int k, int ld,
                               double *d_theta, double *d_W, int rotate, void *d_scratch,
                               size_t scratch_bytes, void *stream) {
    if (!g || !d_theta) return fail(SPED_ERR_INVALID_ARG, "rayleigh_ritz: null");
    if (k < 1 || k > MAXK) return fail(SPED_ERR_UNSUPPORTED, "rayleigh_ritz: k=%d (1..%d)", k, MAXK);
    if (v_t != SPED_F32 && v_t != SPED_F64)
        return fail(SPED_ERR_UNSUPPORTED, "rayleigh_ritz: V must be F32 or F64");
    SPED_TRY(check_layout(d_V, v_t, k, ld, "rayleigh_ritz V"));
    size_t need = 0;
    SPED_TRY(sped_rayleigh_ritz_scratch_size(g, k, &need));
    if (!d_scratch || scratch_bytes < need || ((uintptr_t)d_scratch) % 256)
        return fail(SPED_ERR_SCRATCH, "rayleigh_ritz: scratch needs %zu bytes", need);
    cudaStream_t st = as_stream(stream);
    Scratch scr(d_scratch, scratch_bytes);
    double *Wk = (double *)scr.take(sizeof(double) * k * k);
    const int ldl = padded_ld(k, SPED_F64);
    void *LV = scr.take((size_t)g->n * ldl * 8);
    double *G = (double *)scr.take(sizeof(double) * 4 * k * k);
    if (!Wk || !LV || !G) return fail(SPED_ERR_SCRATCH, "rayleigh_ritz: scratch too small");
    SPED_TRY(launch_poly_step(g, k, d_V, v_t, ld, nullptr, v_t, ld, LV, SPED_F64, ldl, 0.0, 1.0,
                              0.0, 0, scr, st));
    SPED_TRY(launch_gram(g->n, d_V, v_t, ld, k, LV, SPED_F64, ldl, k, G, scr, st));
    SPED_CUDA(cudaFuncSetAttribute(k_rayleigh_ritz, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)RR_SMEM));
    k_rayleigh_ritz<<<1, SMALL_THREADS, RR_SMEM, st>>>(G, k, d_theta, Wk);
    SPED_CHECK_LAUNCH("k_rayleigh_ritz");
    if (d_W) SPED_CUDA(cudaMemcpyAsync(d_W, Wk, sizeof(double) * k * k, cudaMemcpyDeviceToDevice, st));
    if (rotate)  // V <- V W in place: each row is read whole before it is written
        SPED_TRY(sped_block_combine(g->n, k, d_V, ld, Wk, nullptr, 0, nullptr, d_V, ld, v_t, stream));
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
        if (step > 1) so.shadow_valid = 1;  // the previous step left bf16(V) in the shadow
        if (so.mode != SPED_EXACT) so.seed += (uint64_t)(step - 1);  // fresh draws every step
        // the statistics (Rayleigh quotients, residuals, step norms) cost a Cholesky solve and a
        // second k x k product per row, so they are formed on check steps only
        const bool check = step % opts->check_every == 0 || step == opts->max_steps;
        SPED_TRY(sped_eig_step(g, &so, d_V, v_t, k, ld, check ? d_stats : nullptr, d_scratch,
                               body, stream));
        rep.steps = step;
        rep.spmm_count += poly_spmm_count(g, so.mode);
        if (phase == 1) rep.phase1_steps = step;
        if (check) {
            SPED_CUDA(cudaMemcpyAsync(h_stats, d_stats, sizeof(double) * 3 * k,
                                      cudaMemcpyDeviceToHost, st));
            int h_err = 0;
            SPED_CUDA(cudaMemcpyAsync(&h_err, base + coef_off + offsetof(Coefs, err), sizeof(int),
                                      cudaMemcpyDeviceToHost, st));
            SPED_CUDA(cudaStreamSynchronize(st));
            // a bounded wait that gave up leaves a NaN Gram: report the cause, not the symptom
            if (h_err) SPED_TRY(sped_device_status(stream));
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
    SPED_TRY(sped_device_status(stream));
    if (!rep.converged)
        return fail(SPED_ERR_NOT_CONVERGED, "solve_bottom_k: %d steps, residual %.3e > tol %.3e",
                    rep.steps, rep.final_residual, opts->tol);
    return SPED_OK;
}

}  // extern "C"
