// Block moments of a polynomial basis on span(V): Omega_l = V^T B_l V, l = 0..m-1, with B_l = L^l
// or the Chebyshev polynomial T_l(x), x = (2L - (a + b) I) / (b - a). For M = sum_l c_l B_l the
// Rayleigh-Ritz matrix of M on span(V) is sum_l c_l Omega_l, and with the products B_l B_m
// (L^{l+m}, or (T_{l+m} + T_{|l-m|}) / 2) and x B_m ((T_{m+1} + T_{|m-1|}) / 2) every quadratic
// form of V and M V -- (MV)^T (MV), (MV)^T L (MV) -- is an explicit function of the coefficients.
// That is what fitting (meta-learning) the polynomial's coefficients works on; the paper names
// meta-learning them as future work (Section 6) without a method.
//
// Each moment costs one chain-step launch (the basis recurrence: L P, or 2x P_{l-1} - P_{l-2}
// through the step kernel's second block) and one Gram of [V, B_l V]; the k x k block V^T B_l V
// is copied out of the 2k x 2k Gram. Three blocks rotate.
#include <cmath>

#include "sped_internal.cuh"

namespace sped {

static size_t moments_layout(const sped_graph *g, int k, sped_dtype vt, size_t *blk) {
    *blk = align_up((size_t)g->n * padded_ld(k, vt) * dtype_size(vt), 256);
    ScratchPlan p;
    for (int i = 0; i < 3; ++i) p.add(*blk);
    p.add(sizeof(double) * 4 * (size_t)k * k);
    const size_t step = poly_step_scratch(g, k, vt, 0), gram = gram_scratch(g->n, k, k);
    p.add(step > gram ? step : gram);
    return p.total();
}

}  // namespace sped

using namespace sped;

extern "C" {

sped_status sped_poly_moments_scratch_size(const sped_graph *g, int k, sped_dtype v_t,
                                           size_t *bytes) {
    if (!g || !bytes || k < 1 || k > 32 || !dtype_valid(v_t))
        return fail(SPED_ERR_INVALID_ARG, "poly_moments_scratch_size: bad arguments");
    size_t blk;
    *bytes = moments_layout(g, k, v_t, &blk);
    return SPED_OK;
}

sped_status sped_poly_moments(const sped_graph *g, const void *d_V, sped_dtype v_t, int k, int ld,
                              int basis, int n_moments, double a, double b, double *d_out,
                              void *d_scratch, size_t scratch_bytes, void *stream) {
    if (!g || !d_out) return fail(SPED_ERR_INVALID_ARG, "poly_moments: null argument");
    SPED_TRY(check_layout(d_V, v_t, k, ld, "poly_moments V"));
    if (v_t != SPED_F32 && v_t != SPED_F64)
        return fail(SPED_ERR_UNSUPPORTED, "poly_moments: V must be F32 or F64");
    if (k > 32) return fail(SPED_ERR_UNSUPPORTED, "poly_moments: k = %d > 32", k);
    if (basis != 0 && basis != 1) return fail(SPED_ERR_INVALID_ARG, "poly_moments: basis %d", basis);
    if (n_moments < 1) return fail(SPED_ERR_INVALID_ARG, "poly_moments: n_moments < 1");
    if (b == 0.0) b = g->lambda_bound;
    if (basis == 1 && !(b > a && std::isfinite(a) && std::isfinite(b)))
        return fail(SPED_ERR_INVALID_ARG, "poly_moments: interval [%g, %g] is empty", a, b);
    size_t blk;
    const size_t need = moments_layout(g, k, v_t, &blk);
    if (!d_scratch || scratch_bytes < need || ((uintptr_t)d_scratch) % 256)
        return fail(SPED_ERR_SCRATCH, "poly_moments: scratch needs %zu bytes (256-aligned)", need);
    cudaStream_t st = as_stream(stream);
    Scratch scr(d_scratch, scratch_bytes);
    void *blocks[3];
    for (int i = 0; i < 3; ++i) blocks[i] = scr.take(blk);
    double *G2 = (double *)scr.take(sizeof(double) * 4 * (size_t)k * k);
    const size_t off = align_up(scr.used, 256);
    Scratch rest((char *)d_scratch + off, scratch_bytes - off);
    const int ldc = padded_ld(k, v_t);
    const double al = basis == 1 ? 2.0 / (b - a) : 1.0;
    const double be = basis == 1 ? -(a + b) / (b - a) : 0.0;
    // P_l = B_l V: P_0 = V (the caller's layout), P_l in blocks[l % 3]
    auto P = [&](int l) -> const void * { return l == 0 ? d_V : blocks[l % 3]; };
    auto ldP = [&](int l) { return l == 0 ? ld : ldc; };
    for (int l = 0; l < n_moments; ++l) {
        if (l >= 1) {
            rest.used = 0;
            void *y = blocks[l % 3];
            if (basis == 0 || l == 1) {  // L P_{l-1}, or x V = al L V + be V
                SPED_TRY(launch_poly_step(g, k, P(l - 1), v_t, ldP(l - 1), nullptr, v_t, 0, y,
                                          v_t, ldc, 0.0, al, basis == 0 ? 0.0 : be, 0, rest,
                                          st));
            } else {  // T_l V = 2x T_{l-1} V - T_{l-2} V
                SPED_TRY(launch_poly_step_w2(g, k, P(l - 1), v_t, ldP(l - 1), d_V, v_t, ld, y,
                                             v_t, ldc, 0.0, 2.0 * al, 2.0 * be, P(l - 2),
                                             ldP(l - 2), -1.0, 0, rest, st));
            }
        }
        rest.used = 0;
        SPED_TRY(launch_gram(g->n, d_V, v_t, ld, k, P(l), v_t, ldP(l), k, G2, rest, st));
        SPED_CUDA(cudaMemcpy2DAsync(d_out + (size_t)l * k * k, sizeof(double) * k, G2 + k,
                                    sizeof(double) * 2 * k, sizeof(double) * k, k,
                                    cudaMemcpyDeviceToDevice, st));
    }
    return SPED_OK;
}

}  // extern "C"
