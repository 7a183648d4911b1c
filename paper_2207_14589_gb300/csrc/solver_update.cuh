// Internal declarations shared by the solver step and the translation units that hold its
// N x k update kernel (split by width so that the kernel's instantiations compile in parallel).
#pragma once

#include "sped_internal.cuh"

namespace sped {

constexpr int MAXK = 40;

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

// V <- (V A + Y B) diag(scale) for rows of width KM (k <= KM), launched on `blocks` CTAs of 256
// threads; stats selects the variant that also accumulates the step sizes and residuals.
// Instantiated in update_km*.cu.
template <typename Tm, typename Ty, int KM>
sped_status launch_update(int blocks, int64_t n, void *V, int ldv, const void *Y, int ldy, int k,
                          Coefs *cf, int bdiag, int vec, bool stats, __nv_bfloat16 *shadow,
                          int lds, cudaStream_t st);

}  // namespace sped
