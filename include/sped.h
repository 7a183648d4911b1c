/*
 * sped.h -- C ABI of the GB300 (sm_103a) implementation of the hot path of
 * "Stochastic Parallelizable Eigengap Dilation for Large Graph Clustering"
 * (van der Pol, Gemp, Bachrach, Everett; arXiv 2207.14589).
 *
 * The hot path applies an eigenvector-preserving polynomial p(L) of a sparse graph Laplacian
 * to an n x k block V (exactly by chained CSR SpMM, or by the paper's unbiased random-walk
 * estimate) and feeds p(L) V into a bottom-k eigensolver step (mu-EigenGame or Oja).
 *
 * Conventions for every entry point
 *  - Pointers named d_* are CUDA device pointers on the current device; h_* are host pointers.
 *    The caller owns every buffer. Nothing on the per-step path allocates: scratch memory is
 *    passed in, sized by the matching *_scratch_size query. Scratch must be 256-byte aligned.
 *  - Dense blocks are row-major n x k with leading dimension ld (elements, ld >= k). The vector
 *    path needs ld * sizeof(element) to be a multiple of 16 bytes and 16-byte aligned bases;
 *    other layouts are rejected with SPED_ERR_INVALID_ARG.
 *  - stream is a cudaStream_t passed as void* (NULL = legacy default stream). Work is
 *    stream-ordered; entry points return after enqueueing unless documented as synchronising.
 *  - Arguments are validated on the host before any launch; a rejected call launches nothing.
 *    Errors found on the device (invalid CSR, non-positive-definite Gram, a bounded wait that
 *    gave up) are reported by the next synchronising call. sped_last_error() returns a
 *    thread-local message for the last failing call on this thread.
 *  - Graph input: symmetric adjacency in CSR with int32 row_ptr[n+1] and col_idx[nnz],
 *    columns strictly increasing within each row, no self loops; optional float32 weights per
 *    stored entry, equal for (i,j) and (j,i).
 */
#ifndef SPED_H
#define SPED_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sped_graph sped_graph; /* opaque: device metadata of one graph */

typedef enum {
    SPED_OK = 0,
    SPED_ERR_INVALID_ARG = 1,   /* bad pointer, size, layout or option */
    SPED_ERR_BAD_CSR = 2,       /* graph violates the input convention above */
    SPED_ERR_UNSUPPORTED = 3,   /* valid request with no kernel (e.g. dtype combination) */
    SPED_ERR_NUMERIC = 4,       /* NaN/Inf, or a Gram that is not positive definite */
    SPED_ERR_NOT_CONVERGED = 5, /* solver stopped at max_steps above tolerance */
    SPED_ERR_TIMEOUT = 6,       /* a bounded device-side wait gave up */
    SPED_ERR_CUDA = 7,          /* CUDA runtime error (message in sped_last_error) */
    SPED_ERR_SCRATCH = 8        /* scratch buffer too small or misaligned */
} sped_status;

typedef enum { SPED_BF16 = 0, SPED_F32 = 1, SPED_F64 = 2 } sped_dtype;

/* Polynomial families (Table 2 of the paper; reversal of Eq. reveig folded in so that the
 * wanted bottom-k eigenvectors of L are the top-k of the operator M that is applied). */
typedef enum {
    SPED_POLY_LIMIT_EXP = 0,  /* M = (I - sL)^l, l odd: reversed limit form -(I - L/l)^l   */
    SPED_POLY_TAYLOR_EXP = 1, /* M = sum_{i<=l} (-L)^i / i!: reversed Taylor -e^{-L}        */
    SPED_POLY_TAYLOR_LOG = 2, /* M = lambda* I - sum_{i=1}^{l} (-1)^{i+1} (L+(eps-1)I)^i / i */
    SPED_POLY_MONOMIAL = 3,   /* M = sum_i c_i L^i with caller coefficients c_0..c_l        */
    SPED_POLY_SHIFT = 4,      /* M = lambda* I - L: the plain reversed Laplacian, Eq. reveig */
    SPED_POLY_CHEBYSHEV = 5   /* M = sum_i c_i T_i(x), x = (2L - (a+b) I) / (b - a): Chebyshev
                                 series (or filter) on [a, b], caller coefficients c_0..c_l  */
} sped_poly_kind;

typedef enum {
    SPED_EXACT = 0,               /* chained SpMM                                           */
    SPED_STOCHASTIC_IS = 1,       /* random-walk estimate, importance weights (Section 4.3) */
    SPED_STOCHASTIC_REJECT = 2,   /* random-walk estimate, the text's rejection step        */
    SPED_STOCHASTIC_MINIBATCH = 3, /* every multiplication by L from its own edge minibatch */
    SPED_STOCHASTIC_MINIBATCH_STRATIFIED = 4 /* the same, one draw per stratum of the edges */
} sped_mode;

typedef enum { SPED_SOLVER_MU_EG = 0, SPED_SOLVER_OJA = 1 } sped_solver;

/* ------------------------------------------------------------------------------------
 * Graph set-up (Section 2: L = D - A; end of Section 2.1: weighted L = X^T W X).
 * ------------------------------------------------------------------------------------ */

/* Bytes of device workspace sped_build_laplacian needs for a graph with n nodes and nnz
 * stored entries (reverse-entry map, undirected edge ids, edge list, weight copy). */
sped_status sped_workspace_size(int64_t n, int64_t nnz, size_t *bytes);

/* Validate the CSR (when check != 0), derive the reverse-entry map, the undirected edge list
 * (edges numbered by the CSR order of their upper entries a < b), weighted degrees and the
 * spectral bound lambda_max <= 2 max_i d_i (Section 5.4). row_ptr/col_idx (and d_w when not
 * NULL) must stay valid while the graph is used; col_idx and w must be 16-byte aligned (the
 * chain kernel reads them in 16-byte quads); d_workspace holds the derived arrays.
 * Synchronises the stream. On success *out receives a graph handle; the default polynomial
 * is SPED_POLY_SHIFT with lambda* = the spectral bound. */
sped_status sped_build_laplacian(int64_t n, int64_t nnz, const int32_t *d_row_ptr,
                                 const int32_t *d_col_idx, const float *d_w, void *d_workspace,
                                 size_t ws_bytes, int check, void *stream, sped_graph **out);

void sped_graph_destroy(sped_graph *g);

typedef struct {
    int64_t n, nnz, n_edges;
    int32_t max_degree;     /* largest neighbour count deg* (Section 4.3)              */
    double max_wdegree;     /* largest weighted degree                                 */
    double lambda_bound;    /* 2 * max weighted degree >= lambda_max                    */
    int weighted;
    /* resolved polynomial */
    int poly_kind, degree;
    double scale_s, shift, lambda_star;
} sped_graph_info;

sped_status sped_graph_get_info(const sped_graph *g, sped_graph_info *info);

/* Device arrays of the undirected edge list: d_edge_a[e] < d_edge_b[e], e in [0, n_edges).
 * Either output may be NULL. */
sped_status sped_graph_edges(const sped_graph *g, int32_t *d_edge_a, int32_t *d_edge_b,
                             void *stream);

/* Replace the weights by one float32 per undirected edge (edge order as above), e.g. learned
 * weights. Writes the per-entry copy kept in the workspace; the graph uses it from then on.
 * Synchronises (the spectral bound is recomputed). */
sped_status sped_set_edge_weights(sped_graph *g, const float *d_w_edge, void *stream);

/* ------------------------------------------------------------------------------------
 * Polynomial (Sections 4.1-4.2, Table 2).
 *  degree     l >= 1 (odd required for SPED_POLY_LIMIT_EXP so the map is monotone on R).
 *  scale_s    limit form only; 0 = automatic: 1/l when l >= lambda_bound/2, else
 *             2/lambda_bound, so that |1 - s lambda| <= 1 on the whole spectrum.
 *  eps        Taylor log only (the table's eps << 1); 0 = 1e-3.
 *  coeffs     SPED_POLY_MONOMIAL only: l+1 host doubles c_0..c_l.
 *  lambda_star SHIFT and TAYLOR_LOG: 0 = automatic (the spectral bound, or for the log the
 *             series' value bound).
 *  CHEBYSHEV  coeffs: l+1 host doubles c_0..c_l; eps = a and lambda_star = b (0 = the spectral
 *             bound) are the ends of the interval mapped onto [-1, 1], a < b. Evaluated by
 *             Clenshaw's recurrence: l chain steps, each Y = alpha V + gamma X + beta L X -
 *             (the output of the step before last), three chain buffers. A single c_l = 1 is
 *             the Chebyshev filter T_l, which damps [a, b] and grows fastest below a.
 * ------------------------------------------------------------------------------------ */
sped_status sped_set_polynomial(sped_graph *g, sped_poly_kind kind, int degree, double scale_s,
                                double eps, const double *coeffs, double lambda_star);

/* Power-basis coefficients c_0..c_l of the operator M = sum_i c_i L^i (h_out: l+1 doubles). */
sped_status sped_get_power_coeffs(const sped_graph *g, double *h_out, int capacity);

/* Block moments of a polynomial basis on span(V), the data for fitting (meta-learning) the
 * coefficients of M = sum_l c_l B_l, which the paper names as future work (Section 6):
 *   d_out[l*k*k + i*k + j] = (V^T B_l V)_{ij},  l = 0 .. n_moments-1 (FP64, device),
 * basis 0: B_l = L^l; basis 1: B_l = T_l(x), x = (2L - (a + b) I) / (b - a) (b = 0: the
 * spectral bound). Then V^T M V = sum_l c_l Omega_l; for the power basis (MV)^T (MV) =
 * sum_{l,m} c_l c_m Omega_{l+m} and (MV)^T L (MV) = sum c_l c_m Omega_{l+m+1}; for the Chebyshev
 * basis T_l T_m = (T_{l+m} + T_{|l-m|}) / 2 and x T_m = (T_{m+1} + T_{|m-1|}) / 2. One chain step
 * and one Gram per moment. V: F32 or F64, k <= 32. Scratch: sped_poly_moments_scratch_size. */
sped_status sped_poly_moments(const sped_graph *g, const void *d_V, sped_dtype v_t, int k, int ld,
                              int basis, int n_moments, double a, double b, double *d_out,
                              void *d_scratch, size_t scratch_bytes, void *stream);
sped_status sped_poly_moments_scratch_size(const sped_graph *g, int k, sped_dtype v_t,
                                           size_t *bytes);

/* ------------------------------------------------------------------------------------
 * One fused step of the polynomial chain (the hot kernel):
 *   Y[r,:] = alpha V[r,:] + gamma X[r,:] + beta (d_r X[r,:] - sum_j w_rj X[j,:])
 * i.e. Y = alpha V + gamma X + beta L X. d_V may be NULL when alpha == 0. X and Y must not
 * overlap. Supported (x, y) storage pairs: (F64,F64) (F32,F32) (BF16,BF16) (F32,BF16)
 * (BF16,F32) (F32,F64); accumulation in F64 when y is F64, else F32. V (when used) is
 * F32 or F64, or BF16 when x is BF16.
 * split: 0 = automatic, 1 = row-group kernel, 2 = merge-path kernel (needs scratch).
 * ------------------------------------------------------------------------------------ */
sped_status sped_poly_step(const sped_graph *g, int k, const void *d_X, sped_dtype x_t, int ldx,
                           const void *d_V, sped_dtype v_t, int ldv, void *d_Y, sped_dtype y_t,
                           int ldy, double alpha, double beta, double gamma, int split,
                           void *d_scratch, size_t scratch_bytes, void *stream);

sped_status sped_poly_step_scratch_size(const sped_graph *g, int k, sped_dtype x_t, int split,
                                        size_t *bytes);

/* ------------------------------------------------------------------------------------
 * Schedule selection for the chain step (the paper has no counterpart: it names no kernel).
 * sped_autotune times one step X -> X - 0.01 L X of storage type chain_t on this graph for
 * each candidate schedule -- the row-group kernel, and the merge path with shares of 128,
 * 256, 512 and 1024 items (rows + stored entries) -- and records the fastest in the graph, so
 * that every later split = 0 (automatic) step on it uses that schedule. The choice is also kept
 * in a per-process table keyed by the graph's shape (n, nnz, maximum degree, weighted or not,
 * k, chain_t, device); a later call for the same shape takes it from there without timing
 * (report->cached = 1). The call synchronises `stream` (it reads CUDA event times).
 * Scratch (device, 256-byte aligned): sped_autotune_scratch_size bytes; its contents are
 * overwritten. Scratch needs of sped_poly_step / sped_apply_poly / sped_eig_step depend on the
 * chosen schedule, so query them after tuning. On failure the graph keeps its previous
 * schedule. sped_set_schedule fixes it by hand (split 0 = degree rule, 1 = row group,
 * 2 = merge path; merge_ipg 0 = default share, else 32..2^20 items).
 * ------------------------------------------------------------------------------------ */
typedef struct {
    int split;         /* chosen schedule: 1 row group, 2 merge path                          */
    int merge_ipg;     /* merge-path share in items when split == 2, else 0                   */
    int cached;        /* 1: taken from the per-process table, nothing was timed              */
    int n_candidates;  /* entries of ms[] filled                                               */
    double ms[8];      /* mean step time per candidate: [0] row group, [1..4] merge path with
                          shares 128, 256, 512, 1024                                           */
} sped_tune_report;

sped_status sped_autotune_scratch_size(const sped_graph *g, int k, sped_dtype chain_t,
                                       size_t *bytes);
sped_status sped_autotune(sped_graph *g, int k, sped_dtype chain_t, void *d_scratch,
                          size_t scratch_bytes, void *stream, sped_tune_report *report);
sped_status sped_set_schedule(sped_graph *g, int split, int merge_ipg);

/* ------------------------------------------------------------------------------------
 * Y = M V for the graph's polynomial M (Sections 4.2-4.3).
 *  mode SPED_EXACT: the chain of poly steps; intermediate products stored as chain_t
 *    (BF16 halves gather traffic, accumulation stays F32), the last step writes y_t.
 *  mode SPED_STOCHASTIC_IS / _REJECT: Y = c_0 V + mean over `walkers` walks of the sampled
 *    terms (Section 4.3), draws from Philox4x32-10 keyed by seed (documented in walk.cu);
 *    y_t must be F32 or F64; chain_t is ignored.
 *  mode SPED_STOCHASTIC_MINIBATCH: the edges-in-minibatches model of Sections 2 and 6. The
 *    chain of the exact mode runs with multiplication t (factor t of the limit form, step t of
 *    Horner's or Clenshaw's recurrence, t = 0, 1, ... in evaluation order) by its own estimate
 *    L_hat_t = (|E| / B) sum_{j<B} w_{e_j} x_{e_j} x_{e_j}^T, where B = `walkers` and the e_j are
 *    edge ids drawn uniformly with replacement (L = sum_e w_e x_e x_e^T, Section 4.3). Draw j of
 *    multiplication t is the first Lemire bounded draw in [0, |E|) of the Philox4x32-10 word
 *    stream with key `seed` and counters (j, t, 0x4D42, i), i = 0, 1, ... (edges numbered as in
 *    sped_graph_edges). The multiplications are independent, so Y is an unbiased estimate of
 *    M V for every family. chain_t, v_t and y_t: F32 or F64 (the edge terms are added by
 *    atomic adds, so the summation order is not fixed: results match a sequential sum to
 *    rounding, not bit for bit). 1 <= B <= 2^32.
 *  mode SPED_STOCHASTIC_MINIBATCH_STRATIFIED: variance reduction (left to future work in
 *    Section 6). The edge ids are cut into B contiguous strata S_j = [floor(j |E| / B),
 *    floor((j+1) |E| / B)); draw j is uniform in S_j (the first Lemire bounded draw over |S_j|
 *    of the same stream) and L_hat_t = sum_j |S_j| w_{e_j} x_{e_j} x_{e_j}^T (empty strata, when
 *    B > |E|, add nothing). Unbiased; B >= |E| gives L exactly.
 * ------------------------------------------------------------------------------------ */
sped_status sped_apply_poly(const sped_graph *g, int k, const void *d_V, sped_dtype v_t, int ldv,
                            void *d_Y, sped_dtype y_t, int ldy, sped_dtype chain_t,
                            sped_mode mode, int64_t walkers, uint64_t seed, void *d_scratch,
                            size_t scratch_bytes, void *stream);

sped_status sped_apply_poly_scratch_size(const sped_graph *g, int k, sped_dtype chain_t,
                                         sped_mode mode, size_t *bytes);

/* Backward of Y = M V with respect to V: dV = M^T dY = M dY, since M = p(L) is symmetric (L is,
 * Section 2), i.e. the exact chain of sped_apply_poly run on dY (same dtype rules; scratch:
 * sped_apply_poly_scratch_size with SPED_EXACT). The gradient with respect to the edge weights
 * of a utility of (V, M V) is sped_edge_grad. */
sped_status sped_apply_poly_backward(const sped_graph *g, int k, const void *d_dY, sped_dtype dy_t,
                                     int lddy, void *d_dV, sped_dtype dv_t, int lddv,
                                     sped_dtype chain_t, void *d_scratch, size_t scratch_bytes,
                                     void *stream);

/* ------------------------------------------------------------------------------------
 * Edge minibatches fed from outside (Sections 2 and 6: edges arrive in minibatches, or are
 * drawn from a distribution such as a link-prediction model's output).
 * sped_sample_edges writes the minibatch that SPED_STOCHASTIC_MINIBATCH (stratified == 0) or
 * SPED_STOCHASTIC_MINIBATCH_STRATIFIED (stratified != 0) uses for multiplication `step`: for
 * draw j < count, d_a[j] < d_b[j] are the edge's endpoints and d_w[j] its weight (1 for an
 * unweighted graph); with stratified draws d_size[j] = |S_j| (an empty stratum gives
 * a = b = -1, w = 0, size 0; d_size is not written for uniform draws). Any output may be NULL.
 * count <= 2^32, and the graph must have an edge when count > 0.
 * sped_edge_step runs one chain step on a caller-supplied minibatch:
 *   Y = alpha V + gamma X + beta * edge_scale * sum_{j<count} w_j x_j x_j^T X,
 * x_j = e_{a_j} - e_{b_j}; that is Y[a_j] += c_j (X[a_j] - X[b_j]) and Y[b_j] -= c_j (X[a_j] -
 * X[b_j]) with c_j = beta * edge_scale * w_j. d_w may be NULL (all weights 1). edge_scale =
 * |E| / count makes the sum an unbiased estimate of L X when the edges are uniform draws from E.
 * X, V, Y: n x k blocks, F32 or F64; X and Y must not overlap; d_V may be NULL when alpha == 0.
 * Draws with an endpoint outside [0, n) are skipped and counted into *d_skipped (device int32,
 * may be NULL). The edge terms are added by atomic adds (order not fixed).
 * ------------------------------------------------------------------------------------ */
sped_status sped_sample_edges(const sped_graph *g, uint64_t seed, uint32_t step, int64_t count,
                              int stratified, int32_t *d_a, int32_t *d_b, float *d_w,
                              int32_t *d_size, void *stream);

sped_status sped_edge_step(int64_t n, int k, const int32_t *d_a, const int32_t *d_b,
                           const float *d_w, int64_t count, double edge_scale, const void *d_X,
                           sped_dtype x_t, int ldx, const void *d_V, sped_dtype v_t, int ldv,
                           void *d_Y, sped_dtype y_t, int ldy, double alpha, double beta,
                           double gamma, int32_t *d_skipped, void *stream);

/* ------------------------------------------------------------------------------------
 * Gram of a tall-skinny pair: G = [A B]^T [A B], (ka+kb) x (ka+kb) row-major FP64,
 * ka + kb <= 80. d_B may be NULL (kb = 0). Products in F32 for BF16/F32 inputs (exact for
 * BF16), accumulated in F32 over short row tiles and in F64 across tiles and CTAs;
 * F64 inputs use F64 throughout. Deterministic (fixed reduction order).
 * ------------------------------------------------------------------------------------ */
sped_status sped_gram(int64_t n, const void *d_A, sped_dtype a_t, int lda, int ka, const void *d_B,
                      sped_dtype b_t, int ldb, int kb, double *d_G, void *d_scratch,
                      size_t scratch_bytes, void *stream);

sped_status sped_gram_scratch_size(int64_t n, int ka, int kb, size_t *bytes);

/* Device-detected errors that have no synchronising call of their own. Synchronises `stream`,
 * then reads and clears this library's device status word on the current device: returns
 * SPED_ERR_TIMEOUT when a bounded device-side wait gave up since the last read (the tensor-core
 * Gram's waits on its bulk copies and MMAs; the Gram of that call is NaN), else SPED_OK.
 * sped_solve_bottom_k reads the word too and returns SPED_ERR_TIMEOUT in the same case. The
 * word is shared by every stream and host thread using the device. */
sped_status sped_device_status(void *stream);

/* Test control of the tensor-core Gram's bounded waits, for the calling process: wait_limit is
 * the number of polls after which a wait gives up (0 = the default of 2^22 polls); skip_fills
 * != 0 makes the kernel issue no bulk copies (and so no MMAs), so its first wait runs out with
 * nothing in flight: the CTA frees its tensor memory, writes NaN partials and sets the status
 * word read by sped_device_status. For tests of the timeout path only; leave at (0, 0). */
sped_status sped_test_gram_waits(uint32_t wait_limit, int skip_fills);

/* sped_gram for callers that cannot allocate device memory: for example code running inside a
 * host callback, a real-time loop or a plugin host, where cudaMalloc (which may synchronise the
 * device) is not allowed and no device allocator is handed in. The paper has no counterpart;
 * this is a deployment variant of sped_gram with the same arguments minus the scratch buffer
 * and the same result (within the same rounding).
 *  - Scratch: a fixed 4 MiB static device array inside the library (held by every GPU that
 *    loads the library until the process exits). Maximum size: ka + kb <= 64, any n; larger
 *    column counts are rejected with SPED_ERR_UNSUPPORTED before anything is launched.
 *  - Set-up: the first call on each device looks up the array's device address (with that
 *    device current); make that first call before any stream capture.
 *  - Concurrency: all calls share the array and overwrite it; calls that overlap on the GPU
 *    (different streams or host threads) race and must be serialised by the caller.
 *  - Allocates nothing: no cudaMalloc, cudaFree or allocating library routine. */
sped_status sped_gram_noalloc(int64_t n, const void *d_A, sped_dtype a_t, int lda, int ka,
                              const void *d_B, sped_dtype b_t, int ldb, int kb, double *d_G,
                              void *stream);

/* ------------------------------------------------------------------------------------
 * One solver step on the graph's operator M (Section 5.1: mu-EG and Oja; Section 3 for the
 * reversal). V (n x k, F32 or F64 master copy, k <= 40) is updated in place:
 *  mu-EG: delta_i = y_i - sum_{j<i} <v_i,y_j> v_j, r_i = delta_i - <v_i,delta_i> v_i,
 *         v_i <- (v_i + eta r_i)/||.||, all inner products from the Gram [V Y]^T [V Y];
 *  Oja:   V <- (V + eta Y) R^{-1} with R the Cholesky factor of its Gram (eta <= 0: V <- Y R^{-1}).
 * d_stats (device, 3k doubles, may be NULL): Rayleigh quotients <v_i,Mv_i>/<v_i,v_i>; the
 * invariant-subspace residuals ||(I - P_V) y_i|| / ||y_i|| (P_V the orthogonal projector onto
 * span(V) before the step; zero exactly when span(V) is M-invariant); the step sizes
 * ||v_i(new) - v_i||.
 * ------------------------------------------------------------------------------------ */
typedef struct {
    sped_solver solver;
    double eta;
    sped_dtype chain_t; /* storage of intermediate products                           */
    sped_dtype y_t;     /* storage of Y = M V: F32 or F64                              */
    sped_mode mode;     /* exact or stochastic p(L) V                                  */
    int64_t walkers;    /* walks (IS / REJECT) or edges per minibatch (MINIBATCH modes)  */
    uint64_t seed;
    /* optional cudaEvent_t pair (as void*, NULL = none) recorded on the stream immediately
     * before and after the p(L) V chain, for live timing of the dominant kernel */
    void *ev_chain_begin;
    void *ev_chain_end;
    /* optional BF16 shadow of the master V (device, n x shadow_ld BF16, shadow_ld * 2 a
     * multiple of 16 bytes, 16-byte aligned; NULL = none; F32 master only). The update writes
     * bf16(V_new) into it. When shadow_valid is nonzero the caller asserts that it holds
     * bf16(V) on entry (as left by the previous step with the same shadow and no change to V
     * since), and with a BF16 exact chain the first chain launch reads it instead of the F32
     * master (k-column BF16 rows instead of F32 rows). */
    void *v_shadow;
    int shadow_ld;
    int shadow_valid;
} sped_step_opts;

sped_status sped_eig_step(const sped_graph *g, const sped_step_opts *opts, void *d_V,
                          sped_dtype v_t, int k, int ld, double *d_stats, void *d_scratch,
                          size_t scratch_bytes, void *stream);

sped_status sped_eig_step_scratch_size(const sped_graph *g, const sped_step_opts *opts, int k,
                                       size_t *bytes);

/* Rayleigh quotients of the Laplacian itself, lambda_i = <v_i, L v_i>/<v_i, v_i>, in FP64
 * (d_out: k doubles). */
sped_status sped_rayleigh(const sped_graph *g, const void *d_V, sped_dtype v_t, int k, int ld,
                          double *d_out, void *d_scratch, size_t scratch_bytes, void *stream);

sped_status sped_rayleigh_scratch_size(const sped_graph *g, int k, size_t *bytes);

/* Rayleigh-Ritz: the Ritz pairs of L on span(V) in FP64. With R the upper Cholesky factor of
 * V^T V, theta and Z are the eigenvalues (ascending) and eigenvectors of the symmetric k x k
 * matrix R^{-T} (V^T L V) R^{-1} (cyclic Jacobi rotations on one CTA), and W = R^{-1} Z, so the
 * columns of V W are orthonormal Ritz vectors. d_theta: k doubles; d_W: k x k row-major
 * doubles (W[j*k + i] = coefficient of v_j in Ritz vector i), may be NULL; rotate != 0
 * replaces V by V W in place. When V^T V is not positive definite theta is NaN (and V is left
 * unchanged only if rotate == 0). k <= 40, V F32 or F64. */
sped_status sped_rayleigh_ritz(const sped_graph *g, void *d_V, sped_dtype v_t, int k, int ld,
                               double *d_theta, double *d_W, int rotate, void *d_scratch,
                               size_t scratch_bytes, void *stream);

sped_status sped_rayleigh_ritz_scratch_size(const sped_graph *g, int k, size_t *bytes);

/* ------------------------------------------------------------------------------------
 * Iterate eig_step to convergence (synchronising). The convergence measure is the largest
 * invariant-subspace residual max_i ||(I - P_V) y_i|| / ||y_i|| (second block of d_stats), which
 * tracks the sine of the angle between span(V) and span(MV). Phase 1 stores the chain in
 * opts.step.chain_t (e.g. BF16) until the measure is <= switch_tol or phase1_steps steps;
 * phase 2 uses refine_chain_t (e.g. F32) until <= tol. The test reads the statistics every
 * check_every steps. In the stochastic modes step s (from 1) draws with seed opts.step.seed +
 * s - 1, so the estimates of different steps are independent. h_lambda (host, k doubles, may be NULL) receives the
 * Rayleigh quotients of L.
 * ------------------------------------------------------------------------------------ */
typedef struct {
    sped_step_opts step;
    int max_steps;
    int check_every;
    double tol;
    double switch_tol;
    int phase1_steps;
    sped_dtype refine_chain_t;
} sped_solve_opts;

typedef struct {
    int steps;
    int phase1_steps;
    int64_t spmm_count;
    double final_residual; /* largest invariant-subspace residual at exit */
    int converged;
} sped_solve_report;

sped_status sped_solve_bottom_k(const sped_graph *g, const sped_solve_opts *opts, void *d_V,
                                sped_dtype v_t, int k, int ld, double *h_lambda,
                                sped_solve_report *report, void *d_scratch, size_t scratch_bytes,
                                void *stream);

sped_status sped_solve_scratch_size(const sped_graph *g, const sped_solve_opts *opts, int k,
                                    size_t *bytes);

/* ------------------------------------------------------------------------------------
 * Hard clustering (Sections 1 and 2.1): k-means on the rows of V (n x k, any dtype), rows not
 * normalised. k-means++ seeding from Philox4x32-10 (key = seed; centre 0 is a bounded draw
 * from the word stream of counter (0, 0, 0x6B6D, j), centre c >= 1 uses u = (w + 0.5) 2^-32
 * with w the first word of counter (c, 0, 0, 0x6B6D), taking the first row whose running sum
 * of squared distances exceeds u times the total); Lloyd iterations in FP64 until labels stop
 * changing or max_iter; ties to the lowest centroid; an empty cluster restarts at the
 * farthest point; labels renumbered by first occurrence. Synchronises; *h_iters (may be
 * NULL) receives the Lloyd iteration count.
 * ------------------------------------------------------------------------------------ */
sped_status sped_cluster_assign(const void *d_V, sped_dtype v_t, int64_t n, int k, int ld,
                                int n_clusters, uint64_t seed, int max_iter, int32_t *d_labels,
                                int *h_iters, void *d_scratch, size_t scratch_bytes, void *stream);

sped_status sped_cluster_scratch_size(int64_t n, int k, int n_clusters, size_t *bytes);

/* ------------------------------------------------------------------------------------
 * Batched: many independent graphs solved in one persistent launch (the stochastic-block
 * workloads of Section 5.4 at scale). The graphs are given as one block-diagonal CSR: graph g
 * owns rows [node_off[g], node_off[g+1]) and its columns stay in that range (global ids).
 * Each CTA takes whole graphs from a work list ordered by decreasing size and runs complete
 * mu-EG steps on them with the limit form (I - s_g L_g)^l, s_g from the automatic rule of
 * sped_set_polynomial applied to each graph's own spectral bound. No CTA waits on another;
 * one call is a memset plus one kernel launch, so it can be captured in a CUDA graph.
 * ------------------------------------------------------------------------------------ */
typedef struct sped_batch sped_batch;

sped_status sped_batch_workspace_size(int64_t n_graphs, size_t *bytes);

/* h_node_off: host, n_graphs+1 offsets (node_off[0] = 0, every graph non-empty). degree: odd l.
 * check != 0 verifies that columns stay inside their graph, rows sorted, no self loops.
 * Synchronises the stream. */
sped_status sped_batch_create(int64_t n_graphs, const int64_t *h_node_off,
                              const int32_t *d_row_ptr, const int32_t *d_col_idx,
                              const float *d_w, int degree, int check, void *d_workspace,
                              size_t ws_bytes, void *stream, sped_batch **out);

void sped_batch_destroy(sped_batch *b);

/* Per-graph limit-form scale s_g (host, n_graphs doubles). */
sped_status sped_batch_scale(const sped_batch *b, double *h_scale, int capacity);

sped_status sped_batch_scratch_size(const sped_batch *b, int k, sped_dtype chain_t,
                                    size_t *bytes);

/* `steps` mu-EG steps (Section 5.1) on every graph. V: F32, n_total x ld, ld >= 8 (k <= 8) or
 * ld >= 16 (k <= 16), 16-byte aligned, updated in place. chain_t: BF16 or F32 storage of the
 * intermediate products (F32 accumulation). d_ritz: n_graphs x k doubles, the Rayleigh
 * quotients of each graph's operator before its last update. */
sped_status sped_batch_eig_steps(const sped_batch *b, int steps, double eta, sped_dtype chain_t,
                                 float *d_V, int k, int ld, double *d_ritz, void *d_scratch,
                                 size_t scratch_bytes, void *stream);

/* Schedule of the batched launch: threads per CTA (128, 256 or 512; a thread per row, so small
 * graphs idle fewer lanes in smaller CTAs) and CTAs per SM (how many graphs are in flight).
 * Default 512 threads, 2 CTAs per SM. sped_batch_autotune times one solver step (eta = 1) per
 * candidate {512,2} {512,4} {256,4} {256,8} {128,8} {128,16} on a copy of d_V (V itself is not
 * changed), keeps the fastest in the batch handle and in a per-process table keyed by the
 * batch's shape (graphs, nodes, entries, degree, weighted, k, chain dtype, device); a later
 * batch of the same shape takes it from there (report->cached = 1). Synchronises `stream`.
 * Scratch: sped_batch_autotune_scratch_size bytes (256-byte aligned). */
typedef struct {
    int threads;       /* chosen threads per CTA                                 */
    int ctas_per_sm;   /* chosen CTAs per SM                                     */
    int cached;        /* 1: taken from the per-process table, nothing was timed */
    int n_candidates;  /* entries of ms[] filled                                 */
    double ms[8];      /* one solver step per candidate, in the order above      */
} sped_batch_tune_report;

sped_status sped_batch_set_schedule(sped_batch *b, int threads, int ctas_per_sm);
sped_status sped_batch_autotune_scratch_size(const sped_batch *b, int k, sped_dtype chain_t,
                                             size_t *bytes);
sped_status sped_batch_autotune(sped_batch *b, int k, sped_dtype chain_t, const float *d_V,
                                int ld, void *d_scratch, size_t scratch_bytes, void *stream,
                                sped_batch_tune_report *report);

/* ------------------------------------------------------------------------------------
 * Differentiable utilities (the solver family of Section 5.1 as a loss): with H = V^T M V
 * (k x k, e.g. the block H = G[0:k, k:2k] of sped_gram(V, M V), ldh = 2k),
 *   u_i = H_ii - sum_{j<i} H_ij^2 / H_jj.
 * d_g (k doubles, may be NULL): weights of the loss sum_i g_i u_i; d_Hbar (k x k, row-major,
 * needs d_g) receives d(sum g_i u_i)/dH with every entry H_ij treated as independent; d_S
 * (k x k, may be NULL) receives the detached-parents coefficients: du_i/dv_i (v_j, j < i,
 * held fixed) = sum_j y_j S[j][i]. Any output may be NULL. k <= 32, one CTA, FP64.
 * ------------------------------------------------------------------------------------ */
sped_status sped_eg_utilities(int k, const double *d_H, int ldh, const double *d_g, double *d_u,
                              double *d_Hbar, double *d_S, void *stream);

/* Out = A P + B Q for n x k blocks (F32 or F64, type t) and k x k row-major FP64 matrices
 * (Out[r][i] = sum_j A[r][j] P[j][i] + B[r][j] Q[j][i]); d_B may be NULL. Out must not
 * overlap A or B. k <= 40. */
sped_status sped_block_combine(int64_t n, int k, const void *d_A, int lda, const double *d_P,
                               const void *d_B, int ldb, const double *d_Q, void *d_Out, int ldo,
                               sped_dtype t, void *stream);

/* Edge-weight gradient of f(H), H = V^T M V, for the limit form M = B^l, B = I - sL (V fixed):
 *   df/dw_e = -s sum_{t=0}^{l-1} (x_e^T B^t V) Hbar (x_e^T B^{l-1-t} V)^T,
 * x_e the incidence row of undirected edge e (dL/dw_e = x_e x_e^T). d_HbarT: k x k row-major
 * FP64 holding Hbar transposed (d_HbarT[j*k+i] = Hbar[i][j]). d_grad: n_edges doubles, edge
 * order of sped_graph_edges. The chains B^t V and B^u V Hbar^T are kept at every
 * ceil(sqrt(l))-th step and recomputed between, so scratch holds about 2 sqrt(l) blocks.
 * V: F32 or F64 (the chains and the SDDMM run in that type, accumulated in FP64). */
sped_status sped_edge_grad(const sped_graph *g, const void *d_V, sped_dtype v_t, int k, int ld,
                           const double *d_HbarT, double *d_grad, void *d_scratch,
                           size_t scratch_bytes, void *stream);

sped_status sped_edge_grad_scratch_size(const sped_graph *g, int k, sped_dtype v_t,
                                        size_t *bytes);

/* ------------------------------------------------------------------------------------ */
const char *sped_last_error(void);
const char *sped_version(void);

#ifdef __cplusplus
}
#endif

#endif /* SPED_H */
