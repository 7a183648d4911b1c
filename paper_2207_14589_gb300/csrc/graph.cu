// Graph set-up (operator step of the hot path): CSR validation, reverse-entry map, undirected
// edge numbering, degrees and the spectral bound; polynomial selection (Table 2).
//
// Paper: Section 2 (L = D - A, incidence rows x_e), end of Section 2.1 (weighted L = X^T W X),
// Section 5.4 (lambda_max <= 2 max degree), Table 2 (transforms, l odd), Eq. reveig.
#include <cmath>
#include <cstring>
#include <string>

#include "sped_internal.cuh"

namespace sped {

static thread_local char g_err[1024] = "";

void set_error(const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
}

sped_status fail(sped_status st, const char *fmt, ...) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return st;
}

sped_status cuda_fail(cudaError_t e, const char *where) {
    snprintf(g_err, sizeof(g_err), "%s: %s (%s)", where, cudaGetErrorString(e),
             cudaGetErrorName(e));
    return SPED_ERR_CUDA;
}

int device_sm_count() {
    static int cached[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) return 148;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
        cached[dev] = v > 0 ? v : 148;
    }
    return cached[dev];
}

sped_status check_layout(const void *p, sped_dtype t, int k, int ld, const char *name) {
    if (!dtype_valid(t)) return fail(SPED_ERR_INVALID_ARG, "%s: unknown dtype %d", name, (int)t);
    if (p == nullptr) return fail(SPED_ERR_INVALID_ARG, "%s: null pointer", name);
    if (k < 1) return fail(SPED_ERR_INVALID_ARG, "%s: k=%d < 1", name, k);
    if (ld < k) return fail(SPED_ERR_INVALID_ARG, "%s: ld=%d < k=%d", name, ld, k);
    if (((uintptr_t)p) % 16 != 0)
        return fail(SPED_ERR_INVALID_ARG, "%s: base pointer not 16-byte aligned", name);
    if ((ld * dtype_size(t)) % 16 != 0)
        return fail(SPED_ERR_INVALID_ARG, "%s: ld*sizeof=%zu bytes is not a multiple of 16",
                    name, ld * dtype_size(t));
    return SPED_OK;
}

// ---------------------------------------------------------------------------------------
// device-wide exclusive scan of int32 (n elements; data[n] receives the total when
// `with_total`), three passes with per-block sums in `bsum`.
// ---------------------------------------------------------------------------------------
constexpr int SCAN_BLOCK = 1024;

__device__ __forceinline__ int block_exclusive_scan(int v, int *sh, int *total) {
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[wid] = x;
    __syncthreads();
    if (wid == 0) {
        int s = (lane < (int)(blockDim.x >> 5)) ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        sh[lane] = s;
    }
    __syncthreads();
    int incl = x + (wid > 0 ? sh[wid - 1] : 0);
    if (total) *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return incl - v;
}

__global__ void k_scan_blocks(int32_t *data, int64_t n, int32_t *bsum) {
    __shared__ int sh[32];
    int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    int v = i < n ? data[i] : 0;
    int tot;
    int ex = block_exclusive_scan(v, sh, &tot);
    if (i < n) data[i] = ex;
    if (threadIdx.x == 0) bsum[blockIdx.x] = tot;
}

__global__ void k_scan_sums(int32_t *bsum, int64_t nb, int32_t *total_out) {
    __shared__ int sh[32];
    int carry = 0;
    for (int64_t base = 0; base < nb; base += SCAN_BLOCK) {
        int64_t i = base + threadIdx.x;
        int v = i < nb ? bsum[i] : 0;
        int tot;
        int ex = block_exclusive_scan(v, sh, &tot);
        if (i < nb) bsum[i] = ex + carry;
        carry += tot;
    }
    if (threadIdx.x == 0 && total_out) *total_out = carry;
}

__global__ void k_scan_add(int32_t *data, int64_t n, const int32_t *bsum) {
    int64_t i = (int64_t)blockIdx.x * SCAN_BLOCK + threadIdx.x;
    if (i < n) data[i] += bsum[blockIdx.x];
}

static size_t scan_sums_elems(int64_t n) { return (size_t)((n + SCAN_BLOCK - 1) / SCAN_BLOCK) + 1; }

// exclusive scan of data[0..n); data[n] = total
static sped_status exclusive_scan(int32_t *data, int64_t n, int32_t *bsum, cudaStream_t st) {
    int64_t nb = (n + SCAN_BLOCK - 1) / SCAN_BLOCK;
    if (nb == 0) {
        SPED_CUDA(cudaMemsetAsync(data, 0, sizeof(int32_t), st));
        return SPED_OK;
    }
    k_scan_blocks<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(data, n, bsum);
    k_scan_sums<<<1, SCAN_BLOCK, 0, st>>>(bsum, nb, data + n);
    k_scan_add<<<(unsigned)nb, SCAN_BLOCK, 0, st>>>(data, n, bsum);
    SPED_CHECK_LAUNCH("exclusive_scan");
    return SPED_OK;
}

// ---------------------------------------------------------------------------------------
// set-up kernels
// ---------------------------------------------------------------------------------------
enum : int {
    CSR_BAD_ROWPTR = 1,
    CSR_BAD_COL = 2,
    CSR_SELF_LOOP = 4,
    CSR_UNSORTED = 8,
    CSR_ASYMMETRIC = 16,
    CSR_WEIGHT_ASYM = 32,
    CSR_BAD_WEIGHT = 64
};

struct SetupStats {
    int err;
    int bad_row;
    int max_deg;
    int pad;
    unsigned long long max_wdeg_bits;  // non-negative doubles order like their bit patterns
};

// Maximum degree and maximum weighted degree (as the bit patterns of non-negative doubles, which
// order like the values) over a warp, then one atomic each from lane 0; every lane of the warp
// takes part (rows past n contribute zeros).
__device__ __forceinline__ void warp_max_to(int deg, unsigned long long wbits, SetupStats *stats) {
    for (int o = 16; o > 0; o >>= 1) {
        deg = max(deg, __shfl_xor_sync(0xffffffffu, deg, o));
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, wbits, o);
        wbits = ob > wbits ? ob : wbits;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMax(&stats->max_deg, deg);
        atomicMax(&stats->max_wdeg_bits, wbits);
    }
}

__global__ void k_check_rowptr(int64_t n, int64_t nnz, const int32_t *rp, SetupStats *stats) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r > n) return;
    int v = rp[r];
    bool bad = v < 0 || v > nnz;
    if (r == 0 && v != 0) bad = true;
    if (r == n && v != nnz) bad = true;
    if (r < n && rp[r + 1] < v) bad = true;
    if (bad) {
        atomicOr(&stats->err, CSR_BAD_ROWPTR);
        atomicMin(&stats->bad_row, (int)r);
    }
}

// Per row: column checks (checked mode), degree statistics and the number of upper entries.
__global__ void k_rows(int64_t n, const int32_t *rp, const int32_t *ci, const float *w, int check,
                       int32_t *cnt_up, SetupStats *stats) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int deg = 0;
    unsigned long long wbits = 0ull;
    if (r < n) {
        int p0 = rp[r], p1 = rp[r + 1];
        int up = 0, err = 0;
        double wd = 0.0;
        int prev = -1;
        for (int p = p0; p < p1; ++p) {
            int c = ci[p];
            if (check) {
                if (c < 0 || c >= n) err |= CSR_BAD_COL;
                if (c == r) err |= CSR_SELF_LOOP;
                if (c <= prev) err |= CSR_UNSORTED;
            }
            prev = c;
            if (c > r) ++up;
            if (w) {
                float x = w[p];
                if (check && !(x >= 0.0f && isfinite(x))) err |= CSR_BAD_WEIGHT;
                wd += (double)x;
            } else {
                wd += 1.0;
            }
        }
        cnt_up[r] = up;
        if (err) {
            atomicOr(&stats->err, err);
            atomicMin(&stats->bad_row, (int)r);
        }
        deg = p1 - p0;
        wbits = (unsigned long long)__double_as_longlong(wd);
    }
    // the warp's maxima first, then one atomic per warp instead of one per row
    warp_max_to(deg, wbits, stats);
}

// Reverse-entry map by binary search in the neighbour's row; symmetric-weight check.
__global__ void k_reverse(int64_t n, int64_t nnz, const int32_t *rp, const int32_t *ci,
                          const float *w, int32_t *rev, int check, SetupStats *stats) {
    int64_t r = (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
    int lane = threadIdx.x & 31;
    if (r >= n) return;
    int p0 = rp[r], p1 = rp[r + 1];
    for (int p = p0 + lane; p < p1; p += 32) {
        int c = ci[p];
        int lo = rp[c], hi = rp[c + 1];
        int found = -1;
        while (lo < hi) {
            int mid = (lo + hi) >> 1;
            int v = ci[mid];
            if (v < r) lo = mid + 1;
            else hi = mid;
        }
        if (lo < rp[c + 1] && ci[lo] == r) found = lo;
        rev[p] = found < 0 ? p : found;
        if (found < 0) {
            atomicOr(&stats->err, CSR_ASYMMETRIC);
            atomicMin(&stats->bad_row, (int)r);
        } else if (check && w && w[p] != w[found]) {
            atomicOr(&stats->err, CSR_WEIGHT_ASYM);
            atomicMin(&stats->bad_row, (int)r);
        }
    }
}

// Undirected edge ids: upper entries numbered in CSR order; lower entries take the id of
// their reverse entry.
__global__ void k_edges(int64_t n, const int32_t *rp, const int32_t *ci, const int32_t *rev,
                        const int32_t *eoff, int32_t *eid, int32_t *edge_p, int32_t *edge_a,
                        int2 *edge_ab) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (r >= n) return;
    int p0 = rp[r], p1 = rp[r + 1];
    int e = eoff[r];
    for (int p = p0; p < p1; ++p) {
        int c = ci[p];
        if (c > r) {
            eid[p] = e;
            eid[rev[p]] = e;
            edge_p[e] = p;
            edge_a[e] = (int)r;
            edge_ab[e] = make_int2((int)r, c);
            ++e;
        }
    }
}

__global__ void k_edge_weights(int64_t nnz, const int32_t *eid, const float *w_edge, float *w_out) {
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p < nnz) w_out[p] = w_edge[eid[p]];
}

__global__ void k_wdeg_max(int64_t n, const int32_t *rp, const float *w, SetupStats *stats) {
    int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long wbits = 0ull;
    if (r < n) {
        double s = 0.0;
        for (int p = rp[r]; p < rp[r + 1]; ++p) s += (double)w[p];
        wbits = (unsigned long long)__double_as_longlong(s);
    }
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ob = __shfl_xor_sync(0xffffffffu, wbits, o);
        wbits = ob > wbits ? ob : wbits;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(&stats->max_wdeg_bits, wbits);
}

__global__ void k_edge_ends(int64_t ne, const int32_t *ci, const int32_t *edge_p,
                            const int32_t *edge_a, int32_t *a_out, int32_t *b_out) {
    int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= ne) return;
    if (a_out) a_out[e] = edge_a[e];
    if (b_out) b_out[e] = ci[edge_p[e]];
}

static unsigned nblocks(int64_t n, int t) { return (unsigned)((n + t - 1) / t); }

struct WsLayout {
    size_t rev, eid, edge_p, edge_a, edge_ab, eoff, ws_w, bsum, stats, total;
};

static WsLayout ws_layout(int64_t n, int64_t nnz) {
    WsLayout L;
    ScratchPlan p;
    L.rev = p.used; p.add(sizeof(int32_t) * nnz); p.used = align_up(p.used, 256);
    L.eid = p.used; p.add(sizeof(int32_t) * nnz); p.used = align_up(p.used, 256);
    L.edge_p = p.used; p.add(sizeof(int32_t) * (nnz / 2 + 1)); p.used = align_up(p.used, 256);
    L.edge_a = p.used; p.add(sizeof(int32_t) * (nnz / 2 + 1)); p.used = align_up(p.used, 256);
    L.edge_ab = p.used; p.add(sizeof(int2) * (nnz / 2 + 1)); p.used = align_up(p.used, 256);
    L.eoff = p.used; p.add(sizeof(int32_t) * (n + 1)); p.used = align_up(p.used, 256);
    L.ws_w = p.used; p.add(sizeof(float) * nnz); p.used = align_up(p.used, 256);
    L.bsum = p.used; p.add(sizeof(int32_t) * scan_sums_elems(n + 1)); p.used = align_up(p.used, 256);
    L.stats = p.used; p.add(sizeof(SetupStats));
    L.total = p.total();
    return L;
}

static const char *csr_err_name(int e) {
    if (e & CSR_BAD_ROWPTR) return "row_ptr not monotone / out of [0, nnz] / ends != nnz";
    if (e & CSR_BAD_COL) return "column index out of range";
    if (e & CSR_SELF_LOOP) return "self loop";
    if (e & CSR_UNSORTED) return "columns not strictly increasing (duplicates or unsorted)";
    if (e & CSR_ASYMMETRIC) return "adjacency not symmetric";
    if (e & CSR_WEIGHT_ASYM) return "weights of (i,j) and (j,i) differ";
    if (e & CSR_BAD_WEIGHT) return "negative or non-finite weight";
    return "unknown";
}

static sped_status read_stats(SetupStats *d_stats, SetupStats *h, cudaStream_t st) {
    SPED_CUDA(cudaMemcpyAsync(h, d_stats, sizeof(SetupStats), cudaMemcpyDeviceToHost, st));
    SPED_CUDA(cudaStreamSynchronize(st));
    return SPED_OK;
}

}  // namespace sped

using namespace sped;

// ---------------------------------------------------------------------------------------
// polynomial resolution (host)
// ---------------------------------------------------------------------------------------
static double binom(int n, int k) {
    double r = 1.0;
    for (int i = 1; i <= k; ++i) r = r * (double)(n - k + i) / (double)i;
    return r;
}

static void resolve_power(Poly &P) {
    // power-basis coefficients of M = sum_j h_j (L + shift I)^j, or the limit form
    P.power.assign(P.ell + 1, 0.0);
    if (P.kind == SPED_POLY_LIMIT_EXP) {
        for (int i = 0; i <= P.ell; ++i) P.power[i] = binom(P.ell, i) * std::pow(-P.s, (double)i);
        return;
    }
    if (P.kind == SPED_POLY_SHIFT) {
        P.power[0] = P.lambda_star;
        P.power[1] = -1.0;
        return;
    }
    if (P.kind == SPED_POLY_CHEBYSHEV) {
        // T_j(al L + be) in powers of L by the three-term recurrence, summed with c_j
        const double al = 2.0 / (P.cheb_b - P.cheb_a), be = -(P.cheb_a + P.cheb_b) / (P.cheb_b - P.cheb_a);
        std::vector<double> t0(P.ell + 1, 0.0), t1(P.ell + 1, 0.0), t2(P.ell + 1, 0.0);
        t0[0] = 1.0;
        for (int i = 0; i <= P.ell; ++i) P.power[i] += P.cheb[0] * t0[i];
        if (P.ell >= 1) {
            t1[0] = be;
            t1[1] = al;
            for (int i = 0; i <= P.ell; ++i) P.power[i] += P.cheb[1] * t1[i];
        }
        for (int j = 1; j < P.ell; ++j) {
            for (int i = 0; i <= P.ell; ++i)
                t2[i] = 2.0 * (be * t1[i] + (i > 0 ? al * t1[i - 1] : 0.0)) - t0[i];
            for (int i = 0; i <= P.ell; ++i) P.power[i] += P.cheb[j + 1] * t2[i];
            t0.swap(t1);
            t1.swap(t2);
        }
        return;
    }
    for (int i = 0; i <= P.ell; ++i) {
        double c = 0.0;
        for (int j = i; j <= P.ell; ++j)
            c += P.horner[j] * binom(j, i) * std::pow(P.shift, (double)(j - i));
        P.power[i] = c;
    }
}

extern "C" {

const char *sped_last_error(void) { return g_err; }

const char *sped_version(void) { return "sped-gb300 0.1 (sm_103a)"; }

sped_status sped_workspace_size(int64_t n, int64_t nnz, size_t *bytes) {
    if (!bytes || n < 0 || nnz < 0) return fail(SPED_ERR_INVALID_ARG, "workspace_size: bad args");
    if (n >= INT32_MAX || nnz >= INT32_MAX)
        return fail(SPED_ERR_UNSUPPORTED, "n and nnz must fit int32 indexing");
    *bytes = ws_layout(n, nnz).total;
    return SPED_OK;
}

sped_status sped_build_laplacian(int64_t n, int64_t nnz, const int32_t *d_row_ptr,
                                 const int32_t *d_col_idx, const float *d_w, void *d_workspace,
                                 size_t ws_bytes, int check, void *stream, sped_graph **out) {
    if (!out) return fail(SPED_ERR_INVALID_ARG, "build_laplacian: out is NULL");
    *out = nullptr;
    if (n < 1 || nnz < 0) return fail(SPED_ERR_INVALID_ARG, "build_laplacian: n=%lld nnz=%lld",
                                       (long long)n, (long long)nnz);
    if (n >= INT32_MAX || nnz >= INT32_MAX)
        return fail(SPED_ERR_UNSUPPORTED, "n and nnz must fit int32 indexing");
    if (!d_row_ptr || (nnz > 0 && !d_col_idx))
        return fail(SPED_ERR_INVALID_ARG, "build_laplacian: null CSR array");
    if (nnz % 2) return fail(SPED_ERR_BAD_CSR, "odd nnz cannot be a symmetric adjacency");
    if (((uintptr_t)d_col_idx) % 16 || ((uintptr_t)d_w) % 16 || ((uintptr_t)d_row_ptr) % 4)
        return fail(SPED_ERR_INVALID_ARG,
                    "build_laplacian: col_idx and w must be 16-byte aligned (row_ptr 4-byte)");
    WsLayout L = ws_layout(n, nnz);
    if (!d_workspace || ws_bytes < L.total || ((uintptr_t)d_workspace) % 256)
        return fail(SPED_ERR_SCRATCH, "build_laplacian: workspace needs %zu bytes, 256-aligned",
                    L.total);
    cudaStream_t st = as_stream(stream);
    char *ws = (char *)d_workspace;
    int32_t *rev = (int32_t *)(ws + L.rev), *eid = (int32_t *)(ws + L.eid);
    int32_t *edge_p = (int32_t *)(ws + L.edge_p), *edge_a = (int32_t *)(ws + L.edge_a);
    int2 *edge_ab = (int2 *)(ws + L.edge_ab);
    int32_t *eoff = (int32_t *)(ws + L.eoff), *bsum = (int32_t *)(ws + L.bsum);
    SetupStats *stats = (SetupStats *)(ws + L.stats);
    SetupStats h;
    memset(&h, 0, sizeof(h));
    h.bad_row = INT32_MAX;
    SPED_CUDA(cudaMemcpyAsync(stats, &h, sizeof(h), cudaMemcpyHostToDevice, st));
    if (check) {
        k_check_rowptr<<<nblocks(n + 1, 256), 256, 0, st>>>(n, nnz, d_row_ptr, stats);
        SPED_CHECK_LAUNCH("k_check_rowptr");
        SPED_TRY(read_stats(stats, &h, st));
        if (h.err) return fail(SPED_ERR_BAD_CSR, "invalid CSR: %s (row %d)", csr_err_name(h.err),
                               h.bad_row);
    }
    k_rows<<<nblocks(n, 256), 256, 0, st>>>(n, d_row_ptr, d_col_idx, d_w, check, eoff, stats);
    SPED_CHECK_LAUNCH("k_rows");
    if (check) {
        SPED_TRY(read_stats(stats, &h, st));
        if (h.err) return fail(SPED_ERR_BAD_CSR, "invalid CSR: %s (row %d)", csr_err_name(h.err),
                               h.bad_row);
    }
    k_reverse<<<nblocks(n, 8), 256, 0, st>>>(n, nnz, d_row_ptr, d_col_idx, d_w, rev, check, stats);
    SPED_CHECK_LAUNCH("k_reverse");
    SPED_TRY(exclusive_scan(eoff, n, bsum, st));
    SPED_TRY(read_stats(stats, &h, st));
    if (h.err) return fail(SPED_ERR_BAD_CSR, "invalid CSR: %s (row %d)", csr_err_name(h.err),
                           h.bad_row);
    int32_t n_edges = 0;
    SPED_CUDA(cudaMemcpyAsync(&n_edges, eoff + n, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    SPED_CUDA(cudaStreamSynchronize(st));
    if ((int64_t)n_edges * 2 != nnz)
        return fail(SPED_ERR_BAD_CSR, "upper entries %d != nnz/2", n_edges);
    k_edges<<<nblocks(n, 256), 256, 0, st>>>(n, d_row_ptr, d_col_idx, rev, eoff, eid, edge_p,
                                             edge_a, edge_ab);
    SPED_CHECK_LAUNCH("k_edges");
    SPED_CUDA(cudaStreamSynchronize(st));

    sped_graph *g = new sped_graph();
    cudaGetDevice(&g->device);
    g->n = n;
    g->nnz = nnz;
    g->n_edges = n_edges;
    g->rp = d_row_ptr;
    g->ci = d_col_idx;
    g->w = d_w;
    g->rev = rev;
    g->eid = eid;
    g->edge_p = edge_p;
    g->edge_a = edge_a;
    g->edge_ab = edge_ab;
    g->eoff = eoff;
    g->ws_w = (float *)(ws + L.ws_w);
    g->stats = stats;
    g->max_deg = h.max_deg;
    double mw;
    memcpy(&mw, &h.max_wdeg_bits, sizeof(double));
    g->max_wdeg = mw;
    g->lambda_bound = 2.0 * mw;
    g->poly.kind = SPED_POLY_SHIFT;
    g->poly.ell = 1;
    g->poly.lambda_star = g->lambda_bound;
    g->poly.horner = {g->lambda_bound, -1.0};
    resolve_power(g->poly);
    *out = g;
    return SPED_OK;
}

void sped_graph_destroy(sped_graph *g) { delete g; }

sped_status sped_graph_get_info(const sped_graph *g, sped_graph_info *info) {
    if (!g || !info) return fail(SPED_ERR_INVALID_ARG, "graph_get_info: null");
    info->n = g->n;
    info->nnz = g->nnz;
    info->n_edges = g->n_edges;
    info->max_degree = g->max_deg;
    info->max_wdegree = g->max_wdeg;
    info->lambda_bound = g->lambda_bound;
    info->weighted = g->w != nullptr;
    info->poly_kind = g->poly.kind;
    info->degree = g->poly.ell;
    info->scale_s = g->poly.s;
    info->shift = g->poly.shift;
    info->lambda_star = g->poly.lambda_star;
    return SPED_OK;
}

sped_status sped_graph_edges(const sped_graph *g, int32_t *d_edge_a, int32_t *d_edge_b,
                             void *stream) {
    if (!g) return fail(SPED_ERR_INVALID_ARG, "graph_edges: null graph");
    if (g->n_edges == 0 || (!d_edge_a && !d_edge_b)) return SPED_OK;
    k_edge_ends<<<nblocks(g->n_edges, 256), 256, 0, as_stream(stream)>>>(
        g->n_edges, g->ci, g->edge_p, g->edge_a, d_edge_a, d_edge_b);
    SPED_CHECK_LAUNCH("k_edge_ends");
    return SPED_OK;
}

sped_status sped_set_edge_weights(sped_graph *g, const float *d_w_edge, void *stream) {
    if (!g || !d_w_edge) return fail(SPED_ERR_INVALID_ARG, "set_edge_weights: null");
    cudaStream_t st = as_stream(stream);
    if (g->nnz > 0) {
        k_edge_weights<<<nblocks(g->nnz, 256), 256, 0, st>>>(g->nnz, g->eid, d_w_edge, g->ws_w);
        SPED_CHECK_LAUNCH("k_edge_weights");
    }
    g->w = g->ws_w;
    // spectral bound for the new weights (statistics slot of the workspace)
    SetupStats *d_stats = (SetupStats *)g->stats;
    SPED_CUDA(cudaMemsetAsync(d_stats, 0, sizeof(SetupStats), st));
    k_wdeg_max<<<nblocks(g->n, 256), 256, 0, st>>>(g->n, g->rp, g->w, d_stats);
    SPED_CHECK_LAUNCH("k_wdeg_max");
    SetupStats h;
    SPED_TRY(read_stats(d_stats, &h, st));
    double mw;
    memcpy(&mw, &h.max_wdeg_bits, sizeof(double));
    g->max_wdeg = mw;
    g->lambda_bound = 2.0 * mw;
    return SPED_OK;
}

sped_status sped_set_polynomial(sped_graph *g, sped_poly_kind kind, int degree, double scale_s,
                                double eps, const double *coeffs, double lambda_star) {
    if (!g) return fail(SPED_ERR_INVALID_ARG, "set_polynomial: null graph");
    if (degree < 1 || degree > 100000)
        return fail(SPED_ERR_INVALID_ARG, "set_polynomial: degree %d out of [1, 100000]", degree);
    Poly P;
    P.kind = kind;
    P.ell = degree;
    switch (kind) {
    case SPED_POLY_LIMIT_EXP: {
        if (degree % 2 == 0)
            return fail(SPED_ERR_INVALID_ARG,
                        "limit form needs an odd degree (monotone on the whole real line)");
        double s = scale_s;
        if (s == 0.0) {
            double lb = g->lambda_bound;
            s = (lb <= 0.0 || degree >= lb / 2.0) ? 1.0 / degree : 2.0 / lb;
        }
        if (!(s > 0.0) || !std::isfinite(s))
            return fail(SPED_ERR_INVALID_ARG, "limit form: scale must be positive");
        P.s = s;
        break;
    }
    case SPED_POLY_TAYLOR_EXP:
        P.horner.resize(degree + 1);
        {
            double f = 1.0;
            for (int i = 0; i <= degree; ++i) {
                if (i > 0) f *= (double)i;
                P.horner[i] = ((i % 2) ? -1.0 : 1.0) / f;
            }
        }
        P.shift = 0.0;
        break;
    case SPED_POLY_TAYLOR_LOG: {
        double e = eps == 0.0 ? 1e-3 : eps;
        if (!(e > 0.0)) return fail(SPED_ERR_INVALID_ARG, "taylor log: eps must be > 0");
        P.eps = e;
        P.shift = e - 1.0;
        double ls = lambda_star != 0.0 ? lambda_star : std::log(g->lambda_bound + e) + 1.0;
        P.lambda_star = ls;
        P.horner.assign(degree + 1, 0.0);
        P.horner[0] = ls;
        for (int i = 1; i <= degree; ++i) P.horner[i] = -((i % 2) ? 1.0 : -1.0) / (double)i;
        break;
    }
    case SPED_POLY_MONOMIAL:
        if (!coeffs) return fail(SPED_ERR_INVALID_ARG, "monomial: coeffs is NULL");
        P.horner.assign(coeffs, coeffs + degree + 1);
        for (double c : P.horner)
            if (!std::isfinite(c)) return fail(SPED_ERR_INVALID_ARG, "monomial: non-finite c");
        P.shift = 0.0;
        break;
    case SPED_POLY_SHIFT: {
        if (degree != 1) return fail(SPED_ERR_INVALID_ARG, "shift operator has degree 1");
        double ls = lambda_star != 0.0 ? lambda_star : g->lambda_bound;
        P.lambda_star = ls;
        P.horner = {ls, -1.0};
        break;
    }
    case SPED_POLY_CHEBYSHEV: {
        if (!coeffs) return fail(SPED_ERR_INVALID_ARG, "chebyshev: coeffs is NULL");
        P.cheb.assign(coeffs, coeffs + degree + 1);
        for (double c : P.cheb)
            if (!std::isfinite(c)) return fail(SPED_ERR_INVALID_ARG, "chebyshev: non-finite c");
        P.cheb_a = eps;
        P.cheb_b = lambda_star != 0.0 ? lambda_star : g->lambda_bound;
        if (!(P.cheb_b > P.cheb_a) || !std::isfinite(P.cheb_a) || !std::isfinite(P.cheb_b))
            return fail(SPED_ERR_INVALID_ARG, "chebyshev: interval [%g, %g] is empty", P.cheb_a,
                        P.cheb_b);
        break;
    }
    default:
        return fail(SPED_ERR_INVALID_ARG, "set_polynomial: unknown kind %d", (int)kind);
    }
    resolve_power(P);
    g->poly = P;
    return SPED_OK;
}

sped_status sped_get_power_coeffs(const sped_graph *g, double *h_out, int capacity) {
    if (!g || !h_out) return fail(SPED_ERR_INVALID_ARG, "get_power_coeffs: null");
    if (capacity < (int)g->poly.power.size())
        return fail(SPED_ERR_INVALID_ARG, "get_power_coeffs: need %zu", g->poly.power.size());
    for (size_t i = 0; i < g->poly.power.size(); ++i) h_out[i] = g->poly.power[i];
    return SPED_OK;
}

}  // extern "C"
