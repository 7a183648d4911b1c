// Hard clustering on the rows of the eigenvector block (Sections 1 and 2.1: k-means on the
// bottom-k embedding). k-means++ seeding drawn from Philox4x32-10, then Lloyd iterations in FP64.
// Distances sum (x_d - m_d)^2 in dimension order; ties go to the lowest centroid; an empty
// cluster restarts at the point farthest from its centroid (lowest index); labels are renumbered
// by first occurrence in row order.
#include <algorithm>
#include <cmath>
#include <numeric>
#include <vector>

#include "sped_internal.cuh"

namespace sped {

constexpr int KM_THREADS = 256;
constexpr int KM_MAXK = 32;
constexpr int KM_MAXC = 64;
constexpr uint32_t KM_TAG = 0x6B6D;

template <typename T>
__device__ __forceinline__ double dist2(const T *x, const double *c, int k) {
    double s = 0.0;
    for (int d = 0; d < k; ++d) {
        double t = cvt<double>(x[d]) - c[d];
        s += t * t;
    }
    return s;
}

template <typename T>
__global__ void k_km_first(const T *V, int64_t n, int k, int ld, uint64_t seed, double *centers) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    WordStream s(seed, 0u, 0u, KM_TAG);
    int64_t i = (int64_t)s.bounded((uint32_t)n);
    for (int d = 0; d < k; ++d) centers[d] = cvt<double>(V[i * ld + d]);
}

__device__ __forceinline__ double block_sum(double v, double *sh) {
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) sh[threadIdx.x] += sh[threadIdx.x + o];
        __syncthreads();
    }
    double r = sh[0];
    __syncthreads();
    return r;
}

// D2[i] = min(D2[i], ||x_i - centre c||^2) (first call initialises); per-block sums.
template <typename T>
__global__ void k_km_d2(const T *V, int64_t n, int k, int ld, const double *centers, int c,
                        double *D2, double *bsum) {
    __shared__ double sh[KM_THREADS];
    __shared__ double cc[KM_MAXK];
    if ((int)threadIdx.x < k) cc[threadIdx.x] = centers[c * k + threadIdx.x];
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double v = 0.0;
    if (i < n) {
        double d = dist2(V + i * ld, cc, k);
        v = (c == 0) ? d : fmin(D2[i], d);
        D2[i] = v;
    }
    double s = block_sum(v, sh);
    if (threadIdx.x == 0) bsum[blockIdx.x] = s;
}

// pick centre c: first row whose running sum of D2 exceeds u * total
template <typename T>
__global__ void k_km_pick(const T *V, int64_t n, int k, int ld, const double *D2,
                          const double *bsum, int64_t nblocks, uint64_t seed, int c,
                          double *centers) {
    if (threadIdx.x != 0) return;
    uint2 key = make_uint2((uint32_t)seed, (uint32_t)(seed >> 32));
    uint4 wv = philox4x32_10(make_uint4((uint32_t)c, 0u, 0u, KM_TAG), key);
    double u = ((double)wv.x + 0.5) * (1.0 / 4294967296.0);
    double total = 0.0;
    for (int64_t b = 0; b < nblocks; ++b) total += bsum[b];
    double target = u * total;
    double cum = 0.0;
    int64_t pick = n - 1;
    for (int64_t b = 0; b < nblocks; ++b) {
        if (cum + bsum[b] > target) {
            int64_t i0 = b * KM_THREADS, i1 = i0 + KM_THREADS < n ? i0 + KM_THREADS : n;
            for (int64_t i = i0; i < i1; ++i) {
                cum += D2[i];
                if (cum > target) {
                    pick = i;
                    break;
                }
            }
            break;
        }
        cum += bsum[b];
    }
    for (int d = 0; d < k; ++d) centers[c * k + d] = cvt<double>(V[pick * ld + d]);
}

// Lloyd assignment: label = argmin distance (lowest index on ties); sums and counts per cluster.
template <typename T>
__global__ void k_km_assign(const T *V, int64_t n, int k, int ld, const double *centers, int K,
                            int32_t *labels, int first_iter, double *mind, double *sums,
                            int *counts, int *changed) {
    __shared__ double sc[KM_MAXC * KM_MAXK];
    __shared__ double ssum[KM_MAXC * KM_MAXK];
    __shared__ int scnt[KM_MAXC];
    __shared__ int schg;
    for (int e = threadIdx.x; e < K * k; e += blockDim.x) {
        sc[e] = centers[e];
        ssum[e] = 0.0;
    }
    for (int e = threadIdx.x; e < K; e += blockDim.x) scnt[e] = 0;
    if (threadIdx.x == 0) schg = 0;
    __syncthreads();
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) {
        const T *x = V + i * ld;
        int best = 0;
        double bd = dist2(x, sc, k);
        for (int c = 1; c < K; ++c) {
            double d = dist2(x, sc + c * k, k);
            if (d < bd) {
                bd = d;
                best = c;
            }
        }
        mind[i] = bd;
        if (first_iter || labels[i] != best) atomicAdd(&schg, 1);
        labels[i] = best;
        atomicAdd(&scnt[best], 1);
        for (int d = 0; d < k; ++d) atomicAdd(&ssum[best * k + d], cvt<double>(x[d]));
    }
    __syncthreads();
    for (int e = threadIdx.x; e < K * k; e += blockDim.x)
        if (ssum[e] != 0.0) atomicAdd(&sums[e], ssum[e]);
    for (int e = threadIdx.x; e < K; e += blockDim.x)
        if (scnt[e]) atomicAdd(&counts[e], scnt[e]);
    if (threadIdx.x == 0 && schg) atomicAdd(changed, schg);
}

__global__ void k_km_means(int K, int k, const double *sums, const int *counts, double *centers) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= K * k) return;
    int c = e / k;
    if (counts[c] > 0) centers[e] = sums[e] / (double)counts[c];
}

// index of the largest mind (lowest index on ties), single block
__global__ void k_km_argmax(const double *mind, int64_t n, int64_t *out) {
    __shared__ double sv[KM_THREADS];
    __shared__ int64_t si[KM_THREADS];
    double bv = -1.0;
    int64_t bi = 0;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x)
        if (mind[i] > bv) {
            bv = mind[i];
            bi = i;
        }
    sv[threadIdx.x] = bv;
    si[threadIdx.x] = bi;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            double v2 = sv[threadIdx.x + o];
            int64_t i2 = si[threadIdx.x + o];
            if (v2 > sv[threadIdx.x] || (v2 == sv[threadIdx.x] && i2 < si[threadIdx.x])) {
                sv[threadIdx.x] = v2;
                si[threadIdx.x] = i2;
            }
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = si[0];
}

template <typename T>
__global__ void k_km_copy_row(const T *V, int k, int ld, const int64_t *idx, int c,
                              double *centers) {
    int d = threadIdx.x;
    if (d < k) centers[c * k + d] = cvt<double>(V[(*idx) * ld + d]);
}

__global__ void k_km_first_occ(const int32_t *labels, int64_t n, int *first) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) atomicMin(&first[labels[i]], (int)i);
}

__global__ void k_km_relabel(int32_t *labels, int64_t n, const int *remap) {
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) labels[i] = remap[labels[i]];
}

struct KmLayout {
    size_t centers, sums, D2, bsum, counts, changed, first, remap, idx, total;
};

static KmLayout km_layout(int64_t n, int k, int K) {
    KmLayout L;
    ScratchPlan p;
    int64_t nb = (n + KM_THREADS - 1) / KM_THREADS;
    auto put = [&](size_t &off, size_t bytes) {
        p.used = align_up(p.used, 256);
        off = p.used;
        p.add(bytes);
    };
    put(L.centers, sizeof(double) * K * k);
    put(L.sums, sizeof(double) * K * k);
    put(L.D2, sizeof(double) * n);
    put(L.bsum, sizeof(double) * nb);
    put(L.counts, sizeof(int) * K);
    put(L.changed, sizeof(int));
    put(L.first, sizeof(int) * K);
    put(L.remap, sizeof(int) * K);
    put(L.idx, sizeof(int64_t));
    L.total = p.total();
    return L;
}

template <typename T>
static sped_status run_kmeans(const T *V, int64_t n, int k, int ld, int K, uint64_t seed,
                              int max_iter, int32_t *labels, int *h_iters, char *base, KmLayout L,
                              cudaStream_t st) {
    double *centers = (double *)(base + L.centers), *sums = (double *)(base + L.sums);
    double *D2 = (double *)(base + L.D2), *bsum = (double *)(base + L.bsum);
    int *counts = (int *)(base + L.counts), *changed = (int *)(base + L.changed);
    int *first = (int *)(base + L.first), *remap = (int *)(base + L.remap);
    int64_t *idx = (int64_t *)(base + L.idx);
    const int64_t nb = (n + KM_THREADS - 1) / KM_THREADS;
    k_km_first<T><<<1, 1, 0, st>>>(V, n, k, ld, seed, centers);
    for (int c = 1; c < K; ++c) {
        k_km_d2<T><<<(unsigned)nb, KM_THREADS, 0, st>>>(V, n, k, ld, centers, c - 1, D2, bsum);
        k_km_pick<T><<<1, 32, 0, st>>>(V, n, k, ld, D2, bsum, nb, seed, c, centers);
    }
    SPED_CHECK_LAUNCH("kmeans seeding");
    int iters = 0;
    std::vector<int> hc(K);
    for (int it = 0; it < max_iter; ++it) {
        SPED_CUDA(cudaMemsetAsync(sums, 0, sizeof(double) * K * k, st));
        SPED_CUDA(cudaMemsetAsync(counts, 0, sizeof(int) * K, st));
        SPED_CUDA(cudaMemsetAsync(changed, 0, sizeof(int), st));
        k_km_assign<T><<<(unsigned)nb, KM_THREADS, 0, st>>>(V, n, k, ld, centers, K, labels,
                                                          it == 0, D2, sums, counts, changed);
        SPED_CHECK_LAUNCH("k_km_assign");
        int hchg = 0;
        SPED_CUDA(cudaMemcpyAsync(&hchg, changed, sizeof(int), cudaMemcpyDeviceToHost, st));
        SPED_CUDA(cudaMemcpyAsync(hc.data(), counts, sizeof(int) * K, cudaMemcpyDeviceToHost, st));
        SPED_CUDA(cudaStreamSynchronize(st));
        iters = it + 1;
        if (it > 0 && hchg == 0) break;
        k_km_means<<<(K * k + 255) / 256, 256, 0, st>>>(K, k, sums, counts, centers);
        bool empty = false;
        for (int c = 0; c < K; ++c) empty |= hc[c] == 0;
        if (empty) {
            k_km_argmax<<<1, KM_THREADS, 0, st>>>(D2, n, idx);
            for (int c = 0; c < K; ++c)
                if (hc[c] == 0) k_km_copy_row<T><<<1, KM_MAXK, 0, st>>>(V, k, ld, idx, c, centers);
        }
        SPED_CHECK_LAUNCH("kmeans update");
    }
    // canonical relabel by first occurrence
    std::vector<int> init(K, INT32_MAX);
    SPED_CUDA(cudaMemcpyAsync(first, init.data(), sizeof(int) * K, cudaMemcpyHostToDevice, st));
    k_km_first_occ<<<(unsigned)nb, KM_THREADS, 0, st>>>(labels, n, first);
    std::vector<int> hf(K);
    SPED_CUDA(cudaMemcpyAsync(hf.data(), first, sizeof(int) * K, cudaMemcpyDeviceToHost, st));
    SPED_CUDA(cudaStreamSynchronize(st));
    std::vector<int> order(K);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return hf[a] < hf[b]; });
    std::vector<int> rm(K);
    for (int r = 0; r < K; ++r) rm[order[r]] = r;
    SPED_CUDA(cudaMemcpyAsync(remap, rm.data(), sizeof(int) * K, cudaMemcpyHostToDevice, st));
    k_km_relabel<<<(unsigned)nb, KM_THREADS, 0, st>>>(labels, n, remap);
    SPED_CHECK_LAUNCH("k_km_relabel");
    SPED_CUDA(cudaStreamSynchronize(st));
    if (h_iters) *h_iters = iters;
    return SPED_OK;
}

}  // namespace sped

using namespace sped;

extern "C" {

sped_status sped_cluster_scratch_size(int64_t n, int k, int n_clusters, size_t *bytes) {
    if (!bytes || n < 1 || k < 1 || n_clusters < 1)
        return fail(SPED_ERR_INVALID_ARG, "cluster_scratch_size");
    *bytes = km_layout(n, k, n_clusters).total;
    return SPED_OK;
}

sped_status sped_cluster_assign(const void *d_V, sped_dtype v_t, int64_t n, int k, int ld,
                                int n_clusters, uint64_t seed, int max_iter, int32_t *d_labels,
                                int *h_iters, void *d_scratch, size_t scratch_bytes,
                                void *stream) {
    if (!d_V || !d_labels) return fail(SPED_ERR_INVALID_ARG, "cluster_assign: null");
    if (!dtype_valid(v_t) || n < 1 || k < 1 || ld < k)
        return fail(SPED_ERR_INVALID_ARG, "cluster_assign: bad layout");
    if (k > KM_MAXK || n_clusters < 1 || n_clusters > KM_MAXC || n_clusters > n)
        return fail(SPED_ERR_UNSUPPORTED, "cluster_assign: k <= %d, 1 <= clusters <= min(%d, n)",
                    KM_MAXK, KM_MAXC);
    if (n >= INT32_MAX) return fail(SPED_ERR_UNSUPPORTED, "cluster_assign: n too large");
    if (max_iter < 1) return fail(SPED_ERR_INVALID_ARG, "cluster_assign: max_iter < 1");
    KmLayout L = km_layout(n, k, n_clusters);
    if (!d_scratch || scratch_bytes < L.total || ((uintptr_t)d_scratch) % 256)
        return fail(SPED_ERR_SCRATCH, "cluster_assign: scratch needs %zu bytes", L.total);
    cudaStream_t st = as_stream(stream);
    char *base = (char *)d_scratch;
    switch (v_t) {
    case SPED_F64:
        return run_kmeans<double>((const double *)d_V, n, k, ld, n_clusters, seed, max_iter,
                                  d_labels, h_iters, base, L, st);
    case SPED_F32:
        return run_kmeans<float>((const float *)d_V, n, k, ld, n_clusters, seed, max_iter,
                                 d_labels, h_iters, base, L, st);
    default:
        return run_kmeans<__nv_bfloat16>((const __nv_bfloat16 *)d_V, n, k, ld, n_clusters, seed,
                                         max_iter, d_labels, h_iters, base, L, st);
    }
}

}  // extern "C"
