// sfc_locality.cu - section 5.2: the kNN locality histogram H_k and its skewness G1.
//
// For a set of centres (cloud points, given by original index) the kNN lists come from
// the octree's own search; a storage order then gives every point a position, and
// H_k(d) counts the (centre, neighbour) pairs |pos(centre) - pos(neighbour)| = d apart.
// G1 is the Fisher-Pearson skewness of that distribution, from two passes over the pairs
// (the mean first, then the central moments) in float64.  Computed on a small subset of
// centres for each candidate order, it picks the curve before the full index is built
// (choose_encoding).
#include <cuda_runtime.h>
#include <math.h>

#include "sfc_internal.cuh"

namespace sfc {

// rank[perm[p]] = p: the position of every original point in the handle's sorted order
__global__ void __launch_bounds__(256) k_invert_perm(const uint32_t* __restrict__ perm, int64_t n,
                                                     uint32_t* __restrict__ rank) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < n; p += stride)
        rank[perm[p]] = static_cast<uint32_t>(p);
}

// the coordinates of the centres (original ids) as float x3 queries; bit 0 of *bad for an
// id outside the cloud
__global__ void __launch_bounds__(256) k_gather_centres(const float4* __restrict__ pts, const uint32_t* __restrict__ at,
                                                        const int32_t* __restrict__ ids, int64_t m, int64_t n,
                                                        float* __restrict__ q, unsigned int* bad) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < m; i += stride) {
        const int32_t id = ids[i];
        float4 p = make_float4(0.f, 0.f, 0.f, 0.f);
        if (id >= 0 && id < n) p = pts[at ? at[id] : static_cast<uint32_t>(id)];
        else atomicOr(bad, 1u);
        q[3 * i] = p.x;
        q[3 * i + 1] = p.y;
        q[3 * i + 2] = p.z;
    }
}

// codes of another curve for the handle's points, with the handle's transform (section 4),
// written at each point's original index (so a stable sort breaks ties by that index)
template <int ENC>
__global__ void __launch_bounds__(256) k_order_codes(const float4* __restrict__ pts, int64_t n, float lx, float ly,
                                                     float lz, float s, uint64_t* __restrict__ keys,
                                                     uint32_t* __restrict__ ids) {
    __shared__ HilbertTables table;
    if (ENC == SFC_ENC_HILBERT) fill_hilbert_tables(table);
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t p = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; p < n; p += stride) {
        const float4 q = pts[p];
        const uint32_t cx = cell_of(q.x, lx, s), cy = cell_of(q.y, ly, s), cz = cell_of(q.z, lz, s);
        const uint32_t id = __float_as_uint(q.w);
        keys[id] = ENC == SFC_ENC_HILBERT ? hilbert_code(cx, cy, cz, table) : morton_code(cx, cy, cz);
        ids[id] = id;
    }
}

// Pass 1: the histogram (optional) and the sum of the distances; pass 2: the second and
// third central moments about the mean of pass 1.  Pairs with a padding neighbour (-1)
// are skipped.
template <bool PASS2>
__global__ void __launch_bounds__(256) k_locality_pairs(const int32_t* __restrict__ ids, int64_t m, int64_t n, int k,
                                                        const int32_t* __restrict__ nbr, const uint32_t* __restrict__ rank,
                                                        unsigned long long* __restrict__ hist, const double* mean,
                                                        double* __restrict__ acc) {
    double a0 = 0.0, a1 = 0.0;
    const double mu = PASS2 ? *mean : 0.0;
    const int64_t total = m * k;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t t = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; t < total; t += stride) {
        const int32_t j = nbr[t];
        if (j < 0) continue;
        const int32_t i = ids[t / k];
        if (i < 0 || i >= n) continue;  // reported by the gather
        const int64_t pi = rank ? rank[i] : i, pj = rank ? rank[j] : j;
        const int64_t d = pi > pj ? pi - pj : pj - pi;
        if (!PASS2) {
            if (hist) atomicAdd(&hist[d], 1ull);
            a0 += static_cast<double>(d);
            a1 += 1.0;
        } else {
            const double x = static_cast<double>(d) - mu;
            a0 += x * x;
            a1 += x * x * x;
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a0 += __shfl_xor_sync(0xffffffffu, a0, o);
        a1 += __shfl_xor_sync(0xffffffffu, a1, o);
    }
    if (lane_id() == 0) {
        atomicAdd(&acc[0], a0);
        atomicAdd(&acc[1], a1);
    }
}

__global__ void k_locality_mean(double* acc) {  // acc[0] = sum d, acc[1] = pairs -> acc[2] = mean
    acc[2] = acc[1] > 0.0 ? acc[0] / acc[1] : 0.0;
}

// the position of every original point under `order` (nullptr: the input order)
static sfc_status order_ranks(const Octree* t, int order, cudaStream_t s, Scratch& scratch, const uint32_t** rank,
                              unsigned int* fault) {
    *rank = nullptr;
    if (order == SFC_ENC_NONE) return SFC_OK;
    const int64_t n = t->n;
    uint32_t* r = nullptr;
    SFC_TRY(scratch.alloc(&r, n));
    const unsigned int grid = grid_for(n, 256, 152 * 16);
    const bool own = (t->enc == order) || (t->enc == SFC_ENC_NONE && order == SFC_ENC_MORTON);
    if (own) {  // the handle's permutation is that order
        SFC_LAUNCH("locality_rank", s, k_invert_perm, grid, 256, 0, t->perm, n, r);
    } else {
        uint64_t *k0, *k1;
        uint32_t *v0, *v1;
        SFC_TRY(scratch.alloc(&k0, n));
        SFC_TRY(scratch.alloc(&k1, n));
        SFC_TRY(scratch.alloc(&v0, n));
        SFC_TRY(scratch.alloc(&v1, n));
        if (order == SFC_ENC_HILBERT)
            SFC_LAUNCH("locality_codes", s, k_order_codes<SFC_ENC_HILBERT>, grid, 256, 0, t->pts, n, t->lo[0], t->lo[1],
                       t->lo[2], t->scale, k0, v0);
        else
            SFC_LAUNCH("locality_codes", s, k_order_codes<SFC_ENC_MORTON>, grid, 256, 0, t->pts, n, t->lo[0], t->lo[1],
                       t->lo[2], t->scale, k0, v0);
        SFC_TRY(radix_sort_pairs(k0, v0, k1, v1, n, s, scratch, fault));  // stable: equal codes by original index
        SFC_LAUNCH("locality_rank", s, k_invert_perm, grid, 256, 0, v0, n, r);
    }
    *rank = r;
    return SFC_OK;
}

}  // namespace sfc

extern "C" {

sfc_status knn_locality(sfc_octree h, const int32_t* centre_ids, int64_t n_centres, int32_t k, sfc_encoding order,
                        void* cuda_stream, uint64_t* hist, double* g1) {
    if (!h || k < 1 || n_centres < 0 || (n_centres > 0 && !centre_ids) || !g1) return SFC_ERR_INVALID;
    if (order != SFC_ENC_NONE && order != SFC_ENC_MORTON && order != SFC_ENC_HILBERT) return SFC_ERR_INVALID;
    if (k > sfc::kMaxK) return SFC_ERR_TOO_LARGE;
    if (n_centres > 0 && !sfc::is_device_ptr(centre_ids)) return SFC_ERR_NOT_DEVICE_PTR;
    if (hist && !sfc::is_device_ptr(hist)) return SFC_ERR_NOT_DEVICE_PTR;
    const sfc::Octree* t = &h->tree;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    *g1 = 0.0;
    if (hist && t->n > 0) SFC_CUDA(cudaMemsetAsync(hist, 0, sizeof(uint64_t) * t->n, s));
    if (n_centres == 0 || t->n == 0) return SFC_OK;
    sfc::Scratch scratch(s);
    // the centres' kNN lists, from the octree's own search
    uint32_t* at = nullptr;  // position of each original id in the handle's point array
    if (t->enc != SFC_ENC_NONE) {
        SFC_TRY(scratch.alloc(&at, t->n));
        SFC_LAUNCH("locality_rank", s, sfc::k_invert_perm, sfc::grid_for(t->n, 256, 152 * 16), 256, 0, t->perm, t->n,
                   at);
    }
    float* q = nullptr;
    int32_t* nbr = nullptr;
    float* d2 = nullptr;
    unsigned int* bad = nullptr;
    SFC_TRY(scratch.alloc(&q, 3 * n_centres));
    SFC_TRY(scratch.alloc(&nbr, n_centres * k));
    SFC_TRY(scratch.alloc(&d2, n_centres * k));
    SFC_TRY(scratch.alloc(&bad, 1));
    SFC_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned int), s));
    SFC_LAUNCH("locality_centres", s, sfc::k_gather_centres, sfc::grid_for(n_centres, 256, 152 * 16), 256, 0, t->pts,
               at, centre_ids, n_centres, t->n, q, bad);
    SFC_TRY(knn(h, q, n_centres, k, cuda_stream, nbr, d2));
    const uint32_t* rank = nullptr;
    SFC_TRY(sfc::order_ranks(t, order, s, scratch, &rank, bad));
    double* acc = nullptr;
    SFC_TRY(scratch.alloc(&acc, 5));
    SFC_CUDA(cudaMemsetAsync(acc, 0, sizeof(double) * 5, s));
    const unsigned int grid = sfc::grid_for(n_centres * k, 256, 152 * 8);
    SFC_LAUNCH("locality_pairs", s, sfc::k_locality_pairs<false>, grid, 256, 0, centre_ids, n_centres, t->n, k, nbr, rank,
               reinterpret_cast<unsigned long long*>(hist), nullptr, acc);
    SFC_LAUNCH("locality_mean", s, sfc::k_locality_mean, 1, 1, 0, acc);
    SFC_LAUNCH("locality_pairs", s, sfc::k_locality_pairs<true>, grid, 256, 0, centre_ids, n_centres, t->n, k, nbr, rank,
               nullptr, acc + 2, acc + 3);
    double h_acc[5];
    unsigned int hbad = 0;
    SFC_CUDA(cudaMemcpyAsync(h_acc, acc, sizeof h_acc, cudaMemcpyDeviceToHost, s));
    SFC_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof hbad, cudaMemcpyDeviceToHost, s));
    SFC_CUDA(cudaStreamSynchronize(s));
    if (hbad & sfc::kWaitTimedOut) return SFC_ERR_TIMEOUT;
    if (hbad) return SFC_ERR_INVALID;
    const double pairs = h_acc[1];
    const double m2 = pairs > 0 ? h_acc[3] / pairs : 0.0, m3 = pairs > 0 ? h_acc[4] / pairs : 0.0;
    *g1 = m2 > 0.0 ? m3 / (m2 * sqrt(m2)) : 0.0;
    return SFC_OK;
}

sfc_status choose_encoding(sfc_octree h, const int32_t* centre_ids, int64_t n_centres, int32_t k, void* cuda_stream,
                           sfc_encoding* best, double* g1_by_order) {
    if (!best) return SFC_ERR_INVALID;
    const sfc_encoding orders[3] = {SFC_ENC_NONE, SFC_ENC_MORTON, SFC_ENC_HILBERT};
    double g[3];
    for (int i = 0; i < 3; ++i) SFC_TRY(knn_locality(h, centre_ids, n_centres, k, orders[i], cuda_stream, nullptr, &g[i]));
    int b = 0;
    for (int i = 1; i < 3; ++i)
        if (g[i] > g[b]) b = i;
    *best = orders[b];
    if (g1_by_order)
        for (int i = 0; i < 3; ++i) g1_by_order[i] = g[i];
    return SFC_OK;
}

}  // extern "C"
