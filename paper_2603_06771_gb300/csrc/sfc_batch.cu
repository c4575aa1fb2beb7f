// sfc_batch.cu - many clouds in one pass (the batched path).
//
// The clouds arrive concatenated.  Every step of the single-cloud path runs once over the
// whole batch, each kernel finding a point's cloud from a small segment table:
//   - per-cloud bounding box and scale (warp-aggregated atomics per cloud), codes with the
//     cloud's own transform;
//   - one LSD radix sort of (code, index) over all points, then one stable pass on the cloud
//     number, so the batch is ordered by (cloud, code) and every cloud stays contiguous;
//   - the linear-octree kernels with cloud boundaries: no window crosses a cloud, every
//     cloud gets its own root, node-table slice and leaves slice;
//   - the group search kernels with a per-cloud table (root, centre range, r or k, output
//     base), one launch per kernel type / kNN size class for all clouds.
// A batch waits on the device three times in all (node counts, radius output size, the
// end), whatever the number of clouds.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <vector>

#include "sfc_internal.cuh"

namespace sfc {

// cloud of position p: the last segment with p0 <= p (segments are in position order)
__device__ __forceinline__ int seg_of_pos(const int64_t* p0s, int n, int64_t p) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (p0s[mid] <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// stage the segments' first positions in shared memory
__device__ __forceinline__ void load_p0(const BatchSeg* segs, int nsegs, int64_t* p0s) {
    for (int i = threadIdx.x; i < nsegs; i += blockDim.x) p0s[i] = segs[i].p0;
    __syncthreads();
}

__global__ void k_bseg_init(BatchSeg* segs, int nsegs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nsegs) return;
    for (int a = 0; a < 3; ++a) {
        segs[i].mn[a] = 0xffffffffu;
        segs[i].mx[a] = 0u;
        segs[i].lo[a] = 0.f;
    }
    segs[i].scale = 2097152.0f;
    segs[i].bad = 0u;
}

// per-cloud minima / maxima: a warp whose 32 points share a cloud reduces before one
// atomic per value; a warp on a cloud boundary updates per lane
__global__ void __launch_bounds__(256) k_batch_bbox(const float* __restrict__ xyz, int64_t n, BatchSeg* segs,
                                                    int nsegs) {
    __shared__ int64_t p0s[kBatchMax];
    load_p0(segs, nsegs, p0s);
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t base = static_cast<int64_t>(blockIdx.x) * blockDim.x; base < n; base += stride) {
        const int64_t i = base + threadIdx.x;
        const bool valid = i < n;
        const int sg = valid ? seg_of_pos(p0s, nsegs, i) : -1;
        float v[3] = {0.f, 0.f, 0.f};
        bool bad = false;
        if (valid) {
            for (int a = 0; a < 3; ++a) {
                v[a] = xyz[3 * i + a];
                if (!isfinite(v[a])) bad = true;
            }
        }
        const int s0 = __shfl_sync(0xffffffffu, sg, 0);
        const bool uniform = __all_sync(0xffffffffu, !valid || sg == s0) && s0 >= 0;
        if (uniform) {
            for (int a = 0; a < 3; ++a) {
                const unsigned int o = valid ? float_to_ordered(v[a]) : 0xffffffffu;
                const unsigned int mn = __reduce_min_sync(0xffffffffu, o);
                const unsigned int mx = __reduce_max_sync(0xffffffffu, valid ? o : 0u);
                if (lane_id() == 0) {
                    atomicMin(&segs[s0].mn[a], mn);
                    atomicMax(&segs[s0].mx[a], mx);
                }
            }
            const unsigned int b = __reduce_or_sync(0xffffffffu, bad ? 1u : 0u);
            if (lane_id() == 0 && b) atomicOr(&segs[s0].bad, 1u);
        } else if (valid) {
            for (int a = 0; a < 3; ++a) {
                const unsigned int o = float_to_ordered(v[a]);
                atomicMin(&segs[sg].mn[a], o);
                atomicMax(&segs[sg].mx[a], o);
            }
            if (bad) atomicOr(&segs[sg].bad, 1u);
        }
    }
}

__global__ void k_batch_bbox_finish(BatchSeg* segs, int nsegs) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nsegs) return;
    BatchSeg& g = segs[i];
    if (g.n == 0) return;
    float ext = 0.f;
    for (int a = 0; a < 3; ++a) {
        const float lo = ordered_to_float(g.mn[a]);
        const float hi = ordered_to_float(g.mx[a]);
        g.lo[a] = lo;
        const float d = __fsub_rn(hi, lo);
        if (d > ext) ext = d;
    }
    if (!isfinite(ext)) g.bad |= 2u;
    if (ext == 0.f) ext = 1.f;
    g.scale = __fdiv_rn(2097152.0f, ext);
}

__global__ void __launch_bounds__(256) k_batch_cloud_keys(const uint32_t* __restrict__ idx, int64_t n,
                                                          const BatchSeg* segs, int nsegs, uint64_t* ckey) {
    __shared__ int64_t p0s[kBatchMax];
    load_p0(segs, nsegs, p0s);
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += stride)
        ckey[j] = static_cast<uint64_t>(seg_of_pos(p0s, nsegs, idx[j]));
}

__global__ void __launch_bounds__(256) k_batch_gather(const float* __restrict__ xyz, int64_t n,
                                                      const uint64_t* __restrict__ codes, const uint32_t* __restrict__ idx,
                                                      const BatchSeg* segs, int nsegs, uint64_t* __restrict__ keys,
                                                      float4* __restrict__ pts, uint32_t* __restrict__ perm) {
    __shared__ int64_t p0s[kBatchMax];
    load_p0(segs, nsegs, p0s);
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += stride) {
        const int64_t i = idx[j];
        const uint32_t local = static_cast<uint32_t>(i - p0s[seg_of_pos(p0s, nsegs, j)]);
        keys[j] = codes[i];
        pts[j] = make_float4(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], __uint_as_float(local));
        perm[j] = local;
    }
}

// section 5.1 with cloud boundaries: windows never leave the cloud
__global__ void __launch_bounds__(256) k_batch_tree_count(const uint64_t* __restrict__ keys, int64_t n,
                                                          const BatchSeg* segs, int nsegs, uint32_t* __restrict__ cnt) {
    __shared__ int64_t p0s[kBatchMax];
    load_p0(segs, nsegs, p0s);
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += stride) {
        const int sg = seg_of_pos(p0s, nsegs, j);
        const int64_t p0 = p0s[sg];
        const int64_t end = p0 + segs[sg].n;
        const int64_t ncap = segs[sg].ncap;
        uint32_t c = 0;
        if (j + ncap < end) {
            const int first_new = j == p0 ? 0 : common_levels(keys[j - 1], keys[j]) + 1;
            int deepest = common_levels(keys[j], keys[j + ncap]);
            if (deepest > kLevels - 1) deepest = kLevels - 1;
            if (deepest >= first_new) c = static_cast<uint32_t>(deepest - first_new + 1);
        }
        cnt[j] = c;
    }
}

__global__ void k_batch_seg_internal(BatchSeg* segs, int nsegs, const int64_t* __restrict__ first) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nsegs) return;
    segs[i].g0 = first[segs[i].p0];
    segs[i].n_int = first[segs[i].p0 + segs[i].n] - segs[i].g0;
}

__global__ void __launch_bounds__(256) k_batch_tree_emit(const uint64_t* __restrict__ keys, int64_t n,
                                                         const BatchSeg* segs, int nsegs,
                                                         const uint32_t* __restrict__ cnt,
                                                         const int64_t* __restrict__ first,
                                                         uint64_t* __restrict__ ikey, uint8_t* __restrict__ ilevel) {
    __shared__ int64_t p0s[kBatchMax];
    load_p0(segs, nsegs, p0s);
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t j = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; j < n; j += stride) {
        const uint32_t c = cnt[j];
        if (c == 0) continue;
        const int64_t p0 = p0s[seg_of_pos(p0s, nsegs, j)];
        const int first_new = j == p0 ? 0 : common_levels(keys[j - 1], keys[j]) + 1;
        const uint64_t k = keys[j];
        const int64_t g = first[j];
        for (uint32_t t = 0; t < c; ++t) {
            const int l = first_new + static_cast<int>(t);
            ikey[g + t] = k & ~below_level_mask(l);
            ilevel[g + t] = static_cast<uint8_t>(l);
        }
    }
}

// cloud owning internal node g: the last non-empty segment with g0 <= g
__device__ __forceinline__ int seg_of_internal(const BatchSeg* segs, int n, int64_t g) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].g0 <= g) lo = mid;
        else hi = mid - 1;
    }
    while (lo > 0 && segs[lo].n_int == 0) --lo;  // empty clouds share g0 with the next one
    return lo;
}

__device__ __forceinline__ int seg_of_node(const BatchSeg* segs, int n, int64_t s) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].node0 <= s) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_batch_tree_link(const uint64_t* __restrict__ ikey,
                                                         const uint8_t* __restrict__ ilevel, int64_t total_int,
                                                         const BatchSeg* segs, int nsegs, int32_t* __restrict__ child,
                                                         int32_t* __restrict__ islot) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < total_int; g += stride) {
        const BatchSeg& sg = segs[seg_of_internal(segs, nsegs, g)];
        const int64_t local = g - sg.g0;
        if (local == 0) {
            islot[g] = static_cast<int32_t>(sg.node0);
            child[sg.node0] = static_cast<int32_t>(sg.node0 + 1);
            continue;
        }
        const uint64_t k = ikey[g];
        const int l = ilevel[g];
        const uint64_t pk = k & ~below_level_mask(l - 1);
        const int pl = l - 1;
        int64_t lo = sg.g0, hi = g;
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            const uint64_t mk = ikey[mid];
            if (mk < pk || (mk == pk && ilevel[mid] < pl)) lo = mid + 1;
            else hi = mid;
        }
        const int digit = static_cast<int>((k >> (3 * (kLevels - l))) & 7ull);
        const int64_t slot = sg.node0 + 1 + 8 * (lo - sg.g0) + digit;
        child[slot] = static_cast<int32_t>(sg.node0 + 1 + 8 * local);
        islot[g] = static_cast<int32_t>(slot);
    }
}

__device__ __forceinline__ int octal_digit_sum_b(uint64_t k) {
    const uint64_t m0 = 0x1249249249249249ull;
    return __popcll(k & m0) + 2 * __popcll(k & (m0 << 1)) + 4 * __popcll(k & (m0 << 2));
}

__device__ __forceinline__ int64_t lower_bound_range(const uint64_t* a, int64_t lo, int64_t hi, uint64_t key) {
    while (lo < hi) {
        const int64_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(256) k_batch_tree_nodes(const uint64_t* __restrict__ keys,
                                                          const uint64_t* __restrict__ ikey,
                                                          const uint8_t* __restrict__ ilevel, const BatchSeg* segs,
                                                          int nsegs, int64_t total_nodes,
                                                          const int32_t* __restrict__ child, NodeBox* __restrict__ nodes,
                                                          uint64_t* __restrict__ leaves,
                                                          uint32_t* __restrict__ leaf_counts) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; s < total_nodes; s += stride) {
        const BatchSeg& sg = segs[seg_of_node(segs, nsegs, s)];
        const int64_t local = s - sg.node0;
        uint64_t k = 0;
        int l = 0;
        if (local > 0) {
            const int64_t g = sg.g0 + ((local - 1) >> 3);
            const int c = static_cast<int>((local - 1) & 7);
            l = ilevel[g] + 1;
            k = ikey[g] + (static_cast<uint64_t>(c) << (3 * (kLevels - l)));
        }
        const int64_t p_end = sg.p0 + sg.n;
        const int64_t start = lower_bound_range(keys, sg.p0, p_end, k);
        const int64_t end = l == 0 ? p_end : lower_bound_range(keys, sg.p0, p_end, k + (1ull << (3 * (kLevels - l))));
        NodeBox b;
        b.lo = make_float4(INFINITY, INFINITY, INFINITY, __uint_as_float(static_cast<uint32_t>(start)));
        b.hi = make_float4(-INFINITY, -INFINITY, -INFINITY, __uint_as_float(static_cast<uint32_t>(end)));
        nodes[s] = b;
        if (child[s] < 0) {
            const int64_t before = lower_bound_range(ikey, sg.g0, sg.g0 + sg.n_int, k) - sg.g0;
            const int trailing = k == 0 ? kLevels : (__ffsll(static_cast<long long>(k)) - 1) / 3;
            const int64_t rank = octal_digit_sum_b(k) + 7 * (before - (kLevels - trailing));
            if (rank >= 0 && rank <= 7 * sg.n_int) {
                leaves[sg.leaf0 + rank] = k;
                leaf_counts[sg.leaf0 + rank] = static_cast<uint32_t>(end - start);
            }
        }
        if (local == 0) leaves[sg.leaf0 + 7 * sg.n_int + 1] = kWholeRange;
    }
}

__global__ void __launch_bounds__(256) k_batch_tree_boxes(const float4* __restrict__ pts, const BatchSeg* segs,
                                                          int nsegs, NodeBox* nodes, const int32_t* __restrict__ child,
                                                          const int32_t* __restrict__ islot, unsigned int* arrive,
                                                          int64_t total_nodes) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; s < total_nodes; s += stride) {
        if (child[s] >= 0) continue;
        const BatchSeg& sg = segs[seg_of_node(segs, nsegs, s)];
        NodeBox b = nodes[s];
        const uint32_t start = __float_as_uint(b.lo.w), end = __float_as_uint(b.hi.w);
        for (uint32_t j = start; j < end; ++j) {
            const float4 p = pts[j];
            b.lo.x = fminf(b.lo.x, p.x); b.lo.y = fminf(b.lo.y, p.y); b.lo.z = fminf(b.lo.z, p.z);
            b.hi.x = fmaxf(b.hi.x, p.x); b.hi.y = fmaxf(b.hi.y, p.y); b.hi.z = fmaxf(b.hi.z, p.z);
        }
        nodes[s] = b;
        int64_t cur = s;
        for (int hops = 0; cur != sg.node0 && hops <= kLevels; ++hops) {
            const int64_t g = sg.g0 + ((cur - sg.node0 - 1) >> 3);
            __threadfence();
            if (atomicAdd(&arrive[g], 1u) != 7u) break;
            __threadfence();
            const int64_t ps = islot[g];
            const int64_t c0 = sg.node0 + 1 + 8 * (g - sg.g0);
            NodeBox u = nodes[ps];
            u.lo.x = u.lo.y = u.lo.z = INFINITY;
            u.hi.x = u.hi.y = u.hi.z = -INFINITY;
            for (int c = 0; c < 8; ++c) {
                const float4 clo = __ldcg(&nodes[c0 + c].lo);
                const float4 chi = __ldcg(&nodes[c0 + c].hi);
                u.lo.x = fminf(u.lo.x, clo.x); u.lo.y = fminf(u.lo.y, clo.y); u.lo.z = fminf(u.lo.z, clo.z);
                u.hi.x = fmaxf(u.hi.x, chi.x); u.hi.y = fmaxf(u.hi.y, chi.y); u.hi.z = fmaxf(u.hi.z, chi.z);
            }
            nodes[ps] = u;
            cur = ps;
        }
    }
}

__global__ void k_batch_row_bounds(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ where, int n,
                                   int64_t* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = row_ptr[where[i]];
}

}  // namespace sfc

// ---------------------------------------------------------------------------------
// the batch handle
struct sfc_batch_s {
    int32_t n_clouds = 0;
    std::vector<sfc_batch_cloud> clouds;
    std::vector<int64_t> p0;           // first input position of every cloud
    std::vector<int64_t> out0;         // kNN clouds: first output entry
    std::vector<int64_t> row_lo, row_hi;  // radius clouds: row_ptr[p0], row_ptr[p0 + n]
    int64_t n_total = 0;
    int64_t nnz = 0;
    int64_t knn_total = 0;
    int64_t* row_ptr = nullptr;
    int32_t* cols = nullptr;
    int32_t* knn_idx = nullptr;
    float* knn_d2 = nullptr;
};

namespace sfc {

// launch declared in sfc_radius.cu / sfc_knn.cu
sfc_status batch_radius_launch(const float4* pts, const uint32_t* perm, const NodeBox* nodes, const int32_t* child,
                               int64_t total_nodes, const SearchSeg* segs, int nsegs, int64_t ngroups, int kern,
                               bool fill, uint32_t* counts, const int64_t* row_ptr, int32_t* cols, unsigned int* err,
                               int prune, const BatchRecords& rec, cudaStream_t s);
sfc_status batch_knn_launch(const float4* pts, const uint32_t* perm, const NodeBox* nodes, const int32_t* child,
                            int64_t total_nodes, const SearchSeg* segs, int nsegs, int64_t ngroups, int kmax, int window,
                            int32_t* out_idx, float* out_d2, unsigned int* err, cudaStream_t s);

static sfc_status run_batch(sfc_batch_s* B, const float* xyz, sfc_encoding enc, const sfc_build_opts& o,
                            cudaStream_t s) {
    Scratch scratch(s);
    const int nsegs = B->n_clouds;
    const int64_t n = B->n_total;
    std::vector<BatchSeg> hseg(nsegs);
    for (int i = 0; i < nsegs; ++i) {
        memset(&hseg[i], 0, sizeof(BatchSeg));
        hseg[i].p0 = B->p0[i];
        hseg[i].n = B->clouds[i].n_points;
        hseg[i].ncap = o.leaf_capacity;
    }
    BatchSeg* segs = nullptr;
    SFC_TRY(scratch.alloc(&segs, nsegs));
    SFC_CUDA(cudaMemcpyAsync(segs, hseg.data(), sizeof(BatchSeg) * nsegs, cudaMemcpyHostToDevice, s));
    const unsigned int sgrid = grid_for(nsegs, 128);
    const unsigned int grid = grid_for(n, 256, 152 * 16);
    SFC_LAUNCH("batch_bbox_init", s, k_bseg_init, sgrid, 128, 0, segs, nsegs);
    SFC_LAUNCH("batch_bbox", s, k_batch_bbox, grid, 256, 0, xyz, n, segs, nsegs);
    SFC_LAUNCH("batch_bbox_finish", s, k_batch_bbox_finish, sgrid, 128, 0, segs, nsegs);

    // codes, sort by code, then by cloud (stable): order (cloud, code)
    uint64_t *codes, *k0, *k1;
    uint32_t *v0, *v1, *perm;
    float4* pts;
    SFC_TRY(scratch.alloc(&codes, n));
    SFC_TRY(scratch.alloc(&k0, n));
    SFC_TRY(scratch.alloc(&k1, n));
    SFC_TRY(scratch.alloc(&v0, n));
    SFC_TRY(scratch.alloc(&v1, n));
    SFC_TRY(scratch.alloc(&perm, n));
    SFC_TRY(scratch.alloc(&pts, n));
    SFC_TRY(batch_encode(xyz, n, enc, segs, nsegs, codes, v0, s));
    SFC_CUDA(cudaMemcpyAsync(k0, codes, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
    SFC_TRY(radix_sort_pairs(k0, v0, k1, v1, n, s, scratch));
    if (nsegs > 1) {
        SFC_LAUNCH("batch_cloud_keys", s, k_batch_cloud_keys, grid, 256, 0, v0, n, segs, nsegs, k0);
        int bits = 0;
        while ((1 << bits) < nsegs) ++bits;
        SFC_TRY(radix_sort_pairs_bits(k0, v0, k1, v1, n, 0, bits, s, scratch));
    }
    uint64_t* keys = k1;  // the sorted codes
    SFC_LAUNCH("batch_gather", s, k_batch_gather, grid, 256, 0, xyz, n, codes, v0, segs, nsegs, keys, pts, perm);

    // linear octrees
    uint32_t* cnt;
    int64_t* first;
    SFC_TRY(scratch.alloc(&cnt, n));
    SFC_TRY(scratch.alloc(&first, n + 1));
    SFC_LAUNCH("batch_tree_count", s, k_batch_tree_count, grid, 256, 0, keys, n, segs, nsegs, cnt);
    SFC_TRY(scan_u32_to_i64(cnt, first, n, s, scratch));
    SFC_LAUNCH("batch_seg_internal", s, k_batch_seg_internal, sgrid, 128, 0, segs, nsegs, first);
    SFC_CUDA(cudaMemcpyAsync(hseg.data(), segs, sizeof(BatchSeg) * nsegs, cudaMemcpyDeviceToHost, s));
    SFC_CUDA(cudaStreamSynchronize(s));
    int64_t total_int = 0, total_nodes = 0, total_leaves = 0;
    for (int i = 0; i < nsegs; ++i) {
        if (hseg[i].bad) return SFC_ERR_NOT_FINITE;
        hseg[i].node0 = total_nodes;
        hseg[i].leaf0 = total_leaves;
        total_int += hseg[i].n_int;
        total_nodes += 1 + 8 * hseg[i].n_int;
        total_leaves += 7 * hseg[i].n_int + 2;
    }
    if (total_nodes > 0x7fffffffLL) return SFC_ERR_TOO_LARGE;

    // search tables: radius clouds grouped by kernel, kNN clouds by list size; one launch
    // per group, each reading its slice of one table.  They go up with the segment table,
    // while the device is idle, together with the positions whose row_ptr entries bound
    // every cloud's rows.
    std::vector<SearchSeg> radius_sets[4], knn_sets[4];
    int64_t knn_total = 0;
    for (int i = 0; i < nsegs; ++i) {
        const sfc_batch_cloud& cl = B->clouds[i];
        if (cl.n_points == 0) continue;
        SearchSeg q;
        memset(&q, 0, sizeof q);
        q.q0 = hseg[i].p0;
        q.nq = cl.n_points;
        q.root = static_cast<int32_t>(hseg[i].node0);
        q.k = cl.k;
        q.r = cl.r;
        q.r2 = cl.r * cl.r;
        if (cl.search == SFC_SEARCH_RADIUS) {
            if (!(cl.r > 0.f)) continue;  // r <= 0: every row empty
            q.row0 = hseg[i].p0;
            radius_sets[cl.kernel].push_back(q);
        } else {
            q.row0 = knn_total;
            B->out0[i] = knn_total;
            knn_total += cl.n_points * cl.k;
            const int bucket = cl.k <= 8 ? 0 : (cl.k <= 16 ? 1 : (cl.k <= 32 ? 2 : 3));
            knn_sets[bucket].push_back(q);
        }
    }
    std::vector<SearchSeg> table;
    int64_t radius_off[4], radius_groups[4], knn_off[4], knn_groups[4];
    auto append = [&](std::vector<SearchSeg>& v, int64_t* off, int64_t* ngroups) {
        *off = static_cast<int64_t>(table.size());
        int64_t g = 0;
        for (auto& q : v) {
            q.group0 = g;
            g += (q.nq + 31) / 32;
            table.push_back(q);
        }
        *ngroups = g;
    };
    for (int t = 0; t < 4; ++t) append(radius_sets[t], &radius_off[t], &radius_groups[t]);
    for (int t = 0; t < 4; ++t) append(knn_sets[t], &knn_off[t], &knn_groups[t]);
    std::vector<int64_t> where;
    for (int i = 0; i < nsegs; ++i) {
        where.push_back(hseg[i].p0);
        where.push_back(hseg[i].p0 + hseg[i].n);
    }
    SearchSeg* dsearch = nullptr;
    int64_t *dwhere, *dbounds;
    SFC_TRY(scratch.alloc(&dsearch, table.empty() ? 1 : table.size()));
    SFC_TRY(scratch.alloc(&dwhere, where.size()));
    SFC_TRY(scratch.alloc(&dbounds, where.size()));
    SFC_CUDA(cudaMemcpyAsync(segs, hseg.data(), sizeof(BatchSeg) * nsegs, cudaMemcpyHostToDevice, s));
    if (!table.empty())
        SFC_CUDA(cudaMemcpyAsync(dsearch, table.data(), sizeof(SearchSeg) * table.size(), cudaMemcpyHostToDevice, s));
    SFC_CUDA(cudaMemcpyAsync(dwhere, where.data(), sizeof(int64_t) * where.size(), cudaMemcpyHostToDevice, s));

    NodeBox* nodes;
    int32_t *child, *islot;
    uint64_t *ikey, *leaves;
    uint8_t* ilevel;
    uint32_t* leaf_counts;
    unsigned int *arrive, *err;
    SFC_TRY(scratch.alloc(&nodes, total_nodes));
    SFC_TRY(scratch.alloc(&child, total_nodes));
    SFC_TRY(scratch.alloc(&islot, total_int));
    SFC_TRY(scratch.alloc(&ikey, total_int));
    SFC_TRY(scratch.alloc(&ilevel, total_int));
    SFC_TRY(scratch.alloc(&arrive, total_int));
    SFC_TRY(scratch.alloc(&leaves, total_leaves));
    SFC_TRY(scratch.alloc(&leaf_counts, total_leaves));
    SFC_TRY(scratch.alloc(&err, 1));
    SFC_CUDA(cudaMemsetAsync(child, 0xff, sizeof(int32_t) * total_nodes, s));
    SFC_CUDA(cudaMemsetAsync(arrive, 0, sizeof(unsigned int) * (total_int ? total_int : 1), s));
    SFC_CUDA(cudaMemsetAsync(err, 0, sizeof(unsigned int), s));
    if (total_int > 0) {
        SFC_LAUNCH("batch_tree_emit", s, k_batch_tree_emit, grid, 256, 0, keys, n, segs, nsegs, cnt, first, ikey, ilevel);
        SFC_LAUNCH("batch_tree_link", s, k_batch_tree_link, grid_for(total_int, 256, 152 * 16), 256, 0, ikey, ilevel,
                   total_int, segs, nsegs, child, islot);
    }
    const unsigned int ngrid = grid_for(total_nodes, 256, 152 * 16);
    SFC_LAUNCH("batch_tree_nodes", s, k_batch_tree_nodes, ngrid, 256, 0, keys, ikey, ilevel, segs, nsegs, total_nodes,
               child, nodes, leaves, leaf_counts);
    SFC_LAUNCH("batch_tree_boxes", s, k_batch_tree_boxes, ngrid, 256, 0, pts, segs, nsegs, nodes, child, islot, arrive,
               total_nodes);

    // kNN first, then the radius count: the device works through both while the host
    // waits for the radius output size
    B->knn_total = knn_total;
    SFC_TRY(dev_alloc(&B->knn_idx, knn_total, s));
    SFC_TRY(dev_alloc(&B->knn_d2, knn_total, s));
    const int kmax_of[4] = {8, 16, 32, 64};
    for (int bkt = 0; bkt < 4; ++bkt) {
        int window = 16;  // curve neighbours per side for the seeding window (at least k / 2)
        for (auto& q : knn_sets[bkt]) window = std::max(window, (q.k + 1) / 2);
        SFC_TRY(batch_knn_launch(pts, perm, nodes, child, total_nodes, dsearch + knn_off[bkt],
                                 static_cast<int>(knn_sets[bkt].size()), knn_groups[bkt], kmax_of[bkt], window,
                                 B->knn_idx, B->knn_d2, err, s));
    }
    uint32_t* counts = nullptr;
    SFC_TRY(dev_alloc(&B->row_ptr, n + 1, s));
    SFC_TRY(scratch.alloc(&counts, n));
    SFC_CUDA(cudaMemsetAsync(counts, 0, sizeof(uint32_t) * n, s));
    // hit-mask records of the count pass, replayed by the fill; each kernel type's launch
    // gets its slice.  Without memory for them the fill walks the trees again.
    int64_t rec_groups = 0;
    for (int kern = 0; kern < 4; ++kern) rec_groups += radius_groups[kern];
    BatchRecords rec_all;
    if (rec_groups > 0) {
        const int64_t slots = rec_groups * kRecordCap;
        if (cudaMallocAsync(reinterpret_cast<void**>(&rec_all.masks), sizeof(uint32_t) * 32 * slots, s) !=
                cudaSuccess ||
            cudaMallocAsync(reinterpret_cast<void**>(&rec_all.head), sizeof(uint2) * slots, s) != cudaSuccess ||
            cudaMallocAsync(reinterpret_cast<void**>(&rec_all.count), sizeof(uint32_t) * rec_groups, s) !=
                cudaSuccess) {
            cudaGetLastError();
            dev_free(rec_all.masks, s);
            dev_free(rec_all.head, s);
            dev_free(rec_all.count, s);
            rec_all = BatchRecords();
        }
    }
    struct RecGuard {
        BatchRecords& r;
        cudaStream_t s;
        ~RecGuard() {
            dev_free(r.masks, s);
            dev_free(r.head, s);
            dev_free(r.count, s);
        }
    } rec_guard{rec_all, s};
    BatchRecords rec_of[4];
    for (int64_t kern = 0, g = 0; kern < 4; g += radius_groups[kern], ++kern) {
        if (!rec_all.masks) continue;
        rec_of[kern].masks = rec_all.masks + g * kRecordCap * 32;
        rec_of[kern].head = rec_all.head + g * kRecordCap;
        rec_of[kern].count = rec_all.count + g;
    }
    for (int kern = 0; kern < 4; ++kern)
        SFC_TRY(batch_radius_launch(pts, perm, nodes, child, total_nodes, dsearch + radius_off[kern],
                                    static_cast<int>(radius_sets[kern].size()), radius_groups[kern], kern, false,
                                    counts, nullptr, nullptr, err, o.prune, rec_of[kern], s));
    SFC_TRY(scan_u32_to_i64(counts, B->row_ptr, n, s, scratch));
    SFC_CUDA(cudaMemcpyAsync(&B->nnz, B->row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SFC_CUDA(cudaStreamSynchronize(s));
    SFC_TRY(dev_alloc(&B->cols, B->nnz, s));
    for (int kern = 0; kern < 4; ++kern)
        SFC_TRY(batch_radius_launch(pts, perm, nodes, child, total_nodes, dsearch + radius_off[kern],
                                    static_cast<int>(radius_sets[kern].size()), radius_groups[kern], kern, true,
                                    counts, B->row_ptr, B->cols, err, o.prune, rec_of[kern], s));
    // per-cloud row bounds and the guard word
    SFC_LAUNCH("batch_row_bounds", s, k_batch_row_bounds, grid_for(static_cast<int64_t>(where.size()), 128), 128, 0,
               B->row_ptr, dwhere, static_cast<int>(where.size()), dbounds);
    std::vector<int64_t> bounds(where.size());
    unsigned int herr = 0;
    SFC_CUDA(cudaMemcpyAsync(bounds.data(), dbounds, sizeof(int64_t) * bounds.size(), cudaMemcpyDeviceToHost, s));
    SFC_CUDA(cudaMemcpyAsync(&herr, err, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    SFC_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < nsegs; ++i) {
        B->row_lo[i] = bounds[2 * i];
        B->row_hi[i] = bounds[2 * i + 1];
    }
    if (herr & kGuardTripped) return SFC_ERR_INTERNAL;
    return SFC_OK;
}

static void free_batch(sfc_batch_s* B, cudaStream_t s) {
    dev_free(B->row_ptr, s);
    dev_free(B->cols, s);
    dev_free(B->knn_idx, s);
    dev_free(B->knn_d2, s);
    B->row_ptr = nullptr;
    B->cols = nullptr;
    B->knn_idx = nullptr;
    B->knn_d2 = nullptr;
}

}  // namespace sfc

extern "C" {

sfc_status batch_search(const float* points_xyz, const sfc_batch_cloud* clouds, int32_t n_clouds, sfc_encoding enc,
                        const sfc_build_opts* opts, void* cuda_stream, sfc_batch* out) {
    if (!out || !clouds || n_clouds < 1) return SFC_ERR_INVALID;
    *out = nullptr;
    if (n_clouds > sfc::kBatchMax) return SFC_ERR_TOO_LARGE;
    if (enc != SFC_ENC_MORTON && enc != SFC_ENC_HILBERT) return SFC_ERR_INVALID;
    sfc_build_opts o;
    sfc_build_opts_default(&o);
    if (opts) o = *opts;
    if (o.leaf_capacity < 1 || (o.prune != 0 && o.prune != 1)) return SFC_ERR_INVALID;
    int64_t total = 0;
    for (int i = 0; i < n_clouds; ++i) {
        const sfc_batch_cloud& c = clouds[i];
        if (c.n_points < 0) return SFC_ERR_INVALID;
        if (c.search == SFC_SEARCH_RADIUS) {
            if (c.kernel < 0 || c.kernel > 3 || isnan(c.r)) return SFC_ERR_INVALID;
        } else if (c.search == SFC_SEARCH_KNN) {
            if (c.k < 1) return SFC_ERR_INVALID;
            if (c.k > sfc::kMaxK) return SFC_ERR_TOO_LARGE;
        } else {
            return SFC_ERR_INVALID;
        }
        total += c.n_points;
    }
    if (total > 0x7fffffffLL - 1) return SFC_ERR_TOO_LARGE;
    if (total > 0 && (!points_xyz || !sfc::is_device_ptr(points_xyz))) return SFC_ERR_NOT_DEVICE_PTR;
    int dev = 0;
    SFC_CUDA(cudaGetDevice(&dev));
    SFC_TRY(sfc::ensure_pool(dev));
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    sfc_batch_s* B = new (std::nothrow) sfc_batch_s;
    if (!B) return SFC_ERR_OOM;
    B->n_clouds = n_clouds;
    B->clouds.assign(clouds, clouds + n_clouds);
    B->p0.resize(n_clouds);
    B->out0.assign(n_clouds, 0);
    B->row_lo.assign(n_clouds, 0);
    B->row_hi.assign(n_clouds, 0);
    int64_t p = 0;
    for (int i = 0; i < n_clouds; ++i) {
        B->p0[i] = p;
        p += clouds[i].n_points;
    }
    B->n_total = total;
    sfc_status st = total > 0 ? sfc::run_batch(B, points_xyz, enc, o, s) : SFC_OK;
    if (st == SFC_OK && total == 0) {
        st = sfc::dev_alloc(&B->row_ptr, 1, s);
        if (st == SFC_OK && cudaMemsetAsync(B->row_ptr, 0, sizeof(int64_t), s) != cudaSuccess) st = SFC_ERR_CUDA;
    }
    if (st != SFC_OK) {
        sfc::free_batch(B, s);
        delete B;
        return st;
    }
    *out = B;
    return SFC_OK;
}

sfc_status batch_cloud_result(sfc_batch b, int32_t cloud, const int64_t** row_ptr, const int32_t** cols, int64_t* nnz,
                              const int32_t** knn_idx, const float** knn_d2) {
    if (!b || cloud < 0 || cloud >= b->n_clouds) return SFC_ERR_INVALID;
    const sfc_batch_cloud& c = b->clouds[cloud];
    if (row_ptr) *row_ptr = c.search == SFC_SEARCH_RADIUS ? b->row_ptr + b->p0[cloud] : nullptr;
    if (cols) *cols = c.search == SFC_SEARCH_RADIUS ? b->cols : nullptr;
    if (nnz) *nnz = c.search == SFC_SEARCH_RADIUS ? b->row_hi[cloud] - b->row_lo[cloud] : 0;
    if (knn_idx) *knn_idx = c.search == SFC_SEARCH_KNN ? b->knn_idx + b->out0[cloud] : nullptr;
    if (knn_d2) *knn_d2 = c.search == SFC_SEARCH_KNN ? b->knn_d2 + b->out0[cloud] : nullptr;
    return SFC_OK;
}

sfc_status batch_free(sfc_batch b, void* cuda_stream) {
    if (!b) return SFC_ERR_INVALID;
    sfc::free_batch(b, static_cast<cudaStream_t>(cuda_stream));
    delete b;
    return SFC_OK;
}

}  // extern "C"
