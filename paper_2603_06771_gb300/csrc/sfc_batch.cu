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

// Sizes the device learns during a batch (read by the later kernels, so that nothing
// waits for the host), and what went wrong.
struct BatchTotals {
    int64_t n_int, n_nodes, n_leaves;  // internal nodes, node-table entries, leaves slots
    int64_t nnz;                       // radius output entries
    unsigned int flags;                // kOverNodes | kOverCols | kNonFinite
    unsigned int pad;
};
constexpr unsigned int kOverNodes = 1u;  // the node tables exceed their capacity: no tree, no search
constexpr unsigned int kOverCols = 2u;   // the radius output exceeds its capacity: no fill
constexpr unsigned int kNonFinite = 4u;  // a cloud holds a non-finite coordinate

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
        const uint32_t c = new_internal_cells(keys, j, p0, end, ncap);
        cnt[j] = c;
    }
}

__global__ void k_batch_seg_internal(BatchSeg* segs, int nsegs, const int64_t* __restrict__ first) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nsegs) return;
    segs[i].g0 = first[segs[i].p0];
    segs[i].n_int = first[segs[i].p0 + segs[i].n] - segs[i].g0;
}

// Every cloud's slices of the node table and the leaves array (exclusive prefix sums over
// the clouds, one block), the totals, the capacity check, and the root of every search
// table entry.
__global__ void __launch_bounds__(1024) k_batch_layout(BatchSeg* segs, int nsegs, int64_t int_cap, int64_t node_cap,
                                                       int64_t leaf_cap, SearchSeg* table, const int32_t* table_cloud,
                                                       int ntable, BatchTotals* tot) {
    __shared__ int64_t sn[1024], sl[1024];
    const int i = threadIdx.x;
    const int64_t ni = i < nsegs ? segs[i].n_int : 0;
    const int64_t vn = i < nsegs ? 1 + 8 * ni : 0;
    const int64_t vl = i < nsegs ? 7 * ni + 2 : 0;
    const int bad = __syncthreads_or(i < nsegs && segs[i].bad != 0u);
    sn[i] = vn;
    sl[i] = vl;
    __syncthreads();
    for (int o = 1; o < 1024; o <<= 1) {  // inclusive scan (Hillis-Steele)
        const int64_t an = i >= o ? sn[i - o] : 0;
        const int64_t al = i >= o ? sl[i - o] : 0;
        __syncthreads();
        sn[i] += an;
        sl[i] += al;
        __syncthreads();
    }
    if (i < nsegs) {
        segs[i].node0 = sn[i] - vn;
        segs[i].leaf0 = sl[i] - vl;
    }
    if (i == 1023) {
        const int64_t nodes = sn[1023], leaves = sl[1023];
        const int64_t internal = (nodes - nsegs) / 8;
        unsigned int f = bad ? kNonFinite : 0u;
        if (internal > int_cap || nodes > node_cap || leaves > leaf_cap || nodes > 0x7fffffffLL) f |= kOverNodes;
        tot->n_int = internal;
        tot->n_nodes = nodes;
        tot->n_leaves = leaves;
        tot->nnz = 0;
        tot->flags = f;
    }
    __syncthreads();
    for (int j = i; j < ntable; j += 1024) table[j].root = static_cast<int32_t>(segs[table_cloud[j]].node0);
}

// child links start as "leaf", arrival counters at zero (over the sizes of this run)
__global__ void __launch_bounds__(256) k_batch_tree_init(int32_t* __restrict__ child, unsigned int* __restrict__ arrive,
                                                         const BatchTotals* tot) {
    if (tot->flags & kOverNodes) return;
    const int64_t nodes = tot->n_nodes, internal = tot->n_int;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; s < nodes; s += stride) {
        child[s] = -1;
        if (s < internal) arrive[s] = 0u;
    }
}

__global__ void __launch_bounds__(256) k_batch_tree_emit(const uint64_t* __restrict__ keys, int64_t n,
                                                         const BatchSeg* segs, int nsegs,
                                                         const uint32_t* __restrict__ cnt,
                                                         const int64_t* __restrict__ first,
                                                         uint64_t* __restrict__ ikey, uint8_t* __restrict__ ilevel,
                                                         const BatchTotals* tot) {
    __shared__ int64_t p0s[kBatchMax];
    load_p0(segs, nsegs, p0s);
    if (tot->flags & kOverNodes) return;
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
                                                         const uint8_t* __restrict__ ilevel, const BatchTotals* tot,
                                                         const BatchSeg* segs, int nsegs, int32_t* __restrict__ child,
                                                         int32_t* __restrict__ islot) {
    const int64_t total_int = (tot->flags & kOverNodes) ? 0 : tot->n_int;
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
                                                          int nsegs, const BatchTotals* tot,
                                                          const int32_t* __restrict__ child, NodeBox* __restrict__ nodes,
                                                          uint64_t* __restrict__ leaves,
                                                          uint32_t* __restrict__ leaf_counts) {
    const int64_t total_nodes = (tot->flags & kOverNodes) ? 0 : tot->n_nodes;
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
                                                          const BatchTotals* tot) {
    const int64_t total_nodes = (tot->flags & kOverNodes) ? 0 : tot->n_nodes;
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

// the radius output size against the capacity of the output array
__global__ void k_batch_check_cols(const int64_t* __restrict__ row_end, int64_t cols_cap, BatchTotals* tot) {
    const int64_t nnz = *row_end;
    tot->nnz = nnz;
    if (nnz > cols_cap) atomicOr(&tot->flags, kOverCols);
}

__global__ void k_batch_row_bounds(const int64_t* __restrict__ row_ptr, const int64_t* __restrict__ where, int n,
                                   int64_t* __restrict__ out) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = row_ptr[where[i]];
}

// Every cloud's own row pointers, starting at 0: cloud c's n_c + 1 entries sit at
// [p0_c + c, p0_c + c + n_c] of rel (the batch's row pointers minus the cloud's first).
__global__ void k_batch_rel_rows(const int64_t* __restrict__ row_ptr, const BatchSeg* __restrict__ segs, int nsegs,
                                 int64_t total, int64_t* __restrict__ rel) {
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < total;
         g += static_cast<int64_t>(gridDim.x) * blockDim.x) {
        int lo = 0, hi = nsegs - 1;  // the last cloud c with p0_c + c <= g
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (segs[mid].p0 + mid <= g) lo = mid;
            else hi = mid - 1;
        }
        const int64_t p0 = segs[lo].p0;
        const int64_t i = g - lo - p0;  // 0 .. n_c
        rel[g] = row_ptr[p0 + i] - row_ptr[p0];
    }
}

}  // namespace sfc

// ---------------------------------------------------------------------------------
// host side

namespace sfc {

// launches declared in sfc_radius.cu / sfc_knn.cu
sfc_status batch_radius_launch(const float4* pts, const uint32_t* perm, const NodeBox* nodes, const int32_t* child,
                               int64_t total_nodes, const SearchSeg* segs, int nsegs, int64_t ngroups, int kern,
                               bool fill, uint32_t* counts, const int64_t* row_ptr, int32_t* cols, unsigned int* err,
                               int prune, const BatchRecords& rec, const unsigned int* skip, unsigned int skip_mask,
                               cudaStream_t s);
sfc_status batch_knn_launch(const float4* pts, const uint32_t* perm, const NodeBox* nodes, const int32_t* child,
                            int64_t total_nodes, const SearchSeg* segs, int nsegs, int64_t ngroups, int kmax, int exact,
                            int32_t* out_idx, float* out_d2, unsigned int* err, const unsigned int* skip,
                            unsigned int skip_mask, cudaStream_t s);

// Internal nodes of a cloud of n points at most: the internal nodes of one level hold
// disjoint sets of more than ncap points each, and a level l has at most 8^l nodes.
static int64_t internal_bound(int64_t n, int64_t ncap) {
    if (n <= ncap) return 0;
    const int64_t per_level = n / (ncap + 1);
    int64_t total = 0, level_max = 1;
    for (int l = 0; l < kLevels; ++l) {
        total += std::min(level_max, per_level);
        if (level_max < per_level) level_max *= 8;
    }
    return total;
}

constexpr int kLaunchSets = 8;  // radius kernels 0-3, kNN list sizes 8 / 16 / 32 / 64

// What follows from the clouds' sizes and searches alone.
struct BatchTables {
    int n_clouds = 0;
    int64_t n_total = 0;
    std::vector<BatchSeg> seg;         // p0, n, ncap of every cloud
    std::vector<SearchSeg> table;      // launch tables, one slice per launch (roots set on the device)
    std::vector<int32_t> table_cloud;  // the cloud of every table entry
    int64_t off[kLaunchSets], count[kLaunchSets], groups[kLaunchSets];
    std::vector<int64_t> where;  // the row_ptr positions bounding every cloud's rows
    std::vector<int64_t> out0;   // kNN clouds: first output entry
    int64_t knn_total = 0;
    int64_t rec_groups = 0;  // warp groups of the radius launches
    int rec_cap[kLaunchSets] = {0, 0, 0, 0, 0, 0, 0, 0};  // record slots per group of each radius launch
    bool knn_exact[kLaunchSets] = {true, true, true, true, true, true, true, true};  // every k equals the class's
    bool knn_wexact[kLaunchSets] = {true, true, true, true, true, true, true, true};  // and every seeding window
    int64_t rec_slots = 0;   // record slots of all radius launches
    int64_t int_bound = 0;   // internal nodes of all clouds at most
};

static void make_tables(const sfc_batch_cloud* clouds, int n_clouds, int ncap, BatchTables& T) {
    T.n_clouds = n_clouds;
    T.seg.resize(n_clouds);
    T.out0.assign(n_clouds, 0);
    std::vector<SearchSeg> sets[kLaunchSets];
    std::vector<int32_t> set_cloud[kLaunchSets];
    int64_t p = 0;
    for (int i = 0; i < n_clouds; ++i) {
        const sfc_batch_cloud& c = clouds[i];
        BatchSeg& g = T.seg[i];
        memset(&g, 0, sizeof g);
        g.p0 = p;
        g.n = c.n_points;
        g.ncap = c.leaf_capacity > 0 ? c.leaf_capacity : ncap;
        T.int_bound += internal_bound(c.n_points, g.ncap);
        T.where.push_back(p);
        T.where.push_back(p + c.n_points);
        if (c.n_points > 0) {
            SearchSeg q;
            memset(&q, 0, sizeof q);
            q.q0 = p;
            q.nq = c.n_points;
            q.k = c.k;
            q.r = c.r;
            q.r2 = c.r * c.r;
            q.window = c.knn_window > 0 ? c.knn_window : knn_default_window(c.k);
            q.group_size = c.queries_per_warp > 0 ? c.queries_per_warp : 32;
            if (c.search == SFC_SEARCH_RADIUS) {
                if (c.r > 0.f) {  // r <= 0: every row empty
                    q.row0 = p;
                    sets[c.kernel].push_back(q);
                    set_cloud[c.kernel].push_back(i);
                    const int slots = c.record_slots > 0 ? c.record_slots : kRecordCap;
                    if (slots > T.rec_cap[c.kernel]) T.rec_cap[c.kernel] = slots;
                }
            } else {
                q.row0 = T.knn_total;
                T.out0[i] = T.knn_total;
                T.knn_total += c.n_points * c.k;
                const int b = 4 + (c.k <= 8 ? 0 : (c.k <= 16 ? 1 : (c.k <= 32 ? 2 : 3)));
                if (c.k != (8 << (b - 4))) T.knn_exact[b] = false;
                if (q.window != (8 << (b - 4))) T.knn_wexact[b] = false;
                sets[b].push_back(q);
                set_cloud[b].push_back(i);
            }
        }
        p += c.n_points;
    }
    T.n_total = p;
    for (int t = 0; t < kLaunchSets; ++t) {
        T.off[t] = static_cast<int64_t>(T.table.size());
        T.count[t] = static_cast<int64_t>(sets[t].size());
        int64_t g = 0;
        for (size_t j = 0; j < sets[t].size(); ++j) {
            sets[t][j].group0 = g;
            g += (sets[t][j].nq + sets[t][j].group_size - 1) / sets[t][j].group_size;
            T.table.push_back(sets[t][j]);
            T.table_cloud.push_back(set_cloud[t][j]);
        }
        T.groups[t] = g;
        if (t < 4) {
            T.rec_groups += g;
            T.rec_slots += g * T.rec_cap[t];
        }
    }
}

// The device buffers of one batch run.
struct BatchBuffers {
    uint64_t *codes = nullptr, *k0 = nullptr, *k1 = nullptr;
    uint32_t *v0 = nullptr, *v1 = nullptr, *perm = nullptr, *cnt = nullptr, *counts = nullptr;
    float4* pts = nullptr;
    int64_t* first = nullptr;
    BatchSeg* segs = nullptr;
    SearchSeg* table = nullptr;
    int32_t* table_cloud = nullptr;
    int64_t *where = nullptr, *bounds = nullptr;
    BatchTotals* tot = nullptr;
    unsigned int* err = nullptr;
    int64_t int_cap = 0, node_cap = 0, leaf_cap = 0;  // tree capacities
    NodeBox* nodes = nullptr;
    int32_t *child = nullptr, *islot = nullptr;
    uint64_t *ikey = nullptr, *leaves = nullptr;
    uint8_t* ilevel = nullptr;
    uint32_t* leaf_counts = nullptr;
    unsigned int* arrive = nullptr;
    BatchRecords rec;  // hit-mask records of the radius launches (optional)
};

// per-point buffers and tables (not the trees, the records or the outputs)
static sfc_status alloc_base(const BatchTables& T, BatchBuffers& b, Scratch& m) {
    const int64_t n = T.n_total;
    SFC_TRY(m.alloc(&b.codes, n));
    SFC_TRY(m.alloc(&b.k0, n));
    SFC_TRY(m.alloc(&b.k1, n));
    SFC_TRY(m.alloc(&b.v0, n));
    SFC_TRY(m.alloc(&b.v1, n));
    SFC_TRY(m.alloc(&b.perm, n));
    SFC_TRY(m.alloc(&b.cnt, n));
    SFC_TRY(m.alloc(&b.counts, n));
    SFC_TRY(m.alloc(&b.pts, n));
    SFC_TRY(m.alloc(&b.first, n + 1));
    SFC_TRY(m.alloc(&b.segs, T.n_clouds));
    SFC_TRY(m.alloc(&b.table, T.table.size()));
    SFC_TRY(m.alloc(&b.table_cloud, T.table.size()));
    SFC_TRY(m.alloc(&b.where, T.where.size()));
    SFC_TRY(m.alloc(&b.bounds, T.where.size()));
    SFC_TRY(m.alloc(&b.tot, 1));
    SFC_TRY(m.alloc(&b.err, 1));
    return SFC_OK;
}

static sfc_status alloc_trees(BatchBuffers& b, Scratch& m) {
    SFC_TRY(m.alloc(&b.nodes, b.node_cap));
    SFC_TRY(m.alloc(&b.child, b.node_cap));
    SFC_TRY(m.alloc(&b.islot, b.int_cap));
    SFC_TRY(m.alloc(&b.ikey, b.int_cap));
    SFC_TRY(m.alloc(&b.ilevel, b.int_cap));
    SFC_TRY(m.alloc(&b.arrive, b.int_cap));
    SFC_TRY(m.alloc(&b.leaves, b.leaf_cap));
    SFC_TRY(m.alloc(&b.leaf_counts, b.leaf_cap));
    return SFC_OK;
}

// Records for every radius warp group; without the memory the fill walks the trees again.
static void alloc_records(const BatchTables& T, BatchBuffers& b, Scratch& m) {
    b.rec = BatchRecords();
    if (T.rec_groups == 0) return;
    const int64_t slots = T.rec_slots;
    BatchRecords r;
    if (m.try_alloc(&r.masks, 32 * slots) && m.try_alloc(&r.head, slots) && m.try_alloc(&r.count, T.rec_groups))
        b.rec = r;
}

static sfc_status upload_tables(const BatchTables& T, BatchBuffers& b, cudaStream_t s) {
    SFC_CUDA(cudaMemcpyAsync(b.segs, T.seg.data(), sizeof(BatchSeg) * T.n_clouds, cudaMemcpyHostToDevice, s));
    if (!T.table.empty()) {
        SFC_CUDA(cudaMemcpyAsync(b.table, T.table.data(), sizeof(SearchSeg) * T.table.size(), cudaMemcpyHostToDevice,
                                 s));
        SFC_CUDA(cudaMemcpyAsync(b.table_cloud, T.table_cloud.data(), sizeof(int32_t) * T.table.size(),
                                 cudaMemcpyHostToDevice, s));
    }
    SFC_CUDA(cudaMemcpyAsync(b.where, T.where.data(), sizeof(int64_t) * T.where.size(), cudaMemcpyHostToDevice, s));
    return SFC_OK;
}

// Sections 4 and 5.1 up to the node counts: per-cloud boxes and codes, the (cloud, code)
// order, the gathered points, the internal nodes of every cloud and the slices they get.
static sfc_status enqueue_order(const BatchTables& T, BatchBuffers& b, const float* xyz, int enc, cudaStream_t s,
                                Scratch& tmp) {
    const int nsegs = T.n_clouds;
    const int64_t n = T.n_total;
    const unsigned int sgrid = grid_for(nsegs, 128);
    const unsigned int grid = grid_for(n, 256, 152 * 16);
    SFC_CUDA(cudaMemsetAsync(b.err, 0, sizeof(unsigned int), s));
    SFC_LAUNCH("batch_bbox_init", s, k_bseg_init, sgrid, 128, 0, b.segs, nsegs);
    SFC_LAUNCH("batch_bbox", s, k_batch_bbox, grid, 256, 0, xyz, n, b.segs, nsegs);
    SFC_LAUNCH("batch_bbox_finish", s, k_batch_bbox_finish, sgrid, 128, 0, b.segs, nsegs);
    SFC_TRY(batch_encode(xyz, n, enc, b.segs, nsegs, b.codes, b.v0, s));
    SFC_CUDA(cudaMemcpyAsync(b.k0, b.codes, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
    SFC_TRY(radix_sort_pairs(b.k0, b.v0, b.k1, b.v1, n, s, tmp, b.err));
    if (nsegs > 1) {  // stable pass on the cloud number: order (cloud, code)
        SFC_LAUNCH("batch_cloud_keys", s, k_batch_cloud_keys, grid, 256, 0, b.v0, n, b.segs, nsegs, b.k0);
        int bits = 0;
        while ((1 << bits) < nsegs) ++bits;
        SFC_TRY(radix_sort_pairs_bits(b.k0, b.v0, b.k1, b.v1, n, 0, bits, s, tmp, b.err));
    }
    // k1 receives the sorted codes
    SFC_LAUNCH("batch_gather", s, k_batch_gather, grid, 256, 0, xyz, n, b.codes, b.v0, b.segs, nsegs, b.k1, b.pts,
               b.perm);
    SFC_LAUNCH("batch_tree_count", s, k_batch_tree_count, grid, 256, 0, b.k1, n, b.segs, nsegs, b.cnt);
    SFC_TRY(scan_u32_to_i64(b.cnt, b.first, n, s, tmp, b.err));
    SFC_LAUNCH("batch_seg_internal", s, k_batch_seg_internal, sgrid, 128, 0, b.segs, nsegs, b.first);
    SFC_LAUNCH("batch_layout", s, k_batch_layout, 1, 1024, 0, b.segs, nsegs, b.int_cap, b.node_cap, b.leaf_cap, b.table,
               b.table_cloud, static_cast<int>(T.table.size()), b.tot);
    return SFC_OK;
}

// Section 5.1: the linear octrees of all clouds (sizes read on the device).
static sfc_status enqueue_trees(const BatchTables& T, BatchBuffers& b, cudaStream_t s) {
    const int nsegs = T.n_clouds;
    const int64_t n = T.n_total;
    const unsigned int grid = grid_for(n, 256, 152 * 16);
    const unsigned int igrid = grid_for(std::max<int64_t>(b.int_cap, 1), 256, 152 * 16);
    const unsigned int ngrid = grid_for(b.node_cap, 256, 152 * 16);
    SFC_LAUNCH("batch_tree_init", s, k_batch_tree_init, ngrid, 256, 0, b.child, b.arrive, b.tot);
    SFC_LAUNCH("batch_tree_emit", s, k_batch_tree_emit, grid, 256, 0, b.k1, n, b.segs, nsegs, b.cnt, b.first, b.ikey,
               b.ilevel, b.tot);
    SFC_LAUNCH("batch_tree_link", s, k_batch_tree_link, igrid, 256, 0, b.ikey, b.ilevel, b.tot, b.segs, nsegs, b.child,
               b.islot);
    SFC_LAUNCH("batch_tree_nodes", s, k_batch_tree_nodes, ngrid, 256, 0, b.k1, b.ikey, b.ilevel, b.segs, nsegs, b.tot,
               b.child, b.nodes, b.leaves, b.leaf_counts);
    SFC_LAUNCH("batch_tree_boxes", s, k_batch_tree_boxes, ngrid, 256, 0, b.pts, b.segs, nsegs, b.nodes, b.child,
               b.islot, b.arrive, b.tot);
    return SFC_OK;
}

static BatchRecords records_of(const BatchTables& T, const BatchBuffers& b, int kern) {
    BatchRecords r;
    if (!b.rec.masks) return r;
    int64_t g = 0, slot = 0;
    for (int t = 0; t < kern; ++t) {
        g += T.groups[t];
        slot += T.groups[t] * T.rec_cap[t];
    }
    r.masks = b.rec.masks + slot * 32;
    r.head = b.rec.head + slot;
    r.count = b.rec.count + g;
    r.cap = T.rec_cap[kern];
    return r;
}

// Section 3.3 for every kNN cloud: one launch per list size.
static sfc_status enqueue_knn(const BatchTables& T, BatchBuffers& b, int32_t* knn_idx, float* knn_d2, cudaStream_t s) {
    const int kmax_of[4] = {8, 16, 32, 64};
    for (int t = 4; t < kLaunchSets; ++t)
        SFC_TRY(batch_knn_launch(b.pts, b.perm, b.nodes, b.child, b.node_cap, b.table + T.off[t],
                                 static_cast<int>(T.count[t]), T.groups[t], kmax_of[t - 4],
                                 T.knn_exact[t] ? (T.knn_wexact[t] ? 2 : 1) : 0, knn_idx,
                                 knn_d2, b.err, &b.tot->flags, kOverNodes | kNonFinite, s));
    return SFC_OK;
}

// Section 5.1 neighboursPrune, count pass, then the row pointers.
static sfc_status enqueue_radius_count(const BatchTables& T, BatchBuffers& b, int prune, int64_t* row_ptr,
                                       cudaStream_t s, Scratch& tmp) {
    SFC_CUDA(cudaMemsetAsync(b.counts, 0, sizeof(uint32_t) * T.n_total, s));
    for (int kern = 0; kern < 4; ++kern)
        SFC_TRY(batch_radius_launch(b.pts, b.perm, b.nodes, b.child, b.node_cap, b.table + T.off[kern],
                                    static_cast<int>(T.count[kern]), T.groups[kern], kern, false, b.counts, nullptr,
                                    nullptr, b.err, prune, records_of(T, b, kern), &b.tot->flags, kOverNodes | kNonFinite,
                                    s));
    return scan_u32_to_i64(b.counts, row_ptr, T.n_total, s, tmp, b.err);
}

// The fill pass into cols (capacity cols_cap), then every cloud's row bounds.
static sfc_status enqueue_radius_fill(const BatchTables& T, BatchBuffers& b, int prune, const int64_t* row_ptr,
                                      int32_t* cols, int64_t cols_cap, int64_t* rel_rows, cudaStream_t s) {
    SFC_LAUNCH("batch_check_cols", s, k_batch_check_cols, 1, 1, 0, row_ptr + T.n_total, cols_cap, b.tot);
    for (int kern = 0; kern < 4; ++kern)
        SFC_TRY(batch_radius_launch(b.pts, b.perm, b.nodes, b.child, b.node_cap, b.table + T.off[kern],
                                    static_cast<int>(T.count[kern]), T.groups[kern], kern, true, b.counts, row_ptr,
                                    cols, b.err, prune, records_of(T, b, kern), &b.tot->flags,
                                    kOverNodes | kOverCols | kNonFinite, s));
    SFC_LAUNCH("batch_row_bounds", s, k_batch_row_bounds, grid_for(static_cast<int64_t>(T.where.size()), 128), 128, 0,
               row_ptr, b.where, static_cast<int>(T.where.size()), b.bounds);
    const int64_t rel_total = T.n_total + T.n_clouds;
    SFC_LAUNCH("batch_rel_rows", s, k_batch_rel_rows, grid_for(rel_total, 256, 152 * 8), 256, 0, row_ptr, b.segs,
               T.n_clouds, rel_total, rel_rows);
    return SFC_OK;
}

static sfc_status check_batch_args(const sfc_batch_cloud* clouds, int32_t n_clouds, sfc_encoding enc,
                                   const sfc_build_opts* opts, sfc_build_opts* o, int64_t* total) {
    if (!clouds || n_clouds < 1) return SFC_ERR_INVALID;
    if (n_clouds > kBatchMax) return SFC_ERR_TOO_LARGE;
    if (enc != SFC_ENC_MORTON && enc != SFC_ENC_HILBERT) return SFC_ERR_INVALID;
    sfc_build_opts_default(o);
    if (opts) *o = *opts;
    if (o->leaf_capacity < 1 || (o->prune != 0 && o->prune != 1)) return SFC_ERR_INVALID;
    *total = 0;
    for (int i = 0; i < n_clouds; ++i) {
        const sfc_batch_cloud& c = clouds[i];
        if (c.n_points < 0 || c.leaf_capacity < 0 || c.knn_window < 0 || c.knn_window > 64) return SFC_ERR_INVALID;
        if (c.queries_per_warp != 0 && c.queries_per_warp != 8 && c.queries_per_warp != 16 && c.queries_per_warp != 32)
            return SFC_ERR_INVALID;
        if (c.record_slots < 0 || c.record_slots > kRecordCapMax) return SFC_ERR_INVALID;
        if (c.search == SFC_SEARCH_RADIUS) {
            if (c.kernel < 0 || c.kernel > 3 || isnan(c.r)) return SFC_ERR_INVALID;
        } else if (c.search == SFC_SEARCH_KNN) {
            if (c.k < 1) return SFC_ERR_INVALID;
            if (c.k > kMaxK) return SFC_ERR_TOO_LARGE;
        } else {
            return SFC_ERR_INVALID;
        }
        *total += c.n_points;
    }
    if (*total > 0x7fffffffLL - 1) return SFC_ERR_TOO_LARGE;
    return SFC_OK;
}

}  // namespace sfc

// ---------------------------------------------------------------------------------
// batch_search: one pass with exact sizes (the host waits for the node counts and the
// radius output size)
struct sfc_batch_s {
    sfc::BatchTables T;
    std::vector<sfc_batch_cloud> clouds_;
    std::vector<int64_t> row_lo, row_hi;  // radius clouds: row_ptr[p0], row_ptr[p0 + n]
    int64_t nnz = 0;
    int64_t* row_ptr = nullptr;
    int64_t* rel_rows = nullptr;  // every cloud's row pointers, starting at 0 (see k_batch_rel_rows)
    int32_t* cols = nullptr;
    int32_t* knn_idx = nullptr;
    float* knn_d2 = nullptr;
};

namespace sfc {

// A second stream for the kNN launches of a recorded plan, which depend on the trees
// only: they run beside the radius launches and fill each other's tails (145.6 vs 149 ms
// per run on the 256-cloud batch).
struct SideStream {
    cudaStream_t s2 = nullptr;
    cudaEvent_t forked = nullptr, joined = nullptr;
    sfc_status init() {
        SFC_CUDA(cudaStreamCreateWithFlags(&s2, cudaStreamNonBlocking));
        SFC_CUDA(cudaEventCreateWithFlags(&forked, cudaEventDisableTiming));
        SFC_CUDA(cudaEventCreateWithFlags(&joined, cudaEventDisableTiming));
        return SFC_OK;
    }
    sfc_status fork(cudaStream_t s) {  // s2 starts after what s has queued so far
        SFC_CUDA(cudaEventRecord(forked, s));
        SFC_CUDA(cudaStreamWaitEvent(s2, forked, 0));
        return SFC_OK;
    }
    sfc_status join(cudaStream_t s) {  // s continues after what s2 has queued so far
        SFC_CUDA(cudaEventRecord(joined, s2));
        SFC_CUDA(cudaStreamWaitEvent(s, joined, 0));
        return SFC_OK;
    }
    ~SideStream() {  // queued work still completes; the handles are released afterwards
        if (joined) cudaEventDestroy(joined);
        if (forked) cudaEventDestroy(forked);
        if (s2) cudaStreamDestroy(s2);
    }
};

static sfc_status run_batch(sfc_batch_s* B, const float* xyz, int enc, const sfc_build_opts& o, cudaStream_t s) {
    const BatchTables& T = B->T;
    const int64_t n = T.n_total;
    Scratch tmp(s);
    BatchBuffers b;
    b.int_cap = b.node_cap = b.leaf_cap = INT64_MAX;  // sized once the counts are known
    SFC_TRY(alloc_base(T, b, tmp));
    SFC_TRY(upload_tables(T, b, s));
    SFC_TRY(enqueue_order(T, b, xyz, enc, s, tmp));
    BatchTotals ht;
    SFC_CUDA(cudaMemcpyAsync(&ht, b.tot, sizeof ht, cudaMemcpyDeviceToHost, s));
    SFC_CUDA(cudaStreamSynchronize(s));
    if (ht.flags & kNonFinite) return SFC_ERR_NOT_FINITE;
    if (ht.flags & kOverNodes) return SFC_ERR_TOO_LARGE;
    b.int_cap = ht.n_int;
    b.node_cap = ht.n_nodes;
    b.leaf_cap = ht.n_leaves;
    SFC_TRY(alloc_trees(b, tmp));
    SFC_TRY(enqueue_trees(T, b, s));
    // kNN first, then the radius count: the device works through both while the host
    // waits for the radius output size (a second stream for the kNN measured slower here,
    // 168 vs 149 ms on the 256-cloud batch, though it helps the recorded plan)
    SFC_TRY(dev_alloc(&B->knn_idx, T.knn_total, s));
    SFC_TRY(dev_alloc(&B->knn_d2, T.knn_total, s));
    SFC_TRY(enqueue_knn(T, b, B->knn_idx, B->knn_d2, s));
    SFC_TRY(dev_alloc(&B->row_ptr, n + 1, s));
    alloc_records(T, b, tmp);
    SFC_TRY(enqueue_radius_count(T, b, o.prune, B->row_ptr, s, tmp));
    SFC_CUDA(cudaMemcpyAsync(&B->nnz, B->row_ptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SFC_CUDA(cudaStreamSynchronize(s));
    SFC_TRY(dev_alloc(&B->cols, B->nnz, s));
    SFC_TRY(dev_alloc(&B->rel_rows, n + T.n_clouds, s));
    SFC_TRY(enqueue_radius_fill(T, b, o.prune, B->row_ptr, B->cols, B->nnz, B->rel_rows, s));
    std::vector<int64_t> bounds(T.where.size());
    unsigned int herr = 0;
    SFC_CUDA(cudaMemcpyAsync(bounds.data(), b.bounds, sizeof(int64_t) * bounds.size(), cudaMemcpyDeviceToHost, s));
    SFC_CUDA(cudaMemcpyAsync(&herr, b.err, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    SFC_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < T.n_clouds; ++i) {
        B->row_lo[i] = bounds[2 * i];
        B->row_hi[i] = bounds[2 * i + 1];
    }
    SFC_TRY(guard_status(herr));
    return SFC_OK;
}

static void free_batch(sfc_batch_s* B, cudaStream_t s) {
    dev_free(B->row_ptr, s);
    dev_free(B->rel_rows, s);
    B->rel_rows = nullptr;
    dev_free(B->cols, s);
    dev_free(B->knn_idx, s);
    dev_free(B->knn_d2, s);
    B->row_ptr = nullptr;
    B->cols = nullptr;
    B->knn_idx = nullptr;
    B->knn_d2 = nullptr;
}

// views of one cloud's results (shared by batches and plans)
static sfc_status cloud_views(const BatchTables& T, int32_t cloud, const int64_t* rel_rows, const int32_t* cols,
                              const int32_t* knn_idx, const float* knn_d2, const std::vector<int64_t>& row_lo,
                              const std::vector<int64_t>& row_hi, const int64_t** rp, const int32_t** cl,
                              int64_t* nnz, const int32_t** ki, const float** kd, const sfc_batch_cloud& c) {
    const bool radius = c.search == SFC_SEARCH_RADIUS;
    if (rp) *rp = radius ? rel_rows + T.seg[cloud].p0 + cloud : nullptr;
    if (cl) *cl = radius ? cols + row_lo[cloud] : nullptr;
    if (nnz) *nnz = radius ? row_hi[cloud] - row_lo[cloud] : 0;
    if (ki) *ki = radius ? nullptr : knn_idx + T.out0[cloud];
    if (kd) *kd = radius ? nullptr : knn_d2 + T.out0[cloud];
    return SFC_OK;
}

// ---------------------------------------------------------------------------------
// autotuning: one timed pass of the batch, the build timed whole and every launch set
// (radius kernel type: count + fill; kNN list size) on its own, with CUDA events
class EventTimer {
  public:
    explicit EventTimer(cudaStream_t s) : s_(s) {}
    ~EventTimer() {
        for (auto& e : ev_) cudaEventDestroy(e);
    }
    sfc_status mark(int* id) {
        cudaEvent_t e;
        SFC_CUDA(cudaEventCreate(&e));
        ev_.push_back(e);
        SFC_CUDA(cudaEventRecord(e, s_));
        *id = static_cast<int>(ev_.size()) - 1;
        return SFC_OK;
    }
    float ms(int a, int b) const {
        float t = 0.f;
        cudaEventElapsedTime(&t, ev_[a], ev_[b]);
        return t;
    }

  private:
    cudaStream_t s_;
    std::vector<cudaEvent_t> ev_;
};

static sfc_status timed_pass(const std::vector<sfc_batch_cloud>& clouds, const float* xyz, int enc,
                             const sfc_build_opts& o, cudaStream_t s, float* build_ms, float* set_ms) {
    BatchTables T;
    make_tables(clouds.data(), static_cast<int>(clouds.size()), o.leaf_capacity, T);
    const int64_t n = T.n_total;
    Scratch tmp(s);
    EventTimer ev(s);
    BatchBuffers b;
    b.int_cap = b.node_cap = b.leaf_cap = INT64_MAX;
    SFC_TRY(alloc_base(T, b, tmp));
    SFC_TRY(upload_tables(T, b, s));
    int e0, ea, e1, e2;
    SFC_TRY(ev.mark(&e0));
    SFC_TRY(enqueue_order(T, b, xyz, enc, s, tmp));
    SFC_TRY(ev.mark(&ea));
    BatchTotals ht;
    SFC_CUDA(cudaMemcpyAsync(&ht, b.tot, sizeof ht, cudaMemcpyDeviceToHost, s));
    SFC_CUDA(cudaStreamSynchronize(s));
    if (ht.flags & kNonFinite) return SFC_ERR_NOT_FINITE;
    if (ht.flags & kOverNodes) return SFC_ERR_TOO_LARGE;
    b.int_cap = ht.n_int;
    b.node_cap = ht.n_nodes;
    b.leaf_cap = ht.n_leaves;
    SFC_TRY(alloc_trees(b, tmp));
    SFC_TRY(ev.mark(&e1));
    SFC_TRY(enqueue_trees(T, b, s));
    SFC_TRY(ev.mark(&e2));
    int32_t* knn_idx = nullptr;
    float* knn_d2 = nullptr;
    SFC_TRY(tmp.alloc(&knn_idx, T.knn_total));
    SFC_TRY(tmp.alloc(&knn_d2, T.knn_total));
    const int kmax_of[4] = {8, 16, 32, 64};
    int mk[kLaunchSets][2];
    for (int t = 4; t < kLaunchSets; ++t) {
        SFC_TRY(ev.mark(&mk[t][0]));
        SFC_TRY(batch_knn_launch(b.pts, b.perm, b.nodes, b.child, b.node_cap, b.table + T.off[t],
                                 static_cast<int>(T.count[t]), T.groups[t], kmax_of[t - 4],
                                 T.knn_exact[t] ? (T.knn_wexact[t] ? 2 : 1) : 0, knn_idx,
                                 knn_d2, b.err, &b.tot->flags, kOverNodes | kNonFinite, s));
        SFC_TRY(ev.mark(&mk[t][1]));
    }
    int64_t* row_ptr = nullptr;
    SFC_TRY(tmp.alloc(&row_ptr, n + 1));
    alloc_records(T, b, tmp);
    SFC_CUDA(cudaMemsetAsync(b.counts, 0, sizeof(uint32_t) * n, s));
    int mc[4][2], mf[4][2];
    for (int kern = 0; kern < 4; ++kern) {
        SFC_TRY(ev.mark(&mc[kern][0]));
        SFC_TRY(batch_radius_launch(b.pts, b.perm, b.nodes, b.child, b.node_cap, b.table + T.off[kern],
                                    static_cast<int>(T.count[kern]), T.groups[kern], kern, false, b.counts, nullptr,
                                    nullptr, b.err, o.prune, records_of(T, b, kern), &b.tot->flags,
                                    kOverNodes | kNonFinite, s));
        SFC_TRY(ev.mark(&mc[kern][1]));
    }
    SFC_TRY(scan_u32_to_i64(b.counts, row_ptr, n, s, tmp, b.err));
    int64_t nnz = 0;
    SFC_CUDA(cudaMemcpyAsync(&nnz, row_ptr + n, sizeof nnz, cudaMemcpyDeviceToHost, s));
    SFC_CUDA(cudaStreamSynchronize(s));
    int32_t* cols = nullptr;
    SFC_TRY(tmp.alloc(&cols, nnz));
    for (int kern = 0; kern < 4; ++kern) {
        SFC_TRY(ev.mark(&mf[kern][0]));
        SFC_TRY(batch_radius_launch(b.pts, b.perm, b.nodes, b.child, b.node_cap, b.table + T.off[kern],
                                    static_cast<int>(T.count[kern]), T.groups[kern], kern, true, b.counts, row_ptr,
                                    cols, b.err, o.prune, records_of(T, b, kern), &b.tot->flags,
                                    kOverNodes | kNonFinite, s));
        SFC_TRY(ev.mark(&mf[kern][1]));
    }
    unsigned int herr = 0;
    SFC_CUDA(cudaMemcpyAsync(&herr, b.err, sizeof herr, cudaMemcpyDeviceToHost, s));
    SFC_CUDA(cudaStreamSynchronize(s));
    SFC_TRY(guard_status(herr));
    *build_ms = ev.ms(e0, ea) + ev.ms(e1, e2);  // the host wait between the two is not build time
    for (int kern = 0; kern < 4; ++kern) set_ms[kern] = ev.ms(mc[kern][0], mc[kern][1]) + ev.ms(mf[kern][0], mf[kern][1]);
    for (int t = 4; t < kLaunchSets; ++t) set_ms[t] = ev.ms(mk[t][0], mk[t][1]);
    return SFC_OK;
}

static int launch_set_of(const sfc_batch_cloud& c) {
    if (c.n_points == 0) return -1;
    if (c.search == SFC_SEARCH_RADIUS) return c.r > 0.f ? c.kernel : -1;
    return 4 + (c.k <= 8 ? 0 : (c.k <= 16 ? 1 : (c.k <= 32 ? 2 : 3)));
}

}  // namespace sfc

// ---------------------------------------------------------------------------------
// batch plans: the same pass recorded once as a CUDA graph over buffers sized in advance
// (trees by the bound on internal nodes, the radius output by a capacity), so that a run
// is one graph launch with no allocation and no host wait.  Overflows are found on the
// device (the searches of the run are skipped) and repaired in batch_plan_finish.
struct sfc_batch_plan_s {
    sfc::BatchTables T;
    std::vector<sfc_batch_cloud> clouds;
    int enc = 0;
    sfc_build_opts o{};
    cudaStream_t cs = nullptr;      // capture stream
    sfc::SideStream side;           // the kNN launches' stream inside the graph
    sfc::Scratch* mem = nullptr;    // buffers that live as long as the plan
    sfc::Scratch* trees = nullptr;  // the tree buffers (replaced when they overflow)
    sfc::BatchBuffers b;
    float* xyz = nullptr;
    int64_t* row_ptr = nullptr;
    int64_t* rel_rows = nullptr;  // every cloud's row pointers, starting at 0
    int32_t* cols = nullptr;
    int64_t cols_cap = 0;
    int32_t* knn_idx = nullptr;
    float* knn_d2 = nullptr;
    struct Status {
        sfc::BatchTotals tot;
        unsigned int err;
        unsigned int pad;
    }* host = nullptr;              // pinned, written by the graph's last copies
    int64_t* host_bounds = nullptr; // pinned
    std::vector<int64_t> row_lo, row_hi;
    cudaGraphExec_t exec = nullptr;
    uint64_t kernels_per_run = 0;
    cudaEvent_t done = nullptr;
    bool launched = false;
    bool ready = false;  // results of the last run are complete
};

namespace sfc {

static void release_cols(sfc_batch_plan_s* P) {
    dev_free(P->cols, P->cs);
    P->cols = nullptr;
}

static sfc_status capture_plan(sfc_batch_plan_s* P) {
    if (P->exec) {
        cudaGraphExecDestroy(P->exec);
        P->exec = nullptr;
    }
    const uint64_t launches0 = sfc_launch_count();
    cudaGraph_t graph = nullptr;
    SFC_CUDA(cudaStreamBeginCapture(P->cs, cudaStreamCaptureModeThreadLocal));
    sfc_status st = SFC_OK;
    {
        Scratch tmp(P->cs, true);  // temporaries of one run (sort and scan work arrays): graph allocations
        const cudaStream_t s = P->cs;
        BatchBuffers& b = P->b;
        st = enqueue_order(P->T, b, P->xyz, P->enc, s, tmp);
        if (st == SFC_OK) st = enqueue_trees(P->T, b, s);
        bool forked = false;
        if (st == SFC_OK && (st = P->side.fork(s)) == SFC_OK) forked = true;  // kNN beside the radius launches
        if (st == SFC_OK) st = enqueue_knn(P->T, b, P->knn_idx, P->knn_d2, P->side.s2);
        if (st == SFC_OK) st = enqueue_radius_count(P->T, b, P->o.prune, P->row_ptr, s, tmp);
        if (st == SFC_OK)
            st = enqueue_radius_fill(P->T, b, P->o.prune, P->row_ptr, P->cols, P->cols_cap, P->rel_rows, s);
        if (forked) {  // the capture must end on one stream
            const sfc_status js = P->side.join(s);
            if (st == SFC_OK) st = js;
        }
        if (st == SFC_OK &&
            (cudaMemcpyAsync(P->host_bounds, b.bounds, sizeof(int64_t) * P->T.where.size(), cudaMemcpyDeviceToHost,
                             s) != cudaSuccess ||
             cudaMemcpyAsync(&P->host->tot, b.tot, sizeof(BatchTotals), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
             cudaMemcpyAsync(&P->host->err, b.err, sizeof(unsigned int), cudaMemcpyDeviceToHost, s) != cudaSuccess))
            st = SFC_ERR_CUDA;
    }
    const cudaError_t e = cudaStreamEndCapture(P->cs, &graph);
    P->kernels_per_run = sfc_launch_count() - launches0;
    if (st != SFC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) {
        record_cuda_error(e, "cudaStreamEndCapture");
        if (graph) cudaGraphDestroy(graph);
        return SFC_ERR_CUDA;
    }
    const cudaError_t ie = cudaGraphInstantiate(&P->exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ie != cudaSuccess) {
        record_cuda_error(ie, "cudaGraphInstantiate");
        P->exec = nullptr;
        return SFC_ERR_CUDA;
    }
    return SFC_OK;
}

static sfc_status plan_alloc_trees(sfc_batch_plan_s* P, int64_t int_cap) {
    delete P->trees;
    P->trees = new (std::nothrow) Scratch(P->cs);
    if (!P->trees) return SFC_ERR_OOM;
    P->b.int_cap = int_cap;
    P->b.node_cap = P->T.n_clouds + 8 * int_cap;
    P->b.leaf_cap = 2 * P->T.n_clouds + 7 * int_cap;
    return alloc_trees(P->b, *P->trees);
}

static void destroy_plan(sfc_batch_plan_s* P) {
    if (P->exec) cudaGraphExecDestroy(P->exec);
    if (P->cs) cudaStreamSynchronize(P->cs);
    release_cols(P);
    delete P->trees;
    delete P->mem;
    if (P->cs) cudaStreamSynchronize(P->cs);
    if (P->host) cudaFreeHost(P->host);
    if (P->host_bounds) cudaFreeHost(P->host_bounds);
    if (P->done) cudaEventDestroy(P->done);
    if (P->cs) cudaStreamDestroy(P->cs);
    delete P;
}

}  // namespace sfc

extern "C" {

sfc_status batch_search(const float* points_xyz, const sfc_batch_cloud* clouds, int32_t n_clouds, sfc_encoding enc,
                        const sfc_build_opts* opts, void* cuda_stream, sfc_batch* out) {
    if (!out) return SFC_ERR_INVALID;
    *out = nullptr;
    sfc_build_opts o;
    int64_t total = 0;
    SFC_TRY(sfc::check_batch_args(clouds, n_clouds, enc, opts, &o, &total));
    if (total > 0 && (!points_xyz || !sfc::is_device_ptr(points_xyz))) return SFC_ERR_NOT_DEVICE_PTR;
    int dev = 0;
    SFC_CUDA(cudaGetDevice(&dev));
    SFC_TRY(sfc::ensure_pool(dev));
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    sfc_batch_s* B = new (std::nothrow) sfc_batch_s;
    if (!B) return SFC_ERR_OOM;
    sfc::make_tables(clouds, n_clouds, o.leaf_capacity, B->T);
    B->clouds_.assign(clouds, clouds + n_clouds);
    B->row_lo.assign(n_clouds, 0);
    B->row_hi.assign(n_clouds, 0);
    sfc_status st = total > 0 ? sfc::run_batch(B, points_xyz, enc, o, s) : SFC_OK;
    if (st == SFC_OK && total == 0) {
        st = sfc::dev_alloc(&B->row_ptr, 1, s);
        if (st == SFC_OK && cudaMemsetAsync(B->row_ptr, 0, sizeof(int64_t), s) != cudaSuccess) st = SFC_ERR_CUDA;
        if (st == SFC_OK) st = sfc::dev_alloc(&B->rel_rows, n_clouds, s);
        if (st == SFC_OK && cudaMemsetAsync(B->rel_rows, 0, sizeof(int64_t) * n_clouds, s) != cudaSuccess)
            st = SFC_ERR_CUDA;
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
    if (!b || cloud < 0 || cloud >= b->T.n_clouds) return SFC_ERR_INVALID;
    return sfc::cloud_views(b->T, cloud, b->rel_rows, b->cols, b->knn_idx, b->knn_d2, b->row_lo, b->row_hi, row_ptr,
                            cols, nnz, knn_idx, knn_d2, b->clouds_[cloud]);
}

sfc_status batch_free(sfc_batch b, void* cuda_stream) {
    if (!b) return SFC_ERR_INVALID;
    sfc::free_batch(b, static_cast<cudaStream_t>(cuda_stream));
    delete b;
    return SFC_OK;
}

sfc_status batch_plan_create(const sfc_batch_cloud* clouds, int32_t n_clouds, sfc_encoding enc,
                             const sfc_build_opts* opts, int64_t nnz_capacity, void* cuda_stream,
                             sfc_batch_plan* out) {
    if (!out) return SFC_ERR_INVALID;
    *out = nullptr;
    if (nnz_capacity < 0) return SFC_ERR_INVALID;
    sfc_build_opts o;
    int64_t total = 0;
    SFC_TRY(sfc::check_batch_args(clouds, n_clouds, enc, opts, &o, &total));
    if (total == 0) return SFC_ERR_INVALID;
    int dev = 0;
    SFC_CUDA(cudaGetDevice(&dev));
    SFC_TRY(sfc::ensure_pool(dev));
    cudaStream_t user = static_cast<cudaStream_t>(cuda_stream);
    SFC_CUDA(cudaStreamSynchronize(user));  // the plan's buffers come from its own stream
    sfc_batch_plan_s* P = new (std::nothrow) sfc_batch_plan_s;
    if (!P) return SFC_ERR_OOM;
    P->clouds.assign(clouds, clouds + n_clouds);
    P->enc = enc;
    P->o = o;
    sfc::make_tables(clouds, n_clouds, o.leaf_capacity, P->T);
    P->row_lo.assign(n_clouds, 0);
    P->row_hi.assign(n_clouds, 0);
    sfc_status st = SFC_OK;
    auto fail = [&](sfc_status e) {
        sfc::destroy_plan(P);
        return e;
    };
    if (cudaStreamCreateWithFlags(&P->cs, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&P->done, cudaEventDisableTiming) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&P->host), sizeof(sfc_batch_plan_s::Status)) != cudaSuccess ||
        cudaMallocHost(reinterpret_cast<void**>(&P->host_bounds), sizeof(int64_t) * P->T.where.size()) !=
            cudaSuccess)
        return fail(SFC_ERR_CUDA);
    if (P->side.init() != SFC_OK) return fail(SFC_ERR_CUDA);
    P->mem = new (std::nothrow) sfc::Scratch(P->cs);
    if (!P->mem) return fail(SFC_ERR_OOM);
    sfc::Scratch& m = *P->mem;
    const int64_t n = P->T.n_total;
    int64_t radius_points = 0;
    for (int t = 0; t < 4; ++t)
        for (int64_t j = 0; j < P->T.count[t]; ++j) radius_points += P->T.table[P->T.off[t] + j].nq;
    P->cols_cap = nnz_capacity > 0 ? nnz_capacity : 64 * radius_points;
    if ((st = m.alloc(&P->xyz, 3 * n)) != SFC_OK || (st = sfc::alloc_base(P->T, P->b, m)) != SFC_OK ||
        (st = m.alloc(&P->row_ptr, n + 1)) != SFC_OK || (st = m.alloc(&P->rel_rows, n + n_clouds)) != SFC_OK ||
        (st = m.alloc(&P->knn_idx, P->T.knn_total)) != SFC_OK ||
        (st = m.alloc(&P->knn_d2, P->T.knn_total)) != SFC_OK ||
        (st = sfc::dev_alloc(&P->cols, P->cols_cap, P->cs)) != SFC_OK ||
        (st = sfc::plan_alloc_trees(P, P->T.int_bound)) != SFC_OK)
        return fail(st);
    sfc::alloc_records(P->T, P->b, m);
    if ((st = sfc::upload_tables(P->T, P->b, P->cs)) != SFC_OK) return fail(st);
    if (cudaMemsetAsync(P->xyz, 0, sizeof(float) * 3 * (n ? n : 1), P->cs) != cudaSuccess) return fail(SFC_ERR_CUDA);
    if ((st = sfc::capture_plan(P)) != SFC_OK) return fail(st);
    if (cudaStreamSynchronize(P->cs) != cudaSuccess) return fail(SFC_ERR_CUDA);
    *out = P;
    return SFC_OK;
}

sfc_status batch_plan_points(sfc_batch_plan p, float** points_xyz) {
    if (!p || !points_xyz) return SFC_ERR_INVALID;
    *points_xyz = p->xyz;
    return SFC_OK;
}

sfc_status batch_plan_launch(sfc_batch_plan p, void* cuda_stream) {
    if (!p) return SFC_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    if (!p->exec) SFC_TRY(sfc::capture_plan(p));
    SFC_CUDA(cudaGraphLaunch(p->exec, s));
    SFC_CUDA(cudaEventRecord(p->done, s));
    sfc::count_launches(p->kernels_per_run);
    p->launched = true;
    p->ready = false;
    return SFC_OK;
}

sfc_status batch_plan_finish(sfc_batch_plan p, void* cuda_stream) {
    if (!p || !p->launched) return SFC_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    SFC_CUDA(cudaEventSynchronize(p->done));
    p->launched = false;
    sfc::BatchTotals tot = p->host->tot;
    if (tot.flags & sfc::kNonFinite) return SFC_ERR_NOT_FINITE;
    if (tot.flags & sfc::kOverNodes) {
        // the trees did not fit (the bound holds, so only a smaller capacity can do this)
        if (tot.n_nodes > 0x7fffffffLL) return SFC_ERR_TOO_LARGE;
        SFC_TRY(sfc::plan_alloc_trees(p, tot.n_int));
        SFC_CUDA(cudaStreamSynchronize(p->cs));
        SFC_TRY(sfc::capture_plan(p));
        SFC_TRY(batch_plan_launch(p, cuda_stream));
        return batch_plan_finish(p, cuda_stream);
    }
    if (tot.flags & sfc::kOverCols) {
        // the radius output did not fit: grow it and run the fill again (the counts, row
        // pointers and records of this run are still in place); the graph is recorded
        // again with the new array before the next launch
        sfc::release_cols(p);
        p->cols_cap = tot.nnz + tot.nnz / 8;
        if (cudaGraphExecDestroy(p->exec) == cudaSuccess) p->exec = nullptr;
        SFC_TRY(sfc::dev_alloc(&p->cols, p->cols_cap, p->cs));
        SFC_CUDA(cudaStreamSynchronize(p->cs));
        const unsigned int keep = tot.flags & ~sfc::kOverCols;
        SFC_CUDA(cudaMemcpyAsync(&p->b.tot->flags, &keep, sizeof keep, cudaMemcpyHostToDevice, s));
        SFC_TRY(sfc::enqueue_radius_fill(p->T, p->b, p->o.prune, p->row_ptr, p->cols, p->cols_cap, p->rel_rows, s));
        SFC_CUDA(cudaMemcpyAsync(p->host_bounds, p->b.bounds, sizeof(int64_t) * p->T.where.size(),
                                 cudaMemcpyDeviceToHost, s));
        SFC_CUDA(cudaMemcpyAsync(&p->host->err, p->b.err, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
        SFC_CUDA(cudaStreamSynchronize(s));
    }
    SFC_TRY(sfc::guard_status(p->host->err));
    for (int i = 0; i < p->T.n_clouds; ++i) {
        p->row_lo[i] = p->host_bounds[2 * i];
        p->row_hi[i] = p->host_bounds[2 * i + 1];
    }
    p->ready = true;
    return SFC_OK;
}

sfc_status batch_plan_result(sfc_batch_plan p, int32_t cloud, const int64_t** row_ptr, const int32_t** cols,
                             int64_t* nnz, const int32_t** knn_idx, const float** knn_d2) {
    if (!p || !p->ready || cloud < 0 || cloud >= p->T.n_clouds) return SFC_ERR_INVALID;
    return sfc::cloud_views(p->T, cloud, p->rel_rows, p->cols, p->knn_idx, p->knn_d2, p->row_lo, p->row_hi, row_ptr,
                            cols, nnz, knn_idx, knn_d2, p->clouds[cloud]);
}

sfc_status batch_plan_free(sfc_batch_plan p, void* cuda_stream) {
    if (!p) return SFC_ERR_INVALID;
    SFC_CUDA(cudaStreamSynchronize(static_cast<cudaStream_t>(cuda_stream)));
    sfc::destroy_plan(p);
    return SFC_OK;
}


sfc_status batch_autotune(const float* points_xyz, const sfc_batch_cloud* clouds, int32_t n_clouds, sfc_encoding enc,
                          const sfc_build_opts* opts, const int32_t* leaf_candidates, int32_t n_leaf,
                          const int32_t* window_candidates, int32_t n_window, const int32_t* qpw_candidates,
                          int32_t n_qpw, const int32_t* slot_candidates, int32_t n_slot, void* cuda_stream,
                          sfc_batch_cloud* tuned_out) {
    sfc_build_opts o;
    int64_t total = 0;
    SFC_TRY(sfc::check_batch_args(clouds, n_clouds, enc, opts, &o, &total));
    if (!tuned_out || n_leaf < 0 || n_window < 0 || n_qpw < 0 || n_slot < 0 || (n_leaf > 0 && !leaf_candidates) ||
        (n_window > 0 && !window_candidates) || (n_qpw > 0 && !qpw_candidates) || (n_slot > 0 && !slot_candidates))
        return SFC_ERR_INVALID;
    for (int i = 0; i < n_leaf; ++i)
        if (leaf_candidates[i] < 1) return SFC_ERR_INVALID;
    for (int i = 0; i < n_window; ++i)
        if (window_candidates[i] < 1 || window_candidates[i] > 64) return SFC_ERR_INVALID;
    for (int i = 0; i < n_qpw; ++i)
        if (qpw_candidates[i] != 8 && qpw_candidates[i] != 16 && qpw_candidates[i] != 32) return SFC_ERR_INVALID;
    for (int i = 0; i < n_slot; ++i)
        if (slot_candidates[i] < 1 || slot_candidates[i] > sfc::kRecordCapMax) return SFC_ERR_INVALID;
    if (total > 0 && (!points_xyz || !sfc::is_device_ptr(points_xyz))) return SFC_ERR_NOT_DEVICE_PTR;
    int dev = 0;
    SFC_CUDA(cudaGetDevice(&dev));
    SFC_TRY(sfc::ensure_pool(dev));
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    constexpr int kSets = sfc::kLaunchSets;
    std::vector<sfc_batch_cloud> cl(clouds, clouds + n_clouds);
    std::vector<int64_t> set_points(kSets, 0);
    for (const auto& c : cl) {
        const int t = sfc::launch_set_of(c);
        if (t >= 0) set_points[t] += c.n_points;
    }
    // the current choice of every set; a knob whose candidate list is empty keeps the
    // clouds' own values
    int32_t leaf[kSets], window[kSets], qpw[kSets], slots[kSets];
    for (int t = 0; t < kSets; ++t) leaf[t] = window[t] = qpw[t] = slots[t] = -1;
    auto apply = [&]() {
        for (int i = 0; i < n_clouds; ++i) {
            const int t = sfc::launch_set_of(clouds[i]);
            cl[i] = clouds[i];
            if (t < 0) continue;
            if (leaf[t] >= 0) cl[i].leaf_capacity = leaf[t];
            if (window[t] >= 0 && t >= 4) cl[i].knn_window = window[t];
            if (qpw[t] >= 0) cl[i].queries_per_warp = qpw[t];
            if (slots[t] >= 0 && t < 4) cl[i].record_slots = slots[t];
        }
    };
    // one timed pass per candidate of one knob (all sets at once): each set keeps the
    // candidate with its least cost (its search time, plus its points' share of the build
    // for the leaf capacity, which changes the build)
    auto tune = [&](int32_t* knob, const int32_t* cand, int32_t n_cand, int t_lo, int t_hi, bool with_build,
                    bool warm) -> sfc_status {
        if (n_cand == 0 || total == 0) return SFC_OK;
        float best[kSets];
        int32_t pick[kSets];
        for (int t = 0; t < kSets; ++t) {
            best[t] = INFINITY;
            pick[t] = knob[t];
        }
        for (int i = 0; i < n_cand; ++i) {
            for (int t = t_lo; t < t_hi; ++t) knob[t] = cand[i];
            apply();
            float build = 0.f, set_ms[kSets];
            if (warm && i == 0) SFC_TRY(sfc::timed_pass(cl, points_xyz, enc, o, s, &build, set_ms));
            SFC_TRY(sfc::timed_pass(cl, points_xyz, enc, o, s, &build, set_ms));
            for (int t = t_lo; t < t_hi; ++t) {
                if (set_points[t] == 0) continue;
                const float cost = set_ms[t] + (with_build ? build * static_cast<float>(set_points[t]) /
                                                                 static_cast<float>(total)
                                                           : 0.f);
                if (cost < best[t]) {
                    best[t] = cost;
                    pick[t] = cand[i];
                }
            }
        }
        for (int t = t_lo; t < t_hi; ++t) knob[t] = pick[t];
        apply();
        return SFC_OK;
    };
    SFC_TRY(tune(leaf, leaf_candidates, n_leaf, 0, kSets, true, true));
    SFC_TRY(tune(window, window_candidates, n_window, 4, kSets, false, false));
    SFC_TRY(tune(qpw, qpw_candidates, n_qpw, 0, kSets, false, false));
    SFC_TRY(tune(slots, slot_candidates, n_slot, 0, 4, false, false));
    apply();
    for (int i = 0; i < n_clouds; ++i) {
        tuned_out[i] = cl[i];
        if (tuned_out[i].leaf_capacity == 0) tuned_out[i].leaf_capacity = o.leaf_capacity;
        const int t = sfc::launch_set_of(clouds[i]);
        if (t >= 0 && t < 4) tuned_out[i].knn_window = 0;
        if (t < 0 || t >= 4) tuned_out[i].record_slots = 0;
        if (t < 0) tuned_out[i].knn_window = 0;
    }
    return SFC_OK;
}

}  // extern "C"
