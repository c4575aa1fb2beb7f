// sfc_build.cu - the build half of the path: bounding box and scale (section 4),
// Morton / Hilbert codes (sections 4.1, 4.2), reordering (section 4), and the linear
// octree (section 5.1): leaves and counts, internal nodes, internalRanges and a tight
// bounding box per node.
//
// Linear octree construction.  With the codes sorted, the cell of level l that holds
// sorted point i holds more than N_max points exactly when points i' .. i' + N_max share
// their first l octal digits for the cell's first point i'.  So the internal (split)
// cells can be listed without iterating: point i is the first point of its level-l cell
// when it differs from point i - 1 within the first l digits, and that cell is internal
// when l <= 20 and point i + N_max still shares those l digits.  Emitting, for every i,
// those levels in ascending order lists the internal cells in depth-first pre-order
// (ascending first code, parent before child).  Every internal cell has its 8 children
// (complete octree); a child that is not internal is a leaf.  A leaf's index in the
// leaves array (its rank along the curve) follows from its first code K:
//   rank = (sum of the octal digits of K) + 7 * (#internal cells starting below K
//          - #levels above the leaf whose cell does not start at K),
// because [0, K) splits into (digit sum) maximal aligned cells, each of which is a leaf
// or a complete subtree of i internal cells and 7 i + 1 leaves.
// This reproduces exactly the leaves of the top-down splitting of section 5.1.
#include <cuda_runtime.h>

#include <new>

#include "sfc_internal.cuh"

namespace sfc {

// ---------------------------------------------------------------------------------
// section 4, steps 1-2: bounding box, one scale for all axes
__global__ void k_bbox_init(BuildScalars* sc) {
    for (int a = 0; a < 3; ++a) {
        sc->mn[a] = 0xffffffffu;
        sc->mx[a] = 0u;
        sc->lo[a] = 0.f;
    }
    sc->bad = 0u;
    sc->scale = 2097152.0f;
    sc->ext = 1.0f;
}

// Four points at a time: three float4 loads hold x, y, z of four consecutive points (the
// caller's array must be 16-byte aligned for these); point j of the four is p[3j .. 3j+2].
__device__ __forceinline__ void load_four_points(const float* __restrict__ xyz, int64_t q, float p[12]) {
    const float4* v = reinterpret_cast<const float4*>(xyz) + 3 * q;
    const float4 a = __ldg(v), b = __ldg(v + 1), c = __ldg(v + 2);
    p[0] = a.x; p[1] = a.y; p[2] = a.z; p[3] = a.w;
    p[4] = b.x; p[5] = b.y; p[6] = b.z; p[7] = b.w;
    p[8] = c.x; p[9] = c.y; p[10] = c.z; p[11] = c.w;
}

__device__ __forceinline__ void bbox_take(float v, int a, unsigned int mn[3], unsigned int mx[3], unsigned int& bad) {
    if (!isfinite(v)) bad = 1u;
    const unsigned int o = float_to_ordered(v);
    mn[a] = min(mn[a], o);
    mx[a] = max(mx[a], o);
}

// vec: xyz is 16-byte aligned (whole groups of four points by vector loads, the rest singly)
__global__ void __launch_bounds__(256) k_bbox(const float* __restrict__ xyz, int64_t n, BuildScalars* sc, int vec) {
    __shared__ unsigned int part[8][7];
    unsigned int mn[3] = {0xffffffffu, 0xffffffffu, 0xffffffffu};
    unsigned int mx[3] = {0u, 0u, 0u};
    unsigned int bad = 0u;
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    int64_t done = 0;
    if (vec) {
        const int64_t nq = n / 4;
        for (int64_t q = tid; q < nq; q += stride) {
            float p[12];
            load_four_points(xyz, q, p);
#pragma unroll
            for (int j = 0; j < 12; ++j) bbox_take(p[j], j % 3, mn, mx, bad);
        }
        done = 4 * nq;
    }
    for (int64_t i = done + tid; i < n; i += stride) {
#pragma unroll
        for (int a = 0; a < 3; ++a) bbox_take(xyz[3 * i + a], a, mn, mx, bad);
    }
    // warp, then block, then one atomic per quantity and block
    const unsigned int lane = lane_id(), warp = threadIdx.x >> 5;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        mn[a] = __reduce_min_sync(0xffffffffu, mn[a]);
        mx[a] = __reduce_max_sync(0xffffffffu, mx[a]);
    }
    bad = __reduce_or_sync(0xffffffffu, bad);
    if (lane == 0) {
        for (int a = 0; a < 3; ++a) {
            part[warp][a] = mn[a];
            part[warp][3 + a] = mx[a];
        }
        part[warp][6] = bad;
    }
    __syncthreads();
    if (threadIdx.x < 7) {
        const int w_n = static_cast<int>(blockDim.x >> 5);
        unsigned int v = part[0][threadIdx.x];
        for (int w = 1; w < w_n; ++w) {
            const unsigned int u = part[w][threadIdx.x];
            v = threadIdx.x < 3 ? min(v, u) : (threadIdx.x < 6 ? max(v, u) : (v | u));
        }
        if (threadIdx.x < 3) atomicMin(&sc->mn[threadIdx.x], v);
        else if (threadIdx.x < 6) atomicMax(&sc->mx[threadIdx.x - 3], v);
        else if (v) atomicOr(&sc->bad, 1u);
    }
}

__global__ void k_bbox_finish(BuildScalars* sc) {
    float ext = 0.f;
    for (int a = 0; a < 3; ++a) {
        const float lo = ordered_to_float(sc->mn[a]);
        const float hi = ordered_to_float(sc->mx[a]);
        sc->lo[a] = lo;
        const float d = __fsub_rn(hi, lo);
        if (d > ext) ext = d;
    }
    if (!isfinite(ext)) sc->bad |= 2u;
    if (ext == 0.f) ext = 1.f;
    sc->ext = ext;
    sc->scale = __fdiv_rn(2097152.0f, ext);  // correctly rounded binary32 division
}

// ---------------------------------------------------------------------------------
template <int ENC>
__device__ __forceinline__ uint64_t code_of(float x, float y, float z, float lx, float ly, float lz, float s,
                                            const HilbertTables& table) {
    const uint32_t cx = cell_of(x, lx, s), cy = cell_of(y, ly, s), cz = cell_of(z, lz, s);
    return ENC == SFC_ENC_HILBERT ? hilbert_code(cx, cy, cz, table) : morton_code(cx, cy, cz);
}

// vec: xyz, keys and idx are 16-byte aligned (groups of four points by vector loads and
// stores, the rest singly)
template <int ENC>
__global__ void __launch_bounds__(256) k_encode(const float* __restrict__ xyz, int64_t n,
                                                const BuildScalars* __restrict__ sc, uint64_t* __restrict__ keys,
                                                uint32_t* __restrict__ idx, int vec) {
    __shared__ HilbertTables table;
    if (ENC == SFC_ENC_HILBERT) fill_hilbert_tables(table);
    const float lx = sc->lo[0], ly = sc->lo[1], lz = sc->lo[2], s = sc->scale;
    const int64_t tid = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    int64_t done = 0;
    if (vec) {
        const int64_t nq = n / 4;
        for (int64_t q = tid; q < nq; q += stride) {
            float p[12];
            load_four_points(xyz, q, p);
            uint64_t k[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) k[j] = code_of<ENC>(p[3 * j], p[3 * j + 1], p[3 * j + 2], lx, ly, lz, s, table);
            ulonglong2* kv = reinterpret_cast<ulonglong2*>(keys) + 2 * q;
            kv[0] = make_ulonglong2(k[0], k[1]);
            kv[1] = make_ulonglong2(k[2], k[3]);
            const uint32_t i0 = static_cast<uint32_t>(4 * q);
            reinterpret_cast<uint4*>(idx)[q] = make_uint4(i0, i0 + 1, i0 + 2, i0 + 3);
        }
        done = 4 * nq;
    }
    for (int64_t i = done + tid; i < n; i += stride) {
        keys[i] = code_of<ENC>(xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2], lx, ly, lz, s, table);
        idx[i] = static_cast<uint32_t>(i);
    }
}

template <int ENC>
__global__ void __launch_bounds__(256) k_encode_cells(const uint32_t* __restrict__ cells, int64_t n,
                                                      uint64_t* __restrict__ keys) {
    __shared__ HilbertTables table;
    if (ENC == SFC_ENC_HILBERT) fill_hilbert_tables(table);
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t cx = cells[3 * i] & kCellMax, cy = cells[3 * i + 1] & kCellMax, cz = cells[3 * i + 2] & kCellMax;
        keys[i] = ENC == SFC_ENC_HILBERT ? hilbert_code(cx, cy, cz, table) : morton_code(cx, cy, cz);
    }
}

// codes of a batch: each point takes the box and scale of its cloud
template <int ENC>
__global__ void __launch_bounds__(256) k_batch_encode(const float* __restrict__ xyz, int64_t n,
                                                      const BatchSeg* __restrict__ segs, int nsegs,
                                                      uint64_t* __restrict__ keys, uint32_t* __restrict__ idx) {
    __shared__ HilbertTables table;
    __shared__ int64_t p0s[kBatchMax];
    if (ENC == SFC_ENC_HILBERT) fill_hilbert_tables(table);
    for (int i = threadIdx.x; i < nsegs; i += blockDim.x) p0s[i] = segs[i].p0;
    __syncthreads();
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        int lo = 0, hi = nsegs - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (p0s[mid] <= i) lo = mid;
            else hi = mid - 1;
        }
        const BatchSeg& g = segs[lo];
        const uint32_t cx = cell_of(xyz[3 * i], g.lo[0], g.scale);
        const uint32_t cy = cell_of(xyz[3 * i + 1], g.lo[1], g.scale);
        const uint32_t cz = cell_of(xyz[3 * i + 2], g.lo[2], g.scale);
        keys[i] = ENC == SFC_ENC_HILBERT ? hilbert_code(cx, cy, cz, table) : morton_code(cx, cy, cz);
        idx[i] = static_cast<uint32_t>(i);
    }
}

sfc_status batch_encode(const float* xyz, int64_t n, int enc, const BatchSeg* segs, int nsegs, uint64_t* keys,
                        uint32_t* idx, cudaStream_t s) {
    const unsigned int grid = grid_for(n, 256, 152 * 16);
    if (enc == SFC_ENC_HILBERT)
        SFC_LAUNCH("batch_encode", s, k_batch_encode<SFC_ENC_HILBERT>, grid, 256, 0, xyz, n, segs, nsegs, keys, idx);
    else
        SFC_LAUNCH("batch_encode", s, k_batch_encode<SFC_ENC_MORTON>, grid, 256, 0, xyz, n, segs, nsegs, keys, idx);
    return SFC_OK;
}

// ---------------------------------------------------------------------------------
// reorder (section 4): the sorted cloud as float4 (x, y, z, original index bits)
__global__ void __launch_bounds__(256) k_gather_points(const float* __restrict__ xyz, int64_t n,
                                                       const uint32_t* __restrict__ perm, float4* __restrict__ pts) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t j = perm[i];
        pts[i] = make_float4(xyz[3 * (int64_t)j], xyz[3 * (int64_t)j + 1], xyz[3 * (int64_t)j + 2], __uint_as_float(j));
    }
}

// the unordered cloud (SFC_ENC_NONE) and caller centres: input order, w = input index;
// bit 0 of *bad is set for a non-finite coordinate
__global__ void __launch_bounds__(256) k_pack_points(const float* __restrict__ xyz, int64_t n,
                                                     float4* __restrict__ pts, unsigned int* bad) {
    unsigned int b = 0u;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const float x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
        if (!(isfinite(x) && isfinite(y) && isfinite(z))) b = 1u;
        pts[i] = make_float4(x, y, z, __uint_as_float(static_cast<uint32_t>(i)));
    }
    if (bad) {
        b = __reduce_or_sync(0xffffffffu, b);
        if (lane_id() == 0 && b) atomicOr(bad, 1u);
    }
}

// ---------------------------------------------------------------------------------
// section 5.1: linear octree
// first: the exclusive scan of the new internal cells of every position (n + 1 entries)
__global__ void __launch_bounds__(256) k_tree_emit(const uint64_t* __restrict__ keys, int64_t n,
                                                   const int64_t* __restrict__ first, uint64_t* __restrict__ ikey,
                                                   uint8_t* __restrict__ ilevel) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        const uint32_t c = static_cast<uint32_t>(first[i + 1] - first[i]);
        if (c == 0) continue;
        const int first_new = i == 0 ? 0 : common_levels(keys[i - 1], keys[i]) + 1;
        const uint64_t k = keys[i];
        const int64_t g0 = first[i];
        for (uint32_t t = 0; t < c; ++t) {
            const int l = first_new + static_cast<int>(t);
            ikey[g0 + t] = k & ~below_level_mask(l);
            ilevel[g0 + t] = static_cast<uint8_t>(l);
        }
    }
}

// children of internal node g are nodes 1 + 8g .. 8 + 8g; the root is node 0
__global__ void __launch_bounds__(256) k_tree_link(const uint64_t* __restrict__ ikey, const uint8_t* __restrict__ ilevel,
                                                   int64_t n_int, int32_t* __restrict__ child,
                                                   int32_t* __restrict__ islot) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t g = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; g < n_int; g += stride) {
        if (g == 0) {
            islot[0] = 0;
            child[0] = 1;
            continue;
        }
        const uint64_t k = ikey[g];
        const int l = ilevel[g];
        const uint64_t pk = k & ~below_level_mask(l - 1);
        const int pl = l - 1;
        int64_t lo = 0, hi = g;  // the parent precedes g in pre-order
        while (lo < hi) {
            const int64_t mid = (lo + hi) >> 1;
            const uint64_t mk = ikey[mid];
            if (mk < pk || (mk == pk && ilevel[mid] < pl)) lo = mid + 1;
            else hi = mid;
        }
        const int digit = static_cast<int>((k >> (3 * (kLevels - l))) & 7ull);
        const int64_t slot = 1 + 8 * lo + digit;
        child[slot] = static_cast<int32_t>(1 + 8 * g);
        islot[g] = static_cast<int32_t>(slot);
    }
}

__device__ __forceinline__ int octal_digit_sum(uint64_t k) {
    const uint64_t m0 = 0x1249249249249249ull;  // bit 0 of every octal digit
    return __popcll(k & m0) + 2 * __popcll(k & (m0 << 1)) + 4 * __popcll(k & (m0 << 2));
}

__global__ void __launch_bounds__(256) k_tree_nodes(const uint64_t* __restrict__ keys, int64_t n,
                                                    const uint64_t* __restrict__ ikey,
                                                    const uint8_t* __restrict__ ilevel, int64_t n_int,
                                                    const int32_t* __restrict__ child, NodeBox* __restrict__ nodes,
                                                    uint64_t* __restrict__ node_key, uint8_t* __restrict__ node_level,
                                                    uint64_t* __restrict__ leaves, uint32_t* __restrict__ leaf_counts) {
    const int64_t m = 1 + 8 * n_int;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; s < m; s += stride) {
        uint64_t k = 0;
        int l = 0;
        if (s > 0) {
            const int64_t g = (s - 1) >> 3;
            const int c = static_cast<int>((s - 1) & 7);
            l = ilevel[g] + 1;
            k = ikey[g] + (static_cast<uint64_t>(c) << (3 * (kLevels - l)));
        }
        const int64_t start = lower_bound_u64(keys, n, k);
        const int64_t end = l == 0 ? n : lower_bound_u64(keys, n, k + (1ull << (3 * (kLevels - l))));
        node_key[s] = k;
        node_level[s] = static_cast<uint8_t>(l);
        NodeBox b;
        b.lo = make_float4(INFINITY, INFINITY, INFINITY, __uint_as_float(static_cast<uint32_t>(start)));
        b.hi = make_float4(-INFINITY, -INFINITY, -INFINITY, __uint_as_float(static_cast<uint32_t>(end)));
        nodes[s] = b;
        if (child[s] < 0) {
            const int64_t before = lower_bound_u64(ikey, n_int, k);  // internal cells starting below k
            const int trailing = k == 0 ? kLevels : (__ffsll(static_cast<long long>(k)) - 1) / 3;
            const int64_t rank = octal_digit_sum(k) + 7 * (before - (kLevels - trailing));
            if (rank >= 0 && rank <= 7 * n_int) {  // always true for a consistent tree
                leaves[rank] = k;
                leaf_counts[rank] = static_cast<uint32_t>(end - start);
            }
        }
        if (s == 0) leaves[7 * n_int + 1] = kWholeRange;
    }
}

// Tight boxes: each leaf reduces its points, then walks up; the eighth child to arrive at
// an internal node merges the eight children boxes and continues with the parent.
__global__ void __launch_bounds__(256) k_tree_boxes(const float4* __restrict__ pts, const uint32_t* __restrict__ perm,
                                                    int indirect, NodeBox* nodes, const int32_t* __restrict__ child,
                                                    const int32_t* __restrict__ islot, unsigned int* arrive, int64_t m) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; s < m; s += stride) {
        if (child[s] >= 0) continue;
        NodeBox b = nodes[s];
        const uint32_t start = __float_as_uint(b.lo.w), end = __float_as_uint(b.hi.w);
        for (uint32_t j = start; j < end; ++j) {
            const float4 p = indirect ? pts[perm[j]] : pts[j];
            b.lo.x = fminf(b.lo.x, p.x); b.lo.y = fminf(b.lo.y, p.y); b.lo.z = fminf(b.lo.z, p.z);
            b.hi.x = fmaxf(b.hi.x, p.x); b.hi.y = fmaxf(b.hi.y, p.y); b.hi.z = fmaxf(b.hi.z, p.z);
        }
        nodes[s] = b;
        int64_t cur = s;
        for (int hops = 0; cur != 0 && hops <= kLevels; ++hops) {  // at most 21 levels above a leaf
            const int64_t g = (cur - 1) >> 3;
            __threadfence();
            if (atomicAdd(&arrive[g], 1u) != 7u) break;
            __threadfence();
            const int64_t ps = islot[g];
            NodeBox u = nodes[ps];  // keeps its [start, end) from k_tree_nodes
            u.lo.x = u.lo.y = u.lo.z = INFINITY;
            u.hi.x = u.hi.y = u.hi.z = -INFINITY;
            for (int c = 0; c < 8; ++c) {
                const float4 clo = __ldcg(&nodes[1 + 8 * g + c].lo);
                const float4 chi = __ldcg(&nodes[1 + 8 * g + c].hi);
                u.lo.x = fminf(u.lo.x, clo.x); u.lo.y = fminf(u.lo.y, clo.y); u.lo.z = fminf(u.lo.z, clo.z);
                u.hi.x = fmaxf(u.hi.x, chi.x); u.hi.y = fmaxf(u.hi.y, chi.y); u.hi.z = fmaxf(u.hi.z, chi.z);
            }
            nodes[ps] = u;
            cur = ps;
        }
    }
}

__global__ void __launch_bounds__(256) k_export_nodes(const NodeBox* __restrict__ nodes, const uint8_t* __restrict__ lv,
                                                      int64_t m, int32_t* level, uint32_t* start, uint32_t* end,
                                                      float* box) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t s = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; s < m; s += stride) {
        const NodeBox b = nodes[s];
        if (level) level[s] = lv[s];
        if (start) start[s] = __float_as_uint(b.lo.w);
        if (end) end[s] = __float_as_uint(b.hi.w);
        if (box) {
            box[6 * s + 0] = b.lo.x; box[6 * s + 1] = b.lo.y; box[6 * s + 2] = b.lo.z;
            box[6 * s + 3] = b.hi.x; box[6 * s + 4] = b.hi.y; box[6 * s + 5] = b.hi.z;
        }
    }
}

// ---------------------------------------------------------------------------------
// caller centres in processing order
__global__ void __launch_bounds__(256) k_gather_queries(const float* __restrict__ q, int64_t nq,
                                                        const uint32_t* __restrict__ order, float4* __restrict__ q4) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nq; i += stride) {
        const uint32_t j = order[i];
        q4[i] = make_float4(q[3 * (int64_t)j], q[3 * (int64_t)j + 1], q[3 * (int64_t)j + 2], __uint_as_float(j));
    }
}

template <int ENC>
__global__ void __launch_bounds__(256) k_query_codes(const float* __restrict__ q, int64_t nq,
                                                     const BuildScalars* __restrict__ sc, uint64_t* __restrict__ keys,
                                                     uint32_t* __restrict__ idx, unsigned int* bad) {
    __shared__ HilbertTables table;
    if (ENC == SFC_ENC_HILBERT) fill_hilbert_tables(table);
    const float lx = sc->lo[0], ly = sc->lo[1], lz = sc->lo[2], s = sc->scale;
    unsigned int b = 0u;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < nq; i += stride) {
        const float x = q[3 * i], y = q[3 * i + 1], z = q[3 * i + 2];
        if (!(isfinite(x) && isfinite(y) && isfinite(z))) b = 1u;
        // centres outside the cloud's box clamp to the nearest face cell; the code only
        // orders the work, it never decides a result
        const uint32_t cx = cell_of(x, lx, s), cy = cell_of(y, ly, s), cz = cell_of(z, lz, s);
        keys[i] = ENC == SFC_ENC_HILBERT ? hilbert_code(cx, cy, cz, table) : morton_code(cx, cy, cz);
        idx[i] = static_cast<uint32_t>(i);
    }
    b = __reduce_or_sync(0xffffffffu, b);
    if (lane_id() == 0 && b) atomicOr(bad, 1u);
}

sfc_status prepare_queries(const Octree* h, const float* queries, int64_t nq, cudaStream_t s, Scratch& scratch,
                           const float4** q4, unsigned int* bad) {
    if (!queries) {
        *q4 = h->pts;
        return SFC_OK;
    }
    float4* out = nullptr;
    SFC_TRY(scratch.alloc(&out, static_cast<size_t>(nq)));
    *q4 = out;
    if (nq == 0) return SFC_OK;
    const unsigned int grid = grid_for(nq, 256, 152 * 16);
    if (h->enc == SFC_ENC_NONE) {
        SFC_LAUNCH("pack_queries", s, k_pack_points, grid, 256, 0, queries, nq, out, bad);
        return SFC_OK;
    }
    uint64_t *k0, *k1;
    uint32_t *v0, *v1;
    SFC_TRY(scratch.alloc(&k0, nq));
    SFC_TRY(scratch.alloc(&k1, nq));
    SFC_TRY(scratch.alloc(&v0, nq));
    SFC_TRY(scratch.alloc(&v1, nq));
    if (h->enc == SFC_ENC_HILBERT)
        SFC_LAUNCH("query_codes", s, k_query_codes<SFC_ENC_HILBERT>, grid, 256, 0, queries, nq, h->scal, k0, v0, bad);
    else
        SFC_LAUNCH("query_codes", s, k_query_codes<SFC_ENC_MORTON>, grid, 256, 0, queries, nq, h->scal, k0, v0, bad);
    SFC_TRY(radix_sort_pairs(k0, v0, k1, v1, nq, s, scratch, &h->scal->bad));
    SFC_LAUNCH("gather_queries", s, k_gather_queries, grid, 256, 0, queries, nq, v0, out);
    return SFC_OK;
}

// ---------------------------------------------------------------------------------
static void free_octree(Octree* t, cudaStream_t s) {
    dev_free(t->pts, s);
    dev_free(t->perm, s);
    dev_free(t->keys, s);
    dev_free(t->nodes, s);
    dev_free(t->child, s);
    dev_free(t->node_key, s);
    dev_free(t->node_level, s);
    dev_free(t->leaves, s);
    dev_free(t->leaf_counts, s);
    dev_free(t->scal, s);
    release_records(t, s);
}

static sfc_status build_octree(Octree* t, const float* xyz, cudaStream_t s) {
    Scratch scratch(s);
    const int64_t n = t->n;
    const unsigned int grid = grid_for(n, 256, 152 * 16);
    SFC_TRY(dev_alloc(&t->scal, 1, s));
    SFC_TRY(dev_alloc(&t->keys, n, s));
    SFC_TRY(dev_alloc(&t->perm, n, s));
    SFC_TRY(dev_alloc(&t->pts, n, s));
    SFC_LAUNCH("bbox_init", s, k_bbox_init, 1, 1, 0, t->scal);
    int64_t n_int = 0;
    if (n > 0) {
        // section 4: box, scale and codes
        const int vec = (aligned16(xyz) && aligned16(t->keys) && aligned16(t->perm)) ? 1 : 0;
        SFC_LAUNCH("bbox", s, k_bbox, grid, 256, 0, xyz, n, t->scal, vec);
        SFC_LAUNCH("bbox_finish", s, k_bbox_finish, 1, 1, 0, t->scal);
        uint64_t* keys_alt;
        uint32_t* perm_alt;
        SFC_TRY(scratch.alloc(&keys_alt, n));
        SFC_TRY(scratch.alloc(&perm_alt, n));
        if (t->enc == SFC_ENC_HILBERT)
            SFC_LAUNCH("encode", s, k_encode<SFC_ENC_HILBERT>, grid, 256, 0, xyz, n, t->scal, t->keys, t->perm, vec);
        else
            SFC_LAUNCH("encode", s, k_encode<SFC_ENC_MORTON>, grid, 256, 0, xyz, n, t->scal, t->keys, t->perm, vec);
        // section 4: ascending codes, ties in input order
        SFC_TRY(radix_sort_pairs(t->keys, t->perm, keys_alt, perm_alt, n, s, scratch, &t->scal->bad));
        if (t->enc == SFC_ENC_NONE)
            SFC_LAUNCH("pack_points", s, k_pack_points, grid, 256, 0, xyz, n, t->pts, (unsigned int*)nullptr);
        else
            SFC_LAUNCH("gather_points", s, k_gather_points, grid, 256, 0, xyz, n, t->perm, t->pts);
        // section 5.1: the internal cells first seen at each sorted point, counted and scanned
        // in one pass over the codes
        int64_t* first;
        SFC_TRY(scratch.alloc(&first, n + 1));
        SFC_TRY(scan_tree_counts(t->keys, n, static_cast<int64_t>(t->leaf_cap), first, s, scratch, &t->scal->bad));
        BuildScalars hs;
        SFC_CUDA(cudaMemcpyAsync(&n_int, first + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
        SFC_CUDA(cudaMemcpyAsync(&hs, t->scal, sizeof(BuildScalars), cudaMemcpyDeviceToHost, s));
        SFC_CUDA(cudaStreamSynchronize(s));
        if (hs.bad & kWaitTimedOut) return SFC_ERR_TIMEOUT;
        if (hs.bad) return SFC_ERR_NOT_FINITE;
        for (int a = 0; a < 3; ++a) t->lo[a] = hs.lo[a];
        t->scale = hs.scale;
        if (1 + 8 * n_int > 0x7fffffffLL) return SFC_ERR_TOO_LARGE;
        t->n_internal = n_int;
        t->n_nodes = 1 + 8 * n_int;
        t->n_leaves = 7 * n_int + 1;
        SFC_TRY(dev_alloc(&t->nodes, t->n_nodes, s));
        SFC_TRY(dev_alloc(&t->child, t->n_nodes, s));
        SFC_TRY(dev_alloc(&t->node_key, t->n_nodes, s));
        SFC_TRY(dev_alloc(&t->node_level, t->n_nodes, s));
        SFC_TRY(dev_alloc(&t->leaves, t->n_leaves + 1, s));
        SFC_TRY(dev_alloc(&t->leaf_counts, t->n_leaves, s));
        SFC_CUDA(cudaMemsetAsync(t->child, 0xff, sizeof(int32_t) * t->n_nodes, s));
        uint64_t* ikey = nullptr;
        uint8_t* ilevel = nullptr;
        int32_t* islot = nullptr;
        unsigned int* arrive = nullptr;
        SFC_TRY(scratch.alloc(&ikey, n_int));
        SFC_TRY(scratch.alloc(&ilevel, n_int));
        SFC_TRY(scratch.alloc(&islot, n_int));
        SFC_TRY(scratch.alloc(&arrive, n_int));
        if (n_int > 0) {
            SFC_CUDA(cudaMemsetAsync(arrive, 0, sizeof(unsigned int) * n_int, s));
            SFC_LAUNCH("tree_emit", s, k_tree_emit, grid, 256, 0, t->keys, n, first, ikey, ilevel);
            SFC_LAUNCH("tree_link", s, k_tree_link, grid_for(n_int, 256, 152 * 16), 256, 0, ikey, ilevel, n_int,
                       t->child, islot);
        }
        const unsigned int ngrid = grid_for(t->n_nodes, 256, 152 * 16);
        SFC_LAUNCH("tree_nodes", s, k_tree_nodes, ngrid, 256, 0, t->keys, n, ikey, ilevel, n_int, t->child, t->nodes,
                   t->node_key, t->node_level, t->leaves, t->leaf_counts);
        SFC_LAUNCH("tree_boxes", s, k_tree_boxes, ngrid, 256, 0, t->pts, t->perm, t->enc == SFC_ENC_NONE ? 1 : 0,
                   t->nodes, t->child, islot, arrive, t->n_nodes);
    } else {
        // the empty cloud: a single empty root leaf, leaves = {0, 8^21}
        t->n_internal = 0;
        t->n_nodes = 1;
        t->n_leaves = 1;
        SFC_TRY(dev_alloc(&t->nodes, 1, s));
        SFC_TRY(dev_alloc(&t->child, 1, s));
        SFC_TRY(dev_alloc(&t->node_key, 1, s));
        SFC_TRY(dev_alloc(&t->node_level, 1, s));
        SFC_TRY(dev_alloc(&t->leaves, 2, s));
        SFC_TRY(dev_alloc(&t->leaf_counts, 1, s));
        SFC_CUDA(cudaMemsetAsync(t->child, 0xff, sizeof(int32_t), s));
        SFC_LAUNCH("tree_nodes", s, k_tree_nodes, 1, 256, 0, t->keys, static_cast<int64_t>(0), (const uint64_t*)nullptr,
                   (const uint8_t*)nullptr, static_cast<int64_t>(0), t->child, t->nodes, t->node_key, t->node_level,
                   t->leaves, t->leaf_counts);
        t->lo[0] = t->lo[1] = t->lo[2] = 0.f;
        t->scale = 2097152.0f;
    }
    return SFC_OK;
}

}  // namespace sfc

using sfc::Octree;

extern "C" {

sfc_status sfc_build_opts_default(sfc_build_opts* opts) {
    if (!opts) return SFC_ERR_INVALID;
    opts->leaf_capacity = 32;
    opts->prune = 1;
    return SFC_OK;
}

sfc_status octree_build(const float* points_xyz, int64_t n, sfc_encoding enc, const sfc_build_opts* opts,
                        void* cuda_stream, sfc_octree* out) {
    if (!out) return SFC_ERR_INVALID;
    *out = nullptr;
    if (n < 0) return SFC_ERR_INVALID;
    if (n > 0x7fffffffLL - 1) return SFC_ERR_TOO_LARGE;
    if (enc != SFC_ENC_NONE && enc != SFC_ENC_MORTON && enc != SFC_ENC_HILBERT) return SFC_ERR_INVALID;
    sfc_build_opts o;
    sfc_build_opts_default(&o);
    if (opts) o = *opts;
    if (o.leaf_capacity < 1 || (o.prune != 0 && o.prune != 1)) return SFC_ERR_INVALID;
    if (n > 0 && !points_xyz) return SFC_ERR_INVALID;
    if (n > 0 && !sfc::is_device_ptr(points_xyz)) return SFC_ERR_NOT_DEVICE_PTR;
    int dev = 0;
    SFC_CUDA(cudaGetDevice(&dev));
    SFC_TRY(sfc::ensure_pool(dev));
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    sfc_octree_s* h = new (std::nothrow) sfc_octree_s;
    if (!h) return SFC_ERR_OOM;
    Octree* t = &h->tree;
    t->device = dev;
    t->n = n;
    t->enc = enc;
    t->leaf_cap = o.leaf_capacity;
    t->prune = o.prune;
    sfc_status st = sfc::build_octree(t, points_xyz, s);
    if (st != SFC_OK) {
        sfc::free_octree(t, s);
        delete h;
        return st;
    }
    *out = h;
    return SFC_OK;
}

sfc_status octree_free(sfc_octree h, void* cuda_stream) {
    if (!h) return SFC_ERR_INVALID;
    sfc::free_octree(&h->tree, static_cast<cudaStream_t>(cuda_stream));
    delete h;
    return SFC_OK;
}

sfc_status octree_info(sfc_octree h, sfc_octree_info* info) {
    if (!h || !info) return SFC_ERR_INVALID;
    const Octree* t = &h->tree;
    info->n_points = t->n;
    info->n_leaves = t->n_leaves;
    info->n_internal = t->n_internal;
    info->n_nodes = t->n_nodes;
    info->encoding = t->enc;
    info->leaf_capacity = t->leaf_cap;
    info->prune = t->prune;
    info->device = t->device;
    for (int a = 0; a < 3; ++a) info->lo[a] = t->lo[a];
    info->scale = t->scale;
    return SFC_OK;
}

sfc_status octree_export(sfc_octree h, void* cuda_stream, uint64_t* sorted_keys, uint32_t* perm, uint64_t* leaves,
                         uint32_t* leaf_counts) {
    if (!h) return SFC_ERR_INVALID;
    const Octree* t = &h->tree;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const void* outs[4] = {sorted_keys, perm, leaves, leaf_counts};
    for (const void* p : outs)
        if (p && !sfc::is_device_ptr(p)) return SFC_ERR_NOT_DEVICE_PTR;
    if (sorted_keys && t->n)
        SFC_CUDA(cudaMemcpyAsync(sorted_keys, t->keys, sizeof(uint64_t) * t->n, cudaMemcpyDeviceToDevice, s));
    if (perm && t->n) SFC_CUDA(cudaMemcpyAsync(perm, t->perm, sizeof(uint32_t) * t->n, cudaMemcpyDeviceToDevice, s));
    if (leaves)
        SFC_CUDA(cudaMemcpyAsync(leaves, t->leaves, sizeof(uint64_t) * (t->n_leaves + 1), cudaMemcpyDeviceToDevice, s));
    if (leaf_counts)
        SFC_CUDA(cudaMemcpyAsync(leaf_counts, t->leaf_counts, sizeof(uint32_t) * t->n_leaves, cudaMemcpyDeviceToDevice,
                                 s));
    return SFC_OK;
}

sfc_status octree_export_nodes(sfc_octree h, void* cuda_stream, uint64_t* node_key, int32_t* node_level,
                               uint32_t* node_start, uint32_t* node_end, int32_t* node_child, float* node_box) {
    if (!h) return SFC_ERR_INVALID;
    const Octree* t = &h->tree;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const void* outs[6] = {node_key, node_level, node_start, node_end, node_child, node_box};
    for (const void* p : outs)
        if (p && !sfc::is_device_ptr(p)) return SFC_ERR_NOT_DEVICE_PTR;
    const int64_t m = t->n_nodes;
    if (node_key) SFC_CUDA(cudaMemcpyAsync(node_key, t->node_key, sizeof(uint64_t) * m, cudaMemcpyDeviceToDevice, s));
    if (node_child) SFC_CUDA(cudaMemcpyAsync(node_child, t->child, sizeof(int32_t) * m, cudaMemcpyDeviceToDevice, s));
    if (node_level || node_start || node_end || node_box)
        SFC_LAUNCH("export_nodes", s, sfc::k_export_nodes, sfc::grid_for(m, 256, 152 * 16), 256, 0, t->nodes,
                   t->node_level, m, node_level, node_start, node_end, node_box);
    return SFC_OK;
}

sfc_status sfc_encode_cells(const uint32_t* cells, int64_t n, sfc_encoding enc, void* cuda_stream, uint64_t* keys) {
    if (n < 0 || (n > 0 && (!cells || !keys))) return SFC_ERR_INVALID;
    if (enc != SFC_ENC_NONE && enc != SFC_ENC_MORTON && enc != SFC_ENC_HILBERT) return SFC_ERR_INVALID;
    if (n == 0) return SFC_OK;
    if (!sfc::is_device_ptr(cells) || !sfc::is_device_ptr(keys)) return SFC_ERR_NOT_DEVICE_PTR;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    const unsigned int grid = sfc::grid_for(n, 256, 152 * 16);
    if (enc == SFC_ENC_HILBERT)
        SFC_LAUNCH("encode_cells", s, sfc::k_encode_cells<SFC_ENC_HILBERT>, grid, 256, 0, cells, n, keys);
    else
        SFC_LAUNCH("encode_cells", s, sfc::k_encode_cells<SFC_ENC_MORTON>, grid, 256, 0, cells, n, keys);
    return SFC_OK;
}

}  // extern "C"
