// sfc_knn.cu - k nearest neighbours over the linear octree (section 3.3).
//
// The paper pops octants and points from one priority queue ordered by distance.  Here
// each centre keeps its k best (squared distance, original index) pairs (a max-heap in
// shared memory for the warp-group walk, a sorted register list for the walk of one
// centre), and the octree is walked depth first with the children of a node visited
// nearest first; a node is entered only while its box could still hold a better pair.
// The result is the same exact set, in the same (d2, index) order:
//   - an octant's lower bound is the squared distance to its box point nearest to the
//     centre (the clamp of section 3.3), computed with the same rounded operations as a
//     point distance; rounding is monotone, so no point of the box is nearer;
//   - a node is skipped only when that bound exceeds the current k-th distance, so a
//     point tying the k-th distance (which may win on a smaller index) is still seen.
// For a cloud ordered along the curve a warp serves 32 consecutive centres with one
// shared walk (a node is entered when any lane needs it); for the unordered cloud each
// lane walks alone.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include <algorithm>

#include "sfc_internal.cuh"

namespace sfc {

constexpr int kKnnWarps = 1;  // one warp per block: per-warp work varies widely
constexpr uint32_t kNoIndex = 0xffffffffu;

struct KnnArgs {
    const float4* __restrict__ pts;
    const uint32_t* __restrict__ perm;
    const NodeBox* __restrict__ nodes;
    const int32_t* __restrict__ child;
    const float4* __restrict__ q;
    int64_t nq;
    int k;
    int32_t* out_idx;
    float* out_d2;
    unsigned int* err;
    int64_t max_steps;
    int64_t window;   // > 0: seed each warp's lists from this many curve neighbours on each side
    // batched search: nsegs clouds, ngroups warp groups in all (segs == nullptr: one cloud)
    const SearchSeg* segs;
    int nsegs;
    int64_t ngroups;
    // batched search: the launch does nothing when (*skip & skip_mask) != 0 (a capacity
    // overflow found on the device earlier in the same stream)
    const unsigned int* skip;
    unsigned int skip_mask;
    unsigned long long* stats;  // work counters (the STATS copies of the kernels)
};

__device__ __forceinline__ float box_lower_bound(const NodeBox& b, float cx, float cy, float cz) {
    return sq_dist(__fsub_rn(fminf(fmaxf(cx, b.lo.x), b.hi.x), cx), __fsub_rn(fminf(fmaxf(cy, b.lo.y), b.hi.y), cy),
                   __fsub_rn(fminf(fmaxf(cz, b.lo.z), b.hi.z), cz));
}

__device__ __forceinline__ bool pair_less(float da, uint32_t ia, float db, uint32_t ib) {
    return da < db || (da == db && ia < ib);
}

// A (d2, index) pair packed so that unsigned order is pair order: d2 is never negative
// (a sum of rounded squares), and the bits of a non-negative float order like its value.
__device__ __forceinline__ uint64_t pair_key(float d, uint32_t id) {
    return (static_cast<uint64_t>(__float_as_uint(d)) << 32) | id;
}
constexpr uint64_t kNoPair = (static_cast<uint64_t>(0x7f800000u) << 32) | kNoIndex;  // (+inf, no index)

// The KMAX best pairs of one centre, sorted ascending in registers; the k-th (k <= KMAX)
// is the pruning bound.  insert() decides every slot independently from the comparisons
// "slot s stays before the new pair" (true for a prefix of the sorted list): slot s keeps
// its pair, takes the new one, or takes slot s-1's, and the last pair drops off.
template <int KMAX>
struct BestList {
    uint64_t key[KMAX];
    uint64_t kth;  // the k-th pair
    int k;
    __device__ __forceinline__ void init(int kk) {
#pragma unroll
        for (int s = 0; s < KMAX; ++s) key[s] = kNoPair;
        kth = kNoPair;
        k = kk;
    }
    __device__ __forceinline__ void insert(uint64_t nk) {
        bool stays[KMAX];
#pragma unroll
        for (int s = 0; s < KMAX; ++s) stays[s] = key[s] < nk;
#pragma unroll
        for (int s = KMAX - 1; s > 0; --s) key[s] = stays[s] ? key[s] : (stays[s - 1] ? nk : key[s - 1]);
        key[0] = stays[0] ? key[0] : nk;
        if (k == KMAX) {
            kth = key[KMAX - 1];
        } else {
            kth = key[0];
#pragma unroll
            for (int s = 1; s < KMAX; ++s)
                if (s == k - 1) kth = key[s];
        }
    }
    __device__ __forceinline__ float kth_d2() const { return __uint_as_float(static_cast<uint32_t>(kth >> 32)); }
    __device__ __forceinline__ void store(const KnnArgs& a, uint32_t row) const {
        const int64_t base = static_cast<int64_t>(row) * a.k;
#pragma unroll
        for (int s = 0; s < KMAX; ++s)
            if (s < a.k) {
                const uint32_t id = static_cast<uint32_t>(key[s]);
                a.out_idx[base + s] = id == kNoIndex ? -1 : static_cast<int32_t>(id);
                a.out_d2[base + s] = __uint_as_float(static_cast<uint32_t>(key[s] >> 32));
            }
    }
};

// The k best pairs of one lane as a D-ary max-heap in shared memory (root = the k-th
// pair, the pruning bound; the children of slot i are slots D i + 1 .. D i + D),
// lane-interleaved: slot s of lane l is word s * 32 + l, so the 32 lanes of a warp always
// touch 32 different banks whatever slots they visit.  Replacing the root and sifting it
// down costs O(log_D k) levels; finish() heap-sorts the slots ascending.  D = 4 halves the
// levels of a long list (the four children of a level load together): kNN k = 50 on the
// 10M tile 42.2 -> 36.9 ms; for k <= 16 the binary heap is as fast or faster (k = 8: 5.5
// vs 5.9 ms).
// KFIX > 0: the list size is that compile-time constant (every loop over the slots and
// every sift unrolls); 0: the size is k, known at run time.
template <int D, int KFIX = 0>
struct LaneHeap {
    static_assert(D == 2 || D == 4, "binary or 4-ary");
    static_assert(KFIX <= kMaxK, "at most kMaxK pairs");
    // levels a sift can move down in a list of at most kMaxK = 64 pairs, plus the last test
    static constexpr int kSiftSteps = D == 2 ? 7 : 4;
    uint64_t* slot0;  // &heap[0][lane]
    uint64_t kth;     // register copy of the root
    int k_;
    __device__ __forceinline__ int size() const { return KFIX > 0 ? KFIX : k_; }
    __device__ __forceinline__ uint64_t& at(int s) const { return slot0[s * 32]; }
    __device__ __forceinline__ void init(uint64_t* base, int kk) {
        slot0 = base;
        k_ = kk;
        if constexpr (KFIX > 0) {
#pragma unroll
            for (int s = 0; s < KFIX; ++s) at(s) = kNoPair;
        } else {
            for (int s = 0; s < k_; ++s) at(s) = kNoPair;
        }
        kth = kNoPair;
    }
    // the largest of the children c0 .. c0 + D - 1 (those below `size`; c0 < size) and its slot
    __device__ __forceinline__ uint64_t max_child(int c0, int size, int* c) const {
        if constexpr (D == 2) {
            uint64_t cv = at(c0);
            *c = c0;
            if (c0 + 1 < size) {
                const uint64_t rv = at(c0 + 1);
                if (rv > cv) {
                    *c = c0 + 1;
                    cv = rv;
                }
            }
            return cv;
        } else {
            // absent children read as the smallest key, which never moves up
            const uint64_t v0 = at(c0);
            const uint64_t v1 = c0 + 1 < size ? at(c0 + 1) : 0ull;
            const uint64_t v2 = c0 + 2 < size ? at(c0 + 2) : 0ull;
            const uint64_t v3 = c0 + 3 < size ? at(c0 + 3) : 0ull;
            const bool a = v1 > v0, b = v3 > v2;
            const uint64_t m01 = a ? v1 : v0, m23 = b ? v3 : v2;
            const bool hi = m23 > m01;
            *c = hi ? (b ? c0 + 3 : c0 + 2) : (a ? c0 + 1 : c0);
            return hi ? m23 : m01;
        }
    }
    // place x at slot pos of the heap of the first `size` slots and restore the order below it
    __device__ __forceinline__ void sift_down(uint64_t x, int size, int pos = 0) {
#pragma unroll
        for (int step = 0; step < kSiftSteps; ++step) {
            const int c0 = D * pos + 1;
            if (c0 >= size) break;
            int c;
            const uint64_t cv = max_child(c0, size, &c);
            if (cv <= x) break;
            at(pos) = cv;
            pos = c;
        }
        at(pos) = x;
    }
    // replace the root (the k-th pair) by nk < kth; the new root, the larger of nk and the
    // root's largest child, is known before the rest of the sift and stays in a register
    __device__ __forceinline__ void insert(uint64_t nk) {
        if (size() > 1) {
            int c;
            const uint64_t cv = max_child(1, size(), &c);
            if (cv > nk) {
                at(0) = cv;
                kth = cv;
                sift_down(nk, size(), c);
                return;
            }
        }
        at(0) = nk;
        kth = nk;
    }
    // the k slots hold arbitrary pairs: restore the heap order bottom-up
    __device__ __forceinline__ void heapify() {
        for (int i = (size() - 2) / D; i >= 0; --i) sift_down(at(i), size(), i);
        kth = at(0);
    }
    __device__ __forceinline__ void finish() {
        for (int end = size() - 1; end > 0; --end) {
            const uint64_t top = at(0);
            const uint64_t last = at(end);
            at(end) = top;
            sift_down(last, end);
        }
    }
    __device__ __forceinline__ float kth_d2() const { return __uint_as_float(static_cast<uint32_t>(kth >> 32)); }
    __device__ __forceinline__ void store(const KnnArgs& a, int64_t base) const {
        for (int s = 0; s < size(); ++s) {
            const uint64_t key = at(s);
            const uint32_t id = static_cast<uint32_t>(key);
            a.out_idx[base + s] = id == kNoIndex ? -1 : static_cast<int32_t>(id);
            a.out_d2[base + s] = __uint_as_float(static_cast<uint32_t>(key >> 32));
        }
    }
};

// Test the points at sorted positions [lo, hi) against every lane's centre and insert the
// better ones: pass 1 marks, per 32-point chunk, the points that beat the lane's current
// k-th pair; pass 2 lets each lane insert its marked points.
// Points at positions in [skip_lo, skip_lo + skip_n) were already offered to this lane.
template <class List>
__device__ __forceinline__ void scan_points(const KnnArgs& a, uint32_t lo, uint32_t hi, const float4& c, bool need,
                                            List& best, int64_t skip_lo = 0, uint32_t skip_n = 0) {
    for (uint32_t base = lo; base < hi; base += 32) {
        const uint32_t m = min(32u, hi - base);
        uint32_t cand = 0;
#pragma unroll 4
        for (uint32_t t = 0; t < m; ++t) {
            const float4 p = __ldg(&a.pts[base + t]);
            const float d = sq_dist(__fsub_rn(p.x, c.x), __fsub_rn(p.y, c.y), __fsub_rn(p.z, c.z));
            const bool seen = static_cast<uint64_t>(static_cast<int64_t>(base + t) - skip_lo) < skip_n;
            if (pair_key(d, __float_as_uint(p.w)) < best.kth && !seen) cand |= 1u << t;
        }
        if (!need) cand = 0;
        while (__ballot_sync(0xffffffffu, cand != 0)) {
            if (cand) {
                const int t = __ffs(cand) - 1;
                cand &= cand - 1;
                const float4 p = __ldg(&a.pts[base + t]);
                const uint64_t nk =
                    pair_key(sq_dist(__fsub_rn(p.x, c.x), __fsub_rn(p.y, c.y), __fsub_rn(p.z, c.z)), __float_as_uint(p.w));
                if (nk < best.kth) best.insert(nk);
            }
        }
    }
}

// children order key: empty or unreachable children last, then by bound, then by number
__device__ __forceinline__ uint64_t child_order_key(const NodeBox& cb, float gx, float gy, float gz, int ci) {
    const bool empty = __float_as_uint(cb.lo.w) == __float_as_uint(cb.hi.w);
    const uint32_t bound = empty ? 0xffffffffu : float_to_ordered(box_lower_bound(cb, gx, gy, gz));
    return (static_cast<uint64_t>(bound) << 32) | static_cast<uint32_t>(ci);
}

// The same order in 32 bits for the group walk: the bound's order-preserving image with
// its three low bits replaced by the child number (bounds within 8 ulps may swap places,
// which changes the visiting order only); 0xffffffff marks an empty child.
__device__ __forceinline__ uint32_t child_order_key32(const NodeBox& cb, float gx, float gy, float gz, int ci) {
    if (__float_as_uint(cb.lo.w) == __float_as_uint(cb.hi.w)) return 0xffffffffu;
    return (float_to_ordered(box_lower_bound(cb, gx, gy, gz)) & ~7u) | static_cast<uint32_t>(ci);
}

// Squared distance bound between a node box and the box of a group of centres; no
// centre of the group is nearer to any point of the node (rounding is monotone).
__device__ __forceinline__ float group_lower_bound(const NodeBox& b, float glx, float gly, float glz, float ghx,
                                                   float ghy, float ghz) {
    return sq_dist(fmaxf(fmaxf(__fsub_rn(b.lo.x, ghx), __fsub_rn(glx, b.hi.x)), 0.0f),
                   fmaxf(fmaxf(__fsub_rn(b.lo.y, ghy), __fsub_rn(gly, b.hi.y)), 0.0f),
                   fmaxf(fmaxf(__fsub_rn(b.lo.z, ghz), __fsub_rn(glz, b.hi.z)), 0.0f));
}

// warps per block of the group kernel
template <int KMAX>
__host__ __device__ constexpr int knn_warps() { return kKnnWarps; }

// Group kNN walk.  Stack entries carry (an internal node's first child or a leaf's node
// index, lanes needing the node), decided when the parent was expanded; a popped leaf reads
// its point range from the node table; an expansion loads the eight children once (lanes
// 0-7) and stages their boxes in shared memory for every lane.  Points (the seeding window, leaf chunks) are
// staged in shared memory with coalesced loads, and both the tests and the insertions read
// them there.  Per chunk, pass 1 marks the points that beat each lane's current k-th pair
// and pass 2 lets each lane insert its marked points.
// STATS: also accumulate the work counters of sfc_search_stats.
// KFIX: every list has exactly KFIX pairs; WFIX: the seeding window is WFIX positions per
// side (compile-time sizes, so the list and window loops unroll; batches pass 0 for both).
template <int KMAX, bool STATS = false, int KFIX = 0, int WFIX = 0>
// the minimum resident blocks match what shared memory allows for each list size: with
// 8-byte stack entries 32 one-warp blocks fit for k <= 16 at 64 registers (k = 16 on the
// 10M-point tile: 9.51 ms at 26 resident blocks, 9.10 ms at 32)
__global__ void __launch_bounds__(knn_warps<KMAX>() * 32, KMAX <= 16 ? 32 : (KMAX <= 32 ? 20 : 11))
    k_knn_group(KnnArgs a) {
    constexpr int kWarps = knn_warps<KMAX>();
    // staged points: the seeding window (32 + 2 window - 1 positions) or one leaf chunk
    constexpr int kBuf = KMAX <= 16 ? 64 : 32 + 2 * KMAX;
    static_assert(kBuf >= 64, "the walk keeps a chunk and the centres in the staging buffer");
    // x: an internal node's first child, or ~node for a leaf (its point range is read when it
    // is popped); y: the lanes needing the node
    __shared__ int2 stack_e[kWarps][kStackDepth];
    __shared__ uint64_t heaps[kWarps][KMAX][32];
    __shared__ float4 pbuf[kWarps][kBuf];
    const unsigned int lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int64_t group = static_cast<int64_t>(blockIdx.x) * kWarps + warp;
    int64_t first = group * 32, q_lo = 0, q_end = a.nq, out0 = 0;
    int32_t root = 0;
    int k = KFIX > 0 ? KFIX : a.k;
    int64_t window = WFIX > 0 ? WFIX : a.window;
    unsigned int gsize = 32;  // centres of this group (batched clouds may ask for fewer)
    if (a.segs) {
        if (group >= a.ngroups) return;
        if (a.skip && (*a.skip & a.skip_mask)) return;
        const SearchSeg sg = a.segs[find_search_seg(a.segs, a.nsegs, group)];
        gsize = static_cast<unsigned int>(sg.group_size);
        first = sg.q0 + (group - sg.group0) * gsize;
        q_lo = sg.q0;
        q_end = sg.q0 + sg.nq;
        out0 = sg.row0;
        root = sg.root;
        if constexpr (KFIX == 0) k = sg.k;  // else every cloud's k is KFIX
        if constexpr (WFIX == 0) window = sg.window;
    } else if (first >= a.nq) {
        return;
    }
    const int64_t qi = first + lane;
    const bool active = lane < gsize && qi < q_end;
    const float4 c = active ? a.q[qi] : make_float4(0.f, 0.f, 0.f, 0.f);
    // first output entry of this lane's row
    const int64_t out_base = out0 + static_cast<int64_t>(__float_as_uint(c.w)) * k;
    float4* buf = pbuf[warp];
    float4* cbuf = buf + 32;  // during the walk: the centres with their current k-th distance

    // centre (orders the walk) and bounding box (prunes it) of the group's centres
    const unsigned int act = __ballot_sync(0xffffffffu, active);
    const float inv = 1.0f / static_cast<float>(__popc(act));
    float gx = active ? c.x : 0.f, gy = active ? c.y : 0.f, gz = active ? c.z : 0.f;
    float glx = active ? c.x : INFINITY, gly = active ? c.y : INFINITY, glz = active ? c.z : INFINITY;
    float ghx = active ? c.x : -INFINITY, ghy = active ? c.y : -INFINITY, ghz = active ? c.z : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        gx += __shfl_xor_sync(0xffffffffu, gx, o);
        gy += __shfl_xor_sync(0xffffffffu, gy, o);
        gz += __shfl_xor_sync(0xffffffffu, gz, o);
        glx = fminf(glx, __shfl_xor_sync(0xffffffffu, glx, o));
        gly = fminf(gly, __shfl_xor_sync(0xffffffffu, gly, o));
        glz = fminf(glz, __shfl_xor_sync(0xffffffffu, glz, o));
        ghx = fmaxf(ghx, __shfl_xor_sync(0xffffffffu, ghx, o));
        ghy = fmaxf(ghy, __shfl_xor_sync(0xffffffffu, ghy, o));
        ghz = fmaxf(ghz, __shfl_xor_sync(0xffffffffu, ghz, o));
    }
    gx *= inv; gy *= inv; gz *= inv;

    StatAcc st;
    if constexpr (STATS) {
        st.zero();
        st.v[kStWalks] = lane == 0;
    }
    LaneHeap<(KMAX >= 32 ? 4 : 2), KFIX> best;
    best.init(&heaps[warp][0][lane], k);
    auto key_of = [&](const float4& q) {
        return pair_key(sq_dist(__fsub_rn(q.x, c.x), __fsub_rn(q.y, c.y), __fsub_rn(q.z, c.z)), __float_as_uint(q.w));
    };

    // All-points search on a cloud ordered along the curve: lane l's centre is the point at
    // position p = first + l, and its curve neighbours are mostly its space neighbours.  Each
    // lane first offers its list the points at p, p+1, p-1, p+2, ... (2 * window positions,
    // nearest along the curve first): the k nearest fill the heap directly, the others are
    // offered in turn.  That gives a near-final k-th distance before the walk, which then
    // skips those positions.
    int64_t win_lo = 0;
    uint32_t win_n = 0;
    if (window > 0 && 32 + 2 * window - 1 <= kBuf) {
        const int64_t r0 = first - (window - 1);  // staged positions r0 .. r0 + span - 1
        const int span = 32 + 2 * static_cast<int>(window) - 1;
        for (int j = lane; j < span; j += 32) {
            const int64_t pos = r0 + j;
            buf[j] = (pos >= q_lo && pos < q_end) ? __ldg(&a.pts[pos]) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        __syncwarp();
        const int64_t p = qi;
        win_lo = p - window + 1;
        win_n = static_cast<uint32_t>(2 * window);
        auto window_key = [&](int t) -> uint64_t {
            const int64_t pos = p + ((t & 1) ? (t + 1) / 2 : -(t / 2));
            if (!active || pos < q_lo || pos >= q_end) return kNoPair;
            return key_of(buf[pos - r0]);
        };
        const int nfill = min(k, static_cast<int>(2 * window));
        for (int t = 0; t < k; ++t) best.at(t) = t < nfill ? window_key(t) : kNoPair;
        best.heapify();
        if constexpr (STATS) {
            st.v[kStPointTests] += 2 * window;
            st.v[kStNeeded] += active ? 2 * window : 0;
        }
        for (int t0 = nfill; t0 < 2 * window; t0 += 32) {
            const int span = min(32, 2 * static_cast<int>(window) - t0);
            uint32_t cand = 0;
            const float kd = best.kth_d2();
#pragma unroll 8
            for (int u = 0; u < span; ++u) {
                const int t = t0 + u;
                const int64_t pos = p + ((t & 1) ? (t + 1) / 2 : -(t / 2));
                if (active && pos >= q_lo && pos < q_end) {
                    const float4 q = buf[pos - r0];
                    if (sq_dist(__fsub_rn(q.x, c.x), __fsub_rn(q.y, c.y), __fsub_rn(q.z, c.z)) <= kd) cand |= 1u << u;
                }
            }
            if constexpr (STATS) st.v[kStPassed] += __popc(cand);
            while (__ballot_sync(0xffffffffu, cand != 0)) {
                if (cand) {
                    const int u = __ffs(cand) - 1;
                    cand &= cand - 1;
                    const uint64_t nk = window_key(t0 + u);
                    if (nk < best.kth) {
                        best.insert(nk);
                        if constexpr (STATS) st.v[kStInserts] += 1;
                    }
                }
            }
        }
        __syncwarp();
    }

    bool guard_ok = true;
    int sp = 0;
    {
        const NodeBox rb = a.nodes[root];
        const int32_t rc = a.child[root];
        const unsigned int need = __ballot_sync(0xffffffffu, active && box_lower_bound(rb, c.x, c.y, c.z) <= best.kth_d2());
        if constexpr (STATS) st.v[kStBoxTests] += 1;
        if (need) {
            if (lane == 0) stack_e[warp][0] = make_int2(rc >= 0 ? rc : ~root, static_cast<int>(need));
            sp = 1;
        }
        __syncwarp();
    }
    for (int64_t steps = 0; sp > 0; ++steps) {
        if (steps >= a.max_steps) {
            guard_ok = false;
            break;
        }
        --sp;
        const int2 e = stack_e[warp][sp];
        __syncwarp();
        const int32_t fc = e.x;
        const bool need = (static_cast<uint32_t>(e.y) >> lane) & 1u;
        if (fc >= 0) {
            // the largest k-th distance of the group bounds what any lane still needs
            float mkd = active ? best.kth_d2() : -INFINITY;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) mkd = fmaxf(mkd, __shfl_xor_sync(0xffffffffu, mkd, o));
            // reachable children, nearest to the group centre first (bitonic sort, lanes 0..7)
            NodeBox cb;
            int32_t cc = -1;
            uint32_t key = 0xffffffffu;
            if (lane < 8) {
                cb = a.nodes[fc + lane];
                cc = a.child[fc + lane];
                if (group_lower_bound(cb, glx, gly, glz, ghx, ghy, ghz) <= mkd)
                    key = child_order_key32(cb, gx, gy, gz, static_cast<int>(lane));
                // the children's boxes for every lane, in the (idle) staging buffer
                buf[2 * lane] = cb.lo;
                buf[2 * lane + 1] = cb.hi;
            }
#pragma unroll
            for (int size = 2; size <= 8; size <<= 1) {
#pragma unroll
                for (int stride = size >> 1; stride > 0; stride >>= 1) {
                    const uint32_t other = __shfl_xor_sync(0xffffffffu, key, stride);
                    const bool ascending = (lane & size) == 0;
                    const bool lower = (lane & stride) == 0;
                    const bool take = (lower == ascending) ? (other < key) : (other > key);
                    if (lane < 8 && take) key = other;
                }
            }
            const int nvalid = __popc(__ballot_sync(0xffffffffu, lane < 8 && key != 0xffffffffu));
            if constexpr (STATS) {
                st.v[kStExpansions] += lane == 0;
                st.v[kStBoxTests] += nvalid;
            }
            __syncwarp();
            // push the farthest first so that the nearest is popped first
            for (int i = nvalid - 1; i >= 0; --i) {
                const int ci = static_cast<int>(__shfl_sync(0xffffffffu, key, i) & 7u);
                NodeBox b;
                b.lo = buf[2 * ci];
                b.hi = buf[2 * ci + 1];
                const int32_t bc = __shfl_sync(0xffffffffu, cc, ci);
                const unsigned int cneed =
                    __ballot_sync(0xffffffffu, active && box_lower_bound(b, c.x, c.y, c.z) <= best.kth_d2());
                if (cneed) {
                    if (sp < kStackDepth) {
                        if (lane == 0) stack_e[warp][sp] = make_int2(bc >= 0 ? bc : ~(fc + ci), static_cast<int>(cneed));
                        ++sp;
                    } else {
                        guard_ok = false;
                    }
                }
            }
            __syncwarp();
        } else {
            // a leaf: its point range from the node table
            const NodeBox* const lb = a.nodes + ~fc;
            const uint32_t start = __float_as_uint(__ldg(&lb->lo.w)), end = __float_as_uint(__ldg(&lb->hi.w));
            const unsigned int needing = __ballot_sync(0xffffffffu, need);
            const uint32_t n_need = static_cast<uint32_t>(__popc(needing));
            if constexpr (STATS) st.v[kStLeaves] += lane == 0;
            for (uint32_t base = start; base < end; base += 32) {
                const uint32_t m = min(32u, end - base);
                const float4 mine = lane < m ? __ldg(&a.pts[base + lane]) : make_float4(0.f, 0.f, 0.f, 0.f);
                buf[lane] = mine;
                // pass 1 compares distances only (<= keeps ties for the exact test of pass 2)
                const float kd = best.kth_d2();
                cbuf[lane] = make_float4(c.x, c.y, c.z, kd);
                __syncwarp();
                uint32_t cand = 0;
                if (2 * n_need < m) {
                    // few centres for the chunk's points (under half: k = 16 on the 10M tile 9.0
                    // ms, 9.15 ms with the threshold at all of them): every lane holds a point,
                    // the centres come in turn
                    unsigned int todo = needing;
                    while (todo) {
                        const int l = __ffs(todo) - 1;
                        todo &= todo - 1;
                        const float4 cl = cbuf[l];
                        const bool in = lane < m && sq_dist(__fsub_rn(mine.x, cl.x), __fsub_rn(mine.y, cl.y),
                                                            __fsub_rn(mine.z, cl.z)) <= cl.w;
                        const uint32_t b = __ballot_sync(0xffffffffu, in);
                        if (lane == static_cast<unsigned int>(l)) cand = b;
                    }
                } else {
#pragma unroll 8
                    for (uint32_t t = 0; t < m; ++t) {
                        const float4 q = buf[t];
                        if (sq_dist(__fsub_rn(q.x, c.x), __fsub_rn(q.y, c.y), __fsub_rn(q.z, c.z)) <= kd) cand |= 1u << t;
                    }
                }
                // positions this lane already saw in its seeding window
                const int64_t lo = max(win_lo, static_cast<int64_t>(base));
                const int64_t hi = min(win_lo + static_cast<int64_t>(win_n), static_cast<int64_t>(base) + m);
                if (lo < hi) {
                    const uint32_t len = static_cast<uint32_t>(hi - lo);
                    const uint32_t run = len >= 32 ? 0xffffffffu : ((1u << len) - 1u);
                    cand &= ~(run << static_cast<uint32_t>(lo - base));
                }
                if (!need) cand = 0;
                if constexpr (STATS) {
                    st.v[kStPointTests] += 2 * n_need < m ? n_need : m;  // per lane: transposed or not
                    st.v[kStNeeded] += need ? m : 0u;
                    st.v[kStPassed] += __popc(cand);
                }
                while (__ballot_sync(0xffffffffu, cand != 0)) {
                    if (cand) {
                        const int t = __ffs(cand) - 1;
                        cand &= cand - 1;
                        const uint64_t nk = key_of(buf[t]);
                        if (nk < best.kth) {
                            best.insert(nk);
                            if constexpr (STATS) st.v[kStInserts] += 1;
                        }
                    }
                }
                __syncwarp();
            }
        }
    }
    if (active) {
        best.finish();
        best.store(a, out_base);
    }
    if (!guard_ok && lane == 0) atomicOr(a.err, kGuardTripped);
    if constexpr (STATS) st.flush(a.stats);
}

template <int KMAX, bool STATS = false>
__global__ void __launch_bounds__(128) k_knn_lane(KnnArgs a) {
    const int64_t qi = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (qi >= a.nq) return;
    const float4 c = a.q[qi];
    const uint32_t row = __float_as_uint(c.w);
    StatAcc st;
    if constexpr (STATS) {
        st.zero();
        st.v[kStWalks] = 1;
    }
    BestList<KMAX> best;
    best.init(a.k);
    int32_t stk[kStackDepth];
    int sp = 1;
    stk[0] = 0;
    bool guard_ok = true;
    for (int64_t steps = 0; sp > 0; ++steps) {
        if (steps >= a.max_steps) {
            guard_ok = false;
            break;
        }
        const int32_t node = stk[--sp];
        const NodeBox b = a.nodes[node];
        const uint32_t start = __float_as_uint(b.lo.w), end = __float_as_uint(b.hi.w);
        if (start == end) continue;
        if constexpr (STATS) st.v[kStBoxTests] += 1;
        if (box_lower_bound(b, c.x, c.y, c.z) > best.kth_d2()) continue;
        const int32_t fc = a.child[node];
        if (fc >= 0) {
            if constexpr (STATS) {
                st.v[kStExpansions] += 1;
                st.v[kStBoxTests] += 8;
            }
            uint64_t keys[8];
#pragma unroll
            for (int ci = 0; ci < 8; ++ci) keys[ci] = child_order_key(a.nodes[fc + ci], c.x, c.y, c.z, ci);
            // insertion sort, descending, so that the nearest child is pushed last
#pragma unroll
            for (int x = 1; x < 8; ++x)
#pragma unroll
                for (int y = x; y > 0; --y)
                    if (keys[y] > keys[y - 1]) {
                        const uint64_t t = keys[y]; keys[y] = keys[y - 1]; keys[y - 1] = t;
                    }
#pragma unroll
            for (int ci = 0; ci < 8; ++ci)
                if ((keys[ci] >> 32) != 0xffffffffull) {
                    if (sp < kStackDepth) stk[sp++] = fc + static_cast<int32_t>(keys[ci] & 7ull);
                    else guard_ok = false;
                }
        } else {
            if constexpr (STATS) {
                st.v[kStLeaves] += 1;
                st.v[kStPointTests] += end - start;
                st.v[kStNeeded] += end - start;
            }
            for (uint32_t j = start; j < end; ++j) {
                const uint32_t id = a.perm[j];
                const float4 p = a.pts[id];
                const uint64_t nk = pair_key(sq_dist(__fsub_rn(p.x, c.x), __fsub_rn(p.y, c.y), __fsub_rn(p.z, c.z)), id);
                if (nk < best.kth) {
                    best.insert(nk);
                    if constexpr (STATS) {
                        st.v[kStPassed] += 1;
                        st.v[kStInserts] += 1;
                    }
                }
            }
        }
    }
    best.store(a, row);
    if (!guard_ok) atomicOr(a.err, kGuardTripped);
    if constexpr (STATS) {
        // the lanes of this warp that passed the entry test: a prefix of the warp
        const int64_t live = a.nq - (qi - static_cast<int64_t>(lane_id()));
        st.flush(a.stats, live >= 32 ? 0xffffffffu : (1u << live) - 1u);
    }
}

// Lists of exactly KF pairs (and, for all-points searches, a window of KF positions per
// side) run a copy of the group kernel with those sizes fixed at compile time: the list and
// window loops unroll (kNN on the 10M-point tile: k = 16 8.85 -> 8.15 ms, k = 8 5.12 ->
// 4.85 ms).  *done: k is KF and the kernel was launched.
template <int KMAX, int KF>
static sfc_status launch_knn_fixed(const KnnArgs& a, cudaStream_t s, bool* done) {
    static_assert(KF <= KMAX, "the list fits the kernel's shared memory");
    constexpr int kWarps = knn_warps<KMAX>();
    *done = a.k == KF;
    if (!*done) return SFC_OK;
    if (a.window == KF)
        SFC_LAUNCH("knn", s, (k_knn_group<KMAX, false, KF, KF>), grid_for(a.ngroups, kWarps), kWarps * 32, 0, a);
    else
        SFC_LAUNCH("knn", s, (k_knn_group<KMAX, false, KF>), grid_for(a.ngroups, kWarps), kWarps * 32, 0, a);
    return SFC_OK;
}

template <int KMAX>
static sfc_status launch_knn(const Octree* t, const KnnArgs& a, cudaStream_t s) {
    constexpr int kWarps = knn_warps<KMAX>();
    if (a.stats) {  // work counters on: the instrumented copies (same results)
        if (t->enc == SFC_ENC_NONE) SFC_LAUNCH("knn", s, (k_knn_lane<KMAX, true>), grid_for(a.nq, 128), 128, 0, a);
        else SFC_LAUNCH("knn", s, (k_knn_group<KMAX, true>), grid_for(a.ngroups, kWarps), kWarps * 32, 0, a);
    } else if (t->enc == SFC_ENC_NONE) {
        SFC_LAUNCH("knn", s, k_knn_lane<KMAX>, grid_for(a.nq, 128), 128, 0, a);
    } else {
        bool done = false;
        SFC_TRY((launch_knn_fixed<KMAX, KMAX>(a, s, &done)));
        if constexpr (KMAX == 64)  // k = 50 of the LiDAR kNN workloads
            if (!done) SFC_TRY((launch_knn_fixed<KMAX, 50>(a, s, &done)));
        if (done) return SFC_OK;
        SFC_LAUNCH("knn", s, k_knn_group<KMAX>, grid_for(a.ngroups, kWarps), kWarps * 32, 0, a);
    }
    return SFC_OK;
}

template <int KMAX>
static sfc_status launch_batch_knn(const KnnArgs& a, unsigned int grid, int exact, cudaStream_t s) {
    if (exact == 2) SFC_LAUNCH("batch_knn", s, (k_knn_group<KMAX, false, KMAX, KMAX>), grid, kKnnWarps * 32, 0, a);
    else if (exact == 1) SFC_LAUNCH("batch_knn", s, (k_knn_group<KMAX, false, KMAX>), grid, kKnnWarps * 32, 0, a);
    else SFC_LAUNCH("batch_knn", s, k_knn_group<KMAX>, grid, kKnnWarps * 32, 0, a);
    return SFC_OK;
}

// all kNN clouds of one list-size class of a batch, in one launch (sfc_batch.cu)
sfc_status batch_knn_launch(const float4* pts, const uint32_t* perm, const NodeBox* nodes, const int32_t* child,
                            int64_t total_nodes, const SearchSeg* segs, int nsegs, int64_t ngroups, int kmax, int exact,
                            int32_t* out_idx, float* out_d2, unsigned int* err, const unsigned int* skip,
                            unsigned int skip_mask, cudaStream_t s) {
    if (ngroups == 0) return SFC_OK;
    KnnArgs a;
    memset(&a, 0, sizeof a);
    a.pts = pts;
    a.perm = perm;
    a.nodes = nodes;
    a.child = child;
    a.q = pts;
    a.nq = ngroups * 32;
    a.k = kmax;
    a.out_idx = out_idx;
    a.out_d2 = out_d2;
    a.err = err;
    a.max_steps = total_nodes;
    a.window = 0;  // each cloud's own
    a.segs = segs;
    a.nsegs = nsegs;
    a.ngroups = ngroups;
    a.skip = skip;
    a.skip_mask = skip_mask;
    const unsigned int grid = grid_for(ngroups, kKnnWarps);
    // exact 1: every cloud's k is kmax, so the lists have a compile-time size; 2: every
    // seeding window is kmax positions per side as well
    switch (kmax) {
    case 8: SFC_TRY(launch_batch_knn<8>(a, grid, exact, s)); break;
    case 16: SFC_TRY(launch_batch_knn<16>(a, grid, exact, s)); break;
    case 32: SFC_TRY(launch_batch_knn<32>(a, grid, exact, s)); break;
    default: SFC_TRY(launch_batch_knn<64>(a, grid, exact, s)); break;
    }
    return SFC_OK;
}

__global__ void k_knn_pad(int32_t* idx, float* d2, int64_t total) {
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total; i += stride) {
        idx[i] = -1;
        d2[i] = INFINITY;
    }
}

}  // namespace sfc

extern "C" sfc_status knn(sfc_octree h, const float* queries_xyz, int64_t n_queries, int32_t k, void* cuda_stream,
                          int32_t* out_idx, float* out_d2) {
    if (!h || k < 1) return SFC_ERR_INVALID;
    if (k > sfc::kMaxK) return SFC_ERR_TOO_LARGE;
    const sfc::Octree* t = &h->tree;
    int64_t rows;
    if (!queries_xyz) {
        if (n_queries != 0 && n_queries != t->n) return SFC_ERR_INVALID;
        rows = t->n;
    } else {
        if (n_queries < 0) return SFC_ERR_INVALID;
        if (n_queries > 0x7fffffffLL - 1) return SFC_ERR_TOO_LARGE;
        if (n_queries > 0 && !sfc::is_device_ptr(queries_xyz)) return SFC_ERR_NOT_DEVICE_PTR;
        rows = n_queries;
    }
    if (rows == 0) return SFC_OK;
    if (!out_idx || !out_d2) return SFC_ERR_INVALID;
    if (!sfc::is_device_ptr(out_idx) || !sfc::is_device_ptr(out_d2)) return SFC_ERR_NOT_DEVICE_PTR;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    sfc::Scratch scratch(s);
    unsigned int* bad = nullptr;
    if (queries_xyz) {
        SFC_TRY(scratch.alloc(&bad, 1));
        SFC_CUDA(cudaMemsetAsync(bad, 0, sizeof(unsigned int), s));
    }
    const float4* q4 = nullptr;
    SFC_TRY(sfc::prepare_queries(t, queries_xyz, rows, s, scratch, &q4, bad));
    if (t->n == 0) {
        SFC_LAUNCH("knn_pad", s, sfc::k_knn_pad, sfc::grid_for(rows * k, 256, 152 * 16), 256, 0, out_idx, out_d2,
                   rows * k);
    } else {
        sfc::KnnArgs a;
        a.pts = t->pts;
        a.perm = t->perm;
        a.nodes = t->nodes;
        a.child = t->child;
        a.q = q4;
        a.nq = rows;
        a.k = k;
        a.out_idx = out_idx;
        a.out_d2 = out_d2;
        a.err = &t->scal->bad;
        a.max_steps = t->n_nodes;
        a.segs = nullptr;
        a.nsegs = 0;
        a.ngroups = (rows + 31) / 32;
        a.skip = nullptr;
        a.skip_mask = 0;
        a.stats = sfc::stats_counters();
        // curve neighbours per side for the seeding window: k (measured best from k = 8 to
        // 64 on the LiDAR tile; much narrower windows leave the walk many insertions)
        a.window = (!queries_xyz && t->enc != SFC_ENC_NONE) ? sfc::knn_default_window(k) : 0;
        if (k <= 8) SFC_TRY(sfc::launch_knn<8>(t, a, s));
        else if (k <= 16) SFC_TRY(sfc::launch_knn<16>(t, a, s));
        else if (k <= 32) SFC_TRY(sfc::launch_knn<32>(t, a, s));
        else SFC_TRY(sfc::launch_knn<64>(t, a, s));
    }
    if (bad) {
        unsigned int hbad = 0, herr = 0;
        SFC_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
        SFC_CUDA(cudaMemcpyAsync(&herr, &t->scal->bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
        SFC_CUDA(cudaStreamSynchronize(s));
        if (hbad) return SFC_ERR_NOT_FINITE;
        SFC_TRY(sfc::guard_status(herr));
    }
    return SFC_OK;
}
