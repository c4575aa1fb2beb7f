// sfc_radius.cu - fixed-radius search over the linear octree (section 3.2 kernels,
// section 5.1 neighboursPrune / neighboursLin), compacted into CSR by a count pass, an
// exclusive scan and a fill pass that repeats the count pass's decisions exactly.
//
// Work layout.  For a cloud ordered along the curve, a warp takes 32 consecutive
// centres in curve order (they are close in space) and walks the octree once for all of
// them: one lane per centre, the node stack shared in shared memory, a node entered when
// any lane's kernel may reach its box (for a compact group of centres: when the group's box
// may, the lanes deciding at the leaves).  Leaf points are read with warp-uniform loads and
// tested by every lane against its own centre; hits become a 32-bit mask per lane, and
// the warp writes each lane's hits as one contiguous run of its output row.  For the
// unordered cloud (SFC_ENC_NONE) the 32 centres of a warp are scattered, so each lane
// walks the tree on its own and reads points through the permutation.
//
// Count and fill.  The fill pass must repeat the count pass's decisions exactly.  For
// all-points searches the count pass records, per warp, every leaf chunk that produced a
// hit (its position and the 32 lanes' hit masks) and every node taken whole, in walk
// order; the fill pass replays those records and only writes.  A warp whose records do
// not fit its slots walks the tree again in the fill pass (the same code, the same
// decisions).
//
// Exactness of the box tests.  Each node stores the tight bounding box of its points.
// Rounding to nearest is monotone, so with d = fl(p - c) per axis: the box point
// nearest to c (the clamp of section 3.3) has the smallest |d| on every axis, and one of
// the two faces has the largest.  Every kernel test is monotone in |dx|, |dy|, |dz|, so
// when the nearest box point fails the test every point of the box fails it (prune,
// step 1b), and when the farthest corner passes every point passes (take the whole range,
// step 1a).  Both shortcuts therefore give exactly the per-point result.
#include <cuda_runtime.h>
#include <math.h>
#include <string.h>

#include "sfc_internal.cuh"

namespace sfc {

// warps per block of the group kernel (small blocks: per-warp work varies widely)
template <bool FILL>
__host__ __device__ constexpr int radius_warps() { return FILL ? 2 : 1; }

struct RadiusArgs {
    const float4* __restrict__ pts;     // sorted cloud (ordered encodings) or input order (NONE)
    const uint32_t* __restrict__ perm;  // sorted position -> original index
    const NodeBox* __restrict__ nodes;
    const int32_t* __restrict__ child;
    const float4* __restrict__ q;       // centres in processing order, w = output row
    int64_t nq;
    float r, r2;
    int prune;
    uint32_t* counts;                   // count pass: neighbours per row
    const int64_t* row_ptr;             // fill pass
    int32_t* cols;
    int2* runs;                         // range output: [start, end) sorted positions per run
    int out_runs;                       // 1: range output (count runs / write runs)
    unsigned int* err;                  // kGuardTripped is or-ed in when a guard fails
    int64_t max_steps;                  // nodes of the tree: a walk pops each node once at most
    // hit-mask records: mode 1 = this count pass records them, 2 = this fill pass replays
    int rec_mode;
    int rec_cap;
    uint32_t* rec_masks;
    uint2* rec_head;
    uint32_t* rec_count;
    float compact_factor;               // groups narrower than compact_factor * r on every axis skip
                                        // the per-lane tests of internal nodes (0: never)
    // batched search: nsegs clouds, ngroups warp groups in all (segs == nullptr: one cloud)
    const SearchSeg* segs;
    int nsegs;
    int64_t ngroups;
    // batched search: the launch does nothing when (*skip & skip_mask) != 0 (a capacity
    // overflow found on the device earlier in the same stream)
    const unsigned int* skip;
    unsigned int skip_mask;
    unsigned long long* stats;          // work counters (the STATS copies of the count pass)
};

// A record header is (chunk start, chunk size <= 32) for a leaf chunk, or
// (range start, kRangeBit | range end) for a node taken whole (step 1a).
constexpr uint32_t kRangeBit = 0x80000000u;

// 0: no point of the box is inside the kernel; 2: every point is (asked only with
// prune); 1: undecided.
template <int KERN>
__device__ __forceinline__ int classify_box(const NodeBox& b, float cx, float cy, float cz, float r, float r2,
                                            bool prune) {
    const float nx = __fsub_rn(fminf(fmaxf(cx, b.lo.x), b.hi.x), cx);
    const float ny = __fsub_rn(fminf(fmaxf(cy, b.lo.y), b.hi.y), cy);
    const float nz = __fsub_rn(fminf(fmaxf(cz, b.lo.z), b.hi.z), cz);
    if (!kernel_holds<KERN>(nx, ny, nz, r, r2)) return 0;
    if (!prune) return 1;
    const float fx = fmaxf(fabsf(__fsub_rn(b.lo.x, cx)), fabsf(__fsub_rn(b.hi.x, cx)));
    const float fy = fmaxf(fabsf(__fsub_rn(b.lo.y, cy)), fabsf(__fsub_rn(b.hi.y, cy)));
    const float fz = fmaxf(fabsf(__fsub_rn(b.lo.z, cz)), fabsf(__fsub_rn(b.hi.z, cz)));
    return kernel_holds<KERN>(fx, fy, fz, r, r2) ? 2 : 1;
}

// Gap between a box and the box [glo, ghi] of a group of centres, per axis (0 when they
// overlap).  For any centre c in the group box and any point p in the node box,
// |fl(p - c)| >= gap on that axis (rounding is monotone), so a failed kernel test on the
// gaps proves that no centre of the group reaches any point of the node.
__device__ __forceinline__ float axis_gap(float lo, float hi, float glo, float ghi) {
    return fmaxf(fmaxf(__fsub_rn(lo, ghi), __fsub_rn(glo, hi)), 0.0f);
}

// The walk keeps, per pushed node, what its parent's expansion learnt: its first child,
// its point range and which lanes find it undecided or wholly inside their kernel, so a
// pop reads shared memory only.  An expansion loads the eight children once (lanes 0-7),
// drops those no centre of the group can reach, and classifies the rest for every lane.
// Leaf points are staged in shared memory with one coalesced load per 32-point chunk.
// RUNS: the range output (neighboursStruct, section 5.1): each row lists its neighbours as
// maximal runs [start, end) of consecutive sorted positions instead of one id each; the
// count pass counts runs, the fill writes them.
constexpr uint32_t kNoRun = 0xffffffffu;

// Groups whose centres lie within this many radii of each other skip the per-lane
// classification of internal nodes (see k_radius_group).  Measured on the 10M-point tile,
// sphere r = 2 m: count pass 3.51 ms with no group skipping, 3.50 / 3.42 / 3.39 ms at 1 / 2 / 4.
constexpr float kCompactFactor = 4.0f;

// STATS: the count pass also accumulates the work counters of sfc_search_stats.
template <int KERN, bool FILL, bool RUNS, bool STATS = false>
// 18 two-warp fill blocks per SM (at most 56 registers) keep 36 warps resident: the fill
// waits on memory more than the count pass does
__global__ void __launch_bounds__(radius_warps<FILL>() * 32, FILL ? 18 : 32) k_radius_group(RadiusArgs a) {
    static_assert(!STATS || (!FILL && !RUNS), "only the count pass of the CSR output is instrumented");
    constexpr int kRadiusWarps = radius_warps<FILL>();
    __shared__ int4 stack_e[kRadiusWarps][kStackDepth];      // first child, start, end, undecided lanes
    __shared__ uint32_t stack_w[kRadiusWarps][kStackDepth];  // lanes taking the node whole
    __shared__ float4 chunk[kRadiusWarps][32];
    __shared__ float4 centre[FILL ? 1 : kRadiusWarps][32];  // count pass: the warp's centres
    const unsigned int lane = lane_id();
    const int warp = threadIdx.x >> 5;
    const int64_t group = static_cast<int64_t>(blockIdx.x) * kRadiusWarps + warp;
    int64_t first = group * 32, q_end = a.nq, row0 = 0;
    int32_t root = 0;
    unsigned int gsize = 32;  // centres of this group (batched clouds may ask for fewer)
    float r = a.r, r2 = a.r2;
    if (a.segs) {
        if (group >= a.ngroups) return;  // whole warp
        if (a.skip && (*a.skip & a.skip_mask)) return;
        const SearchSeg sg = a.segs[find_search_seg(a.segs, a.nsegs, group)];
        gsize = static_cast<unsigned int>(sg.group_size);
        first = sg.q0 + (group - sg.group0) * gsize;
        q_end = sg.q0 + sg.nq;
        row0 = sg.row0;
        root = sg.root;
        r = sg.r;
        r2 = sg.r2;
    } else if (first >= a.nq) {
        return;  // whole warp
    }
    const int64_t qi = first + lane;
    const bool active = lane < gsize && qi < q_end;
    const float4 c = active ? a.q[qi] : make_float4(0.f, 0.f, 0.f, 0.f);
    const int64_t row = row0 + __float_as_uint(c.w);
    if constexpr (!FILL) centre[warp][lane] = c;  // read by other lanes after the next __syncwarp
    const unsigned int below = lanes_below();
    const bool prune = a.prune != 0;
    StatAcc st;
    if constexpr (STATS) {
        st.zero();
        st.v[kStWalks] = lane == 0;
    }
    uint32_t count = 0;
    int64_t out = (FILL && active) ? a.row_ptr[row] : 0;
    const int64_t out_end = (FILL && active) ? a.row_ptr[row + 1] : 0;
    bool guard_ok = true;

    // ---- emitting (shared by the walk and the replay)
    // range output: the lane's open run [run_s, run_e); positions arrive in ascending order
    uint32_t run_s = 0, run_e = kNoRun;
    auto flush_run = [&]() {
        if (out < out_end) a.runs[out] = make_int2(static_cast<int>(run_s), static_cast<int>(run_e));
        else guard_ok = false;
        ++out;
    };
    auto add_run = [&](uint32_t s0, uint32_t e0) {
        if (s0 == run_e) {
            run_e = e0;
            return;
        }
        if (FILL && run_e != kNoRun) flush_run();
        run_s = s0;
        run_e = e0;
        ++count;
    };
    auto finish_runs = [&]() {
        if (RUNS && FILL && run_e != kNoRun) flush_run();
    };
    // the lanes of `whole` take [start, end) (step 1a)
    auto take_range = [&](unsigned int whole, uint32_t start, uint32_t end, bool mine) {
        if (RUNS) {
            if (mine) add_run(start, end);
            return;
        }
        if (FILL) {
            unsigned int todo = whole;
            while (todo) {
                const int src = __ffs(todo) - 1;
                todo &= todo - 1;
                const int64_t o = __shfl_sync(0xffffffffu, out, src);
                const int64_t e = __shfl_sync(0xffffffffu, out_end, src);
                if (o + (end - start) > e) {
                    guard_ok = false;
                    continue;
                }
                for (uint32_t j = start + lane; j < end; j += 32)
                    a.cols[o + (j - start)] = static_cast<int32_t>(a.perm[j]);
            }
        }
        if (mine) {
            count += end - start;
            out += end - start;
        }
    };
    // the hits of a leaf chunk at positions base + t: lane i's row gets the ids (my_id of
    // lane j) of its mask's bits, or their runs
    auto take_hits = [&](uint32_t hits, int32_t my_id, uint32_t base) {
        if (RUNS) {
            if (!FILL) {  // count runs: starts of runs of ones, the first may extend the open run
                if (hits) {
                    count += __popc(hits & ~(hits << 1));
                    if ((hits & 1u) && base == run_e) --count;
                    run_e = base + 32u - static_cast<uint32_t>(__clz(hits));
                }
                return;
            }
            uint32_t m = hits;
            while (m) {
                const int s0 = __ffs(m) - 1;
                const uint32_t rest = ~(m >> s0);  // zeros where the run of ones continues
                const int len = rest ? __ffs(rest) - 1 : 32 - s0;
                add_run(base + s0, base + s0 + len);
                m = s0 + len >= 32 ? 0u : (m & (~0u << (s0 + len)));
            }
            return;
        }
        count += __popc(hits);
        if (FILL) {
            if (out + __popc(hits) > out_end) {  // never true when the count pass agrees
                guard_ok = false;
                hits = 0;
            }
            unsigned int todo = __ballot_sync(0xffffffffu, hits != 0);
            if (todo) {
                // one row per round: the lane of chunk point t writes its id at the point's
                // rank in the row's hits, so each row's hits go out as one contiguous run
                const uint32_t below = (1u << lane) - 1u;
                while (todo) {
                    const int src = __ffs(todo) - 1;
                    todo &= todo - 1;
                    const uint32_t hh = __shfl_sync(0xffffffffu, hits, src);
                    const int64_t o = __shfl_sync(0xffffffffu, out, src);
                    if ((hh >> lane) & 1u) a.cols[o + __popc(hh & below)] = my_id;
                }
            }
            out += __popc(hits);
        }
    };

    // ---- replay of the count pass's records
    if (FILL && a.rec_mode == 2) {
        const uint32_t nrec = a.rec_count[group];
        if (nrec <= static_cast<uint32_t>(a.rec_cap)) {  // else the records overflowed: walk again
            // three records in flight: while record k is written, record k + 1's ids and
            // record k + 2's header and masks are loading
            const int64_t slot0 = group * a.rec_cap;
            auto head_of = [&](uint32_t k) { return k < nrec ? a.rec_head[slot0 + k] : make_uint2(0u, 0u); };
            auto mask_of = [&](uint32_t k) { return (k < nrec && active) ? a.rec_masks[(slot0 + k) * 32 + lane] : 0u; };
            auto ids_of = [&](uint2 hd) {
                return (!RUNS && !(hd.y & kRangeBit) && lane < hd.y) ? static_cast<int32_t>(a.perm[hd.x + lane]) : 0;
            };
            uint2 hd = head_of(0), hd1 = head_of(1);
            uint32_t mask = mask_of(0), mask1 = mask_of(1);
            int32_t my_id = ids_of(hd);
            for (uint32_t k = 0; k < nrec; ++k) {
                const uint2 hd2 = head_of(k + 2);
                const uint32_t mask2 = mask_of(k + 2);
                const int32_t id1 = ids_of(hd1);
                if (hd.y & kRangeBit) {
                    take_range(__ballot_sync(0xffffffffu, mask != 0), hd.x, hd.y & ~kRangeBit, mask != 0);
                } else {
                    take_hits(mask, my_id, hd.x);
                }
                hd = hd1;
                hd1 = hd2;
                mask = mask1;
                mask1 = mask2;
                my_id = id1;
            }
            finish_runs();
            if (!guard_ok) atomicOr(a.err, kGuardTripped);
            return;
        }
    }

    // ---- the walk
    uint32_t nrec = 0;
    bool rec_overflow = false;
    auto record = [&](uint32_t hx, uint32_t hy, uint32_t mask) {
        if (nrec < static_cast<uint32_t>(a.rec_cap)) {
            const int64_t slot = group * a.rec_cap + nrec;
            a.rec_masks[slot * 32 + lane] = mask;
            if (lane == 0) a.rec_head[slot] = make_uint2(hx, hy);
        } else {
            rec_overflow = true;
        }
        ++nrec;
    };
    const bool recording = !FILL && a.rec_mode == 1;
    uint32_t taken_below = 0;  // positions below this were emitted as a whole range

    // bounding box of the group's centres
    float glx = active ? c.x : INFINITY, gly = active ? c.y : INFINITY, glz = active ? c.z : INFINITY;
    float ghx = active ? c.x : -INFINITY, ghy = active ? c.y : -INFINITY, ghz = active ? c.z : -INFINITY;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        glx = fminf(glx, __shfl_xor_sync(0xffffffffu, glx, o));
        gly = fminf(gly, __shfl_xor_sync(0xffffffffu, gly, o));
        glz = fminf(glz, __shfl_xor_sync(0xffffffffu, glz, o));
        ghx = fmaxf(ghx, __shfl_xor_sync(0xffffffffu, ghx, o));
        ghy = fmaxf(ghy, __shfl_xor_sync(0xffffffffu, ghy, o));
        ghz = fmaxf(ghz, __shfl_xor_sync(0xffffffffu, ghz, o));
    }
    // a compact group (centres within compact_factor * r of each other on every axis) enters
    // an internal node for every lane that reached its parent, without classifying it per
    // lane: the group's gap test has already dropped what none of them can reach, and the
    // per-lane tests at the leaves keep the results exact
    const bool compact = fmaxf(fmaxf(__fsub_rn(ghx, glx), __fsub_rn(ghy, gly)), __fsub_rn(ghz, glz)) <=
                         a.compact_factor * r;

    int sp = 0;
    {
        const NodeBox rb = a.nodes[root];
        const int32_t rc = a.child[root];
        const int cls = active ? classify_box<KERN>(rb, c.x, c.y, c.z, r, r2, prune) : 0;
        if constexpr (STATS) st.v[kStBoxTests] += 1;
        const unsigned int p = __ballot_sync(0xffffffffu, cls == 1);
        const unsigned int w = __ballot_sync(0xffffffffu, cls == 2);
        if (p | w) {
            if (lane == 0) {
                stack_e[warp][0] = make_int4(rc, __float_as_int(rb.lo.w), __float_as_int(rb.hi.w), static_cast<int>(p));
                stack_w[warp][0] = w;
            }
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
        const int4 e = stack_e[warp][sp];
        const uint32_t wmask = stack_w[warp][sp];
        __syncwarp();
        const int32_t fc = e.x;
        const uint32_t start = static_cast<uint32_t>(e.y), end = static_cast<uint32_t>(e.z);
        const bool live = active && end > taken_below;
        const bool my_partial = live && ((static_cast<uint32_t>(e.w) >> lane) & 1u);
        const bool my_whole = live && ((wmask >> lane) & 1u);
        if (fc >= 0) {
            const unsigned int whole = __ballot_sync(0xffffffffu, my_whole);
            const unsigned int partial = __ballot_sync(0xffffffffu, my_partial);
            if (whole) {
                if constexpr (STATS) st.v[kStWhole] += my_whole ? end - start : 0u;
                take_range(whole, start, end, my_whole);
                if (recording) record(start, kRangeBit | end, my_whole ? 0xffffffffu : 0u);
                if (my_whole) taken_below = end;
            }
            if (partial) {
                NodeBox cb;
                int32_t cc = -1;
                bool keep = false;
                if (lane < 8) {
                    cb = a.nodes[fc + lane];
                    cc = a.child[fc + lane];
                    if (__float_as_uint(cb.lo.w) != __float_as_uint(cb.hi.w))
                        keep = kernel_holds<KERN>(axis_gap(cb.lo.x, cb.hi.x, glx, ghx),
                                                  axis_gap(cb.lo.y, cb.hi.y, gly, ghy),
                                                  axis_gap(cb.lo.z, cb.hi.z, glz, ghz), r, r2);
                    // the children for every lane, in the (idle) chunk buffer
                    chunk[warp][2 * lane] = cb.lo;
                    chunk[warp][2 * lane + 1] = cb.hi;
                    chunk[warp][16 + lane] = make_float4(__int_as_float(cc), 0.f, 0.f, 0.f);
                }
                unsigned int kept = __ballot_sync(0xffffffffu, keep);
                if constexpr (STATS) {
                    st.v[kStExpansions] += lane == 0;
                    st.v[kStBoxTests] += __popc(kept);
                }
                __syncwarp();
                // push the last child first so that the first child is popped first
                while (kept) {
                    const int ci = 31 - __clz(kept);
                    kept &= ~(1u << ci);
                    NodeBox b;
                    b.lo = chunk[warp][2 * ci];
                    b.hi = chunk[warp][2 * ci + 1];
                    const int32_t bc = __float_as_int(chunk[warp][16 + ci].x);
                    // a lane that found the parent disjoint or took it whole has nothing here
                    const int cls = !my_partial ? 0
                                    : (compact && bc >= 0) ? 1
                                                           : classify_box<KERN>(b, c.x, c.y, c.z, r, r2, prune);
                    const unsigned int cp = __ballot_sync(0xffffffffu, cls == 1);
                    const unsigned int cw = __ballot_sync(0xffffffffu, cls == 2);
                    if (cp | cw) {
                        if (sp < kStackDepth) {
                            if (lane == 0) {
                                stack_e[warp][sp] = make_int4(bc, __float_as_int(b.lo.w), __float_as_int(b.hi.w),
                                                              static_cast<int>(cp));
                                stack_w[warp][sp] = cw;
                            }
                            ++sp;
                        } else {
                            guard_ok = false;
                        }
                    }
                }
                __syncwarp();
            }
        } else {
            // a leaf: the lanes that reach its box test every point against their own centre
            const bool need = my_partial || my_whole;
            // lanes whose kernel holds for the whole leaf box take every point untested (its
            // farthest corner passed, so every point passes: step 1a); the others test
            const unsigned int testing = __ballot_sync(0xffffffffu, my_partial);
            const uint32_t n_test = static_cast<uint32_t>(__popc(testing));
            if constexpr (STATS) st.v[kStLeaves] += lane == 0;
            for (uint32_t base = start; base < end; base += 32) {
                const uint32_t m = min(32u, end - base);
                const float4 mine = lane < m ? __ldg(&a.pts[base + lane]) : make_float4(0.f, 0.f, 0.f, 0.f);
                uint32_t hits = 0;
                // (swept on the 10M tile at r = 2 m: n_test <= m / 2 3.30 ms, <= 3 m / 4 3.36 ms, <= m 3.74 ms)
                const bool transposed = !FILL && 2 * n_test <= m;
                if (transposed) {
                    // few centres test this chunk: every lane holds a point and the testing
                    // centres come in turn, each lane's hit mask is one ballot
                    unsigned int todo = testing;
                    while (todo) {
                        const int l = __ffs(todo) - 1;
                        todo &= todo - 1;
                        const float4 cl = centre[warp][l];
                        const bool in = lane < m && kernel_holds<KERN>(__fsub_rn(mine.x, cl.x), __fsub_rn(mine.y, cl.y),
                                                                       __fsub_rn(mine.z, cl.z), r, r2);
                        const uint32_t b = __ballot_sync(0xffffffffu, in);
                        if (lane == static_cast<unsigned int>(l)) hits = b;
                    }
                } else {
                    chunk[warp][lane] = mine;
                    __syncwarp();
#pragma unroll 8
                    for (uint32_t t = 0; t < m; ++t) {
                        const float4 p = chunk[warp][t];
                        const bool in = kernel_holds<KERN>(__fsub_rn(p.x, c.x), __fsub_rn(p.y, c.y),
                                                           __fsub_rn(p.z, c.z), r, r2);
                        hits |= static_cast<uint32_t>(in) << t;
                    }
                    __syncwarp();
                }
                if (my_whole) hits = m >= 32u ? 0xffffffffu : (1u << m) - 1u;
                if (!need) hits = 0;
                if constexpr (STATS) {
                    st.v[kStPointTests] += transposed ? n_test : m;
                    st.v[kStNeeded] += my_partial ? m : 0u;
                    st.v[kStPassed] += __popc(hits);
                }
                if (recording && __ballot_sync(0xffffffffu, hits != 0)) record(base, m, hits);
                take_hits(hits, static_cast<int32_t>(__float_as_uint(mine.w)), base);
            }
        }
    }
    finish_runs();
    if (!FILL && active) a.counts[row] = count;
    if (recording && lane == 0) a.rec_count[group] = rec_overflow ? kRecordsOverflow : nrec;
    if (!guard_ok) atomicOr(a.err, kGuardTripped);
    if constexpr (STATS) st.flush(a.stats);
}

// One centre per thread, its own depth-first walk; points through the permutation.
template <int KERN, bool FILL, bool RUNS, bool STATS = false>
__global__ void __launch_bounds__(128) k_radius_lane(RadiusArgs a) {
    static_assert(!STATS || (!FILL && !RUNS), "only the count pass of the CSR output is instrumented");
    const int64_t qi = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
    if (qi >= a.nq) return;
    const float4 c = a.q[qi];
    const uint32_t row = __float_as_uint(c.w);
    const bool prune = a.prune != 0;
    StatAcc st;
    if constexpr (STATS) {
        st.zero();
        st.v[kStWalks] = 1;
    }
    int32_t stk[kStackDepth];
    int sp = 1;
    stk[0] = 0;
    uint32_t count = 0;
    int64_t out = FILL ? a.row_ptr[row] : 0;
    const int64_t out_end = FILL ? a.row_ptr[row + 1] : 0;
    bool guard_ok = true;
    uint32_t run_s = 0, run_e = kNoRun;  // range output: the open run
    auto add_run = [&](uint32_t s0, uint32_t e0) {
        if (s0 == run_e) {
            run_e = e0;
            return;
        }
        if (FILL && run_e != kNoRun) {
            if (out < out_end) a.runs[out] = make_int2(static_cast<int>(run_s), static_cast<int>(run_e));
            else guard_ok = false;
            ++out;
        }
        run_s = s0;
        run_e = e0;
        ++count;
    };
    for (int64_t steps = 0; sp > 0; ++steps) {
        if (steps >= a.max_steps) {
            guard_ok = false;
            break;
        }
        const int32_t node = stk[--sp];
        const NodeBox b = a.nodes[node];
        const uint32_t start = __float_as_uint(b.lo.w), end = __float_as_uint(b.hi.w);
        if (start == end) continue;
        const int cls = classify_box<KERN>(b, c.x, c.y, c.z, a.r, a.r2, prune);
        if constexpr (STATS) st.v[kStBoxTests] += 1;
        if (cls == 0) continue;
        const int32_t fc = a.child[node];
        if (fc >= 0) {
            if (cls == 2) {
                if constexpr (STATS) st.v[kStWhole] += end - start;
                if (RUNS) {
                    add_run(start, end);
                    continue;
                }
                if (FILL) {
                    if (out + (end - start) > out_end) {
                        guard_ok = false;
                        break;
                    }
                    for (uint32_t j = start; j < end; ++j) a.cols[out++] = static_cast<int32_t>(a.perm[j]);
                }
                count += end - start;
                continue;
            }
            if constexpr (STATS) st.v[kStExpansions] += 1;
            if (sp + 8 <= kStackDepth) {
                for (int k = 7; k >= 0; --k) stk[sp++] = fc + k;
            } else {
                guard_ok = false;
            }
        } else {
            if constexpr (STATS) {
                st.v[kStLeaves] += 1;
                st.v[kStPointTests] += end - start;
                st.v[kStNeeded] += cls == 1 ? end - start : 0u;
            }
            for (uint32_t j = start; j < end; ++j) {
                const uint32_t id = a.perm[j];
                const float4 p = a.pts[id];
                if (kernel_holds<KERN>(__fsub_rn(p.x, c.x), __fsub_rn(p.y, c.y), __fsub_rn(p.z, c.z), a.r, a.r2)) {
                    if constexpr (STATS) st.v[kStPassed] += 1;
                    if (RUNS) {
                        add_run(j, j + 1);
                        continue;
                    }
                    if (FILL) {
                        if (out < out_end) a.cols[out++] = static_cast<int32_t>(id);
                        else guard_ok = false;
                    }
                    ++count;
                }
            }
        }
    }
    if (RUNS && FILL && run_e != kNoRun) {
        if (out < out_end) a.runs[out] = make_int2(static_cast<int>(run_s), static_cast<int>(run_e));
        else guard_ok = false;
    }
    if (!FILL) a.counts[row] = count;
    if (!guard_ok) atomicOr(a.err, kGuardTripped);
    if constexpr (STATS) {
        // the lanes of this warp that passed the entry test: a prefix of the warp
        const int64_t live = a.nq - (qi - static_cast<int64_t>(lane_id()));
        st.flush(a.stats, live >= 32 ? 0xffffffffu : (1u << live) - 1u);
    }
}

// the instrumented count pass (work counters on): same decisions, same output
static sfc_status launch_count_stats(const Octree* t, RadiusArgs& a, int kern, const char* name, cudaStream_t s) {
    if (t->enc == SFC_ENC_NONE) {
        const unsigned int grid = grid_for(a.nq, 128);
        switch (kern) {
        case SFC_SPHERE: SFC_LAUNCH(name, s, (k_radius_lane<SFC_SPHERE, false, false, true>), grid, 128, 0, a); break;
        case SFC_CIRCLE: SFC_LAUNCH(name, s, (k_radius_lane<SFC_CIRCLE, false, false, true>), grid, 128, 0, a); break;
        case SFC_CUBE: SFC_LAUNCH(name, s, (k_radius_lane<SFC_CUBE, false, false, true>), grid, 128, 0, a); break;
        default: SFC_LAUNCH(name, s, (k_radius_lane<SFC_SQUARE, false, false, true>), grid, 128, 0, a); break;
        }
    } else {
        constexpr int kWarps = radius_warps<false>();
        const unsigned int grid = grid_for(a.ngroups, kWarps);
        switch (kern) {
        case SFC_SPHERE:
            SFC_LAUNCH(name, s, (k_radius_group<SFC_SPHERE, false, false, true>), grid, kWarps * 32, 0, a);
            break;
        case SFC_CIRCLE:
            SFC_LAUNCH(name, s, (k_radius_group<SFC_CIRCLE, false, false, true>), grid, kWarps * 32, 0, a);
            break;
        case SFC_CUBE:
            SFC_LAUNCH(name, s, (k_radius_group<SFC_CUBE, false, false, true>), grid, kWarps * 32, 0, a);
            break;
        default:
            SFC_LAUNCH(name, s, (k_radius_group<SFC_SQUARE, false, false, true>), grid, kWarps * 32, 0, a);
            break;
        }
    }
    return SFC_OK;
}

template <bool FILL, bool RUNS>
static sfc_status launch_search_as(const Octree* t, RadiusArgs& a, int kern, cudaStream_t s) {
    if (a.nq == 0) return SFC_OK;
    const char* name = RUNS ? (FILL ? "radius_ranges_fill" : "radius_ranges_count")
                            : (FILL ? "radius_fill" : "radius_count");
    if constexpr (!FILL && !RUNS) {
        if (a.stats) return launch_count_stats(t, a, kern, name, s);
    }
    if (t->enc == SFC_ENC_NONE) {
        const unsigned int grid = grid_for(a.nq, 128);
        switch (kern) {
        case SFC_SPHERE: SFC_LAUNCH(name, s, (k_radius_lane<SFC_SPHERE, FILL, RUNS>), grid, 128, 0, a); break;
        case SFC_CIRCLE: SFC_LAUNCH(name, s, (k_radius_lane<SFC_CIRCLE, FILL, RUNS>), grid, 128, 0, a); break;
        case SFC_CUBE: SFC_LAUNCH(name, s, (k_radius_lane<SFC_CUBE, FILL, RUNS>), grid, 128, 0, a); break;
        default: SFC_LAUNCH(name, s, (k_radius_lane<SFC_SQUARE, FILL, RUNS>), grid, 128, 0, a); break;
        }
    } else {
        constexpr int kWarps = radius_warps<FILL>();
        const int64_t groups = a.ngroups;
        const unsigned int grid = grid_for(groups, kWarps);
        switch (kern) {
        case SFC_SPHERE: SFC_LAUNCH(name, s, (k_radius_group<SFC_SPHERE, FILL, RUNS>), grid, kWarps * 32, 0, a); break;
        case SFC_CIRCLE: SFC_LAUNCH(name, s, (k_radius_group<SFC_CIRCLE, FILL, RUNS>), grid, kWarps * 32, 0, a); break;
        case SFC_CUBE: SFC_LAUNCH(name, s, (k_radius_group<SFC_CUBE, FILL, RUNS>), grid, kWarps * 32, 0, a); break;
        default: SFC_LAUNCH(name, s, (k_radius_group<SFC_SQUARE, FILL, RUNS>), grid, kWarps * 32, 0, a); break;
        }
    }
    return SFC_OK;
}

template <bool FILL>
static sfc_status launch_search(const Octree* t, RadiusArgs& a, int kern, cudaStream_t s) {
    return a.out_runs ? launch_search_as<FILL, true>(t, a, kern, s) : launch_search_as<FILL, false>(t, a, kern, s);
}

static RadiusArgs make_args(const Octree* t, const float4* q4, int64_t rows, float r) {
    RadiusArgs a;
    a.pts = t->pts;
    a.perm = t->perm;
    a.nodes = t->nodes;
    a.child = t->child;
    a.q = q4;
    a.nq = rows;
    a.r = r;
    a.r2 = r * r;  // binary32 product, rounded to nearest
    a.prune = t->prune;
    a.counts = nullptr;
    a.row_ptr = nullptr;
    a.cols = nullptr;
    a.err = &t->scal->bad;
    a.max_steps = t->n_nodes;
    a.rec_mode = 0;
    a.rec_cap = 0;
    a.rec_masks = nullptr;
    a.rec_head = nullptr;
    a.rec_count = nullptr;
    a.compact_factor = kCompactFactor;
    a.segs = nullptr;
    a.nsegs = 0;
    a.ngroups = (rows + 31) / 32;
    a.skip = nullptr;
    a.skip_mask = 0;
    a.runs = nullptr;
    a.out_runs = 0;
    a.stats = stats_counters();
    return a;
}

// rows = number of output rows; validates the arguments common to the radius calls
static sfc_status check_radius_args(sfc_octree h, const float* queries, int64_t nq, float r, sfc_kernel kern,
                                    int64_t* rows) {
    if (!h) return SFC_ERR_INVALID;
    if (kern != SFC_SPHERE && kern != SFC_CIRCLE && kern != SFC_CUBE && kern != SFC_SQUARE) return SFC_ERR_INVALID;
    if (isnan(r)) return SFC_ERR_INVALID;
    if (!queries) {
        if (nq != 0 && nq != h->tree.n) return SFC_ERR_INVALID;
        *rows = h->tree.n;
        return SFC_OK;
    }
    if (nq < 0) return SFC_ERR_INVALID;
    if (nq > 0x7fffffffLL - 1) return SFC_ERR_TOO_LARGE;
    if (nq > 0 && !is_device_ptr(queries)) return SFC_ERR_NOT_DEVICE_PTR;
    *rows = nq;
    return SFC_OK;
}

// Allocate the hit-mask records of an all-points count pass (ordered encodings only);
// without memory for them the fill pass simply walks the tree again.
static void setup_records(Octree* t, int64_t rows, float r, int kern, cudaStream_t s, RadiusArgs& a) {
    release_records(t, s);
    if (t->enc == SFC_ENC_NONE) return;
    RadiusRecords& rec = t->records;
    const int64_t groups = (rows + 31) / 32;
    const int64_t slots = groups * kRecordCapSingle;
    if (raw_alloc(reinterpret_cast<void**>(&rec.masks), sizeof(uint32_t) * 32 * slots, s) != cudaSuccess ||
        raw_alloc(reinterpret_cast<void**>(&rec.head), sizeof(uint2) * slots, s) != cudaSuccess ||
        raw_alloc(reinterpret_cast<void**>(&rec.count), sizeof(uint32_t) * groups, s) != cudaSuccess) {
        cudaGetLastError();
        release_records(t, s);
        return;
    }
    rec.groups = groups;
    rec.cap = kRecordCapSingle;
    rec.r = r;
    rec.kern = kern;
    rec.valid = false;  // set once the recording pass is launched
    a.rec_mode = 1;
    a.rec_cap = kRecordCapSingle;
    a.rec_masks = rec.masks;
    a.rec_head = rec.head;
    a.rec_count = rec.count;
}

static sfc_status count_impl(Octree* t, const float4* q4, int64_t rows, float r, int kern, cudaStream_t s,
                             Scratch& scratch, int64_t* row_ptr, const unsigned int* bad, int64_t* nnz,
                             bool all_points, bool runs = false) {
    if (!(r > 0.f) || rows == 0 || t->n == 0) {
        SFC_CUDA(cudaMemsetAsync(row_ptr, 0, sizeof(int64_t) * (rows + 1), s));
    } else {
        uint32_t* counts = nullptr;
        SFC_TRY(scratch.alloc(&counts, rows));
        RadiusArgs a = make_args(t, q4, rows, r);
        a.counts = counts;
        a.out_runs = runs ? 1 : 0;
        if (all_points) setup_records(t, rows, r, kern, s, a);
        const sfc_status st = launch_search<false>(t, a, kern, s);
        if (st != SFC_OK) {
            release_records(t, s);
            return st;
        }
        if (a.rec_mode == 1) t->records.valid = true;
        SFC_TRY(scan_u32_to_i64(counts, row_ptr, rows, s, scratch, &t->scal->bad));
    }
    unsigned int hbad = 0, herr = 0;
    SFC_CUDA(cudaMemcpyAsync(nnz, row_ptr + rows, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    if (bad) SFC_CUDA(cudaMemcpyAsync(&hbad, bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    SFC_CUDA(cudaMemcpyAsync(&herr, &t->scal->bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    SFC_CUDA(cudaStreamSynchronize(s));
    if (hbad) return SFC_ERR_NOT_FINITE;
    SFC_TRY(guard_status(herr));
    return SFC_OK;
}

sfc_status radius_count_presized(const Octree* t, float r, int kern, cudaStream_t s, uint32_t* counts,
                                 int64_t* tile_sums, int64_t* row_ptr, int64_t* nnz) {
    const int64_t rows = t->n;
    if (!(r > 0.f) || rows == 0) {
        SFC_CUDA(cudaMemsetAsync(row_ptr, 0, sizeof(int64_t) * (rows + 1), s));
    } else {
        RadiusArgs a = make_args(t, t->pts, rows, r);
        a.counts = counts;
        SFC_TRY(launch_search<false>(t, a, kern, s));
        SFC_TRY(scan_u32_to_i64_presized(counts, row_ptr, rows, tile_sums, s, &t->scal->bad));
    }
    unsigned int herr = 0;
    SFC_CUDA(cudaMemcpyAsync(nnz, row_ptr + rows, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    SFC_CUDA(cudaMemcpyAsync(&herr, &t->scal->bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    SFC_CUDA(cudaStreamSynchronize(s));
    return guard_status(herr);
}

static sfc_status fill_impl(Octree* t, const float4* q4, int64_t rows, float r, int kern, cudaStream_t s,
                            const int64_t* row_ptr, int32_t* cols, bool all_points, int2* runs = nullptr) {
    if (!(r > 0.f) || rows == 0 || t->n == 0) return SFC_OK;
    RadiusArgs a = make_args(t, q4, rows, r);
    a.row_ptr = row_ptr;
    a.cols = cols;
    a.runs = runs;
    a.out_runs = runs ? 1 : 0;
    const RadiusRecords& rec = t->records;
    uint32_t rb, qb;
    memcpy(&rb, &rec.r, sizeof rb);
    memcpy(&qb, &r, sizeof qb);
    const bool replay = all_points && rec.valid && rec.kern == kern && rb == qb && rec.groups == (rows + 31) / 32;
    if (replay) {
        a.rec_mode = 2;
        a.rec_cap = rec.cap;
        a.rec_masks = rec.masks;
        a.rec_head = rec.head;
        a.rec_count = rec.count;
    }
    const sfc_status st = launch_search<true>(t, a, kern, s);
    if (replay) release_records(t, s);  // stream-ordered after the replay
    return st;
}

static sfc_status check_guard(const Octree* t, cudaStream_t s) {
    unsigned int herr = 0;
    SFC_CUDA(cudaMemcpyAsync(&herr, &t->scal->bad, sizeof(unsigned int), cudaMemcpyDeviceToHost, s));
    SFC_CUDA(cudaStreamSynchronize(s));
    return guard_status(herr);
}

static sfc_status prepare(const Octree* t, const float* queries, int64_t rows, cudaStream_t s, Scratch& scratch,
                          const float4** q4, unsigned int** bad) {
    *bad = nullptr;
    if (queries) {
        SFC_TRY(scratch.alloc(bad, 1));
        SFC_CUDA(cudaMemsetAsync(*bad, 0, sizeof(unsigned int), s));
    }
    return prepare_queries(t, queries, rows, s, scratch, q4, *bad);
}

// all radius clouds of one kernel type of a batch, in one launch (sfc_batch.cu)
sfc_status batch_radius_launch(const float4* pts, const uint32_t* perm, const NodeBox* nodes, const int32_t* child,
                               int64_t total_nodes, const SearchSeg* segs, int nsegs, int64_t ngroups, int kern,
                               bool fill, uint32_t* counts, const int64_t* row_ptr, int32_t* cols, unsigned int* err,
                               int prune, const BatchRecords& rec, const unsigned int* skip, unsigned int skip_mask,
                               cudaStream_t s) {
    if (ngroups == 0) return SFC_OK;
    RadiusArgs a;
    memset(&a, 0, sizeof a);
    a.pts = pts;
    a.perm = perm;
    a.nodes = nodes;
    a.child = child;
    a.q = pts;
    a.nq = ngroups * 32;
    a.prune = prune;
    a.counts = counts;
    a.row_ptr = row_ptr;
    a.cols = cols;
    a.err = err;
    a.max_steps = total_nodes;
    a.segs = segs;
    a.nsegs = nsegs;
    a.ngroups = ngroups;
    a.skip = skip;
    a.skip_mask = skip_mask;
    a.compact_factor = kCompactFactor;
    if (rec.masks) {  // the count pass records hit masks, the fill replays them
        a.rec_mode = fill ? 2 : 1;
        a.rec_cap = rec.cap;
        a.rec_masks = rec.masks;
        a.rec_head = rec.head;
        a.rec_count = rec.count;
    }
    const char* name = fill ? "batch_radius_fill" : "batch_radius_count";
    if (fill) {
        constexpr int kWarps = radius_warps<true>();
        const unsigned int grid = grid_for(ngroups, kWarps);
        switch (kern) {
        case SFC_SPHERE: SFC_LAUNCH(name, s, (k_radius_group<SFC_SPHERE, true, false>), grid, kWarps * 32, 0, a); break;
        case SFC_CIRCLE: SFC_LAUNCH(name, s, (k_radius_group<SFC_CIRCLE, true, false>), grid, kWarps * 32, 0, a); break;
        case SFC_CUBE: SFC_LAUNCH(name, s, (k_radius_group<SFC_CUBE, true, false>), grid, kWarps * 32, 0, a); break;
        default: SFC_LAUNCH(name, s, (k_radius_group<SFC_SQUARE, true, false>), grid, kWarps * 32, 0, a); break;
        }
    } else {
        constexpr int kWarps = radius_warps<false>();
        const unsigned int grid = grid_for(ngroups, kWarps);
        switch (kern) {
        case SFC_SPHERE: SFC_LAUNCH(name, s, (k_radius_group<SFC_SPHERE, false, false>), grid, kWarps * 32, 0, a); break;
        case SFC_CIRCLE: SFC_LAUNCH(name, s, (k_radius_group<SFC_CIRCLE, false, false>), grid, kWarps * 32, 0, a); break;
        case SFC_CUBE: SFC_LAUNCH(name, s, (k_radius_group<SFC_CUBE, false, false>), grid, kWarps * 32, 0, a); break;
        default: SFC_LAUNCH(name, s, (k_radius_group<SFC_SQUARE, false, false>), grid, kWarps * 32, 0, a); break;
        }
    }
    return SFC_OK;
}

void release_records(Octree* t, cudaStream_t s) {
    dev_free(t->records.masks, s);
    dev_free(t->records.head, s);
    dev_free(t->records.count, s);
    t->records = RadiusRecords();
}

}  // namespace sfc

using sfc::Octree;

extern "C" {

sfc_status radius_count(sfc_octree h, const float* queries_xyz, int64_t n_queries, float r, sfc_kernel kern,
                        void* cuda_stream, int64_t* row_ptr, int64_t* nnz) {
    int64_t rows = 0;
    SFC_TRY(sfc::check_radius_args(h, queries_xyz, n_queries, r, kern, &rows));
    if (!row_ptr || !nnz) return SFC_ERR_INVALID;
    if (!sfc::is_device_ptr(row_ptr)) return SFC_ERR_NOT_DEVICE_PTR;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    sfc::Scratch scratch(s);
    const float4* q4 = nullptr;
    unsigned int* bad = nullptr;
    SFC_TRY(sfc::prepare(&h->tree, queries_xyz, rows, s, scratch, &q4, &bad));
    return sfc::count_impl(&h->tree, q4, rows, r, kern, s, scratch, row_ptr, bad, nnz, queries_xyz == nullptr);
}

sfc_status radius_fill(sfc_octree h, const float* queries_xyz, int64_t n_queries, float r, sfc_kernel kern,
                       void* cuda_stream, const int64_t* row_ptr, int32_t* cols) {
    int64_t rows = 0;
    SFC_TRY(sfc::check_radius_args(h, queries_xyz, n_queries, r, kern, &rows));
    if (!row_ptr || !cols) return SFC_ERR_INVALID;
    if (!sfc::is_device_ptr(row_ptr) || !sfc::is_device_ptr(cols)) return SFC_ERR_NOT_DEVICE_PTR;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    sfc::Scratch scratch(s);
    const float4* q4 = nullptr;
    unsigned int* bad = nullptr;
    SFC_TRY(sfc::prepare(&h->tree, queries_xyz, rows, s, scratch, &q4, &bad));
    return sfc::fill_impl(&h->tree, q4, rows, r, kern, s, row_ptr, cols, queries_xyz == nullptr);
}

sfc_status radius_search(sfc_octree h, const float* queries_xyz, int64_t n_queries, float r, sfc_kernel kern,
                         void* cuda_stream, sfc_csr* out) {
    if (!out) return SFC_ERR_INVALID;
    out->n_rows = 0;
    out->nnz = 0;
    out->row_ptr = nullptr;
    out->cols = nullptr;
    int64_t rows = 0;
    SFC_TRY(sfc::check_radius_args(h, queries_xyz, n_queries, r, kern, &rows));
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    sfc_status st;
    int64_t nnz = 0;
    int64_t* row_ptr = nullptr;
    int32_t* cols = nullptr;
    {
        sfc::Scratch scratch(s);
        const float4* q4 = nullptr;
        unsigned int* bad = nullptr;
        st = sfc::prepare(&h->tree, queries_xyz, rows, s, scratch, &q4, &bad);
        if (st == SFC_OK) st = sfc::dev_alloc(&row_ptr, rows + 1, s);
        const bool all = queries_xyz == nullptr;
        if (st == SFC_OK) st = sfc::count_impl(&h->tree, q4, rows, r, kern, s, scratch, row_ptr, bad, &nnz, all);
        if (st == SFC_OK) st = sfc::dev_alloc(&cols, nnz, s);
        if (st == SFC_OK) st = sfc::fill_impl(&h->tree, q4, rows, r, kern, s, row_ptr, cols, all);
        if (st == SFC_OK) st = sfc::check_guard(&h->tree, s);
    }
    if (st != SFC_OK) {
        sfc::dev_free(row_ptr, s);
        sfc::dev_free(cols, s);
        return st;
    }
    out->n_rows = rows;
    out->nnz = nnz;
    out->row_ptr = row_ptr;
    out->cols = cols;
    return SFC_OK;
}

sfc_status radius_search_ranges(sfc_octree h, const float* queries_xyz, int64_t n_queries, float r, sfc_kernel kern,
                                void* cuda_stream, sfc_ranges* out) {
    if (!out) return SFC_ERR_INVALID;
    out->n_rows = 0;
    out->n_runs = 0;
    out->run_ptr = nullptr;
    out->runs = nullptr;
    int64_t rows = 0;
    SFC_TRY(sfc::check_radius_args(h, queries_xyz, n_queries, r, kern, &rows));
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    sfc_status st;
    int64_t n_runs = 0;
    int64_t* run_ptr = nullptr;
    int2* runs = nullptr;
    {
        sfc::Scratch scratch(s);
        const float4* q4 = nullptr;
        unsigned int* bad = nullptr;
        st = sfc::prepare(&h->tree, queries_xyz, rows, s, scratch, &q4, &bad);
        if (st == SFC_OK) st = sfc::dev_alloc(&run_ptr, rows + 1, s);
        const bool all = queries_xyz == nullptr;
        if (st == SFC_OK)
            st = sfc::count_impl(&h->tree, q4, rows, r, kern, s, scratch, run_ptr, bad, &n_runs, all, true);
        if (st == SFC_OK) st = sfc::dev_alloc(&runs, n_runs, s);
        if (st == SFC_OK) st = sfc::fill_impl(&h->tree, q4, rows, r, kern, s, run_ptr, nullptr, all, runs);
        if (st == SFC_OK) st = sfc::check_guard(&h->tree, s);
    }
    if (st != SFC_OK) {
        sfc::dev_free(run_ptr, s);
        sfc::dev_free(runs, s);
        return st;
    }
    out->n_rows = rows;
    out->n_runs = n_runs;
    out->run_ptr = run_ptr;
    out->runs = reinterpret_cast<int32_t*>(runs);
    return SFC_OK;
}

sfc_status sfc_ranges_free(sfc_ranges* ranges, void* cuda_stream) {
    if (!ranges) return SFC_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    sfc::dev_free(ranges->run_ptr, s);
    sfc::dev_free(ranges->runs, s);
    ranges->run_ptr = nullptr;
    ranges->runs = nullptr;
    ranges->n_rows = 0;
    ranges->n_runs = 0;
    return SFC_OK;
}

sfc_status sfc_csr_free(sfc_csr* csr, void* cuda_stream) {
    if (!csr) return SFC_ERR_INVALID;
    cudaStream_t s = static_cast<cudaStream_t>(cuda_stream);
    sfc::dev_free(csr->row_ptr, s);
    sfc::dev_free(csr->cols, s);
    csr->row_ptr = nullptr;
    csr->cols = nullptr;
    csr->n_rows = 0;
    csr->nnz = 0;
    return SFC_OK;
}

}  // extern "C"
