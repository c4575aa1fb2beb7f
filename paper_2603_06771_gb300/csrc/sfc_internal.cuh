// sfc_internal.cuh - types and helpers shared by the translation units of libsfcoct.
//
// Layout of a built octree in device memory (one allocation per array):
//   pts    float4[n]   sorted cloud: x, y, z and the original index (uint32 bits) in w.
//                      For SFC_ENC_NONE: the cloud in input order (w = input index).
//   perm   uint32[n]   sorted position -> original index.
//   keys   uint64[n]   sorted 63-bit codes.
//   nodes  NodeBox[m]  m = 1 + 8 * n_internal: node 0 is the root; the eight children
//                      of the internal node of pre-order rank g are nodes 1 + 8g .. 8 + 8g.
//                      lo.xyz / hi.xyz = tight box of the node's points, lo.w / hi.w =
//                      internalRanges [start, end) as uint32 bits.
//   child  int32[m]    first child of an internal node, -1 for a leaf.
//   node_key uint64[m], node_level uint8[m]: the node's cell (first code, level).
//   leaves uint64[nL + 1], leaf_counts uint32[nL]: the leaves array of section 5.1.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "sfcoct.h"

namespace sfc {

constexpr int kLevels = 21;                        // L of section 4
constexpr uint64_t kWholeRange = 1ull << 63;       // 8^21 codes
constexpr uint32_t kCellMax = (1u << kLevels) - 1;
constexpr int kMaxK = 64;                          // largest k of the kNN kernels
constexpr int kStackDepth = 160;                   // >= 7 * 21 + 8 pending nodes of a depth-first walk
constexpr unsigned int kGuardTripped = 4u;          // BuildScalars::bad bit set by a failed guard
constexpr unsigned int kWaitTimedOut = 8u;          // the same word: a bounded device-side wait gave up

struct __align__(16) NodeBox {
    float4 lo;  // w: start (uint32 bits)
    float4 hi;  // w: end (uint32 bits)
};

// Device-resident scalars of one build.
struct BuildScalars {
    unsigned int mn[3];  // order-preserving uint images of the per-axis minima
    unsigned int mx[3];
    unsigned int bad;    // bit 0: a coordinate is not finite, bit 1: the extent is not finite,
                         // bit 2: a consistency guard of a search kernel tripped
    float lo[3];
    float scale;
    float ext;
};

// Hit masks recorded by an all-points count pass for the fill pass that follows with the
// same radius and kernel (see sfc_radius.cu).  Owned by the handle, released by the
// fill pass that consumes it or by octree_free.
struct RadiusRecords {
    uint32_t* masks = nullptr;   // [groups][cap][32] per-lane hit masks
    uint2* head = nullptr;       // [groups][cap] record headers
    uint32_t* count = nullptr;   // [groups] records of the group, kRecordsOverflow if they did not fit
    int64_t groups = 0;
    int cap = 0;
    float r = 0.f;
    int kern = -1;
    bool valid = false;
};
constexpr uint32_t kRecordsOverflow = 0xffffffffu;
constexpr int kRecordCap = 32;        // record slots per warp group of a batch cloud by default
                                      // (a group with more leaf chunks walks again in the fill)
constexpr int kRecordCapMax = 128;    // the most record slots a batch cloud may ask for
constexpr int kRecordCapSingle = 64;  // record slots per warp group of a single-cloud search

// The records of one batched radius launch: [groups][cap] slots (null: no records)
struct BatchRecords {
    uint32_t* masks = nullptr;
    uint2* head = nullptr;
    uint32_t* count = nullptr;
    int cap = 0;  // slots per group
};

struct Octree {
    int device = 0;
    int64_t n = 0;
    int enc = 0;
    int leaf_cap = 32;
    int prune = 1;
    float4* pts = nullptr;
    uint32_t* perm = nullptr;
    uint64_t* keys = nullptr;
    NodeBox* nodes = nullptr;
    int32_t* child = nullptr;
    uint64_t* node_key = nullptr;
    uint8_t* node_level = nullptr;
    uint64_t* leaves = nullptr;
    uint32_t* leaf_counts = nullptr;
    BuildScalars* scal = nullptr;
    int64_t n_internal = 0, n_nodes = 0, n_leaves = 0;
    float lo[3] = {0, 0, 0};
    float scale = 1;
    RadiusRecords records;
};

void release_records(Octree* t, cudaStream_t s);

// One cloud of a batched search (see sfc_batch.cu): the group kernels take a table of
// these; without one they search the single cloud of a handle (root node 0, all rows).
struct SearchSeg {
    int64_t group0;  // first warp group (global index) of this cloud
    int64_t q0, nq;  // its centres: sorted positions [q0, q0 + nq) of the batch
    int64_t row0;    // radius: its first CSR row; kNN: its first output entry
    int32_t root;    // its root node
    int32_t k;       // kNN: neighbours
    float r, r2;     // radius and fl(r * r)
    int32_t window;  // kNN: curve neighbours per side for the seeding window (0: none)
    int32_t group_size;  // centres per warp group (8, 16 or 32; lanes beyond stay idle)
};

// Index of the cloud that owns warp group `group` (the last entry with group0 <= group).
__device__ __forceinline__ int find_search_seg(const SearchSeg* segs, int n, int64_t group) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (segs[mid].group0 <= group) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// ---------------------------------------------------------------------------------
// runtime (sfc_runtime.cu)
void record_cuda_error(cudaError_t e, const char* where);
// kernels launched by replaying a recorded graph (added to the launch counter)
void count_launches(uint64_t n);
// Called around every kernel launch: counts launches, records profiling events.
void launch_begin(const char* name, cudaStream_t s);
sfc_status launch_end(const char* name, cudaStream_t s);
bool is_device_ptr(const void* p);
sfc_status ensure_pool(int device);

// Work counters of the search kernels (sfc_stats_enable): the counters' device array while
// counting is on, else nullptr.  The searches launch an instrumented copy of their kernel
// when it is not null.
unsigned long long* stats_counters();

// Every device allocation of the library: through the caller's allocator when one is set
// (sfc_set_allocator), else the stream-ordered allocator; `native` always takes the
// latter (allocations recorded into a CUDA graph).  A free must use the same `native`.
cudaError_t raw_alloc(void** p, size_t bytes, cudaStream_t s, bool native = false);
void raw_free(void* p, cudaStream_t s, bool native = false);

// Scratch allocations, released (in stream order) when the guard dies.
class Scratch {
  public:
    explicit Scratch(cudaStream_t s, bool native = false) : s_(s), native_(native) {}
    ~Scratch();
    template <typename T>
    sfc_status alloc(T** p, size_t count) {
        void* v = nullptr;
        cudaError_t e = raw_alloc(&v, (count ? count : 1) * sizeof(T), s_, native_);
        if (e != cudaSuccess) {
            record_cuda_error(e, "device allocation");
            *p = nullptr;
            return e == cudaErrorMemoryAllocation ? SFC_ERR_OOM : SFC_ERR_CUDA;
        }
        ptrs_.push_back(v);
        *p = static_cast<T*>(v);
        return SFC_OK;
    }
    // The same without reporting a failure (for optional buffers).
    template <typename T>
    bool try_alloc(T** p, size_t count) {
        void* v = nullptr;
        if (raw_alloc(&v, (count ? count : 1) * sizeof(T), s_, native_) != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return false;
        }
        ptrs_.push_back(v);
        *p = static_cast<T*>(v);
        return true;
    }
    // Hand an allocation over to the caller (it is no longer freed by the guard).
    void release(const void* p);
    cudaStream_t stream() const { return s_; }

  private:
    cudaStream_t s_;
    bool native_;
    std::vector<void*> ptrs_;
};

template <typename T>
sfc_status dev_alloc(T** p, size_t count, cudaStream_t s) {
    void* v = nullptr;
    cudaError_t e = raw_alloc(&v, (count ? count : 1) * sizeof(T), s);
    if (e != cudaSuccess) {
        record_cuda_error(e, "device allocation");
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? SFC_ERR_OOM : SFC_ERR_CUDA;
    }
    *p = static_cast<T*>(v);
    return SFC_OK;
}
void dev_free(void* p, cudaStream_t s);

// Exclusive scan: out[0] = 0, out[i + 1] = out[i] + in[i], out has n + 1 entries (one
// kernel, tiles chained by a bounded decoupled look-back).  fault (device, may be null)
// gets kWaitTimedOut if a wait gave up (the offsets are then wrong).
sfc_status scan_u32_to_i64(const uint32_t* in, int64_t* out, int64_t n, cudaStream_t s, Scratch& scratch,
                           unsigned int* fault = nullptr);
// The same scan with its look-back words in a caller buffer of scan_tile_count(n) entries.
int64_t scan_tile_count(int64_t n);
sfc_status scan_u32_to_i64_presized(const uint32_t* in, int64_t* out, int64_t n, int64_t* tile_sums, cudaStream_t s,
                                    unsigned int* fault = nullptr);
// The same scan over the new internal cells of every sorted position of one cloud
// (new_internal_cells with ncap), computed from the sorted codes as they are read.
sfc_status scan_tree_counts(const uint64_t* keys, int64_t n, int64_t ncap, int64_t* first, cudaStream_t s,
                            Scratch& scratch, unsigned int* fault = nullptr);
// All-points count pass of the radius search into caller buffers (counts: one entry per
// point, tile_sums: scan_tile_count(n) entries); reads nnz back (one synchronisation).
sfc_status radius_count_presized(const Octree* t, float r, int kern, cudaStream_t s, uint32_t* counts,
                                 int64_t* tile_sums, int64_t* row_ptr, int64_t* nnz);

// Stable LSD radix sort of (key, value) pairs by the 64 bits of key; the result ends in
// keys / vals, keys_alt / vals_alt are work buffers of the same size.  n < 2^32.  fault
// (device, may be null) gets kWaitTimedOut if a tile's bounded wait for the counts of
// the tiles before it gave up (the order is then wrong); the sort never synchronises.
sfc_status radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, int64_t n,
                            cudaStream_t s, Scratch& scratch, unsigned int* fault);

// Centres of a search in processing order: float4 (x, y, z, output row bits).  For
// queries == NULL the tree points themselves; otherwise caller centres, sorted by their
// code under the tree's transform for the sorted encodings.  *bad (device) gets bit 0
// set for a non-finite centre.
sfc_status prepare_queries(const Octree* h, const float* queries, int64_t nq, cudaStream_t s, Scratch& scratch,
                           const float4** q4, unsigned int* bad);

#define SFC_TRY(expr)                      \
    do {                                   \
        sfc_status st_ = (expr);           \
        if (st_ != SFC_OK) return st_;     \
    } while (0)

#define SFC_CUDA(expr)                                        \
    do {                                                      \
        cudaError_t e_ = (expr);                              \
        if (e_ != cudaSuccess) {                              \
            ::sfc::record_cuda_error(e_, #expr);              \
            return SFC_ERR_CUDA;                              \
        }                                                     \
    } while (0)

#define SFC_LAUNCH(name, stream, kernel, grid, block, smem, ...)   \
    do {                                                           \
        ::sfc::launch_begin(name, stream);                         \
        kernel<<<(grid), (block), (smem), (stream)>>>(__VA_ARGS__); \
        SFC_TRY(::sfc::launch_end(name, stream));                  \
    } while (0)

// The status of the guard bits of a BuildScalars::bad (or batch error) word read back.
inline sfc_status guard_status(unsigned int bad) {
    if (bad & kGuardTripped) return SFC_ERR_INTERNAL;
    if (bad & kWaitTimedOut) return SFC_ERR_TIMEOUT;
    return SFC_OK;
}

inline bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

inline unsigned int grid_for(int64_t n, int threads, int64_t cap = 1 << 30) {
    int64_t g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    if (g > cap) g = cap;
    return static_cast<unsigned int>(g);
}

// ---------------------------------------------------------------------------------
// device helpers

// Number of leading octal digits (levels) two 63-bit codes share, 0..21.
__device__ __forceinline__ int common_levels(uint64_t a, uint64_t b) {
    uint64_t x = a ^ b;
    if (x == 0) return kLevels;
    return (__clzll(static_cast<long long>(x)) - 1) / 3;
}

// Internal cells of the linear octree first met at sorted position i (section 5.1): a
// cell is split when it holds more than ncap points, i.e. when the codes at i and i + ncap
// share it; the new ones at i are those below the deepest level i shares with i - 1 (all
// of them from the root at the start of the range), down to the deepest level i shares
// with i + ncap (never level 21).  lo: the first position of the range, end: one past its last.
__device__ __forceinline__ uint32_t cells_from(int first_new, uint64_t code, uint64_t code_ncap_on) {
    int deepest = common_levels(code, code_ncap_on);
    if (deepest > kLevels - 1) deepest = kLevels - 1;  // a level-21 cell is never split
    return deepest >= first_new ? static_cast<uint32_t>(deepest - first_new + 1) : 0u;
}
__device__ __forceinline__ uint32_t new_internal_cells(const uint64_t* keys, int64_t i, int64_t lo, int64_t end,
                                                       int64_t ncap) {
    if (i + ncap >= end) return 0u;
    const int first_new = i == lo ? 0 : common_levels(keys[i - 1], keys[i]) + 1;
    return cells_from(first_new, keys[i], keys[i + ncap]);
}

// Mask of the code bits below level l (the 3 * (21 - l) low bits).
__device__ __forceinline__ uint64_t below_level_mask(int l) {
    return (1ull << (3 * (kLevels - l))) - 1ull;
}

__device__ __forceinline__ int64_t lower_bound_u64(const uint64_t* __restrict__ a, int64_t n, uint64_t key) {
    int64_t lo = 0, hi = n;
    while (lo < hi) {
        int64_t mid = (lo + hi) >> 1;
        if (a[mid] < key) lo = mid + 1;
        else hi = mid;
    }
    return lo;
}

// Order-preserving map float -> uint32 (for atomic min / max of floats).
__device__ __forceinline__ unsigned int float_to_ordered(float f) {
    unsigned int u = __float_as_uint(f);
    return (u & 0x80000000u) ? ~u : (u | 0x80000000u);
}
__device__ __forceinline__ float ordered_to_float(unsigned int u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

__device__ __forceinline__ unsigned int lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned int lanes_below() {
    unsigned int m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

// Discretisation of one coordinate (section 4, steps 1-2): floor((p - lo) * s) in
// binary32, each operation rounded to nearest, clamped into [0, 2^21 - 1].
__device__ __forceinline__ uint32_t cell_of(float p, float lo, float s) {
    float f = floorf(__fmul_rn(__fsub_rn(p, lo), s));
    if (!(f > 0.0f)) return 0u;
    if (f >= static_cast<float>(kCellMax)) return kCellMax;
    return static_cast<uint32_t>(f);
}

// Kernel tests of section 3.2 on d = p - c (each component already rounded), strict "<".
// No fused multiply-add: every product and sum is rounded on its own.
template <int KERN>
__device__ __forceinline__ bool kernel_holds(float dx, float dy, float dz, float r, float r2) {
    if (KERN == SFC_SPHERE) {
        float s = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
        return __fadd_rn(s, __fmul_rn(dz, dz)) < r2;
    } else if (KERN == SFC_CIRCLE) {
        return __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy)) < r2;
    } else if (KERN == SFC_CUBE) {
        return fmaxf(fmaxf(fabsf(dx), fabsf(dy)), fabsf(dz)) < r;
    } else {
        return fmaxf(fabsf(dx), fabsf(dy)) < r;
    }
}

// Work counters of one search launch, in the order of sfc_search_stats (sfcoct.h).  Each
// lane accumulates its own; warp-uniform events are counted by lane 0 alone.
enum StatIndex {
    kStWalks = 0,
    kStExpansions,
    kStBoxTests,
    kStLeaves,
    kStPointTests,
    kStNeeded,
    kStPassed,
    kStWhole,
    kStInserts,
    kStCount
};
struct StatAcc {
    unsigned long long v[kStCount];
    __device__ __forceinline__ void zero() {
#pragma unroll
        for (int i = 0; i < kStCount; ++i) v[i] = 0ull;
    }
    // The lanes of `lanes` (lane 0 and a prefix of the warp) call this once: their sums go
    // to the device counters.
    __device__ __forceinline__ void flush(unsigned long long* out, unsigned int lanes = 0xffffffffu) const {
        const unsigned int lane = threadIdx.x & 31u;
#pragma unroll
        for (int i = 0; i < kStCount; ++i) {
            unsigned long long x = v[i];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                const unsigned long long y = __shfl_down_sync(lanes, x, o);
                if (lane + o < 32u && ((lanes >> (lane + o)) & 1u)) x += y;
            }
            if (lane == 0 && x) atomicAdd(out + i, x);
        }
    }
};

// Squared Euclidean distance used by kNN: (dx*dx + dy*dy) + dz*dz, rounded per operation.
__device__ __forceinline__ float sq_dist(float dx, float dy, float dz) {
    float s = __fadd_rn(__fmul_rn(dx, dx), __fmul_rn(dy, dy));
    return __fadd_rn(s, __fmul_rn(dz, dz));
}

// ---------------------------------------------------------------------------------
// section 4.1: Morton code, bits of x, y, z interleaved x-high per level.  Each 21-bit
// coordinate is spread to every third bit by shift-and-mask steps.
__device__ __forceinline__ uint64_t spread_every_third(uint32_t v) {
    uint64_t x = v & kCellMax;
    x = (x | (x << 32)) & 0x001f00000000ffffull;
    x = (x | (x << 16)) & 0x001f0000ff0000ffull;
    x = (x | (x << 8)) & 0x100f00f00f00f00full;
    x = (x | (x << 4)) & 0x10c30c30c30c30c3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ uint64_t morton_code(uint32_t x, uint32_t y, uint32_t z) {
    return (spread_every_third(x) << 2) | (spread_every_third(y) << 1) | spread_every_third(z);
}

// section 4.2: Hilbert code as a finite-state machine read level by level from the top.
// The state is the transform that the levels above impose on the remaining bits (a
// permutation of the three axes with a flip per axis, 48 possibilities) plus the running
// parity of the code's last bit column (2): 96 states x 8 inputs.  At a level the input
// bits are transformed by the state, the output digit is the Gray code of the transformed
// bits complemented when the parity is odd, and the transform of the lower levels then
// applies, for axes 0, 1, 2 in turn, "complement axis 0" when that axis's transformed bit
// is 1 and "exchange axis 0 with that axis" when it is 0 (the curve of J. Skilling,
// "Programming the Hilbert curve", 2004).  Every block fills the table in shared memory.
constexpr int kHilbertStates = 96;
constexpr int kHilbertTable = kHilbertStates * 8;

__device__ __forceinline__ void axes_of_perm(int p, int s[3]) {
    // p = 2 * first + (1 if the other two are descending)
    s[0] = p >> 1;
    const int a = s[0] == 0 ? 1 : 0;
    const int b = s[0] == 2 ? 1 : 2;
    if (p & 1) { s[1] = b; s[2] = a; }
    else { s[1] = a; s[2] = b; }
}

__device__ __forceinline__ int perm_of_axes(const int s[3]) { return 2 * s[0] + (s[1] > s[2] ? 1 : 0); }

__device__ inline void fill_hilbert_table(uint16_t* table) {
    for (int t = threadIdx.x; t < kHilbertTable; t += blockDim.x) {
        const int input = t & 7;
        const int state = t >> 3;
        const int parity = state & 1;
        const int flips = (state >> 1) & 7;
        int src[3], flip[3], v[3];
        axes_of_perm(state >> 4, src);
        for (int i = 0; i < 3; ++i) flip[i] = (flips >> (2 - i)) & 1;
        const int bits[3] = {(input >> 2) & 1, (input >> 1) & 1, input & 1};
        for (int i = 0; i < 3; ++i) v[i] = bits[src[i]] ^ flip[i];
        const int g0 = v[0], g1 = v[0] ^ v[1], g2 = v[0] ^ v[1] ^ v[2];
        const int digit = ((g0 ^ parity) << 2) | ((g1 ^ parity) << 1) | (g2 ^ parity);
        const int next_parity = parity ^ g2;
        for (int i = 0; i < 3; ++i) {
            if (v[i]) {
                flip[0] ^= 1;
            } else {
                int ts = src[0]; src[0] = src[i]; src[i] = ts;
                int tf = flip[0]; flip[0] = flip[i]; flip[i] = tf;
            }
        }
        const int next = ((perm_of_axes(src) * 8 + ((flip[0] << 2) | (flip[1] << 1) | flip[2])) << 1) | next_parity;
        table[t] = static_cast<uint16_t>(digit | (next << 3));
    }
}

// Two levels per lookup: entry (state, 3 input bits of a level then 3 of the level below)
// = the two levels' 6 code bits | the state after both << 6, composed from the one-level
// table.  Both tables live in shared memory, filled by every block.
constexpr int kHilbertTable2 = kHilbertStates * 64;
struct HilbertTables {
    uint16_t one[kHilbertTable];
    uint16_t two[kHilbertTable2];
};

// Called by every thread of the block (it synchronises the block).
__device__ inline void fill_hilbert_tables(HilbertTables& t) {
    fill_hilbert_table(t.one);
    __syncthreads();
    for (int i = threadIdx.x; i < kHilbertTable2; i += blockDim.x) {
        const uint32_t e1 = t.one[(i >> 6) * 8 + ((i >> 3) & 7)];
        const uint32_t e2 = t.one[(e1 >> 3) * 8 + (i & 7)];
        t.two[i] = static_cast<uint16_t>(((e1 & 7u) << 3) | (e2 & 7u) | ((e2 >> 3) << 6));
    }
    __syncthreads();
}

__device__ __forceinline__ uint32_t level_bits(uint32_t x, uint32_t y, uint32_t z, int l) {
    return (((x >> l) & 1u) << 2) | (((y >> l) & 1u) << 1) | ((z >> l) & 1u);
}

// The code of a cell: the top level alone, then the other 20 two at a time.
__device__ __forceinline__ uint64_t hilbert_code(uint32_t x, uint32_t y, uint32_t z, const HilbertTables& t) {
    static_assert(kLevels % 2 == 1, "one level alone, then pairs");
    const uint32_t e0 = t.one[level_bits(x, y, z, kLevels - 1)];
    uint64_t code = e0 & 7u;
    uint32_t state = e0 >> 3;
#pragma unroll
    for (int l = kLevels - 2; l >= 1; l -= 2) {
        const uint32_t e = t.two[state * 64 + ((level_bits(x, y, z, l) << 3) | level_bits(x, y, z, l - 1))];
        code = (code << 6) | (e & 63u);
        state = e >> 6;
    }
    return code;
}


// One cloud of a batch (see sfc_batch.cu).
struct BatchSeg {
    int64_t p0, n;       // its points: input and sorted positions [p0, p0 + n)
    int64_t g0, n_int;   // its internal nodes: global pre-order ranks [g0, g0 + n_int)
    int64_t node0;       // its node-table slice: [node0, node0 + 1 + 8 n_int)
    int64_t leaf0;       // its leaves slice: [leaf0, leaf0 + 7 n_int + 2)
    int32_t ncap;
    int32_t pad;
    float lo[3];
    float scale;
    unsigned int mn[3], mx[3];
    unsigned int bad;
};
// curve neighbours per side that seed an all-points kNN list (knn, batches)
inline int knn_default_window(int k) { return k < 8 ? 8 : k; }
constexpr int kBatchMax = 1024;  // clouds per batch (segment starts are staged in shared memory)

// codes of a batch, each cloud with its own box and scale (sfc_build.cu)
sfc_status batch_encode(const float* xyz, int64_t n, int enc, const BatchSeg* segs, int nsegs, uint64_t* keys,
                        uint32_t* idx, cudaStream_t s);
// LSD radix sort on bits [begin_bit, end_bit) of the keys; the result ends in keys / vals
sfc_status radix_sort_pairs_bits(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, int64_t n,
                                 int begin_bit, int end_bit, cudaStream_t s, Scratch& scratch, unsigned int* fault);

}  // namespace sfc

// the opaque handle of the C ABI
struct sfc_octree_s {
    sfc::Octree tree;
};
