// sfc_runtime.cu - error reporting, launch accounting and profiling, stream-ordered
// memory, device-wide scans and the LSD radix sort of (code, index) pairs.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "sfc_internal.cuh"

namespace sfc {

// ---------------------------------------------------------------------------------
// errors
static thread_local char t_last_error[256] = "";

void record_cuda_error(cudaError_t e, const char* where) {
    snprintf(t_last_error, sizeof t_last_error, "%s: %s (%s)", where, cudaGetErrorString(e), cudaGetErrorName(e));
}

// ---------------------------------------------------------------------------------
// launch accounting and per-kernel event timing
static std::atomic<uint64_t> g_launches{0};
static std::atomic<bool> g_prof_on{false};
static std::mutex g_prof_mu;
static std::atomic<bool> g_stats_on{false};
static std::mutex g_stats_mu;
static unsigned long long* g_stats = nullptr;  // kStCount counters, kept for the process
static int g_stats_device = -1;                // the device that holds them

// counting happens on the counters' device only (a search on another device is not counted)
unsigned long long* stats_counters() {
    if (!g_stats_on.load(std::memory_order_relaxed)) return nullptr;
    int d = -1;
    if (cudaGetDevice(&d) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return d == g_stats_device ? g_stats : nullptr;
}

struct ProfRecord {
    std::string name;
    cudaEvent_t start, stop;
};
static std::vector<ProfRecord> g_prof;
static thread_local cudaEvent_t t_pending_start = nullptr;

void count_launches(uint64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void launch_begin(const char* name, cudaStream_t s) {
    (void)name;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (g_prof_on.load(std::memory_order_relaxed) && cudaStreamIsCapturing(s, &cap) == cudaSuccess &&
        cap == cudaStreamCaptureStatusNone) {  // launches recorded into a graph are not timed
        cudaEvent_t e;
        if (cudaEventCreate(&e) == cudaSuccess) {
            cudaEventRecord(e, s);
            t_pending_start = e;
        }
    }
}

sfc_status launch_end(const char* name, cudaStream_t s) {
    g_launches.fetch_add(1, std::memory_order_relaxed);
    cudaError_t e = cudaGetLastError();
    if (t_pending_start) {
        cudaEvent_t stop;
        if (cudaEventCreate(&stop) == cudaSuccess) {
            cudaEventRecord(stop, s);
            std::lock_guard<std::mutex> g(g_prof_mu);
            g_prof.push_back({name, t_pending_start, stop});
        } else {
            cudaEventDestroy(t_pending_start);
        }
        t_pending_start = nullptr;
    }
    if (e != cudaSuccess) {
        record_cuda_error(e, name);
        return SFC_ERR_CUDA;
    }
    return SFC_OK;
}

bool is_device_ptr(const void* p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Keep freed stream-ordered memory cached in the device's default pool so that repeated
// builds and searches do not return memory to the driver between calls.
sfc_status ensure_pool(int device) {
    static std::mutex mu;
    static std::vector<int> done;
    std::lock_guard<std::mutex> g(mu);
    for (int d : done)
        if (d == device) return SFC_OK;
    cudaMemPool_t pool;
    SFC_CUDA(cudaDeviceGetDefaultMemPool(&pool, device));
    uint64_t threshold = UINT64_MAX;
    SFC_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &threshold));
    done.push_back(device);
    return SFC_OK;
}

// the caller's allocator, and how many library allocations are alive (it may change only
// while none is)
static std::mutex g_alloc_mu;
static sfc_alloc_fn g_alloc = nullptr;
static sfc_free_fn g_free = nullptr;
static void* g_alloc_ctx = nullptr;
static std::atomic<int64_t> g_live{0};

cudaError_t raw_alloc(void** p, size_t bytes, cudaStream_t s, bool native) {
    sfc_alloc_fn fn = nullptr;
    void* ctx = nullptr;
    if (!native) {
        std::lock_guard<std::mutex> g(g_alloc_mu);
        fn = g_alloc;
        ctx = g_alloc_ctx;
    }
    cudaError_t e = cudaSuccess;
    if (fn) {
        *p = fn(bytes, ctx, s);
        if (!*p) e = cudaErrorMemoryAllocation;
    } else {
        e = cudaMallocAsync(p, bytes, s);
    }
    if (e == cudaSuccess) g_live.fetch_add(1);
    return e;
}

void raw_free(void* p, cudaStream_t s, bool native) {
    if (!p) return;
    sfc_free_fn fn = nullptr;
    void* ctx = nullptr;
    if (!native) {
        std::lock_guard<std::mutex> g(g_alloc_mu);
        fn = g_free;
        ctx = g_alloc_ctx;
    }
    if (fn) fn(p, ctx, s);
    else cudaFreeAsync(p, s);
    g_live.fetch_sub(1);
}

Scratch::~Scratch() {
    for (void* p : ptrs_) raw_free(p, s_, native_);
}

void Scratch::release(const void* p) {
    for (auto& q : ptrs_)
        if (q == p) q = nullptr;
    std::vector<void*> keep;
    for (void* q : ptrs_)
        if (q) keep.push_back(q);
    ptrs_.swap(keep);
}

void dev_free(void* p, cudaStream_t s) { raw_free(p, s); }

// ---------------------------------------------------------------------------------
// exclusive scans: tiles of kScanTile elements.
constexpr int kScanThreads = 512;
constexpr int kScanItems = 8;
constexpr int kScanTile = kScanThreads * kScanItems;

template <typename T>
__device__ __forceinline__ T warp_inclusive_scan(T x) {
    const unsigned int lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= static_cast<unsigned int>(o)) x += y;
    }
    return x;
}

// Exclusive scan of one value per thread over the block; *total receives the block sum.
template <typename T, int THREADS>
__device__ __forceinline__ T block_exclusive_scan(T v, T* total) {
    constexpr int kWarps = THREADS / 32;
    __shared__ T warp_sums[32];
    const unsigned int lane = lane_id();
    const unsigned int warp = threadIdx.x >> 5;
    T x = warp_inclusive_scan(v);
    if (lane == 31) warp_sums[warp] = x;
    __syncthreads();
    if (warp == 0) {
        T s = lane < static_cast<unsigned int>(kWarps) ? warp_sums[lane] : T(0);
        s = warp_inclusive_scan(s);
        if (lane < static_cast<unsigned int>(kWarps)) warp_sums[lane] = s;
    }
    __syncthreads();
    T prefix = warp == 0 ? T(0) : warp_sums[warp - 1];
    *total = warp_sums[kWarps - 1];
    __syncthreads();
    return prefix + x - v;
}

__device__ __forceinline__ void store_relaxed(uint64_t* p, uint64_t v) {
    asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t load_relaxed(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Exclusive scan of uint32 counts into int64 offsets (out[n] = the total) in one pass
// (vec: in and out are 16-byte aligned, whole runs of 8 by vector loads and stores):
// tiles of kScanTile elements take a ticket, scan themselves, publish their sum and learn
// the sum of the tiles before them by decoupled look-back (D. Merrill and M. Garland,
// "Single-pass Parallel Prefix Scan with Decoupled Look-back", 2016), one warp reading 32
// earlier tiles' words at a time.  A tile only waits on tiles that are already running;
// every wait is bounded all the same.
// Look-back words (tiles of them, then the ticket counter): bit 63 the inclusive prefix
// of this and all earlier tiles, bit 62 this tile's own sum, bits 61-0 the value.
constexpr uint64_t kScanPrefix = 1ull << 63;
constexpr uint64_t kScanSum = 1ull << 62;
constexpr uint64_t kScanValue = (1ull << 62) - 1;
constexpr int kScanSpinLimit = 1 << 22;

__device__ __forceinline__ int64_t warp_sum_i64(int64_t v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Inputs of the scan: an array of counts, or the new internal cells of sorted codes.
struct CountsInput {
    const uint32_t* in;
    int vec;  // in is 16-byte aligned
    __device__ __forceinline__ void load(int64_t base, int64_t n, uint32_t v[kScanItems]) const {
        if (vec && base + kScanItems <= n) {
#pragma unroll
            for (int j = 0; j < kScanItems / 4; ++j) {
                const uint4 a = __ldg(reinterpret_cast<const uint4*>(in + base) + j);
                v[4 * j] = a.x; v[4 * j + 1] = a.y; v[4 * j + 2] = a.z; v[4 * j + 3] = a.w;
            }
        } else {
#pragma unroll
            for (int j = 0; j < kScanItems; ++j) v[j] = base + j < n ? in[base + j] : 0u;
        }
    }
};

struct TreeCountsInput {
    const uint64_t* keys;
    int64_t ncap;
    __device__ __forceinline__ void load(int64_t base, int64_t n, uint32_t v[kScanItems]) const {
        if (base + kScanItems + ncap < n && base > 0) {  // every position has its neighbours: each code read once
            uint64_t k[kScanItems + 1], far[kScanItems];
#pragma unroll
            for (int j = 0; j <= kScanItems; ++j) k[j] = __ldg(keys + base - 1 + j);
#pragma unroll
            for (int j = 0; j < kScanItems; ++j) far[j] = __ldg(keys + base + ncap + j);
#pragma unroll
            for (int j = 0; j < kScanItems; ++j) v[j] = cells_from(common_levels(k[j], k[j + 1]) + 1, k[j + 1], far[j]);
        } else {
#pragma unroll
            for (int j = 0; j < kScanItems; ++j)
                v[j] = base + j < n ? new_internal_cells(keys, base + j, 0, n, ncap) : 0u;
        }
    }
};

template <class In>
__global__ void __launch_bounds__(kScanThreads) k_scan(In in, int64_t* __restrict__ out, int64_t n,
                                                       uint64_t* __restrict__ look, int64_t tiles, unsigned int* fault,
                                                       int vec) {
    __shared__ uint32_t s_tile;
    __shared__ int64_t s_before;
    if (threadIdx.x == 0) s_tile = atomicAdd(reinterpret_cast<unsigned int*>(look + tiles), 1u);
    __syncthreads();
    const int64_t tile = s_tile;
    const int64_t base = tile * kScanTile + static_cast<int64_t>(threadIdx.x) * kScanItems;
    static_assert(kScanItems % 4 == 0, "whole 16-byte loads and stores per thread");
    uint32_t v[kScanItems];
    in.load(base, n, v);
    const bool full = vec && base + kScanItems <= n;
    int64_t acc = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) acc += v[j];
    int64_t total;
    const int64_t ex = block_exclusive_scan<int64_t, kScanThreads>(acc, &total);
    if (threadIdx.x < 32) {
        const unsigned int lane = threadIdx.x;
        if (lane == 0) store_relaxed(look + tile, (tile == 0 ? kScanPrefix : kScanSum) | static_cast<uint64_t>(total));
        int64_t before = 0;
        int spins = 0;
        for (int64_t j = tile - 1; j >= 0;) {
            // lane l reads tile j - l (the nearest first); before the first tile there is a prefix of 0
            const uint64_t w = j - static_cast<int64_t>(lane) >= 0 ? load_relaxed(look + j - lane) : kScanPrefix;
            const unsigned int ready = __ballot_sync(0xffffffffu, (w >> 62) != 0);
            const unsigned int prefix = __ballot_sync(0xffffffffu, (w >> 63) != 0);
            const int first_prefix = prefix ? __ffs(prefix) - 1 : 32;
            const int first_missing = ~ready ? __ffs(~ready) - 1 : 32;
            const int use = min(first_missing, first_prefix + 1);  // words added this round
            before += warp_sum_i64(static_cast<int>(lane) < use ? static_cast<int64_t>(w & kScanValue) : 0);
            if (first_prefix < first_missing) break;  // reached an inclusive prefix
            j -= use;
            if (first_missing < 32) {
                if (++spins > kScanSpinLimit) {  // never expected: the tiles before are running
                    if (fault && lane == 0) atomicOr(fault, kWaitTimedOut);
                    break;
                }
                __nanosleep(32);
            }
        }
        if (lane == 0) {
            if (tile > 0) store_relaxed(look + tile, kScanPrefix | static_cast<uint64_t>(before + total));
            s_before = before;
        }
    }
    __syncthreads();
    int64_t run = s_before + ex;
    int64_t o[kScanItems];
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        o[j] = run;
        run += v[j];
    }
    if (full) {
        longlong2* d = reinterpret_cast<longlong2*>(out + base);
#pragma unroll
        for (int j = 0; j < kScanItems / 2; ++j) d[j] = make_longlong2(o[2 * j], o[2 * j + 1]);
    } else {
#pragma unroll
        for (int j = 0; j < kScanItems; ++j)
            if (base + j < n) out[base + j] = o[j];
    }
    // the element one past the end receives the grand total
    if (tile == tiles - 1 && threadIdx.x == 0) out[n] = s_before + total;
}

int64_t scan_tile_count(int64_t n) { return (n + kScanTile - 1) / kScanTile + 1; }

template <class In>
static sfc_status scan_impl(In in, int64_t* out, int64_t n, int64_t* look, cudaStream_t s, unsigned int* fault,
                            int vec) {
    if (n == 0) {
        SFC_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return SFC_OK;
    }
    const int64_t words = scan_tile_count(n);
    SFC_CUDA(cudaMemsetAsync(look, 0, sizeof(int64_t) * words, s));
    SFC_LAUNCH("scan", s, k_scan<In>, static_cast<unsigned int>(words - 1), kScanThreads, 0, in, out, n,
               reinterpret_cast<uint64_t*>(look), words - 1, fault, vec);
    return SFC_OK;
}

sfc_status scan_u32_to_i64_presized(const uint32_t* in, int64_t* out, int64_t n, int64_t* tile_sums, cudaStream_t s,
                                    unsigned int* fault) {
    const int vec = (aligned16(in) && aligned16(out)) ? 1 : 0;
    return scan_impl(CountsInput{in, vec}, out, n, tile_sums, s, fault, vec);
}

sfc_status scan_u32_to_i64(const uint32_t* in, int64_t* out, int64_t n, cudaStream_t s, Scratch& scratch,
                           unsigned int* fault) {
    int64_t* look = nullptr;
    if (n > 0) SFC_TRY(scratch.alloc(&look, static_cast<size_t>(scan_tile_count(n))));
    return scan_u32_to_i64_presized(in, out, n, look, s, fault);
}

sfc_status scan_tree_counts(const uint64_t* keys, int64_t n, int64_t ncap, int64_t* first, cudaStream_t s,
                            Scratch& scratch, unsigned int* fault) {
    int64_t* look = nullptr;
    if (n > 0) SFC_TRY(scratch.alloc(&look, static_cast<size_t>(scan_tile_count(n))));
    return scan_impl(TreeCountsInput{keys, ncap}, first, n, look, s, fault, aligned16(first) ? 1 : 0);
}

// ---------------------------------------------------------------------------------
// LSD radix sort of (code, uint32 index) pairs, 8-bit digits.
// One read of the keys counts the digits of every pass.  Each pass is then one kernel:
// a tile ranks its items stably (match-any within a warp, warps in input order), publishes
// its per-digit counts and learns the counts of all the tiles before it by decoupled
// look-back (D. Merrill and M. Garland, "Single-pass Parallel Prefix Scan with Decoupled
// Look-back", NVIDIA technical report, 2016), then writes its items out in runs that are
// contiguous per digit.  A tile's place in the order comes from a ticket taken when it
// starts, so a tile only waits on tiles that are already running; every wait is bounded
// all the same.  A pass whose digit is the same in every key is skipped, decided on the
// device, so the sort never synchronises.
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 12;
constexpr int kSortTile = kSortThreads * kSortItems;
constexpr int kMaxPasses = 8;
constexpr int kCountItems = 16;  // keys per thread per round of the counting kernel
static_assert(kSortThreads == kRadix, "one thread per digit in the tile bookkeeping");

struct SortState {
    uint32_t count[kMaxPasses][kRadix];   // keys per digit value, per pass
    uint32_t offset[kMaxPasses][kRadix];  // exclusive scan of count: where each digit's run starts
    uint32_t ticket[kMaxPasses];          // tiles started, per pass
    int32_t skip[kMaxPasses];             // every key has the same digit: the pass is the identity
};

// Whether the passes before `pass` that ran leave the pairs in the work buffers.
__device__ __forceinline__ bool pairs_in_alt(const SortState* st, int pass) {
    int alt = 0;
    for (int q = 0; q < pass; ++q) alt ^= st->skip[q] ? 0 : 1;
    return alt != 0;
}

// look-back words, one per (tile, digit): bits 63-62 the kind (0 nothing yet, 1 the tile's
// own count, 2 the count of this tile and all before it), bits 61-56 the pass + 1, bits 55-0
// the count.  Zeroed once per sort; the pass tag tells a word of the previous pass apart.
constexpr uint64_t kLookCount = 1ull << 62;
constexpr uint64_t kLookPrefix = 2ull << 62;
constexpr uint64_t kLookValue = (1ull << 56) - 1;
constexpr int kLookSpinLimit = 1 << 22;  // rounds that find a word not yet written before the wait gives up
constexpr int kLookWindow = 4;           // look-back words read at once


// Digit counts of every pass in one read of the keys (runs of equal digits in a thread's
// keys are added at once, so sorted or clustered keys do not pile atomics on one counter);
// also zeroes the look-back words.
__global__ void __launch_bounds__(kSortThreads) k_radix_count(const uint64_t* __restrict__ keys, int64_t n,
                                                              int begin_bit, int passes, SortState* __restrict__ st,
                                                              uint64_t* __restrict__ look, int64_t look_words) {
    __shared__ uint32_t h[kMaxPasses][kRadix];
    for (int i = threadIdx.x; i < kMaxPasses * kRadix; i += kSortThreads) (&h[0][0])[i] = 0;
    const int64_t gtid = static_cast<int64_t>(blockIdx.x) * kSortThreads + threadIdx.x;
    const int64_t gthreads = static_cast<int64_t>(gridDim.x) * kSortThreads;
    for (int64_t i = gtid; i < look_words; i += gthreads) look[i] = 0;
    __syncthreads();
    const unsigned int lane = lane_id();
    constexpr int64_t kWarpKeys = 32 * kCountItems;
    for (int64_t wb = (gtid >> 5) * kWarpKeys; wb < n; wb += (gthreads >> 5) * kWarpKeys) {
        uint64_t k[kCountItems];
#pragma unroll
        for (int j = 0; j < kCountItems; ++j) {
            const int64_t i = wb + j * 32 + lane;
            k[j] = i < n ? keys[i] : 0ull;
        }
        const int m = static_cast<int>(min(static_cast<int64_t>(kCountItems), (n - wb - lane + 31) / 32));
        for (int p = 0; p < passes; ++p) {
            const int sh = begin_bit + p * kRadixBits;
            uint32_t prev = static_cast<uint32_t>(k[0] >> sh) & (kRadix - 1);
            uint32_t run = m > 0 ? 1u : 0u;
#pragma unroll
            for (int j = 1; j < kCountItems; ++j) {
                if (j < m) {
                    const uint32_t d = static_cast<uint32_t>(k[j] >> sh) & (kRadix - 1);
                    if (d == prev) {
                        ++run;
                    } else {
                        atomicAdd(&h[p][prev], run);
                        prev = d;
                        run = 1;
                    }
                }
            }
            if (run) atomicAdd(&h[p][prev], run);
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < passes * kRadix; i += kSortThreads) {
        const uint32_t c = (&h[0][0])[i];
        if (c) atomicAdd(&(&st->count[0][0])[i], c);
    }
}

// One block per pass: where each digit's run starts, and whether the pass can be skipped.
__global__ void __launch_bounds__(kSortThreads) k_radix_plan(SortState* __restrict__ st, int64_t n) {
    const int p = blockIdx.x;
    const int d = threadIdx.x;
    const uint32_t c = st->count[p][d];
    uint32_t total;
    st->offset[p][d] = block_exclusive_scan<uint32_t, kSortThreads>(c, &total);
    const int whole = __syncthreads_or(static_cast<int64_t>(c) == n);
    if (d == 0) st->skip[p] = whole;
}

// One pass: stable scatter of the tiles by the digit at `shift`.  Tiles of 3072 pairs with
// 4 resident blocks per SM (at most 64 registers; 16 bytes spill): the 8 passes of the
// 10M-point sort take 0.96 ms, against 1.02 ms with 2048 pairs, 0.97 ms with 2560 and
// 1.06 ms with 3072 pairs at 3 resident blocks.
__global__ void __launch_bounds__(kSortThreads, 4) k_radix_scatter(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt,
                                                                uint32_t* vals_alt, int64_t n, int shift, int pass,
                                                                SortState* __restrict__ st,
                                                                uint64_t* __restrict__ look, unsigned int* fault) {
    if (st->skip[pass]) return;
    const bool alt = pairs_in_alt(st, pass);
    const uint64_t* __restrict__ kin = alt ? keys_alt : keys;
    const uint32_t* __restrict__ vin = alt ? vals_alt : vals;
    __shared__ uint32_t warp_count[kSortWarps][kRadix];
    __shared__ uint32_t digit_start[kRadix];
    __shared__ uint32_t digit_out[kRadix];
    __shared__ uint64_t skeys[kSortTile];
    __shared__ uint32_t svals[kSortTile];
    __shared__ uint32_t s_tile;
    const unsigned int lane = lane_id();
    const int warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) s_tile = atomicAdd(&st->ticket[pass], 1u);
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&warp_count[0][0])[i] = 0;
    __syncthreads();

    const int64_t tile = s_tile;
    const int64_t base = tile * kSortTile;
    const int64_t wbase = base + static_cast<int64_t>(warp) * 32 * kSortItems;
    uint64_t k[kSortItems];
    uint32_t v[kSortItems];
    uint32_t rank[kSortItems];
    const unsigned int below = lanes_below();
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        const bool valid = i < n;
        k[j] = valid ? kin[i] : 0ull;
        v[j] = valid ? vin[i] : 0u;
        const uint32_t d = static_cast<uint32_t>(k[j] >> shift) & (kRadix - 1);
        const uint32_t tag = valid ? d : (0x100u | lane);  // padding lanes match nobody
        const unsigned int peers = __match_any_sync(0xffffffffu, tag);
        const uint32_t r = __popc(peers & below);
        const uint32_t before = valid ? warp_count[warp][d] : 0u;
        __syncwarp();
        if (valid && r == 0) warp_count[warp][d] += __popc(peers);
        __syncwarp();
        rank[j] = before + r;
    }
    __syncthreads();

    // per digit (one thread each): offsets of the warps inside the tile and the tile's
    // count, published at once, and the tile's digit starts
    const int dg = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) {
        uint32_t c = warp_count[w][dg];
        warp_count[w][dg] = run;
        run += c;
    }
    const uint64_t tag = static_cast<uint64_t>(pass + 1) << 56;
    uint64_t* mine = look + tile * kRadix + dg;
    store_relaxed(mine, (tile == 0 ? kLookPrefix : kLookCount) | tag | run);
    uint32_t total;
    digit_start[dg] = block_exclusive_scan<uint32_t, kSortThreads>(run, &total);
    __syncthreads();
    // the tile reordered by digit in shared memory, while the tiles before it publish
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        const int64_t i = wbase + j * 32 + lane;
        if (i < n) {
            const uint32_t d = static_cast<uint32_t>(k[j] >> shift) & (kRadix - 1);
            const uint32_t p = digit_start[d] + warp_count[warp][d] + rank[j];
            skeys[p] = k[j];
            svals[p] = v[j];
        }
    }
    // then the counts of the tiles before it: kLookWindow tiles per round (independent
    // loads), added up to the first inclusive prefix; a word not yet written ends the
    // round early
    uint64_t before = 0;
    int spins = 0;
    for (int64_t j = tile - 1; j >= 0;) {
        uint64_t w[kLookWindow];
#pragma unroll
        for (int u = 0; u < kLookWindow; ++u)
            w[u] = j - u >= 0 ? load_relaxed(look + (j - u) * kRadix + dg) : (kLookPrefix | tag);
        int used = 0;
        bool done = false;
#pragma unroll
        for (int u = 0; u < kLookWindow; ++u) {
            if (done || used < u) continue;  // past the prefix or a word not yet written
            const bool ready = (w[u] & ~kLookValue & ~kLookPrefix & ~kLookCount) == tag && (w[u] >> 62) != 0;
            if (!ready) continue;
            before += w[u] & kLookValue;
            used = u + 1;
            done = (w[u] >> 62) == 2;
        }
        if (done) break;
        j -= used;
        if (used < kLookWindow) {
            if (++spins > kLookSpinLimit) {  // never expected: the tiles before are running
                if (fault) atomicOr(fault, kWaitTimedOut);
                break;
            }
            __nanosleep(32);
        }
    }
    if (tile > 0) store_relaxed(mine, kLookPrefix | tag | (before + run));
    digit_out[dg] = st->offset[pass][dg] + static_cast<uint32_t>(before);
    __syncthreads();
    const bool to_keys = pairs_in_alt(st, pass);  // read again rather than held through the tile
    uint64_t* __restrict__ kout = to_keys ? keys : keys_alt;
    uint32_t* __restrict__ vout = to_keys ? vals : vals_alt;
    const int64_t count = n - base < kSortTile ? n - base : kSortTile;
    for (int i = threadIdx.x; i < count; i += kSortThreads) {
        const uint64_t key = skeys[i];
        const uint32_t d = static_cast<uint32_t>(key >> shift) & (kRadix - 1);
        const int64_t g = static_cast<int64_t>(digit_out[d]) + (i - static_cast<int64_t>(digit_start[d]));
        if (g < n) {  // always true when the counts are consistent
            kout[g] = key;
            vout[g] = svals[i];
        }
    }
}

// After an odd number of passes that ran, the pairs are brought back to keys / vals.
__global__ void __launch_bounds__(256) k_radix_copy_back(uint64_t* __restrict__ keys, uint32_t* __restrict__ vals,
                                                         const uint64_t* __restrict__ keys_alt,
                                                         const uint32_t* __restrict__ vals_alt, int64_t n,
                                                         const SortState* __restrict__ st, int passes) {
    if (!pairs_in_alt(st, passes)) return;
    const int64_t stride = static_cast<int64_t>(gridDim.x) * blockDim.x;
    for (int64_t i = static_cast<int64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n; i += stride) {
        keys[i] = keys_alt[i];
        vals[i] = vals_alt[i];
    }
}

sfc_status radix_sort_pairs_bits(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, int64_t n,
                                 int begin_bit, int end_bit, cudaStream_t s, Scratch& scratch, unsigned int* fault) {
    if (n <= 1 || end_bit <= begin_bit) return SFC_OK;
    const int passes = (end_bit - begin_bit + kRadixBits - 1) / kRadixBits;
    if (begin_bit < 0 || end_bit > 64 || passes > kMaxPasses || n > 0xffffffffLL) return SFC_ERR_INVALID;
    const int64_t tiles = (n + kSortTile - 1) / kSortTile;
    SortState* st = nullptr;
    uint64_t* look = nullptr;
    SFC_TRY(scratch.alloc(&st, 1));
    SFC_TRY(scratch.alloc(&look, static_cast<size_t>(kRadix * tiles)));
    SFC_CUDA(cudaMemsetAsync(st, 0, sizeof(SortState), s));
    SFC_LAUNCH("radix_count", s, k_radix_count, grid_for(n, kSortThreads * kCountItems, 152 * 8), kSortThreads, 0, keys,
               n, begin_bit, passes, st, look, kRadix * tiles);
    SFC_LAUNCH("radix_plan", s, k_radix_plan, passes, kSortThreads, 0, st, n);
    for (int p = 0; p < passes; ++p)
        SFC_LAUNCH("radix_scatter", s, k_radix_scatter, static_cast<unsigned int>(tiles), kSortThreads, 0, keys, vals,
                   keys_alt, vals_alt, n, begin_bit + p * kRadixBits, p, st, look, fault);
    SFC_LAUNCH("radix_copy_back", s, k_radix_copy_back, grid_for(n, 256, 152 * 4), 256, 0, keys, vals, keys_alt,
               vals_alt, n, st, passes);
    return SFC_OK;
}

sfc_status radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, int64_t n,
                            cudaStream_t s, Scratch& scratch, unsigned int* fault) {
    return radix_sort_pairs_bits(keys, vals, keys_alt, vals_alt, n, 0, 64, s, scratch, fault);
}

}  // namespace sfc

// ---------------------------------------------------------------------------------
// C ABI: runtime queries
extern "C" {

const char* sfc_status_string(sfc_status s) {
    switch (s) {
    case SFC_OK: return "ok";
    case SFC_ERR_INVALID: return "invalid argument";
    case SFC_ERR_OOM: return "out of device memory";
    case SFC_ERR_CUDA: return "CUDA error";
    case SFC_ERR_TIMEOUT: return "device wait timed out";
    case SFC_ERR_TOO_LARGE: return "size limit exceeded";
    case SFC_ERR_NOT_DEVICE_PTR: return "pointer is not device memory";
    case SFC_ERR_NOT_FINITE: return "non-finite coordinate or extent";
    case SFC_ERR_INTERNAL: return "device-side consistency guard tripped";
    }
    return "unknown status";
}

const char* sfc_last_error(void) { return sfc::t_last_error; }

uint64_t sfc_launch_count(void) { return sfc::g_launches.load(); }

sfc_status sfc_set_allocator(sfc_alloc_fn alloc, sfc_free_fn free_fn, void* ctx) {
    if ((alloc == nullptr) != (free_fn == nullptr)) return SFC_ERR_INVALID;
    std::lock_guard<std::mutex> g(sfc::g_alloc_mu);
    if (sfc::g_live.load() != 0) return SFC_ERR_INVALID;
    sfc::g_alloc = alloc;
    sfc::g_free = free_fn;
    sfc::g_alloc_ctx = ctx;
    return SFC_OK;
}

int64_t sfc_live_allocations(void) { return sfc::g_live.load(); }

sfc_status sfc_stats_enable(int32_t on) {
    std::lock_guard<std::mutex> g(sfc::g_stats_mu);
    if (on) {
        int dev = -1;
        SFC_CUDA(cudaGetDevice(&dev));
        if (sfc::g_stats && dev != sfc::g_stats_device) {  // counting moves to the current device
            SFC_CUDA(cudaSetDevice(sfc::g_stats_device));
            const cudaError_t e = cudaDeviceSynchronize();
            cudaFree(sfc::g_stats);
            sfc::g_stats = nullptr;
            SFC_CUDA(cudaSetDevice(dev));
            SFC_CUDA(e);
        }
        if (!sfc::g_stats) {
            void* p = nullptr;
            SFC_CUDA(cudaMalloc(&p, sizeof(unsigned long long) * sfc::kStCount));
            sfc::g_stats = static_cast<unsigned long long*>(p);
            sfc::g_stats_device = dev;
        }
        SFC_CUDA(cudaDeviceSynchronize());
        SFC_CUDA(cudaMemset(sfc::g_stats, 0, sizeof(unsigned long long) * sfc::kStCount));
        SFC_CUDA(cudaDeviceSynchronize());
    }
    sfc::g_stats_on.store(on != 0);
    return SFC_OK;
}

sfc_status sfc_stats_read(sfc_search_stats* out) {
    if (!out) return SFC_ERR_INVALID;
    static_assert(sizeof(sfc_search_stats) == sizeof(unsigned long long) * sfc::kStCount,
                  "one counter per field");
    std::lock_guard<std::mutex> g(sfc::g_stats_mu);
    memset(out, 0, sizeof *out);
    if (!sfc::g_stats) return SFC_OK;
    int dev = -1;
    SFC_CUDA(cudaGetDevice(&dev));
    SFC_CUDA(cudaSetDevice(sfc::g_stats_device));  // wait for the work of the counters' device
    const cudaError_t e1 = cudaDeviceSynchronize();
    const cudaError_t e2 = e1 == cudaSuccess ? cudaMemcpy(out, sfc::g_stats, sizeof *out, cudaMemcpyDeviceToHost) : e1;
    SFC_CUDA(cudaSetDevice(dev));
    SFC_CUDA(e2);
    return SFC_OK;
}

sfc_status sfc_profile_enable(int32_t on) {
    std::lock_guard<std::mutex> g(sfc::g_prof_mu);
    if (on) {
        for (auto& r : sfc::g_prof) {
            cudaEventSynchronize(r.stop);
            cudaEventDestroy(r.start);
            cudaEventDestroy(r.stop);
        }
        sfc::g_prof.clear();
    }
    sfc::g_prof_on.store(on != 0);
    return SFC_OK;
}

int32_t sfc_profile_read(char* names, int64_t* launches, double* total_ms, int32_t cap) {
    std::lock_guard<std::mutex> g(sfc::g_prof_mu);
    std::vector<std::string> keys;
    std::vector<int64_t> cnt;
    std::vector<double> ms;
    for (auto& r : sfc::g_prof) {
        float t = 0.f;
        cudaEventSynchronize(r.stop);
        cudaEventElapsedTime(&t, r.start, r.stop);
        size_t i = 0;
        while (i < keys.size() && keys[i] != r.name) ++i;
        if (i == keys.size()) {
            keys.push_back(r.name);
            cnt.push_back(0);
            ms.push_back(0.0);
        }
        cnt[i] += 1;
        ms[i] += t;
    }
    for (size_t i = 0; i < keys.size() && static_cast<int32_t>(i) < cap; ++i) {
        if (names) {
            strncpy(names + 64 * i, keys[i].c_str(), 63);
            names[64 * i + 63] = 0;
        }
        if (launches) launches[i] = cnt[i];
        if (total_ms) total_ms[i] = ms[i];
    }
    return static_cast<int32_t>(keys.size());
}

}  // extern "C"
