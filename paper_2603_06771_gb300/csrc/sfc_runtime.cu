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
// exclusive scan: tiles of kScanTile elements; per-tile sums, a single-block scan of
// the tile sums, then each tile is scanned again with its offset added.
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

template <typename TI, typename TO>
__global__ void __launch_bounds__(kScanThreads) k_scan_tile_sums(const TI* __restrict__ in, int64_t n,
                                                                 TO* __restrict__ sums) {
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + static_cast<int64_t>(threadIdx.x) * kScanItems;
    TO acc = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j)
        if (base + j < n) acc += static_cast<TO>(in[base + j]);
    TO total;
    block_exclusive_scan<TO, kScanThreads>(acc, &total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

template <typename TO>
__global__ void __launch_bounds__(1024) k_scan_spine(TO* __restrict__ sums, int64_t m) {
    TO carry = 0;
    for (int64_t base = 0; base < m; base += 1024) {
        int64_t i = base + threadIdx.x;
        TO v = i < m ? sums[i] : TO(0);
        TO total;
        TO ex = block_exclusive_scan<TO, 1024>(v, &total);
        if (i < m) sums[i] = carry + ex;
        carry += total;
    }
}

template <typename TI, typename TO>
__global__ void __launch_bounds__(kScanThreads) k_scan_apply(const TI* in, TO* out, int64_t n,
                                                             const TO* __restrict__ sums) {
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kScanTile + static_cast<int64_t>(threadIdx.x) * kScanItems;
    TO v[kScanItems];
    TO acc = 0;
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        v[j] = base + j < n ? static_cast<TO>(in[base + j]) : TO(0);
        acc += v[j];
    }
    TO total;
    TO run = block_exclusive_scan<TO, kScanThreads>(acc, &total) + sums[blockIdx.x];
#pragma unroll
    for (int j = 0; j < kScanItems; ++j) {
        if (base + j < n) out[base + j] = run;
        run += v[j];
    }
    // the element one past the end receives the grand total
    if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = sums[blockIdx.x] + total;
}

template <typename TI, typename TO>
static sfc_status scan_impl(const TI* in, TO* out, int64_t n, cudaStream_t s, Scratch& scratch) {
    if (n == 0) {
        SFC_CUDA(cudaMemsetAsync(out, 0, sizeof(TO), s));
        return SFC_OK;
    }
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    TO* sums = nullptr;
    SFC_TRY(scratch.alloc(&sums, static_cast<size_t>(tiles)));
    SFC_LAUNCH("scan_tile_sums", s, (k_scan_tile_sums<TI, TO>), static_cast<unsigned int>(tiles), kScanThreads, 0,
               in, n, sums);
    SFC_LAUNCH("scan_spine", s, k_scan_spine<TO>, 1, 1024, 0, sums, tiles);
    SFC_LAUNCH("scan_apply", s, (k_scan_apply<TI, TO>), static_cast<unsigned int>(tiles), kScanThreads, 0, in, out,
               n, sums);
    return SFC_OK;
}

sfc_status scan_u32_to_i64(const uint32_t* in, int64_t* out, int64_t n, cudaStream_t s, Scratch& scratch) {
    return scan_impl<uint32_t, int64_t>(in, out, n, s, scratch);
}
sfc_status scan_u32_to_u32(const uint32_t* in, uint32_t* out, int64_t n, cudaStream_t s, Scratch& scratch) {
    return scan_impl<uint32_t, uint32_t>(in, out, n, s, scratch);
}

int64_t scan_tile_count(int64_t n) { return (n + kScanTile - 1) / kScanTile; }

sfc_status scan_u32_to_i64_presized(const uint32_t* in, int64_t* out, int64_t n, int64_t* tile_sums, cudaStream_t s) {
    if (n == 0) {
        SFC_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), s));
        return SFC_OK;
    }
    const int64_t tiles = scan_tile_count(n);
    SFC_LAUNCH("scan_tile_sums", s, (k_scan_tile_sums<uint32_t, int64_t>), static_cast<unsigned int>(tiles),
               kScanThreads, 0, in, n, tile_sums);
    SFC_LAUNCH("scan_spine", s, k_scan_spine<int64_t>, 1, 1024, 0, tile_sums, tiles);
    SFC_LAUNCH("scan_apply", s, (k_scan_apply<uint32_t, int64_t>), static_cast<unsigned int>(tiles), kScanThreads,
               0, in, out, n, tile_sums);
    return SFC_OK;
}

// ---------------------------------------------------------------------------------
// LSD radix sort of (63-bit code, uint32 index) pairs, 8-bit digits, 8 passes.
// Per pass: per-tile digit histograms (digit-major, so one exclusive scan gives every
// tile's output offset per digit), then a stable scatter: each warp ranks its items in
// input order with match-any, the tile is reordered by digit in shared memory and
// written out in runs that are contiguous per digit.
constexpr int kRadixBits = 8;
constexpr int kRadix = 1 << kRadixBits;
constexpr int kSortThreads = 256;
constexpr int kSortWarps = kSortThreads / 32;
constexpr int kSortItems = 8;
constexpr int kSortTile = kSortThreads * kSortItems;
static_assert(kSortThreads == kRadix, "one thread per digit in the tile bookkeeping");

__global__ void __launch_bounds__(kSortThreads) k_radix_histogram(const uint64_t* __restrict__ keys, int64_t n,
                                                                  int shift, uint32_t* __restrict__ hist,
                                                                  int64_t tiles) {
    __shared__ uint32_t h[kSortWarps][kRadix];
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&h[0][0])[i] = 0;
    __syncthreads();
    const int64_t base = static_cast<int64_t>(blockIdx.x) * kSortTile;
    const int warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < kSortItems; ++j) {
        int64_t i = base + j * kSortThreads + threadIdx.x;
        if (i < n) atomicAdd(&h[warp][(keys[i] >> shift) & (kRadix - 1)], 1u);
    }
    __syncthreads();
    uint32_t sum = 0;
#pragma unroll
    for (int w = 0; w < kSortWarps; ++w) sum += h[w][threadIdx.x];
    hist[static_cast<int64_t>(threadIdx.x) * tiles + blockIdx.x] = sum;
}

// 4 resident blocks per SM (at most 64 registers): 0.85 -> 0.79 ms for the 8 passes of a
// 10M-point sort; larger tiles (fewer resident blocks) measured slower
__global__ void __launch_bounds__(kSortThreads, 4) k_radix_scatter(const uint64_t* __restrict__ kin,
                                                                const uint32_t* __restrict__ vin,
                                                                uint64_t* __restrict__ kout,
                                                                uint32_t* __restrict__ vout, int64_t n, int shift,
                                                                const uint32_t* __restrict__ offsets,
                                                                int64_t tiles) {
    __shared__ uint32_t warp_count[kSortWarps][kRadix];
    __shared__ uint32_t digit_start[kRadix];
    __shared__ uint32_t digit_out[kRadix];
    __shared__ uint64_t skeys[kSortTile];
    __shared__ uint32_t svals[kSortTile];
    const unsigned int lane = lane_id();
    const int warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < kSortWarps * kRadix; i += kSortThreads) (&warp_count[0][0])[i] = 0;
    __syncthreads();

    const int64_t base = static_cast<int64_t>(blockIdx.x) * kSortTile;
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

    // per digit: offsets of the warps inside the tile, then the tile's digit starts
    {
        const int d = threadIdx.x;
        uint32_t run = 0;
#pragma unroll
        for (int w = 0; w < kSortWarps; ++w) {
            uint32_t c = warp_count[w][d];
            warp_count[w][d] = run;
            run += c;
        }
        uint32_t total;
        uint32_t start = block_exclusive_scan<uint32_t, kSortThreads>(run, &total);
        digit_start[d] = start;
        digit_out[d] = offsets[static_cast<int64_t>(d) * tiles + blockIdx.x];
    }
    __syncthreads();
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
    __syncthreads();
    const int64_t count = n - base < kSortTile ? n - base : kSortTile;
    for (int i = threadIdx.x; i < count; i += kSortThreads) {
        const uint64_t key = skeys[i];
        const uint32_t d = static_cast<uint32_t>(key >> shift) & (kRadix - 1);
        const int64_t g = static_cast<int64_t>(digit_out[d]) + (i - static_cast<int64_t>(digit_start[d]));
        if (g < n) {  // always true when the offsets are consistent
            kout[g] = key;
            vout[g] = svals[i];
        }
    }
}

sfc_status radix_sort_pairs_bits(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, int64_t n,
                                 int begin_bit, int end_bit, cudaStream_t s, Scratch& scratch) {
    if (n <= 1 || end_bit <= begin_bit) return SFC_OK;
    const int64_t tiles = (n + kSortTile - 1) / kSortTile;
    uint32_t* hist = nullptr;
    SFC_TRY(scratch.alloc(&hist, static_cast<size_t>(kRadix * tiles + 1)));
    uint64_t* ksrc = keys;
    uint32_t* vsrc = vals;
    uint64_t* kdst = keys_alt;
    uint32_t* vdst = vals_alt;
    for (int shift = begin_bit; shift < end_bit; shift += kRadixBits) {
        SFC_LAUNCH("radix_histogram", s, k_radix_histogram, static_cast<unsigned int>(tiles), kSortThreads, 0, ksrc,
                   n, shift, hist, tiles);
        SFC_TRY(scan_u32_to_u32(hist, hist, kRadix * tiles, s, scratch));
        SFC_LAUNCH("radix_scatter", s, k_radix_scatter, static_cast<unsigned int>(tiles), kSortThreads, 0, ksrc,
                   vsrc, kdst, vdst, n, shift, hist, tiles);
        uint64_t* tk = ksrc; ksrc = kdst; kdst = tk;
        uint32_t* tv = vsrc; vsrc = vdst; vdst = tv;
    }
    if (ksrc != keys) {  // an odd number of passes: bring the result back
        SFC_CUDA(cudaMemcpyAsync(keys, ksrc, sizeof(uint64_t) * n, cudaMemcpyDeviceToDevice, s));
        SFC_CUDA(cudaMemcpyAsync(vals, vsrc, sizeof(uint32_t) * n, cudaMemcpyDeviceToDevice, s));
    }
    return SFC_OK;
}

sfc_status radix_sort_pairs(uint64_t* keys, uint32_t* vals, uint64_t* keys_alt, uint32_t* vals_alt, int64_t n,
                            cudaStream_t s, Scratch& scratch) {
    return radix_sort_pairs_bits(keys, vals, keys_alt, vals_alt, n, 0, 64, s, scratch);
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
