// sfc_static.cu - radius_count_static: the all-points count pass of the radius search for
// callers that must not allocate device memory.
//
// Some callers cannot let a library allocate: an application that reserves the whole
// device budget up front and hands out fixed buffers (so any cudaMalloc/cudaMallocAsync
// inside a call could fail or evict its own pool), or a loop with a hard latency budget in
// which an allocation's occasional cost or failure is not acceptable.  radius_count needs
// device scratch (one count per point, one look-back word per scan tile); this variant takes that
// scratch from one file-scope __device__ array instead, so it allocates nothing.  The
// caller still provides the outputs.
//
// The array is part of the library image: every GPU that loads the library holds it
// (kStaticBytes, about 8 MiB) until the process exits.  Its device address is looked up
// once per device, by the first call on that device, with cudaGetSymbolAddress; make that
// first call before any stream capture.  All calls share the array and it keeps the last
// call's contents, so calls that overlap on the GPU (on different streams, or from
// different host threads without ordering) race on it.
#include <cuda_runtime.h>
#include <math.h>

#include <mutex>

#include "sfc_internal.cuh"

namespace {

// Largest number of points (rows) the static scratch serves.
constexpr int64_t kStaticRows = int64_t(1) << 21;
constexpr int64_t kStaticCountBytes = kStaticRows * sizeof(uint32_t);  // a multiple of 256
constexpr int64_t kStaticTileBytes = 1024 * sizeof(int64_t);            // >= scan words of kStaticRows
constexpr int64_t kStaticBytes = kStaticCountBytes + kStaticTileBytes;

static __device__ __align__(256) unsigned char g_radius_scratch[kStaticBytes];

constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_radius_scratch on the current device (looked up once per device).
sfc_status scratch_address(void** out) {
    int dev = 0;
    SFC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return SFC_ERR_TOO_LARGE;
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void* p = nullptr;
        SFC_CUDA(cudaGetSymbolAddress(&p, g_radius_scratch));
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
    return SFC_OK;
}

}  // namespace

extern "C" sfc_status radius_count_static(sfc_octree h, float r, sfc_kernel kern, void* cuda_stream,
                                          int64_t* row_ptr, int64_t* nnz) {
    if (!h || !row_ptr || !nnz) return SFC_ERR_INVALID;
    if (kern != SFC_SPHERE && kern != SFC_CIRCLE && kern != SFC_CUBE && kern != SFC_SQUARE) return SFC_ERR_INVALID;
    if (isnan(r)) return SFC_ERR_INVALID;
    const sfc::Octree* t = &h->tree;
    if (t->n > kStaticRows) return SFC_ERR_TOO_LARGE;
    if (sfc::scan_tile_count(t->n) * static_cast<int64_t>(sizeof(int64_t)) > kStaticTileBytes)
        return SFC_ERR_TOO_LARGE;
    if (!sfc::is_device_ptr(row_ptr)) return SFC_ERR_NOT_DEVICE_PTR;
    void* base = nullptr;
    SFC_TRY(scratch_address(&base));
    uint32_t* counts = static_cast<uint32_t*>(base);
    int64_t* tile_sums = reinterpret_cast<int64_t*>(static_cast<unsigned char*>(base) + kStaticCountBytes);
    return sfc::radius_count_presized(t, r, kern, static_cast<cudaStream_t>(cuda_stream), counts, tile_sums,
                                      row_ptr, nnz);
}

extern "C" int64_t radius_count_static_max_points(void) { return kStaticRows; }
