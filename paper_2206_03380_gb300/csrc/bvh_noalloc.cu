// mcdi_build_bvh_noalloc: the BVH build of mcdi_build_bvh with its scratch in a
// fixed device array owned by this library, for callers that must not allocate
// device memory themselves.
//
// The array below is a file-scope __device__ object: every GPU that loads the
// library holds kNoallocScratchBytes of it until the process exits.  In host
// code its name is only a host-side stand-in, never a device address, so the
// address handed to the kernels is looked up with cudaGetSymbolAddress with
// the device current.  That address belongs to one CUDA context, so the cache
// is keyed by the current context's unique id (cuCtxGetId): after
// cudaDeviceReset, or with another context current on the same device, the
// address is looked up again.  A lookup is refused while the caller's stream
// is being captured (the first call in a context must come before any
// capture).  All calls in a context share the array and it keeps the previous
// call's contents; the build writes every scratch word it later reads
// (bounds, histograms, parents, arrival counters, boxes), so nothing needs
// clearing between calls.  Calls whose work overlaps on the GPU (two streams,
// or two host threads) race on the array and must be serialised by the
// caller.
#include <stdint.h>

#include <mutex>

#include "internal.h"

namespace {

constexpr int kNoallocMaxTris = MCDI_NOALLOC_MAX_TRIS;
constexpr int kMaxDevices = 64;

constexpr size_t kNoallocScratchBytes = (size_t)7 << 20;
static_assert(mcdi::bvh_scratch_layout(kNoallocMaxTris).total <= kNoallocScratchBytes,
              "the fixed scratch array must hold the build scratch of MCDI_NOALLOC_MAX_TRIS triangles");

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// driver entry points, resolved through the runtime (no link against libcuda)
typedef int (*CtxGetCurrentFn)(void** ctx);
typedef int (*CtxGetIdFn)(void* ctx, unsigned long long* id);

struct CachedAddress {
    unsigned long long ctx_id;  // 0: nothing cached
    void* addr;
};

std::mutex g_setup_mutex;
CtxGetCurrentFn g_ctx_get_current = nullptr;
CtxGetIdFn g_ctx_get_id = nullptr;
CachedAddress g_scratch_addr[kMaxDevices] = {};

mcdi_status noalloc_fail(mcdi_status s, const char* msg) {
    mcdi::set_last_error(msg);
    return s;
}

// caller holds g_setup_mutex
bool resolve_driver_calls() {
    if (g_ctx_get_current && g_ctx_get_id) return true;
    void* a = nullptr;
    void* b = nullptr;
    cudaDriverEntryPointQueryResult qa = cudaDriverEntryPointSymbolNotFound, qb = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &a, 12000, cudaEnableDefault, &qa) != cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &b, 12000, cudaEnableDefault, &qb) != cudaSuccess ||
        qa != cudaDriverEntryPointSuccess || qb != cudaDriverEntryPointSuccess || !a || !b)
        return false;
    g_ctx_get_current = reinterpret_cast<CtxGetCurrentFn>(a);
    g_ctx_get_id = reinterpret_cast<CtxGetIdFn>(b);
    return true;
}

// Device address of the scratch array in the current context; looked up on
// the first call made in that context (not during stream capture).
mcdi_status scratch_in_current_context(cudaStream_t stream, void** out, const char** why) {
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) {
        *why = cudaGetErrorString(e);
        return MCDI_DEVICE_ERROR;
    }
    if (dev < 0 || dev >= kMaxDevices) {
        *why = "device ordinal beyond the supported range";
        return MCDI_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!resolve_driver_calls()) {
        *why = "cuCtxGetCurrent / cuCtxGetId not available from the driver";
        return MCDI_DEVICE_ERROR;
    }
    void* ctx = nullptr;
    if (g_ctx_get_current(&ctx) != 0 || ctx == nullptr) {
        // no context current yet: make the device's primary context current
        e = cudaSetDevice(dev);
        if (e != cudaSuccess || g_ctx_get_current(&ctx) != 0 || ctx == nullptr) {
            *why = "no CUDA context is current on this thread";
            return MCDI_DEVICE_ERROR;
        }
    }
    unsigned long long id = 0;
    if (g_ctx_get_id(ctx, &id) != 0 || id == 0) {
        *why = "cuCtxGetId failed";
        return MCDI_DEVICE_ERROR;
    }
    CachedAddress& c = g_scratch_addr[dev];
    if (c.ctx_id != id) {
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        e = cudaStreamIsCapturing(stream, &cap);
        if (e != cudaSuccess) {
            *why = cudaGetErrorString(e);
            return MCDI_DEVICE_ERROR;
        }
        if (cap != cudaStreamCaptureStatusNone) {
            *why = "the first mcdi_build_bvh_noalloc call in a CUDA context must come before stream capture";
            return MCDI_INVALID_ARG;
        }
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            *why = e != cudaSuccess ? cudaGetErrorString(e) : "cudaGetSymbolAddress returned NULL";
            return MCDI_DEVICE_ERROR;
        }
        c.ctx_id = id;
        c.addr = p;
    }
    *out = c.addr;
    return MCDI_OK;
}

}  // namespace

extern "C" {

mcdi_status mcdi_build_bvh_noalloc(const float* verts, int n_verts, const int* tris, int n_tris, void* nodes,
                                   void* tri_records, void* stream) {
    if (n_tris < 1 || n_tris > kNoallocMaxTris)
        return noalloc_fail(MCDI_INVALID_ARG,
                            "n_tris must be in [1, MCDI_NOALLOC_MAX_TRIS = 65536] for mcdi_build_bvh_noalloc; "
                            "use mcdi_build_bvh with caller scratch for larger meshes");
    if (n_verts < 1 || verts == nullptr || tris == nullptr)
        return noalloc_fail(MCDI_INVALID_ARG, "verts / tris must be non-NULL and n_verts >= 1");
    if (((uintptr_t)verts & 3u) != 0 || ((uintptr_t)tris & 3u) != 0)
        return noalloc_fail(MCDI_INVALID_ARG, "verts / tris must be 4-byte aligned");
    if (nodes == nullptr || tri_records == nullptr || ((uintptr_t)nodes & 255u) != 0 ||
        ((uintptr_t)tri_records & 15u) != 0)
        return noalloc_fail(MCDI_INVALID_ARG, "nodes must be 256-byte aligned, tri_records 16-byte aligned (non-NULL device pointers)");
    const mcdi::BvhScratch L = mcdi::bvh_scratch_layout(n_tris);  // <= the array (static_assert above)
    void* scratch = nullptr;
    const char* why = "";
    mcdi_status s = scratch_in_current_context(static_cast<cudaStream_t>(stream), &scratch, &why);
    if (s != MCDI_OK) return noalloc_fail(s, why);
    cudaError_t e = mcdi::launch_build_bvh(verts, n_verts, tris, n_tris, nodes, tri_records, scratch, L,
                                           static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return noalloc_fail(MCDI_DEVICE_ERROR, cudaGetErrorString(e));
    mcdi::set_last_error("");
    return MCDI_OK;
}

}  // extern "C"
