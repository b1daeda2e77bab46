// mcdi_build_bvh_noalloc: the BVH build of mcdi_build_bvh with its scratch in a
// fixed device array owned by this library, for callers that must not allocate
// device memory themselves.
//
// The array below is a file-scope __device__ object: every GPU that loads the
// library holds kNoallocScratchBytes of it until the process exits.  In host
// code its name is only a host-side stand-in, never a device address, so the
// address handed to the kernels is looked up with cudaGetSymbolAddress once
// per device (with that device current) and cached.  All calls on a device
// share the array and it keeps the previous call's contents; the build writes
// every scratch word it later reads (bounds, histograms, parents, arrival
// counters, boxes), so nothing needs clearing between calls.  Calls whose
// work overlaps on the GPU (two streams, or two host threads) race on the
// array and must be serialised by the caller.
#include <stdint.h>

#include <mutex>

#include "internal.h"

namespace {

constexpr int kNoallocMaxTris = MCDI_NOALLOC_MAX_TRIS;
constexpr int kMaxDevices = 64;

// large enough for bvh_scratch_layout(kNoallocMaxTris): ~92.5 bytes per triangle
constexpr size_t kNoallocScratchBytes = (size_t)6 << 20;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

std::mutex g_setup_mutex;
void* g_scratch_addr[kMaxDevices] = {};

mcdi_status noalloc_fail(mcdi_status s, const char* msg) {
    mcdi::set_last_error(msg);
    return s;
}

// Device address of the scratch array on the current device; looked up on the
// first call made on that device.
mcdi_status scratch_on_current_device(void** out, const char** why) {
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
    if (g_scratch_addr[dev] == nullptr) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            *why = e != cudaSuccess ? cudaGetErrorString(e) : "cudaGetSymbolAddress returned NULL";
            return MCDI_DEVICE_ERROR;
        }
        g_scratch_addr[dev] = p;
    }
    *out = g_scratch_addr[dev];
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
    const mcdi::BvhScratch L = mcdi::bvh_scratch_layout(n_tris);
    if (L.total > kNoallocScratchBytes) return noalloc_fail(MCDI_INVALID_ARG, "mesh needs more scratch than reserved");
    void* scratch = nullptr;
    const char* why = "";
    mcdi_status s = scratch_on_current_device(&scratch, &why);
    if (s != MCDI_OK) return noalloc_fail(s, why);
    cudaError_t e = mcdi::launch_build_bvh(verts, n_verts, tris, n_tris, nodes, tri_records, scratch, L,
                                           static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return noalloc_fail(MCDI_DEVICE_ERROR, cudaGetErrorString(e));
    mcdi::set_last_error("");
    return MCDI_OK;
}

}  // extern "C"
