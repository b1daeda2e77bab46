// Programmatic dependent launch between the library's kernels.  Every kernel
// starts with pdl_prologue(): it waits until the kernel before it in the stream
// has completed and its writes are visible (before touching any global
// memory), then lets the next kernel begin launching, so that kernel's CTAs
// are resident and waiting when this one ends instead of being launched only
// then.  Host code launches through launch_k, which marks the launch as
// allowed to start before its predecessor completes — except while the
// stream is being captured into a CUDA graph, whose replay already launches
// back to back (measured: the mark saves about 80 us per headline step
// launched kernel by kernel; on every node of the replayed graph it costs
// about 40 us).  The convolutions, which allocate tensor memory and load their
// weights before they wait, launch through launch_k_dependent, which keeps
// the mark in the graph too (a programmatic edge from the preceding kernel
// node): 40 us less per replayed headline step.  For a kernel launched without
// the mark the prologue's wait returns at once.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace mcdi {

// whether launch_k_dependent keeps the programmatic dependence in graphs this thread captures (default on;
// mcdi_set_graph_dependent_launch)
extern thread_local bool t_graph_dependent_launch;

__device__ __forceinline__ void pdl_prologue() {
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

// The two halves of pdl_prologue, for kernels with setup that depends on nothing
// the preceding kernel writes: let the next kernel launch, do that setup, then
// wait (every thread, before its first access to data of earlier kernels).
__device__ __forceinline__ void pdl_allow_dependents() {
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k_impl(bool dependent_in_graph, void (*kernel)(KArgs...), dim3 grid, dim3 block,
                                 size_t smem, cudaStream_t stream, Args&&... args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[2]{};
    unsigned n_attr = 0;
    cudaStreamCaptureStatus capture = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(stream, &capture) != cudaSuccess) capture = cudaStreamCaptureStatusNone;
    if (capture == cudaStreamCaptureStatusNone || (dependent_in_graph && t_graph_dependent_launch)) {
        attr[n_attr].id = cudaLaunchAttributeProgrammaticStreamSerialization;
        attr[n_attr++].val.programmaticStreamSerializationAllowed = 1;
    }
    // a stream's priority, also for kernels captured into a graph (their nodes keep it)
    int prio = 0;
    if (cudaStreamGetPriority(stream, &prio) == cudaSuccess && prio != 0) {
        attr[n_attr].id = cudaLaunchAttributePriority;
        attr[n_attr++].val.priority = prio;
    }
    cfg.attrs = n_attr ? attr : nullptr;
    cfg.numAttrs = n_attr;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                            Args&&... args) {
    return launch_k_impl(false, kernel, grid, block, smem, stream, std::forward<Args>(args)...);
}

// launch_k that keeps the programmatic dependence also inside a captured graph
// (a programmatic edge from the preceding kernel node): for kernels whose
// set-up before pdl_wait() is long enough to pay for it
template <typename... KArgs, typename... Args>
inline cudaError_t launch_k_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                                      cudaStream_t stream, Args&&... args) {
    return launch_k_impl(true, kernel, grid, block, smem, stream, std::forward<Args>(args)...);
}

}  // namespace mcdi
