// Launches with programmatic dependent launch: the kernel may be scheduled
// while the previous kernel on the stream finishes its last CTAs, and waits
// (griddepcontrol.wait, first statement of every kernel launched this way)
// until that kernel has completed and its memory is visible.  This hides the
// launch gap between the kernels of an operation.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace catfhe {

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem,
                              cudaStream_t s, Args &&...args) {
    cudaLaunchConfig_t cfg{};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace catfhe
