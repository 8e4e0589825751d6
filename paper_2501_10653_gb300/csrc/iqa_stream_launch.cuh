// iqa_stream_launch.cuh -- host-side launch of iqa_stream_kernel for one
// storage type (included by iqa_stream_<type>.cu).
#pragma once

#include <atomic>
#include <mutex>

#include "iqa_internal.h"
#include "iqa_stream.cuh"

namespace iqa {

template <typename T, int CT, bool A, bool B>
static cudaError_t stream_launch_one(const StreamParams &sp, int grid, size_t smem,
                                     cudaStream_t st)
{
    auto kern = iqa_stream_kernel<T, CT, A, B>;
    // raise the dynamic shared-memory limit when a launch needs more than any
    // earlier one of this instantiation; host threads may launch concurrently,
    // so raises are serialised and the limit only ever grows
    static std::atomic<size_t> allowed{0};
    static std::mutex raise_mu;
    if (smem > allowed.load(std::memory_order_acquire)) {
        std::lock_guard<std::mutex> g(raise_mu);
        if (smem > allowed.load(std::memory_order_relaxed)) {
            cudaError_t e = cudaFuncSetAttribute(
                kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            allowed.store(smem, std::memory_order_release);
        }
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid, 1, 1);
    cfg.blockDim = dim3(CT + 32, 1, 1);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    // programmatic dependent launch: the kernel may start while the previous
    // kernel in the stream finishes; it waits for it (griddepcontrol.wait)
    // before reading work or pixels
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, sp);
}

template <typename T, int CT>
static cudaError_t stream_by_maps(const StreamParams &sp, int maps, int grid, size_t smem,
                                  cudaStream_t st)
{
    switch (maps) {
    case MAPS_A: return stream_launch_one<T, CT, true, false>(sp, grid, smem, st);
    case MAPS_B: return stream_launch_one<T, CT, false, true>(sp, grid, smem, st);
    default: return stream_launch_one<T, CT, true, true>(sp, grid, smem, st);
    }
}

template <typename T>
static cudaError_t launch_stream_t(const StreamParams &sp, int ct, int maps, int grid,
                                   size_t smem, cudaStream_t st)
{
    switch (ct) {
    case 128: return stream_by_maps<T, 128>(sp, maps, grid, smem, st);
    case 256: return stream_by_maps<T, 256>(sp, maps, grid, smem, st);
    case 512: return stream_by_maps<T, 512>(sp, maps, grid, smem, st);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace iqa
