// iqa_stream_f16.cu -- persistent TMA-pipelined kernels for __half pixel storage.
#include "iqa_stream.cuh"
#include "iqa_stream_launch.cuh"

namespace iqa {

cudaError_t launch_stream_f16(const StreamParams &sp, int ct, int maps, int grid,
                              size_t smem, cudaStream_t st)
{
    return launch_stream_t<__half>(sp, ct, maps, grid, smem, st);
}

}  // namespace iqa

IQA_VIOLATION_READER(iqa_read_violations_stream_f16)
