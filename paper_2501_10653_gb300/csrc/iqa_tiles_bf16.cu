// iqa_tiles_bf16.cu -- plain-path tile kernels for __nv_bfloat16 pixel storage.
#include "iqa_tiles.cuh"

namespace iqa {

cudaError_t launch_tiles_bf16(const TileArgs &p, const TileConfig &c, int maps,
                             int rows, cudaStream_t st, int *occ)
{
    return launch_tiles_t<__nv_bfloat16>(p, c, maps, rows, st, occ);
}

}  // namespace iqa

IQA_VIOLATION_READER(iqa_read_violations_tiles_bf16)
