// iqa_tiles_f32.cu -- plain-path tile kernels for float pixel storage.
#include "iqa_tiles.cuh"

namespace iqa {

cudaError_t launch_tiles_f32(const TileArgs &p, const TileConfig &c, int maps,
                             int rows, cudaStream_t st, int *occ)
{
    return launch_tiles_t<float>(p, c, maps, rows, st, occ);
}

}  // namespace iqa

IQA_VIOLATION_READER(iqa_read_violations_tiles_f32)
