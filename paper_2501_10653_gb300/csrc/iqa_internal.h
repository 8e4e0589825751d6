// iqa_internal.h -- host-side declarations shared by the library's translation
// units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include "iqa_device.cuh"

namespace iqa {

// One launch shape.  variant 0 (iqa_tiles_kernel): RH = NT / S,
// LPT = NT / vec, LPU = TX * LPT.  variant 1 (iqa_stream_kernel): threads =
// consumer threads, TX tiles per unit, a ring of `stages` stages of
// stage_kb KB per image, ctas_per_sm persistent CTAs per SM.
struct TileConfig {
    int variant = 0;
    int threads = 256;  // 128, 256 or 512
    int ilp = 4;        // 2, 4 or 8 vectors of each image in flight per thread
    int vec = 0;        // elements per load: the full 16-byte vector, or 1
    int TX = 1;         // whole tiles across a unit
    int RH = 1;         // variant 1: tile rows down a unit
    int S = 1;          // CTAs per tile (cluster along y), 1..8
    int stages = 8;
    int stage_kb = 8;
    int ctas_per_sm = 1;
    int unit_kpx = 16;  // variant 1, batched: target unit size in K pixel pairs
};

enum MapsMask { MAPS_A = 1, MAPS_B = 2, MAPS_AB = 3 };

constexpr int kMaxTX = 64;
constexpr int kMaxCluster = 8;

// Launch the tile kernel for tile rows [p.tile_row0, p.tile_row0 + rows).
// `maps` says which numerator sums are formed (MapsMask).  With occ non-null
// nothing is launched: *occ receives how many CTAs of that kernel fit one SM.
// Defined once per storage type in iqa_tiles_<type>.cu.
cudaError_t launch_tiles_f32(const TileArgs &p, const TileConfig &c, int maps,
                             int rows, cudaStream_t st, int *occ);
cudaError_t launch_tiles_f16(const TileArgs &p, const TileConfig &c, int maps,
                             int rows, cudaStream_t st, int *occ);
cudaError_t launch_tiles_bf16(const TileArgs &p, const TileConfig &c, int maps,
                              int rows, cudaStream_t st, int *occ);

struct StreamParams;
cudaError_t launch_stream_f32(const StreamParams &sp, int ct, int maps, int grid,
                              size_t smem, cudaStream_t st);
cudaError_t launch_stream_f16(const StreamParams &sp, int ct, int maps, int grid,
                              size_t smem, cudaStream_t st);
cudaError_t launch_stream_bf16(const StreamParams &sp, int ct, int maps, int grid,
                               size_t smem, cudaStream_t st);

}  // namespace iqa
