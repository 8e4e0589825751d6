// iqa_internal.h -- host-side declarations shared by the library's translation
// units (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>

#include "iqa_device.cuh"

namespace iqa {

// One launch shape of the tile kernel.  Derived quantities: RH = NT / S,
// LPT = NT / vec, LPU = TX * LPT.
struct TileConfig {
    int threads = 256;  // 128, 256 or 512
    int ilp = 4;        // 2, 4 or 8 vectors of each image in flight per thread
    int vec = 0;        // elements per load: the full 16-byte vector, or 1
    int TX = 1;         // whole tiles across a unit
    int S = 1;          // CTAs per tile (cluster along y), 1..8
};

enum MapsMask { MAPS_A = 1, MAPS_B = 2, MAPS_AB = 3 };

constexpr int kMaxTX = 64;
constexpr int kMaxCluster = 8;

// Launch the tile kernel for tile rows [p.tile_row0, p.tile_row0 + rows).
// `maps` says which numerator sums are formed (MapsMask).  Defined once per
// storage type in iqa_tiles_<type>.cu.
cudaError_t launch_tiles_f32(const TileArgs &p, const TileConfig &c, int maps,
                             int rows, cudaStream_t st);
cudaError_t launch_tiles_f16(const TileArgs &p, const TileConfig &c, int maps,
                             int rows, cudaStream_t st);
cudaError_t launch_tiles_bf16(const TileArgs &p, const TileConfig &c, int maps,
                              int rows, cudaStream_t st);

}  // namespace iqa
