// iqa_tiles.cuh -- the plain-path kernel: one launch computes the LISI (Eq. 1)
// and/or augLISI (Eq. 2) map of one image pair, reading every pixel once.
//
// Grid: x = unit column (TX whole tiles each), y = tile row * S + part, where a
// tile taller than one unit is split over S CTAs that form a thread-block
// cluster along y; the S partial sums meet in distributed shared memory and
// the cluster's rank-0 CTA writes the tile.  Launched with programmatic
// dependent launch: every CTA waits for the previous grid in the stream before
// its first access.  Included once per storage type.
#pragma once

#include <cooperative_groups.h>

#include "iqa_internal.h"

namespace iqa {

namespace cg = cooperative_groups;

template <typename T, int VEC, int ILP, int THREADS, bool DO_A, bool DO_B, bool OVERLAP>
__global__ void __launch_bounds__(THREADS)
    iqa_tiles_kernel(const TileArgs p)
{
    __shared__ float red[4][THREADS];
    __shared__ float part[kMaxTX * 4];

    // programmatic dependent launch: let the next kernel in the stream be
    // scheduled as this grid drains, and wait for the previous one (which may
    // have written these images or maps) before the first access -- or, for
    // an independent call (OVERLAP), only before the first write, so the
    // loads stream while that kernel drains
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    if constexpr (!OVERLAP) asm volatile("griddepcontrol.wait;" ::: "memory");

    const int tile_col0 = blockIdx.x * p.TX;
    const int srank = blockIdx.y % p.S;
    const int tile_row = p.tile_row0 + blockIdx.y / p.S;
    const long long row0 = (long long)tile_row * p.NT + (long long)srank * p.RH;
    const long long col0 = (long long)tile_col0 * p.NT;
    const T *xu = static_cast<const T *>(p.x) + row0 * p.N + col0;
    const T *yu = static_cast<const T *>(p.y) + row0 * p.N + col0;

    float acc[4] = {0.0f, 0.0f, 0.0f, 0.0f};
    // the unit lies inside the image (checked build only)
    if (IQA_CHECK(tile_row < p.T && row0 + p.RH <= p.N &&
                  col0 + (long long)p.TX * p.NT <= p.N && p.LPU * VEC == p.TX * p.NT))
        accumulate_unit<T, VEC, ILP, THREADS, DO_A, DO_B>(xu, yu, p.N, p.RH, p.LPU,
                                                          p.C1f, acc);
    reduce_unit<THREADS>(acc, p.TX, p.LPU, p.LPT, red, part, CtaBarrier());
    if constexpr (OVERLAP) asm volatile("griddepcontrol.wait;" ::: "memory");

    const long long t0 = (long long)tile_row * p.T + tile_col0;
    const bool out_ok = IQA_CHECK(t0 + p.TX <= (long long)p.T * p.T && p.TX <= kMaxTX);
    if (p.S == 1) {
        for (int tl = threadIdx.x; tl < p.TX && out_ok; tl += THREADS)
            write_tile(p, t0 + tl, part[tl * 4 + 0], part[tl * 4 + 1],
                       part[tl * 4 + 2], part[tl * 4 + 3]);
        return;
    }
    // S > 1: the CTAs of this tile form one cluster; combine in rank order.
    cg::cluster_group cluster = cg::this_cluster();
    cluster.sync();
    if (cluster.block_rank() == 0 && out_ok) {
        for (int tl = threadIdx.x; tl < p.TX; tl += THREADS) {
            float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            for (int r = 0; r < p.S; ++r) {
                const float *rp = cluster.map_shared_rank(part, r);
#pragma unroll
                for (int k = 0; k < 4; ++k) s[k] += rp[tl * 4 + k];
            }
            write_tile(p, t0 + tl, s[0], s[1], s[2], s[3]);
        }
    }
    // keep every CTA's shared memory alive until rank 0 has read it
    cluster.sync();
}

// Launches the kernel, or, with occ non-null, stores the number of its CTAs
// that fit one SM at once (no launch).  An independent call (p.overlap) runs
// the OVERLAP instantiation, which only the 16-byte vector paths have; the
// stream-ordered kernels compile exactly as they would without it.
template <typename T, int VEC, int ILP, int THREADS, bool DO_A, bool DO_B, bool OVERLAP>
static cudaError_t launch_one(const TileArgs &p, int rows, cudaStream_t st, int *occ)
{
    if (occ)
        return cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            occ, iqa_tiles_kernel<T, VEC, ILP, THREADS, DO_A, DO_B, OVERLAP>, THREADS, 0);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(p.T / p.TX), (unsigned)(rows * p.S), 1);
    cfg.blockDim = dim3(THREADS, 1, 1);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    if (p.S > 1) {
        attr[1].id = cudaLaunchAttributeClusterDimension;
        attr[1].val.clusterDim.x = 1;
        attr[1].val.clusterDim.y = (unsigned)p.S;
        attr[1].val.clusterDim.z = 1;
        cfg.numAttrs = 2;
    }
    return cudaLaunchKernelEx(&cfg, iqa_tiles_kernel<T, VEC, ILP, THREADS, DO_A, DO_B, OVERLAP>,
                              p);
}

template <typename T, int VEC, int ILP, int THREADS, bool OVERLAP>
static cudaError_t by_maps_o(const TileArgs &p, int maps, int rows, cudaStream_t st, int *occ)
{
    switch (maps) {
    case MAPS_A: return launch_one<T, VEC, ILP, THREADS, true, false, OVERLAP>(p, rows, st, occ);
    case MAPS_B: return launch_one<T, VEC, ILP, THREADS, false, true, OVERLAP>(p, rows, st, occ);
    default: return launch_one<T, VEC, ILP, THREADS, true, true, OVERLAP>(p, rows, st, occ);
    }
}

template <typename T, int VEC, int ILP, int THREADS>
static cudaError_t by_maps(const TileArgs &p, int maps, int rows, cudaStream_t st, int *occ)
{
    if (VEC > 1 && p.overlap) return by_maps_o<T, VEC, ILP, THREADS, true>(p, maps, rows, st, occ);
    return by_maps_o<T, VEC, ILP, THREADS, false>(p, maps, rows, st, occ);
}

template <typename T, int VEC, int ILP>
static cudaError_t by_threads(const TileArgs &p, const TileConfig &c, int maps,
                              int rows, cudaStream_t st, int *occ)
{
    switch (c.threads) {
    case 128: return by_maps<T, VEC, ILP, 128>(p, maps, rows, st, occ);
    case 256: return by_maps<T, VEC, ILP, 256>(p, maps, rows, st, occ);
    case 512: return by_maps<T, VEC, ILP, 512>(p, maps, rows, st, occ);
    default: return cudaErrorInvalidValue;
    }
}

template <typename T>
static cudaError_t launch_tiles_t(const TileArgs &p, const TileConfig &c,
                                  int maps, int rows, cudaStream_t st, int *occ)
{
    constexpr int V = Elem<T>::VEC;
    if (c.vec == 1) {
        // scalar path for unaligned images or tiles that are not a whole
        // number of 16-byte vectors wide: one launch shape only
        if (c.threads != 256 || c.ilp != 8) return cudaErrorInvalidValue;
        return by_maps<T, 1, 8, 256>(p, maps, rows, st, occ);
    }
    if (c.vec != V) return cudaErrorInvalidValue;
    switch (c.ilp) {
    case 2: return by_threads<T, V, 2>(p, c, maps, rows, st, occ);
    case 4: return by_threads<T, V, 4>(p, c, maps, rows, st, occ);
    case 8: return by_threads<T, V, 8>(p, c, maps, rows, st, occ);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace iqa
