// iqa_merge.cu -- Eq. 3 / Eq. 4 (arxiv 2501.10653, Section 3): the LISI and
// augLISI of larger tiles formed by merging m x m blocks of tiles, up to the
// whole image, rebuilt from the per-tile sums without re-reading any pixel.
//
// Eq. 3 multiplies each lisi_t by (max(Sx_t, Sy_t) + C2), which by Eq. 1 is
// D * A_t; Eq. 4 multiplies each auglisi_t by (Sx_t + Sy_t + C), which by Eq. 2
// is Sx_t + Sy_t + C - B_t, and removes the (n - 1) extra C.  Both therefore
// equal Eq. 1 / Eq. 2 applied to the block's summed (A, B, Sx, Sy); the kernels
// sum the four per-tile sums of each block in FP64, in an order fixed by the
// launch shape (so results repeat bit for bit), and apply Eq. 1 / Eq. 2 once.
//
// The work is m^2 tiles of 32 bytes per merged tile, so the launch shape
// follows m: one thread per merged tile for small blocks, one warp for
// middling ones, and for large blocks (up to the whole image) a cluster of
// kClusterCtas CTAs whose partial sums meet in distributed shared memory.
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include "iqa.h"
#include "iqa_ctx.h"

namespace cg = cooperative_groups;

namespace iqa {

constexpr int kMergeThreads = 256;
constexpr int kClusterCtas = 8;
constexpr long long kThreadMaxTiles = 16;    // m^2 <= 16: one thread per merged tile
constexpr long long kWarpMaxTiles = 8192;    // m^2 <= 8192: one warp per merged tile

struct MergeArgs {
    const double *sums;
    int T, m, M;  // tiles per row, merge factor, merged tiles per row
    double C2, C, D;
    float *lisi;
    float *aug;
    double *out_sums;
};

__device__ __forceinline__ void add4(double (&s)[4], const double *p)
{
    if (!p) return;
#pragma unroll
    for (int k = 0; k < 4; ++k) s[k] += p[k];
}

// Tile i (row-major) of merged tile b (nullptr, in the checked build, for an
// index outside the tile grid).
__device__ __forceinline__ const double *tile_of(const MergeArgs &a, long long b, long long i)
{
    const long long R = b / a.M, Cc = b - R * a.M;
    const long long r = R * a.m + i / a.m, c = Cc * a.m + i % a.m;
    if (!IQA_CHECK(r < a.T && c < a.T && b < (long long)a.M * a.M)) return nullptr;
    return a.sums + 4 * (r * a.T + c);
}

__device__ __forceinline__ void write_merged(const MergeArgs &a, long long b, const double (&t)[4])
{
    const double A = t[0], B = t[1], Sx = t[2], Sy = t[3];
    if (a.lisi) a.lisi[b] = (float)(a.D * A / (fmax(Sx, Sy) + a.C2));
    if (a.aug) a.aug[b] = (float)(1.0 - B / (Sx + Sy + a.C));
    if (a.out_sums) {
        double *o = a.out_sums + 4 * b;
        o[0] = A;
        o[1] = B;
        o[2] = Sx;
        o[3] = Sy;
    }
}

// Programmatic dependent launch: the next kernel in the stream may be
// scheduled as this grid drains, and this one waits for the previous grid
// (which wrote the per-tile sums) before its first read.
__device__ __forceinline__ void pdl_enter()
{
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");
}

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// m^2 <= kThreadMaxTiles: thread b sums its block's tiles row by row.
__global__ void __launch_bounds__(kMergeThreads) iqa_merge_thread_kernel(MergeArgs a)
{
    pdl_enter();
    const long long b = (long long)blockIdx.x * kMergeThreads + threadIdx.x;
    if (b >= (long long)a.M * a.M) return;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    const long long n = (long long)a.m * a.m;
    for (long long i = 0; i < n; ++i) add4(s, tile_of(a, b, i));
    write_merged(a, b, s);
}

// m^2 <= kWarpMaxTiles: warp b takes its block's tiles lane-strided, then an
// xor-shuffle tree.
__global__ void __launch_bounds__(kMergeThreads) iqa_merge_warp_kernel(MergeArgs a)
{
    pdl_enter();
    const int lane = threadIdx.x & 31;
    const long long b = ((long long)blockIdx.x * kMergeThreads + threadIdx.x) >> 5;
    if (b >= (long long)a.M * a.M) return;  // whole warps leave together
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    const long long n = (long long)a.m * a.m;
    for (long long i = lane; i < n; i += 32) add4(s, tile_of(a, b, i));
#pragma unroll
    for (int k = 0; k < 4; ++k) s[k] = warp_sum_d(s[k]);
    if (lane == 0) write_merged(a, b, s);
}

// Larger blocks: cluster b (kClusterCtas CTAs) takes merged tile b; CTA rank
// q sums the tiles i = q * kMergeThreads + tid + j * kClusterCtas *
// kMergeThreads, reduces them in shared memory, and rank 0 adds the ranks'
// partials in rank order through distributed shared memory.
__global__ void __launch_bounds__(kMergeThreads) iqa_merge_cluster_kernel(MergeArgs a)
{
    __shared__ double red[4][kMergeThreads / 32];
    __shared__ double part[4];
    pdl_enter();
    cg::cluster_group cluster = cg::this_cluster();
    const int q = (int)cluster.block_rank();
    const long long b = blockIdx.x / kClusterCtas;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    const long long n = (long long)a.m * a.m;
    const long long step = (long long)kClusterCtas * kMergeThreads;
    for (long long i = (long long)q * kMergeThreads + threadIdx.x; i < n; i += step)
        add4(s, tile_of(a, b, i));
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const double v = warp_sum_d(s[k]);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int w = 0; w < kMergeThreads / 32; ++w) t += red[threadIdx.x][w];
        part[threadIdx.x] = t;
    }
    cluster.sync();
    if (q == 0 && threadIdx.x == 0) {
        double t[4] = {0.0, 0.0, 0.0, 0.0};
        for (int r = 0; r < kClusterCtas; ++r) {
            const double *rp = cluster.map_shared_rank(part, r);
#pragma unroll
            for (int k = 0; k < 4; ++k) t[k] += rp[k];
        }
        write_merged(a, b, t);
    }
    cluster.sync();  // keep every rank's shared memory alive until read
}

}  // namespace iqa

IQA_VIOLATION_READER(iqa_read_violations_merge)

using namespace iqa;

extern "C" iqa_status iqa_merge(iqa_ctx *ctx, const double *sums, int T, int m,
                                const iqa_params *params, float *merged_lisi,
                                float *merged_aug, double *merged_sums, iqa_stream stream)
{
    if (!ctx) return IQA_ERR_INVALID_ARG;
    if (!sums || (!merged_lisi && !merged_aug && !merged_sums)) {
        set_error(ctx, "need per-tile sums and at least one output");
        return IQA_ERR_INVALID_ARG;
    }
    if (T < 1 || m < 1 || m > T || T % m) {
        set_error(ctx, "need 1 <= m <= T with m dividing T (T=%d, m=%d)", T, m);
        return IQA_ERR_INVALID_ARG;
    }
    const long long M = T / m;
    const long long n = (long long)m * m;
    if (M * M * kClusterCtas > 0x7fffffffLL) {
        set_error(ctx, "too many merged tiles");
        return IQA_ERR_UNSUPPORTED;
    }
    iqa_params P;
    iqa_status s = resolve_params(ctx, params, &P);
    if (s != IQA_OK) return s;
    MergeArgs a{sums, T, m, (int)M, P.C2, P.C, P.D, merged_lisi, merged_aug, merged_sums};
    cudaStream_t st = (cudaStream_t)stream;
    // every shape launches with programmatic stream serialization (see
    // pdl_enter); the cluster shape adds its cluster dimension
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[2];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.blockDim = dim3(kMergeThreads);
    cfg.stream = st;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    cudaError_t e;
    if (n <= kThreadMaxTiles) {
        cfg.gridDim = dim3((unsigned)((M * M + kMergeThreads - 1) / kMergeThreads));
        e = cudaLaunchKernelEx(&cfg, iqa_merge_thread_kernel, a);
    } else if (n <= kWarpMaxTiles) {
        cfg.gridDim = dim3((unsigned)((M * M * 32 + kMergeThreads - 1) / kMergeThreads));
        e = cudaLaunchKernelEx(&cfg, iqa_merge_warp_kernel, a);
    } else {
        cfg.gridDim = dim3((unsigned)(M * M * kClusterCtas));
        attr[1].id = cudaLaunchAttributeClusterDimension;
        attr[1].val.clusterDim.x = kClusterCtas;
        attr[1].val.clusterDim.y = 1;
        attr[1].val.clusterDim.z = 1;
        cfg.numAttrs = 2;
        e = cudaLaunchKernelEx(&cfg, iqa_merge_cluster_kernel, a);
    }
    if (e != cudaSuccess) return cuda_fail(ctx, e, "merge kernel launch");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "merge kernel launch");
    return IQA_OK;
}
