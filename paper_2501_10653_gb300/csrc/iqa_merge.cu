// iqa_merge.cu -- Eq. 3 / Eq. 4 (arxiv 2501.10653, Section 3): the LISI and
// augLISI of larger tiles formed by merging m x m blocks of tiles, up to the
// whole image, rebuilt from the per-tile sums without re-reading any pixel.
//
// Eq. 3 multiplies each lisi_t by (max(Sx_t, Sy_t) + C2), which by Eq. 1 is
// D * A_t; Eq. 4 multiplies each auglisi_t by (Sx_t + Sy_t + C), which by Eq. 2
// is Sx_t + Sy_t + C - B_t, and removes the (n - 1) extra C.  Both therefore
// equal Eq. 1 / Eq. 2 applied to the block's summed (A, B, Sx, Sy); the kernel
// sums the four per-tile sums of each block in FP64, in a fixed order, and
// applies Eq. 1 / Eq. 2 once.  The data is tiny (32 bytes per tile), so FP64
// costs nothing here.
#include <cuda_runtime.h>

#include "iqa.h"
#include "iqa_ctx.h"

namespace iqa {

constexpr int kMergeThreads = 256;

__device__ __forceinline__ double warp_sum_d(double v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// One CTA per merged tile: threads stride over the block's m*m tiles (row-
// major), then a shuffle tree and shared memory combine them.
__global__ void __launch_bounds__(kMergeThreads)
    iqa_merge_kernel(const double *__restrict__ sums, int T, int m, double C2, double C,
                     double D, float *__restrict__ lisi, float *__restrict__ aug,
                     double *__restrict__ out_sums)
{
    __shared__ double red[4][kMergeThreads / 32];
    const int M = T / m;
    const int R = blockIdx.x / M, Cc = blockIdx.x % M;
    double s[4] = {0.0, 0.0, 0.0, 0.0};
    const long long count = (long long)m * m;
    for (long long i = threadIdx.x; i < count; i += kMergeThreads) {
        const long long r = (long long)R * m + i / m;
        const long long c = (long long)Cc * m + i % m;
        const double *p = sums + 4 * (r * T + c);
#pragma unroll
        for (int k = 0; k < 4; ++k) s[k] += p[k];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double v = warp_sum_d(s[k]);
        if (lane == 0) red[k][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double t[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            t[k] = 0.0;
            for (int w = 0; w < kMergeThreads / 32; ++w) t[k] += red[k][w];
        }
        const double A = t[0], B = t[1], Sx = t[2], Sy = t[3];
        if (lisi) lisi[blockIdx.x] = (float)(D * A / (fmax(Sx, Sy) + C2));
        if (aug) aug[blockIdx.x] = (float)(1.0 - B / (Sx + Sy + C));
        if (out_sums) {
            double *o = out_sums + 4 * (long long)blockIdx.x;
            o[0] = A;
            o[1] = B;
            o[2] = Sx;
            o[3] = Sy;
        }
    }
}

}  // namespace iqa

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
    if (M * M > 0x7fffffffLL) {
        set_error(ctx, "too many merged tiles");
        return IQA_ERR_UNSUPPORTED;
    }
    iqa_params P;
    iqa_status s = resolve_params(ctx, params, &P);
    if (s != IQA_OK) return s;
    iqa_merge_kernel<<<(unsigned)(M * M), kMergeThreads, 0, (cudaStream_t)stream>>>(
        sums, T, m, P.C2, P.C, P.D, merged_lisi, merged_aug, merged_sums);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "merge kernel launch");
    return IQA_OK;
}
