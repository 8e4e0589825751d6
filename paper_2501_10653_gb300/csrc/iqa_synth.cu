// iqa_synth.cu -- device-side synthetic sky epochs for the serving loop.
//
// The serving workload keeps reference skies resident and makes each
// request's second epoch on the device from (reference catalogue, seed): the
// catalogue's Gaussian-beam sources, minus the ones the request drops, plus an
// optional transient, over fresh noise.  This is input generation, not part
// of the LISI / augLISI method; it is written so that a host implementation
// (paper_2501_10653_gb300/synth.py, `render_epoch`) reproduces every pixel
// bit for bit:
//   * noise: the Philox4x32-10 counter-based generator (Salmon, Moraes, Dror
//     and Shaw, SC'11) keyed by the seed, one call per pixel with counter
//     (pixel index low, high, 0x5EED, 0); its four words' top 16 bits give four
//     uniforms u_i = w_i >> 16 scaled by 2^-16; z = (u0+u1+u2+u3 - 2) * sqrt(3)
//     (an Irwin-Hall sum of four, unit variance, bounded at +-sqrt(12)); every
//     step is exact except the final multiply;
//   * sources: each source i has an integer centre (x_i, y_i), a peak flux f_i
//     and a 1-D float32 profile g_i[-h_i..h_i] computed on the host; its
//     contribution to pixel (r, c) is (f_i * g_i[r - y_i]) * g_i[c - x_i],
//     added to the pixel in catalogue order;
//   * pixel = sky + sigma * z, then rounded to nearest into the storage type.
// All float operations use explicitly rounded intrinsics, so no contraction
// into FMA changes the result.
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "iqa_synth.h"

namespace iqa {

// Philox4x32-10 round constants and key increments (published definition).
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = kPhiloxM0 * c.x, hi0 = __umulhi(kPhiloxM0, c.x);
        const uint32_t lo1 = kPhiloxM1 * c.z, hi1 = __umulhi(kPhiloxM1, c.z);
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
        k.x += kPhiloxW0;
        k.y += kPhiloxW1;
    }
    return c;
}

__device__ __forceinline__ float noise_z(unsigned long long pixel, unsigned long long seed)
{
    const uint4 w = philox4x32_10(
        make_uint4((uint32_t)pixel, (uint32_t)(pixel >> 32), 0x5EEDu, 0u),
        make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    const float scale = 1.0f / 65536.0f;
    float s = __fmul_rn((float)(w.x >> 16), scale);
    s = __fadd_rn(s, __fmul_rn((float)(w.y >> 16), scale));
    s = __fadd_rn(s, __fmul_rn((float)(w.z >> 16), scale));
    s = __fadd_rn(s, __fmul_rn((float)(w.w >> 16), scale));
    return __fmul_rn(__fadd_rn(s, -2.0f), 1.7320508075688772f);
}

template <typename T> __device__ __forceinline__ T to_storage(float v);
template <> __device__ __forceinline__ float to_storage<float>(float v) { return v; }
template <> __device__ __forceinline__ __half to_storage<__half>(float v)
{
    return __float2half_rn(v);
}
template <> __device__ __forceinline__ __nv_bfloat16 to_storage<__nv_bfloat16>(float v)
{
    return __float2bfloat16_rn(v);
}

__device__ __forceinline__ bool is_dropped(const SynthJob &j, int src)
{
    for (int k = 0; k < j.ndrop; ++k)
        if (j.drop[k] == src) return true;
    return false;
}

// One thread per pixel, blocks of kSynthBlock x kSynthBlock pixels.  A block
// lies inside one catalogue bin (bins are kSynthBin pixels square), whose
// source list (in catalogue order) it walks for every pixel.  Jobs are read
// from the device table; `blocks_begin` gives each job's first block.
template <typename T>
__global__ void __launch_bounds__(kSynthBlock *kSynthBlock)
    iqa_synth_kernel(const SynthJob *__restrict__ jobs, const long long *__restrict__ header)
{
    const int njobs = (int)header[0];
    const long long total_blocks = header[1];
    for (long long b = blockIdx.x; b < total_blocks; b += gridDim.x) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].blocks_begin <= b) lo = mid;
            else hi = mid - 1;
        }
        const SynthJob &j = jobs[lo];
        const long long lb = b - j.blocks_begin;
        const int bpr = j.N / kSynthBlock;
        const int r = (int)(lb / bpr) * kSynthBlock + threadIdx.x / kSynthBlock;
        const int c = (int)(lb % bpr) * kSynthBlock + threadIdx.x % kSynthBlock;
        const SynthCatalog &cat = *j.cat;
        const int bin = (r / kSynthBin) * cat.bins_per_row + (c / kSynthBin);
        float sky = 0.0f;
        for (int q = cat.bin_start[bin]; q < cat.bin_start[bin + 1]; ++q) {
            const int i = cat.bin_src[q];
            const int h = cat.half[i];
            const int dy = r - cat.y[i], dx = c - cat.x[i];
            if (dy < -h || dy > h || dx < -h || dx > h) continue;
            if (is_dropped(j, i)) continue;
            const float *g = cat.profile + cat.profile_off[i] + h;
            sky = __fadd_rn(sky, __fmul_rn(__fmul_rn(cat.flux[i], g[dy]), g[dx]));
        }
        if (j.add_src >= 0) {
            const int i = j.add_src;
            const int h = cat.half[i];
            const int dy = r - j.add_y, dx = c - j.add_x;
            if (dy >= -h && dy <= h && dx >= -h && dx <= h) {
                const float *g = cat.profile + cat.profile_off[i] + h;
                sky = __fadd_rn(sky, __fmul_rn(__fmul_rn(j.add_flux, g[dy]), g[dx]));
            }
        }
        const unsigned long long pix = (unsigned long long)r * j.N + c;
        const float v = __fadd_rn(sky, __fmul_rn(cat.noise_sigma, noise_z(pix, j.seed)));
        static_cast<T *>(j.out)[pix] = to_storage<T>(v);
    }
}

cudaError_t launch_synth(int dtype, const SynthJob *jobs, const long long *header, int grid,
                         cudaStream_t st)
{
    const dim3 block(kSynthBlock * kSynthBlock);
    switch (dtype) {
    case 0: iqa_synth_kernel<float><<<grid, block, 0, st>>>(jobs, header); break;
    case 1: iqa_synth_kernel<__half><<<grid, block, 0, st>>>(jobs, header); break;
    default: iqa_synth_kernel<__nv_bfloat16><<<grid, block, 0, st>>>(jobs, header); break;
    }
    return cudaGetLastError();
}

}  // namespace iqa
