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
//     and Shaw, SC'11) keyed by the seed, one call per pair of horizontally
//     adjacent pixels with counter (q low, q high, 0x5EED, 0), q = pixel
//     index / 2; words 0-1 serve the even pixel and words 2-3 the odd one, each
//     word giving two 16-bit uniforms (high half, low half) scaled by 2^-16;
//     z = (u0+u1+u2+u3 - 2) * sqrt(3) (an Irwin-Hall sum of four, unit
//     variance, bounded at +-sqrt(12)); every step is exact except the final
//     multiply;
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

// Irwin-Hall sum of four 16-bit uniforms: z = (u0+u1+u2+u3 - 2) * sqrt(3).
__device__ __forceinline__ float irwin_hall4(uint32_t a, uint32_t b)
{
    const float scale = 1.0f / 65536.0f;
    float s = __fmul_rn((float)(a >> 16), scale);
    s = __fadd_rn(s, __fmul_rn((float)(a & 0xFFFFu), scale));
    s = __fadd_rn(s, __fmul_rn((float)(b >> 16), scale));
    s = __fadd_rn(s, __fmul_rn((float)(b & 0xFFFFu), scale));
    return __fmul_rn(__fadd_rn(s, -2.0f), 1.7320508075688772f);
}

// Standardised noise of the two horizontally adjacent pixels 2q, 2q+1 (q =
// pixel index / 2): one Philox call, words (0, 1) for the even pixel and
// (2, 3) for the odd one.
__device__ __forceinline__ float2 noise_pair(unsigned long long q, unsigned long long seed)
{
    const uint4 w = philox4x32_10(make_uint4((uint32_t)q, (uint32_t)(q >> 32), 0x5EEDu, 0u),
                                  make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
    return make_float2(irwin_hall4(w.x, w.y), irwin_hall4(w.z, w.w));
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

// Work unit: one catalogue bin (kSynthBin x kSynthBin pixels) of one job per
// block iteration; thread t takes the column pair 2 (t % 32), 2 (t % 32) + 1
// of rows t / 32 + 8k, k < 8 (one Philox call per pair), so each warp writes
// 64 consecutive pixels per step.  The jobs' first-bin offsets live in shared
// memory (looked up once per bin), and so do the bin's sources (in catalogue
// order, the order every pixel adds them in).
constexpr int kSynthThreads = 256;
constexpr int kSynthMaxJobs = 64;
constexpr int kSynthBinSrc = 64;  // bin sources staged in shared memory

__device__ __forceinline__ float sky_at(const SynthCatalog &cat, const SynthJob &j, int n,
                                        const int *s_x, const int *s_y, const int *s_h,
                                        const int *s_off, const float *s_f, int r, int c)
{
    float sky = 0.0f;
    for (int m = 0; m < n; ++m) {
        const int h = s_h[m];
        const int dy = r - s_y[m], dx = c - s_x[m];
        if (dy < -h || dy > h || dx < -h || dx > h) continue;
        const float *g = cat.profile + s_off[m] + h;
        sky = __fadd_rn(sky, __fmul_rn(__fmul_rn(s_f[m], g[dy]), g[dx]));
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
    return sky;
}

template <typename T>
__global__ void __launch_bounds__(kSynthThreads)
    iqa_synth_kernel(const SynthJob *__restrict__ jobs, const long long *__restrict__ header)
{
    __shared__ long long s_begin[kSynthMaxJobs];
    __shared__ int s_x[kSynthBinSrc], s_y[kSynthBinSrc], s_h[kSynthBinSrc], s_off[kSynthBinSrc];
    __shared__ float s_f[kSynthBinSrc];
    __shared__ int s_n;
    const int njobs = (int)header[0];
    const long long total_bins = header[1];
    for (int i = threadIdx.x; i < njobs; i += kSynthThreads) s_begin[i] = jobs[i].blocks_begin;
    __syncthreads();
    const int lc = 2 * (threadIdx.x % (kSynthBin / 2));  // even column within the bin
    const int lr0 = threadIdx.x / (kSynthBin / 2);       // first row within the bin
    constexpr int kRowStep = kSynthThreads / (kSynthBin / 2);
    for (long long b = blockIdx.x; b < total_bins; b += gridDim.x) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (s_begin[mid] <= b) lo = mid;
            else hi = mid - 1;
        }
        const SynthJob &j = jobs[lo];
        const SynthCatalog &cat = *j.cat;
        const long long lb = b - s_begin[lo];
        const int bpr = cat.bins_per_row;
        const int br = (int)(lb / bpr), bc = (int)(lb % bpr);
        const int bin = br * bpr + bc;
        // stage the bin's non-dropped sources (catalogue order kept)
        if (threadIdx.x == 0) {
            const int q0 = cat.bin_start[bin], q1 = cat.bin_start[bin + 1];
            int n = 0;
            for (int q = q0; q < q1 && n < kSynthBinSrc; ++q) {
                const int i = cat.bin_src[q];
                if (is_dropped(j, i)) continue;
                s_x[n] = cat.x[i];
                s_y[n] = cat.y[i];
                s_h[n] = cat.half[i];
                s_off[n] = cat.profile_off[i];
                s_f[n] = cat.flux[i];
                ++n;
            }
            s_n = n;
        }
        __syncthreads();
        const int c = bc * kSynthBin + lc;
        const int n = s_n;
        const float sigma = cat.noise_sigma;
        T *out = static_cast<T *>(j.out);
        for (int k = 0; k < kSynthBin / kRowStep; ++k) {
            const int r = br * kSynthBin + lr0 + k * kRowStep;
            const unsigned long long pix = (unsigned long long)r * j.N + c;
            const float2 z = noise_pair(pix >> 1, j.seed);
            const float v0 = __fadd_rn(sky_at(cat, j, n, s_x, s_y, s_h, s_off, s_f, r, c),
                                       __fmul_rn(sigma, z.x));
            const float v1 = __fadd_rn(sky_at(cat, j, n, s_x, s_y, s_h, s_off, s_f, r, c + 1),
                                       __fmul_rn(sigma, z.y));
            out[pix] = to_storage<T>(v0);
            out[pix + 1] = to_storage<T>(v1);
        }
        __syncthreads();  // s_* are reused by the next bin
    }
}

cudaError_t launch_synth(int dtype, const SynthJob *jobs, const long long *header, int grid,
                         cudaStream_t st)
{
    const dim3 block(kSynthThreads);
    switch (dtype) {
    case 0: iqa_synth_kernel<float><<<grid, block, 0, st>>>(jobs, header); break;
    case 1: iqa_synth_kernel<__half><<<grid, block, 0, st>>>(jobs, header); break;
    default: iqa_synth_kernel<__nv_bfloat16><<<grid, block, 0, st>>>(jobs, header); break;
    }
    return cudaGetLastError();
}

}  // namespace iqa
