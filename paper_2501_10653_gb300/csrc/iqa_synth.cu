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
//     and Shaw, SC'11) keyed by the seed, one call per four horizontally
//     adjacent pixels with counter (q low, q high, 0x5EED, 0), q = pixel
//     index / 4; word k serves pixel 4q + k: its four bytes, summed as
//     integers to s in [0, 1020], give z = (s - 510) * (sqrt(3) / 256) (an
//     Irwin-Hall sum of four uniforms on the byte centres (b + 1/2) / 256:
//     zero mean, variance 1 - 2^-16, bounded at +-sqrt(12)); the only
//     rounding is the final multiply;
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

#include "iqa_device.cuh"
#include "iqa_synth.h"

namespace iqa {

// Philox4x32-10 round constants and key increments (published definition).
constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

// M independent counters under one key, rounds interleaved: the key schedule
// is shared and the M multiply chains overlap.  Each round multiplies the
// counter's words 0 and 2 by the round constants (one 32 x 32 -> 64-bit
// product each), swaps and XORs the high halves with the other two words and
// the round key, then bumps the key by the Weyl constants.
template <int M>
__device__ __forceinline__ void philox4x32_10(uint4 (&c)[M], uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
#pragma unroll
        for (int i = 0; i < M; ++i) {
            const unsigned long long p0 = (unsigned long long)kPhiloxM0 * c[i].x;
            const unsigned long long p1 = (unsigned long long)kPhiloxM1 * c[i].z;
            c[i] = make_uint4((uint32_t)(p1 >> 32) ^ c[i].y ^ k.x, (uint32_t)p1,
                              (uint32_t)(p0 >> 32) ^ c[i].w ^ k.y, (uint32_t)p0);
        }
        k.x += kPhiloxW0;
        k.y += kPhiloxW1;
    }
}

// Irwin-Hall sum of the four bytes of one Philox word, standardised:
// z = (b0 + b1 + b2 + b3 - 510) * sqrt(3) / 256; the integer is exact in
// float, so the final multiply is the only rounding.
constexpr float kNoiseScale = 1.7320508075688772f / 256.0f;  // exact: a power-of-2 step

// The byte sum s of a word is one four-way byte dot product with (1,1,1,1),
// accumulated onto 0x4B000000: the bits of the float 2^23 + s (s < 2^23),
// so s - 510 comes out exactly in float by subtracting 2^23 + 510, with no
// conversion instruction and no integer-pipe work (the generator is bound
// by the integer pipe, which the Philox rounds already load).
__device__ __forceinline__ float irwin_hall4_bytes(uint32_t w)
{
    const uint32_t biased = __dp4a(w, 0x01010101u, 0x4B000000u);
    return __fmul_rn(__fsub_rn(__uint_as_float(biased), 8389118.0f), kNoiseScale);  // 2^23 + 510
}

// Standardised noise of M quads of horizontally adjacent pixels 4q .. 4q+3
// (q = pixel index / 4): one Philox call per quad, word k for pixel 4q + k.
template <int M>
__device__ __forceinline__ void noise_quads(const unsigned long long (&q)[M],
                                            unsigned long long seed, float4 (&z)[M])
{
    uint4 w[M];
#pragma unroll
    for (int i = 0; i < M; ++i)
        w[i] = make_uint4((uint32_t)q[i], (uint32_t)(q[i] >> 32), 0x5EEDu, 0u);
    philox4x32_10<M>(w, make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
#pragma unroll
    for (int i = 0; i < M; ++i)
        z[i] = make_float4(irwin_hall4_bytes(w[i].x), irwin_hall4_bytes(w[i].y),
                           irwin_hall4_bytes(w[i].z), irwin_hall4_bytes(w[i].w));
}

// Four consecutive pixels rounded to nearest into the storage type and
// written with one vector store (16 bytes for FP32, 8 for 16-bit types; the
// first pixel index is a multiple of 4 and the image 16-byte aligned).
template <typename T> __device__ __forceinline__ void store4(T *out, const float (&v)[4]);
template <> __device__ __forceinline__ void store4<float>(float *out, const float (&v)[4])
{
    *reinterpret_cast<float4 *>(out) = make_float4(v[0], v[1], v[2], v[3]);
}
template <> __device__ __forceinline__ void store4<__half>(__half *out, const float (&v)[4])
{
    const __half2 a = __halves2half2(__float2half_rn(v[0]), __float2half_rn(v[1]));
    const __half2 b = __halves2half2(__float2half_rn(v[2]), __float2half_rn(v[3]));
    uint2 u;
    u.x = *reinterpret_cast<const uint32_t *>(&a);
    u.y = *reinterpret_cast<const uint32_t *>(&b);
    *reinterpret_cast<uint2 *>(out) = u;
}
template <>
__device__ __forceinline__ void store4<__nv_bfloat16>(__nv_bfloat16 *out, const float (&v)[4])
{
    const __nv_bfloat162 a =
        __halves2bfloat162(__float2bfloat16_rn(v[0]), __float2bfloat16_rn(v[1]));
    const __nv_bfloat162 b =
        __halves2bfloat162(__float2bfloat16_rn(v[2]), __float2bfloat16_rn(v[3]));
    uint2 u;
    u.x = *reinterpret_cast<const uint32_t *>(&a);
    u.y = *reinterpret_cast<const uint32_t *>(&b);
    *reinterpret_cast<uint2 *>(out) = u;
}

__device__ __forceinline__ bool is_dropped(const SynthJob &j, int src)
{
    for (int k = 0; k < j.ndrop; ++k)
        if (j.drop[k] == src) return true;
    return false;
}

// Work unit: one catalogue bin (kSynthBin x kSynthBin pixels) of one job per
// block iteration; thread t takes the four columns 4 (t % 16) .. 4 (t % 16) + 3
// of rows t / 16 + 8k, k < 8 (one Philox call and one vector store per four
// pixels, in two batches of four rows), so each warp writes two 64-pixel row
// segments per step and a bin's fixed cost (job and catalogue fields, bin
// index, source staging, barriers) is paid once per 32 pixels of a thread.
// The jobs' first-bin offsets live in shared memory (looked up once per bin),
// and so do the bin's sources (in catalogue order, the order every pixel adds
// them in).
constexpr int kSynthThreads = 128;
constexpr int kSynthMaxJobs = 64;
constexpr int kSynthBinSrc = 64;  // bin sources staged in shared memory
constexpr int kQuadsPerRow = kSynthBin / 4;

// Adds one source's contribution (f * g[dy]) * g[dx] to the four pixels
// (r, c .. c+3), for the pixels inside its window.
__device__ __forceinline__ void add_source(float (&sky)[4], const float *g0, int h, int dy,
                                           int dx0, float f)
{
    if (dy < -h || dy > h || dx0 + 3 < -h || dx0 > h) return;
    const float *g = g0 + h;
    const float fy = __fmul_rn(f, g[dy]);
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int dx = dx0 + k;
        if (dx >= -h && dx <= h) sky[k] = __fadd_rn(sky[k], __fmul_rn(fy, g[dx]));
    }
}

template <typename T>
__global__ void __launch_bounds__(kSynthThreads, kSynthBlocksPerSM)
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
    const int lc = 4 * (threadIdx.x % kQuadsPerRow);  // first column within the bin
    const int lr0 = threadIdx.x / kQuadsPerRow;       // first row within the bin
    constexpr int kRowStep = kSynthThreads / kQuadsPerRow;
    for (long long b = blockIdx.x; b < total_bins; b += gridDim.x) {
        int lo = 0, hi = njobs - 1;
        while (lo < hi) {
            int mid = (lo + hi + 1) >> 1;
            if (s_begin[mid] <= b) lo = mid;
            else hi = mid - 1;
        }
        // the job's and catalogue's fields in registers (the image stores
        // below could otherwise alias them and force reloads)
        const SynthJob &j = jobs[lo];
        const SynthCatalog &cat = *j.cat;
        const int N = j.N;
        const unsigned long long seed = j.seed;
        T *const out = static_cast<T *>(j.out);
        const float *const prof = cat.profile;
        const float sigma = cat.noise_sigma;
        // bin within the job (catalogues have N <= 2^20, so fewer than 2^28
        // bins: a 32-bit division, not the much longer 64-bit routine)
        const int lb = (int)(b - s_begin[lo]);
        const int bpr = cat.bins_per_row;
        const int br = lb / bpr, bc = lb - br * bpr;
        const int bin = br * bpr + bc;
        const int r0 = br * kSynthBin, c0 = bc * kSynthBin;
        // the transient, when its window meets this bin
        const int tsrc = j.add_src;
        const float *tg = prof;
        int th = -1, tx = 0, ty = 0;
        float tf = 0.0f;
        if (tsrc >= 0) {
            th = cat.half[tsrc];
            tg = prof + cat.profile_off[tsrc];
            tx = j.add_x;
            ty = j.add_y;
            tf = j.add_flux;
            if (ty + th < r0 || ty - th >= r0 + kSynthBin || tx + th < c0 ||
                tx - th >= c0 + kSynthBin)
                th = -1;
        }
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
        // the noise of the thread's first batch of quads (it does not depend on
        // the sources, so it overlaps their staging)
        const int c = c0 + lc;
        constexpr int kQuads = kSynthBin / kRowStep;  // rows of a thread in a bin
        constexpr int kBatch = 4;                     // Philox calls interleaved
        float4 zq[kBatch];
        const auto batch_noise = [&](int k0) {
            unsigned long long q[kBatch];
#pragma unroll
            for (int k = 0; k < kBatch; ++k)
                q[k] = ((unsigned long long)(r0 + lr0 + (k0 + k) * kRowStep) * N + c) >> 2;
            noise_quads<kBatch>(q, seed, zq);
        };
        batch_noise(0);
        __syncthreads();
        const int n = s_n;
        // the batches are not unrolled: one copy of the row body keeps the
        // kernel within the instruction cache
#pragma unroll 1
        for (int k0 = 0; k0 < kQuads; k0 += kBatch) {
            if (k0 > 0) batch_noise(k0);
#pragma unroll
            for (int k = 0; k < kBatch; ++k) {
                const int r = r0 + lr0 + (k0 + k) * kRowStep;
                const unsigned long long pix = (unsigned long long)r * N + c;
                const float4 z = zq[k];
                float sky[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                for (int m = 0; m < n; ++m)
                    add_source(sky, prof + s_off[m], s_h[m], r - s_y[m], c - s_x[m], s_f[m]);
                if (th >= 0) add_source(sky, tg, th, r - ty, c - tx, tf);
                const float v[4] = {__fadd_rn(sky[0], __fmul_rn(sigma, z.x)),
                                    __fadd_rn(sky[1], __fmul_rn(sigma, z.y)),
                                    __fadd_rn(sky[2], __fmul_rn(sigma, z.z)),
                                    __fadd_rn(sky[3], __fmul_rn(sigma, z.w))};
                // the four pixels lie in the job's image (checked build only)
                if (IQA_CHECK(r < N && c + 3 < N && pix + 3 < (unsigned long long)N * N))
                    store4<T>(out + pix, v);
            }
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

IQA_VIOLATION_READER(iqa_read_violations_synth)
