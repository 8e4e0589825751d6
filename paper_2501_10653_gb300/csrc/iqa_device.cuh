// iqa_device.cuh -- device building blocks of the tile-wise LISI / augLISI maps.
//
// arxiv 2501.10653, Section 2: negative pixels are set to zero, the images are
// cut into N_T x N_T tiles, and each tile reduces, over its clamped pixels,
//   A  = sum |x+y| / (|x-y| + C1)   (numerator sum of Eq. 1)
//   B  = sum |x+y| |x-y|            (numerator sum of Eq. 2)
//   Sx = sum x,  Sy = sum y         (denominators of Eq. 1 and Eq. 2)
// The paper names this pixel summation as the expensive step and gives it one
// thread block per tile with a shared-memory reduction.  Here a CTA streams a
// "unit": a rectangle of RH rows and TX whole tiles across (or, with a cluster
// of S CTAs along y, 1/S of one tile's rows), with 16-byte non-caching loads,
// the clamp and every term fused into that single read, packed f32x2 running
// sums per thread over a pass of vectors, Kahan-compensated across passes, an
// FP32 shuffle-tree / cross-CTA combine, and the per-tile ratios of Eq. 1 /
// Eq. 2 (FP64 where augLISI cancels).
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

// Bounds checks of the checked build (IQA_CHECKS=1, libiqa_checked.so): every
// kernel checks the geometry of what it is about to read or write (unit and
// tile bounds, TMA box coordinates, stage capacity, output indices) with
// IQA_CHECK(cond); a failed check counts one violation in this translation
// unit's device counter and the access is skipped (nothing traps).  In the
// product build IQA_CHECK(cond) is `true` and the condition is not compiled.
#ifndef IQA_CHECKS
#define IQA_CHECKS 0
#endif
#if IQA_CHECKS
static __device__ unsigned int g_iqa_violations;
__device__ __forceinline__ bool iqa_check_ok(bool ok)
{
    if (!ok) atomicAdd(&g_iqa_violations, 1u);
    return ok;
}
#define IQA_CHECK(cond) iqa_check_ok(cond)
// Host reader of this translation unit's counter (read and cleared).
#define IQA_VIOLATION_READER(name)                                                   \
    extern "C" unsigned int name()                                                   \
    {                                                                                \
        unsigned int v = 0, z = 0;                                                   \
        cudaMemcpyFromSymbol(&v, g_iqa_violations, sizeof v);                        \
        cudaMemcpyToSymbol(g_iqa_violations, &z, sizeof z);                          \
        return v;                                                                    \
    }
#else
#define IQA_CHECK(cond) (true)
#define IQA_VIOLATION_READER(name)
#endif

#include <type_traits>

namespace iqa {

// ---------------------------------------------------------------------------
// Launch arguments shared by the host launchers and the kernels.
struct TileArgs {
    const void *x;
    const void *y;
    long long N;        // image side = row stride in elements
    int NT;             // tile side
    int T;              // tiles per image row = N / NT
    int TX;             // whole tiles across one unit
    int S;              // CTAs per tile along y (cluster size), RH = NT / S
    int RH;             // rows per unit
    int LPU;            // vectors per unit row = TX * NT / VEC
    int LPT;            // vectors per tile row = NT / VEC
    int tile_row0;      // first tile row covered by this launch
    float C1f;          // C1 rounded to float, used in the per-pixel divide
    float C2f, Cf, Df;  // Eq. 1 / Eq. 2 constants of the per-tile combine
    double Cd;          // C, for the FP64 form of Eq. 2 (cancelling tiles)
    float *lisi;        // (T*T) map or nullptr
    float *aug;         // (T*T) map or nullptr
    double *sums;       // (T*T*4) or nullptr
    int overlap;        // 1: an independent call (the kernel before it in the
                        // stream writes none of these images and touches none
                        // of the outputs): wait for that kernel only before
                        // writing; 0: wait before any access
};

// ---------------------------------------------------------------------------
// Loads.  16-byte vector loads through the non-coherent path without L1
// allocation (every pixel is read exactly once), with a 256-byte L2 prefetch
// hint that matches the row segments of a tile.
__device__ __forceinline__ uint4 ld_stream16(const void *p)
{
    uint4 r;
    asm("ld.global.nc.L1::no_allocate.L2::256B.v4.u32 {%0,%1,%2,%3}, [%4];"
        : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
        : "l"(p));
    return r;
}

__device__ __forceinline__ uint32_t ld_stream4(const void *p)
{
    uint32_t r;
    asm("ld.global.nc.L1::no_allocate.u32 %0, [%1];" : "=r"(r) : "l"(p));
    return r;
}

__device__ __forceinline__ uint32_t ld_stream2(const void *p)
{
    unsigned short r;
    asm("ld.global.nc.L1::no_allocate.u16 %0, [%1];" : "=h"(r) : "l"(p));
    return (uint32_t)r;
}

// Storage types: VEC elements per 16-byte vector.
template <typename T> struct Elem;
template <> struct Elem<float> { static constexpr int VEC = 4; };
template <> struct Elem<__half> { static constexpr int VEC = 8; };
template <> struct Elem<__nv_bfloat16> { static constexpr int VEC = 8; };

// Raw register form of VEC elements (VEC == full vector, or 1 = scalar path).
template <typename T, int VEC> struct Raw { uint4 v; };
template <typename T> struct Raw<T, 1> { uint32_t v; };

template <typename T, int VEC>
__device__ __forceinline__ Raw<T, VEC> load_raw(const T *p)
{
    Raw<T, VEC> r;
    if constexpr (VEC == 1) {
        if constexpr (sizeof(T) == 4) r.v = ld_stream4(p);
        else r.v = ld_stream2(p);
    } else {
        r.v = ld_stream16(p);
    }
    return r;
}

template <typename T, int VEC>
__device__ __forceinline__ Raw<T, VEC> zero_raw()
{
    Raw<T, VEC> r;
    if constexpr (VEC == 1) r.v = 0u;
    else r.v = make_uint4(0u, 0u, 0u, 0u);
    return r;
}

__device__ __forceinline__ void h2_to_f(uint32_t w, float &lo, float &hi)
{
    __half2 h = *reinterpret_cast<__half2 *>(&w);
    float2 f = __half22float2(h);
    lo = f.x;
    hi = f.y;
}

__device__ __forceinline__ void b2_to_f(uint32_t w, float &lo, float &hi)
{
    lo = __uint_as_float(w << 16);
    hi = __uint_as_float(w & 0xffff0000u);
}

// Widen VEC stored elements to float (exact for all three storage types).
template <typename T, int VEC>
__device__ __forceinline__ void unpack(const Raw<T, VEC> &r, float (&f)[VEC])
{
    if constexpr (VEC == 1) {
        if constexpr (sizeof(T) == 4) {
            f[0] = __uint_as_float(r.v);
        } else if constexpr (std::is_same<T, __half>::value) {
            __half h = __ushort_as_half((unsigned short)r.v);
            f[0] = __half2float(h);
        } else {
            f[0] = __uint_as_float(r.v << 16);
        }
    } else if constexpr (sizeof(T) == 4) {
        f[0] = __uint_as_float(r.v.x);
        f[1] = __uint_as_float(r.v.y);
        f[2] = __uint_as_float(r.v.z);
        f[3] = __uint_as_float(r.v.w);
    } else if constexpr (std::is_same<T, __half>::value) {
        h2_to_f(r.v.x, f[0], f[1]);
        h2_to_f(r.v.y, f[2], f[3]);
        h2_to_f(r.v.z, f[4], f[5]);
        h2_to_f(r.v.w, f[6], f[7]);
    } else {
        b2_to_f(r.v.x, f[0], f[1]);
        b2_to_f(r.v.y, f[2], f[3]);
        b2_to_f(r.v.z, f[4], f[5]);
        b2_to_f(r.v.w, f[6], f[7]);
    }
}

// ---------------------------------------------------------------------------
// Approximate reciprocal: the PTX rcp.approx.ftz.f32 instruction (about one
// ulp of error by the PTX ISA's bound).  Its argument here is d + C1 >= C1, a
// normal number, and its result is normal for every argument below 2^126, so
// flushing subnormals changes nothing for pixel values in that range (any
// radio image, whose pixels are Jy-scale).
__device__ __forceinline__ float rcp_approx(float v)
{
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(v));
    return r;
}

// Packed running sums of one thread: lane .x takes the even elements of each
// vector, lane .y the odd ones (VEC == 1: lane .x only).
struct Sums2 {
    float2 a, b, x, y;
    __device__ __forceinline__ void zero()
    {
        a = b = x = y = make_float2(0.0f, 0.0f);
    }
};

// Per-pixel terms of Eq. 1 / Eq. 2 for the VEC pixel pairs of one 16-byte
// vector of each image, added in element order to the running sums p:
//   a += s / (d + C1),  b += s * d,  x += x',  y += y'
// with x', y' clamped, s = x' + y' (= |x + y| after the clamp) and
// d = |x' - y'|.  Clamp: max(v, 0) returns 0 for v <= 0 and for NaN (the
// non-NaN operand); 16-bit pixels are clamped two at a time in their packed
// form, then widened to float exactly.  The divide s / (d + C1) is
// s * rcp(d + C1) (denominator >= C1 > 0; about 2 ulp), fused into the
// accumulation, as is s * d.  Two pixel pairs per instruction with the packed
// f32x2 operations (add.f32x2, fma.f32x2); the sums stay packed until the
// caller folds them.
template <typename T, int VEC, bool DO_A, bool DO_B>
__device__ __forceinline__ void vector_terms(const Raw<T, VEC> &rx, const Raw<T, VEC> &ry,
                                             float C1f, Sums2 &p)
{
    float xv[VEC], yv[VEC];
    if constexpr (VEC > 1 && !std::is_same<T, float>::value) {
        // packed clamp of two 16-bit pixels per instruction
        const uint32_t wx[4] = {rx.v.x, rx.v.y, rx.v.z, rx.v.w};
        const uint32_t wy[4] = {ry.v.x, ry.v.y, ry.v.z, ry.v.w};
#pragma unroll
        for (int w = 0; w < 4; ++w) {
            if constexpr (std::is_same<T, __half>::value) {
                const __half2 z = __float2half2_rn(0.0f);
                __half2 hx = __hmax2(*reinterpret_cast<const __half2 *>(&wx[w]), z);
                __half2 hy = __hmax2(*reinterpret_cast<const __half2 *>(&wy[w]), z);
                float2 fx = __half22float2(hx), fy = __half22float2(hy);
                xv[2 * w] = fx.x;
                xv[2 * w + 1] = fx.y;
                yv[2 * w] = fy.x;
                yv[2 * w + 1] = fy.y;
            } else {
                const __nv_bfloat162 z = __float2bfloat162_rn(0.0f);
                __nv_bfloat162 hx =
                    __hmax2(*reinterpret_cast<const __nv_bfloat162 *>(&wx[w]), z);
                __nv_bfloat162 hy =
                    __hmax2(*reinterpret_cast<const __nv_bfloat162 *>(&wy[w]), z);
                uint32_t ux = *reinterpret_cast<uint32_t *>(&hx);
                uint32_t uy = *reinterpret_cast<uint32_t *>(&hy);
                b2_to_f(ux, xv[2 * w], xv[2 * w + 1]);
                b2_to_f(uy, yv[2 * w], yv[2 * w + 1]);
            }
        }
    } else {
        unpack<T, VEC>(rx, xv);
        unpack<T, VEC>(ry, yv);
#pragma unroll
        for (int i = 0; i < VEC; ++i) {
            xv[i] = fmaxf(xv[i], 0.0f);
            yv[i] = fmaxf(yv[i], 0.0f);
        }
    }
    if constexpr (VEC == 1) {
        const float s = xv[0] + yv[0];
        const float d = fabsf(xv[0] - yv[0]);
        if (DO_A) p.a.x = __fmaf_rn(s, rcp_approx(d + C1f), p.a.x);
        if (DO_B) p.b.x = __fmaf_rn(s, d, p.b.x);
        p.x.x += xv[0];
        p.y.x += yv[0];
    } else {
        const float2 neg1 = make_float2(-1.0f, -1.0f);
        const float2 c1 = make_float2(C1f, C1f);
#pragma unroll
        for (int i = 0; i < VEC; i += 2) {
            const float2 x2 = make_float2(xv[i], xv[i + 1]);
            const float2 y2 = make_float2(yv[i], yv[i + 1]);
            const float2 s2 = __fadd2_rn(x2, y2);
            const float2 m2 = __ffma2_rn(y2, neg1, x2);  // x - y, one rounding
            const float2 d2 = make_float2(fabsf(m2.x), fabsf(m2.y));
            if (DO_A) {
                const float2 t2 = __fadd2_rn(d2, c1);
                const float2 r2 = make_float2(rcp_approx(t2.x), rcp_approx(t2.y));
                p.a = __ffma2_rn(s2, r2, p.a);
            }
            if (DO_B) p.b = __ffma2_rn(s2, d2, p.b);
            p.x = __fadd2_rn(p.x, x2);
            p.y = __fadd2_rn(p.y, y2);
        }
    }
}

// Kahan-compensated float accumulator.
struct Kahan {
    float s = 0.0f, c = 0.0f;
    __device__ __forceinline__ void add(float v)
    {
        float yv = v - c;
        float t = s + yv;
        c = (t - s) - yv;
        s = t;
    }
    __device__ __forceinline__ float value() const { return s - c; }
};

// ---------------------------------------------------------------------------
// Streams one unit (RH rows x LPU vectors, top-left at xu / yu, row stride N)
// and returns this thread's four sums.  Vector v = tid + j * THREADS of the
// unit is (row v / LPU, column v % LPU); (row, column) advance incrementally.
// ILP vectors of each image are in flight per thread before any is used.
template <typename T, int VEC, int ILP, int THREADS, bool DO_A, bool DO_B>
__device__ __forceinline__ void accumulate_unit(const T *__restrict__ xu,
                                                const T *__restrict__ yu,
                                                long long N, int RH, int LPU,
                                                float C1f, float (&acc)[4])
{
    const int tid = threadIdx.x;
    int row = tid / LPU;
    int col = tid - row * LPU;
    const int drow = THREADS / LPU;
    const int dcol = THREADS - drow * LPU;
    Kahan ka, kb, kx, ky;
    while (row < RH) {
        Raw<T, VEC> rx[ILP], ry[ILP];
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            if (row < RH) {
                long long off = (long long)row * N + (long long)col * VEC;
                rx[u] = load_raw<T, VEC>(xu + off);
                ry[u] = load_raw<T, VEC>(yu + off);
            } else {
                rx[u] = zero_raw<T, VEC>();
                ry[u] = zero_raw<T, VEC>();
            }
            col += dcol;
            row += drow;
            if (col >= LPU) {
                col -= LPU;
                row += 1;
            }
        }
        Sums2 p;
        p.zero();
#pragma unroll
        for (int u = 0; u < ILP; ++u) {
            // a vector that was not loaded is all zeros and adds exactly 0
            vector_terms<T, VEC, DO_A, DO_B>(rx[u], ry[u], C1f, p);
        }
        if (DO_A) ka.add(p.a.x + p.a.y);
        if (DO_B) kb.add(p.b.x + p.b.y);
        kx.add(p.x.x + p.x.y);
        ky.add(p.y.x + p.y.y);
    }
    acc[0] = ka.value();
    acc[1] = kb.value();
    acc[2] = kx.value();
    acc[3] = ky.value();
}

__device__ __forceinline__ float warp_sum(float v)
{
#pragma unroll
    for (int o = 16; o >= 1; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Barriers for reduce_unit: the whole CTA, or a named barrier over the
// consumer warps of the persistent kernel (its producer warp does not take
// part).
struct CtaBarrier {
    __device__ __forceinline__ void operator()() const { __syncthreads(); }
};
template <int ID, int COUNT> struct NamedBarrier {
    __device__ __forceinline__ void operator()() const
    {
        asm volatile("bar.sync %0, %1;" ::"n"(ID), "n"(COUNT) : "memory");
    }
};

__host__ __device__ __forceinline__ bool is_pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }

// Whether a unit of TX > 1 tiles across, LPU vectors per unit row and LPT per
// tile row takes the segmented shuffle tree of reduce_unit (LPT a power of two
// up to 32, and whole unit rows per warp or whole warps per unit row).
__host__ __device__ __forceinline__ bool segmented_reduce(int TX, int LPU, int LPT)
{
    return TX > 1 && is_pow2(LPT) && LPT <= 32 && (LPU >= 32 || is_pow2(LPU));
}

// Reduction slots of one tile row in the segmented form: one per (group of
// threads that covers a unit row, tile), (THREADS / max(LPU, 32)) * TX.
__host__ __device__ __forceinline__ int segmented_slots(int threads, int TX, int LPU)
{
    return threads / (LPU >= 32 ? LPU : 32) * TX;
}

// Segmented shuffle tree of one tile row (segmented_reduce() holds): each
// tile's LPT lanes are summed (and, when a warp spans several unit rows, the
// same columns of those rows), and the lane heading each segment stores the
// partial of its (row group, tile) in red[k][slot0 + group * TX + tile].
template <int THREADS>
__device__ __forceinline__ void segmented_partials(const float (&acc)[4], int TX, int LPU,
                                                   int LPT, int slot0, float (*red)[THREADS])
{
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    float v[4] = {acc[0], acc[1], acc[2], acc[3]};
    for (int o = 1; o < LPT; o <<= 1) {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    for (int o = LPU; o < 32; o <<= 1) {
#pragma unroll
        for (int k = 0; k < 4; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    }
    const int span = LPU >= 32 ? LPU : 32;  // threads per row group
    const int col = tid % LPU;
    if (col % LPT == 0 && (LPU >= 32 || lane < LPU)) {
        const int slot = slot0 + (tid / span) * TX + col / LPT;
#pragma unroll
        for (int k = 0; k < 4; ++k) red[k][slot] = v[k];
    }
}

// Cross-thread reduction of one unit, in FP32 (the low-rate FP64 pipe of this
// GPU is kept off the per-unit path).  part[tl * 4 + k] receives tile tl's sum
// k (A, B, Sx, Sy).  A thread's column is v % LPU and, for TX > 1, fixed
// (the host guarantees THREADS % LPU == 0), so its tile is (tid % LPU) / LPT.
//  * TX == 1: every warp reduces its lanes with an xor-shuffle tree, then warp
//    0 combines the per-warp partials the same way.
//  * TX > 1, LPT a power of two and the warp rows aligned (LPU >= 32, or LPU a
//    power of two): a segmented shuffle tree sums each tile's LPT lanes (and,
//    when a warp spans several unit rows, the same columns of those rows); the
//    lane heading each segment stores one partial per (row group, tile); then
//    thread tl sums tile tl's row-group partials in order.
//  * otherwise: all four sums go through shared memory and warp w sums tiles
//    w, w + warps, ... lane-wise in a fixed order, then with a shuffle tree.
template <int THREADS, typename Bar>
__device__ __forceinline__ void reduce_unit(const float (&acc)[4], int TX, int LPU, int LPT,
                                            float (*red)[THREADS], float *part, Bar bar)
{
    const int tid = threadIdx.x;
    const int lane = tid & 31, warp = tid >> 5;
    constexpr int WARPS = THREADS / 32;
    if (TX == 1) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float v = warp_sum(acc[k]);
            if (lane == 0) red[k][warp] = v;
        }
        bar();
        if (warp == 0) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float v = lane < WARPS ? red[k][lane] : 0.0f;
                v = warp_sum(v);
                if (lane == 0) part[k] = v;
            }
        }
        bar();
        return;
    }
    if (segmented_reduce(TX, LPU, LPT)) {
        segmented_partials<THREADS>(acc, TX, LPU, LPT, 0, red);
        const int groups = THREADS / (LPU >= 32 ? LPU : 32);
        bar();
        for (int tl = tid; tl < TX; tl += THREADS) {
            float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            for (int g = 0; g < groups; ++g) {
#pragma unroll
                for (int k = 0; k < 4; ++k) s[k] += red[k][g * TX + tl];
            }
#pragma unroll
            for (int k = 0; k < 4; ++k) part[tl * 4 + k] = s[k];
        }
        bar();
        return;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) red[k][tid] = acc[k];
    bar();
    const int count = (THREADS / LPU) * LPT;
    for (int tl = warp; tl < TX; tl += WARPS) {
        float s[4] = {0.0f, 0.0f, 0.0f, 0.0f};
        for (int e = lane; e < count; e += 32) {
            int q = e / LPT;
            int src = q * LPU + tl * LPT + (e - q * LPT);
#pragma unroll
            for (int k = 0; k < 4; ++k) s[k] += red[k][src];
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            float w = warp_sum(s[k]);
            if (lane == 0) part[tl * 4 + k] = w;
        }
    }
    bar();
}

// Eq. 1 / Eq. 2 per-tile combine and the output writes; the optional sums are
// exported widened to FP64.
//
// Per-tile combine of Eq. 1 and Eq. 2 from the tile's four FP32 sums:
//   lisi = D A / (max(Sx, Sy) + C2),   aug = 1 - B / (Sx + Sy + C).
// lisi is a product and quotient of nonnegative values, so FP32 with IEEE
// division (correctly rounded) keeps it within 3 u of the exact ratio of the
// sums.  aug loses relative accuracy to cancellation when r = B/(Sx+Sy+C) is
// close to 1: there (|aug| < r/16, rare on sky images, where aug is close to 1)
// the ratio and the subtraction are redone in FP64 from the same sums and
// rounded once, so aug keeps about 1 u relative on every tile.
__device__ __forceinline__ void combine_tile(float *lisi, float *aug, long long t, float A,
                                             float B, float Sx, float Sy, float C2f, float Cf,
                                             float Df, double Cd)
{
    if (lisi) lisi[t] = __fdiv_rn(Df * A, fmaxf(Sx, Sy) + C2f);
    if (aug) {
        const float r = __fdiv_rn(B, (Sx + Sy) + Cf);
        float v = 1.0f - r;
        if (fabsf(v) < 0.0625f * r)
            v = __double2float_rn(__dadd_rn(
                1.0, -__ddiv_rn((double)B, __dadd_rn(__dadd_rn((double)Sx, (double)Sy), Cd))));
        aug[t] = v;
    }
}

__device__ __forceinline__ void write_tile(const TileArgs &p, long long t,
                                           float A, float B, float Sx, float Sy)
{
    combine_tile(p.lisi, p.aug, t, A, B, Sx, Sy, p.C2f, p.Cf, p.Df, p.Cd);
    if (p.sums) {
        double *o = p.sums + 4 * t;
        o[0] = A;
        o[1] = B;
        o[2] = Sx;
        o[3] = Sy;
    }
}

}  // namespace iqa
