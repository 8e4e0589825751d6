// iqa_stream.cuh -- persistent, TMA-pipelined form of the tile reduction.
//
// Same method as iqa_tiles.cuh (arxiv 2501.10653, Section 2, Eq. 1 and Eq. 2:
// clamp, tile, four per-tile sums, per-tile ratios), laid out for GB300:
//   * one CTA per SM slot loops over units (TX whole tiles across, up to 1024
//     elements wide, x RH tile rows down) of one or many image pairs: a static first
//     grab of consecutive units from its own index (head_units of them), then
//     grabs of consecutive units from a global counter (about 64 KB per image
//     each, fetched one grab ahead, shrinking toward one unit as the work runs
//     out), or round-robin without a counter; the producer
//     tells the consumers which pair a stage holds and the first tile of its
//     unit through per-stage slots in shared memory;
//   * a producer warp streams every unit in chunks of CH rows with TMA tensor
//     copies (cp.async.bulk.tensor: one 2-D box, or one 3-D box of 256-element
//     segments for rows wider than 256) of x and y into a ring of shared-
//     memory stages, signalling completion on per-stage mbarriers;
//   * consumer warps read each stage with 16-byte shared loads, clamp, form
//     the terms, accumulate in registers across a tile row's chunks and
//     release the stage; at the end of each tile row a segmented shuffle tree
//     leaves per-warp partials in shared memory, and at the end of the unit one
//     named barrier lets each thread sum and write one tile, while the
//     producer is already a stage ahead (units of several tile rows take the
//     per-unit work once for all of them);
//   * launches use programmatic dependent launch: the next kernel in the
//     stream may be scheduled while this one drains, and the producer waits
//     for the previous grid before it fetches work or issues a copy;
//   * every mbarrier wait is bounded by a time limit: on expiry the CTA
//     records an error code, stops issuing, waits (bounded) for the copies it
//     has in flight and returns, so the host sees a status instead of a hang.
#pragma once

#include <climits>
#include <cuda.h>

#include "iqa_device.cuh"
#include "iqa_internal.h"

namespace iqa {

// One image pair of a persistent launch.  Lives in global memory (batched
// launches) or inside the kernel's __grid_constant__ parameter (one pair);
// the CUtensorMap members give it the alignment the TMA unit requires.
struct PairDesc {
    CUtensorMap tmx;         // 2-D map of x: dims {N, N}, box {BW, CH}
    CUtensorMap tmy;         // same for y
    float *lisi;
    float *aug;
    double *sums;
    long long unit_begin;    // first global unit index of this pair
    int N, NT, T;            // image side, tile side, tiles per row
    int TX;                  // tiles across a unit
    int RH;                  // tile rows down a unit (T % RH == 0)
    int units_x;             // units per band of RH tile rows = T / TX
    int CH;                  // rows per chunk
    int CPR;                 // chunks per tile row = NT / CH
    int chunks;              // chunks per unit = RH * CPR
    int LPU;                 // 16-byte vectors per unit row = TX * NT / VEC
    int LPT;                 // vectors per tile row = NT / VEC
    int NB;                  // 256-element boxes across a unit row: 1 = 2-D map
                             // {N, N}, box {BW, CH}; > 1 = 3-D map
                             // {256, N/256, N}, box {256, NB, CH}
    float C1f;               // C1 rounded to float, used in the per-pixel divide
    float C2f, Cf, Df;       // Eq. 1 / Eq. 2 constants of the per-tile combine
    double Cd;               // C, for the FP64 form of Eq. 2 (cancelling tiles)
};

struct StreamParams {
    const PairDesc *descs;   // table in global memory, or nullptr: use one_pair
    int npairs;
    int stage_bytes;         // bytes of ONE image per stage
    int stages;
    // units of every CTA's first grab, taken statically (CTA b takes units
    // [b * head_units, (b + 1) * head_units)); dynamic grabs then count from
    // gridDim.x * head_units.  0 or 1 = one unit; only with a work counter.
    int head_units;
    long long total_units;
    int *status;             // error word (nullable), nonzero = failed
    long long timeout_ns;    // bound on every wait
    // Dynamic schedule (nullable: static round-robin instead): [0] = next
    // unit, [1] = CTAs done fetching.  Zero before the launch; the last CTA to
    // finish fetching puts both back to zero, so a stream of launches needs no
    // reset in between (launches sharing a counter must not use it at the same
    // time: even an independent launch waits for the kernel before it first).
    unsigned long long *sched;
    int inject_stall;        // test hook: 1 = the producer issues nothing
    // 1: the launch does not depend on the kernel before it in the stream
    // (an independent plan): each CTA's first grab is copied before waiting
    // for that kernel, and only the shared counter waits for it
    int overlap_head;
    // nullable: {npairs, total_units} in device memory, read at launch in
    // place of the two fields above (a captured graph replayed with new work)
    const long long *dyn;
    PairDesc one_pair;
};

enum StreamError { STREAM_TIMEOUT_FULL = 1, STREAM_TIMEOUT_EMPTY = 2 };

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return done != 0;
}

// Bounded wait on the phase with the given parity.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity,
                                          long long timeout_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = global_ns();
    while (!mbar_try_wait(bar, parity)) {
        if ((long long)(global_ns() - t0) > timeout_ns) return false;
    }
    return true;
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
                 : "memory");
}

// 3-D tiled TMA load of one box at (0, seg, row): the image viewed as rows of
// 256-element segments, so that a box of NB segments lands in shared memory
// as NB * 256 contiguous elements per row.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int seg,
                                            int row, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(0), "r"(seg), "r"(row),
        "r"(smem_addr(bar))
        : "memory");
}

// 2-D tiled TMA load of one box at (col, row) into shared memory.
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, int col,
                                            int row, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_addr(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(col), "r"(row), "r"(smem_addr(bar))
        : "memory");
}

// A tensor map in a global-memory table may have been rewritten since the TMA
// unit last read that address (a plan's re-upload, a server step, a no-alloc
// call): acquire the new contents for the tensor-map proxy before first use.
__device__ __forceinline__ void acquire_tmap(const CUtensorMap *map)
{
    asm volatile("fence.proxy.tensormap::generic.acquire.gpu [%0], 128;" ::"l"(
                     reinterpret_cast<uint64_t>(map))
                 : "memory");
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap *map)
{
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
}

__device__ __forceinline__ void named_bar(int id, int count)
{
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(count) : "memory");
}

// Which pair owns global unit u (pairs are stored in unit order).
__device__ __forceinline__ void write_tile_desc(const PairDesc &d, long long t, float A,
                                                float B, float Sx, float Sy)
{
    combine_tile(d.lisi, d.aug, t, A, B, Sx, Sy, d.C2f, d.Cf, d.Df, d.Cd);
    if (d.sums) {
        double *o = d.sums + 4 * t;
        o[0] = A;
        o[1] = B;
        o[2] = Sx;
        o[3] = Sy;
    }
}

// Dynamic shared memory layout: [stages][2][stage_bytes] ring, then the
// 2*stages mbarriers, the per-stage slots (first tile of the stage's unit
// within its pair, -1 at the end of work; the pair's index), the reduction scratch
// red[4][2 * CT] (the segmented form's per-tile-row slots; reduce_unit views
// its first 4 * CT floats as red[4][CT]) and part[kMaxTX*4], and the abort
// flag.  Host:
// stream_smem_bytes().
template <typename T, int CT, bool DO_A, bool DO_B>
__global__ void __launch_bounds__(CT + 32, 1)
    iqa_stream_kernel(const __grid_constant__ StreamParams sp)
{
    constexpr int VEC = Elem<T>::VEC;
    extern __shared__ __align__(128) unsigned char smem[];
    const int S = sp.stages;
    const int SB = sp.stage_bytes;
    unsigned char *ring = smem;
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)S * 2 * SB);
    uint64_t *empty = full + S;
    long long *stage_unit = reinterpret_cast<long long *>(empty + S);
    int *stage_pair = reinterpret_cast<int *>(stage_unit + S);
    float(*red)[CT] = reinterpret_cast<float(*)[CT]>(stage_unit + 2 * S);
    float(*rows)[2 * CT] = reinterpret_cast<float(*)[2 * CT]>(red);
    float *part = reinterpret_cast<float *>(rows + 4);
    int *abort_flag = reinterpret_cast<int *>(part + kMaxTX * 4);

    const PairDesc *descs = sp.descs ? sp.descs : &sp.one_pair;
    const int npairs = sp.dyn ? (int)sp.dyn[0] : sp.npairs;
    const long long total_units = sp.dyn ? sp.dyn[1] : sp.total_units;
    const int tid = threadIdx.x;
    const bool producer = tid >= CT;

    if (tid == 0) {
        *abort_flag = 0;
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], CT / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        // programmatic dependent launch: the next kernel in the stream may be
        // scheduled once every CTA of this one is resident; it waits (below,
        // griddepcontrol.wait) for this grid to finish before touching memory
        asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    }
    __syncthreads();

    if (producer) {
        // ---------------- producer warp: one elected lane issues the copies
        if (tid != CT) return;
        long long k = 0;  // chunk counter of this CTA
        int ps = 0;         // its stage, k % S
        uint32_t pph = 1u;  // the empty-barrier parity to wait on, ((k / S) & 1) ^ 1
        int last_pair = -1;
        bool ok = true;
        // Work is taken in grabs of consecutive units [u, u_end): one
        // atomicAdd on the shared counter per grab, issued one grab ahead so
        // that its latency hides behind the current grab's copies.  A grab
        // spans about kGrabBytes of each image (several small units, or one).
        // The first grab of every CTA is static: head units from its own
        // index times head (no atomic on the launch's critical path; head > 1
        // makes a grab of small units about as many bytes as one large unit);
        // dynamic grabs then count from gridDim.x * head, and shrink toward
        // one unit as the work runs out (guided), so that the CTAs finish
        // close together.
        constexpr uint32_t kGrabBytes = 65536;
        const long long head = (sp.sched && sp.head_units > 1) ? sp.head_units : 1;
        long long u = blockIdx.x * head, u_end = u + head, nxt = -1, nxt_end = -1, i = 0;
        bool have_next = false;
        // A kernel earlier in the stream (programmatic dependent launch) may
        // still be running: wait for it before any work is fetched or copied.
        // An independent launch (sp.overlap_head) instead issues its first
        // grab's copies at once, overlapping that kernel's drain, and waits
        // before it touches the shared counter, which that kernel may still
        // be using (and so that this grid never completes before it).
        bool waited = sp.overlap_head == 0;
        if (waited) asm volatile("griddepcontrol.wait;" ::: "memory");
        // next grab of units (one atomicAdd on the shared counter, or the
        // static round-robin without one), sized from the current unit
        const auto fetch_next = [&](uint32_t unit_bytes) {
            if (sp.sched) {
                unsigned g = unit_bytes >= kGrabBytes ? 1u : min(8u, kGrabBytes / unit_bytes);
                // guided: at most a quarter of this CTA's share of what is left,
                // (total_units - u) / (4 gridDim.x), tested without a 64-bit
                // division (floor(a / b) < g exactly when a < g b)
                const long long left = total_units - u;
                const long long span = 4LL * gridDim.x;
                if (left < (long long)g * span) {
                    const unsigned share = left > 0 ? (unsigned)left / (unsigned)span : 0u;
                    g = share > 1 ? share : 1u;
                }
                nxt = (long long)gridDim.x * head +
                      (long long)atomicAdd(&sp.sched[0], (unsigned long long)g);
                nxt_end = nxt + g;
            } else {
                nxt = blockIdx.x + (++i) * (long long)gridDim.x;
                nxt_end = nxt + 1;
            }
            have_next = true;
        };
        if (sp.inject_stall) ok = false;  // test hook: issue nothing at all
        // pair of unit u: units are taken in increasing order, so the pair
        // index only moves forward (a binary search only when u passes the
        // next pair's first unit)
        int pi = 0;
        long long next_begin = npairs > 1 ? descs[1].unit_begin : LLONG_MAX;
        while (ok) {
            const bool last = u >= total_units;
            if (!last && u >= next_begin) {
                int lo = pi + 1, hi = npairs - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (descs[mid].unit_begin <= u) lo = mid;
                    else hi = mid - 1;
                }
                pi = lo;
                next_begin = pi + 1 < npairs ? descs[pi + 1].unit_begin : LLONG_MAX;
            }
            const PairDesc &d = descs[pi];
            const int nchunks = last ? 1 : d.chunks;
            int col0 = 0, row0 = 0;
            long long t0 = -1;  // first tile of the unit within its pair
            uint32_t bytes = 0;
            if (!last) {
                if (pi != last_pair) {
                    if (sp.descs) {
                        acquire_tmap(&d.tmx);
                        acquire_tmap(&d.tmy);
                    }
                    prefetch_tmap(&d.tmx);
                    prefetch_tmap(&d.tmy);
                    last_pair = pi;
                }
                const long long lu = u - d.unit_begin;
                // a 32-bit division whenever the unit index fits (every pair
                // below 2^31 units): the 64-bit one is a long subroutine
                const int band = lu <= (long long)INT_MAX ? (int)lu / d.units_x
                                                          : (int)(lu / d.units_x);
                const int ucol = (int)(lu - (long long)band * d.units_x);
                col0 = ucol * d.TX * d.NT;
                row0 = band * d.RH * d.NT;
                t0 = (long long)band * d.RH * d.T + (long long)ucol * d.TX;
                bytes = (uint32_t)(d.CH * d.TX * d.NT * (int)sizeof(T));
                if (!have_next && waited) fetch_next(bytes * (uint32_t)d.chunks);
            }
            for (int c = 0; c < nchunks; ++c, ++k) {
                // ring position of chunk k: stage k % S, and the parity of the
                // empty barrier's phase to wait on, ((k / S) & 1) ^ 1, kept
                // incrementally (no division per chunk)
                const int s = ps;
                const uint32_t par = pph;
                if (!mbar_wait(&empty[s], par, sp.timeout_ns)) {
                    if (sp.status) atomicOr(sp.status, STREAM_TIMEOUT_EMPTY);
                    atomicExch(abort_flag, 1);
                }
                if (*((volatile int *)abort_flag)) {
                    ok = false;
                    break;
                }
                if (last) {
                    // end of work: an empty stage whose unit slot says so
                    stage_unit[s] = -1;
                    mbar_arrive(&full[s]);
                    break;
                }
                // the chunk's box lies inside the image and fits one stage
                // (checked build only; a violation stops the CTA like an abort)
                if (!IQA_CHECK(pi < npairs && d.RH >= 1 && d.T % d.RH == 0 &&
                               u - d.unit_begin < (long long)(d.T / d.RH) * d.units_x &&
                               col0 >= 0 && col0 + d.TX * d.NT <= d.N &&
                               (col0 * (int)sizeof(T)) % 16 == 0 &&
                               (d.NB == 1 || col0 % 256 == 0) &&
                               row0 + (c + 1) * d.CH <= d.N &&
                               bytes <= (uint32_t)SB)) {
                    atomicExch(abort_flag, 1);
                    ok = false;
                    break;
                }
                stage_unit[s] = t0;
                stage_pair[s] = pi;
                mbar_expect_tx(&full[s], 2 * bytes);
                unsigned char *dst = ring + (size_t)s * 2 * SB;
                if (d.NB > 1) {
                    tma_load_3d(dst, &d.tmx, col0 >> 8, row0 + c * d.CH, &full[s]);
                    tma_load_3d(dst + SB, &d.tmy, col0 >> 8, row0 + c * d.CH, &full[s]);
                } else {
                    tma_load_2d(dst, &d.tmx, col0, row0 + c * d.CH, &full[s]);
                    tma_load_2d(dst + SB, &d.tmy, col0, row0 + c * d.CH, &full[s]);
                }
                if (++ps == S) {
                    ps = 0;
                    pph ^= 1u;
                }
            }
            if (!waited && (last || u + 1 >= u_end)) {
                // the first grab is in flight (independent launch)
                asm volatile("griddepcontrol.wait;" ::: "memory");
                waited = true;
                if (!last && ok) fetch_next(bytes * (uint32_t)d.chunks);
            }
            if (last) break;
            if (++u >= u_end) {
                u = nxt;
                u_end = nxt_end;
                have_next = false;
            }
        }
        if (!waited) asm volatile("griddepcontrol.wait;" ::: "memory");
        if (sp.sched) {
            // every CTA has made its final fetch once the count reaches the
            // grid size; the last one puts the counters back to zero (the
            // fence orders this CTA's fetches, including a grab fetched ahead
            // and never used, before its count)
            __threadfence();
            if (atomicAdd(&sp.sched[1], 1ull) == (unsigned long long)gridDim.x - 1) {
                atomicExch(&sp.sched[0], 0ull);
                atomicExch(&sp.sched[1], 0ull);
            }
        }
        // Copies still in flight when leaving (only after an abort): wait,
        // bounded, for every stage's last issued phase before returning.
        if (!ok && k > 0) {
            for (long long j = (k > S ? k - S : 0); j < k; ++j)
                mbar_wait(&full[j % S], (uint32_t)((j / S) & 1), sp.timeout_ns);
        }
        return;
    }

    // -------------------- consumer warps
    // Every consumer thread waits (bounded) for each chunk itself, then all
    // consumers meet at named barrier 2 and read the shared abort flag, so a
    // timeout anywhere makes every consumer leave at the same point and no
    // thread is ever left waiting at a barrier the others skipped.
    const int lane = tid & 31;
    const PairDesc *d = nullptr;
    long long t0 = -1;  // first tile of the current unit within its pair
    int c = 0, V = 0, chunks = 0;
    // chunks per tile row, chunk within the current tile row, that row's
    // index within the unit; seg: the unit takes the segmented reduction, one
    // block of reduction slots per tile row (units of several tile rows)
    int cpr = 0, cr = 0, r = 0, spr = 0;
    bool seg = false;
    float C1f = 0.0f;
    Kahan ka, kb, kx, ky;
    // ring position of chunk k: stage s = k % S, full-barrier parity
    // ph = (k / S) & 1, kept incrementally (no division per chunk)
    int s = 0;
    uint32_t ph = 0u;
    for (;;) {
        if (!mbar_wait(&full[s], ph, sp.timeout_ns)) {
            if (sp.status) atomicOr(sp.status, STREAM_TIMEOUT_FULL);
            atomicExch(abort_flag, 1);
        }
        named_bar(2, CT);
        if (*((volatile int *)abort_flag)) return;
        if (c == 0) {
            // a new unit: its first tile (the producer formed it) and its
            // descriptor fields are read once into registers
            t0 = stage_unit[s];
            if (t0 < 0) return;
            d = &descs[stage_pair[s]];
            V = d->CH * d->LPU;
            chunks = d->chunks;
            cpr = d->CPR;
            seg = segmented_reduce(d->TX, d->LPU, d->LPT);
            spr = segmented_slots(CT, d->TX, d->LPU);
            cr = 0;
            r = 0;
            C1f = d->C1f;
            ka = Kahan();
            kb = Kahan();
            kx = Kahan();
            ky = Kahan();
        }
        // the chunk's vectors fit the stage (checked build only)
        if (!IQA_CHECK(V * 16 <= SB)) V = 0;
        const uint4 *xs = reinterpret_cast<const uint4 *>(ring + (size_t)s * 2 * SB);
        const uint4 *ys = reinterpret_cast<const uint4 *>(ring + (size_t)s * 2 * SB + SB);
        Sums2 p;
        p.zero();
        // Full passes of PASS vectors of each image per thread (eight for FP32,
        // four for 16-bit types, whose vectors hold twice the pixels: the
        // unrolled pass stays small enough for the instruction cache), all
        // of a pass loaded before any is used; then a predicated tail of four
        // (vectors past V read as zeros, which add exactly 0).
        constexpr int PASS = VEC == 4 ? 8 : 4;
        int v0 = tid;
        for (; v0 + (PASS - 1) * CT < V; v0 += PASS * CT) {
            Raw<T, VEC> rx[PASS], ry[PASS];
#pragma unroll
            for (int j = 0; j < PASS; ++j) {
                rx[j].v = xs[v0 + j * CT];
                ry[j].v = ys[v0 + j * CT];
            }
#pragma unroll
            for (int j = 0; j < PASS; ++j)
                vector_terms<T, VEC, DO_A, DO_B>(rx[j], ry[j], C1f, p);
        }
        for (; v0 < V; v0 += 4 * CT) {
            Raw<T, VEC> rx[4], ry[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int v = v0 + j * CT;
                if (v < V) {
                    rx[j].v = xs[v];
                    ry[j].v = ys[v];
                } else {
                    rx[j] = zero_raw<T, VEC>();
                    ry[j] = zero_raw<T, VEC>();
                }
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) vector_terms<T, VEC, DO_A, DO_B>(rx[j], ry[j], C1f, p);
        }
        __syncwarp();
        if (lane == 0) mbar_arrive(&empty[s]);
        if (DO_A) ka.add(p.a.x + p.a.y);
        if (DO_B) kb.add(p.b.x + p.b.y);
        kx.add(p.x.x + p.x.y);
        ky.add(p.y.x + p.y.y);
        ++c;
        if (seg) {
            if (++cr == cpr) {
                // tile row r of the unit is complete: this warp's partials of
                // its tiles go to the row's block of reduction slots (no
                // barrier: the blocks of a unit's rows are disjoint, and every
                // read of the previous unit's slots precedes the named barrier
                // 2 that began this unit)
                cr = 0;
                const float acc[4] = {ka.value(), kb.value(), kx.value(), ky.value()};
                if (IQA_CHECK((r + 1) * spr <= 2 * CT))
                    segmented_partials<2 * CT>(acc, d->TX, d->LPU, d->LPT, r * spr, rows);
                ka = Kahan();
                kb = Kahan();
                kx = Kahan();
                ky = Kahan();
                ++r;
            }
            if (c == chunks) {
                // the unit's RH x TX tiles: thread tl sums tile tl's row-group
                // partials in order and writes it
                c = 0;
                named_bar(1, CT);
                const int TX = d->TX, T = d->T, RH = d->RH;
                const int groups = spr / TX;
                const bool out_ok = IQA_CHECK(t0 + (long long)(RH - 1) * T + TX <=
                                              (long long)T * T && RH * spr <= 2 * CT);
                for (int tl = tid; tl < RH * TX && out_ok; tl += CT) {
                    const int rr = tl / TX, tx = tl - rr * TX;
                    float sm[4] = {0.0f, 0.0f, 0.0f, 0.0f};
                    for (int g = 0; g < groups; ++g) {
#pragma unroll
                        for (int k = 0; k < 4; ++k) sm[k] += rows[k][rr * spr + g * TX + tx];
                    }
                    write_tile_desc(*d, t0 + (long long)rr * T + tx, sm[0], sm[1], sm[2],
                                    sm[3]);
                }
            }
        } else if (c == chunks) {
            c = 0;
            const int TX = d->TX, LPU = d->LPU, LPT = d->LPT;
            float acc[4] = {ka.value(), kb.value(), kx.value(), ky.value()};
            reduce_unit<CT>(acc, TX, LPU, LPT, red, part, NamedBarrier<1, CT>());
            const bool out_ok = IQA_CHECK(t0 + TX <= (long long)d->T * d->T && TX <= kMaxTX &&
                                          d->RH == 1);
            for (int tl = tid; tl < TX && out_ok; tl += CT)
                write_tile_desc(*d, t0 + tl, part[tl * 4 + 0], part[tl * 4 + 1],
                                part[tl * 4 + 2], part[tl * 4 + 3]);
        }
        if (++s == S) {
            s = 0;
            ph ^= 1u;
        }
    }
}

inline size_t stream_smem_bytes(int stages, int stage_bytes, int ct)
{
    return (size_t)stages * 2 * stage_bytes + (size_t)2 * stages * 8 + (size_t)2 * stages * 8 +
           (size_t)8 * ct * 4 + (size_t)kMaxTX * 4 * 4 + 16;
}

}  // namespace iqa
