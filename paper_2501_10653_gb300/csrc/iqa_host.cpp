// iqa_host.cpp -- the end-to-end path from host memory: images in, IQA maps
// out (the paper's host interface, Section 2).  iqa_both_host_many streams a
// sequence of pairs through two device slots: the upload of pair k+1 (copy
// stream) runs while pair k is reduced and its maps are read back (compute
// stream), so the host-to-device link stays busy.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>

#include "iqa.h"
#include "iqa_ctx.h"

using namespace iqa;

namespace {

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// Grows the context's workspace to `need` bytes within its HBM budget.
iqa_status ensure_workspace(iqa_ctx *ctx, size_t need)
{
    if (ctx->ws_bytes >= need) return IQA_OK;
    if (ctx->budget && need > ctx->budget) {
        set_error(ctx, "host-path workspace of %zu bytes exceeds the HBM budget of %zu",
                  need, ctx->budget);
        return IQA_ERR_NOMEM;
    }
    if (ctx->ws) {
        cudaStreamSynchronize(ctx->s_copy);
        cudaStreamSynchronize(ctx->s_comp);
        cudaFree(ctx->ws);
        ctx->ws = nullptr;
        ctx->ws_bytes = 0;
    }
    cudaError_t e = cudaMalloc(&ctx->ws, need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(ctx, "cudaMalloc of %zu bytes failed: %s", need, cudaGetErrorString(e));
        return IQA_ERR_NOMEM;
    }
    ctx->ws_bytes = need;
    return IQA_OK;
}

// Grows the page-locked read-back staging to `need` bytes.
iqa_status ensure_stage(iqa_ctx *ctx, size_t need)
{
    if (ctx->h_stage_bytes >= need) return IQA_OK;
    if (ctx->h_stage) {
        cudaFreeHost(ctx->h_stage);
        ctx->h_stage = nullptr;
        ctx->h_stage_bytes = 0;
    }
    cudaError_t e = cudaMallocHost(&ctx->h_stage, need);
    if (e != cudaSuccess) {
        cudaGetLastError();
        set_error(ctx, "page-locked staging of %zu bytes failed: %s", need,
                  cudaGetErrorString(e));
        return IQA_ERR_NOMEM;
    }
    ctx->h_stage_bytes = need;
    return IQA_OK;
}

struct SlotLayout {
    size_t off_y, off_l, off_a, off_s, bytes;
};

SlotLayout slot_layout(size_t img_bytes, size_t n_tiles)
{
    SlotLayout L;
    L.off_y = round_up(img_bytes, 256);
    L.off_l = L.off_y + round_up(img_bytes, 256);
    L.off_a = L.off_l + round_up(n_tiles * 4, 256);
    L.off_s = L.off_a + round_up(n_tiles * 4, 256);
    L.bytes = L.off_s + round_up(n_tiles * 32, 256);
    return L;
}

}  // namespace

extern "C" iqa_status iqa_both_host_many(iqa_ctx *ctx, const iqa_host_pair *pairs, int npairs,
                                         iqa_dtype dtype, const iqa_params *params)
{
    if (!ctx) return IQA_ERR_INVALID_ARG;
    if (!pairs || npairs < 1) {
        set_error(ctx, "need pairs and npairs >= 1");
        return IQA_ERR_INVALID_ARG;
    }
    if (!dtype_ok(dtype)) {
        set_error(ctx, "unknown dtype %d", (int)dtype);
        return IQA_ERR_INVALID_ARG;
    }
    iqa_params P;
    iqa_status s = resolve_params(ctx, params, &P);
    if (s != IQA_OK) return s;
    size_t max_img = 0, max_tiles = 0, out_bytes = 0;
    for (int i = 0; i < npairs; ++i) {
        const iqa_host_pair &p = pairs[i];
        if (!p.hx || !p.hy) {
            set_error(ctx, "pair %d: hx and hy must be host pointers, got NULL", i);
            return IQA_ERR_INVALID_ARG;
        }
        if (!p.lisi_map && !p.aug_map && !p.sums) {
            set_error(ctx, "pair %d: no output requested", i);
            return IQA_ERR_INVALID_ARG;
        }
        s = check_shape(ctx, p.N, p.NT);
        if (s != IQA_OK) return s;
        const size_t T = p.N / p.NT;
        max_img = std::max(max_img, (size_t)p.N * p.N * elem_size(dtype));
        max_tiles = std::max(max_tiles, T * T);
        out_bytes += T * T * 40;
    }

    std::lock_guard<std::mutex> guard(ctx->host_mu);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
    const SlotLayout L = slot_layout(max_img, max_tiles);
    const int slots = npairs > 1 ? 2 : 1;
    s = ensure_workspace(ctx, L.bytes * slots);
    if (s == IQA_OK) s = ensure_stage(ctx, out_bytes);
    if (s != IQA_OK) {
        cudaSetDevice(prev);
        return s;
    }
    while (ctx->band_events.size() < 4) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cudaSetDevice(prev);
            return cuda_fail(ctx, e, "cudaEventCreate");
        }
        ctx->band_events.push_back(ev);
    }
    cudaEvent_t *loaded = &ctx->band_events[0];  // per slot: images on the device
    cudaEvent_t *done = &ctx->band_events[2];    // per slot: slot free again
    char *stage = static_cast<char *>(ctx->h_stage);
    size_t stage_off = 0;
    for (int i = 0; i < npairs && e == cudaSuccess && s == IQA_OK; ++i) {
        const iqa_host_pair &p = pairs[i];
        const int slot = i % slots;
        char *base = static_cast<char *>(ctx->ws) + (size_t)slot * L.bytes;
        const size_t img = (size_t)p.N * p.N * elem_size(dtype);
        const size_t n = (size_t)(p.N / p.NT) * (p.N / p.NT);
        float *dl = p.lisi_map ? reinterpret_cast<float *>(base + L.off_l) : nullptr;
        float *da = p.aug_map ? reinterpret_cast<float *>(base + L.off_a) : nullptr;
        double *dsm = p.sums ? reinterpret_cast<double *>(base + L.off_s) : nullptr;
        // the slot's previous pair must have been reduced and read back
        if (i >= slots) e = cudaStreamWaitEvent(ctx->s_copy, done[slot], 0);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(base, p.hx, img, cudaMemcpyHostToDevice, ctx->s_copy);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(base + L.off_y, p.hy, img, cudaMemcpyHostToDevice,
                                ctx->s_copy);
        if (e == cudaSuccess) e = cudaEventRecord(loaded[slot], ctx->s_copy);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->s_comp, loaded[slot], 0);
        if (e != cudaSuccess) break;
        const int maps = dsm ? MAPS_AB : ((dl ? MAPS_A : 0) | (da ? MAPS_B : 0));
        TileConfig c = pick_config(ctx, p.N, p.NT, dtype, maps, true);
        std::string why;
        if (!any_config_valid(p.N, p.NT, dtype, c, &why)) {
            set_error(ctx, "no launch shape for N=%d NT=%d: %s", p.N, p.NT, why.c_str());
            s = IQA_ERR_UNSUPPORTED;
            break;
        }
        if (c.variant == 1) {
            s = run_stream_pair(ctx, base, base + L.off_y, dtype, p.N, p.NT, c, P, dl, da,
                                dsm, maps, ctx->s_comp);
        } else {
            TileArgs a = make_args(base, base + L.off_y, p.N, p.NT, c, P, dl, da, dsm);
            e = launch_tiles(a, c, dtype, maps, p.N / p.NT, ctx->s_comp);
        }
        // maps go to page-locked staging (copied out after the last pair)
        if (e == cudaSuccess && s == IQA_OK && p.lisi_map)
            e = cudaMemcpyAsync(stage + stage_off, dl, n * 4, cudaMemcpyDeviceToHost,
                                ctx->s_comp);
        if (e == cudaSuccess && s == IQA_OK && p.aug_map)
            e = cudaMemcpyAsync(stage + stage_off + n * 4, da, n * 4, cudaMemcpyDeviceToHost,
                                ctx->s_comp);
        if (e == cudaSuccess && s == IQA_OK && p.sums)
            e = cudaMemcpyAsync(stage + stage_off + n * 8, dsm, n * 32,
                                cudaMemcpyDeviceToHost, ctx->s_comp);
        stage_off += n * 40;
        if (e == cudaSuccess && s == IQA_OK) e = cudaEventRecord(done[slot], ctx->s_comp);
    }
    cudaError_t e2 = cudaStreamSynchronize(ctx->s_comp);
    cudaError_t e3 = cudaStreamSynchronize(ctx->s_copy);
    if (s == IQA_OK && e == cudaSuccess && e2 == cudaSuccess && e3 == cudaSuccess) {
        stage_off = 0;
        for (int i = 0; i < npairs; ++i) {
            const iqa_host_pair &p = pairs[i];
            const size_t n = (size_t)(p.N / p.NT) * (p.N / p.NT);
            if (p.lisi_map) std::memcpy(p.lisi_map, stage + stage_off, n * 4);
            if (p.aug_map) std::memcpy(p.aug_map, stage + stage_off + n * 4, n * 4);
            if (p.sums) std::memcpy(p.sums, stage + stage_off + n * 8, n * 32);
            stage_off += n * 40;
        }
    }
    cudaSetDevice(prev);
    if (s != IQA_OK) return s;
    if (e != cudaSuccess) return cuda_fail(ctx, e, "host-path enqueue");
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "host-path compute stream");
    if (e3 != cudaSuccess) return cuda_fail(ctx, e3, "host-path copy stream");
    return IQA_OK;
}

extern "C" iqa_status iqa_both_host(iqa_ctx *ctx, const void *hx, const void *hy,
                                    iqa_dtype dtype, int N, int NT,
                                    const iqa_params *params, float *lisi_map,
                                    float *aug_map, double *sums)
{
    if (!ctx) return IQA_ERR_INVALID_ARG;
    iqa_host_pair p;
    p.hx = hx;
    p.hy = hy;
    p.N = N;
    p.NT = NT;
    p.lisi_map = lisi_map;
    p.aug_map = aug_map;
    p.sums = sums;
    return iqa_both_host_many(ctx, &p, 1, dtype, params);
}
