// iqa_host.cpp -- iqa_both_host: images in host memory, maps back in host
// memory (the paper's host interface, Section 2), with the upload of each row
// band overlapped with the kernel of the band before it.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

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

}  // namespace

extern "C" iqa_status iqa_both_host(iqa_ctx *ctx, const void *hx, const void *hy,
                                    iqa_dtype dtype, int N, int NT,
                                    const iqa_params *params, float *lisi_map,
                                    float *aug_map, double *sums)
{
    if (!ctx) return IQA_ERR_INVALID_ARG;
    if (!hx || !hy) {
        set_error(ctx, "hx and hy must be host pointers, got NULL");
        return IQA_ERR_INVALID_ARG;
    }
    if (!lisi_map && !aug_map && !sums) {
        set_error(ctx, "no output requested");
        return IQA_ERR_INVALID_ARG;
    }
    if (!dtype_ok(dtype)) {
        set_error(ctx, "unknown dtype %d", (int)dtype);
        return IQA_ERR_INVALID_ARG;
    }
    iqa_status s = check_shape(ctx, N, NT);
    if (s != IQA_OK) return s;
    iqa_params P;
    s = resolve_params(ctx, params, &P);
    if (s != IQA_OK) return s;

    std::lock_guard<std::mutex> guard(ctx->host_mu);
    int prev = 0;
    cudaGetDevice(&prev);
    cudaError_t e = cudaSetDevice(ctx->device);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");

    const int T = N / NT;
    const size_t n = (size_t)T * T;
    const size_t img = (size_t)N * N * elem_size(dtype);
    const size_t off_y = round_up(img, 256);
    const size_t off_l = off_y + round_up(img, 256);
    const size_t off_a = off_l + round_up(n * 4, 256);
    const size_t off_s = off_a + round_up(n * 4, 256);
    const size_t need = off_s + round_up(n * 32, 256);
    s = ensure_workspace(ctx, need);
    if (s != IQA_OK) {
        cudaSetDevice(prev);
        return s;
    }
    char *ws = static_cast<char *>(ctx->ws);
    void *dx = ws, *dy = ws + off_y;
    float *dl = lisi_map ? reinterpret_cast<float *>(ws + off_l) : nullptr;
    float *da = aug_map ? reinterpret_cast<float *>(ws + off_a) : nullptr;
    double *dsm = sums ? reinterpret_cast<double *>(ws + off_s) : nullptr;

    const int maps = sums ? MAPS_AB : ((dl ? MAPS_A : 0) | (da ? MAPS_B : 0));
    TileConfig c = pick_config(ctx, N, NT, dtype, maps, true);
    std::string why;
    if (!config_valid(N, NT, dtype, c, &why)) {
        cudaSetDevice(prev);
        set_error(ctx, "no launch shape for N=%d NT=%d: %s", N, NT, why.c_str());
        return IQA_ERR_UNSUPPORTED;
    }
    TileArgs a = make_args(dx, dy, N, NT, c, P, dl, da, dsm);

    // Row bands of whole tile rows: about 4 MB of each image per band, at most
    // 16 bands.  Band b's upload runs on s_copy while band b-1 computes on
    // s_comp.
    const size_t row_bytes = (size_t)NT * N * elem_size(dtype);
    int rows_per_band = (int)std::max<size_t>(1, (4u << 20) / std::max<size_t>(1, row_bytes));
    rows_per_band = std::max(rows_per_band, (T + 15) / 16);
    const int bands = (T + rows_per_band - 1) / rows_per_band;
    while ((int)ctx->band_events.size() < bands) {
        cudaEvent_t ev;
        e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
        if (e != cudaSuccess) {
            cudaSetDevice(prev);
            return cuda_fail(ctx, e, "cudaEventCreate");
        }
        ctx->band_events.push_back(ev);
    }
    for (int b = 0; b < bands && e == cudaSuccess; ++b) {
        const int r0 = b * rows_per_band;
        const int r1 = std::min(T, r0 + rows_per_band);
        const size_t off = (size_t)r0 * row_bytes;
        const size_t len = (size_t)(r1 - r0) * row_bytes;
        e = cudaMemcpyAsync(static_cast<char *>(dx) + off,
                            static_cast<const char *>(hx) + off, len,
                            cudaMemcpyHostToDevice, ctx->s_copy);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(static_cast<char *>(dy) + off,
                                static_cast<const char *>(hy) + off, len,
                                cudaMemcpyHostToDevice, ctx->s_copy);
        if (e == cudaSuccess) e = cudaEventRecord(ctx->band_events[b], ctx->s_copy);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(ctx->s_comp, ctx->band_events[b], 0);
        if (e == cudaSuccess) {
            a.tile_row0 = r0;
            e = launch_tiles(a, c, dtype, maps, r1 - r0, ctx->s_comp);
        }
    }
    if (e == cudaSuccess && lisi_map)
        e = cudaMemcpyAsync(lisi_map, dl, n * 4, cudaMemcpyDeviceToHost, ctx->s_comp);
    if (e == cudaSuccess && aug_map)
        e = cudaMemcpyAsync(aug_map, da, n * 4, cudaMemcpyDeviceToHost, ctx->s_comp);
    if (e == cudaSuccess && sums)
        e = cudaMemcpyAsync(sums, dsm, n * 32, cudaMemcpyDeviceToHost, ctx->s_comp);
    cudaError_t e2 = cudaStreamSynchronize(ctx->s_comp);
    cudaError_t e3 = cudaStreamSynchronize(ctx->s_copy);
    cudaSetDevice(prev);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "host-path enqueue");
    if (e2 != cudaSuccess) return cuda_fail(ctx, e2, "host-path compute stream");
    if (e3 != cudaSuccess) return cuda_fail(ctx, e3, "host-path copy stream");
    return IQA_OK;
}
