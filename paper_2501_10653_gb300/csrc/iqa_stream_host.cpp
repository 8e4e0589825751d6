// iqa_stream_host.cpp -- host side of the persistent TMA kernel: launch-shape
// checks, tensor-map encoding, pair descriptors and launches.
#include <cuda.h>
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <string>

#include "iqa.h"
#include "iqa_ctx.h"
#include "iqa_stream.cuh"

namespace iqa {

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *,
                                  const cuuint64_t *, const cuuint64_t *, const cuuint32_t *,
                                  const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion,
                                  CUtensorMapFloatOOBfill);

std::once_flag g_encode_once;
EncodeTiledFn g_encode = nullptr;

EncodeTiledFn encode_fn()
{
    std::call_once(g_encode_once, [] {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                             cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            g_encode = reinterpret_cast<EncodeTiledFn>(fn);
        else
            cudaGetLastError();
    });
    return g_encode;
}

}  // namespace

// Rows per chunk for a unit `BW` elements wide: the stage holds CH rows.
static int chunk_rows(int NT, int BW, int es, int stage_bytes)
{
    int row = BW * es;
    if (row <= 0 || row > stage_bytes) return 0;
    int ch = std::min(stage_bytes / row, NT);
    ch = std::min(ch, 256);
    while (ch > 1 && NT % ch) --ch;
    return ch;
}

bool stream_config_valid(int N, int NT, iqa_dtype dtype, const TileConfig &c,
                         std::string *why)
{
    auto fail = [&](const char *m) {
        if (why) *why = m;
        return false;
    };
    const int es = elem_size(dtype);
    const int V = 16 / es;
    if (c.threads != 128 && c.threads != 256 && c.threads != 512)
        return fail("threads must be 128, 256 or 512");
    if (c.stages < 2 || c.stages > 16) return fail("stages must be 2..16");
    if (c.stage_kb != 2 && c.stage_kb != 4 && c.stage_kb != 8 && c.stage_kb != 16)
        return fail("stage_kb must be 2, 4, 8 or 16");
    if (c.ctas_per_sm < 1 || c.ctas_per_sm > 4) return fail("ctas_per_sm must be 1..4");
    if (NT % V) return fail("the TMA kernel needs NT to be a multiple of 16 bytes");
    const int T = N / NT;
    if (c.TX < 1 || c.TX > kMaxTX || T % c.TX) return fail("tiles_across must divide N/NT");
    const int BW = c.TX * NT;
    if (!unit_boxes(N, BW))
        return fail("tiles_across * NT must be <= 256, or a multiple of 256 up to 1024 "
                    "with N a multiple of 256, for the TMA kernel");
    const int LPU = BW / V;
    if (c.TX > 1 && c.threads % LPU) return fail("threads must be a multiple of the unit row");
    if (c.RH < 1 || T % c.RH) return fail("tile rows per unit must divide N/NT");
    if (c.RH > 1 && !segmented_reduce(c.TX, LPU, NT / V))
        return fail("several tile rows per unit need the segmented reduction");
    if (c.RH > 1 && c.RH * segmented_slots(c.threads, c.TX, LPU) > 2 * c.threads)
        return fail("too many tile rows per unit for the reduction slots");
    if (!chunk_rows(NT, BW, es, c.stage_kb * 1024))
        return fail("a unit row does not fit one stage");
    if ((stream_smem_bytes(c.stages, c.stage_kb * 1024, c.threads) + 1024) * c.ctas_per_sm >
        (size_t)228 * 1024)
        return fail("stages * stage_kb exceed shared memory");
    return true;
}

// A unit row of `BW` elements is copied as one 2-D box (BW <= 256) or as a
// 3-D box of BW / 256 segments of 256 elements (BW a multiple of 256, at most
// 1024, and N a multiple of 256); 0 if neither fits.
int unit_boxes(int N, int BW)
{
    if (BW <= 256) return 1;
    if (BW % 256 || N % 256 || BW > 1024) return 0;
    return BW / 256;
}

// Widest unit (whole tiles, <= unit_px pixel pairs, copied as unit_boxes()
// boxes) whose row of 16-byte vectors divides the consumer thread count.
int stream_tiles_across(int N, int NT, iqa_dtype dtype, int threads, long long unit_px)
{
    const int V = 16 / elem_size(dtype);
    const int T = N / NT;
    int best = 1;
    for (int tx = 2; tx <= kMaxTX && tx * NT <= 1024; ++tx) {
        if (T % tx) continue;
        if ((long long)tx * NT * NT > unit_px) break;
        if (threads % (tx * NT / V)) continue;
        if (!unit_boxes(N, tx * NT)) continue;
        best = tx;
    }
    return best;
}

// Most tile rows down a unit of TX tiles across (dividing N / NT) whose
// pixel pairs stay within unit_px and whose per-row reduction slots fit the
// kernel's 2 * threads; 1 where the unit does not take the segmented reduction.
int stream_unit_rows(int N, int NT, iqa_dtype dtype, int threads, int TX, long long unit_px)
{
    const int V = 16 / elem_size(dtype);
    const int T = N / NT, LPU = TX * NT / V, LPT = NT / V;
    if (!segmented_reduce(TX, LPU, LPT)) return 1;
    const int spr = segmented_slots(threads, TX, LPU);
    int best = 1;
    for (int rh = 2; rh * spr <= 2 * threads && (long long)rh * TX * NT * NT <= unit_px; ++rh)
        if (T % rh == 0) best = rh;
    return best;
}

// The unit of a batched launch: as wide as stream_tiles_across() allows, then
// as many tile rows down as stream_unit_rows() allows, for c.unit_kpx.
void stream_unit_shape(TileConfig &c, int N, int NT, iqa_dtype dtype)
{
    const long long unit_px = (long long)c.unit_kpx * 1024;
    c.TX = stream_tiles_across(N, NT, dtype, c.threads, unit_px);
    c.RH = stream_unit_rows(N, NT, dtype, c.threads, c.TX, unit_px);
}

TileConfig default_stream_config(int N, int NT, iqa_dtype dtype)
{
    TileConfig c;
    c.variant = 1;
    c.threads = 256;
    c.stages = 8;
    c.stage_kb = 8;
    c.ctas_per_sm = 1;
    c.TX = stream_tiles_across(N, NT, dtype, c.threads, 16384);
    return c;
}

iqa_status fill_pair_desc(iqa_ctx *ctx, PairDesc *d, const void *x, const void *y, int N,
                          int NT, iqa_dtype dtype, const TileConfig &c, const iqa_params &P,
                          float *lisi, float *aug, double *sums, long long unit_begin)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc) {
        set_error(ctx, "cuTensorMapEncodeTiled is not available from the driver");
        return IQA_ERR_UNSUPPORTED;
    }
    std::memset(d, 0, sizeof *d);
    const int es = elem_size(dtype);
    const int V = 16 / es;
    const int BW = c.TX * NT;
    const int CH = chunk_rows(NT, BW, es, c.stage_kb * 1024);
    CUtensorMapDataType dt = dtype == IQA_F32   ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                             : dtype == IQA_F16 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT16
                                                : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16;
    const int NB = unit_boxes(N, BW);
    // NB == 1: the image as a 2-D array {N, N}, box {BW, CH}.  NB > 1: the
    // image as {256, N / 256, N} (a row of 256-element segments), box
    // {256, NB, CH}, which lands as CH rows of BW contiguous elements.
    const cuuint32_t rank = NB > 1 ? 3 : 2;
    cuuint64_t dims[3], strides[2];
    cuuint32_t box[3];
    if (NB > 1) {
        dims[0] = 256;
        dims[1] = (cuuint64_t)N / 256;
        dims[2] = (cuuint64_t)N;
        strides[0] = (cuuint64_t)256 * es;
        strides[1] = (cuuint64_t)N * es;
        box[0] = 256;
        box[1] = (cuuint32_t)NB;
        box[2] = (cuuint32_t)CH;
    } else {
        dims[0] = (cuuint64_t)N;
        dims[1] = (cuuint64_t)N;
        strides[0] = (cuuint64_t)N * es;
        box[0] = (cuuint32_t)BW;
        box[1] = (cuuint32_t)CH;
    }
    cuuint32_t estr[3] = {1, 1, 1};
    const void *bases[2] = {x, y};
    CUtensorMap *maps[2] = {&d->tmx, &d->tmy};
    for (int i = 0; i < 2; ++i) {
        CUresult r = enc(maps[i], dt, rank, const_cast<void *>(bases[i]), dims, strides, box,
                         estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                         // 128-byte L2 promotion: against 256 bytes, FP16 plans of 32
                         // N=2048 pairs stream 0.3% (N_T = 16) and 0.1% (N_T = 64)
                         // faster, FP32 the same (same box, alternated twice; no
                         // promotion measured the same as 128 bytes)
                         CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) {
            set_error(ctx, "cuTensorMapEncodeTiled failed (%d) for N=%d NT=%d box %dx%d",
                      (int)r, N, NT, BW, CH);
            return IQA_ERR_INVALID_ARG;
        }
    }
    d->lisi = lisi;
    d->aug = aug;
    d->sums = sums;
    d->unit_begin = unit_begin;
    d->N = N;
    d->NT = NT;
    d->T = N / NT;
    d->TX = c.TX;
    d->RH = c.RH;
    d->units_x = d->T / c.TX;
    d->CH = CH;
    d->CPR = NT / CH;
    d->chunks = c.RH * (NT / CH);
    d->LPU = BW / V;
    d->LPT = NT / V;
    d->NB = NB;
    d->C1f = (float)P.C1;
    d->C2f = (float)P.C2;
    d->Cf = (float)P.C;
    d->Df = (float)P.D;
    d->Cd = P.C;
    return IQA_OK;
}

long long pair_units(int N, int NT, const TileConfig &c)
{
    const long long T = N / NT;
    return (T / c.RH) * (T / c.TX);
}

int stream_grid(iqa_ctx *ctx, const TileConfig &c, long long units)
{
    long long g = (long long)ctx->num_sms * c.ctas_per_sm;
    return (int)std::max<long long>(1, std::min<long long>(g, units));
}

cudaError_t launch_stream(const StreamParams &sp, iqa_dtype dtype, const TileConfig &c,
                          int maps, int grid, cudaStream_t st)
{
    size_t smem = stream_smem_bytes(c.stages, c.stage_kb * 1024, c.threads);
    switch (dtype) {
    case IQA_F32: return launch_stream_f32(sp, c.threads, maps, grid, smem, st);
    case IQA_F16: return launch_stream_f16(sp, c.threads, maps, grid, smem, st);
    default: return launch_stream_bf16(sp, c.threads, maps, grid, smem, st);
    }
}

// One pair through the persistent kernel, descriptor inside the parameters.
iqa_status run_stream_pair(iqa_ctx *ctx, const void *x, const void *y, iqa_dtype dtype,
                           int N, int NT, const TileConfig &c, const iqa_params &P,
                           float *lisi, float *aug, double *sums, int maps,
                           cudaStream_t st)
{
    StreamParams sp;
    std::memset(&sp, 0, sizeof sp);
    iqa_status s = fill_pair_desc(ctx, &sp.one_pair, x, y, N, NT, dtype, c, P, lisi, aug,
                                  sums, 0);
    if (s != IQA_OK) return s;
    sp.descs = nullptr;
    sp.npairs = 1;
    sp.stage_bytes = c.stage_kb * 1024;
    sp.stages = c.stages;
    sp.total_units = pair_units(N, NT, c);
    sp.status = ctx->d_status;
    sp.timeout_ns = ctx->wait_timeout_ns;
    sp.sched = nullptr;
    sp.inject_stall = ctx->inject_stall;
    cudaError_t e = launch_stream(sp, dtype, c, maps, stream_grid(ctx, c, sp.total_units), st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "stream kernel launch");
    return IQA_OK;
}

}  // namespace iqa
