// iqa_api.cpp -- the C ABI of include/iqa.h: contexts, argument checks, launch
// shapes, and the plain (one pair per call) LISI / augLISI map path.
#include <cuda_runtime.h>

#include <chrono>
#include <cfloat>
#include <cmath>
#include <cstdarg>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <tuple>
#include <vector>

#include "iqa.h"
#include "iqa_ctx.h"
#include "iqa_internal.h"

using namespace iqa;

namespace {

thread_local std::string g_create_error;

}  // namespace

namespace iqa {

void set_error(iqa_ctx *ctx, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (ctx) {
        std::lock_guard<std::mutex> g(ctx->err_mu);
        ctx->last_error = buf;
    } else {
        g_create_error = buf;
    }
}

iqa_status cuda_fail(iqa_ctx *ctx, cudaError_t e, const char *what)
{
    set_error(ctx, "%s: %s (%s)", what, cudaGetErrorString(e), cudaGetErrorName(e));
    return IQA_ERR_CUDA;
}

int elem_size(iqa_dtype d) { return d == IQA_F32 ? 4 : 2; }

bool dtype_ok(int d) { return d == IQA_F32 || d == IQA_F16 || d == IQA_BF16; }

iqa_status resolve_params(iqa_ctx *ctx, const iqa_params *in, iqa_params *out)
{
    iqa_params p;
    if (in) {
        p = *in;
    } else {
        p.C1 = 1e-6;
        p.C2 = 1e-6;
        p.C = 1e-6;
        p.D = 0.0;
    }
    if (!(std::isfinite(p.C1) && std::isfinite(p.C2) && std::isfinite(p.C) &&
          std::isfinite(p.D))) {
        set_error(ctx, "constants must be finite");
        return IQA_ERR_INVALID_ARG;
    }
    if (!(p.C1 > 0.0) || p.C2 < 0.0 || p.C < 0.0) {
        set_error(ctx, "need C1 > 0, C2 >= 0, C >= 0 (got C1=%g C2=%g C=%g)",
                  p.C1, p.C2, p.C);
        return IQA_ERR_INVALID_ARG;
    }
    // The per-pixel divide of Eq. 1 runs in float32 on d + C1 with a
    // reciprocal that flushes subnormals: C1 must round to a normal float.
    if (p.C1 < (double)FLT_MIN || (float)p.C1 < FLT_MIN) {
        set_error(ctx, "C1=%g is below the smallest normal float32 (%g)", p.C1,
                  (double)FLT_MIN);
        return IQA_ERR_INVALID_ARG;
    }
    if (p.D <= 0.0) p.D = p.C1 / 2.0;
    *out = p;
    return IQA_OK;
}

iqa_status check_shape(iqa_ctx *ctx, int N, int NT)
{
    if (N < 1 || NT < 1 || NT > N || N % NT != 0) {
        set_error(ctx, "need N >= 1, 1 <= NT <= N and NT dividing N (N=%d, NT=%d)",
                  N, NT);
        return IQA_ERR_INVALID_ARG;
    }
    return IQA_OK;
}

static bool divides(long long a, long long b) { return a > 0 && b % a == 0; }

bool config_valid(int N, int NT, iqa_dtype dtype, const TileConfig &c,
                  std::string *why)
{
    const int V = 16 / elem_size(dtype);
    auto fail = [&](const char *m) {
        if (why) *why = m;
        return false;
    };
    if (c.threads != 128 && c.threads != 256 && c.threads != 512)
        return fail("threads must be 128, 256 or 512");
    if (c.vec != V && c.vec != 1) return fail("vec must be the 16-byte width or 1");
    if (c.vec == 1 && (c.threads != 256 || c.ilp != 8))
        return fail("the scalar path runs 256 threads, ilp 8");
    if (c.ilp != 2 && c.ilp != 4 && c.ilp != 8) return fail("ilp must be 2, 4 or 8");
    if (NT % c.vec != 0) return fail("NT is not a whole number of vectors");
    const int T = N / NT;
    if (c.TX < 1 || c.TX > kMaxTX || !divides(c.TX, T))
        return fail("tiles_across must divide N/NT and be <= 64");
    if (c.S < 1 || c.S > kMaxCluster || !divides(c.S, NT))
        return fail("split must divide NT and be <= 8");
    if (c.TX > 1 && c.S > 1) return fail("tiles_across > 1 needs split == 1");
    const long long LPU = (long long)c.TX * (NT / c.vec);
    if (c.TX > 1 && (LPU > c.threads || c.threads % LPU != 0))
        return fail("tiles_across > 1 needs threads to be a multiple of the unit row");
    if ((long long)T * c.S > 65535) return fail("too many tile rows for one launch");
    return true;
}

bool any_config_valid(int N, int NT, iqa_dtype dtype, const TileConfig &c,
                      std::string *why)
{
    if (c.variant == 0) return config_valid(N, NT, dtype, c, why);
    if (c.variant == 1) return stream_config_valid(N, NT, dtype, c, why);
    if (why) *why = "unknown variant";
    return false;
}

// CTAs of the tile kernel in shape c that one SM holds at once (0 if the
// runtime cannot tell), cached per context.
static int tiles_occupancy(iqa_ctx *ctx, iqa_dtype dtype, const TileConfig &c, int maps)
{
    const auto key = std::make_tuple((int)dtype, c.vec * 1000 + c.ilp, c.threads, maps);
    {
        std::lock_guard<std::mutex> g(ctx->cfg_mu);
        auto it = ctx->occupancy.find(key);
        if (it != ctx->occupancy.end()) return it->second;
    }
    TileArgs none;
    std::memset(&none, 0, sizeof none);
    int occ = 0;
    cudaError_t e = dtype == IQA_F32   ? launch_tiles_f32(none, c, maps, 0, nullptr, &occ)
                    : dtype == IQA_F16 ? launch_tiles_f16(none, c, maps, 0, nullptr, &occ)
                                       : launch_tiles_bf16(none, c, maps, 0, nullptr, &occ);
    if (e != cudaSuccess) {
        cudaGetLastError();
        occ = 0;
    }
    std::lock_guard<std::mutex> g(ctx->cfg_mu);
    ctx->occupancy[key] = occ;
    return occ;
}

// Launch shape when nothing was tuned (measured on GB300: 128-thread CTAs
// with 8 loads of each image in flight per thread, and units of up to 16K
// pixel pairs, stream best).  Units shrink for large images so that there are
// at least about six per SM, for load balance, but not below one tile while
// there are at least as many tiles as SMs.  With fewer tiles than SMs (small
// images), each tile gets its own CTA (256 threads once it has 1024 vectors
// per image), and only tiles above 8K pixel pairs (32 KB per image) are split
// over a cluster of CTAs: a cluster launch costs more than it saves on
// smaller tiles (N=256, N_T=64: 7.4 against 8.8 us per isolated launch).
TileConfig default_config(int N, int NT, iqa_dtype dtype, bool aligned,
                          int num_sms)
{
    TileConfig c;
    const int es = elem_size(dtype);
    const int V = 16 / es;
    const int T = N / NT;
    const long long tile_px = (long long)NT * NT;
    const long long img_px = (long long)N * N;
    long long target = (es == 4 ? 16384 : 32768);
    const int sms = num_sms > 0 ? num_sms : 152;
    const bool few_tiles = (long long)T * T < sms;
    const long long balance = img_px / (6LL * sms);
    const long long floor_px =
        few_tiles ? 32768 / es : std::min<long long>(tile_px, target);
    while (target > floor_px && target > balance) target /= 2;
    c.vec = (aligned && NT % V == 0) ? V : 1;
    c.threads = 128;
    const int LPT = NT / c.vec;
    if (tile_px > target) {
        int want = (int)std::min<long long>(kMaxCluster, tile_px / target);
        int S = 1;
        for (int s = want; s >= 1; --s)
            if (NT % s == 0) {
                S = s;
                break;
            }
        c.S = S;
        if (tile_px / S > 4 * target) c.threads = 512;
    } else if (!few_tiles) {
        int best = 1;
        for (int tx = 2; tx <= kMaxTX && tx <= T; ++tx) {
            if (T % tx) continue;
            if ((long long)tx * tile_px > target) break;
            long long lpu = (long long)tx * LPT;
            if (lpu > c.threads || c.threads % lpu) continue;
            best = tx;
        }
        c.TX = best;
    } else if ((long long)NT * LPT >= 1024) {
        c.threads = 256;
    }
    if (c.vec == 1) {
        c.threads = 256;
        c.ilp = 8;
    } else {
        long long vecs = (long long)(NT / c.S) * c.TX * LPT;
        long long per_thread = vecs / c.threads;
        c.ilp = per_thread >= 8 ? 8 : per_thread >= 4 ? 4 : 2;
    }
    return c;
}

// One wave: when the units of a one-pair launch need more than one but at
// most two waves of resident CTAs (the last wave then runs a fraction of the
// GPU and its ramp and tail are paid twice), units twice as wide that fit one
// wave are used instead (N=2048, N_T=64: 512 CTAs of two tiles, 12.96 against
// 14.3 us per isolated launch).  Residency is that of the kernel forming both
// maps (the most registers), whichever maps are requested, so that a map comes
// out of the same launch shape, and so bit for bit the same, in every call.
static TileConfig fit_one_wave(iqa_ctx *ctx, int N, int NT, iqa_dtype dtype, TileConfig c)
{
    const int maps = MAPS_AB;
    if (c.variant != 0 || c.S != 1 || c.vec == 1) return c;
    const int T = N / NT;
    const long long sms = ctx->num_sms > 0 ? ctx->num_sms : 152;
    const int LPT = NT / c.vec;
    const auto ilp_for = [&](const TileConfig &w) {
        const long long per_thread = (long long)NT * w.TX * LPT / w.threads;
        return per_thread >= 8 ? 8 : per_thread >= 4 ? 4 : 2;
    };
    long long units = (long long)(T / c.TX) * T;
    int occ = tiles_occupancy(ctx, dtype, c, maps);
    if (occ <= 0) return c;
    if (units > occ * sms && units <= 2 * occ * sms) {
        for (int tx = c.TX + 1; tx <= std::min(T, kMaxTX); ++tx) {
            if (T % tx || tx % c.TX) continue;
            const long long lpu = (long long)tx * LPT;
            if (lpu > c.threads || c.threads % lpu) continue;
            TileConfig w = c;
            w.TX = tx;
            w.ilp = ilp_for(w);
            const int occ_w = tiles_occupancy(ctx, dtype, w, maps);
            if (occ_w > 0 && (long long)(T / tx) * T <= occ_w * sms) {
                c = w;
                units = (long long)(T / tx) * T;
                occ = occ_w;
                break;
            }
        }
    }
    // A grid that fills at most half of the resident slots leaves load
    // slots unused: wider CTAs put more loads in flight at once, as long as
    // every thread keeps a full batch of 8 vectors and the grid still fits
    // one wave (N=2048, N_T=128: 256 CTAs of 256 threads, 8.3 against 10.2 us
    // per isolated launch).
    while (c.threads < 512 && 2 * units <= occ * sms) {
        TileConfig w = c;
        w.threads = c.threads * 2;
        if ((long long)NT * c.TX * LPT / w.threads < 8) break;
        w.ilp = ilp_for(w);
        const int occ_w = tiles_occupancy(ctx, dtype, w, maps);
        if (occ_w <= 0 || units > occ_w * sms) break;
        c = w;
        occ = occ_w;
    }
    return c;
}

TileConfig pick_config(iqa_ctx *ctx, int N, int NT, iqa_dtype dtype, int maps,
                       bool aligned)
{
    {
        std::lock_guard<std::mutex> g(ctx->cfg_mu);
        auto it = ctx->pinned.find(std::make_tuple((int)dtype, N, NT, maps));
        if (it != ctx->pinned.end()) {
            const TileConfig &c = it->second;
            if ((c.variant == 0 && c.vec == 1) || aligned) return c;
        }
    }
    return fit_one_wave(ctx, N, NT, dtype, default_config(N, NT, dtype, aligned, ctx->num_sms));
}

cudaError_t launch_tiles(const TileArgs &p, const TileConfig &c, iqa_dtype dtype,
                         int maps, int rows, cudaStream_t st)
{
    switch (dtype) {
    case IQA_F32: return launch_tiles_f32(p, c, maps, rows, st, nullptr);
    case IQA_F16: return launch_tiles_f16(p, c, maps, rows, st, nullptr);
    default: return launch_tiles_bf16(p, c, maps, rows, st, nullptr);
    }
}

TileArgs make_args(const void *x, const void *y, int N, int NT,
                   const TileConfig &c, const iqa_params &P, float *lisi,
                   float *aug, double *sums)
{
    TileArgs a;
    a.x = x;
    a.y = y;
    a.N = N;
    a.NT = NT;
    a.T = N / NT;
    a.TX = c.TX;
    a.S = c.S;
    a.RH = NT / c.S;
    a.LPT = NT / c.vec;
    a.LPU = c.TX * a.LPT;
    a.tile_row0 = 0;
    a.C1f = (float)P.C1;
    a.C2f = (float)P.C2;
    a.Cf = (float)P.C;
    a.Df = (float)P.D;
    a.Cd = P.C;
    a.lisi = lisi;
    a.aug = aug;
    a.sums = sums;
    a.overlap = 0;
    return a;
}

static bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Shared body of iqa_lisi / iqa_auglisi / iqa_both.
static iqa_status run_maps(iqa_ctx *ctx, const void *x, const void *y,
                           iqa_dtype dtype, int N, int NT,
                           const iqa_params *params, float *lisi, float *aug,
                           double *sums, iqa_stream stream)
{
    if (!ctx) return IQA_ERR_INVALID_ARG;
    if (!x || !y) {
        set_error(ctx, "x and y must be device pointers, got NULL");
        return IQA_ERR_INVALID_ARG;
    }
    if (!lisi && !aug && !sums) {
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
    const int maps = sums ? MAPS_AB : ((lisi ? MAPS_A : 0) | (aug ? MAPS_B : 0));
    const bool aligned = aligned16(x) && aligned16(y);
    TileConfig c = pick_config(ctx, N, NT, dtype, maps, aligned);
    std::string why;
    if (!any_config_valid(N, NT, dtype, c, &why)) {
        set_error(ctx, "no launch shape for N=%d NT=%d: %s", N, NT, why.c_str());
        return IQA_ERR_UNSUPPORTED;
    }
    if (c.variant == 1)
        return run_stream_pair(ctx, x, y, dtype, N, NT, c, P, lisi, aug, sums, maps,
                               (cudaStream_t)stream);
    TileArgs a = make_args(x, y, N, NT, c, P, lisi, aug, sums);
    a.overlap = ctx->independent_calls;
    cudaError_t e = launch_tiles(a, c, dtype, maps, N / NT, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "tile kernel launch");
    return IQA_OK;
}

}  // namespace iqa

extern "C" {

const char *iqa_version(void) { return "iqa 0.1.0 sm_103a"; }

iqa_status iqa_default_params(iqa_params *p)
{
    if (!p) return IQA_ERR_INVALID_ARG;
    p->C1 = 1e-6;
    p->C2 = 1e-6;
    p->C = 1e-6;
    p->D = 0.5e-6;
    return IQA_OK;
}

iqa_status iqa_create(iqa_ctx **out, int device, size_t hbm_budget_bytes)
{
    if (!out) {
        set_error(nullptr, "out is NULL");
        return IQA_ERR_INVALID_ARG;
    }
    *out = nullptr;
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDeviceCount");
    if (device < 0 || device >= count) {
        set_error(nullptr, "device %d out of range (%d devices)", device, count);
        return IQA_ERR_INVALID_ARG;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    e = cudaSetDevice(device);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaSetDevice");
    iqa_ctx *ctx = new iqa_ctx();
    ctx->device = device;
    ctx->budget = hbm_budget_bytes;
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    cudaDeviceGetAttribute(&ctx->l2_bytes, cudaDevAttrL2CacheSize, device);
    cudaDeviceGetAttribute(&ctx->cc_major, cudaDevAttrComputeCapabilityMajor, device);
    cudaDeviceGetAttribute(&ctx->cc_minor, cudaDevAttrComputeCapabilityMinor, device);
    e = cudaStreamCreateWithFlags(&ctx->s_copy, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->s_comp, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc(&ctx->d_status, 256);
    if (e == cudaSuccess) e = cudaMemset(ctx->d_status, 0, 256);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        iqa_destroy(ctx);
        return cuda_fail(nullptr, e, "context set-up");
    }
    *out = ctx;
    return IQA_OK;
}

void iqa_destroy(iqa_ctx *ctx)
{
    if (!ctx) return;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    if (ctx->s_copy) cudaStreamSynchronize(ctx->s_copy);
    if (ctx->s_comp) cudaStreamSynchronize(ctx->s_comp);
    for (cudaEvent_t ev : ctx->band_events) cudaEventDestroy(ev);
    if (ctx->ws) cudaFree(ctx->ws);
    if (ctx->h_stage) cudaFreeHost(ctx->h_stage);
    if (ctx->d_status) cudaFree(ctx->d_status);
    if (ctx->s_copy) cudaStreamDestroy(ctx->s_copy);
    if (ctx->s_comp) cudaStreamDestroy(ctx->s_comp);
    cudaSetDevice(prev);
    delete ctx;
}

const char *iqa_last_error(const iqa_ctx *ctx)
{
    if (!ctx) return g_create_error.c_str();
    return ctx->last_error.c_str();
}

iqa_status iqa_lisi(iqa_ctx *ctx, const void *x, const void *y, iqa_dtype dtype,
                    int N, int NT, const iqa_params *params, float *map,
                    double *sums, iqa_stream stream)
{
    if (ctx && !map) {
        set_error(ctx, "map is NULL");
        return IQA_ERR_INVALID_ARG;
    }
    return run_maps(ctx, x, y, dtype, N, NT, params, map, nullptr, sums, stream);
}

iqa_status iqa_auglisi(iqa_ctx *ctx, const void *x, const void *y,
                       iqa_dtype dtype, int N, int NT, const iqa_params *params,
                       float *map, double *sums, iqa_stream stream)
{
    if (ctx && !map) {
        set_error(ctx, "map is NULL");
        return IQA_ERR_INVALID_ARG;
    }
    return run_maps(ctx, x, y, dtype, N, NT, params, nullptr, map, sums, stream);
}

iqa_status iqa_both(iqa_ctx *ctx, const void *x, const void *y, iqa_dtype dtype,
                    int N, int NT, const iqa_params *params, float *lisi_map,
                    float *aug_map, double *sums, iqa_stream stream)
{
    return run_maps(ctx, x, y, dtype, N, NT, params, lisi_map, aug_map, sums,
                    stream);
}

iqa_status iqa_get_config(iqa_ctx *ctx, iqa_dtype dtype, int N, int NT, int maps,
                          iqa_launch_config *out)
{
    if (!ctx || !out) return IQA_ERR_INVALID_ARG;
    if (!dtype_ok(dtype) || maps < 1 || maps > 3) {
        set_error(ctx, "bad dtype or maps");
        return IQA_ERR_INVALID_ARG;
    }
    iqa_status s = check_shape(ctx, N, NT);
    if (s != IQA_OK) return s;
    TileConfig c = pick_config(ctx, N, NT, dtype, maps, true);
    out->variant = c.variant;
    out->threads = c.threads;
    out->ilp = c.ilp;
    out->tiles_across = c.TX;
    out->split = c.S;
    out->vector = c.vec == 1 ? 0 : 1;
    out->stages = c.stages;
    out->stage_kb = c.stage_kb;
    out->ctas_per_sm = c.ctas_per_sm;
    out->unit_kpx = c.unit_kpx;
    return IQA_OK;
}

TileConfig from_public(const iqa_launch_config *cfg, iqa_dtype dtype)
{
    TileConfig c;
    c.variant = cfg->variant;
    c.threads = cfg->threads;
    c.ilp = cfg->ilp;
    c.TX = cfg->tiles_across;
    c.S = cfg->split;
    c.vec = cfg->vector ? 16 / elem_size(dtype) : 1;
    c.stages = cfg->stages;
    c.stage_kb = cfg->stage_kb;
    c.ctas_per_sm = cfg->ctas_per_sm;
    c.unit_kpx = cfg->unit_kpx > 0 ? cfg->unit_kpx : 16;
    if (c.variant == 1) {
        c.S = 1;
        c.vec = 16 / elem_size(dtype);
    }
    return c;
}

iqa_status iqa_set_config(iqa_ctx *ctx, iqa_dtype dtype, int N, int NT, int maps,
                          const iqa_launch_config *cfg)
{
    if (!ctx) return IQA_ERR_INVALID_ARG;
    if (!dtype_ok(dtype) || maps < 1 || maps > 3) {
        set_error(ctx, "bad dtype or maps");
        return IQA_ERR_INVALID_ARG;
    }
    iqa_status s = check_shape(ctx, N, NT);
    if (s != IQA_OK) return s;
    auto key = std::make_tuple((int)dtype, N, NT, maps);
    if (!cfg) {
        std::lock_guard<std::mutex> g(ctx->cfg_mu);
        ctx->pinned.erase(key);
        return IQA_OK;
    }
    if (cfg->variant != 0 && cfg->variant != 1) {
        set_error(ctx, "unknown variant %d", cfg->variant);
        return IQA_ERR_UNSUPPORTED;
    }
    TileConfig c = from_public(cfg, dtype);
    std::string why;
    if (!any_config_valid(N, NT, dtype, c, &why)) {
        set_error(ctx, "invalid launch config: %s", why.c_str());
        return IQA_ERR_INVALID_ARG;
    }
    std::lock_guard<std::mutex> g(ctx->cfg_mu);
    ctx->pinned[key] = c;
    return IQA_OK;
}

iqa_status iqa_set_option(iqa_ctx *ctx, int option, long long value)
{
    if (!ctx) return IQA_ERR_INVALID_ARG;
    switch (option) {
    case IQA_OPT_WAIT_TIMEOUT_US:
        if (value < 1 || value > 60000000LL) {
            set_error(ctx, "wait timeout must be 1 us .. 60 s");
            return IQA_ERR_INVALID_ARG;
        }
        ctx->wait_timeout_ns = value * 1000LL;
        return IQA_OK;
    case IQA_OPT_INJECT_STALL:
        if (value != 0 && value != 1) {
            set_error(ctx, "inject-stall takes 0 or 1");
            return IQA_ERR_INVALID_ARG;
        }
        ctx->inject_stall = (int)value;
        return IQA_OK;
    case IQA_OPT_INDEPENDENT_CALLS:
        if (value != 0 && value != 1) {
            set_error(ctx, "independent-calls takes 0 or 1");
            return IQA_ERR_INVALID_ARG;
        }
        ctx->independent_calls = (int)value;
        return IQA_OK;
    default:
        set_error(ctx, "unknown option %d", option);
        return IQA_ERR_INVALID_ARG;
    }
}

#if IQA_CHECKS
extern "C" unsigned int iqa_read_violations_tiles_f32();
extern "C" unsigned int iqa_read_violations_tiles_f16();
extern "C" unsigned int iqa_read_violations_tiles_bf16();
extern "C" unsigned int iqa_read_violations_stream_f32();
extern "C" unsigned int iqa_read_violations_stream_f16();
extern "C" unsigned int iqa_read_violations_stream_bf16();
extern "C" unsigned int iqa_read_violations_synth();
extern "C" unsigned int iqa_read_violations_merge();
#endif

iqa_status iqa_debug_violations(unsigned long long *count)
{
    if (!count) return IQA_ERR_INVALID_ARG;
    *count = 0;
#if IQA_CHECKS
    cudaDeviceSynchronize();
    *count = (unsigned long long)iqa_read_violations_tiles_f32() +
             iqa_read_violations_tiles_f16() + iqa_read_violations_tiles_bf16() +
             iqa_read_violations_stream_f32() + iqa_read_violations_stream_f16() +
             iqa_read_violations_stream_bf16() + iqa_read_violations_synth() +
             iqa_read_violations_merge();
    return IQA_OK;
#else
    return IQA_ERR_UNSUPPORTED;
#endif
}

iqa_status iqa_wait(iqa_ctx *ctx, iqa_stream stream, int timeout_us)
{
    if (!ctx) return IQA_ERR_INVALID_ARG;
    const auto t0 = std::chrono::steady_clock::now();
    for (;;) {
        cudaError_t e = cudaStreamQuery((cudaStream_t)stream);
        if (e == cudaSuccess) break;
        if (e != cudaErrorNotReady) return cuda_fail(ctx, e, "stream");
        auto us = std::chrono::duration_cast<std::chrono::microseconds>(
                      std::chrono::steady_clock::now() - t0)
                      .count();
        if (timeout_us >= 0 && us > timeout_us) {
            set_error(ctx, "stream still busy after %d us", timeout_us);
            return IQA_ERR_TIMEOUT;
        }
        std::this_thread::sleep_for(std::chrono::microseconds(20));
    }
    int code = 0;
    cudaError_t e = cudaMemcpy(&code, ctx->d_status, sizeof code, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status read");
    if (code != 0) {
        cudaMemset(ctx->d_status, 0, sizeof code);
        set_error(ctx, "a device-side wait ran out of time (code %d)", code);
        return IQA_ERR_TIMEOUT;
    }
    return IQA_OK;
}

}  // extern "C"
