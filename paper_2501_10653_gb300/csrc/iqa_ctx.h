// iqa_ctx.h -- the context object behind the opaque iqa_ctx handle.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "iqa.h"
#include "iqa_internal.h"

struct iqa_ctx {
    int device = 0;
    size_t budget = 0;  // 0 = no cap on the context's own allocations
    int num_sms = 0;
    int l2_bytes = 0;
    int cc_major = 0, cc_minor = 0;

    // device error word written by bounded waits in the persistent kernels
    int *d_status = nullptr;
    long long wait_timeout_ns = 1000000000LL;
    int inject_stall = 0;  // test hook, see IQA_OPT_INJECT_STALL
    int independent_calls = 0;  // see IQA_OPT_INDEPENDENT_CALLS

    std::mutex err_mu;
    std::string last_error;

    // launch shapes pinned by iqa_set_config or chosen by the autotuner,
    // keyed by (dtype, N, NT, maps)
    std::mutex cfg_mu;
    std::map<std::tuple<int, int, int, int>, iqa::TileConfig> pinned;
    // resident CTAs per SM of one-pair kernel shapes, keyed by (dtype,
    // vec * 1000 + ilp, threads, maps)
    std::map<std::tuple<int, int, int, int>, int> occupancy;
    // batched-kernel shape per dtype, set by iqa_plan_autotune
    iqa::TileConfig batch_cfg[3];
    bool has_batch_cfg[3] = {false, false, false};

    // workspace of the host-buffer path (iqa_both_host)
    std::mutex host_mu;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    cudaStream_t s_copy = nullptr;
    cudaStream_t s_comp = nullptr;
    std::vector<cudaEvent_t> band_events;
    // page-locked staging for read-backs, so a pageable destination does not
    // block the host thread between pairs
    void *h_stage = nullptr;
    size_t h_stage_bytes = 0;
};

namespace iqa {

void set_error(iqa_ctx *ctx, const char *fmt, ...);
iqa_status cuda_fail(iqa_ctx *ctx, cudaError_t e, const char *what);
int elem_size(iqa_dtype d);
bool dtype_ok(int d);
iqa_status resolve_params(iqa_ctx *ctx, const iqa_params *in, iqa_params *out);
iqa_status check_shape(iqa_ctx *ctx, int N, int NT);
bool config_valid(int N, int NT, iqa_dtype dtype, const TileConfig &c,
                  std::string *why);
TileConfig default_config(int N, int NT, iqa_dtype dtype, bool aligned,
                          int num_sms);
TileConfig pick_config(iqa_ctx *ctx, int N, int NT, iqa_dtype dtype, int maps,
                       bool aligned);
cudaError_t launch_tiles(const TileArgs &p, const TileConfig &c, iqa_dtype dtype,
                         int maps, int rows, cudaStream_t st);
struct PairDesc;
bool stream_config_valid(int N, int NT, iqa_dtype dtype, const TileConfig &c,
                         std::string *why);
TileConfig default_stream_config(int N, int NT, iqa_dtype dtype);
int unit_boxes(int N, int BW);
int stream_tiles_across(int N, int NT, iqa_dtype dtype, int threads, long long unit_px);
int stream_unit_rows(int N, int NT, iqa_dtype dtype, int threads, int TX, long long unit_px);
void stream_unit_shape(TileConfig &c, int N, int NT, iqa_dtype dtype);
iqa_status fill_pair_desc(iqa_ctx *ctx, PairDesc *d, const void *x, const void *y, int N,
                          int NT, iqa_dtype dtype, const TileConfig &c, const iqa_params &P,
                          float *lisi, float *aug, double *sums, long long unit_begin);
long long pair_units(int N, int NT, const TileConfig &c);
int stream_grid(iqa_ctx *ctx, const TileConfig &c, long long units);
iqa_status run_stream_pair(iqa_ctx *ctx, const void *x, const void *y, iqa_dtype dtype,
                           int N, int NT, const TileConfig &c, const iqa_params &P,
                           float *lisi, float *aug, double *sums, int maps,
                           cudaStream_t st);
cudaError_t launch_stream(const StreamParams &sp, iqa_dtype dtype, const TileConfig &c,
                          int maps, int grid, cudaStream_t st);
bool any_config_valid(int N, int NT, iqa_dtype dtype, const TileConfig &c,
                      std::string *why);
TileArgs make_args(const void *x, const void *y, int N, int NT,
                   const TileConfig &c, const iqa_params &P, float *lisi,
                   float *aug, double *sums);

}  // namespace iqa
