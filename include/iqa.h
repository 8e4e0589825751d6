/*
 * iqa.h -- C ABI of libiqa: tile-wise LISI / augLISI image-quality maps on GB300.
 *
 * Method (arxiv 2501.10653, "GPU Accelerated Image Quality Assessment-Based
 * Software for Transient Detection"):
 *   Section 2   negative pixels of both N x N images are set to zero; the images
 *               are cut into N_T x N_T tiles; every tile gets one value.
 *   Eq. 1       lisi_t = D * A_t / (max(Sx_t, Sy_t) + C2)
 *   Eq. 2       auglisi_t = 1 - B_t / (Sx_t + Sy_t + C)
 *   with, over the clamped pixels of tile t,
 *               A_t  = sum |x+y| / (|x-y| + C1)      B_t  = sum |x+y| |x-y|
 *               Sx_t = sum x                         Sy_t = sum y
 *   Section 3   the per-tile values form the IQA matrix, one entry per tile.
 *
 * Conventions shared by every entry point
 *   - Images are N x N, row-major, contiguous (row stride N elements).  Tile t
 *     is at tile-row r = t / (N/N_T), tile-column c = t % (N/N_T), rows in
 *     memory order.  Maps are (N/N_T) x (N/N_T) float32, row-major, entry t.
 *   - The clamp is "v > 0 ? v : 0": NaN and -0 read as 0.  Inputs are never
 *     written: the clamp happens as pixels are loaded.
 *   - Per-tile sums, where requested, are float64 [n][4] = (A, B, Sx, Sy).
 *   - Device-pointer calls are stream-ordered: they validate, enqueue on the
 *     given stream and return without synchronising.  The stream must belong
 *     to the context's device, and that device must be current.
 *   - The map kernels use programmatic dependent launch: each may be
 *     scheduled while the previous kernel in the stream drains, and waits for
 *     it before its first memory access; each lets the next kernel start
 *     early.  A caller's own kernel that follows on the stream with
 *     programmatic stream serialization enabled must wait for its prerequisite
 *     grid (griddepcontrol.wait) before reading the maps; any other work
 *     follows in plain stream order.
 *   - Nothing throws across the ABI: every call returns an iqa_status, and
 *     iqa_last_error() gives a one-line reason for the latest failure.
 *   - The caller owns every buffer it passes; the context owns its workspace.
 *   - A context may be used from several host threads; calls are serialised
 *     internally where they touch context state.
 */
#ifndef IQA_H
#define IQA_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t; NULL means the legacy default stream. */
typedef struct CUstream_st *iqa_stream;

typedef enum {
    IQA_OK = 0,
    IQA_PENDING = 1,           /* iqa_poll: request not finished yet          */
    IQA_ERR_INVALID_ARG = -1,  /* bad shape, pointer, dtype or constant       */
    IQA_ERR_NOMEM = -2,        /* workspace does not fit the HBM budget       */
    IQA_ERR_CUDA = -3,         /* a CUDA call failed (text in last_error)     */
    IQA_ERR_TIMEOUT = -4,      /* a bounded wait ran out                      */
    IQA_ERR_BUSY = -5,         /* queue or slot table full                    */
    IQA_ERR_UNSUPPORTED = -6   /* valid request the compiled library lacks    */
} iqa_status;

/*
 * Pixel storage type of both input images.  Pixels are widened to float32
 * exactly and every sum runs in float32 (compensated), so the maps match the
 * exact Eq. 1 / Eq. 2 values of the STORED pixels to 1e-5 relative in every
 * type.  Against the float32 originals that were rounded to FP16 / BF16,
 * each tile also carries the storage error, which is bounded from the
 * originals alone (per pixel, the rounding moves a clamped value v by at most
 * e(v) = max(u v, eta), u = 2^-11 / 2^-8, eta = 2^-25 / 2^-134 for FP16 /
 * BF16, and 0 for v = 0; with s = x + y, d = |x - y|, t = d + C1 and
 * es = e(x) + e(y)):
 *   |d lisi| <= D (EA M + A EM) / (M max(C2, M - EM)),
 *       EA = sum es (t + s) / (t max(C1, t - es)),  M = max(Sx, Sy) + C2,
 *       EM = max(sum e(x), sum e(y));
 *   |d aug|  <= (EB Q + B EQ) / (Q max(C, Q - EQ)),
 *       EB = sum (es d + s es + es^2),  Q = Sx + Sy + C,  EQ = sum es.
 * The LISI bound is small only where the storage spacing u v stays well
 * below |x - y| + C1; with C1 = 1e-6 it is of the order of LISI itself for
 * pixels above about 2e-3 (FP16) or 2.6e-4 (BF16), i.e. LISI of noisy skies
 * should be computed from FP32 pixels.  augLISI has no such amplification.
 */
typedef enum {
    IQA_F32 = 0,
    IQA_F16 = 1,
    IQA_BF16 = 2
} iqa_dtype;

/*
 * Constants of Eq. 1 and Eq. 2.  Section 1 only says C1, C2, C << 1 and never
 * defines D.  Defaults (iqa_default_params): C1 = C2 = C = 1e-6 and D = C1/2,
 * the value for which identical inputs give LISI -> 1 and every LISI lies in
 * [0, 1].  D <= 0 on input means "use C1/2".  Requirements: C1 at least the
 * smallest normal float32 (about 1.18e-38; the per-pixel divide of Eq. 1 runs
 * in float32), C2 >= 0, C >= 0, all finite.  Range: the per-pixel terms and
 * the tile sums are float32, so (x + y) / C1 summed over a tile must stay
 * below about 3.4e38 (with C1 = 1e-6, pixels far beyond any sky image).
 */
typedef struct {
    double C1;
    double C2;
    double C;
    double D;
} iqa_params;

typedef struct iqa_ctx iqa_ctx;

/* Library version, e.g. "iqa 0.1.0 sm_103a". */
const char *iqa_version(void);

/* Fills *p with the defaults above.  Returns IQA_ERR_INVALID_ARG if p is NULL. */
iqa_status iqa_default_params(iqa_params *p);

/*
 * Creates a context on CUDA device `device`.  hbm_budget_bytes caps the device
 * memory the context may allocate for its own workspace (0 = no cap).  On
 * success *out owns the context; free it with iqa_destroy.
 * Errors: IQA_ERR_INVALID_ARG (out NULL, bad device), IQA_ERR_CUDA.
 */
iqa_status iqa_create(iqa_ctx **out, int device, size_t hbm_budget_bytes);

/* Frees the context and its workspace after waiting for its own streams.
 * NULL is ignored. */
void iqa_destroy(iqa_ctx *ctx);

/*
 * One-line reason for the latest failed call on ctx (or, when ctx is NULL,
 * of iqa_create and the calls that take no context).  The string belongs to the library and stays valid until the
 * next call on the same context.
 */
const char *iqa_last_error(const iqa_ctx *ctx);

/*
 * LISI map (Eq. 1) of the tiles of x and y, from one read of each pixel.
 *   x, y      device pointers, N*N elements of `dtype`, row-major
 *   N, NT     image side and tile side; NT must divide N
 *   params    constants (NULL = defaults)
 *   map       device pointer, (N/NT)^2 float32, written entry t = r*(N/NT)+c
 *   sums      device pointer or NULL; if given, (N/NT)^2 x 4 float64
 *             (A, B, Sx, Sy) per tile
 *   stream    stream to enqueue on
 * Errors: IQA_ERR_INVALID_ARG (NULL input or map, N < 1, NT < 1, N % NT != 0,
 * bad dtype, bad constants), IQA_ERR_CUDA (launch failed).
 */
iqa_status iqa_lisi(iqa_ctx *ctx, const void *x, const void *y, iqa_dtype dtype,
                    int N, int NT, const iqa_params *params, float *map,
                    double *sums, iqa_stream stream);

/* augLISI map (Eq. 2); arguments and errors as for iqa_lisi. */
iqa_status iqa_auglisi(iqa_ctx *ctx, const void *x, const void *y,
                       iqa_dtype dtype, int N, int NT, const iqa_params *params,
                       float *map, double *sums, iqa_stream stream);

/*
 * Both maps from the same single read of each pixel (Eq. 1 and Eq. 2 share the
 * clamp, |x+y|, |x-y| and the pixel sums).  lisi_map or aug_map may be NULL to
 * skip that map, but not both (unless sums is given).  Other arguments and
 * errors as for iqa_lisi.
 */
iqa_status iqa_both(iqa_ctx *ctx, const void *x, const void *y, iqa_dtype dtype,
                    int N, int NT, const iqa_params *params, float *lisi_map,
                    float *aug_map, double *sums, iqa_stream stream);

/*
 * End-to-end form of iqa_both for images in HOST memory (Section 2's host
 * interface: images in, IQA matrix out).  The context uploads x and y to its
 * device workspace on one of its own streams, reduces them on another, and
 * copies the maps (and sums) back to host memory.  Page-locked host buffers
 * give full copy bandwidth; pageable ones work but are slower.  Synchronous:
 * returns when the host outputs are written.
 *   hx, hy               host pointers, N*N elements of dtype
 *   lisi_map, aug_map    host pointers, (N/NT)^2 float32 each, either NULL
 *   sums                 host pointer or NULL, (N/NT)^2 x 4 float64
 * Errors: as iqa_both, plus IQA_ERR_NOMEM when the workspace (both images,
 * maps and sums of the pair) does not fit the context's HBM budget.
 */
iqa_status iqa_both_host(iqa_ctx *ctx, const void *hx, const void *hy,
                         iqa_dtype dtype, int N, int NT,
                         const iqa_params *params, float *lisi_map,
                         float *aug_map, double *sums);

/* One pair of host buffers for iqa_both_host_many (fields as iqa_both_host). */
typedef struct {
    const void *hx;
    const void *hy;
    int N;
    int NT;
    float *lisi_map;
    float *aug_map;
    double *sums;
} iqa_host_pair;

/*
 * iqa_both_host over a sequence of pairs (any mix of N and N_T, one dtype),
 * pipelined: two device slots, so the upload of pair k+1 overlaps the
 * reduction and read-back of pair k and the host-to-device link stays busy.
 * Synchronous: returns when every pair's host outputs are written.
 * Errors: as iqa_both_host (the workspace is two slots of the largest pair).
 */
iqa_status iqa_both_host_many(iqa_ctx *ctx, const iqa_host_pair *pairs, int npairs,
                              iqa_dtype dtype, const iqa_params *params);

/*
 * Launch shape for one (dtype, N, NT, maps) key.  The paper gives each tile
 * one thread block (Section 2).  Two kernels are built:
 *
 * variant 0, the streaming-load kernel: a CTA streams a "unit" of
 * `tiles_across` whole tiles side by side, or 1/`split` of one tile's rows,
 * with 16-byte non-caching loads; the `split` CTAs of a tile form a thread-
 * block cluster that combines its partial sums in distributed shared memory.
 *   threads        128, 256 or 512 threads per CTA
 *   ilp            2, 4 or 8: 16-byte loads of each image in flight per thread
 *   tiles_across   whole tiles per CTA (divides N/NT, <= 64)
 *   split          CTAs per tile (divides NT, <= 8); split > 1 needs
 *                  tiles_across == 1
 *   vector         1: 16-byte loads (needs 16-byte aligned images and NT a
 *                  multiple of 16 bytes); 0: scalar loads, 256 threads, ilp 8
 *
 * variant 1, the persistent TMA kernel: `ctas_per_sm` CTAs per SM loop over
 * units of `tiles_across` whole tiles; a producer warp streams each unit in
 * chunks with tensor copies (one 2-D box for a unit row of at most 256
 * elements; one 3-D box of 256-element segments for a row of 512 or 1024
 * elements when N is a multiple of 256) into a ring of `stages` shared-memory
 * stages of `stage_kb` KB per image, and `threads` consumer threads reduce
 * them.  Needs 16-byte aligned images, NT a multiple of 16 bytes, and
 * tiles_across * NT <= 256, or 512 or 1024 with N a multiple of 256.
 *   threads        128, 256 or 512 consumer threads (plus one producer warp)
 *   tiles_across   whole tiles per unit (one pair: as given, one tile row
 *                  down; plans choose the unit per pair from unit_kpx: the
 *                  widest unit of at most unit_kpx K pixel pairs, then as many
 *                  tile rows down as still fit and divide N/NT, when the unit
 *                  row is reduced by the segmented shuffle tree)
 *   stages         2..16;   stage_kb  2, 4, 8 or 16;   ctas_per_sm  1..4
 * maps: 1 = LISI only, 2 = augLISI only, 3 = both (also used when sums are
 * requested).  Unused fields are ignored.
 */
typedef struct {
    int variant;
    int threads;
    int ilp;
    int tiles_across;
    int split;
    int vector;
    int stages;
    int stage_kb;
    int ctas_per_sm;
    int unit_kpx;
} iqa_launch_config;

/*
 * The launch shape the next call for this key would use with 16-byte aligned
 * inputs: the pinned (or autotuned) one if any, else the built-in heuristic.
 * Errors: IQA_ERR_INVALID_ARG.
 */
iqa_status iqa_get_config(iqa_ctx *ctx, iqa_dtype dtype, int N, int NT, int maps,
                          iqa_launch_config *out);

/*
 * Pins a launch shape for this key (cfg == NULL removes the pin).  Results do
 * not depend on the shape beyond FP32 summation order.
 * Errors: IQA_ERR_INVALID_ARG (shape not valid for this key; reason in
 * iqa_last_error), IQA_ERR_UNSUPPORTED (unknown variant).
 */
iqa_status iqa_set_config(iqa_ctx *ctx, iqa_dtype dtype, int N, int NT, int maps,
                          const iqa_launch_config *cfg);

/*
 * Eq. 3 and Eq. 4 (Section 3): the LISI and augLISI of larger tiles made by
 * merging every m x m block of tiles -- with m = T the whole image -- from the
 * per-tile sums of a previous map call, without re-reading any pixel.  Eq. 3
 * weights lisi_t by max(Sx_t, Sy_t) + C2 (= D A_t by Eq. 1) and Eq. 4 weights
 * auglisi_t by Sx_t + Sy_t + C (= Sx_t + Sy_t + C - B_t by Eq. 2), so both
 * equal Eq. 1 / Eq. 2 on the block's summed (A, B, Sx, Sy); the kernel forms
 * those sums in FP64 and applies the equations once per merged tile.
 *   sums          device (T*T) x 4 float64 (A, B, Sx, Sy), T = N/N_T, tile
 *                 t = r*T + c, as written by iqa_lisi / iqa_auglisi / iqa_both
 *   m             merge factor, divides T
 *   params        the constants used for the tiles (NULL = defaults)
 *   merged_lisi, merged_aug   device (T/m)^2 float32, row-major, or NULL
 *   merged_sums   device (T/m)^2 x 4 float64, or NULL
 * Stream-ordered.  Errors: IQA_ERR_INVALID_ARG, IQA_ERR_CUDA.
 */
iqa_status iqa_merge(iqa_ctx *ctx, const double *sums, int T, int m,
                     const iqa_params *params, float *merged_lisi, float *merged_aug,
                     double *merged_sums, iqa_stream stream);

/* ---------------------------------------------------------------------------
 * Batched form: many pairs, one persistent launch.
 *
 * A plan fixes a list of image pairs (any mix of N and N_T, one storage dtype,
 * one set of constants) and their outputs.  One launch of the persistent
 * TMA-pipelined kernel then computes every pair's maps: its CTAs take units of
 * whole tiles of all pairs from one work list in device memory (largest units
 * first, handed out by a device-side counter), so small images no longer pay
 * a launch and a ramp-up each.  Results of a pair do not depend on the other
 * pairs of the plan (each tile's summation order depends only on the pair's
 * own N, N_T and the plan's launch shape).
 */
typedef struct {
    const void *x;         /* device pointer, N*N elements, 16-byte aligned  */
    const void *y;         /* device pointer, N*N elements, 16-byte aligned  */
    int N;                 /* image side                                      */
    int NT;                /* tile side: divides N, a multiple of 16 bytes,
                              at most 256                                     */
    float *lisi_map;       /* device (N/NT)^2 float32, or NULL                */
    float *aug_map;        /* device (N/NT)^2 float32, or NULL                */
    double *sums;          /* device (N/NT)^2 x 4 float64, or NULL            */
} iqa_pair;

typedef struct iqa_plan iqa_plan;

/* iqa_plan_create flag: capture the launch as a CUDA graph, replayed by
 * iqa_plan_launch. */
#define IQA_PLAN_GRAPH 1
/* iqa_plan_create flag: the caller promises that, whenever the plan is
 * launched, the kernel just before it on the stream does not write the plan's
 * images, does not read its maps or sums, and writes them, if at all, only
 * with the values this launch writes.  The plan's own previous launch
 * qualifies (a plan's results repeat bit for bit), and so does another
 * plan's launch over other outputs.  Each CTA then starts copying its first
 * grab (about 256 KB of each image, 512 KB for 16-bit storage) while that
 * kernel drains, instead of
 * after it completes; every other access, and the launch's completion, still
 * follow it.  Breaking the
 * promise gives wrong maps, not a fault.  Effective for direct launches (a
 * graph replay waits for the previous work anyway). */
#define IQA_PLAN_INDEPENDENT 2

/*
 * Builds a plan over `npairs` pairs: validates them, encodes one TMA tensor
 * map per image, uploads the work-list descriptors to device memory owned by
 * the plan, and (with IQA_PLAN_GRAPH) captures the launch in a CUDA graph.
 * The pair array is copied; the buffers it points to must stay valid while
 * the plan is used.  Synchronous.  The launch shape is the one the context's
 * last iqa_plan_autotune picked for this dtype, else the default: 128
 * consumer threads, 3 CTAs per SM, 2 stages of 16 KB per image, units of 32K
 * pixel pairs for FP32 and 128K for 16-bit storage (iqa_plan_set_config sets
 * another).
 * Errors: IQA_ERR_INVALID_ARG (bad pair, shape, dtype, constants),
 * IQA_ERR_UNSUPPORTED (a pair the TMA kernel cannot stream: unaligned images,
 * NT not a multiple of 16 bytes or above 256), IQA_ERR_NOMEM, IQA_ERR_CUDA.
 */
iqa_status iqa_plan_create(iqa_ctx *ctx, const iqa_pair *pairs, int npairs,
                           iqa_dtype dtype, const iqa_params *params, int flags,
                           iqa_plan **out);

/*
 * Enqueues the plan's launch (graph replay, or a direct launch) on `stream`.
 * Stream-ordered, returns without synchronising.  Launches of the same plan
 * share its work counter, so they must be ordered: issue them on one stream,
 * or order them with events.  (On one stream, an IQA_PLAN_INDEPENDENT plan's
 * launch overlaps the previous kernel only in its first units' copies; it
 * still waits for that kernel before it touches the counter.)
 */
iqa_status iqa_plan_launch(iqa_plan *plan, iqa_stream stream);

/* Frees the plan (its graph, descriptors and counter).  The caller must make
 * sure no launch of the plan is still running.  NULL is ignored. */
void iqa_plan_destroy(iqa_plan *plan);

typedef struct {
    int npairs;
    long long total_units;          /* work-list length                  */
    int grid;                       /* persistent CTAs per launch        */
    unsigned long long input_bytes; /* algorithmic bytes read per launch */
    int graph;                      /* 1 if launches replay a CUDA graph */
    iqa_launch_config config;       /* variant 1 shape in use            */
} iqa_plan_stats;

iqa_status iqa_plan_info(const iqa_plan *plan, iqa_plan_stats *out);

/*
 * Sets the plan's launch shape (variant 1: threads, stages, stage_kb,
 * ctas_per_sm, unit_kpx in 1..1024; the per-pair unit follows from unit_kpx),
 * rebuilds its descriptors and re-captures its graph.  Synchronous; no launch
 * of the plan may be running.  On error the plan keeps its previous shape
 * (unless restoring it fails with IQA_ERR_CUDA, after which the plan can only
 * be destroyed).
 * Errors: IQA_ERR_INVALID_ARG (not variant 1, unit_kpx out of range, or a
 * shape some pair of the plan cannot take), IQA_ERR_CUDA.
 */
iqa_status iqa_plan_set_config(iqa_plan *plan, const iqa_launch_config *cfg);

/*
 * The unit that a plan of launch shape `cfg` (variant 1) streams one pair of
 * side N and tile side NT in, by the rules iqa_plan_create and
 * iqa_plan_set_config apply: *tiles_across whole tiles across (dividing
 * N/NT), *tile_rows tile rows down (dividing N/NT), and *units units in the
 * pair's work list, (N/NT/tile_rows) * (N/NT/tiles_across), taken in
 * row-major order of their first tiles.  A host-only query: needs no GPU and
 * no context.
 * Errors: IQA_ERR_INVALID_ARG (null argument, bad dtype, N, NT or shape, or a
 * shape the pair cannot take); the reason is in iqa_last_error(NULL).
 */
iqa_status iqa_plan_unit_shape(iqa_dtype dtype, int N, int NT, const iqa_launch_config *cfg,
                               int *tiles_across, int *tile_rows, long long *units);

/*
 * Autotuner: times the plan under several launch shapes of the persistent
 * kernel (consumer threads, ring depth, stage size, CTAs per SM, unit size),
 * `iters` launches each on `stream` (synchronising it), re-times the three
 * fastest with 3 * iters launches each, keeps the fastest of those, re-captures
 * the graph, and remembers the shape for later plans of the same dtype on
 * this context.  *best_out (nullable) receives it.
 */
iqa_status iqa_plan_autotune(iqa_plan *plan, iqa_stream stream, int iters,
                             iqa_launch_config *best_out);

/*
 * Waits, at most timeout_us microseconds (< 0: no limit), for `stream` to
 * drain, then reads the context's device status word, which the persistent
 * kernels set when one of their bounded device-side waits runs out.
 * Returns IQA_OK, IQA_ERR_TIMEOUT (stream still busy, or a device-side wait
 * ran out; the status word is then cleared) or IQA_ERR_CUDA.
 */
iqa_status iqa_wait(iqa_ctx *ctx, iqa_stream stream, int timeout_us);

/*
 * Batched launch for callers that cannot allocate device memory.  The paper
 * has no counterpart to this entry point.
 *
 * Some callers must not call cudaMalloc once they are running: a real-time
 * imaging pipeline that reserves all of the GPU's memory for its own buffers
 * at start-up, or one that cannot afford the device-wide synchronisation an
 * allocation may cause between observations.  This call computes the maps
 * of up to IQA_NOALLOC_MAX_PAIRS pairs in one persistent launch, like a plan,
 * but needs no context and allocates nothing: its work-list descriptors, work
 * counter and status word live in one fixed array in device memory, declared
 * in the library (about 25 KB), which every GPU that loads the library keeps
 * until the process exits.  The caller passes the images and the outputs, as
 * in iqa_pair.
 *
 * Set-up: the first call on each device looks up the array's device address
 * (with that device current); make that first call before any stream capture.
 * Every call passes its descriptors by value, as the argument of a small
 * kernel that writes them into the array and clears the counters on `stream`
 * (no host buffer outlives the call), then launches the map kernel there, and
 * returns without synchronising.  All calls share the one array, which keeps
 * the last call's contents: calls whose work overlaps on the GPU (on
 * different streams, or from different threads) race and give wrong maps, so
 * order them on one stream or with events.  A device-side wait that runs out
 * (bounded at 1 s) leaves maps unwritten and is not reported here (the plan
 * path reports it through iqa_wait); a caller that must detect it fills its
 * maps with NaN before the call and checks that none is left.
 * Errors: IQA_ERR_INVALID_ARG (more than IQA_NOALLOC_MAX_PAIRS pairs, a bad
 * pair, dtype or constants), IQA_ERR_UNSUPPORTED (a pair the TMA kernel cannot
 * stream, as for iqa_plan_create), IQA_ERR_CUDA.  Reason: iqa_last_error(NULL).
 */
#define IQA_NOALLOC_MAX_PAIRS 64
iqa_status iqa_batch_noalloc(const iqa_pair *pairs, int npairs, iqa_dtype dtype,
                             const iqa_params *params, iqa_stream stream);

/* ---------------------------------------------------------------------------
 * Serving loop: continuous batching of image-pair requests.
 *
 * Reference skies (first epochs) stay resident on the device.  A request names
 * a reference, a tile side and a seed; its second epoch is rendered on the
 * device from the reference's catalogue (minus the sources the request drops,
 * plus an optional transient) over fresh seeded noise, then the pair's LISI
 * and augLISI maps are computed (Eq. 1, Eq. 2).  A native worker thread
 * admits pending requests in arrival order while they fit the device pool
 * (the admission budget) and the step has room, and launches each step as one
 * CUDA graph: the work-list uploads, one generator launch and one persistent
 * map kernel over all the step's pairs.  Up to max_inflight_steps steps run
 * at once on separate streams, so requests that arrive while others are on
 * the GPU join the next step as memory and slots free up.  A request's maps
 * do not depend on which other requests shared its step.
 */
typedef struct iqa_server iqa_server;
typedef unsigned long long iqa_handle;

/* A reference catalogue: Gaussian-beam sources at integer centres, each with a
 * float32 1-D profile g[-h..h]; source i adds (flux_i * g[dy]) * g[dx] to the
 * pixel at offset (dy, dx) from its centre.  All arrays are host memory and
 * are copied. */
typedef struct {
    int N;                  /* image side, a multiple of 64, at most 2^20 */
    int nsrc;
    const int *x;           /* source centres, columns */
    const int *y;           /* source centres, rows */
    const float *flux;      /* peak flux */
    const int *half;        /* profile half-width h (window 2h+1, h <= 64) */
    const int *profile_off; /* start of source i's profile in `profile` */
    const float *profile;
    int nprofile;           /* floats in `profile` */
    float noise_sigma;      /* sigma of each epoch's noise */
} iqa_catalog;
/* (at most 64 sources' windows may meet any 64 x 64 block of the image) */

typedef struct {
    iqa_dtype dtype;           /* storage of references and epochs */
    int max_pairs_per_step;    /* 1..64 */
    int max_inflight_steps;    /* 1..8 */
    size_t pool_bytes;         /* device memory for second epochs: the admission
                                  budget (a request needs N*N elements) */
    int one_pair_per_launch;   /* 1: the plain path as a baseline -- one request
                                  per step, the streaming-load kernel, no graph */
    int simulate;              /* 1: no GPU work; a step completes after
                                  bytes / sim_bytes_per_s (host-side tests);
                                  2: steps never complete (a stalled source) */
    double sim_bytes_per_s;
    double step_timeout_ms;    /* host watchdog: a step still running after this
                                  fails its requests with IQA_ERR_TIMEOUT (its
                                  buffers stay reserved until it ends); 0 = 10 s */
    unsigned long long max_step_bytes; /* cap on a step's input bytes (2 N^2 per
                                  pair; a larger request still runs alone), so a
                                  large request does not hold small ones back;
                                  0 = no cap */
    iqa_params params;
    int generator_blocks_per_sm; /* resident epoch-generator blocks per SM,
                                  1..8 (0 = 8, every SM full): fewer leave
                                  room for other steps' map kernels */
    int map_ctas_per_sm;       /* persistent map-kernel CTAs per SM, 1..4
                                  (0 = the context's batched shape) */
    int time_kernels;          /* 1: timing marks around each step's generator
                                  and map kernel (the mean_step_* and *_per_pair
                                  statistics); they cut the launch overlap
                                  between the two kernels, adding about 10 us
                                  to a small step's latency, so 0 by default */
} iqa_server_config;

typedef struct {
    int ref_id;                /* a reference added with iqa_server_add_reference */
    int NT;                    /* tile side: divides N, multiple of 16 bytes, <= 256 */
    unsigned long long seed;   /* noise seed of the second epoch */
    int ndrop;                 /* 0..8 catalogue sources left out of epoch 2 */
    int drop[8];
    int add_src;               /* -1, or a source whose profile a transient uses */
    int add_x, add_y;          /* transient centre */
    float add_flux;            /* transient peak flux */
} iqa_request;

typedef struct {
    long long submitted, completed, failed, pending, inflight, steps;
    double p50_ms, p99_ms, max_ms, mean_ms;  /* submit -> maps on the host */
    double pairs_per_s;        /* completed / (last completion - first submit) */
    double input_gb_per_s;     /* algorithmic input bytes of completed pairs / s */
    double mean_pairs_per_step;
    unsigned long long pool_bytes, pool_peak_bytes;
    /* medians over completed requests of the latency's parts: submission ->
     * the start of its step's launch calls (queueing), the launch calls
     * themselves (host), and the rest (device work, read-back, detection) */
    double p50_queue_ms, p50_launch_ms, p50_device_ms;
    /* device time of the steps' two kernels, from timing marks around them
     * in each step (the epoch generator, then the map kernel): means per step
     * and per completed pair; 0 unless the server was created with
     * time_kernels = 1 */
    double mean_step_generator_ms, mean_step_map_ms;
    double generator_ms_per_pair, map_ms_per_pair;
} iqa_server_stats;

/* Creates a server on ctx's device (ctx may be NULL with simulate = 1) and
 * starts its worker thread.  Allocates the pool and per-step buffers.
 * Errors: IQA_ERR_INVALID_ARG, IQA_ERR_NOMEM, IQA_ERR_CUDA. */
iqa_status iqa_server_create(iqa_ctx *ctx, const iqa_server_config *cfg,
                             iqa_server **out);

/* Renders the reference's first epoch on the device (seed `seed`) and keeps it
 * and its catalogue resident under `ref_id`.  Synchronous.
 * Errors: IQA_ERR_INVALID_ARG (bad catalogue or id in use), IQA_ERR_NOMEM. */
iqa_status iqa_server_add_reference(iqa_server *srv, int ref_id, const iqa_catalog *cat,
                                    unsigned long long seed);

/*
 * The serving loop's sky generator as a call of its own: renders one epoch of
 * `cat` on the device -- its sources minus drop[0..ndrop), plus a transient
 * with source add_src's profile at (add_x, add_y) and peak add_flux when
 * add_src >= 0, over noise from `seed` -- rounded to nearest into `dtype` at
 * `out` (device, N*N elements, 16-byte aligned).  The catalogue is uploaded for the call and
 * freed after it; the call waits for the render to finish.  The recipe (a
 * counter-based Philox4x32-10 draw per four pixels, each word's byte sum an
 * Irwin-Hall standard normal stand-in, sources added in catalogue order) is
 * reproducible on the host bit for bit.
 * Errors: IQA_ERR_INVALID_ARG (bad catalogue, drop list or transient, or a
 * misaligned `out`),
 * IQA_ERR_NOMEM, IQA_ERR_CUDA.
 */
iqa_status iqa_render_epoch(iqa_ctx *ctx, const iqa_catalog *cat, unsigned long long seed,
                            const int *drop, int ndrop, int add_src, int add_x, int add_y,
                            float add_flux, iqa_dtype dtype, void *out);

/* Copies a resident reference image (N*N storage elements) to host memory. */
iqa_status iqa_server_reference_image(iqa_server *srv, int ref_id, void *host_out);

/* Queues a request; *out identifies it.  Returns at once.
 * Errors: IQA_ERR_INVALID_ARG (unknown reference, bad N_T or drop list),
 * IQA_ERR_NOMEM (the request alone exceeds the pool), IQA_ERR_BUSY (queue full). */
iqa_status iqa_submit(iqa_server *srv, const iqa_request *req, iqa_handle *out);

/* Waits at most timeout_us (0: just look) for the request.  Returns IQA_OK
 * (maps ready), IQA_PENDING (not yet), IQA_ERR_TIMEOUT (a device-side wait of
 * its step ran out, see IQA_OPT_WAIT_TIMEOUT_US), IQA_ERR_CUDA, or
 * IQA_ERR_INVALID_ARG (unknown handle). */
iqa_status iqa_poll(iqa_server *srv, iqa_handle h, int timeout_us);

/* For a finished request: copies its maps ((N/NT)^2 float32 each, either
 * pointer may be NULL) and its latency, then forgets the request. */
iqa_status iqa_result(iqa_server *srv, iqa_handle h, float *lisi_map, float *aug_map,
                      double *latency_ms);

iqa_status iqa_server_get_stats(iqa_server *srv, iqa_server_stats *out);

/*
 * Load generator (a simulated imaging cadence): submits reqs[i] at arrival_s[i]
 * seconds after the call, timing each arrival on a steady clock in the calling
 * thread, then waits up to timeout_s for every one of them to finish.  The
 * maps of these requests are dropped when they finish; the latency statistics
 * (iqa_server_get_stats) keep them.  Returns IQA_OK, IQA_ERR_TIMEOUT (not all
 * finished in time), or the first iqa_submit error.
 */
iqa_status iqa_server_run_trace(iqa_server *srv, const iqa_request *reqs,
                                const double *arrival_s, int n, double timeout_s);

/* Stops the worker after the steps in flight, frees everything. */
void iqa_server_destroy(iqa_server *srv);

/* Context options for iqa_set_option. */
typedef enum {
    /* Bound, in microseconds, on every device-side wait of the persistent
     * kernels (default 1000000).  A wait that runs out makes the kernel record
     * an error in the status word, stop, and return (see iqa_wait). */
    IQA_OPT_WAIT_TIMEOUT_US = 1,
    /* Fault injection for tests of the failure path: 1 makes the producer warp
     * of the persistent kernels issue no copies, so every consumer wait runs
     * out; 0 (default) is normal operation. */
    IQA_OPT_INJECT_STALL = 2,
    /* 1: the caller promises, for every later iqa_lisi / iqa_auglisi /
     * iqa_both call on this context that runs the streaming-load kernel, the
     * same as IQA_PLAN_INDEPENDENT does for a plan: the kernel just before the
     * call on the stream does not write the call's images, does not read its
     * maps or sums, and writes them, if at all, only with the values this
     * call writes (a stream of calls over other outputs, or the same call
     * repeated, qualifies).  Each CTA then loads and reduces its pixels while
     * that kernel drains, and waits for it only before writing its maps, so
     * the call's writes and completion still follow it.  Breaking the promise
     * gives wrong maps, not a fault.  0 (default): every CTA waits before its
     * first access. */
    IQA_OPT_INDEPENDENT_CALLS = 3
} iqa_option;

/*
 * Checked build only (libiqa_checked.so, compiled with IQA_CHECKS=1): every
 * kernel checks the geometry of each access -- unit and tile bounds, tensor
 * copy coordinates and their 16-byte alignment, stage capacity, output tile
 * indices, generator pixel indices -- counts each failed check and skips the
 * access.  Synchronises the current device, returns the number of failed
 * checks since the previous call in *count, and resets it.  The product
 * library compiles no checks and returns IQA_ERR_UNSUPPORTED.
 */
iqa_status iqa_debug_violations(unsigned long long *count);

/* Sets a context option.  Errors: IQA_ERR_INVALID_ARG (unknown option or
 * value out of range: the timeout must be 1 us .. 60 s). */
iqa_status iqa_set_option(iqa_ctx *ctx, int option, long long value);

#ifdef __cplusplus
}
#endif

#endif /* IQA_H */
