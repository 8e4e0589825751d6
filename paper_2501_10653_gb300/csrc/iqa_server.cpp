// iqa_server.cpp -- the serving loop: resident reference skies, device-side
// second epochs, admission by a device-memory budget, continuous batching of
// requests into steps, one CUDA graph per step slot, p50/p99 latency.
//
// A native worker thread owns every GPU action.  Each pass it (1) retires
// steps whose completion event has fired (maps copied to the requests, pool
// memory returned), (2) marks steps that ran past the host-side step timeout
// as failed, and (3) if a step slot is free, admits pending requests in
// arrival order while they fit the pool and the step, and launches the step:
// fill the slot's page-locked work tables, replay the slot's graph (table
// uploads -> epoch generator -> persistent map kernel, all reading their work
// counts from device memory), read the maps back, record the event.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "iqa.h"
#include "iqa_ctx.h"
#include "iqa_stream.cuh"
#include "iqa_synth.h"

namespace iqa {
TileConfig default_batch_config(iqa_dtype dtype);
}

using namespace iqa;

namespace {

using Clock = std::chrono::steady_clock;

double ms_between(Clock::time_point a, Clock::time_point b)
{
    return std::chrono::duration<double, std::milli>(b - a).count();
}

size_t round_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// First-fit allocator over the offsets [0, size) of the device pool.
class RangeAllocator {
public:
    void reset(size_t size)
    {
        size_ = size;
        used_ = peak_ = 0;
        free_.clear();
        if (size) free_[0] = size;
    }
    bool alloc(size_t bytes, size_t *off)
    {
        bytes = round_up(bytes, 256);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second < bytes) continue;
            *off = it->first;
            const size_t rest = it->second - bytes, start = it->first + bytes;
            free_.erase(it);
            if (rest) free_[start] = rest;
            used_ += bytes;
            peak_ = std::max(peak_, used_);
            return true;
        }
        return false;
    }
    void release(size_t off, size_t bytes)
    {
        bytes = round_up(bytes, 256);
        used_ -= bytes;
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
    size_t size() const { return size_; }
    size_t peak() const { return peak_; }

private:
    size_t size_ = 0, used_ = 0, peak_ = 0;
    std::map<size_t, size_t> free_;
};

struct Reference {
    int N = 0;
    int nsrc = 0;
    SynthCatalog *d_cat = nullptr;  // device struct
    void *d_arrays = nullptr;       // catalogue arrays
    void *d_image = nullptr;        // resident first epoch
};

enum ReqState { REQ_PENDING, REQ_INFLIGHT, REQ_DONE, REQ_FAILED };

struct Request {
    iqa_handle h = 0;
    iqa_request r{};
    Reference ref;  // copied at submission (references are never removed)
    int N = 0, T = 0;
    size_t epoch_bytes = 0, pool_off = 0;
    ReqState state = REQ_PENDING;
    iqa_status status = IQA_PENDING;
    bool discard = false;  // drop the maps (and the record) when finished
    // submission, the start and the end of its step's launch calls, completion
    Clock::time_point t_submit, t_launch, t_launched, t_done;
    std::vector<float> lisi, aug;
};

struct Slot {
    bool busy = false;
    bool timed_out = false;
    std::vector<std::shared_ptr<Request>> reqs;
    size_t out_floats = 0;
    unsigned long long bytes = 0;
    Clock::time_point t_launch;
    cudaStream_t st = nullptr;
    cudaEvent_t ev = nullptr;
    // timing marks of the step's device work: before the epoch generator,
    // between it and the map kernel, after the map kernel
    cudaEvent_t mark[3] = {nullptr, nullptr, nullptr};
    // the step's work tables, one block in page-locked memory and its device
    // copy (one upload per step): generator header {njobs, total_bins}, map
    // kernel header {npairs, total_units}, generator jobs, pair descriptors
    unsigned char *h_tab = nullptr, *d_tab = nullptr;
    size_t tab_bytes = 0;
    SynthJob *d_jobs = nullptr, *h_jobs = nullptr;
    long long *d_synth_hdr = nullptr, *h_synth_hdr = nullptr;
    PairDesc *d_pairs = nullptr, *h_pairs = nullptr;
    long long *d_dyn = nullptr, *h_dyn = nullptr;
    unsigned long long *d_sched = nullptr;
    // the persistent kernel's error word: page-locked and mapped, so the
    // device writes it (only on a failed wait) and the host reads and clears
    // it with no copies on the step's stream
    int *d_status = nullptr;
    volatile int *h_status = nullptr;
    // the step's maps: h_out is page-locked and mapped (m_out is its device
    // address); a batched step's map kernel writes the maps there directly,
    // the one-pair baseline writes d_out and copies it back
    float *d_out = nullptr, *h_out = nullptr, *m_out = nullptr;
    size_t out_cap = 0;
    // one graph per grid size: a step launches the smallest persistent grid
    // that covers its units, so small steps leave SMs to concurrent steps
    cudaGraph_t graph[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaGraphExec_t exec[4] = {nullptr, nullptr, nullptr, nullptr};
    int grid[4] = {0, 0, 0, 0};
};

}  // namespace

struct iqa_server {
    iqa_ctx *ctx = nullptr;
    iqa_server_config cfg{};
    iqa_params P{};
    TileConfig kcfg;  // persistent-kernel shape
    int es = 4;
    int synth_grid = 0;
    int device = 0;
    double step_timeout_ms = 10000.0;

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::atomic<bool> stop{false};
    std::atomic<unsigned long long> n_submitted{0};  // read by the worker without mu
    std::thread worker;

    std::unordered_map<int, Reference> refs;
    std::deque<std::shared_ptr<Request>> pending;
    std::unordered_map<iqa_handle, std::shared_ptr<Request>> all;
    iqa_handle next_handle = 1;
    std::vector<Slot> slots;
    RangeAllocator pool;
    void *d_pool = nullptr;

    // statistics
    long long submitted = 0, completed = 0, failed = 0, steps = 0, step_pairs = 0;
    std::vector<double> latencies;
    // per completed request: submission -> launch, the launch calls, and the
    // rest (device work, read-back and completion detection)
    std::vector<double> lat_queue, lat_launch, lat_device;
    double bytes_done = 0.0;
    // summed device time of the steps' generator and map kernels
    double gen_ms = 0.0, map_ms = 0.0;
    long long marked_steps = 0, marked_pairs = 0;
    bool have_first = false;
    Clock::time_point t_first, t_last;
    std::string worker_error;
};

namespace {

const size_t kMaxQueue = 1 << 20;
// A batched step's map kernel writes its maps straight to mapped host memory,
// whatever their size: that saves the read-back copy, one operation on the
// step's stream.  Measured on the serving trace (10 s, 2000 req/s, same box,
// twice): against a read-back copy above 64K floats, p99 0.83 instead of
// 0.84-0.86 ms and an idle N = 16384 request 0.473 instead of 0.487 ms; no
// change for small requests, which were direct already.

void free_slot(Slot &s)
{
    for (int g = 0; g < 4; ++g) {
        if (s.exec[g]) cudaGraphExecDestroy(s.exec[g]);
        if (s.graph[g]) cudaGraphDestroy(s.graph[g]);
    }
    cudaFree(s.d_tab);
    cudaFree(s.d_sched);
    cudaFree(s.d_out);
    cudaFreeHost(s.h_tab);
    cudaFreeHost(const_cast<int *>(s.h_status));
    cudaFreeHost(s.h_out);
    if (s.ev) cudaEventDestroy(s.ev);
    for (cudaEvent_t m : s.mark)
        if (m) cudaEventDestroy(m);
    if (s.st) cudaStreamDestroy(s.st);
    s = Slot();
}

StreamParams slot_stream_params(const iqa_server *srv, const Slot &s)
{
    StreamParams sp;
    std::memset(&sp, 0, sizeof sp);
    sp.descs = s.d_pairs;
    sp.stage_bytes = srv->kcfg.stage_kb * 1024;
    sp.stages = srv->kcfg.stages;
    sp.status = s.d_status;
    sp.timeout_ns = srv->ctx->wait_timeout_ns;
    sp.sched = s.d_sched;
    sp.inject_stall = srv->ctx->inject_stall;
    sp.dyn = s.d_dyn;
    return sp;
}

// The slot's graphs: work-table uploads, the epoch generator and the
// persistent map kernel, all sized from device-side headers; graph g = 0..3
// runs the kernels on 1/8, 1/4, 1/2 or all of the full persistent grid.
cudaError_t capture_slot(iqa_server *srv, Slot &s)
{
    const int full = srv->ctx->num_sms * srv->kcfg.ctas_per_sm;
    const int div[4] = {8, 4, 2, 1};
    for (int g = 0; g < 4; ++g) {
        const int grid = std::max(1, full / div[g]);
        const int sgrid = std::max(1, srv->synth_grid / div[g]);
        s.grid[g] = grid;
        cudaError_t e = cudaStreamBeginCapture(s.st, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return e;
        cudaError_t e1 =
            cudaMemcpyAsync(s.d_tab, s.h_tab, s.tab_bytes, cudaMemcpyHostToDevice, s.st);
        const bool marks = srv->cfg.time_kernels != 0;
        if (e1 == cudaSuccess && marks)
            e1 = cudaEventRecordWithFlags(s.mark[0], s.st, cudaEventRecordExternal);
        if (e1 == cudaSuccess)
            e1 = launch_synth((int)srv->cfg.dtype, s.d_jobs, s.d_synth_hdr, sgrid, s.st);
        if (e1 == cudaSuccess && marks)
            e1 = cudaEventRecordWithFlags(s.mark[1], s.st, cudaEventRecordExternal);
        if (e1 == cudaSuccess) {
            StreamParams sp = slot_stream_params(srv, s);
            e1 = launch_stream(sp, srv->cfg.dtype, srv->kcfg, MAPS_AB, grid, s.st);
        }
        if (e1 == cudaSuccess && marks)
            e1 = cudaEventRecordWithFlags(s.mark[2], s.st, cudaEventRecordExternal);
        e = cudaStreamEndCapture(s.st, &s.graph[g]);
        if (e1 != cudaSuccess) return e1;
        if (e != cudaSuccess) return e;
        e = cudaGraphInstantiate(&s.exec[g], s.graph[g], 0);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

cudaError_t alloc_slot(iqa_server *srv, Slot &s)
{
    const int M = srv->cfg.max_pairs_per_step;
    cudaError_t e = cudaStreamCreateWithFlags(&s.st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s.ev, cudaEventDisableTiming);
    for (int m = 0; m < 3 && e == cudaSuccess; ++m) e = cudaEventCreate(&s.mark[m]);
    // table block: headers at 0 and 16, jobs at 64, descriptors 64-aligned
    const size_t off_jobs = 64;
    const size_t off_pairs = round_up(off_jobs + sizeof(SynthJob) * M, 64);
    s.tab_bytes = off_pairs + sizeof(PairDesc) * M;
    if (e == cudaSuccess) e = cudaMalloc(&s.d_tab, s.tab_bytes);
    if (e == cudaSuccess) e = cudaMalloc(&s.d_sched, 256);
    if (e == cudaSuccess) e = cudaMemset(s.d_sched, 0, 256);
    if (e == cudaSuccess) e = cudaMallocHost(&s.h_tab, s.tab_bytes);
    if (e == cudaSuccess) {
        int *hs = nullptr;
        e = cudaHostAlloc(&hs, 256, cudaHostAllocMapped);
        if (e == cudaSuccess) {
            std::memset(hs, 0, 256);
            s.h_status = hs;
            e = cudaHostGetDevicePointer(&s.d_status, hs, 0);
        }
    }
    if (e == cudaSuccess) {
        std::memset(s.h_tab, 0, s.tab_bytes);
        e = cudaMemset(s.d_tab, 0, s.tab_bytes);
        s.h_synth_hdr = reinterpret_cast<long long *>(s.h_tab);
        s.h_dyn = s.h_synth_hdr + 2;
        s.h_jobs = reinterpret_cast<SynthJob *>(s.h_tab + off_jobs);
        s.h_pairs = reinterpret_cast<PairDesc *>(s.h_tab + off_pairs);
        s.d_synth_hdr = reinterpret_cast<long long *>(s.d_tab);
        s.d_dyn = s.d_synth_hdr + 2;
        s.d_jobs = reinterpret_cast<SynthJob *>(s.d_tab + off_jobs);
        s.d_pairs = reinterpret_cast<PairDesc *>(s.d_tab + off_pairs);
    }
    if (e == cudaSuccess && !srv->cfg.one_pair_per_launch) {
        // one launch of each kernel with empty work before capture, so that
        // launch attributes are set outside the capture
        e = launch_synth((int)srv->cfg.dtype, s.d_jobs, s.d_synth_hdr, srv->synth_grid, s.st);
        if (e == cudaSuccess) {
            StreamParams sp = slot_stream_params(srv, s);
            e = launch_stream(sp, srv->cfg.dtype, srv->kcfg, MAPS_AB,
                              srv->ctx->num_sms * srv->kcfg.ctas_per_sm, s.st);
        }
        if (e == cudaSuccess) e = cudaStreamSynchronize(s.st);
        if (e == cudaSuccess) e = capture_slot(srv, s);
    }
    return e;
}

// Makes room for the step's maps in the slot's page-locked buffer and, for a
// step that copies its maps back (device_copy), its device buffer.
cudaError_t ensure_out(Slot &s, size_t floats, bool device_copy)
{
    if (floats <= s.out_cap && (!device_copy || s.d_out)) return cudaSuccess;
    size_t cap = std::max(floats, s.out_cap * 2);
    cudaFree(s.d_out);
    cudaFreeHost(s.h_out);
    s.d_out = nullptr;
    s.h_out = nullptr;
    s.m_out = nullptr;
    s.out_cap = 0;
    cudaError_t e = device_copy ? cudaMalloc(&s.d_out, cap * sizeof(float)) : cudaSuccess;
    if (e == cudaSuccess) e = cudaHostAlloc(&s.h_out, cap * sizeof(float), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer(&s.m_out, s.h_out, 0);
    if (e == cudaSuccess) s.out_cap = cap;
    return e;
}

// Fills the slot's tables for its requests and launches the step.
iqa_status launch_step(iqa_server *srv, Slot &s)
{
    iqa_ctx *ctx = srv->ctx;
    const bool sim = srv->cfg.simulate != 0;
    size_t floats = 0;
    unsigned long long bytes = 0;
    for (auto &r : s.reqs) {
        floats += 2 * (size_t)r->T * r->T;
        bytes += 2ull * r->N * r->N * srv->es;
    }
    s.out_floats = floats;
    s.bytes = bytes;
    s.t_launch = Clock::now();
    s.timed_out = false;
    if (sim) return IQA_OK;

    // maps straight to host memory (no read-back copy), except in the
    // one-pair baseline
    const bool direct = !srv->cfg.one_pair_per_launch;
    cudaError_t e = ensure_out(s, floats, !direct);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "step output buffers");
    // the slot's previous step has finished: clear its error word
    *s.h_status = 0;
    float *out = direct ? s.m_out : s.d_out;
    char *pool = static_cast<char *>(srv->d_pool);
    long long blocks = 0, units = 0;
    size_t o = 0;
    const int n = (int)s.reqs.size();
    for (int k = 0; k < n; ++k) {
        Request &r = *s.reqs[k];
        const Reference &ref = r.ref;
        void *epoch = pool + r.pool_off;
        SynthJob &j = s.h_jobs[k];
        std::memset(&j, 0, sizeof j);
        j.cat = ref.d_cat;
        j.out = epoch;
        j.blocks_begin = blocks;
        j.seed = r.r.seed;
        j.N = r.N;
        j.ndrop = r.r.ndrop;
        for (int d = 0; d < r.r.ndrop; ++d) j.drop[d] = r.r.drop[d];
        j.add_src = r.r.add_src;
        j.add_x = r.r.add_x;
        j.add_y = r.r.add_y;
        j.add_flux = r.r.add_flux;
        blocks += (long long)(r.N / kSynthBin) * (r.N / kSynthBin);
        float *dl = out + o, *da = out + o + (size_t)r.T * r.T;
        o += 2 * (size_t)r.T * r.T;
        if (srv->cfg.one_pair_per_launch) continue;
        TileConfig c = srv->kcfg;
        stream_unit_shape(c, r.N, r.r.NT, srv->cfg.dtype);
        iqa_status st = fill_pair_desc(ctx, &s.h_pairs[k], ref.d_image, epoch, r.N, r.r.NT,
                                       srv->cfg.dtype, c, srv->P, dl, da, nullptr, units);
        if (st != IQA_OK) return st;
        units += pair_units(r.N, r.r.NT, c);
    }
    s.h_synth_hdr[0] = n;
    s.h_synth_hdr[1] = blocks;
    s.h_dyn[0] = n;
    s.h_dyn[1] = units;
    if (srv->cfg.one_pair_per_launch) {
        // baseline: the plain path, one pair, no graph
        Request &r = *s.reqs[0];
        const Reference &ref = r.ref;
        // headers and the one job: the start of the table block
        e = cudaMemcpyAsync(s.d_tab, s.h_tab,
                            reinterpret_cast<unsigned char *>(s.h_jobs + 1) - s.h_tab,
                            cudaMemcpyHostToDevice, s.st);
        const bool marks = srv->cfg.time_kernels != 0;
        if (e == cudaSuccess && marks) e = cudaEventRecord(s.mark[0], s.st);
        if (e == cudaSuccess)
            e = launch_synth((int)srv->cfg.dtype, s.d_jobs, s.d_synth_hdr, srv->synth_grid, s.st);
        if (e == cudaSuccess && marks) e = cudaEventRecord(s.mark[1], s.st);
        if (e == cudaSuccess) {
            TileConfig c = pick_config(ctx, r.N, r.r.NT, srv->cfg.dtype, MAPS_AB, true);
            if (c.variant == 1) {
                iqa_status st = run_stream_pair(ctx, ref.d_image, pool + r.pool_off,
                                                srv->cfg.dtype, r.N, r.r.NT, c, srv->P,
                                                s.d_out, s.d_out + (size_t)r.T * r.T, nullptr,
                                                MAPS_AB, s.st);
                if (st != IQA_OK) return st;
            } else {
                TileArgs a = make_args(ref.d_image, pool + r.pool_off, r.N, r.r.NT, c, srv->P,
                                       s.d_out, s.d_out + (size_t)r.T * r.T, nullptr);
                e = launch_tiles(a, c, srv->cfg.dtype, MAPS_AB, r.T, s.st);
            }
        }
        if (e == cudaSuccess && marks) e = cudaEventRecord(s.mark[2], s.st);
    } else {
        int g = 0;
        while (g < 3 && s.grid[g] < units) ++g;
        e = cudaGraphLaunch(s.exec[g], s.st);
    }
    if (e == cudaSuccess && !direct)
        e = cudaMemcpyAsync(s.h_out, s.d_out, floats * sizeof(float), cudaMemcpyDeviceToHost,
                            s.st);
    if (e == cudaSuccess) e = cudaEventRecord(s.ev, s.st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "step launch");
    return IQA_OK;
}

// True when the slot's step has finished (its GPU work, or its modelled time).
bool step_finished(iqa_server *srv, Slot &s, iqa_status *st)
{
    *st = IQA_OK;
    if (srv->cfg.simulate) {
        // a completion source that stalls (until the server is destroyed)
        if (srv->cfg.simulate == 2) return srv->stop.load();
        const double need_ms = 1e3 * (double)s.bytes / std::max(1.0, srv->cfg.sim_bytes_per_s);
        return ms_between(s.t_launch, Clock::now()) >= need_ms;
    }
    cudaError_t e = cudaEventQuery(s.ev);
    if (e == cudaErrorNotReady) return false;
    if (e != cudaSuccess) {
        *st = IQA_ERR_CUDA;
        return true;
    }
    if (*s.h_status != 0) *st = IQA_ERR_TIMEOUT;
    return true;
}

void finish_request(iqa_server *srv, Request &r, iqa_status st, Clock::time_point now)
{
    r.t_done = now;
    r.status = st;
    r.state = st == IQA_OK ? REQ_DONE : REQ_FAILED;
    if (st == IQA_OK) {
        ++srv->completed;
        srv->latencies.push_back(ms_between(r.t_submit, now));
        srv->lat_queue.push_back(ms_between(r.t_submit, r.t_launch));
        srv->lat_launch.push_back(ms_between(r.t_launch, r.t_launched));
        srv->lat_device.push_back(ms_between(r.t_launched, now));
        srv->bytes_done += 2.0 * r.N * r.N * srv->es;
        srv->t_last = now;
    } else {
        ++srv->failed;
    }
}

// Called with srv->mu held.
void retire(iqa_server *srv, Slot &s)
{
    iqa_status st;
    if (!step_finished(srv, s, &st)) {
        if (!s.timed_out && srv->step_timeout_ms > 0 &&
            ms_between(s.t_launch, Clock::now()) > srv->step_timeout_ms) {
            // host-side watchdog: the step's requests fail now; its buffers stay
            // reserved until its GPU work (if any) really ends
            s.timed_out = true;
            const auto now = Clock::now();
            for (auto &r : s.reqs)
                if (r->state == REQ_INFLIGHT) {
                    finish_request(srv, *r, IQA_ERR_TIMEOUT, now);
                    if (r->discard) srv->all.erase(r->h);
                }
            srv->cv_done.notify_all();
        }
        return;
    }
    const auto now = Clock::now();
    if (st == IQA_OK && !srv->cfg.simulate && srv->cfg.time_kernels) {
        // device time of the step's two kernels, from its timing marks
        float gen = 0.0f, map = 0.0f;
        if (cudaEventElapsedTime(&gen, s.mark[0], s.mark[1]) == cudaSuccess &&
            cudaEventElapsedTime(&map, s.mark[1], s.mark[2]) == cudaSuccess) {
            srv->gen_ms += gen;
            srv->map_ms += map;
            ++srv->marked_steps;
            srv->marked_pairs += (long long)s.reqs.size();
        } else {
            cudaGetLastError();
        }
    }
    size_t o = 0;
    for (auto &rp : s.reqs) {
        Request &r = *rp;
        const size_t n = (size_t)r.T * r.T;
        if (r.state == REQ_INFLIGHT) {
            if (r.discard) {
                // nothing kept
            } else if (st == IQA_OK && !srv->cfg.simulate) {
                r.lisi.assign(s.h_out + o, s.h_out + o + n);
                r.aug.assign(s.h_out + o + n, s.h_out + o + 2 * n);
            } else if (st == IQA_OK) {
                r.lisi.assign(n, 0.0f);
                r.aug.assign(n, 0.0f);
            }
            finish_request(srv, r, st, now);
        }
        if (r.discard) srv->all.erase(r.h);
        o += 2 * n;
        srv->pool.release(r.pool_off, r.epoch_bytes);
    }
    s.reqs.clear();
    s.busy = false;
    srv->cv_done.notify_all();
}

// The worker keeps polling for this long after its last step before it
// blocks on the condition variable (one host core while requests flow).
constexpr double kIdleSpinMs = 5.0;
// Longest stretch of polling without the lock before the worker takes it to
// run its watchdog and admission checks.
constexpr double kPollSliceMs = 0.1;

// True when a busy slot's step looks finished.  Worker thread only: slots are
// written by the worker alone, so this needs no lock.
bool any_step_ready(iqa_server *srv)
{
    for (auto &s : srv->slots) {
        if (!s.busy) continue;
        iqa_status st;
        if (step_finished(srv, s, &st)) return true;
    }
    return false;
}

// Polls, without holding srv->mu, until a step finishes, a request arrives,
// the server stops, or kPollSliceMs pass.
void poll_unlocked(iqa_server *srv, unsigned long long seen)
{
    const auto t0 = Clock::now();
    while (!any_step_ready(srv)) {
        if (srv->n_submitted.load(std::memory_order_acquire) != seen) return;
        if (srv->stop.load()) return;
        if (ms_between(t0, Clock::now()) > kPollSliceMs) return;
        std::this_thread::yield();
    }
}

// The worker holds srv->mu only for bookkeeping (retiring steps, admission,
// statistics); GPU calls and polling run without it, so that submitters and
// pollers never wait behind a launch.
void worker_main(iqa_server *srv)
{
    if (!srv->cfg.simulate) cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lk(srv->mu);
    Clock::time_point t_active = Clock::now();
    while (true) {
        bool any_busy = false;
        for (auto &s : srv->slots) {
            if (s.busy) retire(srv, s);
            any_busy = any_busy || s.busy;
        }
        if (srv->stop && !any_busy) break;
        // admit and launch on a free slot
        Slot *free_slot_p = nullptr;
        for (auto &s : srv->slots)
            if (!s.busy) {
                free_slot_p = &s;
                break;
            }
        bool launched = false;
        if (!srv->stop && free_slot_p && !srv->pending.empty()) {
            Slot &s = *free_slot_p;
            const int cap = srv->cfg.one_pair_per_launch ? 1 : srv->cfg.max_pairs_per_step;
            unsigned long long step_bytes = 0;
            while ((int)s.reqs.size() < cap && !srv->pending.empty()) {
                auto r = srv->pending.front();
                const unsigned long long rb = 2ull * r->epoch_bytes;
                if (srv->cfg.max_step_bytes && !s.reqs.empty() &&
                    step_bytes + rb > srv->cfg.max_step_bytes)
                    break;
                size_t off = 0;
                if (!srv->pool.alloc(r->epoch_bytes, &off)) break;  // arrival order kept
                step_bytes += rb;
                r->pool_off = off;
                r->state = REQ_INFLIGHT;
                srv->pending.pop_front();
                s.reqs.push_back(r);
            }
            if (!s.reqs.empty()) {
                s.busy = true;
                ++srv->steps;
                srv->step_pairs += (long long)s.reqs.size();
                // the slot's requests are the worker's alone until retired
                lk.unlock();
                const iqa_status st = launch_step(srv, s);
                const auto t_launched = Clock::now();
                for (auto &r : s.reqs) {
                    r->t_launch = s.t_launch;
                    r->t_launched = t_launched;
                }
                lk.lock();
                if (st != IQA_OK) {
                    // nothing was enqueued that will complete: fail and release now
                    const auto now = Clock::now();
                    for (auto &r : s.reqs) {
                        finish_request(srv, *r, st, now);
                        srv->pool.release(r->pool_off, r->epoch_bytes);
                        if (r->discard) srv->all.erase(r->h);
                    }
                    srv->worker_error = iqa_last_error(srv->ctx);
                    s.reqs.clear();
                    s.busy = false;
                    srv->cv_done.notify_all();
                }
                launched = true;
            }
        }
        if (launched || any_busy) t_active = Clock::now();
        if (!launched) {
            if (any_busy || ms_between(t_active, Clock::now()) < kIdleSpinMs) {
                // a step is on the GPU, or one ended moments ago: poll at
                // once, without the lock (a timed sleep, or a wake-up through
                // the condition variable, would add the kernel's timer slack
                // or scheduling delay, tens of microseconds, to the next
                // request's latency)
                const unsigned long long seen =
                    srv->n_submitted.load(std::memory_order_acquire);
                lk.unlock();
                poll_unlocked(srv, seen);
                lk.lock();
            } else {
                srv->cv_work.wait_for(lk, std::chrono::microseconds(2000));
            }
        }
    }
}

// Copies a catalogue and its 64x64 bin lists to one device allocation
// (*d_arrays), with the SynthCatalog struct at its end (*d_cat).
iqa_status upload_catalog(iqa_ctx *ctx, const iqa_catalog *cat, void **d_arrays,
                          SynthCatalog **d_cat)
{
    const int N = cat->N, n = cat->nsrc;
    const int bpr = (N + kSynthBin - 1) / kSynthBin;
    // catalogue bins: every source whose window meets a bin, in catalogue order
    std::vector<std::vector<int>> bins((size_t)bpr * bpr);
    for (int i = 0; i < n; ++i) {
        const int h = cat->half[i];
        const int r0 = std::max(0, cat->y[i] - h) / kSynthBin;
        const int r1 = std::min(N - 1, cat->y[i] + h) / kSynthBin;
        const int c0 = std::max(0, cat->x[i] - h) / kSynthBin;
        const int c1 = std::min(N - 1, cat->x[i] + h) / kSynthBin;
        for (int br = r0; br <= r1; ++br)
            for (int bc = c0; bc <= c1; ++bc) bins[(size_t)br * bpr + bc].push_back(i);
    }
    for (const auto &bl : bins)
        if (bl.size() > 64) {
            set_error(ctx, "a 64x64 bin meets %zu sources (at most 64)", bl.size());
            return IQA_ERR_INVALID_ARG;
        }
    std::vector<int> start(bins.size() + 1, 0), flat;
    for (size_t b = 0; b < bins.size(); ++b) {
        start[b + 1] = start[b] + (int)bins[b].size();
        flat.insert(flat.end(), bins[b].begin(), bins[b].end());
    }
    if (flat.empty()) flat.push_back(0);
    // one allocation for every array: x, y, half, poff, flux, profile, bins
    const size_t sz_i = sizeof(int) * (size_t)std::max(n, 1);
    size_t off[9];
    size_t total = 0;
    const size_t sizes[8] = {sz_i, sz_i, sz_i, sz_i, sizeof(float) * (size_t)std::max(n, 1),
                             sizeof(float) * (size_t)std::max(cat->nprofile, 1),
                             sizeof(int) * start.size(), sizeof(int) * flat.size()};
    for (int k = 0; k < 8; ++k) {
        off[k] = total;
        total += round_up(sizes[k], 256);
    }
    off[8] = total;
    total += round_up(sizeof(SynthCatalog), 256);
    cudaError_t e = cudaMalloc(d_arrays, total);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *d_arrays = nullptr;
        set_error(ctx, "catalogue of %zu bytes does not fit: %s", total, cudaGetErrorString(e));
        return IQA_ERR_NOMEM;
    }
    char *base = static_cast<char *>(*d_arrays);
    const void *src[8] = {cat->x, cat->y, cat->half, cat->profile_off, cat->flux,
                          cat->profile, start.data(), flat.data()};
    const size_t copy_sizes[8] = {sizeof(int) * (size_t)n, sizeof(int) * (size_t)n,
                                  sizeof(int) * (size_t)n, sizeof(int) * (size_t)n,
                                  sizeof(float) * (size_t)n,
                                  sizeof(float) * (size_t)cat->nprofile,
                                  sizeof(int) * start.size(), sizeof(int) * flat.size()};
    for (int k = 0; k < 8 && e == cudaSuccess; ++k)
        if (copy_sizes[k])
            e = cudaMemcpy(base + off[k], src[k], copy_sizes[k], cudaMemcpyHostToDevice);
    SynthCatalog hc;
    hc.nsrc = n;
    hc.N = N;
    hc.bins_per_row = bpr;
    hc.noise_sigma = cat->noise_sigma;
    hc.x = reinterpret_cast<const int *>(base + off[0]);
    hc.y = reinterpret_cast<const int *>(base + off[1]);
    hc.half = reinterpret_cast<const int *>(base + off[2]);
    hc.profile_off = reinterpret_cast<const int *>(base + off[3]);
    hc.flux = reinterpret_cast<const float *>(base + off[4]);
    hc.profile = reinterpret_cast<const float *>(base + off[5]);
    hc.bin_start = reinterpret_cast<const int *>(base + off[6]);
    hc.bin_src = reinterpret_cast<const int *>(base + off[7]);
    *d_cat = reinterpret_cast<SynthCatalog *>(base + off[8]);
    if (e == cudaSuccess) e = cudaMemcpy(*d_cat, &hc, sizeof hc, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "catalogue upload");
    return IQA_OK;
}

// Renders one epoch of an uploaded catalogue into `out` and waits for it.
iqa_status render_one(iqa_ctx *ctx, SynthCatalog *d_cat, int N, unsigned long long seed,
                      const int *drop, int ndrop, int add_src, int add_x, int add_y,
                      float add_flux, iqa_dtype dtype, void *out, cudaStream_t st)
{
    SynthJob j;
    std::memset(&j, 0, sizeof j);
    j.cat = d_cat;
    j.out = out;
    j.seed = seed;
    j.N = N;
    j.ndrop = ndrop;
    for (int k = 0; k < ndrop; ++k) j.drop[k] = drop[k];
    j.add_src = add_src;
    j.add_x = add_x;
    j.add_y = add_y;
    j.add_flux = add_flux;
    long long hdr[2] = {1, (long long)(N / kSynthBin) * (N / kSynthBin)};
    void *tmp = nullptr;
    cudaError_t e = cudaMalloc(&tmp, sizeof j + 16);
    if (e == cudaSuccess) e = cudaMemcpy(tmp, &j, sizeof j, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaMemcpy(static_cast<char *>(tmp) + sizeof j, hdr, 16, cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = launch_synth((int)dtype, static_cast<SynthJob *>(tmp),
                         reinterpret_cast<long long *>(static_cast<char *>(tmp) + sizeof j),
                         ctx->num_sms * kSynthBlocksPerSM, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(tmp);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "epoch render");
    return IQA_OK;
}

iqa_status upload_reference(iqa_server *srv, Reference &ref, const iqa_catalog *cat,
                            unsigned long long seed)
{
    iqa_ctx *ctx = srv->ctx;
    iqa_status s = upload_catalog(ctx, cat, &ref.d_arrays, &ref.d_cat);
    if (s != IQA_OK) return s;
    const size_t img_bytes = (size_t)cat->N * cat->N * srv->es;
    cudaError_t e = cudaMalloc(&ref.d_image, img_bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        ref.d_image = nullptr;
        set_error(ctx, "reference of %zu bytes does not fit: %s", img_bytes,
                  cudaGetErrorString(e));
        return IQA_ERR_NOMEM;
    }
    return render_one(ctx, ref.d_cat, cat->N, seed, nullptr, 0, -1, 0, 0, 0.0f,
                      srv->cfg.dtype, ref.d_image, ctx->s_comp);
}

iqa_status check_catalog(iqa_ctx *ctx, const iqa_catalog *c)
{
    if (!c || c->N < kSynthBin || c->N % kSynthBin || c->N > (1 << 20) || c->nsrc < 0 ||
        c->nprofile < 0 ||
        (c->nsrc > 0 && (!c->x || !c->y || !c->flux || !c->half || !c->profile_off ||
                         !c->profile))) {
        set_error(ctx, "bad catalogue (N a multiple of 64 up to 2^20, arrays for nsrc sources)");
        return IQA_ERR_INVALID_ARG;
    }
    for (int i = 0; i < c->nsrc; ++i) {
        if (c->half[i] < 0 || c->half[i] > 64 || c->profile_off[i] < 0 ||
            c->profile_off[i] + 2 * c->half[i] + 1 > c->nprofile || c->x[i] < 0 ||
            c->x[i] >= c->N || c->y[i] < 0 || c->y[i] >= c->N) {
            set_error(ctx, "catalogue source %d out of range", i);
            return IQA_ERR_INVALID_ARG;
        }
    }
    return IQA_OK;
}

}  // namespace

extern "C" {

iqa_status iqa_server_create(iqa_ctx *ctx, const iqa_server_config *cfg, iqa_server **out)
{
    if (!out || !cfg) return IQA_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cfg->simulate && !ctx) return IQA_ERR_INVALID_ARG;
    if (!dtype_ok(cfg->dtype) || cfg->max_pairs_per_step < 1 || cfg->max_pairs_per_step > 64 ||
        cfg->max_inflight_steps < 1 || cfg->max_inflight_steps > 8 || cfg->pool_bytes < 256 ||
        cfg->simulate < 0 || cfg->simulate > 2 || !(cfg->step_timeout_ms >= 0) ||
        cfg->generator_blocks_per_sm < 0 || cfg->generator_blocks_per_sm > kSynthBlocksPerSM ||
        cfg->map_ctas_per_sm < 0 || cfg->map_ctas_per_sm > 4 || cfg->time_kernels < 0 ||
        cfg->time_kernels > 1) {
        set_error(ctx, "bad server config (max_pairs_per_step 1..64, max_inflight_steps "
                       "1..8, pool_bytes > 0, generator_blocks_per_sm 0..8, "
                       "map_ctas_per_sm 0..4, time_kernels 0..1)");
        return IQA_ERR_INVALID_ARG;
    }
    iqa_params P;
    iqa_status s = resolve_params(ctx, &cfg->params, &P);
    if (s != IQA_OK) return s;
    auto srv = std::make_unique<iqa_server>();
    srv->ctx = ctx;
    srv->cfg = *cfg;
    srv->P = P;
    srv->kcfg = default_batch_config(cfg->dtype);
    srv->es = elem_size(cfg->dtype);
    srv->step_timeout_ms = cfg->step_timeout_ms > 0 ? cfg->step_timeout_ms : 10000.0;
    srv->pool.reset(cfg->pool_bytes);
    srv->slots.resize(cfg->max_inflight_steps);
    if (!cfg->simulate) {
        {
            std::lock_guard<std::mutex> g(ctx->cfg_mu);
            if (ctx->has_batch_cfg[cfg->dtype]) srv->kcfg = ctx->batch_cfg[cfg->dtype];
        }
        // serving steps are latency-bound: units of 16K pixel pairs (an eighth
        // of the batched form's 16-bit default) spread a small request over
        // more CTAs (served p50 0.079 against 0.089 ms with 32K units)
        srv->kcfg.unit_kpx = 16;
        if (cfg->map_ctas_per_sm > 0) {
            TileConfig k = srv->kcfg;
            k.ctas_per_sm = cfg->map_ctas_per_sm;
            std::string why;
            // the shape's shared memory must fit the requested CTAs per SM
            if (!stream_config_valid(1024, 64, cfg->dtype, k, &why)) {
                set_error(ctx, "map_ctas_per_sm %d: %s", cfg->map_ctas_per_sm, why.c_str());
                return IQA_ERR_INVALID_ARG;
            }
            srv->kcfg = k;
        }
        srv->device = ctx->device;
        srv->synth_grid = ctx->num_sms * (cfg->generator_blocks_per_sm > 0
                                              ? cfg->generator_blocks_per_sm
                                              : kSynthBlocksPerSM);
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(ctx->device);
        if (ctx->budget && cfg->pool_bytes > ctx->budget) {
            cudaSetDevice(prev);
            set_error(ctx, "pool of %zu bytes exceeds the context's HBM budget",
                      cfg->pool_bytes);
            return IQA_ERR_NOMEM;
        }
        cudaError_t e = cudaMalloc(&srv->d_pool, cfg->pool_bytes);
        if (e != cudaSuccess) {
            cudaGetLastError();
            cudaSetDevice(prev);
            set_error(ctx, "pool of %zu bytes: %s", cfg->pool_bytes, cudaGetErrorString(e));
            return IQA_ERR_NOMEM;
        }
        for (auto &sl : srv->slots) {
            e = alloc_slot(srv.get(), sl);
            if (e != cudaSuccess) break;
        }
        cudaSetDevice(prev);
        if (e != cudaSuccess) {
            iqa_server *raw = srv.release();
            iqa_server_destroy(raw);
            return cuda_fail(ctx, e, "server step buffers");
        }
    }
    iqa_server *raw = srv.release();
    raw->worker = std::thread(worker_main, raw);
    *out = raw;
    return IQA_OK;
}

iqa_status iqa_server_add_reference(iqa_server *srv, int ref_id, const iqa_catalog *cat,
                                    unsigned long long seed)
{
    if (!srv) return IQA_ERR_INVALID_ARG;
    iqa_status s = check_catalog(srv->ctx, cat);
    if (s != IQA_OK) return s;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        if (srv->refs.count(ref_id)) {
            set_error(srv->ctx, "reference %d already added", ref_id);
            return IQA_ERR_INVALID_ARG;
        }
    }
    Reference ref;
    ref.N = cat->N;
    ref.nsrc = cat->nsrc;
    if (!srv->cfg.simulate) {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(srv->device);
        s = upload_reference(srv, ref, cat, seed);
        cudaSetDevice(prev);
        if (s != IQA_OK) {
            cudaFree(ref.d_arrays);
            cudaFree(ref.d_image);
            return s;
        }
    }
    std::lock_guard<std::mutex> g(srv->mu);
    srv->refs[ref_id] = ref;
    return IQA_OK;
}

iqa_status iqa_render_epoch(iqa_ctx *ctx, const iqa_catalog *cat, unsigned long long seed,
                            const int *drop, int ndrop, int add_src, int add_x, int add_y,
                            float add_flux, iqa_dtype dtype, void *out)
{
    if (!ctx || !out) return IQA_ERR_INVALID_ARG;
    if (!dtype_ok(dtype)) {
        set_error(ctx, "unknown dtype %d", (int)dtype);
        return IQA_ERR_INVALID_ARG;
    }
    if (reinterpret_cast<uintptr_t>(out) % 16 != 0) {
        set_error(ctx, "out must be 16-byte aligned");
        return IQA_ERR_INVALID_ARG;
    }
    iqa_status s = check_catalog(ctx, cat);
    if (s != IQA_OK) return s;
    if (ndrop < 0 || ndrop > kSynthMaxDrop || (ndrop && !drop) || add_src >= cat->nsrc ||
        (add_src >= 0 && (add_x < 0 || add_x >= cat->N || add_y < 0 || add_y >= cat->N))) {
        set_error(ctx, "bad drop list or transient");
        return IQA_ERR_INVALID_ARG;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    void *arrays = nullptr;
    SynthCatalog *d_cat = nullptr;
    s = upload_catalog(ctx, cat, &arrays, &d_cat);
    if (s == IQA_OK)
        s = render_one(ctx, d_cat, cat->N, seed, drop, ndrop, add_src, add_x, add_y, add_flux,
                       dtype, out, ctx->s_comp);
    cudaFree(arrays);
    cudaSetDevice(prev);
    return s;
}

iqa_status iqa_server_reference_image(iqa_server *srv, int ref_id, void *host_out)
{
    if (!srv || !host_out || srv->cfg.simulate) return IQA_ERR_INVALID_ARG;
    Reference ref;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        auto it = srv->refs.find(ref_id);
        if (it == srv->refs.end()) {
            set_error(srv->ctx, "unknown reference %d", ref_id);
            return IQA_ERR_INVALID_ARG;
        }
        ref = it->second;
    }
    cudaError_t e = cudaMemcpy(host_out, ref.d_image, (size_t)ref.N * ref.N * srv->es,
                               cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(srv->ctx, e, "reference read-back");
    return IQA_OK;
}

static iqa_status submit_impl(iqa_server *srv, const iqa_request *req, iqa_handle *out,
                              bool discard)
{
    if (!srv || !req || !out) return IQA_ERR_INVALID_ARG;
    auto r = std::make_shared<Request>();
    r->r = *req;
    r->discard = discard;
    r->t_submit = Clock::now();
    std::lock_guard<std::mutex> g(srv->mu);
    auto it = srv->refs.find(req->ref_id);
    if (it == srv->refs.end()) {
        set_error(srv->ctx, "unknown reference %d", req->ref_id);
        return IQA_ERR_INVALID_ARG;
    }
    const int N = it->second.N;
    const int V = 16 / srv->es;
    if (req->NT < 1 || N % req->NT || req->NT % V || req->NT > 256 || req->ndrop < 0 ||
        req->ndrop > kSynthMaxDrop) {
        set_error(srv->ctx, "bad request: NT must divide N=%d, be a multiple of 16 bytes and "
                            "<= 256; at most %d drops", N, kSynthMaxDrop);
        return IQA_ERR_INVALID_ARG;
    }
    if (req->add_src >= 0) {
        // the transient borrows an existing source's profile
        if (req->add_src >= it->second.nsrc || req->add_x < 0 || req->add_x >= N ||
            req->add_y < 0 || req->add_y >= N) {
            set_error(srv->ctx, "transient: source index or centre out of range");
            return IQA_ERR_INVALID_ARG;
        }
    }
    r->ref = it->second;
    r->N = N;
    r->T = N / req->NT;
    r->epoch_bytes = (size_t)N * N * srv->es;
    if (round_up(r->epoch_bytes, 256) > srv->pool.size()) {
        set_error(srv->ctx, "request needs %zu bytes, more than the pool of %zu",
                  r->epoch_bytes, srv->pool.size());
        return IQA_ERR_NOMEM;
    }
    if (srv->pending.size() >= kMaxQueue) {
        set_error(srv->ctx, "queue full");
        return IQA_ERR_BUSY;
    }
    r->h = srv->next_handle++;
    if (!srv->have_first) {
        srv->have_first = true;
        srv->t_first = r->t_submit;
    }
    ++srv->submitted;
    srv->pending.push_back(r);
    srv->all[r->h] = r;
    *out = r->h;
    srv->n_submitted.fetch_add(1, std::memory_order_release);
    srv->cv_work.notify_one();
    return IQA_OK;
}

iqa_status iqa_submit(iqa_server *srv, const iqa_request *req, iqa_handle *out)
{
    return submit_impl(srv, req, out, false);
}

iqa_status iqa_server_run_trace(iqa_server *srv, const iqa_request *reqs,
                                const double *arrival_s, int n, double timeout_s)
{
    if (!srv || !reqs || !arrival_s || n < 0) return IQA_ERR_INVALID_ARG;
    long long base_done;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        base_done = srv->completed + srv->failed;
    }
    const auto t0 = Clock::now();
    for (int i = 0; i < n; ++i) {
        const auto due = t0 + std::chrono::duration_cast<Clock::duration>(
                                  std::chrono::duration<double>(arrival_s[i]));
        while (Clock::now() < due) {
        }
        iqa_handle h;
        iqa_status s = submit_impl(srv, &reqs[i], &h, true);
        if (s != IQA_OK) return s;
    }
    std::unique_lock<std::mutex> lk(srv->mu);
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(timeout_s));
    const bool ok = srv->cv_done.wait_until(lk, deadline, [&] {
        return srv->completed + srv->failed - base_done >= n;
    });
    if (!ok) {
        set_error(srv->ctx, "trace not finished after %.1f s", timeout_s);
        return IQA_ERR_TIMEOUT;
    }
    return IQA_OK;
}

iqa_status iqa_poll(iqa_server *srv, iqa_handle h, int timeout_us)
{
    if (!srv) return IQA_ERR_INVALID_ARG;
    std::unique_lock<std::mutex> lk(srv->mu);
    auto it = srv->all.find(h);
    if (it == srv->all.end()) {
        set_error(srv->ctx, "unknown handle %llu", h);
        return IQA_ERR_INVALID_ARG;
    }
    auto r = it->second;
    auto ready = [&] { return r->state == REQ_DONE || r->state == REQ_FAILED; };
    if (!ready() && timeout_us > 0)
        srv->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), ready);
    if (!ready()) return IQA_PENDING;
    if (r->state == REQ_FAILED && srv->ctx) {
        std::lock_guard<std::mutex> g(srv->ctx->err_mu);
        srv->ctx->last_error = r->status == IQA_ERR_TIMEOUT
                                   ? "request's step ran out of time (device or host watchdog)"
                                   : "request's step failed: " + srv->worker_error;
    }
    return r->status;
}

iqa_status iqa_result(iqa_server *srv, iqa_handle h, float *lisi_map, float *aug_map,
                      double *latency_ms)
{
    if (!srv) return IQA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(srv->mu);
    auto it = srv->all.find(h);
    if (it == srv->all.end()) {
        set_error(srv->ctx, "unknown handle %llu", h);
        return IQA_ERR_INVALID_ARG;
    }
    auto r = it->second;
    if (r->state == REQ_PENDING || r->state == REQ_INFLIGHT) return IQA_PENDING;
    if (r->state == REQ_FAILED) {
        srv->all.erase(it);
        return r->status;
    }
    const size_t n = (size_t)r->T * r->T;
    if (lisi_map) std::memcpy(lisi_map, r->lisi.data(), n * sizeof(float));
    if (aug_map) std::memcpy(aug_map, r->aug.data(), n * sizeof(float));
    if (latency_ms) *latency_ms = ms_between(r->t_submit, r->t_done);
    srv->all.erase(it);
    return IQA_OK;
}

iqa_status iqa_server_get_stats(iqa_server *srv, iqa_server_stats *out)
{
    if (!srv || !out) return IQA_ERR_INVALID_ARG;
    std::lock_guard<std::mutex> g(srv->mu);
    std::memset(out, 0, sizeof *out);
    out->submitted = srv->submitted;
    out->completed = srv->completed;
    out->failed = srv->failed;
    out->pending = (long long)srv->pending.size();
    long long inflight = 0;
    for (auto &s : srv->slots)
        if (s.busy) inflight += (long long)s.reqs.size();
    out->inflight = inflight;
    out->steps = srv->steps;
    out->mean_pairs_per_step = srv->steps ? (double)srv->step_pairs / srv->steps : 0.0;
    out->pool_bytes = srv->pool.size();
    out->pool_peak_bytes = srv->pool.peak();
    if (!srv->latencies.empty()) {
        std::vector<double> v = srv->latencies;
        std::sort(v.begin(), v.end());
        auto q = [&](double p) {
            size_t i = (size_t)std::min<double>(v.size() - 1, std::ceil(p * v.size()) - 1);
            return v[i];
        };
        out->p50_ms = q(0.50);
        out->p99_ms = q(0.99);
        out->max_ms = v.back();
        double sum = 0.0;
        for (double x : v) sum += x;
        out->mean_ms = sum / v.size();
        auto median = [](std::vector<double> w) {
            std::sort(w.begin(), w.end());
            return w.empty() ? 0.0 : w[(w.size() - 1) / 2];
        };
        out->p50_queue_ms = median(srv->lat_queue);
        out->p50_launch_ms = median(srv->lat_launch);
        out->p50_device_ms = median(srv->lat_device);
        if (srv->marked_steps) {
            out->mean_step_generator_ms = srv->gen_ms / srv->marked_steps;
            out->mean_step_map_ms = srv->map_ms / srv->marked_steps;
            out->generator_ms_per_pair = srv->gen_ms / srv->marked_pairs;
            out->map_ms_per_pair = srv->map_ms / srv->marked_pairs;
        }
        const double span_s = ms_between(srv->t_first, srv->t_last) / 1e3;
        if (span_s > 0) {
            out->pairs_per_s = srv->completed / span_s;
            out->input_gb_per_s = srv->bytes_done / span_s / 1e9;
        }
    }
    return IQA_OK;
}

void iqa_server_destroy(iqa_server *srv)
{
    if (!srv) return;
    {
        std::lock_guard<std::mutex> g(srv->mu);
        srv->stop = true;  // a stalled simulated step ends when stop is set
    }
    srv->cv_work.notify_all();
    if (srv->worker.joinable()) srv->worker.join();
    if (!srv->cfg.simulate) {
        int prev = 0;
        cudaGetDevice(&prev);
        cudaSetDevice(srv->device);
        for (auto &s : srv->slots) {
            if (s.st) cudaStreamSynchronize(s.st);
            free_slot(s);
        }
        for (auto &kv : srv->refs) {
            cudaFree(kv.second.d_arrays);
            cudaFree(kv.second.d_image);
        }
        cudaFree(srv->d_pool);
        cudaSetDevice(prev);
    }
    delete srv;
}

}  // extern "C"
