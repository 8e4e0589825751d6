// iqa_noalloc.cu -- iqa_batch_noalloc: the batched persistent launch for
// callers that must not allocate device memory.
//
// The plan path (iqa_plan_create) keeps its work-list descriptors and its work
// counter in device memory it allocates.  This entry point keeps them instead
// in one file-scope __device__ array of fixed size that every GPU loading the
// library holds until the process exits.  The caller still passes the images
// and the output buffers; nothing here calls cudaMalloc, cudaFree or any
// other allocating routine.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>
#include <cstring>
#include <mutex>

#include "iqa.h"
#include "iqa_ctx.h"
#include "iqa_stream.cuh"

namespace iqa {
TileConfig default_batch_config(iqa_dtype dtype);
}

using namespace iqa;

namespace {

constexpr int kMaxDevices = 64;
// Layout of the shared scratch: the descriptor table, then the two work
// counters and the status word.
constexpr size_t kDescBytes = sizeof(PairDesc) * IQA_NOALLOC_MAX_PAIRS;
constexpr size_t kCounterOffset = (kDescBytes + 255) / 256 * 256;
constexpr size_t kScratchBytes = kCounterOffset + 256;

}  // namespace

// The scratch itself.  In host code this name is only a stand-in for the
// device array: its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

// A call's descriptor table, passed by value as the argument of the kernel
// that writes it into the scratch (kernel arguments may take up to 32764
// bytes), so that no host buffer has to outlive the call.
struct NoallocTable {
    PairDesc descs[IQA_NOALLOC_MAX_PAIRS];
    int npairs;
};
static_assert(sizeof(NoallocTable) <= 32764, "descriptor table exceeds a kernel argument");
static_assert(sizeof(PairDesc) % 16 == 0, "descriptors are copied in 16-byte words");

// Writes the call's descriptors into the scratch and clears the work counters
// and the status word.  The map kernel that follows on the stream reads the
// tensor maps through the tensor-map proxy: release these writes to it.
__global__ void __launch_bounds__(256) iqa_noalloc_stage_kernel(const __grid_constant__
                                                                NoallocTable tab)
{
    const uint4 *src = reinterpret_cast<const uint4 *>(tab.descs);
    uint4 *dst = reinterpret_cast<uint4 *>(g_noalloc_scratch);
    const int words = tab.npairs * (int)(sizeof(PairDesc) / 16);
    for (int i = threadIdx.x; i < words; i += blockDim.x) dst[i] = src[i];
    if (threadIdx.x < 16)
        reinterpret_cast<uint4 *>(g_noalloc_scratch + kCounterOffset)[threadIdx.x] =
            make_uint4(0u, 0u, 0u, 0u);
    asm volatile("fence.proxy.tensormap::generic.release.gpu;" ::: "memory");
}

}  // namespace

namespace {

std::mutex g_setup_mu;
void *g_scratch_addr[kMaxDevices] = {};
int g_num_sms[kMaxDevices] = {};

// Per-device set-up, done by the first call on each device (with that device
// current): the array's device address and the SM count.
iqa_status scratch_for_current_device(unsigned char **addr, int *num_sms)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        set_error(nullptr, "device %d beyond the %d this entry point tracks", dev,
                  kMaxDevices);
        return IQA_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> g(g_setup_mu);
    if (!g_scratch_addr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress");
        int sms = 0;
        e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaDeviceGetAttribute");
        g_num_sms[dev] = sms;
        g_scratch_addr[dev] = p;
    }
    *addr = static_cast<unsigned char *>(g_scratch_addr[dev]);
    *num_sms = g_num_sms[dev];
    return IQA_OK;
}

}  // namespace

extern "C" iqa_status iqa_batch_noalloc(const iqa_pair *pairs, int npairs, iqa_dtype dtype,
                                        const iqa_params *params, iqa_stream stream)
{
    if (!pairs || npairs < 1) {
        set_error(nullptr, "need pairs and npairs >= 1");
        return IQA_ERR_INVALID_ARG;
    }
    if (npairs > IQA_NOALLOC_MAX_PAIRS) {
        set_error(nullptr, "iqa_batch_noalloc takes at most %d pairs per call (got %d)",
                  IQA_NOALLOC_MAX_PAIRS, npairs);
        return IQA_ERR_INVALID_ARG;
    }
    if (!dtype_ok(dtype)) {
        set_error(nullptr, "unknown dtype %d", (int)dtype);
        return IQA_ERR_INVALID_ARG;
    }
    iqa_params P;
    iqa_status s = resolve_params(nullptr, params, &P);
    if (s != IQA_OK) return s;
    const int V = 16 / elem_size(dtype);
    for (int i = 0; i < npairs; ++i) {
        const iqa_pair &p = pairs[i];
        if (!p.x || !p.y || (!p.lisi_map && !p.aug_map && !p.sums)) {
            set_error(nullptr, "pair %d: needs x, y and at least one output", i);
            return IQA_ERR_INVALID_ARG;
        }
        s = check_shape(nullptr, p.N, p.NT);
        if (s != IQA_OK) return s;
        if (((uintptr_t)p.x & 15u) || ((uintptr_t)p.y & 15u) || p.NT % V || p.NT > 256) {
            set_error(nullptr, "pair %d: needs 16-byte aligned images and NT a multiple "
                               "of 16 bytes, at most 256", i);
            return IQA_ERR_UNSUPPORTED;
        }
    }
    unsigned char *scratch = nullptr;
    int num_sms = 0;
    s = scratch_for_current_device(&scratch, &num_sms);
    if (s != IQA_OK) return s;

    // Descriptors are built in the staging kernel's argument (on the stack),
    // largest tiles first; that kernel writes them into the device array on
    // the caller's stream.
    NoallocTable tab;
    std::memset(&tab, 0, sizeof tab);
    tab.npairs = npairs;
    PairDesc *host = tab.descs;
    int order[IQA_NOALLOC_MAX_PAIRS];
    for (int i = 0; i < npairs; ++i) order[i] = i;
    std::stable_sort(order, order + npairs,
                     [&](int a, int b) { return pairs[a].NT > pairs[b].NT; });
    TileConfig cfg = default_batch_config(dtype);
    long long units = 0;
    int maps = 0;
    for (int k = 0; k < npairs; ++k) {
        const iqa_pair &p = pairs[order[k]];
        TileConfig c = cfg;
        stream_unit_shape(c, p.N, p.NT, dtype);
        std::string why;
        if (!stream_config_valid(p.N, p.NT, dtype, c, &why)) {
            set_error(nullptr, "pair %d: %s", order[k], why.c_str());
            return IQA_ERR_UNSUPPORTED;
        }
        s = fill_pair_desc(nullptr, &host[k], p.x, p.y, p.N, p.NT, dtype, c, P, p.lisi_map,
                           p.aug_map, p.sums, units);
        if (s != IQA_OK) return s;
        units += pair_units(p.N, p.NT, c);
        if (p.sums) maps = MAPS_AB;
        if (p.lisi_map) maps |= MAPS_A;
        if (p.aug_map) maps |= MAPS_B;
    }
    cudaStream_t st = (cudaStream_t)stream;
    // descriptors in, counters and status word to zero: one kernel whose
    // argument carries the table (launched in full stream order, so a
    // previous call's map kernel on this stream has finished with the array)
    iqa_noalloc_stage_kernel<<<1, 256, 0, st>>>(tab);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "scratch set-up");

    StreamParams sp;
    std::memset(&sp, 0, sizeof sp);
    sp.descs = reinterpret_cast<const PairDesc *>(scratch);
    sp.npairs = npairs;
    sp.stage_bytes = cfg.stage_kb * 1024;
    sp.stages = cfg.stages;
    sp.total_units = units;
    sp.sched = reinterpret_cast<unsigned long long *>(scratch + kCounterOffset);
    sp.status = reinterpret_cast<int *>(scratch + kCounterOffset + 16);
    sp.timeout_ns = 1000000000LL;
    const long long g = (long long)num_sms * cfg.ctas_per_sm;
    const int grid = (int)std::max<long long>(1, std::min<long long>(g, units));
    e = launch_stream(sp, dtype, cfg, maps, grid, st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "no-alloc batch launch");
    return IQA_OK;
}
