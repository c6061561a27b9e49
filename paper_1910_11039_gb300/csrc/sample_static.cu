// Allocation-free sampling: the sampling kernel with its scratch (job state,
// per-slot records and queues) in one file-scope device array instead of
// memory the library allocates.
//
// Who needs this: callers that must not allocate device memory after start-up
// -- services that plan all memory once and forbid allocation on the request
// path, code embedded in a host framework that owns the device allocator, or
// work issued where cudaMalloc is not allowed.  They pass only their own
// inputs (a loaded graph) and outputs (a device counter array).
//
// The array is fixed at kStaticScratchBytes and exists on every device that
// loads this library, for as long as the process runs.  Every call reuses it,
// so calls that overlap on the GPU (different streams, or different host
// threads without ordering) race on it; serialise them.
//
// With lazy module loading (the CUDA default) the array is only reserved
// when this file's device code is first touched on a device.  The library
// touches it in kadabra_graph_load (static_scratch_reserve), so by the time
// a caller holds a graph on a device, sampling from it here loads no code
// and reserves no memory.

#include <cstdint>

#include <cuda_runtime.h>

#include "kadabra.h"
#include "kadabra_internal.h"

namespace kadabra {

constexpr size_t kStaticScratchBytes = size_t(KADABRA_STATIC_SCRATCH_BYTES);
constexpr size_t kStaticJobBytes = 256;   // the Job record, padded to the array's alignment
static_assert(sizeof(Job) <= kStaticJobBytes, "job state must fit its reserved bytes");

static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of the static scratch on the current device.  Looked up on
// every call (cheap once the module is loaded), so a cached address can never
// outlive a device reset.  The host-side symbol g_static_scratch is only a
// stand-in for the device array and is never handed to a kernel.
cudaError_t static_scratch_address(void **out)
{
    void *p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) return e;
    *out = p;
    return cudaSuccess;
}

// Set-up on the current device: loads this file's module, which reserves the
// array.  kadabra_graph_load calls it with the graph's device current.
cudaError_t static_scratch_reserve()
{
    void *p = nullptr;
    return static_scratch_address(&p);
}

}  // namespace kadabra

namespace {

kadabra_status static_fail(kadabra_status st, const char *msg)
{
    return (kadabra_status)kadabra::set_last_error((int)st, msg);
}

kadabra_status static_cuda_fail(cudaError_t e)
{
    return static_fail(e == cudaErrorNoDevice ? KADABRA_ERR_NO_DEVICE : KADABRA_ERR_CUDA, cudaGetErrorString(e));
}

}  // namespace

// Layout of the array for one call, each part starting on a 256-byte
// boundary: [Job | code words: slots * n | qv, ql: slots * n each | qs, qm:
// slots * n each] -- full queue capacity (cap = n), so no sample needs a
// spill slot.
namespace {
size_t up256(size_t b) { return (b + 255) & ~size_t(255); }
size_t static_bytes(size_t slots, size_t n)
{
    return up256(slots * n * 4) + 2 * up256(slots * n * 4) + 2 * up256(slots * n * 8);
}
}  // namespace

extern "C" kadabra_status kadabra_sample_static(const kadabra_graph *g, uint64_t seed, int tag, uint64_t first,
                                                int64_t count, uint32_t *counts, void *cuda_stream)
{
    using namespace kadabra;
    GraphView G;
    if (!graph_view(g, &G)) return static_fail(KADABRA_ERR_INVALID_ARG, "graph is null");
    if (!counts) return static_fail(KADABRA_ERR_INVALID_ARG, "counts is null");
    if (tag != 0 && tag != 1) return static_fail(KADABRA_ERR_INVALID_ARG, "tag must be 0 or 1");
    if (count < 0 || count >= (int64_t(1) << 32)) return static_fail(KADABRA_ERR_INVALID_ARG, "count must be in [0, 2^32)");
    if (G.n < 2) return static_fail(KADABRA_ERR_INVALID_ARG, "sampling pairs needs n >= 2");
    const size_t n = (size_t)G.n;
    if (static_bytes(1, n) > kStaticScratchBytes - kStaticJobBytes)
        return static_fail(KADABRA_ERR_INVALID_ARG,
                           "graph too large for the static scratch: n * 28 bytes (rounded up) must fit in "
                           "KADABRA_STATIC_SCRATCH_BYTES - 256");
    size_t max_slots = 1;
    while (static_bytes(max_slots + 1, n) <= kStaticScratchBytes - kStaticJobBytes) ++max_slots;
    if (count == 0) return KADABRA_OK;
    cudaStream_t st = reinterpret_cast<cudaStream_t>(cuda_stream);
    const int threads = 1024;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = sample_occupancy(threads, G.off64, &per_sm);
    if (e != cudaSuccess) return static_cuda_fail(e);
    size_t slots = (size_t)(sms > 0 ? sms : 1) * (size_t)(per_sm > 0 ? per_sm : 1);
    if (slots > max_slots) slots = max_slots;
    if (slots > (size_t)count) slots = (size_t)count;

    void *base = nullptr;
    e = static_scratch_address(&base);
    if (e != cudaSuccess) return static_cuda_fail(e);
    unsigned char *bytes = static_cast<unsigned char *>(base);
    Job *job = reinterpret_cast<Job *>(bytes);
    SlotSet S;
    size_t off = kStaticJobBytes;
    S.code = reinterpret_cast<uint32_t *>(bytes + off);
    off += up256(slots * n * 4);
    S.qv = reinterpret_cast<uint32_t *>(bytes + off);
    off += up256(slots * n * 4);
    S.ql = reinterpret_cast<uint32_t *>(bytes + off);
    off += up256(slots * n * 4);
    S.qs = reinterpret_cast<unsigned long long *>(bytes + off);
    off += up256(slots * n * 8);
    S.qm = reinterpret_cast<unsigned long long *>(bytes + off);
    S.stride = G.n;
    S.cap = G.n;
    S.count = (int)slots;

    // the sampler requires all-zero code words and counts and a fresh job record
    e = cudaMemsetAsync(S.code, 0, slots * n * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.qs, 0, slots * n * 8, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(S.qm, 0, slots * n * 8, st);
    if (e == cudaSuccess) e = launch_reset_job(job, st, first);
    SampleLaunch a{};
    a.n = G.n;
    a.off = G.off;
    a.off64 = G.off64;
    a.adj = G.adj;
    a.slots = S;
    a.counts = counts;
    a.job = job;
    a.seed = seed;
    a.tag = (uint32_t)tag;
    a.K = kadabra_sigma_bits(G.n, G.max_degree);
    a.epoch_len = count;
    a.grid = (int)slots;
    a.threads = threads;
    a.spin_limit = 1ULL << 24;
    if (e == cudaSuccess) e = launch_sample(a, st);
    unsigned int err = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&err, &job->error, sizeof(err), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return static_cuda_fail(e);
    if (err & kErrSigmaOverflow) return static_fail(KADABRA_ERR_SIGMA_OVERFLOW, "a per-side path count exceeded 2^K");
    if (err & kErrCounterOverflow) return static_fail(KADABRA_ERR_COUNTER_OVERFLOW, "a 32-bit counter wrapped");
    if (err) return static_fail(KADABRA_ERR_CUDA, "internal sampling invariant violated");
    return KADABRA_OK;
}
