// Epoch-boundary kernels: the stopping condition and the result
// (arXiv 1910.11039, Section III-A: f(...) < eps and g(...) < eps for all x,
// checked on a consistent snapshot of (tau, c~), Section III-B).
//
// Compiled with -fmad=false and written with explicit IEEE round-to-nearest
// intrinsics so that every f and g value is the correctly rounded result of
// the same operation sequence a host evaluation uses:
//   f = (L_L/tau) * (1/3 - omega/tau + sqrt((1/3 - omega/tau)^2 + ((2 b~) omega) / L_L))
//   g = (L_U/tau) * (1/3 + omega/tau + sqrt((1/3 + omega/tau)^2 + ((2 b~) omega) / L_U))
// with b~ = c~(x) / tau.  The maxima are exact (comparisons), so the stop
// decision does not depend on the reduction order.
//
// Traffic: one streaming pass of 20 bytes per vertex (u32 counter, two f64
// budgets); the grid is a multiple of the SM count.

#include <cstdint>

#include "kadabra_internal.h"
#include "stop_math.cuh"

namespace kadabra {
namespace {

constexpr int kCheckThreads = 256;

__global__ void __launch_bounds__(kCheckThreads) check_kernel(CheckLaunch a)
{
    __shared__ double sf[kCheckThreads / 32], sg[kCheckThreads / 32];
    Job *job = a.job;
    if (*reinterpret_cast<volatile int *>(&job->stopped)) return;   // stays stopped
    const unsigned long long tau = *reinterpret_cast<volatile unsigned long long *>(&job->tau);

    double mf = 0.0, mg = 0.0;
    if (tau > 0) {
        const StopConsts k = stop_consts(tau, a.omega);
        const long long stride = (long long)gridDim.x * blockDim.x;
        for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < a.n; x += stride) {
            double f, g;
            stop_fg(k, __ldg(a.counts + x), __ldg(a.L + x), f, g);
            mf = fmax_exact(mf, f);
            mg = fmax_exact(mg, g);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mf = fmax_exact(mf, __shfl_xor_sync(0xffffffffu, mf, o));
        mg = fmax_exact(mg, __shfl_xor_sync(0xffffffffu, mg, o));
    }
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) {
        sf[wid] = mf;
        sg[wid] = mg;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 0; i < kCheckThreads / 32; ++i) {
            mf = fmax_exact(mf, sf[i]);
            mg = fmax_exact(mg, sg[i]);
        }
        // f, g >= +0, so their bit patterns order like the values
        atomicMax(&job->maxf_bits, (unsigned long long)__double_as_longlong(mf));
        atomicMax(&job->maxg_bits, (unsigned long long)__double_as_longlong(mg));
        __threadfence();
        const unsigned int prev = atomicAdd(&job->check_done, 1u);
        if (prev == gridDim.x - 1) {
            __threadfence();
            double Mf = __longlong_as_double((long long)*reinterpret_cast<volatile unsigned long long *>(&job->maxf_bits));
            double Mg = __longlong_as_double((long long)*reinterpret_cast<volatile unsigned long long *>(&job->maxg_bits));
            int stop = 0;
            if (tau == 0) {
                Mf = __longlong_as_double(0x7ff0000000000000LL);
                Mg = Mf;
            } else {
                stop = ((double)tau >= a.omega) || (Mf < a.eps && Mg < a.eps);
            }
            job->last_maxf = Mf;
            job->last_maxg = Mg;
            if (stop) {
                unsigned long long now;
                asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
                job->stop_ns = now;
                job->stopped = 1;
                job->stop_epoch = job->epoch;
            }
            job->epoch += 1;
            job->maxf_bits = 0ULL;
            job->maxg_bits = 0ULL;
            job->check_done = 0u;
            __threadfence();
        }
    }
}

__global__ void result_kernel(long long n, const uint32_t *counts, const Job *job, double *btilde)
{
    const double tau_d = (double)job->tau;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride)
        btilde[x] = __ddiv_rn((double)__ldg(counts + x), tau_d);
}

// c~ += delta, tau += samples (one thread block strides, then the tau update)
__global__ void absorb_kernel(long long n, uint32_t *counts, const uint32_t *delta, Job *job,
                              unsigned long long samples)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        const unsigned int d = __ldg(delta + x);
        if (d) {
            const unsigned int old = atomicAdd(counts + x, d);
            if (old + d < old) atomicOr(&job->error, kErrCounterOverflow);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&job->tau, samples);
}

// c~[log[i]] += 1 for i < len, tau += samples: the epoch logs of all shards
// folded into the counters (integer sums, any order)
__global__ void absorb_log_kernel(const uint32_t *log, unsigned long long len, long long n, uint32_t *counts, Job *job,
                                  unsigned long long samples)
{
    const unsigned long long stride = (unsigned long long)gridDim.x * blockDim.x;
    for (unsigned long long i = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; i < len; i += stride) {
        const unsigned int x = __ldg(log + i);
        if ((long long)x >= n) {
            atomicOr(&job->error, kErrSelect);
            continue;
        }
        if (atomicAdd(counts + x, 1u) == 0xffffffffu) atomicOr(&job->error, kErrCounterOverflow);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) atomicAdd(&job->tau, samples);
}

__global__ void clock_kernel(unsigned long long *out)
{
    unsigned long long now;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(now));
    *out = now;
}

__global__ void reset_job_kernel(Job *job, unsigned long long tau)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) {
        Job z;
        unsigned char *p = reinterpret_cast<unsigned char *>(&z);
        for (size_t i = 0; i < sizeof(Job); ++i) p[i] = 0;
        z.stop_epoch = -1;
        z.tau = tau;
        *job = z;
    }
}

int grid_for(long long n, int threads)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (sms <= 0) sms = 1;
    long long want = (n + threads - 1) / threads;
    long long cap = (long long)sms * 8;    // 8 CTAs of 256 threads per SM: full occupancy
    long long g = want < cap ? want : cap;
    return (int)(g > 0 ? g : 1);
}

}  // namespace

cudaError_t launch_check(const CheckLaunch &a, cudaStream_t st)
{
    CheckLaunch b = a;
    if (b.grid <= 0) b.grid = grid_for(a.n, kCheckThreads);
    check_kernel<<<b.grid, kCheckThreads, 0, st>>>(b);
    return cudaGetLastError();
}

cudaError_t launch_result(int64_t n, const uint32_t *counts, const Job *job, double *btilde, cudaStream_t st)
{
    result_kernel<<<grid_for(n, 256), 256, 0, st>>>((long long)n, counts, job, btilde);
    return cudaGetLastError();
}

cudaError_t launch_absorb(int64_t n, uint32_t *counts, const uint32_t *delta, Job *job, uint64_t samples,
                          cudaStream_t st)
{
    absorb_kernel<<<grid_for(n, 256), 256, 0, st>>>((long long)n, counts, delta, job, (unsigned long long)samples);
    return cudaGetLastError();
}

cudaError_t launch_absorb_log(const uint32_t *log, uint64_t len, int64_t n, uint32_t *counts, Job *job, uint64_t samples,
                              cudaStream_t st)
{
    const int grid = len ? grid_for((long long)len, 256) : 1;
    absorb_log_kernel<<<grid, 256, 0, st>>>(log, (unsigned long long)len, (long long)n, counts, job,
                                            (unsigned long long)samples);
    return cudaGetLastError();
}

cudaError_t read_device_clock(unsigned long long *ns, cudaStream_t st)
{
    unsigned long long *d = nullptr;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&d), sizeof(unsigned long long));
    if (e != cudaSuccess) return e;
    clock_kernel<<<1, 1, 0, st>>>(d);
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(ns, d, sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d);
    return e;
}

// ---- budgets from calibration counts (Section III-A, phase 2) -----------
//
// The budget rule depends on a vertex only through its calibration count, so
// the host needs just the number of vertices with each count; every vertex
// then takes the (L_L, L_U) pair of its count's class.

__global__ void cal_max_kernel(long long n, const uint32_t *cal, unsigned int *mx)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    unsigned int m = 0;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const unsigned int c = cal[v];
        m = c > m ? c : m;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned int y = __shfl_xor_sync(0xffffffffu, m, o);
        m = y > m ? y : m;
    }
    if ((threadIdx.x & 31) == 0 && m) atomicMax(mx, m);
}

constexpr int kHistSmem = 4096;

__global__ void cal_hist_kernel(long long n, const uint32_t *cal, unsigned int cmax, unsigned long long *hist)
{
    __shared__ unsigned int h[kHistSmem];
    const unsigned int nb = cmax + 1u < (unsigned int)kHistSmem ? cmax + 1u : (unsigned int)kHistSmem;
    for (unsigned int i = threadIdx.x; i < nb; i += blockDim.x) h[i] = 0;
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_round = (n + 31) & ~31LL;   // whole warps stay in the loop
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n_round; v += stride) {
        const bool in = v < n;
        const unsigned int c = in ? cal[v] : 0xffffffffu;
        const unsigned int peers = __match_any_sync(0xffffffffu, c);
        if (in && (threadIdx.x & 31) == __ffs(peers) - 1) {
            if (c < nb) atomicAdd(&h[c], (unsigned int)__popc(peers));
            else atomicAdd(&hist[c], (unsigned long long)__popc(peers));
        }
    }
    __syncthreads();
    for (unsigned int i = threadIdx.x; i < nb; i += blockDim.x)
        if (h[i]) atomicAdd(&hist[i], (unsigned long long)h[i]);
}

__global__ void fill_budgets_kernel(long long n, const uint32_t *cal, const int *class_of, const double2 *Ltab,
                                    uint32_t *cls, double2 *L)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int k = class_of[cal[v]];
        cls[v] = (uint32_t)k;
        L[v] = Ltab[k];
    }
}

cudaError_t launch_cal_max(int64_t n, const uint32_t *cal, unsigned int *mx, cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(mx, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
    cal_max_kernel<<<grid_for(n, 256), 256, 0, st>>>((long long)n, cal, mx);
    return cudaGetLastError();
}

cudaError_t launch_cal_hist(int64_t n, const uint32_t *cal, unsigned int cmax, unsigned long long *hist,
                            cudaStream_t st)
{
    cudaError_t e = cudaMemsetAsync(hist, 0, ((size_t)cmax + 1) * sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    cal_hist_kernel<<<grid_for(n, 256), 256, 0, st>>>((long long)n, cal, cmax, hist);
    return cudaGetLastError();
}

cudaError_t launch_fill_budgets(int64_t n, const uint32_t *cal, const int *class_of, const double2 *Ltab,
                                uint32_t *cls, double2 *L, cudaStream_t st)
{
    fill_budgets_kernel<<<grid_for(n, 256), 256, 0, st>>>((long long)n, cal, class_of, Ltab, cls, L);
    return cudaGetLastError();
}

// State of every query of a batch step: 0 running, 1 calibration samples
// complete, 2 stopped (or at its sample cap).
__global__ void batch_poll_kernel(const QueryDesc *d, int nq, int *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nq) return;
    const QueryDesc &q = d[i];
    const volatile PipeState *ps = q.ps;
    const volatile Job *job = q.job;
    int r = 0;
    if (q.tag == 0) r = ps->done[0] >= (unsigned int)q.E ? 1 : 0;
    else r = job->stopped ? 2 : 0;
    out[i] = r;
}

cudaError_t launch_batch_poll(const QueryDesc *d, int nq, int *out, cudaStream_t st)
{
    if (nq <= 0) return cudaSuccess;
    batch_poll_kernel<<<(nq + 255) / 256, 256, 0, st>>>(d, nq, out);
    return cudaGetLastError();
}

cudaError_t launch_reset_job(Job *job, cudaStream_t st, unsigned long long tau)
{
    reset_job_kernel<<<1, 32, 0, st>>>(job, tau);
    return cudaGetLastError();
}

}  // namespace kadabra
