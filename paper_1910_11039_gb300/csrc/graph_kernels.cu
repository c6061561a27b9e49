// Graph-wide kernels of the diameter phase (arXiv 1910.11039, Section III-A:
// the diameter is the main ingredient of omega).
//
// The vertex-diameter bound used for omega is, per connected component,
// 2 * ecc(smallest vertex id) + 1, maximised over components.  On the device:
//   1. components by union-find: an edge links the larger of its two roots
//      under the smaller (CAS), so each component's root is its smallest id.
//      Edges are taken in the order of subgraph sampling (Sutton, Ben-Nun and
//      Barak, IPDPS 2018): every vertex first links along its first two
//      adjacency entries; the root that most sampled vertices then share is
//      that of the largest component, whose vertices skip their remaining
//      edges (each such edge is also an edge of its other endpoint, which
//      either lies in the same component or links along it itself);
//   2. one breadth-first search from all roots at once: a vertex's level is its
//      distance from its own component's root, so the largest level is the
//      largest eccentricity and the bound is 2 * (largest level) + 1.
// The search runs in one cooperative launch (all CTAs resident) with a grid
// barrier between levels; every wait in it is bounded and reports an error
// flag instead of hanging.

#include <algorithm>
#include <cstdint>

#include <cuda_runtime.h>

#include "kadabra_internal.h"

namespace kadabra {
namespace {

constexpr unsigned int kUnvisited = 0xffffffffu;
constexpr unsigned long long kSpinLimit = 1ULL << 26;

__device__ __forceinline__ unsigned int find_root(unsigned int *parent, unsigned int x)
{
    // path halving; parents only ever decrease, so racing writes are benign
    unsigned int p = __ldcg(parent + x);
    while (p != x) {
        const unsigned int gp = __ldcg(parent + p);
        if (gp != p) __stcg(parent + x, gp);
        x = p;
        p = gp;
    }
    return x;
}

// Link the trees of u and v: the larger root goes under the smaller one.  The
// link is an atomic minimum, so it always makes progress under contention
// (many vertices linking to one hub): if the larger root had meanwhile been
// linked to some other vertex, the minimum keeps the smaller of the two
// parents and the loop links the displaced one as well.  Parents only ever
// decrease, so every root stays the smallest id of its tree.
__device__ __forceinline__ void hook(unsigned int *parent, unsigned int u, unsigned int v, unsigned int *err)
{
    unsigned long long tries = 0;
    unsigned int ru = find_root(parent, u), rv = find_root(parent, v);
    while (ru != rv) {
        const unsigned int big = ru > rv ? ru : rv, small = ru > rv ? rv : ru;
        const unsigned int old = atomicMin(parent + big, small);
        if (old == big) return;
        if (++tries > kSpinLimit) {
            atomicOr(err, 1u);
            return;
        }
        ru = find_root(parent, old);
        rv = find_root(parent, small);
    }
}

// Round r of the sampling phase: every vertex links along adjacency entry r.
template <typename OffT>
__global__ void cc_link_round_kernel(long long n, const OffT *off, const uint2 *adj, unsigned int *parent, int r,
                                     unsigned int *err)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long u = (long long)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        const long long b = (long long)__ldg(off + u), e = (long long)__ldg(off + u + 1);
        if (b + r < e) hook(parent, (unsigned int)u, __ldg(&adj[b + r].x), err);
    }
}

__global__ void cc_compress_kernel(long long n, unsigned int *parent)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        __stcg(parent + v, find_root(parent, (unsigned int)v));
}

// Roots of m spread-out vertices (a fixed multiplicative stride through the ids).
__global__ void cc_sample_kernel(long long n, unsigned int *parent, unsigned int *out, int m)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m) return;
    const unsigned long long v = ((unsigned long long)i * 2654435761ULL + 40503ULL) % (unsigned long long)n;
    out[i] = find_root(parent, (unsigned int)v);
}

// The remaining adjacency entries (from entry r0 on) of every vertex outside
// the tree rooted at `skip`; one warp per vertex, lanes stride its entries.
template <typename OffT>
__global__ void cc_rest_kernel(long long n, const OffT *off, const uint2 *adj, unsigned int *parent, unsigned int skip,
                               int r0, unsigned int *err)
{
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long u = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); u < n; u += warps) {
        const long long b = (long long)__ldg(off + u), e = (long long)__ldg(off + u + 1);
        if (b + r0 >= e) continue;
        unsigned int ru = 0;
        if (lane == 0) ru = find_root(parent, (unsigned int)u);
        ru = __shfl_sync(0xffffffffu, ru, 0);
        if (ru == skip) continue;
        for (long long i = b + r0 + lane; i < e; i += 32) hook(parent, (unsigned int)u, __ldg(&adj[i].x), err);
    }
}

__global__ void cc_init_kernel(long long n, unsigned int *parent, unsigned int *dist, unsigned int *queue,
                               unsigned int *qlen)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        parent[v] = (unsigned int)v;
        dist[v] = kUnvisited;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) *qlen = 0;
    (void)queue;
}

// Warp-aggregated append of the lanes' `take` vertices to queue q (length
// *len), adding their degrees to *fdeg.
__device__ __forceinline__ void warp_append(bool take, unsigned int v, unsigned long long deg, unsigned int *q,
                                            unsigned int *len, unsigned long long *fdeg)
{
    const unsigned int lane = threadIdx.x & 31;
    const unsigned int active = __activemask();
    const unsigned int m = __ballot_sync(active, take);
    if (!m) return;
    unsigned long long dsum = take ? deg : 0ULL;
    for (int o = 16; o > 0; o >>= 1) dsum += __shfl_xor_sync(active, dsum, o);
    const int leader = __ffs(m) - 1;
    unsigned int base = 0;
    if ((int)lane == leader) {
        base = atomicAdd(len, (unsigned int)__popc(m));
        atomicAdd(fdeg, dsum);
    }
    base = __shfl_sync(active, base, leader);
    if (take) __stcg(q + base + __popc(m & ((1u << lane) - 1u)), v);
}

// roots (parent[v] == v after hooking) start the search at level 0
template <typename OffT>
__global__ void roots_kernel(long long n, const OffT *off, unsigned int *parent, unsigned int *dist,
                             unsigned int *queue, unsigned int *qlen, unsigned long long *fdeg)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_round = (n + 31) & ~31LL;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n_round; v += stride) {
        bool take = false;
        unsigned long long d = 0;
        if (v < n && find_root(parent, (unsigned int)v) == (unsigned int)v) {
            dist[v] = 0;
            take = true;
            d = (unsigned long long)((long long)off[v + 1] - (long long)off[v]);
        }
        warp_append(take, (unsigned int)v, d, queue, qlen, fdeg);
    }
}

struct BfsState {
    unsigned int len[2];       // frontier sizes of the two queues
    unsigned int arrive;       // grid barrier arrivals
    unsigned int gen;          // grid barrier generation
    unsigned int level;        // largest level reached
    unsigned int err;
    unsigned long long fdeg[2];  // degree sums of the two queues' vertices
    unsigned long long explored; // degree sum of every vertex reached so far
    int bottom_up;             // direction of the current level
};

__device__ bool grid_barrier(BfsState *s)
{
    __syncthreads();
    __shared__ int ok;
    if (threadIdx.x == 0) {
        ok = 1;
        volatile unsigned int *gen = &s->gen;
        const unsigned int g = *gen;
        __threadfence();
        if (atomicAdd(&s->arrive, 1u) == gridDim.x - 1) {
            s->arrive = 0;
            __threadfence();
            atomicAdd(&s->gen, 1u);
        } else {
            unsigned long long spins = 0;
            while (*gen == g) {
                if (++spins > kSpinLimit) {
                    atomicOr(&s->err, 2u);
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
    }
    __syncthreads();
    return ok != 0;
}

// Multi-source breadth-first search, direction-optimising (Beamer, Asanovic
// and Patterson, SC 2012): a level expands its frontier top-down (one warp per
// frontier vertex) while the frontier's edges are few against the edges not
// yet explored, and bottom-up (every unreached vertex looks for a neighbour in
// the frontier) while the frontier is large.  Both give every vertex its exact
// distance from its component's root.
template <typename OffT>
__global__ void msbfs_kernel(long long n, const OffT *off, const uint2 *adj, unsigned int *dist, unsigned int *q0,
                             unsigned int *q1, BfsState *s, unsigned long long nnz)
{
    unsigned int *q[2] = {q0, q1};
    int cur = 0;
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long threads = (long long)gridDim.x * blockDim.x;
    int bottom_up = 0;
    for (unsigned int level = 0;; ++level) {
        const unsigned int len = *reinterpret_cast<volatile unsigned int *>(&s->len[cur]);
        if (len == 0) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) s->level = level;
        // direction of this level, decided alike by every CTA from the same state
        const unsigned long long mf = *reinterpret_cast<volatile unsigned long long *>(&s->fdeg[cur]);
        const unsigned long long ex = *reinterpret_cast<volatile unsigned long long *>(&s->explored);
        const unsigned long long mu = nnz > ex ? nnz - ex : 0ULL;
        if (!bottom_up && mf * 14ULL > mu) bottom_up = 1;
        else if (bottom_up && (unsigned long long)len * 24ULL < (unsigned long long)n) bottom_up = 0;
        unsigned int *nextq = q[cur ^ 1];
        unsigned int *nlen = &s->len[cur ^ 1];
        unsigned long long *nfdeg = &s->fdeg[cur ^ 1];
        if (!bottom_up) {
            // one warp per frontier vertex: lanes stride its adjacency
            for (long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < len; i += warps) {
                const unsigned int u = __ldcg(q[cur] + i);
                const long long b = (long long)__ldg(off + u), e = (long long)__ldg(off + u + 1);
                for (long long k0 = b; k0 < e; k0 += 32) {
                    const long long k = k0 + lane;
                    bool take = false;
                    unsigned int w = 0;
                    unsigned long long dw = 0;
                    if (k < e) {
                        const uint2 c = __ldg(&adj[k]);
                        w = c.x;
                        dw = c.y;
                        take = __ldcg(dist + w) == kUnvisited && atomicCAS(dist + w, kUnvisited, level + 1) == kUnvisited;
                    }
                    warp_append(take, w, dw, nextq, nlen, nfdeg);
                }
            }
        } else {
            // every unreached vertex looks for a neighbour at this level
            const long long n_round = (n + 31) & ~31LL;
            for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n_round; v += threads) {
                bool take = false;
                unsigned long long dv = 0;
                if (v < n && __ldcg(dist + v) == kUnvisited) {
                    const long long b = (long long)__ldg(off + v), e = (long long)__ldg(off + v + 1);
                    dv = (unsigned long long)(e - b);
                    for (long long k = b; k < e; ++k) {
                        if (__ldcg(dist + __ldg(&adj[k].x)) == level) {
                            take = true;
                            break;
                        }
                    }
                    if (take) __stcg(dist + v, level + 1);
                }
                warp_append(take, (unsigned int)v, dv, nextq, nlen, nfdeg);
            }
        }
        if (!grid_barrier(s)) return;
        // every CTA has read len[cur] and fdeg[cur]; one clears them for reuse
        // two levels on and books the next frontier's edges as explored
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            s->len[cur] = 0;
            s->fdeg[cur] = 0;
            s->explored += s->fdeg[cur ^ 1];
        }
        if (!grid_barrier(s)) return;
        cur ^= 1;
    }
}

__global__ void max_degree_kernel_i32(long long n, const int *off, unsigned long long *out)
{
    unsigned long long m = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const unsigned long long d = (unsigned long long)((long long)off[v + 1] - (long long)off[v]);
        m = d > m ? d : m;
    }
    atomicMax(out, m);
}

__global__ void max_degree_kernel_i64(long long n, const long long *off, unsigned long long *out)
{
    unsigned long long m = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const unsigned long long d = (unsigned long long)(off[v + 1] - off[v]);
        m = d > m ? d : m;
    }
    atomicMax(out, m);
}

int sm_count()
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms > 0 ? sms : 1;
}

template <typename OffT>
cudaError_t vd_bound_t(int64_t n, const OffT *off, const uint2 *adj, unsigned int *scratch, cudaStream_t st,
                       int64_t *vd)
{
    // scratch: parent[n], dist[n], q0[n], q1[n] (4n u32) followed by BfsState
    unsigned int *parent = scratch;
    unsigned int *dist = scratch + n;
    unsigned int *q0 = scratch + 2 * n;
    unsigned int *q1 = scratch + 3 * n;
    BfsState *s = reinterpret_cast<BfsState *>(scratch + 4 * n);
    const int sms = sm_count();
    const int grid = (int)((n + 255) / 256 < (int64_t)sms * 8 ? (n + 255) / 256 : (int64_t)sms * 8);
    cudaError_t e = cudaMemsetAsync(s, 0, sizeof(BfsState), st);
    if (e != cudaSuccess) return e;
    cc_init_kernel<<<grid, 256, 0, st>>>((long long)n, parent, dist, q0, &s->len[0]);
    constexpr int kRounds = 2, kSamples = 1024;
    for (int r = 0; r < kRounds; ++r) {
        cc_link_round_kernel<OffT><<<grid, 256, 0, st>>>((long long)n, off, adj, parent, r, &s->err);
        cc_compress_kernel<<<grid, 256, 0, st>>>((long long)n, parent);
    }
    // the most frequent root among the sampled vertices (q1, n entries, holds the samples)
    const int m = n < kSamples ? (int)n : kSamples;
    cc_sample_kernel<<<(m + 255) / 256, 256, 0, st>>>((long long)n, parent, q1, m);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    unsigned int roots[kSamples];
    e = cudaMemcpyAsync(roots, q1, (size_t)m * sizeof(unsigned int), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    std::sort(roots, roots + m);
    unsigned int best = roots[0];
    int best_run = 0;
    for (int i = 0; i < m;) {
        int j = i;
        while (j < m && roots[j] == roots[i]) ++j;
        if (j - i > best_run) {
            best_run = j - i;
            best = roots[i];
        }
        i = j;
    }
    cc_rest_kernel<OffT><<<grid, 256, 0, st>>>((long long)n, off, adj, parent, best, kRounds, &s->err);
    roots_kernel<OffT><<<grid, 256, 0, st>>>((long long)n, off, parent, dist, q0, &s->len[0], &s->fdeg[0]);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // cooperative launch: every CTA is resident, so the grid barrier is safe
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, msbfs_kernel<OffT>, 256, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    const int bgrid = sms * (per_sm < 4 ? per_sm : 4);
    long long nn = (long long)n;
    unsigned long long nnz = 0;
    {
        OffT last = 0;
        e = cudaMemcpyAsync(&last, off + n, sizeof(OffT), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) return e;
        nnz = (unsigned long long)last;
    }
    void *args[] = {&nn, (void *)&off, (void *)&adj, &dist, &q0, &q1, &s, &nnz};
    e = cudaLaunchCooperativeKernel((const void *)msbfs_kernel<OffT>, dim3(bgrid), dim3(256), args, 0, st);
    if (e != cudaSuccess) return e;
    BfsState hs;
    e = cudaMemcpyAsync(&hs, s, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if (hs.err) return cudaErrorLaunchTimeout;
    *vd = 2 * (int64_t)hs.level + 1;
    return cudaSuccess;
}

}  // namespace

size_t vd_bound_scratch_bytes(int64_t n) { return (size_t)n * 16 + 64; }

cudaError_t launch_vd_bound(int64_t n, const void *off, int off64, const uint2 *adj, void *scratch, cudaStream_t st,
                            int64_t *vd)
{
    if (n < 1) return cudaErrorInvalidValue;
    if (off64)
        return vd_bound_t<long long>(n, static_cast<const long long *>(off), adj, static_cast<unsigned int *>(scratch),
                                     st, vd);
    return vd_bound_t<int>(n, static_cast<const int *>(off), adj, static_cast<unsigned int *>(scratch), st, vd);
}

cudaError_t launch_max_degree(int64_t n, const void *off, int off64, unsigned long long *out, cudaStream_t st)
{
    const int sms = sm_count();
    const int grid = (int)((n + 255) / 256 < (int64_t)sms * 4 ? (n + 255) / 256 : (int64_t)sms * 4);
    cudaError_t e = cudaMemsetAsync(out, 0, sizeof(unsigned long long), st);
    if (e != cudaSuccess) return e;
    if (off64)
        max_degree_kernel_i64<<<grid > 0 ? grid : 1, 256, 0, st>>>((long long)n, static_cast<const long long *>(off), out);
    else
        max_degree_kernel_i32<<<grid > 0 ? grid : 1, 256, 0, st>>>((long long)n, static_cast<const int *>(off), out);
    return cudaGetLastError();
}

}  // namespace kadabra
