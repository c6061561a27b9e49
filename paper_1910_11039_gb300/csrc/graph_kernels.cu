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
//
// The exact vertex diameter (the paper computes the diameter exactly, with
// iFUB: Crescenzi, Grossi, Habib, Lanzi and Marino, TCS 2013) is computed for
// the largest component: a double sweep from its highest-degree vertex (h ->
// a -> b, each a farthest vertex of the previous search) gives lower bounds
// and the midpoint m of the a-b path; from m, the fringe levels F_i (vertices
// at distance i, from the deepest down) have their eccentricities computed,
// 64 vertices per bit-parallel search, until the largest eccentricity found
// exceeds 2(i - 1): every pair of vertices both closer to m than i is within
// 2(i - 1), so that eccentricity is the diameter.  A fringe too wide for 64
// searches of 64 sources (meshes) ends the search with the upper bound
// max(lb, 2 i) proven so far, flagged as not exact.  Then every other component
// whose bound 2 ecc(root) + 1 still exceeds the best value found gets the
// same treatment (largest bound first; up to 64 components, beyond which the
// remaining bound is used and the result is flagged as not exact).

#include <algorithm>
#include <cstdint>
#include <vector>

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
// *len), adding their degrees to *fdeg (if fdeg is not null).
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
        if (fdeg) atomicAdd(fdeg, dsum);
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
            d = (unsigned long long)((long long)off[v + 1] - (long long)off[v]);
            take = d > 0;     // an isolated vertex is its own whole search (eccentricity 0)
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
// and Patterson, SC 2012): a level expands its frontier top-down (32 frontier
// vertices per warp) while the frontier's edges are few against the edges not
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
            // 32 frontier vertices per warp: their adjacency lists form one
            // range (a warp-wide prefix sum of the degrees) that the lanes
            // stride, so no lane idles on a low-degree vertex
            const long long groups = ((long long)len + 31) / 32;
            for (long long gi = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); gi < groups;
                 gi += warps) {
                const long long i = gi * 32 + lane;
                long long b = 0;
                unsigned long long d = 0;
                if (i < (long long)len) {
                    const unsigned int u = __ldcg(q[cur] + i);
                    b = (long long)__ldg(off + u);
                    d = (unsigned long long)((long long)__ldg(off + u + 1) - b);
                }
                unsigned long long incl = d;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= o) incl += t;
                }
                const unsigned long long excl = incl - d;
                const unsigned long long total = __shfl_sync(0xffffffffu, incl, 31);
                for (unsigned long long k0 = 0; k0 < total; k0 += 32) {
                    const unsigned long long k = k0 + lane;
                    // owner of entry k: the last lane whose exclusive prefix is <= k
                    int lo = 0;
#pragma unroll
                    for (int step = 16; step > 0; step >>= 1) {
                        const int cand = lo + step;
                        const unsigned long long ex = __shfl_sync(0xffffffffu, excl, cand < 32 ? cand : 31);
                        if (cand < 32 && ex <= k) lo = cand;
                    }
                    const long long ob = __shfl_sync(0xffffffffu, b, lo);
                    const unsigned long long oe = __shfl_sync(0xffffffffu, excl, lo);
                    bool take = false;
                    unsigned int w = 0;
                    unsigned long long dw = 0;
                    if (k < total) {
                        const uint2 c = __ldg(&adj[ob + (long long)(k - oe)]);
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

// ---- exact vertex diameter (iFUB) -----------------------------------------

__global__ void fill_u32_kernel(long long n, unsigned int *a, unsigned int v)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) a[i] = v;
}

// single source: dist[src] = 0, queue {src}
template <typename OffT>
__global__ void seed_kernel(const OffT *off, unsigned int src, unsigned int *dist, unsigned int *q0, BfsState *s)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        dist[src] = 0;
        q0[0] = src;
        s->len[0] = 1;
        s->fdeg[0] = (unsigned long long)((long long)off[src + 1] - (long long)off[src]);
    }
}

// key = (degree << 32) | (~v): the maximum is the highest-degree vertex of the
// component rooted at `root`, smallest id among equals
template <typename OffT>
__global__ void argmax_degree_kernel(long long n, const OffT *off, unsigned int *parent, unsigned int root,
                                     unsigned long long *out)
{
    unsigned long long best = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        if (find_root(parent, (unsigned int)v) != root) continue;
        const unsigned long long d = (unsigned long long)((long long)off[v + 1] - (long long)off[v]);
        const unsigned long long key = (d << 32) | (unsigned long long)(0xffffffffu - (unsigned int)v);
        best = key > best ? key : best;
    }
    if (best) atomicMax(out, best);
}

// smallest vertex at distance `level` (a farthest vertex of the search)
__global__ void farthest_kernel(long long n, const unsigned int *dist, unsigned int level, unsigned int *out)
{
    unsigned int best = kUnvisited;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (dist[v] == level && (unsigned int)v < best) best = (unsigned int)v;
    if (best != kUnvisited) atomicMin(out, best);
}

// smallest vertex m with dist_a(m) = half and dist_a(m) + dist_b(m) = d(a, b):
// the middle of a shortest a-b path
__global__ void midpoint_kernel(long long n, const unsigned int *da, const unsigned int *db, unsigned int half,
                                unsigned int dab, unsigned int *out)
{
    unsigned int best = kUnvisited;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (da[v] == half && db[v] != kUnvisited && da[v] + db[v] == dab && (unsigned int)v < best)
            best = (unsigned int)v;
    if (best != kUnvisited) atomicMin(out, best);
}

// vertices at distance `level` (a fringe level), appended to out
__global__ void fringe_kernel(long long n, const unsigned int *dist, unsigned int level, unsigned int *out,
                              unsigned int *len)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long n_round = (n + 31) & ~31LL;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n_round; v += stride) {
        const bool take = v < n && dist[v] == level;
        warp_append(take, (unsigned int)v, 0ULL, out, len, nullptr);
    }
}

// largest distance from a component's root over the vertices outside the
// component rooted at `skip`
__global__ void other_max_kernel(long long n, unsigned int *parent, const unsigned int *dist, unsigned int skip,
                                 unsigned int *out)
{
    unsigned int best = 0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (dist[v] != kUnvisited && dist[v] > best && find_root(parent, (unsigned int)v) != skip) best = dist[v];
    if (best) atomicMax(out, best);
}

__global__ void root_of_kernel(unsigned int *parent, unsigned int v, unsigned int *out)
{
    if (blockIdx.x == 0 && threadIdx.x == 0) *out = find_root(parent, v);
}

// root distances of the component rooted at `root` set to 0 (done with it)
__global__ void clear_component_kernel(long long n, unsigned int *parent, unsigned int *dist, unsigned int root)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (dist[v] != kUnvisited && dist[v] != 0u && find_root(parent, (unsigned int)v) == root) dist[v] = 0u;
}

struct EccState {
    unsigned int len[2];       // active vertices of the current / next level
    unsigned int arrive, gen, err;
    unsigned int pad;
    unsigned long long alive;  // sources with a vertex at the level being settled
};

__device__ bool ecc_barrier(EccState *s)
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

// Eccentricities of up to 64 sources at once: bit k of seen/fr/nx[v] says
// that v has been reached / is at the current level / reaches the next level
// from source k.  Level by level (cooperative launch, grid barriers): every
// active vertex pushes its frontier bits to its neighbours (top-down, one
// warp per vertex); the newly reached bits become the next frontier; a
// source's eccentricity is the last level at which its bit is still new.
template <typename OffT>
__global__ void ecc64_kernel(long long n, const OffT *off, const uint2 *adj, unsigned long long *seen,
                             unsigned long long *fr, unsigned long long *nx, unsigned int *q0, unsigned int *q1,
                             EccState *s, unsigned int *ecc)
{
    unsigned int *q[2] = {q0, q1};
    int cur = 0;
    const int lane = threadIdx.x & 31;
    const long long warps = (long long)gridDim.x * (blockDim.x >> 5);
    const long long threads = (long long)gridDim.x * blockDim.x;
    const long long gtid = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (unsigned int level = 0;; ++level) {
        const unsigned int len = *reinterpret_cast<volatile unsigned int *>(&s->len[cur]);
        if (len == 0) break;
        unsigned int *nextq = q[cur ^ 1];
        unsigned int *nlen = &s->len[cur ^ 1];
        for (long long i = (long long)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < len; i += warps) {
            const unsigned int u = __ldcg(q[cur] + i);
            const unsigned long long fu = __ldcg(fr + u);
            const long long b = (long long)__ldg(off + u), e = (long long)__ldg(off + u + 1);
            for (long long k0 = b; k0 < e; k0 += 32) {
                const long long k = k0 + lane;
                bool take = false;
                unsigned int w = 0;
                if (k < e) {
                    w = __ldg(&adj[k].x);
                    const unsigned long long m = fu & ~__ldcg(seen + w);
                    if (m) take = atomicOr(nx + w, m) == 0ULL;
                }
                warp_append(take, w, 0ULL, nextq, nlen, nullptr);
            }
        }
        if (!ecc_barrier(s)) return;
        // the current level's frontier bits are spent
        for (long long i = gtid; i < len; i += threads) __stcg(fr + __ldcg(q[cur] + i), 0ULL);
        if (!ecc_barrier(s)) return;
        // settle the next level: its new bits join seen and form the frontier
        const unsigned int nl = *reinterpret_cast<volatile unsigned int *>(nlen);
        unsigned long long alive = 0;
        for (long long i = gtid; i < nl; i += threads) {
            const unsigned int w = __ldcg(nextq + i);
            const unsigned long long m = __ldcg(nx + w);
            __stcg(seen + w, __ldcg(seen + w) | m);
            __stcg(fr + w, m);
            __stcg(nx + w, 0ULL);
            alive |= m;
        }
        for (int o = 16; o > 0; o >>= 1) alive |= __shfl_xor_sync(0xffffffffu, alive, o);
        if (lane == 0 && alive) atomicOr(&s->alive, alive);
        if (!ecc_barrier(s)) return;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            const unsigned long long a = s->alive;
            for (int k = 0; k < 64; ++k)
                if ((a >> k) & 1ULL) ecc[k] = level + 1;
            s->alive = 0;
            s->len[cur] = 0;
        }
        if (!ecc_barrier(s)) return;
        cur ^= 1;
    }
}

// ecc64 sources: seen = fr = their bit, queue = the sources
__global__ void ecc_seed_kernel(const unsigned int *src, int k, unsigned long long *seen, unsigned long long *fr,
                                unsigned int *q0, EccState *s, unsigned int *ecc)
{
    const int i = threadIdx.x;
    if (blockIdx.x == 0 && i < 64) {
        if (i < k) {
            seen[src[i]] = 1ULL << i;
            fr[src[i]] = 1ULL << i;
            q0[i] = src[i];
        }
        ecc[i] = 0;
        if (i == 0) s->len[0] = (unsigned int)k;
    }
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
                       int64_t *vd, unsigned int *lcc_root = nullptr)
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
    if (lcc_root) *lcc_root = best;
    return cudaSuccess;
}

// One cooperative single-source search from src into dist (kUnvisited
// elsewhere); *ecc = eccentricity of src.
// Byte offsets of vd_exact_t's scratch parts, each on a 256-byte boundary:
// the bound's 4n words and search state, 4 distance arrays, 3 arrays of
// 64-bit masks, a fringe list, and a block of small words.
struct ExactLayout {
    size_t dist, masks, fringe, words, total;
};
inline size_t up256(size_t b) { return (b + 255) & ~size_t(255); }
inline ExactLayout exact_layout(int64_t n)
{
    ExactLayout L;
    const size_t un = (size_t)n;
    L.dist = up256(un * 16 + 256);        // after parent, root distances, two queues, BfsState
    L.masks = up256(L.dist + un * 16);
    L.fringe = up256(L.masks + un * 24);
    L.words = up256(L.fringe + un * 4);
    L.total = L.words + 1024;
    return L;
}
static_assert(sizeof(BfsState) <= 256, "search state fits its slot");

template <typename OffT>
cudaError_t bfs_from(int64_t n, const OffT *off, const uint2 *adj, unsigned long long nnz, unsigned int src,
                     unsigned int *dist, unsigned int *q0, unsigned int *q1, BfsState *s, int grid, int bgrid,
                     cudaStream_t st, unsigned int *ecc)
{
    cudaError_t e = cudaMemsetAsync(s, 0, sizeof(BfsState), st);
    if (e != cudaSuccess) return e;
    fill_u32_kernel<<<grid, 256, 0, st>>>((long long)n, dist, kUnvisited);
    seed_kernel<OffT><<<1, 32, 0, st>>>(off, src, dist, q0, s);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    long long nn = (long long)n;
    void *args[] = {&nn, (void *)&off, (void *)&adj, &dist, &q0, &q1, &s, &nnz};
    e = cudaLaunchCooperativeKernel((const void *)msbfs_kernel<OffT>, dim3(bgrid), dim3(256), args, 0, st);
    if (e != cudaSuccess) return e;
    BfsState hs;
    e = cudaMemcpyAsync(&hs, s, sizeof(hs), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    if (hs.err) return cudaErrorLaunchTimeout;
    *ecc = hs.level;
    return cudaSuccess;
}

template <typename T>
cudaError_t read_back(const T *d, T *h, cudaStream_t st)
{
    cudaError_t e = cudaMemcpyAsync(h, d, sizeof(T), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

// Exact vertex diameter of the largest component by iFUB from the midpoint of
// a double sweep (see the file header); other components contribute their
// bound 2 ecc(root) + 1.  *exact = 1 if no other component's bound exceeds
// the largest component's exact value.  *searches = searches run.
template <typename OffT>
cudaError_t vd_exact_t(int64_t n, const OffT *off, const uint2 *adj, unsigned int *scratch, cudaStream_t st,
                       int64_t *vd, int *exact, int64_t *searches)
{
    // scratch: the bound's 4n words and state (parent, root distances, queues),
    // then 4 distance arrays, 3 arrays of 64-bit masks, a fringe list, and
    // small words
    unsigned int lcc = 0;
    int64_t bound = 0;
    cudaError_t e = vd_bound_t<OffT>(n, off, adj, scratch, st, &bound, &lcc);
    if (e != cudaSuccess) return e;
    unsigned int *parent = scratch;
    unsigned int *droot = scratch + n;
    unsigned int *q0 = scratch + 2 * n;
    unsigned int *q1 = scratch + 3 * n;
    BfsState *s = reinterpret_cast<BfsState *>(scratch + 4 * n);
    // the rest starts on 256-byte boundaries (64-bit arrays and words need
    // 8-byte alignment whatever n is)
    const ExactLayout L = exact_layout(n);
    unsigned char *bytes = reinterpret_cast<unsigned char *>(scratch);
    unsigned int *dh = reinterpret_cast<unsigned int *>(bytes + L.dist);
    unsigned int *da = dh + n, *db = dh + 2 * n, *dm = dh + 3 * n;
    unsigned long long *seen = reinterpret_cast<unsigned long long *>(bytes + L.masks);
    unsigned long long *fr = seen + n, *nx = seen + 2 * n;
    unsigned int *fringe = reinterpret_cast<unsigned int *>(bytes + L.fringe);
    unsigned long long *w64 = reinterpret_cast<unsigned long long *>(bytes + L.words);
    unsigned int *w32 = reinterpret_cast<unsigned int *>(bytes + L.words + 8);    // 2 words
    unsigned int *ecc = reinterpret_cast<unsigned int *>(bytes + L.words + 256);  // 64 words
    EccState *es = reinterpret_cast<EccState *>(bytes + L.words + 512);
    if ((reinterpret_cast<uintptr_t>(seen) | reinterpret_cast<uintptr_t>(w64) | reinterpret_cast<uintptr_t>(es) |
         reinterpret_cast<uintptr_t>(s)) & 7u)
        return cudaErrorMisalignedAddress;
    const int sms = sm_count();
    const int grid = (int)((n + 255) / 256 < (int64_t)sms * 8 ? (n + 255) / 256 : (int64_t)sms * 8);
    int per_sm = 0, per_sm2 = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, msbfs_kernel<OffT>, 256, 0);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm2, ecc64_kernel<OffT>, 256, 0);
    if (e != cudaSuccess) return e;
    const int bgrid = sms * (per_sm < 1 ? 1 : (per_sm < 4 ? per_sm : 4));
    const int egrid = sms * (per_sm2 < 1 ? 1 : (per_sm2 < 4 ? per_sm2 : 4));
    unsigned long long nnz = 0;
    {
        OffT last = 0;
        if ((e = read_back(off + n, &last, st)) != cudaSuccess) return e;
        nnz = (unsigned long long)last;
    }
    int64_t nsearch = 0;
    auto far = [&](const unsigned int *d, unsigned int lev, unsigned int *out) -> cudaError_t {
        cudaError_t ee = cudaMemsetAsync(w32, 0xff, 4, st);
        if (ee != cudaSuccess) return ee;
        farthest_kernel<<<grid, 256, 0, st>>>((long long)n, d, lev, w32);
        return read_back(w32, out, st);
    };
    // iFUB on the component rooted at r: its diameter (edges), or, once the
    // fringe eccentricities would take more than kMaxSweeps searches of 64
    // sources (meshes: wide fringes), the upper bound max(lb, 2 i) proven so
    // far (*is_exact = 0)
    constexpr int kMaxSweeps = 64;
    auto ifub = [&](unsigned int r, unsigned int *diam, int *is_exact) -> cudaError_t {
        *is_exact = 1;
        int sweeps = 0;
        cudaError_t ee = cudaMemsetAsync(w64, 0, 8, st);
        if (ee != cudaSuccess) return ee;
        argmax_degree_kernel<OffT><<<grid, 256, 0, st>>>((long long)n, off, parent, r, w64);
        unsigned long long key = 0;
        if ((ee = read_back(w64, &key, st)) != cudaSuccess) return ee;
        const unsigned int h = key ? 0xffffffffu - (unsigned int)(key & 0xffffffffULL) : r;
        // double sweep h -> a -> b, and the middle m of the a-b path
        unsigned int ecc_h = 0, ecc_a = 0, ecc_b = 0, ecc_m = 0, a = 0, b = 0, m = 0;
        if ((ee = bfs_from<OffT>(n, off, adj, nnz, h, dh, q0, q1, s, grid, bgrid, st, &ecc_h)) != cudaSuccess) return ee;
        if ((ee = far(dh, ecc_h, &a)) != cudaSuccess) return ee;
        if ((ee = bfs_from<OffT>(n, off, adj, nnz, a, da, q0, q1, s, grid, bgrid, st, &ecc_a)) != cudaSuccess) return ee;
        if ((ee = far(da, ecc_a, &b)) != cudaSuccess) return ee;
        if ((ee = bfs_from<OffT>(n, off, adj, nnz, b, db, q0, q1, s, grid, bgrid, st, &ecc_b)) != cudaSuccess) return ee;
        if ((ee = cudaMemsetAsync(w32, 0xff, 4, st)) != cudaSuccess) return ee;
        midpoint_kernel<<<grid, 256, 0, st>>>((long long)n, da, db, ecc_a / 2, ecc_a, w32);
        if ((ee = read_back(w32, &m, st)) != cudaSuccess) return ee;
        if (m == kUnvisited) m = h;
        if ((ee = bfs_from<OffT>(n, off, adj, nnz, m, dm, q0, q1, s, grid, bgrid, st, &ecc_m)) != cudaSuccess) return ee;
        nsearch += 4;
        unsigned int lb = ecc_h;
        lb = ecc_a > lb ? ecc_a : lb;
        lb = ecc_b > lb ? ecc_b : lb;
        lb = ecc_m > lb ? ecc_m : lb;
        // fringe levels of m, deepest first, until lb > 2 (i - 1); consecutive
        // levels are gathered into one batch of sources until it holds 64
        unsigned int i = ecc_m;
        while (i >= 1 && 2ULL * i > (unsigned long long)lb) {
            unsigned int lo = i, cnt = 0;
            if ((ee = cudaMemsetAsync(w32 + 1, 0, 4, st)) != cudaSuccess) return ee;
            for (;;) {
                fringe_kernel<<<grid, 256, 0, st>>>((long long)n, dm, lo, fringe, w32 + 1);
                if ((ee = read_back(w32 + 1, &cnt, st)) != cudaSuccess) return ee;
                if (cnt >= 64u || lo == 1 || 2ULL * (lo - 1) < (unsigned long long)lb) break;
                --lo;
            }
            if (sweeps + (int)((cnt + 63u) / 64u) > kMaxSweeps) {
                // levels above i are done: D <= max(lb, 2 i)
                *diam = 2 * i > lb ? 2 * i : lb;
                *is_exact = 0;
                return cudaSuccess;
            }
            sweeps += (int)((cnt + 63u) / 64u);
            unsigned int bi = 0;
            for (unsigned int c0 = 0; c0 < cnt; c0 += 64) {
                const int k = (int)(cnt - c0 < 64u ? cnt - c0 : 64u);
                ee = cudaMemsetAsync(seen, 0, (size_t)n * 24, st);
                if (ee == cudaSuccess) ee = cudaMemsetAsync(es, 0, sizeof(EccState), st);
                if (ee != cudaSuccess) return ee;
                ecc_seed_kernel<<<1, 64, 0, st>>>(fringe + c0, k, seen, fr, q0, es, ecc);
                if ((ee = cudaGetLastError()) != cudaSuccess) return ee;
                long long nn = (long long)n;
                void *args[] = {&nn, (void *)&off, (void *)&adj, &seen, &fr, &nx, &q0, &q1, &es, &ecc};
                ee = cudaLaunchCooperativeKernel((const void *)ecc64_kernel<OffT>, dim3(egrid), dim3(256), args, 0, st);
                if (ee != cudaSuccess) return ee;
                unsigned int he[64];
                EccState hs;
                ee = cudaMemcpyAsync(he, ecc, sizeof(he), cudaMemcpyDeviceToHost, st);
                if (ee == cudaSuccess) ee = cudaMemcpyAsync(&hs, es, sizeof(hs), cudaMemcpyDeviceToHost, st);
                if (ee == cudaSuccess) ee = cudaStreamSynchronize(st);
                if (ee != cudaSuccess) return ee;
                if (hs.err) return cudaErrorLaunchTimeout;
                for (int j = 0; j < k; ++j) bi = he[j] > bi ? he[j] : bi;
                ++nsearch;
            }
            lb = bi > lb ? bi : lb;
            // levels lo..i are done: every pair closer to m than lo is within 2 (lo - 1)
            if (lo == 1 || (unsigned long long)lb > 2ULL * (lo - 1)) break;
            i = lo - 1;
        }
        *diam = lb;
        return cudaSuccess;
    };
    // the largest component first, then every component whose bound
    // 2 ecc(root) + 1 still exceeds the best vertex diameter found (largest
    // bound first), at most kMaxExactComponents of them
    constexpr int kMaxExactComponents = 64;
    unsigned int d0 = 0;
    int ex = 1, ex1 = 1;
    if ((e = ifub(lcc, &d0, &ex1)) != cudaSuccess) return e;
    ex &= ex1;
    int64_t best = (int64_t)d0 + 1;
    clear_component_kernel<<<grid, 256, 0, st>>>((long long)n, parent, droot, lcc);
    int done = 1;
    for (;;) {
        unsigned int other = 0;
        if ((e = cudaMemsetAsync(w32, 0, 4, st)) != cudaSuccess) return e;
        other_max_kernel<<<grid, 256, 0, st>>>((long long)n, parent, droot, kUnvisited, w32);
        if ((e = read_back(w32, &other, st)) != cudaSuccess) return e;
        const int64_t bound_other = 2 * (int64_t)other + 1;
        if (other == 0 || bound_other <= best) break;
        if (done >= kMaxExactComponents) {
            best = bound_other;
            ex = 0;
            break;
        }
        unsigned int v = 0, r = 0;
        if ((e = far(droot, other, &v)) != cudaSuccess) return e;
        root_of_kernel<<<1, 32, 0, st>>>(parent, v, w32 + 1);
        if ((e = read_back(w32 + 1, &r, st)) != cudaSuccess) return e;
        unsigned int dc = 0;
        if ((e = ifub(r, &dc, &ex1)) != cudaSuccess) return e;
        ex &= ex1;
        best = (int64_t)dc + 1 > best ? (int64_t)dc + 1 : best;
        clear_component_kernel<<<grid, 256, 0, st>>>((long long)n, parent, droot, r);
        ++done;
    }
    *vd = best;
    *exact = ex;
    *searches = nsearch;
    return cudaSuccess;
}

}  // namespace

size_t vd_bound_scratch_bytes(int64_t n) { return (size_t)n * 16 + 64; }

size_t vd_exact_scratch_bytes(int64_t n) { return exact_layout(n).total; }

cudaError_t launch_vd_exact(int64_t n, const void *off, int off64, const uint2 *adj, void *scratch, cudaStream_t st,
                            int64_t *vd, int *exact, int64_t *searches)
{
    if (n < 1) return cudaErrorInvalidValue;
    if (off64)
        return vd_exact_t<long long>(n, static_cast<const long long *>(off), adj, static_cast<unsigned int *>(scratch),
                                     st, vd, exact, searches);
    return vd_exact_t<int>(n, static_cast<const int *>(off), adj, static_cast<unsigned int *>(scratch), st, vd, exact,
                           searches);
}

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
