// KADABRA sampling kernel for sm_103a (arXiv 1910.11039, Section III-A).
//
// One CTA owns one "slot" (the scratch of one in-flight sample) and takes
// sample indices from a per-launch work counter until the epoch's range is
// exhausted; a launch is one epoch of the adaptive phase (or the calibration
// phase).  Per sample:
//   A1  pair s != t from Philox draw 0;
//   A2  balanced bidirectional BFS: the side whose frontier has the smaller
//       degree sum (ties: s) expands one whole layer; path counts sigma are
//       accumulated with 64-bit atomics (integer sums, so order-free); the
//       search ends when the new layer touches the other ball (meeting set M)
//       or dies out (disconnected pair);
//   A3  meeting vertex w chosen with probability sigma_s(w) sigma_t(w) /
//       sigma_st in ascending-id order (radix select on ids, 128-bit weights),
//       then a walk from w to s and from w to t picking each predecessor with
//       probability proportional to its sigma, predecessors in ascending-id
//       (= CSR) order;
//   A4  c~(x) += 1 for every interior vertex of the path;
//   the last CTA of the launch advances tau (A5: stream order makes the
//   counter vector at the next kernel a consistent snapshot).
//
// Layout in HBM (per slot, see SlotSet): one 32-bit code word per vertex
// (0 = not reached; else the side that reached it and its queue position), a
// queue of `cap` positions shared by both sides (s-side grows from the front,
// t-side from the back; the balls are disjoint until they meet) holding each
// reached vertex's id, BFS level and exact 64-bit path count, a meeting-count
// array beside it, and, for each side, one reached bit per vertex.  The code
// word is the only per-vertex state (4 B per vertex and slot), so many slots
// fit even when n is large; a sample whose balls outgrow `cap` runs again on
// a spill slot with cap = n.  Everything is cleared by the sample that set it,
// so no per-sample O(n) reset is needed.
//
// Latency hiding inside one CTA: the layer expansion assigns adjacency
// entries to threads by a block-wide prefix sum over the frontier's degrees
// (every thread gets the same share whatever the degree skew) and keeps
// kUnroll entries per thread in flight: their column ids, then their code
// words (one 4-byte load), then the claims and the path-count additions,
// issued together and waited on once per batch.  A claim CASes the code word
// to "pending", takes a queue position (warp-aggregated) and publishes it;
// an addition that meets a pending claim waits (bounded) for the position.
// A meeting vertex (a target in the other side's last layer) is never
// claimed: its second path count is added at its existing queue position.
//
// The last layer: as soon as a target of the layer is found on the other
// side, the layer is the last one and only meeting vertices need counts;
// other targets are not claimed, and on graphs of small diameter an edge then
// reads only the other side's reached bit (a dense map that stays in L2)
// before the target's code word.
//
// The meeting-vertex choice and walk steps with at most 32 candidates run in
// warp 0 with shuffles, without block barriers; larger ones use the CTA (and,
// at hubs, the predecessor layer from the BFS queue instead of the hub's
// adjacency).  The path's vertices go to the sink in one flush.
//
// Mutable slot state is read with ld.global.cg (L2) so that values written by
// atomics of other threads in the CTA are never served stale from L1.

#include <cstdint>

#include "kadabra_internal.h"
#include "philox.cuh"
#include "stop_math.cuh"

namespace kadabra {
namespace {

constexpr int kMeetCap = 512;      // candidates kept in shared memory (meeting set, predecessors)
constexpr int kBuckets = 256;      // radix-select digit width: 8 bits
constexpr int kMaxLayers = 64;     // BFS layers whose queue ranges are remembered for the walk
constexpr int kPathCap = 1024;     // path vertices buffered in shared memory before a flush
#ifndef KADABRA_UNROLL
#define KADABRA_UNROLL 4
#endif
constexpr int kUnroll = KADABRA_UNROLL;   // adjacency entries in flight per thread
constexpr unsigned int kNone = 0xffffffffu;
constexpr int kProbeMinLog2 = 15;  // smallest probe bitmap worth a pass (4 KB)
// adjacency entries in flight per thread in the probe pass: 8 for CTAs of
// 1024 threads (one per SM: the pass is the SM's only work), 4 below
template <int NT>
struct ProbeUnroll {
    static constexpr int value = NT >= 1024 ? 8 : 4;
};
constexpr int kProbeMaxLog2 = 20;  // largest probe bitmap (128 KB)

__device__ __forceinline__ unsigned long long ldcg(const unsigned long long *p) { return __ldcg(p); }

// The launch's dynamic shared memory: the probe bitmap (2^probe_log2 bits)
// of the other side's frontier, present when the launch sets probe_log2.
__device__ __forceinline__ uint32_t *probe_map()
{
    extern __shared__ __align__(16) uint32_t kadabra_dyn_smem[];
    return kadabra_dyn_smem;
}
// bit of vertex w in a bitmap of 2^log2b bits (Fibonacci hashing: ids of a
// structured layer, e.g. a grid diagonal, spread over the whole map)
__device__ __forceinline__ unsigned int probe_hash(unsigned int w, int log2b)
{
    return (w * 0x9E3779B1u) >> (32 - log2b);
}

__device__ __forceinline__ int bitlen64(unsigned long long x) { return 64 - __clzll(x); }

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Adjacency entries are (neighbour id, neighbour degree) pairs: the degree
// of a newly reached vertex arrives with its id in the same coalesced load,
// so the frontier degree sums need no random row-offset reads.
template <typename OffT>
struct GraphRef {
    const OffT *off;
    const uint2 *adj;
    long long n;
    __device__ __forceinline__ long long col(long long e) const { return (long long)__ldg(&adj[e].x); }
    __device__ __forceinline__ long long begin(long long v) const { return (long long)__ldg(off + v); }
    __device__ __forceinline__ long long end(long long v) const { return (long long)__ldg(off + v + 1); }
};

template <int NT>
struct Smem {
    // sample
    long long s, t;
    unsigned int qlen[2];            // entries appended to each side's queue
    unsigned int fbeg[2], fend[2];   // current frontier = queue positions [fbeg, fend)
    unsigned int layer[2];           // radius reached by each side
    unsigned long long fdeg[2];      // degree sum of each frontier
    unsigned int lbeg[2][kMaxLayers];// queue range of layer k of each side (k < kMaxLayers)
    unsigned int lend[2][kMaxLayers];
    int X;                           // side expanded this layer
    int status;                      // 0 running, 1 met, 2 disconnected, 3 strict overflow,
                                     // 5 discarded (its query stopped), 6 out of queue positions
    int scaled;
    unsigned int err;
    // per-layer accumulators
    unsigned int new_count;
    unsigned int meet_count;
    int meets;                       // a target of this layer is on the other side: it is the last
    unsigned long long lmax;         // largest path count of the new layer
    unsigned long long ldeg;         // degree sum of the new frontier
    unsigned long long e_scan;       // this sample
    unsigned long long expanded;
    // selection and walk
    unsigned long long r_lo, r_hi;   // residual of the 128-bit choice
    unsigned long long sig_lo, sig_hi;
    unsigned int prefix;
    unsigned int pcnt;
    long long chosen;
    unsigned int pw;                 // queue position of the chosen meeting vertex on the other side
    int ovf;                         // a claim found no free queue position
    int spill_k;                     // spill slot taken by this CTA (-1: none)
    int help_k, help_c;              // help request and chunk taken (-1: none)
    struct {
        uint32_t *code, *qv, *ql;
        unsigned long long *qs, *qm;
        uint32_t *bits;
        long long bw, n;
        const void *off;
        const uint2 *adj;
        unsigned int cap, X, nl, fb, fe, qbase, room, yb, ye, cv;
        int mode, log2b;
        unsigned int id;             // request index << 16 | its generation
    } hl;                            // the helped layer, copied from its request
    long long next_v;
    int found;
    // the probe bitmap holds side pf_Y's queue positions [pf_yb, pf_ye) of
    // this sample (pf_ok = 1), or the frontier of helped request pf_req
    // (pf_ok = 2); pf_ok = 0: nothing valid
    int pf_ok, pf_Y;
    unsigned int pf_yb, pf_ye, pf_req;
    unsigned long long cur;          // work item taken by this CTA
    // back-walk: vertices found so far (flushed to the sink by warp 0) and
    // the state handed between warp 0's steps and the whole CTA's steps
    unsigned int path[kPathCap];
    unsigned int plen;               // entries in path[]
    unsigned int pflushed;           // entries flushed before path[0]
    long long wv;
    unsigned int wl;
    int wstate;
    unsigned long long wk;
    unsigned long long tmp[NT / 32];
    unsigned long long tmp2[NT / 32];
    unsigned int cand[kMeetCap];     // candidate ids (meeting set or predecessors)
    unsigned int cpos[kMeetCap];     // meeting set: queue positions on the other side
    unsigned long long wlo[kMeetCap];
    unsigned long long whi[kMeetCap];
    union {
        struct {
            long long cbeg[NT];
            unsigned long long cpos[NT];
            unsigned long long csig[NT];
        } ex;
        struct {
            unsigned long long blo[kBuckets];
            unsigned long long bhi[kBuckets];
        } sel;
    } u;
};

// ---- block-wide primitives ------------------------------------------------

template <int NT>
__device__ __forceinline__ void block_sum2(unsigned long long &a, unsigned long long &b, Smem<NT> &sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    if (lane == 0) {
        sh.tmp[wid] = a;
        sh.tmp2[wid] = b;
    }
    __syncthreads();
    unsigned long long ta = 0, tb = 0;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) {
        ta += sh.tmp[i];
        tb += sh.tmp2[i];
    }
    __syncthreads();
    a = ta;
    b = tb;
}

template <int NT>
__device__ __forceinline__ unsigned long long block_sum(unsigned long long v, Smem<NT> &sh)
{
    unsigned long long z = 0;
    block_sum2<NT>(v, z, sh);
    return v;
}

template <int NT>
__device__ __forceinline__ unsigned long long block_max(unsigned long long v, Smem<NT> &sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        unsigned long long w = __shfl_xor_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    if (lane == 0) sh.tmp[wid] = v;
    __syncthreads();
    unsigned long long m = 0;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) m = sh.tmp[i] > m ? sh.tmp[i] : m;
    __syncthreads();
    return m;
}

// Exclusive prefix sum over the block; *total receives the block sum.
template <int NT>
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v, unsigned long long *total,
                                                              Smem<NT> &sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) sh.tmp[wid] = incl;
    __syncthreads();
    unsigned long long before = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) {
        if (i < wid) before += sh.tmp[i];
        tot += sh.tmp[i];
    }
    __syncthreads();
    *total = tot;
    return before + incl - v;
}

// The same scan with one barrier: sh.tmp must not be written again before
// the caller's next block barrier (the caller's next barrier protects it).
template <int NT>
__device__ __forceinline__ unsigned long long block_excl_scan_open(unsigned long long v, unsigned long long *total,
                                                                   Smem<NT> &sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) sh.tmp[wid] = incl;
    __syncthreads();
    unsigned long long before = 0, tot = 0;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) {
        if (i < wid) before += sh.tmp[i];
        tot += sh.tmp[i];
    }
    *total = tot;
    return before + incl - v;
}

// 128-bit helpers (lo, hi pairs)
__device__ __forceinline__ void add128(unsigned long long &lo, unsigned long long &hi, unsigned long long blo,
                                       unsigned long long bhi)
{
    const unsigned long long l = lo + blo;
    hi += bhi + (l < lo ? 1ULL : 0ULL);
    lo = l;
}

__device__ __forceinline__ bool less128(unsigned long long alo, unsigned long long ahi, unsigned long long blo,
                                        unsigned long long bhi)
{
    return ahi < bhi || (ahi == bhi && alo < blo);
}

__device__ __forceinline__ void smem_add128(unsigned long long *lo, unsigned long long *hi, unsigned long long vlo,
                                            unsigned long long vhi)
{
    const unsigned long long old = atomicAdd(lo, vlo);
    const unsigned long long carry = (old + vlo < old) ? 1ULL : 0ULL;
    if (vhi + carry) atomicAdd(hi, vhi + carry);
}

template <int NT>
__device__ __forceinline__ void block_sum128(unsigned long long &lo, unsigned long long &hi, Smem<NT> &sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long ol = __shfl_xor_sync(0xffffffffu, lo, o);
        const unsigned long long oh = __shfl_xor_sync(0xffffffffu, hi, o);
        add128(lo, hi, ol, oh);
    }
    if (lane == 0) {
        sh.tmp[wid] = lo;
        sh.tmp2[wid] = hi;
    }
    __syncthreads();
    unsigned long long tl = 0, th = 0;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) add128(tl, th, sh.tmp[i], sh.tmp2[i]);
    __syncthreads();
    lo = tl;
    hi = th;
}

// Weighted choice by vertex id: among the candidates produced by `each`
// (a functor calling its argument with (id, weight_lo, weight_hi) for the
// calling thread's share), return the first id in ascending order whose
// inclusive prefix weight exceeds r = (sh.r_lo, sh.r_hi) < total weight.
// Radix select over the id bits, 8 bits per pass from the top; each pass
// sums 128-bit weights into 256 shared-memory buckets and one warp finds the
// bucket holding r.  Returns -1 if no bucket holds r (broken invariant).
template <int NT, typename Each>
__device__ long long radix_choose(Smem<NT> &sh, int npass, Each each)
{
    const int tid = threadIdx.x;
    if (tid == 0) sh.prefix = 0;
    for (int p = npass - 1; p >= 0; --p) {
        const int shft = 8 * p;
        for (int b = tid; b < kBuckets; b += NT) {
            sh.u.sel.blo[b] = 0;
            sh.u.sel.bhi[b] = 0;
        }
        // every thread has read the previous pass's `found` before this barrier,
        // so `found` is re-armed only after it
        __syncthreads();
        if (tid == 0) sh.found = 0;
        const unsigned int pref = sh.prefix;
        const bool top = (p == npass - 1);
        each([&](unsigned int id, unsigned long long lo, unsigned long long hi) {
            if (!top && (id >> (shft + 8)) != pref) return;
            const int dg = (id >> shft) & 255;
            smem_add128(&sh.u.sel.blo[dg], &sh.u.sel.bhi[dg], lo, hi);
        });
        __syncthreads();
        if (tid < 32) {
            // lane l owns buckets [8l, 8l + 8)
            unsigned long long slo = 0, shi = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) add128(slo, shi, sh.u.sel.blo[tid * 8 + j], sh.u.sel.bhi[tid * 8 + j]);
            unsigned long long ilo = slo, ihi = shi;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const unsigned long long yl = __shfl_up_sync(0xffffffffu, ilo, o);
                const unsigned long long yh = __shfl_up_sync(0xffffffffu, ihi, o);
                if (tid >= o) add128(ilo, ihi, yl, yh);
            }
            unsigned long long elo = ilo - slo;
            unsigned long long ehi = ihi - shi - (ilo < slo ? 1ULL : 0ULL);
            const unsigned long long rlo = sh.r_lo, rhi = sh.r_hi;
            __syncwarp();   // every lane has read r before one lane rewrites it
            if (!less128(rlo, rhi, elo, ehi) && less128(rlo, rhi, ilo, ihi)) {
                for (int j = 0; j < 8; ++j) {
                    unsigned long long nlo = elo, nhi = ehi;
                    add128(nlo, nhi, sh.u.sel.blo[tid * 8 + j], sh.u.sel.bhi[tid * 8 + j]);
                    if (less128(rlo, rhi, nlo, nhi)) {
                        sh.r_lo = rlo - elo;
                        sh.r_hi = rhi - ehi - (rlo < elo ? 1ULL : 0ULL);
                        sh.prefix = (pref << 8) | (unsigned int)(tid * 8 + j);
                        sh.found = 1;
                        break;
                    }
                    elo = nlo;
                    ehi = nhi;
                }
            }
        }
        __syncthreads();
        if (!sh.found) return -1;
    }
    return (long long)sh.prefix;
}

// Warp 0 picks among cnt <= 32 candidates (sh.cand, 64-bit weights sh.wlo)
// the one whose interval, in ascending id order, holds r; sh.next_v.
template <int NT>
__device__ __forceinline__ void warp_pick64(Smem<NT> &sh, unsigned int cnt, unsigned long long r)
{
    if (threadIdx.x >= 32) return;
    const unsigned int lane = threadIdx.x;
    const bool have = lane < cnt;
    const unsigned int id = have ? sh.cand[lane] : 0xffffffffu;
    const unsigned long long wt = have ? sh.wlo[lane] : 0ULL;
    unsigned long long pre = 0;
    for (int j = 0; j < 32; ++j) {
        const unsigned int idj = __shfl_sync(0xffffffffu, id, j);
        const unsigned long long wj = __shfl_sync(0xffffffffu, wt, j);
        if (idj < id) pre += wj;
    }
    const bool mine = have && pre <= r && r < pre + wt;
    const unsigned int m = __ballot_sync(0xffffffffu, mine);
    const unsigned int pick = m ? __shfl_sync(0xffffffffu, id, __ffs(m) - 1) : 0u;
    if (lane == 0) sh.next_v = m ? (long long)pick : -1;
}

// ---- one slot's scratch ----------------------------------------------------

constexpr unsigned int kSideBit = 0x80000000u;
constexpr unsigned int kPosMask = 0x7fffffffu;
constexpr unsigned int kPending = kPosMask;   // position field while a claim is being published

__device__ __forceinline__ unsigned int code_of(int side, unsigned int p) { return (side ? kSideBit : 0u) | (p + 1u); }
__device__ __forceinline__ int side_of(unsigned int c) { return (int)(c >> 31); }
__device__ __forceinline__ bool is_pending(unsigned int c) { return (c & kPosMask) == kPending; }
__device__ __forceinline__ unsigned int pos_of(unsigned int c) { return (c & kPosMask) - 1u; }

// One slot's view of a SlotSet.
struct Slot {
    uint32_t *code;
    uint32_t *qv, *ql;
    unsigned long long *qs, *qm;
    uint32_t *bits;            // null: the sample does not use reached-bit maps
    long long bw;              // words of one side's map
    unsigned int cap;
    // array index of a side's queue position p
    __device__ __forceinline__ unsigned int at(int side, unsigned int p) const { return side ? cap - 1u - p : p; }
};

__device__ __forceinline__ Slot slot_of(const SlotSet &S, int k, bool use_bits)
{
    Slot s;
    s.code = S.code + (size_t)k * (size_t)S.stride;
    s.qv = S.qv + (size_t)k * (size_t)S.cap;
    s.ql = S.ql + (size_t)k * (size_t)S.cap;
    s.qs = S.qs + (size_t)k * (size_t)S.cap;
    s.qm = S.qm + (size_t)k * (size_t)S.cap;
    s.bw = bit_words(S.stride);
    s.bits = (use_bits && S.bits) ? S.bits + (size_t)k * (size_t)(2 * s.bw) : nullptr;
    s.cap = (unsigned int)S.cap;
    return s;
}

// Is `key` in the ascending neighbour list adj[b, b + d)?
__device__ __forceinline__ bool contains(const uint2 *adj, long long b, long long d, long long key)
{
    long long lo = b, hi = b + d;
    while (lo < hi) {
        const long long mid = (lo + hi) >> 1;
        if ((long long)__ldg(&adj[mid].x) < key) lo = mid + 1;
        else hi = mid;
    }
    return lo < b + d && (long long)__ldg(&adj[lo].x) == key;
}

// Path count of u if it was reached by `side` at BFS level `level`, else 0.
__device__ __forceinline__ unsigned long long pred_weight(const Slot &S, int side, long long u, unsigned int level)
{
    const unsigned int c = __ldcg(S.code + u);
    if (c == 0u || side_of(c) != side || is_pending(c)) return 0ULL;
    const unsigned int ph = S.at(side, pos_of(c));
    return __ldcg(S.ql + ph) == level ? __ldcg(S.qs + ph) : 0ULL;
}

// ---- one sample ------------------------------------------------------------

// Where a sample's interior vertices go: straight into c~ (epoch launches,
// calibration), or into the log of the sample's epoch (pipelined launch).
struct CountSink {
    uint32_t *counts;
    uint32_t *log;
    unsigned int *len;
    unsigned int cap;
};

// Warp 0 hands the buffered path vertices path[0, cnt) to the sink (counter
// increments, or one log reservation for all of them); returns error bits.
__device__ __forceinline__ unsigned int sink_flush(const CountSink &sink, const unsigned int *path, unsigned int cnt)
{
    const unsigned int lane = threadIdx.x & 31;
    unsigned int err = 0;
    if (sink.counts) {
        for (unsigned int i = lane; i < cnt; i += 32) {
            const unsigned int old = atomicAdd(&sink.counts[path[i]], 1u);
            if (old == 0xffffffffu) err |= kErrCounterOverflow;
        }
    } else if (sink.log && cnt) {
        unsigned int p0 = 0;
        if (lane == 0) p0 = atomicAdd(sink.len, cnt);
        p0 = __shfl_sync(0xffffffffu, p0, 0);
        for (unsigned int i = lane; i < cnt; i += 32) {
            if (p0 + i >= sink.cap) err |= kErrLogOverflow;
            else __stcg(sink.log + p0 + i, path[i]);
        }
    }
    return __reduce_or_sync(0xffffffffu, err);
}

struct LocalStats {
    unsigned long long samples, connected, e_scan, expanded, touched, interior, walk_scan, scaled;
};

// kinds of a scanned adjacency target (phase 2 of a layer)
enum : int { kTSkip = 0, kTUnseen = 1, kTMeet = 2, kTSame = 3, kTPend = 4 };

// Where a layer's accumulators live: the CTA's shared memory (a layer one
// CTA expands), or a help request in global memory (a layer several CTAs
// expand together).
template <int NT>
struct SmemAcc {
    Smem<NT> &sh;
    __device__ __forceinline__ unsigned int *new_count() const { return &sh.new_count; }
    __device__ __forceinline__ unsigned int *meet_count() const { return &sh.meet_count; }
    __device__ __forceinline__ unsigned int *cand() const { return sh.cand; }
    __device__ __forceinline__ unsigned int *cpos() const { return sh.cpos; }
    __device__ __forceinline__ volatile int *meets() const { return &sh.meets; }
    __device__ __forceinline__ unsigned int *err() const { return &sh.err; }
    __device__ __forceinline__ volatile int *ovf() const { return &sh.ovf; }
    __device__ __forceinline__ unsigned long long *lmax() const { return &sh.lmax; }
    __device__ __forceinline__ unsigned long long *ldeg() const { return &sh.ldeg; }
};

// A layer posted for several CTAs of a persistent launch to expand together:
// a heavy layer (frontier degree sum above the launch's threshold) of one
// sample is split into chunks of frontier vertices; its owner and any CTA
// between two samples take chunks until none is left, then the owner waits
// until all are done and collects the accumulators.  Every claim and count
// is an atomic on the slot's global state, so the result is the same whoever
// expands which chunk.
constexpr int kHelpSlots = 8;
struct HelpReq {
    unsigned long long ticket;     // bits 48..63 generation, 24..47 chunks, 0..23 next chunk
    unsigned int done;             // chunks finished
    int state;                     // 0 free, 1 held by an owner
    // the layer (read by helpers, written before the ticket opens)
    uint32_t *code, *qv, *ql;
    unsigned long long *qs, *qm;
    uint32_t *bits;
    long long bw;
    const void *off;
    const uint2 *adj;
    long long n;
    unsigned int cap, X, nl, fb, fe, qbase, room, yb, ye, cv;
    int mode;                      // 0: expand the layer; 1: probe pass
    int log2b;                     // probe bitmap size of the launch
    // accumulators
    unsigned long long lmax, ldeg, scan;
    unsigned int new_count, meet_count, err;
    int meets, ovf;
    unsigned int cand[kMeetCap], cpos[kMeetCap];
};

struct ReqAcc {
    HelpReq *r;
    __device__ __forceinline__ unsigned int *new_count() const { return &r->new_count; }
    __device__ __forceinline__ unsigned int *meet_count() const { return &r->meet_count; }
    __device__ __forceinline__ unsigned int *cand() const { return r->cand; }
    __device__ __forceinline__ unsigned int *cpos() const { return r->cpos; }
    __device__ __forceinline__ volatile int *meets() const { return &r->meets; }
    __device__ __forceinline__ unsigned int *err() const { return &r->err; }
    __device__ __forceinline__ volatile int *ovf() const { return &r->ovf; }
    __device__ __forceinline__ unsigned long long *lmax() const { return &r->lmax; }
    __device__ __forceinline__ unsigned long long *ldeg() const { return &r->ldeg; }
};

// Takes the next chunk of request R, or -1 if none is left.  The ticket is
// read first, so once the chunks are gone no further add touches it (its
// chunk field never overflows into the count).
__device__ __forceinline__ int take_chunk(HelpReq *R)
{
    const unsigned long long t = *reinterpret_cast<volatile unsigned long long *>(&R->ticket);
    if ((t & 0xffffffULL) >= ((t >> 24) & 0xffffffULL)) return -1;
    const unsigned long long got = atomicAdd(&R->ticket, 1ULL);
    if ((got & 0xffffffULL) >= ((got >> 24) & 0xffffffULL)) return -1;
    return (int)(got & 0xffffffULL);
}

// A help board: a 256-byte header (the count of requests with chunks left)
// and kHelpSlots requests.
__device__ __forceinline__ unsigned int *board_open(void *h) { return reinterpret_cast<unsigned int *>(h); }
__device__ __forceinline__ HelpReq *board_req(void *h)
{
    return reinterpret_cast<HelpReq *>(reinterpret_cast<unsigned char *>(h) + 256);
}

// Expands the frontier vertices [cb, min(cb + NT, fe)) of side X's current
// layer (CTA-wide): every adjacency entry of them is scanned once; unseen
// targets are claimed for level nl, targets already in the new layer get the
// source's path count added, targets in the other side's last layer (queue
// positions [yb, ye)) get it added to their meeting count.  Returns the
// chunk's adjacency-entry count in thread 0 (0 elsewhere).
template <int NT, typename OffT, typename Acc>
__device__ __forceinline__ unsigned long long expand_chunk(const unsigned long long spin_limit, const GraphRef<OffT> &G,
                                                           const Slot &S, Smem<NT> &sh, const Acc &A, const int X,
                                                           const unsigned int nl, const unsigned int cb,
                                                           const unsigned int fe, const unsigned int qbase,
                                                           const unsigned int room, const unsigned int yb,
                                                           const unsigned int ye)
{
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int Y = 1 - X;
    const unsigned int pend_code = (X ? kSideBit : 0u) | kPending;
    unsigned long long my_max = 0, my_scan = 0, my_deg = 0;
        const unsigned int i = cb + tid;
        long long b = 0;
        unsigned long long d = 0, sg = 0;
        if (i < fe) {
            const unsigned int ph = S.at(X, i);
            const unsigned int u = __ldcg(S.qv + ph);
            b = G.begin(u);
            d = (unsigned long long)(G.end(u) - b);
            sg = ldcg(S.qs + ph);
        }
        unsigned long long total;
        // one barrier: sh.tmp is next written after this chunk's closing barrier
        const unsigned long long excl = block_excl_scan_open<NT>(d, &total, sh);
        sh.u.ex.cbeg[tid] = b;
        sh.u.ex.cpos[tid] = excl;
        sh.u.ex.csig[tid] = sg;
        const int cnt = (int)min((unsigned int)NT, fe - cb);
        __syncthreads();
        my_scan = (tid == 0) ? total : 0ULL;
        // warp-uniform batches: lane l of warp k handles entries
        // e0 + l + j*NT, j < kUnroll, with e0 = 32k + (multiple of NT*kUnroll);
        // each phase issues all kUnroll memory operations before waiting
        const unsigned long long wbase = (unsigned long long)(tid & ~31);
        for (unsigned long long e0 = wbase; e0 < total; e0 += (unsigned long long)NT * kUnroll) {
            unsigned int w[kUnroll];
            unsigned int dw[kUnroll];
            int own[kUnroll];
#pragma unroll
            for (int j = 0; j < kUnroll; ++j) {
                const unsigned long long e = e0 + (unsigned long long)lane + (unsigned long long)j * NT;
                w[j] = kNone;
                dw[j] = 0;
                own[j] = 0;
                if (e < total) {
                    // owner: the last k with cpos[k] <= e
                    int lo = j > 0 ? own[j - 1] : 0, hi = cnt - 1;
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (sh.u.ex.cpos[mid] <= e) lo = mid;
                        else hi = mid - 1;
                    }
                    own[j] = lo;
                    const uint2 c = __ldg(G.adj + sh.u.ex.cbeg[lo] + (long long)(e - sh.u.ex.cpos[lo]));
                    w[j] = c.x;
                    dw[j] = c.y;
                }
            }
            // phase 2: the code word of every target (one 4-byte load each);
            // once the layer is known to be the last, only the other side's
            // reached bit first (a dense map that stays in L2), and the code
            // only of targets that have it
            unsigned int cd[kUnroll];
            int kind[kUnroll];
            const bool fast = S.bits != nullptr && *A.meets() != 0;
            if (fast) {
                const uint32_t *ybits = S.bits + (X ? 0 : S.bw);
                unsigned int ymask = 0;
#pragma unroll
                for (int j = 0; j < kUnroll; ++j)
                    if (w[j] != kNone && ((__ldcg(ybits + (w[j] >> 5)) >> (w[j] & 31)) & 1u)) ymask |= 1u << j;
#pragma unroll
                for (int j = 0; j < kUnroll; ++j) cd[j] = ((ymask >> j) & 1u) ? __ldcg(S.code + w[j]) : 0u;
#pragma unroll
                for (int j = 0; j < kUnroll; ++j) kind[j] = ((ymask >> j) & 1u) ? kTMeet : kTSkip;
            } else {
#pragma unroll
                for (int j = 0; j < kUnroll; ++j) cd[j] = w[j] != kNone ? __ldcg(S.code + w[j]) : 0u;
#pragma unroll
                for (int j = 0; j < kUnroll; ++j) {
                    const unsigned int c = cd[j];
                    kind[j] = w[j] == kNone ? kTSkip
                              : c == 0u ? kTUnseen
                              : side_of(c) != X ? kTMeet
                              : is_pending(c) ? kTPend
                              : pos_of(c) >= qbase ? kTSame : kTSkip;
                }
            }
            // a target held by the other side makes this layer the last one:
            // from then on only meeting vertices need counts, so other unseen
            // targets of the last layer are not claimed
#pragma unroll
            for (int j = 0; j < kUnroll; ++j)
                if (kind[j] == kTMeet) *A.meets() = 1;
            const bool last = *A.meets() != 0;
            // phase 3: claims (CAS on the code word to "pending"), path-count
            // additions to targets already in the new layer, and meeting
            // counts (the other side's last layer, indexed by its queue
            // position).  The additions return their old value, so a thread
            // has waited for all of them before the layer's closing barrier
            // and every count is complete when any thread reads it next.
            unsigned int cmask = 0, mfirst = 0, retry = 0;
#pragma unroll
            for (int j = 0; j < kUnroll; ++j) {
                if (kind[j] == kTUnseen) {
                    if (last) {
                        kind[j] = kTSkip;
                    } else {
                        const unsigned int old = atomicCAS(S.code + w[j], 0u, pend_code);
                        if (old == 0u) {
                            cmask |= 1u << j;
                        } else {
                            // claimed in this layer by another thread meanwhile
                            cd[j] = old;
                            kind[j] = is_pending(old) ? kTPend : kTSame;
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < kUnroll; ++j) {
                const unsigned long long su = sh.u.ex.csig[own[j]];
                if (kind[j] == kTMeet) {
                    const unsigned int p = pos_of(cd[j]);
                    if (side_of(cd[j]) != Y || is_pending(cd[j]) || p < yb || p >= ye) {
                        atomicOr(A.err(), kErrSelect);     // broken invariant: never expected
                        continue;
                    }
                    const unsigned long long old = atomicAdd(S.qm + S.at(Y, p), su);
                    if (old == 0ULL) mfirst |= 1u << j;
                    if (old + su < su) atomicOr(A.err(), kErrAddOverflow);
                } else if (kind[j] == kTSame) {
                    const unsigned int p = pos_of(cd[j]);
                    if (side_of(cd[j]) != X || p < qbase) {
                        atomicOr(A.err(), kErrSelect);
                        continue;
                    }
                    const unsigned long long nv = atomicAdd(S.qs + S.at(X, p), su) + su;
                    if (nv < su) atomicOr(A.err(), kErrAddOverflow);      // excluded by the choice of K
                    my_max = nv > my_max ? nv : my_max;
                } else if (kind[j] == kTPend) {
                    retry |= 1u << j;
                }
            }
            // phase 4: claimed targets join the new frontier (warp-aggregated
            // queue positions), get their first path count and publish their
            // position; first-touched meeting vertices join the meeting set
#pragma unroll
            for (int j = 0; j < kUnroll; ++j) {
                const bool claimed = (cmask >> j) & 1u;
                const unsigned int m = __ballot_sync(0xffffffffu, claimed);
                if (m) {
                    const int leader = __ffs(m) - 1;
                    unsigned int slot0 = 0;
                    if (lane == leader) slot0 = atomicAdd(A.new_count(), (unsigned int)__popc(m));
                    slot0 = __shfl_sync(0xffffffffu, slot0, leader);
                    if (claimed) {
                        const unsigned int p = qbase + slot0 + __popc(m & ((1u << lane) - 1u));
                        if (p < room) {
                            const unsigned int ph = S.at(X, p);
                            const unsigned long long su = sh.u.ex.csig[own[j]];
                            __stcg(S.qv + ph, w[j]);
                            __stcg(S.ql + ph, nl);
                            const unsigned long long nv = atomicAdd(S.qs + ph, su) + su;
                            if (nv < su) atomicOr(A.err(), kErrAddOverflow);
                            my_max = nv > my_max ? nv : my_max;
                            __stcg(S.code + w[j], code_of(X, p));
                            my_deg += dw[j];
                            if (S.bits) atomicOr(&S.bits[(X ? S.bw : 0) + (w[j] >> 5)], 1u << (w[j] & 31));
                        } else {
                            // out of queue positions: the sample restarts on a larger slot
                            *A.ovf() = 1;
                            __stcg(S.code + w[j], 0u);
                        }
                    }
                }
                if ((mfirst >> j) & 1u) {
                    const unsigned int p = atomicAdd(A.meet_count(), 1u);
                    if (p < kMeetCap) {
                        A.cand()[p] = w[j];
                        A.cpos()[p] = pos_of(cd[j]);
                    }
                }
            }
            // phase 5: additions to targets whose claim (by another warp) was
            // still being published; this warp published its own claims above
            __syncwarp();
            if (retry) {
#pragma unroll
                for (int j = 0; j < kUnroll; ++j) {
                    if (!((retry >> j) & 1u)) continue;
                    unsigned int c = *reinterpret_cast<volatile unsigned int *>(S.code + w[j]);
                    unsigned long long spins = 0;
                    while (is_pending(c) && ++spins < spin_limit) {
                        __nanosleep(32);
                        c = *reinterpret_cast<volatile unsigned int *>(S.code + w[j]);
                    }
                    if (is_pending(c)) {
                        atomicOr(A.err(), kErrTimeout);
                        continue;
                    }
                    if (c == 0u) continue;      // the claim ran out of positions: the sample restarts
                    const unsigned long long su = sh.u.ex.csig[own[j]];
                    const unsigned long long nv = atomicAdd(S.qs + S.at(X, pos_of(c)), su) + su;
                    if (nv < su) atomicOr(A.err(), kErrAddOverflow);
                    my_max = nv > my_max ? nv : my_max;
                }
            }
        }
        // largest new path count (every count's final value is the largest
        // value its additions returned) and the new frontier's degree sum,
        // folded per warp into shared memory before the chunk's barrier
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) {
            const unsigned long long om = __shfl_xor_sync(0xffffffffu, my_max, o);
            my_max = om > my_max ? om : my_max;
            my_deg += __shfl_xor_sync(0xffffffffu, my_deg, o);
        }
        if (lane == 0) {
            if (my_max) atomicMax(A.lmax(), my_max);
            if (my_deg) atomicAdd(A.ldeg(), my_deg);
        }
        my_max = 0;
        my_deg = 0;
        __syncthreads();
    return my_scan;
}

// ---- probe pass --------------------------------------------------------
// On graphs of small diameter a layer is often the last one: some of its
// targets are in the other side's frontier.  The probe pass scans the layer's
// adjacency once, tests every target against a shared-memory bitmap of that
// frontier, and reads the code word only of targets whose bit is set, so the
// scan costs the adjacency reads alone.  If it finds meeting vertices their
// meeting counts are complete (every adjacency entry was scanned) and the
// layer ends without claiming anything: the next layer is never expanded.  If
// it finds none, no target is on the other side (the bitmap has no false
// negatives) and the layer is expanded as usual.

// Fills the bitmap with side Y's queue positions [yb, ye) (CTA-wide; the
// caller has ensured ye - yb fits the map's load limit).
template <int NT>
__device__ __forceinline__ void probe_build(const int log2b, const Slot &S, const int Y, const unsigned int yb,
                                            const unsigned int ye)
{
    uint4 *m4 = reinterpret_cast<uint4 *>(probe_map());
    const int n4 = 1 << (log2b - 7);
    for (int i = threadIdx.x; i < n4; i += NT) m4[i] = make_uint4(0u, 0u, 0u, 0u);
    __syncthreads();
    uint32_t *m = probe_map();
    for (unsigned int p = yb + threadIdx.x; p < ye; p += NT) {
        const unsigned int h = probe_hash(__ldcg(S.qv + S.at(Y, p)), log2b);
        atomicOr(&m[h >> 5], 1u << (h & 31));
    }
    __syncthreads();
}

// Probes the frontier vertices [cb, min(cb + NT, fe)) of side X's current
// layer (CTA-wide): a target in side Y's frontier (queue positions [yb, ye))
// gets the source's path count added to its meeting count and joins the
// meeting set, exactly as in expand_chunk; nothing else is written.  Returns
// the chunk's adjacency-entry count in thread 0 (0 elsewhere).
template <int NT, typename OffT, typename Acc>
__device__ __forceinline__ unsigned long long probe_chunk(const GraphRef<OffT> &G, const Slot &S, Smem<NT> &sh,
                                                          const Acc &A, const int log2b, const int X,
                                                          const unsigned int cb, const unsigned int fe,
                                                          const unsigned int yb, const unsigned int ye)
{
    constexpr int kProbeUnroll = ProbeUnroll<NT>::value;
    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int Y = 1 - X;
    const uint32_t *m = probe_map();
    const unsigned int i = cb + tid;
    long long b = 0;
    unsigned long long d = 0, sg = 0;
    if (i < fe) {
        const unsigned int ph = S.at(X, i);
        const unsigned int u = __ldcg(S.qv + ph);
        b = G.begin(u);
        d = (unsigned long long)(G.end(u) - b);
        sg = ldcg(S.qs + ph);
    }
    unsigned long long total;
    const unsigned long long excl = block_excl_scan_open<NT>(d, &total, sh);
    sh.u.ex.cbeg[tid] = b;
    sh.u.ex.cpos[tid] = excl;
    sh.u.ex.csig[tid] = sg;
    const int cnt = (int)min((unsigned int)NT, fe - cb);
    __syncthreads();
    const unsigned long long wbase = (unsigned long long)(tid & ~31);
    for (unsigned long long e0 = wbase; e0 < total; e0 += (unsigned long long)NT * kProbeUnroll) {
        unsigned int w[kProbeUnroll];
        int own[kProbeUnroll];
#pragma unroll
        for (int j = 0; j < kProbeUnroll; ++j) {
            const unsigned long long e = e0 + (unsigned long long)lane + (unsigned long long)j * NT;
            w[j] = kNone;
            own[j] = 0;
            if (e < total) {
                int lo = j > 0 ? own[j - 1] : 0, hi = cnt - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (sh.u.ex.cpos[mid] <= e) lo = mid;
                    else hi = mid - 1;
                }
                own[j] = lo;
                w[j] = __ldg(&G.adj[sh.u.ex.cbeg[lo] + (long long)(e - sh.u.ex.cpos[lo])].x);
            }
        }
        unsigned int cd[kProbeUnroll];
#pragma unroll
        for (int j = 0; j < kProbeUnroll; ++j) {
            cd[j] = 0u;
            if (w[j] != kNone) {
                const unsigned int h = probe_hash(w[j], log2b);
                if ((m[h >> 5] >> (h & 31)) & 1u) cd[j] = __ldcg(S.code + w[j]);
            }
        }
#pragma unroll
        for (int j = 0; j < kProbeUnroll; ++j) {
            const unsigned int c = cd[j];
            if (c == 0u || side_of(c) != Y) continue;     // unseen, or on this side
            const unsigned int p = pos_of(c);
            if (is_pending(c) || p < yb || p >= ye) {
                atomicOr(A.err(), kErrSelect);             // broken invariant: never expected
                continue;
            }
            const unsigned long long su = sh.u.ex.csig[own[j]];
            const unsigned long long old = atomicAdd(S.qm + S.at(Y, p), su);
            if (old + su < su) atomicOr(A.err(), kErrAddOverflow);
            *A.meets() = 1;
            if (old == 0ULL) {
                const unsigned int q = atomicAdd(A.meet_count(), 1u);
                if (q < kMeetCap) {
                    A.cand()[q] = w[j];
                    A.cpos()[q] = p;
                }
            }
        }
    }
    __syncthreads();
    return tid == 0 ? total : 0ULL;
}

// Makes the bitmap hold side Y's frontier [yb, ye) of the CTA's own sample
// (CTA-wide; nothing to do if it already does).
template <int NT>
__device__ __forceinline__ void probe_ready(const int log2b, const Slot &S, Smem<NT> &sh, const int Y,
                                            const unsigned int yb, const unsigned int ye)
{
    if (!(sh.pf_ok == 1 && sh.pf_Y == Y && sh.pf_yb == yb && sh.pf_ye == ye)) {
        probe_build<NT>(log2b, S, Y, yb, ye);
        // read next after the layer's closing barrier
        if (threadIdx.x == 0) {
            sh.pf_ok = 1;
            sh.pf_Y = Y;
            sh.pf_yb = yb;
            sh.pf_ye = ye;
        }
    }
}

// The probe pass over side X's whole current layer [fb, fe) by this CTA
// alone.  Returns the layer's adjacency-entry count in thread 0 (0
// elsewhere); after it, sh.meets says whether the layer met side Y.
template <int NT, typename OffT>
__device__ __noinline__ unsigned long long probe_layer(const GraphRef<OffT> &G, const Slot &S, Smem<NT> &sh,
                                                       const int log2b, const int X, const unsigned int fb,
                                                       const unsigned int fe, const unsigned int yb,
                                                       const unsigned int ye)
{
    probe_ready<NT>(log2b, S, sh, 1 - X, yb, ye);
    unsigned long long ps = 0;
    for (unsigned int cb = fb; cb < fe; cb += NT)
        ps += probe_chunk<NT, OffT>(G, S, sh, SmemAcc<NT>{sh}, log2b, X, cb, fe, yb, ye);
    return ps;
}

// A heavy layer of a persistent launch, posted on the help board (mode 0:
// expand, 1: probe): the CTA takes chunks of cv frontier vertices with every
// CTA that joins until none is left, waits (bounded) for the chunks others
// took, and copies the request's accumulators into its own.  Returns false,
// having done nothing, if no request was free.
template <int NT, typename OffT>
__device__ __noinline__ bool help_layer(const SampleLaunch &a, const GraphRef<OffT> &G, const Slot &S, Smem<NT> &sh,
                                        const int mode, const int X, const unsigned int nl, const unsigned int fb,
                                        const unsigned int fe, const unsigned int qbase, const unsigned int room,
                                        const unsigned int yb, const unsigned int ye, unsigned long long &my_scan)
{
    const int tid = threadIdx.x;
    const unsigned int cv = (unsigned int)NT / 8u;
    const unsigned int nch = (fe - fb + cv - 1u) / cv;
    if (tid == 0) {
        HelpReq *board = board_req(a.help);
        int k = -1;
        if (nch < (1u << 23))
            for (int i = 0; i < kHelpSlots && k < 0; ++i)
                if (atomicCAS(&board[i].state, 0, 1) == 0) k = i;
        if (k >= 0) {
            HelpReq *R = board + k;
            R->code = S.code; R->qv = S.qv; R->ql = S.ql; R->qs = S.qs; R->qm = S.qm;
            R->bits = S.bits; R->bw = S.bw; R->off = G.off; R->adj = G.adj; R->n = G.n;
            R->cap = S.cap; R->X = (unsigned int)X; R->nl = nl; R->fb = fb; R->fe = fe; R->qbase = qbase;
            R->room = room; R->yb = yb; R->ye = ye; R->cv = cv;
            R->mode = mode; R->log2b = a.probe_log2;
            R->lmax = 0; R->ldeg = 0; R->scan = 0; R->new_count = 0; R->meet_count = 0; R->err = 0;
            R->meets = 0; R->ovf = 0; R->done = 0;
            __threadfence();
            const unsigned long long gen = (*reinterpret_cast<volatile unsigned long long *>(&R->ticket) >> 48) + 1ULL;
            atomicExch(&R->ticket, ((gen & 0xffffULL) << 48) | ((unsigned long long)nch << 24));
            __threadfence();
            atomicAdd(board_open(a.help), 1u);
        }
        sh.help_k = k;
    }
    __syncthreads();
    const int hk = sh.help_k;
    if (hk < 0) return false;
    HelpReq *R = board_req(a.help) + hk;
    for (;;) {
        if (tid == 0) sh.help_c = take_chunk(R);
        __syncthreads();
        const int c = sh.help_c;
        if (c < 0) break;
        const unsigned int cb = fb + (unsigned int)c * cv;
        const unsigned long long sc =
            mode ? probe_chunk<NT, OffT>(G, S, sh, ReqAcc{R}, a.probe_log2, X, cb, min(cb + cv, fe), yb, ye)
                 : expand_chunk<NT, OffT>(a.spin_limit, G, S, sh, ReqAcc{R}, X, nl, cb, min(cb + cv, fe), qbase,
                                          room, yb, ye);
        if (tid == 0) {
            atomicAdd(&R->scan, sc);
            __threadfence();
            atomicAdd(&R->done, 1u);
        }
    }
    // no chunk left to take; wait (bounded) for the chunks other CTAs took,
    // then collect
    if (tid == 0) {
        atomicSub(board_open(a.help), 1u);
        unsigned long long w = 0;
        while (*reinterpret_cast<volatile unsigned int *>(&R->done) < nch && ++w < a.spin_limit) __nanosleep(256);
        __threadfence();
        if (*reinterpret_cast<volatile unsigned int *>(&R->done) < nch) sh.err |= kErrTimeout;
        sh.new_count = *reinterpret_cast<volatile unsigned int *>(&R->new_count);
        sh.meet_count = *reinterpret_cast<volatile unsigned int *>(&R->meet_count);
        sh.meets = *reinterpret_cast<volatile int *>(&R->meets);
        sh.ovf |= *reinterpret_cast<volatile int *>(&R->ovf);
        sh.err |= *reinterpret_cast<volatile unsigned int *>(&R->err);
        sh.lmax = *reinterpret_cast<volatile unsigned long long *>(&R->lmax);
        sh.ldeg = *reinterpret_cast<volatile unsigned long long *>(&R->ldeg);
        my_scan = *reinterpret_cast<volatile unsigned long long *>(&R->scan);
    }
    __syncthreads();
    const unsigned int mc = min(sh.meet_count, (unsigned int)kMeetCap);
    for (unsigned int i = tid; i < mc; i += NT) {
        sh.cand[i] = __ldcg(R->cand + i);
        sh.cpos[i] = __ldcg(R->cpos + i);
    }
    __syncthreads();
    // the request is free again only if every chunk is done (a request
    // whose wait gave up stays held: a late helper may still write it)
    if (tid == 0 && !(sh.err & kErrTimeout)) {
        __threadfence();
        atomicExch(&R->state, 0);
    }
    return true;
}

// Runs sample `idx` in slot S.  Returns false if the sample's two balls
// outgrew the slot's queue capacity: the slot is then clear again and
// nothing was counted, and the caller runs the sample on a larger slot.
template <int NT, typename OffT>
__device__ bool run_sample(const SampleLaunch &a, const GraphRef<OffT> &G, const Slot &S, Smem<NT> &sh,
                           unsigned long long idx, unsigned long long trace_i, LocalStats &ls, const CountSink &sink)
{
    const int tid = threadIdx.x;
    const long long n = G.n;
    unsigned long long t_start = 0, t_bfs = 0, t_sel = 0, t_walk = 0;

    // A1: pair (draw 0)
    if (tid == 0) {
        if (a.trace) t_start = global_ns();
        const U64x4 x = sample_draw(a.seed, a.tag, idx, 0);
        const unsigned long long s = __umul64hi(x.v[0], (unsigned long long)n);
        unsigned long long t = __umul64hi(x.v[1], (unsigned long long)(n - 1));
        if (t >= s) ++t;
        sh.s = (long long)s;
        sh.t = (long long)t;
        const unsigned int ps = S.at(0, 0u), pt = S.at(1, 0u);
        __stcg(S.code + s, code_of(0, 0u));
        __stcg(S.code + t, code_of(1, 0u));
        __stcg(S.qv + ps, (unsigned int)s);
        __stcg(S.qv + pt, (unsigned int)t);
        __stcg(S.ql + ps, 0u);
        __stcg(S.ql + pt, 0u);
        __stcg(S.qs + ps, 1ULL);
        __stcg(S.qs + pt, 1ULL);
        if (S.bits) {
            atomicOr(&S.bits[s >> 5], 1u << (s & 31));
            atomicOr(&S.bits[S.bw + (t >> 5)], 1u << (t & 31));
        }
        sh.qlen[0] = sh.qlen[1] = 1;
        sh.fbeg[0] = sh.fbeg[1] = 0;
        sh.fend[0] = sh.fend[1] = 1;
        sh.lbeg[0][0] = sh.lbeg[1][0] = 0;
        sh.lend[0][0] = sh.lend[1][0] = 1;
        sh.layer[0] = sh.layer[1] = 0;
        sh.fdeg[0] = (unsigned long long)(G.end(s) - G.begin(s));
        sh.fdeg[1] = (unsigned long long)(G.end(t) - G.begin(t));
        sh.status = 0;
        sh.scaled = 0;
        sh.err = 0;
        sh.ovf = 0;
        sh.e_scan = 0;
        sh.expanded = 0;
        sh.meet_count = 0;
        sh.new_count = 0;
        sh.meets = 0;
        sh.lmax = 0;
        sh.ldeg = 0;
        sh.chosen = -1;
        sh.pf_ok = 0;
        sh.X = (sh.fdeg[0] <= sh.fdeg[1]) ? 0 : 1;
        if (sh.fdeg[sh.X] == 0) {
            // the side expanded first has no edges (the smaller degree sum is
            // 0): its layer is empty, so the pair is disconnected; same result
            // as expanding that layer, without the layer's barriers
            sh.layer[sh.X] = 1;
            sh.expanded = 1;
            if (1u < (unsigned int)kMaxLayers) {
                sh.lbeg[sh.X][1] = 1;
                sh.lend[sh.X][1] = 1;
            }
            sh.status = 2;
        }
    }
    __syncthreads();

    // A2: balanced bidirectional BFS, one whole layer per step.  The side of
    // the next layer is chosen by thread 0 at the end of the previous layer;
    // the layer accumulators are cleared by thread 0 here, before the first
    // barrier of the layer (every thread read the previous layer's values
    // before that layer's closing barrier).
    while (sh.status == 0) {
        if (tid == 0) {
            sh.new_count = 0;
            sh.meet_count = 0;
            sh.meets = 0;
            sh.lmax = 0;
            sh.ldeg = 0;
        }
        const int X = sh.X, Y = 1 - X;
        const unsigned int nl = sh.layer[X] + 1;     // level of the new layer
        const unsigned int fb = sh.fbeg[X], fe = sh.fend[X];
        const unsigned int qbase = sh.qlen[X];       // queue position of the new layer's first vertex
        const unsigned int room = S.cap - sh.qlen[Y];   // positions this side may fill
        const unsigned int yb = sh.fbeg[Y], ye = sh.fend[Y];
        unsigned long long my_scan = 0;

        // probe pass (small-diameter samples): if the layer meets side Y's
        // frontier, its meeting counts are complete and it claims nothing.
        // A heavy layer of a persistent launch is posted for other CTAs to
        // help with, for the probe pass and for the expansion alike.
        const bool heavy = a.help && sh.fdeg[X] >= a.help_edges && fe - fb > (unsigned int)NT / 8u;
        bool probed_last = false;
        if (a.probe_log2 && S.bits && sh.fdeg[X] >= a.probe_edges && ye - yb <= (1u << (a.probe_log2 - 4))) {
            unsigned long long ps = 0;
            bool shared = false;
            if (heavy) {
                probe_ready<NT>(a.probe_log2, S, sh, Y, yb, ye);
                shared = help_layer<NT, OffT>(a, G, S, sh, 1, X, nl, fb, fe, qbase, room, yb, ye, ps);
            }
            if (!shared) ps = probe_layer<NT, OffT>(G, S, sh, a.probe_log2, X, fb, fe, yb, ye);
            if (*reinterpret_cast<volatile int *>(&sh.meets)) {
                probed_last = true;
                my_scan = ps;
            }
        }
        if (!probed_last && !(heavy && help_layer<NT, OffT>(a, G, S, sh, 0, X, nl, fb, fe, qbase, room, yb, ye,
                                                              my_scan))) {
            for (unsigned int cb = fb; cb < fe; cb += NT)
                my_scan += expand_chunk<NT, OffT>(a.spin_limit, G, S, sh, SmemAcc<NT>{sh}, X, nl, cb, fe, qbase, room,
                                                  yb, ye);
        }
        // The layer's outcome (final after the last chunk's barrier), read
        // alike by every thread: if the search goes on, every thread scales
        // its share of the new layer's counts now (keeping them <= 2^K,
        // rounding up so that they stay >= 1) while thread 0 books the layer,
        // and one barrier closes both.
        {
            const unsigned int ncount = *reinterpret_cast<volatile unsigned int *>(&sh.new_count);
            const unsigned int mcl = *reinterpret_cast<volatile unsigned int *>(&sh.meet_count);
            const unsigned long long lmaxl = *reinterpret_cast<volatile unsigned long long *>(&sh.lmax);
            const int ovfl = *reinterpret_cast<volatile int *>(&sh.ovf);
            const int shv = bitlen64(lmaxl) - a.K;
            if (!ovfl && ncount <= room - qbase && mcl == 0 && ncount > 0 && shv > 0 && !a.strict) {
                for (unsigned int i = qbase + tid; i < qbase + ncount; i += NT) {
                    unsigned long long *q = S.qs + S.at(X, i);
                    __stcg(q, ((ldcg(q) - 1ULL) >> shv) + 1ULL);
                }
            }
        }
        if (tid == 0) {
            sh.e_scan += my_scan;
            sh.expanded += fe - fb;
            sh.layer[X] = nl;
            unsigned int nc = sh.new_count;
            if (nc > room - qbase) {
                nc = room - qbase;
                sh.ovf = 1;
            }
            sh.qlen[X] = qbase + nc;
            if (nl < (unsigned int)kMaxLayers) {
                sh.lbeg[X][nl] = qbase;
                sh.lend[X][nl] = qbase + nc;
            }
            if (sh.ovf) {
                sh.status = 6;      // out of queue positions: clear and restart elsewhere
            } else if (sh.meet_count > 0) {
                sh.status = 1;
            } else if (nc == 0) {
                sh.status = 2;
            } else if (a.abandon && *reinterpret_cast<const volatile int *>(a.abandon)) {
                sh.status = 5;      // discarded sample: clear its state and leave
            } else {
                sh.fbeg[X] = qbase;
                sh.fend[X] = qbase + nc;
                sh.fdeg[X] = sh.ldeg;
                const int shv = bitlen64(sh.lmax) - a.K;
                if (shv > 0) {
                    sh.scaled = 1;
                    if (a.strict) sh.status = 3;
                }
                // the next layer: side with the smaller frontier degree sum (ties: s)
                if (sh.status == 0) sh.X = (sh.fdeg[0] <= sh.fdeg[1]) ? 0 : 1;
            }
        }
        __syncthreads();
    }

    // A3 + A4: choose the meeting vertex, walk back, count interior vertices
    if (tid == 0 && a.trace) t_bfs = global_ns();
    const int met = sh.status == 1;
    unsigned long long path_len = 0, walk_scan = 0;
    const int nbits = bitlen64((unsigned long long)(n - 1)) > 0 ? bitlen64((unsigned long long)(n - 1)) : 1;
    const int npass = (nbits + 7) / 8;
    if (met) {
        // The meeting set is the part of Y's last layer that X's last layer
        // reached: weight of w = sigma_Y(w) (qs) * sigma_X(w) (qm).
        const int X = sh.X, Y = 1 - X;
        const unsigned int mcnt = sh.meet_count;
        const bool in_smem = mcnt <= (unsigned int)kMeetCap;
        unsigned long long tlo = 0, thi = 0;
        if (mcnt <= 32u) {
            // small meeting set: warp 0 alone weighs the candidates, orders
            // them by id and picks the one whose prefix interval holds r
            if (tid < 32) {
                const int lane = tid;
                const bool have = (unsigned int)lane < mcnt;
                const unsigned int id = have ? sh.cand[lane] : 0xffffffffu;
                const unsigned int myp = have ? sh.cpos[lane] : 0u;
                unsigned long long lo = 0, hi = 0;
                if (have) {
                    const unsigned int ph = S.at(Y, myp);
                    const unsigned long long p = ldcg(S.qs + ph), q = ldcg(S.qm + ph);
                    lo = p * q;
                    hi = __umul64hi(p, q);
                }
                // exclusive prefix of the weights in ascending id order, and the total
                unsigned long long plo = 0, phi = 0, alo = 0, ahi = 0;
                for (int j = 0; j < 32; ++j) {
                    const unsigned int idj = __shfl_sync(0xffffffffu, id, j);
                    const unsigned long long ljo = __shfl_sync(0xffffffffu, lo, j);
                    const unsigned long long hjo = __shfl_sync(0xffffffffu, hi, j);
                    add128(alo, ahi, ljo, hjo);
                    if (idj < id) add128(plo, phi, ljo, hjo);
                }
                int pick = -1;
                if (mcnt == 1) {
                    pick = 0;
                } else {
                    unsigned long long rlo = 0, rhi = 0;
                    if (lane == 0) {
                        const U64x4 x = sample_draw(a.seed, a.tag, idx, 1);
                        const unsigned __int128 R = ((unsigned __int128)x.v[1] << 64) | x.v[0];
                        const unsigned __int128 T = ((unsigned __int128)ahi << 64) | alo;
                        const unsigned __int128 r = R % T;
                        rlo = (unsigned long long)r;
                        rhi = (unsigned long long)(r >> 64);
                    }
                    rlo = __shfl_sync(0xffffffffu, rlo, 0);
                    rhi = __shfl_sync(0xffffffffu, rhi, 0);
                    unsigned long long elo = plo, ehi = phi;
                    add128(elo, ehi, lo, hi);
                    const bool mine = have && !less128(rlo, rhi, plo, phi) && less128(rlo, rhi, elo, ehi);
                    const unsigned int m = __ballot_sync(0xffffffffu, mine);
                    pick = m ? __ffs(m) - 1 : -1;
                }
                if (lane == 0) {
                    sh.sig_lo = alo;
                    sh.sig_hi = ahi;
                    sh.chosen = pick >= 0 ? (long long)sh.cand[pick] : -1;
                    sh.pw = pick >= 0 ? sh.cpos[pick] : 0u;
                }
            }
            __syncthreads();
        } else {
            if (in_smem) {
                for (unsigned int i = tid; i < mcnt; i += NT) {
                    const unsigned int ph = S.at(Y, sh.cpos[i]);
                    const unsigned long long p = ldcg(S.qs + ph), q = ldcg(S.qm + ph);
                    const unsigned long long lo = p * q, hi = __umul64hi(p, q);
                    sh.wlo[i] = lo;
                    sh.whi[i] = hi;
                    add128(tlo, thi, lo, hi);
                }
            } else {
                for (unsigned int i = sh.fbeg[Y] + tid; i < sh.fend[Y]; i += NT) {
                    const unsigned int ph = S.at(Y, i);
                    const unsigned long long q = ldcg(S.qm + ph);
                    if (q == 0ULL) continue;
                    const unsigned long long p = ldcg(S.qs + ph);
                    add128(tlo, thi, p * q, __umul64hi(p, q));
                }
            }
            block_sum128<NT>(tlo, thi, sh);
            if (tid == 0) {
                sh.sig_lo = tlo;
                sh.sig_hi = thi;
                const U64x4 x = sample_draw(a.seed, a.tag, idx, 1);
                const unsigned __int128 R = ((unsigned __int128)x.v[1] << 64) | x.v[0];
                const unsigned __int128 T = ((unsigned __int128)thi << 64) | tlo;
                const unsigned __int128 r = R % T;
                sh.r_lo = (unsigned long long)r;
                sh.r_hi = (unsigned long long)(r >> 64);
                sh.chosen = -1;
            }
            __syncthreads();
            long long c;
            if (in_smem) {
                c = radix_choose<NT>(sh, npass, [&](auto &&add) {
                    for (unsigned int i = tid; i < mcnt; i += NT) add(sh.cand[i], sh.wlo[i], sh.whi[i]);
                });
            } else {
                const unsigned int yb = sh.fbeg[Y], ye = sh.fend[Y];
                c = radix_choose<NT>(sh, npass, [&](auto &&add) {
                    for (unsigned int i = yb + tid; i < ye; i += NT) {
                        const unsigned int ph = S.at(Y, i);
                        const unsigned long long q = ldcg(S.qm + ph);
                        if (q == 0ULL) continue;
                        const unsigned long long p = ldcg(S.qs + ph);
                        add(__ldcg(S.qv + ph), p * q, __umul64hi(p, q));
                    }
                });
            }
            if (tid == 0) {
                sh.chosen = c;
                const unsigned int cc = (c >= 0 && c < n) ? __ldcg(S.code + c) : 0u;
                sh.pw = pos_of(cc);
            }
            __syncthreads();
        }
        if (tid == 0) {
            // the chosen vertex must be in Y's last layer and reached by X
            const long long c = sh.chosen;
            bool ok = c >= 0 && c < n;
            if (ok) {
                const unsigned int cc = __ldcg(S.code + c);
                ok = cc == code_of(Y, sh.pw) && sh.pw >= sh.fbeg[Y] && sh.pw < sh.fend[Y] &&
                     ldcg(S.qm + S.at(Y, sh.pw)) != 0ULL;
            }
            if (!ok) {
                sh.chosen = -1;
                sh.err |= kErrSelect;
            }
        }
        __syncthreads();

        const long long w = sh.chosen;
        if (tid == 0 && a.trace) t_sel = global_ns();
        if (tid == 0) {
            sh.plen = 0;
            sh.pflushed = 0;
            if (w >= 0 && w != sh.s && w != sh.t) {
                sh.path[sh.plen++] = (unsigned int)w;
                ++path_len;
            }
        }
        // walk towards s (side 0), then towards t (side 1); draws 2, 3, ...
        // w's level: one past X's last expanded layer on side X, its queue
        // level on side Y
        unsigned long long k = 2;
        bool walk_ok = w >= 0;
        const unsigned int lw[2] = {X == 0 ? sh.layer[0] : (walk_ok ? __ldcg(S.ql + S.at(0, sh.pw)) : 0u),
                                    X == 1 ? sh.layer[1] : (walk_ok ? __ldcg(S.ql + S.at(1, sh.pw)) : 0u)};
        for (int Z = 0; Z < 2 && walk_ok; ++Z) {
            long long v = w;
            const long long src = Z == 0 ? sh.s : sh.t;
            unsigned int lz = lw[Z];     // level of v on side Z
            for (;;) {
                // Warp 0 alone takes every step from a vertex of degree <= 32
                // (lanes hold its neighbours) and every step whose predecessor
                // is the side's source, without block barriers; the CTA joins
                // for a step from a larger vertex.  Every step owns one draw
                // index, in path order.
                if (tid < 32) {
                    long long vv = v;
                    unsigned int ll = lz;
                    unsigned long long kk = k;
                    int state = 0;        // 0: a large step at vv, 1: source reached, 2: broken invariant
                    unsigned long long scan = 0;
                    // row of vv, when already known (each lane reads its
                    // candidate's row with its state, so the chosen
                    // predecessor's row comes with the choice)
                    long long bb = -1, be = -1;
                    for (;;) {
                        if (ll == 0) {
                            state = 1;
                            break;
                        }
                        const unsigned int tg = ll - 1;
                        if (ll == 1) {
                            vv = src;
                            ll = tg;
                            ++kk;
                            continue;
                        }
                        if (bb < 0) {
                            bb = G.begin(vv);
                            be = G.end(vv);
                        }
                        const long long dd = be - bb;
                        if (dd > 32) break;
                        const U64x4 xx = sample_draw(a.seed, a.tag, idx, kk);
                        ++kk;
                        long long u = -1, ub = -1, ue = -1;
                        unsigned long long wt = 0;
                        if (tid < dd) {
                            u = G.col(bb + tid);
                            ub = G.begin(u);
                            ue = G.end(u);
                            wt = pred_weight(S, Z, u, tg);
                        }
                        unsigned long long incl = wt;
#pragma unroll
                        for (int o = 1; o < 32; o <<= 1) {
                            const unsigned long long y = __shfl_up_sync(0xffffffffu, incl, o);
                            if (tid >= o) incl += y;
                        }
                        const unsigned long long total = __shfl_sync(0xffffffffu, incl, 31);
                        const unsigned long long ex = incl - wt;
                        const unsigned long long r = __umul64hi(xx.v[0], total);
                        const unsigned int m = __ballot_sync(0xffffffffu, wt > 0 && ex <= r && r < ex + wt);
                        scan += (unsigned long long)dd;
                        if (!m) {
                            state = 2;
                            break;
                        }
                        const int pick = __ffs(m) - 1;
                        vv = __shfl_sync(0xffffffffu, u, pick);
                        bb = __shfl_sync(0xffffffffu, ub, pick);
                        be = __shfl_sync(0xffffffffu, ue, pick);
                        ll = tg;
                        if (tid == 0) sh.path[sh.plen++] = (unsigned int)vv;
                        __syncwarp();
                        if (sh.plen >= (unsigned int)kPathCap) {
                            const unsigned int fe = sink_flush(sink, sh.path, sh.plen);
                            if (tid == 0) sh.err |= fe;
                            __syncwarp();
                            if (tid == 0) {
                                if (a.trace_path)
                                    for (unsigned int i = 0; i < sh.plen; ++i)
                                        if ((long long)(sh.pflushed + i) < a.trace_cap)
                                            a.trace_path[trace_i * a.trace_cap + sh.pflushed + i] = (int32_t)sh.path[i];
                                sh.pflushed += sh.plen;
                                sh.plen = 0;
                            }
                            __syncwarp();
                        }
                    }
                    if (tid == 0) {
                        sh.wv = vv;
                        sh.wl = ll;
                        sh.wk = kk;
                        sh.wstate = state;
                        walk_scan += scan;
                        path_len = sh.pflushed + sh.plen;
                    }
                }
                __syncthreads();
                v = sh.wv;
                lz = sh.wl;
                k = sh.wk;
                const int wstate = sh.wstate;
                __syncthreads();   // sh.w* are rewritten by the next warp phase
                if (wstate == 1) break;
                if (wstate == 2) {
                    if (tid == 0) sh.err |= kErrSelect;
                    walk_ok = false;
                    break;
                }
                const unsigned int target = lz - 1;      // level of the predecessors (>= 1 here)
                const unsigned int P = target;           // their layer index
                const unsigned long long draw = k++;
                {
                    const long long b = G.begin(v);
                    const long long d = G.end(v) - b;
                    const U64x4 x = sample_draw(a.seed, a.tag, idx, draw);
                    const unsigned int lsz = P < (unsigned int)kMaxLayers ? sh.lend[Z][P] - sh.lbeg[Z][P] : 0xffffffffu;
                    if (tid == 0) sh.next_v = -1;
                    if (d > 2 * NT && lsz <= (unsigned int)kMeetCap && (unsigned long long)lsz * 8ULL < (unsigned long long)d) {
                        // hub: test the predecessor layer's vertices for adjacency
                        if (tid == 0) sh.pcnt = 0;
                        __syncthreads();
                        const unsigned int lb = sh.lbeg[Z][P];
                        for (unsigned int i = tid; i < lsz; i += NT) {
                            const unsigned int ph = S.at(Z, lb + i);
                            const unsigned int u = __ldcg(S.qv + ph);
                            const long long bu = G.begin(u), du = G.end(u) - bu;
                            const bool isadj = du <= d ? contains(G.adj, bu, du, v) : contains(G.adj, b, d, u);
                            if (isadj) {
                                const unsigned int p = atomicAdd(&sh.pcnt, 1u);
                                sh.cand[p] = u;
                                sh.wlo[p] = ldcg(S.qs + ph);
                                sh.whi[p] = 0;
                            }
                        }
                        __syncthreads();
                        const unsigned int pc = sh.pcnt;
                        walk_scan += lsz;
                        unsigned long long part = 0;
                        for (unsigned int i = tid; i < pc; i += NT) part += sh.wlo[i];
                        const unsigned long long total = block_sum<NT>(part, sh);
                        if (pc == 1) {
                            if (tid == 0) sh.next_v = sh.cand[0];
                        } else if (pc > 1 && pc <= 32) {
                            warp_pick64<NT>(sh, pc, __umul64hi(x.v[0], total));
                        } else if (pc > 1) {
                            if (tid == 0) {
                                sh.r_lo = __umul64hi(x.v[0], total);
                                sh.r_hi = 0;
                            }
                            __syncthreads();
                            const long long c = radix_choose<NT>(sh, npass, [&](auto &&add) {
                                for (unsigned int i = tid; i < pc; i += NT) add(sh.cand[i], sh.wlo[i], 0ULL);
                            });
                            if (tid == 0) sh.next_v = c;
                        }
                        __syncthreads();
                    } else if (d <= NT) {
                        walk_scan += (unsigned long long)d;
                        __syncthreads();
                        long long u = -1;
                        unsigned long long wt = 0;
                        if (tid < d) {
                            u = G.col(b + tid);
                            wt = pred_weight(S, Z, u, target);
                        }
                        unsigned long long total;
                        const unsigned long long ex = block_excl_scan<NT>(wt, &total, sh);
                        const unsigned long long r = __umul64hi(x.v[0], total);
                        if (wt > 0 && ex <= r && r < ex + wt) sh.next_v = u;
                        __syncthreads();
                    } else {
                        // one pass over the adjacency collects the candidates
                        // (up to kMeetCap) with their weights; more than that
                        // falls back to a second, ordered pass
                        walk_scan += (unsigned long long)d;
                        if (tid == 0) sh.pcnt = 0;
                        __syncthreads();
                        unsigned long long part = 0;
                        for (long long j = tid; j < d; j += NT) {
                            const long long u = G.col(b + j);
                            const unsigned long long su = pred_weight(S, Z, u, target);
                            if (su) {
                                part += su;
                                const unsigned int p = atomicAdd(&sh.pcnt, 1u);
                                if (p < (unsigned int)kMeetCap) {
                                    sh.cand[p] = (unsigned int)u;
                                    sh.wlo[p] = su;
                                }
                            }
                        }
                        const unsigned long long total = block_sum<NT>(part, sh);
                        const unsigned long long r = __umul64hi(x.v[0], total);
                        const unsigned int pc = sh.pcnt;
                        if (pc <= (unsigned int)kMeetCap) {
                            if (pc == 1) {
                                if (tid == 0) sh.next_v = sh.cand[0];
                            } else if (pc <= 32) {
                                warp_pick64<NT>(sh, pc, r);
                            } else {
                                if (tid == 0) {
                                    sh.r_lo = r;
                                    sh.r_hi = 0;
                                }
                                __syncthreads();
                                const long long c = radix_choose<NT>(sh, npass, [&](auto &&add) {
                                    for (unsigned int i = tid; i < pc; i += NT) add(sh.cand[i], sh.wlo[i], 0ULL);
                                });
                                if (tid == 0) sh.next_v = c;
                            }
                            __syncthreads();
                        } else {
                        unsigned long long carry = 0;
                        if (tid == 0) sh.found = 0;
                        __syncthreads();
                        for (long long c0 = 0; c0 < d; c0 += NT) {
                            const long long j = c0 + tid;
                            long long u = -1;
                            unsigned long long wt = 0;
                            if (j < d) {
                                u = G.col(b + j);
                                wt = pred_weight(S, Z, u, target);
                            }
                            unsigned long long ctot;
                            const unsigned long long ex = carry + block_excl_scan<NT>(wt, &ctot, sh);
                            if (wt > 0 && ex <= r && r < ex + wt) {
                                sh.next_v = u;
                                sh.found = 1;
                            }
                            carry += ctot;
                            __syncthreads();
                            if (sh.found) break;
                        }
                        }
                    }
                    v = sh.next_v;
                    if (v < 0 || v >= n || pred_weight(S, Z, v, target) == 0ULL) {
                        // no predecessor found: an invariant is broken; record it, stop the walk
                        if (tid == 0) sh.err |= kErrSelect;
                        walk_ok = false;
                        __syncthreads();
                        break;
                    }
                    lz = target;
                }
                if (tid == 0) {
                    sh.path[sh.plen++] = (unsigned int)v;    // level >= 1: v is interior
                    ++path_len;
                }
                __syncthreads();   // sh.next_v is rewritten by the next step
                if (sh.plen >= (unsigned int)kPathCap - 1u) {
                    if (tid < 32) {
                        const unsigned int fe = sink_flush(sink, sh.path, sh.plen);
                        if (tid == 0) sh.err |= fe;
                        __syncwarp();
                        if (tid == 0) {
                            if (a.trace_path)
                                for (unsigned int i = 0; i < sh.plen; ++i)
                                    if ((long long)(sh.pflushed + i) < a.trace_cap)
                                        a.trace_path[trace_i * a.trace_cap + sh.pflushed + i] = (int32_t)sh.path[i];
                            sh.pflushed += sh.plen;
                            sh.plen = 0;
                        }
                    }
                    __syncthreads();
                }
            }
        }
        // the path's interior vertices still buffered go to the sink
        if (tid < 32) {
            const unsigned int cnt = sh.plen;
            const unsigned int fe = sink_flush(sink, sh.path, cnt);
            if (tid == 0) sh.err |= fe;
            if (a.trace_path)
                for (unsigned int i = tid; i < cnt; i += 32)
                    if ((long long)(sh.pflushed + i) < a.trace_cap)
                        a.trace_path[trace_i * a.trace_cap + sh.pflushed + i] = (int32_t)sh.path[i];
        }
        __syncthreads();
    }

    const bool done = sh.status != 6;
    // per-sample bookkeeping (thread 0); a sample that ran out of queue
    // positions is not counted here (it runs again on a larger slot)
    if (tid == 0 && done) {
        if (a.trace) {
            t_walk = global_ns();
            if (!met) t_sel = t_bfs;
        }
        ls.samples += 1;
        ls.connected += met ? 1 : 0;
        ls.e_scan += sh.e_scan;
        ls.expanded += sh.expanded;
        ls.touched += (unsigned long long)sh.qlen[0] + sh.qlen[1] + (met ? sh.meet_count : 0u);
        ls.interior += path_len;
        ls.walk_scan += walk_scan;
        ls.scaled += sh.scaled ? 1 : 0;
        if (sh.status == 3) sh.err |= kErrSigmaOverflow;
        if (a.trace) {
            TraceRec tr;
            tr.s = sh.s;
            tr.t = sh.t;
            tr.d = met ? (long long)sh.layer[0] + sh.layer[1] : -1;
            tr.sigma_lo = met ? sh.sig_lo : 0;
            tr.sigma_hi = met ? sh.sig_hi : 0;
            tr.meet_size = met ? sh.meet_count : 0;
            tr.chosen = met ? sh.chosen : -1;
            tr.e_scan = (long long)sh.e_scan;
            tr.n_interior = (long long)path_len;
            tr.scaled = sh.scaled;
            tr.overflow = sh.status == 3 ? 1 : 0;
            tr.ns = (long long)(t_walk - t_start);
            tr.phase_ns[0] = (long long)(t_bfs - t_start);
            tr.phase_ns[1] = (long long)(t_sel - t_bfs);
            tr.phase_ns[2] = (long long)(t_walk - t_sel);
            tr.phase_ns[3] = 0;
            a.trace[trace_i] = tr;
        }
    }
    if (tid == 0 && sh.err) atomicOr(&a.job->error, sh.err);

    // clear every code word, path count and meeting count this sample set,
    // restoring the all-zero invariant
    __syncthreads();
    if (sh.meet_count > 0) {
        const int Y = 1 - sh.X;
        for (unsigned int i = sh.fbeg[Y] + tid; i < sh.fend[Y]; i += NT) __stcg(S.qm + S.at(Y, i), 0ULL);
    }
    for (int side = 0; side < 2; ++side) {
        const unsigned int len = sh.qlen[side];
        for (unsigned int i0 = tid; i0 < len; i0 += 4 * NT) {
            unsigned int v[4];
            unsigned int ph[4];
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const unsigned int i = i0 + (unsigned int)j * NT;
                ph[j] = S.at(side, i);
                v[j] = i < len ? __ldcg(S.qv + ph[j]) : kNone;
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                if (v[j] == kNone) continue;
                __stcg(S.code + v[j], 0u);
                __stcg(S.qs + ph[j], 0ULL);
                // every set bit of this side's map belongs to a queued vertex of
                // this sample, so the whole word can go
                if (S.bits) __stcg(S.bits + (side ? S.bw : 0) + (v[j] >> 5), 0u);
            }
        }
    }
    __syncthreads();
    if (tid == 0 && a.trace && done) a.trace[trace_i].phase_ns[3] = (long long)(global_ns() - t_walk);
    return done;
}

// Runs sample `idx` in this CTA's slot; a sample that outgrows the slot runs
// again on a spill slot (queue capacity = n), taken and released under a
// lock word with a bounded wait.  One call site of run_sample, so that it is
// inlined once.
template <int NT, typename OffT>
__device__ void run_sample_any(const SampleLaunch &a, const GraphRef<OffT> &G, const Slot &mine, const SlotSet &spill,
                               bool use_bits, Smem<NT> &sh, unsigned long long idx, unsigned long long trace_i,
                               LocalStats &ls, const CountSink &sink)
{
    Slot S = mine;
    for (int attempt = 0;; ++attempt) {
        if (run_sample<NT, OffT>(a, G, S, sh, idx, trace_i, ls, sink)) break;
        if (threadIdx.x == 0) {
            if (attempt > 0) {
                atomicOr(&a.job->error, kErrScratch);      // a spill slot holds any sample: never expected
                sh.spill_k = -1;
            } else if (spill.count > 0 && spill.lock) {
                int got = -1;
                unsigned long long w = 0;
                for (;;) {
                    for (int k = 0; k < spill.count && got < 0; ++k)
                        if (atomicCAS(spill.lock + k, 0, 1) == 0) got = k;
                    if (got >= 0 || ++w > a.spin_limit) break;
                    __nanosleep(1024);
                }
                if (got < 0) atomicOr(&a.job->error, kErrTimeout);
                sh.spill_k = got;
                __threadfence();
            } else {
                atomicOr(&a.job->error, kErrScratch);
                sh.spill_k = -1;
            }
        }
        __syncthreads();
        if (attempt > 0 || sh.spill_k < 0) break;
        S = slot_of(spill, sh.spill_k, use_bits);
    }
    if (S.code != mine.code) {
        // release the spill slot once this CTA is done with it
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            atomicExch(spill.lock + sh.spill_k, 0);
        }
    }
    __syncthreads();
}

template <int NT, typename OffT>
__global__ void __launch_bounds__(NT, (2048 / NT / 2) > 0 ? (2048 / NT / 2) : 1) sample_kernel(SampleLaunch a)
{
    __shared__ Smem<NT> sh;
    __shared__ unsigned long long s_base;
    __shared__ unsigned long long s_count;
    const int tid = threadIdx.x;
    GraphRef<OffT> G{reinterpret_cast<const OffT *>(a.off), a.adj, (long long)a.n};
    const Slot slot = slot_of(a.slots, blockIdx.x, a.use_bits != 0);
    Job *job = a.job;

    if (tid == 0) {
        const unsigned long long base = *reinterpret_cast<volatile unsigned long long *>(&job->tau);
        const int stopped = a.use_stop ? *reinterpret_cast<volatile int *>(&job->stopped) : 0;
        unsigned long long count = stopped ? 0ULL : (unsigned long long)a.epoch_len;
        if (a.clip) {
            const unsigned long long room = a.clip > base ? a.clip - base : 0ULL;
            count = count < room ? count : room;
        }
        s_base = base;
        s_count = count;
    }
    __syncthreads();
    const unsigned long long base = s_base, count = s_count;

    LocalStats ls = {0, 0, 0, 0, 0, 0, 0, 0};
    for (;;) {
        if (tid == 0) sh.cur = atomicAdd(&job->work, 1ULL);
        __syncthreads();
        const unsigned long long i = sh.cur;
        if (i >= count) break;
        run_sample_any<NT, OffT>(a, G, slot, a.spill, a.use_bits != 0, sh, base + i, i, ls,
                                 CountSink{a.counts, a.log, a.log_len, a.log_cap});
    }

    if (tid == 0) {
        Counters *cs[2] = {&job->total, a.launch_ctr};
        for (int c = 0; c < 2; ++c) {
            if (!cs[c]) continue;
            atomicAdd(&cs[c]->samples, ls.samples);
            atomicAdd(&cs[c]->connected, ls.connected);
            atomicAdd(&cs[c]->e_scan, ls.e_scan);
            atomicAdd(&cs[c]->expanded, ls.expanded);
            atomicAdd(&cs[c]->touched, ls.touched);
            atomicAdd(&cs[c]->interior, ls.interior);
            atomicAdd(&cs[c]->walk_scan, ls.walk_scan);
            atomicAdd(&cs[c]->scaled, ls.scaled);
        }
        // the last CTA out publishes the new tau and re-arms the counters
        __threadfence();
        const unsigned int prev = atomicAdd(&job->done_ctas, 1u);
        if (prev == gridDim.x - 1) {
            __threadfence();
            *reinterpret_cast<volatile unsigned long long *>(&job->tau) = base + count;
            *reinterpret_cast<volatile unsigned long long *>(&job->work) = 0ULL;
            *reinterpret_cast<volatile unsigned int *>(&job->done_ctas) = 0u;
            __threadfence();
        }
    }
}

// ---- pipelined adaptive phase (one or many queries) -------------------------
//
// The paper's epoch framework (Section IV-A/B, Algorithm 2) lets every thread
// keep sampling across an epoch transition: samples are written to the state
// frame of their own epoch, and the stopping condition is checked on the
// aggregate of complete epochs only.  On one GPU the same idea becomes: a
// persistent launch hands out sample indices in order; sample i belongs to
// epoch e = i / E and logs its interior vertices in frame e mod F; the CTA
// that finishes the last sample of epoch e (which must be the next epoch in
// order) folds frame e into c~ and evaluates the stopping condition on exactly
// samples [0, (e+1) E), while every other CTA keeps sampling later epochs.  A
// frame is the epoch's log of interior vertices (at most VD - 2 per sample);
// folding it costs O(E * path length), not O(n).  A CTA may start a sample of
// epoch e only once epoch e - F has been folded (its frame is free); that
// wait is bounded.  Samples of epochs after the
// stopping epoch are discarded, so tau, c~ and the stop epoch are those of
// epoch-by-epoch sampling with the same E.

template <int NT>
struct PipeSmem {
    int take;                 // 1: this CTA has a sample to run
    long long epoch;          // its epoch
    unsigned long long idx;   // its sample index (relative)
    int try_check;
    int acquired;
    int go;                   // inner loop: fold the next epoch
    int again;                // after releasing the checker role: try to take it again
    long long chk_epoch;
    double mf[NT / 32], mg[NT / 32];
};

// Fold one epoch's log into c~ and evaluate the stopping functions (CTA-wide).
//
// The check needs max_x f(c~(x), L(x)) and max_x g(...).  Vertices with the
// same budgets (L_L, L_U) form a class; every step of f and g is a correctly
// rounded monotone operation, so for fixed budgets the computed f and g are
// non-decreasing in c~(x), and the maximum over a class is attained at the
// class's largest counter.  The fold keeps those per-class maxima current
// (counters only grow), so the check evaluates f and g once per class and
// obtains exactly the per-vertex maxima.  Returns error bits.
template <int NT>
__device__ unsigned int fold_and_check(const QueryDesc &P, uint32_t *counts, const uint32_t *log, unsigned int len,
                                       unsigned long long tau, PipeSmem<NT> &ps, double &Mf, double &Mg)
{
    unsigned int err = 0;
    for (unsigned int i = threadIdx.x; i < len; i += NT) {
        const unsigned int x = __ldcg(log + i);
        const unsigned int c = atomicAdd(&counts[x], 1u) + 1u;
        if (c == 0u) err |= kErrCounterOverflow;
        // the old maximum is consumed, so the update completes before the barrier
        const unsigned int before = atomicMax(&P.cmax[__ldg(P.cls + x)], c);
        if (before == 0xffffffffu) err |= kErrCounterOverflow;
    }
    __syncthreads();
    const StopConsts k = stop_consts(tau, P.omega);
    double mf = 0.0, mg = 0.0;
    for (int cl = threadIdx.x; cl < P.nclass; cl += NT) {
        double f, g;
        stop_fg(k, __ldcg(P.cmax + cl), __ldg(P.Ltab + cl), f, g);
        mf = fmax_exact(mf, f);
        mg = fmax_exact(mg, g);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mf = fmax_exact(mf, __shfl_xor_sync(0xffffffffu, mf, o));
        mg = fmax_exact(mg, __shfl_xor_sync(0xffffffffu, mg, o));
    }
    if ((threadIdx.x & 31) == 0) {
        ps.mf[threadIdx.x >> 5] = mf;
        ps.mg[threadIdx.x >> 5] = mg;
    }
    __syncthreads();
    Mf = 0.0;
    Mg = 0.0;
#pragma unroll
    for (int i = 0; i < NT / 32; ++i) {
        Mf = fmax_exact(Mf, ps.mf[i]);
        Mg = fmax_exact(Mg, ps.mg[i]);
    }
    __syncthreads();
    return err;
}

// Sets up a query's pipeline: base = current tau, R samples up to ceil(omega).
// One warp zeroes the state in place, then lane 0 sets its fields.
__global__ void pipe_begin_kernel(PipeState *ps, const Job *job, unsigned long long clip, long long E)
{
    if (blockIdx.x != 0 || threadIdx.x >= 32) return;
    unsigned int *w = reinterpret_cast<unsigned int *>(ps);
    for (size_t i = threadIdx.x; i < sizeof(PipeState) / 4; i += 32) w[i] = 0u;
    __syncwarp();
    if (threadIdx.x == 0) {
        ps->base = job->tau;
        ps->R = clip > ps->base ? clip - ps->base : 0ULL;
        ps->nE = (long long)((ps->R + (unsigned long long)E - 1) / (unsigned long long)E);
    }
}

__device__ __forceinline__ unsigned long long epoch_size(const PipeState *st, long long E, long long e)
{
    const unsigned long long lo = (unsigned long long)e * (unsigned long long)E;
    const unsigned long long R = st->R;
    return R - lo < (unsigned long long)E ? R - lo : (unsigned long long)E;
}

// One persistent launch over the queries of a batch (one query for
// kadabra_run_pipelined).  A CTA repeatedly takes the next sample index of
// some running query (round robin, skipping queries whose epoch logs are all
// in use), runs the sample in its slot, and, if that sample completed the
// query's oldest unchecked epoch, folds and checks that query's complete
// epochs in order.  The launch ends when every query has stopped or reached
// ceil(omega), or once `budget` samples have been handed out; the pipeline
// state persists, so the next launch continues where this one ended.
// Epoch frames a pipelined query may fill ahead of its oldest unchecked
// epoch.  While its stop is far, all F.  Modelling f and g as shrinking like
// 1/sqrt(tau) (their slowest regime: near the stop they fall faster, so the
// prediction is late and the narrowing mild), after the last check (tau
// samples, maxima m of f and g) the stop is expected near tau * (m / eps)^2
// samples: once that is within the frames,
// samples are handed out only up to the predicted stop epoch and one more,
// so that fewer samples are discarded and CTAs without one help heavy layers.
// A late stop only delays later hand-outs: results never depend on it.
__device__ __forceinline__ long long lookahead(const QueryDesc *Q, volatile PipeState *vst, volatile Job *vjob)
{
    if (!Q->lookahead || Q->tag == 0) return Q->F;
    if (vst->next_check < 2) return Q->F;      // no trend yet
    const double m = fmax(vjob->last_maxf, vjob->last_maxg);
    const double r = m / Q->eps;
    if (!(r >= 1.0) || !(r < 4.0)) return Q->F;
    const double ahead = (double)vjob->tau * (r * r - 1.0) / (double)Q->E;    // epochs to the predicted stop
    const long long f = (long long)ceil(ahead) + 1;
    return f < (long long)Q->F ? f : (long long)Q->F;
}

// Lane 0 of warp 0: takes a chunk of a request on the help board, if any,
// and copies the request's layer into sh.hl.  Returns whether it took one.
template <int NT>
__device__ __forceinline__ bool board_take(const BatchLaunch &B, Smem<NT> &sh)
{
    if (!B.help || *reinterpret_cast<volatile unsigned int *>(board_open(B.help)) == 0u) return false;
    HelpReq *board = board_req(B.help);
    for (int i = 0; i < kHelpSlots; ++i) {
        const int c = take_chunk(board + i);
        if (c < 0) continue;
        // the chunk belongs to the layer the request holds now, and the
        // request cannot be reused before this chunk is done
        volatile HelpReq *V = board + i;
        sh.help_k = i;
        sh.help_c = c;
        sh.hl.code = V->code;
        sh.hl.qv = V->qv;
        sh.hl.ql = V->ql;
        sh.hl.qs = V->qs;
        sh.hl.qm = V->qm;
        sh.hl.bits = V->bits;
        sh.hl.bw = V->bw;
        sh.hl.n = V->n;
        sh.hl.off = V->off;
        sh.hl.adj = V->adj;
        sh.hl.cap = V->cap;
        sh.hl.X = V->X;
        sh.hl.nl = V->nl;
        sh.hl.fb = V->fb;
        sh.hl.fe = V->fe;
        sh.hl.qbase = V->qbase;
        sh.hl.room = V->room;
        sh.hl.yb = V->yb;
        sh.hl.ye = V->ye;
        sh.hl.cv = V->cv;
        sh.hl.mode = V->mode;
        sh.hl.log2b = V->log2b;
        sh.hl.id = ((unsigned int)i << 16) | (unsigned int)((V->ticket >> 48) & 0xffffULL);
        return true;
    }
    return false;
}

template <int NT, typename OffT>
__global__ void __launch_bounds__(NT, (2048 / NT / 2) > 0 ? (2048 / NT / 2) : 1) batch_kernel(BatchLaunch B)
{
    __shared__ Smem<NT> sh;
    __shared__ PipeSmem<NT> pm;
    __shared__ QueryDesc qd;
    __shared__ SampleLaunch sa;
    __shared__ int s_qi;
    const int tid = threadIdx.x;
    volatile BatchState *vbs = B.bs;
    if (tid == 0) {
        sh.pf_ok = 0;       // the probe bitmap holds nothing yet
        // one query: its descriptor stays in shared memory for the whole launch
        if (B.nq == 1) qd = B.queries[0];
    }
    __syncthreads();

    for (;;) {
        // Warp 0 picks the next sample: its lanes read the state of 32
        // queries at a time and the first eligible one in scan order (round
        // robin from a per-pick ticket, or array order) is tried.
        // Between two samples a CTA first helps expand a layer another CTA
        // posted (a heavy layer of its sample), one chunk at a time.
        if (tid < 32) {
            const int lane = tid;
            int take = 0;
            bool stop_launch = false;
            int helping = 0;
            if (lane == 0) {
                pm.take = 0;
                s_qi = -1;
                sh.help_k = -1;
                if (board_take<NT>(B, sh)) helping = 1;
                if (!helping) {
                    stop_launch = vbs->abort != 0;
                    if (!stop_launch && B.budget && atomicAdd(&B.bs->taken, 0ULL) >= B.budget) stop_launch = true;
                }
            }
            helping = __shfl_sync(0xffffffffu, helping, 0);
            if (helping) stop_launch = true;     // skip the pick below
            stop_launch = __shfl_sync(0xffffffffu, stop_launch ? 1 : 0, 0) != 0;
            if (!stop_launch) {
                unsigned int start = 0;
                if (B.policy == 0 && B.nq > 1 && lane == 0) start = atomicAdd(&B.bs->ticket, 1u) % (unsigned int)B.nq;
                start = __shfl_sync(0xffffffffu, start, 0);
                unsigned long long polls = 0;
                for (;;) {
                    bool any_running = false;
                    for (int base = 0; base < B.nq && !take; base += 32) {
                        const int k = base + lane;
                        int qi = -1;
                        bool running = false, eligible = false;
                        if (k < B.nq) {
                            qi = (int)((start + (unsigned int)k) % (unsigned int)B.nq);
                            const QueryDesc *Q = B.nq == 1 ? &qd : B.queries + qi;
                            volatile PipeState *vst = Q->ps;
                            volatile Job *vjob = Q->job;
                            if (!vjob->stopped && !vst->abort) {
                                const unsigned long long nx = vst->next_idx;
                                if (nx < vst->R) {
                                    running = true;
                                    eligible = (long long)(nx / (unsigned long long)Q->E) <
                                               vst->next_check + lookahead(Q, vst, vjob);
                                }
                            }
                        }
                        any_running |= __any_sync(0xffffffffu, running);
                        unsigned int mask = __ballot_sync(0xffffffffu, eligible);
                        while (mask && !take) {
                            const int leader = __ffs(mask) - 1;
                            int got = 0;
                            if (lane == leader) {
                                const QueryDesc *Q = B.nq == 1 ? &qd : B.queries + qi;
                                PipeState *st = Q->ps;
                                volatile PipeState *vst = st;
                                volatile Job *vjob = Q->job;
                                const unsigned long long R = vst->R;
                                const unsigned long long i = atomicAdd(&st->next_idx, 1ULL);
                                if (i < R) {
                                    const long long E = Q->E;
                                    const int F = Q->F;
                                    const long long e = (long long)(i / (unsigned long long)E);
                                    // rare: another CTA took the indices in between; wait (bounded) for the log
                                    unsigned long long w = 0;
                                    bool ok = true;
                                    while (e >= vst->next_check + F) {
                                        if (vjob->stopped || vst->abort) {
                                            ok = false;
                                            break;
                                        }
                                        if (++w > B.spin_limit) {
                                            atomicOr(&Q->job->error, kErrTimeout);
                                            vst->abort = 1;
                                            ok = false;
                                            break;
                                        }
                                        __nanosleep(256);
                                    }
                                    __threadfence();
                                    if (ok) {
                                        got = 1;
                                        pm.epoch = e;
                                        pm.idx = i;
                                        s_qi = qi;
                                    }
                                }
                            }
                            take = __shfl_sync(0xffffffffu, got, leader);
                            mask &= ~(1u << leader);
                        }
                    }
                    if (take || !any_running) break;
                    // every running query waits for an epoch check: help with a
                    // posted heavy layer meanwhile, else back off (bounded)
                    int helped = 0;
                    if (lane == 0) helped = board_take<NT>(B, sh) ? 1 : 0;
                    if (__shfl_sync(0xffffffffu, helped, 0)) break;
                    if (++polls > B.spin_limit) {
                        if (lane == 0) {
                            atomicOr(&B.bs->abort, 1u);
                            for (int k = 0; k < B.nq; ++k) atomicOr(&B.queries[k].job->error, kErrTimeout);
                        }
                        break;
                    }
                    __nanosleep(512);
                }
                if (lane == 0 && take) {
                    pm.take = 1;
                    if (B.budget) atomicAdd(&B.bs->taken, 1ULL);
                }
            }
            __syncwarp();
            if (lane == 0 && take) {
                if (B.nq > 1) qd = B.queries[s_qi];
                SampleLaunch t{};
                t.n = qd.n;
                t.off = qd.off;
                t.adj = qd.adj;
                t.job = qd.job;
                t.seed = qd.seed;
                t.tag = qd.tag;
                t.K = qd.K;
                t.strict = qd.strict;
                // a sample still running when its query stops belongs to an
                // epoch after the stopping one and is discarded: end it early
                t.abandon = qd.tag != 0 ? &qd.job->stopped : nullptr;
                t.use_bits = qd.use_bits;
                t.spin_limit = B.spin_limit;
                t.help = B.help;
                t.help_edges = B.help_edges;
                t.probe_log2 = qd.use_bits ? B.probe_log2 : 0;
                t.probe_edges = B.probe_edges;
                sa = t;
            }
        }
        __syncthreads();
        if (sh.help_k >= 0) {
            HelpReq *R = board_req(B.help) + sh.help_k;
            Slot S2;
            S2.code = sh.hl.code;
            S2.qv = sh.hl.qv;
            S2.ql = sh.hl.ql;
            S2.qs = sh.hl.qs;
            S2.qm = sh.hl.qm;
            S2.bits = sh.hl.bits;
            S2.bw = sh.hl.bw;
            S2.cap = sh.hl.cap;
            const GraphRef<OffT> G2{reinterpret_cast<const OffT *>(sh.hl.off), sh.hl.adj, sh.hl.n};
            const unsigned int cb = sh.hl.fb + (unsigned int)sh.help_c * sh.hl.cv;
            unsigned long long sc;
            if (sh.hl.mode) {
                // probe chunk: this CTA's bitmap gets the request's frontier
                // (between two samples the bitmap is free; the next sample of
                // this CTA builds its own)
                if (!(sh.pf_ok == 2 && sh.pf_req == sh.hl.id)) {
                    probe_build<NT>(sh.hl.log2b, S2, 1 - (int)sh.hl.X, sh.hl.yb, sh.hl.ye);
                    if (tid == 0) {
                        sh.pf_ok = 2;
                        sh.pf_req = sh.hl.id;
                    }
                }
                sc = probe_chunk<NT, OffT>(G2, S2, sh, ReqAcc{R}, sh.hl.log2b, (int)sh.hl.X, cb,
                                           min(cb + sh.hl.cv, sh.hl.fe), sh.hl.yb, sh.hl.ye);
            } else {
                sc = expand_chunk<NT, OffT>(B.spin_limit, G2, S2, sh, ReqAcc{R}, (int)sh.hl.X, sh.hl.nl, cb,
                                            min(cb + sh.hl.cv, sh.hl.fe), sh.hl.qbase, sh.hl.room, sh.hl.yb,
                                            sh.hl.ye);
            }
            if (tid == 0) {
                atomicAdd(&R->scan, sc);
                __threadfence();
                atomicAdd(&R->done, 1u);
            }
            __syncthreads();
            continue;
        }
        if (!pm.take) break;
        const long long e = pm.epoch;
        const int f = (int)(e % qd.F);
        PipeState *st = qd.ps;
        volatile PipeState *vst = st;
        volatile Job *vjob = qd.job;
        Job *job = qd.job;
        GraphRef<OffT> G{reinterpret_cast<const OffT *>(qd.off), qd.adj, qd.n};
        LocalStats ls = {0, 0, 0, 0, 0, 0, 0, 0};
        run_sample_any<NT, OffT>(sa, G, slot_of(B.slots, blockIdx.x, qd.use_bits != 0), B.spill, qd.use_bits != 0, sh,
                                 st->base + pm.idx, pm.idx, ls,
                                 qd.tag == 0 ? CountSink{qd.counts, nullptr, nullptr, 0u}
                                             : CountSink{nullptr, qd.logs + (size_t)f * qd.log_cap, &st->log_len[f],
                                                         qd.log_cap});
        if (tid == 0) {
            Counters *cs[2] = {qd.tag != 0 ? &st->fc[f] : &job->total, qd.launch_ctr};
            for (int c = 0; c < 2; ++c) {
                if (!cs[c]) continue;
                atomicAdd(&cs[c]->samples, ls.samples);
                atomicAdd(&cs[c]->connected, ls.connected);
                atomicAdd(&cs[c]->e_scan, ls.e_scan);
                atomicAdd(&cs[c]->expanded, ls.expanded);
                atomicAdd(&cs[c]->touched, ls.touched);
                atomicAdd(&cs[c]->interior, ls.interior);
                atomicAdd(&cs[c]->walk_scan, ls.walk_scan);
                atomicAdd(&cs[c]->scaled, ls.scaled);
            }
            __threadfence();    // this sample's log entries before its completion
            const unsigned int d = atomicAdd(&st->done[f], 1u) + 1u;
            pm.try_check = (qd.tag != 0 && d == epoch_size(st, qd.E, e)) ? 1 : 0;
        }
        __syncthreads();
        if (!pm.try_check) continue;
        // this CTA completed an epoch of the query: fold and check its complete epochs in order
        const long long nE = st->nE;
        for (;;) {
            if (tid == 0) pm.acquired = atomicCAS(&st->checker, 0, 1) == 0;
            __syncthreads();
            if (!pm.acquired) break;
            for (;;) {
                if (tid == 0) {
                    const long long ce = vst->next_check;
                    pm.go = ce < nE && !vjob->stopped && vst->done[ce % qd.F] == epoch_size(st, qd.E, ce);
                    pm.chk_epoch = ce;
                    __threadfence();
                }
                __syncthreads();
                if (!pm.go) break;
                const long long ce = pm.chk_epoch;
                const unsigned long long tau = st->base + (unsigned long long)ce * (unsigned long long)qd.E +
                                               epoch_size(st, qd.E, ce);
                double Mf, Mg;
                const int cf = (int)(ce % qd.F);
                const unsigned int llen = vst->log_len[cf];
                unsigned int ferr = 0;
                if (llen > qd.log_cap) {
                    ferr = kErrLogOverflow;
                    Mf = Mg = 0.0;
                } else {
                    ferr = fold_and_check<NT>(qd, qd.counts, qd.logs + (size_t)cf * qd.log_cap, llen, tau, pm, Mf, Mg);
                }
                if (ferr) {
                    atomicOr(&job->error, ferr);
                    if (tid == 0) vst->abort = 1;
                    __syncthreads();
                    break;
                }
                if (tid == 0) {
                    const int stop = ((double)tau >= qd.omega) || (Mf < qd.eps && Mg < qd.eps);
                    job->tau = tau;
                    job->last_maxf = Mf;
                    job->last_maxg = Mg;
                    if (stop) {
                        job->stop_ns = global_ns();
                        job->stop_epoch = job->epoch;
                        job->stopped = 1;
                    }
                    job->epoch += 1;
                    // the checked epoch's counters join the query's totals
                    volatile Counters *fc = &st->fc[cf];
                    job->total.samples += fc->samples;
                    job->total.connected += fc->connected;
                    job->total.e_scan += fc->e_scan;
                    job->total.expanded += fc->expanded;
                    job->total.touched += fc->touched;
                    job->total.interior += fc->interior;
                    job->total.walk_scan += fc->walk_scan;
                    job->total.scaled += fc->scaled;
                    fc->samples = fc->connected = fc->e_scan = fc->expanded = 0;
                    fc->touched = fc->interior = fc->walk_scan = fc->scaled = 0;
                    st->done[cf] = 0u;
                    st->log_len[cf] = 0u;
                    __threadfence();
                    st->next_check = ce + 1;     // frees the log for epoch ce + F
                    __threadfence();
                }
                __syncthreads();
            }
            // release, then look again: an epoch completed while this CTA held
            // the checker role is picked up here
            if (tid == 0) {
                __threadfence();
                atomicExch(&st->checker, 0);
                __threadfence();
                const long long ce = vst->next_check;
                pm.again = ce < nE && !vjob->stopped && vst->done[ce % qd.F] == epoch_size(st, qd.E, ce);
            }
            __syncthreads();
            if (!pm.again) break;
        }
    }
}

// cmax[class] = max c~ over the class's vertices (cmax zeroed beforehand)
__global__ void class_max_kernel(long long n, const uint32_t *counts, const uint32_t *cls, unsigned int *cmax)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        const unsigned int c = __ldg(counts + x);
        if (c) atomicMax(&cmax[__ldg(cls + x)], c);
    }
}

// adj[e] = (col[e], degree of col[e]) for every adjacency entry
template <typename OffT>
__global__ void degree_kernel(long long n, const OffT *off, uint32_t *deg)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long v = (long long)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        deg[v] = (uint32_t)((long long)__ldg(off + v + 1) - (long long)__ldg(off + v));
}

// adj[e] = (col[e], deg[col[e]]).  col may be page-locked host memory read in
// place over the host link: plain loads (no read-only path), kAdjPer
// independent entries per thread in flight to cover the link's latency.
constexpr int kAdjPer = 8;
__global__ void build_adj_kernel(long long nnz, const uint32_t *deg, const int32_t *col, uint2 *adj)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (; e + (long long)(kAdjPer - 1) * stride < nnz; e += (long long)kAdjPer * stride) {
        int32_t w[kAdjPer];
#pragma unroll
        for (int j = 0; j < kAdjPer; ++j) w[j] = col[e + (long long)j * stride];
        uint32_t d[kAdjPer];
#pragma unroll
        for (int j = 0; j < kAdjPer; ++j) d[j] = __ldg(deg + w[j]);
#pragma unroll
        for (int j = 0; j < kAdjPer; ++j) adj[e + (long long)j * stride] = make_uint2((unsigned int)w[j], d[j]);
    }
    for (; e < nnz; e += stride) {
        const int32_t w = col[e];
        adj[e] = make_uint2((unsigned int)w, __ldg(deg + w));
    }
}

// dynamic shared memory of a launch: the probe bitmap, if any
inline size_t probe_bytes(int log2b) { return log2b ? (size_t)1 << (log2b - 3) : 0; }

template <int NT>
cudaError_t launch_nt(const SampleLaunch &a, cudaStream_t st)
{
    const size_t dyn = probe_bytes(a.probe_log2);
    if (a.off64)
        sample_kernel<NT, long long><<<a.grid, NT, dyn, st>>>(a);
    else
        sample_kernel<NT, int><<<a.grid, NT, dyn, st>>>(a);
    return cudaGetLastError();
}

template <int NT>
cudaError_t occupancy_nt(int off64, int *ctas)
{
    if (off64) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, sample_kernel<NT, long long>, NT, 0);
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, sample_kernel<NT, int>, NT, 0);
}

}  // namespace

cudaError_t launch_sample(const SampleLaunch &a, cudaStream_t st)
{
    if (a.grid <= 0) return cudaSuccess;
    switch (a.threads) {
    case 128: return launch_nt<128>(a, st);
    case 256: return launch_nt<256>(a, st);
    case 512: return launch_nt<512>(a, st);
    case 1024: return launch_nt<1024>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_build_adj(int64_t n, int64_t nnz, const void *off, int off64, const int32_t *col, uint2 *adj,
                             uint32_t *deg_tmp, cudaStream_t st)
{
    if (nnz <= 0) return cudaSuccess;
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long vgrid = (n + 255) / 256 < (long long)sms * 8 ? (n + 255) / 256 : (long long)sms * 8;
    if (off64)
        degree_kernel<long long><<<(int)vgrid, 256, 0, st>>>((long long)n, static_cast<const long long *>(off), deg_tmp);
    else
        degree_kernel<int><<<(int)vgrid, 256, 0, st>>>((long long)n, static_cast<const int *>(off), deg_tmp);
    const long long want = (nnz + 255) / 256;
    const int grid = (int)(want < (long long)sms * 8 ? want : (long long)sms * 8);
    build_adj_kernel<<<grid, 256, 0, st>>>((long long)nnz, deg_tmp, col, adj);
    return cudaGetLastError();
}

template <int NT>
cudaError_t launch_batch_nt(const BatchLaunch &a, cudaStream_t st)
{
    const size_t dyn = probe_bytes(a.probe_log2);
    if (a.off64)
        batch_kernel<NT, long long><<<a.grid, NT, dyn, st>>>(a);
    else
        batch_kernel<NT, int><<<a.grid, NT, dyn, st>>>(a);
    return cudaGetLastError();
}

// Largest probe bitmap (log2 of its bits, 0 if none) that keeps `per_sm` CTAs
// of both kernels resident, and the kernels' dynamic shared memory limit
// raised to it.
template <int NT, typename OffT>
cudaError_t probe_prepare_nt(int per_sm, int *log2b)
{
    size_t a1 = 0, a2 = 0;
    cudaError_t e = cudaOccupancyAvailableDynamicSMemPerBlock(&a1, sample_kernel<NT, OffT>, per_sm, NT);
    if (e == cudaSuccess) e = cudaOccupancyAvailableDynamicSMemPerBlock(&a2, batch_kernel<NT, OffT>, per_sm, NT);
    if (e != cudaSuccess) return e;
    const size_t avail = a1 < a2 ? a1 : a2;
    int lb = kProbeMaxLog2;
    while (lb >= kProbeMinLog2 && probe_bytes(lb) > avail) --lb;
    if (lb < kProbeMinLog2) {
        *log2b = 0;
        return cudaSuccess;
    }
    const int bytes = (int)probe_bytes(lb);
    e = cudaFuncSetAttribute(sample_kernel<NT, OffT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(batch_kernel<NT, OffT>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    *log2b = e == cudaSuccess ? lb : 0;
    return e;
}

template <int NT>
cudaError_t probe_prepare_t(int off64, int per_sm, int *log2b)
{
    return off64 ? probe_prepare_nt<NT, long long>(per_sm, log2b) : probe_prepare_nt<NT, int>(per_sm, log2b);
}

cudaError_t launch_batch(const BatchLaunch &a, cudaStream_t st)
{
    if (a.grid <= 0 || a.nq <= 0) return cudaSuccess;
    switch (a.threads) {
    case 128: return launch_batch_nt<128>(a, st);
    case 256: return launch_batch_nt<256>(a, st);
    case 512: return launch_batch_nt<512>(a, st);
    case 1024: return launch_batch_nt<1024>(a, st);
    default: return cudaErrorInvalidValue;
    }
}

size_t help_board_bytes() { return 256 + sizeof(HelpReq) * (size_t)kHelpSlots; }

cudaError_t launch_pipe_begin(PipeState *ps, const Job *job, unsigned long long clip, long long E, cudaStream_t st)
{
    pipe_begin_kernel<<<1, 32, 0, st>>>(ps, job, clip, E);
    return cudaGetLastError();
}

cudaError_t launch_class_max(int64_t n, const uint32_t *counts, const uint32_t *cls, unsigned int *cmax,
                             cudaStream_t st)
{
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const long long want = (n + 255) / 256;
    const int grid = (int)(want < (long long)sms * 8 ? want : (long long)sms * 8);
    class_max_kernel<<<grid > 0 ? grid : 1, 256, 0, st>>>((long long)n, counts, cls, cmax);
    return cudaGetLastError();
}

cudaError_t probe_prepare(int threads, int off64, int ctas_per_sm, int *log2_bits)
{
    *log2_bits = 0;
    if (ctas_per_sm < 1) ctas_per_sm = 1;
    switch (threads) {
    case 128: return probe_prepare_t<128>(off64, ctas_per_sm, log2_bits);
    case 256: return probe_prepare_t<256>(off64, ctas_per_sm, log2_bits);
    case 512: return probe_prepare_t<512>(off64, ctas_per_sm, log2_bits);
    case 1024: return probe_prepare_t<1024>(off64, ctas_per_sm, log2_bits);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t sample_occupancy(int threads, int off64, int *ctas_per_sm)
{
    switch (threads) {
    case 128: return occupancy_nt<128>(off64, ctas_per_sm);
    case 256: return occupancy_nt<256>(off64, ctas_per_sm);
    case 512: return occupancy_nt<512>(off64, ctas_per_sm);
    case 1024: return occupancy_nt<1024>(off64, ctas_per_sm);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace kadabra
