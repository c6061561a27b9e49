// Internal types shared by the host side (kadabra_api.cpp) and the kernels.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

struct kadabra_graph;

namespace kadabra {

// Sampling scratch of a set of slots, one in-flight sample each.  Per slot:
//   code[stride]  one word per vertex: 0 = not reached; else bit 31 = the side
//                 that reached it (0: s, 1: t) and bits 0..30 = its queue
//                 position + 1, or all ones while the claim that reached it is
//                 being published.  Zero at rest.
//   cap queue positions shared by the two sides (s from the front, t from
//   the back; the balls are disjoint until they meet), in four arrays:
//     qv  vertex id,   ql  BFS level (distance from the side's source),
//     qs  exact path count from the side's source, an exact uint64: a
//         layer's counts are kept at most 2^K with K <= 63 - bitlen(max
//         degree), so a count of the next layer stays below 2^63;
//     qm  for vertices of the other side's last layer: their path count from
//         the expanding side (the meeting vertices' second factor).
//     qs and qm are zero at rest.
//   bits (optional): two reached-bit maps of ceil(stride / 32) words each.
// A sample clears what it set before the slot takes its next sample, so no
// O(n) reset is needed.  A slot with cap < stride serves samples whose two
// balls hold at most cap vertices; a sample that outgrows it is cleared and
// re-run on a spill slot (cap = stride), so results never depend on cap.
struct SlotSet {
    uint32_t *code = nullptr;
    uint32_t *qv = nullptr;
    uint32_t *ql = nullptr;
    unsigned long long *qs = nullptr;
    unsigned long long *qm = nullptr;
    uint32_t *bits = nullptr;
    long long stride = 0;      // largest n the slots serve
    long long cap = 0;         // queue positions per slot (2 <= cap <= stride)
    int count = 0;             // slots
    int *lock = nullptr;       // spill sets: one word per slot, 0 = free
};

// words of one side's reached-bit map for n vertices
inline __host__ __device__ long long bit_words(long long n) { return (n + 31) / 32; }
// The reached-bit maps pay for their upkeep (one bit set per reached vertex)
// only when the last BFS layer is a large share of a sample, i.e. on graphs
// of small diameter; queries whose vertex-diameter bound exceeds this leave
// them alone.
constexpr long long kBitsMaxVD = 64;

// Counters a launch accumulates (one atomicAdd per CTA at exit).
struct Counters {
    unsigned long long samples, connected, e_scan, expanded, touched, interior, walk_scan, scaled;
};

// Device-resident state of one sample stream (adaptive, calibration, trace).
struct Job {
    unsigned long long tau;        // samples already taken by this stream
    unsigned long long work;       // next sample offset inside the running launch (64-bit: every
                                   // CTA takes one offset past the end, so it reaches count + grid)
    unsigned int done_ctas;        // CTAs that finished the running launch
    int stopped;                   // stop flag (adaptive stream)
    long long epoch;               // checks run so far
    long long stop_epoch;          // check that stopped, -1 if none
    unsigned long long maxf_bits;  // running maxima of the check in flight
    unsigned long long maxg_bits;
    unsigned int check_done;       // CTAs that finished the running check
    unsigned int error;            // sticky error bits (kErr*)
    double last_maxf, last_maxg;   // maxima of the last completed check
    unsigned long long stop_ns;    // device global timer when the stop was decided (0: not stopped)
    Counters total;                // since the query started (reset with the query)
};

constexpr int kLaunchLog = 256;    // sampling launches remembered per query

enum : unsigned int {
    kErrSigmaOverflow = 1u,    // strict mode: a layer's path count exceeded 2^K
    kErrAddOverflow = 2u,      // a 64-bit path-count add wrapped (never expected)
    kErrCounterOverflow = 4u,  // a 32-bit c~ counter wrapped
    kErrSelect = 8u,           // weighted choice found no element (never expected)
    kErrDepth = 16u,           // reserved: levels are 32-bit, so no side can run out of them
    kErrTimeout = 32u,         // a bounded wait for a free counter frame gave up
    kErrLogOverflow = 64u,     // an epoch log overflowed (a path longer than VD - 2)
    kErrScratch = 128u,        // a sample outgrew its slot and no spill slot was configured
};

// Per-sample trace record (mirrors kadabra_trace_rec).
struct TraceRec {
    long long s, t, d;
    unsigned long long sigma_lo, sigma_hi;
    long long meet_size, chosen, e_scan, n_interior;
    int scaled, overflow;
    long long ns;              // device time of the sample (global timer), cleanup excluded
    long long phase_ns[4];     // BFS, meeting-vertex choice, back-walk, record clearing
};

struct SampleLaunch {
    int64_t n;
    const void *off;           // int32 or int64 offsets (n + 1)
    int off64;
    const uint2 *adj;          // (neighbour id, neighbour degree) per adjacency entry
    SlotSet slots;             // one per CTA (stride >= n)
    SlotSet spill;             // taken by samples that outgrow their slot (may be empty)
    uint32_t *counts;          // c~[n]; nullptr: do not count (trace runs)
    Job *job;
    Counters *launch_ctr;      // this launch's own counters (zeroed before the launch), may be null
    uint64_t seed;
    uint32_t tag;              // 0 calibration, 1 adaptive
    int K;                     // sigma bits
    int strict;
    int use_stop;              // honour job->stopped
    int64_t epoch_len;         // requested samples
    uint64_t clip;             // never pass this tau (0 = no clip)
    TraceRec *trace;           // optional per-sample records (index - tau)
    int32_t *trace_path;       // optional interior vertices, trace_cap per sample
    int64_t trace_cap;
    int grid;
    int threads;
    const int *abandon;        // optional: a sample stops at its next layer once *abandon != 0
    int use_bits;              // use the slots' reached-bit maps (graphs of small diameter)
    unsigned long long spin_limit;   // bounded waits (spill slot, claims being published)
    void *help;                // persistent launches: board of layers posted for other CTAs (or null)
    unsigned long long help_edges;   // a layer with at least this frontier degree sum is posted
    uint32_t *log;             // optional (counts == nullptr): interior vertices appended here
    unsigned int *log_len;     //   entries appended (may exceed log_cap: then the log overflowed)
    unsigned int log_cap;
    int probe_log2;            // log2 of the bits of the shared-memory frontier bitmap (dynamic
                               //   shared memory of the launch); 0: no bitmap, no probe pass
    unsigned long long probe_edges;  // samples with reached-bit maps probe a layer first when its
                                     //   frontier degree sum is at least this
};

cudaError_t launch_sample(const SampleLaunch &a, cudaStream_t st);
// Device bytes of `count` slots; allocation (zeroed) and release of a slot set.
size_t slot_set_bytes(int count, long long stride, long long cap, bool bits, bool lock);
cudaError_t alloc_slot_set(SlotSet *S, int count, long long stride, long long cap, bool bits, bool lock);
void free_slot_set(SlotSet *S);
// adj[e] = (col[e], degree of col[e]); off in device memory, col in device
// memory or device-accessible page-locked host memory; deg_tmp: n words.
cudaError_t launch_build_adj(int64_t n, int64_t nnz, const void *off, int off64, const int32_t *col, uint2 *adj,
                             uint32_t *deg_tmp, cudaStream_t st);
// diameter phase (graph_kernels.cu)
size_t vd_bound_scratch_bytes(int64_t n);
cudaError_t launch_vd_bound(int64_t n, const void *off, int off64, const uint2 *adj, void *scratch, cudaStream_t st,
                            int64_t *vd);
cudaError_t launch_max_degree(int64_t n, const void *off, int off64, unsigned long long *out, cudaStream_t st);
// exact vertex diameter (iFUB on the largest component; graph_kernels.cu)
size_t vd_exact_scratch_bytes(int64_t n);
cudaError_t launch_vd_exact(int64_t n, const void *off, int off64, const uint2 *adj, void *scratch, cudaStream_t st,
                            int64_t *vd, int *exact, int64_t *searches);
cudaError_t sample_occupancy(int threads, int off64, int *ctas_per_sm);
// Size of the probe bitmap that leaves `ctas_per_sm` sampling CTAs of
// `threads` threads resident on an SM (log2 of its bits; 0 if below 2^15
// bits), with both sampling kernels allowed that much dynamic shared memory.
// Host-side set-up: call outside stream capture.
cudaError_t probe_prepare(int threads, int off64, int ctas_per_sm, int *log2_bits);

// Pipelined adaptive phase: epochs rotate through F epoch logs; one persistent
// launch serves one or many queries (see batch_kernel in sample_kernel.cu).
constexpr int kMaxFrames = 16;

// Per-query pipeline state; persists across launches until the query is
// begun again.
struct PipeState {
    unsigned long long next_idx;        // next sample (relative to base) to hand out
    long long next_check;               // next epoch to fold into c~ and check
    unsigned int done[kMaxFrames];      // finished samples of the epoch each frame holds
    unsigned int log_len[kMaxFrames];   // interior vertices logged by the epoch each frame holds
    int checker;                        // 1 while a CTA folds and checks this query
    int abort;                          // set when a bounded wait gave up
    unsigned long long base;            // tau when the pipeline began
    unsigned long long R;               // samples the pipeline may take (ceil(omega) - base)
    long long nE;                       // epochs in R
    Counters fc[kMaxFrames];            // counters of the epoch each frame holds: added to the
                                        // query's totals when that epoch is checked, so samples
                                        // of epochs after the stop are never counted
};

// One query of a pipelined launch (device memory, written by the host).
struct QueryDesc {
    long long n;
    const void *off;           // offsets (the launch's offset width)
    const uint2 *adj;
    int K;
    int strict;
    unsigned long long seed;
    long long E;               // samples per epoch
    int F;                     // epoch logs in rotation
    unsigned int log_cap;      // entries per log
    uint32_t *logs;            // F logs
    const uint32_t *cls;       // budget class of every vertex
    const double2 *Ltab;       // (L_L, L_U) of every class
    unsigned int *cmax;        // largest c~ in every class
    int nclass;
    int use_bits;              // the query uses the slots' reached-bit maps
    int lookahead;             // 1: near the predicted stop, open only the epochs up to it
                               //    (and one more); 0: always all F frames
    int tag;                   // 1: adaptive phase (epochs, logs, checks); 0: calibration samples
                               //    counted straight into `counts` (E = n_calib, F = 1, no check)
    double omega, eps;
    uint32_t *counts;          // c~
    Job *job;
    PipeState *ps;
    Counters *launch_ctr;      // this launch's counters for the query (may be null)
};

struct BatchState {
    unsigned int ticket;                // round-robin start for query selection
    unsigned int abort;
    unsigned long long taken;           // samples handed out by this launch
};

struct BatchLaunch {
    QueryDesc *queries;        // device array
    int nq;
    SlotSet slots;             // one per CTA; stride = largest n of the batch
    SlotSet spill;             // taken by samples that outgrow their slot (may be empty)
    void *help;                // help board (help_board_bytes(), zeroed once), or null: no helping
    unsigned long long help_edges;   // frontier degree sum from which a layer is posted
    BatchState *bs;
    unsigned long long budget; // samples this launch may hand out (0 = no limit)
    unsigned long long spin_limit;
    int grid, threads, off64;
    int policy;                // 0: round robin over the queries; 1: first in array order
    int probe_log2;            // as in SampleLaunch (queries with use_bits only)
    unsigned long long probe_edges;
};

cudaError_t launch_batch(const BatchLaunch &a, cudaStream_t st);
// Bytes of a help board for persistent launches (allocate once, zeroed).
size_t help_board_bytes();
cudaError_t launch_pipe_begin(PipeState *ps, const Job *job, unsigned long long clip, long long E, cudaStream_t st);
cudaError_t launch_class_max(int64_t n, const uint32_t *counts, const uint32_t *cls, unsigned int *cmax,
                             cudaStream_t st);

struct CheckLaunch {
    int64_t n;
    const uint32_t *counts;
    const double2 *L;          // (L_L, L_U) per vertex
    Job *job;
    double omega;
    double eps;
    int grid;
};

cudaError_t launch_check(const CheckLaunch &a, cudaStream_t st);

// Read-only view of a loaded graph's device arrays (kadabra_api.cpp).
struct GraphView {
    int64_t n, nnz, max_degree;
    int off64;
    const void *off;
    const uint2 *adj;
};
bool graph_view(const struct ::kadabra_graph *g, GraphView *out);
// Record the message returned by kadabra_last_error() on this thread.
int set_last_error(int status, const char *msg);

// Allocation-free sampling (sample_static.cu).
cudaError_t static_scratch_address(void **out);
cudaError_t static_scratch_reserve();
cudaError_t launch_result(int64_t n, const uint32_t *counts, const Job *job, double *btilde,
                          cudaStream_t st);
// Job record reset to its start state (tau = `tau`, no stop, no error).
cudaError_t launch_reset_job(Job *job, cudaStream_t st, unsigned long long tau = 0);
cudaError_t read_device_clock(unsigned long long *ns, cudaStream_t st);
cudaError_t launch_batch_poll(const QueryDesc *d, int nq, int *out, cudaStream_t st);
cudaError_t launch_cal_max(int64_t n, const uint32_t *cal, unsigned int *mx, cudaStream_t st);
cudaError_t launch_cal_hist(int64_t n, const uint32_t *cal, unsigned int cmax, unsigned long long *hist,
                            cudaStream_t st);
cudaError_t launch_fill_budgets(int64_t n, const uint32_t *cal, const int *class_of, const double2 *Ltab,
                                uint32_t *cls, double2 *L, cudaStream_t st);
cudaError_t launch_absorb(int64_t n, uint32_t *counts, const uint32_t *delta, Job *job, uint64_t samples,
                          cudaStream_t st);
cudaError_t launch_absorb_log(const uint32_t *log, uint64_t len, int64_t n, uint32_t *counts, Job *job, uint64_t samples,
                              cudaStream_t st);

}  // namespace kadabra
