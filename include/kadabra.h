/*
 * kadabra.h -- C ABI of the GB300 KADABRA adaptive-sampling betweenness library.
 *
 * The method (arXiv 1910.11039, Section III-A): betweenness
 *   b(x) = 1/(n(n-1)) * sum_{s != t} sigma_st(x) / sigma_st          (Section I)
 * is approximated by sampling pairs s != t, drawing one shortest s-t path
 * uniformly with a bidirectional BFS and adding 1 to the counter c~(x) of each
 * interior vertex x; after tau samples b~(x) = c~(x) / tau.  Sampling is
 * adaptive: after every epoch a stopping condition f(...) < eps and
 * g(...) < eps for all x is evaluated on a consistent snapshot of (tau, c~)
 * (Section III-B; Algorithms 1 and 2), with a hard cap of omega samples.
 * The three phases are diameter -> omega, calibration of delta_L / delta_U,
 * and adaptive sampling (Section III-A).
 *
 * Conventions for every call:
 *   - Every function returns a kadabra_status; nothing throws across the ABI.
 *     On error the outputs are left untouched and kadabra_last_error()
 *     returns a message (thread-local, valid until the next call on the
 *     same thread).
 *   - `cuda_stream` is a cudaStream_t passed as void* (NULL = legacy default
 *     stream).  Calls marked "async" only enqueue work on that stream.
 *   - Vertex ids are int32 (n < 2^31).  Offsets are int32 or int64.
 *   - Objects (kadabra_graph, kadabra_query) are owned by the library and
 *     released with their _free call.  Caller arrays stay owned by the caller.
 *   - A graph's sampling scratch is shared by its queries: queries of one
 *     graph must be driven from one stream (or serialised by the caller).
 */
#ifndef KADABRA_H
#define KADABRA_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum kadabra_status {
    KADABRA_OK = 0,
    KADABRA_ERR_INVALID_ARG = 1,      /* bad argument or malformed CSR            */
    KADABRA_ERR_OOM = 2,              /* device or host allocation failed         */
    KADABRA_ERR_CUDA = 3,             /* a CUDA runtime call failed               */
    KADABRA_ERR_SIGMA_OVERFLOW = 4,   /* strict mode met a path count above 2^K   */
    KADABRA_ERR_COUNTER_OVERFLOW = 5, /* a 32-bit counter would wrap              */
    KADABRA_ERR_TIMEOUT = 6,          /* a bounded device wait gave up            */
    KADABRA_ERR_STATE = 7,            /* call out of order (e.g. result before run)*/
    KADABRA_ERR_NO_DEVICE = 8,        /* no CUDA device / library built without it */
    KADABRA_ERR_DEPTH = 9             /* reserved (BFS levels are 32-bit; unused)  */
} kadabra_status;

typedef struct kadabra_graph kadabra_graph;
typedef struct kadabra_query kadabra_query;

/* flags for kadabra_graph_load */
#define KADABRA_GRAPH_DEVICE_PTRS   1u  /* offsets / cols are device pointers           */
#define KADABRA_GRAPH_SKIP_VALIDATE 2u  /* trust the CSR (no host-side checks)           */

/* kadabra_params.flags */
#define KADABRA_STRICT_SIGMA 1u  /* a per-side path count above 2^K is an error instead
                                    of being scaled down (see kadabra_sigma_bits)        */
#define KADABRA_FULL_LOOKAHEAD 2u /* pipelined launches: keep all epoch frames open until
                                    the stop.  By default, once the last check's maxima
                                    of f and g predict the stop within the frames (both
                                    shrink about as 1/sqrt(tau)), samples are handed out
                                    only up to the predicted stop epoch and one more, and
                                    CTAs without a sample help heavy layers instead.
                                    Results never depend on it                           */

/* kadabra_params.delta_rule */
#define KADABRA_DELTA_UNIFORM  0  /* delta_L = delta_U = delta / (4n)                     */
#define KADABRA_DELTA_BALANCED 1  /* calibrated split, exp(-C eps^2 / bhat) + floor       */

/* Parameters of one betweenness query (Section III-A: eps, delta; the rest
 * are this library's readings of what the paper leaves open). */
typedef struct kadabra_params {
    double eps;               /* additive error bound, 0 < eps < 1                         */
    double delta;             /* failure probability, 0 < delta < 1                        */
    uint64_t seed;            /* Philox key: sample i of stream tag k draws from
                                 counter (i, draw, k, 0) under key (seed, 0)               */
    int64_t vertex_diameter;  /* VD >= 1 if known; 0: upper bound 2*ecc(root)+1 per
                                 component; -1: exact, by iFUB on the device (Section
                                 III-A computes the diameter exactly), for every
                                 component whose bound exceeds the best value; a search
                                 whose fringe needs more than 64 bit-parallel sweeps
                                 (meshes) keeps the upper bound it proved, and
                                 kadabra_query_info.vd_exact says which               */
    int64_t n_calib;          /* calibration samples; <= 0: max(1000, ceil(omega/100))     */
    int32_t delta_rule;       /* KADABRA_DELTA_UNIFORM or KADABRA_DELTA_BALANCED           */
    uint32_t flags;           /* KADABRA_STRICT_SIGMA | KADABRA_FULL_LOOKAHEAD              */
    double beta;              /* balanced rule floor weight (default 1e-3)                 */
    int32_t slots;            /* samples in flight (one CTA each); 0 = fill the GPU        */
    int32_t threads;          /* threads per sampling CTA: 128, 256, 512, 1024; 0 = 1024   */
    double scratch_fraction;  /* max share of free device memory for scratch; 0 = 0.6      */
    int64_t queue_cap;        /* queue positions per slot (the two BFS balls of a sample
                                 together); 0 = n when the slots fit the scratch budget,
                                 else what fits.  A sample that outgrows it runs again on
                                 one of two full-capacity spill slots, so results never
                                 depend on it                                              */
    int64_t coop_edges;       /* pipelined launches: a BFS layer whose frontier degree sum
                                 is at least this is split into chunks that idle CTAs
                                 expand together with the sample's own CTA; 0 = 32768,
                                 < 0 = never.  Results never depend on it               */
    int64_t probe_edges;      /* queries whose vertex-diameter bound is at most 64: a BFS
                                 layer whose frontier degree sum is at least this first
                                 tests its targets against a shared-memory bitmap of the
                                 other side's frontier and, if it meets that frontier,
                                 ends the search without claiming anything; 0 = the
                                 default (256), < 0 = never.  Results never depend on it   */
} kadabra_params;

/* Snapshot of a query (kadabra_query_get_info). */
typedef struct kadabra_query_info {
    double omega;               /* maximal number of samples                               */
    uint64_t omega_ceil;        /* ceil(omega): adaptive sampling never passes it          */
    int64_t vertex_diameter;    /* VD used for omega                                       */
    int64_t n_calib;            /* calibration samples taken                               */
    int32_t sigma_bits;         /* K: per-side path counts are kept <= 2^K                 */
    int32_t stopped;            /* 1 once the stopping condition held                      */
    uint64_t tau;               /* adaptive samples taken                                  */
    int64_t epochs;             /* stop checks run                                         */
    int64_t stop_epoch;         /* index of the check that stopped, -1 if none             */
    double max_f, max_g;        /* maxima of f and g at the last check                     */
    double balance_C;           /* constant of the balanced delta rule                     */
    /* adaptive-phase counters (summed over all epochs) */
    uint64_t samples;           /* samples taken                                            */
    uint64_t connected;         /* samples whose pair was connected                        */
    uint64_t e_scan;            /* adjacency entries scanned by the BFS (traversed edges)  */
    uint64_t expanded;          /* frontier vertices expanded                              */
    uint64_t touched;           /* vertices reached by either BFS side                     */
    uint64_t interior;          /* interior path vertices counted                          */
    uint64_t walk_scan;         /* adjacency entries scanned by the path back-walk         */
    uint64_t scaled;            /* samples whose path counts were scaled                   */
    uint32_t device_error;      /* sticky device error bits (0 = none)                     */
    int32_t slots;              /* samples in flight per launch                            */
    int32_t threads;            /* threads per sampling CTA                                */
    int32_t offsets_64;         /* 1 if the graph uses int64 offsets                       */
    int32_t budget_classes;     /* distinct (L_L, L_U) pairs                               */
    uint64_t stop_ns;           /* device global timer (ns) when the stop was decided, or 0 */
    int32_t phase;              /* 0 created, 1 calibrating in a batch, 2 calibrated        */
    int32_t pad0;
    uint64_t cal_done;          /* calibration samples completed (phase 1), else n_calib    */
    uint64_t device_bytes;      /* device memory the query holds (not the graph's)          */
    int64_t launches;           /* sampling launches logged (kadabra_launch_log), ever      */
    double diameter_ms;         /* host wall time of phase 1 (diameter bound and omega)    */
    double calibration_ms;      /* host wall time of phase 2 (calibration; batch: budgets)  */
    int64_t queue_cap;          /* queue positions per sampling slot (both BFS sides)       */
    int32_t spill_slots;        /* full-capacity slots for samples that outgrow queue_cap   */
    int32_t vd_exact;           /* 1 if vertex_diameter is the exact vertex diameter        */
    int64_t vd_searches;        /* breadth-first searches the diameter phase ran            */
} kadabra_query_info;

/* Per-sample record written by kadabra_sample_trace (one per sample index). */
typedef struct kadabra_trace_rec {
    int64_t s, t;               /* the pair (draw 0)                                       */
    int64_t d;                  /* d(s,t), -1 if disconnected                              */
    uint64_t sigma_lo, sigma_hi;/* sigma_st as used for the choice (128 bits)             */
    int64_t meet_size;          /* size of the meeting set                                 */
    int64_t chosen;             /* meeting vertex picked, -1 if none                       */
    int64_t e_scan;             /* adjacency entries scanned by the BFS                    */
    int64_t n_interior;         /* interior vertices of the sampled path                   */
    int32_t scaled;             /* 1 if a layer's path counts were scaled                  */
    int32_t overflow;           /* 1 strict mode rejected the sample, 2 too many layers    */
    int64_t ns;                 /* device time spent on the sample (ns, global timer)      */
    int64_t phase_ns[4];        /* of which: BFS, meeting-vertex choice, back-walk, and
                                   (not included in ns) clearing the touched records       */
} kadabra_trace_rec;

/* ---- errors and version ------------------------------------------------ */

/* Message of the last failed call on this thread ("" if none). */
const char *kadabra_last_error(void);
/* Static name of a status code. */
const char *kadabra_status_string(kadabra_status s);
/* ABI version of this header (major * 100 + minor). */
int kadabra_abi_version(void);

/* ---- host utilities (no device needed) --------------------------------- */

/* Fill `p` with defaults: eps 0.01, delta 0.1, seed 1, auto VD, default
 * calibration size, balanced rule, beta 1e-3, auto slots, 1024 threads. */
void kadabra_params_default(kadabra_params *p);

/* Check that (offsets, cols) is a symmetric CSR with ascending, duplicate-free
 * neighbour lists, no self-loops and ids in [0, n) (Section III: undirected,
 * unweighted graphs).  Host pointers.  KADABRA_ERR_INVALID_ARG on the first
 * violation, with the reason in kadabra_last_error(). */
kadabra_status kadabra_validate_csr(int64_t n, int64_t nnz, const void *offsets, int offsets_is_64,
                                    const int32_t *cols);

/* omega = (1/2) / eps^2 * (floor(log2(VD - 2)) + 1 + ln(2/delta)), VD - 2
 * clamped to >= 1: the maximal number of samples, computed from the diameter
 * (Section III-A names omega; the formula is this library's reading).
 * Writes NaN and returns KADABRA_ERR_INVALID_ARG for eps or delta outside (0,1). */
kadabra_status kadabra_omega(double eps, double delta, int64_t vertex_diameter, double *omega);

/* K = min(63 - bitlen(max_degree), 63 - bitlen(n)).  Section III-A samples
 * a shortest s-t path uniformly, which needs exact path counts; the paper does
 * not say how counts beyond a machine word are handled.  This library's
 * reading: every per-side path count is an exact uint64.  Counts up to 2^K
 * are exact; a BFS layer whose largest count exceeds 2^K has all its counts
 * shifted right by the excess (rounding up, so they stay >= 1).  Then a count
 * of the next layer (a sum of at most max_degree counts) stays below 2^63, so
 * no 64-bit addition can wrap (each is checked all the same), and every
 * meeting-set weight sum fits 128 bits. */
int kadabra_sigma_bits(int64_t n, int64_t max_degree);

/* Device global timer (ns; the clock of kadabra_query_info.stop_ns), read by a
 * one-thread kernel on `cuda_stream`.  Synchronises. */
kadabra_status kadabra_device_clock(uint64_t *ns, void *cuda_stream);

/* ---- graph ------------------------------------------------------------- */

/* Copy a CSR graph into library-owned device memory, on `cuda_stream`;
 * synchronises before returning (the maximum degree is read back), so the
 * caller's arrays are no longer referenced afterwards.
 *   n        number of vertices (1 <= n < 2^31)
 *   nnz      number of adjacency entries (= offsets[n])
 *   offsets  n+1 entries, int32 if offsets_is_64 == 0 else int64
 *   cols     nnz int32 neighbour ids, each row ascending
 *   flags    KADABRA_GRAPH_DEVICE_PTRS, KADABRA_GRAPH_SKIP_VALIDATE
 * Host inputs are validated (kadabra_validate_csr) unless skipped.  Host
 * columns in page-locked memory (cudaHostAlloc, cudaHostRegister) are read
 * in place by the kernel that builds the device adjacency (one pass over the
 * host link); pageable host columns go through a temporary device copy. */
kadabra_status kadabra_graph_load(int64_t n, int64_t nnz, const void *offsets, int offsets_is_64,
                                  const int32_t *cols, uint32_t flags, void *cuda_stream,
                                  kadabra_graph **out);
kadabra_status kadabra_graph_free(kadabra_graph *g);
kadabra_status kadabra_graph_info(const kadabra_graph *g, int64_t *n, int64_t *nnz,
                                  int64_t *max_degree, int *offsets_is_64);

/* ---- query: the three phases (Section III-A) --------------------------- */

/* Phase 1 alone: VD and omega, and the query's device state (counters,
 * budgets, calibration counts), without calibration samples.  Synchronises.
 * The query then takes its calibration samples inside a batch
 * (kadabra_calibration_begin, kadabra_batch_step until
 * kadabra_query_info.cal_done == n_calib, kadabra_calibration_finish); no
 * other sampling call accepts it before that.  The calibration samples are
 * the same ones kadabra_calibrate takes, so the budgets are identical. */
kadabra_status kadabra_query_create(kadabra_graph *g, const kadabra_params *p, void *cuda_stream,
                                    kadabra_query **out);
/* Hand out calibration sample indices [0, n_calib) (stream tag 0) to the
 * next batch steps that include the query (async).  KADABRA_ERR_STATE unless
 * the query came from kadabra_query_create and has not begun calibrating. */
kadabra_status kadabra_calibration_begin(kadabra_query *q, void *cuda_stream);
/* Phase 2 on the host once all calibration samples completed: delta_L,
 * delta_U and the budget classes, uploaded to the device.  Synchronises.
 * KADABRA_ERR_STATE while samples are outstanding. */
kadabra_status kadabra_calibration_finish(kadabra_query *q, void *cuda_stream);

/* Phases 1 and 2.  Computes VD (or takes it from `p`) and omega, runs the
 * calibration samples on the device (stream tag 0, sample indices
 * [0, n_calib)), derives delta_L(x), delta_U(x) on the host and uploads
 * L_L = -ln delta_L, L_U = -ln delta_U.  Allocates the query's device state.
 * Synchronises `cuda_stream`.  Rejects eps, delta outside (0,1) and omega
 * >= 2^32 (the counters are 32-bit). */
kadabra_status kadabra_calibrate(kadabra_graph *g, const kadabra_params *p, void *cuda_stream,
                                 kadabra_query **out);
kadabra_status kadabra_query_free(kadabra_query *q);

/* Phase 3, one epoch (async).  Takes adaptive samples [tau, tau + m) with
 * m = min(n_samples, omega_ceil - tau) (stream tag 1) and adds each sampled
 * path's interior vertices to c~.  tau lives on the device and advances when
 * the launch ends; if a previous check already stopped the query the launch
 * takes no samples.  Device errors surface at the next synchronising call. */
kadabra_status kadabra_sample_epoch(kadabra_query *q, int64_t n_samples, void *cuda_stream);

/* Stopping condition on the current snapshot (tau, c~): stop iff tau >= omega
 * or max_x f(b~(x), delta_L(x), omega, tau) < eps and max_x g(b~(x),
 * delta_U(x), omega, tau) < eps, evaluated in IEEE double without contraction.
 * The first check that stops records the stop epoch.  Synchronises and writes
 * the host outputs (each may be NULL). */
kadabra_status kadabra_check_stop(kadabra_query *q, int *stopped, double *max_f, double *max_g,
                                  void *cuda_stream);
/* Same check, async: the flag stays on the device, where later
 * kadabra_sample_epoch launches read it. */
kadabra_status kadabra_check_stop_async(kadabra_query *q, void *cuda_stream);

/* Convenience loop: epochs of `epoch_len` samples, each followed by an async
 * check, until the query stops or `max_epochs` checks ran.  The host reads the
 * device flag once every `sync_every` epochs (<= 0: 4).  Writes *stopped. */
kadabra_status kadabra_run(kadabra_query *q, int64_t epoch_len, int64_t max_epochs,
                           int64_t sync_every, void *cuda_stream, int *stopped);

/* Phase 3 as one persistent launch (async), the GPU form of the paper's
 * epoch framework (Section IV-A/B, Algorithm 2: threads keep sampling into the
 * state frame of their epoch while a completed epoch is aggregated and
 * checked).  Sample i belongs to epoch i / epoch_len and logs its interior
 * vertices in frame (epoch mod frames); the CTA that completes the oldest
 * unchecked epoch folds that log into c~ and evaluates the stopping condition
 * on exactly samples [0, (e + 1) epoch_len) while all other CTAs keep
 * sampling later epochs.  The check evaluates f and g once per budget class
 * (vertices with equal (L_L, L_U)) at the class's largest counter, which
 * gives exactly the per-vertex maxima because f and g are monotone in c~.
 * Samples of epochs after the stopping epoch are discarded, so tau, c~ and
 * the stop epoch equal those of repeated kadabra_sample_epoch(epoch_len) +
 * kadabra_check_stop from the same starting tau.
 *   frames: 1..16 epoch logs of epoch_len * (VD - 2) entries (<= 0: 8); a CTA
 *   waits for a free frame before sampling more than `frames` epochs ahead of
 *   the oldest unchecked one.  That wait is bounded; if it gives up, the launch
 *   ends and the next synchronising call returns KADABRA_ERR_TIMEOUT.  A path
 *   with more than VD - 2 interior vertices (a vertex_diameter parameter below
 *   the true one) ends the launch with KADABRA_ERR_INVALID_ARG. */
kadabra_status kadabra_run_pipelined(kadabra_query *q, int64_t epoch_len, int frames, void *cuda_stream);

/* The pipelined phase in steps, and many queries in one launch.
 * kadabra_pipeline_begin prepares a query's pipelined adaptive phase from its
 * current tau (epoch logs, per-query pipeline state; async);
 * kadabra_run_pipelined = begin + one launch run to the end.
 * A kadabra_batch holds sampling scratch for `slots` samples in flight (0 =
 * fill the GPU) on graphs of up to max_n vertices, all with the same offset
 * width.  kadabra_batch_step is one persistent launch over `count` begun
 * queries, possibly on different graphs (async): CTAs take the next sample
 * of the running queries in round robin and check each query's epochs in
 * order exactly as kadabra_run_pipelined does, so every query's tau, c~ and
 * stop epoch are those it has alone.  The launch ends when every query has
 * stopped or reached ceil(omega), or after `sample_budget` samples were
 * handed out (0 = no limit); pipeline state persists, so a later step (with
 * the same or other begun queries) continues where this one ended.  A batch
 * must not be stepped on two streams at once. */
typedef struct kadabra_batch kadabra_batch;
kadabra_status kadabra_pipeline_begin(kadabra_query *q, int64_t epoch_len, int frames, void *cuda_stream);
kadabra_status kadabra_batch_create(int64_t max_n, int32_t slots, int32_t threads, int offsets_is_64,
                                    kadabra_batch **out);
kadabra_status kadabra_batch_free(kadabra_batch *b);
kadabra_status kadabra_batch_step(kadabra_batch *b, kadabra_query *const *qs, int64_t count, uint64_t sample_budget,
                                  void *cuda_stream);
/* Device time (ms) of the most recent step (CUDA events on its stream).  Synchronises. */
kadabra_status kadabra_batch_last_ms(kadabra_batch *b, float *ms);
/* Which running query a CTA serves next.  ROUND_ROBIN (default): each pick
 * starts the scan at the next query in turn, so running queries take samples
 * at equal rates.  IN_ORDER: the first query in the array passed to
 * kadabra_batch_step that can take a sample gets it, so earlier queries run
 * at full width and later ones fill the slots they leave (a priority order,
 * e.g. shortest expected work first or arrival order).  Results do not
 * depend on the policy. */
enum { KADABRA_BATCH_ROUND_ROBIN = 0, KADABRA_BATCH_IN_ORDER = 1 };
/* After a step: the state of each of its `count` queries (in the order they
 * were passed) into states[] (host): 0 running, 1 calibration samples
 * complete (kadabra_calibration_finish may run), 2 stopped or at ceil(omega).
 * One small kernel and one copy on `cuda_stream`.  Synchronises.
 * KADABRA_ERR_INVALID_ARG if count differs from the last step's. */
kadabra_status kadabra_batch_poll(kadabra_batch *b, int32_t *states, int64_t count, void *cuda_stream);
kadabra_status kadabra_batch_set_policy(kadabra_batch *b, int policy);
/* Every wait inside a batch step (a CTA waiting for a free epoch frame, or
 * for any running query to accept a sample) polls at most `polls` times
 * (default 2^24, each poll sleeps ~0.3-0.5 us); a wait that runs out marks its
 * queries with the timeout bit and ends the step, and the next synchronising
 * call on such a query returns KADABRA_ERR_TIMEOUT.  The device stays usable:
 * kadabra_query_reset and kadabra_pipeline_begin restart the query. */
kadabra_status kadabra_batch_set_spin_limit(kadabra_batch *b, uint64_t polls);
/* Samples in flight per step (CTAs), threads per sampling CTA and the largest
 * n the batch serves; each output optional. */
kadabra_status kadabra_batch_info(const kadabra_batch *b, int32_t *slots, int32_t *threads, int64_t *max_n);

/* Sharded sampling (several ranks, one GPU each; Section I-A: samples are
 * independent, so a rank can take any subset of an epoch's sample indices).
 * kadabra_sample_range takes sample indices [first, first + count) of stream
 * `tag` (0 calibration, 1 adaptive) with the query's seed and adds the
 * interior vertices of each sampled path to counts[n] (device pointer,
 * caller-owned, accumulated); the query's tau and c~ are not touched (async).
 * kadabra_absorb is the epoch aggregate: it adds delta[n] (device pointer,
 * e.g. the sum of every rank's counts for one epoch) to c~ and advances tau by
 * `samples` (async); kadabra_check_stop then checks the new snapshot. */
kadabra_status kadabra_sample_range(kadabra_query *q, int tag, uint64_t first, int64_t count, uint32_t *counts,
                                    void *cuda_stream);
kadabra_status kadabra_absorb(kadabra_query *q, const uint32_t *delta, uint64_t samples, void *cuda_stream);

/* The same exchange with epoch logs instead of counter vectors (an epoch's
 * logs hold at most E * (VD - 2) vertex ids, against n counters).
 * kadabra_sample_range_log takes sample indices [first, first + count) of
 * stream `tag` and appends the interior vertices of each sampled path to
 * log[log_cap] (device pointer, caller-owned; order unspecified); *log_len
 * (device word) is set to the number appended -- a value above log_cap means
 * the log overflowed and the entries beyond it were dropped (async).
 * kadabra_absorb_log adds 1 to c~[x] for every entry x of log[len] (device
 * pointer: the concatenated logs of every rank for one epoch, in any order)
 * and advances tau by `samples` (async). */
kadabra_status kadabra_sample_range_log(kadabra_query *q, int tag, uint64_t first, int64_t count, uint32_t *log,
                                        uint32_t log_cap, uint32_t *log_len, void *cuda_stream);
kadabra_status kadabra_absorb_log(kadabra_query *q, const uint32_t *log, uint64_t len, uint64_t samples,
                                  void *cuda_stream);

/* The stream-ordered epochs of kadabra_run as a CUDA graph: the first call
 * for a given (epoch_len, epochs_per_graph) captures epochs_per_graph epochs
 * (sampling launch + stop-check launch each) on a private stream and
 * instantiates the graph; every call then launches the graph on `cuda_stream`
 * until the query stops, max_epochs epochs ran, or tau reaches ceil(omega),
 * reading the device stop flag once per graph launch.  Results equal
 * kadabra_run with the same epoch_len.  Writes *stopped. */
kadabra_status kadabra_run_graph(kadabra_query *q, int64_t epoch_len, int epochs_per_graph, int64_t max_epochs,
                                 void *cuda_stream, int *stopped);

/* Restart phase 3 (tau = 0, c~ = 0, not stopped) keeping omega and the
 * calibrated budgets (async). */
kadabra_status kadabra_query_reset(kadabra_query *q, void *cuda_stream);

/* Checkpoint and resume.  A query's adaptive state is its counters c~, tau
 * and the number of epochs checked; samples are indexed by (seed, stream tag,
 * sample index), so a query restored from that state continues exactly as the
 * checkpointed one would have (same tau, stop epoch and counters at the end).
 * A checkpoint is read with kadabra_result (counts, tau) and
 * kadabra_query_get_info (epochs).  kadabra_query_restore sets c~ from
 * counts[n] (host), tau and the epoch count, and clears the stop flag and
 * error bits; the query must have been calibrated with the parameters of the
 * checkpointed one (graph, eps, delta, seed, n_calib, delta rule, vertex
 * diameter).  A pipelined phase must be begun again.  Synchronises. */
kadabra_status kadabra_query_restore(kadabra_query *q, const uint32_t *counts, uint64_t tau, int64_t epochs,
                                     void *cuda_stream);

/* Result: b~(x) = c~(x) / tau, computed on the device.  Host outputs, each
 * optional: btilde[n] (double), counts[n] (uint32 c~), *tau, *stop_epoch.
 * Synchronises.  KADABRA_ERR_STATE if tau == 0 and btilde is requested. */
kadabra_status kadabra_result(kadabra_query *q, double *btilde, uint32_t *counts, uint64_t *tau,
                              int64_t *stop_epoch, void *cuda_stream);

/* Snapshot of omega, tau, epochs, maxima and counters.  Synchronises. */
kadabra_status kadabra_query_get_info(kadabra_query *q, kadabra_query_info *out, void *cuda_stream);

/* Calibration budgets as uploaded: host L_L[n], L_U[n] (each optional) and the
 * calibration counts cal[n] (optional).  Synchronises. */
kadabra_status kadabra_query_budgets(kadabra_query *q, double *L_L, double *L_U, uint32_t *cal,
                                     void *cuda_stream);

/* Per-sample records for sample indices [first, first + count) of stream
 * `tag` (0 calibration, 1 adaptive), computed by the same sampling kernel
 * without touching the query's counters or tau.  Host outputs: recs[count];
 * interior[count * path_cap] (optional) receives each path's interior
 * vertices in the order meeting vertex, walk towards s, walk towards t,
 * truncated to path_cap.  Synchronises. */
kadabra_status kadabra_sample_trace(kadabra_query *q, int tag, uint64_t first, int64_t count,
                                    kadabra_trace_rec *recs, int32_t *interior, int64_t path_cap,
                                    void *cuda_stream);

/* Per-launch instrumentation of kadabra_sample_epoch: each launch is
 * bracketed by CUDA events on its stream and keeps its own counters; the
 * query remembers its most recent 256 launches. */
typedef struct kadabra_launch_stats {
    float ms;                   /* sampling kernel time between its two events             */
    uint64_t samples, connected, e_scan, expanded, touched, interior, walk_scan;
    int32_t grid, threads;      /* launch shape                                             */
} kadabra_launch_stats;
/* The most recent launch.  Synchronises on its end event. */
kadabra_status kadabra_last_launch(kadabra_query *q, kadabra_launch_stats *out);
/* Up to `max_entries` most recent launches, oldest first, into out[]; *n_out
 * receives the number written.  Synchronises on the newest end event. */
kadabra_status kadabra_launch_log(kadabra_query *q, int64_t max_entries, kadabra_launch_stats *out,
                                  int64_t *n_out);

/* ---- allocation-free sampling ------------------------------------------ */

/* Size of the library's file-scope device scratch array used by
 * kadabra_sample_static.  Every device that loads the library holds it until
 * the process exits. */
#define KADABRA_STATIC_SCRATCH_BYTES (64u << 20)

/* Adaptive-phase style sampling for callers that cannot allocate device
 * memory: for example, a service that plans all memory at start-up and
 * forbids allocation afterwards, or code inside a framework that owns the
 * device allocator.  The paper has no counterpart; this is a packaging of the
 * sampling kernel.
 * Takes sample indices [first, first + count) of stream `tag` (0 calibration,
 * 1 adaptive) under `seed`, exactly as kadabra_sample_epoch / the calibration
 * do, and adds each sampled path's interior vertices to counts[n] (device
 * pointer, caller-owned, accumulated, not cleared).  The scratch lives in a
 * fixed array of KADABRA_STATIC_SCRATCH_BYTES inside the library; nothing is
 * allocated.  Graphs need about n * 28 bytes per in-flight sample, so n must
 * satisfy n * 28 <= KADABRA_STATIC_SCRATCH_BYTES - 256 - 1280 (else
 * KADABRA_ERR_INVALID_ARG),
 * and fewer samples run in parallel as n grows.
 * Set-up: CUDA loads device code lazily, and the array is reserved on a
 * device only when its code is first loaded there.  kadabra_graph_load does
 * that set-up on the graph's device (it looks up the array's address, which
 * loads the code and reserves the 64 MiB), so a call here with a loaded graph
 * neither loads code nor reserves memory.  Each call looks the address up
 * again (cheap once loaded).  All calls share the array and each call clears
 * the part it uses before it samples: calls that overlap on the GPU race and
 * must be serialised by the caller.
 * count must be in [0, 2^32).  Synchronises `cuda_stream` and reports device
 * errors. */
kadabra_status kadabra_sample_static(const kadabra_graph *g, uint64_t seed, int tag, uint64_t first, int64_t count,
                                     uint32_t *counts, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* KADABRA_H */
