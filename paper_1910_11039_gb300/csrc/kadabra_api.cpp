// Host side of the C ABI declared in include/kadabra.h.
//
// Phase 1 (diameter -> omega) and the calibration arithmetic of phase 2 run
// here on the host in IEEE double (built with -ffp-contract=off); the
// sampling, the stop check and the result run in the kernels of
// sample_kernel.cu and check_kernel.cu (arXiv 1910.11039, Section III-A).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <unordered_map>
#include <vector>

#include <cuda_runtime.h>

#include <chrono>

#include <nvtx3/nvToolsExt.h>

#include "kadabra.h"
#include "kadabra_internal.h"

using kadabra::Job;

namespace {

thread_local std::string g_last_error;

kadabra_status fail(kadabra_status st, const std::string &msg)
{
    g_last_error = msg;
    return st;
}

kadabra_status cuda_fail(cudaError_t e, const char *what)
{
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return fail(KADABRA_ERR_OOM, m);
    if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return fail(KADABRA_ERR_NO_DEVICE, m);
    return fail(KADABRA_ERR_CUDA, m);
}

#define KCUDA(call, what)                      \
    do {                                       \
        cudaError_t _e = (call);               \
        if (_e != cudaSuccess) return cuda_fail(_e, what); \
    } while (0)

int bitlen64(uint64_t x)
{
    int b = 0;
    while (x) {
        ++b;
        x >>= 1;
    }
    return b;
}

cudaStream_t as_stream(void *s) { return reinterpret_cast<cudaStream_t>(s); }

}  // namespace

struct kadabra_graph {
    int64_t n = 0, nnz = 0, max_degree = 0;
    int off64 = 0;
    void *d_off = nullptr;
    uint2 *d_adj = nullptr;       // (neighbour, neighbour degree) per adjacency entry
    // sampling scratch shared by the graph's queries
    kadabra::SlotSet ws;          // one slot per CTA
    kadabra::SlotSet spill;       // full-capacity slots for samples that outgrow ws.cap
    int ws_threads = 0;
    int ws_req = 0;               // slots requested when the scratch was sized
    int64_t ws_cap_req = 0;       // queue capacity requested when the scratch was sized
    int probe_log2 = 0;           // probe bitmap of launches with ws_threads threads (0: none)
    void *d_help = nullptr;       // help board of the graph's pipelined launches
};

struct kadabra_query {
    kadabra_graph *g = nullptr;
    kadabra_params p{};
    double omega = 0.0;
    uint64_t omega_ceil = 0;
    int64_t vd = 0;
    int vd_exact = 0;
    int64_t vd_searches = 0;
    int64_t n_calib = 0;
    int K = 0;
    double balance_C = 0.0;
    int slots = 0;
    int threads = 256;
    uint32_t *d_counts = nullptr;
    uint32_t *d_cal = nullptr;
    double2 *d_L = nullptr;
    double *d_btilde = nullptr;
    Job *d_job = nullptr;       // adaptive stream
    Job *d_cal_job = nullptr;   // calibration stream
    Job *d_trace_job = nullptr; // trace runs
    // launch log: event pair, grid and device counters per sampling launch
    cudaEvent_t ev0[kadabra::kLaunchLog] = {};
    cudaEvent_t ev1[kadabra::kLaunchLog] = {};
    int grid_log[kadabra::kLaunchLog] = {};
    kadabra::Counters *d_launch = nullptr;   // kLaunchLog entries
    int64_t launches = 0;
    // budget classes: vertices with equal (L_L, L_U)
    uint32_t *d_cls = nullptr;               // class of every vertex
    double2 *d_Ltab = nullptr;               // budgets of every class
    unsigned int *d_cmax = nullptr;          // largest c~ per class (pipelined launches)
    int nclass = 0;
    // pipelined adaptive phase
    uint32_t *d_logs = nullptr;              // epoch logs of interior vertices
    size_t logs_alloc = 0;                   // entries allocated
    kadabra::PipeState *d_pipe = nullptr;
    kadabra::QueryDesc *d_desc = nullptr;    // descriptor for single-query launches
    kadabra::BatchState *d_bs = nullptr;
    bool pipe_begun = false;
    int phase = 0;                           // 0 created, 1 calibrating in a batch, 2 calibrated
    double diameter_ms = 0.0;                // host wall time of phase 1 (diameter bound, omega)
    double calibration_ms = 0.0;             // host wall time of phase 2 (samples and budgets)
    int64_t pipe_E = 0;
    int pipe_F = 0;
    unsigned int pipe_cap = 0;
    // captured epochs (kadabra_run_graph)
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t graph_exec = nullptr;
    int64_t graph_E = 0;
    int graph_k = 0;
};

struct kadabra_batch {
    int64_t max_n = 0;
    int slots = 0, threads = 0, off64 = 0;
    kadabra::SlotSet ws;
    kadabra::SlotSet spill;
    int probe_log2 = 0;           // probe bitmap of the batch's launches (0: none)
    void *d_help = nullptr;       // help board of the batch's launches
    kadabra::QueryDesc *d_descs = nullptr;
    int64_t descs_cap = 0;
    kadabra::BatchState *d_bs = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    bool have_step = false;
    int policy = 0;
    int64_t last_count = 0;       // queries of the most recent step
    int *d_states = nullptr;      // descs_cap entries
    uint64_t spin_limit = 1ULL << 24;
};

namespace kadabra {

namespace {
constexpr long long kMaxCap = (1LL << 31) - 2;   // queue positions must fit the code word
size_t align256(size_t b) { return (b + 255) & ~size_t(255); }
}  // namespace

size_t slot_set_bytes(int count, long long stride, long long cap, bool bits, bool lock)
{
    const size_t c = (size_t)(count > 0 ? count : 0);
    size_t b = align256(c * (size_t)stride * 4);                          // code
    b += align256(c * (size_t)cap * 4) * 2;                               // qv, ql
    b += align256(c * (size_t)cap * 8) * 2;                               // qs, qm
    if (bits) b += align256(c * 2 * (size_t)bit_words(stride) * 4);       // reached bits
    if (lock) b += align256(c * sizeof(int));
    return b;
}

void free_slot_set(SlotSet *S)
{
    cudaFree(S->code);
    cudaFree(S->qv);
    cudaFree(S->ql);
    cudaFree(S->qs);
    cudaFree(S->qm);
    cudaFree(S->bits);
    cudaFree(S->lock);
    *S = SlotSet{};
}

cudaError_t alloc_slot_set(SlotSet *S, int count, long long stride, long long cap, bool bits, bool lock)
{
    *S = SlotSet{};
    if (count <= 0) return cudaSuccess;
    const size_t c = (size_t)count;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&S->code), c * (size_t)stride * 4);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&S->qv), c * (size_t)cap * 4);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&S->ql), c * (size_t)cap * 4);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&S->qs), c * (size_t)cap * 8);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&S->qm), c * (size_t)cap * 8);
    if (e == cudaSuccess && bits) e = cudaMalloc(reinterpret_cast<void **>(&S->bits), c * 2 * (size_t)bit_words(stride) * 4);
    if (e == cudaSuccess && lock) e = cudaMalloc(reinterpret_cast<void **>(&S->lock), c * sizeof(int));
    // the sampler relies on all-zero code words, counts, bits and locks at rest
    if (e == cudaSuccess) e = cudaMemset(S->code, 0, c * (size_t)stride * 4);
    if (e == cudaSuccess) e = cudaMemset(S->qs, 0, c * (size_t)cap * 8);
    if (e == cudaSuccess) e = cudaMemset(S->qm, 0, c * (size_t)cap * 8);
    if (e == cudaSuccess && bits) e = cudaMemset(S->bits, 0, c * 2 * (size_t)bit_words(stride) * 4);
    if (e == cudaSuccess && lock) e = cudaMemset(S->lock, 0, c * sizeof(int));
    if (e != cudaSuccess) {
        free_slot_set(S);
        return e;
    }
    S->stride = stride;
    S->cap = cap;
    S->count = count;
    return cudaSuccess;
}

// How many slots of what queue capacity fit `budget` bytes for graphs of up
// to `stride` vertices.  Full capacity (cap = stride) when `want` such slots
// fit; otherwise two full-capacity spill slots and `want` slots whose queue
// capacity uses the rest (at least 2^16 positions; fewer slots if even that
// does not fit).  cap_req > 0 forces that capacity (spill slots whenever it
// is below stride).
void plan_slots(long long stride, int want, size_t budget, long long cap_req, int *slots, long long *cap, int *nspill)
{
    const long long full = stride < kMaxCap ? stride : kMaxCap;
    long long c = full;
    if (cap_req > 0) {
        c = cap_req < full ? cap_req : full;
        if (c < 2) c = 2;
    } else if ((size_t)want * slot_set_bytes(1, stride, full, true, false) > budget) {
        const size_t spill_b = 2 * slot_set_bytes(1, stride, full, true, true);
        const size_t rest = budget > spill_b ? budget - spill_b : 0;
        const size_t fixed = slot_set_bytes(1, stride, 0, true, false);
        const size_t per = rest / (size_t)(want > 0 ? want : 1);
        long long fit = per > fixed ? (long long)((per - fixed) / 24) : 0;
        const long long floor_cap = full < (1LL << 16) ? full : (1LL << 16);
        c = fit < floor_cap ? floor_cap : (fit < full ? fit : full);
    }
    const int ns = c < full ? 2 : 0;
    const size_t spill_b = ns ? (size_t)ns * slot_set_bytes(1, stride, full, true, true) : 0;
    const size_t avail = budget > spill_b ? budget - spill_b : 0;
    const size_t per = slot_set_bytes(1, stride, c, true, false);
    const size_t fit = per ? avail / per : (size_t)want;
    *slots = (int)((size_t)want < fit ? (size_t)want : fit);
    *cap = c;
    *nspill = ns;
}

bool graph_view(const kadabra_graph *g, GraphView *out)
{
    if (!g || !out) return false;
    out->n = g->n;
    out->nnz = g->nnz;
    out->max_degree = g->max_degree;
    out->off64 = g->off64;
    out->off = g->d_off;
    out->adj = g->d_adj;
    return true;
}

int set_last_error(int status, const char *msg)
{
    g_last_error = msg;
    return status;
}

}  // namespace kadabra

// ---------------------------------------------------------------------------
// errors, version, params
// ---------------------------------------------------------------------------

extern "C" const char *kadabra_last_error(void) { return g_last_error.c_str(); }

extern "C" const char *kadabra_status_string(kadabra_status s)
{
    switch (s) {
    case KADABRA_OK: return "KADABRA_OK";
    case KADABRA_ERR_INVALID_ARG: return "KADABRA_ERR_INVALID_ARG";
    case KADABRA_ERR_OOM: return "KADABRA_ERR_OOM";
    case KADABRA_ERR_CUDA: return "KADABRA_ERR_CUDA";
    case KADABRA_ERR_SIGMA_OVERFLOW: return "KADABRA_ERR_SIGMA_OVERFLOW";
    case KADABRA_ERR_COUNTER_OVERFLOW: return "KADABRA_ERR_COUNTER_OVERFLOW";
    case KADABRA_ERR_TIMEOUT: return "KADABRA_ERR_TIMEOUT";
    case KADABRA_ERR_STATE: return "KADABRA_ERR_STATE";
    case KADABRA_ERR_NO_DEVICE: return "KADABRA_ERR_NO_DEVICE";
    case KADABRA_ERR_DEPTH: return "KADABRA_ERR_DEPTH";
    }
    return "KADABRA_ERR_UNKNOWN";
}

extern "C" int kadabra_abi_version(void) { return 100; }

extern "C" void kadabra_params_default(kadabra_params *p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->eps = 0.01;
    p->delta = 0.1;
    p->seed = 1;
    p->vertex_diameter = 0;
    p->n_calib = 0;
    p->delta_rule = KADABRA_DELTA_BALANCED;
    p->flags = 0;
    p->beta = 1e-3;
    p->slots = 0;
    p->threads = 1024;
    p->scratch_fraction = 0.6;
}

// ---------------------------------------------------------------------------
// host utilities
// ---------------------------------------------------------------------------

template <typename OffT>
static kadabra_status validate(int64_t n, int64_t nnz, const OffT *off, const int32_t *col)
{
    if (n < 1 || n >= (int64_t(1) << 31)) return fail(KADABRA_ERR_INVALID_ARG, "n must be in [1, 2^31)");
    if (nnz < 0) return fail(KADABRA_ERR_INVALID_ARG, "nnz must be >= 0");
    if (!off || (nnz > 0 && !col)) return fail(KADABRA_ERR_INVALID_ARG, "null CSR array");
    if ((int64_t)off[0] != 0) return fail(KADABRA_ERR_INVALID_ARG, "offsets[0] != 0");
    if ((int64_t)off[n] != nnz) return fail(KADABRA_ERR_INVALID_ARG, "offsets[n] != nnz");
    for (int64_t v = 0; v < n; ++v) {
        const int64_t b = (int64_t)off[v], e = (int64_t)off[v + 1];
        if (e < b) return fail(KADABRA_ERR_INVALID_ARG, "offsets not non-decreasing at vertex " + std::to_string(v));
        for (int64_t i = b; i < e; ++i) {
            const int64_t w = col[i];
            if (w < 0 || w >= n) return fail(KADABRA_ERR_INVALID_ARG, "neighbour id out of range at vertex " + std::to_string(v));
            if (w == v) return fail(KADABRA_ERR_INVALID_ARG, "self-loop at vertex " + std::to_string(v));
            if (i > b && col[i - 1] >= w)
                return fail(KADABRA_ERR_INVALID_ARG, "neighbour list not strictly ascending at vertex " + std::to_string(v));
        }
    }
    // symmetry: every (v, w) has (w, v), found by binary search in w's row
    for (int64_t v = 0; v < n; ++v) {
        for (int64_t i = (int64_t)off[v]; i < (int64_t)off[v + 1]; ++i) {
            const int64_t w = col[i];
            int64_t lo = (int64_t)off[w], hi = (int64_t)off[w + 1];
            while (lo < hi) {
                const int64_t mid = (lo + hi) / 2;
                if (col[mid] < v) lo = mid + 1;
                else hi = mid;
            }
            if (lo == (int64_t)off[w + 1] || col[lo] != v)
                return fail(KADABRA_ERR_INVALID_ARG, "CSR not symmetric: edge " + std::to_string(v) + "->" +
                                                         std::to_string(w) + " has no reverse");
        }
    }
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_device_clock(uint64_t *ns, void *cuda_stream)
{
    if (!ns) return fail(KADABRA_ERR_INVALID_ARG, "ns is null");
    unsigned long long v = 0;
    KCUDA(kadabra::read_device_clock(&v, as_stream(cuda_stream)), "device clock");
    *ns = v;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_validate_csr(int64_t n, int64_t nnz, const void *offsets, int offsets_is_64,
                                               const int32_t *cols)
{
    if (offsets_is_64) return validate(n, nnz, static_cast<const int64_t *>(offsets), cols);
    if (nnz >= (int64_t(1) << 31)) return fail(KADABRA_ERR_INVALID_ARG, "nnz too large for int32 offsets");
    return validate(n, nnz, static_cast<const int32_t *>(offsets), cols);
}

extern "C" kadabra_status kadabra_omega(double eps, double delta, int64_t vertex_diameter, double *omega)
{
    if (!omega) return fail(KADABRA_ERR_INVALID_ARG, "omega is null");
    if (!(eps > 0.0 && eps < 1.0) || !(delta > 0.0 && delta < 1.0)) {
        *omega = NAN;
        return fail(KADABRA_ERR_INVALID_ARG, "eps and delta must lie in (0, 1)");
    }
    int64_t x = vertex_diameter - 2;
    if (x < 1) x = 1;
    const int floor_log2 = bitlen64((uint64_t)x) - 1;
    *omega = (0.5 / (eps * eps)) * ((double)floor_log2 + 1.0 + std::log(2.0 / delta));
    return KADABRA_OK;
}

extern "C" int kadabra_sigma_bits(int64_t n, int64_t max_degree)
{
    const int a = 63 - bitlen64((uint64_t)max_degree);
    const int b = 63 - bitlen64((uint64_t)n);
    return a < b ? a : b;
}

// delta_L / delta_U -> L = -ln(delta).  Balanced rule: bisection for C with
// sum_x exp(-C eps^2 / bhat(x)) <= (1 - beta) delta / 4 (bhat = cal / n_cal),
// delta_L = delta_U = exp(-C eps^2 / bhat) + beta delta / (4n).  Vertices with
// equal calibration counts have equal terms: the sum runs over the distinct
// counts in ascending order, weighted by how many vertices have each.  Both
// rules make the budgets a function of the calibration count, so the budget
// classes (equal (L_L, L_U)) are the distinct counts present (one class for
// the uniform rule); cls[x] receives the class of every vertex.
// Budget table from the number of vertices with each calibration count:
// class_of[c] (-1 where no vertex has count c) and (L_L, L_U) per class.
// Uniform rule: delta_L = delta_U = delta / (4n) for every vertex.  Balanced
// rule: delta_L = delta_U = exp(-C eps^2 / bhat) + beta delta / (4n) with
// bhat = c / n_cal, C found by bisection so that the variable terms sum to at
// most (1 - beta) delta / 4 (zero counts get the floor term alone).
static void budget_table(int64_t n, const std::vector<unsigned long long> &hist, int64_t n_cal, double eps,
                         double delta, int rule, double beta, std::vector<int32_t> &class_of,
                         std::vector<double2> &Ltab, double *C_out)
{
    const uint32_t cmax = (uint32_t)(hist.size() - 1);
    class_of.assign((size_t)cmax + 1, -1);
    Ltab.clear();
    if (rule == KADABRA_DELTA_UNIFORM) {
        const double dl = delta / (4.0 * (double)n);
        Ltab.push_back(make_double2(-std::log(dl), -std::log(dl)));
        for (auto &k : class_of) k = 0;
        *C_out = 0.0;
        return;
    }
    auto term = [&](double C, uint32_t c) {
        const double bhat = (double)c / (double)n_cal;
        return std::exp(-((C * (eps * eps)) / bhat));
    };
    const double budget = (1.0 - beta) * delta / 4.0;
    double lo = 0.0;
    double hi = std::log(4.0 * (double)n / ((1.0 - beta) * delta)) / (eps * eps);
    while (hi - lo > eps / 10.0) {
        const double mid = (lo + hi) / 2.0;
        double sum = 0.0;
        for (uint32_t c = 1; c <= cmax; ++c)
            if (hist[c]) sum += (double)hist[c] * term(mid, c);
        if (sum <= budget) hi = mid;
        else lo = mid;
    }
    const double C = hi;
    const double floor_term = beta * delta / (4.0 * (double)n);
    for (uint32_t c = 0; c <= cmax; ++c) {
        if (!hist[c]) continue;
        const double dl = c == 0 ? floor_term : term(C, c) + floor_term;
        class_of[c] = (int32_t)Ltab.size();
        Ltab.push_back(make_double2(-std::log(dl), -std::log(dl)));
    }
    *C_out = C;
}

// ---------------------------------------------------------------------------
// graph
// ---------------------------------------------------------------------------

static void free_graph_device(kadabra_graph *g)
{
    cudaFree(g->d_off);
    cudaFree(g->d_adj);
    kadabra::free_slot_set(&g->ws);
    kadabra::free_slot_set(&g->spill);
    cudaFree(g->d_help);
    g->d_off = nullptr;
    g->d_adj = nullptr;
    g->d_help = nullptr;
}

extern "C" kadabra_status kadabra_graph_load(int64_t n, int64_t nnz, const void *offsets, int offsets_is_64,
                                             const int32_t *cols, uint32_t flags, void *cuda_stream,
                                             kadabra_graph **out)
{
    if (!out) return fail(KADABRA_ERR_INVALID_ARG, "out is null");
    if (n < 1 || n >= (int64_t(1) << 31)) return fail(KADABRA_ERR_INVALID_ARG, "n must be in [1, 2^31)");
    if (nnz < 0 || !offsets || (nnz > 0 && !cols)) return fail(KADABRA_ERR_INVALID_ARG, "bad CSR arguments");
    if (!offsets_is_64 && nnz >= (int64_t(1) << 31))
        return fail(KADABRA_ERR_INVALID_ARG, "nnz too large for int32 offsets");
    const bool dev = (flags & KADABRA_GRAPH_DEVICE_PTRS) != 0;
    const size_t ob = (size_t)(n + 1) * (offsets_is_64 ? 8 : 4);
    const size_t cb = (size_t)nnz * 4;
    cudaStream_t st = as_stream(cuda_stream);

    kadabra_graph *g = new kadabra_graph();
    g->n = n;
    g->nnz = nnz;
    g->off64 = offsets_is_64 ? 1 : 0;
    // host-side checks (host inputs are read in place; device inputs are
    // copied to the host only when they are to be validated)
    if (!(flags & KADABRA_GRAPH_SKIP_VALIDATE)) {
        std::vector<unsigned char> off_raw;
        std::vector<int32_t> col_raw;
        const void *hoff = offsets;
        const int32_t *hcol = cols;
        if (dev) {
            off_raw.resize(ob);
            col_raw.resize((size_t)nnz);
            cudaError_t e = cudaMemcpyAsync(off_raw.data(), offsets, ob, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess && cb) e = cudaMemcpyAsync(col_raw.data(), cols, cb, cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) {
                delete g;
                return cuda_fail(e, "copy CSR to host for validation");
            }
            hoff = off_raw.data();
            hcol = col_raw.data();
        }
        kadabra_status s = kadabra_validate_csr(n, nnz, hoff, offsets_is_64, hcol);
        if (s != KADABRA_OK) {
            delete g;
            return s;
        }
    }
    // device copy: offsets, and the adjacency as (neighbour, neighbour degree)
    // pairs built on the device from the columns; host columns in page-locked
    // memory are read in place by that kernel (one pass over the host link),
    // other host columns go through a temporary device copy.  The maximum
    // degree is reduced on the device from the copied offsets.
    const int32_t *cols_in = dev ? cols : nullptr;
    if (!dev && cb) {
        cudaPointerAttributes pa{};
        if (cudaPointerGetAttributes(&pa, cols) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer)
            cols_in = static_cast<const int32_t *>(pa.devicePointer);
        else
            cudaGetLastError();     // pageable memory: clear the query's error, if any
    }
    int32_t *d_cols_tmp = nullptr;
    uint32_t *d_deg = nullptr;
    cudaError_t e = cudaMalloc(&g->d_off, ob);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&g->d_adj), (size_t)(nnz > 0 ? nnz : 1) * sizeof(uint2));
    if (e == cudaSuccess && cb) e = cudaMalloc(reinterpret_cast<void **>(&d_deg), (size_t)n * sizeof(uint32_t));
    if (e == cudaSuccess && !cols_in && cb) e = cudaMalloc(reinterpret_cast<void **>(&d_cols_tmp), cb);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(g->d_off, offsets, ob, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && d_cols_tmp) {
        e = cudaMemcpyAsync(d_cols_tmp, cols, cb, cudaMemcpyHostToDevice, st);
        cols_in = d_cols_tmp;
    }
    if (e == cudaSuccess)
        e = kadabra::launch_build_adj(n, nnz, g->d_off, g->off64, cols_in, g->d_adj, d_deg, st);
    unsigned long long *d_md = nullptr;
    unsigned long long md = 0;
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&d_md), sizeof(unsigned long long));
    if (e == cudaSuccess) e = kadabra::launch_max_degree(n, g->d_off, g->off64, d_md, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&md, d_md, sizeof(md), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    g->max_degree = (int64_t)md;
    cudaFree(d_md);
    cudaFree(d_cols_tmp);
    cudaFree(d_deg);
    // reserve kadabra_sample_static's array on this device now, so that
    // sampling from this graph there later loads and reserves nothing
    if (e == cudaSuccess) e = kadabra::static_scratch_reserve();
    if (e != cudaSuccess) {
        free_graph_device(g);
        delete g;
        return cuda_fail(e, "upload CSR");
    }
    *out = g;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_graph_free(kadabra_graph *g)
{
    if (!g) return KADABRA_OK;
    cudaDeviceSynchronize();
    free_graph_device(g);
    delete g;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_graph_info(const kadabra_graph *g, int64_t *n, int64_t *nnz, int64_t *max_degree,
                                             int *offsets_is_64)
{
    if (!g) return fail(KADABRA_ERR_INVALID_ARG, "graph is null");
    if (n) *n = g->n;
    if (nnz) *nnz = g->nnz;
    if (max_degree) *max_degree = g->max_degree;
    if (offsets_is_64) *offsets_is_64 = g->off64;
    return KADABRA_OK;
}

// Sampling scratch of the graph: per slot one code word per vertex, two
// reached-bit maps and a queue of `cap` positions (24 B each); see SlotSet.
static kadabra_status ensure_workspace(kadabra_graph *g, int want_slots, int threads, double fraction, int64_t cap_req)
{
    int dev = 0, sms = 0, per_sm = 0;
    KCUDA(cudaGetDevice(&dev), "cudaGetDevice");
    KCUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    KCUDA(kadabra::sample_occupancy(threads, g->off64, &per_sm), "occupancy");
    if (per_sm < 1) per_sm = 1;
    const int requested = want_slots > 0 ? want_slots : sms * per_sm;
    if (g->ws.count && g->ws_threads == threads && g->ws_cap_req == cap_req &&
        (g->ws.count >= requested || g->ws_req == requested))
        return KADABRA_OK;
    cudaDeviceSynchronize();
    kadabra::free_slot_set(&g->ws);
    kadabra::free_slot_set(&g->spill);
    size_t free_b = 0, total_b = 0;
    KCUDA(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
    if (fraction <= 0.0 || fraction > 0.95) fraction = 0.6;
    const size_t budget = (size_t)((double)free_b * fraction);
    int slots = 0, nspill = 0;
    long long cap = 0;
    kadabra::plan_slots(g->n, requested, budget, cap_req, &slots, &cap, &nspill);
    if (slots < 1) return fail(KADABRA_ERR_OOM, "not enough device memory for one sampling slot");
    cudaError_t e = kadabra::alloc_slot_set(&g->ws, slots, g->n, cap, true, false);
    if (e == cudaSuccess) e = kadabra::alloc_slot_set(&g->spill, nspill, g->n, g->n, true, true);
    if (e != cudaSuccess) {
        kadabra::free_slot_set(&g->ws);
        kadabra::free_slot_set(&g->spill);
        return cuda_fail(e, "allocate sampling scratch");
    }
    g->ws_threads = threads;
    g->ws_req = requested;
    g->ws_cap_req = cap_req;
    KCUDA(kadabra::probe_prepare(threads, g->off64, per_sm, &g->probe_log2), "probe bitmap set-up");
    return KADABRA_OK;
}

// ---------------------------------------------------------------------------
// query
// ---------------------------------------------------------------------------

static void free_query_device(kadabra_query *q)
{
    cudaFree(q->d_counts);
    cudaFree(q->d_cal);
    cudaFree(q->d_L);
    cudaFree(q->d_btilde);
    cudaFree(q->d_job);
    cudaFree(q->d_cal_job);
    cudaFree(q->d_trace_job);
    cudaFree(q->d_launch);
    cudaFree(q->d_cls);
    cudaFree(q->d_Ltab);
    cudaFree(q->d_cmax);
    cudaFree(q->d_logs);
    cudaFree(q->d_pipe);
    cudaFree(q->d_desc);
    cudaFree(q->d_bs);
    if (q->graph_exec) cudaGraphExecDestroy(q->graph_exec);
    if (q->cap_stream) cudaStreamDestroy(q->cap_stream);
    for (int i = 0; i < kadabra::kLaunchLog; ++i) {
        if (q->ev0[i]) cudaEventDestroy(q->ev0[i]);
        if (q->ev1[i]) cudaEventDestroy(q->ev1[i]);
    }
}

static kadabra_status device_error_status(const Job &j)
{
    if (j.error & kadabra::kErrSigmaOverflow)
        return fail(KADABRA_ERR_SIGMA_OVERFLOW, "strict mode: a per-side path count exceeded 2^K");
    if (j.error & kadabra::kErrCounterOverflow) return fail(KADABRA_ERR_COUNTER_OVERFLOW, "a 32-bit counter wrapped");
    if (j.error & kadabra::kErrLogOverflow)
        return fail(KADABRA_ERR_INVALID_ARG, "a sampled path had more interior vertices than VD - 2 (vertex diameter bound too small)");
    if (j.error & kadabra::kErrTimeout)
        return fail(KADABRA_ERR_TIMEOUT, "a pipelined launch gave up waiting for a free counter frame");
    if (j.error & kadabra::kErrScratch)
        return fail(KADABRA_ERR_OOM, "a sample outgrew its slot's queue and no spill slot was available");
    if (j.error & (kadabra::kErrAddOverflow | kadabra::kErrSelect))
        return fail(KADABRA_ERR_CUDA, "internal sampling invariant violated (error bits " + std::to_string(j.error) + ")");
    return KADABRA_OK;
}

// frontier degree sum from which a small-diameter sample probes a layer
static unsigned long long probe_edges_of(const kadabra_params &p)
{
    return p.probe_edges > 0 ? (unsigned long long)p.probe_edges : 256ULL;
}

// probe bitmap of a launch of this query (sized for the threads the graph's
// scratch was planned with; none if the query asks for no probing)
static int probe_log2_of(const kadabra_query *q)
{
    return (q->p.probe_edges >= 0 && q->threads == q->g->ws_threads) ? q->g->probe_log2 : 0;
}

static kadabra::SampleLaunch base_launch(const kadabra_query *q)
{
    kadabra::SampleLaunch a{};
    a.n = q->g->n;
    a.off = q->g->d_off;
    a.off64 = q->g->off64;
    a.adj = q->g->d_adj;
    a.slots = q->g->ws;
    a.spill = q->g->spill;
    a.use_bits = q->vd <= kadabra::kBitsMaxVD ? 1 : 0;
    a.probe_log2 = a.use_bits ? probe_log2_of(q) : 0;
    a.probe_edges = probe_edges_of(q->p);
    a.spin_limit = 1ULL << 24;
    a.seed = q->p.seed;
    a.K = q->K;
    a.strict = (q->p.flags & KADABRA_STRICT_SIGMA) ? 1 : 0;
    a.threads = q->threads;
    return a;
}

// Never launch more CTAs than the graph's scratch has slots (another query
// may have re-sized it), nor more than there are samples.
static int clamp_grid(const kadabra_query *q, int64_t count)
{
    int64_t g = q->slots < q->g->ws.count ? q->slots : q->g->ws.count;
    if (count < g) g = count;
    return (int)g;
}

// An NVTX range (visible to Nsight tools, free otherwise) that also measures
// its host wall time.
struct PhaseScope {
    std::chrono::steady_clock::time_point t0;
    double *out;
    PhaseScope(const char *name, double *ms) : t0(std::chrono::steady_clock::now()), out(ms) { nvtxRangePushA(name); }
    ~PhaseScope()
    {
        nvtxRangePop();
        if (out) *out = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    }
};

// Phase 1 and the query's device state; no sampling yet.
static kadabra_status create_query(kadabra_graph *g, const kadabra_params *pin, cudaStream_t st, kadabra_query **out)
{
    if (!g || !out) return fail(KADABRA_ERR_INVALID_ARG, "graph or out is null");
    kadabra_params p;
    if (pin) p = *pin;
    else kadabra_params_default(&p);
    if (!(p.eps > 0.0 && p.eps < 1.0) || !(p.delta > 0.0 && p.delta < 1.0))
        return fail(KADABRA_ERR_INVALID_ARG, "eps and delta must lie in (0, 1)");
    if (p.delta_rule != KADABRA_DELTA_UNIFORM && p.delta_rule != KADABRA_DELTA_BALANCED)
        return fail(KADABRA_ERR_INVALID_ARG, "unknown delta_rule");
    if (!(p.beta > 0.0 && p.beta < 1.0)) return fail(KADABRA_ERR_INVALID_ARG, "beta must lie in (0, 1)");
    if (p.threads == 0) p.threads = 1024;
    if (p.threads != 128 && p.threads != 256 && p.threads != 512 && p.threads != 1024)
        return fail(KADABRA_ERR_INVALID_ARG, "threads must be 128, 256, 512 or 1024");
    if (g->n < 2) return fail(KADABRA_ERR_INVALID_ARG, "sampling pairs needs n >= 2");

    kadabra_query *q = new kadabra_query();
    q->g = g;
    q->p = p;
    q->threads = p.threads;
    q->K = kadabra_sigma_bits(g->n, g->max_degree);
    // phase 1: diameter -> omega
    PhaseScope scope("kadabra: diameter phase", &q->diameter_ms);
    if (p.vertex_diameter > 0) {
        q->vd = p.vertex_diameter;
        q->vd_exact = 0;
    } else if (p.vertex_diameter == -1) {
        // exact vertex diameter: iFUB on the device for the largest component
        void *scratch = nullptr;
        cudaError_t e = cudaMalloc(&scratch, kadabra::vd_exact_scratch_bytes(g->n));
        if (e == cudaSuccess)
            e = kadabra::launch_vd_exact(g->n, g->d_off, g->off64, g->d_adj, scratch, st, &q->vd, &q->vd_exact,
                                         &q->vd_searches);
        cudaFree(scratch);
        if (e != cudaSuccess) {
            delete q;
            if (e == cudaErrorLaunchTimeout)
                return fail(KADABRA_ERR_TIMEOUT, "diameter phase: a bounded device wait gave up");
            return cuda_fail(e, "diameter phase (exact)");
        }
    } else if (p.vertex_diameter < -1) {
        delete q;
        return fail(KADABRA_ERR_INVALID_ARG, "vertex_diameter must be >= 0 or -1 (exact)");
    } else {
        q->vd_searches = 1;
        // vertex-diameter bound on the device (union-find components, then one
        // breadth-first search from every component's smallest vertex)
        void *scratch = nullptr;
        cudaError_t e = cudaMalloc(&scratch, kadabra::vd_bound_scratch_bytes(g->n));
        if (e == cudaSuccess) e = kadabra::launch_vd_bound(g->n, g->d_off, g->off64, g->d_adj, scratch, st, &q->vd);
        cudaFree(scratch);
        if (e != cudaSuccess) {
            delete q;
            if (e == cudaErrorLaunchTimeout)
                return fail(KADABRA_ERR_TIMEOUT, "diameter phase: a bounded device wait gave up");
            return cuda_fail(e, "diameter phase");
        }
    }
    kadabra_omega(p.eps, p.delta, q->vd, &q->omega);
    q->omega_ceil = (uint64_t)std::ceil(q->omega);
    if (q->omega_ceil >= (uint64_t(1) << 32)) {
        delete q;
        return fail(KADABRA_ERR_INVALID_ARG, "omega >= 2^32: counters are 32-bit");
    }
    q->n_calib = p.n_calib;
    if (q->n_calib <= 0) {
        q->n_calib = (int64_t)std::ceil(q->omega / 100.0);
        if (q->n_calib < 1000) q->n_calib = 1000;
    }
    if (q->n_calib >= (int64_t(1) << 32)) {
        delete q;
        return fail(KADABRA_ERR_INVALID_ARG, "n_calib must be < 2^32");
    }

    const size_t n = (size_t)g->n;
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&q->d_counts), n * 4);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&q->d_cal), n * 4);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&q->d_L), n * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&q->d_btilde), n * sizeof(double));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&q->d_job), sizeof(Job));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&q->d_cal_job), sizeof(Job));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&q->d_trace_job), sizeof(Job));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&q->d_cls), n * 4);
    if (e == cudaSuccess)
        e = cudaMalloc(reinterpret_cast<void **>(&q->d_launch), sizeof(kadabra::Counters) * kadabra::kLaunchLog);
    if (e == cudaSuccess) e = cudaMemsetAsync(q->d_counts, 0, n * 4, st);
    if (e == cudaSuccess) e = cudaMemsetAsync(q->d_cal, 0, n * 4, st);
    if (e == cudaSuccess) e = kadabra::launch_reset_job(q->d_job, st);
    if (e == cudaSuccess) e = kadabra::launch_reset_job(q->d_cal_job, st);
    if (e == cudaSuccess) e = kadabra::launch_reset_job(q->d_trace_job, st);
    if (e != cudaSuccess) {
        free_query_device(q);
        delete q;
        return cuda_fail(e, "allocate query state");
    }
    *out = q;
    return KADABRA_OK;
}

// Event pair of launch-log slot `slot`, created on first use.
static kadabra_status slot_events(kadabra_query *q, int slot)
{
    if (!q->ev0[slot]) KCUDA(cudaEventCreate(&q->ev0[slot]), "create event");
    if (!q->ev1[slot]) KCUDA(cudaEventCreate(&q->ev1[slot]), "create event");
    return KADABRA_OK;
}

// Sampling scratch of the graph for launches that serve this query alone.
static kadabra_status ready_workspace(kadabra_query *q)
{
    kadabra_status s = ensure_workspace(q->g, q->p.slots, q->p.threads, q->p.scratch_fraction, q->p.queue_cap);
    if (s != KADABRA_OK) return s;
    q->slots = q->p.slots > 0 && q->p.slots < q->g->ws.count ? q->p.slots : q->g->ws.count;
    return KADABRA_OK;
}

// Phase 2: budgets from the calibration counts.  The device reduces the
// counts to a histogram, the host runs the budget rule on it, the device
// gives every vertex its class's budgets.  Synchronises.
static kadabra_status finish_calibration(kadabra_query *q, cudaStream_t st)
{
    const int64_t n = q->g->n;
    Job cj{};
    KCUDA(cudaMemcpyAsync(&cj, q->d_cal_job, sizeof(Job), cudaMemcpyDeviceToHost, st), "read calibration state");
    unsigned int *d_mx = nullptr;
    KCUDA(cudaMalloc(reinterpret_cast<void **>(&d_mx), sizeof(unsigned int)), "allocate");
    unsigned int cmax = 0;
    cudaError_t e = kadabra::launch_cal_max(n, q->d_cal, d_mx, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&cmax, d_mx, sizeof(cmax), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_mx);
    if (e != cudaSuccess) return cuda_fail(e, "calibration counts");
    kadabra_status s = device_error_status(cj);
    if (s != KADABRA_OK) return s;
    std::vector<unsigned long long> hist((size_t)cmax + 1, 0ULL);
    unsigned long long *d_hist = nullptr;
    KCUDA(cudaMalloc(reinterpret_cast<void **>(&d_hist), hist.size() * sizeof(unsigned long long)), "allocate");
    e = kadabra::launch_cal_hist(n, q->d_cal, cmax, d_hist, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(hist.data(), d_hist, hist.size() * sizeof(unsigned long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_hist);
    if (e != cudaSuccess) return cuda_fail(e, "calibration histogram");
    std::vector<int32_t> class_of;
    std::vector<double2> Ltab;
    budget_table(n, hist, q->n_calib, q->p.eps, q->p.delta, q->p.delta_rule, q->p.beta, class_of, Ltab,
                 &q->balance_C);
    cudaFree(q->d_Ltab);
    cudaFree(q->d_cmax);
    q->d_Ltab = nullptr;
    q->d_cmax = nullptr;
    q->nclass = (int)Ltab.size();
    int *d_class_of = nullptr;
    e = cudaMalloc(reinterpret_cast<void **>(&q->d_Ltab), Ltab.size() * sizeof(double2));
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&q->d_cmax), Ltab.size() * 4);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&d_class_of), class_of.size() * sizeof(int32_t));
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(q->d_Ltab, Ltab.data(), Ltab.size() * sizeof(double2), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d_class_of, class_of.data(), class_of.size() * sizeof(int32_t), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = kadabra::launch_fill_budgets(n, q->d_cal, d_class_of, q->d_Ltab, q->d_cls, q->d_L, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_class_of);
    if (e != cudaSuccess) return cuda_fail(e, "budgets");
    q->phase = 2;
    q->pipe_begun = false;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_calibrate(kadabra_graph *g, const kadabra_params *pin, void *cuda_stream,
                                            kadabra_query **out)
{
    cudaStream_t st = as_stream(cuda_stream);
    kadabra_query *q = nullptr;
    kadabra_status s = create_query(g, pin, st, &q);
    if (s != KADABRA_OK) return s;
    s = ready_workspace(q);
    if (s != KADABRA_OK) {
        free_query_device(q);
        delete q;
        return s;
    }
    PhaseScope scope("kadabra: calibration phase", &q->calibration_ms);
    // phase 2: calibration samples (stream tag 0) on the device
    kadabra::SampleLaunch a = base_launch(q);
    a.counts = q->d_cal;
    a.job = q->d_cal_job;
    a.tag = 0;
    a.use_stop = 0;
    a.epoch_len = q->n_calib;
    a.clip = 0;
    a.grid = clamp_grid(q, q->n_calib);
    const int slot = (int)(q->launches % kadabra::kLaunchLog);
    a.launch_ctr = q->d_launch + slot;
    s = slot_events(q, slot);
    cudaError_t e = s == KADABRA_OK ? cudaSuccess : cudaErrorMemoryAllocation;
    if (e == cudaSuccess) e = cudaMemsetAsync(a.launch_ctr, 0, sizeof(kadabra::Counters), st);
    if (e == cudaSuccess) e = cudaEventRecord(q->ev0[slot], st);
    if (e == cudaSuccess) e = kadabra::launch_sample(a, st);
    if (e == cudaSuccess) e = cudaEventRecord(q->ev1[slot], st);
    if (e == cudaSuccess) {
        q->grid_log[slot] = a.grid;
        ++q->launches;
    }
    if (e != cudaSuccess) {
        free_query_device(q);
        delete q;
        return cuda_fail(e, "calibration samples");
    }
    s = finish_calibration(q, st);
    if (s != KADABRA_OK) {
        free_query_device(q);
        delete q;
        return s;
    }
    *out = q;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_query_create(kadabra_graph *g, const kadabra_params *p, void *cuda_stream,
                                               kadabra_query **out)
{
    return create_query(g, p, as_stream(cuda_stream), out);
}

static kadabra_status ensure_pipe_state(kadabra_query *q)
{
    if (!q->d_pipe) KCUDA(cudaMalloc(reinterpret_cast<void **>(&q->d_pipe), sizeof(kadabra::PipeState)), "allocate pipeline state");
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_calibration_begin(kadabra_query *q, void *cuda_stream)
{
    if (!q) return fail(KADABRA_ERR_INVALID_ARG, "query is null");
    if (q->phase != 0) return fail(KADABRA_ERR_STATE, "query is already calibrating or calibrated");
    cudaStream_t st = as_stream(cuda_stream);
    kadabra_status s = ensure_pipe_state(q);
    if (s != KADABRA_OK) return s;
    KCUDA(cudaMemsetAsync(q->d_cal, 0, (size_t)q->g->n * 4, st), "clear calibration counts");
    KCUDA(kadabra::launch_reset_job(q->d_cal_job, st), "reset calibration state");
    // one epoch of n_calib samples, no check: the pipeline state only hands
    // out indices [0, n_calib) and counts completions
    KCUDA(kadabra::launch_pipe_begin(q->d_pipe, q->d_cal_job, (unsigned long long)q->n_calib, q->n_calib, st),
          "begin calibration");
    q->phase = 1;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_calibration_finish(kadabra_query *q, void *cuda_stream)
{
    if (!q) return fail(KADABRA_ERR_INVALID_ARG, "query is null");
    if (q->phase != 1) return fail(KADABRA_ERR_STATE, "query is not calibrating (kadabra_calibration_begin)");
    cudaStream_t st = as_stream(cuda_stream);
    kadabra::PipeState ps{};
    KCUDA(cudaMemcpyAsync(&ps, q->d_pipe, sizeof(ps), cudaMemcpyDeviceToHost, st), "read calibration progress");
    KCUDA(cudaStreamSynchronize(st), "synchronise");
    if (ps.done[0] < (unsigned int)q->n_calib) return fail(KADABRA_ERR_STATE, "calibration samples not complete");
    PhaseScope scope("kadabra: calibration budgets", &q->calibration_ms);
    return finish_calibration(q, st);
}

extern "C" kadabra_status kadabra_query_free(kadabra_query *q)
{
    if (!q) return KADABRA_OK;
    cudaDeviceSynchronize();
    free_query_device(q);
    delete q;
    return KADABRA_OK;
}

static kadabra_status need_calibrated(kadabra_query *q)
{
    if (!q) return fail(KADABRA_ERR_INVALID_ARG, "query is null");
    if (q->phase != 2) return fail(KADABRA_ERR_STATE, "query is not calibrated");
    return KADABRA_OK;
}

#define KREADY(q)                                          \
    do {                                                   \
        kadabra_status s_ = need_calibrated(q);            \
        if (s_ == KADABRA_OK) s_ = ready_workspace(q);     \
        if (s_ != KADABRA_OK) return s_;                   \
    } while (0)

extern "C" kadabra_status kadabra_sample_epoch(kadabra_query *q, int64_t n_samples, void *cuda_stream)
{
    KREADY(q);
    if (n_samples < 0 || n_samples >= (int64_t(1) << 32))
        return fail(KADABRA_ERR_INVALID_ARG, "n_samples must be in [0, 2^32)");
    if (n_samples == 0) return KADABRA_OK;
    cudaStream_t st = as_stream(cuda_stream);
    kadabra::SampleLaunch a = base_launch(q);
    a.counts = q->d_counts;
    a.job = q->d_job;
    a.tag = 1;
    a.use_stop = 1;
    a.epoch_len = n_samples;
    a.clip = q->omega_ceil;
    a.grid = clamp_grid(q, n_samples);
    const int slot = (int)(q->launches % kadabra::kLaunchLog);
    a.launch_ctr = q->d_launch + slot;
    KCUDA(cudaMemsetAsync(a.launch_ctr, 0, sizeof(kadabra::Counters), st), "reset launch counters");
    {
        kadabra_status se = slot_events(q, slot);
        if (se != KADABRA_OK) return se;
    }
    KCUDA(cudaEventRecord(q->ev0[slot], st), "event");
    KCUDA(kadabra::launch_sample(a, st), "sampling kernel launch");
    KCUDA(cudaEventRecord(q->ev1[slot], st), "event");
    q->grid_log[slot] = a.grid;
    ++q->launches;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_pipeline_begin(kadabra_query *q, int64_t epoch_len, int frames, void *cuda_stream)
{
    {
        kadabra_status s = need_calibrated(q);
        if (s != KADABRA_OK) return s;
    }
    if (epoch_len <= 0 || epoch_len >= (int64_t(1) << 40)) return fail(KADABRA_ERR_INVALID_ARG, "epoch_len out of range");
    if (frames <= 0) frames = 8;
    if (frames > kadabra::kMaxFrames) return fail(KADABRA_ERR_INVALID_ARG, "frames must be <= 16");
    cudaStream_t st = as_stream(cuda_stream);
    // an epoch logs at most (VD - 2) interior vertices per sample
    const uint64_t per_sample = q->vd > 3 ? (uint64_t)(q->vd - 2) : 1ULL;
    const uint64_t cap = (uint64_t)epoch_len * per_sample;
    if (cap >= (uint64_t(1) << 32)) return fail(KADABRA_ERR_INVALID_ARG, "epoch_len * (VD - 2) must be < 2^32");
    const size_t need = (size_t)frames * (size_t)cap;
    if (q->logs_alloc < need) {
        cudaFree(q->d_logs);
        q->d_logs = nullptr;
        q->logs_alloc = 0;
        KCUDA(cudaMalloc(reinterpret_cast<void **>(&q->d_logs), need * 4), "allocate epoch logs");
        q->logs_alloc = need;
    }
    {
        kadabra_status s = ensure_pipe_state(q);
        if (s != KADABRA_OK) return s;
    }
    KCUDA(kadabra::launch_pipe_begin(q->d_pipe, q->d_job, q->omega_ceil, epoch_len, st), "begin pipeline");
    // per-class maxima of the counters the pipeline starts from
    KCUDA(cudaMemsetAsync(q->d_cmax, 0, (size_t)q->nclass * 4, st), "clear class maxima");
    KCUDA(kadabra::launch_class_max(q->g->n, q->d_counts, q->d_cls, q->d_cmax, st), "class maxima");
    q->pipe_begun = true;
    q->pipe_E = epoch_len;
    q->pipe_F = frames;
    q->pipe_cap = (unsigned int)cap;
    return KADABRA_OK;
}

static kadabra::QueryDesc make_desc(const kadabra_query *q, kadabra::Counters *launch_ctr)
{
    kadabra::QueryDesc d{};
    d.n = q->g->n;
    d.off = q->g->d_off;
    d.adj = q->g->d_adj;
    d.K = q->K;
    d.strict = (q->p.flags & KADABRA_STRICT_SIGMA) ? 1 : 0;
    d.seed = q->p.seed;
    d.E = q->pipe_E;
    d.F = q->pipe_F;
    d.log_cap = q->pipe_cap;
    d.logs = q->d_logs;
    d.cls = q->d_cls;
    d.Ltab = q->d_Ltab;
    d.cmax = q->d_cmax;
    d.nclass = q->nclass;
    d.omega = q->omega;
    d.eps = q->p.eps;
    d.counts = q->d_counts;
    d.job = q->d_job;
    d.ps = q->d_pipe;
    d.launch_ctr = launch_ctr;
    d.use_bits = q->vd <= kadabra::kBitsMaxVD ? 1 : 0;
    d.lookahead = (q->p.flags & KADABRA_FULL_LOOKAHEAD) ? 0 : 1;
    d.tag = 1;
    if (q->phase == 1) {
        // calibration samples: one epoch of n_calib samples counted into the
        // calibration counters, no logs and no check
        d.tag = 0;
        d.E = q->n_calib;
        d.F = 1;
        d.log_cap = 0;
        d.logs = nullptr;
        d.counts = q->d_cal;
        d.job = q->d_cal_job;
    }
    return d;
}

extern "C" kadabra_status kadabra_run_pipelined(kadabra_query *q, int64_t epoch_len, int frames, void *cuda_stream)
{
    KREADY(q);
    PhaseScope scope("kadabra: pipelined adaptive phase (enqueue)", nullptr);
    kadabra_status s = kadabra_pipeline_begin(q, epoch_len, frames, cuda_stream);
    if (s != KADABRA_OK) return s;
    cudaStream_t st = as_stream(cuda_stream);
    if (!q->d_desc) KCUDA(cudaMalloc(reinterpret_cast<void **>(&q->d_desc), sizeof(kadabra::QueryDesc)), "allocate descriptor");
    if (!q->d_bs) KCUDA(cudaMalloc(reinterpret_cast<void **>(&q->d_bs), sizeof(kadabra::BatchState)), "allocate launch state");
    const int slot = (int)(q->launches % kadabra::kLaunchLog);
    kadabra::Counters *ctr = q->d_launch + slot;
    const kadabra::QueryDesc d = make_desc(q, ctr);
    KCUDA(cudaMemcpyAsync(q->d_desc, &d, sizeof(d), cudaMemcpyHostToDevice, st), "upload descriptor");
    KCUDA(cudaMemsetAsync(q->d_bs, 0, sizeof(kadabra::BatchState), st), "clear launch state");
    KCUDA(cudaMemsetAsync(ctr, 0, sizeof(kadabra::Counters), st), "reset launch counters");
    kadabra::BatchLaunch B{};
    B.queries = q->d_desc;
    B.nq = 1;
    B.slots = q->g->ws;
    B.spill = q->g->spill;
    if (q->p.coop_edges >= 0) {
        if (!q->g->d_help) {
            KCUDA(cudaMalloc(&q->g->d_help, kadabra::help_board_bytes()), "allocate help board");
            KCUDA(cudaMemset(q->g->d_help, 0, kadabra::help_board_bytes()), "clear help board");
        }
        B.help = q->g->d_help;
        B.help_edges = q->p.coop_edges > 0 ? (unsigned long long)q->p.coop_edges : 32768ULL;
    }
    B.bs = q->d_bs;
    B.budget = 0;
    B.spin_limit = 1ULL << 24;
    B.grid = clamp_grid(q, int64_t(1) << 40);
    B.threads = q->threads;
    B.off64 = q->g->off64;
    B.probe_log2 = probe_log2_of(q);
    B.probe_edges = probe_edges_of(q->p);
    {
        kadabra_status se = slot_events(q, slot);
        if (se != KADABRA_OK) return se;
    }
    KCUDA(cudaEventRecord(q->ev0[slot], st), "event");
    KCUDA(kadabra::launch_batch(B, st), "pipelined kernel launch");
    KCUDA(cudaEventRecord(q->ev1[slot], st), "event");
    q->grid_log[slot] = B.grid;
    ++q->launches;
    return KADABRA_OK;
}

// ---------------------------------------------------------------------------
// batches: many queries in one persistent launch
// ---------------------------------------------------------------------------

extern "C" kadabra_status kadabra_batch_create(int64_t max_n, int32_t slots, int32_t threads, int offsets_is_64,
                                               kadabra_batch **out)
{
    if (!out) return fail(KADABRA_ERR_INVALID_ARG, "out is null");
    if (max_n < 2 || max_n >= (int64_t(1) << 31)) return fail(KADABRA_ERR_INVALID_ARG, "max_n must be in [2, 2^31)");
    if (threads == 0) threads = 1024;
    if (threads != 128 && threads != 256 && threads != 512 && threads != 1024)
        return fail(KADABRA_ERR_INVALID_ARG, "threads must be 128, 256, 512 or 1024");
    int dev = 0, sms = 0, per_sm = 0;
    KCUDA(cudaGetDevice(&dev), "cudaGetDevice");
    KCUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
    KCUDA(kadabra::sample_occupancy(threads, offsets_is_64 ? 1 : 0, &per_sm), "occupancy");
    if (per_sm < 1) per_sm = 1;
    if (slots <= 0 || slots > sms * per_sm) slots = sms * per_sm;
    kadabra_batch *b = new kadabra_batch();
    b->max_n = max_n;
    b->slots = slots;
    b->threads = threads;
    b->off64 = offsets_is_64 ? 1 : 0;
    size_t free_b = 0, total_b = 0;
    KCUDA(cudaMemGetInfo(&free_b, &total_b), "cudaMemGetInfo");
    int fit = 0, nspill = 0;
    long long cap = 0;
    kadabra::plan_slots(max_n, slots, (size_t)((double)free_b * 0.6), 0, &fit, &cap, &nspill);
    if (fit < 1) {
        delete b;
        return fail(KADABRA_ERR_OOM, "not enough device memory for one sampling slot");
    }
    b->slots = fit;
    cudaError_t e = kadabra::alloc_slot_set(&b->ws, fit, max_n, cap, true, false);
    if (e == cudaSuccess) e = kadabra::alloc_slot_set(&b->spill, nspill, max_n, max_n, true, true);
    if (e == cudaSuccess) e = cudaMalloc(reinterpret_cast<void **>(&b->d_bs), sizeof(kadabra::BatchState));
    if (e == cudaSuccess) e = cudaMalloc(&b->d_help, kadabra::help_board_bytes());
    if (e == cudaSuccess) e = cudaMemset(b->d_help, 0, kadabra::help_board_bytes());
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
    if (e == cudaSuccess) e = kadabra::probe_prepare(threads, b->off64, per_sm, &b->probe_log2);
    if (e != cudaSuccess) {
        kadabra::free_slot_set(&b->ws);
        kadabra::free_slot_set(&b->spill);
        cudaFree(b->d_bs);
        cudaFree(b->d_help);
        delete b;
        return cuda_fail(e, "allocate batch scratch");
    }
    *out = b;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_batch_free(kadabra_batch *b)
{
    if (!b) return KADABRA_OK;
    cudaDeviceSynchronize();
    kadabra::free_slot_set(&b->ws);
    kadabra::free_slot_set(&b->spill);
    cudaFree(b->d_help);
    cudaFree(b->d_descs);
    cudaFree(b->d_states);
    cudaFree(b->d_bs);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    delete b;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_batch_step(kadabra_batch *b, kadabra_query *const *qs, int64_t count,
                                             uint64_t sample_budget, void *cuda_stream)
{
    if (!b || (!qs && count > 0)) return fail(KADABRA_ERR_INVALID_ARG, "batch or queries is null");
    if (count < 0 || count > (int64_t(1) << 20)) return fail(KADABRA_ERR_INVALID_ARG, "count out of range");
    if (count == 0) return KADABRA_OK;
    PhaseScope scope("kadabra: batch step (enqueue)", nullptr);
    cudaStream_t st = as_stream(cuda_stream);
    std::vector<kadabra::QueryDesc> descs((size_t)count);
    for (int64_t i = 0; i < count; ++i) {
        const kadabra_query *q = qs[i];
        if (!q) return fail(KADABRA_ERR_INVALID_ARG, "null query in batch");
        if (q->phase == 0 || (q->phase == 2 && !q->pipe_begun))
            return fail(KADABRA_ERR_STATE, "query not begun (kadabra_pipeline_begin or kadabra_calibration_begin)");
        if (q->g->n > b->max_n) return fail(KADABRA_ERR_INVALID_ARG, "query graph larger than the batch's max_n");
        if (q->g->off64 != b->off64) return fail(KADABRA_ERR_INVALID_ARG, "query offset width differs from the batch's");
        descs[(size_t)i] = make_desc(q, nullptr);
    }
    if (b->descs_cap < count) {
        cudaStreamSynchronize(st);
        cudaFree(b->d_descs);
        b->d_descs = nullptr;
        b->descs_cap = 0;
        cudaFree(b->d_states);
        b->d_states = nullptr;
        KCUDA(cudaMalloc(reinterpret_cast<void **>(&b->d_descs), (size_t)count * sizeof(kadabra::QueryDesc)),
              "allocate descriptors");
        KCUDA(cudaMalloc(reinterpret_cast<void **>(&b->d_states), (size_t)count * sizeof(int)), "allocate states");
        b->descs_cap = count;
    }
    KCUDA(cudaMemcpyAsync(b->d_descs, descs.data(), (size_t)count * sizeof(kadabra::QueryDesc), cudaMemcpyHostToDevice, st),
          "upload descriptors");
    KCUDA(cudaMemsetAsync(b->d_bs, 0, sizeof(kadabra::BatchState), st), "clear launch state");
    kadabra::BatchLaunch B{};
    B.queries = b->d_descs;
    B.nq = (int)count;
    B.slots = b->ws;
    B.spill = b->spill;
    B.help = b->d_help;
    B.help_edges = 32768ULL;
    B.bs = b->d_bs;
    B.budget = sample_budget;
    B.spin_limit = b->spin_limit;
    B.grid = b->slots;
    B.threads = b->threads;
    B.off64 = b->off64;
    B.policy = b->policy;
    B.probe_log2 = b->probe_log2;
    B.probe_edges = 256ULL;
    KCUDA(cudaEventRecord(b->ev0, st), "event");
    KCUDA(kadabra::launch_batch(B, st), "batch kernel launch");
    KCUDA(cudaEventRecord(b->ev1, st), "event");
    b->have_step = true;
    b->last_count = count;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_batch_poll(kadabra_batch *b, int32_t *states, int64_t count, void *cuda_stream)
{
    if (!b || (!states && count > 0)) return fail(KADABRA_ERR_INVALID_ARG, "batch or states is null");
    if (!b->have_step) return fail(KADABRA_ERR_STATE, "no batch step yet");
    if (count != b->last_count) return fail(KADABRA_ERR_INVALID_ARG, "count differs from the last step's");
    if (count == 0) return KADABRA_OK;
    cudaStream_t st = as_stream(cuda_stream);
    KCUDA(kadabra::launch_batch_poll(b->d_descs, (int)count, b->d_states, st), "poll kernel launch");
    KCUDA(cudaMemcpyAsync(states, b->d_states, (size_t)count * sizeof(int32_t), cudaMemcpyDeviceToHost, st),
          "read states");
    KCUDA(cudaStreamSynchronize(st), "synchronise");
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_batch_info(const kadabra_batch *b, int32_t *slots, int32_t *threads, int64_t *max_n)
{
    if (!b) return fail(KADABRA_ERR_INVALID_ARG, "batch is null");
    if (slots) *slots = b->slots;
    if (threads) *threads = b->threads;
    if (max_n) *max_n = b->max_n;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_batch_set_spin_limit(kadabra_batch *b, uint64_t polls)
{
    if (!b) return fail(KADABRA_ERR_INVALID_ARG, "batch is null");
    if (polls == 0) return fail(KADABRA_ERR_INVALID_ARG, "the poll limit must be >= 1");
    b->spin_limit = polls;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_batch_set_policy(kadabra_batch *b, int policy)
{
    if (!b) return fail(KADABRA_ERR_INVALID_ARG, "batch is null");
    if (policy != KADABRA_BATCH_ROUND_ROBIN && policy != KADABRA_BATCH_IN_ORDER)
        return fail(KADABRA_ERR_INVALID_ARG, "unknown batch policy");
    b->policy = policy;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_batch_last_ms(kadabra_batch *b, float *ms)
{
    if (!b || !ms) return fail(KADABRA_ERR_INVALID_ARG, "batch or ms is null");
    if (!b->have_step) return fail(KADABRA_ERR_STATE, "no batch step yet");
    KCUDA(cudaEventSynchronize(b->ev1), "event sync");
    KCUDA(cudaEventElapsedTime(ms, b->ev0, b->ev1), "event time");
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_check_stop_async(kadabra_query *q, void *cuda_stream)
{
    {
        kadabra_status s = need_calibrated(q);
        if (s != KADABRA_OK) return s;
    }
    kadabra::CheckLaunch c{};
    c.n = q->g->n;
    c.counts = q->d_counts;
    c.L = q->d_L;
    c.job = q->d_job;
    c.omega = q->omega;
    c.eps = q->p.eps;
    c.grid = 0;
    KCUDA(kadabra::launch_check(c, as_stream(cuda_stream)), "stop-check kernel launch");
    return KADABRA_OK;
}

static kadabra_status read_job(kadabra_query *q, Job *j, cudaStream_t st)
{
    KCUDA(cudaMemcpyAsync(j, q->d_job, sizeof(Job), cudaMemcpyDeviceToHost, st), "read query state");
    KCUDA(cudaStreamSynchronize(st), "synchronise");
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_check_stop(kadabra_query *q, int *stopped, double *max_f, double *max_g,
                                             void *cuda_stream)
{
    kadabra_status s = kadabra_check_stop_async(q, cuda_stream);
    if (s != KADABRA_OK) return s;
    Job j{};
    s = read_job(q, &j, as_stream(cuda_stream));
    if (s != KADABRA_OK) return s;
    s = device_error_status(j);
    if (s != KADABRA_OK) return s;
    if (stopped) *stopped = j.stopped;
    if (max_f) *max_f = j.last_maxf;
    if (max_g) *max_g = j.last_maxg;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_run(kadabra_query *q, int64_t epoch_len, int64_t max_epochs, int64_t sync_every,
                                      void *cuda_stream, int *stopped)
{
    if (!q) return fail(KADABRA_ERR_INVALID_ARG, "query is null");
    if (epoch_len <= 0 || max_epochs <= 0) return fail(KADABRA_ERR_INVALID_ARG, "epoch_len and max_epochs must be > 0");
    if (sync_every <= 0) sync_every = 4;
    cudaStream_t st = as_stream(cuda_stream);
    Job j{};
    for (int64_t e = 0; e < max_epochs; ++e) {
        kadabra_status s = kadabra_sample_epoch(q, epoch_len, cuda_stream);
        if (s == KADABRA_OK) s = kadabra_check_stop_async(q, cuda_stream);
        if (s != KADABRA_OK) return s;
        if ((e + 1) % sync_every == 0 || e + 1 == max_epochs) {
            s = read_job(q, &j, st);
            if (s != KADABRA_OK) return s;
            s = device_error_status(j);
            if (s != KADABRA_OK) return s;
            if (j.stopped) break;
        }
    }
    if (stopped) *stopped = j.stopped;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_sample_range(kadabra_query *q, int tag, uint64_t first, int64_t count,
                                               uint32_t *counts, void *cuda_stream)
{
    KREADY(q);
    if (!q || !counts) return fail(KADABRA_ERR_INVALID_ARG, "query or counts is null");
    if (tag != 0 && tag != 1) return fail(KADABRA_ERR_INVALID_ARG, "tag must be 0 or 1");
    if (count < 0 || count >= (int64_t(1) << 32)) return fail(KADABRA_ERR_INVALID_ARG, "count must be in [0, 2^32)");
    if (count == 0) return KADABRA_OK;
    cudaStream_t st = as_stream(cuda_stream);
    kadabra::SampleLaunch a = base_launch(q);
    a.counts = counts;
    a.job = q->d_trace_job;
    a.tag = (uint32_t)tag;
    a.use_stop = 0;
    a.epoch_len = count;
    a.clip = 0;
    a.grid = clamp_grid(q, count);
    const unsigned long long tau0 = first;
    KCUDA(kadabra::launch_reset_job(q->d_trace_job, st), "reset range state");
    KCUDA(cudaMemcpyAsync(&q->d_trace_job->tau, &tau0, 8, cudaMemcpyHostToDevice, st), "set range start");
    KCUDA(kadabra::launch_sample(a, st), "sampling kernel launch");
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_sample_range_log(kadabra_query *q, int tag, uint64_t first, int64_t count,
                                                   uint32_t *log, uint32_t log_cap, uint32_t *log_len,
                                                   void *cuda_stream)
{
    KREADY(q);
    if (!q || !log || !log_len) return fail(KADABRA_ERR_INVALID_ARG, "query, log or log_len is null");
    if (tag != 0 && tag != 1) return fail(KADABRA_ERR_INVALID_ARG, "tag must be 0 or 1");
    if (count < 0 || count >= (int64_t(1) << 32)) return fail(KADABRA_ERR_INVALID_ARG, "count must be in [0, 2^32)");
    cudaStream_t st = as_stream(cuda_stream);
    KCUDA(cudaMemsetAsync(log_len, 0, sizeof(uint32_t), st), "clear log length");
    if (count == 0) return KADABRA_OK;
    kadabra::SampleLaunch a = base_launch(q);
    a.counts = nullptr;
    a.log = log;
    a.log_len = log_len;
    a.log_cap = log_cap;
    a.job = q->d_trace_job;
    a.tag = (uint32_t)tag;
    a.use_stop = 0;
    a.epoch_len = count;
    a.clip = 0;
    a.grid = clamp_grid(q, count);
    const unsigned long long tau0 = first;
    KCUDA(kadabra::launch_reset_job(q->d_trace_job, st), "reset range state");
    KCUDA(cudaMemcpyAsync(&q->d_trace_job->tau, &tau0, 8, cudaMemcpyHostToDevice, st), "set range start");
    KCUDA(kadabra::launch_sample(a, st), "sampling kernel launch");
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_absorb_log(kadabra_query *q, const uint32_t *log, uint64_t len, uint64_t samples,
                                            void *cuda_stream)
{
    {
        kadabra_status s = need_calibrated(q);
        if (s != KADABRA_OK) return s;
    }
    if (!q || (!log && len > 0)) return fail(KADABRA_ERR_INVALID_ARG, "query or log is null");
    KCUDA(kadabra::launch_absorb_log(log, len, q->g->n, q->d_counts, q->d_job, samples, as_stream(cuda_stream)),
          "absorb kernel launch");
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_absorb(kadabra_query *q, const uint32_t *delta, uint64_t samples, void *cuda_stream)
{
    {
        kadabra_status s = need_calibrated(q);
        if (s != KADABRA_OK) return s;
    }
    if (!q || !delta) return fail(KADABRA_ERR_INVALID_ARG, "query or delta is null");
    KCUDA(kadabra::launch_absorb(q->g->n, q->d_counts, delta, q->d_job, samples, as_stream(cuda_stream)),
          "absorb kernel launch");
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_run_graph(kadabra_query *q, int64_t epoch_len, int epochs_per_graph, int64_t max_epochs,
                                            void *cuda_stream, int *stopped)
{
    KREADY(q);
    if (!q) return fail(KADABRA_ERR_INVALID_ARG, "query is null");
    if (epoch_len <= 0 || epoch_len >= (int64_t(1) << 32) || epochs_per_graph <= 0 || epochs_per_graph > 4096 ||
        max_epochs <= 0)
        return fail(KADABRA_ERR_INVALID_ARG, "epoch_len, epochs_per_graph or max_epochs out of range");
    cudaStream_t st = as_stream(cuda_stream);
    if (!q->graph_exec || q->graph_E != epoch_len || q->graph_k != epochs_per_graph) {
        if (q->graph_exec) cudaGraphExecDestroy(q->graph_exec);
        q->graph_exec = nullptr;
        if (!q->cap_stream) KCUDA(cudaStreamCreateWithFlags(&q->cap_stream, cudaStreamNonBlocking), "capture stream");
        kadabra::SampleLaunch a = base_launch(q);
        a.counts = q->d_counts;
        a.job = q->d_job;
        a.tag = 1;
        a.use_stop = 1;
        a.epoch_len = epoch_len;
        a.clip = q->omega_ceil;
        a.grid = clamp_grid(q, epoch_len);
        kadabra::CheckLaunch c{};
        c.n = q->g->n;
        c.counts = q->d_counts;
        c.L = q->d_L;
        c.job = q->d_job;
        c.omega = q->omega;
        c.eps = q->p.eps;
        KCUDA(cudaStreamBeginCapture(q->cap_stream, cudaStreamCaptureModeRelaxed), "begin capture");
        cudaError_t e = cudaSuccess;
        for (int k = 0; k < epochs_per_graph && e == cudaSuccess; ++k) {
            e = kadabra::launch_sample(a, q->cap_stream);
            if (e == cudaSuccess) e = kadabra::launch_check(c, q->cap_stream);
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t e2 = cudaStreamEndCapture(q->cap_stream, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&q->graph_exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            q->graph_exec = nullptr;
            return cuda_fail(e, "capture epochs");
        }
        q->graph_E = epoch_len;
        q->graph_k = epochs_per_graph;
    }
    Job j{};
    for (int64_t done = 0; done < max_epochs; done += epochs_per_graph) {
        KCUDA(cudaGraphLaunch(q->graph_exec, st), "graph launch");
        kadabra_status s = read_job(q, &j, st);
        if (s != KADABRA_OK) return s;
        s = device_error_status(j);
        if (s != KADABRA_OK) return s;
        if (j.stopped || j.tau >= q->omega_ceil) break;
    }
    if (stopped) *stopped = j.stopped;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_query_reset(kadabra_query *q, void *cuda_stream)
{
    {
        kadabra_status s = need_calibrated(q);
        if (s != KADABRA_OK) return s;
    }
    if (!q) return fail(KADABRA_ERR_INVALID_ARG, "query is null");
    cudaStream_t st = as_stream(cuda_stream);
    KCUDA(cudaMemsetAsync(q->d_counts, 0, (size_t)q->g->n * 4, st), "reset counters");
    KCUDA(kadabra::launch_reset_job(q->d_job, st), "reset state");
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_query_restore(kadabra_query *q, const uint32_t *counts, uint64_t tau, int64_t epochs,
                                              void *cuda_stream)
{
    {
        kadabra_status s = need_calibrated(q);
        if (s != KADABRA_OK) return s;
    }
    if (!counts) return fail(KADABRA_ERR_INVALID_ARG, "counts is null");
    if (epochs < 0) return fail(KADABRA_ERR_INVALID_ARG, "epochs must be >= 0");
    if (tau > q->omega_ceil) return fail(KADABRA_ERR_INVALID_ARG, "tau beyond ceil(omega)");
    cudaStream_t st = as_stream(cuda_stream);
    KCUDA(cudaMemcpyAsync(q->d_counts, counts, (size_t)q->g->n * 4, cudaMemcpyHostToDevice, st), "upload counters");
    KCUDA(kadabra::launch_reset_job(q->d_job, st), "reset state");
    Job j{};
    KCUDA(cudaMemcpyAsync(&j, q->d_job, sizeof(Job), cudaMemcpyDeviceToHost, st), "read state");
    KCUDA(cudaStreamSynchronize(st), "synchronise");
    j.tau = tau;
    j.epoch = epochs;
    KCUDA(cudaMemcpyAsync(q->d_job, &j, sizeof(Job), cudaMemcpyHostToDevice, st), "write state");
    KCUDA(cudaStreamSynchronize(st), "synchronise");
    q->pipe_begun = false;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_result(kadabra_query *q, double *btilde, uint32_t *counts, uint64_t *tau,
                                         int64_t *stop_epoch, void *cuda_stream)
{
    if (!q) return fail(KADABRA_ERR_INVALID_ARG, "query is null");
    cudaStream_t st = as_stream(cuda_stream);
    Job j{};
    kadabra_status s = read_job(q, &j, st);
    if (s != KADABRA_OK) return s;
    s = device_error_status(j);
    if (s != KADABRA_OK) return s;
    const size_t n = (size_t)q->g->n;
    if (btilde) {
        if (j.tau == 0) return fail(KADABRA_ERR_STATE, "no adaptive samples taken yet");
        KCUDA(kadabra::launch_result(q->g->n, q->d_counts, q->d_job, q->d_btilde, st), "result kernel launch");
        KCUDA(cudaMemcpyAsync(btilde, q->d_btilde, n * sizeof(double), cudaMemcpyDeviceToHost, st), "copy result");
    }
    if (counts) KCUDA(cudaMemcpyAsync(counts, q->d_counts, n * 4, cudaMemcpyDeviceToHost, st), "copy counts");
    KCUDA(cudaStreamSynchronize(st), "synchronise");
    if (tau) *tau = j.tau;
    if (stop_epoch) *stop_epoch = j.stop_epoch;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_query_get_info(kadabra_query *q, kadabra_query_info *out, void *cuda_stream)
{
    if (!q || !out) return fail(KADABRA_ERR_INVALID_ARG, "query or out is null");
    Job j{};
    kadabra_status s = read_job(q, &j, as_stream(cuda_stream));
    if (s != KADABRA_OK) return s;
    kadabra_query_info I;
    std::memset(&I, 0, sizeof(I));
    I.omega = q->omega;
    I.omega_ceil = q->omega_ceil;
    I.vertex_diameter = q->vd;
    I.n_calib = q->n_calib;
    I.sigma_bits = q->K;
    I.stopped = j.stopped;
    I.tau = j.tau;
    I.epochs = j.epoch;
    I.stop_epoch = j.stop_epoch;
    I.max_f = j.last_maxf;
    I.max_g = j.last_maxg;
    I.balance_C = q->balance_C;
    I.samples = j.total.samples;
    I.connected = j.total.connected;
    I.e_scan = j.total.e_scan;
    I.expanded = j.total.expanded;
    I.touched = j.total.touched;
    I.interior = j.total.interior;
    I.walk_scan = j.total.walk_scan;
    I.scaled = j.total.scaled;
    I.device_error = j.error;
    I.slots = q->slots;
    I.threads = q->threads;
    I.offsets_64 = q->g->off64;
    I.budget_classes = q->nclass;
    I.stop_ns = j.stopped ? j.stop_ns : 0ULL;
    I.phase = q->phase;
    I.launches = q->launches;
    I.diameter_ms = q->diameter_ms;
    I.calibration_ms = q->calibration_ms;
    I.queue_cap = q->g->ws.cap;
    I.spill_slots = q->g->spill.count;
    I.vd_exact = q->vd_exact;
    I.vd_searches = q->vd_searches;
    I.cal_done = q->phase == 2 ? (uint64_t)q->n_calib : 0ULL;
    if (q->phase == 1) {
        kadabra::PipeState ps{};
        cudaStream_t st = as_stream(cuda_stream);
        KCUDA(cudaMemcpyAsync(&ps, q->d_pipe, sizeof(ps), cudaMemcpyDeviceToHost, st), "read calibration progress");
        KCUDA(cudaStreamSynchronize(st), "synchronise");
        I.cal_done = ps.done[0];
    }
    const uint64_t n = (uint64_t)q->g->n;
    I.device_bytes = n * (4 + 4 + 16 + 8 + 4) + 3 * sizeof(Job) +
                     sizeof(kadabra::Counters) * kadabra::kLaunchLog + (uint64_t)q->nclass * (16 + 4) +
                     (uint64_t)q->logs_alloc * 4 + (q->d_pipe ? sizeof(kadabra::PipeState) : 0);
    *out = I;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_query_budgets(kadabra_query *q, double *L_L, double *L_U, uint32_t *cal,
                                                void *cuda_stream)
{
    {
        kadabra_status s = need_calibrated(q);
        if (s != KADABRA_OK) return s;
    }
    cudaStream_t st = as_stream(cuda_stream);
    const size_t n = (size_t)q->g->n;
    std::vector<double2> L(n);
    KCUDA(cudaMemcpyAsync(L.data(), q->d_L, n * sizeof(double2), cudaMemcpyDeviceToHost, st), "copy budgets");
    if (cal) KCUDA(cudaMemcpyAsync(cal, q->d_cal, n * 4, cudaMemcpyDeviceToHost, st), "copy calibration counts");
    KCUDA(cudaStreamSynchronize(st), "synchronise");
    for (size_t x = 0; x < n; ++x) {
        if (L_L) L_L[x] = L[x].x;
        if (L_U) L_U[x] = L[x].y;
    }
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_sample_trace(kadabra_query *q, int tag, uint64_t first, int64_t count,
                                               kadabra_trace_rec *recs, int32_t *interior, int64_t path_cap,
                                               void *cuda_stream)
{
    if (!q || !recs) return fail(KADABRA_ERR_INVALID_ARG, "query or recs is null");
    if (tag != 0 && tag != 1) return fail(KADABRA_ERR_INVALID_ARG, "tag must be 0 or 1");
    if (count <= 0 || count >= (int64_t(1) << 31)) return fail(KADABRA_ERR_INVALID_ARG, "count out of range");
    if (interior && path_cap <= 0) return fail(KADABRA_ERR_INVALID_ARG, "path_cap must be > 0");
    static_assert(sizeof(kadabra::TraceRec) == sizeof(kadabra_trace_rec), "trace record layout");
    {
        kadabra_status s = ready_workspace(q);
        if (s != KADABRA_OK) return s;
    }
    cudaStream_t st = as_stream(cuda_stream);
    kadabra::TraceRec *d_tr = nullptr;
    int32_t *d_path = nullptr;
    KCUDA(cudaMalloc(reinterpret_cast<void **>(&d_tr), (size_t)count * sizeof(kadabra::TraceRec)), "trace buffer");
    if (interior) {
        cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&d_path), (size_t)count * (size_t)path_cap * 4);
        if (e != cudaSuccess) {
            cudaFree(d_tr);
            return cuda_fail(e, "trace path buffer");
        }
    }
    kadabra::SampleLaunch a = base_launch(q);
    a.counts = nullptr;
    a.job = q->d_trace_job;
    a.tag = (uint32_t)tag;
    a.use_stop = 0;
    a.epoch_len = count;
    a.clip = 0;
    a.trace = d_tr;
    a.trace_path = d_path;
    a.trace_cap = interior ? path_cap : 0;
    a.grid = clamp_grid(q, count);
    unsigned long long tau0 = first;
    cudaError_t e = kadabra::launch_reset_job(q->d_trace_job, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&q->d_trace_job->tau, &tau0, 8, cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = kadabra::launch_sample(a, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(recs, d_tr, (size_t)count * sizeof(kadabra::TraceRec), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && interior)
        e = cudaMemcpyAsync(interior, d_path, (size_t)count * (size_t)path_cap * 4, cudaMemcpyDeviceToHost, st);
    Job j{};
    if (e == cudaSuccess) e = cudaMemcpyAsync(&j, q->d_trace_job, sizeof(Job), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaFree(d_tr);
    cudaFree(d_path);
    if (e != cudaSuccess) return cuda_fail(e, "trace run");
    return (j.error & ~kadabra::kErrSigmaOverflow) ? device_error_status(j) : KADABRA_OK;
}

extern "C" kadabra_status kadabra_launch_log(kadabra_query *q, int64_t max_entries, kadabra_launch_stats *out,
                                             int64_t *n_out)
{
    if (!q || !out || !n_out || max_entries < 0) return fail(KADABRA_ERR_INVALID_ARG, "bad arguments");
    int64_t have = q->launches < kadabra::kLaunchLog ? q->launches : kadabra::kLaunchLog;
    int64_t m = have < max_entries ? have : max_entries;
    *n_out = 0;
    if (m == 0) return KADABRA_OK;
    const int newest = (int)((q->launches - 1) % kadabra::kLaunchLog);
    KCUDA(cudaEventSynchronize(q->ev1[newest]), "event sync");
    std::vector<kadabra::Counters> c(kadabra::kLaunchLog);
    KCUDA(cudaMemcpy(c.data(), q->d_launch, sizeof(kadabra::Counters) * kadabra::kLaunchLog, cudaMemcpyDeviceToHost),
          "read launch counters");
    for (int64_t k = 0; k < m; ++k) {
        const int slot = (int)((q->launches - m + k) % kadabra::kLaunchLog);
        float ms = 0.f;
        KCUDA(cudaEventElapsedTime(&ms, q->ev0[slot], q->ev1[slot]), "event time");
        kadabra_launch_stats &o = out[k];
        o.ms = ms;
        o.samples = c[slot].samples;
        o.connected = c[slot].connected;
        o.e_scan = c[slot].e_scan;
        o.expanded = c[slot].expanded;
        o.touched = c[slot].touched;
        o.interior = c[slot].interior;
        o.walk_scan = c[slot].walk_scan;
        o.grid = q->grid_log[slot];
        o.threads = q->threads;
    }
    *n_out = m;
    return KADABRA_OK;
}

extern "C" kadabra_status kadabra_last_launch(kadabra_query *q, kadabra_launch_stats *out)
{
    if (!q || !out) return fail(KADABRA_ERR_INVALID_ARG, "query or out is null");
    if (q->launches == 0) return fail(KADABRA_ERR_STATE, "no sampling launch yet");
    int64_t got = 0;
    return kadabra_launch_log(q, 1, out, &got);
}
