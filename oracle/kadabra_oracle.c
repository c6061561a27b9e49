/*
 * KADABRA adaptive-sampling betweenness: plain CPU oracle.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * restatement of the method that the CUDA library is checked against.  Only
 * the tests, the smoke check and the benchmark's CPU-baseline leg may load
 * it.  It shares no code, header, table or constant generator with the CUDA
 * library; both consume the same seeded input graphs.
 *
 * What is computed, and where it comes from (arXiv 1910.11039):
 *   - normalised betweenness b(x) = 1/(n(n-1)) sum_{s!=t} sigma_st(x)/sigma_st
 *     (Section I); exact value by Brandes' accumulation (Section II).
 *   - one KADABRA sample (Section III-A): a pair s != t, a shortest s-t path
 *     drawn uniformly via a bidirectional BFS, +1 on the counter of every
 *     interior path vertex; tau counts samples; b~(x) = c~(x)/tau.
 *   - the three phases (Section III-A): diameter -> omega, calibration of
 *     delta_L / delta_U from a few non-adaptive samples, adaptive sampling
 *     checked after every epoch on a consistent snapshot (Section III-B,
 *     Algorithms 1 and 2: snapshot, aggregate, check, broadcast).
 *
 * The paper does not print the formulas of f, g, omega, delta_L and delta_U
 * (Section III-A defers them to KADABRA's original publication).  The
 * formulas used here are the readings recorded in the design notes.  They are
 * pinned against what they are defined to solve rather than against
 * themselves: f and g against a high-precision root of the deviation-bound
 * equation, omega against hand-worked values and the Table II sample counts,
 * the balanced delta rule against closed-form and high-precision roots of its
 * budget equation, and the whole method against the epsilon guarantee with
 * exact Brandes on small graphs.
 *
 * Determinism contract (a reading; the paper draws from an unspecified RNG):
 *   Philox-4x64-10 (Salmon et al., SC'11), key = (seed, 0),
 *   counter = (sample index, draw index, stream tag, 0).
 *   draw 0: pair; draw 1: meeting vertex; draws 2, 3, ...: back-walk steps,
 *   first towards s, then towards t.  Tag 0 = calibration, 1 = adaptive.
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fPIC -shared -o liboracle.so
 *        kadabra_oracle.c -lm      (no fast-math: IEEE rounding is part of
 *        the stop-check contract)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

typedef unsigned __int128 u128;

/* ------------------------------------------------------------------------ */
/* Philox-4x64-10, from the published round function and key schedule.      */
/* ------------------------------------------------------------------------ */

void orc_philox4x64_10(const uint64_t ctr_in[4], const uint64_t key_in[2], uint64_t out[4])
{
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint64_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; round++) {
        if (round > 0) { k0 += W0; k1 += W1; }
        u128 p0 = (u128)M0 * c0;
        u128 p1 = (u128)M1 * c2;
        uint64_t hi0 = (uint64_t)(p0 >> 64), lo0 = (uint64_t)p0;
        uint64_t hi1 = (uint64_t)(p1 >> 64), lo1 = (uint64_t)p1;
        c0 = hi1 ^ c1 ^ k0;
        c1 = lo1;
        c2 = hi0 ^ c3 ^ k1;
        c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static void draw(uint64_t seed, uint64_t tag, uint64_t idx, uint64_t k, uint64_t out[4])
{
    uint64_t ctr[4] = {idx, k, tag, 0};
    uint64_t key[2] = {seed, 0};
    orc_philox4x64_10(ctr, key, out);
}

/* floor(x * m / 2^64): maps a uniform 64-bit word to [0, m). */
static uint64_t mulhi64(uint64_t x, uint64_t m) { return (uint64_t)(((u128)x * m) >> 64); }

static int bitlen64(uint64_t x) { int b = 0; while (x) { b++; x >>= 1; } return b; }

/* ------------------------------------------------------------------------ */
/* Graph helpers                                                             */
/* ------------------------------------------------------------------------ */

static int64_t deg(const int64_t *off, int64_t v) { return off[v + 1] - off[v]; }

/* Largest shift-free sigma width K.  Section III-A asks for a shortest s-t
 * path drawn uniformly, which needs the exact path counts; it does not say
 * what happens when they outgrow a machine word.  Reading: every per-side
 * count is an exact uint64.  A layer's counts are kept at most 2^K,
 * K = min(63 - bitlen(max degree), 63 - bitlen(n)), so that
 *   - a count of the next layer, a sum of at most max-degree counts of at
 *     most 2^K each, stays below 2^63 (no 64-bit add can wrap), and
 *   - a meeting-set weight sum, at most n products of a count below 2^63
 *     and one of at most 2^K, stays below 2^126 (fits 128 bits).
 * Below 2^K counts are exact; a layer above it is scaled down
 * deterministically (see orc_sample_pair). */
int orc_sigma_bits(int64_t n, int64_t max_degree)
{
    int a = 63 - bitlen64((uint64_t)max_degree);
    int b = 63 - bitlen64((uint64_t)n);
    return a < b ? a : b;
}

/* ------------------------------------------------------------------------ */
/* One KADABRA sample (Section III-A)                                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    int64_t n;
    int64_t *dist[2];      /* dist[0] = from s, dist[1] = from t; -1 = unseen */
    uint64_t *sigma[2];    /* shortest-path counts from s / from t            */
    int32_t *ball[2];      /* all vertices reached by each side, BFS order    */
    int64_t ball_len[2];
    int32_t *meet;         /* meeting set M                                    */
} orc_ws;

orc_ws *orc_ws_create(int64_t n)
{
    orc_ws *w = (orc_ws *)calloc(1, sizeof(orc_ws));
    w->n = n;
    for (int side = 0; side < 2; side++) {
        w->dist[side] = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
        w->sigma[side] = (uint64_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(uint64_t));
        w->ball[side] = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        for (int64_t v = 0; v < n; v++) w->dist[side][v] = -1;
    }
    w->meet = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    return w;
}

void orc_ws_free(orc_ws *w)
{
    if (!w) return;
    for (int side = 0; side < 2; side++) { free(w->dist[side]); free(w->sigma[side]); free(w->ball[side]); }
    free(w->meet);
    free(w);
}

/* Forget everything the previous sample touched. */
static void ws_reset(orc_ws *w)
{
    for (int side = 0; side < 2; side++) {
        for (int64_t i = 0; i < w->ball_len[side]; i++) {
            int32_t v = w->ball[side][i];
            w->dist[side][v] = -1;
            w->sigma[side][v] = 0;
        }
        w->ball_len[side] = 0;
    }
}

typedef struct {
    int64_t s, t;
    int64_t d;             /* d(s,t); -1 when s and t are disconnected       */
    uint64_t sigma_lo;     /* sigma_st (possibly scaled), low / high 64 bits */
    uint64_t sigma_hi;
    int64_t meet_size;     /* |M|                                            */
    int64_t chosen;        /* meeting vertex picked                          */
    int64_t e_scan;        /* adjacency entries scanned by the BFS           */
    int64_t n_interior;    /* interior vertices on the sampled path          */
    int32_t scaled;        /* 1 if some layer's sigma values were shifted    */
    int32_t overflow;      /* 1 if strict mode met a sigma above 2^K         */
} orc_sample_info;

static int cmp_i32(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* Walk from v back to the source of `side`, choosing each predecessor u
 * (a neighbour one layer closer, scanned in CSR order) with probability
 * sigma(u) / sum of sigma over the predecessors.  Appends interior vertices
 * (every vertex but the source) to `path`.  Returns the next draw index. */
static uint64_t walk_back(const int64_t *off, const int32_t *col, orc_ws *w, int side,
                          int64_t v, uint64_t seed, uint64_t tag, uint64_t idx, uint64_t k,
                          int32_t *path, int64_t *np)
{
    const int64_t *dist = w->dist[side];
    const uint64_t *sig = w->sigma[side];
    while (dist[v] > 0) {
        uint64_t total = 0;
        for (int64_t e = off[v]; e < off[v + 1]; e++)
            if (dist[col[e]] == dist[v] - 1) total += sig[col[e]];
        uint64_t x[4];
        draw(seed, tag, idx, k++, x);
        uint64_t r = mulhi64(x[0], total);
        uint64_t prefix = 0;
        int64_t u = -1;
        for (int64_t e = off[v]; e < off[v + 1]; e++) {
            if (dist[col[e]] != dist[v] - 1) continue;
            prefix += sig[col[e]];
            if (prefix > r) { u = col[e]; break; }
        }
        if (dist[u] > 0) path[(*np)++] = (int32_t)u;
        v = u;
    }
    return k;
}

/* Sample a shortest s-t path for a given pair with the balanced
 * bidirectional BFS; draws use (seed, tag, idx).  Writes the interior
 * vertices to `path` (capacity n) and returns their number. */
int64_t orc_sample_pair(int64_t n, const int64_t *off, const int32_t *col, orc_ws *w,
                        int64_t s, int64_t t, uint64_t seed, uint64_t tag, uint64_t idx,
                        int K, int strict, int32_t *path, orc_sample_info *info)
{
    orc_sample_info I;
    memset(&I, 0, sizeof(I));
    I.s = s; I.t = t; I.d = -1; I.chosen = -1;
    (void)n;

    /* the two balls: side 0 grows from s, side 1 from t */
    int64_t src[2] = {s, t};
    int64_t layer[2] = {0, 0};        /* radius reached by each side       */
    int64_t fbeg[2], fend[2];          /* current frontier = ball[fbeg,fend) */
    int64_t fdeg[2];                   /* sum of degrees over the frontier   */
    for (int side = 0; side < 2; side++) {
        w->dist[side][src[side]] = 0;
        w->sigma[side][src[side]] = 1;
        w->ball[side][0] = (int32_t)src[side];
        w->ball_len[side] = 1;
        fbeg[side] = 0; fend[side] = 1;
        fdeg[side] = deg(off, src[side]);
    }

    int64_t meet_len = 0;
    int X = 0;
    for (;;) {
        /* expand the side whose frontier has the smaller degree sum; ties -> s */
        X = (fdeg[0] <= fdeg[1]) ? 0 : 1;
        int Y = 1 - X;
        int64_t *dX = w->dist[X];
        uint64_t *sX = w->sigma[X];
        int64_t next = layer[X] + 1;
        int64_t new_beg = w->ball_len[X];
        meet_len = 0;
        for (int64_t i = fbeg[X]; i < fend[X]; i++) {
            int64_t u = w->ball[X][i];
            I.e_scan += deg(off, u);
            for (int64_t e = off[u]; e < off[u + 1]; e++) {
                int64_t v = col[e];
                if (dX[v] == -1) {
                    dX[v] = next;
                    if (w->dist[Y][v] != -1) w->meet[meet_len++] = (int32_t)v;
                    else w->ball[X][w->ball_len[X]++] = (int32_t)v;
                }
                if (dX[v] == next) sX[v] += sX[u];
            }
        }
        layer[X] = next;
        if (meet_len > 0) break;                       /* balls touch: done */
        if (w->ball_len[X] == new_beg) {                /* frontier died out */
            meet_len = 0;
            break;
        }
        /* keep the new layer's sigma below 2^K + 1 (ceil-shift, stays >= 1) */
        uint64_t mx = 0;
        for (int64_t i = new_beg; i < w->ball_len[X]; i++)
            if (sX[w->ball[X][i]] > mx) mx = sX[w->ball[X][i]];
        int sh = bitlen64(mx) - K;
        if (sh > 0) {
            I.scaled = 1;
            if (strict) { I.overflow = 1; break; }
            for (int64_t i = new_beg; i < w->ball_len[X]; i++) {
                int32_t v = w->ball[X][i];
                sX[v] = ((sX[v] - 1) >> sh) + 1;
            }
        }
        fbeg[X] = new_beg;
        fend[X] = w->ball_len[X];
        fdeg[X] = 0;
        for (int64_t i = fbeg[X]; i < fend[X]; i++) fdeg[X] += deg(off, w->ball[X][i]);
    }

    /* meeting vertices also live in the expanding side's tables; remember
     * them so that the reset after the sample clears them */
    int64_t np = 0;
    if (meet_len > 0 && !I.overflow) {
        int Y = 1 - X;
        I.d = layer[X] + layer[Y];
        I.meet_size = meet_len;
        /* sigma_st = sum over M of sigma_s(w) * sigma_t(w); pick w with
         * probability proportional to its term, M in ascending id order */
        qsort(w->meet, (size_t)meet_len, sizeof(int32_t), cmp_i32);
        u128 total = 0;
        for (int64_t i = 0; i < meet_len; i++) {
            int32_t v = w->meet[i];
            total += (u128)w->sigma[0][v] * w->sigma[1][v];
        }
        I.sigma_lo = (uint64_t)total;
        I.sigma_hi = (uint64_t)(total >> 64);
        uint64_t x[4];
        draw(seed, tag, idx, 1, x);
        u128 R = ((u128)x[1] << 64) | x[0];
        u128 r = R % total;
        u128 prefix = 0;
        int64_t wv = -1;
        for (int64_t i = 0; i < meet_len; i++) {
            int32_t v = w->meet[i];
            prefix += (u128)w->sigma[0][v] * w->sigma[1][v];
            if (prefix > r) { wv = v; break; }
        }
        I.chosen = wv;
        if (wv != s && wv != t) path[np++] = (int32_t)wv;
        uint64_t k = 2;
        k = walk_back(off, col, w, 0, wv, seed, tag, idx, k, path, &np);
        k = walk_back(off, col, w, 1, wv, seed, tag, idx, k, path, &np);
        (void)k;
    }
    /* clear the expanding side's marks on meeting vertices */
    for (int64_t i = 0; i < meet_len; i++) {
        int32_t v = w->meet[i];
        w->dist[X][v] = -1;
        w->sigma[X][v] = 0;
    }
    I.n_interior = np;
    ws_reset(w);
    if (info) *info = I;
    return np;
}

/* Draw the pair for sample `idx` (draw 0): s uniform in [0,n), t uniform in
 * [0,n) minus {s}. */
void orc_draw_pair(int64_t n, uint64_t seed, uint64_t tag, uint64_t idx, int64_t *s, int64_t *t)
{
    uint64_t x[4];
    draw(seed, tag, idx, 0, x);
    uint64_t a = mulhi64(x[0], (uint64_t)n);
    uint64_t b = mulhi64(x[1], (uint64_t)(n - 1));
    if (b >= a) b++;
    *s = (int64_t)a;
    *t = (int64_t)b;
}

int64_t orc_sample(int64_t n, const int64_t *off, const int32_t *col, orc_ws *w,
                   uint64_t seed, uint64_t tag, uint64_t idx, int K, int strict,
                   int32_t *path, orc_sample_info *info)
{
    int64_t s, t;
    orc_draw_pair(n, seed, tag, idx, &s, &t);
    return orc_sample_pair(n, off, col, w, s, t, seed, tag, idx, K, strict, path, info);
}

/* Samples [idx_begin, idx_end): counts[x] += 1 for every interior vertex.
 * Returns the number of samples that met a sigma above 2^K in strict mode. */
typedef struct {
    int64_t samples, e_scan, connected, interior, scaled, overflow;
} orc_run_stats;

/* Same as orc_run_samples, with a caller-owned workspace (reused across
 * calls; every sample leaves it as it found it) and path buffer (n entries). */
int64_t orc_run_samples_ws(int64_t n, const int64_t *off, const int32_t *col, orc_ws *w, int32_t *path,
                           uint64_t seed, uint64_t tag, uint64_t idx_begin, uint64_t idx_end,
                           int K, int strict, uint32_t *counts, orc_run_stats *st)
{
    orc_run_stats S;
    memset(&S, 0, sizeof(S));
    for (uint64_t i = idx_begin; i < idx_end; i++) {
        orc_sample_info I;
        int64_t np = orc_sample(n, off, col, w, seed, tag, i, K, strict, path, &I);
        for (int64_t j = 0; j < np; j++) counts[path[j]] += 1;
        S.samples++;
        S.e_scan += I.e_scan;
        S.connected += (I.d >= 0);
        S.interior += np;
        S.scaled += I.scaled;
        S.overflow += I.overflow;
    }
    if (st) *st = S;
    return S.overflow;
}

int64_t orc_run_samples(int64_t n, const int64_t *off, const int32_t *col,
                        uint64_t seed, uint64_t tag, uint64_t idx_begin, uint64_t idx_end,
                        int K, int strict, uint32_t *counts, orc_run_stats *st)
{
    orc_ws *w = orc_ws_create(n);
    int32_t *path = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int64_t r = orc_run_samples_ws(n, off, col, w, path, seed, tag, idx_begin, idx_end, K, strict, counts, st);
    free(path);
    orc_ws_free(w);
    return r;
}

/* ------------------------------------------------------------------------ */
/* Diameter phase: vertex-diameter upper bound                               */
/* ------------------------------------------------------------------------ */

/* For every connected component, BFS from its smallest vertex id v and take
 * 2*ecc(v) + 1 >= D + 1 = vertex diameter; return the maximum over
 * components (1 for a graph without edges). */
int64_t orc_vertex_diameter_bound(int64_t n, const int64_t *off, const int32_t *col)
{
    int64_t *dist = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t v = 0; v < n; v++) dist[v] = -1;
    int64_t best = 1;
    for (int64_t r = 0; r < n; r++) {
        if (dist[r] != -1) continue;
        int64_t qh = 0, qt = 0, ecc = 0;
        dist[r] = 0; queue[qt++] = r;
        while (qh < qt) {
            int64_t u = queue[qh++];
            if (dist[u] > ecc) ecc = dist[u];
            for (int64_t e = off[u]; e < off[u + 1]; e++)
                if (dist[col[e]] == -1) { dist[col[e]] = dist[u] + 1; queue[qt++] = col[e]; }
        }
        if (2 * ecc + 1 > best) best = 2 * ecc + 1;
    }
    free(dist); free(queue);
    return best;
}

/* Exact vertex diameter (all-pairs BFS): for small graphs only. */
int64_t orc_vertex_diameter_exact(int64_t n, const int64_t *off, const int32_t *col)
{
    int64_t *dist = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t *queue = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    int64_t best = n > 0 ? 1 : 0;
    for (int64_t r = 0; r < n; r++) {
        for (int64_t v = 0; v < n; v++) dist[v] = -1;
        int64_t qh = 0, qt = 0;
        dist[r] = 0; queue[qt++] = r;
        while (qh < qt) {
            int64_t u = queue[qh++];
            if (dist[u] + 1 > best) best = dist[u] + 1;
            for (int64_t e = off[u]; e < off[u + 1]; e++)
                if (dist[col[e]] == -1) { dist[col[e]] = dist[u] + 1; queue[qt++] = col[e]; }
        }
    }
    free(dist); free(queue);
    return best;
}

/* ------------------------------------------------------------------------ */
/* omega, delta_L / delta_U, and the stopping functions (Section III-A)     */
/* formulas not printed in the paper (readings; pinned by what they solve)  */
/* ------------------------------------------------------------------------ */

/* Maximal number of samples: (c / eps^2) * (floor(log2(VD - 2)) + 1 + ln(2/delta)),
 * c = 1/2, VD = vertex diameter (VD - 2 clamped to >= 1). */
double orc_omega(double eps, double delta, int64_t vd)
{
    int64_t x = vd - 2;
    if (x < 1) x = 1;
    int fl = bitlen64((uint64_t)x) - 1;
    return (0.5 / (eps * eps)) * ((double)fl + 1.0 + log(2.0 / delta));
}

/* Per-vertex log failure budgets L_L(x) = -ln delta_L(x), L_U(x) = -ln delta_U(x).
 * rule 0 (uniform):  delta_L = delta_U = delta / (4n).
 * rule 1 (balanced): delta_L = delta_U = exp(-C eps^2 / bhat(x)) + beta delta / (4n),
 *   bhat(x) = cal(x) / n_cal, C the bisection result on [0, ln(4n/((1-beta)delta))/eps^2]
 *   so that sum_x exp(-C eps^2 / bhat(x)) <= (1 - beta) delta / 4, i.e. the
 *   per-vertex budgets sum to at most delta/2 (the rest of delta goes to omega).
 *   The sum runs over calibration counts c (vertices with equal counts have
 *   equal terms): sum_c #{x : cal(x) = c} * exp(-C eps^2 n_cal / c). */
static double balanced_sum(const int64_t *hist, uint32_t cmax, int64_t n_cal, double eps, double C)
{
    /* sum over vertices with a calibration count c > 0 of exp(-C eps^2 / bhat),
     * bhat = c / n_cal, grouped by c in ascending order */
    double sum = 0.0;
    for (uint32_t c = 1; c <= cmax; c++) {
        if (hist[c] == 0) continue;
        double bhat = (double)c / (double)n_cal;
        sum += (double)hist[c] * exp(-((C * (eps * eps)) / bhat));
    }
    return sum;
}

void orc_calibrate_L(int64_t n, const uint32_t *cal, int64_t n_cal, double eps, double delta,
                     int rule, double beta, double *L_L, double *L_U, double *C_out)
{
    if (rule == 0) {
        double dl = delta / (4.0 * (double)n);
        for (int64_t x = 0; x < n; x++) { L_L[x] = -log(dl); L_U[x] = -log(dl); }
        if (C_out) *C_out = 0.0;
        return;
    }
    uint32_t cmax = 0;
    for (int64_t x = 0; x < n; x++) if (cal[x] > cmax) cmax = cal[x];
    int64_t *hist = (int64_t *)calloc((size_t)cmax + 1, sizeof(int64_t));
    for (int64_t x = 0; x < n; x++) hist[cal[x]]++;
    double budget = (1.0 - beta) * delta / 4.0;
    double lo = 0.0;
    double hi = log(4.0 * (double)n / ((1.0 - beta) * delta)) / (eps * eps);
    while (hi - lo > eps / 10.0) {
        double mid = (lo + hi) / 2.0;
        if (balanced_sum(hist, cmax, n_cal, eps, mid) <= budget) hi = mid;
        else lo = mid;
    }
    free(hist);
    double C = hi;
    double floor_term = beta * delta / (4.0 * (double)n);
    for (int64_t x = 0; x < n; x++) {
        double dl;
        if (cal[x] == 0) {
            dl = floor_term;
        } else {
            double bhat = (double)cal[x] / (double)n_cal;
            dl = exp(-((C * (eps * eps)) / bhat)) + floor_term;
        }
        L_L[x] = -log(dl);
        L_U[x] = -log(dl);
    }
    if (C_out) *C_out = C;
}

/* f(b~, delta_L, omega, tau) and g(b~, delta_U, omega, tau), with L = -ln delta:
 *   f = (L/tau) * (1/3 - omega/tau + sqrt((1/3 - omega/tau)^2 + 2 b~ omega / L))
 *   g = (L/tau) * (1/3 + omega/tau + sqrt((1/3 + omega/tau)^2 + 2 b~ omega / L))
 * evaluated in this operation order, IEEE double, no contraction. */
void orc_stop_functions(uint32_t c, uint64_t tau, double omega, double LL, double LU,
                        double *f, double *g)
{
    double tau_d = (double)tau;
    double bt = (double)c / tau_d;
    double r = omega / tau_d;
    double third = 1.0 / 3.0;
    double af = third - r;
    double ag = third + r;
    *f = (LL / tau_d) * (af + sqrt(af * af + ((2.0 * bt) * omega) / LL));
    *g = (LU / tau_d) * (ag + sqrt(ag * ag + ((2.0 * bt) * omega) / LU));
}

/* Stop iff tau >= omega, or max_x f < eps and max_x g < eps.  tau = 0 never
 * stops (and reports +inf maxima). */
int orc_check_stop(int64_t n, const uint32_t *counts, uint64_t tau, double omega, double eps,
                   const double *L_L, const double *L_U, double *max_f, double *max_g)
{
    if (tau == 0) { *max_f = INFINITY; *max_g = INFINITY; return 0; }
    double mf = 0.0, mg = 0.0;
    for (int64_t x = 0; x < n; x++) {
        double f, g;
        orc_stop_functions(counts[x], tau, omega, L_L[x], L_U[x], &f, &g);
        if (f > mf) mf = f;
        if (g > mg) mg = g;
    }
    *max_f = mf; *max_g = mg;
    if ((double)tau >= omega) return 1;
    return (mf < eps && mg < eps) ? 1 : 0;
}

/* ------------------------------------------------------------------------ */
/* The whole method: diameter -> omega -> calibration -> adaptive epochs      */
/* ------------------------------------------------------------------------ */

typedef struct {
    double eps, delta;
    uint64_t seed;
    int64_t vertex_diameter;   /* <= 0: use orc_vertex_diameter_bound */
    int64_t n_calib;           /* <= 0: max(1000, ceil(omega / 100))   */
    int64_t epoch_len;         /* adaptive samples per epoch           */
    int32_t delta_rule;        /* 0 uniform, 1 balanced                */
    int32_t strict;            /* 1: a sigma above 2^K is an error     */
    double beta;               /* balancing floor weight               */
    int64_t max_epochs;        /* safety bound on the loop             */
} orc_params;

typedef struct {
    double omega;
    int64_t vd;
    int64_t n_calib;
    int32_t K;
    int32_t stopped;
    uint64_t tau;
    int64_t epochs;            /* epochs run (the stop epoch is epochs-1) */
    int64_t stop_epoch;        /* -1 if not stopped within max_epochs     */
    double max_f, max_g;       /* at the last check                       */
    double C;                  /* balancing constant                      */
    int64_t e_scan;            /* adaptive phase traversed edges          */
    int64_t overflow;          /* strict-mode sigma overflows             */
} orc_result;

int orc_kadabra(int64_t n, const int64_t *off, const int32_t *col, const orc_params *P,
                uint32_t *counts, uint32_t *cal_counts, double *L_L, double *L_U, orc_result *R)
{
    memset(R, 0, sizeof(*R));
    int64_t maxdeg = 0;
    for (int64_t v = 0; v < n; v++) if (deg(off, v) > maxdeg) maxdeg = deg(off, v);
    int K = orc_sigma_bits(n, maxdeg);
    R->K = K;

    /* phase 1: diameter -> omega */
    int64_t vd = P->vertex_diameter > 0 ? P->vertex_diameter : orc_vertex_diameter_bound(n, off, col);
    R->vd = vd;
    double omega = orc_omega(P->eps, P->delta, vd);
    R->omega = omega;
    uint64_t omega_ceil = (uint64_t)ceil(omega);

    /* phase 2: calibration samples (tag 0) -> delta_L, delta_U */
    int64_t nc = P->n_calib;
    if (nc <= 0) {
        nc = (int64_t)ceil(omega / 100.0);
        if (nc < 1000) nc = 1000;
    }
    R->n_calib = nc;
    memset(cal_counts, 0, sizeof(uint32_t) * (size_t)n);
    orc_run_stats st;
    R->overflow += orc_run_samples(n, off, col, P->seed, 0, 0, (uint64_t)nc, K, P->strict, cal_counts, &st);
    orc_calibrate_L(n, cal_counts, nc, P->eps, P->delta, P->delta_rule, P->beta, L_L, L_U, &R->C);

    /* phase 3: adaptive sampling (tag 1), stop check after every epoch */
    memset(counts, 0, sizeof(uint32_t) * (size_t)n);
    uint64_t tau = 0;
    R->stop_epoch = -1;
    for (int64_t e = 0; e < P->max_epochs; e++) {
        uint64_t m = 0;
        if (tau < omega_ceil) {
            m = omega_ceil - tau;
            if (m > (uint64_t)P->epoch_len) m = (uint64_t)P->epoch_len;
        }
        R->overflow += orc_run_samples(n, off, col, P->seed, 1, tau, tau + m, K, P->strict, counts, &st);
        R->e_scan += st.e_scan;
        tau += m;
        R->epochs = e + 1;
        int stop = orc_check_stop(n, counts, tau, omega, P->eps, L_L, L_U, &R->max_f, &R->max_g);
        if (stop) { R->stopped = 1; R->stop_epoch = e; break; }
    }
    R->tau = tau;
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exact betweenness (Brandes): the definition of b(x), for small graphs     */
/* ------------------------------------------------------------------------ */

/* b(x) = 1/(n(n-1)) sum over ordered pairs s != t of sigma_st(x)/sigma_st. */
void orc_brandes(int64_t n, const int64_t *off, const int32_t *col, double *b)
{
    int64_t *dist = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    double *sigma = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    double *dep = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    int64_t *order = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    for (int64_t x = 0; x < n; x++) b[x] = 0.0;
    for (int64_t s = 0; s < n; s++) {
        for (int64_t v = 0; v < n; v++) { dist[v] = -1; sigma[v] = 0.0; dep[v] = 0.0; }
        int64_t qh = 0, qt = 0;
        dist[s] = 0; sigma[s] = 1.0; order[qt++] = s;
        while (qh < qt) {
            int64_t u = order[qh++];
            for (int64_t e = off[u]; e < off[u + 1]; e++) {
                int64_t v = col[e];
                if (dist[v] == -1) { dist[v] = dist[u] + 1; order[qt++] = v; }
                if (dist[v] == dist[u] + 1) sigma[v] += sigma[u];
            }
        }
        /* dependencies in reverse BFS order */
        for (int64_t i = qt - 1; i >= 0; i--) {
            int64_t v = order[i];
            for (int64_t e = off[v]; e < off[v + 1]; e++) {
                int64_t u = col[e];
                if (dist[u] == dist[v] - 1) dep[u] += sigma[u] / sigma[v] * (1.0 + dep[v]);
            }
            if (v != s) b[v] += dep[v];
        }
    }
    double norm = (double)n * (double)(n - 1);
    for (int64_t x = 0; x < n; x++) b[x] = n > 1 ? b[x] / norm : 0.0;
    free(dist); free(sigma); free(dep); free(order);
}
