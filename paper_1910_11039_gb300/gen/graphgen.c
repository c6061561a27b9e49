/*
 * Native R-MAT graph builder (inputs only: no part of the method).
 *
 * Builds the symmetric CSR of an R-MAT graph (Chakrabarti, Zhan, Faloutsos
 * 2004) with edge_factor * 2^scale edge draws, without noise, with a random
 * relabelling of the vertices, self-loops and duplicate edges removed and
 * every neighbour list in ascending order: the synthetic stand-in for the
 * complex networks of the paper's experiments (Section V-A), at sizes where a
 * numpy builder takes minutes and tens of GB.
 *
 * Randomness is counter-based, so any edge can be drawn again from its index
 * and the result does not depend on the thread count:
 *   h(seed, i, k) = mix(mix(seed * G + i) ^ (k * H + J)), mix = the splitmix64
 *   finaliser (Steele, Lea and Flood 2014);
 *   edge i, level l (0 = most significant bit): a 32-bit uniform u, half of
 *   h(seed, i, l / 2); quadrant a if u < A, b if u < A + B, c if
 *   u < A + B + C, else d, with A = floor(a 2^32) etc.; quadrants b and d set
 *   the column bit, c and d the row bit;
 *   relabelling: Fisher-Yates over [0, n), step j (from n - 1 down to 1)
 *   swapping j with floor(h(seed, j, 2^40) * (j + 1) / 2^64).
 *
 * Construction: one pass counts each vertex's edge ends, a prefix sum gives
 * the row offsets, a second pass (drawing the same edges again) scatters the
 * ends into their rows, then every row is sorted and deduplicated and the rows
 * are packed.  Peak memory: the column array of 2 * edge draws entries plus
 * 16 bytes per vertex.
 *
 * Build: gcc -O3 -std=c11 -fPIC -shared -pthread -o libgraphgen.so graphgen.c
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static inline uint64_t mix(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

static inline uint64_t h3(uint64_t seed, uint64_t i, uint64_t k)
{
    return mix(mix(seed * 0x9E3779B97F4A7C15ULL + i) ^ (k * 0xD1B54A32D192ED03ULL + 0x632BE59BD9B4E019ULL));
}

typedef struct {
    int scale;
    uint64_t seed;
    uint32_t A, AB, ABC;          /* cumulative quadrant thresholds, scaled to 2^32 */
    const int32_t *perm;          /* relabelling (NULL: none) */
} rmat_spec;

static inline void rmat_edge(const rmat_spec *R, uint64_t i, int64_t *u, int64_t *v)
{
    int64_t r = 0, c = 0;
    uint64_t word = 0;
    for (int l = 0; l < R->scale; l++) {
        if ((l & 1) == 0) word = h3(R->seed, i, (uint64_t)(l >> 1));
        const uint32_t x = (l & 1) ? (uint32_t)(word >> 32) : (uint32_t)word;
        const int64_t bit = (int64_t)1 << (R->scale - 1 - l);
        if (x >= R->AB) r |= bit;                         /* quadrants c, d */
        if ((x >= R->A && x < R->AB) || x >= R->ABC) c |= bit;   /* quadrants b, d */
    }
    if (R->perm) {
        r = R->perm[r];
        c = R->perm[c];
    }
    *u = r;
    *v = c;
}

typedef struct {
    const rmat_spec *R;
    uint64_t lo, hi;              /* edge draws [lo, hi) */
    int64_t *cnt;                 /* pass 1: ends per vertex; pass 2: next free slot per row */
    int32_t *cols;                /* pass 2 only */
    int64_t n, *off, *ndeg;       /* row pass */
    int64_t vlo, vhi;
} task;

static void *count_pass(void *arg)
{
    task *T = (task *)arg;
    for (uint64_t i = T->lo; i < T->hi; i++) {
        int64_t u, v;
        rmat_edge(T->R, i, &u, &v);
        if (u == v) continue;
        __atomic_fetch_add(&T->cnt[u], 1, __ATOMIC_RELAXED);
        __atomic_fetch_add(&T->cnt[v], 1, __ATOMIC_RELAXED);
    }
    return NULL;
}

static void *scatter_pass(void *arg)
{
    task *T = (task *)arg;
    for (uint64_t i = T->lo; i < T->hi; i++) {
        int64_t u, v;
        rmat_edge(T->R, i, &u, &v);
        if (u == v) continue;
        const int64_t pu = __atomic_fetch_add(&T->cnt[u], 1, __ATOMIC_RELAXED);
        const int64_t pv = __atomic_fetch_add(&T->cnt[v], 1, __ATOMIC_RELAXED);
        T->cols[pu] = (int32_t)v;
        T->cols[pv] = (int32_t)u;
    }
    return NULL;
}

static int cmp_i32(const void *a, const void *b)
{
    const int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

/* sort and deduplicate rows [vlo, vhi); ndeg[v] = distinct neighbours */
static void *row_pass(void *arg)
{
    task *T = (task *)arg;
    for (int64_t v = T->vlo; v < T->vhi; v++) {
        int32_t *row = T->cols + T->off[v];
        const int64_t d = T->off[v + 1] - T->off[v];
        if (d > 16) {
            qsort(row, (size_t)d, sizeof(int32_t), cmp_i32);
        } else {
            for (int64_t a = 1; a < d; a++) {
                const int32_t x = row[a];
                int64_t b = a - 1;
                while (b >= 0 && row[b] > x) { row[b + 1] = row[b]; b--; }
                row[b + 1] = x;
            }
        }
        int64_t k = 0;
        for (int64_t a = 0; a < d; a++)
            if (k == 0 || row[a] != row[k - 1]) row[k++] = row[a];
        T->ndeg[v] = k;
    }
    return NULL;
}

static int run_threads(int nt, task *tasks, void *(*fn)(void *))
{
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * (size_t)nt);
    if (!th) return -1;
    int started = 0, rc = 0;
    for (int k = 0; k < nt; k++) {
        if (pthread_create(&th[k], NULL, fn, &tasks[k]) != 0) { rc = -1; break; }
        started++;
    }
    for (int k = 0; k < started; k++) pthread_join(th[k], NULL);
    if (rc != 0)   /* finish the rest on this thread */
        for (int k = started; k < nt; k++) fn(&tasks[k]);
    free(th);
    return 0;
}

/*
 * Builds the CSR into caller-owned arrays: off[n + 1] (int64) and cols, which
 * must hold 2 * edge_factor * 2^scale entries (the count before duplicates are
 * removed).  Returns the number of adjacency entries, or -1 on bad arguments
 * or an allocation failure.
 */
int64_t gg_rmat_csr(int scale, int64_t edge_factor, uint64_t seed, double a, double b, double c, int relabel,
                    int nthreads, int64_t *off, int32_t *cols)
{
    if (scale < 1 || scale > 30 || edge_factor < 1 || !off || !cols) return -1;
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    const int64_t n = (int64_t)1 << scale;
    const uint64_t m = (uint64_t)edge_factor << scale;
    rmat_spec R;
    R.scale = scale;
    R.seed = seed;
    R.A = (uint32_t)(a * 4294967296.0);
    R.AB = (uint32_t)((a + b) * 4294967296.0);
    R.ABC = (uint32_t)((a + b + c) * 4294967296.0);
    R.perm = NULL;

    int32_t *perm = NULL;
    if (relabel) {
        perm = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
        if (!perm) return -1;
        for (int64_t v = 0; v < n; v++) perm[v] = (int32_t)v;
        for (int64_t j = n - 1; j >= 1; j--) {
            const uint64_t x = h3(seed, (uint64_t)j, (uint64_t)1 << 40);
            const int64_t k = (int64_t)(((unsigned __int128)x * (uint64_t)(j + 1)) >> 64);
            const int32_t t = perm[j];
            perm[j] = perm[k];
            perm[k] = t;
        }
        R.perm = perm;
    }

    int64_t *cnt = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    int64_t *ndeg = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    task *tasks = (task *)calloc((size_t)nthreads, sizeof(task));
    if (!cnt || !ndeg || !tasks) {
        free(perm); free(cnt); free(ndeg); free(tasks);
        return -1;
    }
    for (int k = 0; k < nthreads; k++) {
        tasks[k].R = &R;
        tasks[k].lo = m * (uint64_t)k / (uint64_t)nthreads;
        tasks[k].hi = m * (uint64_t)(k + 1) / (uint64_t)nthreads;
        tasks[k].cnt = cnt;
        tasks[k].cols = cols;
    }
    run_threads(nthreads, tasks, count_pass);
    off[0] = 0;
    for (int64_t v = 0; v < n; v++) off[v + 1] = off[v] + cnt[v];
    memcpy(cnt, off, sizeof(int64_t) * (size_t)n);
    run_threads(nthreads, tasks, scatter_pass);

    /* rows split into nthreads ranges of about equal entry counts */
    const int64_t total = off[n];
    int64_t v0 = 0;
    for (int k = 0; k < nthreads; k++) {
        const int64_t target = total * (int64_t)(k + 1) / nthreads;
        int64_t v1 = v0;
        if (k == nthreads - 1) v1 = n;
        else while (v1 < n && off[v1] < target) v1++;
        tasks[k].n = n;
        tasks[k].off = off;
        tasks[k].ndeg = ndeg;
        tasks[k].vlo = v0;
        tasks[k].vhi = v1;
        v0 = v1;
    }
    run_threads(nthreads, tasks, row_pass);

    /* pack the deduplicated rows to the left, in order */
    int64_t w = 0;
    for (int64_t v = 0; v < n; v++) {
        const int64_t from = off[v];
        off[v] = w;
        if (from != w && ndeg[v] > 0) memmove(cols + w, cols + from, sizeof(int32_t) * (size_t)ndeg[v]);
        w += ndeg[v];
    }
    off[n] = w;
    free(perm);
    free(cnt);
    free(ndeg);
    free(tasks);
    return w;
}
