/*
 * dls_oracle.c -- slow, plain reference counter for (diagonal, vertically
 * symmetric) Latin squares.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes
 * or calls this file; it exists so that tests, the smoke check and the CPU
 * baseline leg of the benchmark can check the CUDA path against an
 * independent implementation.  It shares no code, header, table or helper
 * with the CUDA path.
 *
 * What it computes (Section 1 and Section 2.2 of the paper, Algorithms 1 and
 * 2): cells of an N x N square are filled one at a time in a given fill order.
 * For each cell every value 0..N-1 is tried in ascending order; a value is
 * accepted when it is not already used in the cell's row or column, nor (for
 * diagonal squares) on the main diagonal when i == j or on the anti-diagonal
 * when i + j == N-1.  Occupancy is kept in value-indexed boolean arrays
 * (rows[i][v], cols[j][v], md[v], ad[v]) exactly as in Algorithm 2 -- the
 * bitmask forms of Algorithms 3 and 4 are deliberately NOT used here.  When
 * the last cell of the order has been filled the square counter is
 * incremented (Algorithm 1).
 *
 * Vertical symmetry (Section 5.4): A[i][j] + A[i][N-1-j] == N-1.  Filling
 * cell (i, j) with v also fills its mirror (i, N-1-j) with N-1-v; both cells
 * are checked against all constraints like any other cell.  A cell in the
 * middle column of an odd order is its own mirror and may only take
 * (N-1)/2.  For odd N the middle-column cells are appended to the given
 * order (they are implied by the definition even when the caller lists only
 * left-half cells), so every vertically symmetric count of odd order N >= 3
 * comes out as 0.
 *
 * Count(P) for a prefix P (values of the first `depth` cells of the order) is
 * the number of ways to assign all remaining cells of the order consistently
 * with P.  When the order covers every cell this is the number of full squares
 * that agree with P; a shorter order counts partial squares (used for the
 * hourglass count of Section 4.2 and the partial counts of Section 5.3).
 *
 * A "node" is one accepted placement of a value into a cell at a position at
 * or after the prefix depth (the last cell's placements included), i.e. one
 * execution of the body of a loop of Algorithm 1 past its occupancy test.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

#define OR_MAXN 16
#define OR_MAXCELLS (OR_MAXN * OR_MAXN)

#define OR_DIAGONAL 1u
#define OR_VSYM 2u

typedef struct {
    int n;
    int diagonal;
    int vsym;
    int len;                           /* number of cells in the fill order */
    int ci[OR_MAXCELLS], cj[OR_MAXCELLS];
    int ls[OR_MAXN][OR_MAXN];          /* -1 = not assigned                 */
    unsigned char rows[OR_MAXN][OR_MAXN]; /* rows[i][v]: v used in row i     */
    unsigned char cols[OR_MAXN][OR_MAXN]; /* cols[j][v]: v used in column j  */
    unsigned char md[OR_MAXN];         /* v used on the main diagonal        */
    unsigned char ad[OR_MAXN];         /* v used on the anti-diagonal        */
    uint64_t count;                    /* completions found                  */
    uint64_t nodes;                    /* accepted placements past the prefix */
    /* prefix-enumeration mode */
    int stop;                          /* emit a record at this position     */
    int prefix_depth;
    uint8_t *out;
    int64_t cap, n_out, parent;
    int64_t *parents_out;
} or_state;

/* May value v go into cell (i, j) given what is already assigned? */
static int or_fits(const or_state *s, int i, int j, int v)
{
    if (s->ls[i][j] >= 0) return 0;
    if (s->rows[i][v]) return 0;
    if (s->cols[j][v]) return 0;
    if (s->diagonal && i == j && s->md[v]) return 0;
    if (s->diagonal && i + j == s->n - 1 && s->ad[v]) return 0;
    return 1;
}

static void or_mark(or_state *s, int i, int j, int v, int on)
{
    s->ls[i][j] = on ? v : -1;
    s->rows[i][v] = (unsigned char)on;
    s->cols[j][v] = (unsigned char)on;
    if (s->diagonal && i == j) s->md[v] = (unsigned char)on;
    if (s->diagonal && i + j == s->n - 1) s->ad[v] = (unsigned char)on;
}

/* Assign v to (i, j) -- and N-1-v to the mirror cell when vertically
 * symmetric.  Returns 1 and leaves the assignment in place on success,
 * returns 0 and changes nothing otherwise. */
static int or_assign(or_state *s, int i, int j, int v)
{
    if (v < 0 || v >= s->n) return 0;
    if (!or_fits(s, i, j, v)) return 0;
    if (!s->vsym) {
        or_mark(s, i, j, v, 1);
        return 1;
    }
    int mj = s->n - 1 - j, mv = s->n - 1 - v;
    if (mj == j) {                     /* middle column: its own mirror */
        if (mv != v) return 0;
        or_mark(s, i, j, v, 1);
        return 1;
    }
    or_mark(s, i, j, v, 1);
    if (!or_fits(s, i, mj, mv)) {
        or_mark(s, i, j, v, 0);
        return 0;
    }
    or_mark(s, i, mj, mv, 1);
    return 1;
}

static void or_unassign(or_state *s, int i, int j)
{
    int v = s->ls[i][j];
    or_mark(s, i, j, v, 0);
    if (s->vsym) {
        int mj = s->n - 1 - j;
        if (mj != j) or_mark(s, i, mj, s->n - 1 - v, 0);
    }
}

/* Algorithm 1 written as a recursion over positions of the fill order. */
static void or_search(or_state *s, int t)
{
    if (s->out != NULL && t == s->stop) {
        if (s->n_out < s->cap) {
            uint8_t *rec = s->out + (size_t)s->n_out * (size_t)s->stop;
            for (int u = 0; u < s->stop; ++u)
                rec[u] = (uint8_t)s->ls[s->ci[u]][s->cj[u]];
            if (s->parents_out) s->parents_out[s->n_out] = s->parent;
        }
        s->n_out++;
        return;
    }
    if (t == s->len) {
        s->count++;
        return;
    }
    int i = s->ci[t], j = s->cj[t];
    for (int v = 0; v < s->n; ++v) {
        if (!or_assign(s, i, j, v)) continue;
        if (t >= s->prefix_depth) s->nodes++;
        or_search(s, t + 1);
        or_unassign(s, i, j);
    }
}

/* Set up the state for one order; returns 0 on bad arguments. */
static int or_init(or_state *s, int n, unsigned flags, const uint8_t *order,
                   int order_len)
{
    if (n < 1 || n > OR_MAXN || order_len < 0 || order_len > n * n) return 0;
    memset(s, 0, sizeof(*s));
    s->n = n;
    s->diagonal = (flags & OR_DIAGONAL) != 0;
    s->vsym = (flags & OR_VSYM) != 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) s->ls[i][j] = -1;
    for (int t = 0; t < order_len; ++t) {
        s->ci[t] = order[2 * t];
        s->cj[t] = order[2 * t + 1];
        if (s->ci[t] >= n || s->cj[t] >= n) return 0;
    }
    s->len = order_len;
    if (s->vsym && (n % 2) == 1) {
        /* the middle column is part of every vertically symmetric square */
        int m = n / 2;
        for (int i = 0; i < n; ++i) {
            int listed = 0;
            for (int t = 0; t < order_len; ++t)
                if (s->ci[t] == i && s->cj[t] == m) listed = 1;
            if (!listed) {
                s->ci[s->len] = i;
                s->cj[s->len] = m;
                s->len++;
            }
        }
    }
    return 1;
}

/* Apply a prefix; returns 1 if every value could be placed. */
static int or_apply_prefix(or_state *s, const uint8_t *prefix, int depth)
{
    for (int t = 0; t < depth; ++t)
        if (!or_assign(s, s->ci[t], s->cj[t], prefix[t])) return 0;
    return 1;
}

/* ---------------------------------------------------------------- API -- */

/* Count completions of one prefix.  Returns 0 on success, -1 on bad args. */
int oracle_count(int n, unsigned flags, const uint8_t *order, int order_len,
                 const uint8_t *prefix, int depth, uint64_t *count_out,
                 uint64_t *nodes_out)
{
    or_state *s = (or_state *)malloc(sizeof(or_state));
    if (!s) return -1;
    if (!or_init(s, n, flags, order, order_len) || depth < 0 ||
        depth > order_len) {
        free(s);
        return -1;
    }
    s->prefix_depth = depth;
    if (or_apply_prefix(s, prefix, depth)) or_search(s, depth);
    if (count_out) *count_out = s->count;
    if (nodes_out) *nodes_out = s->nodes;
    free(s);
    return 0;
}

typedef struct {
    int n;
    unsigned flags;
    const uint8_t *order;
    int order_len;
    const uint8_t *prefixes;
    int depth;
    int64_t n_prefixes;
    uint64_t *counts;
    uint64_t *nodes;
    int64_t next;
    pthread_mutex_t lock;
    int failed;
} or_job;

static void *or_worker(void *arg)
{
    or_job *job = (or_job *)arg;
    for (;;) {
        pthread_mutex_lock(&job->lock);
        int64_t p = job->next++;
        pthread_mutex_unlock(&job->lock);
        if (p >= job->n_prefixes) break;
        uint64_t c = 0, nd = 0;
        if (oracle_count(job->n, job->flags, job->order, job->order_len,
                         job->prefixes + (size_t)p * (size_t)job->depth,
                         job->depth, &c, &nd) != 0)
            job->failed = 1;
        job->counts[p] = c;
        if (job->nodes) job->nodes[p] = nd;
    }
    return NULL;
}

/* Count every prefix of a batch (prefixes are `depth` bytes each, packed)
 * on `threads` POSIX threads that take prefixes one at a time. */
int oracle_count_many(int n, unsigned flags, const uint8_t *order,
                      int order_len, const uint8_t *prefixes, int depth,
                      int64_t n_prefixes, uint64_t *counts_out,
                      uint64_t *nodes_out, int threads)
{
    or_job job;
    memset(&job, 0, sizeof(job));
    job.n = n;
    job.flags = flags;
    job.order = order;
    job.order_len = order_len;
    job.prefixes = prefixes;
    job.depth = depth;
    job.n_prefixes = n_prefixes;
    job.counts = counts_out;
    job.nodes = nodes_out;
    pthread_mutex_init(&job.lock, NULL);
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    pthread_t tid[256];
    int started = 0;
    for (int t = 1; t < threads; ++t)
        if (pthread_create(&tid[started], NULL, or_worker, &job) == 0) started++;
    or_worker(&job);
    for (int t = 0; t < started; ++t) pthread_join(tid[t], NULL);
    pthread_mutex_destroy(&job.lock);
    return job.failed ? -1 : 0;
}

/* Enumerate every valid assignment of the first `depth` cells of the order
 * that extends one of the base prefixes (each `base_depth` bytes), in
 * ascending lexicographic order of values along the fill order, base
 * prefixes in the given order.  Writes at most `cap` records of `depth`
 * bytes to `out` (and the index of the base prefix each came from to
 * `parents_out`, if not NULL).  Returns the total number of records, which
 * may exceed `cap`, or -1 on bad arguments. */
int64_t oracle_extend(int n, unsigned flags, const uint8_t *order,
                      int order_len, const uint8_t *base, int base_depth,
                      int64_t n_base, int depth, uint8_t *out, int64_t cap,
                      int64_t *parents_out)
{
    or_state *s = (or_state *)malloc(sizeof(or_state));
    if (!s) return -1;
    if (!or_init(s, n, flags, order, order_len) || base_depth < 0 ||
        depth < base_depth || depth > order_len || out == NULL) {
        free(s);
        return -1;
    }
    s->stop = depth;
    s->out = out;
    s->cap = cap;
    s->parents_out = parents_out;
    s->prefix_depth = depth;
    for (int64_t b = 0; b < n_base; ++b) {
        for (int i = 0; i < n; ++i)
            for (int j = 0; j < n; ++j)
                if (s->ls[i][j] >= 0) or_unassign(s, i, j);
        s->parent = b;
        if (!or_apply_prefix(s, base + (size_t)b * (size_t)base_depth,
                             base_depth))
            continue;
        or_search(s, base_depth);
    }
    int64_t total = s->n_out;
    free(s);
    return total;
}

/* Draw-driven random prefix ("random walk"), used to build the partial
 * squares of the serving workload.  Cells F[0..depth-1] are filled in order;
 * the order must list each row's cells contiguously.  For each cell the
 * values that may be placed are listed in ascending order and the next draw
 * picks one of them (draw modulo the number of choices).  If a cell has no
 * value left, every cell of its row that was filled in this row pass is
 * cleared and the row starts again (a restart takes no draw).  Returns the
 * number of draws used, or -1 if they ran out first (or on bad arguments). */
int64_t oracle_sample_prefix(int n, unsigned flags, const uint8_t *order,
                             int order_len, int depth, const uint32_t *draws,
                             int64_t n_draws, uint8_t *out)
{
    or_state *s = (or_state *)malloc(sizeof(or_state));
    if (!s) return -1;
    if (!or_init(s, n, flags, order, order_len) || depth < 0 ||
        depth > order_len) {
        free(s);
        return -1;
    }
    int64_t used = 0;
    int t = 0;
    while (t < depth) {
        int i = s->ci[t], j = s->cj[t];
        int choices[OR_MAXN], nc = 0;
        for (int v = 0; v < n; ++v) {
            if (or_assign(s, i, j, v)) {
                choices[nc++] = v;
                or_unassign(s, i, j);
            }
        }
        if (nc == 0) {
            /* clear this row's cells of the current pass and restart it */
            int r = t;
            while (r > 0 && s->ci[r - 1] == i) r--;
            for (int u = r; u < t; ++u) or_unassign(s, s->ci[u], s->cj[u]);
            t = r;
            continue;
        }
        if (used >= n_draws) {
            free(s);
            return -1;
        }
        int v = choices[draws[used++] % (uint32_t)nc];
        or_assign(s, i, j, v);
        out[t] = (uint8_t)v;
        t++;
    }
    free(s);
    return used;
}

/* ------------------------------------------------ symmetry breaking --
 *
 * Section 4.  An hourglass design has row 0, the last row and both diagonals
 * filled.  The M-transformations that keep hourglasses (Section 4.2) are
 * generated by
 *   - the vertical mirror, column j -> N-1-j (not for vertically symmetric
 *     squares: there it only renames the symbols, Section 5.4);
 *   - for any subset S of {0..N/2-1}: swap rows k, N-1-k and columns k,
 *     N-1-k for every k in S (the second type of Section 4.1);
 *   - for any permutation s of {1..N/2-1}: row and column k -> s(k) and
 *     N-1-k -> N-1-s(k) (the third type, with index 0 kept in place so that
 *     row 0 only ever trades places with the last row).
 * After a transformation the symbols are renamed so that row 0 reads
 * 0..N-1 (Section 4.1).  Algorithm 5: an hourglass is canonic when no image
 * is lexicographically smaller (cells compared in row-major order); its class
 * size is the number of distinct images. */

typedef struct {
    int n;
    int a[OR_MAXN][OR_MAXN];   /* -1 = empty */
} or_grid;

static void or_apply(const or_grid *src, or_grid *dst, int mirror,
                     unsigned subset, const int *perm)
{
    int n = src->n, h = n / 2;
    or_grid t1, t2;
    /* vertical mirror */
    t1.n = n;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            t1.a[i][j] = mirror ? src->a[i][n - 1 - j] : src->a[i][j];
    /* symmetric row+column pair swaps */
    int sw[OR_MAXN];
    for (int k = 0; k < n; ++k) sw[k] = k;
    for (int k = 0; k < h; ++k)
        if (subset >> k & 1u) {
            sw[k] = n - 1 - k;
            sw[n - 1 - k] = k;
        }
    t2.n = n;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) t2.a[sw[i]][sw[j]] = t1.a[i][j];
    /* paired permutation of the left-half indices and their mirrors */
    int pm[OR_MAXN];
    for (int k = 0; k < n; ++k) pm[k] = k;
    for (int k = 0; k < h; ++k) {
        pm[k] = perm[k];
        pm[n - 1 - k] = n - 1 - perm[k];
    }
    dst->n = n;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) dst->a[pm[i]][pm[j]] = t2.a[i][j];
    /* rename the symbols so that row 0 reads 0..N-1 */
    int ren[OR_MAXN];
    for (int j = 0; j < n; ++j) ren[dst->a[0][j]] = j;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j)
            if (dst->a[i][j] >= 0) dst->a[i][j] = ren[dst->a[i][j]];
}

static int or_grid_cmp(const or_grid *x, const or_grid *y)
{
    for (int i = 0; i < x->n; ++i)
        for (int j = 0; j < x->n; ++j)
            if (x->a[i][j] != y->a[i][j]) return x->a[i][j] < y->a[i][j] ? -1 : 1;
    return 0;
}

/* next permutation of p[0..m-1] in lexicographic order; 0 when done */
static int or_next_perm(int *p, int m)
{
    int i = m - 2;
    while (i >= 0 && p[i] >= p[i + 1]) i--;
    if (i < 0) return 0;
    int j = m - 1;
    while (p[j] <= p[i]) j--;
    int t = p[i]; p[i] = p[j]; p[j] = t;
    for (int a = i + 1, b = m - 1; a < b; ++a, --b) {
        t = p[a]; p[a] = p[b]; p[b] = t;
    }
    return 1;
}

/* Class size of one hourglass if it is canonic, else 0 (Algorithm 5).  The
 * hourglass is given as the values of the first `len` cells of `order`
 * (row 0 must be 0..N-1); with vertical symmetry the cells are left-half
 * cells and their mirrors are filled in.  Orders 2..11.  Returns -1 on bad
 * arguments. */
long oracle_hourglass_class(int n, unsigned flags, const uint8_t *order, int len,
                            const uint8_t *values)
{
    if (n < 2 || n > 11 || len < 0 || len > n * n) return -1;
    int vsym = (flags & OR_VSYM) != 0;
    or_grid H;
    H.n = n;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) H.a[i][j] = -1;
    for (int t = 0; t < len; ++t) {
        int i = order[2 * t], j = order[2 * t + 1];
        H.a[i][j] = values[t];
        if (vsym) H.a[i][n - 1 - j] = n - 1 - values[t];
    }
    for (int j = 0; j < n; ++j)
        if (H.a[0][j] != j) return -1;
    int h = n / 2;
    /* at most 2 * 2^5 * 4! = 1536 images for N <= 11 */
    static __thread or_grid eqc[2 * (1 << 5) * 24];
    long k = 0;
    int perm[OR_MAXN];
    for (int mirror = 0; mirror < (vsym ? 1 : 2); ++mirror) {
        for (unsigned subset = 0; subset < (1u << h); ++subset) {
            for (int t = 0; t < h; ++t) perm[t] = t;
            do {
                or_grid T;
                or_apply(&H, &T, mirror, subset, perm);
                if (or_grid_cmp(&T, &H) < 0) return 0;
                if (k < (long)(sizeof(eqc) / sizeof(eqc[0]))) eqc[k] = T;
                k++;
            } while (or_next_perm(perm + 1, h - 1));
        }
    }
    /* ComputeDistinct: count images not equal to an earlier image */
    long distinct = 0;
    for (long x = 0; x < k; ++x) {
        int seen = 0;
        for (long y = 0; y < x && !seen; ++y)
            if (or_grid_cmp(&eqc[x], &eqc[y]) == 0) seen = 1;
        if (!seen) distinct++;
    }
    return distinct;
}

typedef struct {
    int n;
    unsigned flags;
    const uint8_t *order;
    int len;
    const uint8_t *values;
    int64_t count;
    long *out;
    int64_t next;
    pthread_mutex_t lock;
} or_canon_job;

static void *or_canon_worker(void *arg)
{
    or_canon_job *job = (or_canon_job *)arg;
    for (;;) {
        pthread_mutex_lock(&job->lock);
        int64_t lo = job->next;
        job->next += 256;
        pthread_mutex_unlock(&job->lock);
        if (lo >= job->count) break;
        int64_t hi = lo + 256 < job->count ? lo + 256 : job->count;
        for (int64_t q = lo; q < hi; ++q)
            job->out[q] = oracle_hourglass_class(job->n, job->flags, job->order, job->len,
                                                 job->values + (size_t)q * job->len);
    }
    return NULL;
}

/* oracle_hourglass_class over many hourglasses on `threads` threads. */
int oracle_hourglass_classes(int n, unsigned flags, const uint8_t *order, int len,
                             const uint8_t *values, int64_t count, long *out,
                             int threads)
{
    or_canon_job job;
    memset(&job, 0, sizeof(job));
    job.n = n;
    job.flags = flags;
    job.order = order;
    job.len = len;
    job.values = values;
    job.count = count;
    job.out = out;
    pthread_mutex_init(&job.lock, NULL);
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    pthread_t tid[256];
    int started = 0;
    for (int t = 1; t < threads; ++t)
        if (pthread_create(&tid[started], NULL, or_canon_worker, &job) == 0) started++;
    or_canon_worker(&job);
    for (int t = 0; t < started; ++t) pthread_join(tid[t], NULL);
    pthread_mutex_destroy(&job.lock);
    return 0;
}
