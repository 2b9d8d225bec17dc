/*
 * dls.h -- C ABI of the GB300 enumerator of diagonal Latin squares
 * (Kochemazov, Vatutin, Zaikin, "Fast Algorithm for Enumerating Diagonal
 * Latin Squares of Small Order").
 *
 * Definitions (Section 1): a Latin square of order N is an N x N array over
 * {0..N-1} whose rows and columns are permutations.  It is diagonal when the
 * main diagonal and the anti-diagonal are permutations too, and vertically
 * symmetric when A[i][N-1-j] == N-1-A[i][j] for all i, j (Section 5.4).
 *
 * The method (Sections 2-3): cells are filled one at a time in a fixed fill
 * order; one bitmask per row, column and diagonal records the values in use;
 * a cell's admissible values are ALL & ~(row | column | diagonals) and are
 * visited lowest bit first (Algorithm 4).  The search tree is split at a
 * fixed depth into independent subproblems ("prefixes", Section 5.2) whose
 * counts are summed.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - n: the order, 1 <= n <= DLS_MAX_N.
 * - flags: OR of DLS_DIAGONAL and DLS_VSYM (0 = ordinary Latin squares).
 * - order: host array of order_len (i, j) byte pairs, the fill order.  Cells
 *   must be distinct and inside the square.  With DLS_VSYM every cell must be
 *   in the left half (j < n/2); its mirror (i, n-1-j) is filled with the
 *   mirrored value at the same time.  The order need not cover the square:
 *   a shorter order counts partial squares (Section 5.3 counts the first k
 *   cells in row-major order that way).
 * - prefix: the values of the first `depth` cells of the order, one byte per
 *   cell (0..n-1), prefixes packed back to back (`depth` bytes each).  Row 0
 *   is not special: to fix it to 0..n-1 (Section 2.2), start the order with
 *   row 0 and put 0..n-1 (left half with DLS_VSYM) in every prefix.
 * - Count(prefix) = number of ways to give every remaining cell of the order
 *   (and its mirror with DLS_VSYM) a value so that no value repeats in a row,
 *   a column and, with DLS_DIAGONAL, on either diagonal, among the cells
 *   assigned.  A prefix that breaks a constraint or holds a value >= n has
 *   count 0.  With DLS_VSYM and odd n >= 3 every count is 0: the middle
 *   column would have to hold (n-1)/2 in every row.
 * - All counts are exact unsigned 64-bit integers.
 * - Return value: DLS_OK (0) or a dls_status code; dls_strerror() names it.
 *   Device work is asynchronous on the given CUDA stream (NULL = legacy
 *   default stream); errors raised by the GPU while it runs are reported by
 *   the next call that synchronises.
 */
#ifndef DLS_H
#define DLS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DLS_MAX_N 16
#define DLS_MAX_CELLS (DLS_MAX_N * DLS_MAX_N)

/* flags */
#define DLS_DIAGONAL 1u
#define DLS_VSYM 2u

typedef enum {
    DLS_OK = 0,
    DLS_ERR_INVALID_N = 1,    /* n outside 1..DLS_MAX_N                      */
    DLS_ERR_BAD_ORDER = 2,    /* repeated / out-of-range / right-half cell   */
    DLS_ERR_BAD_ARG = 3,      /* NULL pointer, negative size, bad depth ...  */
    DLS_ERR_CAPACITY = 4,     /* output buffer too small; *n_out = needed    */
    DLS_ERR_CUDA = 5,         /* a CUDA call failed (dls_last_cuda_error())  */
    DLS_ERR_TIMEOUT = 6,      /* a count ran out of its iteration budget     */
    DLS_ERR_ABORTED = 7,      /* stopped through dls_server_abort() or a
                                 count's abort flag                         */
    DLS_ERR_NO_MEMORY = 8,    /* host or device allocation failed            */
    DLS_ERR_BAD_STATE = 9,    /* object used after release / wrong sequence  */
    DLS_ERR_INTERNAL = 10     /* a kernel met a state its bounds exclude
                                 (its counts are not to be trusted)          */
} dls_status;

/* kinds of fill order for dls_fill_order() */
typedef enum {
    /* rows 0..first_rows-1, then the main diagonal, then the anti-diagonal,
     * then the remaining cells row by row (Section 2.3 fills the diagonals
     * first; Section 4.3 keeps them first) */
    DLS_ORDER_MD_AD_ROWS = 0,
    /* row by row, left to right (the trivial order of Sections 2.1, 5.3) */
    DLS_ORDER_ROW_MAJOR = 1,
    /* row 0, both diagonals, last row, then the rest: the cells of an
     * hourglass design first (Section 4.2); left half with DLS_VSYM */
    DLS_ORDER_HOURGLASS = 2,
    /* the greedy most-constrained-cell order of Section 2.3 with its
     * forced-last-cell rule (Fig. 1 for order 9) */
    DLS_ORDER_HEURISTIC = 3,
    /* not in the paper: the same greedy rule with V = the sum of the
     * squares of the assigned-cell counts of the cell's lines (a cell on one
     * nearly complete line goes before one on several half-filled lines);
     * on the order-8 split after both diagonals and row 1 it searches ~16 %
     * fewer nodes per square -- an autotuner candidate */
    DLS_ORDER_HEURISTIC_SQ = 4
} dls_order_kind;

typedef struct {
    uint64_t lo, hi;
} dls_u128;

/* ------------------------------------------------------------------ info */

/* Name of a status code (static string, never NULL). */
const char *dls_strerror(int code);

/* Last CUDA error string seen by the library on this thread ("" if none). */
const char *dls_last_cuda_error(void);

/* Library version, (major << 16) | minor. */
int dls_version(void);

/* ------------------------------------------------------ host-side setup */

/* Fill order of the given kind (Sections 2.3, 4.2).  Writes up to `cap` (i,j)
 * pairs to ij_out (2*cap bytes) and their number to *len_out.  first_rows
 * (>= 1) only affects DLS_ORDER_MD_AD_ROWS.  With DLS_VSYM only left-half
 * cells are listed.  Host memory; caller owns both buffers.  Errors:
 * INVALID_N, BAD_ARG, CAPACITY (*len_out = needed). */
int dls_fill_order(int n, uint32_t flags, int kind, int first_rows,
                   uint8_t *ij_out, int cap, int *len_out);

/* Completes a fill order: keeps its first `keep` cells and appends every
 * other cell of the square (left half with DLS_VSYM) by the rule of `kind`
 * applied from the kept cells -- DLS_ORDER_HEURISTIC: the greedy
 * most-constrained-cell order with the forced-last-cell rule of Section 2.3
 * (the cell values never matter, so the completion depends only on which
 * cells are kept); DLS_ORDER_HEURISTIC_SQ: its squared-count variant;
 * DLS_ORDER_MD_AD_ROWS: remaining diagonal cells, then the
 * rest row by row; DLS_ORDER_ROW_MAJOR: the rest row by row.  Counts do not
 * depend on the order of the cells after a prefix, so this changes only the
 * size of the search (Section 2.3).  Host memory, caller-owned.  Errors as
 * dls_fill_order, BAD_ORDER for a bad kept part. */
int dls_order_complete(int n, uint32_t flags, const uint8_t *order, int keep,
                       int kind, uint8_t *ij_out, int cap, int *len_out);

/* Shortens a fill order that lists every cell of the square, without
 * changing any count.  First, of the order's last `window` cells (none
 * before position `keep`), those on the row of the last cell move to the
 * end, in their order; or those on its column, whichever leaves the longer
 * run below.  Then the run of cells at the end that lie on that one line
 * and on neither diagonal (with DLS_DIAGONAL) is dropped, leaving at least
 * one cell after `keep`.
 * Why the count stays: once every other cell is filled, each dropped cell
 * is the last open cell of its column (of its row, for a column run), so
 * its value is the one that column lacks (Section 2.4.1 computes such a
 * value directly).  Counting each value's occurrences in the full rows and
 * columns shows that these values are exactly the values the run's line
 * lacks, each once; no diagonal is involved.  So every filling of the kept
 * cells has exactly one completion, and a count over the shortened order
 * -- which counts fillings of its cells -- equals the count over the full
 * order.  The cells before `keep` (a prefix) keep their places, so
 * prefixes made with either order are the same.  The search gets shorter
 * by the dropped cells, and moving the line's cells within the window
 * lets more of them drop (window 0: only the run already at the end).
 * With DLS_VSYM (left-half cells; Section 5.4) only a row's run drops: each
 * cell is still the last open cell of its column, and since every full row
 * holds one value of each pair {v, N-1-v} in its left half and every left
 * column holds both, the forced values give the run's row one value of
 * each pair it lacks and none of a pair it has; a column's last left cell
 * is not forced (either value of a pair may fit).  An order that does not
 * list every cell (every left-half cell with DLS_VSYM; a partial order,
 * whose count is of partial squares), or DLS_VSYM with odd N, is copied
 * unchanged.
 * Writes up to `cap` (i,j) pairs to ij_out and their number to *len_out.
 * Host memory, caller-owned.  Errors: as dls_fill_order, BAD_ORDER for a bad
 * order, BAD_ARG for keep outside [0, order_len] or window < 0. */
int dls_order_trim(int n, uint32_t flags, const uint8_t *order, int order_len,
                   int keep, int window, uint8_t *ij_out, int cap, int *len_out);

/* The prefix split of Section 5.2: every valid assignment of the first
 * `depth` order cells that extends one of the n_base base prefixes (each
 * base_depth bytes), base prefixes in turn, each one's extensions in
 * ascending lexicographic order of the values along the fill order.  Writes
 * at most `cap` records of `depth` bytes to out and, if parents_out is not
 * NULL, the index of the base prefix of each record; *n_out = number of
 * records (also when it exceeds cap, with DLS_ERR_CAPACITY).  Invalid base
 * prefixes have no extensions.  Host memory, caller-owned. */
int dls_extend_prefixes(int n, uint32_t flags, const uint8_t *order,
                        int order_len, const uint8_t *base, int base_depth,
                        int64_t n_base, int depth, uint8_t *out, int64_t cap,
                        int64_t *parents_out, int64_t *n_out);

/* A random valid prefix built from caller-supplied uniform draws (used for
 * the partial squares of the serving workload).  Cells are filled in order;
 * each row's cells must be contiguous in the order.  For each cell the
 * admissible values are listed in ascending order and draws[k] % count picks
 * one (one draw per cell filled); when a cell has no admissible value, the
 * cells of its row filled in the current pass are cleared and the row starts
 * again, taking no draw.  Writes `depth` bytes to out and the number of
 * draws used to *draws_used.  DLS_ERR_CAPACITY if the draws run out first.
 * Host memory, caller-owned. */
int dls_sample_prefix(int n, uint32_t flags, const uint8_t *order,
                      int order_len, int depth, const uint32_t *draws,
                      int64_t n_draws, uint8_t *out, int64_t *draws_used);

/* An estimate of the size of the search below one prefix: the number of
 * values the search of Algorithm 4 places after the prefix (every accepted
 * placement, the last cell's included) -- the `nodes` a counting pass
 * reports.  Not a method of the paper: it is D. E. Knuth's random-descent
 * estimate ("Estimating the efficiency of backtrack programs", Math. Comp.
 * 29, 1975).  Each of `probes` descents fills the cells after the prefix in
 * order with an admissible value drawn uniformly at random, multiplying up
 * the numbers of admissible values met (d_1, d_1 d_2, ...) and summing those
 * products until a cell has none or the last cell is reached; *nodes_out =
 * the mean of the sums, an unbiased estimate.  The draws are splitmix64
 * (Steele, Lea and Flood 2014) of the counter (probe << 32 | cell position)
 * XORed with splitmix64(seed), taken modulo the number of admissible
 * values: the result is a pure function of the arguments.  The serving path
 * sizes its work items with it (seed = job id, 256 probes).  An invalid
 * prefix gives 0.  prefix: `depth` value bytes along the order, host
 * memory.  Errors: INVALID_N, BAD_ORDER, BAD_ARG (unknown flags, depth
 * outside [0, order_len], probes < 1, NULL nodes_out). */
int dls_estimate_nodes(int n, uint32_t flags, const uint8_t *order, int order_len,
                       const uint8_t *prefix, int depth, uint64_t seed, int probes,
                       double *nodes_out);

/* Number of squares represented by one square whose row 0 is 0..n-1:
 * n! for diagonal and ordinary Latin squares (Section 2.2; the order-9 total
 * of Section 5.2.1 is the fixed-row count times 9!), 2^(n/2) (n/2)! for
 * vertically symmetric ones of even order (the relabellings that commute
 * with v -> n-1-v), 1 for odd vertically symmetric orders. */
dls_u128 dls_multiplier(int n, uint32_t flags);

/* 128-bit a * b and a + b (totals of order 9 and above exceed 64 bits). */
dls_u128 dls_mul_u64(uint64_t a, dls_u128 b);
dls_u128 dls_add_u128(dls_u128 a, dls_u128 b);

/* -------------------------------------------------------- GPU counting */

typedef enum {
    DLS_KERNEL_PERSISTENT = 0, /* one resident grid, atomic work queue,
                                  in-warp work donation                     */
    DLS_KERNEL_PLAIN = 1       /* one thread per (prefix, lane) work item     */
} dls_kernel_kind;

/* Launch shape.  Zero fields take the defaults. */
typedef struct {
    int kernel;           /* dls_kernel_kind                                 */
    int block_threads;    /* 32..512, multiple of 32 (default 128)           */
    int blocks_per_sm;    /* persistent grid: blocks per SM (default: all that
                             fit)                                            */
    int lanes_per_prefix; /* 1,2,4,...,32 work items per prefix (default 1); a
                             prefix's item s takes the nodes at order
                             position split_pos whose DFS index is s mod
                             lanes_per_prefix                                */
    int split_pos;        /* order position of that split (default depth+2)  */
    int donate;           /* persistent only: 1 = idle lanes take work from
                             busy lanes of their warp once the queue is empty
                             (default), -1 = off                            */
    int check_every;      /* iterations between donation checks (persistent
                             kernels) and between checks of the budget and
                             abort flag (power of two, default 64)           */
    int words;            /* where a lane keeps its row and column words:
                             0 = registers when they fit (n <= 8, or even
                             n <= 10 with DLS_VSYM, or the snapshot search's
                             wide words for n = 9 with at most 8 rows after
                             the prefix), else shared memory; 1 = shared
                             memory; 2 = registers (BAD_ARG if they do not
                             fit)                                            */
    int stack;            /* the search's stack --
                             1 = one entry per order position (Algorithm 4's
                             L and LS per cell; backing out of a cell is one
                             step);
                             2 = snapshots: an entry (the line words, the
                             position and its untried candidates) only where
                             candidates remain after the one placed, so a
                             dead end returns to the deepest open cell in one
                             step (persistent and plain kernels alike);
                             register words and one lane per prefix only
                             (BAD_ARG otherwise); entries per lane =
                             positions after the prefix whose cell is not
                             forced by a line with all other cells earlier;
                             0 = snapshots where they apply (default)        */
    int lookahead;        /* 1 = lookahead (Section 2.4.2) in the persistent
                             snapshot search: a placement after which the cell
                             after the next one has no candidate is a dead end
                             at once; only where no cell after the prefix lies
                             on a diagonal and without DLS_VSYM (BAD_ARG
                             otherwise); same counts, fewer nodes.  0 = off
                             (default)                                       */
    int fuse;             /* the snapshot search's fused step: when the cell
                             after a placement has exactly one candidate (and
                             is not the last cell), the same iteration places
                             it -- the next iteration's move, so the counts,
                             nodes and stack entries are unchanged and the
                             iterations fewer; only where no cell after the
                             prefix lies on a diagonal and without the
                             lookahead.  1 = on (BAD_ARG where it
                             does not apply), -1 = off, 0 = on where it
                             applies, except with DLS_VSYM (default; with
                             the mirrored words the fused placement costs
                             more than it saves there)                      */
    int64_t budget;       /* stop early after this many search iterations per
                             lane (the lanes of a warp step together; 0 = no
                             limit) -- see "Stopping early" below          */
    int stack_cap;        /* snapshot entries per lane: 0 = the default --
                             the bound that no search can exceed, or for the
                             wide words of order 9 (32-byte entries) the
                             largest cap with which two blocks fit an SM,
                             where a cap applies; a smaller value leaves
                             more lanes resident -- see "Stack cap" below   */
    const volatile int *abort_flag; /* NULL, or a word the kernel polls (device
                             memory, or host memory the GPU can read, e.g.
                             pinned and mapped): once it reads nonzero, the
                             kernel stops early                             */
} dls_launch_t;

/* Stopping early (Section 5.2's workunits are restartable; this makes a long
 * launch restartable too).  With a budget or an abort flag, each warp checks
 * every check_every iterations (and whenever a lane finishes its prefix):
 * once its iterations reach the budget, or the flag reads nonzero, it stops.
 * A lane still searching gives up its prefix: bit 63 (DLS_UNFINISHED) of the
 * prefix's count is set (counts are below 2^63 for every order the library
 * takes), and the warp takes no further prefix.  The count's status (the
 * host-buffer entries' return value, or dls_stream_status /
 * dls_plan_status) becomes DLS_ERR_TIMEOUT or DLS_ERR_ABORTED when work was
 * left, and prefixes_started says how many leading prefixes were handed to
 * lanes.  To finish the job, count again the prefixes whose count has bit 63
 * set and those from prefixes_started on; every other count is exact.  The
 * total (d_total) is then partial.  No wait in the kernel depends on the
 * flag: a warp only reads it. */
#define DLS_UNFINISHED (1ull << 63)

/* Stack cap (dls_launch_t.stack_cap).  The snapshot search's stack has as
 * many entries per lane as the order has positions after the prefix whose
 * cell is not forced by a line -- a bound no search can exceed -- but real
 * searches stay far below it (order 8, split 25 cells into the order: bound
 * 25, deepest stack 19, and 0.15 % of the prefixes deeper than 16).  A
 * smaller cap leaves more lanes resident.  A lane whose stack would outgrow
 * the cap finishes its prefix at once and marks it; a second pass of the
 * same kernel, with the full bound, then counts the marked prefixes again
 * from zero (its idle lanes share their searches through donation), and the
 * total is summed from the counts.  Counts stay exact; both passes are
 * enqueued on the stream (and captured by plans).  The cap applies only with
 * per-prefix counts (d_counts), without a node count, a budget or an abort
 * flag; otherwise the bound is kept. */

/* What a dls_count_ex call with this shape runs. */
typedef enum {
    DLS_RUN_PERSISTENT = 0,     /* persistent grid, one stack entry per
                                   position                                 */
    DLS_RUN_PLAIN = 1,          /* one thread per work item, one stack entry
                                   per position                             */
    DLS_RUN_SNAPSHOT = 2,       /* persistent grid, snapshot stack          */
    DLS_RUN_PLAIN_SNAPSHOT = 3  /* one thread per prefix, snapshot stack    */
} dls_run_kind;

typedef struct {
    int run;              /* dls_run_kind                                    */
    int words;            /* 1 = row/column words in shared memory,
                             2 = in registers                                */
    int block_threads;
    int grid_blocks;      /* 0 = nothing to launch                           */
    int smem_bytes;       /* dynamic shared memory per block                 */
    int stack_entries;    /* snapshot entries per lane (0 otherwise)         */
    int fused;            /* 1 = the snapshot search takes the fused step    */
    int step;             /* the search step: 0 = one entry per position,
                             1 = snapshots with field shifts (vertical
                             symmetry), 2 = snapshots with byte words (n <= 8
                             without vertical symmetry), 3 = snapshots with
                             wide words (n = 9: values 0-7 in byte slots,
                             value 8 a bit per line)                         */
} dls_launch_info;

/* Resolves the kernel and launch shape that dls_count_ex would use for these
 * arguments, with per-prefix counts and no node count (same validation and
 * errors), without enqueueing anything.
 * Queries the current CUDA device (occupancy).  out: HOST, caller-owned. */
int dls_describe_launch(int n, uint32_t flags, const uint8_t *order,
                        int order_len, int depth, int64_t n_prefixes,
                        const dls_launch_t *cfg, dls_launch_info *out);

/* Count completions of every prefix on the GPU (Algorithm 4 on the device).
 * d_prefixes: DEVICE, n_prefixes * depth bytes (caller-owned).
 * d_counts:   DEVICE, n_prefixes uint64 (caller-owned) or NULL; overwritten
 *             with Count(prefix) for each prefix.
 * d_total:    DEVICE, one uint64 (caller-owned) or NULL; overwritten with the
 *             sum of all counts (exact; the caller must know it fits 64 bits).
 * stream:     cudaStream_t (NULL = default stream).
 * Uses a small per-(device, stream) work area that the library allocates on
 * first use and keeps until dls_release(); call once before capturing the
 * stream into a CUDA graph.  Asynchronous.  Errors: INVALID_N, BAD_ORDER,
 * BAD_ARG (depth outside 0..order_len, n_prefixes < 0, both outputs NULL),
 * CUDA, NO_MEMORY.  The persistent kernel is used (dls_count_ex selects). */
int dls_count(int n, uint32_t flags, const uint8_t *order, int order_len,
              const uint8_t *d_prefixes, int depth, int64_t n_prefixes,
              uint64_t *d_counts, uint64_t *d_total, void *stream);

/* Same counts from the plain one-thread-per-prefix launch (the comparison
 * baseline): no queue, no donation, one grid thread per prefix. */
int dls_count_plain(int n, uint32_t flags, const uint8_t *order,
                    int order_len, const uint8_t *d_prefixes, int depth,
                    int64_t n_prefixes, uint64_t *d_counts, uint64_t *d_total,
                    void *stream);

/* dls_count with an explicit launch shape (cfg may be NULL = defaults).
 * d_nodes: DEVICE, one uint64, or NULL.  If given, it is overwritten with
 * the number of nodes of the search -- accepted placements of a value into
 * a cell at order positions >= depth, the last position included (one pass
 * of the body of a loop of Algorithm 1 past its occupancy test) -- counted
 * by a separately compiled variant of the kernel. */
int dls_count_ex(int n, uint32_t flags, const uint8_t *order, int order_len,
                 const uint8_t *d_prefixes, int depth, int64_t n_prefixes,
                 uint64_t *d_counts, uint64_t *d_total, uint64_t *d_nodes,
                 const dls_launch_t *cfg, void *stream);

/* Host-buffer entry point: copies h_prefixes (HOST, n_prefixes*depth bytes;
 * page-locked memory makes the copy asynchronous) to the device, counts, and
 * copies the counts back to h_counts (HOST, n_prefixes uint64, may be NULL)
 * and the sum to *total_out (may be NULL; the plain 128-bit sum of the
 * counts -- multiply by dls_multiplier() for whole-square totals).  A count
 * that stops early returns DLS_ERR_TIMEOUT or DLS_ERR_ABORTED with its
 * counts copied back (unfinished ones marked DLS_UNFINISHED, those never
 * started 0) and *total_out not written.
 * Synchronous: returns after the copies back have landed.  The device
 * buffers come from a per-(device, stream) area that grows on demand and
 * lives until dls_release().  Calls on the same stream from several host
 * threads at once share that area (one may even reallocate it under the
 * other's kernel) and race: serialise them, or give each thread its own
 * stream.  Also returns DLS_ERR_INTERNAL if the snapshot
 * search reported a stack overflow (excluded by its entry bound; the kernel
 * drops the entry rather than write past its stack). */
int dls_count_host(int n, uint32_t flags, const uint8_t *order,
                   int order_len, const uint8_t *h_prefixes, int depth,
                   int64_t n_prefixes, uint64_t *h_counts,
                   dls_u128 *total_out, const dls_launch_t *cfg,
                   void *stream);

/* What the last count on a work area reported.  status: DLS_OK;
 * DLS_ERR_INTERNAL when the snapshot search reported a stack overflow
 * (excluded by its entry bound; the kernel drops the entry rather than write
 * past its stack, so the counts are not to be trusted); DLS_ERR_TIMEOUT or
 * DLS_ERR_ABORTED when it stopped early with work left (see "Stopping
 * early").  prefixes_started: the prefixes of which at least one work item
 * was handed to a lane (all of them once a count has run to its end). */
typedef struct {
    int status;
    int64_t prefixes_started;
} dls_count_status;

/* Status of the last count enqueued on `stream` (of the current device)
 * through dls_count, dls_count_plain or dls_count_ex: waits for the stream,
 * then reads the status word that each such count clears before its kernel
 * and the kernel sets.  This is how callers of the device-buffer entries
 * learn of a stack overflow (the host-buffer entries return it themselves).
 * out: HOST, caller-owned.  Returns DLS_OK when *out was filled; BAD_ARG
 * (out NULL), BAD_STATE (nothing counted on that stream since
 * dls_release()), CUDA. */
int dls_stream_status(void *stream, dls_count_status *out);

/* Counts every prefix (as dls_count_ex) and sums weight x Count over all of
 * them in 128 bits on the device: Algorithm 6's Total += Cnt * multiple
 * (Section 4.3), where the weight of an item is the class size of the
 * canonical hourglass it extends (Corollary 1), and with unit weights the
 * plain 128-bit total.  d_weights: DEVICE, n_prefixes uint32 (caller-owned),
 * or NULL for all 1.  d_counts: DEVICE, n_prefixes uint64 receiving the
 * counts, or NULL to keep them in the library's work area for `stream`
 * (grown on demand, shared with dls_count_host: the same race applies).
 * multiply: nonzero multiplies the total by dls_multiplier(n, flags) (row 0
 * fixed -> all squares, Section 2.2).  *total_out: HOST.  Synchronous.
 * Errors as dls_count_ex, BAD_ARG for a NULL total_out, and the count's
 * status (INTERNAL, TIMEOUT, ABORTED) with *total_out not written. */
int dls_count_weighted(int n, uint32_t flags, const uint8_t *order, int order_len,
                       const uint8_t *d_prefixes, int depth, int64_t n_prefixes,
                       const uint32_t *d_weights, uint64_t *d_counts, int multiply,
                       dls_u128 *total_out, const dls_launch_t *cfg, void *stream);

/* ---------------------------------------------------- symmetry breaking */

/* Canonical hourglasses (Section 4.2, Algorithm 5).  An hourglass design has
 * row 0, the last row and both diagonals filled; `order` lists exactly those
 * cells (left half with DLS_VSYM) -- e.g. the first cells of
 * DLS_ORDER_HOURGLASS -- and d_hourglasses (DEVICE, count * len bytes) holds
 * their values, one hourglass per record.  For each, d_class_size (DEVICE,
 * count uint32) receives the size of its class under the M-transformations
 * that keep hourglasses (Section 4.1: vertical mirror -- not with DLS_VSYM,
 * Section 5.4 --, symmetric row+column pair swaps, paired permutations of
 * the indices 1..n/2-1) if it is the lexicographically least member after
 * row 0 is renamed to 0..n-1, else 0.  By Proposition 1 / Corollary 1 the
 * number of squares with row 0 fixed is the sum over canonical hourglasses
 * of class size x completions.  DLS_DIAGONAL required; 2 <= n <= 11 (even n
 * with DLS_VSYM).  Asynchronous on `stream`.  Errors: INVALID_N, BAD_ARG,
 * BAD_ORDER (cells are not the hourglass cells), CUDA. */
int dls_hourglass_classes(int n, uint32_t flags, const uint8_t *order, int len,
                          const uint8_t *d_hourglasses, int64_t count,
                          uint32_t *d_class_size, void *stream);

/* ------------------------------------------------------------ serving */

/* A continuous-batching server for counting jobs of mixed order, flags and
 * prefix (the job answer is Count(prefix), as for dls_count).  Jobs are split
 * on the host into work items (the prefix split of Section 5.2, extended
 * until a job has one item per lane, or more for a big job -- see
 * item_nodes), wait in arrival order, and are
 * admitted at an epoch boundary when a job slot and enough free chunks of the
 * device item arena (the memory budget) are free; an admitted job's items
 * are copied to the arena.  Each dls_server_step() reads the results of the
 * previous epoch, admits, feeds the device work queue -- items for the idle
 * lanes plus a backlog, first from the admitted job with the least estimated
 * work not yet fed (shortest remaining work first), so a new job is served
 * within an epoch or two even while a big one still has most of its items to
 * go -- and launches one epoch: every lane of
 * a resident grid resumes the search it saved in device memory, or takes the
 * next queued item, runs `budget` search iterations and saves what is
 * unfinished.  Search stacks
 * and per-job counters stay on the device; jobs that arrive while others run
 * share the GPU with them from the next epoch on.  One server uses one CUDA
 * stream of its own and is driven from one host thread at a time. */
typedef struct dls_server dls_server;

typedef struct {
    int max_jobs;          /* device job slots (default 1024)                */
    size_t arena_bytes;    /* device memory for the items of admitted jobs
                              (default 256 MiB)                              */
    size_t chunk_bytes;    /* arena allocation unit (default 64 KiB)         */
    int64_t queue_items;   /* work-queue ring capacity (default 4 Mi)        */
    int max_order;         /* largest n a job may have (default 10)          */
    int budget;            /* search iterations per lane per epoch (4096)    */
    int block_threads;     /* 32..256 (default 128)                          */
    int blocks_per_sm;     /* 0 = as many as fit                             */
    int items_per_job;     /* most items a job is split into (0 = default:
                              16 per lane of the grid, at most 4 Mi)         */
    int min_backlog;       /* queue items kept beyond the idle lanes (default
                              1024; twice the items taken in the last epoch
                              when that is more)                             */
    int64_t item_nodes;    /* search nodes aimed at per item (default 2^17):
                              a job is split into one item per lane, or into
                              its estimated nodes / item_nodes items if that
                              is more (at most items_per_job), the estimate
                              being Knuth's random-descent estimate of the
                              size of its search tree (256 descents)         */
} dls_server_cfg;

typedef struct {
    int64_t submitted, admitted, completed, pending, active, epochs;
    uint64_t squares;      /* sum of the counts of completed jobs            */
    int64_t lanes;         /* lanes of the resident grid                     */
    size_t device_bytes;   /* device memory held by the server               */
    size_t free_arena_bytes;
} dls_server_stats;

/* Fills *cfg with the defaults above. */
void dls_server_default_cfg(dls_server_cfg *cfg);
/* Allocates the server's device memory (cfg NULL = defaults) on the current
 * device and starts its worker threads (at most 4).  Errors: BAD_ARG,
 * NO_MEMORY, CUDA. */
int dls_server_create(const dls_server_cfg *cfg, dls_server **out);
/* Queues a job (host arguments, copied; conventions as dls_count with one
 * prefix of `depth` bytes) and returns at once: *job_id receives its id, and
 * the job is split into work items on one of the server's worker threads
 * (never beyond half the arena, so every job can be admitted) before it
 * waits for admission.  A job whose prefix is invalid, or that leaves
 * nothing to search, completes without the GPU.  Errors: INVALID_N (also
 * n > max_order), BAD_ORDER, BAD_ARG, NO_MEMORY. */
int dls_server_submit(dls_server *srv, int n, uint32_t flags,
                      const uint8_t *order, int order_len,
                      const uint8_t *prefix, int depth, int64_t *job_id);
/* One epoch (see above).  Blocks only to read the previous epoch's results. */
int dls_server_step(dls_server *srv);
/* Moves up to cap completed jobs (ids and exact counts) out of the server;
 * *n_done receives how many. */
int dls_server_poll(dls_server *srv, int64_t *ids, uint64_t *counts, int cap,
                    int *n_done);
int dls_server_get_stats(dls_server *srv, dls_server_stats *out);
/* Stops the server; may be called from any thread, also while another
 * thread is inside dls_server_step().  The next dls_server_step() reads the
 * running epoch's results and returns DLS_ERR_ABORTED instead of launching
 * another; so do all later steps and submissions.  Jobs completed so far
 * stay available to dls_server_poll(); unfinished ones never complete.
 * Then call dls_server_destroy().  Errors: BAD_ARG (NULL). */
int dls_server_abort(dls_server *srv);
/* Waits for the running epoch and frees everything. */
void dls_server_destroy(dls_server *srv);

/* Allocation-free variant of dls_count_host() -- the paper has no
 * counterpart; it exists for callers that cannot let a library call
 * cudaMalloc: programs whose own pool already owns the device memory, and
 * latency-critical paths that must not pay the implicit device
 * synchronisation of cudaMalloc/cudaFree.  The staged prefixes, the staged
 * counts and the persistent kernel's queue head live in one fixed array of
 * DLS_NOALLOC_SCRATCH_BYTES compiled into the library (held on every GPU
 * that loads the library until the process exits).  A call needs 256 +
 * (n_prefixes * depth rounded up to 256) + 8 * n_prefixes bytes of it;
 * bigger calls return DLS_ERR_CAPACITY before any copy.  Arguments and
 * results are those of dls_count_host() (h_counts or total_out may be NULL,
 * not both).  Synchronous.  Every call shares the array: calls that overlap
 * on the GPU race and give wrong counts, so serialise them.  The first call
 * on a device looks up the array's device address (cudaGetSymbolAddress);
 * make it before any stream capture.  After cudaDeviceReset(), call
 * dls_release() (which forgets that address) before the next call.  Like
 * dls_count_host() it returns DLS_ERR_INTERNAL when the snapshot search
 * reported a stack overflow.  Allocates no device memory and calls no
 * cudaMalloc/cudaFree. */
#define DLS_NOALLOC_SCRATCH_BYTES (4u << 20)
int dls_count_host_noalloc(int n, uint32_t flags, const uint8_t *order,
                           int order_len, const uint8_t *h_prefixes, int depth,
                           int64_t n_prefixes, uint64_t *h_counts,
                           dls_u128 *total_out, const dls_launch_t *cfg,
                           void *stream);

/* Free the library's per-(device, stream) work areas and forget the device
 * address of the allocation-free entry's array. */
void dls_release(void);

/* ------------------------------------------------------------ plans */

/* A plan freezes one dls_count_ex call (all pointers and sizes) into a CUDA
 * graph so that repeated launches cost one graph launch.  The buffers must
 * stay valid while the plan lives.  dls_plan_create captures on its own
 * private stream. */
typedef struct dls_plan dls_plan;

int dls_plan_create(dls_plan **plan_out, int n, uint32_t flags,
                    const uint8_t *order, int order_len,
                    const uint8_t *d_prefixes, int depth, int64_t n_prefixes,
                    uint64_t *d_counts, uint64_t *d_total,
                    const dls_launch_t *cfg);
int dls_plan_launch(dls_plan *plan, void *stream);
/* Status of the plan's last launch (as dls_stream_status; every launch
 * clears the plan's own status word first): waits for `stream`, the stream
 * the plan was last launched on.  Errors: BAD_STATE (no plan), BAD_ARG,
 * CUDA. */
int dls_plan_status(dls_plan *plan, void *stream, dls_count_status *out);
void dls_plan_destroy(dls_plan *plan);

#ifdef __cplusplus
}
#endif

#endif /* DLS_H */
