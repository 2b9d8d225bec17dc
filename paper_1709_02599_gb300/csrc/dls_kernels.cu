// dls_kernels.cu -- the batch kernels (Algorithm 4 of the paper on sm_103a)
// and the C-ABI entry points that launch them.
//
// Two per-lane searches: the one-entry-per-position search of
// dls_search.cuh, whose row/column words and stack live in shared memory in
// a thread-minor layout (word w of thread t at w * blockDim + t, so a warp's
// accesses hit 32 distinct banks whatever positions its lanes are at) or,
// where they fit, with the row and column words packed into two 64-bit
// registers; and the snapshot search of dls_snapshot.cuh (register words, a
// stack entry only where candidates remain), the default where the words fit
// registers.
//
// Kernels:
//   k_plain      -- one thread per work item, per-position search: the
//                   comparison baseline of the paper's loop structure.
//   k_plain_snap -- one thread per prefix, snapshot search: the baseline
//                   with the batched kernel's own search step.
//   k_persistent -- a resident grid; warps take work items from a global
//                   atomic queue as lanes go idle, and once the queue is empty
//                   idle lanes take the shallowest untried subtree of a busy
//                   lane in the same warp (ballot + shuffle + shared memory).
//   k_snapshot   -- the same grid, queue and donation with the snapshot
//                   search, so that a dead end returns to the deepest open
//                   cell in one step; optional lookahead (Section 2.4.2);
//                   the fused step (a following single-candidate cell
//                   placed in the same iteration) where it applies, in
//                   k_plain_snap too.
//   All keep per-lane totals, reduce them per block in shared memory and add
//   one 64-bit atomic per block to the global total.
//
// Work items: prefix p is split into `lanes` items (p, s); item s keeps the
// nodes at order position split_pos whose index in depth-first order is
// s mod lanes (all items walk the few positions above split_pos).

#include <cuda_runtime.h>

#include <algorithm>
#include <numeric>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "dls_internal.h"
#include "dls_search.cuh"
#include "dls_snapshot.cuh"

namespace dls {

// Status word of a count (word 1 of its work area, after the queue head):
// bits the kernels set, read back by the host entry points and by
// dls_stream_status / dls_plan_status.
constexpr unsigned ST_OVERFLOW = 1u;  // a snapshot stack would have overflowed
constexpr unsigned ST_TIMEOUT = 2u;   // stopped early: iteration budget spent
constexpr unsigned ST_ABORTED = 4u;   // stopped early: abort flag seen
constexpr unsigned ST_DEFERRED = 8u;  // a capped stack deferred prefixes to the recount pass
// Count mark of a prefix deferred by a capped stack (counted again, from 0,
// by the recount pass; never left in a count returned to the caller).
constexpr unsigned long long RECOUNT = 1ull << 62;
// iterations between two reads of a count's abort flag (a read of mapped
// host memory takes microseconds)
constexpr long long POLL_EVERY = 4096;

__device__ __forceinline__ void raise_status(const unsigned long long *queue, unsigned bit) {
  atomicOr(reinterpret_cast<unsigned *>(const_cast<unsigned long long *>(queue + 1)), bit);
}

struct KParams {
  Geo g;                 // order size, admissible values, prefix length, last
  Split sp;              // item split over lanes
  int order_len;
  int check_mask;        // donation check period - 1
  int donate;
  int count_store;       // 1: counts[p] = cnt (one item per prefix, no donation)
  int wr, wc;            // register words: bit width of a row / column field
  long long n_prefixes;
  long long n_items;
  const uint8_t *prefixes;
  unsigned long long *counts;
  unsigned long long *total;
  unsigned long long *nodes;
  unsigned long long *queue;  // [0] queue head, [1] status word
  int snap_cap;               // snapshot stack entries per lane
  long long budget;           // search iterations per lane before stopping (0: none)
  const volatile int *abort_flag;  // polled; nonzero stops the count (NULL: none)
  int defer;                  // a stack overflow defers the prefix to the recount pass
  int recount;                // the recount pass: only deferred prefixes are searched
  int diag_words;             // DLS_DIAGONAL (the wide load checks the diagonals)
  // k_snapshot hands out queue place k as item k * qstride mod n_items (0:
  // in order): a stride near n_items / 64, coprime with n_items, interleaves
  // the runs of neighbouring prefixes, whose search sizes are alike, so the
  // heavy ones of a run are not all taken at the end of the queue
  unsigned long long qstride;
  int8_t rslot[DLS_MAX_N];    // wide words: byte slot of each row / column (-1: none)
  int8_t cslot[DLS_MAX_N];
  uint8_t ci[DLS_MAX_CELLS];
  uint8_t cj[DLS_MAX_CELLS];
};

// Load work item `item` into the lane.  Returns true if it is already
// finished (invalid prefix, or nothing left to search).
template <bool REG, bool VSYM, bool NODES>
__device__ bool load_item(Lane<REG> &s, const KParams &p, long long item,
                          const Cell *tbl, unsigned B) {
  const Geo &g = p.g;
  s.prefix = item >> p.sp.lanes_log2;
  s.sub = (uint32_t)(item & ((1ll << p.sp.lanes_log2) - 1));
  s.cnt = 0ull;
  s.splitc = 0u;
  s.w.clear(2 * g.n, B);
  if (!place_prefix<REG, VSYM>(s.w, g, p.prefixes + (size_t)s.prefix * (size_t)g.depth, tbl))
    return true;
  if (g.depth == p.order_len) {
    s.cnt = (s.sub == 0u) ? 1ull : 0ull;
    return true;
  }
  const Cell info = tbl[g.depth];
  const uint32_t L = s.w.template cands<VSYM>(info, g);
  if (g.depth == g.last) {
    if (s.sub == 0u) {
      s.cnt = (unsigned)__popc(L);
      if (NODES) s.nodes += (unsigned)__popc(L);
    }
    return true;
  }
  s.p = g.depth;
  s.L = L;
  s.v = 0u;
  s.info = info;
  return L == 0u;
}

__device__ __forceinline__ void flush_count(long long prefix, unsigned long long cnt,
                                            const KParams &p,
                                            unsigned long long &lane_total) {
  if (prefix < 0) return;  // a prefix the recount pass skips
  lane_total += cnt;
  if (p.counts != nullptr) {
    if (p.count_store)
      p.counts[prefix] = cnt;
    else if (cnt)
      atomicAdd(p.counts + prefix, cnt);
  }
}

// A finished item of a snapshot search: counted, unless the lane's stack
// overflowed during it -- then, with a capped stack, the prefix is marked for
// the recount pass (which searches it again with the full bound); without a
// cap (where the bound excludes an overflow) the count's status reports it.
__device__ __forceinline__ void finish_snapshot_item(long long prefix, unsigned long long cnt,
                                                     const KParams &p, uint32_t &ovf,
                                                     unsigned long long &lane_total) {
  if (!ovf) {
    flush_count(prefix, cnt, p, lane_total);
    return;
  }
  ovf = 0u;
  if (p.defer && prefix >= 0) {
    if (p.count_store)
      p.counts[prefix] = RECOUNT;
    else
      atomicOr(p.counts + prefix, RECOUNT);
    atomicOr(reinterpret_cast<unsigned *>(p.queue + 1), ST_DEFERRED);
  } else {
    atomicOr(reinterpret_cast<unsigned *>(p.queue + 1), ST_OVERFLOW);
  }
}

// The recount pass takes only the prefixes the first pass deferred (and
// clears their count); any other one is skipped (prefix -1: nothing is
// stored for it).  Returns true for a skipped one.
__device__ __forceinline__ bool recount_skip(const KParams &p, long long item) {
  if (!p.recount) return false;
  if ((p.counts[item] & RECOUNT) == 0ull) return true;
  p.counts[item] = 0ull;
  return false;
}

// Stopping early.  `spent` = search iterations the warp has made (the same
// in every lane); returns the status bit to stop with, or 0.  Lane 0 reads
// the abort flag every POLL_EVERY iterations and shares what it read.
__device__ __forceinline__ unsigned stop_due(const KParams &p, long long spent,
                                             long long &next_poll, int lane) {
  if (p.budget > 0 && spent >= p.budget) return ST_TIMEOUT;
  if (p.abort_flag != nullptr && spent >= next_poll) {
    next_poll = spent + POLL_EVERY;
    int f = 0;
    if (lane == 0) f = *p.abort_flag;
    if (__shfl_sync(FULL, f, 0) != 0) return ST_ABORTED;
  }
  return 0u;
}

// A warp that stops: a lane still searching marks its prefix unfinished
// (with a stored count, the partial count goes with the mark), and the
// count's status records why, if work was left (a lane was searching, or
// the queue still held items the warp would have taken).
__device__ __forceinline__ void stop_warp(const KParams &p, unsigned why, bool busy,
                                          long long prefix, unsigned long long cnt, bool queued,
                                          int lane) {
  if (busy && p.counts != nullptr) {
    if (p.count_store)
      p.counts[prefix] = cnt | DLS_UNFINISHED;
    else
      atomicOr(p.counts + prefix, DLS_UNFINISHED);
  }
  unsigned long long head = 0ull;
  if (queued && lane == 0) head = *reinterpret_cast<volatile unsigned long long *>(p.queue);
  head = __shfl_sync(FULL, head, 0);
  const bool left = __any_sync(FULL, busy) || (queued && (long long)head < p.n_items);
  if (left && lane == 0) raise_status(p.queue, why);
}

// Per-block reduction of the lane totals, one global atomic per block.
__device__ void block_reduce_add(unsigned long long v, unsigned long long *dst,
                                 unsigned long long *red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULL, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long s = 0ull;
    for (unsigned w = 0; w < (blockDim.x >> 5); ++w) s += red[w];
    if (dst != nullptr && s) atomicAdd(dst, s);
  }
}

// Shared memory: [table: one Cell (8 bytes) per order position]
//                [words: 2n * B, shared-memory variant only]
//                [stack: (last - depth) * B]
template <bool REG>
__device__ __forceinline__ void setup(const KParams &p, int diag, uint32_t *smem,
                                      const Cell *&tbl, uint32_t *&stk, Lane<REG> &s) {
  const unsigned B = blockDim.x;
  Cell *t = reinterpret_cast<Cell *>(smem);
  for (int idx = threadIdx.x; idx < p.order_len; idx += B)
    t[idx] = REG ? describe_regs(p.ci[idx], p.cj[idx], p.g.n, diag != 0, p.wr, p.wc)
                 : describe_shared(p.ci[idx], p.cj[idx], p.g.n, diag != 0, B, p.g.n);
  uint32_t *st = smem + 2 * ((p.order_len + 31) & ~31);
  s.w.tb = reinterpret_cast<char *>(st + threadIdx.x);
  stk = st + (REG ? 0 : 2 * p.g.n * (int)B) + threadIdx.x;
  tbl = t;
  s.nodes = 0ull;
  s.prefix = 0;
  s.sub = 0u;
  s.p = 0;
  s.L = s.v = 0u;
  s.info = make_uint2(0u, 0u);
  s.cnt = 0ull;
  s.w.dg = 0u;
  s.w.R = s.w.C = 0ull;
  __syncthreads();
}

template <bool REG, bool VSYM, bool NODES, bool SPLIT>
__global__ void __launch_bounds__(512) k_plain(const __grid_constant__ KParams p,
                                               int diag) {
  extern __shared__ uint32_t smem[];
  __shared__ unsigned long long red[16];
  const unsigned B = blockDim.x;
  const Cell *tbl;
  uint32_t *stk;
  Lane<REG> s;
  setup(p, diag, smem, tbl, stk, s);
  uint32_t *sbase = stk - p.g.depth * (int)B;

  unsigned long long lane_total = 0ull;
  const long long item = (long long)blockIdx.x * B + threadIdx.x;
  bool busy = false;
  if (item < p.n_items) {
    busy = !load_item<REG, VSYM, NODES>(s, p, item, tbl, B);
    if (!busy) flush_count(s.prefix, s.cnt, p, lane_total);
  }
  const bool stoppable = p.budget > 0 || p.abort_flag != nullptr;
  long long spent = 0, next_poll = 0;
  unsigned stopped = 0u;
  int k = 0;
  while (__any_sync(FULL, busy)) {
    if (busy && dfs_step<REG, VSYM, NODES, SPLIT>(s, p.g, p.sp, sbase, tbl, B)) {
      busy = false;
      flush_count(s.prefix, s.cnt, p, lane_total);
    }
    if (stoppable && ++k > p.check_mask) {
      spent += k;
      k = 0;
      stopped = stop_due(p, spent, next_poll, threadIdx.x & 31);
      if (stopped) break;
    }
  }
  if (stopped) stop_warp(p, stopped, busy, s.prefix, s.cnt, false, threadIdx.x & 31);
  block_reduce_add(lane_total, p.total, red);
  if (NODES) block_reduce_add(s.nodes, p.nodes, red);
}

// Position of the (r+1)-th set bit of m (r = 0 -> lowest set bit).
__device__ __forceinline__ int nth_set_bit(unsigned m, int r) {
  for (int k = 0; k < r; ++k) m &= m - 1u;
  return __ffs(m) - 1;
}

// In-warp work donation: each idle lane is paired with a busy lane that has
// an untried candidate at some position pd (the shallowest such position at
// or below the item split); the idle lane copies the busy lane's words and
// path, undoes its placements below pd and takes the untried candidates of
// pd, which the busy lane gives up.
template <bool REG, bool VSYM>
__device__ void donate(Lane<REG> &s, bool &busy, const KParams &p, uint32_t *stk,
                       const Cell *tbl, int lane, unsigned B) {
  const Geo &g = p.g;
  const unsigned idle = __ballot_sync(FULL, !busy);
  if (idle == 0u || idle == FULL) return;
  const int lo = max(g.depth, p.sp.pos + 1);
  int pd = -1;
  uint32_t Lpd = 0u, vpd = 0u;
  if (busy) {
    for (int q = lo; q < s.p; ++q) {
      const uint32_t e = stk[(q - g.depth) * B];
      if (e & 0xffffu) {
        pd = q;
        Lpd = e & 0xffffu;
        vpd = e >> 16;
        break;
      }
    }
    if (pd < 0 && s.p >= lo && s.L != 0u) {
      pd = s.p;
      Lpd = s.L;
      vpd = s.v;
    }
  }
  const unsigned donors = __ballot_sync(FULL, pd >= 0);
  if (donors == 0u) return;
  const int pairs = min(__popc(idle), __popc(donors));
  const unsigned below = (1u << lane) - 1u;
  int partner = lane;  // the lane this one reads from (itself if unpaired)
  bool receiver = false, giver = false;
  if (!busy) {
    const int r = __popc(idle & below);
    if (r < pairs) {
      partner = nth_set_bit(donors, r);
      receiver = true;
    }
  } else if (pd >= 0) {
    giver = __popc(donors & below) < pairs;
  }
  const int d_pd = __shfl_sync(FULL, pd, partner);
  const uint32_t d_L = __shfl_sync(FULL, Lpd, partner);
  const uint32_t d_vpd = __shfl_sync(FULL, vpd, partner);
  const int d_p = __shfl_sync(FULL, s.p, partner);
  const uint32_t d_v = __shfl_sync(FULL, s.v, partner);
  const uint32_t d_dg = __shfl_sync(FULL, s.w.dg, partner);
  const unsigned long long d_R = __shfl_sync(FULL, s.w.R, partner);
  const unsigned long long d_C = __shfl_sync(FULL, s.w.C, partner);
  const long long d_prefix = __shfl_sync(FULL, s.prefix, partner);
  const uint32_t d_sub = __shfl_sync(FULL, s.sub, partner);
  if (receiver) {
    const int dl = partner - lane;  // donor's thread offset from this one
    if (REG) {
      s.w.R = d_R;
      s.w.C = d_C;
    } else {
      uint32_t *mine = reinterpret_cast<uint32_t *>(s.w.tb);
      const uint32_t *theirs = mine + dl;
      for (int w = 0; w < 2 * g.n; ++w) mine[w * B] = theirs[w * B];
    }
    const uint32_t *dstk = stk + dl;
    for (int q = g.depth; q < d_pd; ++q)
      stk[(q - g.depth) * B] = dstk[(q - g.depth) * B] & 0xffff0000u;
    s.w.dg = d_dg;
    // undo the donor's placements below pd
    for (int q = d_pd + 1; q <= d_p; ++q) {
      const uint32_t vq = (q < d_p) ? (dstk[(q - g.depth) * B] >> 16) : d_v;
      if (vq) s.w.template toggle<VSYM>(tbl[q], vq, g);
    }
    s.p = d_pd;
    s.L = d_L;
    s.v = d_vpd;
    s.info = tbl[d_pd];
    s.prefix = d_prefix;
    s.sub = d_sub;
    s.splitc = 0u;
    s.cnt = 0ull;
    busy = true;
  }
  __syncwarp();
  if (giver) {
    if (pd < s.p)
      stk[(pd - g.depth) * B] &= 0xffff0000u;
    else
      s.L = 0u;
  }
  __syncwarp();
}

template <bool REG, bool VSYM, bool NODES, bool SPLIT>
__global__ void __launch_bounds__(512)
    k_persistent(const __grid_constant__ KParams p, int diag) {
  extern __shared__ uint32_t smem[];
  __shared__ unsigned long long red[16];
  const unsigned B = blockDim.x;
  const int lane = threadIdx.x & 31;
  const Cell *tbl;
  uint32_t *stk;
  Lane<REG> s;
  setup(p, diag, smem, tbl, stk, s);
  uint32_t *sbase = stk - p.g.depth * (int)B;

  unsigned long long lane_total = 0ull;
  bool busy = false;
  bool qdone = false;
  const bool stoppable = p.budget > 0 || p.abort_flag != nullptr;
  long long spent = 0, next_poll = 0;
  unsigned stopped = 0u;

  for (;;) {
    if (stoppable && (stopped = stop_due(p, spent, next_poll, lane)) != 0u) break;
    // hand queue items to idle lanes, one atomic per warp
    unsigned idle = __ballot_sync(FULL, !busy);
    while (idle != 0u && !qdone) {
      const int nidle = __popc(idle);
      unsigned long long base = 0ull;
      if (lane == 0) base = atomicAdd(p.queue, (unsigned long long)nidle);
      base = __shfl_sync(FULL, base, 0);
      if (!busy) {
        const long long item = (long long)base + __popc(idle & ((1u << lane) - 1u));
        if (item < p.n_items) {
          busy = !load_item<REG, VSYM, NODES>(s, p, item, tbl, B);
          if (!busy) flush_count(s.prefix, s.cnt, p, lane_total);
        }
      }
      if ((long long)(base + (unsigned long long)nidle) >= p.n_items) qdone = true;
      idle = __ballot_sync(FULL, !busy);
    }
    if (idle == FULL) break;  // queue drained and every lane idle
    if (!qdone) {
      // every lane is busy here: step until one finishes its item (or, when
      // the count may stop early, at most check_every iterations)
      bool fin;
      if (!stoppable) {
        do {
          fin = dfs_step<REG, VSYM, NODES, SPLIT>(s, p.g, p.sp, sbase, tbl, B);
        } while (!__any_sync(FULL, fin));
      } else {
        int k = 0;
        do {
          fin = dfs_step<REG, VSYM, NODES, SPLIT>(s, p.g, p.sp, sbase, tbl, B);
        } while (!__any_sync(FULL, fin) && ++k <= p.check_mask);
        spent += k + 1;
      }
      if (fin) {
        busy = false;
        flush_count(s.prefix, s.cnt, p, lane_total);
      }
    } else {
      for (int it = 0; it <= p.check_mask; ++it) {
        if (busy && dfs_step<REG, VSYM, NODES, SPLIT>(s, p.g, p.sp, sbase, tbl, B)) {
          busy = false;
          flush_count(s.prefix, s.cnt, p, lane_total);
        }
      }
      spent += p.check_mask + 1;
      if (p.donate) donate<REG, VSYM>(s, busy, p, stk, tbl, lane, B);
    }
  }
  if (stopped) stop_warp(p, stopped, busy, s.prefix, s.cnt, true, lane);
  block_reduce_add(lane_total, p.total, red);
  if (NODES) block_reduce_add(s.nodes, p.nodes, red);
}

// ---------------------------------------------------- snapshot search --

// Load work item (= prefix) `item` into a snapshot lane.  Returns true if it
// is already finished (invalid prefix, or nothing left to search).
template <bool VSYM, bool NODES>
__device__ bool snap_load(SnapLane &s, const KParams &p, long long item, const Cell *tbl,
                          const SnapTable &tb) {
  const Geo &g = p.g;
  s.cnt = 0ull;
  s.sp = s.bot = 0;
  s.prefix = recount_skip(p, item) ? -1 : item;
  if (s.prefix < 0) return true;
  s.w.clear(0, 0u);
  if (!place_prefix<true, VSYM>(s.w, g, p.prefixes + (size_t)item * (size_t)g.depth, tbl))
    return true;
  if (g.depth == p.order_len) {
    s.cnt = 1ull;
    return true;
  }
  const uint32_t L = s.w.template cands<VSYM>(tbl[g.depth], g);
  if (g.depth == g.last) {
    s.cnt = (unsigned)__popc(L);
    if (NODES) s.nodes += (unsigned)__popc(L);
    return true;
  }
  s.p = g.depth;
  s.L = L;
  s.sh = tb.sh[g.depth];
  s.dm = tb.dm[g.depth];
  return L == 0u;
}

// The same for a byte-word lane (orders n <= 8 without vertical symmetry):
// the prefix is placed into the 64-bit words, which are then split into the
// four byte words.
template <bool VSYM, bool NODES>
__device__ bool snap_load(BLane &s, const KParams &p, long long item, const Cell *tbl,
                          const BRow *tb) {
  static_assert(!VSYM, "byte words: no vertical symmetry");
  const Geo &g = p.g;
  s.cnt = 0ull;
  s.sp = s.bot = 0;
  s.prefix = recount_skip(p, item) ? -1 : item;
  if (s.prefix < 0) return true;
  Words<true> w;
  w.tb = nullptr;
  w.clear(0, 0u);
  const bool ok =
      place_prefix<true, false>(w, g, p.prefixes + (size_t)item * (size_t)g.depth, tbl);
  s.R0 = (uint32_t)w.R;
  s.R1 = (uint32_t)(w.R >> 32);
  s.C0 = (uint32_t)w.C;
  s.C1 = (uint32_t)(w.C >> 32);
  s.dg = w.dg;
  if (!ok) return true;
  if (g.depth == p.order_len) {
    s.cnt = 1ull;
    return true;
  }
  const uint32_t L = w.template cands<false>(tbl[g.depth], g);
  if (g.depth == g.last) {
    s.cnt = (unsigned)__popc(L);
    if (NODES) s.nodes += (unsigned)__popc(L);
    return true;
  }
  s.p = g.depth;
  s.L = L;
  const BRow &row = tb[g.depth];
  s.a = row.a;
  s.b = row.b;
  s.c = row.c;
  return L == 0u;
}

// The same for a wide-word lane (order 9): the prefix is checked and placed
// with plain line masks, which are then written into the row and column
// slots and the value-8 word.
template <bool VSYM, bool NODES>
__device__ bool snap_load(WLane &s, const KParams &p, long long item, const Cell *,
                          const WRow *tb) {
  static_assert(!VSYM, "wide words: no vertical symmetry");
  const Geo &g = p.g;
  const int n = g.n;
  s.cnt = 0ull;
  s.sp = s.bot = 0;
  s.prefix = recount_skip(p, item) ? -1 : item;
  if (s.prefix < 0) return true;
  uint32_t rows[DLS_MAX_N], cols[DLS_MAX_N];
  for (int k = 0; k < n; ++k) rows[k] = cols[k] = 0u;
  uint32_t md = 0u, ad = 0u;
  const uint8_t *rec = p.prefixes + (size_t)item * (size_t)g.depth;
  bool ok = true;
  for (int t = 0; t < g.depth && ok; ++t) {
    const int i = p.ci[t], j = p.cj[t];
    const uint32_t v = rec[t];
    const uint32_t b = v < (uint32_t)n ? (1u << v) : 0u;
    const bool on_md = p.diag_words && i == j, on_ad = p.diag_words && i + j == n - 1;
    const uint32_t used = rows[i] | cols[j] | (on_md ? md : 0u) | (on_ad ? ad : 0u);
    ok = b != 0u && (used & b) == 0u;
    rows[i] |= b;
    cols[j] |= b;
    md |= on_md ? b : 0u;
    ad |= on_ad ? b : 0u;
  }
  uint32_t R0 = 0u, R1 = 0u, C0 = 0u, C1 = 0u, C2 = 0u, V8 = 0u;
  for (int k = 0; k < n; ++k) {
    const int rs = p.rslot[k], cs = p.cslot[k];
    const uint32_t rb = rows[k] & 0xffu, cb = cols[k] & 0xffu;
    if (rs >= 0) {
      R0 |= rb * byte_mult(rs, 0);
      R1 |= rb * byte_mult(rs, 1);
    }
    if (cs >= 0) {
      C0 |= cb * wide_col_mult(cs, 0);
      C1 |= cb * wide_col_mult(cs, 1);
      C2 |= cb * wide_col_mult(cs, 2);
    }
    V8 |= ((rows[k] >> 8) & 1u) << k;
    V8 |= ((cols[k] >> 8) & 1u) << (16 + k);
  }
  s.R0 = R0;
  s.R1 = R1;
  s.C0 = C0;
  s.C1 = C1;
  s.C2 = C2;
  s.V8 = V8;
  s.dg = md | (ad << 16);
  if (!ok) return true;
  if (g.depth == p.order_len) {
    s.cnt = 1ull;
    return true;
  }
  const int i = p.ci[g.depth], j = p.cj[g.depth];
  const bool on_md = p.diag_words && i == j, on_ad = p.diag_words && i + j == n - 1;
  const uint32_t L = g.all & ~(rows[i] | cols[j] | (on_md ? md : 0u) | (on_ad ? ad : 0u));
  if (g.depth == g.last) {
    s.cnt = (unsigned)__popc(L);
    if (NODES) s.nodes += (unsigned)__popc(L);
    return true;
  }
  s.p = g.depth;
  s.L = L;
  s.r = tb[g.depth];
  return L == 0u;
}

// In-warp work donation for snapshot lanes: each idle lane is paired with a
// busy lane that holds a stack entry; it takes the busy lane's bottom entry
// (the shallowest open cell: the largest untried subtree) and the busy lane
// drops it by raising its bottom index.
// Restores a lane's words from an entry (line words, packed word) and loads
// the table row of its position.
template <bool VSYM, bool DG>
__device__ __forceinline__ void snap_take(SnapLane &s, const KParams &p, uint4 a, uint32_t wv,
                                          const SnapTable &tb) {
  s.w.R = ((unsigned long long)a.y << 32) | a.x;
  s.w.C = ((unsigned long long)a.w << 32) | a.z;
  uint32_t dg;
  snap_unpack<VSYM>(wv, p.g.n, dg, s.p, s.L);
  if (DG) s.w.dg = dg;
  s.sh = tb.sh[s.p];
  s.dm = tb.dm[s.p];
}

template <bool VSYM, bool DG>
__device__ __forceinline__ void snap_take(BLane &s, const KParams &p, uint4 a, uint32_t wv,
                                          const BRow *tb) {
  s.R0 = a.x;
  s.R1 = a.y;
  s.C0 = a.z;
  s.C1 = a.w;
  uint32_t dg;
  snap_unpack<false>(wv, p.g.n, dg, s.p, s.L);
  if (DG) s.dg = dg;
  const BRow &row = tb[s.p];
  s.a = row.a;
  s.b = row.b;
  s.c = row.c;
}

// A wide-word entry: R0, R1, C0, C1 in sa, then (C2, V8, diagonal words,
// position | untried candidates << 16) in the stack's second array.
template <bool VSYM, bool DG>
__device__ __forceinline__ void snap_take(WLane &s, const KParams &, uint4 a, uint4 b,
                                          const WRow *tb) {
  s.R0 = a.x;
  s.R1 = a.y;
  s.C0 = a.z;
  s.C1 = a.w;
  s.C2 = b.x;
  s.V8 = b.y;
  if (DG) s.dg = b.z;
  s.p = (int)(b.w & 0xffffu);
  s.L = b.w >> 16;
  s.r = tb[s.p];
}

// The second word of entry `off` (a 32-bit packed word, or 16 bytes for
// wide words).
__device__ __forceinline__ uint32_t entry_word(const SnapLane &, const SnapStack &st, int off) {
  return st.sw[off];
}
__device__ __forceinline__ uint32_t entry_word(const BLane &, const SnapStack &st, int off) {
  return st.sw[off];
}
__device__ __forceinline__ uint4 entry_word(const WLane &, const SnapStack &st, int off) {
  return reinterpret_cast<const uint4 *>(st.sw)[off];
}

template <bool VSYM, bool DG, class LaneT, class TableT>
__device__ void snap_donate(LaneT &s, bool &busy, const KParams &p, const SnapStack &st,
                            const TableT &tb, int lane, unsigned B) {
  const unsigned idle = __ballot_sync(FULL, !busy);
  if (idle == 0u || idle == FULL) return;
  const unsigned donors = __ballot_sync(FULL, busy && s.sp > s.bot);
  if (donors == 0u) return;
  const int pairs = min(__popc(idle), __popc(donors));
  const unsigned below = (1u << lane) - 1u;
  int partner = lane;
  bool receiver = false, giver = false;
  if (!busy) {
    const int r = __popc(idle & below);
    if (r < pairs) {
      partner = nth_set_bit(donors, r);
      receiver = true;
    }
  } else if ((donors >> lane) & 1u) {
    giver = __popc(donors & below) < pairs;
  }
  const int d_bot = __shfl_sync(FULL, s.bot, partner);
  const long long d_prefix = __shfl_sync(FULL, s.prefix, partner);
  if (receiver) {
    const int off = (d_bot + 1) * (int)B + (partner - lane);
    snap_take<VSYM, DG>(s, p, st.sa[off], entry_word(s, st, off), tb);
    s.sp = s.bot = 0;
    s.prefix = d_prefix;
    s.cnt = 0ull;
    busy = true;
  }
  __syncwarp();
  if (giver) s.bot++;
}

// The three snapshot searches: byte words (orders n <= 8 without vertical
// symmetry; BLane, bsnap_step), register words with field shifts (vertically
// symmetric orders; SnapLane, snap_step) and wide words (order 9; WLane,
// wsnap_step).  W2 = 4-byte words in the second part of an entry.
constexpr int KIND_BYTE = 0, KIND_SHIFT = 1, KIND_WIDE = 2;

template <int KIND>
struct SnapKind {
  using Lane = BLane;
  using Table = const BRow *;
  static constexpr int W2 = 1;
  template <bool NODES, bool DG, bool LA, bool FU>
  static __device__ __forceinline__ bool step(Lane &s, const Geo &g, const SnapStack &st,
                                              const Table &tb, unsigned B, uint32_t &ovf) {
    return bsnap_step<NODES, DG, LA, FU>(s, g, st, tb, B, ovf);
  }
};

template <>
struct SnapKind<KIND_SHIFT> {
  using Lane = SnapLane;
  using Table = SnapTable;
  static constexpr int W2 = 1;
  template <bool NODES, bool DG, bool LA, bool FU>
  static __device__ __forceinline__ bool step(Lane &s, const Geo &g, const SnapStack &st,
                                              const Table &tb, unsigned B, uint32_t &ovf) {
    return snap_step<true, NODES, DG, LA, FU>(s, g, st, tb, B, ovf);
  }
};

template <>
struct SnapKind<KIND_WIDE> {
  using Lane = WLane;
  using Table = const WRow *;
  static constexpr int W2 = 4;
  template <bool NODES, bool DG, bool LA, bool FU>
  static __device__ __forceinline__ bool step(Lane &s, const Geo &g, const SnapStack &st,
                                              const Table &tb, unsigned B, uint32_t &ovf) {
    return wsnap_step<NODES, DG, LA, FU>(s, g, st, tb, B, ovf);
  }
};

template <bool VSYM, bool WIDE>
struct SnapKindOf {
  static constexpr int value = VSYM ? KIND_SHIFT : (WIDE ? KIND_WIDE : KIND_BYTE);
};

// Position tables in shared memory; returns where the stacks start.
// [cell table: 8 bytes per position, rounded to 32 positions]
// [position table: 24 bytes per position (shifts and diagonal masks), or 48
//  (byte-word rows), same rounding]
__device__ __forceinline__ uint4 *snap_tables(const KParams &p, int diag, bool dgw,
                                              uint32_t *smem, const Cell *&tbl, SnapTable &tb,
                                              bool two_on) {
  const unsigned B = blockDim.x;
  const int rows = (p.order_len + 31) & ~31;
  Cell *t = reinterpret_cast<Cell *>(smem);
  uint4 *tsh = reinterpret_cast<uint4 *>(smem + 2 * rows);
  uint2 *tdm = reinterpret_cast<uint2 *>(tsh + rows);
  for (int idx = threadIdx.x; idx < p.order_len; idx += B) {
    t[idx] = describe_regs(p.ci[idx], p.cj[idx], p.g.n, diag != 0, p.wr, p.wc);
    const int nx = min(idx + 1, p.order_len - 1);
    snap_row(p.g.n, diag != 0, p.wr, p.wc, p.ci[idx], p.cj[idx], p.ci[nx], p.cj[nx], tsh[idx],
             tdm[idx]);
    if (two_on) {
      // lookahead or fused step: the field shifts of the cell two positions
      // on (the last cell stands in past the end, where neither uses it)
      const int n2 = min(idx + 2, p.order_len - 1);
      tdm[idx] = make_uint2((uint32_t)(p.ci[n2] * p.wr), (uint32_t)(p.cj[n2] * p.wc));
    }
  }
  tbl = t;
  tb.sh = tsh;
  tb.dm = tdm;
  return reinterpret_cast<uint4 *>(tdm + rows);
}

__device__ __forceinline__ uint4 *snap_tables(const KParams &p, int diag, bool dgw,
                                              uint32_t *smem, const Cell *&tbl,
                                              const BRow *&tb, bool) {
  const unsigned B = blockDim.x;
  const int rows = (p.order_len + 31) & ~31;
  Cell *t = reinterpret_cast<Cell *>(smem);
  BRow *rw = reinterpret_cast<BRow *>(smem + 2 * rows);
  for (int idx = threadIdx.x; idx < p.order_len; idx += B) {
    t[idx] = describe_regs(p.ci[idx], p.cj[idx], p.g.n, diag != 0, 8, 8);
    rw[idx] = brow_make(p.g.n, diag != 0, dgw, p.ci, p.cj, idx, p.order_len);
  }
  tbl = t;
  tb = rw;
  return reinterpret_cast<uint4 *>(rw + rows);
}

__device__ __forceinline__ uint4 *snap_tables(const KParams &p, int diag, bool dgw,
                                              uint32_t *smem, const Cell *&tbl,
                                              const WRow *&tb, bool) {
  const unsigned B = blockDim.x;
  const int rows = (p.order_len + 31) & ~31;
  Cell *t = reinterpret_cast<Cell *>(smem);
  WRow *rw = reinterpret_cast<WRow *>(smem + 2 * rows);
  int rs[DLS_MAX_N], cs[DLS_MAX_N];
  for (int k = 0; k < DLS_MAX_N; ++k) {
    rs[k] = p.rslot[k];
    cs[k] = p.cslot[k];
  }
  for (int idx = threadIdx.x; idx < p.order_len; idx += B) {
    t[idx] = describe_regs(p.ci[idx], p.cj[idx], p.g.n, diag != 0, 8, 8);
    rw[idx] = wrow_make(p.g.n, diag != 0, dgw, p.ci, p.cj, idx, p.order_len, rs, cs);
  }
  tbl = t;
  tb = rw;
  return reinterpret_cast<uint4 *>(rw + rows);
}

// Shared memory: the position tables (snap_tables), then the stacks:
// (cap + 2) * B entries of 16 bytes, then as many of 4 * W2.
template <int W2, class LaneT, class TableT>
__device__ __forceinline__ void snap_setup(const KParams &p, int diag, bool dgw,
                                           uint32_t *smem, const Cell *&tbl, TableT &tb,
                                           SnapStack &st, LaneT &s, bool two_on) {
  const unsigned B = blockDim.x;
  uint4 *sa0 = snap_tables(p, diag, dgw, smem, tbl, tb, two_on);
  st.sa = sa0 + threadIdx.x;
  st.sw = reinterpret_cast<uint32_t *>(sa0 + (size_t)(p.snap_cap + 2) * B) + threadIdx.x * W2;
  st.cap = p.snap_cap;
  s = LaneT{};
  __syncthreads();
}

// The plain launch with the snapshot search: one thread per prefix, no
// queue, no donation (the baseline the batched kernel is measured against,
// with the same search step).
template <bool VSYM, bool NODES, bool DG, bool FU, bool WIDE = false>
__global__ void __launch_bounds__(512)
    k_plain_snap(const __grid_constant__ KParams p, int diag) {
  extern __shared__ uint32_t smem[];
  __shared__ unsigned long long red[16];
  const unsigned B = blockDim.x;
  using K = SnapKind<SnapKindOf<VSYM, WIDE>::value>;
  const Cell *tbl;
  typename K::Table tb;
  SnapStack st;
  typename K::Lane s;
  snap_setup<K::W2>(p, diag, DG, smem, tbl, tb, st, s, FU);
  uint32_t ovf = 0u;
  unsigned long long lane_total = 0ull;
  const long long item = (long long)blockIdx.x * B + threadIdx.x;
  bool busy = false;
  if (item < p.n_items) {
    busy = !snap_load<VSYM, NODES>(s, p, item, tbl, tb);
    if (!busy) finish_snapshot_item(s.prefix, s.cnt, p, ovf, lane_total);
  }
  const bool stoppable = p.budget > 0 || p.abort_flag != nullptr;
  long long spent = 0, next_poll = 0;
  unsigned stopped = 0u;
  int k = 0;
  while (__any_sync(FULL, busy)) {
    if (busy && K::template step<NODES, DG, false, FU>(s, p.g, st, tb, B, ovf)) {
      busy = false;
      finish_snapshot_item(s.prefix, s.cnt, p, ovf, lane_total);
    }
    if (stoppable && ++k > p.check_mask) {
      spent += k;
      k = 0;
      stopped = stop_due(p, spent, next_poll, threadIdx.x & 31);
      if (stopped) break;
    }
  }
  if (stopped) stop_warp(p, stopped, busy, s.prefix, s.cnt, false, threadIdx.x & 31);
  block_reduce_add(lane_total, p.total, red);
  if (NODES) block_reduce_add(s.nodes, p.nodes, red);
}

template <bool VSYM, bool NODES, bool DG, bool LA, bool FU, bool WIDE = false>
__global__ void __launch_bounds__(512)
    k_snapshot(const __grid_constant__ KParams p, int diag) {
  extern __shared__ uint32_t smem[];
  __shared__ unsigned long long red[16];
  const unsigned B = blockDim.x;
  const int lane = threadIdx.x & 31;
  using K = SnapKind<SnapKindOf<VSYM, WIDE>::value>;
  const Cell *tbl;
  typename K::Table tb;
  SnapStack st;
  typename K::Lane s;
  snap_setup<K::W2>(p, diag, DG, smem, tbl, tb, st, s, LA || FU);
  uint32_t ovf = 0u;

  unsigned long long lane_total = 0ull;
  bool busy = false;
  bool qdone = false;
  const bool stoppable = p.budget > 0 || p.abort_flag != nullptr;
  long long spent = 0, next_poll = 0;
  unsigned stopped = 0u;
  for (;;) {
    if (stoppable && (stopped = stop_due(p, spent, next_poll, lane)) != 0u) break;
    unsigned idle = __ballot_sync(FULL, !busy);
    while (idle != 0u && !qdone) {
      const int nidle = __popc(idle);
      unsigned long long base = 0ull;
      if (lane == 0) base = atomicAdd(p.queue, (unsigned long long)nidle);
      base = __shfl_sync(FULL, base, 0);
      if (!busy) {
        const long long k = (long long)base + __popc(idle & ((1u << lane) - 1u));
        if (k < p.n_items) {
          const long long item =
              p.qstride ? (long long)(((unsigned long long)k * p.qstride) %
                                      (unsigned long long)p.n_items)
                        : k;
          busy = !snap_load<VSYM, NODES>(s, p, item, tbl, tb);
          if (!busy) finish_snapshot_item(s.prefix, s.cnt, p, ovf, lane_total);
        }
      }
      if ((long long)(base + (unsigned long long)nidle) >= p.n_items) qdone = true;
      idle = __ballot_sync(FULL, !busy);
    }
    if (idle == FULL) break;  // queue drained and every lane idle
    if (!qdone) {
      // every lane is busy here: step until one finishes (or, when the
      // count may stop early, at most check_every iterations)
      bool fin;
      if (!stoppable) {
        do {
          fin = K::template step<NODES, DG, LA, FU>(s, p.g, st, tb, B, ovf);
        } while (!__any_sync(FULL, fin));
      } else {
        int k = 0;
        do {
          fin = K::template step<NODES, DG, LA, FU>(s, p.g, st, tb, B, ovf);
        } while (!__any_sync(FULL, fin) && ++k <= p.check_mask);
        spent += k + 1;
      }
      if (fin) {
        busy = false;
        finish_snapshot_item(s.prefix, s.cnt, p, ovf, lane_total);
      }
    } else {
      for (int it = 0; it <= p.check_mask; ++it) {
        if (busy && K::template step<NODES, DG, LA, FU>(s, p.g, st, tb, B, ovf)) {
          busy = false;
          finish_snapshot_item(s.prefix, s.cnt, p, ovf, lane_total);
        }
      }
      spent += p.check_mask + 1;
      if (p.donate) snap_donate<VSYM, DG>(s, busy, p, st, tb, lane, B);
    }
  }
  if (stopped) stop_warp(p, stopped, busy, s.prefix, s.cnt, true, lane);
  block_reduce_add(lane_total, p.total, red);
  if (NODES) block_reduce_add(s.nodes, p.nodes, red);
}

// --------------------------------------------------- weighted 128-bit sum --

// 128-bit (hi, lo) += 64-bit x * 32-bit y
__device__ __forceinline__ void acc_mul(unsigned long long &hi, unsigned long long &lo,
                                        unsigned long long x, unsigned y) {
  const unsigned long long plo = x * (unsigned long long)y;
  const unsigned long long phi = __umul64hi(x, (unsigned long long)y);
  lo += plo;
  hi += phi + (lo < plo ? 1ull : 0ull);
}

__device__ __forceinline__ void acc_add(unsigned long long &hi, unsigned long long &lo,
                                        unsigned long long ohi, unsigned long long olo) {
  lo += olo;
  hi += ohi + (lo < olo ? 1ull : 0ull);
}

// Sum over k of counts[k] * weights[k] (weights NULL: 1) into out[0] (low
// 64 bits) and out[1] (high 64 bits): per-thread 128-bit sums, a warp and a
// block reduction, then one pair of atomics per block (the carry of the low
// word is detected from the value it replaced).
__global__ void __launch_bounds__(256) k_weighted_sum(const unsigned long long *counts,
                                                      const uint32_t *weights, long long n,
                                                      unsigned long long *out) {
  __shared__ unsigned long long rh[8];
  __shared__ unsigned long long rl[8];
  unsigned long long hi = 0ull, lo = 0ull;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    acc_mul(hi, lo, counts[k], weights ? weights[k] : 1u);
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long h2 = __shfl_down_sync(FULL, hi, o);
    const unsigned long long l2 = __shfl_down_sync(FULL, lo, o);
    acc_add(hi, lo, h2, l2);
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) {
    rh[warp] = hi;
    rl[warp] = lo;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    hi = lo = 0ull;
    for (unsigned w = 0; w < (blockDim.x >> 5); ++w) acc_add(hi, lo, rh[w], rl[w]);
    const unsigned long long old = atomicAdd(out, lo);
    if (old + lo < old) hi += 1ull;
    if (hi) atomicAdd(out + 1, hi);
  }
}

// ------------------------------------------------------------ host side --

// What the last count on a work area launched (for its status query).
struct LaunchRecord {
  int64_t n_prefixes = -1;  // -1: nothing counted yet
  int lanes_log2 = 0;
  bool queued = false;      // a persistent kernel that takes items from the queue
};

struct Workspace {
  unsigned long long *scratch = nullptr;  // [0] queue head, [1] status word
  uint8_t *h2d = nullptr;                 // host-entry prefix buffer
  size_t h2d_bytes = 0;
  unsigned long long *d2h = nullptr;      // host-entry counts buffer
  size_t d2h_count = 0;
  LaunchRecord last;
};

static std::mutex g_ws_mutex;
static std::map<std::pair<int, cudaStream_t>, Workspace> g_ws;

static int cuda_fail(cudaError_t e) {
  set_cuda_error(cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? DLS_ERR_NO_MEMORY : DLS_ERR_CUDA;
}

static int get_workspace(cudaStream_t stream, Workspace **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  std::lock_guard<std::mutex> g(g_ws_mutex);
  Workspace &w = g_ws[{dev, stream}];
  if (w.scratch == nullptr) {
    e = cudaMalloc(&w.scratch, 256);
    if (e != cudaSuccess) {
      w.scratch = nullptr;
      return cuda_fail(e);
    }
  }
  *out = &w;
  return DLS_OK;
}

struct DevInfo {
  int sms = 0;
  size_t smem_optin = 0;
  size_t smem_per_sm = 0;
};

static int dev_info(DevInfo *d) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  static std::mutex m;
  static std::map<int, DevInfo> cache;
  std::lock_guard<std::mutex> g(m);
  auto it = cache.find(dev);
  if (it == cache.end()) {
    DevInfo di;
    int v = 0;
    e = cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    if (e != cudaSuccess) return cuda_fail(e);
    di.sms = v;
    e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (e != cudaSuccess) return cuda_fail(e);
    di.smem_optin = (size_t)v;
    e = cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e != cudaSuccess) return cuda_fail(e);
    di.smem_per_sm = (size_t)v;
    it = cache.emplace(dev, di).first;
  }
  *d = it->second;
  return DLS_OK;
}

static int ilog2_exact(int x) {
  int r = 0;
  while ((1 << r) < x) ++r;
  return ((1 << r) == x) ? r : -1;
}

// Resolved launch shape.
struct Shape {
  int kernel;
  int block;
  int blocks_per_sm;
  int lanes_log2;
  int split_pos;
  int donate;
  int check_mask;
  int words;  // 0 auto, 1 shared memory, 2 registers
  int stack;  // 0 auto, 1 one entry per position, 2 snapshots
  int lookahead;
  int fuse;   // -1 off, 0 where it applies, 1 on
  long long budget;
  int stack_cap;
  const volatile int *abort_flag;
};

static int resolve_shape(const dls_launch_t *cfg, int depth, int last,
                         Shape *sh) {
  dls_launch_t c;
  std::memset(&c, 0, sizeof(c));
  if (cfg) c = *cfg;
  sh->kernel = c.kernel;
  if (sh->kernel != DLS_KERNEL_PERSISTENT && sh->kernel != DLS_KERNEL_PLAIN)
    return DLS_ERR_BAD_ARG;
  sh->block = c.block_threads ? c.block_threads : 128;
  if (sh->block < 32 || sh->block > 512 || sh->block % 32) return DLS_ERR_BAD_ARG;
  sh->blocks_per_sm = c.blocks_per_sm;
  if (sh->blocks_per_sm < 0) return DLS_ERR_BAD_ARG;
  int lanes = c.lanes_per_prefix ? c.lanes_per_prefix : 1;
  sh->lanes_log2 = ilog2_exact(lanes);
  if (sh->lanes_log2 < 0 || lanes > 32) return DLS_ERR_BAD_ARG;
  // the split needs a position with a stack entry below it
  if (depth >= last) sh->lanes_log2 = 0;
  if (sh->lanes_log2 > 0) {
    int sp = c.split_pos ? c.split_pos : std::min(depth + 2, last - 1);
    if (sp < depth || sp > last - 1) return DLS_ERR_BAD_ARG;
    sh->split_pos = sp;
  } else {
    sh->split_pos = -1;
  }
  sh->donate = (c.donate >= 0) ? 1 : 0;
  int every = c.check_every ? c.check_every : 64;
  if (ilog2_exact(every) < 0) return DLS_ERR_BAD_ARG;
  sh->check_mask = every - 1;
  sh->words = c.words;
  if (sh->words < 0 || sh->words > 2) return DLS_ERR_BAD_ARG;
  sh->stack = c.stack;
  if (sh->stack < 0 || sh->stack > 2) return DLS_ERR_BAD_ARG;
  sh->lookahead = c.lookahead;
  if (sh->lookahead < 0 || sh->lookahead > 1) return DLS_ERR_BAD_ARG;
  sh->fuse = c.fuse;
  if (sh->fuse < -1 || sh->fuse > 1) return DLS_ERR_BAD_ARG;
  if (c.budget < 0) return DLS_ERR_BAD_ARG;
  sh->budget = c.budget;
  sh->abort_flag = c.abort_flag;
  if (c.stack_cap < 0) return DLS_ERR_BAD_ARG;
  sh->stack_cap = c.stack_cap;
  return DLS_OK;
}

// Entries a snapshot stack needs: the order positions from depth to the one
// before the last whose cell can have two or more candidates.  A cell on a
// line that has all its other cells earlier in the order has at most one
// (the value the line misses), and entries are only made where a candidate
// remains after the one placed, at strictly increasing positions of a path.
// Lines: rows, columns and, with DLS_DIAGONAL, the two diagonals; with
// DLS_VSYM (left-half cells) a row holds n/2 cells whose last one still has
// a value pair to choose from, so only the columns (n cells each) and the
// diagonal line -- the left cell of each row on either diagonal, n cells
// that fix the n values of the main diagonal -- force a cell.
static int snapshot_entries(const OrderInfo &info, int n, uint32_t flags, int depth) {
  const bool diag = (flags & DLS_DIAGONAL) != 0, vsym = (flags & DLS_VSYM) != 0;
  int rowc[DLS_MAX_N] = {0}, colc[DLS_MAX_N] = {0};
  int mdc = 0, adc = 0, dline = 0;
  int cap = 0;
  for (int t = 0; t + 1 < info.len; ++t) {
    const int i = info.i[t], j = info.j[t];
    const bool md = diag && i == j, ad = diag && i + j == n - 1;
    bool forced;
    if (vsym)
      forced = colc[j] == n - 1 || ((md || ad) && dline == n - 1);
    else
      forced = rowc[i] == n - 1 || colc[j] == n - 1 || (md && mdc == n - 1) ||
               (ad && adc == n - 1);
    if (t >= depth && !forced) ++cap;
    ++rowc[i];
    ++colc[j];
    mdc += md ? 1 : 0;
    adc += ad ? 1 : 0;
    dline += (md || ad) ? 1 : 0;
  }
  return cap;
}

template <bool REG, bool VSYM, bool NODES, bool SPLIT>
static const void *kernel_ptr(int kind) {
  return kind == DLS_KERNEL_PLAIN ? (const void *)k_plain<REG, VSYM, NODES, SPLIT>
                                  : (const void *)k_persistent<REG, VSYM, NODES, SPLIT>;
}

template <bool REG, bool VSYM, bool NODES>
static const void *pick3(int kind, bool split) {
  return split ? kernel_ptr<REG, VSYM, NODES, true>(kind)
               : kernel_ptr<REG, VSYM, NODES, false>(kind);
}

template <bool REG>
static const void *pick2(int kind, bool vsym, bool nodes, bool split) {
  if (vsym) return nodes ? pick3<REG, true, true>(kind, split) : pick3<REG, true, false>(kind, split);
  return nodes ? pick3<REG, false, true>(kind, split) : pick3<REG, false, false>(kind, split);
}

static const void *pick_kernel(int kind, bool reg, bool vsym, bool nodes, bool split) {
  return reg ? pick2<true>(kind, vsym, nodes, split) : pick2<false>(kind, vsym, nodes, split);
}

template <bool VSYM, bool NODES, bool DG, bool WIDE>
static const void *snapshot_ptr(bool plain) {
  return plain ? (const void *)k_plain_snap<VSYM, NODES, DG, false, WIDE>
               : (const void *)k_snapshot<VSYM, NODES, DG, false, false, WIDE>;
}

template <bool VSYM, bool WIDE>
static const void *pick_snapshot2(bool plain, bool nodes, bool dg) {
  if (dg) return nodes ? snapshot_ptr<VSYM, true, true, WIDE>(plain)
                       : snapshot_ptr<VSYM, false, true, WIDE>(plain);
  return nodes ? snapshot_ptr<VSYM, true, false, WIDE>(plain)
               : snapshot_ptr<VSYM, false, false, WIDE>(plain);
}

// the fused step (no diagonal words) or the lookahead (no diagonal words,
// no vertical symmetry)
template <bool WIDE>
static const void *pick_snapshot_fl(bool plain, bool nodes, bool la) {
  if (!la && plain) return nodes ? (const void *)k_plain_snap<false, true, false, true, WIDE>
                                 : (const void *)k_plain_snap<false, false, false, true, WIDE>;
  if (!la) return nodes ? (const void *)k_snapshot<false, true, false, false, true, WIDE>
                        : (const void *)k_snapshot<false, false, false, false, true, WIDE>;
  return nodes ? (const void *)k_snapshot<false, true, false, true, false, WIDE>
               : (const void *)k_snapshot<false, false, false, true, false, WIDE>;
}

static const void *pick_snapshot_vsym_fu(bool plain, bool nodes) {
  if (plain) return nodes ? (const void *)k_plain_snap<true, true, false, true>
                          : (const void *)k_plain_snap<true, false, false, true>;
  return nodes ? (const void *)k_snapshot<true, true, false, false, true>
               : (const void *)k_snapshot<true, false, false, false, true>;
}

// dg: some cell at or after the prefix depth lies on a diagonal (the
// diagonal words change during the search); la: the persistent kernel with
// the lookahead (no diagonal words, no vertical symmetry); fu: the fused
// step (no diagonal words); wide: the wide-word search of order 9
static const void *pick_snapshot(bool plain, bool vsym, bool wide, bool nodes, bool dg, bool la,
                                 bool fu) {
  if (fu && vsym) return pick_snapshot_vsym_fu(plain, nodes);
  if (fu || la) return wide ? pick_snapshot_fl<true>(plain, nodes, la)
                            : pick_snapshot_fl<false>(plain, nodes, la);
  if (vsym) return pick_snapshot2<true, false>(plain, nodes, dg);
  return wide ? pick_snapshot2<false, true>(plain, nodes, dg)
              : pick_snapshot2<false, false>(plain, nodes, dg);
}

static bool diagonal_cells_after(const OrderInfo &info, int n, uint32_t flags, int depth) {
  if (!(flags & DLS_DIAGONAL)) return false;
  for (int t = depth; t < info.len; ++t)
    if (info.i[t] == info.j[t] || info.i[t] + info.j[t] == n - 1) return true;
  return false;
}

// Do all row words and all column words fit one 64-bit register each?
// Field widths: 8 bits per row and column for n <= 8; with vertical
// symmetry n/2 bits per row (value pairs) and n bits per left column.
static bool words_fit_registers(int n, bool vsym, int *wr, int *wc) {
  if (!vsym) {
    if (n > 8) return false;
    *wr = 8;
    *wc = 8;
    return true;
  }
  if (n % 2) return false;
  *wr = n / 2;
  *wc = n;
  return n * (n / 2) <= 64;
}

static size_t smem_bytes(int order_len, int n, int depth, int last, int block,
                         bool reg) {
  const int stack = std::max(0, last - depth);
  return (size_t)((order_len + 31) & ~31) * 8u + (size_t)((reg ? 0 : 2 * n) + stack) * block * 4u;
}

// Snapshot kernels: the cell table and the position table (8 + 24 bytes per
// position with vertical symmetry, 8 + 48 with byte words, 8 + 80 with wide
// words), then 20 bytes (32 with wide words) per entry slot and lane (cap + 2
// slots).
static size_t smem_bytes_snapshot(int order_len, int entries, int block, bool vsym,
                                  bool wide = false) {
  const size_t row = vsym ? 32u : (wide ? 88u : 56u);
  return (size_t)((order_len + 31) & ~31) * row +
         (size_t)(entries + 2) * block * (wide ? 32u : 20u);
}

// A resolved launch: the parameter block, the kernel and its shape.
// dls_launch_t.fuse = 0 takes the fused step where it applies.
static constexpr bool kFuseByDefault = true;

struct Prepared {
  KParams kp;
  const void *fn = nullptr;
  int run = DLS_RUN_PERSISTENT;  // dls_run_kind
  int diag = 0;
  bool reg = false;
  int block = 0;
  unsigned grid = 0;  // 0 = nothing to launch
  size_t smem = 0;
  bool store = false;
  bool fused = false;  // snapshot search with the fused step
  bool wide = false;   // the wide-word search (order 9)
  int bound = 0;       // snapshot entries no search can exceed
  // a capped stack: the recount pass (same kernel, full bound, deferred
  // prefixes only) and the total summed from the counts afterwards
  bool recount = false;
  KParams kp2;
  int block2 = 0;
  unsigned grid2 = 0;
  size_t smem2 = 0;
  uint64_t *total_out = nullptr;
};

// Validates the arguments and resolves the kernel and its launch shape
// (no device work).  grid stays 0 when there is nothing to launch (no
// prefixes, or odd vertically symmetric orders whose counts are all 0).
static int prepare_launch(int n, uint32_t flags, const uint8_t *order, int order_len,
                          const uint8_t *d_prefixes, int depth, int64_t n_prefixes,
                          uint64_t *d_counts, uint64_t *d_total, uint64_t *d_nodes,
                          const dls_launch_t *cfg, Prepared *pr) {
  OrderInfo info;
  int rc = validate_order(n, flags, order, order_len, &info);
  if (rc) return rc;
  if (depth < 0 || depth > order_len || n_prefixes < 0) return DLS_ERR_BAD_ARG;
  Shape sh;
  rc = resolve_shape(cfg, depth, order_len - 1, &sh);
  if (rc) return rc;
  const bool zero_all = vsym_all_zero(n, flags);
  pr->store = sh.kernel == DLS_KERNEL_PLAIN && sh.lanes_log2 == 0;

  KParams &kp = pr->kp;
  std::memset(&kp, 0, sizeof(kp));
  kp.g.n = n;
  kp.g.all = (1u << n) - 1u;
  kp.g.pairmask = (1u << (n / 2)) - 1u;
  kp.g.depth = depth;
  kp.g.last = order_len - 1;
  kp.order_len = order_len;
  kp.sp.lanes_log2 = sh.lanes_log2;
  kp.sp.pos = sh.split_pos;
  kp.check_mask = sh.check_mask;
  kp.budget = sh.budget;
  kp.abort_flag = sh.abort_flag;
  kp.donate = sh.donate;
  kp.count_store = pr->store ? 1 : 0;
  kp.n_prefixes = n_prefixes;
  kp.n_items = n_prefixes << sh.lanes_log2;
  kp.prefixes = d_prefixes;
  kp.qstride = 0ull;
  kp.counts = reinterpret_cast<unsigned long long *>(d_counts);
  kp.total = reinterpret_cast<unsigned long long *>(d_total);
  kp.nodes = reinterpret_cast<unsigned long long *>(d_nodes);
  for (int t = 0; t < order_len; ++t) {
    kp.ci[t] = info.i[t];
    kp.cj[t] = info.j[t];
  }
  pr->diag = (flags & DLS_DIAGONAL) ? 1 : 0;
  const bool vsym = (flags & DLS_VSYM) != 0;
  int wr = 0, wc = 0;
  bool reg = words_fit_registers(n, vsym, &wr, &wc);
  if (sh.words == 1) reg = false;
  kp.wr = wr;
  kp.wc = wc;
  // the snapshot search: register words, one lane per prefix; order
  // positions must fit its packed entry.  Order 9 without vertical symmetry
  // takes the wide words when at most 8 rows have cells after the prefix.
  int rs9[DLS_MAX_N], cs9[DLS_MAX_N];
  const bool wide = !vsym && n == 9 && sh.lanes_log2 == 0 && sh.words != 1 &&
                    wide_slots(n, info.i, info.j, order_len, depth, rs9, cs9);
  if (wide) {
    for (int k = 0; k < DLS_MAX_N; ++k) {
      kp.rslot[k] = (int8_t)(k < n ? rs9[k] : -1);
      kp.cslot[k] = (int8_t)(k < n ? cs9[k] : -1);
    }
  }
  kp.diag_words = (flags & DLS_DIAGONAL) ? 1 : 0;
  const bool snap_ok = (reg || wide) && sh.lanes_log2 == 0 && order_len <= (vsym ? 64 : 256);
  if (sh.stack == 2 && !snap_ok) return DLS_ERR_BAD_ARG;
  bool snap = snap_ok && sh.stack != 1;
  kp.snap_cap = snap ? std::max(1, snapshot_entries(info, n, flags, depth)) : 0;
  pr->bound = kp.snap_cap;
  // a stack cap below the bound needs per-prefix counts to defer to (and no
  // node count, budget or abort flag); otherwise the bound stays
  const bool can_defer = d_counts != nullptr && d_nodes == nullptr && sh.budget == 0 &&
                         sh.abort_flag == nullptr;
  DevInfo di;
  rc = dev_info(&di);
  if (rc) return rc;
  // static shared memory of the kernels: the 16-entry reduction buffer
  const size_t static_smem = 16 * sizeof(unsigned long long);
  // the wide words' 32-byte entries leave one block of 128 lanes per SM at
  // the full bound of a typical order-9 split; by default they take the
  // largest cap with which two blocks fit (canonical order-9 hourglasses
  // split 4 cells deeper: bound 31, 1 block, 3.7e9 squares/s; cap 20, 5.2e9;
  // cap 24, 5.6e9)
  int cap_asked = sh.stack_cap;
  if (cap_asked == 0 && wide && snap) {
    const int blk = sh.block;
    cap_asked = kp.snap_cap;
    while (cap_asked > 1 &&
           2 * (smem_bytes_snapshot(order_len, cap_asked, blk, false, true) + static_smem +
                1024) > di.smem_per_sm)
      --cap_asked;
  }
  if (snap && cap_asked > 0 && cap_asked < kp.snap_cap && can_defer) {
    kp.snap_cap = cap_asked;
    pr->recount = true;
    kp.defer = 1;
    pr->total_out = d_total;
    kp.total = nullptr;  // summed from the counts after the recount pass
  }
  const bool default_block = cfg == nullptr || cfg->block_threads == 0;
  // by default, an explicit block size whose snapshot stacks do not fit
  // falls back to the per-position stack (a fifth of the bytes per entry)
  if (snap && sh.stack == 0 && !default_block &&
      smem_bytes_snapshot(order_len, kp.snap_cap, sh.block, vsym, wide) + static_smem >
          di.smem_optin) {
    snap = false;
    kp.snap_cap = 0;
  }
  // words in registers: the 64-bit fields, or the wide words of a snapshot
  if (sh.words == 2 && !reg && !(snap && wide)) return DLS_ERR_BAD_ARG;
  pr->reg = reg;
  const bool plain = sh.kernel == DLS_KERNEL_PLAIN;
  pr->run = snap ? (plain ? DLS_RUN_PLAIN_SNAPSHOT : DLS_RUN_SNAPSHOT)
                 : (plain ? DLS_RUN_PLAIN : DLS_RUN_PERSISTENT);
  const bool dgw = diagonal_cells_after(info, n, flags, depth);
  const bool la = snap && !plain && sh.lookahead && !dgw && !vsym;
  if (sh.lookahead && !la) return DLS_ERR_BAD_ARG;
  // the fused step: snapshot search without diagonal words; not with the
  // lookahead
  const bool fu_fits = snap && !dgw && !la;
  if (sh.fuse == 1 && !fu_fits) return DLS_ERR_BAD_ARG;
  // (by default not with vertical symmetry: there the second placement, with
  // its mirrored words, costs more than the iterations it saves)
  const bool fu = fu_fits && (sh.fuse == 1 || (sh.fuse == 0 && kFuseByDefault && !vsym));
  pr->fused = fu;
  pr->wide = snap && wide;
  pr->fn = snap ? pick_snapshot(plain, vsym, pr->wide, d_nodes != nullptr, dgw, la, fu)
                : pick_kernel(sh.kernel, reg, vsym, d_nodes != nullptr, sh.lanes_log2 > 0);
  auto smem_for = [&](int block) {
    return snap ? smem_bytes_snapshot(order_len, kp.snap_cap, block, vsym, pr->wide)
                : smem_bytes(order_len, n, depth, order_len - 1, block, reg);
  };
  size_t smem = smem_for(sh.block);
  while (default_block && smem + static_smem > di.smem_optin && sh.block > 32) {
    sh.block /= 2;
    smem = smem_for(sh.block);
  }
  if (smem + static_smem > di.smem_optin) return DLS_ERR_NO_MEMORY;
  pr->block = sh.block;
  pr->smem = smem;
  pr->grid = 0;
  if (n_prefixes == 0 || zero_all) return DLS_OK;
  cudaError_t e = cudaFuncSetAttribute(pr->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return cuda_fail(e);
  auto grid_for = [&](int block, size_t sm, unsigned *grid) -> int {
    if (sh.kernel == DLS_KERNEL_PLAIN) {
      long long g = (kp.n_items + block - 1) / block;
      if (g > 0x7fffffffll) return DLS_ERR_BAD_ARG;
      *grid = (unsigned)g;
      return DLS_OK;
    }
    int per_sm = sh.blocks_per_sm;
    if (per_sm == 0) {
      cudaError_t e2 = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, pr->fn, block, sm);
      if (e2 != cudaSuccess) return cuda_fail(e2);
      if (per_sm < 1) return DLS_ERR_NO_MEMORY;
    }
    long long want = (long long)di.sms * per_sm;
    long long need = (kp.n_items + 31) / 32;  // warps with at least one item
    long long blocks_needed = (need * 32 + block - 1) / block;
    *grid = (unsigned)std::max(1ll, std::min(want, blocks_needed));
    return DLS_OK;
  };
  rc = grid_for(sh.block, smem, &pr->grid);
  if (rc) return rc;
  // the batched byte-word search takes its queue in a strided order (see
  // KParams::qstride) where the lanes of the grid get few prefixes each (at
  // most 16: the end of the queue is then a large part of the pass; with
  // more -- the symmetric order-10 workload, 32 per lane -- the given order
  // measured faster); not where a count may stop early, whose report of the
  // prefixes handed out ("every prefix from here on") needs the given order
  if (snap && !plain && !vsym && !pr->wide && sh.budget == 0 && sh.abort_flag == nullptr &&
      kp.n_items >= 4096 && kp.n_items < (1ll << 32) &&
      kp.n_items <= 16ll * (long long)pr->grid * (long long)sh.block) {
    unsigned long long a = (unsigned long long)(kp.n_items + 63) / 64ull;
    while (std::gcd(a, (unsigned long long)kp.n_items) != 1ull) ++a;
    kp.qstride = a;
  }
  if (pr->recount) {
    // the recount pass: the full bound, a smaller block where its stacks
    // need it; it takes only the deferred prefixes
    pr->kp2 = kp;
    pr->kp2.snap_cap = pr->bound;
    pr->kp2.defer = 0;
    pr->kp2.recount = 1;
    int b2 = sh.block;
    size_t sm2 = smem_bytes_snapshot(order_len, pr->bound, b2, vsym, pr->wide);
    while (sm2 + static_smem > di.smem_optin && b2 > 32) {
      b2 /= 2;
      sm2 = smem_bytes_snapshot(order_len, pr->bound, b2, vsym, pr->wide);
    }
    if (sm2 + static_smem > di.smem_optin) return DLS_ERR_NO_MEMORY;
    if (sm2 > smem) {
      e = cudaFuncSetAttribute(pr->fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm2);
      if (e != cudaSuccess) return cuda_fail(e);
    }
    pr->block2 = b2;
    pr->smem2 = sm2;
    const int saved = sh.blocks_per_sm;
    sh.blocks_per_sm = 0;  // the occupancy of the recount pass's own shape
    rc = grid_for(b2, sm2, &pr->grid2);
    sh.blocks_per_sm = saved;
    if (rc) return rc;
  }
  return DLS_OK;
}

// Sum of n counts into *total (64 bits; the total of one count call).
__global__ void __launch_bounds__(256) k_sum_counts(const unsigned long long *counts,
                                                    long long n, unsigned long long *total) {
  __shared__ unsigned long long red[8];
  unsigned long long v = 0ull;
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < n;
       k += (long long)gridDim.x * blockDim.x)
    v += counts[k];
  block_reduce_add(v, total, red);
}

// Validates, fills the parameter block and enqueues the whole pass on
// `stream`: zero the outputs, reset the queue, launch.
static int enqueue_count(int n, uint32_t flags, const uint8_t *order,
                         int order_len, const uint8_t *d_prefixes, int depth,
                         int64_t n_prefixes, uint64_t *d_counts,
                         uint64_t *d_total, uint64_t *d_nodes,
                         const dls_launch_t *cfg, cudaStream_t stream,
                         unsigned long long *scratch = nullptr,
                         LaunchRecord *rec = nullptr) {
  if (n_prefixes > 0 && d_counts == nullptr && d_total == nullptr) return DLS_ERR_BAD_ARG;
  if (n_prefixes > 0 && depth > 0 && d_prefixes == nullptr) return DLS_ERR_BAD_ARG;
  Prepared pr;
  int rc = prepare_launch(n, flags, order, order_len, d_prefixes, depth, n_prefixes, d_counts,
                          d_total, d_nodes, cfg, &pr);
  if (rc) return rc;
  cudaError_t e;
  if (d_total) {
    e = cudaMemsetAsync(d_total, 0, sizeof(uint64_t), stream);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (d_nodes) {
    e = cudaMemsetAsync(d_nodes, 0, sizeof(uint64_t), stream);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  if (d_counts && n_prefixes > 0 && (!pr.store || pr.grid == 0)) {
    e = cudaMemsetAsync(d_counts, 0, (size_t)n_prefixes * sizeof(uint64_t), stream);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  // the work area: queue head and status word, cleared for every count so
  // that the status always describes the last one
  Workspace *ws = nullptr;
  if (scratch == nullptr) {
    rc = get_workspace(stream, &ws);
    if (rc) return rc;
    scratch = ws->scratch;
  }
  pr.kp.queue = scratch;
  e = cudaMemsetAsync(scratch, 0, 2 * sizeof(unsigned long long), stream);
  if (e != cudaSuccess) return cuda_fail(e);
  LaunchRecord r;
  r.n_prefixes = n_prefixes;
  r.lanes_log2 = pr.kp.sp.lanes_log2;
  r.queued = pr.grid != 0 && (pr.run == DLS_RUN_PERSISTENT || pr.run == DLS_RUN_SNAPSHOT);
  if (ws != nullptr) {
    std::lock_guard<std::mutex> g(g_ws_mutex);
    ws->last = r;
  }
  if (rec != nullptr) *rec = r;
  if (pr.grid == 0) return DLS_OK;
  void *args[] = {&pr.kp, (void *)&pr.diag};
  e = cudaLaunchKernel(pr.fn, dim3(pr.grid), dim3(pr.block), args, pr.smem, stream);
  if (e != cudaSuccess) return cuda_fail(e);
  if (pr.recount) {
    // the recount pass over the deferred prefixes, from a fresh queue head
    pr.kp2.queue = scratch;
    e = cudaMemsetAsync(scratch, 0, sizeof(unsigned long long), stream);
    if (e != cudaSuccess) return cuda_fail(e);
    void *args2[] = {&pr.kp2, (void *)&pr.diag};
    e = cudaLaunchKernel(pr.fn, dim3(pr.grid2), dim3(pr.block2), args2, pr.smem2, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    if (pr.total_out) {
      DevInfo di;
      rc = dev_info(&di);
      if (rc) return rc;
      const long long np = (long long)n_prefixes;
      const unsigned gs = (unsigned)std::max(1ll, std::min<long long>((np + 255) / 256,
                                                                      4ll * di.sms));
      unsigned long long *tot = reinterpret_cast<unsigned long long *>(pr.total_out);
      const unsigned long long *cnt = reinterpret_cast<const unsigned long long *>(d_counts);
      k_sum_counts<<<gs, 256, 0, stream>>>(cnt, np, tot);
      e = cudaGetLastError();
      if (e != cudaSuccess) return cuda_fail(e);
    }
  }
  return DLS_OK;
}

// The status code a count's status word stands for: a stack overflow makes
// its counts untrustworthy (DLS_ERR_INTERNAL).
int status_code(unsigned word) {
  if (word & ST_OVERFLOW) return DLS_ERR_INTERNAL;
  if (word & ST_ABORTED) return DLS_ERR_ABORTED;
  if (word & ST_TIMEOUT) return DLS_ERR_TIMEOUT;
  return DLS_OK;
}

// Reads a work area's queue head and status word after `stream` has
// finished, and fills *out from them and the record of the count.
static int read_status(const unsigned long long *scratch, const LaunchRecord &rec,
                       cudaStream_t stream, dls_count_status *out) {
  if (rec.n_prefixes < 0) return DLS_ERR_BAD_STATE;
  unsigned long long w[2] = {0ull, 0ull};
  cudaError_t e = cudaStreamSynchronize(stream);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaMemcpy(w, scratch, sizeof(w), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e);
  out->status = status_code((unsigned)w[1]);
  int64_t started = rec.n_prefixes;
  if (rec.queued) {
    // items handed out (warps take a few past the end); a prefix is started
    // when its first item was
    const int64_t lanes = (int64_t)1 << rec.lanes_log2;
    const int64_t items = (int64_t)std::min<unsigned long long>(
        w[0], (unsigned long long)(rec.n_prefixes * lanes));
    started = std::min<int64_t>(rec.n_prefixes, (items + lanes - 1) / lanes);
  }
  out->prefixes_started = started;
  return DLS_OK;
}

// The persistent or plain launch of enqueue_count with the queue head at a
// caller-chosen device address (used by the allocation-free entry point).
int enqueue_count_with_scratch(int n, uint32_t flags, const uint8_t *order,
                               int order_len, const uint8_t *d_prefixes,
                               int depth, int64_t n_prefixes,
                               uint64_t *d_counts, const dls_launch_t *cfg,
                               cudaStream_t stream,
                               unsigned long long *scratch) {
  return enqueue_count(n, flags, order, order_len, d_prefixes, depth, n_prefixes,
                       d_counts, nullptr, nullptr, cfg, stream, scratch);
}

}  // namespace dls

using namespace dls;

extern "C" {

int dls_count_ex(int n, uint32_t flags, const uint8_t *order, int order_len,
                 const uint8_t *d_prefixes, int depth, int64_t n_prefixes,
                 uint64_t *d_counts, uint64_t *d_total, uint64_t *d_nodes,
                 const dls_launch_t *cfg, void *stream) {
  return enqueue_count(n, flags, order, order_len, d_prefixes, depth, n_prefixes,
                       d_counts, d_total, d_nodes, cfg,
                       reinterpret_cast<cudaStream_t>(stream));
}

int dls_describe_launch(int n, uint32_t flags, const uint8_t *order, int order_len,
                        int depth, int64_t n_prefixes, const dls_launch_t *cfg,
                        dls_launch_info *out) {
  if (out == nullptr) return DLS_ERR_BAD_ARG;
  // as a count with per-prefix counts and no node count would launch (the
  // pointer only enables the stack cap; nothing is launched)
  static uint64_t no_counts;
  Prepared pr;
  int rc = prepare_launch(n, flags, order, order_len, nullptr, depth, n_prefixes, &no_counts,
                          nullptr, nullptr, cfg, &pr);
  if (rc) return rc;
  out->run = pr.run;
  out->words = (pr.reg || pr.wide) ? 2 : 1;
  out->block_threads = pr.block;
  out->grid_blocks = (int)pr.grid;
  out->smem_bytes = (int)pr.smem;
  out->stack_entries = pr.kp.snap_cap;
  out->fused = pr.fused ? 1 : 0;
  const bool snapshot = pr.run == DLS_RUN_SNAPSHOT || pr.run == DLS_RUN_PLAIN_SNAPSHOT;
  out->step = !snapshot ? 0 : ((flags & DLS_VSYM) ? 1 : (pr.wide ? 3 : 2));
  return DLS_OK;
}

int dls_count(int n, uint32_t flags, const uint8_t *order, int order_len,
              const uint8_t *d_prefixes, int depth, int64_t n_prefixes,
              uint64_t *d_counts, uint64_t *d_total, void *stream) {
  dls_launch_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.kernel = DLS_KERNEL_PERSISTENT;
  return dls_count_ex(n, flags, order, order_len, d_prefixes, depth, n_prefixes,
                      d_counts, d_total, nullptr, &cfg, stream);
}

int dls_count_plain(int n, uint32_t flags, const uint8_t *order,
                    int order_len, const uint8_t *d_prefixes, int depth,
                    int64_t n_prefixes, uint64_t *d_counts, uint64_t *d_total,
                    void *stream) {
  dls_launch_t cfg;
  std::memset(&cfg, 0, sizeof(cfg));
  cfg.kernel = DLS_KERNEL_PLAIN;
  return dls_count_ex(n, flags, order, order_len, d_prefixes, depth, n_prefixes,
                      d_counts, d_total, nullptr, &cfg, stream);
}

int dls_count_host(int n, uint32_t flags, const uint8_t *order,
                   int order_len, const uint8_t *h_prefixes, int depth,
                   int64_t n_prefixes, uint64_t *h_counts,
                   dls_u128 *total_out, const dls_launch_t *cfg,
                   void *stream) {
  if (n_prefixes < 0 || depth < 0) return DLS_ERR_BAD_ARG;
  if (n_prefixes > 0 && depth > 0 && h_prefixes == nullptr) return DLS_ERR_BAD_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Workspace *ws = nullptr;
  int rc = get_workspace(st, &ws);
  if (rc) return rc;
  const size_t in_bytes = (size_t)n_prefixes * (size_t)depth;
  const size_t n_cnt = (size_t)n_prefixes;
  cudaError_t e;
  {
    std::lock_guard<std::mutex> g(g_ws_mutex);
    if (ws->h2d_bytes < in_bytes) {
      if (ws->h2d) cudaFree(ws->h2d);
      ws->h2d = nullptr;
      ws->h2d_bytes = 0;
      e = cudaMalloc(&ws->h2d, in_bytes);
      if (e != cudaSuccess) return cuda_fail(e);
      ws->h2d_bytes = in_bytes;
    }
    if (ws->d2h_count < n_cnt + 1) {
      if (ws->d2h) cudaFree(ws->d2h);
      ws->d2h = nullptr;
      ws->d2h_count = 0;
      e = cudaMalloc(&ws->d2h, (n_cnt + 1) * sizeof(unsigned long long));
      if (e != cudaSuccess) return cuda_fail(e);
      ws->d2h_count = n_cnt + 1;
    }
  }
  if (in_bytes) {
    e = cudaMemcpyAsync(ws->h2d, h_prefixes, in_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  uint64_t *d_counts = reinterpret_cast<uint64_t *>(ws->d2h);
  rc = enqueue_count(n, flags, order, order_len, ws->h2d, depth, n_prefixes,
                     d_counts, nullptr, nullptr, cfg, st);
  if (rc) return rc;
  if (h_counts && n_cnt) {
    e = cudaMemcpyAsync(h_counts, d_counts, n_cnt * sizeof(uint64_t),
                        cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) return cuda_fail(e);
  }
  unsigned long long flag = 0ull;
  e = cudaMemcpyAsync(&flag, ws->scratch + 1, sizeof(flag), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  rc = status_code((unsigned)flag);
  if (rc) return rc;
  if (total_out) {
    dls_u128 t = {0, 0};
    if (h_counts) {
      for (size_t k = 0; k < n_cnt; ++k) t = dls_add_u128(t, dls_u128{h_counts[k], 0});
    } else {
      std::vector<uint64_t> tmp(n_cnt);
      if (n_cnt) {
        e = cudaMemcpy(tmp.data(), d_counts, n_cnt * sizeof(uint64_t), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e);
      }
      for (size_t k = 0; k < n_cnt; ++k) t = dls_add_u128(t, dls_u128{tmp[k], 0});
    }
    *total_out = t;
  }
  return DLS_OK;
}

int dls_count_weighted(int n, uint32_t flags, const uint8_t *order, int order_len,
                       const uint8_t *d_prefixes, int depth, int64_t n_prefixes,
                       const uint32_t *d_weights, uint64_t *d_counts, int multiply,
                       dls_u128 *total_out, const dls_launch_t *cfg, void *stream) {
  if (total_out == nullptr || n_prefixes < 0) return DLS_ERR_BAD_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  Workspace *ws = nullptr;
  int rc = get_workspace(st, &ws);
  if (rc) return rc;
  cudaError_t e;
  if (d_counts == nullptr && n_prefixes > 0) {
    // the counts go to the work area's buffer (shared with dls_count_host)
    std::lock_guard<std::mutex> g(g_ws_mutex);
    if (ws->d2h_count < (size_t)n_prefixes + 1) {
      if (ws->d2h) cudaFree(ws->d2h);
      ws->d2h = nullptr;
      ws->d2h_count = 0;
      e = cudaMalloc(&ws->d2h, ((size_t)n_prefixes + 1) * sizeof(unsigned long long));
      if (e != cudaSuccess) return cuda_fail(e);
      ws->d2h_count = (size_t)n_prefixes + 1;
    }
    d_counts = reinterpret_cast<uint64_t *>(ws->d2h);
  }
  rc = enqueue_count(n, flags, order, order_len, d_prefixes, depth, n_prefixes, d_counts,
                     nullptr, nullptr, cfg, st);
  if (rc) return rc;
  // words 2-3 of the work area: the 128-bit sum
  unsigned long long *sum = ws->scratch + 2;
  e = cudaMemsetAsync(sum, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_fail(e);
  if (n_prefixes > 0) {
    DevInfo di;
    rc = dev_info(&di);
    if (rc) return rc;
    const long long want = (n_prefixes + 255) / 256;
    const unsigned grid = (unsigned)std::max(1ll, std::min<long long>(want, 4ll * di.sms));
    const unsigned long long *cnt = reinterpret_cast<const unsigned long long *>(d_counts);
    const long long np = (long long)n_prefixes;
    k_weighted_sum<<<grid, 256, 0, st>>>(cnt, d_weights, np, sum);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
  }
  unsigned long long h[4] = {0ull, 0ull, 0ull, 0ull};  // head, status, sum lo, sum hi
  e = cudaMemcpyAsync(h, ws->scratch, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) return cuda_fail(e);
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(e);
  rc = status_code((unsigned)h[1]);
  if (rc) return rc;
  dls_u128 t = {h[2], h[3]};
  if (multiply) {
    const dls_u128 m = dls_multiplier(n, flags);
    t = dls_mul_u64(m.lo, t);  // the multiplier is below 2^64 for every order taken
  }
  *total_out = t;
  return DLS_OK;
}

void dls_release(void) {
  noalloc_forget();
  std::lock_guard<std::mutex> g(g_ws_mutex);
  for (auto &kv : g_ws) {
    int cur = 0;
    cudaGetDevice(&cur);
    cudaSetDevice(kv.first.first);
    if (kv.second.scratch) cudaFree(kv.second.scratch);
    if (kv.second.h2d) cudaFree(kv.second.h2d);
    if (kv.second.d2h) cudaFree(kv.second.d2h);
    cudaSetDevice(cur);
  }
  g_ws.clear();
}

int dls_stream_status(void *stream, dls_count_status *out) {
  if (out == nullptr) return DLS_ERR_BAD_ARG;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e);
  const unsigned long long *scratch = nullptr;
  LaunchRecord rec;
  {
    std::lock_guard<std::mutex> g(g_ws_mutex);
    auto it = g_ws.find({dev, st});
    if (it == g_ws.end()) return DLS_ERR_BAD_STATE;
    scratch = it->second.scratch;
    rec = it->second.last;
  }
  return read_status(scratch, rec, st, out);
}

// ------------------------------------------------------------------ plans

}  // extern "C"

struct dls_plan {
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaStream_t capture = nullptr;
  unsigned long long *scratch = nullptr;  // the plan's own queue head, status word
  dls::LaunchRecord rec;
};

extern "C" {

int dls_plan_create(dls_plan **plan_out, int n, uint32_t flags,
                    const uint8_t *order, int order_len,
                    const uint8_t *d_prefixes, int depth, int64_t n_prefixes,
                    uint64_t *d_counts, uint64_t *d_total,
                    const dls_launch_t *cfg) {
  if (plan_out == nullptr) return DLS_ERR_BAD_ARG;
  *plan_out = nullptr;
  dls_plan *pl = new (std::nothrow) dls_plan();
  if (!pl) return DLS_ERR_NO_MEMORY;
  cudaError_t e = cudaStreamCreateWithFlags(&pl->capture, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    delete pl;
    return cuda_fail(e);
  }
  // the plan's own work area, allocated before capture (no allocation while
  // capturing)
  int rc = DLS_OK;
  e = cudaMalloc(&pl->scratch, 256);
  if (e != cudaSuccess) {
    pl->scratch = nullptr;
    rc = cuda_fail(e);
  }
  if (rc == DLS_OK) {
    e = cudaStreamBeginCapture(pl->capture, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) rc = cuda_fail(e);
  }
  if (rc == DLS_OK) {
    rc = enqueue_count(n, flags, order, order_len, d_prefixes, depth, n_prefixes,
                       d_counts, d_total, nullptr, cfg, pl->capture, pl->scratch, &pl->rec);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(pl->capture, &g);
    if (rc == DLS_OK && e != cudaSuccess) rc = cuda_fail(e);
    pl->graph = g;
  }
  if (rc == DLS_OK) {
    e = cudaGraphInstantiate(&pl->exec, pl->graph, 0);
    if (e != cudaSuccess) rc = cuda_fail(e);
  }
  if (rc != DLS_OK) {
    dls_plan_destroy(pl);
    return rc;
  }
  *plan_out = pl;
  return DLS_OK;
}

int dls_plan_launch(dls_plan *plan, void *stream) {
  if (plan == nullptr || plan->exec == nullptr) return DLS_ERR_BAD_STATE;
  cudaError_t e = cudaGraphLaunch(plan->exec, reinterpret_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e);
  return DLS_OK;
}

int dls_plan_status(dls_plan *plan, void *stream, dls_count_status *out) {
  if (plan == nullptr || plan->exec == nullptr) return DLS_ERR_BAD_STATE;
  if (out == nullptr) return DLS_ERR_BAD_ARG;
  return read_status(plan->scratch, plan->rec, reinterpret_cast<cudaStream_t>(stream), out);
}

void dls_plan_destroy(dls_plan *plan) {
  if (!plan) return;
  if (plan->exec) cudaGraphExecDestroy(plan->exec);
  if (plan->graph) cudaGraphDestroy(plan->graph);
  if (plan->capture) cudaStreamDestroy(plan->capture);
  if (plan->scratch) cudaFree(plan->scratch);
  delete plan;
}

}  // extern "C"
