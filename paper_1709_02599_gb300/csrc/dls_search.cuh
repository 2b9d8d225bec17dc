// dls_search.cuh -- the per-lane search of Algorithm 4, shared by the batch
// kernels (dls_kernels.cu) and the serving kernel (dls_serve.cu).
//
// One lane runs one depth-first search over the order positions after its
// prefix.  Its state is the bitmask form of Section 3 -- a word per row and
// per column holding the values in use, plus the two diagonal words -- and a
// stack of (untried candidates, placed value) per position, i.e. the
// L[i][j] / LS[i][j] pairs of Algorithm 4 kept as an explicit stack instead of
// nested loops.
#pragma once

#include <cstdint>

#include "dls_internal.h"

namespace dls {

constexpr unsigned FULL = 0xffffffffu;

// Shape of one search.
struct Geo {
  int n;
  uint32_t all;       // admissible values: (1 << n) - 1, without (n-1)/2
                      // for odd vertically symmetric orders (its mirror
                      // would repeat it in the same row)
  uint32_t pairmask;  // (1 << n/2) - 1: value pairs of a symmetric row
  int depth;          // prefix length = first position with a stack entry
  int last;           // order length - 1
  uint32_t vsmask;    // all ones with vertical symmetry, else 0 (read only by
                      // the step that takes the flag at run time)
};

// Work-item split of a prefix over several lanes (SPLIT kernels only).
struct Split {
  int pos;            // order position of the split (-1 = none)
  int lanes_log2;     // items per prefix = 1 << lanes_log2
};

// A cell descriptor, one per order position:
//   x: where the cell's row word and column word are -- byte offsets from the
//      lane's first word (bits 0-15, 16-31) in shared memory, or bit shifts
//      (bits 0-5, 8-13) into the packed registers;
//   y: diagonal masks -- 0xffff in bits 0-15 if the cell lies on the main
//      diagonal, 0xffff in bits 16-31 if on the anti-diagonal.
typedef uint2 Cell;

__host__ __device__ inline Cell describe_shared(int i, int j, int n, bool diag,
                                                unsigned B, int col_base) {
  Cell c;
  c.y = ((diag && i == j) ? 0x0000ffffu : 0u) | ((diag && i + j == n - 1) ? 0xffff0000u : 0u);
  c.x = ((uint32_t)i * B * 4u) | (((uint32_t)(col_base + j) * B * 4u) << 16);
  return c;
}

__host__ __device__ inline Cell describe_regs(int i, int j, int n, bool diag, int wr,
                                              int wc) {
  Cell c;
  c.y = ((diag && i == j) ? 0x0000ffffu : 0u) | ((diag && i + j == n - 1) ? 0xffff0000u : 0u);
  c.x = (uint32_t)(i * wr) | ((uint32_t)(j * wc) << 8);
  return c;
}

__device__ __forceinline__ uint32_t &word_at(char *tb, uint32_t off) {
  return *reinterpret_cast<uint32_t *>(tb + off);
}

// Value v -> n-1-v on a one-hot (or two-hot) word.
template <bool VSYM>
__device__ __forceinline__ uint32_t mirror(uint32_t d, int n) {
  return VSYM ? (__brev(d) >> (32 - n)) : 0u;
}

// The row/column/diagonal words of one lane (Section 3: one word per line,
// bit v set when value v is used on it).
//
// REG = false: row and column words in shared memory, word w of thread t at
//   st[w * blockDim + t]; the descriptor gives their byte offsets.
// REG = true: every row word packed into one 64-bit register R and every
//   column word into C; the descriptor gives their shifts.  With vertical
//   symmetry a row field records the value pairs {v, n-1-v} in use (bit
//   min(v, n-1-v)) -- a row takes each pair exactly once -- which halves its
//   width.
// dg holds both diagonal words: the main diagonal in bits 0-15 and the
// anti-diagonal in bits 16-31, so that one AND with a descriptor's masks
// selects the diagonals a cell lies on.
template <bool REG>
struct Words {
  unsigned long long R, C;
  char *tb;
  uint32_t dg;

  // Admissible values of the cell: ALL & ~(row | col | md | ad).
  template <bool VSYM>
  __device__ __forceinline__ uint32_t cands(Cell c, const Geo &g) const {
    uint32_t f;
    if (REG) {
      uint32_t r = (uint32_t)(R >> (c.x & 63u));
      if (VSYM) {
        r &= g.pairmask;
        r |= mirror<true>(r, g.n);
      }
      f = r | (uint32_t)(C >> ((c.x >> 8) & 63u));
    } else {
      f = word_at(tb, c.x & 0xffffu) | word_at(tb, c.x >> 16);
    }
    const uint32_t t = dg & c.y;
    return g.all & ~(f | t | (t >> 16));
  }
  // XOR value bits d (the old value and/or the new one) into the words of the
  // cell; with vertical symmetry the mirror cell (i, n-1-j) takes n-1-v, and
  // the mirror of a main-diagonal cell lies on the anti-diagonal and vice
  // versa.
  template <bool VSYM>
  __device__ __forceinline__ void toggle(Cell c, uint32_t d, const Geo &g) {
    const uint32_t dm = mirror<VSYM>(d, g.n);
    if (REG) {
      const uint32_t rd = VSYM ? ((d ^ dm) & g.pairmask) : d;
      R ^= (unsigned long long)rd << (c.x & 63u);
      C ^= (unsigned long long)d << ((c.x >> 8) & 63u);
    } else {
      word_at(tb, c.x & 0xffffu) ^= d ^ dm;
      word_at(tb, c.x >> 16) ^= d;
    }
    // d < 2^16, so d * 0x10001 puts d in both halves
    if (VSYM) {
      const uint32_t swapped = __byte_perm(c.y, 0u, 0x1032u);
      dg ^= ((d * 0x10001u) & c.y) ^ ((dm * 0x10001u) & swapped);
    } else {
      dg ^= (d * 0x10001u) & c.y;
    }
  }
  // toggle() with vertical symmetry decided at run time by g.vsmask (one
  // step body for lanes of a warp that serve different jobs); shared-memory
  // words only.  With dm = 0 the symmetric update reduces to the plain one.
  __device__ __forceinline__ void toggle_rt(Cell c, uint32_t d, const Geo &g) {
    static_assert(!REG, "runtime symmetry flag: shared-memory words only");
    const uint32_t dm = (__brev(d) >> (32 - g.n)) & g.vsmask;
    word_at(tb, c.x & 0xffffu) ^= d ^ dm;
    word_at(tb, c.x >> 16) ^= d;
    const uint32_t swapped = __byte_perm(c.y, 0u, 0x1032u);
    dg ^= ((d * 0x10001u) & c.y) ^ ((dm * 0x10001u) & swapped);
  }
  __device__ __forceinline__ void clear(int words, unsigned B) {
    dg = 0u;
    if (REG) {
      R = C = 0ull;
    } else {
      for (int w = 0; w < words; ++w) word_at(tb, (uint32_t)w * B * 4u) = 0u;
    }
  }
};

// Per-lane search state.
template <bool REG>
struct Lane {
  Words<REG> w;
  int p;                 // current order position
  uint32_t L;            // untried candidates at p
  uint32_t v;            // value placed at p (one-hot), 0 = none yet
  Cell info;             // cell descriptor of p
  uint32_t splitc;       // nodes met at the split position so far
  uint32_t sub;          // residue class of split nodes this item keeps
  long long prefix;      // prefix (or item) index of the current work
  unsigned long long cnt;    // completions found for the current item
  unsigned long long nodes;  // placements made (node counting variant)
};

// One search iteration.  Returns true when the lane's item is finished.
//
// One iteration of a lane:
//   nv = lowest bit of L        (Algorithm 4: LS = L & -L)
//   d  = v ^ nv                 (take the old value out, put the new one in:
//                                the two XOR steps of Algorithm 4 fused)
//   nv == 0: the loop of this cell is exhausted -> pop to the previous one
//   else:    candidates of the next cell; at the last cell add their
//            popcount (each completes a square, Algorithm 1's innermost
//            loop), an empty set is a dead end, else push and descend.
// Written without data-dependent branches so that the lanes of a warp -- each
// at its own position of its own subtree -- stay converged: every lane
// computes the candidates of the next cell, writes the stack slot of its
// position and reads the one below it, and the outcome only selects which
// registers change.
//
// sbase is the lane's stack base moved back by depth entries, so that the
// entry of position k is sbase[k * B] (k >= depth).
// RTV: vertical symmetry from g.vsmask at run time (VSYM is then ignored).
template <bool REG, bool VSYM, bool NODES, bool SPLIT, bool RTV = false>
__device__ __forceinline__ bool dfs_step(Lane<REG> &s, const Geo &g, const Split &sp,
                                         uint32_t *sbase, const Cell *tbl, unsigned B) {
  const uint32_t nv = s.L & (0u - s.L);
  if constexpr (RTV)
    s.w.toggle_rt(s.info, s.v ^ nv, g);
  else
    s.w.template toggle<VSYM>(s.info, s.v ^ nv, g);
  s.L ^= nv;
  s.v = nv;
  const bool pop = nv == 0u;
  bool skip = false;
  if (SPLIT) {
    const bool at = (s.p == sp.pos) && !pop;
    skip = at && ((s.splitc & ((1u << sp.lanes_log2) - 1u)) != s.sub);
    s.splitc += at ? 1u : 0u;
    if (NODES && !pop && !skip && (s.p >= sp.pos || s.sub == 0u)) s.nodes++;
  } else if (NODES && !pop) {
    s.nodes++;
  }
  const int q = s.p + 1;  // <= last: a lane never stands on the last cell
  const Cell info1 = tbl[q];
  const uint32_t L1 = s.w.template cands<VSYM>(info1, g);
  const bool live = !pop && !skip;
  const bool leaf = q == g.last;
  const unsigned leaves = (live && leaf) ? (unsigned)__popc(L1) : 0u;
  s.cnt += leaves;
  if (NODES) s.nodes += leaves;
  const bool down = live && !leaf && L1 != 0u;
  // entry = untried candidates (bits 0-15) | placed value (bits 16-31);
  // written unconditionally: the slot of the current position is live only
  // once the lane descends below it, which is when this write matters
  sbase[s.p * (int)B] = __byte_perm(s.L, s.v, 0x5410u);
  const int pp = s.p - 1;
  const bool up = pop && pp >= g.depth;
  // read unconditionally (used only when popping; clamped into the stack)
  const int pr = max(pp, g.depth);
  const uint32_t e = sbase[pr * (int)B];
  const Cell infoP = tbl[pr];
  s.p = down ? q : (pop ? pp : s.p);
  s.L = down ? L1 : (up ? (e & 0xffffu) : s.L);
  s.v = down ? 0u : (up ? (e >> 16) : s.v);
  s.info.x = down ? info1.x : (up ? infoP.x : s.info.x);
  s.info.y = down ? info1.y : (up ? infoP.y : s.info.y);
  return pop && !up;
}

// Place the prefix values rec[0..depth-1] into cleared words.  Returns
// false if a value is out of range or breaks a constraint (count 0).
template <bool REG, bool VSYM>
__device__ __forceinline__ bool place_prefix(Words<REG> &w, const Geo &g, const uint8_t *rec,
                                             const Cell *tbl) {
  for (int t = 0; t < g.depth; ++t) {
    const Cell info = tbl[t];
    const uint32_t val = rec[t];
    const uint32_t b = (val < (uint32_t)g.n) ? (1u << val) : 0u;
    if ((w.template cands<VSYM>(info, g) & b) == 0u) return false;
    w.template toggle<VSYM>(info, b, g);
  }
  return true;
}

}  // namespace dls
