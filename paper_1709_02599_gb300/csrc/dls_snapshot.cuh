// dls_snapshot.cuh -- the per-lane search of Algorithm 4 with a stack of
// state snapshots (the batch kernel k_snapshot in dls_kernels.cu).
//
// Algorithm 4 keeps, per cell, the untried candidates L[i][j] and the value
// LS[i][j] placed there; backing out of a cell undoes its placement.  On a
// GPU lane that costs one loop iteration per cell on the way back, and in an
// order where most cells are forced (one candidate: Section 2.3 completes
// lines as soon as they miss one cell) most iterations are such pops.
//
// This search keeps a stack entry only for a cell that still has untried
// candidates after the one being placed, and the entry is the whole line
// state before that placement (row words R, column words C, diagonal words,
// position, untried candidates).  A dead end or a counted leaf then returns
// to the deepest such cell in one step and the following iteration places
// its next candidate.  Every iteration places one value (or two: the fused
// step below also fills a following cell that has a single candidate), so
// iterations <= search nodes without the last cell.
//
// An iteration writes the entry it would push (the state before its
// placement) to the first free slot and reads back the entry a dead end
// would resume -- that one, or the deepest live one -- plus the
// position-table row of the position it ends at (two cells' field shifts and
// diagonal masks, used by the next iteration).  Both accesses happen every
// time (a push keeps the slot, anything else leaves it free), so the step
// has no branch at all and the lanes of a warp never split; and a dead end
// takes its whole state from the one entry read, one select per register.
//
// A position whose cell lies on a line (row, column or diagonal) that has
// all its other cells earlier in the order has at most one candidate, so it
// never makes an entry.  The number of other positions after the prefix
// bounds the stack (dls_kernels.cu computes it per order): entries are made
// at strictly increasing positions along a path.
//
// Only register-packed words (Words<true>: n <= 8, or even n <= 10 with
// vertical symmetry).  An entry is 20 bytes: R and C as one 16-byte word and
// a 32-bit word packing the diagonal words, the position and the untried
// candidates; a lane has cap + 2 entry slots (entry e in slot e + 1; slot 0
// is read when the stack is empty and never holds a live entry; slot cap + 1
// takes the writes a push does not keep once the stack is full).
#pragma once

#include <cstdint>

#include "dls_search.cuh"

namespace dls {

// 32-bit part of an entry.
//   plain / diagonal (n <= 8): main diagonal bits 0-7, anti-diagonal bits
//     16-23 (where the diagonal words keep them), position bits 8-15,
//     untried candidates bits 24-31;
//   vertically symmetric (n <= 10, order <= 64 cells): main diagonal bits
//     0-15 (the anti-diagonal word is its mirror: the mirror of a cell on
//     one diagonal lies on the other), position bits 16-21, untried
//     candidates bits 22-31.
template <bool VSYM>
__device__ __forceinline__ uint32_t snap_pack(uint32_t dg, int p, uint32_t L) {
  if (VSYM) return (dg & 0xffffu) | ((uint32_t)p << 16) | (L << 22);
  return (dg & 0x00ff00ffu) | ((uint32_t)p << 8) | (L << 24);
}

template <bool VSYM>
__device__ __forceinline__ void snap_unpack(uint32_t w, int n, uint32_t &dg, int &p,
                                            uint32_t &L) {
  if (VSYM) {
    const uint32_t md = w & 0xffffu;
    dg = md | (mirror<true>(md, n) << 16);
    p = (int)((w >> 16) & 63u);
    L = w >> 22;
  } else {
    dg = w & 0x00ff00ffu;
    p = (int)((w >> 8) & 0xffu);
    L = w >> 24;
  }
}

// Position table, one row per order position p: sh = shifts of the row and
// column fields of the cells at p and p + 1 (rs_p, cs_p, rs_p+1, cs_p+1),
// dm = their diagonal masks (as Cell::y).  The row of the last position
// repeats its own cell as the next one.
struct SnapTable {
  const uint4 *sh;
  const uint2 *dm;
};

__host__ __device__ inline void snap_row(int n, bool diag, int wr, int wc, int i0, int j0,
                                         int i1, int j1, uint4 &sh, uint2 &dm) {
  sh = make_uint4((uint32_t)(i0 * wr), (uint32_t)(j0 * wc), (uint32_t)(i1 * wr),
                  (uint32_t)(j1 * wc));
  const Cell c0 = describe_regs(i0, j0, n, diag, wr, wc);
  const Cell c1 = describe_regs(i1, j1, n, diag, wr, wc);
  dm = make_uint2(c0.y, c1.y);
}

// Per-lane state.
struct SnapLane {
  Words<true> w;             // line words of the current path
  int p;                     // position whose candidates L are being tried
  uint32_t L;                // untried candidates at p
  uint4 sh;                  // table row of p
  uint2 dm;
  int sp;                    // entries [bot, sp) are live; entries below
  int bot;                   // bot were given to other lanes
  long long prefix;          // prefix index of the current work
  unsigned long long cnt;    // completions found for the current work
  unsigned long long nodes;  // placements made (node counting variant)
};

// Stack of one lane: entry e at sa[e * B] (line words) and sw[e * B]
// (packed word), thread-minor so that a warp's accesses are conflict-free
// whatever entries its lanes are at.
struct SnapStack {
  uint4 *sa;
  uint32_t *sw;
  int cap;                   // entries per lane
};

// Admissible values of a cell (fields at shifts rs, cs, diagonal mask m).
// DG = false: no cell searched lies on a diagonal, the diagonal words are
// left out.
template <bool VSYM, bool DG>
__device__ __forceinline__ uint32_t snap_cands(const Words<true> &w, uint32_t rs, uint32_t cs,
                                               uint32_t m, const Geo &g) {
  uint32_t r = (uint32_t)(w.R >> rs);
  if (VSYM) {
    r &= g.pairmask;
    r |= mirror<true>(r, g.n);
  }
  const uint32_t f = r | (uint32_t)(w.C >> cs);
  if (!DG) return g.all & ~f;
  const uint32_t t = w.dg & m;
  return g.all & ~(f | t | (t >> 16));
}

// Place value bits d at a cell (Words::toggle with explicit shifts).
template <bool VSYM, bool DG>
__device__ __forceinline__ void snap_place(Words<true> &w, uint32_t rs, uint32_t cs, uint32_t m,
                                           uint32_t d, const Geo &g) {
  const uint32_t dm = mirror<VSYM>(d, g.n);
  const uint32_t rd = VSYM ? ((d ^ dm) & g.pairmask) : d;
  w.R ^= (unsigned long long)rd << rs;
  w.C ^= (unsigned long long)d << cs;
  if (!DG) return;
  if (VSYM) {
    const uint32_t swapped = __byte_perm(m, 0u, 0x1032u);
    w.dg ^= ((d * 0x10001u) & m) ^ ((dm * 0x10001u) & swapped);
  } else {
    w.dg ^= (d * 0x10001u) & m;
  }
}

// Shared-memory accesses under a predicate.  On the GPU they are single
// predicated instructions (a C++ `if` around them would become a branch,
// and the lanes of a warp would split); a lane whose predicate is off makes
// no access and its registers keep their values.
#ifdef __CUDA_ARCH__
// (the base's shared-window address is loop-invariant and computed once)
__device__ __forceinline__ uint32_t smem_addr(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void st_shared_if(bool c, uint4 *base, int k, uint4 v) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n"
      " @q st.shared.v4.u32 [%1], {%2, %3, %4, %5};\n}\n" ::"r"((uint32_t)c),
      "r"(smem_addr(base) + (uint32_t)k * 16u), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
      : "memory");
}
__device__ __forceinline__ void st_shared_if(bool c, uint32_t *base, int k, uint32_t v) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.u32 q, %0, 0;\n"
      " @q st.shared.u32 [%1], %2;\n}\n" ::"r"((uint32_t)c),
      "r"(smem_addr(base) + (uint32_t)k * 4u), "r"(v)
      : "memory");
}
__device__ __forceinline__ void ld_shared_if(bool c, const uint4 *base, int k, uint4 &v) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.u32 q, %4, 0;\n"
      " @q ld.shared.v4.u32 {%0, %1, %2, %3}, [%5];\n}\n"
      : "+r"(v.x), "+r"(v.y), "+r"(v.z), "+r"(v.w)
      : "r"((uint32_t)c), "r"(smem_addr(base) + (uint32_t)k * 16u)
      : "memory");
}
__device__ __forceinline__ void ld_shared_if(bool c, const uint32_t *base, int k, uint32_t &v) {
  asm volatile(
      "{\n .reg .pred q;\n setp.ne.u32 q, %1, 0;\n"
      " @q ld.shared.u32 %0, [%2];\n}\n"
      : "+r"(v)
      : "r"((uint32_t)c), "r"(smem_addr(base) + (uint32_t)k * 4u)
      : "memory");
}
#else
inline void st_shared_if(bool c, uint4 *base, int k, uint4 v) {
  if (c) base[k] = v;
}
inline void st_shared_if(bool c, uint32_t *base, int k, uint32_t v) {
  if (c) base[k] = v;
}
inline void ld_shared_if(bool c, const uint4 *base, int k, uint4 &v) {
  if (c) v = base[k];
}
inline void ld_shared_if(bool c, const uint32_t *base, int k, uint32_t &v) {
  if (c) v = base[k];
}
#endif

// One search iteration.  Returns true when the lane's work is finished.
//   nv = lowest untried candidate at p (Algorithm 4's L & -L), removed from L
//   place nv; candidates of the next cell: at the last cell their popcount
//   is added (each completes a square), none is a dead end
//   no dead end: if candidates remain at p, the state before placing nv is
//   pushed as an entry; descend
//   dead end or leaf: resume at p itself if candidates remain there (that
//   state is the entry just written, read back), else at the deepest entry.
// ovf is set (and the stack index held at cap, so every access stays in the
// lane's cap + 2 slots) if a lane ever needs more entries than cap -- which
// the bound on cap excludes, and which a capped stack turns into a deferred
// prefix.
// LA (lookahead, Section 2.4.2; only without diagonal words and without
// vertical symmetry): the cell after the next one must still have a
// candidate, or the placement is a dead end already -- placing the next cell
// only removes candidates.  Its field shifts are in dm (the diagonal masks
// are not needed there).
// FU (fused forced placement; no diagonal words, dm as for LA; with or
// without vertical symmetry): when the next cell is left with exactly one
// candidate and is not the last cell, that value is placed in the same
// iteration and the lane moves two cells on.
// It is the move the next iteration would make -- a single candidate makes
// no entry -- so the counts, the nodes and the entries are those of the
// plain step; only the iterations are fewer.  On the order-8 split after
// row 1, the cell after a placement has one candidate after 54 % of the
// iterations, and fusing one such cell cuts the iterations by 34 %.
template <bool VSYM, bool NODES, bool DG, bool LA = false, bool FU = false>
__device__ __forceinline__ bool snap_step(SnapLane &s, const Geo &g, const SnapStack &st,
                                          const SnapTable &tb, unsigned B, uint32_t &ovf) {
  static_assert(!LA || (!DG && !VSYM), "lookahead: no diagonal words, no symmetry");
  static_assert(!FU || (!DG && !LA), "fused step: no diagonal words, no lookahead");
  const uint32_t nv = s.L & (0u - s.L);
  const uint32_t Lr = s.L ^ nv;
  const bool keep = Lr != 0u;
  const bool has = s.sp > s.bot;
  int q = s.p + 1;  // <= last: a lane never stands on the last cell
  const unsigned long long R0 = s.w.R, C0 = s.w.C;
  const uint32_t dg0 = s.w.dg;
  snap_place<VSYM, DG>(s.w, s.sh.x, s.sh.y, s.dm.x, nv, g);
  if (NODES) s.nodes++;
  uint32_t L1 = snap_cands<VSYM, DG>(s.w, s.sh.z, s.sh.w, s.dm.y, g);
  if (FU) {
    // one candidate at q (q not the last cell): place it too (placing 0
    // changes nothing); L1 becomes the candidates of the cell after q
    const bool f = q != g.last && L1 != 0u && (L1 & (L1 - 1u)) == 0u;
    snap_place<VSYM, false>(s.w, s.sh.z, s.sh.w, 0u, f ? L1 : 0u, g);
    const uint32_t L2 = snap_cands<VSYM, false>(s.w, s.dm.x, s.dm.y, 0u, g);
    if (NODES) s.nodes += f ? 1u : 0u;
    L1 = f ? L2 : L1;
    q = f ? q + 1 : q;
  }
  const bool leaf = q == g.last;
  const unsigned leaves = leaf ? (unsigned)__popc(L1) : 0u;
  s.cnt += leaves;
  if (NODES) s.nodes += leaves;
  bool dead = leaf || L1 == 0u;
  if (LA) dead = dead || snap_cands<false, false>(s.w, s.dm.x, s.dm.y, 0u, g) == 0u;
  // entry e lives in slot e + 1 (slot 0 is never live, slot cap + 1 is
  // spare): the state before placing nv is written to the first free slot
  // every iteration; a push keeps it
  st.sa[(s.sp + 1) * (int)B] = make_uint4((uint32_t)R0, (uint32_t)(R0 >> 32), (uint32_t)C0,
                                          (uint32_t)(C0 >> 32));
  st.sw[(s.sp + 1) * (int)B] = snap_pack<VSYM>(DG ? dg0 : 0u, s.p, Lr);
  // a dead end resumes the entry just written if candidates remain at p,
  // else the deepest live one (read back after the write; used only on a
  // dead end).  A lane that finishes -- no candidate left, no live entry --
  // reads the entry just written as well, so that every position read back
  // is a valid one (it indexes the position table below).
  const int rd = (keep || s.sp <= s.bot) ? s.sp + 1 : s.sp;
  const uint4 ea = st.sa[rd * (int)B];
  const uint32_t ew = st.sw[rd * (int)B];
  const bool push = keep && !dead;
  const bool pop = dead && !keep && has;
  ovf |= (push && s.sp >= st.cap) ? 1u : 0u;
  uint32_t edg, eL;
  int ep;
  snap_unpack<VSYM>(ew, g.n, edg, ep, eL);
  const unsigned long long eR = ((unsigned long long)ea.y << 32) | ea.x;
  const unsigned long long eC = ((unsigned long long)ea.w << 32) | ea.z;
  s.w.R = dead ? eR : s.w.R;
  s.w.C = dead ? eC : s.w.C;
  if (DG) s.w.dg = dead ? edg : s.w.dg;
  s.L = dead ? eL : L1;
  s.p = dead ? ep : q;
  s.sp = min(s.sp + (push ? 1 : 0) - (pop ? 1 : 0), st.cap);
  // table row of the new position, for the next iteration
  s.sh = tb.sh[s.p];
  s.dm = tb.dm[s.p];
  return dead && !keep && !has;
}

// ------------------------------------------------------------ byte words --
//
// Orders n <= 8 without vertical symmetry keep every row word and every
// column word in one byte: rows 0-3 are the bytes of R0 and rows 4-7 those
// of R1, columns 0-3 of C0 and 4-7 of C1.  A cell's admissible values are
// then two byte permutes (one per word pair, picking the cell's row byte and
// column byte) and one three-input logic operation; a value is placed with
// four multiply-adds, one per word, by the multipliers 2^(8k) or 0 of the
// cell's row and column (the bit placed is always clear, so adding it sets
// it).  The multiply-adds run on the FMA pipe, leaving the integer ALU --
// the unit the search is bound by -- the rest of the step.  The stack and its
// entries are those of the search above: R0, R1, C0, C1 as one 16-byte word,
// and the packed word (diagonal words, position, untried candidates).

// Position table row for order position p (48 bytes):
//   a: multipliers that place a value at p (row into R0 / R1, column into
//      C0 / C1);
//   b: the same for p + 1 (the fused step), or, with diagonal words, the
//      diagonal masks of p and of p + 1 (as Cell::y) in b.x and b.y;
//   c: byte selectors of the row and the column of p + 1, then of p + 2
//      (the lookahead and the fused step read p + 2).
// Positions past the last repeat the last cell; no step uses them.
struct BRow {
  uint4 a, b, c;
};

__host__ __device__ inline uint32_t byte_mult(int k, int half) {
  return (k >> 2) == half ? (1u << (8 * (k & 3))) : 0u;
}

__host__ __device__ inline BRow brow_make(int n, bool diag, bool dgw, const uint8_t *ci,
                                          const uint8_t *cj, int p, int len) {
  const int q = p + 1 < len ? p + 1 : len - 1;
  const int q2 = p + 2 < len ? p + 2 : len - 1;
  BRow r;
  r.a = make_uint4(byte_mult(ci[p], 0), byte_mult(ci[p], 1), byte_mult(cj[p], 0),
                   byte_mult(cj[p], 1));
  if (dgw) {
    const Cell c0 = describe_regs(ci[p], cj[p], n, diag, 8, 8);
    const Cell c1 = describe_regs(ci[q], cj[q], n, diag, 8, 8);
    r.b = make_uint4(c0.y, c1.y, 0u, 0u);
  } else {
    r.b = make_uint4(byte_mult(ci[q], 0), byte_mult(ci[q], 1), byte_mult(cj[q], 0),
                     byte_mult(cj[q], 1));
  }
  r.c = make_uint4(ci[q], cj[q], ci[q2], cj[q2]);
  return r;
}

// Per-lane state of the byte-word search.
struct BLane {
  uint32_t R0, R1, C0, C1;   // row and column bytes of the current path
  uint32_t dg;               // diagonal words (as Words::dg)
  int p;                     // position whose candidates L are being tried
  uint32_t L;                // untried candidates at p
  uint4 a, b, c;             // table row of p
  int sp, bot;               // live entries [bot, sp)
  long long prefix;
  unsigned long long cnt;
  unsigned long long nodes;
};

// Admissible values at the cell whose byte selectors are (sr, sc).
__device__ __forceinline__ uint32_t bcands(uint32_t R0, uint32_t R1, uint32_t C0, uint32_t C1,
                                           uint32_t sr, uint32_t sc, uint32_t all) {
  return all & ~(__byte_perm(R0, R1, sr) | __byte_perm(C0, C1, sc));
}

// One search iteration of the byte-word search: the moves of snap_step (see
// there), with the stack and table traffic cut to what each lane needs.
// Only a push writes its entry (the state before placing nv); only a move
// back to an older cell reads one, loaded over the registers that hold the
// state before the placement -- so a dead end with candidates left at p
// resumes from those registers, and one select per register picks the new
// state; only a move to another position reads a table row.  Returns true
// when the lane's work is finished (then it stays on p with no candidate).
// (The same predicated traffic in snap_step, with field shifts and vertical
// symmetry, measured 2 % slower than its unconditional write and read.)
template <bool NODES, bool DG, bool LA = false, bool FU = false>
__device__ __forceinline__ bool bsnap_step(BLane &s, const Geo &g, const SnapStack &st,
                                           const BRow *tb, unsigned B, uint32_t &ovf) {
  static_assert(!LA || !DG, "lookahead: no diagonal words");
  static_assert(!FU || (!DG && !LA), "fused step: no diagonal words, no lookahead");
  const uint32_t nv = s.L & (0u - s.L);
  const uint32_t Lr = s.L ^ nv;
  const bool keep = Lr != 0u;
  const bool has = s.sp > s.bot;
  int q = s.p + 1;  // <= last: a lane never stands on the last cell
  const uint32_t dg0 = s.dg;
  uint4 e = make_uint4(s.R0, s.R1, s.C0, s.C1);  // the state before placing nv
  uint32_t r0 = nv * s.a.x + e.x, r1 = nv * s.a.y + e.y;
  uint32_t c0 = nv * s.a.z + e.z, c1 = nv * s.a.w + e.w;
  uint32_t L1 = bcands(r0, r1, c0, c1, s.c.x, s.c.y, g.all);
  uint32_t dg = dg0;
  if (DG) {
    dg += (nv * 0x10001u) & s.b.x;
    const uint32_t t = dg & s.b.y;
    L1 &= ~(t | (t >> 16));
  }
  if (NODES) s.nodes++;
  if (FU) {
    // one candidate at q (q not the last cell): place it too
    const bool f = q != g.last && L1 != 0u && (L1 & (L1 - 1u)) == 0u;
    const uint32_t d2 = f ? L1 : 0u;
    r0 = d2 * s.b.x + r0;
    r1 = d2 * s.b.y + r1;
    c0 = d2 * s.b.z + c0;
    c1 = d2 * s.b.w + c1;
    const uint32_t L2 = bcands(r0, r1, c0, c1, s.c.z, s.c.w, g.all);
    if (NODES) s.nodes += f ? 1u : 0u;
    L1 = f ? L2 : L1;
    q = f ? q + 1 : q;
  }
  const bool leaf = q == g.last;
  const unsigned leaves = leaf ? (unsigned)__popc(L1) : 0u;
  s.cnt += leaves;
  if (NODES) s.nodes += leaves;
  bool dead = leaf || L1 == 0u;
  if (LA) dead = dead || bcands(r0, r1, c0, c1, s.c.z, s.c.w, g.all) == 0u;
  const bool push = keep && !dead;
  const bool pop = dead && !keep && has;
  ovf |= (push && s.sp >= st.cap) ? 1u : 0u;
  uint32_t ew = snap_pack<false>(DG ? dg0 : 0u, s.p, Lr);
  // entry e lives in slot e + 1; a full stack pushes into the spare slot
  // cap + 1, which the index clamp below never makes live
  st_shared_if(push, st.sa, (s.sp + 1) * (int)B, e);
  st_shared_if(push, st.sw, (s.sp + 1) * (int)B, ew);
  ld_shared_if(pop, st.sa, s.sp * (int)B, e);
  ld_shared_if(pop, st.sw, s.sp * (int)B, ew);
  uint32_t edg, eL;
  int ep;
  snap_unpack<false>(ew, g.n, edg, ep, eL);
  s.R0 = dead ? e.x : r0;
  s.R1 = dead ? e.y : r1;
  s.C0 = dead ? e.z : c0;
  s.C1 = dead ? e.w : c1;
  if (DG) s.dg = dead ? edg : dg;
  s.L = dead ? eL : L1;
  const int np = dead ? ep : q;
  const bool moved = np != s.p;
  s.p = np;
  s.sp = min(s.sp + (push ? 1 : 0) - (pop ? 1 : 0), st.cap);
  // table row of the new position, for the next iteration
  const uint4 *rows = reinterpret_cast<const uint4 *>(tb);
  ld_shared_if(moved, rows, 3 * s.p, s.a);
  ld_shared_if(moved, rows, 3 * s.p + 1, s.b);
  ld_shared_if(moved, rows, 3 * s.p + 2, s.c);
  return dead && !keep && !has;
}

// ------------------------------------------------------------ wide words --
//
// Order 9 without vertical symmetry: the values 0-7 of a line keep their
// byte (as with byte words) and the value 8 a bit of its own.
//   row bytes:    the rows that have cells after the prefix get slots 0-7,
//                 slot k is byte k of {R1:R0} (at most 8 such rows);
//   column bytes: slot s of a column is byte s of C0 (s < 4), byte s - 4 of
//                 C1 (4 <= s < 7) or byte s - 7 of C2 (s = 7, 8); byte 3 of
//                 C1 and bytes 2-3 of C2 stay 0, so two byte permutes reach
//                 any column (the other one picks a zero byte);
//   value 8:      V8 bit i = row i holds 8, bit 16 + j = column j holds 8.
// A cell's admissible values: ~(row byte | column bytes) for 0-7 in one
// three-input logic op (the second permute fills bytes 1-3 with ones so the
// result keeps only byte 0), and bit 8 set when V8 has neither the cell's
// row bit nor its column bit (mask m8).  A value is placed by multiply-adds:
// its low byte into R0, R1, C0, C1, C2 by the cell's multipliers (2^(8k) or
// 0), its bit 8 into V8 by m8.  An entry is 32 bytes: R0, R1, C0, C1, then
// C2, V8, the diagonal words and (position | untried candidates << 16).

// Position table row for order position p (80 bytes):
//   a  = byte multipliers of p (R0, R1, C0, C1);
//   a2 = (C2 multiplier of p, m8 of p, diagonal mask of p, and the diagonal
//        mask of p + 1 with diagonal words, else the C2 multiplier of p + 1);
//   b  = byte multipliers of p + 1 (the fused step);
//   c  = (row selector, column selectors A and B, m8) of p + 1;
//   c2 = the same for p + 2.
struct WRow {
  uint4 a, a2, b, c, c2;
};

// Slot maps of an order after its prefix: rslot[i] (-1: row i has no cell
// after the prefix), cslot[j].  Returns false if more than 8 rows do.
__host__ __device__ inline bool wide_slots(int n, const uint8_t *ci, const uint8_t *cj, int len,
                                           int depth, int *rslot, int *cslot) {
  for (int k = 0; k < n; ++k) rslot[k] = cslot[k] = -1;
  int nr = 0, nc = 0;
  for (int t = depth; t < len; ++t) {
    if (rslot[ci[t]] < 0) rslot[ci[t]] = nr++;
    if (cslot[cj[t]] < 0) cslot[cj[t]] = nc++;
  }
  return nr <= 8 && nc <= 9;
}

__host__ __device__ inline uint32_t wide_row_sel(int rs) { return rs < 0 ? 0u : (uint32_t)rs; }
__host__ __device__ inline uint32_t wide_col_sel_a(int cs) {
  return (cs >= 0 && cs < 7) ? (uint32_t)cs : 7u;
}
__host__ __device__ inline uint32_t wide_col_sel_b(int cs) {
  return (cs >= 7) ? (0x7650u | (uint32_t)(cs - 7)) : 0x7654u;
}
__host__ __device__ inline uint32_t wide_col_mult(int cs, int word) {
  if (cs < 0) return 0u;
  const int w = cs < 4 ? 0 : (cs < 7 ? 1 : 2);
  const int b = cs < 4 ? cs : (cs < 7 ? cs - 4 : cs - 7);
  return w == word ? (1u << (8 * b)) : 0u;
}

__host__ __device__ inline WRow wrow_make(int n, bool diag, bool dgw, const uint8_t *ci,
                                          const uint8_t *cj, int p, int len, const int *rslot,
                                          const int *cslot) {
  const int q = p + 1 < len ? p + 1 : len - 1;
  const int q2 = p + 2 < len ? p + 2 : len - 1;
  auto m8 = [&](int t) { return (1u << ci[t]) | (1u << (16 + cj[t])); };
  auto sel = [&](int t) {
    return make_uint4(wide_row_sel(rslot[ci[t]]), wide_col_sel_a(cslot[cj[t]]),
                      wide_col_sel_b(cslot[cj[t]]), m8(t));
  };
  auto bytes = [&](int t) {
    const int rs = rslot[ci[t]], cs = cslot[cj[t]];
    return make_uint4(rs >= 0 ? byte_mult(rs, 0) : 0u, rs >= 0 ? byte_mult(rs, 1) : 0u,
                      wide_col_mult(cs, 0), wide_col_mult(cs, 1));
  };
  WRow r;
  r.a = bytes(p);
  const Cell d0 = describe_regs(ci[p], cj[p], n, diag, 8, 8);
  const Cell d1 = describe_regs(ci[q], cj[q], n, diag, 8, 8);
  r.a2 = make_uint4(wide_col_mult(cslot[cj[p]], 2), m8(p), dgw ? d0.y : 0u,
                    dgw ? d1.y : wide_col_mult(cslot[cj[q]], 2));
  r.b = bytes(q);
  r.c = sel(q);
  r.c2 = sel(q2);
  return r;
}

// Per-lane state of the wide-word search.
struct WLane {
  uint32_t R0, R1, C0, C1, C2, V8;
  uint32_t dg;
  int p;
  uint32_t L;
  WRow r;                    // table row of p
  int sp, bot;
  long long prefix;
  unsigned long long cnt;
  unsigned long long nodes;
};

// Admissible values at a cell with selectors / mask c = (row, column A,
// column B, m8).
__device__ __forceinline__ uint32_t wcands(uint32_t R0, uint32_t R1, uint32_t C0, uint32_t C1,
                                           uint32_t C2, uint32_t V8, uint4 c) {
  const uint32_t lo = ~(__byte_perm(R0, R1, c.x) | __byte_perm(C0, C1, c.y) |
                        __byte_perm(C2, 0xffffff00u, c.z));
  return lo | ((V8 & c.w) == 0u ? 0x100u : 0u);
}

// The wide-word search iteration: the moves of snap_step / bsnap_step, with
// the same predicated stack and table traffic as bsnap_step.
template <bool NODES, bool DG, bool LA = false, bool FU = false>
__device__ __forceinline__ bool wsnap_step(WLane &s, const Geo &g, const SnapStack &st,
                                           const WRow *tb, unsigned B, uint32_t &ovf) {
  static_assert(!LA || !DG, "lookahead: no diagonal words");
  static_assert(!FU || (!DG && !LA), "fused step: no diagonal words, no lookahead");
  const uint32_t nv = s.L & (0u - s.L);
  const uint32_t Lr = s.L ^ nv;
  const bool keep = Lr != 0u;
  const bool has = s.sp > s.bot;
  int q = s.p + 1;  // <= last: a lane never stands on the last cell
  uint4 e = make_uint4(s.R0, s.R1, s.C0, s.C1);  // the state before placing nv
  uint4 e2 = make_uint4(s.C2, s.V8, s.dg, (uint32_t)s.p | (Lr << 16));
  const uint32_t lo = nv & 0xffu, hi = nv >> 8;
  uint32_t r0 = lo * s.r.a.x + e.x, r1 = lo * s.r.a.y + e.y;
  uint32_t c0 = lo * s.r.a.z + e.z, c1 = lo * s.r.a.w + e.w;
  uint32_t c2 = lo * s.r.a2.x + e2.x, v8 = hi * s.r.a2.y + e2.y;
  uint32_t L1 = wcands(r0, r1, c0, c1, c2, v8, s.r.c);  // bits 0-8 only
  uint32_t dg = e2.z;
  if (DG) {
    dg += (nv * 0x10001u) & s.r.a2.z;
    const uint32_t t = dg & s.r.a2.w;
    L1 &= ~(t | (t >> 16));
  }
  if (NODES) s.nodes++;
  if (FU) {
    const bool f = q != g.last && L1 != 0u && (L1 & (L1 - 1u)) == 0u;
    const uint32_t d2 = f ? L1 : 0u;
    const uint32_t lo2 = d2 & 0xffu, hi2 = d2 >> 8;
    r0 = lo2 * s.r.b.x + r0;
    r1 = lo2 * s.r.b.y + r1;
    c0 = lo2 * s.r.b.z + c0;
    c1 = lo2 * s.r.b.w + c1;
    c2 = lo2 * s.r.a2.w + c2;
    v8 = hi2 * s.r.c.w + v8;
    const uint32_t L2 = wcands(r0, r1, c0, c1, c2, v8, s.r.c2);
    if (NODES) s.nodes += f ? 1u : 0u;
    L1 = f ? L2 : L1;
    q = f ? q + 1 : q;
  }
  const bool leaf = q == g.last;
  const unsigned leaves = leaf ? (unsigned)__popc(L1) : 0u;
  s.cnt += leaves;
  if (NODES) s.nodes += leaves;
  bool dead = leaf || L1 == 0u;
  if (LA) dead = dead || wcands(r0, r1, c0, c1, c2, v8, s.r.c2) == 0u;
  const bool push = keep && !dead;
  const bool pop = dead && !keep && has;
  ovf |= (push && s.sp >= st.cap) ? 1u : 0u;
  // entries: R0, R1, C0, C1 in sa; C2, V8, diagonal words, packed in sb
  // (the stack's second array of 16-byte slots)
  uint4 *sb = reinterpret_cast<uint4 *>(st.sw);
  st_shared_if(push, st.sa, (s.sp + 1) * (int)B, e);
  st_shared_if(push, sb, (s.sp + 1) * (int)B, e2);
  ld_shared_if(pop, st.sa, s.sp * (int)B, e);
  ld_shared_if(pop, sb, s.sp * (int)B, e2);
  s.R0 = dead ? e.x : r0;
  s.R1 = dead ? e.y : r1;
  s.C0 = dead ? e.z : c0;
  s.C1 = dead ? e.w : c1;
  s.C2 = dead ? e2.x : c2;
  s.V8 = dead ? e2.y : v8;
  if (DG) s.dg = dead ? e2.z : dg;
  s.L = dead ? (e2.w >> 16) : L1;
  const int np = dead ? (int)(e2.w & 0xffffu) : q;
  const bool moved = np != s.p;
  s.p = np;
  s.sp = min(s.sp + (push ? 1 : 0) - (pop ? 1 : 0), st.cap);
  const uint4 *rows = reinterpret_cast<const uint4 *>(tb);
  ld_shared_if(moved, rows, 5 * s.p, s.r.a);
  ld_shared_if(moved, rows, 5 * s.p + 1, s.r.a2);
  ld_shared_if(moved, rows, 5 * s.p + 2, s.r.b);
  ld_shared_if(moved, rows, 5 * s.p + 3, s.r.c);
  ld_shared_if(moved, rows, 5 * s.p + 4, s.r.c2);
  return dead && !keep && !has;
}

}  // namespace dls
