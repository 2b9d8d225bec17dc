// step_check.cpp -- runs the kernels' per-lane search steps (bsnap_step and snap_step of
// dls_snapshot.cuh, dfs_step of dls_search.cuh, compiled for the host
// through shim.h) on one lane per work item, with no warp and no donation,
// for tests/test_host_step.py.
//
//   step_check n flags mode order.bin prefixes.bin depth cap [lanes_log2 split_pos]
//
// mode, the snapshot step (the byte-word step without vertical symmetry,
// the field-shift step with it): 0 = plain (diagonal words when a cell
// after the prefix lies on a diagonal), 1 = lookahead, 2 = fused step (1 and
// 2 only without diagonal words and without vertical symmetry; exit 2
// otherwise).
// mode, the per-position step (one stack entry per position): 10 = words in
// registers (exit 2 where they do not fit), 11 = words in the shared-memory
// layout, 12 = as 11 with vertical symmetry taken at run time (the serving
// kernel's step).  lanes_log2 / split_pos (per-position step only): each
// prefix is split into 2^lanes_log2 work items at order position split_pos,
// run one after the other and summed.
// order.bin: the fill order as (i, j) byte pairs; prefixes.bin: depth value
// bytes per prefix.  cap: stack entries per lane (snapshot step).  The
// tables are built as the kernels' setup builds them.  Every stack slot
// starts as 0xff bytes, so a read of a slot never written shows up.
//
// stdout: "count nodes" per prefix.  stderr: one line
// "iters I maxsp M overflow O badpos B".  Exit 3 when a step leaves the lane
// at a position outside the order or a stack index outside its stack.
#include "shim.h"

#include <cstdio>
#include <cstdlib>
#include <vector>

#include "dls_snapshot.cuh"

using namespace dls;

namespace {

struct Run {
  unsigned long long iters = 0;
  int maxsp = 0;
  uint32_t ovf = 0u;
  int badpos = 0;
};

// The byte-word step (orders n <= 8 without vertical symmetry).
template <bool DG, bool LA, bool FU>
bool bsearch(BLane &s, const Geo &g, const SnapStack &st, const BRow *tb, int len, Run &run) {
  for (;;) {
    ++run.iters;
    const bool fin = bsnap_step<true, DG, LA, FU>(s, g, st, tb, 1u, run.ovf);
    if (s.p < 0 || s.p >= len || s.sp < 0 || s.sp > st.cap) {
      ++run.badpos;
      return false;
    }
    run.maxsp = std::max(run.maxsp, s.sp);
    if (fin) return true;
  }
}

// The wide-word step (order 9 without vertical symmetry).
template <bool DG, bool LA, bool FU>
bool wsearch(WLane &s, const Geo &g, const SnapStack &st, const WRow *tb, int len, Run &run) {
  for (;;) {
    ++run.iters;
    const bool fin = wsnap_step<true, DG, LA, FU>(s, g, st, tb, 1u, run.ovf);
    if (s.p < 0 || s.p >= len || s.sp < 0 || s.sp > st.cap) {
      ++run.badpos;
      return false;
    }
    run.maxsp = std::max(run.maxsp, s.sp);
    if (fin) return true;
  }
}

// Wide-word runs: each prefix placed with plain line masks, written into the
// slots as the kernel's load does, then searched.
int run_wide(int n, uint32_t flags, int mode, const std::vector<uint8_t> &ob,
             const std::vector<uint8_t> &pre, int depth, int cap) {
  const bool diag = (flags & 1u) != 0;
  const int len = (int)ob.size() / 2;
  std::vector<uint8_t> ci(len), cj(len);
  for (int t = 0; t < len; ++t) {
    ci[t] = ob[2 * t];
    cj[t] = ob[2 * t + 1];
  }
  int rs[DLS_MAX_N], cs[DLS_MAX_N];
  if (!wide_slots(n, ci.data(), cj.data(), len, depth, rs, cs)) return 2;
  bool dg = false;
  for (int t = depth; t < len; ++t)
    if (diag && (ci[t] == cj[t] || ci[t] + cj[t] == n - 1)) dg = true;
  if ((mode == 1 || mode == 2) && dg) return 2;
  std::vector<WRow> rows(len);
  for (int t = 0; t < len; ++t)
    rows[t] = wrow_make(n, diag, dg, ci.data(), cj.data(), t, len, rs, cs);
  Geo g;
  g.n = n;
  g.all = (1u << n) - 1u;
  g.pairmask = 0u;
  g.depth = depth;
  g.last = len - 1;
  g.vsmask = 0u;
  std::vector<uint4> sa((size_t)cap + 2, make_uint4(~0u, ~0u, ~0u, ~0u));
  std::vector<uint4> sb((size_t)cap + 2, make_uint4(~0u, ~0u, ~0u, ~0u));
  const SnapStack st{sa.data(), reinterpret_cast<uint32_t *>(sb.data()), cap};
  const long long P = depth ? (long long)pre.size() / depth : 1;
  Run run;
  for (long long k = 0; k < P; ++k) {
    const uint8_t *rec = pre.data() + (size_t)k * (size_t)depth;
    uint32_t rw[DLS_MAX_N] = {0}, cl[DLS_MAX_N] = {0}, md = 0u, ad = 0u;
    bool ok = true;
    for (int t = 0; t < depth && ok; ++t) {
      const int i = ci[t], j = cj[t];
      const uint32_t b = rec[t] < n ? (1u << rec[t]) : 0u;
      const bool om = diag && i == j, oa = diag && i + j == n - 1;
      ok = b != 0u && ((rw[i] | cl[j] | (om ? md : 0u) | (oa ? ad : 0u)) & b) == 0u;
      rw[i] |= b;
      cl[j] |= b;
      md |= om ? b : 0u;
      ad |= oa ? b : 0u;
    }
    unsigned long long cnt = 0, nodes = 0;
    if (ok && depth == len) {
      cnt = 1;
    } else if (ok) {
      const int i = ci[depth], j = cj[depth];
      const bool om = diag && i == j, oa = diag && i + j == n - 1;
      const uint32_t L = g.all & ~(rw[i] | cl[j] | (om ? md : 0u) | (oa ? ad : 0u));
      if (depth == g.last) {
        cnt = nodes = (unsigned)__popc(L);
      } else if (L != 0u) {
        WLane w{};
        for (int x = 0; x < n; ++x) {
          if (rs[x] >= 0) {
            w.R0 |= (rw[x] & 0xffu) * byte_mult(rs[x], 0);
            w.R1 |= (rw[x] & 0xffu) * byte_mult(rs[x], 1);
          }
          if (cs[x] >= 0) {
            w.C0 |= (cl[x] & 0xffu) * wide_col_mult(cs[x], 0);
            w.C1 |= (cl[x] & 0xffu) * wide_col_mult(cs[x], 1);
            w.C2 |= (cl[x] & 0xffu) * wide_col_mult(cs[x], 2);
          }
          w.V8 |= ((rw[x] >> 8) & 1u) << x;
          w.V8 |= ((cl[x] >> 8) & 1u) << (16 + x);
        }
        w.dg = md | (ad << 16);
        w.p = depth;
        w.L = L;
        w.r = rows[depth];
        bool done;
        if (mode == 1)
          done = wsearch<false, true, false>(w, g, st, rows.data(), len, run);
        else if (mode == 2)
          done = wsearch<false, false, true>(w, g, st, rows.data(), len, run);
        else
          done = dg ? wsearch<true, false, false>(w, g, st, rows.data(), len, run)
                    : wsearch<false, false, false>(w, g, st, rows.data(), len, run);
        if (!done) {
          std::fprintf(stderr, "iters %llu maxsp %d overflow %u badpos %d\n", run.iters,
                       run.maxsp, run.ovf, run.badpos);
          return 3;
        }
        cnt = w.cnt;
        nodes = w.nodes;
      }
    }
    std::printf("%llu %llu\n", cnt, nodes);
  }
  std::fprintf(stderr, "iters %llu maxsp %d overflow %u badpos %d\n", run.iters, run.maxsp,
               run.ovf, run.badpos);
  return 0;
}

template <bool VSYM, bool DG, bool LA, bool FU>
bool search(SnapLane &s, const Geo &g, const SnapStack &st, const SnapTable &tb, int len,
            Run &run) {
  for (;;) {
    ++run.iters;
    const bool fin = snap_step<VSYM, true, DG, LA, FU>(s, g, st, tb, 1u, run.ovf);
    if (s.p < 0 || s.p >= len || s.sp < 0 || s.sp > st.cap) {
      ++run.badpos;
      return false;
    }
    run.maxsp = std::max(run.maxsp, s.sp);
    if (fin) return true;
  }
}

// The per-position step over one work item (the kernels' load_item, then
// dfs_step until the item is done).  words: 2n words of the lane for the
// shared-memory layout (stride 1); stk: one entry per order position.
template <bool REG, bool VSYM, bool SPLIT, bool RTV>
bool search_pos(const Geo &g, const Split &sp, const Cell *tbl, int len, const uint8_t *rec,
                uint32_t sub, uint32_t *words, uint32_t *stk, unsigned long long &cnt,
                unsigned long long &nodes, Run &run) {
  Lane<REG> s{};
  s.w.tb = reinterpret_cast<char *>(words);
  s.w.clear(2 * g.n, 1u);
  s.sub = sub;
  s.splitc = 0u;
  s.cnt = 0ull;
  s.nodes = 0ull;
  cnt = nodes = 0ull;
  if (!place_prefix<REG, VSYM>(s.w, g, rec, tbl)) return true;
  if (g.depth == len) {
    cnt = sub == 0u ? 1ull : 0ull;
    return true;
  }
  const uint32_t L = s.w.template cands<VSYM>(tbl[g.depth], g);
  if (g.depth == g.last) {
    if (sub == 0u) cnt = nodes = (unsigned)__popc(L);
    return true;
  }
  if (L == 0u) return true;
  s.p = g.depth;
  s.L = L;
  s.v = 0u;
  s.info = tbl[g.depth];
  for (;;) {
    ++run.iters;
    // with the run-time flag the step is the serving kernel's: VSYM = false
    // (only the prefix placement above takes the flag at compile time)
    const bool fin = dfs_step<REG, RTV ? false : VSYM, true, SPLIT, RTV>(s, g, sp, stk, tbl, 1u);
    if (fin) break;
    // a lane that goes on stands on a cell after the prefix, before the last
    if (s.p < g.depth || s.p >= g.last) {
      ++run.badpos;
      return false;
    }
    run.maxsp = std::max(run.maxsp, s.p - g.depth);
  }
  cnt = s.cnt;
  nodes = s.nodes;
  return true;
}

std::vector<uint8_t> read_file(const char *path) {
  std::vector<uint8_t> out;
  FILE *f = std::fopen(path, "rb");
  if (!f) return out;
  uint8_t buf[4096];
  size_t k;
  while ((k = std::fread(buf, 1, sizeof(buf), f)) > 0) out.insert(out.end(), buf, buf + k);
  std::fclose(f);
  return out;
}

template <bool REG, bool VSYM, bool RTV>
int run_items(const Geo &g, const Split &sp, const Cell *tbl, int len,
              const std::vector<uint8_t> &pre) {
  const int depth = g.depth;
  const long long P = depth ? (long long)pre.size() / depth : 1;
  std::vector<uint32_t> words(2 * (size_t)g.n);
  std::vector<uint32_t> stk((size_t)len, ~0u);
  Run run;
  for (long long k = 0; k < P; ++k) {
    const uint8_t *rec = pre.data() + (size_t)k * (size_t)depth;
    unsigned long long cnt = 0, nodes = 0;
    for (uint32_t sub = 0; sub < (1u << sp.lanes_log2); ++sub) {
      unsigned long long c = 0, nd = 0;
      const bool ok = sp.lanes_log2 > 0
                          ? search_pos<REG, VSYM, true, RTV>(g, sp, tbl, len, rec, sub,
                                                             words.data(), stk.data(), c, nd, run)
                          : search_pos<REG, VSYM, false, RTV>(g, sp, tbl, len, rec, sub,
                                                              words.data(), stk.data(), c, nd,
                                                              run);
      if (!ok) {
        std::fprintf(stderr, "iters %llu maxsp %d overflow %u badpos %d\n", run.iters,
                     run.maxsp, run.ovf, run.badpos);
        return 3;
      }
      cnt += c;
      nodes += nd;
    }
    std::printf("%llu %llu\n", cnt, nodes);
  }
  std::fprintf(stderr, "iters %llu maxsp %d overflow %u badpos %d\n", run.iters, run.maxsp,
               run.ovf, run.badpos);
  return 0;
}

// The per-position step (modes 10-12): cell descriptors for register words
// (bit shifts) or for the shared-memory layout (byte offsets of the lane's
// 2n words: rows, then columns), as the kernels' setup makes them.
int run_pos(int n, uint32_t flags, int mode, const std::vector<uint8_t> &ob,
            const std::vector<uint8_t> &pre, int depth, const Split &sp) {
  const bool diag = (flags & 1u) != 0, vsym = (flags & 2u) != 0;
  const int len = (int)ob.size() / 2;
  std::vector<Cell> tbl(len);
  for (int t = 0; t < len; ++t) {
    const int i = ob[2 * t], j = ob[2 * t + 1];
    tbl[t] = mode == 10 ? describe_regs(i, j, n, diag, vsym ? n / 2 : 8, vsym ? n : 8)
                        : describe_shared(i, j, n, diag, 1u, n);
  }
  Geo g;
  g.n = n;
  g.all = (1u << n) - 1u;
  g.pairmask = (1u << (n / 2)) - 1u;
  g.depth = depth;
  g.last = len - 1;
  g.vsmask = vsym ? 0xffffffffu : 0u;
  if (mode == 10)
    return vsym ? run_items<true, true, false>(g, sp, tbl.data(), len, pre)
                : run_items<true, false, false>(g, sp, tbl.data(), len, pre);
  if (mode == 12)
    return vsym ? run_items<false, true, true>(g, sp, tbl.data(), len, pre)
                : run_items<false, false, true>(g, sp, tbl.data(), len, pre);
  return vsym ? run_items<false, true, false>(g, sp, tbl.data(), len, pre)
              : run_items<false, false, false>(g, sp, tbl.data(), len, pre);
}

}  // namespace

int main(int argc, char **argv) {
  if (argc != 8 && argc != 10) {
    std::fprintf(stderr,
                 "usage: step_check n flags mode order.bin prefixes.bin depth cap "
                 "[lanes_log2 split_pos]\n");
    return 1;
  }
  const int n = std::atoi(argv[1]);
  const uint32_t flags = (uint32_t)std::atoi(argv[2]);
  const int mode = std::atoi(argv[3]);
  const std::vector<uint8_t> ob = read_file(argv[4]);
  const std::vector<uint8_t> pre = read_file(argv[5]);
  const int depth = std::atoi(argv[6]);
  const int cap = std::atoi(argv[7]);
  const int len = (int)ob.size() / 2;
  const bool diag = (flags & 1u) != 0, vsym = (flags & 2u) != 0;
  const bool pos = mode >= 10;
  if (n < 2 || n > (pos ? DLS_MAX_N : 10) || len < 1 || depth < 0 || depth > len || cap < 1)
    return 1;
  if (vsym && (n % 2)) return 1;  // no such squares; the library answers 0
  Split sp{-1, 0};
  if (argc == 10) {
    sp.lanes_log2 = std::atoi(argv[8]);
    sp.pos = std::atoi(argv[9]);
    if (!pos || sp.lanes_log2 < 0 || sp.lanes_log2 > 5 || sp.pos < depth || sp.pos > len - 2)
      return 1;
  }
  if (mode == 10 && (vsym ? n * (n / 2) > 64 : n > 8)) return 2;
  // register words: 8-bit fields without symmetry, n/2 value pairs with it
  const int wr = vsym ? n / 2 : 8, wc = vsym ? n : 8;
  bool dg = false;
  for (int t = depth; t < len; ++t) {
    const int i = ob[2 * t], j = ob[2 * t + 1];
    if (diag && (i == j || i + j == n - 1)) dg = true;
  }
  if ((mode == 1 && (dg || vsym)) || (mode == 2 && dg)) return 2;
  if (pos) return run_pos(n, flags, mode, ob, pre, depth, sp);
  if (!vsym && n == 9) return run_wide(n, flags, mode, ob, pre, depth, cap);

  std::vector<Cell> tbl(len);
  std::vector<uint4> tsh(len);
  std::vector<uint2> tdm(len);
  for (int t = 0; t < len; ++t) {
    const int i = ob[2 * t], j = ob[2 * t + 1];
    tbl[t] = describe_regs(i, j, n, diag, wr, wc);
    const int nx = std::min(t + 1, len - 1);
    snap_row(n, diag, wr, wc, i, j, ob[2 * nx], ob[2 * nx + 1], tsh[t], tdm[t]);
    if (mode != 0) {
      const int n2 = std::min(t + 2, len - 1);
      tdm[t] = make_uint2((uint32_t)(ob[2 * n2] * wr), (uint32_t)(ob[2 * n2 + 1] * wc));
    }
  }
  const SnapTable tb{tsh.data(), tdm.data()};
  std::vector<uint8_t> ci(len), cj(len);
  for (int t = 0; t < len; ++t) {
    ci[t] = ob[2 * t];
    cj[t] = ob[2 * t + 1];
  }
  std::vector<BRow> brows(len);
  for (int t = 0; t < len; ++t) brows[t] = brow_make(n, diag, dg, ci.data(), cj.data(), t, len);
  Geo g;
  g.n = n;
  g.all = (1u << n) - 1u;
  g.pairmask = (1u << (n / 2)) - 1u;
  g.depth = depth;
  g.last = len - 1;
  g.vsmask = vsym ? 0xffffffffu : 0u;

  std::vector<uint4> sa((size_t)cap + 2, make_uint4(~0u, ~0u, ~0u, ~0u));
  std::vector<uint32_t> sw((size_t)cap + 2, ~0u);
  const SnapStack st{sa.data(), sw.data(), cap};

  const long long P = depth ? (long long)pre.size() / depth : 1;
  Run run;
  for (long long k = 0; k < P; ++k) {
    SnapLane s{};
    s.w.tb = nullptr;
    s.w.R = s.w.C = 0ull;
    s.w.dg = 0u;
    unsigned long long cnt = 0, nodes = 0;
    const uint8_t *rec = pre.data() + (size_t)k * (size_t)depth;
    const bool ok = vsym ? place_prefix<true, true>(s.w, g, rec, tbl.data())
                         : place_prefix<true, false>(s.w, g, rec, tbl.data());
    if (ok && depth == len) {
      cnt = 1;
    } else if (ok) {
      const uint32_t L = vsym ? s.w.cands<true>(tbl[depth], g) : s.w.cands<false>(tbl[depth], g);
      if (depth == g.last) {
        cnt = nodes = (unsigned)__popc(L);
      } else if (L != 0u && !vsym) {
        // byte words: the kernels' search for every order without symmetry
        BLane b{};
        b.R0 = (uint32_t)s.w.R;
        b.R1 = (uint32_t)(s.w.R >> 32);
        b.C0 = (uint32_t)s.w.C;
        b.C1 = (uint32_t)(s.w.C >> 32);
        b.dg = s.w.dg;
        b.p = depth;
        b.L = L;
        b.a = brows[depth].a;
        b.b = brows[depth].b;
        b.c = brows[depth].c;
        bool done;
        if (mode == 1)
          done = bsearch<false, true, false>(b, g, st, brows.data(), len, run);
        else if (mode == 2)
          done = bsearch<false, false, true>(b, g, st, brows.data(), len, run);
        else
          done = dg ? bsearch<true, false, false>(b, g, st, brows.data(), len, run)
                    : bsearch<false, false, false>(b, g, st, brows.data(), len, run);
        if (!done) {
          std::fprintf(stderr, "iters %llu maxsp %d overflow %u badpos %d\n", run.iters,
                       run.maxsp, run.ovf, run.badpos);
          return 3;
        }
        cnt = b.cnt;
        nodes = b.nodes;
      } else if (L != 0u) {
        s.p = depth;
        s.L = L;
        s.sh = tsh[depth];
        s.dm = tdm[depth];
        s.sp = s.bot = 0;
        s.cnt = 0ull;
        s.nodes = 0ull;
        bool done;
        if (mode == 1)
          done = search<false, false, true, false>(s, g, st, tb, len, run);
        else if (mode == 2)
          done = vsym ? search<true, false, false, true>(s, g, st, tb, len, run)
                      : search<false, false, false, true>(s, g, st, tb, len, run);
        else if (vsym)
          done = dg ? search<true, true, false, false>(s, g, st, tb, len, run)
                    : search<true, false, false, false>(s, g, st, tb, len, run);
        else
          done = dg ? search<false, true, false, false>(s, g, st, tb, len, run)
                    : search<false, false, false, false>(s, g, st, tb, len, run);
        if (!done) {
          std::fprintf(stderr, "iters %llu maxsp %d overflow %u badpos %d\n", run.iters,
                       run.maxsp, run.ovf, run.badpos);
          return 3;
        }
        cnt = s.cnt;
        nodes = s.nodes;
      }
    }
    std::printf("%llu %llu\n", cnt, nodes);
  }
  std::fprintf(stderr, "iters %llu maxsp %d overflow %u badpos %d\n", run.iters, run.maxsp,
               run.ovf, run.badpos);
  return 0;
}
