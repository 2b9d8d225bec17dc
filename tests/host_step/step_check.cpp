// step_check.cpp -- runs the kernels' snapshot search step (snap_step of
// dls_snapshot.cuh, compiled for the host through shim.h) on one lane per
// prefix, with no warp and no donation, for tests/test_host_step.py.
//
//   step_check n flags mode order.bin prefixes.bin depth cap
//
// mode: 0 = the plain step (diagonal words when a cell after the prefix lies
// on a diagonal), 1 = lookahead, 2 = fused step (1 and 2 only without
// diagonal words and without vertical symmetry; exit 2 otherwise).
// order.bin: the fill order as (i, j) byte pairs; prefixes.bin: depth value
// bytes per prefix.  cap: stack entries per lane.  The position table is
// built as the kernels' setup builds it.  Every stack slot starts as 0xff
// bytes, so a read of a slot never written shows up as a bad position.
//
// stdout: "count nodes" per prefix.  stderr: one line
// "iters I maxsp M overflow O badpos B".  Exit 3 when a step leaves the lane
// at a position outside the order or a stack index outside [0, cap].
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

}  // namespace

int main(int argc, char **argv) {
  if (argc != 8) {
    std::fprintf(stderr, "usage: step_check n flags mode order.bin prefixes.bin depth cap\n");
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
  if (n < 2 || n > 10 || len < 1 || depth < 0 || depth > len || cap < 1) return 1;
  if (vsym && (n % 2)) return 1;  // no such squares; the library answers 0
  // register words: 8-bit fields without symmetry, n/2 value pairs with it
  const int wr = vsym ? n / 2 : 8, wc = vsym ? n : 8;
  bool dg = false;
  for (int t = depth; t < len; ++t) {
    const int i = ob[2 * t], j = ob[2 * t + 1];
    if (diag && (i == j || i + j == n - 1)) dg = true;
  }
  if (mode != 0 && (dg || vsym)) return 2;

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
          done = search<false, false, false, true>(s, g, st, tb, len, run);
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
