// dls_host.cpp -- host-side part of the C ABI: fill orders, the prefix split,
// the draw-driven prefix sampler, multipliers, 128-bit helpers, status names.
//
// Everything here runs on the CPU and prepares the input of the GPU search
// (dls_kernels.cu).  The search state is the bitmask form of Section 3: one
// word per row, column and diagonal holding the values in use, candidates
// ALL & ~(row | col | md | ad), lowest set bit first (Algorithm 4).

#include "dls_internal.h"

#include <algorithm>
#include <cstring>
#include <deque>
#include <mutex>
#include <string>
#include <vector>

namespace dls {

thread_local std::string g_last_cuda_error;

void set_cuda_error(const char *what) { g_last_cuda_error = what ? what : ""; }

// ------------------------------------------------------------ validation --

int validate_order(int n, uint32_t flags, const uint8_t *order, int order_len,
                   OrderInfo *info) {
  if (n < 1 || n > DLS_MAX_N) return DLS_ERR_INVALID_N;
  if (order_len < 0 || order_len > n * n) return DLS_ERR_BAD_ORDER;
  if (order_len > 0 && order == nullptr) return DLS_ERR_BAD_ARG;
  if (flags & ~(DLS_DIAGONAL | DLS_VSYM)) return DLS_ERR_BAD_ARG;
  bool seen[DLS_MAX_N][DLS_MAX_N] = {};
  const bool vsym = (flags & DLS_VSYM) != 0;
  for (int t = 0; t < order_len; ++t) {
    int i = order[2 * t], j = order[2 * t + 1];
    if (i >= n || j >= n) return DLS_ERR_BAD_ORDER;
    if (vsym && j >= n / 2 && n > 1) return DLS_ERR_BAD_ORDER;
    if (seen[i][j]) return DLS_ERR_BAD_ORDER;
    seen[i][j] = true;
    if (info) {
      info->i[t] = (uint8_t)i;
      info->j[t] = (uint8_t)j;
    }
  }
  if (vsym && n == 1 && order_len > 0) return DLS_ERR_BAD_ORDER;
  if (info) {
    info->n = n;
    info->flags = flags;
    info->len = order_len;
  }
  return DLS_OK;
}

bool vsym_all_zero(int n, uint32_t flags) {
  return (flags & DLS_VSYM) && (n % 2 == 1) && n >= 3;
}

// ------------------------------------------------------------ fill orders --

static void order_md_ad_rows(int n, bool vsym, int first_rows,
                             std::vector<std::pair<int, int>> &out) {
  const int w = vsym ? n / 2 : n;
  bool used[DLS_MAX_N][DLS_MAX_N] = {};
  auto add = [&](int i, int j) {
    if (j >= w || used[i][j]) return;
    used[i][j] = true;
    out.push_back({i, j});
  };
  for (int i = 0; i < first_rows && i < n; ++i)
    for (int j = 0; j < w; ++j) add(i, j);
  for (int i = 0; i < n; ++i) add(i, i);
  for (int i = 0; i < n; ++i) add(i, n - 1 - i);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < w; ++j) add(i, j);
}

static void order_hourglass(int n, bool vsym, std::vector<std::pair<int, int>> &out) {
  const int w = vsym ? n / 2 : n;
  bool used[DLS_MAX_N][DLS_MAX_N] = {};
  auto add = [&](int i, int j) {
    if (j >= w || used[i][j]) return;
    used[i][j] = true;
    out.push_back({i, j});
  };
  for (int j = 0; j < n; ++j) add(0, j);
  for (int i = 0; i < n; ++i) add(i, i);
  for (int i = 0; i < n; ++i) add(i, n - 1 - i);
  for (int j = 0; j < n; ++j) add(n - 1, j);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) add(i, j);
}

// Section 2.3: after row 0, repeatedly take the unassigned cell with the
// largest V = r_i + c_j + md(i,j) + ad(i,j) -- the numbers of assigned cells
// in its row, its column and, when the cell lies on them, the two diagonals
// -- ties broken by the first cell in row-major order.  Whenever placing a
// cell leaves exactly one unassigned cell in one of its lines (row, column,
// main diagonal, anti-diagonal, checked in that order), that cell is queued
// and taken next, queued cells first-in first-out.  Only which cells are
// assigned matters, never their values.  This reproduces Fig. 1 for order 9.
// With vsym the cells are the left half: a row has n/2 of them, a column n,
// and the two diagonals become one line (the left cells on the main diagonal
// and those on the anti-diagonal, whose mirrors complete the main diagonal).
// squares = true is this library's variant (DLS_ORDER_HEURISTIC_SQ): V is
// the sum of the squares of those counts, which prefers a cell on one nearly
// complete line to a cell on several half-filled ones; everything else is
// the same.
static void order_heuristic(int n, bool diag, bool vsym,
                            const std::vector<std::pair<int, int>> &kept,
                            std::vector<std::pair<int, int>> &out, bool squares = false) {
  const int w = vsym ? n / 2 : n;
  std::vector<std::vector<std::pair<int, int>>> lines;
  std::vector<std::vector<int>> of_cell(n * w);
  for (int i = 0; i < n; ++i) {
    std::vector<std::pair<int, int>> l;
    for (int j = 0; j < w; ++j) l.push_back({i, j});
    lines.push_back(l);
  }
  for (int j = 0; j < w; ++j) {
    std::vector<std::pair<int, int>> l;
    for (int i = 0; i < n; ++i) l.push_back({i, j});
    lines.push_back(l);
  }
  if (diag && !vsym) {
    std::vector<std::pair<int, int>> m, a;
    for (int i = 0; i < n; ++i) m.push_back({i, i});
    for (int i = 0; i < n; ++i) a.push_back({i, n - 1 - i});
    lines.push_back(m);
    lines.push_back(a);
  } else if (diag && vsym) {
    // left cells of the main diagonal (rows above the middle) and of the
    // anti-diagonal (rows below it); an odd order's centre is not a left cell
    std::vector<std::pair<int, int>> m;
    for (int i = 0; i < n; ++i) {
      if (i < w) m.push_back({i, i});
      else if (i >= n - w) m.push_back({i, n - 1 - i});
    }
    lines.push_back(m);
  }
  for (int l = 0; l < (int)lines.size(); ++l)
    for (auto &c : lines[l]) of_cell[c.first * w + c.second].push_back(l);
  std::vector<int> filled(lines.size(), 0);
  std::vector<char> asg(n * w, 0);
  std::deque<std::pair<int, int>> queue;
  auto assign = [&](int i, int j, bool forced_rule) {
    asg[i * w + j] = 1;
    out.push_back({i, j});
    for (int l : of_cell[i * w + j]) {
      filled[l]++;
      if (forced_rule && filled[l] == (int)lines[l].size() - 1)
        for (auto &c : lines[l])
          if (!asg[c.first * w + c.second]) queue.push_back(c);
    }
  };
  // the kept cells (row 0 for a whole order) are assigned without queuing
  for (auto &c : kept) assign(c.first, c.second, false);
  const int total = n * w;
  while ((int)out.size() < total) {
    std::pair<int, int> cell{-1, -1};
    while (!queue.empty()) {
      auto q = queue.front();
      queue.pop_front();
      if (!asg[q.first * w + q.second]) {
        cell = q;
        break;
      }
    }
    if (cell.first < 0) {
      int best = -1;
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < w; ++j) {
          if (asg[i * w + j]) continue;
          int v = 0;
          for (int l : of_cell[i * w + j]) v += squares ? filled[l] * filled[l] : filled[l];
          if (v > best) {
            best = v;
            cell = {i, j};
          }
        }
    }
    assign(cell.first, cell.second, true);
  }
}

// ------------------------------------------------------ size estimate --

uint64_t splitmix64(uint64_t x) {
  x += 0x9e3779b97f4a7c15ull;
  x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ull;
  x = (x ^ (x >> 27)) * 0x94d049bb133111ebull;
  return x ^ (x >> 31);
}

// Knuth's estimate of the size of the search below a prefix (D. E. Knuth,
// "Estimating the efficiency of backtrack programs", 1975): a random descent
// along the order takes, at each cell, the product of the numbers of
// admissible values met so far as its estimate of the nodes at that depth
// and adds them up, stopping at a dead end or the last cell; the mean over
// descents is an unbiased estimate of the number of search nodes.  (The
// same estimate of the completions alone is nearly always 0 here: most
// descents end at a dead end.)  The serving path uses it only to choose how
// finely a job is split -- no count depends on it.
double estimate_nodes(const OrderInfo &info, const uint8_t *prefix, int depth, uint64_t key,
                      int probes) {
  HostState base;
  base.init(info);
  for (int t = 0; t < depth; ++t)
    if (!base.place(t, prefix[t])) return 0.0;
  double sum = 0.0;
  for (int pr = 0; pr < probes; ++pr) {
    HostState s = base;
    double w = 1.0;
    for (int t = depth; t < info.len; ++t) {
      const uint32_t c = s.candidates(t);
      const int k = __builtin_popcount(c);
      w *= (double)k;
      sum += w;
      if (k == 0 || t == info.len - 1) break;
      const uint64_t r = splitmix64(key ^ splitmix64(((uint64_t)pr << 32) | (uint64_t)t));
      uint32_t v = c;
      for (int q = (int)(r % (uint64_t)k); q > 0; --q) v &= v - 1u;
      s.toggle(t, v & (0u - v));
    }
  }
  return probes > 0 ? sum / probes : 0.0;
}

// ------------------------------------------------------ order trimming --

// Cells at the end of `cells` that share coordinate `axis` (0 row, 1 column)
// with the last cell and lie on no diagonal (with the diagonal flag), at
// most `most`.
static int tail_run(const std::vector<std::pair<int, int>> &cells, int axis, int n,
                    bool diag, int most) {
  if (cells.empty()) return 0;
  const auto key = [axis](const std::pair<int, int> &c) { return axis ? c.second : c.first; };
  const int line = key(cells.back());
  int k = 0;
  for (auto it = cells.rbegin(); it != cells.rend() && k < most; ++it) {
    if (key(*it) != line) break;
    if (diag && (it->first == it->second || it->first + it->second == n - 1)) break;
    ++k;
  }
  return k;
}

}  // namespace dls

using namespace dls;

extern "C" {

const char *dls_strerror(int code) {
  switch (code) {
    case DLS_OK: return "ok";
    case DLS_ERR_INVALID_N: return "order n outside 1..16";
    case DLS_ERR_BAD_ORDER: return "bad fill order (repeated, out-of-range or right-half cell)";
    case DLS_ERR_BAD_ARG: return "bad argument";
    case DLS_ERR_CAPACITY: return "output buffer too small";
    case DLS_ERR_CUDA: return "CUDA error";
    case DLS_ERR_TIMEOUT: return "stopped: iteration budget spent";
    case DLS_ERR_ABORTED: return "aborted";
    case DLS_ERR_NO_MEMORY: return "out of memory";
    case DLS_ERR_BAD_STATE: return "object in the wrong state";
    case DLS_ERR_INTERNAL: return "a kernel exceeded a bound it relies on";
    default: return "unknown status";
  }
}

const char *dls_last_cuda_error(void) { return g_last_cuda_error.c_str(); }

int dls_version(void) { return (1 << 16) | 2; }

int dls_fill_order(int n, uint32_t flags, int kind, int first_rows,
                   uint8_t *ij_out, int cap, int *len_out) {
  if (n < 1 || n > DLS_MAX_N) return DLS_ERR_INVALID_N;
  if (len_out == nullptr || cap < 0 || (cap > 0 && ij_out == nullptr))
    return DLS_ERR_BAD_ARG;
  if (flags & ~(DLS_DIAGONAL | DLS_VSYM)) return DLS_ERR_BAD_ARG;
  const bool vsym = (flags & DLS_VSYM) != 0;
  const bool diag = (flags & DLS_DIAGONAL) != 0;
  std::vector<std::pair<int, int>> cells;
  switch (kind) {
    case DLS_ORDER_MD_AD_ROWS:
      if (first_rows < 1) first_rows = 1;
      order_md_ad_rows(n, vsym, first_rows, cells);
      break;
    case DLS_ORDER_ROW_MAJOR:
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < (vsym ? n / 2 : n); ++j) cells.push_back({i, j});
      break;
    case DLS_ORDER_HOURGLASS:
      order_hourglass(n, vsym, cells);
      break;
    case DLS_ORDER_HEURISTIC:
    case DLS_ORDER_HEURISTIC_SQ: {
      std::vector<std::pair<int, int>> row0;
      for (int j = 0; j < (vsym ? n / 2 : n); ++j) row0.push_back({0, j});
      order_heuristic(n, diag, vsym, row0, cells, kind == DLS_ORDER_HEURISTIC_SQ);
      break;
    }
    default:
      return DLS_ERR_BAD_ARG;
  }
  *len_out = (int)cells.size();
  if ((int)cells.size() > cap) return DLS_ERR_CAPACITY;
  for (size_t t = 0; t < cells.size(); ++t) {
    ij_out[2 * t] = (uint8_t)cells[t].first;
    ij_out[2 * t + 1] = (uint8_t)cells[t].second;
  }
  return DLS_OK;
}

int dls_order_complete(int n, uint32_t flags, const uint8_t *order, int keep,
                       int kind, uint8_t *ij_out, int cap, int *len_out) {
  if (n < 1 || n > DLS_MAX_N) return DLS_ERR_INVALID_N;
  if (len_out == nullptr || keep < 0 || cap < 0 || (cap > 0 && ij_out == nullptr))
    return DLS_ERR_BAD_ARG;
  OrderInfo info;
  int rc = validate_order(n, flags, order, keep, &info);
  if (rc) return rc;
  const bool vsym = (flags & DLS_VSYM) != 0;
  const bool diag = (flags & DLS_DIAGONAL) != 0;
  const int w = vsym ? n / 2 : n;
  std::vector<std::pair<int, int>> kept, cells;
  for (int t = 0; t < keep; ++t) kept.push_back({info.i[t], info.j[t]});
  if (kind == DLS_ORDER_HEURISTIC || kind == DLS_ORDER_HEURISTIC_SQ) {
    order_heuristic(n, diag, vsym, kept, cells, kind == DLS_ORDER_HEURISTIC_SQ);
  } else if (kind == DLS_ORDER_MD_AD_ROWS || kind == DLS_ORDER_ROW_MAJOR) {
    bool used[DLS_MAX_N][DLS_MAX_N] = {};
    for (auto &c : kept) {
      used[c.first][c.second] = true;
      cells.push_back(c);
    }
    auto add = [&](int i, int j) {
      if (j >= w || used[i][j]) return;
      used[i][j] = true;
      cells.push_back({i, j});
    };
    if (kind == DLS_ORDER_MD_AD_ROWS) {
      for (int i = 0; i < n; ++i) add(i, i);
      for (int i = 0; i < n; ++i) add(i, n - 1 - i);
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < w; ++j) add(i, j);
  } else {
    return DLS_ERR_BAD_ARG;
  }
  *len_out = (int)cells.size();
  if ((int)cells.size() > cap) return DLS_ERR_CAPACITY;
  for (size_t t = 0; t < cells.size(); ++t) {
    ij_out[2 * t] = (uint8_t)cells[t].first;
    ij_out[2 * t + 1] = (uint8_t)cells[t].second;
  }
  return DLS_OK;
}

int dls_order_trim(int n, uint32_t flags, const uint8_t *order, int order_len, int keep,
                   int window, uint8_t *ij_out, int cap, int *len_out) {
  if (n < 1 || n > DLS_MAX_N) return DLS_ERR_INVALID_N;
  if (len_out == nullptr || cap < 0 || (cap > 0 && ij_out == nullptr) || window < 0)
    return DLS_ERR_BAD_ARG;
  OrderInfo info;
  int rc = validate_order(n, flags, order, order_len, &info);
  if (rc) return rc;
  if (keep < 0 || keep > order_len) return DLS_ERR_BAD_ARG;
  std::vector<std::pair<int, int>> cells;
  for (int t = 0; t < order_len; ++t) cells.push_back({info.i[t], info.j[t]});
  const bool diag = (flags & DLS_DIAGONAL) != 0;
  const bool vsym = (flags & DLS_VSYM) != 0;
  const int w = vsym ? n / 2 : n;
  if (!(vsym && n % 2) && order_len == n * w && order_len > keep + 1) {
    const int most = order_len - keep - 1;  // one cell after keep stays
    const int start = std::max(keep, order_len - window);
    std::vector<std::pair<int, int>> best;
    int best_k = 0;  // nothing to drop: the order stays as it is
    // with vertical symmetry a row's last left cell is not forced (two
    // values of a symmetric pair may fit), so only row runs go
    for (int axis = 0; axis < (vsym ? 1 : 2); ++axis) {
      // the window's cells on the last cell's line move to the end
      const int line = axis ? cells.back().second : cells.back().first;
      std::vector<std::pair<int, int>> moved(cells.begin(), cells.begin() + start), on;
      for (int t = start; t < order_len; ++t) {
        const int c = axis ? cells[t].second : cells[t].first;
        (c == line ? on : moved).push_back(cells[t]);
      }
      moved.insert(moved.end(), on.begin(), on.end());
      const int k = tail_run(moved, axis, n, diag, most);
      if (k > best_k) {
        best_k = k;
        best.swap(moved);
      }
    }
    if (best_k > 0) {
      best.resize(best.size() - (size_t)best_k);
      cells.swap(best);
    }
  }
  *len_out = (int)cells.size();
  if ((int)cells.size() > cap) return DLS_ERR_CAPACITY;
  for (size_t t = 0; t < cells.size(); ++t) {
    ij_out[2 * t] = (uint8_t)cells[t].first;
    ij_out[2 * t + 1] = (uint8_t)cells[t].second;
  }
  return DLS_OK;
}

int dls_extend_prefixes(int n, uint32_t flags, const uint8_t *order,
                        int order_len, const uint8_t *base, int base_depth,
                        int64_t n_base, int depth, uint8_t *out, int64_t cap,
                        int64_t *parents_out, int64_t *n_out) {
  OrderInfo info;
  int rc = validate_order(n, flags, order, order_len, &info);
  if (rc) return rc;
  if (n_out == nullptr || n_base < 0 || cap < 0 || base_depth < 0 ||
      depth < base_depth || depth > order_len)
    return DLS_ERR_BAD_ARG;
  if ((n_base > 0 && base_depth > 0 && base == nullptr) ||
      (cap > 0 && depth > 0 && out == nullptr))
    return DLS_ERR_BAD_ARG;
  *n_out = 0;
  if (vsym_all_zero(n, flags)) return DLS_OK;
  int64_t produced = 0;
  HostState s;
  uint32_t L[DLS_MAX_CELLS + 1];
  uint32_t cur[DLS_MAX_CELLS + 1];
  uint8_t vals[DLS_MAX_CELLS];
  for (int64_t b = 0; b < n_base; ++b) {
    s.init(info);
    bool ok = true;
    const uint8_t *bp = base + (size_t)b * (size_t)base_depth;
    for (int t = 0; t < base_depth && ok; ++t) {
      ok = s.place(t, bp[t]);
      vals[t] = bp[t];
    }
    if (!ok) continue;
    if (depth == base_depth) {
      if (produced < cap) {
        if (depth) std::memcpy(out + (size_t)produced * depth, vals, depth);
        if (parents_out) parents_out[produced] = b;
      }
      produced++;
      continue;
    }
    // iterative DFS over positions base_depth..depth-1 (Algorithm 4)
    int t = base_depth;
    L[t] = s.candidates(t);
    cur[t] = 0;
    while (t >= base_depth) {
      if (cur[t]) {
        s.toggle(t, cur[t]);
        cur[t] = 0;
      }
      if (L[t] == 0) {
        --t;
        continue;
      }
      uint32_t v = L[t] & (0u - L[t]);
      L[t] &= L[t] - 1u;
      s.toggle(t, v);
      cur[t] = v;
      vals[t] = (uint8_t)__builtin_ctz(v);
      if (t + 1 == depth) {
        if (produced < cap) {
          std::memcpy(out + (size_t)produced * depth, vals, depth);
          if (parents_out) parents_out[produced] = b;
        }
        produced++;
        continue;
      }
      ++t;
      L[t] = s.candidates(t);
      cur[t] = 0;
    }
  }
  *n_out = produced;
  return produced > cap ? DLS_ERR_CAPACITY : DLS_OK;
}

int dls_estimate_nodes(int n, uint32_t flags, const uint8_t *order, int order_len,
                       const uint8_t *prefix, int depth, uint64_t seed, int probes,
                       double *nodes_out) {
  OrderInfo info;
  int rc = validate_order(n, flags, order, order_len, &info);
  if (rc) return rc;
  if (nodes_out == nullptr || depth < 0 || depth > order_len || probes < 1 ||
      (depth > 0 && prefix == nullptr))
    return DLS_ERR_BAD_ARG;
  *nodes_out = vsym_all_zero(n, flags) ? 0.0
                                       : estimate_nodes(info, prefix, depth, splitmix64(seed),
                                                        probes);
  return DLS_OK;
}

int dls_sample_prefix(int n, uint32_t flags, const uint8_t *order,
                      int order_len, int depth, const uint32_t *draws,
                      int64_t n_draws, uint8_t *out, int64_t *draws_used) {
  OrderInfo info;
  int rc = validate_order(n, flags, order, order_len, &info);
  if (rc) return rc;
  if (depth < 0 || depth > order_len || n_draws < 0 ||
      (depth > 0 && out == nullptr) || (n_draws > 0 && draws == nullptr))
    return DLS_ERR_BAD_ARG;
  if (draws_used) *draws_used = 0;
  HostState s;
  s.init(info);
  uint32_t placed[DLS_MAX_CELLS];
  int64_t used = 0;
  int t = 0;
  while (t < depth) {
    uint32_t cand = s.candidates(t);
    if (cand == 0) {
      int r = t;
      while (r > 0 && info.i[r - 1] == info.i[t]) --r;
      for (int u = t - 1; u >= r; --u) s.toggle(u, placed[u]);
      t = r;
      continue;
    }
    if (used >= n_draws) return DLS_ERR_CAPACITY;
    int k = (int)(draws[used++] % (uint32_t)__builtin_popcount(cand));
    uint32_t v = cand;
    for (int q = 0; q < k; ++q) v &= v - 1u;
    v &= 0u - v;
    s.toggle(t, v);
    placed[t] = v;
    out[t] = (uint8_t)__builtin_ctz(v);
    ++t;
  }
  if (draws_used) *draws_used = used;
  return DLS_OK;
}

dls_u128 dls_mul_u64(uint64_t a, dls_u128 b) {
  unsigned __int128 lo = (unsigned __int128)a * b.lo;
  unsigned __int128 hi = (unsigned __int128)a * b.hi;
  dls_u128 r;
  r.lo = (uint64_t)lo;
  r.hi = (uint64_t)(lo >> 64) + (uint64_t)hi;
  return r;
}

dls_u128 dls_add_u128(dls_u128 a, dls_u128 b) {
  dls_u128 r;
  r.lo = a.lo + b.lo;
  r.hi = a.hi + b.hi + (r.lo < a.lo ? 1u : 0u);
  return r;
}

dls_u128 dls_multiplier(int n, uint32_t flags) {
  dls_u128 m = {1, 0};
  if (n < 1 || n > DLS_MAX_N) return dls_u128{0, 0};
  if (flags & DLS_VSYM) {
    if (n % 2 == 1) return m;
    int h = n / 2;
    for (int k = 2; k <= h; ++k) m = dls_mul_u64((uint64_t)k, m);
    for (int k = 0; k < h; ++k) m = dls_mul_u64(2u, m);
    return m;
  }
  for (int k = 2; k <= n; ++k) m = dls_mul_u64((uint64_t)k, m);
  return m;
}

}  // extern "C"
