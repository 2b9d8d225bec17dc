// dls_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cstdint>
#include <cstring>

#include "../../include/dls.h"

namespace dls {

// A validated fill order.
struct OrderInfo {
  int n = 0;
  uint32_t flags = 0;
  int len = 0;
  uint8_t i[DLS_MAX_CELLS];
  uint8_t j[DLS_MAX_CELLS];
};

// Checks n, flags and the cells of an order (distinct, inside the square,
// left half with DLS_VSYM); fills *info when not NULL.
int validate_order(int n, uint32_t flags, const uint8_t *order, int order_len,
                   OrderInfo *info);

// Vertically symmetric squares of odd order >= 3 do not exist (the middle
// column would be constant), so every count is 0.
bool vsym_all_zero(int n, uint32_t flags);

// Records the text of the last CUDA error for dls_last_cuda_error().
void set_cuda_error(const char *what);

// The status code that a count's status word (bits set by the kernels)
// stands for (dls_kernels.cu).
int status_code(unsigned word);

// Forgets the device addresses of the allocation-free entry's array
// (dls_noalloc.cu; called by dls_release()).
void noalloc_forget();

// splitmix64 (Steele, Lea, Flood 2014), the library's counter-based
// generator for random probes.
uint64_t splitmix64(uint64_t x);

// Knuth's random-descent estimate of the search nodes below a prefix
// (dls_estimate_nodes), probes keyed by `key`; 0 for an invalid prefix.
double estimate_nodes(const OrderInfo &info, const uint8_t *prefix, int depth, uint64_t key,
                      int probes);

// Host bitmask search state (Section 3).
struct HostState {
  int n;
  bool diag, vsym;
  uint32_t all;
  uint32_t row[DLS_MAX_N], col[DLS_MAX_N], md, ad;
  const OrderInfo *o;

  void init(const OrderInfo &info) {
    o = &info;
    n = info.n;
    diag = (info.flags & DLS_DIAGONAL) != 0;
    vsym = (info.flags & DLS_VSYM) != 0;
    all = (n >= 32) ? 0xffffffffu : ((1u << n) - 1u);
    // odd order with vertical symmetry: a left cell holding (n-1)/2 would put
    // the same value in its mirror cell, in the same row
    if (vsym && (n & 1)) all &= ~(1u << (n / 2));
    std::memset(row, 0, sizeof(row));
    std::memset(col, 0, sizeof(col));
    md = ad = 0;
  }
  uint32_t mirror(uint32_t m) const {
    // bit v -> bit n-1-v
    uint32_t r = 0;
    for (int v = 0; v < n; ++v)
      if (m >> v & 1u) r |= 1u << (n - 1 - v);
    return r;
  }
  bool on_md(int t) const { return diag && o->i[t] == o->j[t]; }
  bool on_ad(int t) const { return diag && o->i[t] + o->j[t] == n - 1; }
  uint32_t candidates(int t) const {
    uint32_t f = row[o->i[t]] | col[o->j[t]];
    if (on_md(t)) f |= md;
    if (on_ad(t)) f |= ad;
    return all & ~f;
  }
  // toggle one-hot (or two-hot) value bits d at order position t
  void toggle(int t, uint32_t d) {
    uint32_t dm = vsym ? mirror(d) : 0u;
    row[o->i[t]] ^= d ^ dm;
    col[o->j[t]] ^= d;
    if (on_md(t)) md ^= d;
    if (on_ad(t)) ad ^= d;
    if (vsym) {
      if (on_md(t)) ad ^= dm;  // mirror cell (i, n-1-i) is on the anti-diagonal
      if (on_ad(t)) md ^= dm;  // mirror cell (i, i) is on the main diagonal
    }
  }
  bool place(int t, int value) {
    if (value < 0 || value >= n) return false;
    uint32_t b = 1u << value;
    if (!(candidates(t) & b)) return false;
    toggle(t, b);
    return true;
  }
};

}  // namespace dls
