// dls_symmetry.cu -- symmetry breaking on the GPU (Section 4).
//
// An hourglass design is a square with only row 0, the last row and both
// diagonals filled (Section 4.2).  The M-transformations that map hourglasses
// to hourglasses (Section 4.1) form a group G generated by
//   - the vertical mirror, column j -> n-1-j (left out for vertically
//     symmetric squares, where it only renames the symbols; Section 5.4);
//   - the swap of rows k, n-1-k together with columns k, n-1-k, for each k in
//     a subset of {0..n/2-1};
//   - a permutation s of {1..n/2-1} applied to rows and columns as
//     k -> s(k), n-1-k -> n-1-s(k) (index 0 stays, so row 0 can only trade
//     places with the last row);
// |G| = 2 (or 1) * 2^(n/2) * (n/2 - 1)!.  After a transformation the symbols
// are renamed so that row 0 reads 0..n-1.  Algorithm 5 keeps an hourglass
// when no image is lexicographically smaller (cells in row-major order) and
// weights it by its class size; Proposition 1 makes every member of a class
// have the same number of completions (Corollary 1).
//
// k_canon: one thread per hourglass.  Each transformation is applied on the
// fly through its inverse row and column maps; the image is compared cell by
// cell with the hourglass and abandoned at the first difference.  The class
// size is |G| / |stabiliser| (the images equal to the hourglass itself).

#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "dls_internal.h"

namespace dls {

constexpr int SB_MAXN = 11;       // 2 * 2^5 * 4! = 1536 transformations at most
constexpr int SB_MAXPERM = 24;    // (5 - 1)!

struct CanonParams {
  int n, h, vsym, len;
  int n_mirror, n_subset, n_perm;
  int n_cmp;                      // comparison cells (row-major, row 0 left out)
  long long count;
  const uint8_t *hg;              // [count][len] hourglass values
  uint32_t *out;                  // class size, or 0 when not canonic
  uint8_t ci[4 * DLS_MAX_N], cj[4 * DLS_MAX_N];     // hourglass cells, given order
  uint8_t mi[4 * DLS_MAX_N], mj[4 * DLS_MAX_N];     // comparison cells
  uint8_t perm[SB_MAXPERM][SB_MAXN];                // s on {0..h-1}, s(0) = 0
  uint8_t pinv[SB_MAXPERM][SB_MAXN];
};

__global__ void __launch_bounds__(128) k_canon(const __grid_constant__ CanonParams P) {
  const long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= P.count) return;
  const int n = P.n, h = P.h;
  uint8_t g[SB_MAXN][SB_MAXN];  // the hourglass, 0xff = empty
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) g[i][j] = 0xff;
  const uint8_t *rec = P.hg + (size_t)q * P.len;
  for (int t = 0; t < P.len; ++t) {
    const int i = P.ci[t], j = P.cj[t];
    g[i][j] = rec[t];
    if (P.vsym) g[i][n - 1 - j] = (uint8_t)(n - 1 - rec[t]);
  }
  // rename so that row 0 reads 0..n-1
  uint8_t ren0[SB_MAXN];
  for (int j = 0; j < n; ++j) ren0[g[0][j] < n ? g[0][j] : 0] = (uint8_t)j;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (g[i][j] != 0xff) g[i][j] = ren0[g[i][j] < n ? g[i][j] : 0];

  int stab = 0;
  bool canonic = true;
  for (int m = 0; m < P.n_mirror && canonic; ++m) {
    for (int S = 0; S < P.n_subset && canonic; ++S) {
      for (int k = 0; k < P.n_perm; ++k) {
        // inverse maps: image index -> source index.  Forward: columns are
        // mirrored, then pair-swapped, then permuted; rows pair-swapped, then
        // permuted.  Undo in reverse.
        uint8_t rinv[SB_MAXN], cinv[SB_MAXN];
        for (int x = 0; x < n; ++x) {
          // undo the permutation
          int y = x;
          if (x < h) y = P.pinv[k][x];
          else if (x >= n - h) y = n - 1 - P.pinv[k][n - 1 - x];
          // undo the pair swaps
          if (y < h && ((S >> y) & 1)) y = n - 1 - y;
          else if (y >= n - h && ((S >> (n - 1 - y)) & 1)) y = n - 1 - y;
          rinv[x] = (uint8_t)y;
          cinv[x] = (uint8_t)(m ? n - 1 - y : y);
        }
        // renaming of the image: its row 0 is source row rinv[0]
        uint8_t ren[SB_MAXN];
        for (int j = 0; j < n; ++j) ren[g[rinv[0]][cinv[j]]] = (uint8_t)j;
        int c = 0;
        for (int t = 0; t < P.n_cmp; ++t) {
          const int i = P.mi[t], j = P.mj[t];
          const int a = ren[g[rinv[i]][cinv[j]]];
          const int b = g[i][j];
          if (a != b) {
            c = a < b ? -1 : 1;
            break;
          }
        }
        if (c < 0) {
          canonic = false;
          break;
        }
        if (c == 0) stab++;
      }
    }
  }
  const int order = P.n_mirror * P.n_subset * P.n_perm;
  P.out[q] = canonic ? (uint32_t)(order / stab) : 0u;
}

}  // namespace dls

using namespace dls;

extern "C" {

int dls_hourglass_classes(int n, uint32_t flags, const uint8_t *order, int len,
                          const uint8_t *d_hourglasses, int64_t count,
                          uint32_t *d_class_size, void *stream) {
  if (n < 2 || n > SB_MAXN) return DLS_ERR_INVALID_N;
  if (!(flags & DLS_DIAGONAL)) return DLS_ERR_BAD_ARG;
  OrderInfo info;
  int rc = validate_order(n, flags, order, len, &info);
  if (rc) return rc;
  if (count < 0 || (count > 0 && (d_hourglasses == nullptr || d_class_size == nullptr)))
    return DLS_ERR_BAD_ARG;
  const bool vsym = (flags & DLS_VSYM) != 0;
  if (vsym && (n % 2)) return DLS_ERR_INVALID_N;
  const int w = vsym ? n / 2 : n;
  // the given cells must be exactly the hourglass cells (left half with vsym)
  bool want[DLS_MAX_N][DLS_MAX_N] = {}, got[DLS_MAX_N][DLS_MAX_N] = {};
  int n_want = 0;
  auto mark = [&](int i, int j) {
    if (j < w && !want[i][j]) {
      want[i][j] = true;
      n_want++;
    }
  };
  for (int j = 0; j < n; ++j) {
    mark(0, j);
    mark(n - 1, j);
  }
  for (int i = 0; i < n; ++i) {
    mark(i, i);
    mark(i, n - 1 - i);
  }
  if (len != n_want) return DLS_ERR_BAD_ORDER;
  for (int t = 0; t < len; ++t) {
    if (!want[info.i[t]][info.j[t]]) return DLS_ERR_BAD_ORDER;
    got[info.i[t]][info.j[t]] = true;
  }
  if (count == 0) return DLS_OK;
  CanonParams P;
  std::memset(&P, 0, sizeof(P));
  P.n = n;
  P.h = n / 2;
  P.vsym = vsym ? 1 : 0;
  P.len = len;
  P.count = count;
  P.hg = d_hourglasses;
  P.out = d_class_size;
  for (int t = 0; t < len; ++t) {
    P.ci[t] = info.i[t];
    P.cj[t] = info.j[t];
  }
  // comparison cells: row-major, row 0 left out (it is 0..n-1 in every image)
  for (int i = 1; i < n; ++i)
    for (int j = 0; j < w; ++j)
      if (got[i][j]) {
        P.mi[P.n_cmp] = (uint8_t)i;
        P.mj[P.n_cmp] = (uint8_t)j;
        P.n_cmp++;
      }
  P.n_mirror = vsym ? 1 : 2;
  P.n_subset = 1 << P.h;
  std::vector<uint8_t> s(P.h);
  for (int t = 0; t < P.h; ++t) s[t] = (uint8_t)t;
  int k = 0;
  do {
    for (int t = 0; t < P.h; ++t) {
      P.perm[k][t] = s[t];
      P.pinv[k][s[t]] = (uint8_t)t;
    }
    k++;
  } while (P.h > 1 && std::next_permutation(s.begin() + 1, s.end()));
  P.n_perm = k;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int block = 128;
  const long long grid = (count + block - 1) / block;
  k_canon<<<(unsigned)grid, block, 0, st>>>(P);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_cuda_error(cudaGetErrorString(e));
    return DLS_ERR_CUDA;
  }
  return DLS_OK;
}

}  // extern "C"
