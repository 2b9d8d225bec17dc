// dls_internal.h -- declarations shared by the library's translation units.
#pragma once

#include <cstdint>

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

}  // namespace dls
