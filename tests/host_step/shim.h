// shim.h -- host definitions of the few CUDA builtins and vector types that
// the per-lane search headers (dls_search.cuh, dls_snapshot.cuh) use, so
// that the kernels' own search step compiles and runs on the CPU for the
// tests.  Each builtin is written from its documented meaning.
#pragma once

#include <algorithm>
#include <cstdint>

#define __device__
#define __host__
#define __forceinline__ inline

struct uint2 {
  uint32_t x, y;
};
struct uint4 {
  uint32_t x, y, z, w;
};

inline uint2 make_uint2(uint32_t x, uint32_t y) { return {x, y}; }
inline uint4 make_uint4(uint32_t x, uint32_t y, uint32_t z, uint32_t w) { return {x, y, z, w}; }

// number of set bits
inline int __popc(uint32_t v) {
  int c = 0;
  for (; v != 0u; v &= v - 1u) ++c;
  return c;
}

// bit i of the result = bit 31 - i of v
inline uint32_t __brev(uint32_t v) {
  uint32_t r = 0u;
  for (int i = 0; i < 32; ++i) r |= ((v >> i) & 1u) << (31 - i);
  return r;
}

// byte k of the result = byte ((s >> 4k) & 7) of the eight bytes y:x
// (x holds bytes 0-3, y bytes 4-7)
inline uint32_t __byte_perm(uint32_t x, uint32_t y, uint32_t s) {
  const uint64_t v = ((uint64_t)y << 32) | x;
  uint32_t r = 0u;
  for (int k = 0; k < 4; ++k) {
    const uint32_t sel = (s >> (4 * k)) & 7u;
    r |= (uint32_t)((v >> (8 * sel)) & 0xffu) << (8 * k);
  }
  return r;
}

using std::max;
using std::min;
