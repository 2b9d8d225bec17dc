// cuda_runtime.h -- a CPU stand-in for the parts of the CUDA runtime and of
// the device language that the library's kernel source uses, so that
// dls_kernels.cu compiles with the host compiler and runs on the CPU for
// tests/test_host_kernels.py.  Test infrastructure only: the library itself
// is always built with nvcc for sm_103a and never sees this file.
//
// Execution model (simt.cpp): every CUDA thread of a launch is a cooperative
// fiber on one OS thread.  A fiber runs until it reaches a warp intrinsic
// (vote, shuffle, __syncwarp) or __syncthreads and then waits; a warp
// intrinsic completes once every lane of the warp waits at it, a block
// barrier once every live thread of the block does.  All blocks of a grid
// are resident at once and interleave at those points, so the global work
// queue is shared as on the device.  Memory calls are synchronous host
// memory operations; stream capture records the calls and a graph launch
// replays them.
#pragma once

#include <cstddef>
#include <cstdint>
#include <cstring>

#include "shim.h"

#define __global__
#define __launch_bounds__(...)
#define __grid_constant__
#define __align__(n) __attribute__((aligned(n)))

struct dim3 {
  unsigned x, y, z;
  constexpr dim3(unsigned a = 1, unsigned b = 1, unsigned c = 1) : x(a), y(b), z(c) {}
};

// the running fiber's indices (set by the scheduler before it resumes one)
extern dim3 threadIdx, blockIdx, blockDim, gridDim;

// ---------------------------------------------------------- device side --

inline int __ffs(int v) {
  const uint32_t u = (uint32_t)v;
  if (u == 0u) return 0;
  int k = 1;
  while (((u >> (k - 1)) & 1u) == 0u) ++k;
  return k;
}

// no preemption between synchronisation points: a plain add is atomic here
inline unsigned long long atomicAdd(unsigned long long *a, unsigned long long v) {
  const unsigned long long old = *a;
  *a = old + v;
  return old;
}
inline unsigned atomicSub(unsigned *a, unsigned v) {
  const unsigned old = *a;
  *a = old - v;
  return old;
}
inline unsigned atomicOr(unsigned *a, unsigned v) {
  const unsigned old = *a;
  *a = old | v;
  return old;
}
// high 64 bits of the 128-bit product
inline unsigned long long __umul64hi(unsigned long long a, unsigned long long b) {
  return (unsigned long long)(((unsigned __int128)a * b) >> 64);
}
inline unsigned long long atomicOr(unsigned long long *a, unsigned long long v) {
  const unsigned long long old = *a;
  *a = old | v;
  return old;
}

namespace shim {
// warp operations: the calling lane waits until all lanes of its warp call
// the same one
unsigned warp_ballot(unsigned pred);
uint64_t warp_shfl(uint64_t v, int src_lane);
uint64_t warp_shfl_down(uint64_t v, int delta);
void warp_sync();
void block_sync();
// the block's dynamic shared memory, and a block-private array standing in
// for a static __shared__ one (id tells the arrays of a kernel apart)
void *dynamic_smem();
void *block_shared(size_t bytes, int id);

template <class T>
uint64_t to_bits(T v) {
  static_assert(sizeof(T) <= 8, "shuffle of at most 8 bytes");
  uint64_t b = 0;
  std::memcpy(&b, &v, sizeof(T));
  return b;
}
template <class T>
T from_bits(uint64_t b) {
  T v;
  std::memcpy(&v, &b, sizeof(T));
  return v;
}
}  // namespace shim

inline unsigned __ballot_sync(unsigned, int pred) { return shim::warp_ballot(pred ? 1u : 0u); }
inline int __any_sync(unsigned, int pred) { return shim::warp_ballot(pred ? 1u : 0u) != 0u; }
template <class T>
T __shfl_sync(unsigned, T v, int src) {
  return shim::from_bits<T>(shim::warp_shfl(shim::to_bits(v), src));
}
template <class T>
T __shfl_down_sync(unsigned, T v, unsigned delta) {
  return shim::from_bits<T>(shim::warp_shfl_down(shim::to_bits(v), (int)delta));
}
inline void __syncwarp(unsigned = 0xffffffffu) { shim::warp_sync(); }
inline void __syncthreads() { shim::block_sync(); }

// ----------------------------------------------------------- host side --

typedef enum {
  cudaSuccess = 0,
  cudaErrorInvalidValue = 1,
  cudaErrorMemoryAllocation = 2,
} cudaError_t;

struct CUstream_st;
struct CUgraph_st;
struct CUevent_st;
typedef CUstream_st *cudaStream_t;
typedef CUevent_st *cudaEvent_t;
typedef CUgraph_st *cudaGraph_t;
typedef CUgraph_st *cudaGraphExec_t;

enum cudaMemcpyKind {
  cudaMemcpyHostToHost = 0,
  cudaMemcpyHostToDevice = 1,
  cudaMemcpyDeviceToHost = 2,
  cudaMemcpyDeviceToDevice = 3,
  cudaMemcpyDefault = 4
};
enum cudaDeviceAttr {
  cudaDevAttrMultiProcessorCount = 16,
  cudaDevAttrMaxSharedMemoryPerMultiprocessor = 81,
  cudaDevAttrMaxSharedMemoryPerBlockOptin = 97
};
enum cudaFuncAttribute { cudaFuncAttributeMaxDynamicSharedMemorySize = 8 };
enum cudaStreamCaptureMode {
  cudaStreamCaptureModeGlobal = 0,
  cudaStreamCaptureModeThreadLocal = 1,
  cudaStreamCaptureModeRelaxed = 2
};
#define cudaStreamNonBlocking 0x01
#define cudaEventDisableTiming 0x02

const char *cudaGetErrorString(cudaError_t e);
cudaError_t cudaGetDevice(int *dev);
cudaError_t cudaSetDevice(int dev);
cudaError_t cudaDeviceGetAttribute(int *v, cudaDeviceAttr a, int dev);
cudaError_t cudaFuncSetAttribute(const void *fn, cudaFuncAttribute a, int v);
cudaError_t cudaOccupancyMaxActiveBlocksPerMultiprocessor(int *n, const void *fn, int block,
                                                          size_t smem);
// kernels passed by name, as the runtime's template overloads allow
template <class F>
cudaError_t cudaFuncSetAttribute(F *fn, cudaFuncAttribute a, int v) {
  return cudaFuncSetAttribute((const void *)fn, a, v);
}
template <class F>
cudaError_t cudaOccupancyMaxActiveBlocksPerMultiprocessor(int *n, F *fn, int block, size_t smem) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(n, (const void *)fn, block, smem);
}
cudaError_t cudaMalloc(void **p, size_t bytes);
template <class T>
cudaError_t cudaMalloc(T **p, size_t bytes) {
  return cudaMalloc(reinterpret_cast<void **>(p), bytes);
}
cudaError_t cudaFree(void *p);
cudaError_t cudaMallocHost(void **p, size_t bytes);
template <class T>
cudaError_t cudaMallocHost(T **p, size_t bytes) {
  return cudaMallocHost(reinterpret_cast<void **>(p), bytes);
}
cudaError_t cudaFreeHost(void *p);
cudaError_t cudaGetLastError();
// a __device__ variable is an ordinary one here
template <class T>
cudaError_t cudaGetSymbolAddress(void **p, const T &symbol) {
  *p = const_cast<void *>(static_cast<const void *>(&symbol));
  return cudaSuccess;
}
cudaError_t cudaEventCreateWithFlags(cudaEvent_t *e, unsigned flags);
cudaError_t cudaEventRecord(cudaEvent_t e, cudaStream_t s = nullptr);
cudaError_t cudaEventSynchronize(cudaEvent_t e);
cudaError_t cudaEventDestroy(cudaEvent_t e);
cudaError_t cudaMemsetAsync(void *p, int v, size_t bytes, cudaStream_t s = nullptr);
cudaError_t cudaMemcpyAsync(void *dst, const void *src, size_t bytes, cudaMemcpyKind k,
                            cudaStream_t s = nullptr);
cudaError_t cudaMemcpy(void *dst, const void *src, size_t bytes, cudaMemcpyKind k);
cudaError_t cudaStreamSynchronize(cudaStream_t s);
cudaError_t cudaStreamCreateWithFlags(cudaStream_t *s, unsigned flags);
cudaError_t cudaStreamDestroy(cudaStream_t s);
cudaError_t cudaStreamBeginCapture(cudaStream_t s, cudaStreamCaptureMode m);
cudaError_t cudaStreamEndCapture(cudaStream_t s, cudaGraph_t *g);
cudaError_t cudaGraphInstantiate(cudaGraphExec_t *e, cudaGraph_t g, unsigned long long flags);
cudaError_t cudaGraphLaunch(cudaGraphExec_t e, cudaStream_t s);
cudaError_t cudaGraphExecDestroy(cudaGraphExec_t e);
cudaError_t cudaGraphDestroy(cudaGraph_t g);
// defined next to the kernels (it needs their parameter type)
cudaError_t cudaLaunchKernel(const void *fn, dim3 grid, dim3 block, void **args, size_t smem,
                             cudaStream_t s);

#include <functional>

namespace shim {
// Enqueues a launch of `body` on every thread of the grid (run at once, or
// recorded while the stream is being captured).
cudaError_t launch(cudaStream_t s, dim3 grid, dim3 block, size_t smem,
                   std::function<void()> body);
}  // namespace shim
