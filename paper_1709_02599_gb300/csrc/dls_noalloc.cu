// dls_noalloc.cu -- dls_count_host_noalloc(): the host-buffer count without
// any device allocation.
//
// Why: dls_count_host() stages the caller's prefixes and counts in device
// buffers that the library cudaMalloc()s on first use, and the persistent
// kernel's work-queue head lives in another small allocation.  Some callers
// cannot let a library do that: code that owns all of the device memory
// through its own pool (a framework that reserved the GPU up front, so a
// foreign cudaMalloc fails or breaks its budget), and code on a
// latency-critical path that must never hit the implicit device
// synchronisation of cudaMalloc/cudaFree.  This entry point keeps the staged
// prefixes, the staged counts and the queue head in one fixed array compiled
// into the library instead, so a call allocates nothing on the device.
//
// The array is NOALLOC_SCRATCH_BYTES (4 MiB) of device memory that every GPU
// which loads the library holds until the process exits.  A call needs
// 256 bytes (queue head) + n_prefixes * depth rounded up to 256 + 8 bytes per
// prefix; larger calls are rejected with DLS_ERR_CAPACITY before anything
// is copied.  Every call shares the array and it keeps the last call's
// contents; the call clears the queue head and the counts itself.  Calls
// that overlap on the GPU (two host threads, or two streams, at once) race on
// the array and give wrong counts: serialise them.
//
// The device address of the array is looked up once per device with
// cudaGetSymbolAddress() on the first call made while that device is
// current (the host-side symbol is only a stand-in and must never be handed
// to a kernel).  That first call is synchronous like every call of this
// entry point; make it before any stream capture.  dls_release() forgets
// the addresses; after cudaDeviceReset() call it before the next call, since
// the array can then live at another address.

#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <vector>

#include "dls_internal.h"

namespace dls {

// declared in dls_kernels.cu
int enqueue_count_with_scratch(int n, uint32_t flags, const uint8_t *order,
                               int order_len, const uint8_t *d_prefixes,
                               int depth, int64_t n_prefixes,
                               uint64_t *d_counts, const dls_launch_t *cfg,
                               cudaStream_t stream,
                               unsigned long long *scratch);

constexpr size_t NOALLOC_SCRATCH_BYTES = DLS_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];

static std::mutex g_noalloc_mutex;
static std::map<int, unsigned char *> g_noalloc_addr;  // device -> address

static int noalloc_address(unsigned char **out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    set_cuda_error(cudaGetErrorString(e));
    return DLS_ERR_CUDA;
  }
  std::lock_guard<std::mutex> g(g_noalloc_mutex);
  auto it = g_noalloc_addr.find(dev);
  if (it == g_noalloc_addr.end()) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || p == nullptr) {
      set_cuda_error(cudaGetErrorString(e));
      return DLS_ERR_CUDA;
    }
    it = g_noalloc_addr.emplace(dev, static_cast<unsigned char *>(p)).first;
  }
  *out = it->second;
  return DLS_OK;
}

static size_t round256(size_t x) { return (x + 255u) & ~size_t(255u); }

// Forgets the looked-up addresses (dls_release): after a device reset the
// library's module can be loaded again at another address.
void noalloc_forget() {
  std::lock_guard<std::mutex> g(g_noalloc_mutex);
  g_noalloc_addr.clear();
}

}  // namespace dls

using namespace dls;

extern "C" {

int dls_count_host_noalloc(int n, uint32_t flags, const uint8_t *order,
                           int order_len, const uint8_t *h_prefixes, int depth,
                           int64_t n_prefixes, uint64_t *h_counts,
                           dls_u128 *total_out, const dls_launch_t *cfg,
                           void *stream) {
  if (n_prefixes < 0 || depth < 0) return DLS_ERR_BAD_ARG;
  if (n_prefixes > 0 && depth > 0 && h_prefixes == nullptr) return DLS_ERR_BAD_ARG;
  if (n_prefixes > 0 && h_counts == nullptr && total_out == nullptr)
    return DLS_ERR_BAD_ARG;
  const size_t in_bytes = (size_t)n_prefixes * (size_t)depth;
  const size_t need = 256u + round256(in_bytes) + (size_t)n_prefixes * sizeof(uint64_t);
  if ((double)n_prefixes * (depth + 8.0) > (double)NOALLOC_SCRATCH_BYTES ||
      need > NOALLOC_SCRATCH_BYTES)
    return DLS_ERR_CAPACITY;
  unsigned char *base = nullptr;
  int rc = noalloc_address(&base);
  if (rc) return rc;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  unsigned long long *queue = reinterpret_cast<unsigned long long *>(base);
  uint8_t *d_pre = base + 256;
  uint64_t *d_counts = reinterpret_cast<uint64_t *>(base + 256 + round256(in_bytes));
  cudaError_t e;
  if (in_bytes) {
    e = cudaMemcpyAsync(d_pre, h_prefixes, in_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      set_cuda_error(cudaGetErrorString(e));
      return DLS_ERR_CUDA;
    }
  }
  // word 1 of the array is the count's status word (the snapshot search's
  // stack-overflow flag); the launch clears it, and it is read back with the
  // counts
  rc = enqueue_count_with_scratch(n, flags, order, order_len, d_pre, depth, n_prefixes,
                                  d_counts, cfg, st, queue);
  if (rc) return rc;
  std::vector<uint64_t> tmp;
  uint64_t *host_counts = h_counts;
  if (host_counts == nullptr && n_prefixes > 0) {
    tmp.resize((size_t)n_prefixes);
    host_counts = tmp.data();
  }
  if (n_prefixes > 0) {
    e = cudaMemcpyAsync(host_counts, d_counts, (size_t)n_prefixes * sizeof(uint64_t),
                        cudaMemcpyDeviceToHost, st);
    if (e != cudaSuccess) {
      set_cuda_error(cudaGetErrorString(e));
      return DLS_ERR_CUDA;
    }
  }
  unsigned long long status = 0ull;
  e = cudaMemcpyAsync(&status, queue + 1, sizeof(status), cudaMemcpyDeviceToHost, st);
  if (e != cudaSuccess) {
    set_cuda_error(cudaGetErrorString(e));
    return DLS_ERR_CUDA;
  }
  e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    set_cuda_error(cudaGetErrorString(e));
    return DLS_ERR_CUDA;
  }
  // a stack overflow (the kernel dropped a stack entry rather than write past
  // its stack) makes the counts untrustworthy, as dls_count_host reports it
  rc = status_code((unsigned)status);
  if (rc) return rc;
  if (total_out) {
    dls_u128 t = {0, 0};
    for (int64_t k = 0; k < n_prefixes; ++k) t = dls_add_u128(t, dls_u128{host_counts[k], 0});
    *total_out = t;
  }
  return DLS_OK;
}

}  // extern "C"
