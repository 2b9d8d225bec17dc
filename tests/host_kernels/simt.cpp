// simt.cpp -- the CPU stand-in behind tests/host_kernels/cuda_runtime.h:
// a cooperative scheduler that runs every CUDA thread of a launch as a
// fiber, the warp and block synchronisation points, and host-memory
// versions of the runtime calls.  Test infrastructure only.
//
// Scheduling: blocks are resident in waves of at most kResident (a
// persistent grid of the stand-in device -- two multiprocessors -- fits in
// one wave, so its blocks share the work queue); the fibers of a wave run
// in turn, each until it reaches a synchronisation point.  When none can
// run, every warp whose live lanes all wait at the same warp operation gets
// its results and runs again, and every block whose live threads all wait
// at __syncthreads is released.  A
// warp operation reached by only some lanes of a warp while the others have
// exited, two different warp operations met at once, or a state where
// nothing can proceed end the program with a message (exit status 4): each
// is a bug in the kernel under test.
#include "cuda_runtime.h"

#include <ucontext.h>

#include <cstdio>
#include <cstdlib>
#include <functional>
#include <map>
#include <memory>
#include <utility>
#include <vector>

dim3 threadIdx, blockIdx, blockDim, gridDim;

struct CUstream_st {
  bool capturing = false;
  std::vector<std::function<void()>> rec;
};
struct CUgraph_st {
  std::vector<std::function<void()>> ops;
};
struct CUevent_st {};

namespace shim {

namespace {

enum State { RUNNABLE, AT_WARP, AT_BLOCK, DONE };
enum Op { OP_BALLOT, OP_SHFL, OP_SHFL_DOWN, OP_SYNCWARP };

constexpr size_t kStack = 64 * 1024;
constexpr unsigned kResident = 8;

struct Fiber {
  ucontext_t ctx;
  std::unique_ptr<char[]> stack;  // left untouched until the fiber runs
  State state = RUNNABLE;
  Op op = OP_SYNCWARP;
  uint64_t val = 0;
  int arg = 0;
  uint64_t res = 0;
  unsigned tid = 0, bid = 0;
};

struct GridRun {
  std::vector<Fiber> f;
  const std::function<void()> *body = nullptr;
  unsigned threads = 0, blocks = 0, first = 0;  // blocks [first, first + blocks)
  std::vector<std::vector<char>> smem;
  std::vector<std::map<int, std::vector<char>>> statics;
  size_t cur = 0;
  ucontext_t sched;
};

GridRun *G = nullptr;

[[noreturn]] void fail(const char *what) {
  std::fprintf(stderr, "simt: %s\n", what);
  std::fflush(stderr);
  std::exit(4);
}

void fiber_entry() {
  (*G->body)();
  G->f[G->cur].state = DONE;  // uc_link returns to the scheduler
}

uint64_t wait_warp(Op op, uint64_t val, int arg) {
  if (G == nullptr) fail("warp operation outside a kernel");
  Fiber &me = G->f[G->cur];
  me.op = op;
  me.val = val;
  me.arg = arg;
  me.state = AT_WARP;
  swapcontext(&me.ctx, &G->sched);
  return G->f[G->cur].res;
}

// Completes the warp operation of warp w of block b if all its live lanes
// wait at it.  Returns true if it did.
bool resolve_warp(unsigned b, unsigned w) {
  const size_t base = (size_t)b * G->threads + (size_t)w * 32u;
  const unsigned lanes = std::min(32u, G->threads - w * 32u);
  unsigned waiting = 0, done = 0;
  for (unsigned l = 0; l < lanes; ++l) {
    const State s = G->f[base + l].state;
    if (s == AT_WARP) ++waiting;
    if (s == DONE) ++done;
  }
  if (waiting == 0 || waiting + done != lanes) return false;
  if (done != 0) fail("warp operation reached while lanes of the warp have exited");
  const Op op = G->f[base].op;
  for (unsigned l = 1; l < lanes; ++l)
    if (G->f[base + l].op != op) fail("lanes of a warp wait at different warp operations");
  if (op == OP_BALLOT) {
    uint64_t m = 0;
    for (unsigned l = 0; l < lanes; ++l) m |= (G->f[base + l].val ? 1ull : 0ull) << l;
    for (unsigned l = 0; l < lanes; ++l) G->f[base + l].res = m;
  } else if (op == OP_SHFL) {
    for (unsigned l = 0; l < lanes; ++l) {
      const unsigned src = (unsigned)G->f[base + l].arg & 31u;
      if (src >= lanes) fail("shuffle from a lane outside the block");
      G->f[base + l].res = G->f[base + src].val;
    }
  } else if (op == OP_SHFL_DOWN) {
    for (unsigned l = 0; l < lanes; ++l) {
      const unsigned src = l + (unsigned)G->f[base + l].arg;
      G->f[base + l].res = src < lanes ? G->f[base + src].val : G->f[base + l].val;
    }
  }
  for (unsigned l = 0; l < lanes; ++l) G->f[base + l].state = RUNNABLE;
  return true;
}

bool resolve_block(unsigned b) {
  const size_t base = (size_t)b * G->threads;
  unsigned waiting = 0, done = 0;
  for (unsigned t = 0; t < G->threads; ++t) {
    const State s = G->f[base + t].state;
    if (s == AT_BLOCK) ++waiting;
    if (s == DONE) ++done;
  }
  if (waiting == 0 || waiting + done != G->threads) return false;
  for (unsigned t = 0; t < G->threads; ++t)
    if (G->f[base + t].state == AT_BLOCK) G->f[base + t].state = RUNNABLE;
  return true;
}

// Runs blocks [first, first + count) of the grid to completion.
void run_wave(unsigned first, unsigned count, dim3 grid, dim3 block, size_t smem,
              const std::function<void()> &body) {
  GridRun run;
  G = &run;
  run.body = &body;
  run.threads = block.x;
  run.blocks = count;
  run.first = first;
  run.smem.assign(count, std::vector<char>(smem, (char)0xcd));
  run.statics.resize(count);
  run.f.resize((size_t)count * block.x);
  for (size_t k = 0; k < run.f.size(); ++k) {
    Fiber &f = run.f[k];
    f.tid = (unsigned)(k % block.x);
    f.bid = first + (unsigned)(k / block.x);
    f.stack.reset(new char[kStack]);
    getcontext(&f.ctx);
    f.ctx.uc_stack.ss_sp = f.stack.get();
    f.ctx.uc_stack.ss_size = kStack;
    f.ctx.uc_link = &run.sched;
    makecontext(&f.ctx, fiber_entry, 0);
  }
  blockDim = block;
  gridDim = grid;
  for (;;) {
    bool ran = false;
    for (size_t k = 0; k < run.f.size(); ++k) {
      if (run.f[k].state != RUNNABLE) continue;
      run.cur = k;
      threadIdx = dim3(run.f[k].tid);
      blockIdx = dim3(run.f[k].bid);
      swapcontext(&run.sched, &run.f[k].ctx);
      ran = true;
    }
    bool released = false;
    for (unsigned b = 0; b < run.blocks; ++b) {
      for (unsigned w = 0; w * 32u < run.threads; ++w) released |= resolve_warp(b, w);
      released |= resolve_block(b);
    }
    bool all_done = true;
    for (const Fiber &f : run.f) all_done = all_done && f.state == DONE;
    if (all_done) break;
    if (!ran && !released) fail("no thread can proceed (a barrier or warp operation that "
                                "some threads never reach)");
  }
  G = nullptr;
}

void run_grid(dim3 grid, dim3 block, size_t smem, const std::function<void()> &body) {
  if (G != nullptr) fail("nested launch");
  if (block.x == 0 || block.y != 1 || block.z != 1 || grid.y != 1 || grid.z != 1)
    fail("launch shape outside what the kernels use");
  for (unsigned first = 0; first < grid.x; first += kResident)
    run_wave(first, std::min(kResident, grid.x - first), grid, block, smem, body);
}

bool capturing(cudaStream_t s) { return s != nullptr && s->capturing; }

cudaError_t enqueue(cudaStream_t s, std::function<void()> op) {
  if (capturing(s))
    s->rec.push_back(std::move(op));
  else
    op();
  return cudaSuccess;
}

}  // namespace

unsigned warp_ballot(unsigned pred) { return (unsigned)wait_warp(OP_BALLOT, pred, 0); }
uint64_t warp_shfl(uint64_t v, int src) { return wait_warp(OP_SHFL, v, src); }
uint64_t warp_shfl_down(uint64_t v, int delta) { return wait_warp(OP_SHFL_DOWN, v, delta); }
void warp_sync() { wait_warp(OP_SYNCWARP, 0, 0); }

void block_sync() {
  if (G == nullptr) fail("__syncthreads outside a kernel");
  Fiber &me = G->f[G->cur];
  me.state = AT_BLOCK;
  swapcontext(&me.ctx, &G->sched);
}

void *dynamic_smem() {
  if (G == nullptr) fail("shared memory outside a kernel");
  std::vector<char> &m = G->smem[blockIdx.x - G->first];
  return m.empty() ? nullptr : m.data();
}

void *block_shared(size_t bytes, int id) {
  if (G == nullptr) fail("shared memory outside a kernel");
  std::vector<char> &m = G->statics[blockIdx.x - G->first][id];
  if (m.empty()) m.assign(bytes, (char)0xcd);
  return m.data();
}

// Runs a launch (called by the cudaLaunchKernel next to the kernels).
cudaError_t launch(cudaStream_t s, dim3 grid, dim3 block, size_t smem,
                   std::function<void()> body) {
  return enqueue(s, [=]() { run_grid(grid, block, smem, body); });
}

}  // namespace shim

// ------------------------------------------------------------- runtime --

const char *cudaGetErrorString(cudaError_t e) {
  return e == cudaSuccess ? "no error" : "emulated CUDA error";
}
cudaError_t cudaGetDevice(int *dev) {
  *dev = 0;
  return cudaSuccess;
}
cudaError_t cudaSetDevice(int) { return cudaSuccess; }
cudaError_t cudaDeviceGetAttribute(int *v, cudaDeviceAttr a, int) {
  // two multiprocessors, so that grids have a few blocks; GB300's shared
  // memory: 227 KB per block (opt-in), 228 KB per SM
  *v = a == cudaDevAttrMultiProcessorCount ? 2
       : a == cudaDevAttrMaxSharedMemoryPerMultiprocessor ? 233472 : 232448;
  return cudaSuccess;
}
cudaError_t cudaFuncSetAttribute(const void *, cudaFuncAttribute, int) { return cudaSuccess; }
cudaError_t cudaOccupancyMaxActiveBlocksPerMultiprocessor(int *n, const void *, int block,
                                                          size_t smem) {
  const size_t per_sm = 233472;
  const size_t by_smem = smem ? per_sm / (smem + 1024) : 32;
  const size_t by_threads = 2048 / (size_t)block;
  *n = (int)std::min<size_t>(2, std::min(by_smem, by_threads));
  return cudaSuccess;
}
cudaError_t cudaMalloc(void **p, size_t bytes) {
  *p = std::malloc(bytes ? bytes : 1);
  if (*p == nullptr) return cudaErrorMemoryAllocation;
  std::memset(*p, 0xa5, bytes);  // device memory starts undefined
  return cudaSuccess;
}
cudaError_t cudaFree(void *p) {
  std::free(p);
  return cudaSuccess;
}
cudaError_t cudaMemsetAsync(void *p, int v, size_t bytes, cudaStream_t s) {
  return shim::enqueue(s, [=]() { std::memset(p, v, bytes); });
}
cudaError_t cudaMemcpyAsync(void *dst, const void *src, size_t bytes, cudaMemcpyKind,
                            cudaStream_t s) {
  return shim::enqueue(s, [=]() { std::memcpy(dst, src, bytes); });
}
cudaError_t cudaMemcpy(void *dst, const void *src, size_t bytes, cudaMemcpyKind) {
  std::memcpy(dst, src, bytes);
  return cudaSuccess;
}
cudaError_t cudaStreamSynchronize(cudaStream_t) { return cudaSuccess; }
cudaError_t cudaMallocHost(void **p, size_t bytes) {
  *p = std::malloc(bytes ? bytes : 1);
  return *p ? cudaSuccess : cudaErrorMemoryAllocation;
}
cudaError_t cudaFreeHost(void *p) {
  std::free(p);
  return cudaSuccess;
}
cudaError_t cudaGetLastError() { return cudaSuccess; }
// every call completes before it returns, so an event is always reached
cudaError_t cudaEventCreateWithFlags(cudaEvent_t *e, unsigned) {
  *e = new CUevent_st();
  return cudaSuccess;
}
cudaError_t cudaEventRecord(cudaEvent_t, cudaStream_t) { return cudaSuccess; }
cudaError_t cudaEventSynchronize(cudaEvent_t) { return cudaSuccess; }
cudaError_t cudaEventDestroy(cudaEvent_t e) {
  delete e;
  return cudaSuccess;
}
cudaError_t cudaStreamCreateWithFlags(cudaStream_t *s, unsigned) {
  *s = new CUstream_st();
  return cudaSuccess;
}
cudaError_t cudaStreamDestroy(cudaStream_t s) {
  delete s;
  return cudaSuccess;
}
cudaError_t cudaStreamBeginCapture(cudaStream_t s, cudaStreamCaptureMode) {
  if (s == nullptr || s->capturing) return cudaErrorInvalidValue;
  s->capturing = true;
  s->rec.clear();
  return cudaSuccess;
}
cudaError_t cudaStreamEndCapture(cudaStream_t s, cudaGraph_t *g) {
  if (s == nullptr || !s->capturing) return cudaErrorInvalidValue;
  s->capturing = false;
  *g = new CUgraph_st();
  (*g)->ops.swap(s->rec);
  return cudaSuccess;
}
cudaError_t cudaGraphInstantiate(cudaGraphExec_t *e, cudaGraph_t g, unsigned long long) {
  *e = new CUgraph_st(*g);
  return cudaSuccess;
}
cudaError_t cudaGraphLaunch(cudaGraphExec_t e, cudaStream_t s) {
  const std::vector<std::function<void()>> ops = e->ops;
  return shim::enqueue(s, [ops]() {
    for (const auto &op : ops) op();
  });
}
cudaError_t cudaGraphExecDestroy(cudaGraphExec_t e) {
  delete e;
  return cudaSuccess;
}
cudaError_t cudaGraphDestroy(cudaGraph_t g) {
  delete g;
  return cudaSuccess;
}
