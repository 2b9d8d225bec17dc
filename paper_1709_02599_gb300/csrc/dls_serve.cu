// dls_serve.cu -- continuous-batching server for counting jobs of mixed
// order, flags and prefix.
//
// A job is one count: an order n, flags, a fill order and one prefix; its
// answer is Count(prefix) as defined in dls.h.  At submission the host splits
// the job into work items -- the valid extensions of its prefix a few cells
// deeper (the prefix split of Section 5.2) -- and queues it.  Each call of
// dls_server_step() is one epoch:
//   1. results of the previous epoch are read: a job whose items are all
//      finished is complete, and its job slot and arena chunks are freed;
//   2. queued jobs are admitted in arrival order while a job slot, enough
//      free chunks of the device item arena (the memory budget) and queue
//      room are available; their items are copied to the arena and appended
//      to the device work queue;
//   3. one launch of k_serve runs every lane of a resident grid for a fixed
//      number of search iterations.  A lane resumes the search it saved at
//      the end of the previous epoch, or takes the next queued item of any
//      job; when an item is finished its count is added to the job's counter
//      and the job's remaining-item counter is decremented.  At the end of
//      the epoch every unfinished search (position, candidate stack, row /
//      column / diagonal words, partial count) is written back to the lane's
//      slot in device memory.
// Jobs that arrive while others are on the GPU therefore start at the next
// epoch boundary and share the device with them; search stacks and counters
// stay on the device between epochs.  The search itself is Algorithm 4 as in
// dls_kernels.cu, with the order, flags and size read per lane from the job
// table so that lanes of one warp may work on different jobs.

#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <vector>

#include "dls_internal.h"
#include "dls_search.cuh"

namespace dls {

constexpr int SV_WORDS = 2 * DLS_MAX_N;   // row words 0..15, column words 16..31
constexpr int SV_HDR = 10;                // slot header words

struct ServeJob {            // device job descriptor
  Geo g;                     // order size, admissible values, item length, last
  uint32_t flags;
  int order_len;
  Cell cells[DLS_MAX_CELLS]; // descriptor of each order position (shared-memory
                             // words, column words from word 16)
};

struct ServeParams {
  const ServeJob *jobs;
  unsigned long long *job_count;   // per slot: completions found so far
  unsigned int *job_left;          // per slot: items not finished
  const uint8_t *arena;            // item prefixes
  const uint2 *queue;              // (job slot, arena byte offset)
  unsigned long long *head;        // items handed out (device counter)
  unsigned long long tail;         // items queued so far
  unsigned long long qcap;         // queue ring capacity
  uint32_t *slots;                 // lane slots, word w of lane g at w * G + g
  long long G;                     // lanes in the grid
  int budget;                      // search iterations per lane per epoch
};

// A lane of the server: the search state plus its job's shape.
struct SvLane {
  Lane<false> s;
  int job;          // job slot, -1 = idle
  bool vsym;
  Geo g;
  const Cell *tbl;  // the job's descriptor table (global memory)
};

__device__ __forceinline__ void sv_bind(SvLane &l, const ServeParams &P, int job) {
  const ServeJob &J = P.jobs[job];
  l.job = job;
  l.g = J.g;
  l.vsym = (J.flags & DLS_VSYM) != 0;
  l.tbl = J.cells;
}

// Finishes an item: its count goes to the job, one item fewer is left.
__device__ __forceinline__ void sv_finish(SvLane &l, const ServeParams &P) {
  if (l.s.cnt) atomicAdd(P.job_count + l.job, l.s.cnt);
  atomicSub(P.job_left + l.job, 1u);
  l.job = -1;
}

// Loads an item; returns true if the lane now has a search to run.
__device__ bool sv_load(SvLane &l, const ServeParams &P, uint2 item, unsigned B) {
  sv_bind(l, P, (int)item.x);
  Lane<false> &s = l.s;
  s.cnt = 0ull;
  s.w.clear(SV_WORDS, B);
  const uint8_t *rec = P.arena + item.y;
  const bool ok = l.vsym ? place_prefix<false, true>(s.w, l.g, rec, l.tbl)
                         : place_prefix<false, false>(s.w, l.g, rec, l.tbl);
  if (!ok) {
    sv_finish(l, P);
    return false;
  }
  const int order_len = l.g.last + 1;
  if (l.g.depth == order_len) {
    s.cnt = 1ull;
    sv_finish(l, P);
    return false;
  }
  s.info = l.tbl[l.g.depth];
  s.L = l.vsym ? s.w.template cands<true>(s.info, l.g) : s.w.template cands<false>(s.info, l.g);
  if (l.g.depth == l.g.last || s.L == 0u) {
    s.cnt = (l.g.depth == l.g.last) ? (unsigned)__popc(s.L) : 0ull;
    sv_finish(l, P);
    return false;
  }
  s.p = l.g.depth;
  s.v = 0u;
  return true;
}

// Items handed out beyond the queued ones are taken back after an epoch
// (their fetches failed), so the next epoch starts at the first unserved item.
__global__ void k_serve_clamp(unsigned long long *head, unsigned long long tail) {
  if (*head > tail) *head = tail;
}

// Shared memory per lane: SV_WORDS words + the stack, thread-minor.
__global__ void __launch_bounds__(256) k_serve(const __grid_constant__ ServeParams P) {
  extern __shared__ uint32_t smem[];
  const unsigned B = blockDim.x;
  const long long gl = (long long)blockIdx.x * B + threadIdx.x;
  uint32_t *stk = smem + SV_WORDS * B + threadIdx.x;
  uint32_t *slot = P.slots + gl;
  const long long G = P.G;
  const Split nosplit = {-1, 0};

  SvLane l;
  l.s.w.tb = reinterpret_cast<char *>(smem + threadIdx.x);
  l.s.w.R = l.s.w.C = 0ull;
  l.s.nodes = 0ull;
  l.job = -1;
  bool busy = slot[0] != 0u;
  if (busy) {
    sv_bind(l, P, (int)slot[1 * G]);
    Lane<false> &s = l.s;
    s.p = (int)slot[2 * G];
    s.L = slot[3 * G];
    s.v = slot[4 * G];
    s.w.dg = slot[5 * G];
    s.cnt = (unsigned long long)slot[7 * G] | ((unsigned long long)slot[8 * G] << 32);
    for (int w = 0; w < SV_WORDS; ++w) word_at(s.w.tb, (uint32_t)w * B * 4u) = slot[(SV_HDR + w) * G];
    for (int k = 0; k < s.p - l.g.depth; ++k) stk[k * B] = slot[(SV_HDR + SV_WORDS + k) * G];
    s.info = l.tbl[s.p];
  }
  // The epoch: idle lanes of a warp take queued items together (one atomic
  // per warp); while every lane of the warp is busy it steps until one
  // finishes; once the queue is drained the remaining searches step on.
  // Lanes may serve different jobs: one step body decides vertical symmetry
  // from the job at run time, so the warp never splits on it.
  const int lane = threadIdx.x & 31;
  bool drained = false;
  int it = 0;
  while (it < P.budget) {
    unsigned idle = __ballot_sync(FULL, !busy);
    if (idle != 0u && !drained) {
      const int nidle = __popc(idle);
      unsigned long long base = 0ull;
      if (lane == 0) base = atomicAdd(P.head, (unsigned long long)nidle);
      base = __shfl_sync(FULL, base, 0);
      if (!busy) {
        const unsigned long long idx = base + (unsigned)__popc(idle & ((1u << lane) - 1u));
        if (idx < P.tail) busy = sv_load(l, P, P.queue[idx % P.qcap], B);
      }
      if (base + (unsigned long long)nidle >= P.tail) drained = true;
      ++it;
      continue;
    }
    if (idle == FULL) break;  // drained and nothing left to search
    uint32_t *sbase = stk - l.g.depth * (int)B;
    bool fin = false;
    if (idle == 0u) {
      do {
        fin = dfs_step<false, false, false, false, true>(l.s, l.g, nosplit, sbase, l.tbl, B);
        ++it;
      } while (!__any_sync(FULL, fin) && it < P.budget);
    } else {
      if (busy) fin = dfs_step<false, false, false, false, true>(l.s, l.g, nosplit, sbase, l.tbl, B);
      ++it;
    }
    if (fin) {
      sv_finish(l, P);
      busy = false;
    }
  }
  slot[0] = busy ? 1u : 0u;
  if (busy) {
    const Lane<false> &s = l.s;
    slot[1 * G] = (uint32_t)l.job;
    slot[2 * G] = (uint32_t)s.p;
    slot[3 * G] = s.L;
    slot[4 * G] = s.v;
    slot[5 * G] = s.w.dg;
    slot[7 * G] = (uint32_t)s.cnt;
    slot[8 * G] = (uint32_t)(s.cnt >> 32);
    for (int w = 0; w < SV_WORDS; ++w) slot[(SV_HDR + w) * G] = word_at(s.w.tb, (uint32_t)w * B * 4u);
    for (int k = 0; k < s.p - l.g.depth; ++k) slot[(SV_HDR + SV_WORDS + k) * G] = stk[k * B];
  }
}

}  // namespace dls

using namespace dls;

// ------------------------------------------------------------ host side --

struct HostJob {
  int64_t id;
  int slot = -1;
  int n;
  uint32_t flags;
  std::vector<uint8_t> order;   // 2 * order_len
  int depth;                    // item length
  std::vector<uint8_t> items;   // n_items * depth
  int64_t n_items;
  int64_t fed = 0;              // items appended to the device queue so far
  size_t per_chunk = 0;         // items per arena chunk
  double est_nodes = 0.0;       // estimated search nodes of the whole job
  std::vector<int> chunks;
};

struct dls_server {
  dls_server_cfg cfg;
  int dev = 0;
  cudaStream_t stream = nullptr;
  // device
  ServeJob *d_jobs = nullptr;
  unsigned long long *d_count = nullptr;
  unsigned int *d_left = nullptr;
  uint8_t *d_arena = nullptr;
  uint2 *d_queue = nullptr;
  unsigned long long *d_head = nullptr;
  uint32_t *d_slots = nullptr;
  long long G = 0;
  int grid = 0;
  size_t smem = 0;
  // host
  ServeJob *h_job_stage = nullptr;       // pinned, one per slot
  unsigned long long *h_count = nullptr; // pinned readback
  unsigned int *h_left = nullptr;
  uint8_t *h_item_stage = nullptr;       // pinned, arena-sized staging
  uint2 *h_queue_stage = nullptr;        // pinned, queue-sized staging
  unsigned long long *h_zero = nullptr;
  unsigned long long *h_head = nullptr;  // pinned readback of the queue head
  unsigned long long tail = 0;
  unsigned long long head_known = 0;     // queue head after the last epoch
  unsigned long long taken_last = 0;     // items handed out in the last epoch
  int64_t finished_done = 0;             // items of completed jobs
  std::vector<int> free_slots;
  std::vector<int> free_chunks;
  std::vector<HostJob *> active;         // by slot
  std::deque<HostJob *> pending;
  std::vector<std::pair<int64_t, uint64_t>> done;
  int64_t next_id = 0;
  bool in_flight = false;
  cudaEvent_t ev = nullptr;
  dls_server_stats stats;
  std::mutex mu;
  // submitted jobs are split on worker threads, off the caller's path
  std::deque<HostJob *> to_split;
  int64_t splitting = 0;                 // submitted, not yet pending or done
  std::condition_variable cv;
  bool stopping = false;
  std::vector<std::thread> workers;
  // set by dls_server_abort from any thread; read without the lock
  std::atomic<bool> aborted{false};
};

// Splits a submitted job into work items (worker thread, no lock held but
// at the end): the prefix is extended a few cells deeper (Section 5.2), at
// most to two cells before the end, until there are enough items -- one per
// lane, or more for a big job: its estimated search nodes / item_nodes, at
// most items_per_job -- so that no item of a big job is long, while small
// jobs are not cut finer than the grid needs; and never beyond half the
// item arena, so that every job can be admitted.  Then the job waits for
// admission (or completes at once if nothing is left for the GPU).
static void sv_split(dls_server *s, HostJob *j) {
  const int n = j->n;
  const uint32_t flags = j->flags;
  const int order_len = (int)(j->order.size() / 2);
  const uint8_t *order = j->order.data();
  OrderInfo info;
  int rc = validate_order(n, flags, order, order_len, &info);
  std::vector<uint8_t> cur;
  cur.swap(j->items);
  int d = j->depth;
  int64_t m = 0;
  if (rc == DLS_OK && !vsym_all_zero(n, flags)) {
    int64_t need = 0;
    rc = dls_extend_prefixes(n, flags, order, order_len, cur.data(), d, 1, d, nullptr, 0,
                             nullptr, &need);
    m = (rc == DLS_OK || rc == DLS_ERR_CAPACITY) ? need : 0;  // 1 if the prefix is valid
    int64_t target = std::min<int64_t>(s->G, s->cfg.items_per_job);
    if (m > 0) {
      const double est = estimate_nodes(info, cur.data(), d, splitmix64((uint64_t)j->id), 256);
      j->est_nodes = est;
      const double want = est / (double)s->cfg.item_nodes;
      if (want > (double)target)
        target = (int64_t)std::min<double>(want, (double)s->cfg.items_per_job);
    }
    std::vector<uint8_t> next;
    while (m > 0 && m < target && d < order_len - 2) {
      rc = dls_extend_prefixes(n, flags, order, order_len, cur.data(), d, m, d + 1,
                               nullptr, 0, nullptr, &need);
      if ((rc != DLS_OK && rc != DLS_ERR_CAPACITY) ||
          (double)need * (d + 1) > 0.5 * (double)s->cfg.arena_bytes)
        break;
      next.assign((size_t)need * (d + 1), 0);
      int64_t got = 0;
      rc = dls_extend_prefixes(n, flags, order, order_len, cur.data(), d, m, d + 1,
                               next.data(), need, nullptr, &got);
      if (rc) break;
      cur.swap(next);
      ++d;
      m = got;
    }
  }
  if (m == 0) cur.clear();
  j->depth = d;
  j->n_items = m;
  j->items.swap(cur);
  std::lock_guard<std::mutex> g(s->mu);
  s->splitting--;
  if (m == 0 || d == order_len) {
    // nothing for the GPU: no valid extension, or complete assignments
    s->done.push_back({j->id, (uint64_t)(d == order_len ? m : 0)});
    s->stats.completed++;
    s->stats.squares += (uint64_t)(d == order_len ? m : 0);
    delete j;
    return;
  }
  s->pending.push_back(j);
}

static void sv_worker(dls_server *s) {
  for (;;) {
    HostJob *j = nullptr;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      s->cv.wait(lk, [&] { return s->stopping || !s->to_split.empty(); });
      if (s->stopping) return;
      j = s->to_split.front();
      s->to_split.pop_front();
    }
    sv_split(s, j);
  }
}

static int sv_fail(cudaError_t e) {
  set_cuda_error(cudaGetErrorString(e));
  return e == cudaErrorMemoryAllocation ? DLS_ERR_NO_MEMORY : DLS_ERR_CUDA;
}

static void sv_free(dls_server *s) {
  {
    std::lock_guard<std::mutex> g(s->mu);
    s->stopping = true;
  }
  s->cv.notify_all();
  for (auto &t : s->workers) t.join();
  for (auto *j : s->to_split) delete j;
  if (s->ev) cudaEventDestroy(s->ev);
  if (s->stream) cudaStreamDestroy(s->stream);
  cudaFree(s->d_jobs);
  cudaFree(s->d_count);
  cudaFree(s->d_left);
  cudaFree(s->d_arena);
  cudaFree(s->d_queue);
  cudaFree(s->d_head);
  cudaFree(s->d_slots);
  cudaFreeHost(s->h_job_stage);
  cudaFreeHost(s->h_count);
  cudaFreeHost(s->h_left);
  cudaFreeHost(s->h_item_stage);
  cudaFreeHost(s->h_queue_stage);
  cudaFreeHost(s->h_zero);
  cudaFreeHost(s->h_head);
  for (auto *j : s->active) delete j;
  for (auto *j : s->pending) delete j;
  delete s;
}

extern "C" {

void dls_server_default_cfg(dls_server_cfg *cfg) {
  if (!cfg) return;
  std::memset(cfg, 0, sizeof(*cfg));
  cfg->max_jobs = 1024;
  cfg->arena_bytes = size_t(256) << 20;
  cfg->chunk_bytes = size_t(64) << 10;
  cfg->queue_items = int64_t(1) << 22;
  cfg->max_order = 10;
  cfg->budget = 4096;
  cfg->block_threads = 128;
  cfg->blocks_per_sm = 0;
  cfg->items_per_job = 0;
  cfg->min_backlog = 1024;
  cfg->item_nodes = int64_t(1) << 17;
}

int dls_server_create(const dls_server_cfg *cfg_in, dls_server **out) {
  if (out == nullptr) return DLS_ERR_BAD_ARG;
  *out = nullptr;
  dls_server_cfg cfg;
  dls_server_default_cfg(&cfg);
  if (cfg_in) cfg = *cfg_in;
  if (cfg.max_jobs < 1 || cfg.chunk_bytes < 256 || cfg.arena_bytes < cfg.chunk_bytes ||
      cfg.queue_items < 1 || cfg.max_order < 1 || cfg.max_order > DLS_MAX_N ||
      cfg.budget < 1 || cfg.block_threads < 32 || cfg.block_threads > 256 ||
      cfg.block_threads % 32 || cfg.items_per_job < 0 || cfg.blocks_per_sm < 0 ||
      cfg.min_backlog < 1 || cfg.item_nodes < 1)
    return DLS_ERR_BAD_ARG;
  dls_server *s = new (std::nothrow) dls_server();
  if (!s) return DLS_ERR_NO_MEMORY;
  s->cfg = cfg;
  std::memset(&s->stats, 0, sizeof(s->stats));
  cudaError_t e = cudaGetDevice(&s->dev);
  const int stack_words = cfg.max_order * cfg.max_order;
  const int slot_words = SV_HDR + SV_WORDS + stack_words;
  const size_t n_chunks = cfg.arena_bytes / cfg.chunk_bytes;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&s->ev, cudaEventDisableTiming);
  int sms = 0, per_sm = 0;
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, s->dev);
  s->smem = (size_t)(SV_WORDS + stack_words) * cfg.block_threads * 4u;
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(k_serve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s->smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_serve, cfg.block_threads, s->smem);
  if (e == cudaSuccess && per_sm < 1) {
    sv_free(s);
    return DLS_ERR_NO_MEMORY;
  }
  if (e == cudaSuccess) {
    if (cfg.blocks_per_sm) per_sm = std::min(per_sm, cfg.blocks_per_sm);
    s->grid = sms * per_sm;
    s->G = (long long)s->grid * cfg.block_threads;
    // by default a job may be split into up to 16 items per lane: a big
    // job's slowest item, which bounds its latency, is then a small part of it
    if (s->cfg.items_per_job == 0)
      s->cfg.items_per_job = (int)std::min<long long>(16 * s->G, 1 << 22);
  }
  if (e == cudaSuccess) e = cudaMalloc(&s->d_jobs, sizeof(ServeJob) * cfg.max_jobs);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_count, sizeof(unsigned long long) * cfg.max_jobs);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_left, sizeof(unsigned int) * cfg.max_jobs);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_arena, n_chunks * cfg.chunk_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_queue, sizeof(uint2) * cfg.queue_items);
  if (e == cudaSuccess) e = cudaMalloc(&s->d_head, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMalloc(&s->d_slots, sizeof(uint32_t) * (size_t)slot_words * s->G);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_job_stage, sizeof(ServeJob) * cfg.max_jobs);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_count, sizeof(unsigned long long) * cfg.max_jobs);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_left, sizeof(unsigned int) * cfg.max_jobs);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_item_stage, n_chunks * cfg.chunk_bytes);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_queue_stage, sizeof(uint2) * cfg.queue_items);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_zero, 64);
  if (e == cudaSuccess) e = cudaMallocHost(&s->h_head, sizeof(unsigned long long));
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_head, 0, sizeof(unsigned long long), s->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(s->d_slots, 0, sizeof(uint32_t) * s->G, s->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) {
    int rc = sv_fail(e);
    sv_free(s);
    return rc;
  }
  std::memset(s->h_zero, 0, 64);
  *s->h_head = 0ull;
  for (int k = cfg.max_jobs - 1; k >= 0; --k) s->free_slots.push_back(k);
  for (int k = (int)n_chunks - 1; k >= 0; --k) s->free_chunks.push_back(k);
  s->active.assign(cfg.max_jobs, nullptr);
  const unsigned hw = std::thread::hardware_concurrency();
  const int n_workers = (int)std::max(1u, std::min(4u, hw ? hw / 2 : 1u));
  for (int w = 0; w < n_workers; ++w) s->workers.emplace_back(sv_worker, s);
  s->stats.lanes = s->G;
  s->stats.device_bytes = sizeof(ServeJob) * cfg.max_jobs + 12u * cfg.max_jobs +
                          n_chunks * cfg.chunk_bytes + sizeof(uint2) * cfg.queue_items +
                          sizeof(uint32_t) * (size_t)slot_words * s->G;
  *out = s;
  return DLS_OK;
}

int dls_server_submit(dls_server *s, int n, uint32_t flags, const uint8_t *order,
                      int order_len, const uint8_t *prefix, int depth,
                      int64_t *job_id) {
  if (s == nullptr || job_id == nullptr) return DLS_ERR_BAD_ARG;
  if (s->aborted.load()) return DLS_ERR_ABORTED;
  OrderInfo info;
  int rc = validate_order(n, flags, order, order_len, &info);
  if (rc) return rc;
  if (n > s->cfg.max_order) return DLS_ERR_INVALID_N;
  if (depth < 0 || depth > order_len || (depth > 0 && prefix == nullptr)) return DLS_ERR_BAD_ARG;
  HostJob *j = new (std::nothrow) HostJob();
  if (!j) return DLS_ERR_NO_MEMORY;
  j->n = n;
  j->flags = flags;
  j->order.assign(order, order + 2 * order_len);
  j->items.assign(prefix, prefix + depth);  // the prefix, until it is split
  j->depth = depth;
  {
    std::lock_guard<std::mutex> g(s->mu);
    j->id = s->next_id++;
    *job_id = j->id;
    s->stats.submitted++;
    s->to_split.push_back(j);
    s->splitting++;
  }
  s->cv.notify_one();
  return DLS_OK;
}

// Reads the finished epoch's counters; completes jobs whose items are done.
static int sv_collect(dls_server *s) {
  if (!s->in_flight) return DLS_OK;
  cudaError_t e = cudaEventSynchronize(s->ev);
  if (e != cudaSuccess) return sv_fail(e);
  s->in_flight = false;
  s->taken_last = *s->h_head - s->head_known;
  s->head_known = *s->h_head;
  for (int slot = 0; slot < s->cfg.max_jobs; ++slot) {
    HostJob *j = s->active[slot];
    if (j == nullptr || s->h_left[slot] != 0u) continue;
    s->done.push_back({j->id, (uint64_t)s->h_count[slot]});
    s->stats.completed++;
    s->stats.squares += s->h_count[slot];
    s->finished_done += j->n_items;
    for (int c : j->chunks) s->free_chunks.push_back(c);
    s->free_slots.push_back(slot);
    s->active[slot] = nullptr;
    delete j;
  }
  return DLS_OK;
}

int dls_server_step(dls_server *s) {
  if (s == nullptr) return DLS_ERR_BAD_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  int rc = sv_collect(s);
  if (rc) return rc;
  if (s->aborted.load()) return DLS_ERR_ABORTED;  // no further epoch
  cudaError_t e;
  int prev;
  if (cudaGetDevice(&prev) == cudaSuccess && prev != s->dev) cudaSetDevice(s->dev);
  // admission, in arrival order, by job slots, arena chunks and queue room
  size_t qn = 0;
  unsigned long long q0 = s->tail;
  while (!s->pending.empty()) {
    HostJob *j = s->pending.front();
    const size_t per_chunk = s->cfg.chunk_bytes / (size_t)j->depth;
    const size_t need = (size_t)((j->n_items + (int64_t)per_chunk - 1) / (int64_t)per_chunk);
    if (s->free_slots.empty() || s->free_chunks.size() < need) break;
    s->pending.pop_front();
    j->slot = s->free_slots.back();
    s->free_slots.pop_back();
    ServeJob &dj = s->h_job_stage[j->slot];
    std::memset(&dj, 0, sizeof(dj));
    dj.flags = j->flags;
    dj.order_len = (int)(j->order.size() / 2);
    dj.g.n = j->n;
    dj.g.all = (1u << j->n) - 1u;
    // odd order with vertical symmetry: no left cell may hold (n-1)/2
    if ((j->flags & DLS_VSYM) && (j->n & 1)) dj.g.all &= ~(1u << (j->n / 2));
    dj.g.pairmask = (1u << (j->n / 2)) - 1u;
    dj.g.vsmask = (j->flags & DLS_VSYM) ? 0xffffffffu : 0u;
    dj.g.depth = j->depth;
    dj.g.last = dj.order_len - 1;
    for (int t = 0; t < dj.order_len; ++t)
      dj.cells[t] = describe_shared(j->order[2 * t], j->order[2 * t + 1], j->n,
                                    (j->flags & DLS_DIAGONAL) != 0,
                                    (unsigned)s->cfg.block_threads, DLS_MAX_N);
    s->h_count[j->slot] = 0ull;
    s->h_left[j->slot] = (unsigned int)j->n_items;
    e = cudaMemcpyAsync(s->d_jobs + j->slot, &dj, sizeof(ServeJob), cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->d_count + j->slot, s->h_count + j->slot, sizeof(unsigned long long),
                          cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(s->d_left + j->slot, s->h_left + j->slot, sizeof(unsigned int),
                          cudaMemcpyHostToDevice, s->stream);
    int64_t k = 0;
    for (size_t c = 0; c < need && e == cudaSuccess; ++c) {
      const int chunk = s->free_chunks.back();
      s->free_chunks.pop_back();
      j->chunks.push_back(chunk);
      const size_t base = (size_t)chunk * s->cfg.chunk_bytes;
      const int64_t take = std::min<int64_t>((int64_t)per_chunk, j->n_items - k);
      std::memcpy(s->h_item_stage + base, j->items.data() + (size_t)k * j->depth,
                  (size_t)take * j->depth);
      e = cudaMemcpyAsync(s->d_arena + base, s->h_item_stage + base, (size_t)take * j->depth,
                          cudaMemcpyHostToDevice, s->stream);
      k += take;
    }
    if (e != cudaSuccess) return sv_fail(e);
    std::vector<uint8_t>().swap(j->items);
    j->per_chunk = per_chunk;
    j->fed = 0;
    s->active[j->slot] = j;
    s->stats.admitted++;
  }
  // feed the device queue: enough items for the lanes that are idle plus a
  // margin for those that free up during the epoch (twice the items taken
  // in the last epoch, at least min_backlog), taken first from the admitted
  // job with the least estimated work not yet fed (shortest remaining work
  // first) -- so a job admitted now is served within an epoch or two even
  // while a big job still has most of its items left, and of two big jobs
  // one finishes first instead of both finishing last
  {
    int64_t finished = s->finished_done;
    std::vector<HostJob *> feed;
    for (int slot = 0; slot < s->cfg.max_jobs; ++slot) {
      HostJob *j = s->active[slot];
      if (j == nullptr) continue;
      finished += j->n_items - (int64_t)s->h_left[slot];
      if (j->fed < j->n_items) feed.push_back(j);
    }
    const long long busy = (long long)s->head_known - (long long)finished;
    const long long idle = std::max(0ll, (long long)s->G - std::max(0ll, busy));
    const long long backlog = (long long)(s->tail - s->head_known);
    const long long margin = std::max<long long>(s->cfg.min_backlog, 2 * (long long)s->taken_last);
    const long long room = (long long)s->cfg.queue_items - backlog;
    long long want = std::min(room, idle + margin - backlog);
    auto unfed_work = [](const HostJob *j) {
      return j->est_nodes * (double)(j->n_items - j->fed) / (double)j->n_items;
    };
    std::stable_sort(feed.begin(), feed.end(), [&](const HostJob *a, const HostJob *b) {
      return unfed_work(a) < unfed_work(b);
    });
    for (HostJob *j : feed) {
      if (want <= 0) break;
      const long long take = std::min(want, (long long)(j->n_items - j->fed));
      for (long long t = 0; t < take; ++t) {
        const int64_t item = j->fed + t;
        const size_t base = (size_t)j->chunks[(size_t)(item / (int64_t)j->per_chunk)] *
                                s->cfg.chunk_bytes +
                            (size_t)(item % (int64_t)j->per_chunk) * j->depth;
        const unsigned long long pos = (q0 + qn) % (unsigned long long)s->cfg.queue_items;
        s->h_queue_stage[pos] = make_uint2((unsigned)j->slot, (unsigned)base);
        ++qn;
      }
      j->fed += take;
      want -= take;
    }
  }
  // new queue entries (the ring may wrap)
  if (qn) {
    const unsigned long long cap = (unsigned long long)s->cfg.queue_items;
    const unsigned long long a = q0 % cap;
    const unsigned long long first = std::min<unsigned long long>(qn, cap - a);
    e = cudaMemcpyAsync(s->d_queue + a, s->h_queue_stage + a, first * sizeof(uint2),
                        cudaMemcpyHostToDevice, s->stream);
    if (e == cudaSuccess && first < qn)
      e = cudaMemcpyAsync(s->d_queue, s->h_queue_stage, (qn - first) * sizeof(uint2),
                          cudaMemcpyHostToDevice, s->stream);
    if (e != cudaSuccess) return sv_fail(e);
    s->tail += qn;
  }
  bool any = false;
  for (auto *j : s->active) any = any || (j != nullptr);
  if (!any) return DLS_OK;
  // one epoch
  ServeParams P;
  P.jobs = s->d_jobs;
  P.job_count = s->d_count;
  P.job_left = s->d_left;
  P.arena = s->d_arena;
  P.queue = s->d_queue;
  P.head = s->d_head;
  P.tail = s->tail;
  P.qcap = (unsigned long long)s->cfg.queue_items;
  P.slots = s->d_slots;
  P.G = s->G;
  P.budget = s->cfg.budget;
  k_serve<<<s->grid, s->cfg.block_threads, s->smem, s->stream>>>(P);
  // lanes that found the queue empty advanced the head past the tail
  k_serve_clamp<<<1, 1, 0, s->stream>>>(s->d_head, s->tail);
  e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->h_count, s->d_count, sizeof(unsigned long long) * s->cfg.max_jobs,
                        cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->h_left, s->d_left, sizeof(unsigned int) * s->cfg.max_jobs,
                        cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(s->h_head, s->d_head, sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, s->stream);
  if (e == cudaSuccess) e = cudaEventRecord(s->ev, s->stream);
  if (e != cudaSuccess) return sv_fail(e);
  s->in_flight = true;
  s->stats.epochs++;
  return DLS_OK;
}

int dls_server_poll(dls_server *s, int64_t *ids, uint64_t *counts, int cap, int *n_done) {
  if (s == nullptr || n_done == nullptr || cap < 0 || (cap > 0 && (!ids || !counts)))
    return DLS_ERR_BAD_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  const int k = (int)std::min<size_t>((size_t)cap, s->done.size());
  for (int t = 0; t < k; ++t) {
    ids[t] = s->done[t].first;
    counts[t] = s->done[t].second;
  }
  s->done.erase(s->done.begin(), s->done.begin() + k);
  *n_done = k;
  return DLS_OK;
}

int dls_server_get_stats(dls_server *s, dls_server_stats *out) {
  if (s == nullptr || out == nullptr) return DLS_ERR_BAD_ARG;
  std::lock_guard<std::mutex> g(s->mu);
  *out = s->stats;
  out->pending = (int64_t)s->pending.size() + s->splitting;
  int64_t act = 0;
  for (auto *j : s->active) act += (j != nullptr);
  out->active = act;
  out->free_arena_bytes = s->free_chunks.size() * s->cfg.chunk_bytes;
  return DLS_OK;
}

int dls_server_abort(dls_server *s) {
  if (s == nullptr) return DLS_ERR_BAD_ARG;
  s->aborted.store(true);
  return DLS_OK;
}

void dls_server_destroy(dls_server *s) {
  if (!s) return;
  if (s->in_flight) cudaEventSynchronize(s->ev);
  sv_free(s);
}

}  // extern "C"
