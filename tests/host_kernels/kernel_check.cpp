// kernel_check.cpp -- calls the library's C entry points with the kernels
// running on the CPU (the library source built against the stand-in
// cuda_runtime.h of this folder), for tests/test_host_kernels.py.
//
//   kernel_check ENTRY n flags order.bin prefixes.bin depth
//                kernel block blocks_per_sm lanes split_pos donate check_every
//                words stack lookahead fuse budget abort stack_cap
//   kernel_check classes n flags order.bin hourglasses.bin len
//   kernel_check serve jobs.txt mode max_jobs arena_bytes chunk_bytes budget
//                block_threads items_per_job max_order
//
// ENTRY: count (dls_count_ex with node counting, then dls_stream_status),
// host (dls_count_host), noalloc (dls_count_host_noalloc), weighted
// (dls_count_weighted with weights (k % 5) + 1 and the multiplier), plan
// (dls_plan_create, then two dls_plan_launch and dls_plan_status), describe
// (dls_describe_launch).  "Device" buffers are host memory here.  Output:
// "rc R" and, when R = 0, "total T nodes N" (nodes 0 where the entry does
// not count them; count and plan add "status S started K") and one count per
// prefix; describe prints "run W block grid smem entries fused step" instead.
//
// classes: dls_hourglass_classes over `len`-byte hourglass records; prints
// "rc R" and one class size per record.
//
// serve: a dls_server with that configuration (0 = default) counts the jobs
// of jobs.txt (one per line: n flags order_len depth, then the order's
// 2 * order_len bytes and the prefix's depth bytes, as integers).  mode
// "all" submits every job before the first step, "stream" one job per
// step, "alone" the next job only once the previous one is done, "abort"
// every job, then dls_server_abort from another thread once two epochs have
// run (and one more submission after the next step).  Steps
// until every job is done (at most 100000 steps).  Prints "rc R" for each
// submission in order, then "job ID COUNT" per completed job, then "stats
// submitted admitted completed epochs max_pending min_free_arena" (the last
// two over the steps).
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <string>
#include <thread>
#include <utility>
#include <vector>

#include "dls.h"

namespace {

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

void print_counts(int rc, unsigned long long total, unsigned long long nodes,
                  const std::vector<uint64_t> &counts, const dls_count_status *st = nullptr) {
  std::printf("rc %d\n", rc);
  if (rc != 0) return;
  if (st)
    std::printf("total %llu nodes %llu status %d started %lld\n", total, nodes, st->status,
                (long long)st->prefixes_started);
  else
    std::printf("total %llu nodes %llu\n", total, nodes);
  for (uint64_t c : counts) std::printf("%llu\n", (unsigned long long)c);
}

}  // namespace

int run_classes(int argc, char **argv) {
  if (argc != 7) return 1;
  const int n = std::atoi(argv[2]);
  const uint32_t flags = (uint32_t)std::atoi(argv[3]);
  const std::vector<uint8_t> order = read_file(argv[4]);
  std::vector<uint8_t> hg = read_file(argv[5]);
  const int len = std::atoi(argv[6]);
  const int64_t count = len ? (int64_t)hg.size() / len : 0;
  if (hg.empty()) hg.push_back(0);
  std::vector<uint32_t> sizes((size_t)count + 1, 0xdeadbeefu);
  const int rc = dls_hourglass_classes(n, flags, order.data(), (int)order.size() / 2,
                                       hg.data(), count, sizes.data(), nullptr);
  std::printf("rc %d\n", rc);
  if (rc == 0)
    for (int64_t k = 0; k < count; ++k) std::printf("%u\n", sizes[(size_t)k]);
  return 0;
}

struct Job {
  int n = 0;
  uint32_t flags = 0;
  std::vector<uint8_t> order, prefix;
};

int run_serve(int argc, char **argv) {
  if (argc != 11) return 1;
  std::vector<Job> jobs;
  FILE *f = std::fopen(argv[2], "r");
  if (!f) return 1;
  int n, fl, ol, d;
  while (std::fscanf(f, "%d %d %d %d", &n, &fl, &ol, &d) == 4) {
    Job j;
    j.n = n;
    j.flags = (uint32_t)fl;
    for (int k = 0; k < 2 * ol + d; ++k) {
      int v = 0;
      if (std::fscanf(f, "%d", &v) != 1) return 1;
      (k < 2 * ol ? j.order : j.prefix).push_back((uint8_t)v);
    }
    jobs.push_back(std::move(j));
  }
  std::fclose(f);
  const std::string mode = argv[3];
  dls_server_cfg cfg;
  dls_server_default_cfg(&cfg);
  if (std::atoi(argv[4])) cfg.max_jobs = std::atoi(argv[4]);
  if (std::atoll(argv[5])) cfg.arena_bytes = (size_t)std::atoll(argv[5]);
  if (std::atoll(argv[6])) cfg.chunk_bytes = (size_t)std::atoll(argv[6]);
  if (std::atoi(argv[7])) cfg.budget = std::atoi(argv[7]);
  if (std::atoi(argv[8])) cfg.block_threads = std::atoi(argv[8]);
  if (std::atoi(argv[9])) cfg.items_per_job = std::atoi(argv[9]);
  if (std::atoi(argv[10])) cfg.max_order = std::atoi(argv[10]);
  dls_server *srv = nullptr;
  int rc = dls_server_create(&cfg, &srv);
  std::printf("create %d\n", rc);
  if (rc) return 0;
  std::vector<std::pair<int64_t, uint64_t>> done;
  size_t next = 0;
  int64_t accepted = 0;
  auto submit = [&](const Job &j) {
    int64_t id = -1;
    const int r = dls_server_submit(srv, j.n, j.flags, j.order.data(), (int)j.order.size() / 2,
                                    j.prefix.data(), (int)j.prefix.size(), &id);
    std::printf("rc %d\n", r);
    if (r == 0) ++accepted;
  };
  if (mode == "all" || mode == "abort")
    for (; next < jobs.size(); ++next) submit(jobs[next]);
  int64_t max_pending = 0;
  bool abort_sent = false;
  size_t min_free = (size_t)-1;
  for (int step = 0; step < 100000 && ((int64_t)done.size() < accepted || next < jobs.size());
       ++step) {
    if (next < jobs.size() &&
        (mode == "stream" || (mode == "alone" && (int64_t)done.size() == accepted)))
      submit(jobs[next++]);
    if (mode == "abort" && !abort_sent) {
      dls_server_stats ran;
      dls_server_get_stats(srv, &ran);
      if (ran.epochs >= 2) {
        std::thread stopper([srv]() { dls_server_abort(srv); });
        stopper.join();
        abort_sent = true;
      }
    }
    rc = dls_server_step(srv);
    if (mode == "abort" && rc == DLS_ERR_ABORTED) {
      std::printf("step %d\n", rc);
      submit(jobs[0]);
      int64_t ids[64];
      uint64_t counts[64];
      int got = 0;
      dls_server_poll(srv, ids, counts, 64, &got);
      for (int k = 0; k < got; ++k) done.emplace_back(ids[k], counts[k]);
      break;
    }
    dls_server_stats now;
    dls_server_get_stats(srv, &now);
    max_pending = std::max(max_pending, now.pending);
    min_free = std::min(min_free, now.free_arena_bytes);
    if (rc) {
      std::printf("step %d\n", rc);
      break;
    }
    int64_t ids[64];
    uint64_t counts[64];
    int got = 0;
    do {
      rc = dls_server_poll(srv, ids, counts, 64, &got);
      for (int k = 0; k < got; ++k) done.emplace_back(ids[k], counts[k]);
    } while (rc == 0 && got == 64);
  }
  for (const auto &x : done)
    std::printf("job %lld %llu\n", (long long)x.first, (unsigned long long)x.second);
  dls_server_stats st;
  dls_server_get_stats(srv, &st);
  std::printf("stats %lld %lld %lld %lld %lld %llu\n", (long long)st.submitted,
              (long long)st.admitted, (long long)st.completed, (long long)st.epochs,
              (long long)max_pending, (unsigned long long)min_free);
  dls_server_destroy(srv);
  return 0;
}

int main(int argc, char **argv) {
  if (argc >= 2 && std::string(argv[1]) == "classes") return run_classes(argc, argv);
  if (argc >= 2 && std::string(argv[1]) == "serve") return run_serve(argc, argv);
  if (argc != 21) {
    std::fprintf(stderr, "usage: kernel_check ENTRY n flags order.bin prefixes.bin depth "
                         "kernel block blocks_per_sm lanes split_pos donate check_every "
                         "words stack lookahead fuse budget abort stack_cap\n");
    return 1;
  }
  const std::string entry = argv[1];
  const int n = std::atoi(argv[2]);
  const uint32_t flags = (uint32_t)std::atoi(argv[3]);
  const std::vector<uint8_t> order = read_file(argv[4]);
  std::vector<uint8_t> pre = read_file(argv[5]);
  const int depth = std::atoi(argv[6]);
  dls_launch_t cfg;
  cfg.kernel = std::atoi(argv[7]);
  cfg.block_threads = std::atoi(argv[8]);
  cfg.blocks_per_sm = std::atoi(argv[9]);
  cfg.lanes_per_prefix = std::atoi(argv[10]);
  cfg.split_pos = std::atoi(argv[11]);
  cfg.donate = std::atoi(argv[12]);
  cfg.check_every = std::atoi(argv[13]);
  cfg.words = std::atoi(argv[14]);
  cfg.stack = std::atoi(argv[15]);
  cfg.lookahead = std::atoi(argv[16]);
  cfg.fuse = std::atoi(argv[17]);
  cfg.budget = std::atoll(argv[18]);
  // abort: 0 = no flag, 1 = a flag already set, 2 = a flag that stays clear
  static int abort_word = 0;
  const int abort_mode = std::atoi(argv[19]);
  abort_word = abort_mode == 1 ? 1 : 0;
  cfg.abort_flag = abort_mode ? &abort_word : nullptr;
  cfg.stack_cap = std::atoi(argv[20]);
  const int len = (int)order.size() / 2;
  const int64_t P = depth ? (int64_t)pre.size() / depth : 1;
  if (pre.empty()) pre.push_back(0);  // a valid pointer for depth 0

  if (entry == "describe") {
    dls_launch_info info;
    const int rc = dls_describe_launch(n, flags, order.data(), len, depth, P, &cfg, &info);
    std::printf("rc %d\n", rc);
    if (rc == 0)
      std::printf("%d %d %d %d %d %d %d %d\n", info.run, info.words, info.block_threads,
                  info.grid_blocks, info.smem_bytes, info.stack_entries, info.fused, info.step);
    return 0;
  }
  std::vector<uint64_t> counts((size_t)P, 0xdeadbeefull);
  uint64_t total = 0xdeadbeefull, nodes = 0;
  if (entry == "count") {
    int rc = dls_count_ex(n, flags, order.data(), len, pre.data(), depth, P,
                          counts.data(), &total, &nodes, &cfg, nullptr);
    dls_count_status st{-1, -1};
    if (rc == 0) rc = dls_stream_status(nullptr, &st);
    print_counts(rc, total, nodes, counts, &st);
  } else if (entry == "host" || entry == "noalloc") {
    dls_u128 t{0, 0};
    const int rc = entry == "host"
                       ? dls_count_host(n, flags, order.data(), len, pre.data(), depth, P,
                                        counts.data(), &t, &cfg, nullptr)
                       : dls_count_host_noalloc(n, flags, order.data(), len, pre.data(), depth,
                                                P, counts.data(), &t, &cfg, nullptr);
    // total_out: the plain 128-bit sum of the counts
    std::printf("rc %d\n", rc);
    if (rc == 0) {
      std::printf("total %llu nodes 0 hi %llu\n", (unsigned long long)t.lo,
                  (unsigned long long)t.hi);
      for (uint64_t c : counts) std::printf("%llu\n", (unsigned long long)c);
    }
  } else if (entry == "weighted") {
    // weights (k % 5) + 1, total times the row-0 multiplier
    std::vector<uint32_t> w((size_t)P);
    for (int64_t k = 0; k < P; ++k) w[(size_t)k] = (uint32_t)(k % 5) + 1u;
    dls_u128 t{0, 0};
    const int rc = dls_count_weighted(n, flags, order.data(), len, pre.data(), depth, P,
                                      w.data(), counts.data(), 1, &t, &cfg, nullptr);
    std::printf("rc %d\n", rc);
    if (rc == 0) {
      std::printf("total %llu nodes 0 hi %llu\n", (unsigned long long)t.lo,
                  (unsigned long long)t.hi);
      for (uint64_t c : counts) std::printf("%llu\n", (unsigned long long)c);
    }
  } else if (entry == "plan") {
    dls_plan *plan = nullptr;
    int rc = dls_plan_create(&plan, n, flags, order.data(), len, pre.data(), depth, P,
                             counts.data(), &total, &cfg);
    if (rc == 0) rc = dls_plan_launch(plan, nullptr);
    const std::vector<uint64_t> first = counts;
    const uint64_t first_total = total;
    if (rc == 0) {
      counts.assign(counts.size(), 0xdeadbeefull);
      total = 0xdeadbeefull;
      rc = dls_plan_launch(plan, nullptr);
    }
    dls_count_status st{-1, -1};
    if (rc == 0) rc = dls_plan_status(plan, nullptr, &st);
    if (plan) dls_plan_destroy(plan);
    if (rc == 0 && (first != counts || first_total != total)) rc = 99;  // replays differ
    print_counts(rc, total, 0, counts, &st);
  } else {
    std::fprintf(stderr, "unknown entry %s\n", entry.c_str());
    return 1;
  }
  return 0;
}
