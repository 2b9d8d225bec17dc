// kernel_check.cpp -- calls the library's C entry points with the kernels
// running on the CPU (the library source built against the stand-in
// cuda_runtime.h of this folder), for tests/test_host_kernels.py.
//
//   kernel_check ENTRY n flags order.bin prefixes.bin depth
//                kernel block blocks_per_sm lanes split_pos donate check_every
//                words stack lookahead fuse
//
// ENTRY: count (dls_count_ex with node counting), host (dls_count_host),
// plan (dls_plan_create, then two dls_plan_launch), describe
// (dls_describe_launch).  "Device" buffers are host memory here.
// Output: "rc R" and, when R = 0, "total T nodes N" (nodes 0 where the entry
// does not count them) and one count per prefix; describe prints
// "run W block grid smem entries fused" instead of the counts.
#include <cstdio>
#include <cstdlib>
#include <string>
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
                  const std::vector<uint64_t> &counts) {
  std::printf("rc %d\n", rc);
  if (rc != 0) return;
  std::printf("total %llu nodes %llu\n", total, nodes);
  for (uint64_t c : counts) std::printf("%llu\n", (unsigned long long)c);
}

}  // namespace

int main(int argc, char **argv) {
  if (argc != 18) {
    std::fprintf(stderr, "usage: kernel_check ENTRY n flags order.bin prefixes.bin depth "
                         "kernel block blocks_per_sm lanes split_pos donate check_every "
                         "words stack lookahead fuse\n");
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
  const int len = (int)order.size() / 2;
  const int64_t P = depth ? (int64_t)pre.size() / depth : 1;
  if (pre.empty()) pre.push_back(0);  // a valid pointer for depth 0

  if (entry == "describe") {
    dls_launch_info info;
    const int rc = dls_describe_launch(n, flags, order.data(), len, depth, P, &cfg, &info);
    std::printf("rc %d\n", rc);
    if (rc == 0)
      std::printf("%d %d %d %d %d %d %d\n", info.run, info.words, info.block_threads,
                  info.grid_blocks, info.smem_bytes, info.stack_entries, info.fused);
    return 0;
  }
  std::vector<uint64_t> counts((size_t)P, 0xdeadbeefull);
  uint64_t total = 0xdeadbeefull, nodes = 0;
  if (entry == "count") {
    const int rc = dls_count_ex(n, flags, order.data(), len, pre.data(), depth, P,
                                counts.data(), &total, &nodes, &cfg, nullptr);
    print_counts(rc, total, nodes, counts);
  } else if (entry == "host") {
    dls_u128 t{0, 0};
    const int rc = dls_count_host(n, flags, order.data(), len, pre.data(), depth, P,
                                  counts.data(), &t, &cfg, nullptr);
    // total_out: the plain 128-bit sum of the counts
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
    if (plan) dls_plan_destroy(plan);
    if (rc == 0 && (first != counts || first_total != total)) rc = 99;  // replays differ
    print_counts(rc, total, 0, counts);
  } else {
    std::fprintf(stderr, "unknown entry %s\n", entry.c_str());
    return 1;
  }
  return 0;
}
