"""The library built for the CPU on the stand-in CUDA runtime of
tests/host_kernels, for the CPU tests of its kernels (test_host_kernels.py,
test_host_serving.py).

Every CUDA source of the library is copied into a temporary folder with
three mechanical changes that the host compiler needs, and built with the
library's own host code, the stand-in runtime (simt.cpp) and the driver
program kernel_check.cpp. The changes:
- the dynamic shared array becomes a per-block buffer;
- each static shared array becomes a per-block buffer too;
- each `kernel<<<grid, block, smem, stream>>>(args)` launch becomes a call to
  the stand-in launcher.
The kernels launched through cudaLaunchKernel get the stand-in version of
that call appended (launch_kparams.inc). This build is test infrastructure:
the library itself is built only with nvcc, and its Python binding loads
only that build."""
import os
import re
import shutil
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(ROOT, "paper_1709_02599_gb300", "csrc")
HK = os.path.join(HERE, "host_kernels")
SOURCES = ["dls_kernels.cu", "dls_serve.cu", "dls_symmetry.cu", "dls_noalloc.cu"]
FIELDS = ["kernel", "block_threads", "blocks_per_sm", "lanes_per_prefix", "split_pos",
          "donate", "check_every", "words", "stack", "lookahead", "fuse", "budget", "abort",
          "stack_cap"]

_SHARED = re.compile(r"__shared__\s+([A-Za-z_][\w ]*?)\s+(\w+)\[(\d+)\];")
_LAUNCH = re.compile(r"(\w+)<<<([^;]*?)>>>\(([^;]*)\);")


def host_source(text, name):
    """The CUDA source `text` (file `name`) with the changes above."""
    text = text.replace("extern __shared__ uint32_t smem[];",
                        "uint32_t *smem = static_cast<uint32_t *>(::shim::dynamic_smem());")
    lines = text.split("\n")
    for k, line in enumerate(lines):
        m = _SHARED.search(line)
        if m:
            t, var, count = m.groups()
            lines[k] = (line[:m.start()] + "%s *%s = static_cast<%s *>(::shim::block_shared("
                        "sizeof(%s) * %s, %d));" % (t, var, t, t, count, k) + line[m.end():])
        m = _LAUNCH.search(lines[k])
        if m:
            fn, conf, args = m.groups()
            parts = [p.strip() for p in conf.split(",")]
            assert len(parts) == 4, (name, lines[k])
            grid, block, smem, stream = parts
            lines[k] = (lines[k][:m.start()] + "::shim::launch(%s, dim3(%s), dim3(%s), %s, "
                        "[=]() { %s(%s); });" % (stream, grid, block, smem, fn, args)
                        + lines[k][m.end():])
    text = "\n".join(lines)
    if name == "dls_kernels.cu":
        # test hook of this build only: DLS_STANDIN_SNAP_CAP, when set, replaces
        # the snapshot stack's entry bound, so that a test can make the stack
        # overflow and see the entry points report it
        cap = "kp.snap_cap = snap ? std::max(1, snapshot_entries(info, n, flags, depth)) : 0;"
        assert cap in text
        text = text.replace(cap, cap + ' if (snap && std::getenv("DLS_STANDIN_SNAP_CAP")) '
                            'kp.snap_cap = std::atoi(std::getenv("DLS_STANDIN_SNAP_CAP"));')
        text = "#include <cstdlib>\n" + text
        text += '\n#include "launch_kparams.inc"\n'
    assert "__shared__" not in text and "<<<" not in text, name
    return text


def build(outdir):
    """Builds the driver program in `outdir`; returns its path (None when no
    host C++ compiler is available)."""
    gxx = shutil.which("g++")
    if gxx is None:
        return None
    srcs = []
    for name in SOURCES:
        with open(os.path.join(CSRC, name)) as f:
            text = f.read()
        out = os.path.join(outdir, name.replace(".cu", "_host.cpp"))
        with open(out, "w") as f:
            f.write(host_source(text, name))
        srcs.append(out)
    exe = os.path.join(outdir, "kernel_check")
    r = subprocess.run([gxx, "-O1", "-std=c++17", "-w", "-pthread", "-I", HK,
                        "-I", os.path.join(HERE, "host_step"), "-I", CSRC,
                        "-I", os.path.join(ROOT, "include")] + srcs
                       + [os.path.join(CSRC, "dls_host.cpp"), os.path.join(HK, "simt.cpp"),
                          os.path.join(HK, "kernel_check.cpp"), "-o", exe],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("building the CPU stand-in failed:\n" + r.stderr[-4000:])
    return exe


class Emulated:
    """Runs the driver program; every call writes its inputs to `workdir`."""

    def __init__(self, exe, workdir):
        self.exe, self.d = exe, workdir

    def _run(self, args, timeout=600, env=None):
        full_env = None
        if env:
            full_env = dict(os.environ)
            full_env.update({k: str(v) for k, v in env.items()})
        r = subprocess.run([self.exe] + [str(a) for a in args], capture_output=True, text=True,
                           timeout=timeout, env=full_env)
        assert r.returncode == 0, (r.returncode, r.stderr[-2000:])
        return r.stdout.split("\n")

    def _files(self, order, records):
        o = os.path.join(self.d, "order.bin")
        p = os.path.join(self.d, "records.bin")
        np.ascontiguousarray(order, dtype=np.uint8).tofile(o)
        np.ascontiguousarray(records, dtype=np.uint8).tofile(p)
        return o, p

    def count(self, entry, n, flags, order, prefixes, env=None, **launch):
        """entry: count, host, noalloc, plan or describe.  Returns (rc,
        result): (counts, total, nodes) for the counting entries, a dict for
        describe, None when rc != 0.  After count and plan, self.last_status
        holds (status, prefixes started) of dls_stream_status /
        dls_plan_status.  env: extra environment of the driver process."""
        prefixes = np.ascontiguousarray(prefixes, dtype=np.uint8)
        depth = prefixes.shape[1] if prefixes.ndim == 2 else 0
        o, p = self._files(order, prefixes)
        lines = self._run([entry, n, flags, o, p, depth] + [launch.get(k, 0) for k in FIELDS],
                          env=env)
        rc = int(lines[0].split()[1])
        self.last_status = None
        if rc != 0:
            return rc, None
        if entry == "describe":
            keys = ["run", "words", "block_threads", "grid_blocks", "smem_bytes",
                    "stack_entries", "fused", "step"]
            return 0, dict(zip(keys, map(int, lines[1].split())))
        head = lines[1].split()
        if "hi" in head:
            self.last_total128 = int(head[head.index("hi") + 1]) << 64 | int(head[1])
        if "status" in head:
            k = head.index("status")
            self.last_status = (int(head[k + 1]), int(head[k + 3]))
        counts = np.array([int(x) for x in lines[2:] if x.strip()], dtype=np.uint64)
        return 0, (counts, int(head[1]), int(head[3]))

    def classes(self, n, flags, order, hourglasses):
        hourglasses = np.ascontiguousarray(hourglasses, dtype=np.uint8)
        o, p = self._files(order, hourglasses)
        lines = self._run(["classes", n, flags, o, p, hourglasses.shape[1]])
        rc = int(lines[0].split()[1])
        return rc, (np.array([int(x) for x in lines[1:] if x.strip()], dtype=np.int64)
                    if rc == 0 else None)

    def serve(self, jobs, mode="all", max_jobs=0, arena_bytes=0, chunk_bytes=0, budget=0,
              block_threads=0, items_per_job=0, max_order=0):
        """jobs: dicts with n, flags, order (uint8 [L, 2]), prefix (uint8
        [d]); mode: all, stream, alone or abort (kernel_check.cpp).  Returns
        (create_rc, submit_rcs, {job id: count}, stats)."""
        path = os.path.join(self.d, "jobs.txt")
        with open(path, "w") as f:
            for j in jobs:
                order = np.asarray(j["order"], dtype=np.uint8).reshape(-1, 2)
                prefix = np.asarray(j["prefix"], dtype=np.uint8).ravel()
                vals = [j["n"], j["flags"], len(order), len(prefix)]
                vals += [int(x) for x in order.ravel()] + [int(x) for x in prefix]
                f.write(" ".join(map(str, vals)) + "\n")
        # a correct server finishes these jobs in seconds; a search that was
        # resumed wrongly can run for very long instead
        lines = self._run(["serve", path, mode, max_jobs, arena_bytes, chunk_bytes, budget,
                           block_threads, items_per_job, max_order], timeout=120)
        create = int(lines[0].split()[1])
        if create != 0:
            return create, [], {}, None
        rcs, done, stats, stats_step = [], {}, None, None
        for line in lines[1:]:
            w = line.split()
            if not w:
                continue
            if w[0] == "rc":
                rcs.append(int(w[1]))
            elif w[0] == "job":
                done[int(w[1])] = int(w[2])
            elif w[0] == "stats":
                stats = dict(zip(["submitted", "admitted", "completed", "epochs",
                                  "max_pending", "min_free_arena"], map(int, w[1:])))
            elif w[0] == "step":
                if mode != "abort":
                    raise AssertionError("dls_server_step returned %s" % w[1])
                stats_step = int(w[1])
        if stats is not None and stats_step is not None:
            stats["step_rc"] = stats_step
        return create, rcs, done, stats
