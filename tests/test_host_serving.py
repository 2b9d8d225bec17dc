"""CPU tests of the serving kernel and server, and of the symmetry-breaking
kernel, on the library built for the CPU on the stand-in CUDA runtime
(host_emulation.py).

They mirror the GPU tests of test_serving.py and test_symmetry.py.  Each
job's count must be the oracle's when it runs alone and when it runs in the
mix: all jobs at once, or one more per epoch while others run, with a small
epoch budget so that searches are saved and resumed many times.  Admission
must wait for arena memory.  Bad jobs must be refused, and degenerate jobs
must complete at once.  Hourglass class sizes must be the oracle's
(Algorithm 5)."""
import numpy as np

import oracle
from gpu_cases import make_jobs, oracle_counts
from oracle import orders

D, V = 1, 2
ERR_INVALID_N, ERR_BAD_ORDER, ERR_ABORTED = 1, 2, 7
SMALL_ARENA = dict(arena_bytes=4 << 20, max_jobs=64)


def _counts_in_submission_order(rcs, done):
    # ids are handed out in submission order, from 0, to accepted jobs only
    assert all(rc == 0 for rc in rcs)
    return [done[k] for k in range(len(rcs))]


def test_mix_equals_alone_equals_oracle(dls, emulated):
    jobs = make_jobs(dls, 40)
    assert len({(j["n"], j["flags"]) for j in jobs}) >= 5
    ref = oracle_counts(jobs)
    assert sum(ref) > 0
    for mode, budget in (("stream", 256), ("all", 64)):
        create, rcs, done, st = emulated.serve(jobs, mode=mode, budget=budget,
                                               items_per_job=64, **SMALL_ARENA)
        assert create == 0
        assert _counts_in_submission_order(rcs, done) == ref, mode
        assert st["completed"] == len(jobs) and st["epochs"] > 1, st
    create, rcs, done, st = emulated.serve(jobs, mode="alone", budget=4096, **SMALL_ARENA)
    assert create == 0 and _counts_in_submission_order(rcs, done) == ref


def test_admission_waits_for_memory(dls, emulated):
    jobs = make_jobs(dls, 16, seed=5)
    ref = oracle_counts(jobs)
    # an arena of 3 small chunks: most jobs have to wait for earlier ones
    create, rcs, done, st = emulated.serve(jobs, mode="all", budget=128, items_per_job=32,
                                           chunk_bytes=1024, arena_bytes=3 * 1024)
    assert create == 0
    assert _counts_in_submission_order(rcs, done) == ref
    assert st["max_pending"] > 0 and st["min_free_arena"] <= 3 * 1024


def test_server_rejects_bad_jobs(dls, emulated):
    o6 = dls.fill_order(6, D)
    jobs = [dict(n=9, flags=D, order=dls.fill_order(9, D), prefix=np.arange(9)),  # > max_order
            dict(n=6, flags=D, order=[(0, 0), (0, 0)], prefix=[0]),              # repeated cell
            dict(n=6, flags=D, order=o6, prefix=[0, 1, 2, 3, 4, 5, 0]),          # invalid prefix
            dict(n=7, flags=D | V, order=dls.fill_order(7, D | V), prefix=[0, 1, 2])]  # odd, sym.
    create, rcs, done, st = emulated.serve(jobs, mode="all", max_order=8, **SMALL_ARENA)
    assert create == 0
    assert rcs == [ERR_INVALID_N, ERR_BAD_ORDER, 0, 0]
    assert done == {0: 0, 1: 0}  # both complete at once with 0
    assert st["submitted"] == 2 and st["completed"] == 2


def _hourglass_case(n, flags):
    vs = bool(flags & V)
    hc = orders.hourglass_cells(n, vs)
    full = hc + [c for c in orders.md_ad_rows(n, vsym=vs) if c not in hc]
    hg, _ = oracle.extend(n, flags, full, np.array([orders.identity(n, vs)], np.uint8), len(hc))
    return hc, full, hg


def test_hourglass_classes_against_oracle(dls, emulated):
    for n, flags, step in ((5, D, 1), (6, D, 1), (7, D, 1), (6, D | V, 1), (8, D | V, 1),
                           (8, D, 1109)):
        hc, full, hg = _hourglass_case(n, flags)
        hg = hg[::step]
        ref = oracle.hourglass_classes(n, flags, full, hg, threads=4)
        rc, sizes = emulated.classes(n, flags, np.array(hc, np.uint8), hg)
        assert rc == 0 and (sizes == ref).all(), (n, flags)
        if step == 1:
            # every hourglass lies in exactly one class: the sizes of the
            # canonical ones add up to the number of hourglasses
            assert int(sizes.sum()) == len(hg), (n, flags)
    # the hourglass cells may come in any order (values in the same order);
    # another set of cells is refused
    hc, full, hg = _hourglass_case(6, D)
    ref = oracle.hourglass_classes(6, D, full, hg, threads=4)
    rc, sizes = emulated.classes(6, D, np.array(hc[::-1], np.uint8), hg[:, ::-1])
    assert rc == 0 and (sizes == ref).all()
    other = [c for c in full if c not in hc][0]
    rc, _ = emulated.classes(6, D, np.array(hc[:-1] + [other], np.uint8), hg)
    assert rc == ERR_BAD_ORDER


def test_abort_from_another_thread(dls, emulated):
    """dls_server_abort from another thread once two epochs have run: the next step
    and later submissions return DLS_ERR_ABORTED and no epoch follows; the
    jobs completed by then keep their exact counts."""
    jobs = make_jobs(dls, 16, seed=5)
    ref = oracle_counts(jobs)
    create, rcs, done, st = emulated.serve(jobs, mode="abort", budget=16, items_per_job=32,
                                           **SMALL_ARENA)
    assert create == 0
    assert rcs == [0] * len(jobs) + [ERR_ABORTED]
    assert st["step_rc"] == ERR_ABORTED and st["epochs"] == 2
    assert len(done) == st["completed"] < len(jobs)
    assert all(done[k] == ref[k] for k in done)
