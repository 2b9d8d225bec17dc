"""Serving: jobs of mixed order, flags and partial square, counted by the
continuous-batching server.  Each job's count must be the same when it runs
alone, when it runs in the mix, and in the oracle."""
import numpy as np
import pytest

from gpu_cases import make_jobs, oracle_counts

pytestmark = pytest.mark.gpu
D, V = 1, 2


def test_mix_equals_alone_equals_oracle(dls):
    from paper_1709_02599_gb300 import serving
    jobs = make_jobs(dls, 40)
    assert len({(j["n"], j["flags"]) for j in jobs}) >= 5
    ref = oracle_counts(jobs)
    assert sum(ref) > 0
    # in the mix: a small epoch budget makes searches stop and resume often
    srv = serving.Server(budget=256, items_per_job=64)
    ids = {}
    for k, j in enumerate(jobs):
        ids[srv.submit(j["n"], j["flags"], j["order"], j["prefix"])] = k
        if k % 7 == 3:
            srv.step()          # jobs keep arriving while others run
    got = dict(srv.drain())
    st = srv.stats()
    srv.close()
    mix = [got[i] for i in sorted(ids, key=ids.get)]
    assert mix == ref
    assert st["completed"] == len(jobs) and st["epochs"] > 1
    # alone: one job in the server at a time
    srv = serving.Server(budget=4096)
    for k, j in enumerate(jobs):
        jid = srv.submit(j["n"], j["flags"], j["order"], j["prefix"])
        res = dict(srv.drain())
        assert res == {jid: ref[k]}
    srv.close()


def test_admission_waits_for_memory(dls):
    from paper_1709_02599_gb300 import serving
    jobs = make_jobs(dls, 16, seed=5)
    ref = oracle_counts(jobs)
    # an arena of 3 small chunks: most jobs have to wait for earlier ones
    srv = serving.Server(budget=128, items_per_job=32, chunk_bytes=1024, arena_bytes=3 * 1024)
    ids = [srv.submit(j["n"], j["flags"], j["order"], j["prefix"]) for j in jobs]
    waited = 0
    got = {}
    for _ in range(100000):
        srv.step()
        got.update(dict(srv.poll()))
        st = srv.stats()
        waited = max(waited, st["pending"])
        assert st["free_arena_bytes"] <= 3 * 1024
        if len(got) == len(jobs):
            break
    srv.close()
    assert waited > 0
    assert [got[i] for i in ids] == ref


def test_real_time_stream(dls):
    from paper_1709_02599_gb300 import serving
    jobs = make_jobs(dls, 24, seed=23)
    ref = oracle_counts(jobs)
    t = np.linspace(0.0, 0.2, len(jobs))
    for j, a in zip(jobs, t):
        j["arrival"] = float(a)
    srv = serving.Server(budget=1024)
    done, makespan = serving.run_stream(srv, jobs)
    srv.close()
    assert sorted(done) == list(range(len(jobs)))
    assert [done[k][1] for k in range(len(jobs))] == ref
    assert all(done[k][0] >= 0 for k in done)


def test_server_rejects_bad_jobs(dls):
    from paper_1709_02599_gb300 import serving
    srv = serving.Server(max_order=8)
    with pytest.raises(dls.DlsError):
        srv.submit(9, D, dls.fill_order(9, D), np.arange(9, dtype=np.uint8))
    with pytest.raises(dls.DlsError):
        srv.submit(6, D, [(0, 0), (0, 0)], [0])
    # invalid prefix and odd vertically symmetric order complete at once with 0
    a = srv.submit(6, D, dls.fill_order(6, D), [0, 1, 2, 3, 4, 5, 0])
    b = srv.submit(7, D | V, dls.fill_order(7, D | V), [0, 1, 2])
    res = dict(srv.drain())
    assert res == {a: 0, b: 0}
    srv.close()


def test_abort_from_another_thread(dls):
    import threading
    from paper_1709_02599_gb300 import serving
    jobs = make_jobs(dls, 16, seed=5)
    ref = oracle_counts(jobs)
    srv = serving.Server(budget=16, items_per_job=32)
    ids = [srv.submit(j["n"], j["flags"], j["order"], j["prefix"]) for j in jobs]
    got = {}
    for _ in range(100000):
        srv.step()
        got.update(dict(srv.poll()))
        if srv.stats()["epochs"] >= 2:
            break
    stopper = threading.Thread(target=srv.abort)
    stopper.start()
    stopper.join()
    with pytest.raises(dls.DlsError) as e:
        srv.step()
    assert e.value.code == 7
    with pytest.raises(dls.DlsError) as e:
        srv.submit(jobs[0]["n"], jobs[0]["flags"], jobs[0]["order"], jobs[0]["prefix"])
    assert e.value.code == 7
    got.update(dict(srv.poll()))
    srv.close()
    want = dict(zip(ids, ref))
    assert all(got[i] == want[i] for i in got)
