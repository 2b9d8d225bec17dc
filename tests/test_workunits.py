"""CPU tests of the workunit runner (Section 5.2: independent workunits, a
quorum of two copies, results accumulated across restarts).  Failures are
made on the host: a counter that raises part way, one that returns a wrong
count, a checkpoint cut short or changed on disk."""
import dataclasses
import json

import numpy as np
import pytest

import gpu_cases
import oracle

D = 1


@pytest.fixture(scope="module")
def problem(dls):
    wl = gpu_cases.split(dls, 6, D, 9)
    ref, _ = oracle.count_many(6, D, wl.oracle_order, wl.oracle_prefixes)
    return wl, ref


def oracle_counter(wl):
    """Counts from the oracle, for the prefixes the runner hands over."""
    o_order = wl.oracle_order

    def counter(prefixes, launch):
        c, _ = oracle.count_many(6, D, o_order, prefixes)
        return c
    return counter


def test_counts_equal_the_oracle(dls, problem, tmp_path):
    from paper_1709_02599_gb300 import Launch, KERNEL_PLAIN, workunits
    wl, ref = problem
    res = workunits.run_workunits(6, D, wl.order, wl.prefixes, str(tmp_path / "a.jsonl"),
                                  batch=7, quorum=(Launch(), Launch(kernel=KERNEL_PLAIN)),
                                  counter=oracle_counter(wl))
    assert (res["counts"] == ref).all() and res["total"] == int(ref.sum()) == 128
    assert res["units"] == (len(ref) + 6) // 7 == res["units_counted"]
    assert res["units_resumed"] == 0 and res["disagreements"] == 0
    # a second run finds every workunit done
    again = workunits.run_workunits(6, D, wl.order, wl.prefixes, str(tmp_path / "a.jsonl"),
                                    batch=7, counter=oracle_counter(wl))
    assert again["units_resumed"] == res["units"] and again["units_counted"] == 0
    assert (again["counts"] == ref).all()


def test_an_interrupted_run_resumes(dls, problem, tmp_path):
    from paper_1709_02599_gb300 import workunits
    wl, ref = problem
    path = str(tmp_path / "b.jsonl")
    good = oracle_counter(wl)
    calls = []

    def dies_after_three(prefixes, launch):
        if len(calls) == 3:
            raise RuntimeError("worker lost")
        calls.append(1)
        return good(prefixes, launch)

    with pytest.raises(RuntimeError):
        workunits.run_workunits(6, D, wl.order, wl.prefixes, path, batch=5,
                                counter=dies_after_three)
    res = workunits.run_workunits(6, D, wl.order, wl.prefixes, path, batch=5, counter=good)
    assert res["units_resumed"] == 3 and res["units_counted"] == res["units"] - 3
    assert (res["counts"] == ref).all() and res["total"] == 128


def test_a_torn_last_line_costs_one_unit_once(dls, problem, tmp_path):
    # a run killed while writing a record leaves half a line; the next run
    # counts that unit again, and the run after it resumes every unit (the
    # new record was not glued to the fragment)
    from paper_1709_02599_gb300 import workunits
    wl, ref = problem
    path = str(tmp_path / "t.jsonl")
    good = oracle_counter(wl)
    res = workunits.run_workunits(6, D, wl.order, wl.prefixes, path, batch=5, counter=good)
    units = res["units"]
    text = open(path).read()
    cut = text.rstrip("\n").rfind("\n") + 1
    open(path, "w").write(text[:cut] + text[cut:cut + 20])  # last record torn
    res = workunits.run_workunits(6, D, wl.order, wl.prefixes, path, batch=5, counter=good)
    assert res["units_counted"] == 1 and res["units_resumed"] == units - 1
    res = workunits.run_workunits(6, D, wl.order, wl.prefixes, path, batch=5, counter=good)
    assert res["units_counted"] == 0 and res["units_resumed"] == units
    assert (res["counts"] == ref).all() and res["total"] == 128


def test_quorum_recounts_a_disagreement_and_refuses_a_persistent_one(dls, problem, tmp_path):
    from paper_1709_02599_gb300 import Launch, KERNEL_PLAIN, workunits
    wl, ref = problem
    good = oracle_counter(wl)
    quorum = (Launch(), Launch(kernel=KERNEL_PLAIN))
    bad_once = {"left": 1}

    def flaky(prefixes, launch):
        c = good(prefixes, launch)
        if launch.kernel == KERNEL_PLAIN and bad_once["left"] and c.sum() > 0:
            bad_once["left"] -= 1
            c = c.copy()
            c[np.argmax(c)] += 1  # one wrong count in one copy
        return c

    res = workunits.run_workunits(6, D, wl.order, wl.prefixes, str(tmp_path / "c.jsonl"),
                                  batch=9, quorum=quorum, counter=flaky)
    assert res["disagreements"] == 1 and (res["counts"] == ref).all()
    lines = [json.loads(l) for l in open(tmp_path / "c.jsonl").read().split("\n")[1:] if l]
    assert sorted(r["rounds"] for r in lines)[-1] == 2

    def always_wrong(prefixes, launch):
        c = good(prefixes, launch)
        return c + 1 if launch.kernel == KERNEL_PLAIN else c

    with pytest.raises(RuntimeError, match="quorum"):
        workunits.run_workunits(6, D, wl.order, wl.prefixes, str(tmp_path / "d.jsonl"),
                                batch=9, quorum=quorum, counter=always_wrong, max_rounds=2)


def test_checkpoint_damage_is_recounted_and_other_problems_refused(dls, problem, tmp_path):
    from paper_1709_02599_gb300 import workunits
    wl, ref = problem
    path = str(tmp_path / "e.jsonl")
    good = oracle_counter(wl)
    res = workunits.run_workunits(6, D, wl.order, wl.prefixes, path, batch=4, counter=good)
    units = res["units"]
    # the last line cut short, and a count changed in the sidecar file
    text = open(path).read().rstrip("\n")
    open(path, "w").write(text[:-10])
    side = np.memmap(path + ".counts", dtype=np.uint64, mode="r+", shape=(len(ref),))
    k = int(np.argmax(ref))
    side[k] += 5
    side.flush()
    del side
    res = workunits.run_workunits(6, D, wl.order, wl.prefixes, path, batch=4, counter=good)
    assert res["units_counted"] == 2 and res["units_resumed"] == units - 2
    assert (res["counts"] == ref).all()
    # another problem (other prefixes, or another batch size) is refused
    with pytest.raises(ValueError):
        workunits.run_workunits(6, D, wl.order, wl.prefixes[:-1], path, batch=4, counter=good)
    with pytest.raises(ValueError):
        workunits.run_workunits(6, D, wl.order, wl.prefixes, path, batch=5, counter=good)


def test_quorum_of_the_two_kernel_families_on_the_stand_in(dls, problem, emulated, tmp_path):
    """The library's own kernels (built for the CPU on the stand-in runtime)
    as the two copies: the batched snapshot kernel and the plain
    per-position one."""
    from paper_1709_02599_gb300 import Launch, KERNEL_PLAIN, workunits
    wl, ref = problem

    def kernels(prefixes, launch):
        rc, res = emulated.count("count", 6, D, wl.order, prefixes, **dataclasses.asdict(launch))
        assert rc == 0
        return res[0]

    res = workunits.run_workunits(6, D, wl.order, wl.prefixes, str(tmp_path / "f.jsonl"),
                                  batch=64, counter=kernels,
                                  quorum=(Launch(), Launch(kernel=KERNEL_PLAIN, stack=1)))
    assert (res["counts"] == ref).all() and res["disagreements"] == 0


@pytest.mark.gpu
def test_default_counter_on_the_gpu(dls, tmp_path):
    """The default counter (the library on the GPU) with the two kernel
    families as the quorum."""
    from paper_1709_02599_gb300 import Launch, KERNEL_PLAIN, workunits
    wl = gpu_cases.split(dls, 7, D, 10)
    ref, _ = oracle.count_many(7, D, wl.oracle_order, wl.oracle_prefixes, threads=8)
    res = workunits.run_workunits(7, D, wl.order, wl.prefixes, str(tmp_path / "g.jsonl"),
                                  batch=1000,
                                  quorum=(Launch(), Launch(kernel=KERNEL_PLAIN, stack=1)))
    assert (res["counts"] == ref).all() and res["total"] == 171200
    assert res["disagreements"] == 0 and res["units"] == 3


def test_count_split_on_the_stand_in(dls, emulated, tmp_path):
    """count_split (the command line's run): order 6 split 4 cells past row 0,
    a quorum of the two kernel families on the stand-in runtime."""
    from paper_1709_02599_gb300 import ORDER_HEURISTIC, workunits
    order = dls.fill_order(6, D, ORDER_HEURISTIC)

    def kernels(prefixes, launch):
        rc, res = emulated.count("count", 6, D, order, prefixes, **dataclasses.asdict(launch))
        assert rc == 0
        return res[0]

    res = workunits.count_split(6, D, 10, str(tmp_path / "h.jsonl"), batch=16, quorum=2,
                                counter=kernels)
    assert res["row0_fixed"] == 128 and res["squares"] == 92160
    assert res["disagreements"] == 0 and res["units"] == (res["prefixes"] + 15) // 16


def test_count_split_makes_the_order9_workunits(dls, tmp_path):
    """Section 5.2: row 0 and the first 10 cells of the Fig. 1 order give
    1 255 884 workunits (the number the assignments of those cells have)."""
    from paper_1709_02599_gb300 import workunits

    def zeros(prefixes, launch):
        return np.zeros(len(prefixes), np.uint64)

    res = workunits.count_split(9, D, 19, str(tmp_path / "i.jsonl"), counter=zeros)
    assert res["prefixes"] == 1255884 and res["units"] == 2 and res["total"] == 0
