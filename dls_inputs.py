"""Seeded synthetic inputs shared by the oracle side and the CUDA side.

This module draws random numbers only -- it holds none of the counting
method's arithmetic.  Anything that needs the Latin-square constraints (which
prefixes are valid, how draws become a partial square) is computed by each
side separately from these numbers.  All generators are numpy PCG64 with an
explicit seed.

Workload recipes (sizes follow the paper's experiments, Sections 5.1-5.4):

* ``dls6_single``: order 6, row 0 = identity, one subproblem.
* ``dls7_split10``: order 7, row 0 = identity, split 10 cells past row 0.
* ``dls8_diag64``: order 8, row 0 = identity; ``choose(n_fillings, 64,
  seed=0)`` picks 64 main-diagonal fillings out of all of them, each split 20
  cells past row 0 (both diagonals and the rest of row 1).
* ``vsym10_rows2``: order 10, vertically symmetric; ``choose(n_prefixes,
  2000, seed=0)`` picks 2000 of the valid fillings of rows 1 and 2.
* Monte Carlo (Section 5.3): ``ranks(N^k, m, seed)`` -- m uniform ranks of
  k-cell partial squares, each side selecting the partial square of a rank
  itself.
* serving: ``serving_jobs(n, seed)`` -- Poisson arrivals at 200 req/s, order
  uniform in {6, 7, 8, 9}, flag uniform in {diagonal, vertically symmetric},
  k uniform in {2, ..., N-3} fixed rows, and 4096 uint32 draws per job from
  which each side builds the job's random partial square.
"""
import numpy as np

WORKLOADS = {
    "dls6_single": dict(n=6, vsym=False, split_after_row0=0),
    "dls7_split10": dict(n=7, vsym=False, split_after_row0=10),
    "dls8_diag64": dict(n=8, vsym=False, diag_fillings=64, split_after_row0=20, seed=0),
    "vsym10_rows2": dict(n=10, vsym=True, sample=2000, seed=0),
}


def rng(seed, stream=0):
    return np.random.Generator(np.random.PCG64([int(seed), int(stream)]))


def choose(population, k, seed=0):
    """k distinct indices out of range(population), sorted ascending."""
    k = min(int(k), int(population))
    g = np.random.Generator(np.random.PCG64(int(seed)))
    return np.sort(g.choice(int(population), size=k, replace=False)).astype(np.int64)


def draws(count, seed, stream=0):
    """``count`` uniform uint32 numbers."""
    return rng(seed, stream).integers(0, 2**32, size=int(count), dtype=np.uint32)


def ranks(total, count, seed, stream=3):
    """``count`` uniform integers in [0, total) (Monte Carlo sample ranks)."""
    return rng(seed, stream).integers(0, int(total), size=int(count), dtype=np.int64)


def poisson_arrivals(rate_hz, n_jobs, seed=0):
    """Arrival times (seconds from 0) of a Poisson process."""
    g = rng(seed, 1)
    gaps = g.exponential(1.0 / float(rate_hz), size=int(n_jobs))
    return np.cumsum(gaps)


def serving_jobs(n_jobs, seed=0, orders=(6, 7, 8, 9), draws_per_job=4096,
                 rate_hz=200.0):
    """Job descriptions for the serving workload (random numbers only)."""
    g = rng(seed, 2)
    times = poisson_arrivals(rate_hz, n_jobs, seed)
    jobs = []
    for q in range(int(n_jobs)):
        n = int(g.choice(orders))
        vsym = bool(g.integers(0, 2))
        k = int(g.integers(2, n - 3 + 1))
        jobs.append(dict(id=q, arrival=float(times[q]), n=n, vsym=vsym, rows=k,
                         draws=draws(draws_per_job, seed, 1000 + q)))
    return jobs
