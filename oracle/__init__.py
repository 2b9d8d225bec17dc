"""Reference (oracle) implementation of the counting method.

TEST INFRASTRUCTURE ONLY: imported by ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py``; never by the product package.  It
shares no code with the CUDA path.

* ``dls_oracle.c`` -- recursive counter with value-indexed boolean occupancy
  arrays (Algorithms 1 and 2 of the paper), prefix enumeration and the
  draw-driven prefix sampler.
* ``orders.py`` -- fill orders written from their definitions, and
  ``trim_tail``, the shortened order whose count equals the whole order's
  (pinned in tests/test_oracle.py on known totals and brute force).
* ``brute.py`` -- row-permutation brute force for tiny orders (independent of
  any cell-by-cell search).
"""
from .core import (  # noqa: F401
    DIAGONAL,
    VSYM,
    build,
    count,
    count_many,
    extend,
    hourglass_classes,
    sample_prefix,
    multiplier,
)
from . import orders  # noqa: F401
