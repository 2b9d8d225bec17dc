import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a)")
    config.addinivalue_line("markers", "slow: takes more than a few seconds")


def golden_counts():
    """Parse tests/golden/paper_counts.txt into {key: int}."""
    out = {}
    with open(os.path.join(ROOT, "tests", "golden", "paper_counts.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, val = line.split()[:2]
            out[key] = int(val)
    return out


def fig1_order():
    """The Fig. 1 fill order as a list of (i, j), positions 1..72."""
    pos = {}
    with open(os.path.join(ROOT, "tests", "golden", "fig1_order_dls9.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for i, r in enumerate(rows):
        for j, tok in enumerate(r):
            if tok != "-":
                pos[int(tok)] = (i, j)
    return [pos[k] for k in sorted(pos)]


@pytest.fixture(scope="session")
def golden():
    return golden_counts()


@pytest.fixture(scope="session")
def dls():
    """The product binding, with libdls.so built in-tree if needed (nvcc)."""
    from paper_1709_02599_gb300 import build as _build
    _build.build()
    import paper_1709_02599_gb300 as m
    m.lib()
    return m


@pytest.fixture(scope="session")
def emulated(tmp_path_factory):
    """The library built for the CPU on the stand-in CUDA runtime of
    tests/host_kernels (see host_emulation.py); skipped without g++."""
    import host_emulation
    d = tmp_path_factory.mktemp("host_emulation")
    exe = host_emulation.build(str(d))
    if exe is None:
        pytest.skip("g++ is not available")
    return host_emulation.Emulated(exe, str(d))
