import os
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")


@pytest.fixture(scope="session")
def olib():
    from oracle import oracle
    return oracle.load()


@pytest.fixture(scope="session")
def torch_philox_bin(tmp_path_factory):
    """PyTorch's header-only Philox4x32-10 engine, compiled as a tiny filter program."""
    torch = pytest.importorskip("torch")
    inc = os.path.join(os.path.dirname(torch.__file__), "include")
    if not os.path.exists(os.path.join(inc, "ATen", "core", "PhiloxRNGEngine.h")):
        pytest.skip("torch headers not available")
    out = str(tmp_path_factory.mktemp("tp") / "torch_philox")
    src = os.path.join(ROOT, "tests", "helpers", "torch_philox.cpp")
    subprocess.run(["g++", "-std=c++17", "-O1", "-I", inc, "-o", out, src], check=True)
    return out


def torch_philox_blocks(binary, rows):
    """rows: iterable of (k0, k1, c0, c1, c2, c3) -> (n, 4) uint32 from PyTorch's engine."""
    text = "\n".join(" ".join(str(int(v)) for v in r) for r in rows) + "\n"
    res = subprocess.run([binary], input=text, capture_output=True, text=True, check=True)
    return np.array([[int(v) for v in line.split()] for line in res.stdout.strip().splitlines()],
                    dtype=np.uint64).astype(np.uint32)
