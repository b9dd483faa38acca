"""The bounded device waits on the GPU: co-resident CTAs wait at the sweep kernels' grid barrier
for an arrival that nothing makes.  The wait must give up on its own, record ISF_ERR_TIMEOUT in
the status word the host reads, and leave the context usable: a film run right after is still
bit-exact with the oracle.  No fault, no trap, no hang."""
import time

import numpy as np
import pytest

from paper_1205_5588_gb300 import workloads as W
from tests.gpu_common import assert_same_run, gpu_lib, run_gpu, run_oracle

pytestmark = pytest.mark.gpu

ISF_ERR_TIMEOUT = -6


@pytest.fixture(scope="module")
def I():
    return gpu_lib()


def test_grid_barrier_wait_gives_up_and_reports(I):
    t0 = time.perf_counter()
    status, where = I.debug_wait_timeout(4)
    elapsed = time.perf_counter() - t0
    assert status == ISF_ERR_TIMEOUT and where == 1, (status, where)
    assert elapsed < 60.0, elapsed           # bounded: the wait gives up by itself
    # the context is still usable: a film runs and matches the oracle
    spec = {"heights": W.fractal_heights(24, 40, 0.7, 1, 3, seed=11), "layers": 3, "seed": 5, "init": "random"}
    sched = W.schedule(np.array([2.5, 4.0]), np.array([0.5, -0.5]), np.array([1, 0]), np.array([3, 4]))
    assert_same_run(run_gpu(I, spec, sched), run_oracle(spec, sched))
