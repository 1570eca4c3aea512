"""Failure detection without a GPU fault: a device wait on a status word that
nothing sets runs out its bound, the kernel records a timeout and returns,
the host reads DDQMC_ERR_TIMEOUT, and the context keeps working."""
import time

import numpy as np
import pytest

from oracle import oracle as O
from tests import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ddqmc():
    import __graft_entry__ as g
    g.build()
    from paper_1802_05931_gb300 import ddqmc as d
    return d


def test_bounded_wait_reports_timeout_and_context_survives(ddqmc):
    t0 = time.perf_counter()
    rc = ddqmc.ddqmc_wait_selftest()
    el = time.perf_counter() - t0
    assert rc == -5                     # DDQMC_ERR_TIMEOUT
    assert el < 30.0
    # the same process keeps stepping bit-exact with the oracle
    args, kw = W.run_kwargs(W.C1)
    gpu = ddqmc.Run(*args, **kw)
    cpu = O.OracleRun(*args, **kw)
    gpu.step(50)
    cpu.step(50)
    for a, b in zip(gpu.export(), cpu.export()):
        assert np.array_equal(a, b)
