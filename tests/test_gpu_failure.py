"""Failure detection without a GPU fault: the library's bounded device waits.

Every spin-wait in the library's kernels (bulk-copy completions of the
persistent Green pass, tensor-core commits of the convolution) is bounded by
a wall-clock limit; when it runs out the kernel drains its own copies in
flight, sets a device error word and returns, and the host call reports
FH_ERR_TIMEOUT with the context still usable.  These tests make a wait run
out on purpose -- on an mbarrier that nothing completes, with nothing in
flight -- and check the status and the recovery, and check that an explicit
limit leaves the waits that do complete correct.  Nothing here faults, traps
or hangs a GPU.
"""
import numpy as np
import pytest

import oracle
from paper_1004_1122_gb300 import microstructure as micro

from gpu_util import cuda_or_skip

pytestmark = pytest.mark.gpu

TIMEOUT = 8  # FH_ERR_TIMEOUT


def test_wait_on_a_barrier_nothing_completes_gives_up():
    """fh_wait_selftest waits on an mbarrier that nothing completes: the wait
    must spin for its limit, give up, and report FH_ERR_TIMEOUT; the device
    stays usable afterwards."""
    torch = cuda_or_skip()
    import time

    from paper_1004_1122_gb300 import fh

    assert fh.wait_selftest(1e-3) == TIMEOUT
    t0 = time.perf_counter()
    assert fh.wait_selftest(0.2) == TIMEOUT
    assert time.perf_counter() - t0 >= 0.2  # it waited its whole limit, no longer bounded by anything else
    # the device is still usable: a solve right after succeeds
    phase = micro.centred_disk(27, 0.3)
    L = micro.isotropic_table([1.0, 10.0], 2)
    with fh.Solver(phase, L, precision="fp64") as s:
        _, _, info = s.solve([1.0, 0.0], tol=1e-10)
    assert info["status"] == "FH_OK"


def test_persistent_green_pass_with_an_explicit_wait_limit(monkeypatch):
    """With an explicit limit the bulk-copy waits of the persistent Green pass
    cap their suspension by it; a generous explicit limit leaves the solve
    unchanged (oracle parity), and restoring the default keeps it so."""
    torch = cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    monkeypatch.setenv("FH_GREEN_PIPE", "1")   # select the persistent Green pass
    monkeypatch.setenv("FH_TUNE_CACHE", "")    # no cached shape overrides the choice
    phase = micro.rsa_disks(243, 0.3, 6, 14, seed=micro.config_seed(9, 1))
    L = micro.isotropic_table([1.0, 10.0], 2)
    L0 = oracle.reference_medium(L)
    xo, _ = oracle.cg(phase, L, L0, [1.0, 0.0], tol=1e-13)
    for limit in (1.0, 0.0):
        try:
            fh.set_wait_limit(limit)
            with fh.Solver(phase, L, precision="fp32_refined") as s:
                x, _, info = s.solve([1.0, 0.0], tol=1e-9, method="cg")
        finally:
            fh.set_wait_limit(0.0)
        assert info["status"] == "FH_OK", (limit, info)
        err = np.linalg.norm(x.cpu().numpy() - xo) / np.linalg.norm(xo)
        assert err < 1e-6, (limit, err)


def test_wait_limit_arguments():
    cuda_or_skip()
    from paper_1004_1122_gb300 import fh

    with pytest.raises(fh.FhError):
        fh.set_wait_limit(-1.0)
    assert fh.wait_selftest(0.0) == 1  # FH_ERR_ARG
