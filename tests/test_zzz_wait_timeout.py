"""Failure detection without a GPU fault: a bounded device-side wait is made to run out and
its error reaches the host, after which the same handle solves correctly.

The bulge chasing (S1c) pipelines sweeps across the CTAs of one cooperative launch; step k of
sweep s waits for step k+1 of sweep s-1 to be published.  The test hook drops every progress
message of sweep 0 (a message dropped on the host's orders), so sweep 1's wait runs out after
the short limit set here; it records GEP_ERR_TIMEOUT and returns, the waits behind it see the
error and return, and the launch ends.  No trap, assert, bad address or unbounded loop is
involved.  This file sorts last so that it runs after every other GPU test.
"""
import numpy as np
import pytest

import gep_inputs as gi

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gep():
    import torch
    assert torch.cuda.is_available(), "GPU tests need CUDA"
    from paper_1504_06443_gb300 import build
    build.build()
    import paper_1504_06443_gb300 as g
    g.load()
    return g


def test_bulge_wait_times_out_and_handle_recovers(gep, oracle_lib):
    import torch
    M, b = 300, 16
    C = gi.random_symmetric(M, seed=11)
    Cd = torch.as_tensor(C, device="cuda")
    h = gep.Handle()
    try:
        h.set_wait_fault(drop_sweep=0, wait_limit_s=0.05)
        gep.tridiag_2stage(Cd, b=b, handle=h)      # enqueues; the error is on the device
        assert h.info() == gep.ERR_TIMEOUT
        # the hook and the recorded error cleared, the same handle and context work again
        h.set_wait_fault(drop_sweep=-1, wait_limit_s=4.0)
        h.reset_info()
        d, e, _, _, _ = gep.tridiag_2stage(Cd, b=b, handle=h)
        assert h.info() == 0
        w_ref, _, info = oracle_lib.gep_solve(C, np.eye(M), want_vectors=False)
        assert info == 0
        wT = np.sort(oracle_lib.bisect(d.cpu().numpy(), e.cpu().numpy()))
        nC = max(float(np.max(np.abs(w_ref))), 1.0)
        assert np.max(np.abs(wT - np.sort(w_ref))) <= 200 * M * 2.0 ** -52 * nC
    finally:
        h.close()


def test_wait_fault_arguments_checked(gep):
    h = gep.Handle()
    try:
        for bad in [(-2, 1.0), (0, 0.0), (0, 5.0), (0, float("nan"))]:
            with pytest.raises(gep.GepError):
                h.set_wait_fault(*bad)
        h.set_wait_fault(-1, 4.0)
    finally:
        h.close()
