"""The device-side failure path without a GPU fault: a bounded wait that runs
out raises the context's error flag, the next syncing call reports
LBM_ERR_TIMEOUT and clears it, and the context keeps working (the step kernels'
waits for staged rows use the same bounded wait)."""
import numpy as np
import pytest

import workloads as W
from lbmtest import gpu_sim, split_preset

pytestmark = pytest.mark.gpu


def test_wait_timeout_is_reported_and_the_context_stays_usable():
    from paper_1902_00530_gb300 import _abi
    model, d = split_preset("CIL_RHO1")
    sim = gpu_sim(model, d, 64, 32, W.seed(1), W.INIT_CONFIG2, tuning=(4, 16, 2, 3))
    sim.step(5)
    before = sim.get_state(host=True).numpy().copy()
    assert sim.lib.lbm_check_wait_timeout(sim.ctx) == _abi.LBM_ERR_TIMEOUT
    assert b"timed out" in sim.lib.lbm_last_error(sim.ctx)
    # the flag was cleared and nothing else changed: the context steps on
    np.testing.assert_array_equal(sim.get_state(host=True).numpy(), before)
    sim.step(5)
    ob = sim.observables()  # a syncing call that reads the flag: clean
    assert np.isfinite(ob["phi"]) and ob["t"] == 10
    sim.close()
