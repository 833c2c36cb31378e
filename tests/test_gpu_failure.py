"""Failure detection on the GPU without a fault: the bounded device-side wait that every
mbarrier wait of the library uses is made to run out (a barrier that nothing arrives on,
bounded at ~1 ms); the kernel records LBM_ETIMEOUT in a status word instead of trapping,
the host reads it, and the context stays usable - a following FP64 step still matches the
oracle."""
import os

import numpy as np
import pytest

from oracle import eos
from oracle import lbm as olbm
from paper_2301_12869_gb300 import _build, inputs, lbm

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def cuda_lib():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    if not os.path.exists(lbm.LIB_PATH):
        _build.build()
    lbm.load()


def test_bounded_wait_gives_up_and_the_context_stays_usable():
    for cycles in (2_000_000, 50_000):
        assert lbm.lbm_wait_bound_selftest(cycles) == lbm.LBM_ETIMEOUT
    with pytest.raises(lbm.LbmError, match="cycles"):
        lbm.lbm_wait_bound_selftest(0)
    _, Tc, _ = eos.critical_point(0.25, 4.0, 1.0)
    rv, rl, _ = eos.maxwell(0.85 * Tc, 0.25, 4.0, 1.0)
    nx, ny = 8, 24
    rho0 = inputs.column_rho0(nx, ny, rl, rv, ny // 2, width=3.0)
    p = lbm.make_params(nx, ny, 0.85 * Tc, "fp64", a=0.25, form=1, g=(0.0, -2e-5))
    h = lbm.lbm_init(p, rho0)
    try:
        f0 = np.empty((9, ny, nx))
        lbm.lbm_get_state(h, f0)
        lbm.lbm_step(h, 3)
        f = np.empty_like(f0)
        lbm.lbm_get_state(h, f)
        assert lbm.lbm_status(h) == lbm.LBM_OK
    finally:
        lbm.lbm_destroy(h)
    op = olbm.Params(nx=nx, ny=ny, a=0.25, T=0.85 * Tc, g=(0.0, -2e-5), form=1)
    assert np.max(np.abs(f - olbm.run(f0, op, 3))) <= 1e-14
