"""What the FP32 path costs in accuracy on the single-domain workload (1024 x 4096,
(rho - <rho>) g with g_y = -1e-4, T = 0.8 T_c, noise +-1e-3): FP32 populations with FP64
reductions against the FP64 GPU run from the same initial state (the FP64 run is held to
the FP64 oracle at 1e-12 by test_gpu_parity.py), over the workload's physical window
(400 steps; it leaves the physical regime after ~500).

Bounds (measured values in the comment beside each, from the report bench.py prints):
max |rho_32 - rho_64| over the domain, the interface height (first crossing of the
coexistence midpoint by the x-averaged profile) and the liquid / vapour densities (max /
min of that profile).
"""
import os

import pytest

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


def test_fp32_against_fp64_on_the_domain_workload():
    import bench

    _, Tc, _ = lbm.lbm_critical_point(bench.A, bench.B, bench.R)
    rv, rl, _ = lbm.lbm_coexistence(bench.A, bench.B, bench.R, bench.TR * Tc)
    rho0 = inputs.column_rho0(bench.NX, bench.NY, rl, rv, bench.LIQUID_ROWS, noise_amp=bench.NOISE, seed=bench.SEED)
    rep = bench.precision_report(lbm, rho0, Tc)
    for row in rep["samples"]:
        assert row["status_fp32"] == lbm.LBM_OK and row["status_fp64"] == lbm.LBM_OK
    assert rep["max_abs_drho"] <= 1.5e-5                # measured 4.2e-6
    assert rep["max_abs_interface_error"] <= 2e-4       # measured 4.5e-5 lattice units
    assert rep["max_abs_rho_l_rel_error"] <= 2.5e-6     # measured 7.1e-7
    assert rep["max_abs_rho_v_rel_error"] <= 2e-4       # measured 6.6e-5 (the vapour thins as it falls)
