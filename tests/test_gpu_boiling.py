"""The paper's phase-formation example (Sec. V) on the GPU: the onset of boiling at the hot
wall falls between the two temperature differences the paper prints
(tests/golden/paper_theory_examples.txt): Delta T / T_c = 0.3381 keeps the liquid at the
bottom wall, 0.3382 forms a vapour layer there. Thermal column of 101 wet nodes (Zou-He
walls), a = 0.5, <rho> = 1.3344 rho_c, rho g with g = 1.5e-5, T_med = 0.75 T_c, c_v = 5,
kappa = 0.02, FP64."""
import os

import numpy as np
import pytest

from oracle import eos
from paper_2301_12869_gb300 import _build, inputs, lbm

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

A, B, R = 0.5, 4.0, 1.0
RHO_C, T_C, _ = eos.critical_point(A, B, R)
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_theory_examples.txt")


@pytest.fixture(scope="module", autouse=True)
def cuda_lib():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    if not os.path.exists(lbm.LIB_PATH):
        _build.build()
    lbm.load()


def golden():
    out = {}
    for line in open(GOLDEN):
        line = line.split("#")[0].strip()
        if line:
            k, v = line.split()[:2]
            out[k] = float(v)
    return out


def layer_forms(dT, post_steps=400000):
    G = golden()
    ny, nx = 101, 4
    T_bot, T_top = (G["T_med_reduced"] + dT / 2) * T_C, (G["T_med_reduced"] - dT / 2) * T_C
    rv, rl, _ = eos.maxwell(G["T_med_reduced"] * T_C, A, B, R)
    rho0 = inputs.column_rho0(nx, ny, rl, rv, 54)
    rho0 *= G["mean_rho_reduced"] * RHO_C / rho0.mean()
    p = lbm.make_params(nx, ny, 0.75 * T_C, "fp64", a=A, form=1, g=(0.0, -G["example2_g"]), thermal=1, T_bot=T_bot,
                        T_top=G["boil_T_top_prerun"] * T_C, wall=lbm.LBM_WALL_ZOU_HE)
    h = lbm.lbm_init(p, rho0)
    try:
        res, steps = np.inf, 0
        while res >= 1e-10 and steps < 2000000:  # equilibrate at the warmer top wall
            lbm.lbm_step(h, 49999)
            lbm.lbm_reduce(h, lbm.LBM_REDUCE_RESIDUAL)
            lbm.lbm_step(h, 1)
            res = lbm.lbm_reduce(h, lbm.LBM_REDUCE_RESIDUAL)[0]
            steps += 50000
        assert res < 1e-10
        p.T_top = T_top
        lbm.lbm_set_params(h, p)
        rho, T = np.empty((ny, nx)), np.empty((ny, nx))
        for _ in range(post_steps // 20000):
            lbm.lbm_step(h, 20000)
            lbm.lbm_moments(h, rho)
            lbm.lbm_get_temperature(h, T)
            rv2, rl2, _ = eos.maxwell(min(T[2, 0], 0.999 * T_C), A, B, R)
            if rho[2, 0] < 0.5 * (rv2 + rl2):
                return True
        assert lbm.lbm_status(h) == 0
        return False
    finally:
        lbm.lbm_destroy(h)


def test_boiling_onset_between_the_papers_values():
    G = golden()
    assert not layer_forms(G["boil_dT_stays"])
    assert layer_forms(G["boil_dT_boils"])
