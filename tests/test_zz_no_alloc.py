"""lbm_step_noalloc, the entry point that allocates no device memory.

Some callers cannot call cudaMalloc (a host loop that must not stall other
streams on an allocation's implicit synchronisation, a process whose device
memory another allocator reserved up front, a plug-in that may not allocate).
For them liblbm runs one step on caller-owned arrays with its scratch in a
static __device__ array. This test calls it through the C ABI twice in a row,
each call continuing from the previous call's output, and compares each result
with lbm_step on a handle from the same initial state, within the tolerances of
the parity tests (1e-14 for FP64, 1e-6 for FP32). The file sorts last so that a
run stopping at the first failure has already run every other test.
"""
import os

import numpy as np
import pytest

from paper_2301_12869_gb300 import _build, inputs, lbm

pytestmark = pytest.mark.gpu

A, B, R = 0.25, 4.0, 1.0
W = inputs.LATTICE_WEIGHTS


@pytest.fixture(scope="module", autouse=True)
def cuda_lib():
    import torch

    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    if not os.path.exists(lbm.LIB_PATH):
        _build.build()
    lbm.load()


@pytest.mark.parametrize("precision, nx, ny, tol, form, wall", [
    ("fp64", 64, 40, 1e-14, 2, "bounce_back"),
    ("fp32", 64, 40, 1e-6, 2, "bounce_back"),
    ("fp32", 1028, 300, 1e-6, 2, "bounce_back"),
    # Eq. Gravity_1: no mass partials are formed for the call
    ("fp64", 64, 40, 1e-14, 1, "bounce_back"),
    ("fp32", 64, 40, 1e-6, 1, "bounce_back"),
    # Zou-He wet-node walls, both gravity forms
    ("fp64", 64, 40, 1e-14, 1, "zou_he"),
    ("fp64", 64, 40, 1e-14, 2, "zou_he"),
    ("fp32", 68, 24, 1e-6, 2, "zou_he"),
])
def test_noalloc_step_matches_handle_two_calls_in_a_row(precision, nx, ny, tol, form, wall):
    import torch

    _, Tc, _ = lbm.lbm_critical_point(A, B, R)
    T = 0.8 * Tc
    rv, rl, _ = lbm.lbm_coexistence(A, B, R, T)
    rho0 = inputs.column_rho0(nx, ny, rl, rv, ny // 2, noise_amp=1e-3)
    rho_ref = 0.0 if precision == "fp64" else float(rho0.mean())
    wall_id = lbm.LBM_WALL_ZOU_HE if wall == "zou_he" else lbm.LBM_WALL_BOUNCE_BACK
    kw = dict(a=A, b=B, R=R, form=form, g=(1e-5, -1e-4), rho_ref=rho_ref, wall=wall_id)
    h = lbm.lbm_init(lbm.make_params(nx, ny, T, precision, **kw), rho0)
    try:
        f_abs = np.empty((9, ny, nx))
        lbm.lbm_get_state(h, f_abs)
        dev = (f_abs - W[:, None, None] * rho_ref)          # the handle's stored deviations
        dtype = torch.float32 if precision == "fp32" else torch.float64
        f_in = torch.from_numpy(dev).to("cuda", dtype)
        f_a = torch.empty_like(f_in)
        f_b = torch.empty_like(f_in)
        q = lbm.make_params(nx, ny, T, precision, **kw)
        for src, dst in ((f_in, f_a), (f_a, f_b)):
            lbm.lbm_step_noalloc(q, src, dst)
            lbm.lbm_step(h, 1)
            lbm.lbm_get_state(h, f_abs)
            got = dst.double().cpu().numpy() + W[:, None, None] * rho_ref
            assert np.max(np.abs(got - f_abs)) <= tol
    finally:
        lbm.lbm_destroy(h)


def test_noalloc_reports_a_nonphysical_state():
    """A node with negative density makes the call return LBM_ENONPHYS (a status word the
    kernel sets, read back by the call), and the next call on a physical state is clean:
    the status word of the shared array is cleared at the start of every call."""
    import torch

    nx, ny = 16, 12
    p = lbm.make_params(nx, ny, 0.07, "fp64", a=A, form=2, g=(0.0, -1e-5))
    good = torch.from_numpy(np.repeat(W[:, None, None] * 0.1, ny, 1).repeat(nx, 2)).cuda()
    bad = good.clone()
    bad[:, 5, 7] = torch.from_numpy(-0.2 * W).cuda()  # rho = -0.2 at (x, y) = (7, 5)
    out = torch.empty_like(good)
    with pytest.raises(lbm.LbmError, match="LBM_ENONPHYS"):
        lbm.lbm_step_noalloc(p, bad, out)
    lbm.lbm_step_noalloc(p, good, out)
    assert torch.allclose(out, good, rtol=0, atol=1e-15)  # the uniform rest state is a fixed point


def test_noalloc_rejects_bad_arguments():
    import ctypes

    import torch

    p = lbm.make_params(8, 8, 0.02, "fp32", a=A)
    buf = torch.zeros((9, 8, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(lbm.LbmError, match="distinct"):
        lbm.lbm_step_noalloc(p, buf, buf)
    # the binding refuses host tensors, another real type and a wrong element count ...
    with pytest.raises(ValueError, match="CUDA"):
        lbm.lbm_step_noalloc(p, buf.cpu(), torch.empty_like(buf))
    with pytest.raises(ValueError, match="float32"):
        lbm.lbm_step_noalloc(p, buf.double(), torch.empty_like(buf))
    with pytest.raises(ValueError, match="9 nx ny"):
        lbm.lbm_step_noalloc(p, buf[:8], torch.empty_like(buf))
    # ... and the C side refuses a host address passed straight through the ABI
    host = np.zeros(9 * 8 * 8, dtype=np.float32)
    rc = lbm.load().lbm_step_noalloc(ctypes.byref(p), ctypes.c_void_p(host.ctypes.data),
                                     ctypes.c_void_p(torch.empty_like(buf).data_ptr()), None)
    assert rc == lbm.LBM_EINVAL
    assert b"device memory" in lbm.load().lbm_last_error(None)
    # a device address off the 16-byte boundary the step's bulk copies need (nothing launched)
    out = torch.empty_like(buf)
    rc = lbm.load().lbm_step_noalloc(ctypes.byref(p), ctypes.c_void_p(buf.data_ptr() + 4),
                                     ctypes.c_void_p(out.data_ptr()), None)
    assert rc == lbm.LBM_EINVAL
    assert b"16-byte" in lbm.load().lbm_last_error(None)
    p.nx = 6
    with pytest.raises(lbm.LbmError, match="multiple of 4"):
        lbm.lbm_step_noalloc(p, buf[:, :, :6].contiguous(), torch.empty_like(buf[:, :, :6]).contiguous())
