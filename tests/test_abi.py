"""C-ABI checks that need no GPU: the library builds and loads, exports every
symbol include/lbm.h declares, validates parameters before touching the device,
and its host thermodynamics (an equal-chemical-potential solver) agrees with the
oracle's equal-area Maxwell construction."""
import ctypes
import math
import os
import re

import pytest

from paper_2301_12869_gb300 import _build, lbm

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    if not os.path.exists(lbm.LIB_PATH):
        _build.build()
    return lbm.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "lbm.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(lbm_[a-z_]+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert len(names) >= 15
    for n in names:
        assert hasattr(lib, n), n
    assert sorted(lbm.EXPORTS) == names


def test_params_struct_layout_matches(lib):
    p = lbm.lbm_params_default()
    assert p.size == ctypes.sizeof(lbm.lbm_params)
    # paper defaults: a = 0.5, b = 4, R = 1, sigma = 1.385, every tau = 1 (Sec. IV)
    assert (p.a, p.b, p.R, p.sigma, p.G) == (0.5, 4.0, 1.0, 1.385, -1.0)
    assert all(getattr(p, t) == 1.0 for t in ("tau_rho", "tau_e", "tau_varsigma", "tau_j", "tau_q", "tau_nu"))
    assert math.isnan(p.rho_ref)
    # isothermal by default; c_v = 5 and kappa = 0.02 of Sec. IV for the thermal variant
    assert p.thermal == 0 and (p.c_v, p.kappa) == (5.0, 0.02)


@pytest.mark.parametrize(
    "change, fragment",
    [
        (dict(nx=3), "multiple of 2"),
        (dict(nx=0), "positive"),
        (dict(tau_nu=0.5), "> 1/2"),
        (dict(G=1.0), "negative"),
        (dict(gravity_form=3), "gravity_form"),
        (dict(size=8), "params.size"),
        (dict(T=-1.0), "T > 0"),
        (dict(thermal=2), "thermal must be 0 or 1"),
        (dict(wall=2), "wall must be"),
        (dict(reserved1=1), "reserved1"),
        (dict(thermal=1), "T_bot > 0"),  # wall temperatures unset
        (dict(thermal=1, T_bot=0.02, T_top=0.02, c_v=0.0), "c_v > 0"),
        (dict(thermal=1, T_bot=0.02, T_top=0.02, kappa=-1.0), "kappa >= 0"),
    ],
)
def test_init_rejects_bad_parameters(lib, change, fragment):
    import numpy as np

    p = lbm.make_params(4, 10, 0.02, "fp64")
    for k, v in change.items():
        setattr(p, k, v)
    with pytest.raises(lbm.LbmError) as ei:
        lbm.lbm_init(p, np.full((10, 4), 0.1))
    assert ei.value.code == lbm.LBM_EINVAL
    assert fragment in str(ei.value)


def test_fp32_needs_16_byte_rows(lib):
    import numpy as np

    p = lbm.make_params(6, 10, 0.02, "fp32")
    with pytest.raises(lbm.LbmError, match="multiple of 4"):
        lbm.lbm_init(p, np.full((10, 6), 0.1))


def test_null_rho0_rejected(lib):
    p = lbm.make_params(4, 10, 0.02)
    h = ctypes.c_void_p()
    rc = lib.lbm_init(ctypes.byref(p), None, 0, None, ctypes.byref(h))
    assert rc == lbm.LBM_EINVAL and "NULL" in lbm.lbm_last_error()


@pytest.mark.parametrize("a", [0.25, 0.5])
def test_host_thermodynamics_agree_with_oracle(lib, a):
    from oracle import eos

    rc_o, Tc_o, pc_o = eos.critical_point(a, 4.0, 1.0)
    rc_l, Tc_l, pc_l = lbm.lbm_critical_point(a, 4.0, 1.0)
    assert rc_l == pytest.approx(rc_o, rel=1e-12)
    assert Tc_l == pytest.approx(Tc_o, rel=1e-12)
    assert pc_l == pytest.approx(pc_o, rel=1e-12)
    for Tr in (0.7, 0.8, 0.85, 0.95):
        rv_o, rl_o, ps_o = eos.maxwell(Tr * Tc_o, a, 4.0, 1.0)
        rv_l, rl_l, ps_l = lbm.lbm_coexistence(a, 4.0, 1.0, Tr * Tc_o)
        assert rv_l == pytest.approx(rv_o, rel=1e-10)
        assert rl_l == pytest.approx(rl_o, rel=1e-10)
        assert ps_l == pytest.approx(ps_o, rel=1e-10)


def test_coexistence_rejects_supercritical(lib):
    _, Tc, _ = lbm.lbm_critical_point(0.25, 4.0, 1.0)
    with pytest.raises(lbm.LbmError):
        lbm.lbm_coexistence(0.25, 4.0, 1.0, 1.01 * Tc)


def test_binding_defines_each_name_once():
    """A later `def` of the same name would silently replace an earlier one in the binding."""
    import ast

    for mod in ("lbm.py", "partition.py"):
        path = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "paper_2301_12869_gb300", mod)
        tree = ast.parse(open(path).read())
        names = [n.name for n in tree.body if isinstance(n, (ast.FunctionDef, ast.ClassDef))]
        dup = {n for n in names if names.count(n) > 1}
        assert not dup, (mod, dup)


def test_slab_calls_reach_the_library_without_a_gpu():
    """The slab wrappers marshal their arguments and the library answers (no device here:
    LBM_ECUDA from the device query, or the binding's own refusal of host tensors)."""
    import torch

    p = lbm.make_params(16, 10, 0.02, "fp64", a=0.25)
    s = lbm.make_slab(0, 5)
    try:
        n = lbm.lbm_slab_partials(p, s)
        assert n >= 1  # a machine with a GPU
    except lbm.LbmError as exc:
        assert exc.code == lbm.LBM_ECUDA
    with pytest.raises(lbm.LbmError, match="outside"):
        lbm.lbm_slab_partials(p, lbm.make_slab(8, 4))
    f = torch.zeros((9, 9, 16), dtype=torch.float64)
    with pytest.raises(ValueError, match="CUDA"):
        lbm.lbm_slab_step(p, s, f, f, None, f, f)
