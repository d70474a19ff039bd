"""CPU checks of the C-ABI library: it loads, exports every function that
include/lbc.h declares, validates parameters before touching the GPU, and its
host-side building blocks (quadrature rules, discrete equilibrium) agree with
the oracle's independent derivation."""
import ctypes as C
import math

import numpy as np
import pytest

from oracle import quadrature as oq
from oracle.oracle import Oracle
from paper_1810_07803_gb300 import build, lbc


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build()


def test_exports_every_declared_symbol():
    names = lbc.declared_functions()
    assert len(names) >= 11
    raw = C.CDLL(lbc.LIB_PATH)
    for n in names:
        assert hasattr(raw, n), n


def test_build_variant_flag():
    assert lbc.lib().lbc_checked_build() == (1 if lbc.LIB_PATH == build.LIB_CHECKED else 0)


def test_checked_build_exports_every_declared_symbol_and_says_so():
    """The range-checked variant (kernels compiled with LBC_CHECKED) links, exports the same
    functions and reports itself as the checked build (a host call: no GPU needed)."""
    path = build.build(checked=True)
    raw = C.CDLL(path)
    for n in lbc.declared_functions():
        assert hasattr(raw, n), n
    raw.lbc_checked_build.restype = C.c_int
    assert raw.lbc_checked_build() == 1


@pytest.mark.parametrize("bad,msg", [
    (dict(Qx=0), "Qx"), (dict(Qy=65), "Qx and Qy"), (dict(Nx=4), "Nx"), (dict(delta=-1.0), "delta"),
    (dict(T_left=0.0), "temperatures"), (dict(stretch_A=1.0), "stretch_A"), (dict(Nexp_x=4), "Nexp_x"),
    (dict(Qy=2), "Nexp_y"), (dict(Pr=0.0), "Pr"), (dict(u_right=float("nan")), "velocities"),
    (dict(local_dt=2), "local_dt"), (dict(local_dt=1, dt=1e-3), "automatic"), (dict(half_channel=3), "half_channel"),
    (dict(half_channel=1, u_left=0.1, u_right=0.1), "symmetric walls"),
    (dict(half_channel=1, T_left=0.9, T_right=1.1), "symmetric walls"),
    (dict(compensated=2, precision="fp32"), "compensated"), (dict(compensated=1), "FP32 state only"),
])
def test_create_rejects_bad_parameters(bad, msg):
    with pytest.raises(lbc.LbcError) as e:
        lbc.Solver(bad)
    assert e.value.status == lbc.EINVAL
    assert msg in str(e.value)


@pytest.mark.parametrize("Q", [1, 2, 4, 7, 16, 24, 50])
def test_host_half_range_rule_matches_oracle(Q):
    z, w = lbc.quadrature(Q, True)
    r = oq.HalfRangeRule(Q)
    np.testing.assert_allclose(z, [float(v) for v in r.z], rtol=2e-14 if Q < 30 else 1e-13)
    np.testing.assert_allclose(w, [float(v) for v in r.w], rtol=5e-14 if Q < 30 else 1e-12)


@pytest.mark.parametrize("Q", [1, 3, 4, 7, 20, 24])
def test_host_full_range_rule_matches_oracle(Q):
    y, w = lbc.quadrature(Q, False)
    r = oq.FullRangeRule(Q)
    np.testing.assert_allclose(y, [float(v) for v in r.y], rtol=1e-14, atol=1e-15)
    np.testing.assert_allclose(w, [float(v) for v in r.w], rtol=1e-13)


def test_quadrature_rejects_bad_order():
    with pytest.raises(lbc.LbcError):
        lbc.quadrature(0, True)
    with pytest.raises(lbc.LbcError):
        lbc.quadrature(65, False)


@pytest.mark.parametrize("Qx,Qy,p0", [(4, 4, 1.0), (7, 7, 1.0), (16, 20, 1.0), (24, 24, 1.0), (10, 6, 1.3)])
@pytest.mark.parametrize("u,T", [(0.0, 1.0), (0.2, 1.3), (-0.35, 0.6), (0.05, 0.18), (0.4, 1.82)])
def test_host_equilibrium_matches_oracle(Qx, Qy, p0, u, T):
    """The product's stable Gauss-sum projection against the oracle's binary128
    evaluation of Eqs. gx and gy: weighted values agree to ~1e-14."""
    params = dict(Qx=Qx, Qy=Qy, p0=p0, Nx=8)
    gx, gy = lbc.equilibrium(params, u, -0.7 * u, T)
    o = Oracle(params)
    rx, ry = o.equilibrium_factors(u, -0.7 * u, T)
    wx = np.concatenate([o.tab["wx"], o.tab["wx"]])
    wy = o.tab["wy"]
    assert np.max(np.abs(wx * (gx - rx))) <= 2e-14 * np.max(np.abs(wx * rx))
    assert np.max(np.abs(wy * (gy - ry))) <= 2e-14 * np.max(np.abs(wy * ry))


def test_library_is_not_a_cpu_fallback():
    """Without a GPU the solver refuses to run instead of computing on the CPU."""
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(lbc.LbcError) as e:
        lbc.Solver(dict(Qx=4, Qy=4, Nx=16))
    assert e.value.status == lbc.ECUDA


@pytest.mark.parametrize("bad,msg", [
    (dict(tab_T=[1.0], tab_mu=[1.0], tab_Pr=[0.7]), "2 to 256 entries"),
    (dict(tab_T=[1.0, 0.5], tab_mu=[1.0, 1.2], tab_Pr=[0.7, 0.7]), "strictly increasing"),
    (dict(tab_T=[0.5, 1.0], tab_mu=[1.0, -1.2], tab_Pr=[0.7, 0.7]), "viscosities"),
    (dict(tab_T=[0.5, 1.0], tab_mu=[1.0, 1.2], tab_Pr=[0.7, 0.0]), "Prandtl"),
])
def test_create_rejects_bad_viscosity_tables(bad, msg):
    with pytest.raises(lbc.LbcError) as e:
        lbc.Solver(dict(mu_law="table", **bad))
    assert e.value.status == lbc.EINVAL
    assert msg in str(e.value)


@pytest.mark.parametrize("opt,msg", [(dict(local_dt=1), "local_dt"), (dict(compensated=1, precision="fp32"), "compensated")])
def test_noalloc_rejects_options_it_has_no_room_for(opt, msg):
    """The allocation-free path refuses local steps (their reference mass would not survive from
    one call to the next) and the compensated state (no remainder buffer), before any device
    access: the state pointer below is never dereferenced."""
    with pytest.raises(lbc.LbcError) as e:
        lbc.step_noalloc(dict(Nx=16, Qx=4, Qy=4, **opt), 0x1000, 1)
    assert e.value.status == lbc.EINVAL
    assert msg in str(e.value)
