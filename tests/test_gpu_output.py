"""Pressure and transmission-loss snapshots (PE3D_OPT_OUTPUT) against the
oracle (needs a GB300).

The library forms p = u H0^(1)(k0 r) (Sec. 2; Fig. 2), with H0^(1)
evaluated in FP64 per range step, and TL = -20 log10 |p| (Fig. 2) in
the snapshot stores.  The oracle applies the same definitions to its own FP64
march (scipy's hankel1, pinned in test_oracle_output.py).

Tolerances: p is compared in relative L2 per snapshot like the field (FP64
1e-10; FP32 2e-5, the field's bound plus one complex64 rounding of H).  TL is
compared through |p| = 10^(-TL/20), whose relative L2 error carries the same
bounds; this also holds near nodes of the field, where TL itself is
ill-conditioned.
"""
import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {False: 1e-10, True: 2e-5}


@pytest.fixture(scope="module")
def P():
    from paper_1711_00005_gb300 import build
    build.build()
    import paper_1711_00005_gb300 as P
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return P


def _march(P, wl, fp32, output, exec_mode=None, rc_every=0):
    g = wl.grid
    cdt = np.complex64 if fp32 else np.complex128
    with P.Plan.for_grid(g, fp32=fp32, output=output, exec_mode=exec_mode) as plan:
        if rc_every:
            P.pe3d_set_option(plan.h, P.PE3D_OPT_RC_EVERY, rc_every)
        plan.set_medium(torch.from_numpy(wl.n2).cuda(), wl.slice_r)
        out = plan.march(torch.from_numpy(wl.u0.astype(cdt)).cuda(), g.r0, g.steps, g.stride)
        torch.cuda.synchronize()
    return out.cpu().numpy()


def _rel(a, b):
    return max(np.linalg.norm((x - y).ravel()) / np.linalg.norm(y.ravel()) for x, y in zip(a, b))


CASES = [(300, 70, False, 3, 12, 4, 11), (257, 33, True, 2, 10, 5, 12), (5, 2, False, 1, 6, 2, 13)]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}{'p' if c[2] else 'w'}")
@pytest.mark.parametrize("fp32", [False, True], ids=["fp64", "fp32"])
@pytest.mark.parametrize("exec_mode", [None, 1], ids=["persistent", "stream"])
def test_pressure_and_tl(P, oracle_lib, case, fp32, exec_mode):
    Nz, Nt, periodic, K, steps, stride, seed = case
    wl = workloads.random_case(Nz, Nt, periodic=periodic, K=K, steps=steps, seed=seed, stride=stride)
    g = wl.grid
    u_ref = oracle_lib.march(g, wl.n2, wl.slice_r, wl.u0)
    p_ref = oracle.pressure(u_ref, oracle.snapshot_ranges(g.r0, g.dr, g.steps, g.stride), g.k0)
    p = _march(P, wl, fp32, P.PE3D_OUT_PRESSURE, exec_mode)
    assert p.dtype == (np.complex64 if fp32 else np.complex128)
    assert _rel(p, p_ref) <= TOL[fp32]
    tl = _march(P, wl, fp32, P.PE3D_OUT_TL, exec_mode)
    assert tl.dtype == (np.float32 if fp32 else np.float64) and tl.shape == p_ref.shape
    assert _rel(10.0 ** (-tl.astype(np.float64) / 20.0), np.abs(p_ref)) <= TOL[fp32]
    # the field itself is unchanged by the option
    u = _march(P, wl, fp32, P.PE3D_OUT_FIELD, exec_mode)
    assert _rel(u, u_ref) <= TOL[fp32]


def test_tl_through_host_buffers_and_correction(P, oracle_lib):
    """TL into a host buffer (staged copy of half-size real snapshots) and on
    the steps the FP64 residual correction stores itself."""
    wl = workloads.random_case(200, 40, periodic=False, K=2, steps=12, seed=14, stride=3)
    g = wl.grid
    u_ref = oracle_lib.march(g, wl.n2, wl.slice_r, wl.u0)
    p_ref = oracle.pressure(u_ref, oracle.snapshot_ranges(g.r0, g.dr, g.steps, g.stride), g.k0)
    with P.Plan.for_grid(g, fp32=True, output=P.PE3D_OUT_TL) as plan:
        P.pe3d_set_option(plan.h, P.PE3D_OPT_RC_EVERY, 3)
        plan.set_medium(wl.n2, wl.slice_r)
        host = np.full((g.steps // g.stride, g.Ntheta, g.Nz), np.nan, np.float32)
        P.pe3d_march(plan.h, wl.u0.astype(np.complex64), g.r0, g.steps, g.stride, host)
    assert np.all(np.isfinite(host))
    assert _rel(10.0 ** (-host.astype(np.float64) / 20.0), np.abs(p_ref)) <= TOL[True]


def test_output_option_is_checked(P):
    g = workloads.random_case(8, 4, periodic=False, steps=2).grid
    with P.Plan.for_grid(g) as plan:
        with pytest.raises(P.PE3DError):
            P.pe3d_set_option(plan.h, P.PE3D_OPT_OUTPUT, 3)
        P.pe3d_set_option(plan.h, P.PE3D_OPT_OUTPUT, P.PE3D_OUT_TL)
        assert P.pe3d_get_option(plan.h, P.PE3D_OPT_OUTPUT) == P.PE3D_OUT_TL
