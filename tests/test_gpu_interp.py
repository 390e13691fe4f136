"""Range-dependent medium refreshed every step: n^2 interpolated linearly in
range between the slices around r* and the depth systems set up in FP64 for
every range step (Fig. 2's update of A, run per step), against the oracle's
interpolating march (pinned in tests/pins.py:check_interp_linear).

Tolerances as in test_gpu_parity.py: 1e-10 for the FP64 march, 2e-5 for
FP32 on these short cases, 2e-6 for FP32 corrected every step.
"""
import numpy as np
import pytest

import workloads
from test_gpu_parity import TOL32, TOL64, gpu_march, relerrs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1711_00005_gb300 import build
    build.build()
    import paper_1711_00005_gb300 as P
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return P


@pytest.mark.parametrize("periodic", [False, True], ids=["walled", "periodic"])
@pytest.mark.parametrize("exec_mode", [1, 3], ids=["stream", "persistent"])
@pytest.mark.parametrize("fp32", [False, True], ids=["fp64", "fp32"])
def test_interp_parity(P, oracle_lib, periodic, exec_mode, fp32):
    """Five slices over twelve steps (several tiles, ragged tails)."""
    wl = workloads.random_case(300, 41, periodic=periodic, K=5, steps=12, seed=141 + periodic, stride=3)
    ref = oracle_lib.march(wl.grid, wl.n2, wl.slice_r, wl.u0, interp=True)
    got, _ = gpu_march(P, wl, fp32=fp32, exec_mode=exec_mode, interp=True)
    assert relerrs(got, ref).max() < (TOL32 if fp32 else TOL64)
    # the interpolated medium is a different march from the piecewise one
    assert relerrs(got, oracle_lib.march(wl.grid, wl.n2, wl.slice_r, wl.u0)).max() > 1e-6


@pytest.mark.parametrize("fp32", [False, True], ids=["fp64", "fp32"])
def test_interp_linear_medium(P, oracle_lib, fp32):
    """Slices sampling a medium linear in range, steps before, inside and after
    their span, with the centred Y as well."""
    wl = workloads.range_linear_case(257, 40, periodic=True, steps=9, seed=143, stride=1)
    for mid in (False, True):
        ref = oracle_lib.march(wl.grid, wl.n2, wl.slice_r, wl.u0, interp=True, y_midpoint=mid)
        got, _ = gpu_march(P, wl, fp32=fp32, interp=True, y_midpoint=mid)
        assert relerrs(got, ref).max() < (TOL32 if fp32 else TOL64)


def test_interp_with_correction(P, oracle_lib):
    """The FP64 residual forms the interpolated n^2 of each step."""
    wl = workloads.random_case(120, 33, periodic=False, K=4, steps=8, seed=145, stride=2)
    ref = oracle_lib.march(wl.grid, wl.n2, wl.slice_r, wl.u0, interp=True)
    with P.Plan.for_grid(wl.grid, fp32=True, interp=True) as plan:
        P.pe3d_set_option(plan.h, P.PE3D_OPT_RC_EVERY, 1)
        plan.set_medium(torch.from_numpy(wl.n2).cuda(), wl.slice_r)
        got = plan.march(torch.from_numpy(wl.u0.astype(np.complex64)).cuda(), wl.grid.r0, wl.grid.steps,
                         wl.grid.stride).cpu().numpy()
    assert relerrs(got, ref).max() < 2e-6


@pytest.mark.parametrize("fp32", [False, True], ids=["fp64", "fp32"])
def test_interp_exec_modes_bitwise_equal(P, fp32):
    wl = workloads.random_case(500, 96, periodic=True, K=4, steps=9, seed=147, stride=3)
    outs = [gpu_march(P, wl, fp32=fp32, exec_mode=m, interp=True)[0] for m in (1, 2, 3)]
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[0], outs[2])


def test_interp_toggle_and_resume(P, oracle_lib):
    """Turning interpolation off again rebuilds the per-slice systems; a march
    split in two from the stored field equals the whole one."""
    wl = workloads.random_case(200, 40, periodic=False, K=4, steps=10, seed=149, stride=5)
    g = wl.grid
    piecewise, _ = gpu_march(P, wl, fp32=False)
    with P.Plan.for_grid(g, fp32=False, interp=True) as plan:
        plan.set_medium(torch.from_numpy(wl.n2).cuda(), wl.slice_r)
        u0 = torch.from_numpy(wl.u0).cuda()
        full = plan.march(u0, g.r0, g.steps, g.stride).cpu().numpy()
        half = plan.march(u0, g.r0, 5, 5)
        rest = plan.march(half[-1].contiguous(), g.r0 + 5 * g.dr, 5, 5).cpu().numpy()
        assert np.array_equal(full[-1], rest[-1])
        P.pe3d_set_option(plan.h, P.PE3D_OPT_MEDIUM_INTERP, 0)
        back = plan.march(u0, g.r0, g.steps, g.stride).cpu().numpy()
    assert np.array_equal(back, piecewise)
    ref = oracle_lib.march(g, wl.n2, wl.slice_r, wl.u0, interp=True)
    assert relerrs(full, ref).max() < TOL64


def test_interp_in_batch(P, oracle_lib):
    """An interpolating march inside a batched launch (beside a piecewise one)
    is bit-identical to the same march alone."""
    wls = [workloads.random_case(300, 70, periodic=False, K=4, steps=9, seed=151, stride=1),
           workloads.random_case(37, 257, periodic=True, K=3, steps=5, seed=152, stride=1)]
    interp = [True, False]
    plans, u0s, outs = [], [], []
    for wl, it in zip(wls, interp):
        pl = P.Plan.for_grid(wl.grid, fp32=True, interp=it)
        pl.set_medium(torch.from_numpy(wl.n2).cuda(), wl.slice_r)
        plans.append(pl)
        u0s.append(torch.from_numpy(wl.u0).to(torch.complex64).cuda())
        outs.append(torch.zeros((wl.grid.steps, wl.grid.Ntheta, wl.grid.Nz), dtype=torch.complex64, device="cuda"))
    P.pe3d_march_batched([p.h for p in plans], u0s, [wl.grid.r0 for wl in wls], [wl.grid.steps for wl in wls],
                         [1, 1], outs)
    torch.cuda.synchronize()
    for wl, it, out in zip(wls, interp, outs):
        alone, _ = gpu_march(P, wl, fp32=True, interp=it, exec_mode=3)
        assert np.array_equal(out.cpu().numpy(), alone)
        ref = oracle_lib.march(wl.grid, wl.n2, wl.slice_r, wl.u0, interp=it)
        assert relerrs(alone, ref).max() < TOL32
    for pl in plans:
        pl.close()


def test_interp_full_grid(P, oracle_lib):
    """The 100 Hz walled grid (1067 x 256) with slices every 100 m,
    interpolated, for 40 steps across two slice intervals."""
    wl = workloads.config2(steps=40)
    g = wl.grid
    assert len(wl.slice_r) >= 3
    ref = oracle_lib.march(g, wl.n2, wl.slice_r, wl.u0, steps=40, stride=20, interp=True)
    got, _ = gpu_march(P, wl, fp32=True, steps=40, stride=20, interp=True)
    assert relerrs(got, ref).max() < TOL32


@pytest.mark.parametrize("fp32", [False, True], ids=["fp64", "fp32"])
def test_interp_wide_long_march(P, oracle_lib, fp32):
    """Ntheta = 1024 over 96 steps and six slices: the persistent launch equals
    the stream launch bit for bit and matches the oracle; so does a march with
    the FP64 correction.  One march is four launches: the per-step depth
    set-up, the azimuth set-up, the prologue and the persistent march."""
    steps = 96
    wl = workloads.random_case(64, 1024, periodic=True, K=6, steps=steps, seed=153, stride=24)
    ref = oracle_lib.march(wl.grid, wl.n2, wl.slice_r, wl.u0, interp=True)
    per, info = gpu_march(P, wl, fp32=fp32, exec_mode=3, interp=True)
    assert info["launches"] == 4
    stream, _ = gpu_march(P, wl, fp32=fp32, exec_mode=1, interp=True)
    assert np.array_equal(per, stream)
    assert relerrs(per, ref).max() < (TOL32 if fp32 else TOL64)
    if fp32:
        with P.Plan.for_grid(wl.grid, fp32=True, interp=True) as plan:
            P.pe3d_set_option(plan.h, P.PE3D_OPT_RC_EVERY, 1)
            plan.set_medium(torch.from_numpy(wl.n2).cuda(), wl.slice_r)
            got = plan.march(torch.from_numpy(wl.u0.astype(np.complex64)).cuda(), wl.grid.r0, steps,
                             wl.grid.stride).cpu().numpy()
        assert relerrs(got, ref).max() < 2e-6
