"""The Taylor form of Eq. 3 (depth factor [1 -+ (d/2)(X/2 - X^2/8)]) on the GPU
against the oracle's pentadiagonal march (pinned in tests/pins.py:
check_dense(taylor=True), check_eigenmodes(taylor=True), penta).

The GPU solves the pentadiagonal factor as two tridiagonal factors
(I + a1 X)(I + a2 X) combined by partial fractions; the oracle assembles it
and uses banded elimination, so agreement checks the factorisation too.
Tolerances as in test_gpu_parity.py: FP64 1e-10, FP32 2e-5.
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


CASES = [
    # (Nz, Ntheta, periodic, K, steps): several tiles, ragged tails, the four chunk classes
    (300, 41, False, 3, 9),
    (257, 40, True, 2, 7),
    (1067, 24, False, 3, 4),
    (33, 5, True, 1, 6),
]


@pytest.mark.parametrize("case", CASES, ids=[f"{c[0]}x{c[1]}{'p' if c[2] else 'w'}" for c in CASES])
@pytest.mark.parametrize("exec_mode", [1, 2, 3], ids=["stream", "graph", "persistent"])
@pytest.mark.parametrize("fp32", [False, True], ids=["fp64", "fp32"])
def test_taylor_parity(P, oracle_lib, case, exec_mode, fp32):
    Nz, Nt, periodic, K, steps = case
    wl = workloads.random_case(Nz, Nt, periodic=periodic, K=K, steps=steps, seed=170 + Nz, stride=1)
    ref = oracle_lib.march(wl.grid, wl.n2, wl.slice_r, wl.u0, taylor=True)
    got, info = gpu_march(P, wl, fp32=fp32, exec_mode=exec_mode, scheme=P.PE3D_SCHEME_TAYLOR)
    assert info["exec"] == exec_mode
    assert relerrs(got, ref).max() < (TOL32 if fp32 else TOL64)
    # a different scheme from Eq. 4
    assert relerrs(got, oracle_lib.march(wl.grid, wl.n2, wl.slice_r, wl.u0)).max() > 1e-6
    if exec_mode == 3:   # the persistent launch runs the same per-system arithmetic as the per-step launches
        stepwise, _ = gpu_march(P, wl, fp32=fp32, exec_mode=1, scheme=P.PE3D_SCHEME_TAYLOR)
        assert np.array_equal(got, stepwise)


@pytest.mark.parametrize("zthreads", [32, 64, 256])
def test_taylor_layouts(P, oracle_lib, zthreads):
    """Other depth layouts (threads per system, hence chunk classes) and the
    centred Y with the automatic launch (the persistent launch for this scheme
    when its three-column depth unit fits)."""
    wl = workloads.random_case(700, 20, periodic=False, K=2, steps=5, seed=180, stride=5)
    for mid in (False, True):
        ref = oracle_lib.march(wl.grid, wl.n2, wl.slice_r, wl.u0, taylor=True, y_midpoint=mid)
        got, info = gpu_march(P, wl, fp32=True, zthreads=zthreads, scheme=P.PE3D_SCHEME_TAYLOR, y_midpoint=mid)
        assert info["exec"] == 3                      # persistent
        assert relerrs(got, ref).max() < TOL32


def test_taylor_refusals(P):
    wl = workloads.random_case(20, 5, periodic=False, K=1, steps=2, seed=9)
    n2 = torch.from_numpy(wl.n2).cuda()
    u0 = torch.from_numpy(wl.u0.astype(np.complex64)).cuda()
    with P.Plan.for_grid(wl.grid, fp32=True, scheme=P.PE3D_SCHEME_TAYLOR) as plan:
        plan.set_medium(n2, wl.slice_r)
        for opt in (P.PE3D_OPT_MEDIUM_INTERP, P.PE3D_OPT_RC_EVERY):
            with pytest.raises(P.PE3DError) as e:
                P.pe3d_set_option(plan.h, opt, 1)
            assert e.value.code == P.PE3D_ERR_ARG
        with pytest.raises(P.PE3DError) as e:        # the scheme is fixed once a medium is set
            P.pe3d_set_option(plan.h, P.PE3D_OPT_SCHEME, P.PE3D_SCHEME_PADE)
        assert e.value.code == P.PE3D_ERR_STATE
        P.pe3d_set_option(plan.h, P.PE3D_OPT_EXEC, 4)
        with pytest.raises(P.PE3DError) as e:        # no resident launch
            plan.march(u0, wl.grid.r0, 2, 1)
        assert e.value.code == P.PE3D_ERR_ARG
        out = torch.zeros((2, 5, 20), dtype=torch.complex64, device="cuda")
        with pytest.raises(P.PE3DError) as e:        # no batched launch
            P.pe3d_march_batched([plan.h], [u0], [wl.grid.r0], [2], [1], [out])
        assert e.value.code == P.PE3D_ERR_ARG


def test_taylor_set_medium_batched(P):
    """A Taylor plan among Eq. 4 plans in pe3d_set_medium_batched gets its two
    factors, bit-identical to its own pe3d_set_medium."""
    wls = [workloads.random_case(90, 12, periodic=False, K=2, steps=3, seed=190 + i, stride=1) for i in range(3)]
    schemes = [P.PE3D_SCHEME_PADE, P.PE3D_SCHEME_TAYLOR, P.PE3D_SCHEME_PADE]
    ref = [gpu_march(P, wl, fp32=True, scheme=sc)[0] for wl, sc in zip(wls, schemes)]
    plans = [P.Plan.for_grid(wl.grid, fp32=True, scheme=sc) for wl, sc in zip(wls, schemes)]
    P.pe3d_set_medium_batched([pl.h for pl in plans], [torch.from_numpy(wl.n2).cuda() for wl in wls],
                              [wl.slice_r for wl in wls])
    for pl, wl, r in zip(plans, wls, ref):
        got = pl.march(torch.from_numpy(wl.u0.astype(np.complex64)).cuda(), wl.grid.r0, wl.grid.steps, 1)
        assert np.array_equal(got.cpu().numpy(), r)
        pl.close()
