"""The resident march (PE3D_EXEC_RESIDENT) against the FP64 oracle (needs a GB300).

Each CTA of the resident march keeps a block of azimuths x depths in shared
memory; a step exchanges two complex numbers per system and block.  Its
rounding order differs from the other launches, so it is checked against the
oracle at the FP32 tolerance of the short cases (2e-5), on grids whose
layouts cover one block along an axis, many blocks, ragged last blocks, both
boundaries, every output mode and the centred Y.
"""
import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 2e-5
RESIDENT = 4


@pytest.fixture(scope="module")
def P():
    from paper_1711_00005_gb300 import build
    build.build()
    import paper_1711_00005_gb300 as P
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return P


def relerrs(got, ref):
    got, ref = np.asarray(got), np.asarray(ref)
    assert got.shape == ref.shape
    return np.array([np.linalg.norm((a - b).ravel()) / max(np.linalg.norm(b.ravel()), 1e-300)
                     for a, b in zip(got, ref)])


def march(P, wl, exec_mode=RESIDENT, **opts):
    g = wl.grid
    with P.Plan.for_grid(g, fp32=True, exec_mode=exec_mode, **opts) as plan:
        plan.set_medium(torch.from_numpy(wl.n2).cuda(), wl.slice_r)
        out = plan.march(torch.from_numpy(wl.u0.astype(np.complex64)).cuda(), g.r0, g.steps, g.stride)
        torch.cuda.synchronize()
        return out.cpu().numpy(), plan.info()


CASES = [
    # (Nz, Ntheta, periodic, K, steps, seed)
    (300, 70, False, 3, 12, 901),
    (300, 70, True, 3, 12, 902),
    (1, 1, False, 1, 4, 903),
    (2, 3, True, 1, 4, 904),
    (5, 2, False, 2, 6, 905),
    (33, 31, True, 2, 6, 906),
    (257, 5, False, 1, 5, 907),
    (7, 257, True, 1, 5, 908),
    (1067, 64, False, 4, 8, 909),
    (1067, 256, False, 5, 25, 910),
    (1067, 1024, True, 3, 6, 911),
    (2400, 40, True, 2, 5, 912),
    (60, 900, False, 2, 5, 913),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}x{c[1]}{'p' if c[2] else 'w'}")
def test_resident_parity(P, oracle_lib, case):
    Nz, Nt, periodic, K, steps, seed = case
    wl = workloads.random_case(Nz, Nt, periodic=periodic, K=K, steps=steps, seed=seed, stride=1)
    ref = oracle_lib.march(wl.grid, wl.n2, wl.slice_r, wl.u0)
    got, info = march(P, wl)
    assert info["exec"] == RESIDENT
    err = relerrs(got, ref)
    assert err.max() < TOL32, err


@pytest.mark.parametrize("output", [1, 2], ids=["pressure", "tl"])
@pytest.mark.parametrize("periodic", [False, True], ids=["walled", "periodic"])
def test_resident_outputs(P, oracle_lib, output, periodic):
    import oracle
    wl = workloads.random_case(400, 96, periodic=periodic, K=2, steps=12, seed=920 + periodic, stride=4)
    g = wl.grid
    ref = oracle_lib.march(g, wl.n2, wl.slice_r, wl.u0)
    p_ref = oracle.pressure(ref, oracle.snapshot_ranges(g.r0, g.dr, g.steps, g.stride), g.k0)
    got, _ = march(P, wl, output=output)
    if output == 1:
        assert relerrs(got, p_ref).max() < TOL32
    else:
        assert relerrs(10.0 ** (-got.astype(np.float64) / 20.0), np.abs(p_ref)).max() < TOL32


def test_resident_y_midpoint(P, oracle_lib):
    wl = workloads.random_case(150, 41, periodic=True, K=3, steps=9, seed=930, stride=3)
    ref = oracle_lib.march(wl.grid, wl.n2, wl.slice_r, wl.u0, y_midpoint=True)
    got, _ = march(P, wl, y_midpoint=True)
    assert relerrs(got, ref).max() < TOL32


def test_resident_with_many_slices(P, oracle_lib):
    """A new medium slice every step: the depth blocks' constants are rebuilt
    and exchanged at every step."""
    wl = workloads.random_case(700, 96, periodic=False, K=20, steps=20, seed=940, stride=5)
    ref = oracle_lib.march(wl.grid, wl.n2, wl.slice_r, wl.u0)
    got, _ = march(P, wl)
    assert relerrs(got, ref).max() < TOL32


def test_auto_and_refusals(P):
    wl = workloads.random_case(200, 48, periodic=False, K=2, steps=4, seed=950, stride=2)
    _, info = march(P, wl, exec_mode=0)
    assert info["exec"] == 3                                 # AUTO: persistent unless the autotuner chose it
    g = wl.grid
    for kind in ("fp64", "rc", "interp", "taylor"):
        plan = P.Plan.for_grid(g, fp32=(kind != "fp64"), exec_mode=RESIDENT,
                               interp=(kind == "interp") or None,
                               scheme=(P.PE3D_SCHEME_TAYLOR if kind == "taylor" else None))
        if kind == "rc":
            P.pe3d_set_option(plan.h, P.PE3D_OPT_RC_EVERY, 4)
        plan.set_medium(torch.from_numpy(wl.n2).cuda(), wl.slice_r)
        cdt = np.complex128 if kind == "fp64" else np.complex64
        with pytest.raises(P.PE3DError) as e:
            plan.march(torch.from_numpy(wl.u0.astype(cdt)).cuda(), g.r0, g.steps, g.stride)
        assert e.value.code == P.PE3D_ERR_ARG, kind
        plan.close()


def test_resident_close_to_persistent(P):
    """Both launches solve the same systems: their fields differ by rounding only."""
    wl = workloads.random_case(1067, 128, periodic=True, K=3, steps=40, seed=960, stride=10)
    a, _ = march(P, wl, exec_mode=RESIDENT)
    b, _ = march(P, wl, exec_mode=3)
    assert relerrs(a, b).max() < 1e-5
    assert not np.array_equal(a, b)


def test_resident_wait_gives_up(P):
    """One poll per exchange wait: the march ends with PE3D_ERR_TIMEOUT and the
    next march with the default limit succeeds."""
    wl = workloads.random_case(1067, 256, periodic=False, K=2, steps=6, seed=970, stride=3)
    g = wl.grid
    with P.Plan.for_grid(g, fp32=True, exec_mode=RESIDENT) as plan:
        P.pe3d_set_option(plan.h, P.PE3D_OPT_WAIT_LIMIT, 1)
        plan.set_medium(torch.from_numpy(wl.n2).cuda(), wl.slice_r)
        u0 = torch.from_numpy(wl.u0.astype(np.complex64)).cuda()
        with pytest.raises(P.PE3DError) as e:
            plan.march(u0, g.r0, g.steps, g.stride)
        assert e.value.code == P.PE3D_ERR_TIMEOUT
        P.pe3d_set_option(plan.h, P.PE3D_OPT_WAIT_LIMIT, 0)
        out = plan.march(u0, g.r0, g.steps, g.stride).cpu().numpy()
    assert np.all(np.isfinite(out))
