"""Broadband synthesis on the GPU against the oracle's (pinned in
tests/test_oracle_synthesis.py), alone and after a batched multi-frequency
march with pressure output (the paper's 8-frequency run, scaled down).

Tolerances (relative L2 over all receivers and samples):
  * synthesis alone: FP64 1e-12; FP32 1e-5 (complex64 inputs and phasors,
    ~1e-7 per term, summed over 2F terms in FP32);
  * after the march: FP64 1e-10; FP32 1e-4, the march's own bound.
"""
import numpy as np
import pytest

import oracle
import workloads

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


def relerr(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


@pytest.mark.parametrize("F,R,T", [(37, 1000, 300), (1, 129, 7), (120, 600, 1024)])
@pytest.mark.parametrize("fp32", [False, True], ids=["fp64", "fp32"])
def test_synthesis_parity(P, F, R, T, fp32):
    """Ragged receiver and sample counts (tiles of 128 and 64), one and many frequencies."""
    rng = np.random.default_rng(F + R)
    freqs = 40.0 + 20.0 * rng.random(F)
    W = rng.normal(size=F) + 1j * rng.normal(size=F)
    p = rng.normal(size=(F, R)) + 1j * rng.normal(size=(F, R))
    t0, dt = 3.21, 1.0 / 200.0
    cdt = torch.complex64 if fp32 else torch.complex128
    rdt = torch.float32 if fp32 else torch.float64
    ps = [torch.from_numpy(p[i]).to(cdt).cuda() for i in range(F)]
    out = torch.full((R, T), float("nan"), dtype=rdt, device="cuda")
    P.pe3d_synthesize(P.PE3D_FP32 if fp32 else P.PE3D_FP64, freqs, W, ps, T, t0, dt, out)
    got = out.cpu().numpy()
    pin = np.array([x.cpu().numpy() for x in ps]) if fp32 else p     # the same rounded inputs
    ref = oracle.synthesize(freqs, W, pin, t0, dt, T)
    assert np.isfinite(got).all()
    assert relerr(got, ref) < (1e-5 if fp32 else 1e-12)


def test_synthesis_arguments(P):
    ps = [torch.zeros(10, dtype=torch.complex64, device="cuda")]
    out = torch.zeros((10, 4), dtype=torch.float32, device="cuda")
    P.pe3d_synthesize(P.PE3D_FP32, [50.0], [1.0], ps, 0, 0.0, 0.01, out)          # T = 0: nothing to do
    with pytest.raises(P.PE3DError) as e:                                          # host pressure
        P.pe3d_synthesize(P.PE3D_FP32, [50.0], [1.0], [torch.zeros(10, dtype=torch.complex64)], 4, 0.0, 0.01, out)
    assert e.value.code == P.PE3D_ERR_ARG
    with pytest.raises(P.PE3DError) as e:                                          # host output
        P.pe3d_synthesize(P.PE3D_FP32, [50.0], [1.0], ps, 4, 0.0, 0.01, torch.zeros((10, 4)))
    assert e.value.code == P.PE3D_ERR_ARG
    with pytest.raises(P.PE3DError) as e:
        P.pe3d_synthesize(P.PE3D_FP32, [float("nan")], [1.0], ps, 4, 0.0, 0.01, out)
    assert e.value.code == P.PE3D_ERR_ARG


@pytest.mark.parametrize("fp32", [False, True], ids=["fp64", "fp32"])
def test_broadband_march_and_synthesis(P, oracle_lib, fp32):
    """Eight frequencies on one grid in one batched launch with pressure
    output, then the time series at every grid point of the last range."""
    bb = workloads.broadband(F=8, Nz=96, Ntheta=24, steps=40, T=256)
    cdt = torch.complex64 if fp32 else torch.complex128
    rdt = torch.float32 if fp32 else torch.float64
    plans, u0s, outs = [], [], []
    for wl in bb.members:
        pl = P.Plan.for_grid(wl.grid, fp32=fp32, output=P.PE3D_OUT_PRESSURE)
        pl.set_medium(torch.from_numpy(wl.n2).cuda(), wl.slice_r)
        plans.append(pl)
        u0s.append(torch.from_numpy(wl.u0).to(cdt).cuda())
        outs.append(torch.zeros((1, wl.grid.Ntheta, wl.grid.Nz), dtype=cdt, device="cuda"))
    g = bb.members[0].grid
    P.pe3d_march_batched([pl.h for pl in plans], u0s, [g.r0] * len(plans), [g.steps] * len(plans),
                         [g.steps] * len(plans), outs)
    s = torch.empty((g.Ntheta * g.Nz, bb.T), dtype=rdt, device="cuda")
    P.pe3d_synthesize(P.PE3D_FP32 if fp32 else P.PE3D_FP64, bb.freqs, bb.W, outs, bb.T, bb.t0, bb.dt, s)
    got = s.cpu().numpy()
    for pl in plans:
        pl.close()
    p_ref = []
    for wl in bb.members:
        u = oracle_lib.march(wl.grid, wl.n2, wl.slice_r, wl.u0)
        p_ref.append(oracle.pressure(u, oracle.snapshot_ranges(g.r0, g.dr, g.steps, g.steps), wl.grid.k0)[0])
    ref = oracle.synthesize(bb.freqs, bb.W, np.array(p_ref).reshape(len(p_ref), -1), bb.t0, bb.dt, bb.T)
    assert relerr(got, ref) < (1e-4 if fp32 else 1e-10)
