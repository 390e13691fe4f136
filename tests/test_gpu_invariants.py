"""Exact properties of the scheme (Eq. 4) checked on the GPU march itself,
independently of the oracle (FP64 marches; the properties hold exactly, so
the tolerances bound rounding only: about 1e-14 per step here, checked at
1e-11 and above):
  * norm conservation for real, theta-independent media (X and Y commute
    and both factors are Cayley transforms of real symmetric operators);
  * linearity in the starter;
  * a theta-uniform field in a theta-independent full circle stays uniform;
  * mirror symmetry of a walled sector with a symmetric medium and starter.
"""
import numpy as np
import pytest

import workloads
from test_gpu_parity import gpu_march

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


def rel(a, b):
    return float(np.linalg.norm((np.asarray(a) - b).ravel()) / np.linalg.norm(np.asarray(b).ravel()))


@pytest.mark.parametrize("periodic", [False, True], ids=["walled", "periodic"])
@pytest.mark.parametrize("exec_mode", [1, 3], ids=["stream", "persistent"])
def test_norm_conservation(P, periodic, exec_mode):
    wl = workloads.random_case(150, 24, periodic=periodic, K=4, steps=40, seed=11, lossy=False,
                               theta_dependent=False, stride=1)
    got, _ = gpu_march(P, wl, fp32=False, exec_mode=exec_mode)
    n0 = np.linalg.norm(wl.u0)
    drift = np.abs(np.linalg.norm(got.reshape(got.shape[0], -1), axis=1) - n0) / n0
    assert np.all(drift <= 1e-11 * np.arange(1, got.shape[0] + 1)), drift.max()


def test_lossy_medium_absorbs(P):
    """With Im(n^2) > 0 (delta = +i k0 dr) the field loses energy over the march."""
    wl = workloads.random_case(150, 24, periodic=True, K=1, steps=20, seed=31, lossy=True,
                               theta_dependent=False, stride=20)
    got, _ = gpu_march(P, wl, fp32=False)
    assert np.linalg.norm(got[-1]) < 0.999 * np.linalg.norm(wl.u0)


@pytest.mark.parametrize("scheme", [0, 1], ids=["pade", "taylor"])
def test_linearity(P, scheme):
    wl = workloads.random_case(200, 40, periodic=False, K=3, steps=8, seed=13, stride=4)
    rng = np.random.default_rng(14)
    v0 = rng.normal(size=wl.u0.shape) + 1j * rng.normal(size=wl.u0.shape)
    a, b = 0.7 - 0.2j, -1.3 + 0.4j
    f = lambda u: gpu_march(P, wl, fp32=False, u0=u, scheme=scheme)[0]
    assert rel(f(a * wl.u0 + b * v0), a * f(wl.u0) + b * f(v0)) < 1e-11


def test_theta_uniform_stays_uniform(P):
    wl = workloads.random_case(300, 32, periodic=True, K=2, steps=10, seed=15, theta_dependent=False, stride=5)
    col = wl.u0[0]
    u0 = np.broadcast_to(col, wl.u0.shape).copy()
    got, _ = gpu_march(P, wl, fp32=False, u0=u0)
    for snap in got:
        assert rel(snap, np.broadcast_to(snap[0], snap.shape)) < 1e-11


def test_mirror_symmetry(P):
    wl = workloads.random_case(250, 31, periodic=False, K=2, steps=10, seed=16, stride=5)
    n2 = 0.5 * (wl.n2 + wl.n2[:, ::-1, :])
    u0 = 0.5 * (wl.u0 + wl.u0[::-1, :])
    sym = workloads.Workload(wl.grid, wl.slice_r, np.ascontiguousarray(n2), np.ascontiguousarray(u0), wl.meta)
    got, _ = gpu_march(P, sym, fp32=False)
    for snap in got:
        assert rel(snap[::-1, :], snap) < 1e-11
