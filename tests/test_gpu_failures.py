"""Failure detection and the FP64 reciprocal of the coefficient set-up (needs a GB300).

None of these faults, traps or hangs the GPU.  A bounded wait is made to give
up by lowering its poll limit (PE3D_OPT_WAIT_LIMIT): the kernel records
PE3D_ERR_TIMEOUT, lets its copies in flight land and returns, and the context
stays usable.  A NaN in the medium must be reported as a singular system, and
a request whose set-up fails must end as PE3D_REQ_FAILED without stopping the
request loop.
"""
import ctypes
import os
import subprocess
import time

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def P():
    from paper_1711_00005_gb300 import build
    build.build()
    import paper_1711_00005_gb300 as P
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return P


def _march(P, wl, *, wait_limit=0, exec_mode=None):
    g = wl.grid
    with P.Plan.for_grid(g, fp32=True, exec_mode=exec_mode) as plan:
        P.pe3d_set_option(plan.h, P.PE3D_OPT_WAIT_LIMIT, wait_limit)
        plan.set_medium(torch.from_numpy(wl.n2).cuda(), wl.slice_r)
        out = plan.march(torch.from_numpy(wl.u0.astype(np.complex64)).cuda(), g.r0, g.steps, g.stride)
        torch.cuda.synchronize()
        return out.cpu().numpy()


def test_grid_barrier_wait_gives_up(P):
    """One poll per wait: with 100+ CTAs the first to arrive at a grid barrier
    cannot see all the others, so the march ends with PE3D_ERR_TIMEOUT; the
    same plan settings with the default limit then march normally."""
    wl = workloads.random_case(1067, 256, periodic=False, K=2, steps=6, seed=700, stride=3)
    with pytest.raises(P.PE3DError) as e:
        _march(P, wl, wait_limit=1, exec_mode=P.PE3D_EXEC_PERSISTENT)
    assert e.value.code == P.PE3D_ERR_TIMEOUT
    assert "gave up" in str(e.value)
    a = _march(P, wl, exec_mode=P.PE3D_EXEC_PERSISTENT)
    b = _march(P, wl, exec_mode=P.PE3D_EXEC_STREAM)
    assert np.all(np.isfinite(a)) and np.array_equal(a, b)


def test_batched_wait_gives_up(P):
    wls = [workloads.random_case(400 + 50 * i, 96, periodic=bool(i % 2), K=2, steps=5, seed=710 + i, stride=5)
           for i in range(4)]
    plans = []
    for i, wl in enumerate(wls):
        pl = P.Plan.for_grid(wl.grid, fp32=True)
        if i == 0:                                  # the first plan's limit governs the launch
            P.pe3d_set_option(pl.h, P.PE3D_OPT_WAIT_LIMIT, 1)
        pl.set_medium(torch.from_numpy(wl.n2).cuda(), wl.slice_r)
        plans.append(pl)
    u0s = [torch.from_numpy(wl.u0.astype(np.complex64)).cuda() for wl in wls]
    outs = [torch.zeros((1, wl.grid.Ntheta, wl.grid.Nz), dtype=torch.complex64, device="cuda") for wl in wls]
    with pytest.raises(P.PE3DError) as e:
        P.pe3d_march_batched([p.h for p in plans], u0s, [wl.grid.r0 for wl in wls], [5] * 4, [5] * 4, outs)
    assert e.value.code == P.PE3D_ERR_TIMEOUT
    P.pe3d_set_option(plans[0].h, P.PE3D_OPT_WAIT_LIMIT, 0)
    P.pe3d_march_batched([p.h for p in plans], u0s, [wl.grid.r0 for wl in wls], [5] * 4, [5] * 4, outs)
    torch.cuda.synchronize()
    for wl, o in zip(wls, outs):
        assert np.array_equal(o.cpu().numpy(), _march(P, wl, exec_mode=P.PE3D_EXEC_PERSISTENT))
    for pl in plans:
        pl.close()


@pytest.mark.parametrize("where", ["water", "bottom"])
def test_nan_medium_is_singular(P, where):
    wl = workloads.random_case(120, 30, periodic=False, K=2, steps=3, seed=720)
    bad = wl.n2.copy()
    bad[1, 7, 5 if where == "water" else 119] = np.nan
    with P.Plan.for_grid(wl.grid, fp32=True) as plan:
        with pytest.raises(P.PE3DError) as e:
            plan.set_medium(bad, wl.slice_r)
        assert e.value.code == P.PE3D_ERR_SINGULAR
        plan.set_medium(wl.n2, wl.slice_r)          # recovers


def test_failed_request_does_not_stop_the_loop(P):
    good = workloads.random_case(80, 20, periodic=False, K=1, steps=6, seed=730, stride=6)
    bad = workloads.random_case(80, 20, periodic=False, K=1, steps=6, seed=731, stride=6)
    bad.n2[0, 3, 10] = np.nan
    srv = P.pe3d_server_create(1 << 30, 8, 4)
    try:
        rb, kb = P.make_request(bad.grid, bad.n2, bad.slice_r, bad.u0, fp32=True)
        rg, kg = P.make_request(good.grid, good.n2, good.slice_r, good.u0, fp32=True)
        id_bad = P.pe3d_submit(srv, rb)
        id_good = P.pe3d_submit(srv, rg)
        t0 = time.perf_counter()
        failed = False
        while not failed:
            assert time.perf_counter() - t0 < 60
            try:
                st, _ = P.pe3d_poll(srv, id_bad)
            except P.PE3DError as e:
                assert "request failed" in str(e) and "singular" in str(e).lower()
                failed = True
            else:
                assert st in (P.PE3D_REQ_PENDING, P.PE3D_REQ_RUNNING)
                time.sleep(0.005)
        while P.pe3d_poll(srv, id_good)[0] != P.PE3D_REQ_DONE:
            assert time.perf_counter() - t0 < 60
            time.sleep(0.005)
        out = np.empty((1, 20, 80), np.complex64)
        P.pe3d_poll(srv, id_good, out)
        stats = P.pe3d_server_stats(srv)
        assert stats["failed"] == 1 and stats["finished"] == 1
    finally:
        P.pe3d_server_destroy(srv)
    assert np.array_equal(out, _march(P, good, exec_mode=P.PE3D_EXEC_PERSISTENT))


def test_recip_newton_against_cuda_division(tmp_path):
    """The set-up's reciprocal of |den|^2 (rcp.approx.ftz.f64 and two
    Newton-Raphson steps) against CUDA's IEEE 1.0 / x over the whole range the
    set-up admits, [2^-53, 2^996): a log-uniform sample, the range ends and
    powers of two.  Bound: 1 ulp of the correctly rounded quotient."""
    from paper_1711_00005_gb300 import build
    src = os.path.join(ROOT, "tests", "gpu_helpers", "recip_check.cu")
    lib = str(tmp_path / "librecip.so")
    cmd = [build.nvcc(), *build.ARCH, "-O3", "-std=c++17", "--expt-relaxed-constexpr", "-shared", "-Xcompiler",
           "-fPIC", "-I", os.path.join(ROOT, "paper_1711_00005_gb300", "csrc"), "-I", os.path.join(ROOT, "include"),
           src, "-o", lib]
    subprocess.run(cmd, check=True, capture_output=True)
    L = ctypes.CDLL(lib)
    L.recip_check.argtypes = [ctypes.c_void_p] * 3 + [ctypes.c_longlong]
    rng = np.random.default_rng(7)
    lo, hi = -53.0, 996.0
    x = np.exp2(rng.uniform(lo, hi, 1 << 20))
    top = np.nextafter(np.exp2(hi), 0.0)
    ends = np.array([np.exp2(lo), np.nextafter(np.exp2(lo), np.inf), top, 1.0, np.nextafter(1.0, 0.0),
                     np.nextafter(1.0, 2.0), 3.0, 0.1, 1e300])
    x = np.concatenate([x, ends, np.exp2(np.arange(-53.0, 996.0))])
    x = x[(x >= np.exp2(lo)) & (x < np.exp2(hi))]
    yn = np.empty_like(x)
    yd = np.empty_like(x)
    assert L.recip_check(x.ctypes.data, yn.ctypes.data, yd.ctypes.data, len(x)) == 0
    ulp = np.abs(yn - yd) / np.spacing(yd)
    print(f"\nrecip_newton vs 1.0/x over {len(x)} inputs: max {ulp.max():.2f} ulp, "
          f"{np.mean(ulp > 0) * 100:.3f} % not equal")
    assert np.all(np.isfinite(yn))
    assert ulp.max() <= 1.0
