"""Request loop (continuous batching) on the GPU: each request's result is the
same alone and in the mix; admission respects the memory budget; invalid or
oversized requests are refused."""
import time

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    from paper_1711_00005_gb300 import build
    build.build()
    import paper_1711_00005_gb300 as P
    return P


def alone(P, wl, fp32):
    """The same march alone, in the persistent launch: the request loop runs
    the batched kernel, whose per-system arithmetic the persistent launch shares
    (the resident launch rounds in another order)."""
    g = wl.grid
    cdt = np.complex64 if fp32 else np.complex128
    with P.Plan.for_grid(g, fp32=fp32, exec_mode=P.PE3D_EXEC_PERSISTENT) as plan:
        plan.set_medium(wl.n2, wl.slice_r)
        out = np.zeros((g.steps // g.stride, g.Ntheta, g.Nz), cdt)
        P.pe3d_march(plan.h, wl.u0.astype(cdt), g.r0, g.steps, g.stride, out)
    return out


def serve(P, items, budget=8 << 30, max_active=64, chunk=16, stagger=0.0):
    srv = P.pe3d_server_create(budget, max_active, chunk)
    try:
        ids, keep = [], []
        for wl, fp32 in items:
            req, k = P.make_request(wl.grid, wl.n2, wl.slice_r, wl.u0, fp32=fp32)
            keep.append(k)
            ids.append(P.pe3d_submit(srv, req))
            if stagger:
                time.sleep(stagger)
        outs, times = [], []
        for (wl, fp32), rid in zip(items, ids):
            g = wl.grid
            out = np.zeros((g.steps // g.stride, g.Ntheta, g.Nz), np.complex64 if fp32 else np.complex128)
            t0 = time.time()
            while True:
                st, tm = P.pe3d_poll(srv, rid)
                if st == P.PE3D_REQ_DONE:
                    P.pe3d_poll(srv, rid, out)
                    break
                assert st in (P.PE3D_REQ_PENDING, P.PE3D_REQ_RUNNING), st
                assert time.time() - t0 < 120
                time.sleep(0.002)
            outs.append(out)
            times.append(tm)
        stats = P.pe3d_server_stats(srv)
    finally:
        P.pe3d_server_destroy(srv)
    return outs, times, stats


def test_alone_equals_mix(P, oracle_lib):
    specs = [(300, 70, False, 40, False), (37, 257, True, 25, True), (1067, 64, False, 13, True),
             (5, 3, True, 30, False), (128, 130, False, 64, True), (411, 45, True, 17, False)]
    items = [(workloads.random_case(Nz, Nt, periodic=per, K=3, steps=st, seed=200 + i, stride=1), fp32)
             for i, (Nz, Nt, per, st, fp32) in enumerate(specs)]
    outs, times, stats = serve(P, items, stagger=0.003)
    assert stats["finished"] == len(items) and stats["failed"] == 0
    # every turn launches the batched march, every request its own set-up
    assert stats["launches"] >= stats["ticks"] + len(items)
    for (wl, fp32), got in zip(items, outs):
        ref = alone(P, wl, fp32)
        assert np.array_equal(got, ref)          # same arithmetic alone and in the mix
        orc = oracle_lib.march(wl.grid, wl.n2, wl.slice_r, wl.u0)
        err = max(np.linalg.norm(a - b) / np.linalg.norm(b) for a, b in zip(got, orc))
        assert err < (2e-5 if fp32 else 1e-10)
    for ts, ta, td in times:
        assert ts <= ta <= td


def test_admission_by_memory(P):
    """A budget that fits one request at a time still serves them all, in order."""
    items = [(workloads.random_case(500, 64, periodic=False, K=2, steps=20, seed=300 + i, stride=5), True)
             for i in range(4)]
    outs, times, stats = serve(P, items, budget=5 << 20, chunk=8)
    assert stats["finished"] == 4
    starts = [t[1] for t in times]
    dones = [t[2] for t in times]
    for i in range(1, 4):                       # each waits for the previous one's memory
        assert starts[i] >= dones[i - 1] - 1e-3
    for (wl, fp32), got in zip(items, outs):
        assert np.array_equal(got, alone(P, wl, fp32))


def test_refusals(P):
    srv = P.pe3d_server_create(1 << 20, 4, 8)
    try:
        wl = workloads.random_case(2000, 128, periodic=False, K=4, steps=50, seed=1)
        req, keep = P.make_request(wl.grid, wl.n2, wl.slice_r, wl.u0)
        with pytest.raises(P.PE3DError) as e:
            P.pe3d_submit(srv, req)
        assert e.value.code == P.PE3D_ERR_ARG and "budget" in str(e.value)
        with pytest.raises(P.PE3DError):
            P.pe3d_poll(srv, 12345)
    finally:
        P.pe3d_server_destroy(srv)
