"""The FP64 residual correction in batched launches (needs a GB300).

A batch mixes marches with and without the correction, with different
correction periods, step counts and boundaries, so that corrected steps fall
at different batched steps, at the first and the last step of a launch, and
on snapshot steps.  Every march must give the bit-identical field of the same
march run alone in the persistent launch (which corrects in-kernel), and
match the FP64 oracle within the FP32 tolerance; a march corrected every step
comes within 2e-6 of it.
"""
import time

import numpy as np
import pytest

import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 2e-5


@pytest.fixture(scope="module")
def P():
    from paper_1711_00005_gb300 import build
    build.build()
    import paper_1711_00005_gb300 as P
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return P


def relerrs(got, ref):
    return np.array([np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()) for a, b in zip(got, ref)])


def alone(P, wl, rc):
    g = wl.grid
    with P.Plan.for_grid(g, fp32=True, exec_mode=P.PE3D_EXEC_PERSISTENT) as plan:
        if rc:
            P.pe3d_set_option(plan.h, P.PE3D_OPT_RC_EVERY, rc)
        plan.set_medium(torch.from_numpy(wl.n2).cuda(), wl.slice_r)
        out = plan.march(torch.from_numpy(wl.u0.astype(np.complex64)).cuda(), g.r0, g.steps, g.stride)
        torch.cuda.synchronize()
        return out.cpu().numpy()


SPECS = [
    # (Nz, Ntheta, periodic, steps, stride, rc_every, seed)
    (200, 48, False, 40, 5, 7, 501),
    (150, 40, True, 33, 3, 1, 502),
    (300, 70, False, 25, 5, 0, 503),
    (97, 130, True, 40, 8, 8, 504),
    (1067, 64, False, 20, 4, 5, 505),
    (33, 31, False, 14, 7, 14, 506),
]


def test_batched_correction_matches_alone_and_oracle(P, oracle_lib):
    wls = [workloads.random_case(Nz, Nt, periodic=per, K=3, steps=st, seed=seed, stride=sd, lossy=True,
                                 theta_dependent=True)
           for Nz, Nt, per, st, sd, rc, seed in SPECS]
    rcs = [s[5] for s in SPECS]
    plans, u0s, outs = [], [], []
    for wl, rc in zip(wls, rcs):
        g = wl.grid
        pl = P.Plan.for_grid(g, fp32=True)
        if rc:
            P.pe3d_set_option(pl.h, P.PE3D_OPT_RC_EVERY, rc)
        pl.set_medium(torch.from_numpy(wl.n2).cuda(), wl.slice_r)
        plans.append(pl)
        u0s.append(torch.from_numpy(wl.u0.astype(np.complex64)).cuda())
        outs.append(torch.zeros((g.n_out, g.Ntheta, g.Nz), dtype=torch.complex64, device="cuda"))
    P.pe3d_march_batched([p.h for p in plans], u0s, [wl.grid.r0 for wl in wls], [wl.grid.steps for wl in wls],
                         [wl.grid.stride for wl in wls], outs)
    torch.cuda.synchronize()
    # the batch split at every batched step that some march corrects: a launch
    # up to it and a correction launch after it
    corrected = {t for wl, rc in zip(wls, rcs) if rc for t in range(wl.grid.steps) if (t + 1) % rc == 0}
    ends = sorted(corrected)
    batched_launches = len(ends) + (1 if not ends or ends[-1] < max(wl.grid.steps for wl in wls) - 1 else 0)
    info = P.pe3d_plan_info(plans[0].h)
    assert info["launches"] == batched_launches + len(ends) + len(wls) + 1
    for wl, rc, out in zip(wls, rcs, outs):
        got = out.cpu().numpy()
        assert np.array_equal(got, alone(P, wl, rc)), f"rc={rc}: batched differs from the march alone"
        ref = oracle_lib.march(wl.grid, wl.n2, wl.slice_r, wl.u0)
        err = relerrs(got, ref)
        assert err.max() < (2e-6 if rc == 1 else TOL32), (rc, err)
    for pl in plans:
        pl.close()


def test_served_correction_matches_alone(P):
    """Requests with the correction through the request loop, in chunks of 16
    steps (so corrections every 7 steps fall inside and across ticks):
    bit-identical to the march alone."""
    wls = [workloads.random_case(120 + 10 * i, 24 + 8 * i, periodic=bool(i % 2), K=2, steps=45, seed=600 + i,
                                 stride=9) for i in range(5)]
    rcs = [7, 0, 16, 1, 64]
    srv = P.pe3d_server_create(8 << 30, 8, 16)
    try:
        ids, keep = [], []
        for wl, rc in zip(wls, rcs):
            req, k = P.make_request(wl.grid, wl.n2, wl.slice_r, wl.u0, fp32=True, rc_every=rc)
            ids.append(P.pe3d_submit(srv, req))
            keep.append(k)
        for rid, wl, rc in zip(ids, wls, rcs):
            t0 = time.perf_counter()
            while P.pe3d_poll(srv, rid)[0] != P.PE3D_REQ_DONE:
                assert time.perf_counter() - t0 < 120
                time.sleep(0.005)
            g = wl.grid
            got = np.empty((g.n_out, g.Ntheta, g.Nz), np.complex64)
            P.pe3d_poll(srv, rid, got)
            assert np.array_equal(got, alone(P, wl, rc)), f"rc={rc}"
    finally:
        P.pe3d_server_destroy(srv)


def test_correction_refused_for_fp64_requests(P):
    wl = workloads.random_case(20, 6, periodic=False, K=1, steps=4, seed=9)
    srv = P.pe3d_server_create(1 << 30, 4, 8)
    try:
        req, keep = P.make_request(wl.grid, wl.n2, wl.slice_r, wl.u0, fp32=False, rc_every=4)
        with pytest.raises(P.PE3DError) as e:
            P.pe3d_submit(srv, req)
        assert e.value.code == P.PE3D_ERR_ARG
    finally:
        P.pe3d_server_destroy(srv)
