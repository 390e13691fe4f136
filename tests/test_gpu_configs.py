"""The measured configurations at their specified size, against the FP64 oracle
(needs a GB300; the oracle runs on the host's cores, about two minutes in all).

* Periodic 200 Hz (1067 x 1024, cyclic azimuth solve, 4000 range steps,
  complex FP32): every stored step within 1e-4 relative L2 of the oracle.
* Batched multi-frequency launch: the four lowest and the two highest of the
  32 log-spaced frequencies (25-400 Hz) at full grid size, their first 500
  range steps in one batched launch, each within 1e-4 of the oracle.
* Served: 32 requests of the Poisson stream (seed 5; 30 drawn at random and
  two full-circle ones), truncated to 500 range steps, complex FP32 with the
  FP64 residual correction every 64 steps, through the request loop: each
  within 1e-4 of the oracle and bit-identical to the same request marched
  alone.

Each test prints the error against range, so a run's log carries the curves.
"""
import time

import numpy as np
import pytest

import oracle
import workloads

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL32 = 1e-4


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
    assert got.shape == ref.shape, (got.shape, ref.shape)
    return np.array([np.linalg.norm((a - b).ravel()) / np.linalg.norm(b.ravel()) for a, b in zip(got, ref)])


def test_config3_periodic_200Hz_full(P, oracle_lib):
    wl = workloads.config3()
    g = wl.grid
    assert (g.Nz, g.Ntheta, g.steps, g.periodic) == (1067, 1024, 4000, True)
    t = time.perf_counter()
    ref = oracle_lib.march(g, wl.n2, wl.slice_r, wl.u0)
    t_or = time.perf_counter() - t
    ranges = oracle.snapshot_ranges(g.r0, g.dr, g.steps, g.stride)
    for exec_mode in (P.PE3D_EXEC_PERSISTENT, P.PE3D_EXEC_RESIDENT):
        with P.Plan.for_grid(g, fp32=True, exec_mode=exec_mode) as plan:
            plan.set_medium(torch.from_numpy(wl.n2).cuda(), wl.slice_r)
            got = plan.march(torch.from_numpy(wl.u0.astype(np.complex64)).cuda(), g.r0, g.steps, g.stride)
            torch.cuda.synchronize()
            ran = plan.info()["exec"]
        err = relerrs(got.cpu().numpy(), ref)
        print(f"\nperiodic 200 Hz, FP32 (exec {ran}), oracle {t_or:.1f} s; rel-L2 vs range:")
        for r, e in zip(ranges, err):
            print(f"  r = {r:8.1f} m  rel-L2 = {e:.3e}")
        assert err.max() < TOL32, err


def test_config4_frequency_subset(P, oracle_lib):
    grids = workloads.config4_grids()
    assert len(grids) == 32
    pick = grids[:4] + grids[-2:]
    steps = 500
    wls = []
    for g in pick:
        g.steps = min(g.steps, steps)
        g.stride = 100
        wls.append(workloads.config4_member(g))
    plans, u0s, outs = [], [], []
    for wl in wls:
        g = wl.grid
        pl = P.Plan.for_grid(g, fp32=True)
        plans.append(pl)
        u0s.append(torch.from_numpy(wl.u0.astype(np.complex64)).cuda())
        outs.append(torch.empty((g.n_out, g.Ntheta, g.Nz), dtype=torch.complex64, device="cuda"))
    P.pe3d_set_medium_batched([p.h for p in plans], [torch.from_numpy(wl.n2).cuda() for wl in wls],
                              [wl.slice_r for wl in wls])
    P.pe3d_march_batched([p.h for p in plans], u0s, [wl.grid.r0 for wl in wls], [wl.grid.steps for wl in wls],
                         [wl.grid.stride for wl in wls], outs)
    torch.cuda.synchronize()
    worst = 0.0
    for wl, out in zip(wls, outs):
        g = wl.grid
        ref = oracle_lib.march(g, wl.n2, wl.slice_r, wl.u0)
        err = relerrs(out.cpu().numpy(), ref)
        print(f"\n{g.name} ({g.Nz} x {g.Ntheta}, {g.steps} steps): rel-L2 vs range "
              + np.array2string(err, precision=2))
        worst = max(worst, err.max())
    for pl in plans:
        pl.close()
    assert worst < TOL32


def test_slice_boundaries_on_step_ranges(P, oracle_lib):
    """Slice k starts exactly at a step's range, R_k = r0 + (j_k + 1) dr as the
    definition rounds it (product, then sum).  The step at R_k must use slice k
    on the GPU as in the oracle: a host that fused the expression into one FMA
    could land an ulp below R_k and keep the previous slice (the served
    request 9891 of the Poisson stream did, at 3e-3 error)."""
    worst = 0.0
    for i, f in enumerate((373.5077, 101.3, 222.2, 57.7)):
        lam = 1500.0 / f
        wl = workloads.random_case(40, 6, periodic=False, K=6, steps=60, seed=800 + i, stride=10, lossy=True,
                                   theta_dependent=True, k0=2 * np.pi * f / 1500.0, dz=lam / 8.0, dr=lam / 4.0)
        g = wl.grid
        jk = np.array([-1, 9, 20, 31, 42, 53])
        wl.slice_r[:] = np.array([g.r0 + float(j + 1) * g.dr for j in jk])
        ref = oracle_lib.march(g, wl.n2, wl.slice_r, wl.u0)
        with P.Plan.for_grid(g, fp32=False) as plan:
            plan.set_medium(torch.from_numpy(wl.n2).cuda(), wl.slice_r)
            got = plan.march(torch.from_numpy(wl.u0).cuda(), g.r0, g.steps, g.stride).cpu().numpy()
        worst = max(worst, relerrs(got, ref).max())
    assert worst < 1e-10, worst


def _config5_sample():
    reqs = workloads.config5_stream(rate=200.0, duration=60.0, seed=5)
    rng = np.random.default_rng(0)
    full_circle = [i for i, r in enumerate(reqs) if workloads.config5_grid(r, max_steps=500).periodic][:2]
    rest = [i for i in range(len(reqs)) if i not in full_circle]
    idx = sorted(list(rng.choice(rest, 30, replace=False)) + full_circle)
    out = []
    for i in idx:
        g = workloads.config5_grid(reqs[i], max_steps=500)
        g.stride = 100
        out.append((int(i), workloads.config5_member(reqs[i], g)))
    return out


def test_config5_served_sample_with_correction(P, oracle_lib):
    sample = _config5_sample()
    assert len(sample) == 32 and any(wl.grid.periodic for _, wl in sample)
    rc = 64
    srv = P.pe3d_server_create(64 << 30, 64, 64)
    ids, keep = [], []
    try:
        for _, wl in sample:
            req, k = P.make_request(wl.grid, wl.n2, wl.slice_r, wl.u0, fp32=True, rc_every=rc)
            ids.append(P.pe3d_submit(srv, req))
            keep.append(k)
        results = {}
        t0 = time.perf_counter()
        while len(results) < len(ids):
            assert time.perf_counter() - t0 < 600, "request loop did not finish"
            for rid, (i, wl) in zip(ids, sample):
                if rid in results:
                    continue
                st, _ = P.pe3d_poll(srv, rid)
                if st == P.PE3D_REQ_DONE:
                    g = wl.grid
                    out = np.empty((g.n_out, g.Ntheta, g.Nz), np.complex64)
                    P.pe3d_poll(srv, rid, out)
                    results[rid] = out
            time.sleep(0.01)
        stats = P.pe3d_server_stats(srv)
    finally:
        P.pe3d_server_destroy(srv)
    assert stats["failed"] == 0 and stats["finished"] == 32
    worst = 0.0
    for rid, (i, wl) in zip(ids, sample):
        g = wl.grid
        got = results[rid]
        with P.Plan.for_grid(g, fp32=True) as plan:              # the same request alone
            P.pe3d_set_option(plan.h, P.PE3D_OPT_RC_EVERY, rc)
            plan.set_medium(wl.n2, wl.slice_r)
            alone = np.zeros_like(got)
            P.pe3d_march(plan.h, wl.u0.astype(np.complex64), g.r0, g.steps, g.stride, alone)
        assert np.array_equal(got, alone), f"request {i}: served result differs from the march alone"
        ref = oracle_lib.march(g, wl.n2, wl.slice_r, wl.u0)
        err = relerrs(got, ref)
        print(f"\nrequest {i} ({g.freq:.1f} Hz, {g.Nz} x {g.Ntheta}{' periodic' if g.periodic else ''}): "
              f"rel-L2 vs range " + np.array2string(err, precision=2))
        worst = max(worst, err.max())
    assert worst < TOL32
