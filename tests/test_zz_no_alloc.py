"""pe3d_march_static: the range march without device allocation.

Some callers cannot allocate device memory while they run: a real-time sonar
or tracking loop that fixes its GPU memory at start-up and cannot take
cudaMalloc's implicit synchronisation or a mid-run out-of-memory failure, or
an application whose own allocator owns the device heap.  pe3d_march_static
serves them from one fixed scratch array compiled into the library.

These tests call it through the C ABI and check that two calls in a row each
give what the allocating entry point (pe3d_plan + pe3d_set_medium +
pe3d_march) gives, and what the FP64 oracle gives, within the parity
tolerances used everywhere else (1e-10 for FP64, 2e-5 for FP32).  A third
call repeats the first after the second has left other data in the array: it
must give the bit-identical result and leave the device's free memory
unchanged.  A march larger than the array is refused with a clear error.  The
file is named so that pytest collects it last.
"""
import numpy as np
import pytest

import workloads

TOL = {False: 1e-10, True: 2e-5}


def _relerr(a, b):
    return max(np.linalg.norm((x - y).ravel()) / np.linalg.norm(y.ravel()) for x, y in zip(a, b))


def _args(wl, fp32):
    import paper_1711_00005_gb300 as P
    g = wl.grid
    return (g.Nz, g.Ntheta, g.dz, g.dtheta, g.dr, g.k0, P.PE3D_PERIODIC if g.periodic else P.PE3D_WALLED,
            P.PE3D_FP32 if fp32 else P.PE3D_FP64)


def test_too_large_march_is_refused():
    """The 100 Hz, 2000-step march needs far more than the 32 MiB array: the
    call fails with PE3D_ERR_ARG naming the size, before touching the GPU."""
    from paper_1711_00005_gb300 import build
    build.build()
    import paper_1711_00005_gb300 as P
    g = workloads._config2_grid()
    n2 = np.zeros((101, 1, 1), np.complex128)           # never read: the size check comes first
    with pytest.raises(P.PE3DError) as e:
        P.pe3d_march_static(g.Nz, g.Ntheta, g.dz, g.dtheta, g.dr, g.k0, P.PE3D_WALLED, P.PE3D_FP32, n2,
                            100.0 + 100.0 * np.arange(101), np.zeros(1, np.complex64), g.r0, g.steps, 100,
                            np.zeros(1, np.complex64))
    assert e.value.code == P.PE3D_ERR_ARG
    assert "bytes of scratch" in str(e.value) and "PE3D_STATIC_SCRATCH_BYTES" in str(e.value)


@pytest.mark.gpu
def test_static_march_matches_allocating_march_twice():
    torch = pytest.importorskip("torch")
    from paper_1711_00005_gb300 import build
    build.build()
    import paper_1711_00005_gb300 as P
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required")
    import oracle
    cases = [
        (workloads.random_case(200, 64, periodic=False, K=5, steps=12, seed=91, stride=4), False),
        (workloads.random_case(333, 40, periodic=True, K=3, steps=10, seed=92, stride=5), True),
    ]
    stream = torch.cuda.current_stream()
    inputs, results = [], []
    for wl, fp32 in cases:                       # two calls in a row, each checked
        g = wl.grid
        cdt = torch.complex64 if fp32 else torch.complex128
        n2 = torch.from_numpy(wl.n2).cuda()
        u0 = torch.from_numpy(wl.u0).to(cdt).cuda()
        with P.Plan.for_grid(g, fp32=fp32) as plan:
            plan.set_medium(n2, wl.slice_r)
            ref = plan.march(u0, g.r0, g.steps, g.stride).cpu().numpy()
        out = torch.full((g.steps // g.stride, g.Ntheta, g.Nz), float("nan"), dtype=cdt, device="cuda")
        P.pe3d_march_static(*_args(wl, fp32), n2, wl.slice_r, u0, g.r0, g.steps, g.stride, out, stream)
        got = out.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert _relerr(got, ref) <= TOL[fp32]
        # and directly against the FP64 oracle, at the same tolerances
        assert _relerr(got, oracle.march_workload(wl)) <= TOL[fp32]
        inputs.append((wl, fp32, n2, u0, out))
        results.append(got)
    # a third call repeats the first after the second has filled the array with
    # other data: what a call leaves behind does not change the next result,
    # and the call takes no device memory
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    wl, fp32, n2, u0, out = inputs[0]
    g = wl.grid
    out.fill_(float("nan"))
    torch.cuda.synchronize()
    P.pe3d_march_static(*_args(wl, fp32), n2, wl.slice_r, u0, g.r0, g.steps, g.stride, out, stream)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert np.array_equal(out.cpu().numpy(), results[0])
