"""pe3d_set_medium from device memory, page-locked host memory and pageable host
memory gives bit-identical marches (needs a GB300).

The depth set-up reads a medium in device memory in place and writes the
plan's own copy as it goes; a host medium is copied first.  The copy must
hold the medium afterwards: the FP64 correction and the interpolated medium
read it during the march, and the caller may reuse its buffer as soon as
pe3d_set_medium returns.
"""
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
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    return P


def march(P, wl, source, *, fp32, clobber=False, rc=0, **opts):
    g = wl.grid
    cdt = np.complex64 if fp32 else np.complex128
    n2 = np.ascontiguousarray(wl.n2)
    if source == "device":
        buf = torch.from_numpy(n2.copy()).cuda()
    elif source == "pinned":
        buf = torch.from_numpy(n2.copy()).pin_memory()
        assert buf.is_pinned()
    else:
        buf = n2.copy()
    with P.Plan.for_grid(g, fp32=fp32, **opts) as plan:
        if rc:
            P.pe3d_set_option(plan.h, P.PE3D_OPT_RC_EVERY, rc)
        plan.set_medium(buf, wl.slice_r)
        if clobber:   # the caller reuses its buffer: the plan must hold its own copy
            if source == "pageable":
                buf[...] = np.nan
            else:
                buf.fill_(complex("nan"))
            torch.cuda.synchronize()
        u0 = torch.from_numpy(np.ascontiguousarray(wl.u0, dtype=cdt)).cuda()
        out = plan.march(u0, g.r0, g.steps, g.stride)
        torch.cuda.synchronize()
    return out.cpu().numpy()


CASES = [
    # (id, Nz, Ntheta, periodic, K, steps, fp32, options)
    ("pade-fp32", 300, 37, False, 3, 12, True, {}),
    ("pade-fp64-periodic", 129, 24, True, 2, 8, False, {}),
    ("rc4-fp32", 211, 33, False, 3, 12, True, {"rc": 4}),
    ("interp-fp32", 180, 20, False, 3, 10, True, {"interp": 1}),
    ("taylor-fp64", 150, 18, False, 2, 8, False, {"scheme": 1}),   # PE3D_SCHEME_TAYLOR
]


@pytest.mark.parametrize("case", CASES, ids=[c[0] for c in CASES])
def test_sources_bit_identical(P, case):
    _, Nz, Nt, per, K, steps, fp32, opts = case
    wl = workloads.random_case(Nz, Nt, periodic=per, K=K, steps=steps, seed=900 + Nz, stride=2)
    ref = march(P, wl, "pageable", fp32=fp32, **opts)
    assert np.isfinite(ref).all()
    for source in ("device", "pinned"):
        got = march(P, wl, source, fp32=fp32, **opts)
        assert np.array_equal(got, ref), f"{source} medium differs from the pageable one"
    for source in ("device", "pinned", "pageable"):
        got = march(P, wl, source, fp32=fp32, clobber=True, **opts)
        assert np.array_equal(got, ref), f"{source} medium: the march read the caller's buffer after set-up"


def test_medium_replaced_from_another_source(P):
    """A plan re-set from pinned memory after a device medium marches the new medium."""
    a = workloads.random_case(200, 30, periodic=False, K=2, steps=6, seed=951, stride=3)
    b = workloads.random_case(200, 30, periodic=False, K=2, steps=6, seed=952, stride=3)
    g = a.grid
    u0 = torch.from_numpy(np.ascontiguousarray(a.u0, dtype=np.complex64)).cuda()
    with P.Plan.for_grid(g, fp32=True) as plan:
        P.pe3d_set_option(plan.h, P.PE3D_OPT_RC_EVERY, 3)
        plan.set_medium(torch.from_numpy(np.ascontiguousarray(a.n2)).cuda(), a.slice_r)
        out_a = plan.march(u0, g.r0, g.steps, g.stride).cpu().numpy()
        plan.set_medium(torch.from_numpy(np.ascontiguousarray(b.n2)).pin_memory(), b.slice_r)
        out_b = plan.march(u0, g.r0, g.steps, g.stride).cpu().numpy()
    with P.Plan.for_grid(g, fp32=True) as plan:
        P.pe3d_set_option(plan.h, P.PE3D_OPT_RC_EVERY, 3)
        plan.set_medium(np.ascontiguousarray(b.n2), b.slice_r)
        ref_b = plan.march(u0, g.r0, g.steps, g.stride).cpu().numpy()
    assert not np.array_equal(out_a, out_b)
    assert np.array_equal(out_b, ref_b)
