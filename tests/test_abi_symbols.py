"""The C ABI builds for sm_103a, loads, and exports every function the public
header declares (CPU only: no compute call is made without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "pe3d.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pe3d_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def lib():
    from paper_1711_00005_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = declared_functions()
    for need in ("pe3d_plan", "pe3d_set_medium", "pe3d_march", "pe3d_submit", "pe3d_poll",
                 "pe3d_server_create", "pe3d_server_destroy", "pe3d_destroy", "pe3d_last_error",
                 "pe3d_march_batched"):
        assert need in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, f"not exported: {missing}"


def test_binding_covers_header():
    import paper_1711_00005_gb300 as P
    missing = [n for n in declared_functions() if not hasattr(P, n)]
    assert not missing, f"binding lacks: {missing}"


def test_errors_without_gpu_are_reported(lib):
    """On a machine without a usable GPU the plan call fails with a CUDA status
    and a message, never a crash; argument errors are caught before CUDA."""
    import paper_1711_00005_gb300 as P
    with pytest.raises(P.PE3DError) as e:
        P.pe3d_plan(0, 4, 1.0, 0.1, 1.0, 0.5)
    assert e.value.code == P.PE3D_ERR_ARG
    with pytest.raises(P.PE3DError) as e:
        P.pe3d_plan(8, 2, 1.0, 0.1, 1.0, 0.5, P.PE3D_PERIODIC)
    assert e.value.code == P.PE3D_ERR_ARG
    with pytest.raises(P.PE3DError) as e:
        P.pe3d_plan(8, 8, -1.0, 0.1, 1.0, 0.5)
    assert e.value.code == P.PE3D_ERR_ARG


def test_kernels_compiled_for_sm103a():
    """The build log lists sm_103a entry points for every march kernel."""
    log = os.path.join(ROOT, "paper_1711_00005_gb300", "_build", "pe3d_f32.cu.log")
    text = open(log).read()
    for k in ("k_phaseA", "k_phaseB", "k_march_persistent", "k_setupA", "k_setupB", "k_prologue"):
        assert re.search(rf"Compiling entry function '\S*{k}\S*' for 'sm_103a'", text), k
