"""CPU checks of the boundary: the library builds, loads, and exports every
symbol include/mpi_gb300.h declares (no compute calls without a GPU)."""

import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "mpi_gb300.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(mpi_[a-z0-9_]+)\s*\(", txt)))


@pytest.fixture(scope="module")
def lib():
    from paper_2008_09042_gb300 import _lib, build

    if not os.path.exists(_lib.LIB_PATH):
        build.build()
    return _lib.load()


def test_every_declared_symbol_is_exported(lib):
    names = _declared()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n


def test_binding_covers_header():
    from paper_2008_09042_gb300 import _lib

    assert sorted(_lib.EXPORTS) == _declared()


def test_null_context_is_rejected_without_gpu(lib):
    import ctypes

    assert lib.mpi_ctx_create(None, 0, None) == 1  # MPI_ERR_ARG
    assert lib.mpi_forward(None, None, None, None, 1, None, None, 0) == 1
    assert lib.mpi_last_error(None) == b"null context"
    # context settings and queries take a null context without touching a device
    assert lib.mpi_ctx_tf32_reading(None) == -1
    assert lib.mpi_ctx_set_tf32x3(None, 0) == 1
    assert lib.mpi_ctx_set_wait_limit(None, 10**6) == 1
    assert lib.mpi_ctx_workspace_bytes(None) == -1
    # no device here: creating a context reports a CUDA error instead of faulting
    h = ctypes.c_void_p()
    st = lib.mpi_ctx_create(ctypes.byref(h), 0, None)
    import torch

    if not torch.cuda.is_available():
        assert st == 3
