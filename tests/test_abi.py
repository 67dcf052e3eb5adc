"""The C-ABI library builds for sm_103a, loads, and exports every function
include/rambo.h declares (no GPU needed: nothing here launches a kernel)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    text = open(os.path.join(ROOT, "include", "rambo.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = set(re.findall(r"\b(rambo_[a-z0-9_]+)\s*\(", text))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    from paper_1910_02611_gb300 import build

    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("rambo_create", "rambo_destroy", "rambo_insert_batch", "rambo_insert_seq_batch",
                     "rambo_query_batch", "rambo_query_seq_batch", "rambo_export_index", "rambo_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_1910_02611_gb300.rambo import SIGNATURES

    assert sorted(SIGNATURES) == _declared_functions()


def test_strerror_without_gpu(lib):
    lib.rambo_strerror.restype = ctypes.c_char_p
    lib.rambo_strerror.argtypes = [ctypes.c_int]
    assert lib.rambo_strerror(0) == b"ok"
    assert b"sequence" in lib.rambo_strerror(-3)


def test_create_rejects_bad_parameters_before_touching_the_gpu(lib):
    # parameter checks come first, so these fail the same way with or without a GPU
    lib.rambo_create.restype = ctypes.c_int
    lib.rambo_create.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64,
                                 ctypes.c_uint32, ctypes.c_uint64, ctypes.POINTER(ctypes.c_void_p)]
    h = ctypes.c_void_p()
    for args in [(10, 4, 2, 1000, 2), (10, 0, 2, 1024, 2), (10, 4, 17, 1024, 2), (10, 4, 2, 1024, 5),
                 (0, 4, 2, 1024, 2), (10, 65536, 2, 1024, 2), (10, 4, 2, 1 << 33, 2)]:
        assert lib.rambo_create(*args, 1, ctypes.byref(h)) == -1
        assert not h.value


def test_kernels_are_compiled_for_sm103a():
    from paper_1910_02611_gb300 import build

    assert "arch=compute_103a,code=sm_103a" in build.ARCH
    assert all("-gencode" == a or "sm_103a" in a for a in build.ARCH)


def test_no_cpu_fallback_without_a_gpu():
    # The product path has no CPU fallback: without a CUDA device, creating an
    # index fails loudly with RAMBO_ECUDA instead of answering on the host.
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1910_02611_gb300 import ECUDA, Rambo, RamboError

    with pytest.raises(RamboError) as e:
        Rambo(100, 10, 3, 1 << 20, 2, 42)
    assert e.value.code == ECUDA


def test_parameter_checks_precede_the_gpu():
    # invalid parameters are rejected before any CUDA call (RAMBO_EINVAL even
    # without a device)
    from paper_1910_02611_gb300 import EINVAL, Rambo, RamboError

    for args in ((0, 10, 3, 1 << 20, 2), (100, 0, 3, 1 << 20, 2), (100, 10, 0, 1 << 20, 2),
                 (100, 10, 3, 1000, 2), (100, 10, 3, 1 << 20, 0), (100, 10, 17, 1 << 20, 2),
                 (100, 65536, 3, 1 << 20, 2), (100, 10, 3, 1 << 20, 5)):
        with pytest.raises(RamboError) as e:
            Rambo(*args, 42)
        assert e.value.code == EINVAL, args
