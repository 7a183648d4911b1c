"""The C ABI library loads without a GPU, exports every entry point include/sped.h declares, and
rejects bad arguments on the host before touching a device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "sped.h")


def _declared():
    text = open(HEADER).read()
    pat = r"^\s*(?:const\s+)?(?:sped_status|void|const char)\s*\*?\s*(sped_\w+)\s*\("
    return sorted(set(re.findall(pat, text, re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2207_14589_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for want in ["sped_build_laplacian", "sped_set_polynomial", "sped_apply_poly",
                 "sped_eig_step", "sped_solve_bottom_k", "sped_cluster_assign"]:
        assert want in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing


def test_host_validation_without_gpu(lib):
    lib.sped_last_error.restype = ctypes.c_char_p
    size = ctypes.c_size_t()
    assert lib.sped_workspace_size(ctypes.c_int64(-1), ctypes.c_int64(0), ctypes.byref(size)) == 1
    assert lib.sped_workspace_size(ctypes.c_int64(100), ctypes.c_int64(400),
                                   ctypes.byref(size)) == 0
    assert size.value > 400 * 4
    out = ctypes.c_void_p()
    # odd nnz cannot be symmetric: rejected before any launch
    st = lib.sped_build_laplacian(ctypes.c_int64(4), ctypes.c_int64(3), ctypes.c_void_p(16),
                                  ctypes.c_void_p(16), None, None, ctypes.c_size_t(0), 1, None,
                                  ctypes.byref(out))
    assert st == 2 and b"odd" in lib.sped_last_error()
    assert lib.sped_set_polynomial(None, 0, 3, ctypes.c_double(0), ctypes.c_double(0), None,
                                   ctypes.c_double(0)) == 1
    assert lib.sped_gram_scratch_size(ctypes.c_int64(1000), 20, 20, ctypes.byref(size)) == 0
    assert size.value > 0
    # misaligned / bad layouts are rejected on the host
    assert lib.sped_gram(ctypes.c_int64(10), ctypes.c_void_p(0), 1, 4, 4, None, 1, 0, 0,
                         ctypes.c_void_p(64), None, ctypes.c_size_t(0), None) == 1
    assert lib.sped_cluster_scratch_size(ctypes.c_int64(10), 3, 2, ctypes.byref(size)) == 0
    lib.sped_version.restype = ctypes.c_char_p
    assert b"sm_103a" in lib.sped_version()


def test_python_binding_fails_loudly_without_device():
    import torch
    import paper_2207_14589_gb300 as sped
    if torch.cuda.is_available():
        pytest.skip("a device is present")
    with pytest.raises(Exception):
        sped.Graph(torch.zeros(3, dtype=torch.int32), torch.zeros(0, dtype=torch.int32))
