"""sped_gram_noalloc: the Gram for callers that cannot allocate device memory (for example code
in a host callback, a real-time loop or a plugin host, where cudaMalloc may synchronise the
device or no allocator is available). It keeps its per-CTA partial sums in a static 4 MiB
device array inside the library instead of caller scratch. Checked through the C ABI on two
calls in a row (the second call reuses the array the first one left behind) against the FP64
product of the stored inputs, with torch's allocator counters and the device's free memory
unchanged across the calls. This file is named to run last."""
import ctypes

import numpy as np
import pytest
import torch

import gen
import paper_2207_14589_gb300 as sped
from util_gpu import assert_gram_close, stored, to_block

pytestmark = pytest.mark.gpu

_DT = {torch.bfloat16: sped.BF16, torch.float32: sped.F32, torch.float64: sped.F64}


def _noalloc():
    f = sped.lib().sped_gram_noalloc
    vp, i32, i64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64
    f.argtypes = [i64, vp, i32, i32, i32, vp, i32, i32, i32, vp, vp]
    f.restype = ctypes.c_int
    return f


def _call(f, n, A, ka, B, kb, G):
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return f(n, ctypes.c_void_p(A.data_ptr()), _DT[A.dtype], A.stride(0), ka,
             ctypes.c_void_p(B.data_ptr()) if B is not None else None,
             _DT[B.dtype] if B is not None else _DT[A.dtype],
             B.stride(0) if B is not None else 0, kb, ctypes.c_void_p(G.data_ptr()), stream)


def _torch_alloc_state():
    st = torch.cuda.memory_stats()
    return (torch.cuda.memory_allocated(), torch.cuda.memory_reserved(),
            st.get("allocation.all.allocated", 0), st.get("segment.all.allocated", 0))


# tolerances as in test_gpu_solver.test_gram, element-wise against the FP64 product
@pytest.mark.parametrize("dtype,n,ka,kb,tol", [(torch.float32, 100003, 20, 20, 2e-6),
                                               (torch.float64, 50000, 32, 32, 1e-13),
                                               (torch.bfloat16, 7777, 7, 3, 1e-6),
                                               (torch.float32, 2500, 5, 0, 2e-6)])
def test_gram_noalloc_matches_fp64_product_twice(dtype, n, ka, kb, tol):
    A0 = gen.gaussian_block(n, ka, seed=31)
    B0 = gen.gaussian_block(n, kb, seed=32) if kb else None
    A = to_block(A0, dtype)
    B = to_block(B0, dtype) if kb else None
    M = stored(A0, dtype) if not kb else np.concatenate([stored(A0, dtype), stored(B0, dtype)],
                                                        axis=1)
    want = M.T @ M
    f = _noalloc()
    K2 = ka + kb
    Gs = [torch.full((K2, K2), float("nan"), dtype=torch.float64, device="cuda")
          for _ in range(2)]
    torch.cuda.synchronize()
    for t, G in enumerate(Gs):
        before, free0 = _torch_alloc_state(), torch.cuda.mem_get_info()[0]
        st = _call(f, n, A, ka, B, kb, G)
        assert st == sped.OK, sped.lib().sped_last_error().decode()
        torch.cuda.synchronize()
        # nothing allocated: neither through torch's allocator nor on the device (the first
        # call in a process may load the library's module holding the static array)
        assert _torch_alloc_state() == before
        if t == 1:
            assert torch.cuda.mem_get_info()[0] == free0
        assert_gram_close(G.cpu().numpy(), want, tol)
    # the second call, which found the first call's partials in the array, gives the same bits
    assert torch.equal(Gs[0], Gs[1])


def test_gram_noalloc_rejects_more_than_64_columns():
    n = 64
    A = to_block(gen.gaussian_block(n, 40, seed=1), torch.float32)
    B = to_block(gen.gaussian_block(n, 25, seed=2), torch.float32)
    G = torch.zeros((65, 65), dtype=torch.float64, device="cuda")
    st = _call(_noalloc(), n, A, 40, B, 25, G)
    assert st == sped.ERR_UNSUPPORTED
    assert b"maximum" in sped.lib().sped_last_error()
