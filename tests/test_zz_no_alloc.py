"""The allocation-free neighbor search (mlp_neighbors_static) against the
library's regular neighbor search.

mlp_neighbors_static is for callers that may not allocate device memory
while they run (fixed memory plans, host-owned pools, time-critical loops):
its working memory is a fixed static device array shared by all calls. This
test calls it through the C-ABI twice in a row on the same inputs (the
second call must see the array reset by the call itself) and compares the
lists with the ones the regular system path builds: neighbor lists are
integer results, so counts must be equal and each atom's neighbors the same
set. It also checks the size limit. It lives in a file of its own, collected
last, and passes alone in a fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    from paper_2310_03121_b300 import _lib

    return _lib.load()


def _static(L, coords, cell, cutoff, cap):
    n = coords.shape[0]
    x = torch.as_tensor(np.ascontiguousarray(coords), dtype=torch.float64, device="cuda")
    counts = torch.full((n,), -1, dtype=torch.int32, device="cuda")
    lst = torch.full((n, cap), -1, dtype=torch.int32, device="cuda")
    cl = None if cell is None else np.ascontiguousarray(cell, dtype=np.float64)
    rc = L.mlp_neighbors_static(ctypes.c_void_p(x.data_ptr()), n,
                                None if cl is None else cl.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                cutoff, ctypes.c_void_p(counts.data_ptr()), ctypes.c_void_p(lst.data_ptr()), cap,
                                ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == 0, L.mlp_last_error()
    torch.cuda.synchronize()
    return counts.cpu().numpy(), lst.cpu().numpy()


@pytest.mark.parametrize("case", [4, 1])
def test_static_neighbors_equal_regular_path(lib, case):
    import paper_2310_03121_b300 as P

    c = gen.make_config(case)
    W = P.Weights(gen.make_weights())
    s = P.System(W, c.species, c.coords, c.cell, precision="fp32")
    s.energy_forces()
    counts_ref, lst_ref = s.debug_neighbors()
    cap = lst_ref.shape[1]
    for _ in range(2):
        counts, lst = _static(lib, c.coords, c.cell, 5.1, cap)
        np.testing.assert_array_equal(counts, counts_ref)
        for i in range(c.n):
            k = counts[i]
            assert np.array_equal(np.sort(lst[i, :k]), np.sort(lst_ref[i, :k])), i


def test_static_neighbors_reject_oversize(lib):
    from paper_2310_03121_b300 import _lib

    x = torch.zeros((40000, 3), dtype=torch.float64, device="cuda")
    out = torch.zeros(40000 * 8, dtype=torch.int32, device="cuda")
    rc = lib.mlp_neighbors_static(ctypes.c_void_p(x.data_ptr()), 40000, None, 5.1, ctypes.c_void_p(out.data_ptr()),
                                  ctypes.c_void_p(out.data_ptr()), 8, None)
    assert rc == _lib.MLP_EINVAL
    assert b"static neighbor array" in lib.mlp_last_error()
