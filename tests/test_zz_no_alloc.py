"""The allocation-free neighbor search (mlp_neighbors_static) against the
library's regular neighbor search.

mlp_neighbors_static is for callers that may not allocate device memory
while they run (fixed memory plans, host-owned pools, time-critical loops):
its working memory is a fixed static device array shared by all calls. This
test calls it through the C-ABI twice in a row on the same inputs (the
second call must see the array reset by the call itself) and compares the
lists with the ones the regular system path builds: neighbor lists are
integer results, so counts must be equal and each atom's neighbors the same
set. It also checks the size limit, and, against the FP64 oracle's neighbor
sets: a periodic box with fewer than three cells per axis (every cell
visited once), lists shorter than the true neighbor counts (the counts stay
the true counts, the stored entries are true neighbors), and boxes whose cell
grid at the requested cutoff would exceed the static array (fewer, wider
cells). It lives in a file of its own, collected last, and passes alone in a
fresh process as well as after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

import gen
import oracle

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


def _oracle_sets(coords, cell, cutoff):
    """Neighbors every correct search must find (outside the rounding band of
    the cutoff) and those it may find (inside it), per atom."""
    pairs, band = oracle.neighbors(coords, cell, cutoff)
    n = coords.shape[0]
    must = [set() for _ in range(n)]
    may = [set() for _ in range(n)]
    for (i, j), b in zip(pairs, band):
        (may if b else must)[int(i)].add(int(j))
    return must, may


def _check_against_oracle(counts, lst, must, may, cap):
    for i in range(len(must)):
        k = int(counts[i])
        assert len(must[i]) <= k <= len(must[i]) + len(may[i]), (i, k, len(must[i]))
        stored = lst[i, :min(k, cap)]
        assert len(set(stored.tolist())) == stored.size, i           # no duplicates
        assert set(stored.tolist()) <= must[i] | may[i], i            # only true neighbors
        if k <= cap:
            assert must[i] <= set(stored.tolist()), i                 # all of them when they fit


@pytest.mark.parametrize("cutoff,cap", [(5.1, 256), (3.5, 4)])
def test_static_neighbors_two_cells_per_axis(lib, cutoff, cap):
    """L = 12 A: floor(12 / 5.1) = 2 cells per axis, so every cell is visited
    once along each axis instead of the three relative cells."""
    c = gen.random_molecule(173, 5, density=0.1, periodic=True)
    if cutoff == 5.1:
        assert np.all(c.cell // cutoff == 2)
    must, may = _oracle_sets(c.coords, c.cell, cutoff)
    assert max(len(m) for m in must) > cap or cap == 256
    for _ in range(2):
        counts, lst = _static(lib, c.coords, c.cell, cutoff, cap)
        _check_against_oracle(counts, lst, must, may, cap)


def test_static_neighbors_short_list(lib):
    """cap smaller than the largest neighbor count: the counts are the true
    counts (the MD pair guard reads only those), the rows hold cap true
    neighbors, nothing is written past a row."""
    c = gen.make_config(1)
    must, may = _oracle_sets(c.coords, None, 3.5)
    cap = 4
    assert max(len(m) for m in must) > 3 * cap
    counts, lst = _static(lib, c.coords, None, 3.5, cap)
    _check_against_oracle(counts, lst, must, may, cap)


@pytest.mark.parametrize("cutoff", [0.5, 1.2])
def test_static_neighbors_fewer_wider_cells(lib, cutoff):
    """The 59.5 A box at a short cutoff needs 119^3 (0.5 A) or 49^3 (1.2 A)
    cells, more than the array holds: the call uses at most its 32,768 cells
    (wider ones) and still finds exactly the oracle's pairs (1.2 A: the O-H
    bonds of the waters; 0.5 A: none, as the MD guard expects)."""
    c = gen.make_config(4)
    must, may = _oracle_sets(c.coords, c.cell, cutoff)
    for _ in range(2):
        counts, lst = _static(lib, c.coords, c.cell, cutoff, 4)
        _check_against_oracle(counts, lst, must, may, 4)
    if cutoff == 0.5:
        assert counts.max() == 0


def test_static_neighbors_huge_box(lib):
    """A 1,300 A periodic box with a 1 A cutoff: 1300^3 cells would overflow a
    32-bit count; the grid is capped and the result is still exact."""
    c = gen.make_config(0)
    cell = np.array([1300.0, 1300.0, 1300.0])
    x = c.coords + 640.0
    must, may = _oracle_sets(x, cell, 1.2)
    counts, lst = _static(lib, x, cell, 1.2, 8)
    _check_against_oracle(counts, lst, must, may, 8)
