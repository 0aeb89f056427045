"""Neighbor capacities through the C-ABI.

An atom with more neighbors inside the 5.1 A list than a system's rows hold
(160 by default) makes the system grow its rows to 256 once and redo the
evaluation: the result matches the oracle. More than 60 neighbors inside the
3.5 A angular cutoff is an error (MLP_EOVERFLOW, reported, never a wrong
result), and the system evaluates ordinary coordinates afterwards.
"""
import numpy as np
import pytest
import torch

import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_2310_03121_b300 as P

    P.load()
    return P


@pytest.fixture(scope="module")
def wts():
    return gen.make_weights()


def _shell(n_shell=176, radius=4.3, seed=2):
    """A central atom and n_shell atoms spread over a sphere (Fibonacci
    lattice): the centre has n_shell neighbors inside 5.1 A and none inside
    3.5 A; a shell atom has ~30 angular neighbors."""
    k = np.arange(n_shell) + 0.5
    phi = np.arccos(1 - 2 * k / n_shell)
    th = np.pi * (1 + 5 ** 0.5) * k
    pts = radius * np.stack([np.cos(th) * np.sin(phi), np.sin(th) * np.sin(phi), np.cos(phi)], 1)
    xyz = np.concatenate([np.zeros((1, 3)), pts])
    sp = np.random.default_rng(seed).integers(0, 4, size=n_shell + 1).astype(np.int8)
    return sp, xyz


def test_rows_grow_for_a_crowded_atom(P, wts):
    sp, xyz = _shell()
    E_ref, F_ref = oracle.energy_forces(sp, xyz, None, oracle.Weights(wts))
    s = P.System(P.Weights(wts), sp, xyz, None, precision="fp32")
    E, F = s.energy_forces()
    assert abs(E - E_ref) <= 1e-6 * abs(E_ref), (E, E_ref)
    assert np.abs(F - F_ref).max() <= 1e-4
    counts, _ = s.debug_neighbors()
    assert counts[0] == len(sp) - 1 > 160


def test_angular_overflow_is_an_error_and_the_system_recovers(P, wts):
    from paper_2310_03121_b300 import _lib

    rng = np.random.default_rng(4)
    n = 80
    ball = rng.normal(size=(n, 3))
    ball *= (2.4 * rng.uniform(size=(n, 1)) ** (1 / 3)) / np.linalg.norm(ball, axis=1, keepdims=True)
    sp = rng.integers(0, 4, size=n).astype(np.int8)
    spread = gen.random_molecule(n, seed=9).coords   # ordinary density, same atom count
    s = P.System(P.Weights(wts), sp, spread, None, precision="fp32")
    with pytest.raises(P.MLPError) as ei:
        s.energy_forces(ball)
    assert ei.value.code == _lib.MLP_EOVERFLOW
    E, F = s.energy_forces(spread)
    E_ref, F_ref = oracle.energy_forces(sp, spread, None, oracle.Weights(wts))
    assert abs(E - E_ref) <= 1e-6 * abs(E_ref)
    assert np.abs(F - F_ref).max() <= 1e-4
