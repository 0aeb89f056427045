"""Neighbor capacities through the C-ABI.

An atom with more neighbors inside the 5.1 A list than a system's rows hold
(160 by default) makes the system grow its rows to 256 once and redo the
evaluation: the result matches the oracle. An atom with more than 48
neighbors inside the 3.5 A angular cutoff is done by the AEV's and the force
kernel's second launches (up to 256 angular neighbors, more than a row
holds): crowded atoms alone, mixed with ordinary ones, in a batch, at both
precisions, against the oracle, and the system evaluates ordinary
coordinates afterwards.
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


def _ball(n=80, radius=2.4, seed=4):
    """n atoms inside a 2.4 A ball: most have more than 48 angular neighbors."""
    rng = np.random.default_rng(seed)
    ball = rng.normal(size=(n, 3))
    ball *= (radius * rng.uniform(size=(n, 1)) ** (1 / 3)) / np.linalg.norm(ball, axis=1, keepdims=True)
    sp = rng.integers(0, 4, size=n).astype(np.int8)
    return sp, ball


def _check(E, F, E_ref, F_ref, precision, e_abs):
    """The path's bars, with the energy bar taken per atom (against e_abs =
    sum_i |e_i|): these crowded geometries (14x water density, AEV entries up
    to ~35 instead of ~4) make per-atom energies of both signs and large
    AEV sums, so FP32 rounding that is 1e-6 of each atom's energy can exceed
    1e-6 of the total."""
    if precision == "fp32":
        assert abs(E - E_ref) <= 1e-6 * e_abs, (E, E_ref)
        assert np.abs(F - F_ref).max() <= 1e-4, np.abs(F - F_ref).max()
    else:
        assert abs(E - E_ref) <= 1e-3 * e_abs, (E, E_ref)
        assert np.sqrt(np.mean((F - F_ref) ** 2)) <= 2e-2
    print(f"{precision}: |dE| {abs(E - E_ref):.2e} (|E| {abs(E_ref):.2f}, sum|e_i| {e_abs:.2f}), "
          f"max |dF| {np.abs(F - F_ref).max():.2e}")


def _e_abs(OW, sp, x, cell=None):
    return float(np.abs(oracle.atom_energies(sp, x, cell, OW)).sum())


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_crowded_atoms_take_the_second_launch(P, wts, precision):
    OW = oracle.Weights(wts)
    sp, ball = _ball()
    spread = gen.random_molecule(len(sp), seed=9).coords   # ordinary density, same atom count
    s = P.System(P.Weights(wts), sp, spread, None, precision=precision)
    E, F = s.energy_forces(ball)
    _check(E, F, *oracle.energy_forces(sp, ball, None, OW), precision, _e_abs(OW, sp, ball))
    if precision == "bf16":   # the second launch's AEV rows, element by element
        G = s.debug_aev().astype(np.float64)
        G_ref = oracle.aev(sp, ball, None)
        assert (np.abs(G - G_ref) <= 2e-5 * np.maximum(1.0, np.abs(G_ref)) + 2.0 ** -16 * np.abs(G_ref)).all()
    E, F = s.energy_forces(spread)   # and ordinary coordinates afterwards
    E_ref, F_ref = oracle.energy_forces(sp, spread, None, OW)
    _check(E, F, E_ref, F_ref, precision, abs(E_ref))


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_crowded_and_ordinary_atoms_mixed(P, wts, precision):
    """The ball inside the ligand-in-water system (its atoms placed 14 A from
    the centre): a few atoms take the second launch, the rest the first."""
    OW = oracle.Weights(wts)
    c = gen.make_config(1)
    sp_b, ball = _ball(70, 2.3, 5)
    sp = np.concatenate([c.species, sp_b])
    x = np.concatenate([c.coords, ball + np.array([14.0, 0.0, 0.0]) + c.coords.mean(0)])
    s = P.System(P.Weights(wts), sp, x, None, precision=precision)
    E, F = s.energy_forces()
    _check(E, F, *oracle.energy_forces(sp, x, None, OW), precision, _e_abs(OW, sp, x))


def test_crowded_molecule_in_a_batch(P, wts):
    OW = oracle.Weights(wts)
    st = gen.served_stream(count=12)
    sp_b, ball = _ball(90, 2.6, 6)
    mols = [(st.molecule(m).species, st.molecule(m).coords) for m in range(6)] + [(sp_b, ball)] + \
        [(st.molecule(m).species, st.molecule(m).coords) for m in range(6, 12)]
    ms = np.cumsum([0] + [len(q) for q, _ in mols]).astype(np.int32)
    sp = np.concatenate([q for q, _ in mols])
    xyz = np.concatenate([x for _, x in mols])
    for precision in ("fp32", "bf16"):
        b = P.Batch(P.Weights(wts), precision=precision, max_atoms=int(ms[-1]), max_mols=len(mols))
        E, F = b.run(ms, sp, xyz)
        b.close()
        E_ref, F_ref = oracle.energy_forces_batch(ms, sp, xyz, OW)
        e_abs = np.abs(E_ref)
        e_abs[6] = _e_abs(OW, sp_b, ball)        # the crowded molecule: per-atom bar (see _check)
        if precision == "fp32":
            assert (np.abs(E - E_ref) <= 1e-6 * e_abs).all()
            assert np.abs(F - F_ref).max() <= 1e-4
        else:
            assert (np.abs(E - E_ref) <= 1e-3 * e_abs).all()
            assert np.sqrt(np.mean((F - F_ref) ** 2)) <= 2e-2
