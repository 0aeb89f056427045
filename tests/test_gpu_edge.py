"""Degenerate inputs through the C-ABI against the oracle: a lone atom (AEV
all zero: the energy is the network's value at G = 0, the force zero), two
atoms beyond the cutoff, two atoms inside it (radial terms only: every
angular column zero), three atoms (one angular pair), a system of one
element, one atom of each of the seven elements, and a batch that mixes
one-atom, two-atom and 256-atom molecules (the largest a request may have)
with ordinary ones.

Bars as everywhere: FP32 path energy relative error <= 1e-6 (absolute 1e-9
where the energy is ~0) and max force error <= 1e-4 eV/A; BF16 path energy
relative error <= 1e-3 and force RMS <= 2e-2 eV/A.
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


@pytest.fixture(scope="module")
def W(P, wts):
    return P.Weights(wts)


@pytest.fixture(scope="module")
def OW(wts):
    return oracle.Weights(wts)


def _systems():
    rng = np.random.default_rng(17)
    out = {
        "one atom": (np.array([1], np.int8), np.array([[0.3, -0.2, 0.1]])),
        "two far": (np.array([0, 3], np.int8), np.array([[0.0, 0.0, 0.0], [5.25, 0.0, 0.0]])),
        "two near": (np.array([1, 0], np.int8), np.array([[0.0, 0.0, 0.0], [1.1, 0.2, -0.1]])),
        "three": (np.array([1, 0, 3], np.int8), np.array([[0.0, 0.0, 0.0], [1.1, 0.0, 0.0], [-0.4, 1.3, 0.2]])),
    }
    c = gen.random_molecule(40, seed=5)
    out["one element"] = (np.zeros(40, np.int8), c.coords)
    c7 = gen.random_molecule(7, seed=6)
    out["seven elements"] = (np.arange(7, dtype=np.int8), c7.coords)
    return out


SYSTEMS = _systems()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
@pytest.mark.parametrize("name", list(SYSTEMS))
def test_degenerate_systems(P, W, OW, name, precision):
    sp, x = SYSTEMS[name]
    E_ref, F_ref = oracle.energy_forces(sp, x, None, OW)
    s = P.System(W, sp, x, None, precision=precision)
    E, F = s.energy_forces()
    if precision == "fp32":
        assert abs(E - E_ref) <= 1e-6 * abs(E_ref) + 1e-9, (E, E_ref)
        assert np.abs(F - F_ref).max() <= 1e-4
    else:
        assert abs(E - E_ref) <= 1e-3 * abs(E_ref) + 1e-9, (E, E_ref)
        assert np.sqrt(np.mean((F - F_ref) ** 2)) <= 2e-2
    if name in ("one atom", "two far"):
        assert np.all(F == 0.0)
    if name in ("one atom", "two far", "two near"):
        G = P.System(W, sp, x, None, precision="fp32")
        G.energy_forces()
        assert np.all(G.debug_aev()[:, 112:] == 0.0)   # no angular pair


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_batch_with_extreme_molecule_sizes(P, W, OW, precision):
    st = gen.served_stream(count=30)
    mols = [(np.array([2], np.int8), np.array([[1.0, 2.0, 3.0]])),
            (np.array([0, 0], np.int8), np.array([[0.0, 0.0, 0.0], [0.9, 0.3, 0.0]]))]
    big = gen.random_molecule(256, seed=8)
    mols.append((big.species, big.coords))
    mols += [(st.molecule(m).species, st.molecule(m).coords) for m in range(st.count)]
    mols.append((np.array([6], np.int8), np.array([[-4.0, 0.0, 1.0]])))
    ms = np.cumsum([0] + [len(s) for s, _ in mols]).astype(np.int32)
    sp = np.concatenate([s for s, _ in mols])
    xyz = np.concatenate([x for _, x in mols])
    b = P.Batch(W, precision=precision, max_atoms=int(ms[-1]), max_mols=len(mols))
    E, F = b.run(ms, sp, xyz)
    b.close()
    E_ref, F_ref = oracle.energy_forces_batch(ms, sp, xyz, OW)
    if precision == "fp32":
        assert (np.abs(E - E_ref) <= 1e-6 * np.abs(E_ref) + 1e-9).all()
        assert np.abs(F - F_ref).max() <= 1e-4
    else:
        assert (np.abs(E - E_ref) <= 1e-3 * np.abs(E_ref) + 1e-9).all()
        assert np.sqrt(np.mean((F - F_ref) ** 2)) <= 2e-2
    assert np.all(F[0] == 0.0) and np.all(F[-1] == 0.0)   # the lone atoms


def test_huge_periodic_box(P, W, OW):
    """Three copies of the 24-atom molecule far apart in a 1,300 A periodic
    box: floor(1300 / 5.1)^3 cells would overflow a 32-bit count, so the grid
    is capped (fewer, wider cells) and the result equals the oracle's."""
    c = gen.make_config(0)
    cell = np.array([1300.0, 1300.0, 1300.0])
    sp = np.concatenate([c.species] * 3)
    x = np.concatenate([c.coords + off for off in (300.0, 700.0, 1297.0)])   # the last copy straddles the boundary
    E_ref, F_ref = oracle.energy_forces(sp, x, cell, OW)
    s = P.System(W, sp, x, cell, precision="fp32")
    E, F = s.energy_forces()
    assert abs(E - E_ref) <= 1e-6 * abs(E_ref), (E, E_ref)
    assert np.abs(F - F_ref).max() <= 1e-4
