"""ML/MM mechanical embedding (section "OpenMM-ML": a listed subset of the
atoms is modeled with the MLP, the rest and the interaction between the two
regions with a conventional force field supplied by the caller) through
mlp_energy_forces_subset_device, against the oracle's ML region.

Bars: FP32 path energy relative error <= 1e-6, max force error <= 1e-4
eV/A; BF16 path energy relative error <= 1e-3, force RMS <= 2e-2 eV/A. Rows
outside the region are never touched: equal bit for bit to what the caller
put there.
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


def _region(P, W, c, idx, precision):
    s = P.System(W, c.species[idx], None, c.cell, precision=precision)
    x = torch.from_numpy(np.ascontiguousarray(c.coords)).cuda()
    it = torch.from_numpy(np.ascontiguousarray(idx, dtype=np.int32)).cuda()
    return s, x, it


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_ligand_region_in_solvent(P, W, OW, precision):
    """Workload 1: the 72-atom ligand is the ML region, the 600 water atoms
    are classical; the caller's forces on every row are kept and the ML
    forces added to the ligand rows."""
    c = gen.make_config(1)
    idx = np.arange(72)
    E_ref, F_ref = oracle.ml_region(c.species, c.coords, c.cell, OW, idx)
    s, x, it = _region(P, W, c, idx, precision)
    mm = torch.from_numpy(np.random.default_rng(0).normal(size=(c.n, 3)).astype(np.float32)).cuda()
    F = mm.clone()
    E, F = s.energy_forces_subset_device(x, it, forces_full=F, accumulate=True)
    s.sync()
    E, F, mm = float(E.item()), F.cpu().numpy(), mm.cpu().numpy()
    assert np.array_equal(F[72:], mm[72:])
    dF = F[:72].astype(np.float64) - mm[:72] - F_ref[:72]
    if precision == "fp32":
        assert abs(E - E_ref) <= 1e-6 * abs(E_ref), (E, E_ref)
        assert np.abs(dF).max() <= 1e-4 + 1e-6, np.abs(dF).max()   # + FP32 rounding of the sum with mm
    else:
        assert abs(E - E_ref) <= 1e-3 * abs(E_ref), (E, E_ref)
        assert np.sqrt(np.mean(dF ** 2)) <= 2e-2


def test_overwrite_and_order(P, W, OW):
    """accumulate = 0 writes the region's rows only; the region's atoms may be
    listed in any order (the system's elements follow that order)."""
    c = gen.make_config(1)
    idx = np.random.default_rng(4).permutation(np.concatenate([np.arange(0, 72, 2), np.arange(300, 330)]))
    E_ref, F_ref = oracle.ml_region(c.species, c.coords, c.cell, OW, idx)
    s, x, it = _region(P, W, c, idx, "fp32")
    F = torch.full((c.n, 3), 7.5, dtype=torch.float32, device="cuda")
    E, F = s.energy_forces_subset_device(x, it, forces_full=F, accumulate=False)
    s.sync()
    E, F = float(E.item()), F.cpu().numpy()
    rest = np.setdiff1d(np.arange(c.n), idx)
    assert np.all(F[rest] == 7.5)
    assert abs(E - E_ref) <= 1e-6 * abs(E_ref)
    assert np.abs(F[idx] - F_ref[idx]).max() <= 1e-4


def test_periodic_region(P, W, OW):
    """Workload 2 (periodic water box): 40 waters as the ML region, evaluated
    with the box's minimum-image convention."""
    c = gen.make_config(2)
    idx = np.arange(120)
    E_ref, F_ref = oracle.ml_region(c.species, c.coords, c.cell, OW, idx)
    s, x, it = _region(P, W, c, idx, "fp32")
    E, F = s.energy_forces_subset_device(x, it)
    s.sync()
    E, F = float(E.item()), F.cpu().numpy()
    assert abs(E - E_ref) <= 1e-6 * abs(E_ref)
    assert np.abs(F - F_ref).max() <= 1e-4


def test_repeated_calls_follow_the_full_coordinates(P, W, OW):
    """The region's positions are gathered on every call: moving the full
    array moves the region (the neighbor list follows)."""
    c = gen.make_config(1)
    idx = np.arange(72)
    s, x, it = _region(P, W, c, idx, "fp32")
    E1, _ = s.energy_forces_subset_device(x, it)
    x2 = c.coords.copy()
    x2[:72] += np.random.default_rng(9).normal(scale=0.05, size=(72, 3))
    x.copy_(torch.from_numpy(x2))
    E2, F2 = s.energy_forces_subset_device(x, it)
    s.sync()
    E_ref, F_ref = oracle.ml_region(c.species, x2, c.cell, OW, idx)
    assert abs(float(E2.item()) - E_ref) <= 1e-6 * abs(E_ref)
    assert np.abs(F2.cpu().numpy() - F_ref).max() <= 1e-4


def test_index_out_of_range_is_reported(P, W):
    c = gen.make_config(1)
    idx = np.arange(72)
    s, x, it = _region(P, W, c, idx, "fp32")
    bad = it.clone()
    bad[5] = c.n                                     # one past the end
    with pytest.raises(P.MLPError):
        s.energy_forces_subset_device(x, bad)
        s.sync()
    with pytest.raises(P.MLPError):                  # n_full smaller than the region
        s.energy_forces_subset_device(x[:10].contiguous(), it)
    E, _ = s.energy_forces_subset_device(x, it)      # the system stays usable
    s.sync()
    assert np.isfinite(float(E.item()))
