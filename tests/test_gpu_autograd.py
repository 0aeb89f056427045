"""Differentiation through the torch.autograd.Function (forward: energy;
backward: hand-written network backward + AEV-backward force kernel) on the
6,561-atom periodic water box, against the FP64 oracle: its analytic
gradient on 48 sampled atoms, and central finite differences of its energy
(h = 1e-4 A) on 16 of them. The finite difference moves one atom, so only
that atom's neighborhood changes energy: it is taken on the local energy
(atoms within 5.1 A + 0.2 A of it), which equals the full difference
(pinned in tests/test_oracle.py).

Tolerances: FP32 path max |dF| <= 1e-4 eV/A against the analytic gradient;
against the finite differences <= 1e-4 + the FD truncation (h^2 f''' ~ 1e-8).
"""
import numpy as np
import pytest
import torch

import gen
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_2310_03121_b300 as P
    from paper_2310_03121_b300.autograd import MLPEnergy

    wts = gen.make_weights()
    W = P.Weights(wts)
    c = gen.make_config(2)
    return P, MLPEnergy, W, oracle.Weights(wts), c


@pytest.mark.parametrize("keep_aev", [True, False])
def test_autograd_forces_fp32(setup, keep_aev):
    P, MLPEnergy, W, OW, c = setup
    s = P.System(W, c.species, c.coords, c.cell, precision="fp32")
    x = torch.tensor(c.coords, dtype=torch.float64, device="cuda", requires_grad=True)
    E = MLPEnergy.apply(x, s, keep_aev)
    E.backward()
    F = -x.grad.cpu().numpy()
    E_host, F_host = s.energy_forces()
    assert abs(E.item() - E_host) <= 1e-12 * abs(E_host)
    assert np.abs(F - F_host).max() <= 1e-6 * max(1.0, np.abs(F_host).max())
    idx = np.random.default_rng(5).choice(c.n, 48, replace=False)
    F_ref = oracle.forces_subset(c.species, c.coords, c.cell, OW, idx)
    assert np.abs(F[idx] - F_ref).max() <= 1e-4
    # central finite differences of the oracle energy on 16 atoms
    h = 1e-4
    for m in idx[:16]:
        ctr = c.coords[m].copy()
        for a in range(3):
            xp = c.coords.copy()
            xp[m, a] += h
            Ep = oracle.local_energy(c.species, xp, c.cell, OW, int(m), ctr)
            xp[m, a] -= 2 * h
            Em = oracle.local_energy(c.species, xp, c.cell, OW, int(m), ctr)
            assert abs(F[m, a] - (-(Ep - Em) / (2 * h))) <= 1e-4


def test_autograd_scales_with_upstream_gradient(setup):
    P, MLPEnergy, W, OW, c = setup
    s = P.System(W, c.species, c.coords, c.cell, precision="fp32")
    x = torch.tensor(c.coords, dtype=torch.float64, device="cuda", requires_grad=True)
    (3.0 * MLPEnergy.apply(x, s)).backward()
    g3 = x.grad.clone()
    x.grad = None
    MLPEnergy.apply(x, s).backward()
    assert torch.allclose(g3, 3.0 * x.grad, rtol=1e-6, atol=1e-9)


def test_autograd_bf16(setup):
    P, MLPEnergy, W, OW, c = setup
    s = P.System(W, c.species, c.coords, c.cell, precision="bf16")
    x = torch.tensor(c.coords, dtype=torch.float64, device="cuda", requires_grad=True)
    E = MLPEnergy.apply(x, s, False)
    E.backward()
    F = -x.grad.cpu().numpy()
    idx = np.random.default_rng(6).choice(c.n, 48, replace=False)
    F_ref = oracle.forces_subset(c.species, c.coords, c.cell, OW, idx)
    assert np.sqrt(np.mean((F[idx] - F_ref) ** 2)) <= 2e-2
    E_ref = float(np.sum(oracle.atom_energies(c.species, c.coords, c.cell, OW)))
    assert abs(E.item() - E_ref) <= 1e-3 * abs(E_ref)
