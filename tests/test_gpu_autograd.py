"""Differentiation through the torch.autograd.Function (forward: energy;
backward: hand-written network backward + AEV-backward force kernel) on the
6,561-atom periodic water box, against the FP64 oracle on 64 random atoms:
its analytic gradient, and central finite differences of its energy
(h = 1e-4 A). The finite difference moves one atom, so only that atom's
neighborhood changes energy: it is taken on the local energy (atoms within
5.1 A + 0.2 A of it), which equals the full difference (pinned in
tests/test_oracle.py).

Tolerances: FP32 path max |dF| <= 1e-4 eV/A against the analytic gradient;
against the finite differences <= 1e-4 + the FD truncation (h^2 f''' ~ 1e-8).
BF16 path (network on tensor cores): force RMS <= 2e-2 eV/A against both,
energy relative error <= 1e-3.
"""
import numpy as np
import pytest
import torch

import gen
import oracle

pytestmark = pytest.mark.gpu

FD_ATOMS = 64


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


@pytest.fixture(scope="module")
def reference(setup):
    """(atoms, oracle analytic forces, oracle central-difference forces) on
    64 random atoms of the water box."""
    P, MLPEnergy, W, OW, c = setup
    idx = np.random.default_rng(5).choice(c.n, FD_ATOMS, replace=False)
    F_ref = oracle.forces_subset(c.species, c.coords, c.cell, OW, idx)
    h = 1e-4
    F_fd = np.zeros((FD_ATOMS, 3))
    for q, m in enumerate(idx):
        ctr = c.coords[m].copy()
        for a in range(3):
            xp = c.coords.copy()
            xp[m, a] += h
            Ep = oracle.local_energy(c.species, xp, c.cell, OW, int(m), ctr)
            xp[m, a] -= 2 * h
            Em = oracle.local_energy(c.species, xp, c.cell, OW, int(m), ctr)
            F_fd[q, a] = -(Ep - Em) / (2 * h)
    # the oracle's two gradients agree to the FD truncation (pinned on small systems)
    assert np.abs(F_fd - F_ref).max() <= 1e-6 * max(1.0, np.abs(F_ref).max())
    return idx, F_ref, F_fd


@pytest.mark.parametrize("keep_aev", [True, False])
def test_autograd_forces_fp32(setup, reference, keep_aev):
    P, MLPEnergy, W, OW, c = setup
    idx, F_ref, F_fd = reference
    s = P.System(W, c.species, c.coords, c.cell, precision="fp32")
    x = torch.tensor(c.coords, dtype=torch.float64, device="cuda", requires_grad=True)
    E = MLPEnergy.apply(x, s, keep_aev)
    E.backward()
    F = -x.grad.cpu().numpy()
    E_host, F_host = s.energy_forces()
    assert abs(E.item() - E_host) <= 1e-12 * abs(E_host)
    assert np.abs(F - F_host).max() <= 1e-6 * max(1.0, np.abs(F_host).max())
    assert np.abs(F[idx] - F_ref).max() <= 1e-4
    assert np.abs(F[idx] - F_fd).max() <= 1e-4 + 1e-8
    print(f"fp32 autograd: max |dF| {np.abs(F[idx] - F_ref).max():.2e} (analytic), "
          f"{np.abs(F[idx] - F_fd).max():.2e} (FD, {FD_ATOMS} atoms)")


def test_autograd_scales_with_upstream_gradient(setup):
    P, MLPEnergy, W, OW, c = setup
    s = P.System(W, c.species, c.coords, c.cell, precision="fp32")
    x = torch.tensor(c.coords, dtype=torch.float64, device="cuda", requires_grad=True)
    (3.0 * MLPEnergy.apply(x, s)).backward()
    g3 = x.grad.clone()
    x.grad = None
    MLPEnergy.apply(x, s).backward()
    assert torch.allclose(g3, 3.0 * x.grad, rtol=1e-6, atol=1e-9)


@pytest.mark.parametrize("keep_aev", [True, False])
def test_autograd_bf16(setup, reference, keep_aev):
    P, MLPEnergy, W, OW, c = setup
    idx, F_ref, F_fd = reference
    s = P.System(W, c.species, c.coords, c.cell, precision="bf16")
    x = torch.tensor(c.coords, dtype=torch.float64, device="cuda", requires_grad=True)
    E = MLPEnergy.apply(x, s, keep_aev)
    E.backward()
    F = -x.grad.cpu().numpy()
    rms_a = np.sqrt(np.mean((F[idx] - F_ref) ** 2))
    rms_fd = np.sqrt(np.mean((F[idx] - F_fd) ** 2))
    assert rms_a <= 2e-2 and rms_fd <= 2e-2, (rms_a, rms_fd)
    E_ref = float(np.sum(oracle.atom_energies(c.species, c.coords, c.cell, OW)))
    assert abs(E.item() - E_ref) <= 1e-3 * abs(E_ref)
    print(f"bf16 autograd: force RMS {rms_a:.2e} (analytic), {rms_fd:.2e} (FD, {FD_ATOMS} atoms), "
          f"energy rel {abs(E.item() - E_ref) / abs(E_ref):.2e}")
