"""Pins for the FP64 oracle: closed forms, library routines, invariants and
finite differences. Nothing here compares the oracle with itself or with the
CUDA path."""
import math

import numpy as np
import pytest
import torch

import gen
import oracle

RC_R, RC_A = 5.1, 3.5
ETA_R = 19.7
R_SHIFTS = np.linspace(0.8, 4.9, 16)
A_SHIFTS = 0.8 + np.arange(4) * (3.5 - 0.8) / 4
Z_SHIFTS = (2 * np.arange(8) + 1) * np.pi / 16


@pytest.fixture(scope="module")
def W():
    return oracle.Weights(gen.make_weights())


# ------------------------------------------------------------------ cutoff / celu
def test_cutoff_special_values():
    for rc in (RC_R, RC_A):
        assert oracle.cutoff(0.0, rc) == pytest.approx(1.0, abs=1e-15)
        assert oracle.cutoff(rc / 2, rc) == pytest.approx(0.5, abs=1e-15)
        assert oracle.cutoff(rc, rc) == 0.0
        assert oracle.cutoff(rc + 0.3, rc) == 0.0
        # just inside: fc ~ (pi d / rc)^2 / 4 for small d = rc - r
        d = 1e-3
        assert oracle.cutoff(rc - d, rc) == pytest.approx((math.pi * d / rc) ** 2 / 4, rel=1e-5)
        assert oracle.cutoff_deriv(rc / 2, rc) == pytest.approx(-math.pi / (2 * rc), rel=1e-14)
        assert oracle.cutoff_deriv(0.0, rc) == 0.0
        assert oracle.cutoff_deriv(rc + 0.1, rc) == 0.0


def test_cutoff_derivative_matches_fd():
    for r in np.linspace(0.3, 5.0, 11):
        h = 1e-6
        fd = (oracle.cutoff(r + h, RC_R) - oracle.cutoff(r - h, RC_R)) / (2 * h)
        assert oracle.cutoff_deriv(r, RC_R) == pytest.approx(fd, abs=1e-8)


def test_celu_matches_torch():
    xs = torch.linspace(-3, 3, 241, dtype=torch.float64, requires_grad=True)
    ref = torch.nn.functional.celu(xs, alpha=0.1)
    ref.sum().backward()
    for x, y, g in zip(xs.detach().tolist(), ref.detach().tolist(), xs.grad.tolist()):
        assert oracle.celu(x) == pytest.approx(y, abs=1e-15)
        if abs(x) > 1e-12:
            # torch forms the derivative as (y + alpha) / alpha, which cancels for x << 0
            assert oracle.celu_deriv(x) == pytest.approx(g, rel=1e-6)
            hh = 1e-6
            fd = (oracle.celu(x + hh) - oracle.celu(x - hh)) / (2 * hh)
            if abs(x) > 2e-6:
                assert oracle.celu_deriv(x) == pytest.approx(fd, rel=1e-7, abs=1e-9)
    assert oracle.celu(-50.0) == pytest.approx(-0.1)
    assert oracle.celu(-0.1 * math.log(2)) == pytest.approx(-0.05, rel=1e-14)


def test_pair_index_enumerates_upper_triangle():
    seen = []
    for a in range(7):
        for b in range(a, 7):
            seen.append(oracle.pair_index(a, b))
            assert oracle.pair_index(b, a) == oracle.pair_index(a, b)
    assert seen == list(range(28))


# ------------------------------------------------------------------ neighbors
def _kdtree_pairs(x, cell, rc):
    from scipy.spatial import cKDTree

    if cell is not None:
        t = cKDTree(np.mod(x, cell), boxsize=cell)
    else:
        t = cKDTree(x)
    P = t.query_pairs(rc, output_type="ndarray")
    return {(int(i), int(j)) for i, j in P} | {(int(j), int(i)) for i, j in P}


@pytest.mark.parametrize("which", ["open", "periodic"])
def test_neighbors_match_kdtree(which):
    if which == "open":
        c = gen.make_config(1)
    else:
        c = gen.random_molecule(700, seed=5, density=0.1, periodic=True)
    for rc in (RC_R, RC_A):
        pairs, band = oracle.neighbors(c.coords, c.cell, rc)
        inside = {(int(i), int(j)) for (i, j), b in zip(pairs, band) if b != 2}
        clear = {(int(i), int(j)) for (i, j), b in zip(pairs, band) if b == 0}
        ref = _kdtree_pairs(c.coords, c.cell, rc)
        assert clear <= ref
        assert ref <= inside | {(int(i), int(j)) for (i, j), b in zip(pairs, band) if b}
        assert len(inside ^ ref) <= int((band > 0).sum())
        # full list: each pair stored in both directions
        assert inside == {(j, i) for i, j in inside}


# ------------------------------------------------------------------ AEV special cases
def test_two_atom_radial_block():
    k = 5
    r = R_SHIFTS[k]
    species = np.array([1, 3])  # C, O
    x = np.array([[0.0, 0.0, 0.0], [r, 0.0, 0.0]])
    G = oracle.aev(species, x)
    fc = 0.5 * np.cos(np.pi * r / RC_R) + 0.5
    # atom 0 sees an O neighbor: only columns 16*3..16*3+15 are non-zero
    nz0 = np.nonzero(G[0])[0]
    assert set(nz0) <= set(range(48, 64))
    nz1 = np.nonzero(G[1])[0]
    assert set(nz1) <= set(range(16, 32))
    assert np.allclose(G[0, 48:64], G[1, 16:32], rtol=0, atol=1e-15)
    # Gaussian centred on shift k: value 0.25 fc at the centre ...
    assert G[0, 48 + k] == pytest.approx(0.25 * fc, rel=1e-14)
    # ... symmetric about it on the even grid of shifts ...
    for q in (1, 2, 3):
        assert G[0, 48 + k - q] == pytest.approx(G[0, 48 + k + q], rel=1e-12)
    # ... and each step of width D = 4.1/15 multiplies by exp(-eta D^2 (2q-1))
    D = 4.1 / 15
    assert G[0, 48 + k + 1] / G[0, 48 + k] == pytest.approx(math.exp(-ETA_R * D * D), rel=1e-12)
    assert G[0, 48 + k + 2] / G[0, 48 + k + 1] == pytest.approx(math.exp(-3 * ETA_R * D * D), rel=1e-12)
    assert np.all(G[:, 112:] == 0.0)


def test_two_atom_beyond_cutoff_is_zero():
    G = oracle.aev(np.array([0, 0]), np.array([[0, 0, 0], [RC_R + 1e-9, 0, 0.0]]))
    assert np.all(G == 0.0)


def test_three_atom_angular_peak():
    """theta' = Z_z and r_ij = r_ik = A_a: the angular factor is 2 * 1 * 1 * fc^2."""
    a, z = 1, 2
    r = A_SHIFTS[a]
    theta = math.acos(math.cos(Z_SHIFTS[z]) / 0.95)  # 0.95 cos(theta) = cos(Z_z)
    species = np.array([0, 1, 2])  # H centre, C and N neighbours
    x = np.array([[0.0, 0, 0], [r, 0, 0], [r * math.cos(theta), r * math.sin(theta), 0.0]])
    G = oracle.aev(species, x)
    fc = 0.5 * math.cos(math.pi * r / RC_A) + 0.5
    p = oracle.pair_index(1, 2)
    col = 112 + 32 * p + 8 * a + z
    assert G[0, col] == pytest.approx(2 * fc * fc, rel=1e-12)
    # only the (C, N) pair block of atom 0 is populated
    nz = np.nonzero(G[0, 112:])[0] // 32
    assert set(nz) == {p}
    # cos(theta' - Z) is symmetric about Z_z: sections z-1 and z+1 agree when
    # the three sections are evenly spaced around theta' = Z_z
    assert G[0, col - 1] == pytest.approx(G[0, col + 1], rel=1e-12)
    # one section away the angular factor is ((1 + cos(pi/8)) / 2)^zeta, zeta = 14.1
    assert G[0, col + 1] / G[0, col] == pytest.approx(((1 + math.cos(math.pi / 8)) / 2) ** 14.1, rel=1e-12)
    # one radial shift away (spacing 0.675 A) the Gaussian is exp(-eta_A 0.675^2), eta_A = 12.5
    assert G[0, col + 8] / G[0, col] == pytest.approx(math.exp(-12.5 * 0.675**2), rel=1e-12)
    # swapping which neighbour is C and which is N leaves the block unchanged
    G2 = oracle.aev(np.array([0, 2, 1]), x)
    assert np.allclose(G2[0], G[0], rtol=1e-14, atol=0)


def test_angular_requires_both_inside_rc_ang():
    x = np.array([[0.0, 0, 0], [1.0, 0, 0], [0, RC_A + 0.01, 0.0]])
    G = oracle.aev(np.array([0, 0, 0]), x)
    assert np.all(G[0, 112:] == 0.0)
    assert G[0, :16].sum() > 0


# ------------------------------------------------------------------ network
def test_network_matches_torch(W):
    w = gen.make_weights()
    rng = np.random.default_rng(7)
    for s in range(7):
        G = rng.uniform(0, 1.5, size=1008) * (rng.uniform(size=1008) < 0.3)
        net = torch.nn.Sequential(
            torch.nn.Linear(1008, 256), torch.nn.CELU(0.1), torch.nn.Linear(256, 192), torch.nn.CELU(0.1),
            torch.nn.Linear(192, 160), torch.nn.CELU(0.1), torch.nn.Linear(160, 1)).double()
        with torch.no_grad():
            for li, lay in enumerate([0, 2, 4, 6]):
                Wt = w[f"W{li + 1}"][s]
                net[lay].weight.copy_(torch.from_numpy(Wt.reshape(-1, Wt.shape[-1]) if li < 3 else Wt[None, :]))
                net[lay].bias.copy_(torch.from_numpy(np.atleast_1d(w[f"b{li + 1}"][s])))
        Gt = torch.tensor(G, requires_grad=True)
        et = net(Gt)[0]
        et.backward()
        e, g = oracle.atom_energy(s, G, W, grad=True)
        assert e == pytest.approx(et.item(), rel=1e-13, abs=1e-14)
        # torch's CELU backward, (y + alpha) / alpha, loses ~1e-7 relative for z << 0
        np.testing.assert_allclose(g, Gt.grad.numpy(), rtol=0, atol=1e-8 * np.abs(g).max())
        # and the gradient against central differences of the oracle energy
        for c in rng.choice(1008, size=6, replace=False):
            Gp, Gm = G.copy(), G.copy()
            Gp[c] += 1e-5
            Gm[c] -= 1e-5
            fd = (oracle.atom_energy(s, Gp, W) - oracle.atom_energy(s, Gm, W)) / 2e-5
            assert g[c] == pytest.approx(fd, rel=1e-6, abs=1e-10)


def test_single_path_network_by_hand():
    z = {k: np.zeros_like(v) for k, v in gen.make_weights().items()}
    z["W1"][2, 0, 5] = 2.0
    z["W2"][2, 0, 0] = 3.0
    z["W3"][2, 0, 0] = 0.5
    z["W4"][2, 0] = 1.5
    z["b4"][2] = 0.25
    Wz = oracle.Weights(z)
    G = np.zeros(1008)
    G[5] = 0.4  # 0.8 -> 2.4 -> 1.2 -> 1.5 * 1.2 + 0.25
    e, g = oracle.atom_energy(2, G, Wz, grad=True)
    assert e == pytest.approx(2.05, abs=1e-14)
    assert g[5] == pytest.approx(1.5 * 0.5 * 3.0 * 2.0, abs=1e-13)
    assert np.count_nonzero(g) == 1
    G[5] = -0.1  # negative branch: alpha (exp(x / alpha) - 1)
    h1 = 0.1 * (math.exp(-0.2 / 0.1) - 1)
    h2 = 0.1 * (math.exp(3 * h1 / 0.1) - 1)
    h3 = 0.1 * (math.exp(0.5 * h2 / 0.1) - 1)
    assert oracle.atom_energy(2, G, Wz) == pytest.approx(1.5 * h3 + 0.25, abs=1e-14)
    # other elements see all-zero weights: energy equals their (zero) b4
    assert oracle.atom_energy(0, G, Wz) == 0.0


def _torch_net(w, k, s):
    """Net k (of an ensemble dict with a leading [nets] axis), element s, as torch layers."""
    net = torch.nn.Sequential(
        torch.nn.Linear(1008, 256), torch.nn.CELU(0.1), torch.nn.Linear(256, 192), torch.nn.CELU(0.1),
        torch.nn.Linear(192, 160), torch.nn.CELU(0.1), torch.nn.Linear(160, 1)).double()
    with torch.no_grad():
        for li, lay in enumerate([0, 2, 4, 6]):
            Wt = w[f"W{li + 1}"][k, s]
            net[lay].weight.copy_(torch.from_numpy(Wt if li < 3 else Wt[None, :]))
            net[lay].bias.copy_(torch.from_numpy(np.atleast_1d(w[f"b{li + 1}"][k, s])))
    return net


@pytest.mark.parametrize("nets", [2, 8])
def test_ensemble_is_mean_of_torch_nets(nets):
    """Section "Performance of MLPs": the ANI-2x ensemble averages eight
    independently trained models; energy and dE/dG are the means over nets."""
    w = gen.make_weights(nets=nets)
    We = oracle.Weights(w)
    assert We.nets == nets
    rng = np.random.default_rng(70 + nets)
    for s in (0, 3, 6):
        G = rng.uniform(0, 1.5, size=1008) * (rng.uniform(size=1008) < 0.3)
        Gt = torch.tensor(G, requires_grad=True)
        et = sum(_torch_net(w, k, s)(Gt)[0] for k in range(nets)) / nets
        et.backward()
        e, g = oracle.atom_energy(s, G, We, grad=True)
        assert e == pytest.approx(et.item(), rel=1e-13, abs=1e-14)
        np.testing.assert_allclose(g, Gt.grad.numpy(), rtol=0, atol=1e-8 * np.abs(g).max())


def test_ensemble_single_path_by_hand():
    """Two nets, each with one live path through element 2: e is the mean of
    the two hand-computed outputs and so is dE/dG."""
    z = {k: np.zeros_like(v) for k, v in gen.make_weights(nets=2).items()}
    z["W1"][0, 2, 0, 5] = 2.0
    z["W2"][0, 2, 0, 0] = 3.0
    z["W3"][0, 2, 0, 0] = 0.5
    z["W4"][0, 2, 0] = 1.5
    z["b4"][0, 2] = 0.25        # net 0: 1.5 * (0.5 * 3 * 2 * 0.4) + 0.25 = 2.05
    z["W1"][1, 2, 7, 9] = 1.0
    z["W2"][1, 2, 4, 7] = 1.0
    z["W3"][1, 2, 9, 4] = 1.0
    z["W4"][1, 2, 9] = -2.0
    z["b4"][1, 2] = 1.0         # net 1: -2 * 0.7 + 1 = -0.4
    G = np.zeros(1008)
    G[5], G[9] = 0.4, 0.7
    e, g = oracle.atom_energy(2, G, oracle.Weights(z), grad=True)
    assert e == pytest.approx((2.05 - 0.4) / 2, abs=1e-14)
    assert g[5] == pytest.approx(1.5 * 0.5 * 3.0 * 2.0 / 2, abs=1e-13)
    assert g[9] == pytest.approx(-2.0 / 2, abs=1e-13)
    assert np.count_nonzero(g) == 2


# ------------------------------------------------------------------ forces
def _fd_forces(c, W, atoms, h):
    out = np.zeros((len(atoms), 3))
    for q, m in enumerate(atoms):
        for a in range(3):
            x = c.coords.copy()
            x[m, a] += h
            Ep = oracle.energy(c.species, x, c.cell, W)
            x[m, a] -= 2 * h
            Em = oracle.energy(c.species, x, c.cell, W)
            out[q, a] = -(Ep - Em) / (2 * h)
    return out


@pytest.mark.parametrize("n", [2, 3, 5, 24])
def test_forces_match_central_differences(W, n):
    if n == 24:
        c = gen.make_config(0)
    else:
        c = gen.random_molecule(n, seed=11, density=0.3)
    E, F = oracle.energy_forces(c.species, c.coords, c.cell, W)
    atoms = list(range(min(n, 6)))
    f4 = _fd_forces(c, W, atoms, 1e-4)
    f5 = _fd_forces(c, W, atoms, 1e-5)
    scale = max(np.abs(F).max(), 1e-3)
    # the two step sizes agree to O(h^2), and both agree with the analytic force
    assert np.abs(f4 - f5).max() <= 1e-6 * scale
    assert np.abs(F[atoms] - f4).max() <= 1e-6 * scale
    assert np.abs(F[atoms] - f5).max() <= 1e-6 * scale


@pytest.mark.parametrize("periodic", [False, True])
def test_forces_from_dEdG_match_central_differences(periodic):
    """The AEV backward alone: for a fixed random g (every column, positive
    and negative), F = -d/dr sum_i g_i . G_i(r), by central differences of
    the oracle's AEV (h = 1e-4 and 1e-5 A)."""
    if periodic:
        c = gen.random_molecule(40, seed=23, density=0.1, periodic=True)
    else:
        c = gen.random_molecule(12, seed=13, density=0.3)
    g = np.random.default_rng(3).normal(size=(c.n, oracle.AEV_LEN))
    F = oracle.forces_from_dEdG(c.species, c.coords, c.cell, g)

    def phi(x):
        return float((g * oracle.aev(c.species, x, c.cell)).sum())

    atoms = [0, 1, c.n // 2, c.n - 1]
    scale = np.abs(F).max()
    fd = {}
    for h in (1e-4, 1e-5):
        out = np.zeros((len(atoms), 3))
        for q, m in enumerate(atoms):
            for a in range(3):
                x = c.coords.copy()
                x[m, a] += h
                p = phi(x)
                x[m, a] -= 2 * h
                out[q, a] = -(p - phi(x)) / (2 * h)
        fd[h] = out
    assert np.abs(fd[1e-4] - fd[1e-5]).max() <= 1e-6 * scale
    assert np.abs(F[atoms] - fd[1e-4]).max() <= 1e-6 * scale
    if not periodic:
        assert np.abs(F.sum(0)).max() <= 1e-10 * np.abs(F).sum()     # translation invariance of g . G


def test_forces_from_dEdG_with_network_gradient_equal_forces(W):
    """With dE/dG from the oracle's network, the AEV backward alone gives the
    forces of the whole evaluation (same arithmetic, same order: equal)."""
    for c in (gen.make_config(0), gen.random_molecule(60, seed=4, density=0.1, periodic=True)):
        E, F = oracle.energy_forces(c.species, c.coords, c.cell, W)
        e, g = oracle.aev_grad(c.species, c.coords, c.cell, W)
        F2 = oracle.forces_from_dEdG(c.species, c.coords, c.cell, g)
        assert np.array_equal(F, F2)
        g2 = np.random.default_rng(1).normal(size=g.shape)       # and it is linear in dE/dG
        Fa = oracle.forces_from_dEdG(c.species, c.coords, c.cell, 2.0 * g - 3.0 * g2)
        Fb = 2.0 * F2 - 3.0 * oracle.forces_from_dEdG(c.species, c.coords, c.cell, g2)
        assert np.abs(Fa - Fb).max() <= 1e-12 * np.abs(Fa).max()


def test_ensemble_forces_match_central_differences():
    We = oracle.Weights(gen.make_weights(nets=3))
    c = gen.random_molecule(9, seed=5, density=0.3)
    E, F = oracle.energy_forces(c.species, c.coords, c.cell, We)
    atoms = [0, 4, 8]
    fd = _fd_forces(c, We, atoms, 1e-4)
    assert np.abs(F[atoms] - fd).max() <= 1e-6 * max(np.abs(F).max(), 1e-3)
    assert np.abs(F.sum(0)).max() <= 1e-10 * max(np.abs(F).max(), 1.0)


def test_ml_region_mechanical_embedding(W):
    """Section "OpenMM-ML": the ML part of a mixed system depends on the ML
    atoms only. Moving the other atoms leaves E_ML and its forces unchanged,
    their force rows are zero, and the ML rows are minus the finite-difference
    gradient of E_ML."""
    c = gen.make_config(1)
    idx = np.arange(0, 72, 3)                        # a subset of the ligand
    E, F = oracle.ml_region(c.species, c.coords, c.cell, W, idx)
    rest = np.setdiff1d(np.arange(c.n), idx)
    assert np.all(F[rest] == 0.0)
    x2 = c.coords.copy()
    x2[rest] += np.random.default_rng(3).normal(scale=0.3, size=(rest.size, 3))
    E2, F2 = oracle.ml_region(c.species, x2, c.cell, W, idx)
    assert E2 == E and np.array_equal(F2, F)
    for m in (idx[0], idx[5], rest[0]):
        for a in range(3):
            xp, xm = c.coords.copy(), c.coords.copy()
            xp[m, a] += 1e-5
            xm[m, a] -= 1e-5
            fd = -(oracle.ml_region(c.species, xp, c.cell, W, idx)[0] -
                   oracle.ml_region(c.species, xm, c.cell, W, idx)[0]) / 2e-5
            assert abs(F[m, a] - fd) <= 1e-6 * max(np.abs(F).max(), 1e-3)


def test_forces_fd_periodic(W):
    c = gen.random_molecule(60, seed=3, density=0.1, periodic=True)
    E, F = oracle.energy_forces(c.species, c.coords, c.cell, W)
    atoms = [0, 17, 42]
    fd = _fd_forces(c, W, atoms, 1e-4)
    assert np.abs(F[atoms] - fd).max() <= 1e-6 * max(np.abs(F).max(), 1e-3)


def test_net_force_and_torque_vanish_open(W):
    c = gen.make_config(0)
    E, F = oracle.energy_forces(c.species, c.coords, None, W)
    s = np.abs(F).sum()
    assert np.abs(F.sum(0)).max() <= 1e-12 * s
    tau = np.cross(c.coords, F).sum(0)
    assert np.abs(tau).max() <= 1e-10 * s * np.abs(c.coords).max()


# ------------------------------------------------------------------ invariances
def test_translation_rotation_permutation_invariance(W):
    c = gen.make_config(0)
    E = oracle.energy(c.species, c.coords, None, W)
    x = c.coords + np.array([3.3, -1.7, 12.25])
    assert oracle.energy(c.species, x, None, W) == pytest.approx(E, rel=1e-12)
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1]])
    R = R @ np.array([[1, 0, 0], [0, math.cos(1.1), -math.sin(1.1)], [0, math.sin(1.1), math.cos(1.1)]])
    assert oracle.energy(c.species, c.coords @ R.T, None, W) == pytest.approx(E, rel=1e-12)
    # forces rotate with the frame
    _, F = oracle.energy_forces(c.species, c.coords, None, W)
    _, FR = oracle.energy_forces(c.species, c.coords @ R.T, None, W)
    np.testing.assert_allclose(FR, F @ R.T, atol=1e-12 * np.abs(F).max())
    # permutation of atoms (of any species, carried with their coordinates)
    perm = np.random.default_rng(1).permutation(c.n)
    Ep, ep = oracle.energy(c.species[perm], c.coords[perm], None, W, per_atom=True)
    assert Ep == pytest.approx(E, rel=1e-12)
    _, e = oracle.energy(c.species, c.coords, None, W, per_atom=True)
    np.testing.assert_allclose(ep, e[perm], rtol=1e-12, atol=1e-15)


def test_same_species_swap_invariance(W):
    c = gen.make_config(0)
    E, e = oracle.energy(c.species, c.coords, None, W, per_atom=True)
    h = np.nonzero(c.species == 0)[0][:2]
    x = c.coords.copy()
    x[[h[0], h[1]]] = x[[h[1], h[0]]]
    E2, e2 = oracle.energy(c.species, x, None, W, per_atom=True)
    assert E2 == pytest.approx(E, rel=1e-13)
    assert e2[h[0]] == pytest.approx(e[h[1]], rel=1e-13)


def test_periodic_translation_invariance(W):
    c = gen.random_molecule(80, seed=9, density=0.1, periodic=True)
    E, F = oracle.energy_forces(c.species, c.coords, c.cell, W)
    x = np.mod(c.coords + np.array([5.3, -2.2, 7.9]), c.cell)
    E2, F2 = oracle.energy_forces(c.species, x, c.cell, W)
    assert E2 == pytest.approx(E, rel=1e-12)
    np.testing.assert_allclose(F2, F, atol=1e-11 * np.abs(F).max())


def test_cutoff_smoothness(W):
    sp = np.array([1, 3])
    Es, Fs = [], []
    for r in (RC_R - 1e-4, RC_R - 1e-7, RC_R, RC_R + 1e-7):
        E, F = oracle.energy_forces(sp, np.array([[0, 0, 0.0], [r, 0, 0]]), None, W)
        Es.append(E)
        Fs.append(np.abs(F).max())
    # energy is continuous across the cutoff and the force goes to zero
    assert abs(Es[1] - Es[3]) < 1e-12
    assert abs(Es[0] - Es[3]) < 1e-6
    assert Fs[1] < 1e-9 and Fs[2] == 0.0


# ------------------------------------------------------------------ subset / local
def test_forces_subset_equals_full(W):
    for c in (gen.make_config(0), gen.random_molecule(60, seed=4, density=0.1, periodic=True)):
        E, F = oracle.energy_forces(c.species, c.coords, c.cell, W)
        idx = [0, 5, c.n - 1]
        np.testing.assert_allclose(oracle.forces_subset(c.species, c.coords, c.cell, W, idx), F[idx],
                                   rtol=1e-12, atol=1e-14)


def test_local_energy_difference_equals_full(W):
    c = gen.random_molecule(80, seed=9, density=0.1, periodic=True)
    m, h = 7, 1e-4
    center = c.coords[m].copy()
    x = c.coords.copy()
    x[m, 1] += h
    dl = oracle.local_energy(c.species, x, c.cell, W, m, center)
    df = oracle.energy(c.species, x, c.cell, W)
    x[m, 1] -= 2 * h
    dl -= oracle.local_energy(c.species, x, c.cell, W, m, center)
    df -= oracle.energy(c.species, x, c.cell, W)
    assert dl == pytest.approx(df, rel=1e-9, abs=1e-15)


def test_batch_driver_equals_single(W):
    s = gen.served_stream(count=6)
    E, F = oracle.energy_forces_batch(s.mol_start, s.species, s.coords, W, nthreads=2)
    for m in range(6):
        mol = s.molecule(m)
        Em, Fm = oracle.energy_forces(mol.species, mol.coords, None, W)
        assert E[m] == Em
        np.testing.assert_array_equal(F[s.mol_start[m]:s.mol_start[m + 1]], Fm)


def test_golden_config0(W):
    import json
    import os

    with open(os.path.join(os.path.dirname(__file__), "golden", "config0_oracle.json")) as f:
        g = json.load(f)
    c = gen.make_config(0)
    E, F, e = oracle.energy_forces(c.species, c.coords, c.cell, W, per_atom=True)
    assert E == pytest.approx(g["energy"], rel=1e-13)
    np.testing.assert_allclose(e, g["atom_energies"], rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(F, g["forces"], rtol=1e-11, atol=1e-15)


def test_parallel_atom_energies_equal_serial(W):
    c = gen.make_config(1)
    E, e = oracle.energy(c.species, c.coords, None, W, per_atom=True)
    e2 = oracle.atom_energies(c.species, c.coords, None, W, nthreads=4)
    np.testing.assert_array_equal(e2, e)
    G = oracle.aev(c.species, c.coords)
    idx = [3, 100, 671]
    np.testing.assert_array_equal(oracle.aev_subset(c.species, c.coords, None, idx), G[idx])


# ------------------------------------------------------------------ Langevin (LF-Middle)
ACC_UNITS = 9.648533212e-3   # (eV / A) / amu in A / fs^2
KE_UNITS = 103.6426965       # amu A^2 / fs^2 in eV
KB_EV = 8.617333262e-5       # eV / K
MASS = np.array([1.008, 12.011, 14.007, 15.999, 32.06, 18.998, 35.45])


@pytest.mark.parametrize("counter,key", [([1, 0, 0, 0], [123, 456]), ([7, 3, 0, 0], [2**63 + 5, 0]),
                                         ([0, 1, 0, 0], [1, 2]), ([12345, 678, 9, 10], [2**64 - 1, 2**64 - 1])])
def test_philox_matches_numpy(counter, key):
    """Philox4x64-10 against numpy.random.Philox, which implements the same
    published generator (it advances its counter before each block)."""
    c = np.array(counter, dtype=object)
    prev = [int(x) for x in c]
    for w in range(4):                              # counter - 1 with borrow
        if prev[w] > 0:
            prev[w] -= 1
            break
        prev[w] = 2**64 - 1
    bg = np.random.Philox(key=np.array(key, dtype=np.uint64), counter=np.array(prev, dtype=np.uint64))
    ref = bg.random_raw(4)
    out = oracle.philox4x64(np.array(counter, dtype=np.uint64), np.array(key, dtype=np.uint64))
    assert np.array_equal(out, ref)


def test_langevin_normals_distribution():
    R = oracle.langevin_normals(2024, 17, 40000).ravel()
    n = R.size
    assert abs(R.mean()) < 4 / np.sqrt(n)
    assert abs(R.var() - 1.0) < 4 * np.sqrt(2.0 / n)
    assert abs(np.mean(R ** 4) - 3.0) < 0.1
    p = np.mean(R < 1.0)                            # Phi(1) = 0.841344746
    assert abs(p - 0.841344746) < 4 * np.sqrt(p * (1 - p) / n)
    Rm = R.reshape(-1, 3)
    assert abs(np.corrcoef(Rm[:, 0], Rm[:, 1])[0, 1]) < 4 / np.sqrt(Rm.shape[0])
    assert abs(np.corrcoef(Rm[:, 1], Rm[:, 2])[0, 1]) < 4 / np.sqrt(Rm.shape[0])
    assert not np.array_equal(oracle.langevin_normals(2024, 18, 10), oracle.langevin_normals(2024, 17, 10))
    assert np.array_equal(oracle.langevin_normals(2024, 17, 10), Rm[:10])


def test_lfmiddle_without_friction_is_leapfrog():
    """No friction, no temperature: the step is leapfrog, which for a harmonic
    force F = -k x conserves v_(n-1/2) v_(n+1/2) + w^2 x_n^2 (w^2 = k / m in
    A / fs^2 units) exactly, step after step."""
    sp = np.array([0, 1, 3, 6, 4])
    rng = np.random.default_rng(1)
    x = rng.normal(size=(5, 3))
    v = rng.normal(scale=0.01, size=(5, 3))
    k = 2.5
    w2 = (k * ACC_UNITS / MASS[sp])[:, None]
    inv = []
    for step in range(400):
        F = -k * x
        x_new, v_new = oracle.lfmiddle_step(sp, x, v, F, 2.0, 0.0, 0.0, 9, step)
        inv.append(v * v_new + w2 * x * x)
        x, v = x_new, v_new
    inv = np.array(inv)
    assert np.abs(inv - inv[0]).max() <= 1e-12 * np.abs(inv[0]).max()


def test_lfmiddle_equipartition_and_decay():
    """Free particles: the friction step leaves the Maxwell-Boltzmann
    distribution invariant (<m v^2> = k T per component) and shrinks the
    velocity memory by a = exp(-gamma dt) per step."""
    n, T, gamma, dt = 20000, 300.0, 5.0, 2.0
    sp = np.random.default_rng(2).integers(0, 7, size=n)
    m = MASS[sp][:, None]
    x = np.zeros((n, 3))
    v = np.zeros((n, 3))
    F = np.zeros((n, 3))
    for step in range(400):
        x, v = oracle.lfmiddle_step(sp, x, v, F, dt, gamma, T, 11, step)
    a = np.exp(-gamma * 1e-3 * dt)
    T_est = np.sum(m * v * v) * KE_UNITS / (3 * n * KB_EV)
    assert abs(T_est - T * (1 - a ** 800)) < 0.01 * T
    x2, v2 = oracle.lfmiddle_step(sp, x, v, F, dt, gamma, T, 11, 400)
    slope = np.sum(v * v2 * m) / np.sum(v * v * m)
    assert abs(slope - a) < 0.005
