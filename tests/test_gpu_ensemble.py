"""The 8-net ensemble (section "Performance of MLPs", Table 3: ANI-2x is the
average of eight independently trained nets; one AEV, eight network passes)
through the C-ABI, against the FP64 oracle's ensemble.

Bars as for one net: FP32 path energy relative error <= 1e-6 and max force
error <= 1e-4 eV/A; BF16 path energy relative error <= 1e-3 and force RMS
<= 2e-2 eV/A. The network alone (mlp_debug_network) is compared per row:
FP32 against the oracle, BF16 against a float64 emulation of the kernel's
arithmetic net by net (dE/dG of each net in FP32, scaled by 1/8 and summed).
"""
import numpy as np
import pytest
import torch

import gen
import oracle
from test_gpu_parity import _emulate_bf16_network

pytestmark = pytest.mark.gpu

K = 8
E_REL_FP32, F_MAX_FP32 = 1e-6, 1e-4
E_REL_BF16, F_RMS_BF16 = 1e-3, 2e-2


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_2310_03121_b300 as P

    P.load()
    return P


@pytest.fixture(scope="module")
def wts():
    return gen.make_weights(nets=K)


@pytest.fixture(scope="module")
def W(P, wts):
    w = P.Weights(wts)
    assert w.n_nets == K
    return w


@pytest.fixture(scope="module")
def OW(wts):
    return oracle.Weights(wts)


def _rows(n, seed):
    rng = np.random.default_rng(seed)
    c = gen.make_config(1)
    G_all = oracle.aev(c.species, c.coords)
    pick = rng.choice(c.n, size=n, replace=n > c.n)
    sp = c.species[pick].copy()
    sp[: min(n, 7)] = np.arange(min(n, 7))   # every element present when n >= 7
    return sp, G_all[pick].astype(np.float32)


@pytest.mark.parametrize("n", [1, 129, 400])
def test_network_fp32_ensemble(P, W, OW, n):
    sp, G = _rows(n, 200 + n)
    e, g = P.debug_network(W, "fp32", sp, G)
    for q in range(n):
        er, gr = oracle.atom_energy(int(sp[q]), G[q].astype(np.float64), OW, grad=True)
        assert abs(e[q] - er) <= 1e-5 * max(1.0, abs(er))
        assert np.abs(g[q] - gr).max() <= 1e-5 * max(1.0, np.abs(gr).max())


@pytest.mark.parametrize("n", [129, 400])
@pytest.mark.parametrize("mode", ["bf16", "bf16_1pass"])
def test_network_bf16_ensemble_matches_emulation(P, W, wts, n, mode):
    sp, G = _rows(n, 300 + n)
    e, g = P.debug_network(W, mode, sp, G)
    e_ref, g_ref = np.zeros(n), np.zeros((n, 1008))
    for k in range(K):
        ek, gk = _emulate_bf16_network({a: v[k] for a, v in wts.items()}, sp, G, split=(mode == "bf16"),
                                       round_out=False)
        e_ref += ek / K
        g_ref += gk / K
    tol_e = 2e-5 if mode == "bf16" else 2e-3
    assert np.abs(e - e_ref).max() <= tol_e * max(1.0, np.abs(e_ref).max()), np.abs(e - e_ref).max()
    assert np.abs(g - g_ref).max() <= 2e-2 * np.abs(g_ref).max(), (np.abs(g - g_ref).max(), np.abs(g_ref).max())
    assert np.sqrt(np.mean((g - g_ref) ** 2)) <= 2e-3 * np.sqrt(np.mean(g_ref ** 2))


def test_ensemble_differs_from_each_net(P, W, wts):
    """The mean is not any single member: net 0 alone gives other energies."""
    sp, G = _rows(129, 7)
    e8, _ = P.debug_network(W, "fp32", sp, G)
    W0 = P.Weights({a: v[0] for a, v in wts.items()})
    e0, _ = P.debug_network(W0, "fp32", sp, G)
    assert np.abs(e8 - e0).max() > 1e-3 * np.abs(e0).max()


def _small_periodic(n=300, seed=21):
    return gen.random_molecule(n, seed=seed, density=0.1, periodic=True)


CASES = {
    "config0": lambda: gen.make_config(0),
    "config1": lambda: gen.make_config(1),
    "box300": lambda: _small_periodic(300),
}


@pytest.mark.parametrize("case", ["config0", "config1", "box300"])
def test_energy_forces_ensemble_fp32(P, W, OW, case):
    c = CASES[case]()
    E_ref, F_ref = oracle.energy_forces(c.species, c.coords, c.cell, OW)
    s = P.System(W, c.species, c.coords, c.cell, precision="fp32")
    E, F = s.energy_forces()
    assert abs(E - E_ref) <= E_REL_FP32 * abs(E_ref), (E, E_ref)
    assert np.abs(F - F_ref).max() <= F_MAX_FP32, np.abs(F - F_ref).max()


@pytest.mark.parametrize("case", ["config0", "config1", "box300"])
def test_energy_forces_ensemble_bf16(P, W, OW, case):
    c = CASES[case]()
    E_ref, F_ref = oracle.energy_forces(c.species, c.coords, c.cell, OW)
    s = P.System(W, c.species, c.coords, c.cell, precision="bf16")
    E, F = s.energy_forces()
    assert abs(E - E_ref) <= E_REL_BF16 * abs(E_ref), (E, E_ref)
    assert np.sqrt(np.mean((F - F_ref) ** 2)) <= F_RMS_BF16


def test_ensemble_full_size_sampled(P, W, OW):
    """21,080-atom periodic box, BF16 network: per-atom energies of 64 sampled
    atoms and forces on 12 sampled atoms against the oracle evaluated one by
    one (the whole box is beyond the oracle's budget for eight nets)."""
    c = gen.make_config(4)
    s = P.System(W, c.species, c.coords, c.cell, precision="bf16")
    E, F = s.energy_forces()
    e, _ = s.debug_atom_energies(grad=False)
    assert abs(E - float(np.sum(e.astype(np.float64)))) <= 1e-9 * abs(E) + 1e-6
    rng = np.random.default_rng(5)
    idx = rng.choice(c.n, 64, replace=False)
    e_ref = oracle.atom_energies(c.species, c.coords, c.cell, OW, idx=idx)
    assert np.abs(e[idx] - e_ref).max() <= E_REL_BF16 * np.abs(e_ref).max()
    fidx = idx[:12]
    F_ref = oracle.forces_subset(c.species, c.coords, c.cell, OW, fidx)
    assert np.sqrt(np.mean((F[fidx] - F_ref) ** 2)) <= F_RMS_BF16


def test_batch_ensemble_bf16(P, W, OW):
    st = gen.served_stream(count=64)
    b = P.Batch(W, precision="bf16", max_atoms=st.n_atoms, max_mols=64)
    E, F = b.run(st.mol_start, st.species, st.coords)
    E_ref, F_ref = oracle.energy_forces_batch(st.mol_start, st.species, st.coords, OW)
    assert (np.abs(E - E_ref) / np.abs(E_ref)).max() <= E_REL_BF16
    assert np.sqrt(np.mean((F - F_ref) ** 2)) <= F_RMS_BF16


def test_server_ensemble_equals_batch(P, W):
    st = gen.served_stream(count=200)
    srv = P.Server(W, precision="bf16", max_batch_atoms=8192, max_batch_mols=64, streams=2)
    tickets = [srv.submit(st.molecule(m).species, st.molecule(m).coords) for m in range(st.count)]
    res = [srv.wait(t, 60) for t in tickets]
    srv.close()
    E = np.array([r[0] for r in res])
    F = np.concatenate([r[1] for r in res])
    b = P.Batch(W, precision="bf16", max_atoms=st.n_atoms, max_mols=st.count)
    Eb, Fb = b.run(st.mol_start, st.species, st.coords)
    np.testing.assert_array_equal(E, Eb)
    assert np.abs(F - Fb).max() <= 1e-6 * max(1.0, np.abs(Fb).max())
