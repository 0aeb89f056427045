"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Tolerances (FP32 network path): energy relative error <= 1e-6, max force
error <= 1e-4 eV/A; neighbor lists equal as sets outside the rounding band
|r^2 - rc^2| < 1e-5 rc^2. AEV rows: FP32 arithmetic on O(1) values with
transcendental functions accurate to a few ulp, summed over <= 160
neighbors / ~2000 triples -> |dG| <= 2e-5 * max(1, |G|) per element.
"""
import numpy as np
import pytest
import torch

import gen
import oracle

pytestmark = pytest.mark.gpu

E_REL_FP32 = 1e-6
F_MAX_FP32 = 1e-4


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


def _small_periodic(n=300, seed=21):
    return gen.random_molecule(n, seed=seed, density=0.1, periodic=True)


CASES = {
    "config0": lambda: gen.make_config(0),
    "config1": lambda: gen.make_config(1),
    "config2": lambda: gen.make_config(2),
    "config4": lambda: gen.make_config(4),
    "box300": lambda: _small_periodic(300),     # 4 x 4 x 4 cells
    "box173": lambda: _small_periodic(173, 5),  # L = 12 A: two cells per axis
    # open systems of more than 1,024 atoms take the cell list; smaller open
    # systems (config0, config1) the all-pairs search of one molecule
    "open1500": lambda: gen.random_molecule(1500, seed=31, density=0.1),
}


# ------------------------------------------------------------------ neighbors
@pytest.mark.parametrize("case", ["config0", "config1", "config2", "config4", "box300", "box173", "open1500"])
def test_neighbor_sets(P, W, case):
    c = CASES[case]()
    s = P.System(W, c.species, c.coords, c.cell, precision="fp32")
    s.energy_forces()
    counts, lst = s.debug_neighbors()
    assert counts.max() <= lst.shape[1]
    got = set()
    for i in range(c.n):
        for j in lst[i, :counts[i]]:
            got.add((i, int(j)))
    assert len(got) == counts.sum(), "duplicate neighbors"
    pairs, band = oracle.neighbors(c.coords, c.cell, 5.1)
    must = {(int(i), int(j)) for (i, j), b in zip(pairs, band) if b == 0}
    may = {(int(i), int(j)) for (i, j), b in zip(pairs, band) if b != 0}
    assert must <= got
    assert got <= must | may


# ------------------------------------------------------------------ AEV
@pytest.mark.parametrize("case", ["config0", "config1", "box300", "box173"])
def test_aev_rows(P, W, case):
    c = CASES[case]()
    s = P.System(W, c.species, c.coords, c.cell, precision="fp32")
    s.energy_forces()
    G = s.debug_aev()
    R = oracle.aev(c.species, c.coords, c.cell)
    err = np.abs(G - R)
    tol = 2e-5 * np.maximum(1.0, np.abs(R))
    assert (err <= tol).all(), (err.max(), np.unravel_index(err.argmax(), err.shape))
    # every structurally zero column stays exactly zero
    assert (G[R == 0.0] == 0.0).all()


def test_aev_rows_config4_sample(P, W):
    c = CASES["config4"]()
    s = P.System(W, c.species, c.coords, c.cell, precision="fp32")
    s.energy_forces()
    G = s.debug_aev()
    idx = np.random.default_rng(0).choice(c.n, 96, replace=False)
    idx = np.concatenate([idx, np.arange(80)])   # the solute atoms
    R = oracle.aev_subset(c.species, c.coords, c.cell, idx)
    assert (np.abs(G[idx] - R) <= 2e-5 * np.maximum(1.0, np.abs(R))).all()


# ------------------------------------------------------------------ network
@pytest.mark.parametrize("n", [1, 127, 129, 400])
def test_network_fp32_ragged_tiles(P, W, OW, n):
    rng = np.random.default_rng(n)
    c = gen.make_config(1)
    G_all = oracle.aev(c.species, c.coords)
    pick = rng.choice(c.n, size=n, replace=n > c.n)
    sp = c.species[pick].copy()
    sp[: min(n, 7)] = np.arange(min(n, 7))   # every element present when n >= 7
    G = G_all[pick]
    e, g = P.debug_network(W, "fp32", sp, G)
    for q in range(n):
        er, gr = oracle.atom_energy(int(sp[q]), G[q].astype(np.float32).astype(np.float64), OW, grad=True)
        assert abs(e[q] - er) <= 1e-5 * max(1.0, abs(er))
        assert np.abs(g[q] - gr).max() <= 1e-5 * max(1.0, np.abs(gr).max())


# ------------------------------------------------------------------ whole path, FP32
def _check_fp32(E, F, E_ref, F_ref):
    assert abs(E - E_ref) <= E_REL_FP32 * abs(E_ref), (E, E_ref, abs(E - E_ref) / abs(E_ref))
    assert np.abs(F - F_ref).max() <= F_MAX_FP32, np.abs(F - F_ref).max()


@pytest.mark.parametrize("case", ["config0", "config1", "box300", "box173", "open1500"])
def test_energy_forces_fp32(P, W, OW, case):
    c = CASES[case]()
    E_ref, F_ref, e_ref = oracle.energy_forces(c.species, c.coords, c.cell, OW, per_atom=True)
    s = P.System(W, c.species, c.coords, c.cell, precision="fp32")
    E, F = s.energy_forces()
    _check_fp32(E, F, E_ref, F_ref)
    e, _ = s.debug_atom_energies(grad=False)
    assert np.abs(e - e_ref).max() <= 1e-5 * max(1.0, np.abs(e_ref).max())


@pytest.mark.parametrize("case", ["config2", "config4"])
def test_energy_forces_fp32_full_size(P, W, OW, case):
    """Full-size boxes: every per-atom energy (oracle threaded over atoms),
    and forces on a sample of atoms (oracle restricted to their neighborhoods)."""
    c = CASES[case]()
    s = P.System(W, c.species, c.coords, c.cell, precision="fp32")
    E, F = s.energy_forces()
    e_ref = oracle.atom_energies(c.species, c.coords, c.cell, OW)
    E_ref = float(np.sum(e_ref))
    assert abs(E - E_ref) <= E_REL_FP32 * abs(E_ref), (E, E_ref)
    idx = np.random.default_rng(1).choice(c.n, 48, replace=False)
    F_ref = oracle.forces_subset(c.species, c.coords, c.cell, OW, idx)
    assert np.abs(F[idx] - F_ref).max() <= F_MAX_FP32
    # zero net force holds at any size only for open systems; periodic: sum ~ 0 too
    assert np.abs(F.astype(np.float64).sum(0)).max() <= 1e-3 * np.abs(F).sum() / c.n


def test_repeat_is_deterministic_energy(P, W):
    c = CASES["config1"]()
    s = P.System(W, c.species, c.coords, None, precision="fp32")
    E1, F1 = s.energy_forces()
    E2, F2 = s.energy_forces()
    assert E1 == E2
    assert np.abs(F1 - F2).max() <= 1e-6


# ------------------------------------------------------------------ persistent neighbor list (skin)
def test_skin_list_reuse_and_guard(P, W, OW):
    c = _small_periodic(400, 33)
    s = P.System(W, c.species, c.coords, c.cell, precision="fp32", skin=0.5)
    E0, F0 = s.energy_forces()
    rng = np.random.default_rng(2)
    x1 = c.coords + rng.normal(0, 0.05, size=c.coords.shape)   # below skin/2: list reused
    E1, F1 = s.energy_forces(x1)
    E1r, F1r = oracle.energy_forces(c.species, x1, c.cell, OW)
    _check_fp32(E1, F1, E1r, F1r)
    x2 = x1.copy()
    x2[5] += np.array([0.6, 0.0, 0.0])                           # beyond skin/2: guard rebuilds
    E2, F2 = s.energy_forces(x2)
    E2r, F2r = oracle.energy_forces(c.species, x2, c.cell, OW)
    _check_fp32(E2, F2, E2r, F2r)


# ------------------------------------------------------------------ batches of molecules
def test_batch_fp32_matches_oracle(P, W, OW):
    st = gen.served_stream(count=300)
    b = P.Batch(W, precision="fp32", max_atoms=st.n_atoms, max_mols=300)
    E, F = b.run(st.mol_start, st.species, st.coords)
    E_ref, F_ref = oracle.energy_forces_batch(st.mol_start, st.species, st.coords, OW)
    rel = np.abs(E - E_ref) / np.abs(E_ref)
    assert rel.max() <= E_REL_FP32, rel.max()
    assert np.abs(F - F_ref).max() <= F_MAX_FP32


def test_batch_alone_equals_in_mix(P, W):
    st = gen.served_stream(count=200)
    b = P.Batch(W, precision="fp32", max_atoms=st.n_atoms, max_mols=200)
    E, F = b.run(st.mol_start, st.species, st.coords)
    for m in (0, 57, 199):
        a, z = st.mol_start[m], st.mol_start[m + 1]
        E1, F1 = b.run(np.array([0, z - a]), st.species[a:z], st.coords[a:z])
        assert E1[0] == E[m]          # per-row network + fixed-order FP64 sum: bitwise
        assert np.abs(F1 - F[a:z]).max() <= 1e-6 * max(1.0, np.abs(F1).max())


# ------------------------------------------------------------------ bad inputs
def test_invalid_inputs(P, W):
    from paper_2310_03121_b300 import _lib

    c = gen.make_config(0)
    with pytest.raises(P.MLPError) as ei:
        P.System(W, np.full(c.n, 9, np.int8), c.coords, None)
    assert ei.value.code == _lib.MLP_EINVAL
    x = c.coords.copy()
    x[3, 1] = np.nan
    with pytest.raises(P.MLPError):
        P.System(W, c.species, x, None)
    with pytest.raises(P.MLPError):
        P.System(W, c.species, c.coords, np.array([8.0, 8.0, 8.0]))   # box < 2 rc
    s = P.System(W, c.species, c.coords, None)
    with pytest.raises(P.MLPError):
        s.energy_forces(x)


def test_allocation_failure_is_reported(P, W):
    from paper_2310_03121_b300 import _lib

    c = gen.make_config(0)
    P.fail_next_allocation(0)
    with pytest.raises(P.MLPError) as ei:
        P.System(W, c.species, c.coords, None)
    assert ei.value.code == _lib.MLP_ENOMEM
    s = P.System(W, c.species, c.coords, None)   # the next one works
    s.energy_forces()


# ------------------------------------------------------------------ BF16 tensor-core network
E_REL_BF16 = 1e-3
F_RMS_BF16 = 2e-2


def _bf16(x):
    return torch.as_tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64)


def _split(x):
    """FP32 value -> (BF16 hi, BF16 rounding of the remainder), as float64."""
    x32 = torch.as_tensor(x, dtype=torch.float64).float()
    hi = x32.to(torch.bfloat16)
    lo = (x32 - hi.float()).to(torch.bfloat16)
    return hi.double(), lo.double()


def _emulate_bf16_network(wts, sp, G, split=True, round_out=True):
    """The tensor-core kernel's arithmetic in float64. Forward GEMMs: BF16
    operands (split = False) or A_hi B_hi + A_lo B_hi + A_hi B_lo from hi/lo
    BF16 pairs (split = True); backward: BF16 operands; celu'(z) of the
    hidden layers recovered from the stored BF16 activation; dE/dG rounded
    to BF16 on output (one net) or left unrounded (round_out = False: an
    ensemble member, whose dE/dG leaves the kernel in FP32)."""
    e = np.zeros(len(sp))
    g = np.zeros((len(sp), 1008))
    cel = lambda z: torch.where(z > 0, z, 0.1 * (torch.exp(z / 0.1) - 1))
    dcel = lambda h: torch.where(h > 0, torch.ones_like(h), h / 0.1 + 1)

    def fwd(a, W):
        ah, al = _split(a)
        wh, wl = _split(W)
        return ah @ wh.T + al @ wh.T + ah @ wl.T if split else ah @ wh.T

    for s in range(7):
        idx = np.nonzero(sp == s)[0]
        if idx.size == 0:
            continue
        W1, W2, W3 = (torch.as_tensor(wts[k][s], dtype=torch.float32).double() for k in ("W1", "W2", "W3"))
        b1, b2, b3, w4 = (torch.as_tensor(wts[k][s], dtype=torch.float32).double() for k in ("b1", "b2", "b3", "W4"))
        b4 = float(np.float32(wts["b4"][s]))
        A = torch.as_tensor(G[idx], dtype=torch.float32).double()
        h1 = cel(fwd(A, W1) + b1).float().double()
        h2 = cel(fwd(h1, W2) + b2).float().double()
        z3 = fwd(h2, W3) + b3
        e[idx] = (cel(z3) @ w4 + b4).numpy()
        h1b, h2b = _bf16(h1), _bf16(h2)
        g3 = _bf16(w4 * torch.where(z3 > 0, torch.ones_like(z3), torch.exp(z3 / 0.1)))
        g2 = _bf16((g3 @ _bf16(W3)) * dcel(h2b))
        g1 = _bf16((g2 @ _bf16(W2)) * dcel(h1b))
        gg = g1 @ _bf16(W1)
        g[idx] = (_bf16(gg) if round_out else gg).numpy()   # one net: dE/dG leaves the kernel as BF16
    return e, g


@pytest.mark.parametrize("n", [1, 129, 400])
@pytest.mark.parametrize("mode", ["bf16", "bf16_1pass"])
def test_network_bf16_matches_emulation(P, W, wts, n, mode):
    rng = np.random.default_rng(100 + n)
    c = gen.make_config(1)
    G_all = oracle.aev(c.species, c.coords)
    pick = rng.choice(c.n, size=n, replace=n > c.n)
    sp = c.species[pick].copy()
    sp[: min(n, 7)] = np.arange(min(n, 7))
    G = G_all[pick].astype(np.float32)
    e, g = P.debug_network(W, mode, sp, G)
    e_ref, g_ref = _emulate_bf16_network(wts, sp, G, split=(mode == "bf16"))
    # remaining differences: FP32 accumulation order, and BF16 re-rounding of
    # activations that sit on a rounding boundary
    tol_e = 2e-5 if mode == "bf16" else 2e-3
    assert np.abs(e - e_ref).max() <= tol_e * max(1.0, np.abs(e_ref).max()), np.abs(e - e_ref).max()
    assert np.abs(g - g_ref).max() <= 2e-2 * np.abs(g_ref).max(), (np.abs(g - g_ref).max(), np.abs(g_ref).max())
    assert np.sqrt(np.mean((g - g_ref) ** 2)) <= 2e-3 * np.sqrt(np.mean(g_ref ** 2))


def _check_bf16(E, F, E_ref, F_ref):
    assert abs(E - E_ref) <= E_REL_BF16 * abs(E_ref), (E, E_ref, abs(E - E_ref) / abs(E_ref))
    rms = float(np.sqrt(np.mean((F - F_ref) ** 2)))
    assert rms <= F_RMS_BF16, rms


@pytest.mark.parametrize("case", ["config0", "config1", "box300"])
def test_energy_forces_bf16(P, W, OW, case):
    c = CASES[case]()
    E_ref, F_ref = oracle.energy_forces(c.species, c.coords, c.cell, OW)
    s = P.System(W, c.species, c.coords, c.cell, precision="bf16")
    E, F = s.energy_forces()
    _check_bf16(E, F, E_ref, F_ref)


@pytest.mark.parametrize("case", ["config2", "config4"])
def test_energy_forces_bf16_full_size(P, W, OW, case):
    c = CASES[case]()
    s = P.System(W, c.species, c.coords, c.cell, precision="bf16")
    E, F = s.energy_forces()
    E_ref = float(np.sum(oracle.atom_energies(c.species, c.coords, c.cell, OW)))
    idx = np.random.default_rng(3).choice(c.n, 48, replace=False)
    F_ref = oracle.forces_subset(c.species, c.coords, c.cell, OW, idx)
    _check_bf16(E, F[idx], E_ref, F_ref)


def test_batch_bf16_matches_oracle(P, W, OW):
    st = gen.served_stream(count=300)
    b = P.Batch(W, precision="bf16", max_atoms=st.n_atoms, max_mols=300)
    E, F = b.run(st.mol_start, st.species, st.coords)
    E_ref, F_ref = oracle.energy_forces_batch(st.mol_start, st.species, st.coords, OW)
    rel = np.abs(E - E_ref) / np.abs(E_ref)
    assert rel.max() <= E_REL_BF16, rel.max()
    assert np.sqrt(np.mean((F - F_ref) ** 2)) <= F_RMS_BF16
