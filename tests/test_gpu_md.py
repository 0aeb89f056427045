"""Velocity-Verlet harness.

* Energy conservation of the ML potential alone on the 672-atom open system
  (FP32 path, 0.1 fs, 100 steps: with random-init weights the potential has
  no repulsive core and the first pairs come closer than 0.5 A after ~25 fs,
  so this check stays inside that window).
* The caller's repulsive wall (md.RepulsiveWall, pairs from the
  allocation-free neighbor search): its forces equal central differences of
  its energy, open and periodic.
* The ligand-in-water system with the wall for 10,000 steps of 0.5 fs (5 ps,
  FP32 path): no collapse, total-energy drift below 2e-3 eV per atom per ps
  (the random-init potential heats the system to ~1,200 K, kT ~ 0.1 eV: at
  most 10 meV per atom over the run; measured 2.2e-4).
* The persistent skin list on the 21,080-atom periodic box (list radius
  5.6 A, rebuilt every 10 steps or by the displacement guard): after a short
  random walk the persistent system's energy and forces (FP32 network) equal
  a fresh evaluation at the same coordinates up to FP32 summation order;
  then 1,000 velocity-Verlet steps of 0.5 fs with the wall on the BF16 path
  complete with finite energies (the system heats to ~2,700 K).
"""
import numpy as np
import pytest
import torch

import gen

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def P():
    if not torch.cuda.is_available():
        pytest.fail("GPU tests need a CUDA device")
    import paper_2310_03121_b300 as P

    return P


def test_energy_conservation_fp32(P):
    from paper_2310_03121_b300 import md

    c = gen.make_config(1)
    W = P.Weights(gen.make_weights())
    s = P.System(W, c.species, c.coords, None, precision="fp32")
    res = md.run(s, c.species, c.coords, None, dt_fs=0.1, steps=100, report_every=5, guard_every=0)
    assert res["aborted"] is None
    # total energy drift well below the kinetic energy scale (kT ~ 0.026 eV per atom)
    assert abs(res["drift_eV_per_atom_per_ps"]) < 1e-3, res
    assert res["etot_rms_fluct_eV_per_atom"] < 1e-4, res


def _wall_energy64(x, cell, sigma, eps, r_soft):
    """The wall's energy in float64 by brute force over all pairs (the form the
    harness documents), for central differences."""
    d = x[None, :, :] - x[:, None, :]
    if cell is not None:
        d -= cell * np.round(d / cell)
    r = np.sqrt((d * d).sum(-1))
    iu = np.triu_indices(len(x), 1)
    r = r[iu]
    r = r[r < sigma]
    rr = np.maximum(r, r_soft)
    q12 = (sigma / rr) ** 12
    u = eps * (q12 - 1.0 + 12.0 * (rr / sigma - 1.0))
    dudr = eps * 12.0 * (1.0 / sigma - q12 / rr)
    u += np.where(r < rr, dudr * (r - rr), 0.0)
    return float(u.sum())


@pytest.mark.parametrize("periodic", [False, True])
def test_repulsive_wall_forces_are_its_gradient(P, periodic):
    """The harness's wall (FP32 pair terms over the allocation-free search's
    pairs): its energy equals the brute-force float64 sum over all pairs, and
    its forces equal central differences (h = 1e-5 A) of that sum."""
    from paper_2310_03121_b300 import md

    rng = np.random.default_rng(3)
    n = 60
    cell = np.array([6.0, 6.0, 6.0]) if periodic else None
    pts = []                                    # dense, pairs no closer than 0.6 A: many inside the wall
    while len(pts) < n:
        p = rng.uniform(0, 6.0, size=3)
        d = np.array(pts) - p if pts else np.zeros((0, 3))
        if periodic:
            d -= 6.0 * np.round(d / 6.0)
        if not pts or np.sqrt((d * d).sum(1)).min() > 0.6:
            pts.append(p)
    x0 = np.array(pts)
    w = md.RepulsiveWall(n, cell, cap=32)
    x = torch.as_tensor(x0, device="cuda").contiguous()
    F = torch.zeros((n, 3), dtype=torch.float32, device="cuda")
    E = float(w.energy_forces(x, F).item())
    assert not w.overflow()
    E64 = _wall_energy64(x0, cell, w.sigma, w.eps, w.r_soft)
    assert E64 > 0 and abs(E - E64) <= 1e-5 * E64, (E, E64)
    F = F.cpu().numpy().astype(np.float64)
    h = 1e-5
    for i in range(n):
        for a in range(3):
            xp = x0.copy()
            xp[i, a] += h
            Ep = _wall_energy64(xp, cell, w.sigma, w.eps, w.r_soft)
            xp[i, a] -= 2 * h
            Em = _wall_energy64(xp, cell, w.sigma, w.eps, w.r_soft)
            assert abs(F[i, a] + (Ep - Em) / (2 * h)) <= 1e-4 * max(1.0, abs(F[i, a])), (i, a)


def test_ligand_in_water_10000_steps_with_wall(P):
    from paper_2310_03121_b300 import md

    c = gen.make_config(1)
    W = P.Weights(gen.make_weights())
    s = P.System(W, c.species, c.coords, None, precision="fp32")
    res = md.run(s, c.species, c.coords, None, dt_fs=0.5, steps=10000, report_every=20, guard_every=0,
                 wall=md.RepulsiveWall(c.n))
    print(res)
    assert res["aborted"] is None and res["steps"] == 10000
    assert abs(res["drift_eV_per_atom_per_ps"]) < 2e-3, res


def test_skin_list_trajectory_matches_fresh(P):
    from paper_2310_03121_b300 import md

    c = gen.make_config(4)
    W = P.Weights(gen.make_weights())
    # FP32 network: the comparison isolates the list logic from BF16 rounding
    s = P.System(W, c.species, c.coords, c.cell, precision="fp32", skin=0.5)
    x = torch.as_tensor(c.coords, device="cuda").contiguous()
    E = torch.zeros(1, dtype=torch.float64, device="cuda")
    F = torch.zeros((c.n, 3), dtype=torch.float32, device="cuda")
    rng = np.random.default_rng(0)
    for step in range(25):   # random walk of 0.01 A per step: several rebuilds by the 10-step policy
        x += torch.as_tensor(rng.normal(0, 0.01, size=c.coords.shape), device="cuda")
        s.energy_forces_device(x, E, F)
    s.sync()
    fresh = P.System(W, c.species, x.cpu().numpy(), c.cell, precision="fp32")
    E2, F2 = fresh.energy_forces()
    assert abs(E.item() - E2) <= 1e-7 * abs(E2)
    assert np.abs(F.cpu().numpy() - F2).max() <= 1e-5
    sb = P.System(W, c.species, c.coords, c.cell, precision="bf16", skin=0.5)
    res = md.run(sb, c.species, c.coords, c.cell, dt_fs=0.5, steps=1000, report_every=50, guard_every=0,
                 wall=md.RepulsiveWall(c.n, c.cell))
    print(res)
    assert res["aborted"] is None and res["steps"] == 1000 and res["atom_steps_per_s"] > 0
    assert np.isfinite(res["etot_last"]) and abs(res["drift_eV_per_atom_per_ps"]) < 0.1, res
