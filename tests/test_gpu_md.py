"""Velocity-Verlet harness: energy conservation on the 672-atom open system
(FP32 path, 0.1 fs, 100 steps: with random-init weights the potential has no
repulsive core and the first pairs come closer than 0.5 A after ~25 fs, so
the check stays inside that window) and the persistent skin list on the
21,080-atom periodic box (list radius 5.6 A, rebuilt every 10 steps or by
the displacement guard): after a short random walk the persistent system's
energy and forces (FP32 network) equal a fresh evaluation at the same
coordinates up to FP32 summation order (the skin list holds the neighbors in
another order); a short BF16 trajectory then runs on the skin list.
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
    sb = P.System(W, c.species, x.cpu().numpy(), c.cell, precision="bf16", skin=0.5)
    res = md.run(sb, c.species, x.cpu().numpy(), c.cell, dt_fs=0.5, steps=50, report_every=10, guard_every=50)
    assert res["steps"] > 0 and res["atom_steps_per_s"] > 0
