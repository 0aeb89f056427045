"""LF-Middle Langevin dynamics (section "New Integrators"; Table 3 runs the
ML simulations with a Langevin integrator at 2 fs) through mlp_langevin_*,
against the oracle's integrator.

The update itself is FP64 on both sides with the same counter-based normal
deviates: given the GPU's own forces, one step agrees with the oracle's step
to 1e-12. Whole trajectories differ only through the force errors of the
path (FP32 bar: 1e-4 eV/A), which grow quadratically over a few steps.
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


def _start(c, seed=0, T=300.0):
    """Maxwell-Boltzmann velocities (A / fs) at T."""
    m = np.array([1.008, 12.011, 14.007, 15.999, 32.06, 18.998, 35.45])[c.species][:, None]
    rng = np.random.default_rng(seed)
    return rng.normal(size=(c.n, 3)) * np.sqrt(8.617333262e-5 * T / (m * 103.6426965))


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64)).cuda()


def test_normals_match_oracle(P):
    for seed, step in ((0, 0), (12345, 987654321), (2**63 + 7, 3)):
        g = P.debug_langevin_normals(seed, step, 777)
        r = oracle.langevin_normals(seed, step, 777)
        assert np.abs(g - r).max() <= 1e-12, np.abs(g - r).max()


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_one_step_equals_oracle_update(P, W, precision):
    """One step from (x, v) with the GPU's own forces at x: the update
    matches the oracle's LF-Middle step to FP64 rounding."""
    c = gen.make_config(1)
    s = P.System(W, c.species, c.coords, c.cell, precision=precision)
    v0 = _start(c)
    x, v = _dev(c.coords), _dev(v0)
    _, F = s.energy_forces_device(x)
    F = F.cpu().numpy().astype(np.float64)
    L = P.Langevin(s, dt_fs=2.0, friction_per_ps=1.0, temperature_K=300.0, seed=77, use_graph=False)
    L.run(x, v, 5, 1)
    xr, vr = oracle.lfmiddle_step(c.species, c.coords, v0, F, 2.0, 1.0, 300.0, 77, 5)
    assert np.abs(x.cpu().numpy() - xr).max() <= 1e-12 * np.abs(xr).max()
    assert np.abs(v.cpu().numpy() - vr).max() <= 1e-12 * np.abs(vr).max()


def test_trajectory_follows_oracle_fp32(P, W, wts):
    """24-atom workload, FP32 path, 2 fs, 20 steps: positions, velocities and
    per-step potential energies against the oracle's trajectory."""
    c = gen.make_config(0)
    s = P.System(W, c.species, c.coords, c.cell, precision="fp32")
    v0 = _start(c, 1)
    x, v = _dev(c.coords), _dev(v0)
    L = P.Langevin(s, dt_fs=2.0, friction_per_ps=1.0, temperature_K=300.0, seed=5)
    E = L.run(x, v, 0, 20).cpu().numpy()
    xr, vr, Er = oracle.langevin_run(c.species, c.coords, v0, c.cell, oracle.Weights(wts), 2.0, 1.0, 300.0, 5, 0, 20)
    # force errors <= 1e-4 eV/A move an H atom by <= dt^2 (F/m units) * n^2 / 2 ~ 8e-4 A in 20 steps
    assert np.abs(x.cpu().numpy() - xr).max() <= 1e-3
    assert np.abs(v.cpu().numpy() - vr).max() <= 1e-4
    assert np.abs(E - Er).max() <= 1e-4 * np.abs(Er).max()
    assert abs(E[0] - Er[0]) <= 1e-6 * abs(Er[0])


def test_graph_replay_equals_plain_launches_and_runs_concatenate(P, W):
    """The captured-graph step is the same computation, and two runs of 10
    steps equal one run of 20 (equal up to the rounding order of the FP64
    force atomics, which can flip the last bit of an FP32 force)."""
    c = gen.make_config(1)
    v0 = _start(c, 2)
    out = []
    for use_graph, split in ((False, False), (True, False), (True, True)):
        s = P.System(W, c.species, c.coords, c.cell, precision="bf16")
        L = P.Langevin(s, dt_fs=2.0, friction_per_ps=1.0, temperature_K=300.0, seed=9, use_graph=use_graph)
        x, v = _dev(c.coords), _dev(v0)
        if split:
            E1 = L.run(x, v, 0, 10)
            E2 = L.run(x, v, 10, 10)
            E = torch.cat([E1, E2])
        else:
            E = L.run(x, v, 0, 20)
        out.append((x.cpu().numpy(), v.cpu().numpy(), E.cpu().numpy()))
    for o in out[1:]:
        for a, b in zip(o, out[0]):
            assert np.abs(a - b).max() <= 1e-9 * max(1.0, np.abs(b).max())


def test_skin_list_periodic_box(P, W):
    """21,080-atom periodic box with a 0.5 A skin (the list is rebuilt on the
    device when an atom has moved more than half the skin): after 30 steps the
    integrator's potential energy equals a fresh evaluation (no skin, new
    list) at the same positions."""
    c = gen.make_config(4)
    s = P.System(W, c.species, c.coords, c.cell, precision="bf16", skin=0.5)
    L = P.Langevin(s, dt_fs=2.0, friction_per_ps=1.0, temperature_K=300.0, seed=3)
    x, v = _dev(c.coords), _dev(_start(c, 3))
    L.run(x, v, 0, 30, energies=False)
    x30 = x.clone()
    E = L.run(x, v, 30, 1)                          # E[0]: energy at x30
    assert torch.isfinite(x).all() and torch.isfinite(v).all()
    fresh = P.System(W, c.species, None, c.cell, precision="bf16")
    Ef, _ = fresh.energy_forces_device(x30)
    e0, ef = float(E[0].item()), float(Ef.item())
    assert abs(e0 - ef) <= 1e-5 * abs(ef), (e0, ef)


def test_bad_parameters(P, W):
    c = gen.make_config(0)
    s = P.System(W, c.species, c.coords, None, precision="fp32")
    for kw in ({"dt_fs": 0.0}, {"friction_per_ps": -1.0}, {"temperature_K": -5.0}):
        with pytest.raises(P.MLPError):
            P.Langevin(s, **kw)


def test_checkpoint_and_resume(P, W):
    """A trajectory is a function of (x, v, seed, step): saving x, v and the
    step to the host and resuming in a fresh system and integrator gives the
    run that never stopped."""
    c = gen.make_config(1)
    v0 = _start(c, 4)
    s = P.System(W, c.species, c.coords, c.cell, precision="bf16")
    L = P.Langevin(s, dt_fs=2.0, friction_per_ps=1.0, temperature_K=300.0, seed=21)
    x, v = _dev(c.coords), _dev(v0)
    L.run(x, v, 0, 24, energies=False)
    xa, va = x.cpu().numpy(), v.cpu().numpy()
    s1 = P.System(W, c.species, c.coords, c.cell, precision="bf16")
    L1 = P.Langevin(s1, dt_fs=2.0, friction_per_ps=1.0, temperature_K=300.0, seed=21)
    x1, v1 = _dev(c.coords), _dev(v0)
    L1.run(x1, v1, 0, 12, energies=False)
    ckpt = (x1.cpu().numpy(), v1.cpu().numpy(), 12)       # host checkpoint
    L1.close()
    s2 = P.System(W, c.species, ckpt[0], c.cell, precision="bf16")
    L2 = P.Langevin(s2, dt_fs=2.0, friction_per_ps=1.0, temperature_K=300.0, seed=21)
    x2, v2 = _dev(ckpt[0]), _dev(ckpt[1])
    L2.run(x2, v2, ckpt[2], 12, energies=False)
    assert np.abs(x2.cpu().numpy() - xa).max() <= 1e-9 * max(1.0, np.abs(xa).max())
    assert np.abs(v2.cpu().numpy() - va).max() <= 1e-9 * max(1.0, np.abs(va).max())
