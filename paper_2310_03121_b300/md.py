"""Velocity-Verlet test harness around the energy+force evaluation.

With random-init weights the potential has no repulsive core: after some
hundreds of femtoseconds atoms fall into attractive regions and pairs
collapse. A caller that runs dynamics therefore adds a short-range
repulsion, as a classical force field's non-bonded term would
(RepulsiveWall: a shifted r^-12 wall inside sigma with bounded curvature,
zero with its force at sigma and beyond). It is the caller's term, outside
the ML potential: its forces are written first and the library adds the ML
forces onto them (mlp_energy_forces_subset_device with accumulate, the
ML/MM path). Its pairs come from the library's allocation-free neighbor
search (mlp_neighbors_static). Without the wall the harness guards the
trajectory (closest pair below 0.5 A, or a neighbor-capacity error from the
library) and reports the steps completed.

Not part of the evaluation itself: a driver that integrates Newton's
equations with the library's forces, to check energy conservation (the
672-atom ligand-in-water system, 10,000 steps of 0.5 fs) and to time a
persistent system with a skin neighbor list (the 21,080-atom periodic box:
list radius 5.1 + 0.5 A, rebuilt every 10 steps or when an atom moved more
than half the skin; 1,000 steps of 0.5 fs).

Units: A, fs, amu, eV. Acceleration F/m in eV/(A amu) = 9.6485e-3 A/fs^2;
kinetic energy 0.5 m v^2 (amu A^2/fs^2) = 103.6427 eV per unit.
Positions and velocities stay on the device; the host reads the potential
and kinetic energy every `report_every` steps.

    python -m paper_2310_03121_b300.md --workload 1 --steps 10000 --precision fp32
"""
from __future__ import annotations

import argparse
import ctypes
import json
import time

import numpy as np

ACC = 9.648533212e-3        # (eV / A / amu) -> A / fs^2
KE = 103.6426965           # amu A^2 / fs^2 -> eV
KB = 8.617333262e-5         # eV / K
MASSES = np.array([1.008, 12.011, 14.007, 15.999, 32.06, 18.998, 35.45])


def _min_pair_distance_ok(coords_t, cell, limit, lib):
    """True if no pair is closer than `limit` (allocation-free neighbor search
    with a list of 4 entries per atom: the counts are the true counts even
    where they exceed the list, which is all this check reads). Raises
    MLPError when the search refuses the input (more atoms than its static
    array holds), so that the guard is never skipped silently."""
    import torch

    from ._lib import check

    n = coords_t.shape[0]
    counts = torch.zeros(n, dtype=torch.int32, device=coords_t.device)
    lst = torch.zeros((n, 4), dtype=torch.int32, device=coords_t.device)
    cl = None if cell is None else np.ascontiguousarray(cell, dtype=np.float64)
    rc = lib.mlp_neighbors_static(ctypes.c_void_p(coords_t.data_ptr()), n,
                                  None if cl is None else cl.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                  float(limit), ctypes.c_void_p(counts.data_ptr()), ctypes.c_void_p(lst.data_ptr()),
                                  4, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    check(rc, "mlp_neighbors_static (MD pair-distance guard)")
    return int(counts.max().item()) == 0


class RepulsiveWall:
    """The caller's short-range repulsion, summed over pairs closer than
    sigma (A): U(r) = eps [(sigma / r)^12 - 1 + 12 (r / sigma - 1)] (eV),
    zero with its derivative at sigma, and below r_soft continued linearly
    (constant force, so its curvature stays bounded and a 0.5 fs step stays
    stable when a hot atom hits it; the r^-12 wall alone made the 21,080-atom
    box blow up). The random-init network's energy keeps falling as atoms
    crowd (AEV entries grow with the number of close neighbors), so the wall
    must start before the collapse: sigma 1.0 A, eps 0.2 eV, r_soft 0.85 A
    held the 672-atom system for 10,000 steps and the box for 1,000. Pairs
    within sigma come from mlp_neighbors_static (up to `cap` per atom; more
    is reported, never silently dropped from the sum)."""

    def __init__(self, n, cell=None, sigma=1.0, eps=0.2, cap=16, r_soft=0.85):
        import torch

        self.n, self.sigma, self.eps, self.cap = n, float(sigma), float(eps), cap
        self.r_soft = float(r_soft)   # below it the wall continues linearly (bounded curvature)
        self.cell = None if cell is None else np.ascontiguousarray(cell, dtype=np.float64)
        dev = torch.device("cuda")
        self.counts = torch.zeros(n, dtype=torch.int32, device=dev)
        self.list = torch.zeros((n, cap), dtype=torch.int32, device=dev)
        self.slot = torch.arange(cap, device=dev, dtype=torch.int32)[None, :]
        self.L = None if cell is None else torch.as_tensor(self.cell, device=dev)
        self.max_seen = torch.zeros((), dtype=torch.int32, device=dev)   # largest count since creation

    def energy_forces(self, x, F):
        """Writes the wall's forces (float32) into F [n, 3]; returns its energy
        as a float64 device tensor [1]."""
        import torch

        from ._lib import check, load

        lib = load()
        cl = None if self.cell is None else self.cell.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        check(lib.mlp_neighbors_static(ctypes.c_void_p(x.data_ptr()), self.n, cl, self.sigma,
                                       ctypes.c_void_p(self.counts.data_ptr()), ctypes.c_void_p(self.list.data_ptr()),
                                       self.cap, ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)),
              "mlp_neighbors_static (repulsive wall)")
        torch.maximum(self.max_seen, self.counts.max(), out=self.max_seen)
        # every (atom, slot) of the list, unused slots masked: fixed shapes, so
        # the host never waits for the device here
        valid = self.slot < self.counts[:, None]
        j = torch.where(valid, self.list, 0).long()
        d = x[j] - x[:, None, :]
        if self.L is not None:
            d = d - self.L * torch.round(d / self.L)
        # the pair terms in FP32 (the forces are FP32; FP64 arithmetic is slow on this GPU)
        d = d.float()
        r = d.norm(dim=2).clamp_min(1e-3)
        rr = r.clamp_min(self.r_soft) if self.r_soft > 0.0 else r
        q2 = (self.sigma / rr) ** 2
        q6 = q2 * q2 * q2
        q12 = q6 * q6
        inside = valid & (r < self.sigma)
        u = torch.where(inside, self.eps * (q12 - 1.0 + 12.0 * (rr / self.sigma - 1.0)), torch.zeros_like(r))
        dudr = torch.where(inside, self.eps * 12.0 * (1.0 / self.sigma - q12 / rr), torch.zeros_like(r))
        if self.r_soft > 0.0:
            u = u + torch.where(inside & (r < rr), dudr * (r - rr), torch.zeros_like(r))
        # force on i from the pair (i, j): -dU/dr along -d/r, summed over i's slots
        F.copy_(((dudr / r)[:, :, None] * d).sum(1))
        return (0.5 * u.sum(dtype=torch.float64)).reshape(1)     # each pair is listed from both ends

    def overflow(self):
        """True if any call so far found more pairs of an atom than the list holds."""
        return int(self.max_seen.item()) > self.cap


def run(system, species, coords, cell=None, dt_fs=0.5, steps=1000, temperature=300.0, seed=0, report_every=10,
        guard_every=1000, min_pair=0.5, wall=None):
    """Integrates `steps` velocity-Verlet steps; returns a dict of results.
    wall: a RepulsiveWall (the caller's repulsion, added to the ML forces),
    or None (the ML potential alone, with the collapse guard)."""
    import torch

    from . import _lib

    dev = torch.device("cuda")
    m = torch.as_tensor(MASSES[np.asarray(species)], dtype=torch.float64, device=dev)[:, None]
    x = torch.as_tensor(np.asarray(coords, dtype=np.float64), device=dev).contiguous()
    rng = np.random.default_rng(seed)
    sigma = np.sqrt(KB * temperature / (MASSES[np.asarray(species)] * KE))[:, None]
    v0 = rng.normal(size=(len(species), 3)) * sigma
    mass = MASSES[np.asarray(species)][:, None]
    v0 -= (mass * v0).sum(0) / mass.sum()              # no centre-of-mass motion
    v = torch.as_tensor(v0, device=dev)
    E = torch.zeros(1, dtype=torch.float64, device=dev)
    F = torch.zeros((len(species), 3), dtype=torch.float32, device=dev)
    lib = _lib.load()
    index = torch.arange(len(species), dtype=torch.int32, device=dev)

    def forces():
        """Potential energy (device [1]) and total forces into F."""
        if wall is None:
            system.energy_forces_device(x, E, F)
            return E
        E_w = wall.energy_forces(x, F)
        system.energy_forces_subset_device(x, index, forces_full=F, energy=E, accumulate=True)
        return E + E_w

    Epot = forces()
    a = F.double() * (ACC / m)
    t_series, e_pot, e_kin = [], [], []
    aborted = None
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    from ._lib import MLPError

    step = 0
    for step in range(1, steps + 1):
        v.add_(a, alpha=0.5 * dt_fs)
        x.add_(v, alpha=dt_fs)
        try:
            Epot = forces()
        except MLPError as e:          # e.g. neighbor capacity exceeded after a collapse
            aborted = f"step {step}: {e}"
            step -= 1
            break
        a = F.double() * (ACC / m)
        v.add_(a, alpha=0.5 * dt_fs)
        if step % report_every == 0:
            ke = 0.5 * KE * float((m * v * v).sum().item())
            t_series.append(step * dt_fs)
            e_pot.append(float(Epot.item()))
            e_kin.append(ke)
            if wall is not None and wall.overflow():
                aborted = f"by step {step}: more than {wall.cap} pairs of an atom inside the wall"
                break
        if guard_every and step % guard_every == 0 and not _min_pair_distance_ok(x, cell, min_pair, lib):
            aborted = f"pair closer than {min_pair} A at step {step}"
            break
    torch.cuda.synchronize()
    wall_s = time.perf_counter() - t0
    if aborted is None and wall is not None and wall.overflow():
        aborted = f"by step {step}: more than {wall.cap} pairs of an atom inside the wall"
    try:
        system.sync()
    except MLPError as e:
        aborted = aborted or f"after step {step}: {e}"
    if not t_series:
        t_series, e_pot, e_kin = [0.0], [float("nan")], [float("nan")]
    n = len(species)
    tt = np.array(t_series)
    et = np.array(e_pot) + np.array(e_kin)
    slope = float(np.polyfit(tt, et, 1)[0]) if len(tt) > 2 else float("nan")   # eV / fs
    done = step if aborted is None else step
    return {"atoms": n, "steps": done, "dt_fs": dt_fs, "wall_s": wall_s, "atom_steps_per_s": n * done / wall_s,
            "drift_eV_per_atom_per_ps": slope * 1000.0 / n,
            "etot_rms_fluct_eV_per_atom": float(np.std(et - np.polyval(np.polyfit(tt, et, 1), tt)) / n)
            if len(tt) > 2 else None,
            "etot_first": float(et[0]) if len(et) else None, "etot_last": float(et[-1]) if len(et) else None,
            "temperature_K_last": float(2 * e_kin[-1] / (3 * n * KB)) if e_kin else None, "aborted": aborted,
            "repulsive_wall": None if wall is None else {"sigma_A": wall.sigma, "eps_eV": wall.eps,
                                                         "r_soft_A": wall.r_soft}}


def main():
    import gen

    from . import System, Weights

    ap = argparse.ArgumentParser()
    ap.add_argument("--workload", type=int, default=1, choices=[1, 4])
    ap.add_argument("--steps", type=int, default=None)
    ap.add_argument("--dt", type=float, default=0.5)
    ap.add_argument("--precision", default=None)
    args = ap.parse_args()
    c = gen.make_config(args.workload)
    W = Weights(gen.make_weights())
    if args.workload == 1:
        steps = args.steps or 10000
        prec = args.precision or "fp32"
        s = System(W, c.species, c.coords, c.cell, precision=prec)
    else:
        steps = args.steps or 1000
        prec = args.precision or "bf16"
        s = System(W, c.species, c.coords, c.cell, precision=prec, skin=0.5)
    res = run(s, c.species, c.coords, c.cell, dt_fs=args.dt, steps=steps, guard_every=0,
              wall=RepulsiveWall(c.n, c.cell))
    res.update({"workload": c.name, "precision": prec})
    print(json.dumps(res))


if __name__ == "__main__":
    main()
