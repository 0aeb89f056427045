"""Seeded synthetic inputs for the ANI-2x-shaped energy+force workloads.

This module is shared by the FP64 oracle tests, the GPU parity tests and the
benchmark. It holds no arithmetic of the potential itself: it only draws
geometries (species, coordinates, box) and random-init network weights.

Workloads (stand-ins for the paper's ligand-in-solvent and solvated-protein
systems of its Results section; no dataset is used):

  0  24 atoms, C6 N2 O2 H14, uniform in a 6 A cube, min pair 0.95 A, open.
  1  72-atom drug-like blob + 200 waters (672 atoms), open boundary.
  2  2,187 waters (6,561 atoms) in a 40.4 A periodic cube, min O-O 2.5 A.
  3  20,000 molecules, N log-uniform in [8, 256], each uniform in a cube of
     side 6 (N/24)^(1/3) A (workload 0's density), open boundary.
  4  7,000 waters + 80-atom solute (21,080 atoms), 59.5 A periodic cube.

Species codes: H=0, C=1, N=2, O=3, S=4, F=5, Cl=6 (the seven ANI-2x
elements, paper section "OpenMM-ML").
"""
from __future__ import annotations

import functools
import math

import numpy as np

SPECIES = ("H", "C", "N", "O", "S", "F", "Cl")
NSPECIES = 7
# ANI-2x-shaped per-element network widths: 1008-256-192-160-1.
LAYER_DIMS = (1008, 256, 192, 160, 1)
# Drug-like composition (C, H, N, O, S, F, Cl) -> our species order.
LIGAND_FREQ = np.array([0.45, 0.35, 0.07, 0.08, 0.02, 0.02, 0.01])  # H C N O S F Cl
MASSES = np.array([1.008, 12.011, 14.007, 15.999, 32.06, 18.998, 35.45])

WATER_OH = 0.96
WATER_HOH_DEG = 104.5
MIN_PAIR = 0.95


class Config:
    """One molecule or periodic box: species[int8 N], coords[f64 N x 3] in A,
    cell[f64 3] box lengths in A (orthorhombic) or None for open boundary."""

    def __init__(self, species, coords, cell=None, name=""):
        self.species = np.ascontiguousarray(species, dtype=np.int8)
        self.coords = np.ascontiguousarray(coords, dtype=np.float64)
        self.cell = None if cell is None else np.ascontiguousarray(cell, dtype=np.float64)
        self.name = name

    @property
    def n(self):
        return int(self.species.shape[0])

    def __repr__(self):
        return f"Config({self.name!r}, n={self.n}, cell={None if self.cell is None else self.cell.tolist()})"


# ----------------------------------------------------------------------------- helpers
def _min_image(d, cell):
    if cell is None:
        return d
    return d - cell * np.rint(d / cell)


def _random_rotation(rng):
    # Uniform random rotation from a random unit quaternion.
    q = rng.normal(size=4)
    q /= np.linalg.norm(q)
    a, b, c, d = q
    return np.array([
        [a * a + b * b - c * c - d * d, 2 * (b * c - a * d), 2 * (b * d + a * c)],
        [2 * (b * c + a * d), a * a - b * b + c * c - d * d, 2 * (c * d - a * b)],
        [2 * (b * d - a * c), 2 * (c * d + a * b), a * a - b * b - c * c + d * d],
    ])


def _water_template():
    half = math.radians(WATER_HOH_DEG) / 2
    o = np.zeros(3)
    h1 = WATER_OH * np.array([math.sin(half), math.cos(half), 0.0])
    h2 = WATER_OH * np.array([-math.sin(half), math.cos(half), 0.0])
    return np.stack([o, h1, h2])


def _uniform_cube(rng, n, side, min_pair=MIN_PAIR, max_rounds=10000):
    """n points uniform in [0, side)^3, re-drawing the later atom of every pair
    closer than min_pair until none is left (open boundary)."""
    from scipy.spatial import cKDTree

    x = rng.uniform(0.0, side, size=(n, 3))
    for _ in range(max_rounds):
        pairs = cKDTree(x).query_pairs(min_pair, output_type="ndarray")
        if pairs.shape[0] == 0:
            return x
        redo = np.unique(pairs.max(axis=1))
        x[redo] = rng.uniform(0.0, side, size=(redo.size, 3))
    raise RuntimeError("rejection sampling did not converge")


class _Grid:
    """Spatial hash for rejection sampling of many atoms (open or periodic)."""

    def __init__(self, cell_size, box=None):
        self.h = cell_size
        self.box = box
        self.cells = {}
        self.pts = []

    def _key(self, p):
        return tuple(int(math.floor(c / self.h)) for c in p)

    def near(self, p, rmin):
        k = self._key(p)
        out_min = np.inf
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    kk = (k[0] + dx, k[1] + dy, k[2] + dz)
                    if self.box is not None:
                        nb = [int(math.floor(b / self.h)) for b in self.box]
                        kk = tuple(kk[a] % nb[a] for a in range(3))
                    for idx in self.cells.get(kk, ()):
                        d = _min_image(self.pts[idx][0] - p, self.box)
                        r = float(np.sqrt(d @ d))
                        if r < out_min:
                            out_min = r
        return out_min

    def near_typed(self, p, tag, rmin_same, rmin_other):
        """True if p is clear: distance >= rmin_same to points with the same tag
        and >= rmin_other to every point."""
        k = self._key(p)
        for dx in (-1, 0, 1):
            for dy in (-1, 0, 1):
                for dz in (-1, 0, 1):
                    kk = (k[0] + dx, k[1] + dy, k[2] + dz)
                    if self.box is not None:
                        nb = [int(math.floor(b / self.h)) for b in self.box]
                        kk = tuple(kk[a] % nb[a] for a in range(3))
                    for idx in self.cells.get(kk, ()):
                        q, t = self.pts[idx]
                        d = _min_image(q - p, self.box)
                        r2 = float(d @ d)
                        if r2 < rmin_other * rmin_other:
                            return False
                        if t == tag and r2 < rmin_same * rmin_same:
                            return False
        return True

    def add(self, p, tag=None):
        k = self._key(p)
        if self.box is not None:
            nb = [int(math.floor(b / self.h)) for b in self.box]
            k = tuple(k[a] % nb[a] for a in range(3))
        self.cells.setdefault(k, []).append(len(self.pts))
        self.pts.append((np.asarray(p, dtype=np.float64), tag))


def _place_waters(rng, n_waters, grid, inside, box=None, min_oo=None, max_tries=2_000_000):
    """Random sequential insertion of rigid waters (O at random, random
    orientation). `inside(p)` restricts the O position; every new atom must be
    >= 0.95 A from every placed atom, and O >= min_oo from every placed O."""
    tmpl = _water_template()
    out = []
    tries = 0
    while len(out) < n_waters:
        tries += 1
        if tries > max_tries:
            raise RuntimeError("water placement did not converge")
        o = inside(rng)
        if o is None:
            continue
        R = _random_rotation(rng)
        atoms = tmpl @ R.T + o
        if box is not None:
            atoms = atoms % box
        ok = True
        for a_idx, p in enumerate(atoms):
            tag = "O" if a_idx == 0 else "H"
            if not grid.near_typed(p, tag, (min_oo if (tag == "O" and min_oo) else MIN_PAIR), MIN_PAIR):
                ok = False
                break
        if not ok:
            continue
        for a_idx, p in enumerate(atoms):
            grid.add(p, "O" if a_idx == 0 else "H")
        out.append(atoms)
    return np.concatenate(out, axis=0) if out else np.zeros((0, 3))


def _water_species(n_waters):
    return np.tile(np.array([3, 0, 0], dtype=np.int8), n_waters)


def _ligand_species(rng, n):
    return rng.choice(NSPECIES, size=n, p=LIGAND_FREQ).astype(np.int8)


def _blob(rng, n, density, center, min_pair=MIN_PAIR):
    """n atoms uniform in a sphere holding `density` atoms/A^3."""
    radius = (3 * n / (4 * math.pi * density)) ** (1 / 3)
    pts = []
    grid = _Grid(2.0)
    while len(pts) < n:
        p = rng.uniform(-radius, radius, size=3)
        if p @ p > radius * radius:
            continue
        p = p + center
        if grid.near(p, min_pair) < min_pair:
            continue
        grid.add(p)
        pts.append(p)
    return np.array(pts), radius, grid


# ----------------------------------------------------------------------------- configs
CONFIG0_DENSITY = 24 / 6.0**3  # atoms / A^3


@functools.lru_cache(maxsize=None)
def _config0(seed=0):
    rng = np.random.default_rng(seed)
    species = np.array([1] * 6 + [2] * 2 + [3] * 2 + [0] * 14, dtype=np.int8)
    species = species[rng.permutation(24)]
    x = _uniform_cube(rng, 24, 6.0)
    return Config(species, x, None, "config0: 24 atoms C6N2O2H14, open")


@functools.lru_cache(maxsize=None)
def _config1(seed=1):
    rng = np.random.default_rng(seed)
    lig_sp = _ligand_species(rng, 72)
    lig, r_lig, grid = _blob(rng, 72, CONFIG0_DENSITY, np.zeros(3))
    # Waters at 1 g/cm^3 (0.0334 waters/A^3) in a shell around the ligand blob.
    vol = 200 / 0.0334
    R = ((3 / (4 * math.pi)) * vol + r_lig**3) ** (1 / 3)

    def inside(rng_):
        p = rng_.uniform(-R, R, size=3)
        rr = float(np.sqrt(p @ p))
        return p if (rr <= R and rr >= r_lig - 0.5) else None

    grid2 = _Grid(2.5)
    for p in lig:
        grid2.add(p, "L")
    wat = _place_waters(rng, 200, grid2, inside, None, min_oo=2.5)
    species = np.concatenate([lig_sp, _water_species(200)])
    x = np.concatenate([lig, wat])
    c = Config(species, x, None, f"config1: 72-atom ligand + 200 waters (672 atoms), open, shell R={R:.2f} A")
    c.shell_radius = R
    return c


@functools.lru_cache(maxsize=None)
def _config2(seed=2):
    rng = np.random.default_rng(seed)
    L = 40.4
    box = np.array([L, L, L])
    grid = _Grid(L / 16, box)
    wat = _place_waters(rng, 2187, grid, lambda r: r.uniform(0, L, size=3), box, min_oo=2.5)
    return Config(_water_species(2187), wat, box, "config2: 2,187 waters (6,561 atoms), periodic L=40.4 A")


@functools.lru_cache(maxsize=None)
def _config4(seed=4):
    rng = np.random.default_rng(seed)
    L = 59.5
    box = np.array([L, L, L])
    center = box / 2
    sol_sp = _ligand_species(rng, 80)
    sol, r_sol, _ = _blob(rng, 80, CONFIG0_DENSITY, center)
    grid = _Grid(L / 23, box)
    for p in sol:
        grid.add(p, "L")
    wat = _place_waters(rng, 7000, grid, lambda r: r.uniform(0, L, size=3), box, min_oo=2.5)
    species = np.concatenate([sol_sp, _water_species(7000)])
    x = np.concatenate([sol, wat])
    return Config(species, x, box, "config4: 7,000 waters + 80-atom solute (21,080 atoms), periodic L=59.5 A")


def molecule_sizes(count=20000, seed=3, lo=8, hi=256):
    """Atom counts N = round(exp(U(ln lo, ln hi))) of the served stream."""
    rng = np.random.default_rng([seed, 0])
    return np.rint(np.exp(rng.uniform(math.log(lo), math.log(hi), size=count))).astype(np.int64)


def served_molecule(m, n_atoms, seed=3):
    """Molecule m of the served stream: species with the drug-like composition,
    uniform in a cube of side 6 (N/24)^(1/3) A, min pair 0.95 A, open."""
    rng = np.random.default_rng([seed, 1, int(m)])
    sp = _ligand_species(rng, int(n_atoms))
    side = 6.0 * (n_atoms / 24.0) ** (1 / 3)
    x = _uniform_cube(rng, int(n_atoms), side)
    return Config(sp, x, None, f"config3 molecule {m}: {n_atoms} atoms")


class ServedStream:
    """The 20,000-request stream (or its first `count` molecules), packed:
    species[int8 sum N], coords[f64 sum N x 3], mol_start[int64 M+1]."""

    def __init__(self, count=20000, seed=3):
        sizes = molecule_sizes(20000, seed)[:count]
        mols = [served_molecule(m, int(n), seed) for m, n in enumerate(sizes)]
        self.sizes = sizes
        self.mol_start = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int64)
        self.species = np.concatenate([m.species for m in mols]).astype(np.int8)
        self.coords = np.concatenate([m.coords for m in mols]).astype(np.float64)
        self.count = count

    @property
    def n_atoms(self):
        return int(self.mol_start[-1])

    def molecule(self, m):
        a, b = int(self.mol_start[m]), int(self.mol_start[m + 1])
        return Config(self.species[a:b], self.coords[a:b], None, f"config3 molecule {m}")


@functools.lru_cache(maxsize=4)
def served_stream(count=20000, seed=3):
    return ServedStream(count, seed)


def make_config(k, seed=None):
    """Workload k (0, 1, 2 or 4) as a Config; workload 3 is `served_stream()`."""
    k = int(k)
    if k == 0:
        return _config0(0 if seed is None else seed)
    if k == 1:
        return _config1(1 if seed is None else seed)
    if k == 2:
        return _config2(2 if seed is None else seed)
    if k == 4:
        return _config4(4 if seed is None else seed)
    raise ValueError("workload 3 is a stream: use served_stream()")


def random_molecule(n, seed, density=CONFIG0_DENSITY, species=None, periodic=False):
    """Small seeded test molecule (or periodic box when periodic=True)."""
    rng = np.random.default_rng([seed, 99, n])
    side = (n / density) ** (1 / 3)
    if species is None:
        species = _ligand_species(rng, n)
    if periodic:
        box = np.array([side, side, side])
        grid = _Grid(side / max(1, int(side // 2.0)), box)
        pts = []
        while len(pts) < n:
            p = rng.uniform(0, side, size=3)
            if grid.near(p, MIN_PAIR) < MIN_PAIR:
                continue
            grid.add(p)
            pts.append(p)
        return Config(species, np.array(pts), box, f"random periodic box n={n}")
    return Config(species, _uniform_cube(rng, n, side), None, f"random molecule n={n}")


# ----------------------------------------------------------------------------- weights
def make_weights(seed=1234, dims=LAYER_DIMS, nets=1):
    """Random-init ANI-2x-shaped per-element networks.

    W ~ N(0, 2 / (fan_in + fan_out)) (Xavier-normal), b ~ U(-0.1, 0.1), one
    seeded stream per (net, species, layer). Returns a dict of float64 arrays
    W1[7,256,1008] b1[7,256] W2[7,192,256] b2[7,192] W3[7,160,192] b3[7,160]
    W4[7,160] b4[7]; with nets > 1 each array gets a leading [nets] axis.
    """
    out = {}
    for layer in range(4):
        fin, fout = dims[layer], dims[layer + 1]
        std = math.sqrt(2.0 / (fin + fout))
        Ws, bs = [], []
        for net in range(nets):
            Wn, bn = [], []
            for s in range(NSPECIES):
                rng = np.random.default_rng([seed, net, s, layer])
                Wn.append(rng.normal(0.0, std, size=(fout, fin)))
                bn.append(rng.uniform(-0.1, 0.1, size=(fout,)))
            Ws.append(np.stack(Wn))
            bs.append(np.stack(bn))
        W = np.stack(Ws)
        b = np.stack(bs)
        if layer == 3:
            W = W[:, :, 0, :]
            b = b[:, :, 0]
        if nets == 1:
            W, b = W[0], b[0]
        out[f"W{layer + 1}"] = np.ascontiguousarray(W)
        out[f"b{layer + 1}"] = np.ascontiguousarray(b)
    return out
