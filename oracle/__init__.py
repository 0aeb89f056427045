"""FP64 CPU oracle (test infrastructure only).

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
may import this module. The product library never imports it: it is the
independent reference that the CUDA path is checked against.

`oracle.c` is a plain, slow C implementation of the ANI-2x-shaped potential
(brute-force O(N^2) neighbors, loop-form AEVs, naive matrix-vector network,
hand-derived forces); this module compiles it to `liboracle.so` and wraps it
with ctypes. See `oracle.c` for the definitions and the paper passages.

Parity status per function (what pins it, from tests/test_oracle.py):
  oracle_cutoff, oracle_celu ........ closed-form special values, torch.nn.functional.celu
  oracle_pair_index ................. enumeration of the 28 unordered pairs
  oracle_neighbors .................. scipy.spatial.cKDTree on periodic/open boxes
  oracle_aev ........................ 2- and 3-atom special cases, invariances
  oracle_atom_energy ................ torch Linear+CELU chain, single-path network;
                                      ensemble: K copies of one net, net-by-net means
  oracle_energy_forces .............. central finite differences, zero net force/torque
  oracle_forces_from_dEdG ........... central differences of g . G(r) for a random g; equality
                                      with oracle_energy_forces for the network's own dE/dG
  oracle_forces_subset / local energy  equality with the full evaluation
  oracle_ml_region .................. invariance to the classical region, zero rows, finite differences
  oracle_philox4x64 ................. numpy.random.Philox (the same published generator)
  oracle_langevin_normals ........... moments and quantiles of the normal distribution
  oracle_lfmiddle_step .............. leapfrog invariant (no friction), equipartition and velocity decay
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
AEV_LEN = 1008


def build(force=False):
    """Compile oracle.c -> liboracle.so (gcc, -O2, OpenMP for the batch driver)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    cmd = ["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-std=c11", _SRC, "-o", _LIB, "-lm"]
    subprocess.check_call(cmd)
    return _LIB


class _Weights(ctypes.Structure):
    _fields_ = [(n, ctypes.POINTER(ctypes.c_double)) for n in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")] + \
        [("nets", ctypes.c_int)]


_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_lib = None


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB)
        L.oracle_cutoff.restype = ctypes.c_double
        L.oracle_cutoff.argtypes = [ctypes.c_double, ctypes.c_double]
        L.oracle_cutoff_deriv.restype = ctypes.c_double
        L.oracle_cutoff_deriv.argtypes = [ctypes.c_double, ctypes.c_double]
        L.oracle_celu.restype = ctypes.c_double
        L.oracle_celu.argtypes = [ctypes.c_double]
        L.oracle_celu_deriv.restype = ctypes.c_double
        L.oracle_celu_deriv.argtypes = [ctypes.c_double]
        L.oracle_pair_index.restype = ctypes.c_int
        L.oracle_pair_index.argtypes = [ctypes.c_int, ctypes.c_int]
        L.oracle_neighbors.restype = ctypes.c_long
        L.oracle_neighbors.argtypes = [ctypes.c_int, _dp, _dp, ctypes.c_double, ctypes.c_long, _ip,
                                       ctypes.POINTER(ctypes.c_ubyte)]
        L.oracle_aev.restype = None
        L.oracle_aev.argtypes = [ctypes.c_int, _ip, _dp, _dp, _dp]
        L.oracle_atom_energy.restype = ctypes.c_double
        L.oracle_atom_energy.argtypes = [ctypes.c_int, _dp, ctypes.POINTER(_Weights), _dp]
        L.oracle_energy.restype = ctypes.c_double
        L.oracle_energy.argtypes = [ctypes.c_int, _ip, _dp, _dp, ctypes.POINTER(_Weights), _dp]
        L.oracle_energy_forces.restype = ctypes.c_double
        L.oracle_energy_forces.argtypes = [ctypes.c_int, _ip, _dp, _dp, ctypes.POINTER(_Weights), _dp, _dp]
        L.oracle_forces_from_dEdG.restype = None
        L.oracle_forces_from_dEdG.argtypes = [ctypes.c_int, _ip, _dp, _dp, _dp, _dp]
        L.oracle_aev_grad.restype = None
        L.oracle_aev_grad.argtypes = [ctypes.c_int, _ip, _dp, _dp, ctypes.POINTER(_Weights), _dp, _dp]
        L.oracle_forces_subset.restype = None
        L.oracle_forces_subset.argtypes = [ctypes.c_int, _ip, _dp, _dp, ctypes.POINTER(_Weights), ctypes.c_int,
                                           _ip, _dp]
        L.oracle_local_energy.restype = ctypes.c_double
        L.oracle_local_energy.argtypes = [ctypes.c_int, _ip, _dp, _dp, ctypes.POINTER(_Weights), ctypes.c_int,
                                          _dp, ctypes.c_double]
        L.oracle_atom_energies.restype = None
        L.oracle_atom_energies.argtypes = [ctypes.c_int, _ip, _dp, _dp, ctypes.POINTER(_Weights), ctypes.c_int, _ip,
                                           _dp, ctypes.c_int]
        L.oracle_aev_subset.restype = None
        L.oracle_aev_subset.argtypes = [ctypes.c_int, _ip, _dp, _dp, ctypes.c_int, _ip, _dp]
        u64 = ctypes.c_uint64
        u64p = ctypes.POINTER(ctypes.c_uint64)
        L.oracle_philox4x64.restype = None
        L.oracle_philox4x64.argtypes = [u64p, u64p, u64p]
        L.oracle_langevin_normals.restype = None
        L.oracle_langevin_normals.argtypes = [u64, ctypes.c_int64, ctypes.c_int, _dp]
        L.oracle_lfmiddle_step.restype = None
        L.oracle_lfmiddle_step.argtypes = [ctypes.c_int, _ip, _dp, _dp, _dp, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, u64, ctypes.c_int64]
        L.oracle_langevin_run.restype = None
        L.oracle_langevin_run.argtypes = [ctypes.c_int, _ip, _dp, _dp, _dp, ctypes.POINTER(_Weights), ctypes.c_double,
                                          ctypes.c_double, ctypes.c_double, u64, ctypes.c_int64, ctypes.c_int, _dp]
        L.oracle_ml_region.restype = ctypes.c_double
        L.oracle_ml_region.argtypes = [ctypes.c_int, _ip, _dp, _dp, ctypes.POINTER(_Weights), ctypes.c_int, _ip, _dp]
        L.oracle_energy_forces_batch.restype = None
        L.oracle_energy_forces_batch.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_long), _ip, _dp, _dp,
                                                 ctypes.POINTER(_Weights), _dp, _dp, ctypes.c_int]
        _lib = L
    return _lib


def _d(a):
    return a.ctypes.data_as(_dp)


def _i(a):
    return a.ctypes.data_as(_ip)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i32(a):
    return np.ascontiguousarray(a, dtype=np.int32)


def _cell(cell):
    return None if cell is None else _f64(cell)


class Weights:
    """FP64 weights for the oracle (dict from gen.make_weights).

    A single net has W1[7,256,1008] ...; an ensemble of K nets carries a
    leading [K] axis on every array, and the model is the mean of the K nets
    (energy and dE/dG alike)."""

    def __init__(self, w):
        self.arrays = {k: _f64(w[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")}
        shp = self.arrays["W1"].shape
        if shp == (7, 256, AEV_LEN):
            self.nets = 1
        else:
            assert len(shp) == 4 and shp[1:] == (7, 256, AEV_LEN), shp
            self.nets = shp[0]
        for k, v in self.arrays.items():
            assert v.shape[0] == self.nets or self.nets == 1, (k, v.shape)
        self.struct = _Weights(*[_d(self.arrays[k]) for k in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")],
                               self.nets)

    def ref(self):
        return ctypes.byref(self.struct)


def _as_weights(w):
    return w if isinstance(w, Weights) else Weights(w)


def cutoff(r, rc):
    return lib().oracle_cutoff(float(r), float(rc))


def cutoff_deriv(r, rc):
    return lib().oracle_cutoff_deriv(float(r), float(rc))


def celu(x):
    return lib().oracle_celu(float(x))


def celu_deriv(x):
    return lib().oracle_celu_deriv(float(x))


def pair_index(a, b):
    return lib().oracle_pair_index(int(a), int(b))


def neighbors(coords, cell, rc):
    """All ordered pairs (i, j) with |d_ij| < rc: (pairs[P, 2] int32,
    band[P] uint8: 0 = clear, 1 = inside but within the rounding band,
    2 = outside but within the band)."""
    x = _f64(coords)
    n = x.shape[0]
    c = _cell(cell)
    L = lib()
    cnt = L.oracle_neighbors(n, _d(x), None if c is None else _d(c), rc, 0, None, None)
    pairs = np.zeros((max(cnt, 1), 2), dtype=np.int32)
    band = np.zeros(max(cnt, 1), dtype=np.uint8)
    L.oracle_neighbors(n, _d(x), None if c is None else _d(c), rc, cnt, _i(pairs),
                       band.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte)))
    return pairs[:cnt], band[:cnt]


def aev(species, coords, cell=None):
    x = _f64(coords)
    s = _i32(species)
    n = x.shape[0]
    G = np.zeros((n, AEV_LEN))
    c = _cell(cell)
    lib().oracle_aev(n, _i(s), _d(x), None if c is None else _d(c), _d(G))
    return G


def atom_energy(s, G, w, grad=False):
    w = _as_weights(w)
    G = _f64(G)
    g = np.zeros(AEV_LEN) if grad else None
    e = lib().oracle_atom_energy(int(s), _d(G), w.ref(), None if g is None else _d(g))
    return (e, g) if grad else e


def energy(species, coords, cell, w, per_atom=False):
    w = _as_weights(w)
    x = _f64(coords)
    s = _i32(species)
    n = x.shape[0]
    e = np.zeros(n)
    c = _cell(cell)
    E = lib().oracle_energy(n, _i(s), _d(x), None if c is None else _d(c), w.ref(), _d(e))
    return (E, e) if per_atom else E


def energy_forces(species, coords, cell, w, per_atom=False):
    w = _as_weights(w)
    x = _f64(coords)
    s = _i32(species)
    n = x.shape[0]
    e = np.zeros(n)
    F = np.zeros((n, 3))
    c = _cell(cell)
    E = lib().oracle_energy_forces(n, _i(s), _d(x), None if c is None else _d(c), w.ref(), _d(e), _d(F))
    return (E, F, e) if per_atom else (E, F)


def philox4x64(counter, key):
    """Philox4x64-10 block: 4 uint64 words of counter (4 words) under key (2 words)."""
    c = np.ascontiguousarray(counter, dtype=np.uint64)
    k = np.ascontiguousarray(key, dtype=np.uint64)
    out = np.zeros(4, dtype=np.uint64)
    p = ctypes.POINTER(ctypes.c_uint64)
    lib().oracle_philox4x64(c.ctypes.data_as(p), k.ctypes.data_as(p), out.ctypes.data_as(p))
    return out


def langevin_normals(seed, step, n):
    """Normal deviates [n, 3] of atoms 0..n-1 at `step` (Philox counter (step, i), key (seed, 0))."""
    out = np.zeros((n, 3))
    for i in range(n):
        lib().oracle_langevin_normals(int(seed), int(step), i, _d(out[i]))
    return out


def lfmiddle_step(species, x, v, F, dt, friction_per_ps, temperature, seed, step):
    """One LF-Middle update from forces F; returns new (x, v)."""
    x = _f64(x).copy()
    v = _f64(v).copy()
    F = _f64(F)
    s = _i32(species)
    lib().oracle_lfmiddle_step(s.shape[0], _i(s), _d(x), _d(v), _d(F), float(dt), float(friction_per_ps),
                               float(temperature), int(seed), int(step))
    return x, v


def langevin_run(species, x, v, cell, w, dt, friction_per_ps, temperature, seed, step0, n_steps):
    """n_steps LF-Middle steps with the oracle's forces: (x, v, E_pot[n_steps])."""
    w = _as_weights(w)
    x = _f64(x).copy()
    v = _f64(v).copy()
    s = _i32(species)
    E = np.zeros(max(1, n_steps))
    c = _cell(cell)
    lib().oracle_langevin_run(s.shape[0], _i(s), _d(x), _d(v), None if c is None else _d(c), w.ref(), float(dt),
                              float(friction_per_ps), float(temperature), int(seed), int(step0), int(n_steps), _d(E))
    return x, v, E[:n_steps]


def ml_region(species, coords, cell, w, index):
    """ML part of a mechanically embedded system: (E_ML, F_full[n_full, 3])
    with the subset's forces in rows `index` and zeros elsewhere."""
    w = _as_weights(w)
    x = _f64(coords)
    s = _i32(species)
    idx = _i32(index)
    F = np.zeros_like(x)
    c = _cell(cell)
    E = lib().oracle_ml_region(x.shape[0], _i(s), _d(x), None if c is None else _d(c), w.ref(), idx.shape[0],
                               _i(idx), _d(F))
    return E, F


def aev_grad(species, coords, cell, w):
    """(e_atoms[n], dE/dG[n, 1008])."""
    w = _as_weights(w)
    x = _f64(coords)
    s = _i32(species)
    n = x.shape[0]
    e = np.zeros(n)
    g = np.zeros((n, AEV_LEN))
    c = _cell(cell)
    lib().oracle_aev_grad(n, _i(s), _d(x), None if c is None else _d(c), w.ref(), _d(e), _d(g))
    return e, g


def forces_from_dEdG(species, coords, cell, dEdG):
    """F[n, 3] = -sum_i dEdG[i] . dG_i/dr (the AEV backward for a given dE/dG)."""
    x = _f64(coords)
    s = _i32(species)
    n = x.shape[0]
    g = _f64(dEdG)
    assert g.shape == (n, AEV_LEN)
    F = np.zeros((n, 3))
    c = _cell(cell)
    lib().oracle_forces_from_dEdG(n, _i(s), _d(x), None if c is None else _d(c), _d(g), _d(F))
    return F


def forces_subset(species, coords, cell, w, idx):
    w = _as_weights(w)
    x = _f64(coords)
    s = _i32(species)
    idx = _i32(idx)
    out = np.zeros((idx.shape[0], 3))
    c = _cell(cell)
    lib().oracle_forces_subset(x.shape[0], _i(s), _d(x), None if c is None else _d(c), w.ref(), idx.shape[0],
                               _i(idx), _d(out))
    return out


def local_energy(species, coords, cell, w, m, center, margin=0.2):
    w = _as_weights(w)
    x = _f64(coords)
    s = _i32(species)
    ctr = _f64(center)
    c = _cell(cell)
    return lib().oracle_local_energy(x.shape[0], _i(s), _d(x), None if c is None else _d(c), w.ref(), int(m),
                                     _d(ctr), float(margin))


def atom_energies(species, coords, cell, w, idx=None, nthreads=None):
    """e_i for the listed atoms (all atoms if idx is None), threads over atoms."""
    w = _as_weights(w)
    x = _f64(coords)
    s = _i32(species)
    n = x.shape[0]
    idx = np.arange(n, dtype=np.int32) if idx is None else _i32(idx)
    e = np.zeros(idx.shape[0])
    c = _cell(cell)
    nt = int(nthreads or os.cpu_count() or 1)
    lib().oracle_atom_energies(n, _i(s), _d(x), None if c is None else _d(c), w.ref(), idx.shape[0], _i(idx), _d(e),
                               nt)
    return e


def aev_subset(species, coords, cell, idx):
    x = _f64(coords)
    s = _i32(species)
    idx = _i32(idx)
    G = np.zeros((idx.shape[0], AEV_LEN))
    c = _cell(cell)
    lib().oracle_aev_subset(x.shape[0], _i(s), _d(x), None if c is None else _d(c), idx.shape[0], _i(idx), _d(G))
    return G


def energy_forces_batch(mol_start, species, coords, w, nthreads=None):
    """Independent open-boundary molecules back to back; returns (E[M], F[N,3])."""
    w = _as_weights(w)
    ms = np.ascontiguousarray(mol_start, dtype=np.int64)
    x = _f64(coords)
    s = _i32(species)
    nmol = ms.shape[0] - 1
    E = np.zeros(nmol)
    F = np.zeros((x.shape[0], 3))
    nt = int(nthreads or os.cpu_count() or 1)
    lib().oracle_energy_forces_batch(nmol, ms.ctypes.data_as(ctypes.POINTER(ctypes.c_long)), _i(s), _d(x), None,
                                     w.ref(), _d(E), _d(F), nt)
    return E, F
