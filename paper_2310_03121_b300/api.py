"""Python binding of libmlp with the C-ABI's names (argument marshalling only).

Host paths take and return numpy arrays; device paths take torch CUDA
tensors (torch provides device memory and streams) and pass raw pointers.
"""
from __future__ import annotations

import ctypes

import numpy as np

from . import _lib
from ._lib import MLP_BF16, MLP_BF16_1PASS, MLP_FP32, MLPError, check, load

PRECISIONS = {"fp32": MLP_FP32, "bf16": MLP_BF16, "bf16_1pass": MLP_BF16_1PASS, MLP_FP32: MLP_FP32,
              MLP_BF16: MLP_BF16, MLP_BF16_1PASS: MLP_BF16_1PASS}


def _prec(p):
    try:
        return PRECISIONS[p]
    except KeyError:
        raise ValueError(f"precision must be 'fp32', 'bf16' or 'bf16_1pass', got {p!r}") from None


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != shape:
        a = a.reshape(shape)
    return a


def _ptr(a, ctype):
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _stream_ptr(stream):
    import torch

    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _tptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class Weights:
    """Per-element network weights on the device (mlp_weights_create).

    `w` is a dict of arrays W1[7,256,1008] b1[7,256] W2[7,192,256] b2[7,192]
    W3[7,160,192] b3[7,160] W4[7,160] b4[7], or with a leading [K] axis an
    ensemble of K <= 8 nets whose mean is the model (n_nets is taken from
    the arrays when not given)."""

    def __init__(self, w, n_nets=None):
        L = load()
        self._arrays = {k: np.ascontiguousarray(w[k], dtype=np.float32) for k in
                        ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")}
        shp = self._arrays["W1"].shape
        inferred = shp[0] if len(shp) == 4 else 1
        if n_nets is None:
            n_nets = inferred
        if n_nets != inferred or shp[-3:] != (7, 256, 1008):
            raise ValueError(f"W1 of shape {shp} does not hold {n_nets} net(s) of [7, 256, 1008]")
        host = _lib.WeightsHost(*[_ptr(self._arrays[k], ctypes.c_float) for k in
                                  ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")])
        h = ctypes.c_void_p()
        check(L.mlp_weights_create(ctypes.byref(host), int(n_nets), ctypes.byref(h)), "mlp_weights_create")
        self.handle = h
        self.n_nets = n_nets

    def close(self):
        if getattr(self, "handle", None):
            load().mlp_weights_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class System:
    """One molecule or periodic box with a persistent neighbor list (mlp_create)."""

    def __init__(self, weights, species, coords=None, cell=None, precision="fp32", skin=0.0):
        L = load()
        self.species = np.ascontiguousarray(species, dtype=np.int8)
        self.n = int(self.species.shape[0])
        self.weights = weights
        self.precision = _prec(precision)
        cut = _lib.Cutoffs(5.1, 3.5, float(skin))
        c = None if coords is None else _f64(coords, (self.n, 3))
        cl = None if cell is None else _f64(cell)
        h = ctypes.c_void_p()
        check(L.mlp_create(_ptr(self.species, ctypes.c_int8), None if c is None else _ptr(c, ctypes.c_double),
                           self.n, None if cl is None else _ptr(cl, ctypes.c_double), ctypes.byref(cut),
                           weights.handle, self.precision, ctypes.byref(h)), "mlp_create")
        self.handle = h

    def energy_forces(self, coords=None, forces=True):
        """Host path (mlp_energy_forces): returns (E, F[n,3] float32 or None)."""
        c = None if coords is None else _f64(coords, (self.n, 3))
        E = ctypes.c_double()
        F = np.empty((self.n, 3), dtype=np.float32) if forces else None
        check(load().mlp_energy_forces(self.handle, None if c is None else _ptr(c, ctypes.c_double),
                                       ctypes.byref(E), None if F is None else _ptr(F, ctypes.c_float)),
              "mlp_energy_forces")
        return E.value, F

    def energy_forces_device(self, coords, energy=None, forces=None, stream=None):
        """Device path (mlp_energy_forces_device): coords torch.float64 [n,3] on
        CUDA; returns (E float64 [1], F float32 [n,3]) device tensors."""
        import torch

        assert coords.is_cuda and coords.dtype == torch.float64 and coords.is_contiguous()
        if energy is None:
            energy = torch.empty(1, dtype=torch.float64, device=coords.device)
        if forces is None:
            forces = torch.empty((self.n, 3), dtype=torch.float32, device=coords.device)
        check(load().mlp_energy_forces_device(self.handle, _tptr(coords), _tptr(energy), _tptr(forces),
                                              _stream_ptr(stream)), "mlp_energy_forces_device")
        return energy, forces

    def energy_forces_subset_device(self, coords_full, index, forces_full=None, energy=None, accumulate=True,
                                    stream=None):
        """ML/MM mechanical embedding (mlp_energy_forces_subset_device): this
        system is the ML region; `index` (torch.int32 [n] on CUDA) gives its
        rows in `coords_full` (torch.float64 [n_full,3] on CUDA). The ML forces
        go to those rows of `forces_full` (float32 [n_full,3], created zeroed
        if None), added to its contents when `accumulate`. Returns
        (E float64 [1], forces_full)."""
        import torch

        assert coords_full.is_cuda and coords_full.dtype == torch.float64 and coords_full.is_contiguous()
        assert index.is_cuda and index.dtype == torch.int32 and index.is_contiguous() and index.numel() == self.n
        n_full = coords_full.shape[0]
        if energy is None:
            energy = torch.empty(1, dtype=torch.float64, device=coords_full.device)
        if forces_full is None:
            forces_full = torch.zeros((n_full, 3), dtype=torch.float32, device=coords_full.device)
        assert forces_full.dtype == torch.float32 and forces_full.is_contiguous() and forces_full.shape[0] == n_full
        check(load().mlp_energy_forces_subset_device(self.handle, _tptr(coords_full), int(n_full), _tptr(index),
                                                     _tptr(energy), _tptr(forces_full), 1 if accumulate else 0,
                                                     _stream_ptr(stream)), "mlp_energy_forces_subset_device")
        return energy, forces_full

    def forward_device(self, coords, energy, keep_aev=True, stream=None):
        check(load().mlp_forward_device(self.handle, _tptr(coords), _tptr(energy), int(bool(keep_aev)),
                                        _stream_ptr(stream)), "mlp_forward_device")

    def backward_device(self, coords, grad_energy, grad_coords, stream=None):
        check(load().mlp_backward_device(self.handle, _tptr(coords), _tptr(grad_energy), _tptr(grad_coords),
                                         _stream_ptr(stream)), "mlp_backward_device")

    def sync(self):
        check(load().mlp_sync(self.handle), "mlp_sync")

    # kernel-level access (tests)
    def debug_neighbors(self):
        L = load()
        cap = check(L.mlp_debug_neighbors(self.handle, None, None, 0), "mlp_debug_neighbors")
        counts = np.zeros(self.n, dtype=np.int32)
        lst = np.zeros((self.n, cap), dtype=np.int32)
        check(L.mlp_debug_neighbors(self.handle, _ptr(counts, ctypes.c_int32), _ptr(lst, ctypes.c_int32), cap),
              "mlp_debug_neighbors")
        return counts, lst

    def debug_aev(self):
        G = np.zeros((self.n, 1008), dtype=np.float32)
        check(load().mlp_debug_aev(self.handle, _ptr(G, ctypes.c_float)), "mlp_debug_aev")
        return G

    def debug_aev_split(self):
        """(G_hi, G_lo) [n, 1008] float32: the BF16 rows of the last evaluation."""
        hi = np.zeros((self.n, 1008), dtype=np.float32)
        lo = np.zeros((self.n, 1008), dtype=np.float32)
        check(load().mlp_debug_aev_split(self.handle, _ptr(hi, ctypes.c_float), _ptr(lo, ctypes.c_float)),
              "mlp_debug_aev_split")
        return hi, lo

    def debug_forces(self, dEdG):
        """The force kernel alone on the last evaluation's positions and
        neighbors for a given dE/dG [n, 1008]: forces [n, 3] float64."""
        g = np.ascontiguousarray(dEdG, dtype=np.float32)
        assert g.shape == (self.n, 1008)
        F = np.zeros((self.n, 3))
        check(load().mlp_debug_forces(self.handle, _ptr(g, ctypes.c_float), _ptr(F, ctypes.c_double)),
              "mlp_debug_forces")
        return F

    def debug_atom_energies(self, grad=True):
        e = np.zeros(self.n, dtype=np.float32)
        g = np.zeros((self.n, 1008), dtype=np.float32) if grad else None
        check(load().mlp_debug_atom_energies(self.handle, _ptr(e, ctypes.c_float),
                                             None if g is None else _ptr(g, ctypes.c_float)),
              "mlp_debug_atom_energies")
        return e, g

    def close(self):
        if getattr(self, "handle", None):
            load().mlp_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Langevin:
    """LF-Middle Langevin dynamics of a System (mlp_langevin_*): positions
    and velocities stay on the device (torch.float64 [n, 3]); run() advances
    them in place and returns the potential energy at the start of each step.
    Units: A, fs, amu, eV; friction in 1/ps, temperature in K."""

    def __init__(self, system, dt_fs=2.0, friction_per_ps=1.0, temperature_K=300.0, seed=0, use_graph=True):
        L = load()
        self.system = system
        p = _lib.LangevinParams(float(dt_fs), float(friction_per_ps), float(temperature_K), int(seed),
                                1 if use_graph else 0)
        h = ctypes.c_void_p()
        check(L.mlp_langevin_create(system.handle, ctypes.byref(p), ctypes.byref(h)), "mlp_langevin_create")
        self.handle = h

    def run(self, x, v, step0, n_steps, energies=True, stream=None):
        import torch

        for t in (x, v):
            assert t.is_cuda and t.dtype == torch.float64 and t.is_contiguous() and t.shape == (self.system.n, 3)
        E = torch.empty(max(1, n_steps), dtype=torch.float64, device=x.device) if energies else None
        check(load().mlp_langevin_run(self.handle, _tptr(x), _tptr(v), int(step0), int(n_steps),
                                      None if E is None else _tptr(E), _stream_ptr(stream)), "mlp_langevin_run")
        return E[:n_steps] if E is not None else None

    def close(self):
        if getattr(self, "handle", None):
            load().mlp_langevin_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_langevin_normals(seed, step, n):
    """The device generator's normal deviates of atoms 0..n-1 at `step` ([n, 3])."""
    out = np.zeros((n, 3))
    check(load().mlp_debug_langevin_normals(int(seed), int(step), int(n), out.ctypes.data_as(ctypes.POINTER(
        ctypes.c_double))), "mlp_debug_langevin_normals")
    return out

def debug_wait_timeout():
    """(timed_out, code) of the network kernels' bounded barrier wait run on a
    phase that never completes (mlp_debug_wait_timeout); takes ~2 s."""
    t, c = ctypes.c_int32(0), ctypes.c_int32(0)
    check(load().mlp_debug_wait_timeout(ctypes.byref(t), ctypes.byref(c)), "mlp_debug_wait_timeout")
    return int(t.value), int(c.value)


class Batch:
    """Many small open-boundary molecules per launch sequence (mlp_batch_create)."""

    def __init__(self, weights, precision="bf16", max_atoms=131072, max_mols=4096, max_atoms_per_mol=256):
        h = ctypes.c_void_p()
        check(load().mlp_batch_create(weights.handle, _prec(precision), int(max_atoms), int(max_mols),
                                      int(max_atoms_per_mol), ctypes.byref(h)), "mlp_batch_create")
        self.handle = h
        self.weights = weights

    def run(self, mol_start, species, coords, forces=True):
        """Host path: returns (E[n_mols] float64, F[n_atoms,3] float32)."""
        ms = np.ascontiguousarray(mol_start, dtype=np.int32)
        sp = np.ascontiguousarray(species, dtype=np.int8)
        n = int(ms[-1])
        x = _f64(coords, (n, 3))
        E = np.zeros(ms.shape[0] - 1)
        F = np.zeros((n, 3), dtype=np.float32) if forces else None
        check(load().mlp_batch_run(self.handle, ms.shape[0] - 1, _ptr(ms, ctypes.c_int32), _ptr(sp, ctypes.c_int8),
                                   _ptr(x, ctypes.c_double), _ptr(E, ctypes.c_double),
                                   None if F is None else _ptr(F, ctypes.c_float)), "mlp_batch_run")
        return E, F

    def run_device(self, n_mols, n_atoms, mol_start, species, coords, energy, forces, stream=None):
        """Device path (mlp_batch_run_device) on torch tensors; asynchronous."""
        check(load().mlp_batch_run_device(self.handle, int(n_mols), int(n_atoms), _tptr(mol_start), _tptr(species),
                                          _tptr(coords), _tptr(energy), _tptr(forces), _stream_ptr(stream)),
              "mlp_batch_run_device")

    def sync(self):
        check(load().mlp_batch_sync(self.handle), "mlp_batch_sync")

    def close(self):
        if getattr(self, "handle", None):
            load().mlp_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching serving loop (mlp_server_create / mlp_submit / mlp_poll)."""

    def __init__(self, weights, precision="bf16", **opts):
        L = load()
        o = _lib.ServerOpts()
        L.mlp_server_opts_default(ctypes.byref(o))
        o.precision = _prec(precision)
        for k, v in opts.items():
            setattr(o, k, int(v))
        h = ctypes.c_void_p()
        check(L.mlp_server_create(weights.handle, ctypes.byref(o), ctypes.byref(h)), "mlp_server_create")
        self.handle = h
        self.weights = weights
        self.opts = o

    def submit(self, species, coords):
        sp = np.ascontiguousarray(species, dtype=np.int8)
        x = _f64(coords, (sp.shape[0], 3))
        t = ctypes.c_uint64()
        rc = load().mlp_submit(self.handle, sp.shape[0], _ptr(sp, ctypes.c_int8), _ptr(x, ctypes.c_double),
                               ctypes.byref(t))
        check(rc, "mlp_submit")
        return t.value, sp.shape[0]

    def poll(self, ticket):
        """None while pending, else (E, F)."""
        t, n = ticket
        E = ctypes.c_double()
        F = np.zeros((n, 3), dtype=np.float32)
        rc = load().mlp_poll(self.handle, t, ctypes.byref(E), _ptr(F, ctypes.c_float))
        if rc == _lib.MLP_PENDING:
            return None
        check(rc, "mlp_poll")
        return E.value, F

    def wait(self, ticket, timeout_s=60.0):
        t, n = ticket
        E = ctypes.c_double()
        F = np.zeros((n, 3), dtype=np.float32)
        check(load().mlp_wait(self.handle, t, int(timeout_s * 1e9), ctypes.byref(E), _ptr(F, ctypes.c_float)),
              "mlp_wait")
        return E.value, F

    def stats(self):
        s = _lib.ServerStats()
        check(load().mlp_server_get_stats(self.handle, ctypes.byref(s)), "mlp_server_get_stats")
        return {k: getattr(s, k) for k, _ in _lib.ServerStats._fields_}

    def latencies(self, cap=1 << 22):
        out = np.zeros(cap, dtype=np.int64)
        k = check(load().mlp_server_latencies(self.handle, _ptr(out, ctypes.c_int64), cap), "mlp_server_latencies")
        return out[:k]

    def replay(self, arrival_ns, mol_start, species, coords, forces=True, out=None, clients=1):
        """Open-loop arrivals (mlp_server_replay_clients with `clients` native
        client threads); returns (E, F, wall_s).

        out = (E float64 [n_req], F float32 [n_atoms, 3] or None): result
        arrays to reuse (a serving process keeps its output buffers).
        """
        arr = np.ascontiguousarray(arrival_ns, dtype=np.int64)
        ms = np.ascontiguousarray(mol_start, dtype=np.int32)
        sp = np.ascontiguousarray(species, dtype=np.int8)
        n = int(ms[-1])
        x = _f64(coords, (n, 3))
        if out is not None:
            E, F = out
            if E.dtype != np.float64 or E.shape != (arr.shape[0],) or not E.flags.c_contiguous:
                raise ValueError("out[0] must be a contiguous float64 array of one energy per request")
            if F is not None and (F.dtype != np.float32 or F.shape != (n, 3) or not F.flags.c_contiguous):
                raise ValueError("out[1] must be a contiguous float32 [n_atoms, 3] array")
        else:
            E = np.zeros(arr.shape[0])
            F = np.zeros((n, 3), dtype=np.float32) if forces else None
        wall = ctypes.c_int64()
        check(load().mlp_server_replay_clients(self.handle, arr.shape[0], _ptr(arr, ctypes.c_int64),
                                               _ptr(ms, ctypes.c_int32), _ptr(sp, ctypes.c_int8),
                                               _ptr(x, ctypes.c_double), _ptr(E, ctypes.c_double),
                                               None if F is None else _ptr(F, ctypes.c_float), int(clients),
                                               ctypes.byref(wall)),
              "mlp_server_replay_clients")
        return E, F, wall.value * 1e-9

    def close(self):
        if getattr(self, "handle", None):
            load().mlp_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_network(weights, precision, species, G):
    """Network only (mlp_debug_network): (e[n] float32, dE/dG[n,1008] float32)."""
    sp = np.ascontiguousarray(species, dtype=np.int8)
    G = np.ascontiguousarray(G, dtype=np.float32)
    n = sp.shape[0]
    e = np.zeros(n, dtype=np.float32)
    g = np.zeros((n, 1008), dtype=np.float32)
    check(load().mlp_debug_network(weights.handle, _prec(precision), n, _ptr(sp, ctypes.c_int8),
                                   _ptr(G, ctypes.c_float), _ptr(e, ctypes.c_float), _ptr(g, ctypes.c_float)),
          "mlp_debug_network")
    return e, g


def launch_count():
    return int(load().mlp_launch_count())


def profile_enable(on=True):
    return load().mlp_profile_enable(1 if on else 0)


def profile_reset():
    load().mlp_profile_reset()


def profile_read():
    """{kernel name: (total_ms, launches)} of the event-timed launches."""
    L = load()
    k = L.mlp_profile_read(None, None, None, 0)
    names = (ctypes.c_char_p * max(k, 1))()
    ms = np.zeros(max(k, 1))
    cnt = np.zeros(max(k, 1), dtype=np.int64)
    k = L.mlp_profile_read(names, _ptr(ms, ctypes.c_double), _ptr(cnt, ctypes.c_int64), k)
    return {names[q].decode(): (float(ms[q]), int(cnt[q])) for q in range(k)}


def fail_next_allocation(after=0):
    load().mlp_debug_fail_alloc(int(after))


__all__ = ["Weights", "System", "Batch", "Server", "debug_network", "launch_count", "profile_enable",
           "profile_reset", "profile_read", "MLPError", "fail_next_allocation"]
