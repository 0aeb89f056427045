"""ctypes declarations of libmlp.so (the C-ABI of include/mlp.h).

Argument marshalling only: every step of an evaluation runs in the library's
CUDA kernels. Importing this module fails loudly if the library is missing;
there is no fallback implementation.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmlp.so")

MLP_OK = 0
MLP_PENDING = 1
MLP_EINVAL = -1
MLP_ENOMEM = -2
MLP_EAGAIN = -3
MLP_ETIMEDOUT = -4
MLP_ECUDA = -5
MLP_ENOTFOUND = -6
MLP_EOVERFLOW = -7
MLP_FP32 = 0
MLP_BF16 = 1
MLP_BF16_1PASS = 2

_NAMES = {0: "MLP_OK", 1: "MLP_PENDING", -1: "MLP_EINVAL", -2: "MLP_ENOMEM", -3: "MLP_EAGAIN",
          -4: "MLP_ETIMEDOUT", -5: "MLP_ECUDA", -6: "MLP_ENOTFOUND", -7: "MLP_EOVERFLOW"}


class MLPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class WeightsHost(ctypes.Structure):
    _fields_ = [(n, ctypes.POINTER(ctypes.c_float)) for n in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")]


class Cutoffs(ctypes.Structure):
    _fields_ = [("rc_rad", ctypes.c_double), ("rc_ang", ctypes.c_double), ("skin", ctypes.c_double)]


class LangevinParams(ctypes.Structure):
    _fields_ = [("dt_fs", ctypes.c_double), ("friction_per_ps", ctypes.c_double), ("temperature_K", ctypes.c_double),
                ("seed", ctypes.c_uint64), ("use_graph", ctypes.c_int)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("max_batch_atoms", ctypes.c_int32), ("max_batch_mols", ctypes.c_int32),
                ("max_atoms_per_mol", ctypes.c_int32), ("streams", ctypes.c_int32),
                ("queue_capacity", ctypes.c_int32), ("budget_bytes", ctypes.c_int64),
                ("min_batch_atoms", ctypes.c_int32), ("max_wait_us", ctypes.c_int32)]


class ServerStats(ctypes.Structure):
    _fields_ = [("submitted", ctypes.c_int64), ("completed", ctypes.c_int64), ("batches", ctypes.c_int64),
                ("atoms", ctypes.c_int64), ("inflight_bytes", ctypes.c_int64),
                ("peak_inflight_bytes", ctypes.c_int64), ("mean_batch_atoms", ctypes.c_double),
                ("slot_bytes", ctypes.c_int64), ("slots", ctypes.c_int32)]


vp = ctypes.c_void_p
ip = ctypes.c_int
i32 = ctypes.c_int32
i64 = ctypes.c_int64
dp = ctypes.POINTER(ctypes.c_double)
fp = ctypes.POINTER(ctypes.c_float)
i8p = ctypes.POINTER(ctypes.c_int8)
i32p = ctypes.POINTER(ctypes.c_int32)
i64p = ctypes.POINTER(ctypes.c_int64)
u64 = ctypes.c_uint64

# name: (restype, argtypes)
SIGNATURES = {
    "mlp_weights_create": (ip, [ctypes.POINTER(WeightsHost), ip, ctypes.POINTER(vp)]),
    "mlp_weights_destroy": (None, [vp]),
    "mlp_create": (ip, [i8p, dp, i32, dp, ctypes.POINTER(Cutoffs), vp, ip, ctypes.POINTER(vp)]),
    "mlp_destroy": (None, [vp]),
    "mlp_energy_forces": (ip, [vp, dp, dp, fp]),
    "mlp_energy_forces_device": (ip, [vp, vp, vp, vp, vp]),
    "mlp_energy_forces_subset_device": (ip, [vp, vp, i64, vp, vp, vp, ip, vp]),
    "mlp_forward_device": (ip, [vp, vp, vp, ip, vp]),
    "mlp_backward_device": (ip, [vp, vp, vp, vp, vp]),
    "mlp_sync": (ip, [vp]),
    "mlp_batch_create": (ip, [vp, ip, i32, i32, i32, ctypes.POINTER(vp)]),
    "mlp_batch_destroy": (None, [vp]),
    "mlp_batch_run_device": (ip, [vp, i32, i32, vp, vp, vp, vp, vp, vp]),
    "mlp_batch_run": (ip, [vp, i32, i32p, i8p, dp, dp, fp]),
    "mlp_batch_sync": (ip, [vp]),
    "mlp_server_opts_default": (None, [ctypes.POINTER(ServerOpts)]),
    "mlp_server_create": (ip, [vp, ctypes.POINTER(ServerOpts), ctypes.POINTER(vp)]),
    "mlp_server_destroy": (None, [vp]),
    "mlp_submit": (ip, [vp, i32, i8p, dp, ctypes.POINTER(u64)]),
    "mlp_poll": (ip, [vp, u64, dp, fp]),
    "mlp_wait": (ip, [vp, u64, i64, dp, fp]),
    "mlp_server_get_stats": (ip, [vp, ctypes.POINTER(ServerStats)]),
    "mlp_server_latencies": (ip, [vp, i64p, ip]),
    "mlp_server_replay": (ip, [vp, i32, i64p, i32p, i8p, dp, dp, fp, i64p]),
    "mlp_server_replay_clients": (ip, [vp, i32, i64p, i32p, i8p, dp, dp, fp, i32, i64p]),
    "mlp_neighbors_static": (ip, [vp, i32, dp, ctypes.c_double, vp, vp, i32, vp]),
    "mlp_set_allocator": (None, [vp, vp, vp]),
    "mlp_debug_fail_alloc": (None, [ctypes.c_longlong]),
    "mlp_last_error": (ctypes.c_char_p, []),
    "mlp_launch_count": (i64, []),
    "mlp_profile_enable": (ip, [ip]),
    "mlp_profile_read": (ip, [ctypes.POINTER(ctypes.c_char_p), dp, i64p, ip]),
    "mlp_profile_reset": (None, []),
    "mlp_debug_neighbors": (ip, [vp, i32p, i32p, i32]),
    "mlp_debug_aev": (ip, [vp, fp]),
    "mlp_debug_aev_split": (ip, [vp, fp, fp]),
    "mlp_debug_forces": (ip, [vp, fp, dp]),
    "mlp_debug_atom_energies": (ip, [vp, fp, fp]),
    "mlp_debug_network": (ip, [vp, ip, i32, i8p, fp, fp, fp]),
    "mlp_langevin_create": (ip, [vp, ctypes.POINTER(LangevinParams), ctypes.POINTER(vp)]),
    "mlp_langevin_destroy": (None, [vp]),
    "mlp_langevin_run": (ip, [vp, vp, vp, i64, i32, vp, vp]),
    "mlp_debug_langevin_normals": (ip, [u64, i64, i32, dp]),
    "mlp_debug_wait_timeout": (ip, [i32p, i32p]),
}

_lib = None


def load():
    """The loaded libmlp.so with argument types set (raises if not built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libmlp.so not built ({LIB_PATH}); run __graft_entry__.build() or "
                              "python -m paper_2310_03121_b300.build")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def check(code, what=""):
    if code < 0:
        msg = load().mlp_last_error().decode(errors="replace")
        raise MLPError(code, f"{what}: {msg}" if what else msg)
    return code
