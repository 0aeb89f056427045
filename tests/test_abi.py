"""C-ABI checks that need no GPU: the library loads, exports every entry point
declared in include/mlp.h, and rejects bad arguments before any CUDA work."""
import ctypes
import os
import re

import numpy as np
import pytest

import gen

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            names |= set(re.findall(r"^MLP_API[^(]*?\b(mlp_\w+)\(", txt, flags=re.M))
    return names


@pytest.fixture(scope="module")
def L():
    from paper_2310_03121_b300 import _lib

    return _lib.load()


def test_every_declared_symbol_is_exported(L):
    names = _declared()
    assert len(names) >= 30
    for n in sorted(names):
        assert hasattr(L, n), n


def test_binding_covers_every_symbol():
    from paper_2310_03121_b300 import _lib

    assert _declared() == set(_lib.SIGNATURES)


def test_null_arguments_are_rejected(L):
    from paper_2310_03121_b300 import _lib

    out = ctypes.c_void_p()
    assert L.mlp_weights_create(None, 1, ctypes.byref(out)) == _lib.MLP_EINVAL
    assert b"NULL" in L.mlp_last_error()
    assert L.mlp_create(None, None, 3, None, None, None, 0, ctypes.byref(out)) == _lib.MLP_EINVAL
    assert L.mlp_energy_forces(None, None, None, None) == _lib.MLP_EINVAL
    assert L.mlp_submit(None, 1, None, None, None) == _lib.MLP_EINVAL
    assert L.mlp_poll(None, 1, None, None) == _lib.MLP_EINVAL
    assert L.mlp_batch_run(None, 1, None, None, None, None, None) == _lib.MLP_EINVAL


def test_bad_weight_count_rejected(L):
    from paper_2310_03121_b300 import _lib

    w = {k: np.ascontiguousarray(v, dtype=np.float32) for k, v in gen.make_weights().items()}
    host = _lib.WeightsHost(*[w[k].ctypes.data_as(ctypes.POINTER(ctypes.c_float))
                              for k in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")])
    out = ctypes.c_void_p()
    assert L.mlp_weights_create(ctypes.byref(host), 0, ctypes.byref(out)) == _lib.MLP_EINVAL
    assert L.mlp_weights_create(ctypes.byref(host), 9, ctypes.byref(out)) == _lib.MLP_EINVAL


def test_weights_binding_checks_ensemble_shape(L):
    """The binding takes K from the arrays' leading axis and refuses a
    count that does not match them, before anything reaches the library."""
    from paper_2310_03121_b300 import api

    w2 = gen.make_weights(nets=2)
    with pytest.raises(ValueError):
        api.Weights(w2, n_nets=3)
    with pytest.raises(ValueError):
        api.Weights(gen.make_weights(), n_nets=2)
    with pytest.raises(ValueError):
        api.Weights({k: v[..., :-1] if k == "W1" else v for k, v in w2.items()})


def test_no_gpu_means_error_not_fallback(L):
    """Without a usable device the compute entry points fail (no CPU path)."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_2310_03121_b300 import _lib

    w = {k: np.ascontiguousarray(v, dtype=np.float32) for k, v in gen.make_weights().items()}
    host = _lib.WeightsHost(*[w[k].ctypes.data_as(ctypes.POINTER(ctypes.c_float))
                              for k in ("W1", "b1", "W2", "b2", "W3", "b3", "W4", "b4")])
    out = ctypes.c_void_p()
    assert L.mlp_weights_create(ctypes.byref(host), 1, ctypes.byref(out)) == _lib.MLP_ECUDA
    assert out.value is None


def test_server_defaults(L):
    from paper_2310_03121_b300 import _lib

    o = _lib.ServerOpts()
    L.mlp_server_opts_default(ctypes.byref(o))
    assert o.precision == _lib.MLP_BF16
    assert o.max_atoms_per_mol == 256 and o.streams == 3
    assert o.budget_bytes == 40 * 10**9


def test_launch_counter_and_profile_without_gpu(L):
    assert L.mlp_launch_count() >= 0
    L.mlp_profile_enable(1)
    assert L.mlp_profile_read(None, None, None, 0) >= 0
    L.mlp_profile_enable(0)
    L.mlp_profile_reset()
