"""B300-native energy+force evaluation of an ANI-2x-shaped neural-network
potential (the hot path of OpenMM 8's machine-learning-potential
simulations): cell-list neighbors, AEVs, per-element networks (FP32 SIMT or
BF16 tcgen05 tensor cores) and the analytic force backward, as hand-written
sm_103a CUDA kernels behind the C-ABI of include/mlp.h (libmlp.so).

This package is the Python binding of that C-ABI (argument marshalling
only). There is no CPU fallback: without the built library every call into
the binding raises ImportError (build it with
`python -m paper_2310_03121_b300.build`).
"""
from ._lib import MLP_BF16, MLP_FP32, MLPError, load  # noqa: F401
from .api import (Batch, Langevin, Server, System, Weights, debug_langevin_normals, debug_network,  # noqa: F401
                  debug_wait_timeout, fail_next_allocation, launch_count, profile_enable, profile_read,
                  profile_reset)
