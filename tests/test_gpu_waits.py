"""Failure detection without a GPU fault: the tensor-core kernels' bounded
barrier wait, run on a phase that nothing completes, gives up after its
limit (2 s), records the waiting warp and barrier, and the kernel returns;
the host reads the status and the context stays usable (an evaluation
afterwards matches the oracle)."""
import time

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


def test_bounded_wait_times_out_and_context_survives(P):
    t0 = time.perf_counter()
    timed_out, code = P.debug_wait_timeout()
    dt = time.perf_counter() - t0
    assert timed_out == 1
    assert code & 0x40000000, hex(code)             # a timed-out wait was recorded
    assert ((code >> 20) & 0x3F) == 0                 # by warp 0, the waiting thread's warp
    assert 1.5 <= dt <= 30.0, dt                      # the 2 s limit, not an endless wait
    w = gen.make_weights()
    c = gen.make_config(0)
    E_ref, _ = oracle.energy_forces(c.species, c.coords, None, oracle.Weights(w))
    s = P.System(P.Weights(w), c.species, c.coords, None, precision="bf16")
    E, F = s.energy_forces()
    assert abs(E - E_ref) <= 1e-3 * abs(E_ref) and np.isfinite(F).all()
