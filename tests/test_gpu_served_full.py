"""The whole served stream at full size (20,000 molecules, N log-uniform in
[8, 256], 1,426,039 atoms) in the benchmark's launch configuration: batches
of at most 131,072 atoms and 4,096 molecules packed oldest first, BF16
network. The oracle evaluates sampled molecules one by one (the first, the
last, the largest, the smallest, the first and last of every batch, and 40
more at random); every other molecule is checked for finite results, and the
serving loop's results for the same stream equal the batch path's.

Bars: energy relative error <= 1e-3 and force RMS <= 2e-2 eV/A against the
FP64 oracle. A molecule's energy does not depend on its batch (per-row
network, per-molecule FP64 sum in a fixed order): equal bit for bit between
the two paths; forces agree to FP64-atomic rounding.
"""
import numpy as np
import pytest
import torch

import gen
import oracle

pytestmark = pytest.mark.gpu

MAX_ATOMS, MAX_MOLS = 262144, 8192


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


@pytest.fixture(scope="module")
def stream():
    return gen.served_stream(count=20000)


def _chunks(mol_start):
    out, m0, M = [], 0, len(mol_start) - 1
    while m0 < M:
        m1 = m0
        while m1 < M and mol_start[m1 + 1] - mol_start[m0] <= MAX_ATOMS and m1 - m0 < MAX_MOLS:
            m1 += 1
        out.append((m0, m1))
        m0 = m1
    return out


@pytest.fixture(scope="module")
def batch_results(P, W, stream):
    st = stream
    b = P.Batch(W, precision="bf16", max_atoms=MAX_ATOMS, max_mols=MAX_MOLS)
    E = np.empty(st.count)
    F = np.empty((st.n_atoms, 3), dtype=np.float32)
    chunks = _chunks(st.mol_start)
    for m0, m1 in chunks:
        a0, a1 = int(st.mol_start[m0]), int(st.mol_start[m1])
        ms = (st.mol_start[m0:m1 + 1] - a0).astype(np.int32)
        E[m0:m1], F[a0:a1] = b.run(ms, st.species[a0:a1], st.coords[a0:a1])
    b.close()
    return E, F, chunks


def test_full_stream_sampled_against_oracle(stream, wts, batch_results):
    st = stream
    E, F, chunks = batch_results
    assert st.n_atoms == 1426039 and len(chunks) >= 6
    assert np.isfinite(E).all() and np.isfinite(F).all()
    sizes = np.diff(st.mol_start)
    pick = {0, st.count - 1, int(np.argmax(sizes)), int(np.argmin(sizes))}
    for m0, m1 in chunks:
        pick.update((m0, m1 - 1))
    pick.update(np.random.default_rng(11).choice(st.count, 40, replace=False).tolist())
    OW = oracle.Weights(wts)
    errs, sq, n = [], 0.0, 0
    for m in sorted(pick):
        a0, a1 = int(st.mol_start[m]), int(st.mol_start[m + 1])
        E_ref, F_ref = oracle.energy_forces(st.species[a0:a1], st.coords[a0:a1], None, OW)
        errs.append(abs(E[m] - E_ref) / abs(E_ref))
        sq += float(np.sum((F[a0:a1] - F_ref) ** 2))
        n += 3 * (a1 - a0)
    assert max(errs) <= 1e-3, max(errs)
    assert np.sqrt(sq / n) <= 2e-2


def test_full_stream_server_equals_batches(P, W, stream, batch_results):
    st = stream
    E, F, _ = batch_results
    srv = P.Server(W, precision="bf16", max_batch_atoms=MAX_ATOMS, max_batch_mols=MAX_MOLS, streams=2)
    out = (np.empty(st.count), np.empty((st.n_atoms, 3), dtype=np.float32))
    Es, Fs, _ = srv.replay(np.zeros(st.count, dtype=np.int64), st.mol_start, st.species, st.coords, out=out)
    srv.close()
    np.testing.assert_array_equal(Es, E)
    assert np.abs(Fs - F).max() <= 1e-6 * max(1.0, float(np.abs(F).max()))
