"""Serving loop through the C-ABI: results against the oracle and against the
batch path, a molecule's result alone vs in a mix, poll / wait semantics,
timeouts, queue and HBM-budget admission, bad requests, open-loop replay.

Tolerances: BF16 network (the server's default) energy relative error <=
1e-3 and force RMS <= 2e-2 eV/A against the FP64 oracle. A molecule's energy
does not depend on the batch it is packed into (per-row network, per-molecule
FP64 sum in fixed order): equal bit for bit; its forces agree to FP64-atomic
rounding (1e-6 relative).
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


@pytest.fixture(scope="module")
def stream():
    return gen.served_stream(count=400)


def _submit_all(srv, st, idx):
    return [srv.submit(st.molecule(m).species, st.molecule(m).coords) for m in idx]


def test_server_matches_oracle_and_batch(P, W, wts, stream):
    st = stream
    srv = P.Server(W, precision="bf16", max_batch_atoms=8192, max_batch_mols=64, streams=2)
    tickets = _submit_all(srv, st, range(st.count))
    res = [srv.wait(t, 60) for t in tickets]
    E = np.array([r[0] for r in res])
    F = np.concatenate([r[1] for r in res])
    E_ref, F_ref = oracle.energy_forces_batch(st.mol_start, st.species, st.coords, oracle.Weights(wts))
    assert (np.abs(E - E_ref) / np.abs(E_ref)).max() <= 1e-3
    assert np.sqrt(np.mean((F - F_ref) ** 2)) <= 2e-2
    b = P.Batch(W, precision="bf16", max_atoms=st.n_atoms, max_mols=st.count)
    Eb, Fb = b.run(st.mol_start, st.species, st.coords)
    np.testing.assert_array_equal(E, Eb)
    assert np.abs(F - Fb).max() <= 1e-6 * max(1.0, np.abs(Fb).max())
    s = srv.stats()
    assert s["completed"] == st.count and s["batches"] >= st.n_atoms // 8192
    srv.close()


def test_alone_equals_in_mix(P, W, stream):
    st = stream
    srv = P.Server(W, precision="bf16", max_batch_atoms=16384, max_batch_mols=256, streams=2)
    for m in (0, 123, 399):
        mol = st.molecule(m)
        E1, F1 = srv.wait(srv.submit(mol.species, mol.coords), 60)   # alone
        others = _submit_all(srv, st, range(0, 300))
        tk = srv.submit(mol.species, mol.coords)                     # in the mix
        others += _submit_all(srv, st, range(300, 400))
        E2, F2 = srv.wait(tk, 60)
        for t in others:
            srv.wait(t, 60)
        assert E1 == E2
        assert np.abs(F1 - F2).max() <= 1e-6 * max(1.0, np.abs(F1).max())
    srv.close()


def test_poll_wait_semantics(P, W, stream):
    from paper_2310_03121_b300 import _lib

    st = stream
    srv = P.Server(W, precision="bf16", max_batch_atoms=4096, max_batch_mols=64, streams=2)
    with pytest.raises(P.MLPError) as ei:
        srv.poll((987654321, 4))
    assert ei.value.code == _lib.MLP_ENOTFOUND
    tickets = _submit_all(srv, st, range(st.count))
    # the newest request cannot be done a microsecond after it was queued
    with pytest.raises(P.MLPError) as ei:
        srv.wait(tickets[-1], timeout_s=1e-6)
    assert ei.value.code == _lib.MLP_ETIMEDOUT
    out = srv.wait(tickets[-1], 60)          # the ticket stayed valid
    assert np.isfinite(out[0])
    while True:                               # poll: pending until done, then released
        r = srv.poll(tickets[0])
        if r is not None:
            break
    with pytest.raises(P.MLPError) as ei:
        srv.poll(tickets[0])
    assert ei.value.code == _lib.MLP_ENOTFOUND
    for t in tickets[1:-1]:
        srv.wait(t, 60)
    srv.close()


def test_queue_full_and_bad_requests(P, W, stream):
    from paper_2310_03121_b300 import _lib

    st = stream
    srv = P.Server(W, precision="bf16", max_batch_atoms=2048, max_batch_mols=16, streams=1, queue_capacity=8,
                   max_atoms_per_mol=256)
    codes, ok = [], []
    for m in range(200):
        mol = st.molecule(m)
        try:
            ok.append(srv.submit(mol.species, mol.coords))
        except P.MLPError as e:
            codes.append(e.code)
    assert codes and all(c == _lib.MLP_EAGAIN for c in codes)
    for t in ok:
        srv.wait(t, 60)
    big = gen.random_molecule(300, seed=1)
    with pytest.raises(P.MLPError) as ei:
        srv.submit(big.species, big.coords)
    assert ei.value.code == _lib.MLP_EINVAL
    mol = st.molecule(0)
    with pytest.raises(P.MLPError) as ei:
        srv.submit(np.full(mol.n, 7, np.int8), mol.coords)
    assert ei.value.code == _lib.MLP_EINVAL
    srv.close()


def test_hbm_budget_admission(P, W, stream):
    from paper_2310_03121_b300 import _lib

    with pytest.raises(P.MLPError) as ei:
        P.Server(W, precision="bf16", max_batch_atoms=4096, max_batch_mols=64, budget_bytes=1 << 20)
    assert ei.value.code == _lib.MLP_ENOMEM
    probe = P.Server(W, precision="bf16", max_batch_atoms=4096, max_batch_mols=64, streams=2)
    slot = probe.stats()["slot_bytes"]
    assert probe.stats()["slots"] == 2
    probe.close()
    # a budget of 1.5 slots: one slot, one batch in flight, in-flight bytes within the budget
    srv = P.Server(W, precision="bf16", max_batch_atoms=4096, max_batch_mols=64, streams=4,
                   budget_bytes=int(1.5 * slot))
    assert srv.stats()["slots"] == 1
    tickets = _submit_all(srv, stream, range(100))
    for t in tickets:
        srv.wait(t, 60)
    s = srv.stats()
    assert s["completed"] == 100
    assert 0 < s["peak_inflight_bytes"] <= int(1.5 * slot)
    srv.close()


def test_replay_open_loop(P, W, stream):
    st = stream
    srv = P.Server(W, precision="bf16", max_batch_atoms=16384, max_batch_mols=256, streams=2)
    n = 300
    arr = (np.cumsum(np.random.default_rng(0).exponential(1 / 20000.0, size=n)) * 1e9).astype(np.int64)
    ms = st.mol_start[: n + 1]
    E, F, wall = srv.replay(arr, ms, st.species[: ms[-1]], st.coords[: ms[-1]])
    b = P.Batch(W, precision="bf16", max_atoms=int(ms[-1]), max_mols=n)
    Eb, Fb = b.run(ms, st.species[: ms[-1]], st.coords[: ms[-1]])
    np.testing.assert_array_equal(E, Eb)
    lat = srv.latencies()
    assert lat.shape[0] == n and (lat > 0).all()
    assert wall >= arr[-1] * 1e-9
    srv.close()


def test_replay_several_clients(P, W, stream):
    """Three client threads: every request answered, results equal to the
    batch path bit for bit (energies) and to FP64-atomic rounding (forces)."""
    st = stream
    srv = P.Server(W, precision="bf16", max_batch_atoms=16384, max_batch_mols=256, streams=2)
    n = 400
    arr = np.zeros(n, dtype=np.int64)
    ms = st.mol_start[: n + 1]
    E, F, wall = srv.replay(arr, ms, st.species[: ms[-1]], st.coords[: ms[-1]], clients=3)
    b = P.Batch(W, precision="bf16", max_atoms=int(ms[-1]), max_mols=n)
    Eb, Fb = b.run(ms, st.species[: ms[-1]], st.coords[: ms[-1]])
    np.testing.assert_array_equal(E, Eb)
    assert np.abs(F - Fb).max() <= 1e-6 * max(1.0, np.abs(Fb).max())
    assert srv.stats()["completed"] == n and wall > 0
    from paper_2310_03121_b300 import _lib

    with pytest.raises(P.MLPError) as ei:
        srv.replay(arr, ms, st.species[: ms[-1]], st.coords[: ms[-1]], clients=65)
    assert ei.value.code == _lib.MLP_EINVAL
    srv.close()


def test_batching_under_load(P, W, stream):
    """With a batch on the device, a free slot waits for min_batch_atoms (or
    max_wait_us) instead of launching whatever is queued. A burst (every
    request due at once) is then served in at most 2 + ceil(atoms /
    min_batch_atoms) batches: the first, launched on an idle device, batches
    of at least min_batch_atoms, and the remainder. Results equal those of
    greedy launching (which may split the burst either way, depending on
    timing)."""
    st = stream
    arr = np.zeros(st.count, dtype=np.int64)
    batches, outs = {}, {}
    for mb in (0, 16384):
        srv = P.Server(W, precision="bf16", max_batch_atoms=131072, max_batch_mols=4096, streams=2,
                       min_batch_atoms=mb, max_wait_us=20000)
        srv.replay(arr, st.mol_start, st.species, st.coords)
        s0 = srv.stats()
        E, F, _ = srv.replay(arr, st.mol_start, st.species, st.coords)
        batches[mb] = srv.stats()["batches"] - s0["batches"]
        outs[mb] = (E, F)
        srv.close()
    assert batches[16384] <= 2 + -(-st.n_atoms // 16384), batches
    np.testing.assert_array_equal(outs[0][0], outs[16384][0])
    assert np.abs(outs[0][1] - outs[16384][1]).max() <= 1e-6 * max(1.0, np.abs(outs[0][1]).max())
