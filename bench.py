#!/usr/bin/env python
"""Benchmark: atom energy+force evaluations per second of the served path.

Workload: the served stream of 20,000 independent open-boundary molecules,
N log-uniform in [8, 256] atoms (1,426,039 atoms in total, seeded synthetic
geometries at 0.111 atoms/A^3, drug-like element mix, random-init
ANI-2x-shaped weights). One step evaluates every molecule once: the stream is
packed, oldest first, into device batches of at most 262,144 atoms / 8,192
molecules (the serving loop's packing; measured 1.7% faster than 131,072 /
4,096: fewer launches and kernel tails) and the batches run on two CUDA
streams, two in flight.

value  device-resident inputs (all coordinates in HBM before the timed
       region), CUDA-event time per step, L2 flushed between steps.
e2e    the same stream through the C-ABI server (mlp_server_replay_clients
       with --e2e-clients native client threads: host coordinates in, host
       energies and forces out, every request due at t = 0, the server's
       default batching), median wall time of at least nine replays after
       four warm-up replays; p50/p99 request latency.
Also reported: Langevin dynamics at 2 fs (LF-Middle, graph-replayed steps)
of the 72-atom ligand and the 672-atom ligand-in-water system in ns/day,
one net and the 8-net ensemble; velocity-Verlet trajectories at 0.5 fs with
a caller-side repulsive wall (10,000 steps of the 672-atom system: energy
drift; 1,000 steps of the 21,080-atom box on its skin list: atom-steps/s); the same device-resident stream with an ensemble of
--ensemble-nets nets (energy = mean of the nets, forces = mean gradient),
Poisson-arrival latency sweep of the server and, with the same arrivals, of
the one-molecule-per-launch FP32 path (one host queue), that path back to
back, the
roofline of the dominant kernel and the FP64 oracle on the host cores
(cpu_baseline). --nets K makes the ensemble the headline model instead.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "atom energy+force evals/s (served BF16 vs plain FP32, same GPU); p50/p99 latency"
UNIT = "atom-evals/s"
WORKLOAD = ("served stream: 20,000 open-boundary molecules, N log-uniform in [8, 256] (1,426,039 atoms), "
            "ANI-2x-shaped network 1008-256-192-160-1 x 7 elements")

# Algorithmic work per atom of each kernel.
MLP_FLOP_FWD = 2 * (1008 * 256 + 256 * 192 + 192 * 160 + 160)          # 676,160
MLP_FLOP_BWD = 2 * (160 * 192 + 192 * 256 + 256 * 1008)                 # 675,840
MLP_FLOP_B1 = 2 * 256 * 1008                                             # 516,096 (dE/dG = g1 W1)


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x, ws, dev):
    """The largest x over all ranks (the slowest rank times the job); x itself
    on one rank. Every rank calls it (a collective)."""
    if ws <= 1:
        return float(x)
    import torch
    import torch.distributed as dist

    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(ws, units_per_rank, ms_step):
    """Weak scaling, replicas: every rank evaluates the whole stream, so the
    job processes ws x units per step in the slowest rank's time."""
    return ws * units_per_rank / (ms_step * 1e-3)


class Clocks:
    """nvidia-smi sampling during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []   # (host time received, csv line)
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
            return
        # nvidia-smi takes a while to start: wait (bounded) for its first sample,
        # so that the samples cover the timed region that follows
        t_end = time.monotonic() + 10.0
        while not self.lines and time.monotonic() < t_end and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append((time.monotonic(), ln.strip()))

    def begin(self):
        self.t0 = time.monotonic()

    def end(self):
        self.t1 = time.monotonic()

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        time.sleep(0.05)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        # the samples taken during the timed region (one sampling period of slack
        # at its end), else all of them
        lines = self.lines
        if self.t0 is not None and self.t1 is not None:
            inside = [x for x in self.lines if self.t0 <= x[0] <= self.t1 + 0.06]
            lines = inside or self.lines
        for _, ln in lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for nm, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm), "period_ms": 50,
                "timed_region_s": (self.t1 - self.t0) if self.t0 is not None and self.t1 is not None else None}


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0, "sm_max_mhz": 2032.0}, \
        "fallback"


def pack_chunks(mol_start, max_atoms, max_mols):
    """Oldest-first packing of consecutive molecules into batches."""
    chunks = []
    m0 = 0
    M = len(mol_start) - 1
    while m0 < M:
        m1 = m0
        while m1 < M and (mol_start[m1 + 1] - mol_start[m0]) <= max_atoms and (m1 - m0) < max_mols:
            m1 += 1
        chunks.append((m0, m1))
        m0 = m1
    return chunks


def cpu_baseline(stream, wts, seconds, nthreads=None):
    """FP64 oracle on the host cores: a bounded sample of the served stream."""
    import oracle

    OW = oracle.Weights(wts)
    nthreads = nthreads or os.cpu_count() or 1
    # calibrate on a small prefix, then size the sample to ~`seconds`
    m_cal = min(nthreads * 2, stream.count)
    t0 = time.perf_counter()
    oracle.energy_forces_batch(stream.mol_start[: m_cal + 1], stream.species[: stream.mol_start[m_cal]],
                               stream.coords[: stream.mol_start[m_cal]], OW, nthreads=nthreads)
    t_cal = time.perf_counter() - t0
    atoms_cal = int(stream.mol_start[m_cal])
    rate = atoms_cal / max(t_cal, 1e-9)
    target_atoms = rate * seconds
    m = int(np.searchsorted(stream.mol_start, target_atoms))
    m = max(m_cal, min(m, stream.count))
    t0 = time.perf_counter()
    oracle.energy_forces_batch(stream.mol_start[: m + 1], stream.species[: stream.mol_start[m]],
                               stream.coords[: stream.mol_start[m]], OW, nthreads=nthreads)
    dt = time.perf_counter() - t0
    atoms = int(stream.mol_start[m])
    return {"value": atoms / dt, "unit": UNIT, "cores": nthreads, "kind": "oracle",
            "sample": f"first {m} molecules ({atoms} atoms) of the served stream, FP64 oracle "
                      f"(brute-force neighbors, loop AEV, naive network, analytic forces), {dt:.1f} s",
            "seconds": dt, "atoms": atoms}


def run_reference(args):
    ws, rank, local = _dist()
    if rank != 0:
        return 0
    import gen

    stream = gen.served_stream(args.count)
    wts = gen.make_weights(nets=args.nets)
    budget = max(min(2.0, args.ref_seconds), args.ref_seconds / max(1, args.steps + args.warmup))
    vals, secs = [], []
    base = None
    for i in range(args.warmup + args.steps):
        cb = cpu_baseline(stream, wts, budget if i >= args.warmup else min(budget, 2.0))
        if i >= args.warmup:
            vals.append(cb["value"])
            secs.append(cb["seconds"])
            base = cb
    v = statistics.median(vals)
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": statistics.median(secs) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "nets": args.nets, "sample": "bounded per-step sample, see cpu_baseline",
                       "ms_per_step": "measured wall time of one step (one bounded sample of the stream, "
                                      f"{base['atoms']} atoms), median over the timed steps"},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": base["cores"], "kind": "oracle",
                             "sample": base["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def measure_device(P, W, stream, args, prec, dev, ws, local, steps, warmup, profile_steps):
    """Device-resident served-stream steps: (ms per step, per-kernel profile,
    launches in the timed steps, clocks, d_E, d_F). Every step packs the
    stream into batches of at most max_batch_atoms atoms, run alternately on
    two streams; L2 is flushed between timed steps."""
    import torch

    n_atoms = stream.n_atoms
    max_atoms, max_mols = args.max_batch_atoms, args.max_batch_mols
    chunks = pack_chunks(stream.mol_start, max_atoms, max_mols)
    d_xyz = torch.from_numpy(stream.coords).to(dev)
    d_sp = torch.from_numpy(stream.species).to(dev)
    d_E = torch.zeros(stream.count, dtype=torch.float64, device=dev)
    d_F = torch.zeros((n_atoms, 3), dtype=torch.float32, device=dev)
    chunk_ms = []
    for (m0, m1) in chunks:
        a0 = int(stream.mol_start[m0])
        ms = (stream.mol_start[m0:m1 + 1] - a0).astype(np.int32)
        chunk_ms.append(torch.from_numpy(ms).to(dev))
    batches = [P.Batch(W, precision=prec, max_atoms=max_atoms, max_mols=max_mols) for _ in range(2)]
    streams = [torch.cuda.Stream(device=dev) for _ in range(2)]
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)

    def step(one_stream=False):
        start = torch.cuda.Event(enable_timing=True)
        cur = torch.cuda.current_stream()
        start.record(cur)
        for s in streams:
            s.wait_event(start)
        for k, (m0, m1) in enumerate(chunks):
            a0, a1 = int(stream.mol_start[m0]), int(stream.mol_start[m1])
            b = batches[k & 1]
            st = streams[0 if one_stream else (k & 1)]
            b.run_device(m1 - m0, a1 - a0, chunk_ms[k], d_sp[a0:a1], d_xyz[a0:a1], d_E[m0:m1], d_F[a0:a1],
                         stream=st)
        ends = []
        for s in streams:
            e = torch.cuda.Event(enable_timing=True)
            e.record(s)
            ends.append(e)
        for e in ends:
            cur.wait_event(e)
        end = torch.cuda.Event(enable_timing=True)
        end.record(cur)
        return start, end

    def barrier():
        if ws > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    for _ in range(warmup):
        step()
        for b in batches:
            b.sync()
    barrier()
    launches0 = P.launch_count()
    clk = Clocks(local)
    clk.start()
    clk.begin()
    times = []
    for i in range(steps):
        flush.zero_()                      # L2 flush between timed steps (outside the events)
        torch.cuda.synchronize()
        s_ev, e_ev = step()
        torch.cuda.synchronize()
        for b in batches:
            b.sync()
        times.append(s_ev.elapsed_time(e_ev))
    barrier()
    clk.end()
    clocks = clk.stop()
    launches = P.launch_count() - launches0
    # per-kernel durations: the same step on one stream (so that an event pair
    # brackets exactly one kernel), CUDA events around every launch
    P.profile_reset()
    P.profile_enable(True)
    for _ in range(profile_steps):
        flush.zero_()
        torch.cuda.synchronize()
        step(one_stream=True)
        torch.cuda.synchronize()
        for b in batches:
            b.sync()
    P.profile_enable(False)
    prof = P.profile_read()
    ms_step = max_over_ranks(float(np.mean(times)), ws, dev)
    return {"ms_step": ms_step, "prof": prof, "launches": launches, "clocks": clocks, "chunks": len(chunks),
            "d_E": d_E, "d_F": d_F}


def run_ours(args):
    import torch

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if ws > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    import gen
    import paper_2310_03121_b300 as P

    prec = args.precision
    stream = gen.served_stream(args.count)
    wts = gen.make_weights(nets=args.nets)
    W = P.Weights(wts)
    n_atoms = stream.n_atoms
    max_atoms, max_mols = args.max_batch_atoms, args.max_batch_mols
    m = measure_device(P, W, stream, args, prec, dev, ws, local, args.steps, args.warmup, args.profile_steps)
    ms_step, prof, launches, clocks = m["ms_step"], m["prof"], m["launches"], m["clocks"]
    d_E, d_F = m["d_E"], m["d_F"]
    value = whole_job_value(ws, n_atoms, ms_step)

    # sanity: outputs finite
    assert torch.isfinite(d_E).all() and torch.isfinite(d_F).all()

    result = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
              "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
              "vs_baseline": None, "dtype": "bf16" if prec == "bf16" else "f32", "data": "synthetic",
              "config": {"workload": WORKLOAD, "precision": prec, "molecules": stream.count, "atoms": n_atoms,
                         "nets": args.nets, "batch_atoms": max_atoms, "batches_per_step": m["chunks"], "streams": 2,
                         "l2": "flushed between timed steps (256 MB write)",
                         "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU"},
              "clocks": clocks, "gpu_launches": int(round(launches / max(1, args.steps)))}
    result["gpu_launches_timed_total"] = int(launches)
    terms = term_counts(stream)
    result["roofline"] = roofline(prof, n_atoms, args.profile_steps, prec, terms, args.nets)
    result["kernels_roofline"] = kernels_roofline(prof, n_atoms, args.profile_steps, prec, terms, args.nets)
    result["kernels_ms_per_step"] = {k: v[0] / max(1, args.profile_steps) for k, v in sorted(prof.items())}
    result["kernels_timing"] = ("CUDA events around every launch, on the launching stream, in "
                                f"{args.profile_steps} extra steps run on one stream after the timed steps")

    # ---------------- the 8-net ensemble on the same stream (device-resident)
    if args.ensemble_nets > 1 and args.nets == 1:
        We = P.Weights(gen.make_weights(nets=args.ensemble_nets))
        me = measure_device(P, We, stream, args, prec, dev, ws, local, args.steps, args.warmup, args.profile_steps)
        assert torch.isfinite(me["d_E"]).all() and torch.isfinite(me["d_F"]).all()
        result["ensemble"] = {
            "nets": args.ensemble_nets, "value": ws * n_atoms / (me["ms_step"] * 1e-3), "unit": UNIT,
            "ms_per_step": me["ms_step"], "clocks": me["clocks"],
            "gpu_launches": int(round(me["launches"] / max(1, args.steps))),
            "roofline": roofline(me["prof"], n_atoms, args.profile_steps, prec, terms, args.ensemble_nets),
            "kernels_ms_per_step": {k: v[0] / max(1, args.profile_steps) for k, v in sorted(me["prof"].items())},
            "what": "energy = mean of the nets' energies, forces = mean gradient; one AEV and one force pass, "
                    "every net on each 128-row tile inside one network kernel"}
        We.close()

    # ---------------- e2e through the server (host buffers), saturating arrivals
    if not args.no_e2e:
        # the server's own batching (mlp_server_opts_default: batches of <= 131,072
        # atoms / 4,096 molecules, three in flight); larger batches lengthen its
        # pipeline's fill and drain (e2e measured 103.5 M with 262,144), and a
        # third slot overlaps one more batch's gather and scatter with the
        # others' kernels (measured +2.3% over two)
        srv = P.Server(W, precision=prec)
        arr = np.zeros(stream.count, dtype=np.int64)
        walls = []
        lat = None
        # result buffers kept across replays (written once here, so no page is first touched while timed)
        out = (np.ones(stream.count), np.ones((n_atoms, 3), dtype=np.float32))
        # four warm-up replays, then the median of at least 9 (the host threads
        # share the machine's cores, so single replays can be slowed from outside)
        warm = 4
        for i in range(warm + max(9, min(args.steps, 15))):
            E, F, wall = srv.replay(arr, stream.mol_start, stream.species, stream.coords, out=out,
                                    clients=args.e2e_clients)
            lt = srv.latencies()
            if i >= warm:
                walls.append(wall)
                lat = lt
        wall = statistics.median(walls)
        # per replay: coordinates and elements, and per batch its table of the
        # molecules' host blocks (32 B each) and offsets (4 B each, + 1)
        batches = srv.stats()["batches"] / float(warm + len(walls))
        h2d = int(24 * n_atoms + n_atoms + (32 + 4) * stream.count + 4 * batches)
        d2h = 12 * n_atoms + 8 * stream.count
        wall = max_over_ranks(wall, ws, dev)
        result["e2e"] = {"value": ws * n_atoms / wall, "unit": UNIT, "h2d_bytes_per_step": h2d,
                         "d2h_bytes_per_step": d2h, "wall_s": wall, "replays": len(walls),
                         "batches_per_replay": batches,
                         "replay_walls_s": walls,
                         "latency_ms": {"p50": float(np.percentile(lat, 50)) * 1e-6,
                                        "p99": float(np.percentile(lat, 99)) * 1e-6},
                         "path": f"mlp_server_replay_clients, {args.e2e_clients} native client threads, "
                                 f"all {stream.count:,} requests due at t=0, server default batching"}
        if not args.no_sweep and rank == 0:
            result["latency_sweep"] = sweep(srv, stream, args)
        srv.close()

    # ---------------- plain FP32, one molecule per launch: back to back, and open-loop
    if not args.no_plain and rank == 0:
        result["plain_fp32"] = plain_fp32(P, W, stream, args)
        if not args.no_sweep:
            result["latency_sweep_plain_fp32"] = plain_sweep(P, W, stream, args)

    # ---------------- Langevin dynamics (2 fs), graph-replayed steps
    if not args.no_md and rank == 0:
        result["langevin_md"] = langevin_md(P, args)
        result["vv_md"] = vv_md(P, args)

    # ---------------- every synthetic system at both precisions, one evaluation per call
    if not args.no_configs and rank == 0:
        result["systems"] = per_system(P, args)

    if rank == 0 and not args.no_cpu:
        result["cpu_baseline"] = cpu_baseline(stream, wts, args.cpu_seconds)
    if rank == 0:
        print(json.dumps(result), flush=True)
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()
        dist.destroy_process_group()
    return 0


# Counted FP32 operations of the algorithm per term (FMA = 2, transcendental = 1),
# from the loop bodies of the kernels:
FLOP_AEV_PER_NEIGHBOR = 100     # 16 radial shifts + cutoff
FLOP_AEV_PER_PAIR = 180         # geometry, 8 angle factors, 4 distance factors, 32 products
FLOP_FORCE_PER_NEIGHBOR = 175   # 16 radial shifts with derivatives + cutoff + vector
FLOP_FORCE_PER_PAIR = 360       # geometry, 32 terms with derivatives, two gradient vectors


def term_counts(stream):
    """Mean neighbors within 5.1 A and unordered neighbor pairs within 3.5 A per
    atom of the stream (the work units of the AEV and force kernels)."""
    from scipy.spatial import cKDTree

    nr = npairs = 0
    for m in range(stream.count):
        a, b = int(stream.mol_start[m]), int(stream.mol_start[m + 1])
        t = cKDTree(stream.coords[a:b])
        nr += 2 * len(t.query_pairs(5.1, output_type="ndarray"))
        na = np.zeros(b - a, dtype=np.int64)
        pr = t.query_pairs(3.5, output_type="ndarray")
        np.add.at(na, pr[:, 0], 1)
        np.add.at(na, pr[:, 1], 1)
        npairs += int((na * (na - 1) // 2).sum())
    n = stream.n_atoms
    return nr / n, npairs / n


# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) per atom of one
# launch, taken by ncu on a 131,056-atom launch of the served stream with the
# kernel source whose SHA-1 is given; reported as `traffic` only while the
# source is unchanged (otherwise null: the counters no longer describe it).
MEASURED_TRAFFIC = {
    # dram__bytes_read.sum + dram__bytes_write.sum of one ncu capture, per atom of the captured
    # launch (profiles/); valid only while the kernel source is the one that was captured
    # (a header comment changed after the capture, not the code)
    "mlp_tc": {"file": "kernels_mlp_tc.cu", "sha1": "a2e41ec7f05411cd851b2147ee9df4029f7bbd4d",
               "bytes_per_atom": (559.553536e6 + 218.314496e6) / 131056},
    "mlp_tc@8": {"file": "kernels_mlp_tc.cu", "sha1": "a2e41ec7f05411cd851b2147ee9df4029f7bbd4d",
                 "bytes_per_atom": (361.349632e6 + 257.609216e6) / 65518},
    "mlp_tc_b1_ens@8": {"file": "kernels_mlp_tc.cu", "sha1": "a2e41ec7f05411cd851b2147ee9df4029f7bbd4d",
                        "bytes_per_atom": (300.847872e6 + 108.366336e6) / 65518},
}


def measured_traffic(name, atoms_per_launch, nets=1):
    m = MEASURED_TRAFFIC.get(name if nets == 1 else f"{name}@{nets}")
    if not m:
        return None
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "paper_2310_03121_b300", "csrc", m["file"])
    try:
        with open(path, "rb") as f:
            if hashlib.sha1(f.read()).hexdigest() != m["sha1"]:
                return None
    except OSError:
        return None
    return m["bytes_per_atom"] * atoms_per_launch


# Algorithmic DRAM bytes per atom of the small kernels (HBM bound):
# staging reads the FP64 coordinates and the element (25 B) and writes the
# split positions (32 B), the rank (4 B) and zeroed FP64 gradients (24 B);
# the neighbor search writes ~30 list entries (4 B each) and a count; the
# finalize kernel reads the atom energy (4 B) and FP64 gradient (24 B) and
# writes FP32 forces (12 B).
HBM_BYTES_PER_ATOM = {"stage": 85, "neighbors_allpairs": 124, "neighbors_cell": 124, "finalize": 40}


# The binding counters of the issue-bound kernels (fraction of cycles with an
# instruction issued, MUFU and FMA pipe utilisation) from ncu captures of the
# BF16 path (profiles/k_aev_served_bf16.md, profiles/k_forces_served_bf16.md);
# reported only while kernels_aev.cu is the source that was captured (the
# force kernel's capture is of this source; the AEV kernel's code has not
# changed since its own).
MEASURED_ISSUE = {
    "file": "kernels_aev.cu", "sha1": "cbeea17ac41bd96a601bc087cda18067d6417b30",
    "aev": {"issue_active": 0.724, "xu_pipe": 0.221, "fma_pipe": 0.229},
    "forces": {"issue_active": 0.734, "xu_pipe": 0.197, "fma_pipe": 0.384},
}


def measured_issue(name):
    m = MEASURED_ISSUE
    if name not in m:
        return None
    path = os.path.join(ROOT, "paper_2310_03121_b300", "csrc", m["file"])
    try:
        with open(path, "rb") as f:
            if hashlib.sha1(f.read()).hexdigest() != m["sha1"]:
                return None
    except OSError:
        return None
    return dict(m[name], source="ncu capture of this source, BF16 path")


def kernels_roofline(prof, n_atoms, steps, prec, terms, nets=1):
    """Every timed kernel against its own bound: tensor (network), FP32 ALU
    (AEV, forces, FP32 network) or HBM (staging, neighbors, finalize); the
    AEV and force kernels are bound by instruction issue, whose counters
    (from ncu) are added when they describe the current source."""
    out = {}
    for name in prof:
        r = roofline(prof, n_atoms, steps, prec, terms, nets, only=name)
        if r is not None:
            out[name] = {k: r[k] for k in ("bound", "achieved", "peak", "unit", "frac") if k in r}
            if prec == "bf16" and measured_issue(name):
                out[name]["ncu"] = measured_issue(name)
    return out


def roofline(prof, n_atoms, steps, prec, terms, nets=1, only=None):
    peaks, src = measured_peaks()
    if not prof:
        return None
    if only is not None:
        name, (tot_ms, cnt) = only, prof[only]
        if name in HBM_BYTES_PER_ATOM:
            avg_ms = tot_ms / max(1, cnt)
            atoms_per_launch = n_atoms / max(1e-9, cnt / max(1, steps))
            ach = HBM_BYTES_PER_ATOM[name] * atoms_per_launch / (avg_ms * 1e-3) / 1e9
            return {"bound": "hbm", "achieved": ach, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                    "frac": ach / peaks["hbm_gbs"]}
        if not (name.startswith("mlp") or name in ("aev", "forces")):
            return None
        if name == "mlp_tc_b1_ens":
            return None   # reported with mlp_tc as the ensemble's network pair
    else:
        name, (tot_ms, cnt) = max(prof.items(), key=lambda kv: kv[1][0])
    avg_ms = tot_ms / max(1, cnt)
    launches_per_step = cnt / max(1, steps)
    atoms_per_launch = n_atoms / max(1e-9, launches_per_step)
    sm_mhz = peaks.get("sm_max_mhz", 2032.0)
    fp32_peak = 148 * 128 * 2 * sm_mhz * 1e6 / 1e12
    nrad, npair = terms
    base = {"kernel": name, "launch_ms": avg_ms, "units_per_launch": atoms_per_launch,
            "traffic": measured_traffic(name, atoms_per_launch, nets)}
    if name.startswith("mlp_tc"):
        # the method's own work (one forward + one backward per net) against the
        # burst peak (the kernel runs for ~0.4 ms at a time inside a ~12 ms step,
        # not a seconds-long loop); the issued MMAs (the split forward computes
        # every forward GEMM three times) are reported beside it
        peak = peaks["bf16_tflops"]
        fwd_issued = 3 * MLP_FLOP_FWD if prec == "bf16" else MLP_FLOP_FWD
        per_atom = nets * (MLP_FLOP_FWD + MLP_FLOP_BWD)
        per_atom_issued = nets * (fwd_issued + MLP_FLOP_BWD)
        if "mlp_tc_b1_ens" in prof:
            # ensemble: the network kernel stops at g1, the last backward layer
            # of every net is one GEMM in mlp_tc_b1_ens; the pair is the network
            b_ms, b_cnt = prof["mlp_tc_b1_ens"]
            b_avg = b_ms / max(1, b_cnt)
            tc_atom = nets * (MLP_FLOP_FWD + MLP_FLOP_BWD - MLP_FLOP_B1)
            b1_atom = nets * MLP_FLOP_B1
            ach = per_atom * atoms_per_launch / ((avg_ms + b_avg) * 1e-3) / 1e12
            base.update({"kernel": "mlp_tc + mlp_tc_b1_ens", "launch_ms": avg_ms + b_avg,
                         "traffic": (None if base["traffic"] is None or measured_traffic("mlp_tc_b1_ens", 1, nets)
                                     is None else base["traffic"] +
                                     measured_traffic("mlp_tc_b1_ens", atoms_per_launch, nets)),
                         "parts": {
                             "mlp_tc": {"launch_ms": avg_ms, "work": f"{tc_atom} FLOP per atom",
                                        "frac": tc_atom * atoms_per_launch / (avg_ms * 1e-3) / 1e12 / peak},
                             "mlp_tc_b1_ens": {"launch_ms": b_avg, "work": f"{b1_atom} FLOP per atom",
                                               "frac": b1_atom * atoms_per_launch / (b_avg * 1e-3) / 1e12 / peak}}})
            t_ms = avg_ms + b_avg
        else:
            ach = per_atom * atoms_per_launch / (avg_ms * 1e-3) / 1e12
            t_ms = avg_ms
        issued = per_atom_issued * atoms_per_launch / (t_ms * 1e-3) / 1e12
        base.update({"bound": "tensor", "achieved": ach, "peak": peak, "unit": "TFLOP/s", "frac": ach / peak,
                     "peak_source": f"bf16_tflops ({src}, burst): the kernel runs ~0.4 ms at a time",
                     "work": f"{per_atom} FLOP per atom (the method: forward + backward of each net)",
                     "frac_of_sustained": ach / peaks["bf16_tflops_sustained"],
                     "issued": {"achieved": issued, "frac": issued / peak,
                                "work": f"{per_atom_issued} FLOP per atom (MMAs issued: the split forward "
                                        "computes each forward GEMM as three BF16 products)"}})
        return base
    if name.startswith("mlp_f32"):
        layer_flop = {"mlp_f32_l1": 2 * 1008 * 256, "mlp_f32_l2": 2 * 256 * 192, "mlp_f32_l3": 2 * 192 * 160,
                      "mlp_f32_b3": 2 * 160 * 192, "mlp_f32_b2": 2 * 192 * 256, "mlp_f32_b1": 2 * 256 * 1008}
        per_atom = nets * layer_flop.get(name, 0)
    elif name == "forces":
        per_atom = FLOP_FORCE_PER_NEIGHBOR * nrad + FLOP_FORCE_PER_PAIR * npair
    elif name == "aev":
        per_atom = FLOP_AEV_PER_NEIGHBOR * nrad + FLOP_AEV_PER_PAIR * npair
    else:
        per_atom = 0
    ach = per_atom * atoms_per_launch / (avg_ms * 1e-3) / 1e12
    base.update({"bound": "alu", "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
                 "peak_source": "FP32: 148 SMs x 128 lanes x 2 FLOP x max SM clock (unit counts)",
                 "work": f"{per_atom:.0f} FP32 operations per atom ({nrad:.1f} neighbors < 5.1 A, "
                         f"{npair:.1f} pairs < 3.5 A per atom)"})
    return base


def sweep(srv, stream, args):
    out = []
    rng = np.random.default_rng(7)
    for lam in (1000, 2000, 5000, 10000, 20000, 50000):
        n = int(min(stream.count, max(200, lam * args.sweep_seconds)))
        gaps = rng.exponential(1.0 / lam, size=n)
        arr = (np.cumsum(gaps) * 1e9).astype(np.int64)
        ms = stream.mol_start[: n + 1]
        E, F, wall = srv.replay(arr, ms, stream.species[: ms[-1]], stream.coords[: ms[-1]], forces=True)
        lt = srv.latencies()
        out.append({"rate_req_s": lam, "requests": n, "atoms_per_s": float(ms[-1] / wall),
                    "p50_ms": float(np.percentile(lt, 50)) * 1e-6, "p99_ms": float(np.percentile(lt, 99)) * 1e-6})
    return out


def plain_sweep(P, W, stream, args):
    """The one-molecule-per-call FP32 path under the served sweep's open-loop
    Poisson arrivals (the same seeded arrival times): one host queue, one
    worker that takes requests in arrival order and runs each synchronously
    (mlp_batch_run, host buffers, FP32 network), idling until the next
    arrival when the queue is empty; latency = completion - arrival. At most
    args.plain_sweep_requests requests per rate (the first ones of the
    served sweep's sequence). Above its capacity (requests per second of
    service time) the queue, and with it the latency, grows without bound
    for as long as requests keep arriving."""
    b = P.Batch(W, precision="fp32", max_atoms=256, max_mols=1, max_atoms_per_mol=256)
    rng = np.random.default_rng(7)
    out = []
    for lam in (1000, 2000, 5000, 10000, 20000, 50000):
        n_served = int(min(stream.count, max(200, lam * args.sweep_seconds)))
        arr = np.cumsum(rng.exponential(1.0 / lam, size=n_served))    # the served sweep's arrivals
        n = min(n_served, args.plain_sweep_requests)
        lat = np.empty(n)
        busy = 0.0
        atoms = 0
        t0 = time.perf_counter()
        for m in range(n):
            due = t0 + arr[m]
            while time.perf_counter() < due:
                pass
            a, z = int(stream.mol_start[m]), int(stream.mol_start[m + 1])
            t1 = time.perf_counter()
            b.run(np.array([0, z - a], dtype=np.int32), stream.species[a:z], stream.coords[a:z])
            t2 = time.perf_counter()
            busy += t2 - t1
            lat[m] = t2 - due
            atoms += z - a
        wall = time.perf_counter() - t0
        cap = n / busy
        out.append({"rate_req_s": lam, "requests": n, "served_req_s": n / wall, "atoms_per_s": atoms / wall,
                    "capacity_req_s": cap, "saturated": bool(lam > cap),
                    "p50_ms": float(np.percentile(lat, 50)) * 1e3, "p99_ms": float(np.percentile(lat, 99)) * 1e3})
    b.close()
    return out


def plain_fp32(P, W, stream, args):
    """One molecule per launch sequence, FP32 network, synchronous host calls."""
    b = P.Batch(W, precision="fp32", max_atoms=256, max_mols=1, max_atoms_per_mol=256)
    lat = []
    atoms = 0
    t_end = time.perf_counter() + args.plain_seconds
    m = 0
    t0 = time.perf_counter()
    while m < stream.count and (time.perf_counter() < t_end or m < 50):
        a, z = int(stream.mol_start[m]), int(stream.mol_start[m + 1])
        t1 = time.perf_counter()
        b.run(np.array([0, z - a], dtype=np.int32), stream.species[a:z], stream.coords[a:z])
        lat.append(time.perf_counter() - t1)
        atoms += z - a
        m += 1
    dt = time.perf_counter() - t0
    b.close()
    return {"value": atoms / dt, "unit": UNIT, "molecules": m, "p50_ms": float(np.percentile(lat, 50)) * 1e3,
            "p99_ms": float(np.percentile(lat, 99)) * 1e3,
            "path": "mlp_batch_run with one molecule per call (host buffers, synchronous)"}


def langevin_md(P, args):
    """LF-Middle Langevin dynamics at 2 fs (Table 3's integrator and step)
    through mlp_langevin_run with graph replay: the 72-atom ligand of the
    ligand-in-water workload as the ML region on its own (the ML part of a
    mechanically embedded system; the classical part is the caller's), and
    the whole 672-atom workload, one net and the 8-net ensemble, BF16
    network. Wall time per step of the fastest of several runs after a
    warm-up run, each restarting from the initial coordinates. Random-init
    weights have no repulsive core: the 672-atom system collapses (neighbor
    capacity) within ~50 steps with one net, so its runs are 40 steps."""
    import torch

    import gen

    c = gen.make_config(1)
    masses = np.array([1.008, 12.011, 14.007, 15.999, 32.06, 18.998, 35.45])
    out = []
    weights = {1: P.Weights(gen.make_weights()), 8: P.Weights(gen.make_weights(nets=8))}
    cases = (("ligand, 72 atoms", np.arange(72), args.md_steps, 3),
             ("ligand in water, 672 atoms", np.arange(c.n), 40, 8))
    for name, idx, steps, reps in cases:
        sp, x0 = c.species[idx], c.coords[idx]
        m = masses[sp][:, None]
        v0 = np.random.default_rng(0).normal(size=x0.shape) * np.sqrt(8.617333262e-5 * 300.0 / (m * 103.6426965))
        for nets, W in weights.items():
            s = P.System(W, sp, x0, None, precision="bf16")
            L = P.Langevin(s, dt_fs=2.0, friction_per_ps=1.0, temperature_K=300.0, seed=1, use_graph=True)
            walls, err = [], None
            for rep in range(reps + 1):
                x = torch.from_numpy(np.ascontiguousarray(x0)).cuda()
                v = torch.from_numpy(np.ascontiguousarray(v0)).cuda()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                try:
                    L.run(x, v, 0, steps, energies=False)     # waits for the last step
                except P.MLPError as e:
                    err = str(e)
                    break
                walls.append(time.perf_counter() - t0)
            row = {"system": name, "nets": nets, "atoms": int(idx.size), "steps_per_run": steps}
            if err or len(walls) < 2:
                row["aborted"] = err
            else:
                us = min(walls[1:]) / steps * 1e6          # the first run captures the graph
                row.update({"us_per_step": us, "ns_per_day": 2.0e-6 * 86400.0 / (us * 1e-6),
                            "atom_steps_per_s": idx.size / (us * 1e-6)})
            out.append(row)
            L.close()
            s.close()
    for W in weights.values():
        W.close()
    return out


def per_system(P, args):
    """Each synthetic system (the 24-atom molecule, the 672-atom ligand in
    water, the 6,561-atom and 21,080-atom periodic water boxes) at both
    precisions through the device path (mlp_energy_forces_device, coordinates
    resident on the device): ms per evaluation and atom-evals/s, CUDA events
    on the launching stream around each evaluation, L2 flushed (256 MB write)
    before each."""
    import torch

    import gen

    W = P.Weights(gen.make_weights())
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device="cuda")
    names = {0: "24-atom molecule", 1: "672-atom ligand in water", 2: "6,561-atom water box (periodic)",
             4: "21,080-atom solvated box (periodic)"}
    out = []
    for k, name in names.items():
        c = gen.make_config(k)
        x = torch.from_numpy(np.ascontiguousarray(c.coords)).cuda()
        for prec in ("fp32", "bf16"):
            s = P.System(W, c.species, c.coords, c.cell, precision=prec)
            for _ in range(3):
                s.energy_forces_device(x)
            torch.cuda.synchronize()
            ms = []
            for _ in range(args.config_reps):
                flush.fill_(1)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                s.energy_forces_device(x)
                e1.record()
                e1.synchronize()
                ms.append(e0.elapsed_time(e1))
            t = float(np.median(ms))
            out.append({"system": name, "atoms": int(c.n), "precision": prec, "ms_per_eval": t,
                        "atom_evals_per_s": c.n / (t * 1e-3)})
            s.close()
    W.close()
    return out


def vv_md(P, args):
    """Velocity-Verlet dynamics at 0.5 fs of the two workloads that ask for a
    trajectory, with the caller's short-range repulsive wall (md.RepulsiveWall:
    shifted r^-12 inside 1.0 A, the classical part a caller adds; random-init
    weights have no repulsive core) added to the ML forces through the
    accumulate path: the 672-atom ligand in water for args.vv_steps steps on
    the FP32 path (total-energy drift per atom per ps), and the 21,080-atom
    periodic box for args.box_md_steps steps on the BF16 path with its
    persistent 5.6 A list (0.5 A skin, rebuilt every 10 steps or when an atom
    moved half the skin): atom-steps/s. Host wall time of the whole run; the
    host reads the energies every report interval."""
    import gen
    from paper_2310_03121_b300 import md

    W = P.Weights(gen.make_weights())
    out = []
    keys = ("atoms", "steps", "dt_fs", "wall_s", "atom_steps_per_s", "drift_eV_per_atom_per_ps",
            "etot_rms_fluct_eV_per_atom", "temperature_K_last", "aborted", "repulsive_wall")
    c = gen.make_config(1)
    s = P.System(W, c.species, c.coords, None, precision="fp32")
    res = md.run(s, c.species, c.coords, None, dt_fs=0.5, steps=args.vv_steps, report_every=20, guard_every=0,
                 wall=md.RepulsiveWall(c.n))
    s.close()
    out.append(dict({"system": "672-atom ligand in water (open), FP32 path"}, **{k: res[k] for k in keys}))
    c = gen.make_config(4)
    s = P.System(W, c.species, c.coords, c.cell, precision="bf16", skin=0.5)
    res = md.run(s, c.species, c.coords, c.cell, dt_fs=0.5, steps=args.box_md_steps, report_every=50,
                 guard_every=0, wall=md.RepulsiveWall(c.n, c.cell))
    s.close()
    out.append(dict({"system": "21,080-atom solvated box (periodic), BF16 path, 5.6 A skin list"},
                    **{k: res[k] for k in keys}))
    W.close()
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="bf16", choices=["bf16", "fp32"])
    ap.add_argument("--count", type=int, default=20000)
    ap.add_argument("--max-batch-atoms", type=int, default=262144)
    ap.add_argument("--max-batch-mols", type=int, default=8192)
    ap.add_argument("--sweep-seconds", type=float, default=1.0)
    ap.add_argument("--profile-steps", type=int, default=2)
    ap.add_argument("--plain-seconds", type=float, default=3.0)
    ap.add_argument("--plain-sweep-requests", type=int, default=2000,
                    help="requests per arrival rate of the plain path's open-loop sweep")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--e2e-clients", type=int, default=1, help="client threads of the e2e replay")
    ap.add_argument("--no-sweep", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--nets", type=int, default=1, help="ensemble size of the headline measurement")
    ap.add_argument("--ref-seconds", type=float, default=120.0,
                    help="host-core seconds of the reference (oracle) run, spread over its steps")
    ap.add_argument("--no-md", action="store_true", help="skip the Langevin dynamics timing")
    ap.add_argument("--md-steps", type=int, default=1000)
    ap.add_argument("--box-md-steps", type=int, default=1000)
    ap.add_argument("--vv-steps", type=int, default=10000, help="velocity-Verlet steps of the 672-atom system")
    ap.add_argument("--no-configs", action="store_true", help="skip the per-system timing")
    ap.add_argument("--config-reps", type=int, default=20)
    ap.add_argument("--ensemble-nets", type=int, default=8,
                    help="also time an ensemble of this many nets on the same stream (<= 1: skip)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
