"""Multi-rank path on CPU (gloo, world size 2): ranks take disjoint shares of the
random vectors, compute their DOS moments (with the oracle, on the CPU) and
average them with one all-reduce; the result equals the single-process average
over all vectors, and the timing maximum is the largest rank's."""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import gqt_synth as S
from paper_1705_01387_gb300.replicas import average_moments, max_over_ranks, shard_vectors

R_TOTAL, M = 5, 40


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _model():
    lat = S.honeycomb(6, 5, -2.7, 1.0, seed=2)
    return lat, S.energy_scale_rule(3, -2.7, 1.0)


def _worker(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle as O
    lat, dE = _model()
    h = O.Hamiltonian(lat, dE)
    first, count = shard_vectors(R_TOTAL, world, rank)
    phis = S.random_phase(lat.n, count, seed=11, first_vector=first)
    local = torch.zeros(M, dtype=torch.float64)
    for r in range(count):
        local += torch.from_numpy(h.dos_moments(phis[:, r], M))
    mean = average_moments(local, count)
    tmax = max_over_ranks(1.0 + rank)
    q.put((rank, mean.numpy(), tmax))
    dist.destroy_process_group()


def test_shard_vectors_partition():
    for total in (0, 1, 5, 32):
        for world in (1, 2, 3, 8):
            got = [shard_vectors(total, world, r) for r in range(world)]
            covered = [v for f, c in got for v in range(f, f + c)]
            assert covered == list(range(total))


def test_two_rank_average_equals_single_process():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    import oracle as O
    lat, dE = _model()
    h = O.Hamiltonian(lat, dE)
    phis = S.random_phase(lat.n, R_TOTAL, seed=11)
    ref = np.mean([h.dos_moments(phis[:, r], M) for r in range(R_TOTAL)], axis=0)
    for rank, mean, tmax in res:
        assert np.max(np.abs(mean - ref)) < 1e-14
        assert tmax == 2.0
