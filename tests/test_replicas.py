"""Replicas across ranks (CPU, gloo, world size 2).

Each rank answers its own shard of the queries; gathering the shards in rank
order must give exactly the single-process answer, and the job time is the
slowest rank's.  The per-rank search here is the CPU oracle (no GPU in this
test); on GPUs bench.py runs mih_knn in the same sharding.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1307_2982_gb300 import replicas, synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, out_dir):
    import oracle

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        db = synth.uniform_codes(4000, 128, 0)
        qs = synth.uniform_codes(101, 128, 1)          # ragged: 51 + 50
        lo, hi = replicas.shard(len(qs), world, rank)
        ids, d = oracle.knn(db, qs[lo:hi], 17, nthreads=2)
        local = torch.from_numpy(np.concatenate([ids.view(np.int32), d], axis=1))
        full = replicas.gather_rows(local, len(qs))
        slow = replicas.max_over_ranks(1.0 + rank)
        if rank == 0:
            np.save(os.path.join(out_dir, "gathered.npy"), full.numpy())
            np.save(os.path.join(out_dir, "slow.npy"), np.array([slow]))
    finally:
        dist.destroy_process_group()


def test_shard_covers_everything():
    for n in (0, 1, 7, 100, 101):
        for world in (1, 2, 3, 8):
            spans = [replicas.shard(n, world, r) for r in range(world)]
            assert spans[0][0] == 0 and spans[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(spans, spans[1:]))
            assert max(h - l for l, h in spans) - min(h - l for l, h in spans) <= 1


def test_two_ranks_gloo_equal_single_process(tmp_path, orc):
    world = 2
    mp.spawn(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    got = np.load(tmp_path / "gathered.npy")
    db = synth.uniform_codes(4000, 128, 0)
    qs = synth.uniform_codes(101, 128, 1)
    ids, d = orc.knn(db, qs, 17)
    assert np.array_equal(got[:, :17].view(np.uint32), ids)
    assert np.array_equal(got[:, 17:], d)
    assert float(np.load(tmp_path / "slow.npy")[0]) == 2.0     # the slowest rank's time
