"""Several ranks (CPU, gloo, world size 2).

Replicas: each rank answers its own shard of the queries; gathering the
shards in rank order must give exactly the single-process answer, and the job
time is the slowest rank's.  Database shards: each rank answers every query
over its own id range; the all-gather of the ranks' answers, merged by
(distance, global id), must give the answer over the whole database.  The
per-rank search here is the CPU oracle and the merge a plain sort in the
test (no GPU); on GPUs the ranks run mih_knn and the merge is the library's
mih_merge_topk (tested against the oracle in test_gpu_parity.py).
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


def _db_rank_main(rank, world, port, out_dir):
    import oracle

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        db = synth.uniform_codes(3001, 64, 4)          # ragged: 1501 + 1500
        qs = synth.uniform_codes(40, 64, 5)
        lo, hi = replicas.db_shard(len(db), world, rank)
        ids, d = oracle.knn(db[lo:hi], qs, 23, nthreads=2)          # ids relative to the range
        pi, pd = replicas.all_gather_parts(torch.from_numpy(ids.view(np.int32)), torch.from_numpy(d))
        if rank == 0:
            np.save(os.path.join(out_dir, "ids.npy"), pi.numpy())
            np.save(os.path.join(out_dir, "dist.npy"), pd.numpy())
    finally:
        dist.destroy_process_group()


def test_db_shards_two_ranks_gloo(tmp_path, orc):
    world = 2
    mp.spawn(_db_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    pi = np.load(tmp_path / "ids.npy").view(np.uint32)
    pd = np.load(tmp_path / "dist.npy")
    assert pi.shape == (world, 40, 23)
    bases = [replicas.db_shard(3001, world, r)[0] for r in range(world)]
    assert bases == [0, 1501]
    db = synth.uniform_codes(3001, 64, 4)
    qs = synth.uniform_codes(40, 64, 5)
    want_ids, want_d = orc.knn(db, qs, 23)
    for i in range(40):
        cand = [(int(pd[r, i, j]), int(pi[r, i, j]) + bases[r]) for r in range(world) for j in range(23)
                if pd[r, i, j] >= 0]
        cand.sort()
        assert [c[1] for c in cand[:23]] == list(want_ids[i])
        assert [c[0] for c in cand[:23]] == list(want_d[i])


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
