"""Host logic of runs on several GPUs (paper_1802_10453_gb300.replicas),
tested as two gloo ranks on the CPU: the timing reduction (max over ranks),
the whole-job rate, and the by-matrix split of a batch.  Each rank factors
its own share of a small batch with the oracle (standing in for a GPU), with
no collective on the data path; the test alone gathers the shares to check
that every matrix was factored exactly once and as the whole batch would be."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1802_10453_gb300 import inputs  # noqa: E402
from paper_1802_10453_gb300.replicas import batch_shard, dist_env, max_over_ranks, whole_job_rate  # noqa: E402


def test_batch_shard_covers_every_matrix_once_and_balances_work():
    rng = np.random.default_rng(3)
    for world in (1, 2, 3, 8):
        ns = [int(v) for v in rng.integers(0, 513, size=97)]
        shards = [batch_shard(ns, r, world) for r in range(world)]
        flat = sorted(i for s in shards for i in s)
        assert flat == list(range(len(ns)))
        work = [sum(ns[i] ** 3 for i in s) for s in shards]
        assert max(work) - min(work) <= max(ns) ** 3
    assert batch_shard([], 0, 2) == []
    with pytest.raises(ValueError):
        batch_shard([5], 2, 2)


def test_whole_job_rate_and_env(monkeypatch):
    assert whole_job_rate(10.0, 4, 2.0) == 20.0
    with pytest.raises(ValueError):
        whole_job_rate(1.0, 1, 0.0)
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert dist_env() == (1, 2, 1)
    monkeypatch.setenv("RANK", "2")
    with pytest.raises(ValueError):
        dist_env()
    assert max_over_ranks(3.5, 1) == 3.5


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    r, w, _ = dist_env()
    dist.init_process_group("gloo", rank=r, world_size=w)
    try:
        from oracle import oracle as o
        p = 65521
        ns, rs = inputs.batch_shapes(12, 8, 40, 77)
        mine = batch_shard(ns, r, w)
        ranks = {}
        for i in mine:  # this rank's share, no communication
            n, rk = int(ns[i]), int(rs[i])
            A, _, _ = inputs.planted_matrix(n, rk, rk // 4, p, inputs.batch_seed(77, i))
            ranks[i] = o.ldlt_rpm(np.tril(np.asarray(A, dtype=np.int64)).astype(np.uint32), p)["rank"]
        t = max_over_ranks(1.0 + r, w)                  # the timing reduction
        rate = whole_job_rate(len(mine), w, t)
        gathered = [None] * w
        dist.all_gather_object(gathered, ranks)         # test-side check only
        np.save(os.path.join(out_dir, "r%d.npy" % r),
                np.array([t, rate, len(mine)] + [len(g) for g in gathered], dtype=np.float64))
        if r == 0:
            merged = {}
            for g in gathered:
                assert not set(g) & set(merged)
                merged.update(g)
            np.save(os.path.join(out_dir, "merged.npy"), np.array(sorted(merged.items()), dtype=np.int64))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    r0 = np.load(tmp_path / "r0.npy")
    r1 = np.load(tmp_path / "r1.npy")
    assert r0[0] == r1[0] == 2.0                        # max over ranks
    assert r0[3] + r0[4] == 12                          # every matrix factored once
    merged = np.load(tmp_path / "merged.npy")
    assert [int(i) for i in merged[:, 0]] == list(range(12))
    # the same ranks as factoring the whole batch on one rank
    from oracle import oracle as o
    p = 65521
    ns, rs = inputs.batch_shapes(12, 8, 40, 77)
    for i, rk in merged:
        assert int(rk) == int(rs[int(i)])                # the planted rank
        n = int(ns[int(i)])
        A, _, _ = inputs.planted_matrix(n, int(rs[int(i)]), int(rs[int(i)]) // 4, p, inputs.batch_seed(77, int(i)))
        assert o.ldlt_rpm(np.tril(np.asarray(A, dtype=np.int64)).astype(np.uint32), p)["rank"] == int(rk)
