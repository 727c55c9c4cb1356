"""Row-sharded exact k-NN: two gloo ranks on the CPU (each rank's local search
is the oracle's brute force on its row range) must return the unsharded
oracle answer; on a GPU, shards on one device merge to the unsharded index's
answer."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import datagen
import oracle
from paper_2009_01614_gb300 import shard

N, n = 6000, 64


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, k, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    X = datagen.rows("walk", 60, 0, N, n)
    Q, _ = datagen.queries("walk", 60, N, n, 61, 6, 4, 0.05)
    r0, r1 = shard.shard_range(N, rank, world)

    def local(Qb, kk):
        i, d2 = oracle.bruteforce_knn(X[r0:r1], Qb, kk)
        return i, np.sqrt(d2).astype(np.float32)

    gi, gd = shard.sharded_knn(local, Q, k, N, rank, world)
    np.save(os.path.join(out_dir, "idx_%d.npy" % rank), gi)
    np.save(os.path.join(out_dir, "dist_%d.npy" % rank), gd)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("k", [1, 7])
def test_two_gloo_ranks_merge_to_the_unsharded_answer(tmp_path, k):
    world = 2
    mp.start_processes(_rank_main, args=(world, _free_port(), k, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    X = datagen.rows("walk", 60, 0, N, n)
    Q, _ = datagen.queries("walk", 60, N, n, 61, 6, 4, 0.05)
    ref_i, ref_d2 = oracle.bruteforce_knn(X, Q, k)
    for r in range(world):
        gi = np.load(tmp_path / ("idx_%d.npy" % r))
        gd = np.load(tmp_path / ("dist_%d.npy" % r))
        np.testing.assert_array_equal(gi, ref_i)
        np.testing.assert_allclose(gd, np.sqrt(ref_d2), rtol=1e-6)


def test_merge_orders_ties_by_row():
    i, d = shard.merge_knn([[[5, 9]], [[2, 7]]], [[[1.0, 2.0]], [[1.0, 3.0]]], 3)
    np.testing.assert_array_equal(i, [[2, 5, 9]])
    np.testing.assert_array_equal(d, [[1.0, 1.0, 2.0]])


@pytest.mark.gpu
def test_shards_on_one_gpu_merge_to_the_unsharded_index():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2009_01614_gb300 as pkg
    Nl, nl, S, k = 40000, 256, 3, 5
    X = datagen.rows("walk", 62, 0, Nl, nl)
    Q, _ = datagen.queries("walk", 62, Nl, nl, 63, 8, 4, 0.05)
    full = pkg.Index(torch.from_numpy(X).cuda(), leaf_size=400)
    ref_i, ref_d = full.query_batch(Q, k)
    parts_i, parts_d = [], []
    for s in range(S):
        r0, r1 = shard.shard_range(Nl, s, S)
        ix = pkg.Index(torch.from_numpy(X[r0:r1]).cuda(), leaf_size=400)
        i, d = ix.query_batch(Q, k)
        parts_i.append(i + r0)
        parts_d.append(d)
        ix.close()
    gi, gd = shard.merge_knn(parts_i, parts_d, k)
    np.testing.assert_array_equal(gi, ref_i)
    np.testing.assert_array_equal(gd, ref_d)
