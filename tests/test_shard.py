"""Row-sharded exact k-NN: two gloo ranks on the CPU (each rank's local search
is the oracle's brute force on its row range) must return the unsharded
oracle answer, including a planted cross-shard near-tie: two rows on different
shards whose fp32 distances to the query are equal while their FP64 squared
distances differ, the higher row being the nearer.  On a GPU, shards on one
device, each answered by its own index with isax_exact_d2 distances, merge to
the oracle's answer."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import datagen
import oracle
from paper_2009_01614_gb300 import shard

N, n = 6000, 64
NEAR_LOW, NEAR_HIGH = 100, 4000  # rows on shards 0 and 1 of 2


def _collection():
    """Random walks with two planted rows near the zero query: |x|^2 = 1 + 2^-24
    (row NEAR_LOW) and 1 + 2^-26 (row NEAR_HIGH), both exactly representable and
    both at fp32 distance 1.0f; every walk is at distance 8 (z-normalised)."""
    X = datagen.rows("walk", 60, 0, N, n).copy()
    X[NEAR_LOW] = 0.0
    X[NEAR_LOW, 0], X[NEAR_LOW, 1] = 1.0, 2.0 ** -12
    X[NEAR_HIGH] = 0.0
    X[NEAR_HIGH, 0], X[NEAR_HIGH, 1] = 1.0, 2.0 ** -13
    Q, _ = datagen.queries("walk", 60, N, n, 61, 6, 4, 0.05)
    Q = np.concatenate([Q, np.zeros((1, n), np.float32)])
    return X, Q


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
    X, Q = _collection()
    r0, r1 = shard.shard_range(N, rank, world)

    def local(Qb, kk):
        i, d2 = oracle.bruteforce_knn(X[r0:r1], Qb, kk)
        return i, np.sqrt(d2).astype(np.float32), d2

    gi, gd, gd2 = shard.sharded_knn(local, Q, k, N, rank, world)
    np.save(os.path.join(out_dir, "idx_%d.npy" % rank), gi)
    np.save(os.path.join(out_dir, "d2_%d.npy" % rank), gd2)
    dist.barrier()
    dist.destroy_process_group()


def test_planted_rows_tie_in_fp32_but_not_in_fp64():
    X, Q = _collection()
    _, d2 = oracle.bruteforce_knn(X, Q[-1:], 2)
    assert d2[0, 0] == 1.0 + 2.0 ** -26 and d2[0, 1] == 1.0 + 2.0 ** -24
    assert np.float32(np.sqrt(d2[0, 0])) == np.float32(np.sqrt(d2[0, 1])) == np.float32(1.0)


@pytest.mark.parametrize("k", [1, 7])
def test_two_gloo_ranks_merge_to_the_unsharded_answer(tmp_path, k):
    world = 2
    assert shard.shard_range(N, 0, world)[0] <= NEAR_LOW < shard.shard_range(N, 0, world)[1]
    assert shard.shard_range(N, 1, world)[0] <= NEAR_HIGH < shard.shard_range(N, 1, world)[1]
    mp.start_processes(_rank_main, args=(world, _free_port(), k, str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    X, Q = _collection()
    ref_i, ref_d2 = oracle.bruteforce_knn(X, Q, k)
    assert ref_i[-1, 0] == NEAR_HIGH
    for r in range(world):
        gi = np.load(tmp_path / ("idx_%d.npy" % r))
        gd2 = np.load(tmp_path / ("d2_%d.npy" % r))
        np.testing.assert_array_equal(gi, ref_i)
        np.testing.assert_array_equal(gd2, ref_d2)


def test_merge_orders_by_fp64_then_row():
    # rows 5 and 2 tie in fp32 (1.0) but not in FP64: the nearer (5) comes first;
    # rows 9 and 7 tie exactly: the lower row (7) comes first
    i, d, d2 = shard.merge_knn([[[5, 9]], [[2, 7]]], [[[1.0, 2.0]], [[1.0, 2.0]]],
                               [[[1.0 + 2.0 ** -26, 4.0]], [[1.0 + 2.0 ** -24, 4.0]]], 4)
    np.testing.assert_array_equal(i, [[5, 2, 7, 9]])
    np.testing.assert_array_equal(d, [[1.0, 1.0, 2.0, 2.0]])


def test_merge_by_fp32_distance_would_pick_the_wrong_row():
    # the ordering the merge replaces: (fp32 distance, row) takes the lower row
    # of an fp32 tie, which is not the definition's nearest here
    rows = np.array([NEAR_LOW, NEAR_HIGH])
    dist32 = np.array([1.0, 1.0], np.float32)
    assert rows[np.lexsort((rows, dist32))][0] == NEAR_LOW
    i, _, _ = shard.merge_knn([[[NEAR_LOW]], [[NEAR_HIGH]]], [[[1.0]], [[1.0]]],
                              [[[1.0 + 2.0 ** -24]], [[1.0 + 2.0 ** -26]]], 1)
    assert i[0, 0] == NEAR_HIGH


@pytest.mark.gpu
def test_shards_on_one_gpu_merge_to_the_oracle_answer():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    import __graft_entry__
    __graft_entry__.build()
    import paper_2009_01614_gb300 as pkg
    X, Q = _collection()
    S = 2
    for k in (1, 5):
        ref_i, ref_d2 = oracle.bruteforce_knn(X, Q, k)
        parts_i, parts_d, parts_d2 = [], [], []
        for s in range(S):
            r0, r1 = shard.shard_range(N, s, S)
            for in_place in (False, True):
                ix = pkg.Index(torch.from_numpy(X[r0:r1].copy()).cuda(), leaf_size=200,
                               rows_in_place=in_place)
                i, d = ix.query_batch(Q, k)
                d2 = ix.exact_d2(Q, i)
                ix.close()
                if in_place:
                    np.testing.assert_array_equal(d2, prev_d2)
                prev_d2 = d2
            parts_i.append(i + r0)
            parts_d.append(d)
            parts_d2.append(d2)
        gi, gd, gd2 = shard.merge_knn(parts_i, parts_d, parts_d2, k)
        np.testing.assert_array_equal(gi, ref_i)
        np.testing.assert_array_equal(gd2, ref_d2)  # isax_exact_d2 is the definition, bit for bit
        np.testing.assert_allclose(gd, np.sqrt(ref_d2), rtol=1e-5, atol=0)
        assert gi[-1, 0] == NEAR_HIGH
