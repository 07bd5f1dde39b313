"""The replica split over ranks (one process per GPU, independent instances),
on two CPU ranks of a gloo process group: the ranks' shares partition the
global batch, each rank's generated instances are the global batch's
instances of its share, and the timing reduction returns the slowest rank's
values to every rank."""
import os
import socket

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as tmp  # noqa: E402

from paper_1205_4139_gb300 import replicas  # noqa: E402

WORLD, PER_RANK = 2, 3
SHAPE = dict(kind="dft", N=64, M=24, K=3, snr_db=40.0, prec="fp32")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        idx = list(replicas.shard(rank, WORLD, PER_RANK))
        inst = synth.make_batch(**SHAPE, B=PER_RANK, seed=replicas.shard_seed(rank, PER_RANK), omega_seed=0)
        # every rank reports its share, its instances and a distinct "time"
        times = [10.0 * (rank + 1), 5.0 - rank]
        red = replicas.max_over_ranks(times)
        gathered = [None] * WORLD
        dist.all_gather_object(gathered, {"idx": idx, "Y": inst["Y"], "omega": inst["omega"], "red": red})
        if rank == 0:
            np.save(os.path.join(out_dir, "ok.npy"), np.array([1]))
            torch.save(gathered, os.path.join(out_dir, "gathered.pt"))
    finally:
        dist.destroy_process_group()


def test_replica_split_two_gloo_ranks(tmp_path):
    tmp.spawn(_rank_main, args=(_free_port(), str(tmp_path)), nprocs=WORLD, join=True)
    gathered = torch.load(os.path.join(tmp_path, "gathered.pt"), weights_only=False)
    idx = [i for g in gathered for i in g["idx"]]
    assert sorted(idx) == list(range(WORLD * PER_RANK)) and len(set(idx)) == len(idx)
    full = synth.make_batch(**SHAPE, B=WORLD * PER_RANK, seed=0)
    for g in gathered:
        assert np.array_equal(g["omega"], full["omega"])
        assert np.array_equal(g["Y"], full["Y"][g["idx"]])
        assert g["red"] == [20.0, 5.0]  # the slowest rank's value in each slot


def _argmax_rank(rank, port, out_dir, hs):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=WORLD)
    try:
        res = []
        for h in hs:
            n = len(h) // WORLD
            sl = h[rank * n:(rank + 1) * n]
            a = np.abs(sl) ** 2
            loc = int(np.flatnonzero(a == a.max())[0])  # lowest j at the slice's maximum
            res.append(replicas.argmax_over_ranks(float(a.max()), rank * n + loc))
        gathered = [None] * WORLD
        dist.all_gather_object(gathered, res)
        if rank == 0:
            torch.save(gathered, os.path.join(out_dir, "argmax.pt"))
    finally:
        dist.destroy_process_group()


def test_argmax_over_two_gloo_ranks(tmp_path):
    """One instance sharded by output index over two ranks: the exchanged
    arg-max equals the arg-max of the whole vector, with ties to the lower
    index across the ranks' slices."""
    rng = np.random.default_rng(3)
    h1 = rng.standard_normal(64) + 1j * rng.standard_normal(64)
    h2 = np.zeros(64)
    h2[[7, 40]] = 2.0          # equal maxima in both slices: j = 7 wins
    h3 = np.zeros(64)
    h3[[45, 50]] = -3.0        # both in rank 1's slice: j = 45
    hs = [h1, h2, h3]
    tmp.spawn(_argmax_rank, args=(_free_port(), str(tmp_path), hs), nprocs=WORLD, join=True)
    gathered = torch.load(os.path.join(tmp_path, "argmax.pt"), weights_only=False)
    for h, got0, got1 in zip(hs, gathered[0], gathered[1]):
        a = np.abs(h) ** 2
        want = int(np.flatnonzero(a == a.max())[0])
        assert got0 == got1 and got0[1] == want and got0[0] == a.max()


def test_shard_host_rules():
    assert list(replicas.shard(1, 4, 5)) == [5, 6, 7, 8, 9]
    assert replicas.shard_seed(2, 1024) == 2048
    assert replicas.max_over_ranks([1.5, 2.0]) == [1.5, 2.0]  # no process group: unchanged
    with pytest.raises(ValueError):
        replicas.shard(2, 2, 3)
