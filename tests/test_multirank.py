"""Host logic of the multi-rank path, on CPU with world_size 2 over gloo: the batched form
splits its independent pencils over ranks (longest-processing-time shares of M^3, no
exchange on the data path) and reports the slowest rank's time (MAX over ranks)."""
import json
import os
import socket

import pytest

import gep_inputs as gi


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_path):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1504_06443_gb300 import shard_batch
    orders = gi.batch_orders(512, seed=1000)
    mine = shard_batch(orders, world)[rank]
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    load = torch.tensor([float(sum(float(orders[i]) ** 3 for i in mine))], dtype=torch.float64)
    loads = [torch.zeros(1, dtype=torch.float64) for _ in range(world)]
    dist.all_gather(loads, load)
    dist.all_reduce(load, op=dist.ReduceOp.MAX)
    if rank == 0:
        with open(out_path, "w") as f:
            json.dump({"parts": gathered, "loads": [x.item() for x in loads], "max": load.item()}, f)
    dist.destroy_process_group()


def test_batch_shards_over_two_gloo_ranks(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    out = str(tmp_path / "ranks.json")
    mp.spawn(_worker, args=(2, _free_port(), out), nprocs=2, join=True)
    res = json.load(open(out))
    orders = gi.batch_orders(512, seed=1000)
    parts = res["parts"]
    flat = sorted(i for p in parts for i in p)
    assert flat == list(range(len(orders)))  # every pencil exactly once
    loads = [sum(float(orders[i]) ** 3 for i in p) for p in parts]
    assert loads == pytest.approx(res["loads"])
    assert res["max"] == pytest.approx(max(loads))  # the time that is reported
    # LPT: the heaviest share exceeds the mean by at most one pencil
    assert max(loads) <= sum(loads) / 2 + max(float(m) ** 3 for m in orders)


def test_shard_batch_single_rank_and_ties():
    from paper_1504_06443_gb300 import shard_batch
    assert shard_batch([64, 128], 1) == [[0, 1]]
    # equal orders alternate over ranks in index order, lower rank first
    assert shard_batch([100, 100, 100, 100], 2) == [[0, 2], [1, 3]]
    assert shard_batch([], 3) == [[], [], []]


def test_size_buckets_and_autotuner_default():
    """Pencils are grouped by the smallest bucket that holds them (the largest bucket takes
    everything above it); an untuned bucket falls back to the tensor-core engine."""
    import paper_1504_06443_gb300 as gep
    assert [gep._bucket(m) for m in (1, 128, 129, 256, 257, 2048, 2049, 4096, 99999)] == \
        [128, 128, 256, 256, 512, 2048, 4096, 4096, 4096]
    t = gep.Autotuner()
    assert t.precision_for(300) == "fp64_emulated"
    t.choice[512] = "fp64"
    assert t.precision_for(300) == "fp64" and t.precision_for(600) == "fp64_emulated"


def test_make_options_maps_names_to_codes():
    import paper_1504_06443_gb300 as gep
    o = gep.make_options(reducer="explicit_inv", sep="2stage", precision="mixed_refined", want_vectors=False,
                         timers=True, bandwidth=32, refine_iters=3)
    assert (o.reducer, o.sep, o.precision) == (gep.RED_EXPLICIT_INV, gep.SEP_2STAGE, gep.PREC_MIXED_REFINED)
    assert (o.want_vectors, o.timers, o.bandwidth, o.refine_iters) == (0, 1, 32, 3)
    with pytest.raises(KeyError):
        gep.make_options(sep="3stage")
