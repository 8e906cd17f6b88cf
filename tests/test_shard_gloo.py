"""Multi-rank path of the batched form on CPU: two gloo ranks each take
their share of the graphs (longest-processing-time by stored edges), cluster
it (the oracle stands in for the GPU step here), and rank 0 gathers the
results; they must equal a single-process run graph for graph."""
import os

import numpy as np
import pytest

import graphgen as gg
from paper_2608_01503_gb300 import shard


def test_assign_covers_every_item_once_and_balances():
    rng = np.random.default_rng(0)
    w = rng.integers(1, 1000, size=500).tolist()
    for world in (1, 2, 3, 8):
        parts = shard.assign(w, world)
        assert sorted(i for p in parts for i in p) == list(range(500))
        loads = [sum(w[i] for i in p) for p in parts]
        # LPT bound: max load <= mean + largest item
        assert max(loads) <= sum(w) / world + max(w)
        assert parts == shard.assign(w, world)  # deterministic


def test_assign_edge_cases():
    assert shard.assign([], 2) == [[], []]
    assert shard.assign([5], 3) == [[0], [], []]
    with pytest.raises(ValueError):
        shard.assign([1], 0)


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist

    import oracle

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    graphs = gg.batched_sbms(24, seed=5, threads=2, n_hi=3000)
    weights = [g.nnz for g in graphs]
    mine = shard.local(weights, rank, world)
    results = []
    for k in mine:
        lab, res, _ = oracle.louvain_plus(graphs[k])
        results.append((lab.tolist(), res["phi"]))
    merged = shard.gather(mine, results)
    if rank == 0:
        import pickle

        with open(os.path.join(out_dir, "merged.pkl"), "wb") as f:
            pickle.dump(merged, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_match_single_process(tmp_path):
    import socket

    import torch.multiprocessing as mp

    import oracle

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    import pickle

    merged = pickle.load(open(tmp_path / "merged.pkl", "rb"))
    graphs = gg.batched_sbms(24, seed=5, threads=2, n_hi=3000)
    assert len(merged) == len(graphs)
    for g, (lab, phi) in zip(graphs, merged):
        ref, res, _ = oracle.louvain_plus(g)
        assert lab == ref.tolist() and phi == res["phi"]
