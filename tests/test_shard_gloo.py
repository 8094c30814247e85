"""Multi-rank network inference on CPU: world size 2 over gloo, each rank
running its targets with the oracle's greedy loop; the gathered network must
equal the single-process one, every target inferred exactly once."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle  # noqa: E402
from paper_1807_10459_gb300 import shard, synth  # noqa: E402

KW = dict(n_past=2, min_lag=1, max_lag=2, k=4, n_surr=20, alpha=0.05, seed=3, max_parents=2)


def _select(series, target, **kw):
    r = oracle.select_target(series, target, **kw)
    return dict(parents=r["parents"], steps=r["steps"])


def _series():
    return synth.var_network(n_nodes=4, order=2, T=300, density=0.5, weight=0.6, seed=5).series


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        net = shard.infer_network(_series(), 4, select=_select, **KW)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"),
                np.array([(t, tuple(net[t]["parents"])) for t in sorted(net)], dtype=object),
                allow_pickle=True)
    finally:
        dist.destroy_process_group()


def test_targets_of_rank_partition():
    for n in (0, 1, 5, 50):
        for world in (1, 2, 3, 8):
            parts = [shard.targets_of_rank(n, world, r) for r in range(world)]
            flat = sorted(t for p in parts for t in p)
            assert flat == list(range(n))
    with pytest.raises(ValueError):
        shard.targets_of_rank(4, 2, 2)


def test_two_ranks_over_gloo_match_one_process(tmp_path):
    single = shard.infer_network(_series(), 4, select=_select, **KW)
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    want = [(t, tuple(single[t]["parents"])) for t in sorted(single)]
    for rank in range(2):
        got = np.load(tmp_path / f"rank{rank}.npy", allow_pickle=True).tolist()
        assert [tuple(x) for x in got] == [tuple(x) for x in want]
