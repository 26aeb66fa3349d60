"""Multi-rank host logic on CPU: world size 2 over gloo (127.0.0.1).

The sharded path gives each rank a contiguous range of spins and sums the ranks' signals once
(§5.3.2: the signal is additive over spin subsets).  Here each rank runs the oracle on its shard,
the signals are summed with the same helper the benchmark uses, and the sum must equal the
oracle's signal of the whole object; the max-over-ranks step time and the weak-scaling seeds are
checked as well.  No GPU is involved.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from paper_1305_6861_gb300 import distributed as D  # noqa: E402
from paper_1305_6861_gb300 import workloads as W  # noqa: E402


def _free_port():
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import signal as oracle_signal

        w = W.config1()
        part = D.shard_phantom(w.phantom, rank, world)
        s = oracle_signal(part, w.sequence)
        sig = torch.from_numpy(np.ascontiguousarray(np.stack([s.real, s.imag], -1).ravel()))
        D.reduce_signal(sig)
        t_max = D.max_over_ranks(1.0 + rank)
        np.save(os.path.join(out_dir, f"rank{rank}.npy"), np.concatenate([sig.numpy(), [t_max, part.n]]))
    finally:
        dist.destroy_process_group()


def test_spin_ranges_partition():
    for n in (0, 1, 7, 4096, 262145):
        for world in (1, 2, 3, 8):
            ranges = [D.spin_range(n, r, world) for r in range(world)]
            assert ranges[0][0] == 0 and ranges[-1][1] == n
            assert all(a[1] == b[0] for a, b in zip(ranges, ranges[1:]))
            sizes = [b - a for a, b in ranges]
            assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        D.spin_range(10, 2, 2)


def test_weak_scaling_seeds_distinct():
    seeds = [D.rank_seed(W.SEED_BASE, 2, r) for r in range(8)]
    assert seeds[0] is None  # rank 0 keeps the config's own seed
    assert len(set(seeds[1:])) == 7 and W.SEED_BASE + 2 not in seeds[1:]


def test_two_gloo_ranks_sum_to_whole_object(tmp_path, oracle_mod):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    ref = oracle_mod.signal(W.config1())
    ref_il = np.stack([ref.real, ref.imag], -1).ravel()
    outs = [np.load(tmp_path / f"rank{r}.npy") for r in range(world)]
    n_total = 0
    for o in outs:
        sig, t_max, n_part = o[:-2], o[-2], int(o[-1])
        assert np.linalg.norm(sig - ref_il) <= 1e-12 * np.linalg.norm(ref_il)
        assert t_max == 2.0  # max over ranks of (1 + rank)
        n_total += n_part
    assert n_total == W.config1().phantom.n
