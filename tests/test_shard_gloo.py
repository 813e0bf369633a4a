"""q-parallel pass (paper_2011_01400_gb300/shard.py) on CPU: two gloo ranks on 127.0.0.1.

Each rank adds planted per-q Sigma_c terms for the q points of its part of the partition; after
the sum over ranks every rank must hold the sum over all q, which is known in closed form. The
partition itself must cover the mesh exactly once and balance the work with q = 0 weighted."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist            # noqa: E402
import torch.multiprocessing as mp          # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
from paper_2011_01400_gb300 import shard    # noqa: E402

NK, NSIG, NW = 27, 3, 5


def planted_term(q):
    """Sigma_c term of point q: (q + 1) * (1 + 2i) * B with B[k][n][w] = k + 10 n + 100 w."""
    k, n, w = np.meshgrid(np.arange(NK), np.arange(NSIG), np.arange(NW), indexing="ij")
    return (q + 1) * (1 + 2j) * (k + 10 * n + 100 * w).astype(np.complex128)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        seen = []

        def accumulate(qs, acc):
            seen.extend(qs)
            for q in qs:
                acc += torch.from_numpy(planted_term(q))

        acc = shard.sharded_sigma(accumulate, NK, NSIG, NW, "cpu")
        np.save(os.path.join(out_dir, f"sig{rank}.npy"), acc.numpy())
        np.save(os.path.join(out_dir, f"qs{rank}.npy"), np.array(seen))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_sum_their_q_terms(tmp_path):
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    k, n, w = np.meshgrid(np.arange(NK), np.arange(NSIG), np.arange(NW), indexing="ij")
    total = (NK * (NK + 1) // 2) * (1 + 2j) * (k + 10 * n + 100 * w)     # sum_q (q + 1) = NK (NK + 1) / 2
    qs = [set(np.load(tmp_path / f"qs{r}.npy").tolist()) for r in range(world)]
    assert qs[0].isdisjoint(qs[1]) and qs[0] | qs[1] == set(range(NK))
    assert len(qs[0]) > 0 and len(qs[1]) > 0
    for r in range(world):
        assert np.array_equal(np.load(tmp_path / f"sig{r}.npy"), total)


@pytest.mark.parametrize("n_q,world", [(1, 1), (8, 3), (27, 2), (216, 8), (5, 8)])
def test_partition_covers_the_mesh_once_and_balances(n_q, world):
    parts = shard.q_partition(n_q, world)
    flat = [q for p in parts for q in p]
    assert sorted(flat) == list(range(n_q))
    assert all(p == sorted(p) for p in parts)
    work = [sum(shard.Q0_WEIGHT if q == 0 else 1.0 for q in p) for p in parts]
    assert max(work) - min(work) <= max(1.0, shard.Q0_WEIGHT)
    assert 0 in parts[0]


def test_single_process_needs_no_group():
    acc = shard.sharded_sigma(lambda qs, a: a.add_(len(qs)), 4, 1, 1, "cpu")
    assert float(acc.real.sum()) == 16.0


@pytest.mark.parametrize("nk", [(2, 2, 2), (3, 3, 3), (4, 2, 1), (6, 6, 6), (5, 1, 3)])
def test_minus_q_is_the_mesh_inversion(nk):
    n_q = nk[0] * nk[1] * nk[2]
    assert shard.minus_q(nk, 0) == 0
    for q in range(n_q):
        mq = shard.minus_q(nk, q)
        assert 0 <= mq < n_q and shard.minus_q(nk, mq) == q
        i = (q // (nk[1] * nk[2]), (q // nk[2]) % nk[1], q % nk[2])
        j = (mq // (nk[1] * nk[2]), (mq // nk[2]) % nk[1], mq % nk[2])
        assert all((a + b) % n == 0 for a, b, n in zip(i, j, nk))      # k + (-k) on the mesh


@pytest.mark.parametrize("nk", [(2, 2, 2), (3, 3, 3), (4, 2, 1), (6, 6, 6)])
@pytest.mark.parametrize("world", [1, 2, 3, 8])
def test_pair_partition_keeps_q_and_minus_q_together(nk, world):
    """With time-reversal pairing every rank's list is closed under q -> -q (its q loop computes
    chi0 / eps~ / W^c once per pair), the mesh is covered once, and the ranks' work differs by at
    most one unit."""
    n_q = nk[0] * nk[1] * nk[2]
    parts = shard.q_partition(n_q, world, nk=nk)
    flat = [q for p in parts for q in p]
    assert sorted(flat) == list(range(n_q))
    for p in parts:
        assert p == sorted(p)
        assert all(shard.minus_q(nk, q) in p for q in p)
    units = shard.q_units(n_q, nk)
    cost = {u[0]: shard.unit_cost(u, nk=nk) for u in units}
    work = [sum(cost[u[0]] for u in units if u[0] in p) for p in parts]
    assert max(work) - min(work) <= max(cost.values()) + 1e-12
    # without pairing nothing changes
    assert shard.q_partition(n_q, world) == shard.q_partition(n_q, world, nk=None)
