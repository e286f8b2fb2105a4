"""k-point sharding (Sec. 5.2): the partition of the k-points over ranks and the
final gather of eigenvalues and residuals, on CPU at world size 2 and 3 over gloo."""
import json
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_0707_3405_gb300 import kshard  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("nk,ws", [(10, 2), (10, 3), (2, 4), (1, 1), (7, 8), (0, 2)])
def test_partition_covers_every_kpoint_once(nk, ws):
    parts = kshard.partition(nk, ws)
    assert len(parts) == ws
    flat = sorted(k for p in parts for k in p)
    assert flat == list(range(nk))
    sizes = [len(p) for p in parts]
    assert max(sizes) - min(sizes) <= 1          # equal costs: counts differ by at most one
    assert all(p == sorted(p) for p in parts)


def test_partition_balances_uneven_costs():
    # the 10 k-point 72^3 cell has spheres of 24.4k-24.5k plane waves; with one heavy point
    cost = [24483, 24426, 24451, 24440, 24470, 24424, 24435, 24460, 24432, 100000]
    parts = kshard.partition(10, 2, cost)
    loads = [sum(cost[k] for k in p) for p in parts]
    assert 9 in parts[0]                         # heaviest first, to rank 0
    assert abs(loads[0] - loads[1]) <= max(cost)
    assert all(p == sorted(p) for p in parts)    # each rank's list ascending whatever the deal order
    with pytest.raises(ValueError):
        kshard.partition(3, 2, [1.0, 2.0])


def _worker(rank, ws, nk, M, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_0707_3405_gb300 import kshard as ks
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    mine = ks.partition(nk, ws)[rank]
    # each rank "solves" its k-points: eigenvalue j of k-point k = 1000 k + j, residual = -k
    local = {k: (1000.0 * k + np.arange(M), np.full(M, -float(k))) for k in mine}
    eig, res = ks.gather_results(local, nk, ws)
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as f:
        json.dump({"mine": mine, "eig": eig.tolist(), "res": res.tolist()}, f)
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("ws", [2, 3])
def test_gather_reassembles_in_k_order_gloo(tmp_path, ws):
    import torch.multiprocessing as mp
    nk, M = 10, 6
    mp.spawn(_worker, args=(ws, nk, M, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    outs = [json.load(open(tmp_path / f"r{r}.json")) for r in range(ws)]
    owned = sorted(k for o in outs for k in o["mine"])
    assert owned == list(range(nk))
    for o in outs:                               # every rank holds the whole result
        eig, res = np.array(o["eig"]), np.array(o["res"])
        assert eig.shape == (nk, M)
        for k in range(nk):
            assert np.array_equal(eig[k], 1000.0 * k + np.arange(M))
            assert np.all(res[k] == -k)


def _dup_worker(rank, ws, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_0707_3405_gb300 import kshard as ks
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    local = {0: ([1.0], [0.0])}                   # both ranks claim k-point 0; k-point 1 is absent
    if rank == 1:
        local[1] = ([2.0], [0.0])
    try:
        ks.gather_results(local, 2, ws)
        msg = ""
    except RuntimeError as e:
        msg = str(e)
    with open(os.path.join(out_dir, f"d{rank}.txt"), "w") as f:
        f.write(msg)
    dist.barrier()
    dist.destroy_process_group()


def test_gather_rejects_a_kpoint_solved_twice_gloo(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_dup_worker, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        assert "two ranks" in (tmp_path / f"d{r}.txt").read_text()


def test_gather_rejects_missing_and_duplicate_kpoints():
    with pytest.raises(RuntimeError):
        kshard.gather_results({0: ([1.0], [0.0])}, 2, 1)
    eig, res = kshard.gather_results({1: ([2.0], [0.5]), 0: ([1.0], [0.0])}, 2, 1)
    assert eig.tolist() == [[1.0], [2.0]] and res.tolist() == [[0.0], [0.5]]
