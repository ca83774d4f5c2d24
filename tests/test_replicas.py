"""Replica coordination across ranks (the benchmark's N > 1 path), on CPU with
gloo and two ranks: barrier, max / sum reductions, the whole-job throughput
and independent white-noise keys per rank."""
import json
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from inputs import philox as px
    import bench
    from paper_2306_15511_gb300.replicas import Replicas, w1_key, w2_key
    rep = Replicas("gloo")
    rep.barrier()
    # rank r "took" 1 + r seconds for 10 (r + 1) iterations
    res = {"rank": rep.rank, "world": rep.world,
           "max": rep.max(1.0 + rank), "sum": rep.sum(10.0 * (rank + 1)),
           "rate": rep.throughput(10.0 * (rank + 1), 1.0 + rank)}
    key = w2_key(rank, 0)
    draw = px.normal_torch(key if key is not None else 3, px.STREAM_W2, 8, 0, torch.device("cpu"))
    gathered = [None] * world
    dist.all_gather_object(gathered, draw.tolist())
    res["draws"] = gathered
    k1 = w1_key(rank, 0)
    d1 = px.normal_torch(k1 if k1 is not None else 3, px.STREAM_W1, 8, 0, torch.device("cpu"))
    g1 = [None] * world
    dist.all_gather_object(g1, d1.tolist())
    res["draws_w1"] = g1
    # the bench's whole-job timing: rank r ran 4 steps of 100 (1 + r) ms with 40 iterations each
    ms, total, value = bench.rank_summary(rep, 100.0 * (1 + rank), 40.0 * 4, 4)
    res["bench"] = [ms, total, value]
    rep.barrier()
    rep.close()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)


def test_two_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mp.start_processes(_worker, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r, x in enumerate(res):
        assert x["rank"] == r and x["world"] == world
        assert x["max"] == 2.0                      # slowest rank's time
        assert x["sum"] == 30.0                     # all ranks' iterations
        assert x["rate"] == pytest.approx(15.0)     # whole-job rate = 30 / 2
    d0, d1 = np.array(res[0]["draws"][0]), np.array(res[0]["draws"][1])
    assert not np.allclose(d0, d1)                  # independent chains per rank
    assert res[0]["draws"] == res[1]["draws"]       # every rank saw the same gather
    w0, w1 = np.array(res[0]["draws_w1"][0]), np.array(res[0]["draws_w1"][1])
    assert not np.allclose(w0, w1)                  # harmonic white noise differs too
    for x in res:
        ms, total, value = x["bench"]
        assert ms == 200.0 and total == 320.0
        assert value == pytest.approx(320.0 / 0.8)  # all ranks' iterations / slowest rank's time


def _launched(out_dir):
    from paper_2306_15511_gb300.replicas import Replicas
    rep = Replicas("gloo")
    total = rep.sum(1.0 + rep.rank)
    rep.close()
    with open(os.path.join(out_dir, f"launched{rep.rank}.json"), "w") as f:
        json.dump({"rank": rep.rank, "world": rep.world, "local": rep.local, "sum": total}, f)


def test_launch_local_spawns_ranks(tmp_path):
    """The bench's own launcher for --gpus N outside torchrun: N spawned ranks
    with the torchrun environment."""
    from paper_2306_15511_gb300.replicas import launch_local
    launch_local(2, _launched, (str(tmp_path),))
    res = [json.load(open(tmp_path / f"launched{r}.json")) for r in range(2)]
    for r, x in enumerate(res):
        assert x == {"rank": r, "world": 2, "local": r, "sum": 3.0}


def test_single_rank_needs_no_process_group(monkeypatch):
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    from paper_2306_15511_gb300.replicas import Replicas, w2_key
    rep = Replicas("gloo")
    assert (rep.rank, rep.world) == (0, 1)
    assert rep.max(3.5) == 3.5 and rep.sum(4.0) == 4.0 and rep.throughput(8.0, 2.0) == 4.0
    rep.barrier()
    rep.close()
    assert w2_key(0, 3) is None and w2_key(1, 0) != w2_key(2, 0) and w2_key(1, 0) != w2_key(1, 1)
    from paper_2306_15511_gb300.replicas import w1_key
    assert w1_key(0, 3) is None and w1_key(1, 0) != w1_key(2, 0) and w1_key(1, 0) != w2_key(1, 0)
