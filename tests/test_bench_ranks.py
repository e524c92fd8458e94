"""The multi-GPU path of bench.py on the CPU: two ranks over gloo (world size 2).

Knots are independent problems, so bench.py shards them by seed with no data-path
collective; the only collective is the max over ranks of the step time.  Here each
rank plans its own shard on a host-only context and reports a stand-in step time; the
reduction, the whole-job rate and the disjointness of the shards are checked."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, outdir):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import paper_1807_02119_gb300 as pk
    knots = bench.workload(rank, n=2)
    ctx = pk.Context(-1)
    plans = [pk.Plan(ctx, pk.Knot.from_pd(ctx, gk.pd, outer=gk.outer), q)
             for gk in knots for q in (2, 3, 5)]
    step_ms = 10.0 + 5.0 * rank                 # stand-in for this rank's measured step
    worst = bench.max_over_ranks(step_ms, dist, "cpu")
    rate = bench.job_rate(world, len(plans), worst)
    seeds = [None] * world
    dist.all_gather_object(seeds, [gk.seed for gk in knots])
    with open(os.path.join(outdir, f"rank{rank}.json"), "w") as f:
        json.dump({"worst": worst, "rate": rate, "evals": len(plans), "seeds": seeds,
                   "shard": bench.shard_seeds(rank)}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_shard_and_reduce(tmp_path):
    mp = pytest.importorskip("torch.multiprocessing")
    world = 2
    mp.spawn(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["worst"] == 15.0                        # the slowest rank's step
        assert r["rate"] == pytest.approx(world * 6 / 0.015)
    s0, s1 = res[0]["shard"], res[1]["shard"]
    assert s0 == list(range(1, 65)) and s1 == list(range(65, 129))
    assert not set(s0) & set(s1)
    assert res[0]["seeds"] == [[1, 2], [65, 66]] == res[1]["seeds"]


def test_reference_arm_other_ranks_exit(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    args = type("A", (), {"qs": "2,3,5", "warmup": 3, "steps": 2, "gpus": 2})()
    bench.run_reference(args)                            # returns at once, prints nothing
    assert capsys.readouterr().out == ""
