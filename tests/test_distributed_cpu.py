"""The multi-rank path of bench.py on CPU: two gloo ranks (one process per
rank, as torchrun starts them) go through the barrier, take the maximum of
their timed regions and form the whole-job aggregate; the reference arm runs
on rank 0 only."""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ws, r, _ = bench._dist()
    bench._barrier(ws)
    t_ms = 10.0 + 5.0 * rank                       # rank 1 is the slower one
    t_max = bench._max_over_ranks(t_ms, ws)
    value = bench._aggregate(81920, 20, t_max, ws)
    # the reference arm: rank 0 alone does the work and prints
    class A:
        warmup, steps, ref_rows, leaf, p = 0, 1, 8, 64, 10
    ran = []
    orig = bench.cpu_baseline
    bench.cpu_baseline = lambda mol, rows=None, budget_s=None: ran.append(1) or {
        "value": 1.0, "unit": "Mpanels/s", "cores": 1, "kind": "oracle", "sample": "stub"}
    bench.workload = lambda: None
    try:
        bench.run_reference(A)
    finally:
        bench.cpu_baseline = orig
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"ws": ws, "rank": r, "t_max": t_max, "value": value, "ref_ran": len(ran)}, f)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.spawn(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True)
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    for r, d in enumerate(res):
        assert d["ws"] == 2 and d["rank"] == r
        assert d["t_max"] == 15.0                 # the max over ranks, on every rank
        assert abs(d["value"] - 2 * 81920 * 20 / 15e-3 / 1e6) < 1e-9
    assert res[0]["ref_ran"] == 1 and res[1]["ref_ran"] == 0
