"""The multi-rank path of bench.py on CPU: two gloo ranks (one process each, as torchrun
starts them) agree on the job's time (the maximum over ranks) and the whole-job throughput;
the reference arm runs on rank 0 only."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, ws, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(ws), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    import torch.distributed as dist
    import bench
    w, r, loc = bench._dist()
    dist.init_process_group("gloo", rank=r, world_size=w)
    ms = bench._job_ms(dist, 10.0 + 5.0 * r, "cpu")
    mlups = bench._job_mlups(1000, 20, w, ms)
    dist.barrier()
    dist.destroy_process_group()
    out[r] = (w, r, loc, ms, mlups)


def test_two_gloo_ranks_agree_on_job_time_and_value():
    import torch.multiprocessing as mp
    ws = 2
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r, (w, rr, loc, ms, mlups) in res.items():
        assert (w, rr, loc) == (2, r, r)
        assert ms == 15.0                                    # the slower rank's time
        assert mlups == pytest.approx(1000 * 20 * 2 / 15e-3 / 1e6)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    ns = type("A", (), {"gpus": 2, "steps": 1, "warmup": 3, "workload": "c0", "impl": "reference"})()
    assert bench.run_reference(ns) == 0
    assert capsys.readouterr().out == ""
