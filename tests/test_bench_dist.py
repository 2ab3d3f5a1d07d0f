"""The N > 1 path of bench.py (one replica of the workload per rank): the job's
step time is the slowest rank's and the throughput counts the work of all
ranks.  Two gloo ranks on the CPU, rendezvous on 127.0.0.1."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, ms_per_rank, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    ms = bench.max_over_ranks(ms_per_rank[rank], dist, "cpu")
    out[rank] = (ms, bench.job_throughput(1000, world, ms))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_all_work():
    world = 2
    ms_per_rank = [10.0, 15.0]
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, _free_port(), ms_per_rank, out), nprocs=world, join=True)
        res = dict(out)
    for r in range(world):
        ms, value = res[r]
        assert ms == 15.0
        assert value == pytest.approx(2 * 1000 / 0.015)


def test_single_process_needs_no_group():
    import bench

    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_throughput(500, 1, 2.0) == pytest.approx(250000.0)


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")

    class Args:
        workload, steps, warmup, gpus = "sph17", 1, 1, 2

    bench.run_reference(Args())
    assert capsys.readouterr().out == ""


def test_traffic_is_taken_only_from_a_capture_of_the_current_source(tmp_path, monkeypatch):
    """roofline.traffic scales the committed DRAM bytes per segment to a launch,
    and is withheld ("stale") once the march source differs from the one captured."""
    import hashlib
    import json

    import bench

    d = json.load(open(os.path.join(bench.ROOT, "profiles", "march_sw_traffic.json")))
    src = open(bench.MARCH_SRC, "rb").read()
    value, why = bench.ncu_traffic(1.0e6)
    if d["source_sha256"] == hashlib.sha256(src).hexdigest():
        assert value == pytest.approx(d["dram_bytes_per_segment"] * 1.0e6)
        assert why == d["capture"]
    else:
        assert (value, why) == (None, "stale")
    edited = tmp_path / "fs_sw.cu"
    edited.write_bytes(src + b"\n// edited\n")
    monkeypatch.setattr(bench, "MARCH_SRC", str(edited))
    assert bench.ncu_traffic(1.0e6) == (None, "stale")


def test_peak_falls_back_without_measured_peaks(tmp_path, monkeypatch):
    import json

    import bench

    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    assert bench.hbm_peak() == (bench.DEFAULT_HBM_FALLBACK, "fallback")
    (tmp_path / "MEASURED_PEAKS.json").write_text(json.dumps({"hbm_gbs": 6500.0}))
    assert bench.hbm_peak() == (6500.0, "measured")
