"""Host logic of bench.py: the multi-rank aggregation (max time, summed units)
over world_size 2 gloo ranks on CPU, and the clock / traffic helpers."""
import os
import socket

import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, q):
    import torch.distributed as dist

    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    secs, units = bench.aggregate(1.0 + rank, 20 * (rank + 1), world)
    q.put((rank, secs, units))
    dist.destroy_process_group()


def test_aggregate_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, secs, units in out:
        assert secs == 2.0          # max over ranks
        assert units == 60.0        # sum over ranks


def test_aggregate_single_rank_is_identity():
    import bench
    assert bench.aggregate(1.5, 7, 1) == (1.5, 7.0)


def test_clock_summary_parsing():
    import bench
    c = bench.ClockSampler(0)
    c.lines = ["0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
               "0, 1995, 2070, 1300.0, 0x4, Not Active, Not Active, Not Active, Active",
               "0, 2010, 2070, 1250.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    s = c.summary()
    assert s["sm_mhz"] == 2010.0 and s["sm_max_mhz"] == 2070.0
    assert s["reasons"] == ["sw_power_cap"]


def test_traffic_is_null_when_sources_changed(tmp_path, monkeypatch):
    import bench
    f = tmp_path / "t.txt"
    f.write_text("kernel_hash = deadbeef\nbytes_per_launch_full = 1\n")
    monkeypatch.setattr(bench, "PROFILE_TRAFFIC", str(f))
    assert bench.read_traffic() is None
    f.write_text(f"kernel_hash = {bench.kernel_hash()}\nbytes_per_launch_full = 123\n")
    assert bench.read_traffic() == 123.0


def test_reference_arm_prints_the_contract_line(monkeypatch, capsys):
    # bench.py --impl reference times the FP64 oracle on the host (no GPU): one
    # JSON line with the arm's metric, unit and direction, a cpu_baseline that
    # describes the run and an e2e object with no host-device bytes; a rank
    # other than 0 under torchrun exits 0 without work.  Run in process on the
    # 32^3 survey (the bench's own 256^3 survey takes minutes to set up here).
    import json

    import bench
    for k in ("RANK", "WORLD_SIZE", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setattr(bench, "WORKLOAD", "survey32")
    argv = ["--impl", "reference", "--steps", "1", "--warmup", "0"]
    assert bench.main(argv) == 0
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC and line["unit"] == bench.UNIT
    assert line["higher_is_better"] is True and line["value"] > 0 and line["steps"] == 1
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] == 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
    assert line["config"]["workload"].startswith("survey32") and "at 32^3 with 1 subsamples" in cb["sample"]
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("LOCAL_RANK", "1")
    assert bench.main(argv) == 0
    assert not capsys.readouterr().out.strip()
