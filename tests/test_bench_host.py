"""Host logic of bench.py: the multi-rank aggregation (max time, summed units)
over world_size 2 gloo ranks on CPU, the clock / traffic helpers and the
z pass's algorithmic byte count."""
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


def test_z_pass_bytes_against_line_by_line_count():
    """Algorithmic bytes of the force z pass, counted line by line: a z line
    that meets the survey (R > 0 in any subsample) reads its half-spectrum row
    of W; every line writes its row; a and c are read over the line's support,
    from its first observed voxel rounded down to a multiple of four to its
    last observed voxel + 1 rounded up to one (the spans the data check
    kernel records)."""
    import numpy as np

    import bench
    N = 16
    rng = np.random.default_rng(3)
    R = np.zeros((2, N, N, N), dtype=np.float32)
    R[0][rng.random((N, N, N)) < 0.05] = 0.5
    R[1, 3, 4, 7] = 1.0                          # a single voxel: support [4, 8)
    R[1, 5, 5, N - 1] = 1.0                      # the line's last voxel: support ends at N
    R[:, 9, 2, :] = 0.0                          # a line with no support
    row = (N // 2 + 1) * 8
    total, support = 0, 0
    for x in range(N):
        for y in range(N):
            idx = np.flatnonzero((R[:, x, y, :] > 0).any(axis=0))
            total += row                                 # W written
            if idx.size:
                lo, hi = (idx[0] // 4) * 4, -(-(idx[-1] + 1) // 4) * 4
                assert lo <= idx[0] and hi > idx[-1] and hi <= N
                total += row + 2 * 4 * (hi - lo)         # W read, a and c over [lo, hi)
                support += hi - lo
    got, info = bench.z_pass_bytes(R, N)
    assert got == total
    assert info["support_voxels"] == support / N ** 3
    assert info["dense_bytes"] == 2 * row * N * N + 2 * 4 * N ** 3
    # a survey that covers every voxel costs the dense pass
    assert bench.z_pass_bytes(np.ones((1, N, N, N), np.float32), N)[0] == info["dense_bytes"]
