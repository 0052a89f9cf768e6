#!/usr/bin/env python
"""Throughput of the sampler's hot path on GB300.

One step = one full Gibbs iteration of the multiple-block scan at 256^3
(L = 1000 Mpc/h, six luminosity subsamples, 32 k bins): an HMC move of the
density field with 20 leapfrog steps, the power-spectrum draw, the P-delta jump
(10 leapfrog steps in ln P), the bias and normalisation draws and the rebuild of
the local fields.  The metric counts the density-field leapfrog steps (20 per
step); everything else in the iteration is inside the timed region too.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) every rank runs its own chain on its own GPU (replicas:
the single-chain path has no data-parallel split), the time is the maximum over
ranks and the value the total over ranks.  Rank 0 prints one JSON line.
"""
import argparse
import hashlib
import json
import math
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "HMC leapfrog steps/sec and P(k) effective samples/sec at 256³ vs plain FP32"
UNIT = "leapfrog steps/s"
WORKLOAD = "survey256"
PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "xleap_survey256_traffic.txt")
KERNEL_SOURCES = [os.path.join(ROOT, "paper_1306_1821_gb300", "csrc", f)
                  for f in ("bps_passes.cu", "bps_passes.cuh", "bps_common.cuh")]
XPASS_END = b"// ------------------------------------------------------------------ y pass\n"
KERNEL_NAMES = ["x pass (kick+drift+IFFT_x)", "y pass inverse", "z pass (C2R, local force, R2C)", "y pass forward"]
PROFILE_EVERY = 10      # one event-timed iteration per this many in the timed region


# ---------------------------------------------------------------- helpers
def kernel_hash():
    """Hash of the x-pass kernel's sources: bps_passes.cu up to the y-pass banner
    (the pass modes, arguments, helpers and the x-pass kernel) and the two
    headers it includes."""
    h = hashlib.sha256()
    for p in KERNEL_SOURCES:
        with open(p, "rb") as f:
            data = f.read()
        if p.endswith("bps_passes.cu"):
            b = data.find(XPASS_END)
            if b > 0:
                data = data[:b]
        h.update(data)
    return h.hexdigest()[:16]


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(seconds, units, world_size, device=None):
    """(max seconds over ranks, sum of units over ranks); identity for one rank."""
    if world_size <= 1:
        return float(seconds), float(units)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(seconds)], dtype=torch.float64, device=device)
    u = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index):
        self.dev = device_index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "100", "-i", str(self.dev)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        time.sleep(0.3)
        return self

    def __exit__(self, *a):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.2)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unavailable"], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def z_pass_bytes(R, N):
    """Algorithmic bytes of one force z pass on this survey.  a and c vanish
    outside the voxels with R > 0, so the pass needs: W read on the z lines that
    meet the survey, W written on every line, and a and c over each line's
    support [lo, hi) (its first and last observed voxel, widened to multiples of
    four floats for 16-byte copies)."""
    import numpy as np
    obs = (np.asarray(R) > 0).any(axis=0).reshape(N * N, N)
    has = obs.any(axis=1)
    first = np.argmax(obs, axis=1)
    last = N - 1 - np.argmax(obs[:, ::-1], axis=1)
    lo = first & ~3
    hi = (last + 4) & ~3
    span = np.where(has, hi - lo, 0).astype(np.int64)
    row = (N // 2 + 1) * 8
    total = row * (int(has.sum()) + N * N) + 2 * 4 * int(span.sum())
    info = {"lines_with_support": float(has.mean()), "support_voxels": float(span.sum()) / N ** 3,
            "dense_bytes": 2 * row * N * N + 2 * 4 * N ** 3}
    return total, info


def read_traffic():
    """DRAM bytes per x-pass launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    if not os.path.exists(PROFILE_TRAFFIC):
        return None
    kv = {}
    with open(PROFILE_TRAFFIC) as f:
        for ln in f:
            if "=" in ln and not ln.startswith("#"):
                k, v = ln.split("=", 1)
                kv[k.strip()] = v.strip()
    if kv.get("kernel_hash") != kernel_hash():
        return None
    try:
        return float(kv["bytes_per_launch_full"])
    except (KeyError, ValueError):
        return None


# ---------------------------------------------------------------- oracle (CPU) leg
def cpu_model():
    """The host CPU's model name (/proc/cpuinfo, else lscpu, else the machine type)."""
    import platform
    import subprocess
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.machine()


def host_info():
    return {"threads_used": 1, "host_cores": os.cpu_count(), "cpu_model": cpu_model(),
            "note": "the oracle is plain numpy: its FFTs and loops run on one host thread"}


def oracle_gibbs_iteration_seconds(name="survey128"):
    """One full Gibbs iteration (HMC with its leapfrog steps, P draw, jump, b and
    Nbar draws, rebuild) of the FP64 oracle on the named workload."""
    from oracle import grid, gibbs
    from paper_1306_1821_gb300 import inputs
    wl = inputs.WORKLOADS[name]
    _, counts, R = inputs.make_survey(wl)
    geom = grid.Geometry(wl.N, wl.box, wl.n_bins)
    P, b, nbar = inputs.initial_state(wl)
    ch = gibbs.Chain(geom, counts, R, P, b, nbar, alpha=wl.alpha, n_leapfrog=wl.n_leapfrog, eps_max=wl.eps_max,
                     jump=True, jump_leapfrog=wl.jump_leapfrog, jump_eps_max=wl.jump_eps_max,
                     fixed_bias=wl.fixed_bias, seed=1)
    t0 = time.perf_counter()
    ch.iterate()
    return time.perf_counter() - t0, wl


def oracle_leapfrog_rate(wl, counts, R, n_steps=4):
    """The FP64 oracle's leapfrog on host cores: n_steps leapfrog steps of one
    trajectory (n_steps + 1 force evaluations, so the first one is amortised)
    at the full workload."""
    import numpy as np

    from oracle import grid, hmc, model
    from paper_1306_1821_gb300 import inputs
    geom = grid.Geometry(wl.N, wl.box, wl.n_bins)
    P, b, nbar = inputs.initial_state(wl)
    a, c = model.local_fields(counts, R, b, nbar)
    M, invM = model.mass_diag(geom, P, float(a.mean()))
    dh = np.zeros((wl.N, wl.N, wl.N // 2 + 1), dtype=np.complex128)
    p0 = hmc.draw_momentum(geom, M, 1, 0)
    t0 = time.perf_counter()
    hmc.leapfrog(geom, dh, p0, 0.1, n_steps, P, a, c, invM)
    dt = time.perf_counter() - t0
    return n_steps / dt, dt


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_1306_1821_gb300 import inputs
    wl = inputs.WORKLOADS[WORKLOAD]
    _, counts, R = inputs.make_survey(wl)
    steps = min(args.steps, 8)
    warm = min(args.warmup, 1)
    L = 3
    for _ in range(warm):
        oracle_leapfrog_rate(wl, counts, R, n_steps=1)
    tot = 0.0
    for _ in range(steps):
        _, dt = oracle_leapfrog_rate(wl, counts, R, n_steps=L)
        tot += dt
    value = steps * L / tot
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000.0 * tot / (steps * L),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(wl, "cpu"),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{steps} trajectories of {L} leapfrog steps ({L + 1} force evaluations each) "
                                   f"at {wl.N}^3 with {wl.n_sub} subsamples, numpy FP64 FFT, one thread, "
                                   f"after {warm} warm-up", **host_info()},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def config_dict(wl, where):
    return {"workload": f"{wl.name}: {wl.N}^3 grid, L={wl.box:g} Mpc/h, {wl.n_sub} subsamples, "
                        f"{wl.n_bins} k bins, {wl.n_leapfrog} leapfrog steps per HMC move, jump on "
                        f"({wl.jump_leapfrog} steps), one Gibbs iteration per step",
            "grid": wl.N, "box_mpc_h": wl.box, "n_sub": wl.n_sub, "n_bins": wl.n_bins,
            "leapfrog_per_step": wl.n_leapfrog, "jump_leapfrog_per_step": wl.jump_leapfrog,
            "l2": "inputs larger than L2 (each half spectrum 68 MB; a, c 67 MB each)",
            "parallelism": "replicas (one chain per GPU)" if where != "cpu" else "single host thread"}


# ---------------------------------------------------------------- GPU leg
def gpu_mock_timing(s, wl, stream, dev, host_seconds):
    """The benchmark survey made on the device (Sec. 5 mock: true field, cap x
    radial response, Poisson counts of every subsample) timed with CUDA events
    on the library's stream, beside the host recipe's wall time."""
    import numpy as np
    import torch

    from paper_1306_1821_gb300 import bps, inputs
    N, box = wl.N, wl.box
    n2 = np.arange(3 * (N // 2) ** 2 + 1, dtype=np.float64)
    P = inputs.true_spectrum(2.0 * np.pi * np.sqrt(n2) / box, N, box)
    P[0] = 0.0
    n_r = 4097
    r = np.arange(n_r) * (box / 2 / (n_r - 1))
    table = np.broadcast_to(np.exp(-(r / wl.r0) ** 2), (wl.n_sub, n_r)).copy()
    with torch.cuda.stream(stream):
        d = torch.empty((N, N, N), dtype=torch.float32, device=dev)
        Rd = torch.empty((wl.n_sub, N, N, N), dtype=torch.float32, device=dev)
        c = torch.empty((wl.n_sub, N, N, N), dtype=torch.int32, device=dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    ms = []
    for rep in range(3):
        e0.record(stream)
        bps.bps_mock_field(s.ctx, 100 + rep, P, d)
        bps.bps_mock_response(s.ctx, wl.f_sky, (0.0, 0.0, 1.0), table, Rd)
        bps.bps_mock_counts(s.ctx, 100 + rep, d, Rd, wl.b, wl.nbar, 0, c)
        e1.record(stream)
        stream.synchronize()
        ms.append(e0.elapsed_time(e1))
    total = int(c.sum().item())
    del d, Rd, c
    return {"gpu_ms": min(ms[1:]), "host_s": host_seconds, "galaxies": total,
            "what": f"{N}^3 true field, cap x radial response and Poisson counts of {wl.n_sub} subsamples: "
                    f"on the device (bps_mock_*, CUDA events, best of 2 after one warm-up) and by the host "
                    f"numpy recipe (inputs.make_survey, wall time)"}


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if ws > 1 else 0)
    torch.cuda.set_device(dev)
    from paper_1306_1821_gb300 import bps, inputs
    if not os.path.exists(bps.LIB_PATH):
        from paper_1306_1821_gb300 import build as b
        b.build()
    bps.load()

    wl = inputs.WORKLOADS[WORKLOAD]
    t_host = time.perf_counter()
    delta, counts, R = inputs.make_survey(wl, seed=wl.seed + rank)
    t_host = time.perf_counter() - t_host
    P0, b0, nbar0 = inputs.initial_state(wl)
    stream = torch.cuda.Stream(device=dev)
    s = bps.Sampler(wl.N, wl.box, wl.n_sub, wl.n_bins, stream=stream, n_leapfrog=wl.n_leapfrog,
                    eps_max=wl.eps_max, jump=1, jump_leapfrog=wl.jump_leapfrog, jump_eps_max=wl.jump_eps_max,
                    fixed_bias_index=wl.fixed_bias, seed=1 + rank)
    with torch.cuda.stream(stream):
        cnt_d = torch.from_numpy(counts).to(dev)
        R_d = torch.from_numpy(R).to(dev)
        d_d = torch.from_numpy(delta.astype(np.float32)).to(dev)
    stream.synchronize()
    bps.bps_set_data(s.ctx, cnt_d, R_d)
    bps.bps_set_state(s.ctx, d_d, P0, b0, nbar0, 0)
    del cnt_d, R_d, d_d
    mock_timing = gpu_mock_timing(s, wl, stream, dev, t_host)

    # warm-up iterations (also moves the chain off its starting point)
    if args.warmup > 0:
        bps.bps_gibbs_iterate(s.ctx, args.warmup)

    # ---- device-timed region: K Gibbs iterations, inputs resident in HBM.  Every
    # PROFILE_EVERY-th iteration replays the iteration's graph with event-record
    # nodes around the leapfrog kernels; the others replay the plain graph.
    bps.bps_profile_read(s.ctx)
    l0 = bps.bps_kernel_launches(s.ctx)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    recs = []
    with ClockSampler(dev.index) as clk:
        if ws > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize(dev)
        e0.record(stream)
        done = 0
        while done < args.steps:
            n = min(PROFILE_EVERY, args.steps - done)
            bps.bps_profile(s.ctx, 1)
            recs.append(bps.bps_gibbs_iterate(s.ctx, 1, s.rec_len))
            bps.bps_profile(s.ctx, 0)
            if n > 1:
                recs.append(bps.bps_gibbs_iterate(s.ctx, n - 1, s.rec_len))
            done += n
        e1.record(stream)
        torch.cuda.synchronize(dev)
    rec = np.concatenate(recs, 0)
    launches = bps.bps_kernel_launches(s.ctx) - l0
    kms, kn = bps.bps_profile_read(s.ctx)
    local_s = e0.elapsed_time(e1) / 1000.0
    secs, units = aggregate(local_s, args.steps * wl.n_leapfrog, ws, dev)
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()
    acc_rate = float(np.mean(rec[:, -1])) if len(rec) else float("nan")

    # ---- end to end through the public API with host buffers: every step
    # uploads its survey from pinned memory, runs one Gibbs iteration and reads
    # the chain record back.  The upload of step k + 1 is staged
    # (bps_stage_data_host_u16) before step k runs, so it overlaps step k; all
    # uploads and read-backs lie inside the timed region.
    k_e2e = min(args.steps, 40)
    cnt_h = torch.from_numpy(counts.astype(np.uint16)).pin_memory().numpy()   # counts <= 65535: 16-bit upload
    R_h = torch.from_numpy(R).pin_memory().numpy()
    rec_h = torch.zeros(s.rec_len, dtype=torch.float64).pin_memory().numpy()
    # untimed warm-up of this path (the first host upload creates the copy streams)
    for _ in range(2):
        bps.bps_stage_data_host_u16(s.ctx, cnt_h, R_h)
        rec_h[:] = bps.bps_gibbs_iterate(s.ctx, 1, s.rec_len)[0]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    bps.bps_stage_data_host_u16(s.ctx, cnt_h, R_h)
    for k in range(k_e2e):
        if k + 1 < k_e2e:
            bps.bps_stage_data_host_u16(s.ctx, cnt_h, R_h)
        out = bps.bps_gibbs_iterate(s.ctx, 1, s.rec_len)
        rec_h[:] = out[0]
    torch.cuda.synchronize(dev)
    e2e_s = time.perf_counter() - t0
    e2e_secs, e2e_units = aggregate(e2e_s, k_e2e * wl.n_leapfrog, ws, dev)

    # ---- P(k) effective samples per second of this (plain diagonal mass) chain:
    # ESS of ln P_m over a further run of Gibbs iterations, timed with events
    pk = None
    if args.ess_iters > 0:
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize(dev)
        f0.record(stream)
        rec_e = bps.bps_gibbs_iterate(s.ctx, args.ess_iters, s.rec_len)
        f1.record(stream)
        torch.cuda.synchronize(dev)
        pk = pk_ess(rec_e, wl.n_bins, wl.N, f0.elapsed_time(f1) / 1000.0)
        pk["mass"] = "plain diagonal Fourier mass (Eq. Mass_matrix)"

    # ---- what a plain streaming update of this size reaches: torch's in-place
    # scale of a tensor as large as one half spectrum (read + write), CUDA
    # events, L2 flushed before each launch.  Context for the roofline: at
    # tens of microseconds per launch a kernel cannot reach the copy peak.
    stream_ref = None
    if rank == 0:
        S_bytes = wl.N * wl.N * (wl.N // 2 + 1) * 8
        buf = torch.zeros(S_bytes // 4, dtype=torch.float32, device=dev)
        flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
        ts = []
        for i in range(13):
            flush.fill_(i)
            g0 = torch.cuda.Event(enable_timing=True)
            g1 = torch.cuda.Event(enable_timing=True)
            g0.record()
            buf.mul_(1.0000001)
            g1.record()
            torch.cuda.synchronize(dev)
            if i >= 3:
                ts.append(g0.elapsed_time(g1))
        ms = sum(ts) / len(ts)
        stream_ref = {"bytes": 2 * S_bytes, "ms": ms, "GBps": 2 * S_bytes / (ms * 1e-3) / 1e9,
                      "what": "torch in-place scale of one half-spectrum-sized float32 tensor (read + write), "
                              "mean of 10 launches after L2 flush"}
        del buf, flush

    # ---- roofline of the dominant kernel (the x pass), from the live events
    S_c = wl.N * wl.N * (wl.N // 2 + 1) * 8
    z_bytes, z_info = z_pass_bytes(R, wl.N)
    bytes_kind = [6 * S_c, 2 * S_c, z_bytes, 2 * S_c]
    per_launch_ms = [kms[i] / max(kn[i], 1) for i in range(4)]
    shares = [kms[i] / max(sum(kms), 1e-30) for i in range(4)]
    peak, peak_kind = measured_peaks()
    dom = int(np.argmax(kms))
    achieved = bytes_kind[dom] / (per_launch_ms[dom] * 1e-3) / 1e9
    leap_ms = sum(per_launch_ms)
    leap_bytes = 10 * S_c + z_bytes
    traffic = read_traffic() if dom == 0 else None

    if rank == 0:
        line = {
            "metric": METRIC,
            "value": units / secs,
            "unit": UNIT,
            "n_gpus": ws,
            "steps": args.steps,
            "warmup": args.warmup,
            "ms_per_step": 1000.0 * secs / args.steps,
            "higher_is_better": True,
            "scaling": "weak",
            "vs_baseline": None,
            "dtype": "f32",
            "data": "synthetic",
            "config": config_dict(wl, "gpu"),
            "gibbs_iterations_per_s": ws * args.steps / secs,
            "hmc_acceptance": acc_rate,
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": traffic,
                         "kernel": KERNEL_NAMES[dom], "peak_source": f"{peak_kind} hbm_gbs (MEASURED_PEAKS.json)"
                         if peak_kind == "measured" else "fallback 6.8 TB/s",
                         "algorithmic_bytes_per_launch": bytes_kind[dom], "launch_ms": per_launch_ms[dom]},
            "leapfrog_kernels": {KERNEL_NAMES[i]: {"ms": per_launch_ms[i], "timed_launches": int(kn[i]),
                                                   "share": shares[i], "bytes": bytes_kind[i],
                                                   "GBps": bytes_kind[i] / (per_launch_ms[i] * 1e-3) / 1e9,
                                                   **(z_info if i == 2 else {})}
                                 for i in range(4)},
            "profiled_iterations": f"1 in {PROFILE_EVERY} replays a second CUDA graph of the iteration with "
                                   f"event-record nodes around each leapfrog kernel; the rest replay the "
                                   f"iteration's plain graph",
            "leapfrog_roofline": {"bytes": leap_bytes, "ms": leap_ms,
                                  "GBps": leap_bytes / (leap_ms * 1e-3) / 1e9,
                                  "frac": leap_bytes / (leap_ms * 1e-3) / 1e9 / peak},
            "e2e": {"value": e2e_units / e2e_secs, "unit": UNIT,
                    "h2d_bytes_per_step": int(cnt_h.nbytes + R_h.nbytes),
                    "d2h_bytes_per_step": int(8 * s.rec_len),
                    "steps": k_e2e,
                    "pipelined": "each step's survey upload (bps_stage_data_host_u16) runs during the previous "
                                 "step's Gibbs iteration"},
            "gpu_launches": int(launches),
            "clocks": clk.summary(),
            "tuning": {"z_line_pairs": bps.bps_z_line_pairs(s.ctx), "x_pass_variant": bps.bps_x_pass_variant(s.ctx)},
        }
        if pk is not None:
            line["pk_ess"] = pk
        line["mock_generation"] = mock_timing
        if stream_ref is not None:
            stream_ref["x_pass_frac_of_this"] = achieved / stream_ref["GBps"]
            line["streaming_reference"] = stream_ref
        if ws == 1 and not args.no_cpu_baseline:
            v, dt = oracle_leapfrog_rate(wl, counts, R, n_steps=4)
            git, wl_g = oracle_gibbs_iteration_seconds("survey128")
            line["cpu_baseline"] = {"value": v, "unit": UNIT, "cores": 1, "kind": "oracle",
                                    "sample": f"4 leapfrog steps (5 force evaluations) of one trajectory at "
                                              f"256^3 with 6 subsamples, FP64 numpy on one host thread, "
                                              f"{dt:.1f} s; plus one full Gibbs iteration at 128^3",
                                    "s_per_leapfrog": 1.0 / v,
                                    "s_per_gibbs_iteration_128": git,
                                    "gibbs_iteration_128": f"{wl_g.name}: {wl_g.N}^3, {wl_g.n_sub} subsamples, "
                                                           f"{wl_g.n_leapfrog} leapfrog steps, jump on "
                                                           f"({wl_g.jump_leapfrog} steps)",
                                    **host_info()}
        print(json.dumps(line), flush=True)
    s.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------------------- batched chains
def run_batch(args):
    """Aggregate throughput of 96 independent chains on 32^3 / 64^3 / 96^3 grids
    (32 each), one CUDA graph replay per Gibbs iteration of the whole batch."""
    import numpy as np
    import torch

    from paper_1306_1821_gb300 import bps, inputs
    if not os.path.exists(bps.LIB_PATH):
        from paper_1306_1821_gb300 import build as b
        b.build()
    bps.load()
    wls = inputs.batch_workloads()
    stream = torch.cuda.Stream()
    cfg = bps.make_config(16, n_leapfrog=10, eps_max=0.1, jump=1, jump_leapfrog=5, jump_eps_max=0.05,
                          fixed_bias_index=0, seed=1000)
    batch = bps.bps_create_batch([w.N for w in wls], [w.box for w in wls], [w.n_sub for w in wls], cfg, stream)
    t0 = time.time()
    for j, wl in enumerate(wls):
        delta, counts, R = inputs.make_survey(wl)
        P, b, nbar = inputs.initial_state(wl)
        with torch.cuda.stream(stream):
            c_d = torch.from_numpy(counts).cuda()
            r_d = torch.from_numpy(R).cuda()
            d_d = torch.from_numpy(delta.astype(np.float32)).cuda()
        stream.synchronize()
        bps.bps_batch_set_chain(batch, j, c_d, r_d, d_d, P, b, nbar, 0)
    setup_s = time.time() - t0
    bps.bps_batch_gibbs_iterate(batch, max(args.warmup, 3))
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    l0 = bps.bps_kernel_launches(batch)
    with ClockSampler(torch.cuda.current_device()) as clk:
        torch.cuda.synchronize()
        e0.record(stream)
        rec = bps.bps_batch_gibbs_iterate(batch, args.steps, len(wls))
        e1.record(stream)
        torch.cuda.synchronize()
    secs = e0.elapsed_time(e1) / 1000.0
    launches = bps.bps_kernel_launches(batch) - l0
    vox = sum(w.N ** 3 for w in wls)
    per_iter = launches / max(args.steps, 1)
    floor_us = graph_node_floor_us(stream, int(round(per_iter)))
    acc = float(np.mean([rec[:, bps.bps_batch_record_slot(batch, j), 16 + 2 * w.n_sub + 1]
                         for j, w in enumerate(wls)]))
    line = {
        "metric": "aggregate voxel-leapfrog steps/s, 96 batched chains",
        "value": vox * cfg.n_leapfrog * args.steps / secs,
        "unit": "voxel-leapfrogs/s",
        "n_gpus": 1, "steps": args.steps, "warmup": max(args.warmup, 3),
        "ms_per_step": 1000.0 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": "batch96: 32 chains each of 32^3, 64^3, 96^3 (L = 500 N/32 Mpc/h), caps of "
                               "20-60% sky, 1-4 subsamples, 16 bins, 10 leapfrog steps, jump on (5 steps); "
                               "one CUDA graph replay per Gibbs iteration of all chains",
                   "chains": len(wls), "voxels": vox},
        "gibbs_iterations_per_s": len(wls) * args.steps / secs,
        "hmc_acceptance": acc,
        "gpu_launches": int(launches),
        "launch_floor": {"kernels_per_iteration": per_iter, "us_per_graph_node": floor_us,
                         "share_of_iteration": per_iter * floor_us / (1000.0 * 1000.0 * secs / args.steps),
                         "what": "replay time per node of a CUDA graph of as many trivial kernels as one batch "
                                 "iteration launches (torch fill of one element): the most a single persistent "
                                 "kernel could save by removing the launches"},
        "setup_s": setup_s,
        "clocks": clk.summary(),
    }
    print(json.dumps(line), flush=True)
    bps.bps_destroy(batch)
    return 0


def graph_node_floor_us(stream, n_nodes, reps=20):
    """Microseconds per node of a captured graph of n_nodes trivial kernels."""
    import torch
    x = torch.zeros(1, device="cuda")
    g = torch.cuda.CUDAGraph()
    with torch.cuda.stream(stream):
        x.fill_(0.0)
        torch.cuda.synchronize()
        with torch.cuda.graph(g, stream=stream):
            for _ in range(n_nodes):
                x.fill_(1.0)
        g.replay()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            g.replay()
        e1.record(stream)
        torch.cuda.synchronize()
    return 1000.0 * e0.elapsed_time(e1) / (reps * max(n_nodes, 1))


# ---------------------------------------------------------------- learned mass vs plain
def pk_ess(rec, n_bins, N, secs):
    """ESS of ln P_m per bin (Geyer) from a chain record, and ESS/s summaries over
    the bins that lie inside the Nyquist sphere (|n| <= N/2); the corner bins
    beyond it hold only shot-noise-dominated modes."""
    import numpy as np

    from paper_1306_1821_gb300 import diagnostics
    P = rec[:, :n_bins]
    lnP = np.log(P)
    ess = np.array([diagnostics.ess_geyer(lnP[:, m]) for m in range(n_bins)])
    inside = [m for m in range(n_bins) if (m + 1) * math.sqrt(3.0) * N / 2 / n_bins <= N / 2]
    # standard error of each bin's ESS from four consecutive quarters of the
    # chain (their ESS summed estimates the whole chain's; the spread of the
    # quarters gives its error); an ESS below ~50 is itself poorly determined
    q = len(rec) // 4
    seg = np.array([[diagnostics.ess_geyer(lnP[i * q:(i + 1) * q, m]) for i in range(4)] for m in range(n_bins)])
    ess_se = 2.0 * seg.std(1, ddof=1)
    m_min = inside[int(np.argmin(ess[inside]))]
    return {"ess_per_bin": [round(float(e), 1) for e in ess],
            "ess_se_per_bin": [round(float(e), 1) for e in ess_se],
            "bins_inside_nyquist": inside,
            "min_ess_per_s": float(ess[inside].min() / secs),
            "min_ess_bin": int(m_min), "min_ess": float(ess[m_min]), "min_ess_se": float(ess_se[m_min]),
            "min_ess_reliable": bool(ess[m_min] >= 50.0),
            "median_ess_per_s": float(np.median(ess[inside]) / secs),
            "correlation_length_median": float(np.median([diagnostics.correlation_length(lnP[:, m])
                                                          for m in inside])),
            "iterations": int(len(rec)), "seconds": secs,
            "mean_lnP": [round(float(v), 4) for v in np.log(P).mean(0)],
            "sd_lnP": [round(float(v), 4) for v in np.log(P).std(0)]}


DAMPED = 0.6          # damping of the second network arm (it learns 0.6 ln s)
PRECOND_RUNS = {
    # workload: (survey, training surveys, mass bins)
    "precond128": ("survey128", 5000, 64),
    "precond256": ("survey256", 256, 64),
}


def run_precond(args):
    """P(k) effective samples per second of the full sampler with the plain
    diagonal mass and with the trained network mass (gamma = 1, and damped to
    gamma = 0.6), on the 128^3 survey (precond128) or the 256^3 survey of the
    headline (precond256), over several seeds per arm.  The network
    (2 n_bins -> 128 -> 128 -> 64, BF16 operands) is trained on the device on
    statistics of plain chains on random surveys of the same recipe (random caps
    and spectra), made on the device; the benchmark survey itself is held out.
    Equal accuracy: the per-bin posterior means of ln P of each network arm and
    the plain arm, pooled over seeds, must agree within three combined Monte
    Carlo standard errors (reported as the largest z)."""
    import numpy as np
    import torch

    from paper_1306_1821_gb300 import bps, inputs, precond
    if not os.path.exists(bps.LIB_PATH):
        from paper_1306_1821_gb300 import build as b
        b.build()
    bps.load()
    survey, n_train_default, n_mass = PRECOND_RUNS[args.workload]
    n_train = args.train_examples or n_train_default
    wl = inputs.WORKLOADS[survey]
    jeps = 0.15
    t0 = time.time()
    probs = precond.random_problems(wl, n_train, 5000, p_jitter=0.3)
    # chains per batch context: ~200 MB each at 128^3, ~1.6 GB at 256^3
    F, T = precond.measure(probs, n_mass, n_moves=args.stat_moves, burn_in=100, device_mocks=True,
                           chunk=256 if wl.N <= 128 else 48)
    t_stats = time.time() - t0
    nets = {}
    for arm, gamma in (("network", 1.0), ("network_damped", DAMPED)):
        pc = precond.Preconditioner(F.shape[1], n_mass, seed=1)
        loss = pc.fit(F, T, steps=4000, batch=128, damping=gamma)
        nets[arm] = (pc, loss)
    train_s = time.time() - t0
    delta, counts, R = inputs.make_survey(wl)
    P0, b0, n0 = inputs.initial_state(wl)
    cnt = torch.from_numpy(counts).cuda()
    Rt = torch.from_numpy(R).cuda()
    d32 = torch.from_numpy(delta.astype(np.float32)).cuda()
    arms = {a: [] for a in ("plain", "network", "network_damped")}
    lnPs = {a: [] for a in arms}
    for k in range(args.seeds):
        for arm in arms:
            s = bps.Sampler(wl.N, wl.box, wl.n_sub, wl.n_bins, n_leapfrog=wl.n_leapfrog, eps_max=wl.eps_max,
                            jump=1, jump_leapfrog=10, jump_eps_max=jeps, fixed_bias_index=0, seed=3 + 101 * k)
            bps.bps_set_data(s.ctx, cnt, Rt)
            bps.bps_set_state(s.ctx, d32, P0, b0, n0, 0)
            if arm != "plain":
                nets[arm][0].install(s.ctx)
            bps.bps_gibbs_iterate(s.ctx, max(args.warmup, 300))
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize()
            e0.record()
            rec = bps.bps_gibbs_iterate(s.ctx, args.ess_iters, s.rec_len)
            e1.record()
            torch.cuda.synchronize()
            secs = e0.elapsed_time(e1) / 1000.0
            r = pk_ess(rec, wl.n_bins, wl.N, secs)
            r["hmc_acceptance"] = float(np.mean(rec[:, -1]))
            r["ms_per_iteration"] = 1000.0 * secs / args.ess_iters
            r["seed"] = 3 + 101 * k
            s.close()
            arms[arm].append(r)
            lnPs[arm].append(np.log(rec[:, :wl.n_bins]))
    inside = arms["plain"][0]["bins_inside_nyquist"]

    def stats(vals):
        v = np.asarray(vals, dtype=np.float64)
        se = float(v.std(ddof=1) / math.sqrt(len(v))) if len(v) > 1 else None
        return {"per_seed": [round(float(x), 4) for x in v], "mean": float(v.mean()), "se": se}

    summary = {}
    for arm in arms:
        summary[arm] = {"min_ess_per_s": stats([r["min_ess_per_s"] for r in arms[arm]]),
                        "median_ess_per_s": stats([r["median_ess_per_s"] for r in arms[arm]]),
                        "hmc_acceptance": stats([r["hmc_acceptance"] for r in arms[arm]]),
                        "ms_per_iteration": stats([r["ms_per_iteration"] for r in arms[arm]])}
    ratios, accuracy = {}, {}
    for arm in ("network", "network_damped"):
        ratios[arm] = {
            "min_ess_per_s": stats([a["min_ess_per_s"] / p["min_ess_per_s"] for a, p in zip(arms[arm], arms["plain"])]),
            "median_ess_per_s": stats([a["median_ess_per_s"] / p["median_ess_per_s"]
                                       for a, p in zip(arms[arm], arms["plain"])])}
        # equal accuracy, pooled over seeds: per-bin posterior means of ln P
        za = []
        for m in inside:
            mu = [np.mean([x[:, m].mean() for x in lnPs[a]]) for a in (arm, "plain")]
            sd = np.mean([x[:, m].std() for x in lnPs["plain"]])
            ess = [np.sum([r["ess_per_bin"][m] for r in arms[a]]) for a in (arm, "plain")]
            za.append(abs(mu[0] - mu[1]) / (sd * math.sqrt(1.0 / max(ess[0], 1.0) + 1.0 / max(ess[1], 1.0))))
        accuracy[arm] = {"max_z_over_bins": float(np.max(za)), "bins_over_3": int(np.sum(np.array(za) > 3.0))}
    line = {
        "metric": "P(k) effective samples/s, learned mass vs plain diagonal mass (min over bins inside the "
                  "Nyquist sphere)",
        "value": summary["network"]["min_ess_per_s"]["mean"],
        "unit": "effective samples/s",
        "n_gpus": 1, "steps": args.ess_iters, "warmup": max(args.warmup, 300),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32 (network bf16)",
        "data": "synthetic",
        "config": {"workload": f"{wl.name}: {wl.N}^3 grid, L={wl.box:g} Mpc/h, {wl.n_sub} subsamples, "
                               f"{wl.f_sky:.0%} sky, {wl.radial} radial selection, {wl.n_bins} k bins, "
                               f"{wl.n_leapfrog} leapfrog steps (eps_max {wl.eps_max}), jump on (10 steps, "
                               f"eps_max {jeps}); network {2 * wl.n_bins}-128-128-{n_mass} trained on {len(F)} "
                               f"(feature, target) pairs from plain chains ({args.stat_moves} HMC moves each) on "
                               "random surveys of the same recipe made on the device; the survey itself held out; "
                               f"{args.seeds} seeds x {args.ess_iters} iterations per arm"},
        "summary": summary, "ratio_to_plain": ratios, "equal_accuracy": accuracy,
        "damping_of_network_damped": DAMPED,
        "per_seed": arms,
        "training": {"seconds": train_s, "statistics_seconds": t_stats, "examples": int(len(F)),
                     "final_minibatch_loss": {a: nets[a][1] for a in nets}},
    }
    print(json.dumps(line), flush=True)
    for a in nets:
        nets[a][0].close()
    return 0


def run_schechter(args):
    """Gibbs iterations per second on the paper's own setup (Sec. 5): 128^3, L =
    750 Mpc/h, fifteen luminosity subsamples with the Schechter selection, the
    mean numbers per magnitude bin and the luminosity bias law, a 25% cap; the
    survey is made on the device (bps_mock_*).  Beside it, the same sampler on
    the six-subsample 128^3 survey, to show what the nine extra subsamples cost
    (the a, c rebuild and the bias and normalisation sums grow with n_sub; the
    leapfrog does not)."""
    import numpy as np
    import torch

    from paper_1306_1821_gb300 import bps, inputs
    if not os.path.exists(bps.LIB_PATH):
        from paper_1306_1821_gb300 import build as b
        b.build()
    bps.load()
    out = {}
    for name in ("schechter128", "survey128"):
        wl = inputs.WORKLOADS[name]
        N, box = wl.N, wl.box
        mock = bps.Sampler(N, box, wl.n_sub, wl.n_bins)
        n2 = np.arange(3 * (N // 2) ** 2 + 1, dtype=np.float64)
        Pk = inputs.true_spectrum(2.0 * np.pi * np.sqrt(n2) / box, N, box)
        Pk[0] = 0.0
        if wl.radial == "schechter":
            table, _ = bps.bps_schechter_tables(np.asarray(wl.extra["M_edges"]), box / 2, 4097)
        else:
            r = np.arange(4097) * (box / 2 / 4096)
            table = np.broadcast_to(np.exp(-(r / wl.r0) ** 2), (wl.n_sub, 4097)).copy()
        d = torch.empty((N, N, N), dtype=torch.float32, device="cuda")
        R = torch.empty((wl.n_sub, N, N, N), dtype=torch.float32, device="cuda")
        c = torch.empty((wl.n_sub, N, N, N), dtype=torch.int32, device="cuda")
        bps.bps_mock_field(mock.ctx, 9, Pk, d)
        bps.bps_mock_response(mock.ctx, wl.f_sky, (0.0, 0.0, 1.0), table, R)
        bps.bps_mock_counts(mock.ctx, 9, d, R, wl.b, wl.nbar, 0, c)
        torch.cuda.synchronize()
        mock.close()
        P0, b0, n0 = inputs.initial_state(wl)
        s = bps.Sampler(N, box, wl.n_sub, wl.n_bins, n_leapfrog=wl.n_leapfrog, eps_max=wl.eps_max, jump=1,
                        jump_leapfrog=wl.jump_leapfrog, jump_eps_max=0.15, fixed_bias_index=wl.fixed_bias, seed=2)
        bps.bps_set_data(s.ctx, c, R)
        bps.bps_set_state(s.ctx, d, P0, b0, n0, 0)
        del c, R, d
        bps.bps_gibbs_iterate(s.ctx, max(args.warmup, 300))
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record()
        rec = bps.bps_gibbs_iterate(s.ctx, args.ess_iters, s.rec_len)
        e1.record()
        torch.cuda.synchronize()
        secs = e0.elapsed_time(e1) / 1000.0
        r = pk_ess(rec, wl.n_bins, N, secs)
        r.update({"n_sub": wl.n_sub, "gibbs_iterations_per_s": args.ess_iters / secs,
                  "ms_per_iteration": 1000.0 * secs / args.ess_iters,
                  "leapfrog_steps_per_s": args.ess_iters * wl.n_leapfrog / secs,
                  "hmc_acceptance": float(np.mean(rec[:, -1])),
                  "mean_b": [round(float(v), 4) for v in rec[:, wl.n_bins:wl.n_bins + wl.n_sub].mean(0)],
                  "true_b": [round(float(v), 4) for v in wl.b]})
        s.close()
        out[name] = r
    line = {"metric": "Gibbs iterations/s on the paper's fifteen-subsample setup (Sec. 5)",
            "value": out["schechter128"]["gibbs_iterations_per_s"], "unit": "Gibbs iterations/s",
            "n_gpus": 1, "steps": args.ess_iters, "warmup": max(args.warmup, 300), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic (made on the device)",
            "config": {"workload": "schechter128: 128^3, L=750 Mpc/h, 15 subsamples (M from -23 to -17 in 0.4 "
                                   "bins), Schechter selection in 14.5 < r < 17.77, bias law Eq. rel_bias, 25% cap, "
                                   "16 k bins, 10 leapfrog steps, jump on (10 steps); beside it survey128 "
                                   "(6 subsamples)"},
            "schechter128": out["schechter128"], "survey128": out["survey128"]}
    print(json.dumps(line), flush=True)
    return 0


def run_bare(args):
    """The 256^3 survey chain alone, for profiler captures of a small case: the
    same survey, state and seeds as the timed leg, set up through the C ABI,
    then --warmup and --steps Gibbs iterations; no other buffers, no timing and
    no JSON line (about 2 GB on the device)."""
    import numpy as np
    import torch

    from paper_1306_1821_gb300 import bps, inputs
    if not os.path.exists(bps.LIB_PATH):
        from paper_1306_1821_gb300 import build as b
        b.build()
    bps.load()
    wl = inputs.WORKLOADS[WORKLOAD]
    delta, counts, R = inputs.make_survey(wl, seed=wl.seed)
    P0, b0, nbar0 = inputs.initial_state(wl)
    s = bps.Sampler(wl.N, wl.box, wl.n_sub, wl.n_bins, n_leapfrog=wl.n_leapfrog, eps_max=wl.eps_max, jump=1,
                    jump_leapfrog=wl.jump_leapfrog, jump_eps_max=wl.jump_eps_max, fixed_bias_index=wl.fixed_bias,
                    seed=1)
    try:
        cnt = torch.from_numpy(counts).cuda()
        Rd = torch.from_numpy(R).cuda()
        bps.bps_set_data(s.ctx, cnt, Rd)
        bps.bps_set_state(s.ctx, torch.from_numpy(delta.astype(np.float32)).cuda(), P0, b0, nbar0, 0)
        del cnt, Rd
        torch.cuda.empty_cache()
        if args.warmup > 0:
            bps.bps_gibbs_iterate(s.ctx, args.warmup)
        rec = bps.bps_gibbs_iterate(s.ctx, args.steps, s.rec_len)
        print(f"bare: {args.steps} Gibbs iterations of {wl.name}, HMC acceptance {float(np.mean(rec[:, -1])):.2f}")
    finally:
        s.close()
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--workload", default=WORKLOAD,
                    choices=[WORKLOAD, "batch96", "precond128", "precond256", "schechter128"])
    ap.add_argument("--train-examples", type=int, default=None,
                    help="(feature, target) pairs of the preconditioner training set (precond* workloads)")
    ap.add_argument("--stat-moves", type=int, default=300, help="HMC moves per training statistic (precond*)")
    ap.add_argument("--seeds", type=int, default=3, help="chain seeds per arm (precond*)")
    ap.add_argument("--ess-iters", type=int, default=None,
                    help="Gibbs iterations of the P(k) ESS run (default 4000 at 256^3, 20000 per arm of precond128; "
                         "0 skips it)")
    ap.add_argument("--bare", action="store_true",
                    help="only the 256^3 chain: --warmup then --steps Gibbs iterations, no timing (profiler captures)")
    args = ap.parse_args(argv)
    if args.bare:
        return run_bare(args)
    if args.warmup < 3 and args.impl == "ours":
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch96":
        return run_batch(args)
    if args.workload in PRECOND_RUNS:
        if args.ess_iters is None:
            args.ess_iters = 20000
        return run_precond(args)
    if args.workload == "schechter128":
        if args.ess_iters is None:
            args.ess_iters = 4000
        return run_schechter(args)
    if args.ess_iters is None:
        args.ess_iters = 4000
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
