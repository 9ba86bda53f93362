"""Benchmark of the single-pass ID hot path on the streamed channel-field workload.

One step = one pass of the whole hot path over one snapshot matrix:
reset -> stream the 1000 snapshots in chunks of 32 (both sketches and the
coarse rows in one read of A) -> id_factor (pivoted QR of W, solve for P) ->
id_coarse_factor (sub-sampled ID of A_c) -> id_reconstruct_error (A(:,J)P).

Workload: 128 x 96 x 128 grid x 3 components (m = 4,718,592 rows) x 1000
snapshots, FP32 (18.87 GB, larger than L2, resident in HBM), l = 60, k = 50,
coarse grid 4x per direction.  Metric: GB/s of snapshot data per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

N > 1 runs under torchrun: each rank compresses its own matrix (replicas, weak
scaling, no collective on the data path).  ``--impl reference`` times the FP64
oracle on the host cores on a bounded row sample of the same workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "single-pass ID GB/s of snapshot data at fixed rel. error; % of HBM roofline"
UNIT = "GB/s"
GRID = (128, 96, 128)
NCOMP = 3
NSNAP = 1000
CHUNK = 32
K_RANK = 50
L_SKETCH = 60
STRIDE = (4, 4, 4)
SEED = 0
FALLBACK_HBM_GBS = 6800.0


def workload(grid=GRID, n=NSNAP):
    m = NCOMP * grid[0] * grid[1] * grid[2]
    return {"workload": f"streamed channel field {grid[0]}x{grid[1]}x{grid[2]}x{NCOMP} = "
                        f"{m} rows x {n} snapshots FP32, chunks of {CHUNK}, l={L_SKETCH}, "
                        f"k={K_RANK}, coarse {STRIDE[0]}x per direction",
            "m": m, "n": n, "l": L_SKETCH, "k": K_RANK, "chunk": CHUNK,
            "coarse_stride": list(STRIDE), "bytes_per_step": 4 * m * n,
            "l2": "inputs larger than L2 (18.9 GB vs 129 MB); no flush needed",
            "parallelism": "replicas (one independent matrix per GPU)"}


# ------------------------------------------------------------------ helpers

def max_over_ranks(ms, device, world):
    """The job's step time: the slowest rank's (an all-reduce MAX over the
    process group; the value itself on one rank)."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, bytes_per_rank_step, ms):
    """Whole-job GB/s: the bytes every rank processed in one step over the
    job's step time (weak scaling: one independent matrix per rank)."""
    return world * bytes_per_rank_step / (ms / 1e3) / 1e9


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            d = json.load(f)
        for key in ("hbm_gbs", "hbm_GBs", "hbm"):
            if key in d:
                return float(d[key]), "measured"
    except (OSError, ValueError):
        pass
    return FALLBACK_HBM_GBS, "fallback"


def kernel_traffic(kernel_file, kernel_name):
    """DRAM bytes per launch from a committed ncu summary, if it matches the
    current kernel source; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            d = json.load(f)
        src = open(os.path.join(ROOT, "paper_1905_13257_gb300", "csrc", kernel_file), "rb").read()
        ent = d.get(kernel_name)
        if ent and ent.get("source_sha256") == hashlib.sha256(src).hexdigest():
            return float(ent["traffic_bytes_per_launch"])
    except (OSError, ValueError, KeyError):
        pass
    return None


def pinned_host(shape, how):
    """A pinned FP32 host tensor: torch's pinned allocator ("torch"), or an
    anonymous mapping advised for transparent huge pages and registered with
    CUDA ("thp"), whose pages the copy engines walk in 2 MB steps when the
    kernel can supply them.  Returns (tensor, handle for release_pinned)."""
    import torch
    if how == "torch":
        return torch.empty(shape, dtype=torch.float32, pin_memory=True), None
    import mmap
    import numpy as np
    nbytes = 4 * int(np.prod(shape))
    mm = mmap.mmap(-1, nbytes, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
    mm.madvise(mmap.MADV_HUGEPAGE)
    arr = np.frombuffer(mm, dtype=np.float32).reshape(shape)
    t = torch.from_numpy(arr)
    err = torch.cuda.cudart().cudaHostRegister(t.data_ptr(), nbytes, 0)
    if int(err) != 0:
        raise RuntimeError(f"cudaHostRegister failed ({err})")
    return t, (mm, arr)


def release_pinned(t, keep):
    import torch
    if keep is not None:
        torch.cuda.cudart().cudaHostUnregister(t.data_ptr())


def gpu_numa_cpus(dev_index):
    """(node, cpus): the host NUMA node sysfs reports for the GPU's PCI device
    and the CPUs of that node this process may run on; None if unknown."""
    import subprocess as sp
    try:
        out = sp.run(["nvidia-smi", "-i", str(dev_index), "--query-gpu=pci.bus_id",
                      "--format=csv,noheader"], capture_output=True, text=True, timeout=30)
        bus = out.stdout.strip().splitlines()[0].strip().lower()
        parts = bus.split(":")
        if len(parts) == 3 and len(parts[0]) > 4:   # 00000000:xx:yy.z
            bus = parts[0][-4:] + ":" + parts[1] + ":" + parts[2]
        node = int(open(f"/sys/bus/pci/devices/{bus}/numa_node").read().strip())
        if node < 0:
            return None
        cpus = set()
        for rng in open(f"/sys/devices/system/node/node{node}/cpulist").read().strip().split(","):
            if "-" in rng:
                lo, hi = rng.split("-")
                cpus.update(range(int(lo), int(hi) + 1))
            elif rng:
                cpus.add(int(rng))
        cpus &= set(os.sched_getaffinity(0))
        return (node, cpus) if cpus else None
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, dev_uuid):
        self.proc = None
        self.uuid = dev_uuid

    def start(self):
        try:
            cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                   "-lms", "100"]
            if self.uuid:
                cmd += ["-i", self.uuid]
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except OSError:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        out, _ = self.proc.communicate(timeout=10)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in out.strip().splitlines():
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_step(A_rows, grid_rows, ncomp_rows, n, k, l, seed):
    """The oracle's hot path on a row sample: sketches, randomized ID, sub-sampled
    ID of the sample's coarse rows, reconstruction error."""
    import numpy as np
    import oracle
    A64 = np.asarray(A_rows, dtype=np.float64)
    m = A64.shape[0]
    Psi = oracle.psi(l, m, seed)
    Om = oracle.omega(n, l, seed)
    W, Y = oracle.sketch(A64, Psi, Om)
    J, P, kout, _ = oracle.column_id(W, k)
    rows = oracle.coarse_rows(grid_rows, ncomp_rows, STRIDE)
    Jc, Pc, kc, _ = oracle.column_id(A64[rows], k)
    fro, mx = oracle.recon_error(A64, J, P)
    return fro


def cpu_sample(A_host_rows, n, reps=1):
    """Time the oracle on a row sample (the first y-planes of component u)."""
    import numpy as np
    nx, ny, nz = GRID
    m_s = A_host_rows.shape[0]
    ny_s = m_s // (nx * nz)
    t0 = time.perf_counter()
    for _ in range(reps):
        oracle_step(A_host_rows, (nx, ny_s, nz), 1, n, K_RANK, L_SKETCH, SEED)
    dt = (time.perf_counter() - t0) / reps
    return dt, f"rows 0..{m_s - 1} (component u, y-planes 0..{ny_s - 1}) x {n} snapshots"


# --------------------------------------------------------------- reference

def run_reference(args):
    import numpy as np
    import torch
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    from synthetic.channel import factors
    nx, ny, nz = GRID
    ny_s = args.ref_planes
    S, T = factors(GRID, NCOMP, NSNAP, SEED)
    A_s = (S[: nx * nz * ny_s] @ T).to(torch.float32).numpy()
    del S
    cores = len(os.sched_getaffinity(0))
    for _ in range(args.warmup):
        cpu_sample(A_s, NSNAP)
    times = []
    for _ in range(args.steps):
        dt, desc = cpu_sample(A_s, NSNAP)
        times.append(dt)
    ms = 1e3 * statistics.mean(times)
    gbs = 4.0 * A_s.shape[0] * NSNAP / (ms / 1e3) / 1e9
    cfg = workload()
    line = {"impl": "reference", "metric": METRIC, "value": gbs, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic channel field (seeded), FP32 values, oracle arithmetic FP64",
            "config": cfg,
            "cpu_baseline": {"value": gbs, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": desc},
            "e2e": {"value": gbs, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------- ours

def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_1905_13257_gb300 import IdSketch, load
    from synthetic import channel_field

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    lib = load()

    grid = tuple(int(x) for x in args.grid.split(",")) if args.grid else GRID
    cfgd = workload(grid, args.n)
    m, n = cfgd["m"], cfgd["n"]
    A = channel_field(grid, NCOMP, n, seed=SEED + rank, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    sk = IdSketch(m, n, K_RANK, L_SKETCH, seed=SEED, dtype=torch.float32, grid=grid,
                  ncomp=NCOMP, coarse_stride=STRIDE, want_Y=True, want_coarse=True,
                  window_cols=n, stream=stream, prec=args.prec)

    ev = lambda: torch.cuda.Event(enable_timing=True)   # noqa: E731
    phase_ms = {"sketch": 0.0, "factor": 0.0, "coarse": 0.0, "recon": 0.0}
    result = {}

    def step(record):
        e0, e1, e2, e3, e4 = ev(), ev(), ev(), ev(), ev()
        e0.record(stream)
        sk.reset()
        for j0 in range(0, n, CHUNK):
            sk.stream_columns(A[:, j0:j0 + CHUNK])
        sk.flush()
        e1.record(stream)
        J, P, kout = sk.factor()
        e2.record(stream)
        Jc, Pc, kc = sk.coarse_factor()
        e3.record(stream)
        fro, mx = sk.reconstruct_error(A, J[:kout], P[:kout])
        e4.record(stream)
        if record:
            e4.synchronize()
            phase_ms["sketch"] += e0.elapsed_time(e1)
            phase_ms["factor"] += e1.elapsed_time(e2)
            phase_ms["coarse"] += e2.elapsed_time(e3)
            phase_ms["recon"] += e3.elapsed_time(e4)
        result.update(fro=fro, rel_max=mx, kout=kout, kc=kc)

    for _ in range(args.warmup):
        step(False)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    # per-kernel launch durations: CUDA events on the library's stream around
    # each launch of the fused sketch kernel and of the error-pass kernel
    sk.timing(True)
    for which in ("sketch", "recon"):
        sk.read_timing(which)
    clocks = ClockSampler(uuid)
    clocks.start()
    l0 = lib.id_kernel_launches()
    t_start, t_end = ev(), ev()
    torch.cuda.synchronize()
    t_start.record(stream)
    for _ in range(args.steps):
        step(True)
    t_end.record(stream)
    torch.cuda.synchronize()
    launches = lib.id_kernel_launches() - l0
    clk = clocks.stop()
    kt = {w: sk.read_timing(w) for w in ("sketch", "recon")}
    sk.timing(False)
    ms = max_over_ranks(t_start.elapsed_time(t_end) / args.steps, dev, world)
    if world > 1:
        dist.barrier()
    value = job_throughput(world, 4.0 * m * n, ms)

    # roofline of the dominant kernel: the fused sketch (FP32 data takes the
    # tensor-core kernel, 512 columns per launch).  Algorithmic bytes of one
    # step: read A once, write Y once per launch plus one read of Y per later
    # launch (read-modify-write across windows).  A_c is copied by its own
    # small kernel after each window's sketch (not counted here).
    per_phase = {k: v / args.steps for k, v in phase_ms.items()}
    peak, peak_kind = measured_peaks()
    window = 512
    launches_per_step = math.ceil(n / window)
    sketch_bytes = 4.0 * m * n + 4.0 * m * L_SKETCH * (2 * launches_per_step - 1)
    ms_s, cnt_s = kt["sketch"]
    sketch_launch_ms = ms_s / max(cnt_s, 1)
    kname = "sketch_tc_kernel<2>" if args.prec == "exact" else "sketch_tc_kernel<1>"
    rl_sketch = {"kernel": kname, "bound": "hbm",
                 "achieved": (sketch_bytes / launches_per_step / (sketch_launch_ms / 1e3) / 1e9
                              if cnt_s else None),
                 "peak": peak, "peak_kind": f"of {peak_kind}", "unit": "GB/s",
                 "traffic": kernel_traffic("sketch_tc.cu", kname),
                 "algorithmic_bytes_per_launch": sketch_bytes / launches_per_step,
                 "launch_ms": sketch_launch_ms, "launches_timed": cnt_s,
                 "launches_per_step": launches_per_step,
                 "timing": "CUDA events around each launch on the library stream"}
    recon_bytes = 4.0 * m * n   # one read of A; the skeleton rows are re-reads of A
    ms_r, cnt_r = kt["recon"]
    recon_launch_ms = ms_r / max(cnt_r, 1)
    rl_recon = {"kernel": "recon_tc_kernel", "bound": "hbm",
                "achieved": recon_bytes / (recon_launch_ms / 1e3) / 1e9 if cnt_r else None,
                "peak": peak,
                "peak_kind": f"of {peak_kind}", "unit": "GB/s",
                "traffic": kernel_traffic("recon_tc.cu", "recon_tc_kernel"),
                "algorithmic_bytes_per_launch": recon_bytes, "launch_ms": recon_launch_ms,
                "launches_timed": cnt_r, "launches_per_step": 1,
                "timing": "CUDA events around each launch on the library stream"}
    for rl in (rl_sketch, rl_recon):
        rl["frac"] = rl["achieved"] / peak if rl["achieved"] is not None else None
    dominant = rl_sketch if ms_s >= ms_r else rl_recon
    roofline = dict(dominant)
    roofline["phase_ms"] = per_phase
    roofline["all"] = [rl_sketch, rl_recon]

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        # the pinned host buffer is allocated (and its pages placed) from the
        # CPUs of the GPU's own NUMA node, so that the copies do not cross
        # to the other socket's memory
        numa = gpu_numa_cpus(local)
        aff = os.sched_getaffinity(0)
        if numa:
            os.sched_setaffinity(0, numa[1])
        A_host, host_keep = pinned_host((n, m), args.host_alloc)
        A_host.copy_(A.T)
        if numa:
            os.sched_setaffinity(0, aff)
        A_host_v = A_host.T
        # Two device buffers: the host-to-device copies of step k + 1 run on a
        # copy stream while step k computes (a stream of snapshot matrices
        # arriving from the host).  Every step still copies its own inputs
        # and reads its results back inside the timed region.
        bufs = [torch.empty_like(A_host, device=dev).T for _ in range(2)]
        copy_stream = torch.cuda.Stream(device=dev)
        copied = [torch.cuda.Event() for _ in range(2)]
        consumed = [torch.cuda.Event() for _ in range(2)]
        used = [False, False]

        def enqueue_copy(k):
            b = k % 2
            with torch.cuda.stream(copy_stream):
                if used[b]:
                    copy_stream.wait_event(consumed[b])   # step k - 2 has read it
                for j0 in range(0, n, CHUNK):
                    bufs[b][:, j0:j0 + CHUNK].copy_(A_host_v[:, j0:j0 + CHUNK],
                                                    non_blocking=True)
                copied[b].record(copy_stream)

        def compute(k):
            b = k % 2
            Ad = bufs[b]
            stream.wait_event(copied[b])
            sk.reset()
            for j0 in range(0, n, CHUNK):
                sk.stream_columns(Ad[:, j0:j0 + CHUNK])
            J, P, kout = sk.factor(device="cpu")
            Jc, Pc, kc = sk.coarse_factor(device="cpu")
            fro, mx = sk.reconstruct_error(Ad, J[:kout], P[:kout])
            consumed[b].record(stream)
            used[b] = True
            return J, P, Jc, Pc

        def e2e_run(steps):
            copy_stream.wait_stream(stream)   # copies start after the timing event
            enqueue_copy(0)
            out = None
            for k in range(steps):
                if k + 1 < steps:
                    enqueue_copy(k + 1)
                out = compute(k)
            return out

        e2e_run(max(1, args.warmup))
        torch.cuda.synchronize()
        # the host link's own rate at this moment (one chunk, outside the
        # timed region): it bounds e2e, and it has varied between calls
        p0, p1 = ev(), ev()
        p0.record(stream)
        bufs[0][:, :CHUNK].copy_(A_host_v[:, :CHUNK], non_blocking=True)
        p1.record(stream)
        torch.cuda.synchronize()
        h2d_probe = 4.0 * m * CHUNK / (p0.elapsed_time(p1) / 1e3) / 1e9
        s0, s1 = ev(), ev()
        s0.record(stream)
        J, P, Jc, Pc = e2e_run(args.steps)
        s1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = s0.elapsed_time(s1) / args.steps
        d2h = J.numel() * 4 + P.numel() * 8 + Jc.numel() * 4 + Pc.numel() * 8 + 16
        e2e = {"value": world * 4.0 * m * n / (e2e_ms / 1e3) / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 4 * m * n, "d2h_bytes_per_step": int(d2h),
               "ms_per_step": e2e_ms,
               "overlap": "host-to-device copies of step k + 1 under the compute of step k",
               "host_numa_node": numa[0] if numa else None,
               "h2d_probe_gbs": h2d_probe, "host_alloc": args.host_alloc}
        release_pinned(A_host, host_keep)
        del A_host, bufs

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        nx, ny, nz = grid
        rows = nx * nz * args.cpu_planes
        A_rows = A[:rows].T.contiguous().cpu().numpy().T
        dt, desc = cpu_sample(A_rows, n)
        cpu = {"value": 4.0 * rows * n / dt / 1e9, "unit": UNIT,
               "cores": len(os.sched_getaffinity(0)), "kind": "oracle", "sample": desc,
               "seconds": dt}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": {"exact": "f32", "bf16": "bf16", "fp8": "fp8e4m3"}[args.prec],
                "data": "synthetic channel field (seeded), resident in HBM",
                "config": dict(cfgd, sketch_precision={
                    "exact": "FP32-accurate (two bfloat16 pieces)",
                    "bf16": "bfloat16 products, FP32 accumulation",
                    "fp8": "FP8-E4M3 values with per-column power-of-two scales (a scale pass "
                           "reads each window once more), products on the bfloat16 tensor cores "
                           "(E4M3 values are exact there), FP32 accumulation"}[args.prec]),
                "roofline": roofline, "e2e": e2e, "gpu_launches": launches,
                "clocks": clk, "cpu_baseline": cpu,
                "errors": {"rel_fro": result.get("fro"), "rel_max": result.get("rel_max"),
                           "k_out": result.get("kout"), "k_coarse": result.get("kc")}}
        print(json.dumps(line), flush=True)
    sk.close()
    if world > 1:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------ batched form

def batched_problems(count=64, seed=1, max_rows=2_000_000):
    """Sizes of the batched workload: 64 channel fields of uneven size, m ~
    U[50k, 2M] rounded to 3 nx ny nz with nx = nz = 2 ny, n ~ U[64, 512],
    k ~ U[10, 80], l = k + 10 (up to 90), seeds 1..64, FP32 data, every
    other problem in the BF16 sketch form.  count and max_rows (m capped
    before rounding) give smaller cases of the same mix, for profiling."""
    import numpy as np
    rng = np.random.default_rng(seed)
    out = []
    for b in range(count):
        mrow = min(rng.uniform(50_000, 2_000_000), max_rows)
        ny = max(2, int(round((mrow / 12.0) ** (1.0 / 3.0))))
        n = int(rng.integers(64, 513))
        k = int(rng.integers(10, 81))
        out.append(dict(grid=(2 * ny, ny, 2 * ny), n=n, k=k, l=k + 10, seed=b + 1,
                        prec="bf16" if b % 2 else "exact"))
    return out


def run_batched(args):
    import torch

    from paper_1905_13257_gb300 import IdBatch, load
    from synthetic import channel_field

    lib = load()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    spec = batched_problems(args.batch_count, max_rows=args.batch_max_rows)
    probs, nbytes = [], 0
    for p in spec:
        A = channel_field(p["grid"], NCOMP, p["n"], seed=p["seed"], dtype=torch.float32,
                          device=dev)
        probs.append(dict(A=A, k=p["k"], l=p["l"], seed=p["seed"], prec=p["prec"]))
        nbytes += 4 * A.shape[0] * A.shape[1]
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    bt = IdBatch(probs, stream=stream)
    tune_choice, tune_ms = bt.tune()     # the project's autotuner: work split of the sketches
    for _ in range(args.warmup):
        bt.run()
    bt.wait()
    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    clocks.start()
    l0 = lib.id_kernel_launches()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    t0.record(stream)
    for _ in range(args.steps):
        bt.run()
    t1.record(stream)
    torch.cuda.synchronize()
    launches = lib.id_kernel_launches() - l0
    clk = clocks.stop()
    res = bt.wait()
    ms = t0.elapsed_time(t1) / args.steps
    gbs = nbytes / (ms / 1e3) / 1e9
    peak, kind = measured_peaks()
    ms_ = [A["A"].shape[0] for A in probs]
    line = {
        "metric": "batched randomized ID GB/s of snapshot data", "value": gbs, "unit": UNIT,
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic channel fields (seeded), resident in HBM",
        "config": {"workload": f"{len(probs)} channel fields of uneven size in one graph launch "
                               "(one persistent kernel: work-list sketches, each matrix's W "
                               "sums, QR and solve by the CTA that completes it): "
                               f"m ~ U[50k, {args.batch_max_rows / 1e6:g}M] (3 x 2ny x ny x 2ny), "
                               "n ~ U[64, 512], "
                               f"k ~ U[10, 80], l = k + 10, seeds 1..{len(probs)}, FP32, "
                               "every other problem BF16 sketch",
                   "problems": len(probs), "bytes_per_step": nbytes,
                   "m_range": [min(ms_), max(ms_)],
                   "n_range": [min(p["n"] for p in spec), max(p["n"] for p in spec)],
                   "k_range": [min(p["k"] for p in spec), max(p["k"] for p in spec)],
                   "l2": f"inputs larger than L2 ({nbytes / 1e9:.1f} GB); no flush needed"},
        "roofline": {"kernel": "whole batch (one graph launch of one persistent kernel)",
                     "bound": "hbm", "achieved": gbs, "peak": peak, "peak_kind": "of " + kind,
                     "unit": "GB/s", "frac": gbs / peak, "traffic": None},
        "gpu_launches": launches, "clocks": clk,
        "autotune": {"work_item_mb": tune_choice,
                     "ms_per_launch_by_candidate": {str(k): v for k, v in tune_ms.items()}},
        "k_out_short": sum(1 for (_, _, ko), p in zip(res, spec) if ko < p["k"]),
    }
    # Equal-error comparison (outside the timed region): each problem sketched
    # in the BF16 form against the plain FP32-accurate form of the same matrix
    # and the same Psi, both errors from the library's error pass (k <= 64).
    from paper_1905_13257_gb300 import IdSketch
    ratios = []
    for (J, P, ko), p in zip(res, probs):
        if p["prec"] != "bf16" or p["k"] > 64:
            continue
        A = p["A"]
        sk = IdSketch(A.shape[0], A.shape[1], p["k"], p["l"], seed=p["seed"],
                      dtype=torch.float32, want_Y=False, stream=stream)
        sk.stream_columns(A)
        J0, P0, k0 = sk.factor()
        e_plain, _ = sk.reconstruct_error(A, J0[:k0], P0[:k0])
        e_bf16, _ = sk.reconstruct_error(A, J[:ko], P[:ko])
        ratios.append(e_bf16 / e_plain)
        sk.close()
    if ratios:
        r = sorted(ratios)
        line["equal_error"] = {
            "what": "relative Frobenius error of the batch's BF16-sketch ID / that of the "
                    "FP32-accurate-sketch ID of the same matrix (same Psi); the BF16 "
                    "problems with k <= 64 (the error pass's limit)",
            "problems": len(r), "min": r[0], "median": r[len(r) // 2], "max": r[-1],
            "within_1.05": sum(1 for x in r if x <= 1.05)}
    print(json.dumps(line))
    bt.close()
    return 0


# ---------------------------------------------------------- learned proposal

def run_learned(args):
    """The learned skeleton proposal on the bench's snapshot stream: train the
    network on the plain ID's skeletons of 200 earlier 512-snapshot windows,
    then compare, on later windows, the plain randomized ID with the learned
    proposal (2k candidates, restricted pivoted QR, fallback at 1.05x the
    plain error): errors, fallback rate, candidate recall, and the time of
    one window's ID (sketch + QR + error pass) of each form."""
    import numpy as np
    import torch

    from paper_1905_13257_gb300 import IdSketch, load
    from paper_1905_13257_gb300.learned import (LearnedProposal, bce, compare_on_window,
                                                plain_skeleton)
    from synthetic.channel import channel_field, snapshot_step

    load()
    torch.cuda.set_device(0)
    grid = tuple(int(x) for x in args.grid.split(",")) if args.grid else GRID
    nwin, ntrain, nheld = 512, args.train_windows, args.held_windows
    m = NCOMP * grid[0] * grid[1] * grid[2]
    dt = snapshot_step(NSNAP)

    def window(w):
        return channel_field(grid, NCOMP, nwin, seed=SEED, dtype=torch.float32, device="cuda",
                             first=w * nwin, dt=dt)

    stride = (grid[0] // 16, grid[1] // 16, grid[2] // 16)
    sk = IdSketch(m, nwin, K_RANK, L_SKETCH, seed=SEED, dtype=torch.float32, want_Y=False)
    prop = LearnedProposal(grid, K_RANK, stride=stride, seed=1)
    untrained = LearnedProposal(grid, K_RANK, stride=stride, seed=1)
    t0 = time.perf_counter()
    data = []
    for w in range(ntrain):
        A = window(w)
        J, _ = plain_skeleton(sk, A)
        y = torch.zeros(nwin, dtype=torch.float32, device="cuda")
        y[J.long()] = 1.0
        data.append((prop.features(A), y))
        del A
    t_data = time.perf_counter() - t0
    pw = (nwin - K_RANK) / K_RANK
    losses = []
    t0 = time.perf_counter()
    for _ in range(args.epochs):
        tot = 0.0
        for X, y in data:
            s = prop.train_step(X, y, lr=args.lr, pos_weight=pw)
            tot += bce(s.cpu().numpy(), y.cpu().numpy(), pw)
        losses.append(tot / len(data))
    prop.net.check()
    t_train = time.perf_counter() - t0
    untrained.scale = prop.scale
    rng = np.random.default_rng(7)
    rows = []
    for w in range(ntrain, ntrain + nheld):
        rows.append(compare_on_window(prop, sk, window(w), rng, untrained=untrained))
    # one window's ID, each form: stream (sketch) + QR (+ proposal) + error pass
    A = window(ntrain)
    X = prop.features(A)

    def plain_form():
        sk.reset()
        for j0 in range(0, nwin, CHUNK):
            sk.stream_columns(A[:, j0:j0 + CHUNK])
        J, P, kout = sk.factor()
        return sk.reconstruct_error(A, J[:kout], P[:kout])

    def learned_form():
        sk.reset()
        for j0 in range(0, nwin, CHUNK):
            sk.stream_columns(A[:, j0:j0 + CHUNK])
        cand = prop.propose(prop.features(A))
        J, P, kout = sk.factor_restricted(cand)
        return sk.reconstruct_error(A, J[:kout], P[:kout])

    times = {}
    for name, fn in (("plain", plain_form), ("learned", learned_form)):
        for _ in range(args.warmup):
            fn()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(args.steps):
            fn()
        e1.record()
        torch.cuda.synchronize()
        times[name] = e0.elapsed_time(e1) / args.steps
    wbytes = 4.0 * m * nwin
    ratio_l = [r["err_learned"] / r["err_plain"] for r in rows]
    ratio_r = [r["err_random"] / r["err_plain"] for r in rows]
    ratio_u = [r["err_untrained"] / r["err_plain"] for r in rows]
    line = {
        "metric": "learned skeleton proposal vs plain randomized ID at equal error (<= 1.05x)",
        "value": wbytes / (times["learned"] / 1e3) / 1e9, "unit": UNIT, "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": times["learned"],
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic channel-field stream (seeded), windows of 512 snapshots",
        "config": {"workload": f"learned proposal: {ntrain} training + {nheld} held-out windows "
                               f"of {grid[0]}x{grid[1]}x{grid[2]}x{NCOMP} = {m} rows x {nwin} "
                               f"snapshots FP32, k={K_RANK}, l={L_SKETCH}, 2 candidates in each "
                               f"of k ranges of snapshots, "
                               f"4096 features, 256 hidden units, BF16 products",
                   "epochs": args.epochs, "lr": args.lr},
        "plain_ms_per_window": times["plain"],
        "plain_GBs": wbytes / (times["plain"] / 1e3) / 1e9,
        "training": {"loss_per_epoch": losses, "data_s": t_data, "train_s": t_train},
        "held_out": {"err_ratio_learned": ratio_l, "err_ratio_random": ratio_r,
                     "err_ratio_untrained": ratio_u,
                     "recall_untrained": float(np.mean([r["recall_untrained"] for r in rows])),
                     "proposal_used": int(sum(r["use_learned"] for r in rows)),
                     "windows": len(rows),
                     "recall_learned": float(np.mean([r["recall_learned"] for r in rows])),
                     "recall_random": float(np.mean([r["recall_random"] for r in rows])),
                     "err_plain": [r["err_plain"] for r in rows],
                     "qr_plain_ms": 1e3 * float(np.median([r["qr_plain_s"] for r in rows])),
                     "proposal_and_qr_ms":
                         1e3 * float(np.median([r["proposal_and_qr_s"] for r in rows]))},
    }
    print(json.dumps(line), flush=True)
    sk.close()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--n", type=int, default=NSNAP)
    ap.add_argument("--grid", type=str, default=None,
                    help="nx,ny,nz of a smaller case (profiling); default 128,96,128")
    ap.add_argument("--coarse-stride", type=str, default=None,
                    help="sx,sy,sz of the coarse grid (profiling); default 4,4,4")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--cpu-planes", type=int, default=8,
                    help="y-planes of component u in the CPU-baseline sample")
    ap.add_argument("--workload", choices=["channel", "batched64", "learned"],
                    default="channel",
                    help="batched64: the batched form (64 matrices of uneven size); "
                         "learned: the learned skeleton proposal (training + comparison)")
    ap.add_argument("--prec", choices=["exact", "bf16", "fp8"], default="exact",
                    help="sketch precision of the channel workload: FP32-accurate (default), "
                         "the bfloat16 or the FP8-E4M3 precision form")
    ap.add_argument("--host-alloc", choices=["torch", "thp"], default="thp",
                    help="pinned host buffer of the end-to-end run")
    ap.add_argument("--batch-count", type=int, default=64,
                    help="batched workload: the first N problems of the mix (profiling)")
    ap.add_argument("--batch-max-rows", type=int, default=2_000_000,
                    help="batched workload: cap on each problem's rows (profiling)")
    ap.add_argument("--train-windows", type=int, default=200)
    ap.add_argument("--held-windows", type=int, default=10)
    ap.add_argument("--epochs", type=int, default=4)
    ap.add_argument("--lr", type=float, default=0.05)
    ap.add_argument("--ref-planes", type=int, default=8,
                    help="y-planes of component u per step of the reference arm's sample "
                         "(the same sample as cpu_baseline by default)")
    args = ap.parse_args()
    if args.coarse_stride:
        global STRIDE
        STRIDE = tuple(int(x) for x in args.coarse_stride.split(","))
    if args.warmup < 3:
        print("warning: fewer than 3 warm-up steps", file=sys.stderr)
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batched64":
        return run_batched(args)
    if args.workload == "learned":
        return run_learned(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
