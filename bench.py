"""Benchmark: voxel-driven cone-beam back-projection on GB300.

One step = one back-projection of all 496 views of 1248x960 FP32 filtered
projections into a 512^3 FP32 volume (6.66e10 voxel updates), inputs resident
in HBM.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the slow, plain definition) on
the host cores on a bounded sample of the same workload.  Under torchrun
(N > 1) every rank runs an independent replica of the workload (the path
needs no exchange between GPUs); the value is the total update rate.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("GUp/s (voxel updates/s) at 512³×496 views, fwd+adjoint; "
          "% of roofline at stated error")
UNIT = "GUp/s"
SM_COUNT = 152
FP32_LANES_PER_SM = 128
ISSUE_SLOTS_PER_UPDATE = 27      # FP32 issue slots per update: 15 FP32 ops, 1 reciprocal, 2 floor, 2 int
                                 # conversions, 1 address, 2 bounds tests, 4 loads
PAPER_PHI_GUPS = {"clipped": 8.5, "full": 12.9}   # Xeon Phi 5110P, assembly, 512^3
# DRAM bytes (read + write) per back-projection launch, the mean of a step's
# launches, from an ncu capture (dram__bytes_read.sum + dram__bytes_write.sum);
# valid only while the kernel sources hash to the value they were taken with.
KERNEL_SOURCES = ["paper_1401_3615_gb300/csrc/fdk_bp_kernel.cuh", "paper_1401_3615_gb300/csrc/fdk_tile.cuh",
                  "paper_1401_3615_gb300/csrc/fdk_internal.cuh", "paper_1401_3615_gb300/csrc/fdk_bp_ldg32.cu",
                  "paper_1401_3615_gb300/csrc/fdk_bp_stage.cu", "paper_1401_3615_gb300/csrc/fdk_stage.cuh"]
MEASURED_TRAFFIC = {("fdk512", 496, 0, 0): {"bytes": (6610201600 + 562296576 + 5338257920 + 554663168) / 2,
                                           "sources": "3811f62f6354a703"}}


def _sources_sha() -> str:
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int, out_path=None):
        self.gpu = gpu_index
        self.out_path = out_path
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for ln in self.proc.stdout:
            self.lines.append(ln.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, val in zip(names, parts[5:9]):
                if val.lower() == "active":
                    reasons.add(n)
        if self.out_path:
            with open(self.out_path, "w") as f:
                f.write("\n".join(self.lines) + "\n")
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else platform)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.strip().lower().startswith("model name"):
                return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for ln in f:
                if ln.lower().startswith("model name"):
                    return ln.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def _accuracy(args, scan, proj, mats, vs, org, dims):
    """One back-projection of the step's workload into a zeroed volume, every
    voxel against the FP64 oracle run on all host cores: max|diff| over
    max|f_oracle| and PSNR (peak max|f_oracle|), the accuracy bar being
    max|diff| <= 1e-4 max|f| and PSNR >= 80 dB."""
    import torch
    import oracle
    from paper_1401_3615_gb300 import fdk
    oracle.build()
    threads = os.cpu_count() or 1
    vol = torch.zeros((int(dims[2]), int(dims[1]), int(dims[0])), dtype=torch.float32, device=proj.device)
    fdk.fdk_backproject(vol, proj, mats, vs, org, fetch=args.fetch, tile=args.tile)
    got = vol.cpu().numpy()
    del vol
    t = time.perf_counter()
    ref = oracle.backproject(proj.float().cpu().numpy(), mats, dims, vs, org, threads=threads)
    dt = time.perf_counter() - t
    peak = float(np.abs(ref).max())
    diff = got.astype(np.float64) - ref
    err = float(np.abs(diff).max())
    mse = float(np.mean(diff * diff))
    return {"max_abs_diff_over_peak": err / peak,
            "psnr_db": float(10 * np.log10(peak * peak / mse)) if mse > 0 else float("inf"),
            "voxels": int(ref.size), "against": "FP64 oracle, whole volume, same inputs",
            "bar": "max|diff| <= 1e-4 max|f_oracle| and PSNR >= 80 dB",
            "meets_bar": bool(err <= 1e-4 * peak and (mse == 0 or 10 * np.log10(peak * peak / mse) >= 80.0)),
            "oracle_seconds": dt, "oracle_threads": threads}


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def _max_over_ranks(x: float, world: int, dev) -> float:
    """The largest x over all ranks: a replicated job takes as long as its
    slowest replica.  Needs an initialised process group when world > 1."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _job_rate(world: int, updates_per_replica: float, seconds: float) -> float:
    """Whole-job GUp/s: the updates of every replica over the slowest one's time."""
    return world * updates_per_replica / seconds / 1e9


def _cpu_sample(cfg, scan_proj, mats, dims, vs, org, target_s: float, threads: int):
    """Time the oracle on a central z-slab of the workload sized to about
    target_s seconds; returns (updates/s, description)."""
    import oracle
    nx, ny, nz = int(dims[0]), int(dims[1]), int(dims[2])
    n = mats.shape[0]

    def run(planes):
        z0 = nz // 2 - planes // 2
        org2 = np.array(org, dtype=np.float64)
        org2[2] = float(org[2]) + z0 * float(vs[2])
        d2 = (nx, ny, planes)
        t = time.perf_counter()
        oracle.backproject(scan_proj, mats, d2, vs, org2.astype(np.float32), threads=threads)
        return time.perf_counter() - t, nx * ny * planes * n

    dt, upd = run(1)
    rate = upd / max(dt, 1e-9)
    planes = int(max(1, min(nz, round(target_s * rate / (nx * ny * n)))))
    dt, upd = run(planes)
    desc = (f"central slab {nx}x{ny}x{planes} of the {nx}x{ny}x{nz} volume, all {n} views "
            f"({upd:.3e} updates, {dt:.1f} s)")
    return upd / dt, desc, dt


def _workload(args, cfg) -> str:
    """The workload's name, the same on both arms."""
    return (f"{args.config}: {cfg.nx}x{cfg.ny}x{cfg.nz} FP32 volume ({cfg.voxel} mm), {cfg.n_views} views of "
            f"{cfg.det_w}x{cfg.det_h} {args.proj_dtype.upper()} filtered projections, 200-degree short scan")


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    import synth
    import torch
    oracle.build()
    cfg = synth.PRESETS[args.config]
    threads = os.cpu_count() or 1
    torch.set_num_threads(threads)
    geo = synth.geometry(cfg)
    dims, vs, org = synth.volume_geometry(cfg)
    # inputs: a band of detector rows is all a central slab needs, but the
    # oracle is given the whole filtered projection stack as generated
    proj = synth.projections(cfg, geo, synth.phantom(cfg), device="cuda" if torch.cuda.is_available() else "cpu")
    proj = proj.cpu().numpy()
    mats = geo["mats"]
    per_step = args.ref_step_seconds
    rate, desc, _ = _cpu_sample(cfg, proj, mats, dims, vs, org, per_step, threads)
    planes = int(desc.split("x")[2].split(" ")[0])
    nx, ny = int(dims[0]), int(dims[1])
    z0 = int(dims[2]) // 2 - planes // 2
    org2 = np.array(org, dtype=np.float32)
    org2[2] = float(org[2]) + z0 * float(vs[2])
    for _ in range(args.warmup):
        oracle.backproject(proj, mats, (nx, ny, planes), vs, org2, threads=threads)
    t = time.perf_counter()
    for _ in range(args.steps):
        oracle.backproject(proj, mats, (nx, ny, planes), vs, org2, threads=threads)
    dt = (time.perf_counter() - t) / max(args.steps, 1)
    upd = nx * ny * planes * cfg.n_views
    value = upd / dt / 1e9
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": _workload(args, cfg), "updates_per_step": cfg.updates,
                   "sample": "bounded slab per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "cpu_model": _cpu_model(),
                         "kind": "oracle",
                         "sample": f"central slab {nx}x{ny}x{planes}, all {cfg.n_views} views per step"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def _precision_report(args, cfg, scan, proj, proj32, vol, mats, vs, org):
    """Error of the low-precision-storage result, reported per result: against
    the FP32-storage GPU result on the whole volume, and against the FP64
    oracle (given the stored values and the FP32 values) on a seeded 64^3
    sub-block."""
    import torch
    import oracle
    from paper_1401_3615_gb300 import fdk
    low = torch.zeros_like(vol)
    fdk.fdk_backproject(low, proj, mats, vs, org, fetch=args.fetch, tile=args.tile)
    ref = torch.zeros_like(vol)
    fdk.fdk_backproject(ref, proj32, mats, vs, org, fetch=args.fetch, tile=args.tile)
    torch.cuda.synchronize()
    peak = float(ref.abs().max())
    diff = (low.double() - ref.double())
    out = {"storage": args.proj_dtype,
           "vs_fp32_storage_gpu": {"max_abs_over_peak": float(diff.abs().max()) / peak,
                                   "psnr_db": float(10 * np.log10(peak ** 2 / float((diff ** 2).mean())))}}
    del diff
    rng = np.random.default_rng(1024)
    n0 = rng.integers(0, np.array([cfg.nx, cfg.ny, cfg.nz]) - 64 + 1)
    # keep the block inside the middle 5/8 of the volume, where the phantom is
    lo = (np.array([cfg.nx, cfg.ny, cfg.nz]) * 5) // 16
    n0 = np.minimum(np.maximum(n0, lo), np.array([cfg.nx, cfg.ny, cfg.nz]) - lo - 64)
    zz, yy, xx = np.meshgrid(*(np.arange(n0[a], n0[a] + 64) for a in (2, 1, 0)), indexing="ij")
    xyz = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1)
    threads = os.cpu_count() or 1
    import concurrent.futures as cf
    chunks = np.array_split(np.arange(len(xyz)), threads)

    def orc(p):
        with cf.ThreadPoolExecutor(threads) as ex:
            return np.concatenate(list(ex.map(lambda idx: oracle.backproject_voxels(
                p, mats, vs, org, xyz[idx]), chunks)))
    stored = proj.float().cpu().numpy()
    exact = proj32.cpu().numpy()
    o_stored, o_exact = orc(stored), orc(exact)
    g = low[xyz[:, 2], xyz[:, 1], xyz[:, 0]].cpu().numpy().astype(np.float64)
    pk = float(np.abs(o_exact).max())
    out["subblock_64"] = {"origin_voxel": [int(v) for v in n0],
                          "gpu_vs_oracle_same_stored_values": float(np.abs(g - o_stored).max()) / pk,
                          "gpu_vs_oracle_fp32_values": float(np.abs(g - o_exact).max()) / pk,
                          "storage_rounding_alone": float(np.abs(o_stored - o_exact).max()) / pk}
    return out


def _adjoint_timing(args, world, dev, proj, vol, mats, vs, org, upd_full, fwd_ms):
    """Time the transpose (voxel-driven splat) on the same workload: the
    volume is read and every view's projection accumulated (+=)."""
    import torch
    import torch.distributed as dist
    from paper_1401_3615_gb300 import fdk
    out = torch.zeros(proj.shape, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream()
    steps = max(1, min(args.steps, 5))
    for _ in range(2):
        fdk.fdk_forwardproject_adjoint(out, vol, mats, vs, org)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        fdk.fdk_forwardproject_adjoint(out, vol, mats, vs, org)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = _max_over_ranks(t0.elapsed_time(t1) / steps, world, dev)
    del out
    return {"value": _job_rate(world, upd_full, ms * 1e-3), "unit": UNIT, "ms_per_step": ms,
            "steps": steps, "ratio_to_forward": ms / fwd_ms,
            "what": "fdk_forwardproject_adjoint (transpose splat) on the same workload"}


def _preprocess_timing(args, world, dev, proj, mats, cfg):
    """Time the FDK pre-processing step on the workload's images: cosine
    pre-weighting and Ram-Lak row filtering (fdk_preweight_filter) of n raw
    line-integral images into filtered ones.  The step's projections serve
    as the raw input (the values do not change the work)."""
    import torch
    from paper_1401_3615_gb300 import fdk
    out = torch.empty_like(proj)
    dbeta = np.deg2rad(cfg.arc_deg) / max(cfg.n_views - 1, 1)
    scale = float(dbeta / (cfg.pixel * cfg.sid / cfg.sdd))
    stream = torch.cuda.current_stream()
    for _ in range(2):
        fdk.fdk_preweight_filter(out, proj, mats, scale)
    torch.cuda.synchronize()
    steps = max(1, min(args.steps, 5))
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(steps):
        fdk.fdk_preweight_filter(out, proj, mats, scale)
    t1.record(stream)
    torch.cuda.synchronize()
    ms = _max_over_ranks(t0.elapsed_time(t1) / steps, world, dev)
    del out
    nbytes = 2 * proj.numel() * 4
    hbm = float(_peaks().get("hbm_gbs", 6800.0))
    return {"ms_per_step": ms, "steps": steps, "GB_per_s": nbytes / (ms * 1e-3) / 1e9,
            "hbm_frac": nbytes / (ms * 1e-3) / 1e9 / hbm, "bytes": nbytes,
            "what": (f"fdk_preweight_filter: cosine pre-weight + Ram-Lak row filter of {proj.shape[0]} images "
                     f"of {proj.shape[2]}x{proj.shape[1]} (row FFT length {_fft_len(proj.shape[2])})")}


def _fft_len(W: int) -> int:
    """The library's row FFT length: 2560 for rows of 1025..1280 pixels, else
    the power of two >= 2W (at least 4)."""
    n = 1
    while n < 2 * W:
        n <<= 1
    n = max(n, 4)
    return 2560 if n == 4096 and 2 * W <= 2560 else n


def _e2e(args, world, dev, proj, vol, mats, vs, org, upd_full):
    """End to end through the C-ABI entry point for host buffers
    (fdk_backproject_host, overwrite): every step copies the projections from
    pinned host memory to the device in chunks of views whose copies overlap
    the back-projection, and the resulting volume back to pinned memory in
    z-slabs that overlap the last chunk's back-projection."""
    import torch
    import torch.distributed as dist
    from paper_1401_3615_gb300 import fdk
    h_proj = torch.empty(proj.shape, dtype=proj.dtype, pin_memory=True)
    h_proj.copy_(proj)
    h_vol = torch.zeros(vol.shape, dtype=vol.dtype, pin_memory=True)
    # at least 20 steps: the host link has periodic slow phases (about every
    # 0.5 s), and the mean should not hinge on whether one falls in a short run
    e2e_steps = min(max(args.steps, 20), 40)

    def e2e_step():
        fdk.fdk_backproject_host(h_vol, h_proj, mats, vs, org, fetch=args.fetch, tile=args.tile,
                                 overwrite=True)

    for _ in range(max(args.warmup, 3)):
        e2e_step()
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    # each call synchronises before it returns, so per-step wall times are exact
    w0 = time.perf_counter()
    marks = [w0]
    for _ in range(e2e_steps):
        e2e_step()
        marks.append(time.perf_counter())
    torch.cuda.synchronize()
    e2e_s = _max_over_ranks((time.perf_counter() - w0) / e2e_steps, world, dev)
    step_ms = [(b - a) * 1e3 for a, b in zip(marks, marks[1:])]
    vol_bytes = int(vol.numel() * vol.element_size())
    # the same host link without the library: plain copies of the step's
    # projections from the same pinned buffer, timed with CUDA events; stalls
    # seen here come from the host side of the copies, not from the library
    dst = torch.empty_like(proj)
    st = torch.cuda.current_stream()
    copy_ms = []
    for _ in range(e2e_steps):
        c0, c1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        c0.record(st)
        dst.copy_(h_proj, non_blocking=True)
        c1.record(st)
        torch.cuda.synchronize()
        copy_ms.append(c0.elapsed_time(c1))
    del dst
    return {"value": _job_rate(world, upd_full, e2e_s), "unit": UNIT,
            "h2d_bytes_per_step": int(proj.numel() * proj.element_size()),
            "d2h_bytes_per_step": vol_bytes, "ms_per_step": e2e_s * 1e3, "steps": e2e_steps,
            "ms_per_step_median": float(np.median(step_ms)), "step_ms": [round(t, 2) for t in step_ms],
            "plain_h2d_copy_ms": {"median": float(np.median(copy_ms)), "max": float(max(copy_ms)),
                                  "each": [round(t, 2) for t in copy_ms],
                                  "what": "cudaMemcpyAsync of the step's projections from the same pinned "
                                          "buffer, no library call, CUDA events"},
            "how": "fdk_backproject_host(overwrite) on pinned host buffers: projections in chunks of "
                   "views that double in size (31, 62, 124, 279 for 496) and whose copies overlap the "
                   "back-projection, the last chunk in z-slabs copied out while the next is computed; "
                   "wall clock"}


def run_ours(args):
    import torch
    import torch.distributed as dist

    import synth
    from paper_1401_3615_gb300 import fdk

    world, rank, local = _dist()
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device (no CPU fallback)")
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    cfg = synth.PRESETS[args.config]
    if args.views:
        cfg = synth.preset(args.config, n_views=args.views)
    dev = torch.device("cuda", local)
    scan = synth.make_scan(cfg, device=dev)
    proj, mats = scan["proj"], scan["mats"]
    proj32 = None
    if args.proj_dtype != "f32":
        # storage-precision form: the same filtered projections stored as
        # BF16/FP16; interpolation and accumulation stay FP32
        proj32 = proj
        proj = proj32.to(torch.bfloat16 if args.proj_dtype == "bf16" else torch.float16)
    dims, vs, org = scan["dims"], scan["voxel_size"], scan["origin"]
    vol = torch.zeros((cfg.nz, cfg.ny, cfg.nx), dtype=torch.float32, device=dev)
    upd_full = cfg.updates
    upd_clip = fdk.fdk_count_updates(dims, (cfg.det_w, cfg.det_h), mats, vs, org)
    # launches per step: each 512-view pass runs one launch per ray orientation
    # present (rays mostly along x, mostly along y), as the library does for
    # host matrices on the LDG path
    along_x = np.abs(mats[:, 2, 0]) > np.abs(mats[:, 2, 1])
    passes = 0
    for p0 in range(0, cfg.n_views, 512):
        grp = along_x[p0:p0 + 512]
        passes += (1 if grp.any() else 0) + (1 if (~grp).any() else 0)
    if args.fetch == 2:
        passes = (cfg.n_views + 511) // 512
    stream = torch.cuda.current_stream()

    def step():
        fdk.fdk_backproject(vol, proj, mats, vs, org, fetch=args.fetch, tile=args.tile)

    for _ in range(max(args.warmup, 3)):
        step()
    torch.cuda.synchronize()
    # per-launch durations (a step's launches run back to back), CUDA events on the launching stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    clocks = ClockSampler(local, args.clocks_csv)
    clocks.start()
    time.sleep(0.3)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for k in range(args.steps):
        ev[k][0].record(stream)
        step()
        ev[k][1].record(stream)
    t1.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    total_ms = _max_over_ranks(t0.elapsed_time(t1), world, dev)
    launch_ms = [a.elapsed_time(b) / passes for a, b in ev]
    ms_step = total_ms / args.steps
    value = _job_rate(world, upd_full, ms_step * 1e-3)

    precision = None
    if proj32 is not None:
        precision = _precision_report(args, cfg, scan, proj, proj32, vol, mats, vs, org)

    adjoint = None
    if not args.no_adjoint and proj32 is None:
        adjoint = _adjoint_timing(args, world, dev, proj, vol, mats, vs, org, upd_full, ms_step)

    preprocess = None
    if not args.no_preprocess and proj32 is None:
        preprocess = _preprocess_timing(args, world, dev, proj, mats, cfg)

    e2e = None
    if not args.no_e2e:
        e2e = _e2e(args, world, dev, proj, vol, mats, vs, org, upd_full)

    # the training-system forms on their own workloads, beside the plain FP32 form
    batched = None
    if world == 1 and not args.no_batched and proj32 is None:
        batched = {key: _batched_leg(args, cfgs, label, max(1, min(args.steps, 5)))
                   for key, cfgs, label in _batched_workloads(args)}
    if world == 1 and not args.no_precision and proj32 is None:
        precision = _precision_leg(args)

    out = None
    if rank == 0:
        peaks = _peaks()
        sm_max = float(peaks.get("sm_max_mhz", 2070.0))
        peak_gups = SM_COUNT * FP32_LANES_PER_SM * sm_max * 1e6 / ISSUE_SLOTS_PER_UPDATE / 1e9
        mean_launch = float(np.mean(launch_ms))
        achieved = upd_clip / passes / (mean_launch * 1e-3) / 1e9   # per launch = per step
        tr = MEASURED_TRAFFIC.get((args.config, cfg.n_views, args.fetch, args.tile))
        traffic = tr["bytes"] if tr and tr["sources"] == _sources_sha() else None
        roofline = {"bound": "alu", "achieved": achieved, "peak": peak_gups, "unit": UNIT,
                    "frac": achieved / peak_gups, "traffic": traffic,
                    "traffic_unit": "bytes per launch (ncu dram read + write)",
                    "peak_basis": (f"{SM_COUNT} SMs x {FP32_LANES_PER_SM} FP32 lanes x {sm_max:.0f} MHz "
                                   f"/ {ISSUE_SLOTS_PER_UPDATE} issue slots per update"),
                    "achieved_basis": (f"clipped updates {upd_clip:.4e} per step / step time "
                                       f"({passes} launches of the same kernel per step)"),
                    "achieved_full_count": upd_full / passes / (mean_launch * 1e-3) / 1e9}
        if clk.get("sm_mhz"):
            roofline["peak_at_measured_clock"] = peak_gups * clk["sm_mhz"] / sm_max
        # the other ceilings, in the same clipped updates: HBM at the algorithmic bytes of a step
        # (the volume read and written once per launch, every view read once)
        alg_bytes = passes * 2 * vol.numel() * 4 + proj.numel() * proj.element_size()
        hbm = float(peaks.get("hbm_gbs", 6800.0))
        roofline["ceilings"] = {
            "issue_gups": peak_gups,
            "hbm_measured_gups": hbm * 1e9 / (alg_bytes / upd_clip) / 1e9,
            "hbm_nominal_gups": 7900.0 * 1e9 / (alg_bytes / upd_clip) / 1e9,
            "algorithmic_bytes_per_step": alg_bytes,
            "binding": "issue",
        }
        accuracy = None
        if not args.no_accuracy and proj32 is None:
            accuracy = _accuracy(args, scan, proj, mats, vs, org, dims)
        cpu = None
        if world == 1 and not args.no_cpu:
            import oracle
            oracle.build()
            threads = os.cpu_count() or 1
            rate, desc, _ = _cpu_sample(cfg, proj.float().cpu().numpy(), mats, dims, vs, org,
                                        args.cpu_seconds, threads)
            cpu = {"value": rate / 1e9, "unit": UNIT, "cores": threads, "cpu_model": _cpu_model(),
                   "kind": "oracle", "sample": desc}
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": _workload(args, cfg),
                       "updates_per_step": upd_full, "clipped_updates_per_step": upd_clip,
                       "l2": (f"inputs larger than L2 (projections {proj.numel() * proj.element_size() / 1e9:.2f} GB, "
                              f"volume {vol.numel() * 4 / 2**20:.0f} MiB)"),
                       "fetch": args.fetch, "tile": args.tile,
                       "parallelism": "replicas" if world > 1 else "single GPU"},
            "value_is": ("the forward back-projection (fdk_backproject): voxel updates nx*ny*nz*N per step "
                         "over the step time (the full count); the adjoint is reported under 'adjoint' and "
                         "both under 'figures' in both update counts"),
            "figures": {
                "forward": {"ms_per_step": ms_step, "gups_full_count": value,
                            "gups_clipped": _job_rate(world, upd_clip, ms_step * 1e-3)},
                "adjoint": None if adjoint is None else {
                    "ms_per_step": adjoint["ms_per_step"], "gups_full_count": adjoint["value"],
                    "gups_clipped": _job_rate(world, upd_clip, adjoint["ms_per_step"] * 1e-3),
                    "ratio_to_forward": adjoint["ratio_to_forward"]},
                "update_counts": {"full": upd_full, "clipped": upd_clip,
                                  "clipped_is": "voxel/view pairs with w > 0, -1 < u < W, -1 < v < H "
                                                "(the paper's GUp/s basis)"}},
            "accuracy": accuracy,
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": e2e,
            "adjoint": adjoint,
            "preprocess": preprocess,
            "precision": precision,
            "batched": batched,
            "gpu_launches": args.steps * passes,
            "clocks": clk,
            "clipped_gups": _job_rate(world, upd_clip, ms_step * 1e-3),
            "paper_context": {"xeon_phi_5110p_asm_512": PAPER_PHI_GUPS},
        }
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


def _batched_leg(args, cfgs, label: str, steps: int) -> dict:
    """The batched form on one set of scans: one autotuned plan (executed,
    and replayed from a CUDA graph) against sequential fdk_backproject calls
    with default options; the batch's volumes are compared with the
    sequential ones bit for bit."""
    import torch
    import synth
    from paper_1401_3615_gb300 import fdk
    scans = []
    for c in cfgs:
        sc = synth.make_scan(c, device="cuda")
        scans.append((torch.zeros((c.nz, c.ny, c.nx), device="cuda"), sc["proj"], sc["mats"],
                      sc["voxel_size"], sc["origin"]))
        del sc
    updates = sum(c.updates for c in cfgs)
    stream = torch.cuda.current_stream()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

    def timed(fn):
        for _ in range(max(args.warmup, 3)):
            fn()
        torch.cuda.synchronize()
        t0.record(stream)
        for _ in range(steps):
            fn()
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / steps

    def sequential_default():
        for vol, proj, mats, vs, org in scans:
            fdk.fdk_backproject(vol, proj, mats, vs, org)

    plan = fdk.fdk_batch_plan_create(scans, autotune=True)
    staged = sum(plan.scan_fetch(i) == fdk.FETCH_STAGE for i in range(len(scans)))
    ms_seq = timed(sequential_default)
    ms_batch = timed(plan.execute)
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    s.wait_stream(stream)
    with torch.cuda.graph(g, stream=s):
        plan.execute(stream=s)
    ms_graph = timed(g.replay)
    # one execution from zero against the same sequential calls: bit for bit
    equal = True
    for i, (vol, proj, mats, vs, org) in enumerate(scans):
        ref = torch.zeros_like(vol)
        if plan.scan_fetch(i) == fdk.FETCH_STAGE:
            fdk.fdk_backproject(ref, proj, mats, vs, org, fetch=fdk.FETCH_STAGE)
        else:
            fdk.fdk_backproject(ref, proj, mats, vs, org, fetch=fdk.FETCH_LDG, tile=plan.tile)
        vol.zero_()
        scans[i] = (ref, proj, mats, vs, org, vol)
    plan.execute()
    torch.cuda.synchronize()
    for ref, *_rest, vol in scans:
        equal = equal and bool(torch.equal(ref, vol))
    tile = plan.tile
    plan.close()
    del scans, g
    torch.cuda.empty_cache()
    return {"workload": label, "scans": len(cfgs), "views_total": sum(c.n_views for c in cfgs),
            "updates_per_step": updates, "autotuned_tile": tile, "staged_scans": staged,
            "batch_ms": ms_batch, "graph_replay_ms": ms_graph, "sequential_default_ms": ms_seq,
            "batch_gups": updates / (ms_graph * 1e-3) / 1e9, "sequential_gups": updates / (ms_seq * 1e-3) / 1e9,
            "speedup_vs_sequential": ms_seq / ms_graph, "bitwise_equal_to_sequential_calls": equal}


def _batched_workloads(args):
    """The two batched workloads; a count of 0 leaves that workload out."""
    import synth
    out = []
    if args.batch_scans > 0:
        out.append((f"uneven_{args.batch_scans}_scans", synth.batch_scan_configs(args.batch_scans),
                    f"{args.batch_scans} seeded scans: volumes 64..384 per axis, 120..496 views, detectors "
                    "640x480..1248x960, FP32 (each fills the GPU alone)"))
    if args.small_batch_scans > 0:
        out.append((f"small_{args.small_batch_scans}_scans", synth.small_batch_scan_configs(args.small_batch_scans),
                    f"{args.small_batch_scans} seeded small scans: volumes 32..96 per axis, 60..180 views, "
                    "detectors 320x240..640x480, FP32 (each under-fills the GPU alone)"))
    return out


def run_batched(args):
    """The batched form (one JSON line): an autotuned plan against
    sequential default calls on 32 uneven scans and on many small ones."""
    import torch
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    work = _batched_workloads(args)
    if not work:
        raise SystemExit("--batched needs --batch-scans or --small-batch-scans above 0")
    legs = [_batched_leg(args, cfgs, label, args.steps) for _key, cfgs, label in work]
    main = legs[0]
    line = {
        "metric": "GUp/s, scans of uneven size in one persistent launch (batched form)",
        "value": main["batch_gups"], "unit": UNIT, "n_gpus": 1, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": main["graph_replay_ms"], "higher_is_better": True, "dtype": "f32",
        "data": "synthetic", "config": {"workload": main["workload"]}, "legs": legs,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def _precision_leg(args) -> dict:
    """The storage-precision form at 1024^3 x 496 views of 1248x960: FP32
    storage (the default staged path) against BF16 and FP16 storage with FP32
    interpolation and accumulation, each timed, with its error against the
    FP32-storage GPU result on the whole volume and against the FP64 oracle
    on a seeded 64^3 sub-block (given the same stored values, and the FP32
    values)."""
    import torch
    import oracle
    import synth
    from paper_1401_3615_gb300 import fdk
    cfg = synth.PRESETS["fdk1024"]
    scan = synth.make_scan(cfg, device="cuda")
    proj32, mats, vs, org = scan["proj"], scan["mats"], scan["voxel_size"], scan["origin"]
    stream = torch.cuda.current_stream()
    vol = torch.zeros((cfg.nz, cfg.ny, cfg.nx), dtype=torch.float32, device="cuda")
    steps = max(1, min(args.steps, 3))

    def timed(p):
        for _ in range(2):
            fdk.fdk_backproject(vol, p, mats, vs, org)
        torch.cuda.synchronize()
        t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0.record(stream)
        for _ in range(steps):
            fdk.fdk_backproject(vol, p, mats, vs, org)
        t1.record(stream)
        torch.cuda.synchronize()
        return t0.elapsed_time(t1) / steps

    out = {"workload": f"fdk1024: {cfg.nx}^3 FP32 volume, {cfg.n_views} views of {cfg.det_w}x{cfg.det_h}",
           "fp32": {"ms_per_step": timed(proj32)}}
    out["fp32"]["gups"] = cfg.updates / (out["fp32"]["ms_per_step"] * 1e-3) / 1e9
    ref = torch.zeros_like(vol)
    fdk.fdk_backproject(ref, proj32, mats, vs, org)
    torch.cuda.synchronize()
    peak = float(ref.abs().max())
    rng = np.random.default_rng(1024)
    n = np.array([cfg.nx, cfg.ny, cfg.nz])
    lo = (n * 5) // 16
    n0 = np.minimum(np.maximum(rng.integers(0, n - 64 + 1), lo), n - lo - 64)
    zz, yy, xx = np.meshgrid(*(np.arange(n0[a], n0[a] + 64) for a in (2, 1, 0)), indexing="ij")
    xyz = np.stack([xx.ravel(), yy.ravel(), zz.ravel()], 1)
    threads = os.cpu_count() or 1
    import concurrent.futures as cf
    chunks = np.array_split(np.arange(len(xyz)), threads)

    def orc(p):
        with cf.ThreadPoolExecutor(threads) as ex:
            return np.concatenate(list(ex.map(lambda idx: oracle.backproject_voxels(
                p, mats, vs, org, xyz[idx]), chunks)))
    o_exact = orc(proj32.cpu().numpy())
    pk = float(np.abs(o_exact).max())
    for name, dt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
        p16 = proj32.to(dt)
        ms = timed(p16)
        low = torch.zeros_like(vol)
        fdk.fdk_backproject(low, p16, mats, vs, org)
        torch.cuda.synchronize()
        diff = (low.double() - ref.double())
        mse = float((diff ** 2).mean())
        mx = float(diff.abs().max())
        del diff
        o_stored = orc(p16.float().cpu().numpy())
        g = low[xyz[:, 2], xyz[:, 1], xyz[:, 0]].cpu().numpy().astype(np.float64)
        out[name] = {"ms_per_step": ms, "gups": cfg.updates / (ms * 1e-3) / 1e9,
                     "vs_fp32_storage_gpu_whole_volume": {
                         "max_abs_over_peak": mx / peak,
                         "psnr_db": float(10 * np.log10(peak ** 2 / mse)) if mse > 0 else float("inf")},
                     "subblock_64_vs_oracle_same_stored_values": float(np.abs(g - o_stored).max()) / pk,
                     "subblock_64_vs_oracle_fp32_values": float(np.abs(g - o_exact).max()) / pk,
                     "storage_rounding_alone": float(np.abs(o_stored - o_exact).max()) / pk}
        del low, p16
    out["subblock_origin_voxel"] = [int(v) for v in n0]
    del vol, ref, scan, proj32
    torch.cuda.empty_cache()
    return out


def run_micro(args):
    """Gather micro-benchmarks (the GB300 counterpart of the paper's gather
    table, Sec. V): one JSON line."""
    import torch
    from paper_1401_3615_gb300 import fdk
    world, rank, local = _dist()
    torch.cuda.set_device(local)
    res = {
        "ldg_warp_loads_per_sm_cycle_by_lines": {str(d): fdk.fdk_microbench(fdk.MICRO_LDG, d)
                                                 for d in (1, 2, 4, 8, 16, 32)},
        "lds_warp_loads_per_sm_cycle_by_conflict": {str(c): fdk.fdk_microbench(fdk.MICRO_LDS, c)
                                                    for c in (1, 2, 4, 8, 32)},
        "tld4_warp_gathers_per_sm_cycle": {str(n): fdk.fdk_microbench(fdk.MICRO_TLD4, n) for n in (64, 1248)},
        "rcp_warp_instr_per_sm_cycle": fdk.fdk_microbench(fdk.MICRO_RCP, 0),
        "dependent_load_cycles_by_ring_kib": {str(k): fdk.fdk_microbench(fdk.MICRO_CHASE, k)
                                              for k in (16, 32768, 1048576)},
    }
    line = {"metric": "gather micro-benchmarks", "impl": "ours", "n_gpus": 1, "data": "synthetic",
            "results": res,
            "notes": ("warp loads / SM / cycle for 4-byte loads whose 32 lanes touch 1..32 distinct 128-byte "
                      "lines (L1-resident); shared loads at 1..32-way bank conflicts; 2x2 texture gathers; "
                      "rcp.approx; one thread's dependent-load latency over 16 KiB (L1), 32 MiB (L2) and "
                      "1 GiB (HBM) rings")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="fdk512")
    ap.add_argument("--fetch", type=int, default=0)
    ap.add_argument("--tile", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--ref-step-seconds", type=float, default=4.0)
    ap.add_argument("--clocks-csv", default=None,
                    help="also write the raw nvidia-smi samples of the timed region to this file")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--no-preprocess", action="store_true")
    ap.add_argument("--no-accuracy", action="store_true",
                    help="skip the whole-volume comparison with the oracle (about 40 s of host time)")
    ap.add_argument("--batched", action="store_true", help="time the batched form instead")
    ap.add_argument("--micro", action="store_true", help="run the gather micro-benchmarks instead")
    ap.add_argument("--batch-scans", type=int, default=32)
    ap.add_argument("--small-batch-scans", type=int, default=128)
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-form key of the line")
    ap.add_argument("--no-precision", action="store_true", help="skip the storage-precision key of the line")
    ap.add_argument("--views", type=int, default=0, help="override the view count (profiling)")
    ap.add_argument("--proj-dtype", default="f32", choices=["f32", "bf16", "f16"],
                    help="projection storage type (the storage-precision form)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.batched:
        return run_batched(args)
    if args.micro:
        return run_micro(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
