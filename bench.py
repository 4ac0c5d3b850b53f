"""Benchmark of the iterative ensemble composite on one GB300 (or N replicas).

Workload (the streaming-sweep point this line is quoted on): 1024 flood masks
of 4096 x 4096 uint8 from the seeded terrain generator (synth), composited
into uint16 counts, overlap classes and RGBA colours.  One step is one pass
of the hot path over the whole ensemble: clear, accumulate every member,
render.

* ``value``: member-pixels/s with the ensemble resident in HBM (the kernel
  reads the members in place); timed with CUDA events on the compute stream.
* ``e2e``: the same metric through the C ABI from pinned HOST memory: every
  step uploads all members through two staging buffers (copy stream,
  events) and reads the rendered buckets and colours back to the host.
* ``roofline``: the accumulation kernel against the measured HBM copy peak,
  its launches timed with CUDA events inside the timed region.
* ``cpu_baseline``: the CPU oracle, single threaded, on a bounded sample of
  the same workload; ``cpu_baseline_all_cores`` runs the same oracle in one
  process per host core (spawned), each on its own members, started together.

``--impl reference`` times the CPU oracle itself on the same workload (each
step a bounded sample of members) and prints its own line.
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

METRIC = "composited member-pixels/s"
UNIT = "member-px/s"
L2_BYTES = 129 * 2 ** 20
HBM_FALLBACK_GBS = 6800.0


def parse_args():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=10)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--width", type=int, default=4096)
    p.add_argument("--height", type=int, default=4096)
    p.add_argument("--members", type=int, default=1024)
    p.add_argument("--chunk", type=int, default=0, help="members per chunk; 0 = the library's automatic depth")
    p.add_argument("--staging", type=int, default=2)
    p.add_argument("--read-path", default="linear", choices=["linear", "texture", "tma"])
    p.add_argument("--seed", type=int, default=2)
    p.add_argument("--cpu-seconds", type=float, default=10.0,
                   help="target CPU time of the oracle baseline sample")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-cpu-all-cores", action="store_true", help="skip the all-cores oracle timing")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--sweep", choices=["readpath", "layout", "streaming", "tiny", "batched", "serving", "ingest",
                                       "compressed", "render"],
                   default=None,
                   help="print one JSON line per point of a workload sweep instead of the bench line")
    p.add_argument("--resident", type=int, default=2048, help="serving: members resident in HBM")
    p.add_argument("--overflow", type=int, default=4096, help="serving: members in pinned host memory")
    p.add_argument("--sessions", type=int, default=16, help="serving: open sessions")
    p.add_argument("--requests", type=int, default=200, help="serving: requests per offered rate")
    p.add_argument("--max-batch", type=int, default=64, help="serving: requests per cycle")
    p.add_argument("--poll-us", type=float, default=100.0, help="serving: host back-off between idle polls")
    p.add_argument("--batch-requests", type=int, default=64,
                   help="batched: requests in the mix (64 is the workload; fewer make a small profiling case)")
    p.add_argument("--batched-streamed", type=int, default=1,
                   help="batched: 1 = also run the 64 requests streamed from pinned host memory")
    p.add_argument("--plain-arm", type=int, default=1,
                   help="serving: 1 = also time the plain per-request pipeline (recompute with the plain calls)")
    p.add_argument("--engine-count-bits", type=int, choices=[16, 32], default=16,
                   help="batched: count width of the engine's planes")
    p.add_argument("--paths", nargs="+", choices=["linear", "texture", "tma"], default=["linear", "texture", "tma"],
                   help="readpath: read paths to time")
    p.add_argument("--formats", nargs="+", choices=["bytes", "bits"], default=["bytes", "bits"],
                   help="compressed: resident mask formats to time (--no-e2e skips the streamed forms)")
    p.add_argument("--staging-mib", type=int, default=1024,
                   help="serving: size of one overflow staging half, MiB (members = this / raster bytes)")
    p.add_argument("--mask-format", choices=["bytes", "bits"], default="bytes",
                   help="serving: store the ensemble as byte or bit-packed masks")
    p.add_argument("--rates", type=float, nargs="+", default=[50, 100, 200, 500],
                   help="serving: offered request rates (per second)")
    p.add_argument("--e2e-mode", choices=["staged", "host_read"], default="staged",
                   help="which host-to-device path the e2e value reports (both are measured)")
    return p.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during the run."""

    QUERY = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.rows = []
        self.windows = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.QUERY}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, ValueError):
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append((time.time(), [x.strip() for x in line.split(",")]))

    def window(self, t0, t1):
        self.windows.append((t0, t1))

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        inside = [r for t, r in self.rows if any(a - 0.15 <= t <= b + 0.15 for a, b in self.windows)]
        rows = inside or [r for _, r in self.rows]
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None

        sm = [num(r[2]) for r in rows if len(r) > 9 and num(r[2]) is not None]
        mx = [num(r[3]) for r in rows if len(r) > 9 and num(r[3]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows if len(r) > 9 for i in range(4)
                          if r[6 + i].lower() in ("active", "1")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows), "samples_in_timed_region": len(inside)}


def max_over_ranks(x: float, world: int, device=None) -> float:
    """The largest of every rank's x (the slowest rank's time); x itself on
    one rank.  Needs an initialised process group when world > 1."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, ms: float) -> float:
    """Units all ranks processed per second, over the slowest rank's time."""
    return world * units_per_rank / (ms * 1e-3)


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": HBM_FALLBACK_GBS}, "fallback"


def profiled_traffic(workload_key: str):
    """DRAM bytes per launch of the accumulation kernel, from the JSON record
    that paper_2104_14667_gb300.ncu_traffic wrote from an ncu capture; None
    unless it was taken on the current kernel source and this workload."""
    from paper_2104_14667_gb300 import ncu_traffic
    path = os.path.join(ROOT, "profiles", f"dram_traffic_count_linear_{workload_key}.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    if rec.get("kernel_source_sha256_16") != ncu_traffic.kernel_source_hash() or rec.get("workload") != workload_key:
        return None
    return float(rec["dram_bytes_per_launch"])


def make_ensemble(args, torch, device):
    import synth
    ens = synth.ensemble(args.seed, args.width, args.height, args.members)
    terrain_dev = torch.from_numpy(ens.terrain).to(device)
    dev = torch.empty((args.members, args.height, args.width), dtype=torch.uint8, device=device)
    synth.fill_masks_torch(ens, dev, terrain_t=terrain_dev)
    del terrain_dev
    return ens, dev


def _oracle_fill(ens, buf, ids, mode):
    import synth
    if mode == "count":
        synth.fill_masks(ens, buf, ids)
    else:
        buf[:] = synth.depths(ens, members=ids)


def _oracle_apply(acc, buf, mode):
    import oracle
    if mode == "count":
        oracle.count_apply(acc, buf, 1)
    else:
        oracle.depth_apply(acc, buf, 1)


def _oracle_buffers(n, h, w, mode):
    if mode == "count":
        return np.empty((n, h, w), dtype=np.uint8), np.zeros((h, w), dtype=np.int64)
    return np.empty((n, h, w), dtype=np.float32), np.zeros((h, w), dtype=np.float64)


def cpu_oracle_rate(ens, members: int, target_s: float, batch: int = 4, mode: str = "count"):
    """The oracle (plain C, one thread) over batches of members of the same
    workload until about target_s seconds of CPU work; member-px/s.  mode
    "count" folds uint8 masks into int64 counts, "mean_depth" float32 depths
    into FP64 sums."""
    h, w = ens.height, ens.width
    buf, acc = _oracle_buffers(batch, h, w, mode)
    done, spent = 0, 0.0
    cycle = target_s > 0 and members < 64     # a small workload is passed over again until target_s
    while done == 0 or (spent < target_s and (cycle or done < members)):
        b = batch if cycle else min(batch, members - done)
        _oracle_fill(ens, buf[:b], [(done + j) % members for j in range(b)], mode)
        t0 = time.perf_counter()
        _oracle_apply(acc, buf[:b], mode)
        spent += time.perf_counter() - t0
        done += b
    return done * w * h / spent, done, spent


def _oracle_worker(seed, width, height, members, first, target_s, barrier, out, mode="count"):
    # one process of the all-cores CPU baseline: members first, first + P, ...
    import synth
    ens = synth.ensemble(seed, width, height, members)
    stride = out["procs"]
    buf, acc = _oracle_buffers(1, height, width, mode)
    ids = list(range(first, members, stride)) or [first % members]
    _oracle_fill(ens, buf, ids[:1], mode)
    _oracle_apply(acc, buf, mode)               # warm: library load, page faults
    barrier.wait()
    done, spent, i = 0, 0.0, 0
    t_start = time.perf_counter()
    while time.perf_counter() - t_start < target_s:
        _oracle_fill(ens, buf, [ids[i % len(ids)]], mode)
        t0 = time.perf_counter()
        _oracle_apply(acc, buf, mode)
        spent += time.perf_counter() - t0
        done += 1
        i += 1
    out[first] = (done, spent, time.perf_counter() - t_start)


def cpu_oracle_rate_all_cores(args, target_s: float, seed=None, width=None, height=None, members=None,
                              mode: str = "count"):
    """The oracle, unchanged, in one spawned process per host core, each on
    its own members of the workload, all starting at one barrier; member-px/s
    = all processes' member-pixels / the longest process's oracle time."""
    import multiprocessing as mp
    seed = args.seed if seed is None else seed
    width = args.width if width is None else width
    height = args.height if height is None else height
    members = args.members if members is None else members
    procs = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict(procs=procs)
        barrier = mgr.Barrier(procs)
        ps = [ctx.Process(target=_oracle_worker, args=(seed, width, height, members, i,
                                                       target_s, barrier, out, mode)) for i in range(procs)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(timeout=600)
        res = [out.get(i) for i in range(procs)]
    if any(r is None for r in res):
        return None
    done = sum(r[0] for r in res)
    spent = max(r[1] for r in res)
    return {"value": done * width * height / spent, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": f"{done} member passes over {procs} processes, one member at a time "
                      f"({spent:.1f} s of oracle time in the longest process)"}


def cpu_baseline_line(args, sweep: str, seed: int, width: int, height: int, members: int, mode: str):
    """One JSON line: the oracle timed on a bounded sample of a sweep's
    workload, one thread and one process per host core (spawned after the GPU
    work, so no process is forked from a CUDA context)."""
    import synth
    ens = synth.ensemble(seed, width, height, members)
    rate, done, spent = cpu_oracle_rate(ens, members, args.cpu_seconds, batch=1, mode=mode)
    one = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{done} member passes over the {members} members of the {width}x{height} workload "
                     f"({spent:.1f} s, one thread)"}
    allc = cpu_oracle_rate_all_cores(args, args.cpu_seconds, seed, width, height, members, mode)
    print(json.dumps({"sweep": sweep, "cpu_baseline": True, "mode": mode, "width": width, "height": height,
                      "members": members, "seed": seed, "one_thread": one, "all_cores": allc}), flush=True)


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    import synth
    ens = synth.ensemble(args.seed, args.width, args.height, args.members)
    per_step = max(1, min(args.members, 4))
    rates = []
    for i in range(args.warmup + args.steps):
        rate, done, spent = cpu_oracle_rate(ens, per_step, 0.0, batch=per_step)
        if i >= args.warmup:
            rates.append((done, spent))
    total_px = sum(d for d, _ in rates) * args.width * args.height
    total_s = sum(s for _, s in rates)
    value = total_px / total_s
    sample = f"{per_step} of {args.members} members of the {args.width}x{args.height} workload per step"
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u8",
        "data": "synthetic",
        "config": workload_config(args),
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def workload_config(args):
    return {"workload": f"{args.members} flood masks of {args.width}x{args.height} uint8 (a streaming-sweep "
                        f"point), uint16 counts, bucket + RGBA render",
            "value_regime": "device resident: the masks already in HBM, one pass = clear + accumulate + render",
            "e2e_regime": "streamed: the masks in pinned host memory, uploaded through the staging buffers "
                          "(or read in place with --e2e-mode host_read), outputs read back to the host",
            "width": args.width, "height": args.height, "members": args.members,
            "read_path": args.read_path, "chunk_members": args.chunk, "staging_buffers": args.staging,
            "seed": args.seed, "l2": "inputs larger than L2 (no flush needed)"}


# How the last pinned_host_buffer was made, for the bench line.
HOST_BUFFER_NOTE = {}


def _h2d_rate(torch, flat, nbytes, reps=2):
    """Best host -> device cudaMemcpyAsync rate (GB/s) of flat[:nbytes]."""
    dst = torch.empty(nbytes, dtype=torch.uint8, device="cuda")
    s = torch.cuda.Stream()
    best = 0.0
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            a.record()
            dst.copy_(flat[:nbytes], non_blocking=True)
            b.record()
        b.synchronize()
        best = max(best, nbytes / (a.elapsed_time(b) * 1e-3) / 1e9)
    del dst
    return best


def pinned_host_buffer(torch, shape):
    """A page-locked host buffer for the e2e leg: anonymous memory advised to
    use transparent huge pages, faulted in, then registered with the driver
    (mapped, so the in-place read path can use it too).  Copy engines read
    buffers of fragmented small pages more slowly: on one box successive
    processes that pinned 17 GB each saw the staged rate fall from 209 to 132
    GB/s while the kernel's own loads held 210, and on another the copy
    engines read a registered 17 GB buffer at 27 GB/s while a 1 GiB buffer of
    torch's pinned allocator went at 210.  So the registered buffer's copy
    rate is probed on its first GiB against such a buffer's, and below 0.9 of
    it the registered buffer is replaced by one from torch's pinned allocator
    (also the fall-back when registering fails).  Returns (tensor, handle for
    release_host_buffer); HOST_BUFFER_NOTE says which buffer it is."""
    import mmap
    n = int(np.prod(shape))
    HOST_BUFFER_NOTE.clear()
    try:
        m = mmap.mmap(-1, n, flags=mmap.MAP_PRIVATE | mmap.MAP_ANONYMOUS)
        if hasattr(mmap, "MADV_HUGEPAGE"):
            m.madvise(mmap.MADV_HUGEPAGE)
        arr = np.frombuffer(m, dtype=np.uint8).reshape(shape)
        arr.fill(0)
        t = torch.from_numpy(arr)
        rc = torch.cuda.cudart().cudaHostRegister(t.data_ptr(), n, 3)   # portable | mapped
        if int(rc) == 0:
            nb = min(n, 1 << 30)
            try:
                probe = _h2d_rate(torch, t.view(-1), nb)
                ref_buf = torch.empty(nb, dtype=torch.uint8, pin_memory=True)
                ref = _h2d_rate(torch, ref_buf, nb)
                del ref_buf
            except Exception:   # no room for the probe: keep the registered buffer
                probe = ref = None
            HOST_BUFFER_NOTE.update(registered_probe_gbs=probe, pinned_probe_gbs=ref)
            if probe is None or probe >= 0.9 * ref:
                HOST_BUFFER_NOTE["kind"] = "huge-page advised, registered"
                return t, (m, t.data_ptr())
            torch.cuda.synchronize()
            torch.cuda.cudart().cudaHostUnregister(t.data_ptr())
            HOST_BUFFER_NOTE["kind"] = "cudaHostAlloc (the registered buffer copied below 0.9 of it)"
        del t, arr
        m.close()   # before the replacement is pinned
    except Exception:
        pass
    HOST_BUFFER_NOTE.setdefault("kind", "cudaHostAlloc")
    return torch.empty(shape, dtype=torch.uint8, pin_memory=True), None


def release_host_buffer(torch, t, handle):
    if handle is not None:
        m, ptr = handle
        torch.cuda.synchronize()
        torch.cuda.cudart().cudaHostUnregister(ptr)
        del t
        try:
            m.close()
        except BufferError:
            pass


def link_peak_gbs(torch, device, nbytes=1 << 30, reps=5):
    """Pinned host -> device cudaMemcpyAsync rate, best of reps (GB/s)."""
    src = torch.empty(nbytes, dtype=torch.uint8, pin_memory=True)
    dst = torch.empty(nbytes, dtype=torch.uint8, device=device)
    s = torch.cuda.Stream(device)
    best = 0.0
    for _ in range(reps + 1):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with torch.cuda.stream(s):
            a.record()
            dst.copy_(src, non_blocking=True)
            b.record()
        b.synchronize()
        best = max(best, nbytes / (a.elapsed_time(b) * 1e-3) / 1e9)
    del src, dst
    return best


def run_ours(args):
    import torch
    from paper_2104_14667_gb300 import binding, metrics

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA device")
    torch.cuda.set_device(local)
    device = torch.device("cuda", local)
    binding.load()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    W, H, N = args.width, args.height, args.members
    P = W * H
    ens, dev_masks = make_ensemble(args, torch, device)
    # a real (non-NULL) stream: the library runs its kernels on it, and the
    # CUDA events below are recorded on the same stream
    stream = torch.cuda.Stream(device)
    torch.cuda.set_stream(stream)
    sampler = ClockSampler(local) if rank == 0 else None
    if sampler:
        sampler.start()

    # ---- value: device-resident ensemble ---------------------------------
    comp = binding.Composite(W, H, read_path=args.read_path, staging_buffers=args.staging,
                             chunk_members=args.chunk, stream=stream.cuda_stream)
    bucket = torch.empty((H, W), dtype=torch.uint8, device=device)
    rgba = torch.empty((H, W, 4), dtype=torch.uint8, device=device)
    k_events = []

    def device_step(timed: bool):
        comp.clear()
        if timed:
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
        comp.add(dev_masks)
        if timed:
            b.record(stream)
            k_events.append((a, b))
        comp.render(bucket_out=bucket, rgba_out=rgba)

    for _ in range(args.warmup):
        device_step(False)
    comp.sync()
    barrier()
    t_start, t_stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    w0 = time.time()
    t_start.record(stream)
    for _ in range(args.steps):
        device_step(True)
    t_stop.record(stream)
    barrier()
    w1 = time.time()
    if sampler:
        sampler.window(w0, w1)
    comp.sync()
    dev_ms = t_start.elapsed_time(t_stop)
    dev_ms = max_over_ranks(dev_ms, world, device)
    kernel_ms = [a.elapsed_time(b) for a, b in k_events]
    kernel_avg_ms = sum(kernel_ms) / len(kernel_ms)
    value = whole_job_rate(args.steps * N * P, world, dev_ms)
    comp.close()

    # roofline of the accumulation kernel (one launch per step on this path)
    peaks, peak_src = measured_peaks()
    alg_bytes = N * P + 2 * 2 * P     # every mask byte once + uint16 count read and write
    achieved = alg_bytes / (kernel_avg_ms * 1e-3) / 1e9
    traffic = profiled_traffic(f"{W}x{H}x{N}") if args.read_path == "linear" else None
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": achieved / peaks["hbm_gbs"], "traffic": traffic,
                "kernel": f"count_linear_kernel<uint16_t> ({args.read_path} read path)",
                "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": kernel_avg_ms,
                "peak_source": f"{peak_src} hbm_gbs (copy test)"}

    # ---- e2e: pinned host ensemble through the C ABI -----------------------
    e2e = None
    link = None
    e2e_launches = 0
    if not args.no_e2e:
        host, host_handle = pinned_host_buffer(torch, (N, H, W))
        host_note = dict(HOST_BUFFER_NOTE)
        host.copy_(dev_masks)
        del dev_masks
        torch.cuda.empty_cache()
        peak_link = link_peak_gbs(torch, device)
        h_bucket = torch.empty((H, W), dtype=torch.uint8, pin_memory=True)
        h_rgba = torch.empty((H, W, 4), dtype=torch.uint8, pin_memory=True)

        def e2e_run(host_read: bool) -> float:
            comp = binding.Composite(W, H, read_path=args.read_path, staging_buffers=args.staging,
                                     chunk_members=args.chunk, stream=stream.cuda_stream,
                                     host_read=host_read)

            def host_step():
                comp.clear()
                comp.add(host)
                comp.render(bucket_out=h_bucket.numpy(), rgba_out=h_rgba.numpy())

            for _ in range(args.warmup):
                host_step()
            barrier()
            w0 = time.time()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                host_step()
            barrier()
            host_s = time.perf_counter() - t0
            if sampler:
                sampler.window(w0, time.time())
            comp.close()
            return max_over_ranks(1e3 * host_s, world, device)

        staged_ms = e2e_run(False)
        direct_ms = e2e_run(True) if args.read_path == "linear" else None
        use_direct = args.e2e_mode == "host_read" and direct_ms is not None
        e2e_ms = direct_ms if use_direct else staged_ms
        e2e_value = whole_job_rate(args.steps * N * P, world, e2e_ms)
        h2d_gbs = N * P / (e2e_ms * 1e-3 / args.steps) / 1e9
        # one traced staged step (outside the timed region) for the overlap fraction
        traced = binding.Composite(W, H, read_path=args.read_path, staging_buffers=args.staging,
                                   chunk_members=args.chunk, stream=stream.cuda_stream, trace=True)
        traced.add(host)
        rec = traced.trace()
        traced.close()
        copies = [(float(a), float(b)) for k, a, b in rec if int(k) == 0]
        kernels = [(float(a), float(b)) for k, a, b in rec if int(k) != 0]
        overlap = metrics.overlap_fraction(copies, kernels)
        copy_busy = sum(b - a for a, b in copies)
        n_chunks = sum(1 for k, _, _ in rec if int(k) == 2)
        chunk_used = -(-N // max(1, n_chunks))
        e2e_launches = 2 if use_direct else n_chunks + 1     # accumulate launches + the render
        e2e = {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": N * P,
               "d2h_bytes_per_step": 5 * P, "ms_per_step": e2e_ms / args.steps,
               "mode": "host_read (kernel loads pinned host memory over the link)" if use_direct
               else f"staged ({args.staging} staging buffers, chunks of {chunk_used} members"
                    f"{' (automatic depth)' if args.chunk == 0 else ''}, copy stream + events)"}
        link = {"h2d_gbs": h2d_gbs, "link_peak_gbs": peak_link, "link_frac": h2d_gbs / peak_link,
                "link_peak_how": "best of 5 pinned 1 GiB cudaMemcpyAsync host->device",
                "staged_h2d_gbs": N * P / (staged_ms * 1e-3 / args.steps) / 1e9,
                "host_read_h2d_gbs": (N * P / (direct_ms * 1e-3 / args.steps) / 1e9) if direct_ms else None,
                "overlap_fraction": overlap, "upload_busy_ms": copy_busy, "chunks": len(copies),
                "host_buffer": dict(host_note)}
        release_host_buffer(torch, host, host_handle)
        del host

    clocks = sampler.stop() if sampler else None

    cpu = cpu_all = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:   # the oracle baseline: rank 0 at N = 1 only
        rate, done, spent = cpu_oracle_rate(ens, N, args.cpu_seconds)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"{done} of {N} members of the {W}x{H} workload ({spent:.1f} s, one thread)"}
        if not args.no_cpu_all_cores:
            cpu_all = cpu_oracle_rate_all_cores(args, args.cpu_seconds)

    if rank == 0:
        launches_per_step = 2
        launches_e2e = e2e_launches if e2e else 0
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": dev_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u8", "data": "synthetic",
            "config": workload_config(args), "roofline": roofline, "cpu_baseline": cpu,
            "cpu_baseline_all_cores": cpu_all, "e2e": e2e,
            "gpu_launches": args.steps * (launches_per_step + (launches_e2e if e2e else 0)),
            "clocks": clocks, "link": link,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


# ---- sweeps: the workload configs' other measurements (one JSON line each) ----

def identity_rows_exact(comp, terrain, levels, rows=(0, 1, -2, -1)) -> bool:
    """Renders the composite's counts and checks sampled rows against the
    nested-threshold identity: every member thresholds the same terrain, so
    count(p) = #{m : w_m > terrain(p)} over the members' water levels (with
    repeats when members cycle through a pool)."""
    got = comp.render_host()["counts"].astype(np.int64)
    lv = np.sort(np.asarray(levels, np.float32))
    rows = sorted({r % terrain.shape[0] for r in rows})
    ident = len(lv) - np.searchsorted(lv, terrain[rows].ravel(), side="right").reshape(len(rows), -1)
    return bool(np.array_equal(got[rows], ident))


def depth_identity_max_error(comp, terrain, levels, rows=(0, 1, -2, -1)) -> float:
    """Renders the mean depth and returns the largest deviation of sampled rows
    from its closed form: every depth is max(w_m - terrain(p), 0), so the sum
    over the members is the sum of the levels above terrain(p) minus their
    number times terrain(p) (FP64, levels sorted once)."""
    got = comp.render_host()["mean"].astype(np.float64)
    lv = np.sort(np.asarray(levels, np.float32)).astype(np.float64)
    suffix = np.append(np.cumsum(lv[::-1])[::-1], 0.0)
    rows = sorted({r % terrain.shape[0] for r in rows})
    t = terrain[rows].astype(np.float64)
    i = np.searchsorted(lv, t.ravel(), side="right").reshape(t.shape)
    ident = (suffix[i] - (len(lv) - i) * t) / len(lv)
    return float(np.abs(got[rows] - ident).max())


def _timed(torch, stream, fn, steps: int, warmup: int) -> float:
    """Average ms of fn() over `steps` runs (CUDA events on `stream`)."""
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for _ in range(steps):
        fn()
    b.record(stream)
    torch.cuda.synchronize()
    return a.elapsed_time(b) / steps


def _busy(rec, kinds):
    return sum(float(e) - float(s) for k, s, e in rec if int(k) in kinds)


def sweep_readpath(args, torch, binding, device, stream):
    """Kernel over 256 device-resident members at 4096x4096 through the
    linear, texture and TMA read paths, uint8 masks and float32 depths."""
    import synth
    W = H = 4096
    N = 256
    P = W * H
    ens = synth.ensemble(3, W, H, N)
    terrain_t = torch.from_numpy(ens.terrain).to(device)
    peaks, _ = measured_peaks()
    for mode in ("count", "mean_depth"):
        elem = 1 if mode == "count" else 4
        if mode == "count":
            data = torch.empty((N, H, W), dtype=torch.uint8, device=device)
            synth.fill_masks_torch(ens, data, terrain_t=terrain_t)
        else:
            data = torch.empty((N, H, W), dtype=torch.float32, device=device)
            synth.fill_depths_torch(ens, data, terrain_t=terrain_t)
        for path, box, conv in (("linear", 0, "kernel"), ("texture", 0, "copy"), ("texture", 0, "kernel"),
                                ("tma", 64, "kernel"), ("tma", 128, "kernel"), ("tma", 256, "kernel")):
            if path not in args.paths:
                continue
            cfg = dict(read_path=path, chunk_members=args.chunk or 32, staging_buffers=args.staging,
                       mode=mode, stream=stream.cuda_stream, tma_box_bytes=box, layout_converter=conv)
            with binding.Composite(W, H, **cfg) as comp:
                def step():
                    comp.clear()
                    comp.add(data)
                ms = _timed(torch, stream, step, args.steps, args.warmup)
                comp.sync()
            with binding.Composite(W, H, trace=True, **cfg) as comp:
                comp.add(data)
                rec = comp.trace()
                if mode == "count":
                    exact, depth_err = identity_rows_exact(comp, ens.terrain, ens.levels), None
                else:
                    depth_err = depth_identity_max_error(comp, ens.terrain, ens.levels)
                    exact = depth_err <= 1e-5 * N
            launches = int(sum(1 for k, _, _ in rec if int(k) == 2))
            kernel_ms = _busy(rec, (2,))
            convert_ms = _busy(rec, (1,))
            plane_rmw = (4 if mode == "count" else 8) * P * launches
            kernel_bytes = N * P * elem + plane_rmw
            line = {"sweep": "readpath", "mode": mode, "read_path": path, "tma_box_bytes": box or None,
                    "layout_converter": conv if path == "texture" else None,
                    "width": W, "height": H,
                    "members": N, "chunk_members": args.chunk or 32, "ms_per_pass": ms,
                    "member_px_per_s": N * P / (ms * 1e-3), "kernel_launches": launches,
                    "kernel_busy_ms": kernel_ms, "conversion_busy_ms": convert_ms,
                    "kernel_alg_gbs": kernel_bytes / (kernel_ms * 1e-3) / 1e9,
                    "kernel_frac_of_hbm": kernel_bytes / (kernel_ms * 1e-3) / 1e9 / peaks["hbm_gbs"],
                    "conversion_gbs": (N * P * elem / (convert_ms * 1e-3) / 1e9) if convert_ms else None,
                    "exact_sampled_rows": exact, "depth_max_abs_error_sampled_rows": depth_err,
                    "depth_tolerance": 1e-5 * N if mode != "count" else None}
            print(json.dumps(line), flush=True)
        del data
        torch.cuda.empty_cache()


def sweep_layout(args, torch, binding, device, stream):
    """Linear buffer -> layered cudaArray conversion rate for every power-of-two
    width and height in 64..16384 (the buffer-to-image transform study)."""
    sides = [64 << i for i in range(9)]
    reps = 4
    for h in sides:
        for w in sides:
            data = torch.randint(0, 2, (reps, h, w), dtype=torch.uint8, device=device)
            line = {"sweep": "layout", "width": w, "height": h, "bytes": w * h}
            for converter in ("copy", "kernel"):
                with binding.Composite(w, h, read_path="texture", chunk_members=1, staging_buffers=2,
                                       trace=True, stream=stream.cuda_stream, layout_converter=converter) as comp:
                    comp.add(data)
                    comp.sync()
                    comp.clear()
                    comp.add(data)
                    rec = comp.trace()
                conv = sorted(float(e) - float(s) for k, s, e in rec if int(k) == 1)
                med = conv[len(conv) // 2]
                line[f"{converter}_ms"] = med
                line[f"{converter}_gbs"] = w * h / (med * 1e-3) / 1e9
            print(json.dumps(line), flush=True)
            del data


def sweep_streaming(args, torch, binding, device, stream, sides=None, counts=None, chunks=None,
                    stagings=None, pool_bytes=16 << 30, plan=None):
    """Members streamed from pinned host memory: member-px/s, H2D GB/s against
    the measured pinned copy rate, copy/compute overlap, MB per 100 ms.  A plan
    entry is (side, members, chunk depth (0 = automatic), staging buffers[,
    read path]); the texture path's conversion runs between each upload and
    its kernel, so its busy time is reported beside the kernel's."""
    import synth
    from paper_2104_14667_gb300 import metrics
    peak = link_peak_gbs(torch, device)
    sides = sides or [512, 1024, 2048, 4096, 8192]
    counts = counts or [16, 64, 256, 1024, 4096]
    if plan is None:
        plan = [(s, n, c, args.staging) for c in sorted({args.chunk or 32, 0}, reverse=True) for s in sides for n in counts]
        for c in (chunks or []):
            plan.append((4096, 1024, c, args.staging))
        for k in (stagings or []):
            plan.append((4096, 1024, args.chunk or 32, k))
        for path in ("texture", "tma"):
            for c in sorted({args.chunk or 32, 0}, reverse=True):
                for k in (2, 3):
                    plan.append((4096, 1024, c, k, path))
        for side in (1024, 4096):
            plan.append((side, 1024, 0, 2, "host_read"))
    plan = [tuple(e) + ("linear",) * (5 - len(e)) for e in plan]
    counts = sorted({e[1] for e in plan})
    pools = {}
    pool_notes = {}   # side -> how its pinned pool was made
    for side, n, chunk, k, path in plan:
        P = side * side
        if side not in pools:
            for old_host, _, old_handle in pools.values():
                release_host_buffer(torch, old_host, old_handle)
            pools.clear()
            torch.cuda.empty_cache()
            pool_n = max(1, min(max(counts), pool_bytes // P))
            ens = synth.ensemble(2, side, side, pool_n)
            dev = torch.empty((pool_n, side, side), dtype=torch.uint8, device=device)
            synth.fill_masks_torch(ens, dev)
            # huge-page advised and registered, like the e2e leg's buffer
            # (and replaced the same way when its copies are slow)
            host, handle = pinned_host_buffer(torch, (pool_n, side, side))
            pool_notes[side] = dict(HOST_BUFFER_NOTE)
            host.copy_(dev)
            del dev
            pools[side] = (host, ens, handle)
        host, ens, _ = pools[side]
        pool_n = host.shape[0]

        def add_all(comp):
            done = 0
            while done < n:
                take = min(pool_n, n - done)
                comp.add(host[:take])
                done += take

        # "host_read": the linear kernel loads the pinned rasters over the link itself
        cfg = dict(chunk_members=chunk, staging_buffers=k, stream=stream.cuda_stream,
                   read_path="linear" if path == "host_read" else path, host_read=path == "host_read")
        with binding.Composite(side, side, **cfg) as comp:
            for _ in range(args.warmup):
                comp.clear()
                add_all(comp)
                comp.sync()
            passes = []
            for _ in range(args.steps):
                t0 = time.perf_counter()
                comp.clear()
                add_all(comp)
                comp.sync()
                passes.append(1e3 * (time.perf_counter() - t0))
            # the median pass: a host link shared with other GPUs' jobs can dip
            # for one pass (copies at a fraction of the rate the same buffer
            # reaches in the next); min and max are reported beside it
            ms = float(np.median(passes))
        with binding.Composite(side, side, trace=True, **cfg) as comp:
            add_all(comp)
            rec = comp.trace()
            exact = identity_rows_exact(comp, ens.terrain, [ens.levels[m % pool_n] for m in range(n)])
        copies = [(float(a), float(b)) for kk, a, b in rec if int(kk) == 0]
        kernels = [(float(a), float(b)) for kk, a, b in rec if int(kk) != 0]
        gbs = n * P / (ms * 1e-3) / 1e9
        # Section 7.1's model over the traced chunks: copy c_i, layout
        # transform m_i (texture path; none on the others), processing p_i;
        # beside the traced wall
        model = {}
        ups = sorted(copies)
        ks = sorted((float(a), float(b)) for kk, a, b in rec if int(kk) == 2)
        ms_conv = sorted((float(a), float(b)) for kk, a, b in rec if int(kk) == 1)
        if ups and len(ups) == len(ks) and len(ms_conv) in (0, len(ks)):
            c = [b - a for a, b in ups]
            pk = [b - a for a, b in ks]
            mk = [b - a for a, b in ms_conv] or [0.0] * len(c)
            model = {"model_wall_ms": metrics.pipeline_wall(c, mk, pk),
                     "traced_wall_ms": max(b for _, b in ks) - min(a for a, _ in ups),
                     "paper_e": metrics.pipeline_ratio(c, mk, pk), "traced_chunks": len(c)}
        busy = {"upload_busy_ms": _busy(rec, (0,)), "conversion_busy_ms": _busy(rec, (1,)),
                "kernel_busy_ms": _busy(rec, (2,))}
        print(json.dumps({"sweep": "streaming", "side": side, "members": n, "chunk_members": chunk,
                          "read_path": path, "staging_buffers": k, "pool_members": pool_n, "ms_per_pass": ms,
                          "ms_per_pass_min": min(passes), "ms_per_pass_max": max(passes), "passes": len(passes),
                          "member_px_per_s": n * P / (ms * 1e-3), "h2d_gbs": gbs,
                          "link_peak_gbs": peak, "link_frac": gbs / peak,
                          "overlap_fraction": metrics.overlap_fraction(copies, kernels),
                          "mb_per_100ms": gbs * 100.0, **model, **busy, "exact_sampled_rows": exact,
                          "host_buffer": pool_notes.get(side)}), flush=True)
    for old_host, _, old_handle in pools.values():
        release_host_buffer(torch, old_host, old_handle)
    pools.clear()


def sweep_batched(args, torch, binding, device, stream):
    """64 composite requests of uneven member counts and raster shapes,
    device resident: 64 sequential plain runs (one context each: clear, add,
    render) against the engine's captured graph (clear every plane, one
    persistent accumulate launch, one persistent render launch), after the
    engine's autotuner picked slab depth and CTAs per SM."""
    import synth
    reqs = synth.batched_requests(4, args.batch_requests)
    terrains, data = {}, []
    for r, (w, h, n) in enumerate(reqs):
        if (w, h) not in terrains:
            t = synth.terrain(4, w, h)
            terrains[(w, h)] = (t, np.sort(t, axis=None), torch.from_numpy(t).to(device))
        t, srt, tdev = terrains[(w, h)]
        ens = synth.ensemble_from_terrain(4, t, n, member_offset=r * 4096, flat_sorted=srt)
        dev = torch.empty((n, h, w), dtype=torch.uint8, device=device)
        synth.fill_masks_torch(ens, dev, terrain_t=tdev)
        data.append(dev)
    terrains.clear()
    member_px = sum(w * h * n for w, h, n in reqs)
    out_plain = [(torch.empty((h, w), dtype=torch.uint8, device=device),
                  torch.empty((h, w, 4), dtype=torch.uint8, device=device)) for w, h, _ in reqs]
    out_batch = [(torch.empty((h, w), dtype=torch.uint8, device=device),
                  torch.empty((h, w, 4), dtype=torch.uint8, device=device)) for w, h, _ in reqs]
    ctxs = [binding.Composite(w, h, staging_buffers=1, chunk_members=1, stream=stream.cuda_stream)
            for w, h, _ in reqs]

    def plain_all():
        for ctx, dev, (b, c) in zip(ctxs, data, out_plain):
            ctx.clear()
            ctx.add(dev)
            ctx.render(bucket_out=b, rgba_out=c)

    ms_plain = _timed(torch, stream, plain_all, args.steps, args.warmup)
    for ctx in ctxs:
        ctx.sync()
        ctx.close()
    eng = binding.Engine(stream=stream.cuda_stream)
    # 16-bit planes, like the plain runs' counts: no request exceeds 65535 members
    bits = args.engine_count_bits
    planes = [eng.add_plane(w, h, bits) for w, h, _ in reqs]
    ops = [eng.op(p, dev) for p, dev in zip(planes, data)]
    rops = [eng.render_op(p, None, b, c) for p, (b, c) in zip(planes, out_batch)]
    t0 = time.perf_counter()
    slab, ctas = eng.tune(ops, repeats=2)
    tune_s = time.perf_counter() - t0
    tuned_cfg = eng.config()
    eng.capture(ops, rops)
    ms_graph = _timed(torch, stream, eng.replay, args.steps, args.warmup)
    eng.sync()
    same = all(torch.equal(a, b) and torch.equal(c, d) for (a, c), (b, d) in zip(out_plain, out_batch))

    def direct():
        eng.clear_many(planes)
        eng.submit(ops)
        eng.render(rops)

    ms_direct = _timed(torch, stream, direct, args.steps, args.warmup)
    eng.sync()
    eng.close()
    peaks, _ = measured_peaks()
    hbm = lambda ms: member_px / (ms * 1e-3) / 1e9
    print(json.dumps({
        "sweep": "batched", "requests": len(reqs), "member_px": member_px,
        "members_total": sum(n for _, _, n in reqs),
        "plain_sequential_ms": ms_plain, "batched_graph_ms": ms_graph, "batched_no_graph_ms": ms_direct,
        "plain_composites_per_s": len(reqs) / (ms_plain * 1e-3),
        "batched_composites_per_s": len(reqs) / (ms_graph * 1e-3),
        "speedup": ms_plain / ms_graph, "plain_member_px_per_s": member_px / (ms_plain * 1e-3),
        "batched_member_px_per_s": member_px / (ms_graph * 1e-3),
        "batched_mask_gbs": hbm(ms_graph), "batched_frac_of_hbm": hbm(ms_graph) / peaks["hbm_gbs"],
        "engine_count_bits": bits,
        "tuned_slab_members": slab, "tuned_ctas_per_sm": ctas, "tune_seconds": tune_s,
        "tuned_config": tuned_cfg, "outputs_identical": bool(same)}), flush=True)
    if args.batched_streamed:
        sweep_batched_streamed(args, torch, binding, device, stream, reqs, data, member_px)


def sweep_batched_streamed(args, torch, binding, device, stream, reqs, data, member_px):
    """The same 64 requests with their masks in pinned host memory: 64 plain
    runs, each streamed through its context's staging buffers (automatic
    chunk depth), against one engine submit of 64 host ops streamed through
    the engine's staging buffers, after the tuner picked slab, schedule, item
    size, staging count and buffer size; one render per request / one render
    launch.  Passes of the two forms alternate; median pass time with CUDA
    events; outputs compared."""
    total = sum(int(d.numel()) for d in data)
    flat, handle = pinned_host_buffer(torch, (total,))
    hosts, off = [], 0
    for d in data:
        n = int(d.numel())
        hosts.append(flat[off:off + n].view(d.shape))
        hosts[-1].copy_(d)
        off += n
    del data
    torch.cuda.empty_cache()
    out_plain = [(torch.empty((h, w), dtype=torch.uint8, device=device),
                  torch.empty((h, w, 4), dtype=torch.uint8, device=device)) for w, h, _ in reqs]
    out_batch = [(torch.empty((h, w), dtype=torch.uint8, device=device),
                  torch.empty((h, w, 4), dtype=torch.uint8, device=device)) for w, h, _ in reqs]
    ctxs = [binding.Composite(w, h, staging_buffers=2, chunk_members=0, stream=stream.cuda_stream)
            for w, h, _ in reqs]

    def plain_all():
        for ctx, src, (b, c) in zip(ctxs, hosts, out_plain):
            ctx.clear()
            ctx.add(src)
            ctx.render(bucket_out=b, rgba_out=c)

    eng = binding.Engine(stream=stream.cuda_stream)
    planes = [eng.add_plane(w, h, args.engine_count_bits) for w, h, _ in reqs]
    ops = [eng.op(p, src) for p, src in zip(planes, hosts)]
    rops = [eng.render_op(p, None, b, c) for p, (b, c) in zip(planes, out_batch)]
    t0 = time.perf_counter()
    eng.tune(ops, repeats=1)
    tune_s = time.perf_counter() - t0
    cfg = eng.config()

    def batched():
        eng.clear_many(planes)
        eng.submit(ops)
        eng.render(rops)

    # The two forms alternate pass by pass, so that a dip of the host link
    # (a link shared with other jobs has them) falls on both alike; medians
    # reported.
    plain_ms, batch_ms = [], []
    for i in range(args.warmup + args.steps):
        a = _timed(torch, stream, plain_all, 1, 0)
        b = _timed(torch, stream, batched, 1, 0)
        if i >= args.warmup:
            plain_ms.append(a)
            batch_ms.append(b)
    ms_plain, ms_batch = float(np.median(plain_ms)), float(np.median(batch_ms))
    eng.sync()
    eng.close()
    for ctx in ctxs:
        ctx.sync()
        ctx.close()
    same = all(torch.equal(a, b) and torch.equal(c, d) for (a, c), (b, d) in zip(out_plain, out_batch))
    peak = link_peak_gbs(torch, device)
    gbs = lambda ms: member_px / (ms * 1e-3) / 1e9
    print(json.dumps({
        "sweep": "batched_streamed", "requests": len(reqs), "member_px": member_px,
        "plain_sequential_ms": ms_plain, "batched_ms": ms_batch, "speedup": ms_plain / ms_batch,
        "plain_ms_each": plain_ms, "batched_ms_each": batch_ms,
        "plain_composites_per_s": len(reqs) / (ms_plain * 1e-3),
        "batched_composites_per_s": len(reqs) / (ms_batch * 1e-3),
        "plain_h2d_gbs": gbs(ms_plain), "batched_h2d_gbs": gbs(ms_batch), "link_peak_gbs": peak,
        "batched_link_frac": gbs(ms_batch) / peak, "tuned_config": cfg, "tune_seconds": tune_s,
        "outputs_identical": bool(same)}), flush=True)
    release_host_buffer(torch, flat, handle)


def sweep_ingest(args, torch, binding, device, stream):
    """Host ingest (step a2): pageable host rasters copied into the pinned
    ring, then uploaded through the staging buffers, against pinned rasters
    uploaded directly; 256 masks of 4096x4096 (4.3 GB), wall clock per pass."""
    import synth
    W = H = 4096
    N = args.members if args.members != 1024 else 256
    ens = synth.ensemble(7, W, H, N)
    dev = torch.empty((N, H, W), dtype=torch.uint8, device=device)
    synth.fill_masks_torch(ens, dev)
    pageable = dev.cpu().numpy()
    pinned = torch.empty((N, H, W), dtype=torch.uint8, pin_memory=True)
    pinned.copy_(dev)
    del dev
    torch.cuda.empty_cache()
    peak = link_peak_gbs(torch, device)
    for kind, data, threads, mode in (("pinned", pinned, 0, "auto"), ("pageable", pageable, 1, "ring"),
                                      ("pageable", pageable, 4, "ring"), ("pageable", pageable, 8, "ring"),
                                      ("pageable", pageable, 0, "ring"), ("pageable", pageable, 0, "auto")):
        with binding.Composite(W, H, chunk_members=args.chunk, staging_buffers=args.staging,
                               stream=stream.cuda_stream, ingest_threads=threads, pageable_ingest=mode) as comp:
            def step():
                comp.clear()
                comp.add(data)
                comp.sync()
            for _ in range(args.warmup):
                step()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                step()
            ms = 1e3 * (time.perf_counter() - t0) / args.steps
            exact = identity_rows_exact(comp, ens.terrain, ens.levels)
        gbs = N * W * H / (ms * 1e-3) / 1e9
        print(json.dumps({"sweep": "ingest", "input": kind, "ingest_threads": threads or "default",
                          "pageable_ingest": mode if kind == "pageable" else None,
                          "width": W, "height": H, "members": N,
                          "chunk_members": args.chunk, "staging_buffers": args.staging, "ms_per_pass": ms,
                          "member_px_per_s": N * W * H / (ms * 1e-3), "gbs": gbs, "link_peak_gbs": peak,
                          "link_frac": gbs / peak, "exact_sampled_rows": exact}), flush=True)

    # The host's own copy rate, pageable -> pinned, in the ring copy's shape
    # (pieces of 4 MiB on a pool of threads), without the GPU: the bound the
    # pageable path cannot beat while it copies through a pinned ring.
    import ctypes
    from concurrent.futures import ThreadPoolExecutor
    piece = 4 << 20
    total = N * W * H
    src_addr = pageable.ctypes.data
    dst_addr = pinned.data_ptr()
    offsets = list(range(0, total, piece))
    for threads in (1, 4, 8, 16):
        with ThreadPoolExecutor(max_workers=threads) as ex:
            def copy_all():
                list(ex.map(lambda o: ctypes.memmove(dst_addr + o, src_addr + o, min(piece, total - o)), offsets))
            copy_all()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                copy_all()
            ms = 1e3 * (time.perf_counter() - t0) / args.steps
        print(json.dumps({"sweep": "ingest", "input": "host memcpy pageable->pinned (no GPU)", "threads": threads,
                          "piece_bytes": piece, "bytes": total, "ms_per_pass": ms,
                          "gbs": total / (ms * 1e-3) / 1e9}), flush=True)

    # The same by hand, outside the library: register the pageable batch with
    # the driver for the call (page-locking it in place), upload it as pinned
    # memory, and unregister it afterwards.
    cudart = torch.cuda.cudart()
    with binding.Composite(W, H, chunk_members=args.chunk, staging_buffers=args.staging,
                           stream=stream.cuda_stream) as comp:
        def step_registered():
            rc = cudart.cudaHostRegister(src_addr, total, 0)
            if int(rc) != 0:
                raise RuntimeError(f"cudaHostRegister failed: {rc}")
            try:
                comp.clear()
                comp.add(pageable)
                comp.sync()
            finally:
                cudart.cudaHostUnregister(src_addr)
        step_registered()
        reg_ms = []
        for _ in range(args.steps):
            t0 = time.perf_counter()
            step_registered()
            reg_ms.append(1e3 * (time.perf_counter() - t0))
        exact = identity_rows_exact(comp, ens.terrain, ens.levels)
    ms = sum(reg_ms) / len(reg_ms)
    gbs = total / (ms * 1e-3) / 1e9
    print(json.dumps({"sweep": "ingest", "input": "pageable, registered for the call (cudaHostRegister + add + "
                      "unregister)", "width": W, "height": H, "members": N, "ms_per_pass": ms, "gbs": gbs,
                      "link_peak_gbs": peak, "link_frac": gbs / peak, "exact_sampled_rows": exact}), flush=True)


def sweep_serving(args, torch, binding, device, stream):
    """The interactive server: a resident ensemble in HBM plus overflow members
    in pinned host memory, sessions toggling member subsets on a Poisson
    trace; continuous batching against serving one request at a time, on the
    same trace.  Latency = completion seen by the host - scheduled arrival."""
    import synth
    from paper_2104_14667_gb300 import metrics
    W = H = args.width
    R, O = args.resident, args.overflow
    try:
        ram = os.sysconf("SC_PAGE_SIZE") * os.sysconf("SC_PHYS_PAGES")
    except (ValueError, OSError):
        ram = 0
    if ram and O * W * H > 0.4 * ram:
        O = int(0.4 * ram // (W * H))
    t_setup = time.perf_counter()
    ens = synth.ensemble(5, W, H, R + O)
    tdev = torch.from_numpy(ens.terrain).to(device)
    bits = args.mask_format == "bits"
    WB = W // 8 if bits else W
    step = 256
    tmp = torch.empty((step, H, W), dtype=torch.uint8, device=device)
    resident = torch.empty((R, H, WB), dtype=torch.uint8, device=device)
    for m0 in range(0, R, step):
        m1 = min(R, m0 + step)
        synth.fill_masks_torch(ens, tmp[: m1 - m0], range(m0, m1), terrain_t=tdev)
        resident[m0:m1] = synth.pack_masks_torch(tmp[: m1 - m0]) if bits else tmp[: m1 - m0]
    overflow = torch.empty((O, H, WB), dtype=torch.uint8, pin_memory=True) if O else None
    for m0 in range(0, O, step):
        m1 = min(O, m0 + step)
        synth.fill_masks_torch(ens, tmp[: m1 - m0], range(R + m0, R + m1), terrain_t=tdev)
        overflow[m0:m1].copy_(synth.pack_masks_torch(tmp[: m1 - m0]) if bits else tmp[: m1 - m0])
    del tmp
    torch.cuda.synchronize()
    setup_s = time.perf_counter() - t_setup
    sorted_levels = ens.levels
    n_sessions = args.sessions
    outs = [(torch.empty((H, W), dtype=torch.uint8, device=device),
             torch.empty((H, W, 4), dtype=torch.uint8, device=device)) for _ in range(n_sessions)]

    staging = max(1, min(4096, (args.staging_mib << 20) // (H * WB)))

    def run(trace, max_batch, cycles_in_flight):
        checks = {}
        with binding.Server(resident, overflow, max_sessions=n_sessions, max_batch=max_batch,
                            staging_members=staging, max_cycles_in_flight=cycles_in_flight,
                            stream=stream.cuda_stream, mask_format=args.mask_format,
                            width=W if bits else None) as srv:
            sessions = [srv.open_session() for _ in range(n_sessions)]
            sets = [np.zeros(R + O, bool) for _ in range(n_sessions)]
            arrival, done_at = {}, {}
            t0 = time.perf_counter()
            i = 0
            while i < len(trace) or len(done_at) < len(trace):
                now = time.perf_counter() - t0
                while i < len(trace) and trace[i][0] <= now:
                    t_arr, s, ids = trace[i]
                    for t in ids:
                        sets[s][t] ^= True
                    if i % 25 == 0:
                        c = torch.empty((H, W), dtype=torch.int32, device=device)
                        rid = srv.request(sessions[s], ids, c, None, None)
                        checks[rid] = (c, np.flatnonzero(sets[s]))
                    else:
                        rid = srv.request(sessions[s], ids, None, *outs[s])
                    arrival[rid] = t_arr
                    i += 1
                done = srv.pump()
                for rid in done:
                    done_at[rid] = time.perf_counter() - t0
                if not done and (i >= len(trace) or trace[i][0] > time.perf_counter() - t0):
                    time.sleep(args.poll_us * 1e-6)     # back off: hot polling slows the host link
                if time.perf_counter() - t0 > 300:
                    raise RuntimeError("serving run exceeded 300 s")
            wall = max(done_at.values()) - trace[0][0]
            stats = srv.stats()
        torch.cuda.synchronize()
        lat = [1e3 * (done_at[r] - arrival[r]) for r in done_at]
        # exactness: sampled requests against the terrain-threshold identity
        exact = True
        for rid, (c, members) in checks.items():
            lv = np.sort(sorted_levels[members])
            ident = len(members) - np.searchsorted(lv, ens.terrain.ravel(), side="right").reshape(H, W)
            exact &= bool(np.array_equal(c.cpu().numpy().astype(np.int64), ident))
        return {"composites_per_s": len(trace) / wall, "p50_ms": metrics.percentile(lat, 50),
                "p99_ms": metrics.percentile(lat, 99), "mean_ms": float(np.mean(lat)), "wall_s": wall,
                "cycles": stats["cycles"], "overflow_uploads": stats["overflow_uploads"],
                "members_added": stats["members_added"], "members_removed": stats["members_removed"],
                "recomputes": stats["recomputes"], "checked": len(checks), "exact": exact,
                "cycle_device_s": stats["cycle_device_us"] * 1e-6, "enqueue_host_s": stats["enqueue_host_us"] * 1e-6}

    def runs_of(ids):
        """Maximal runs of consecutive ids as (first, length)."""
        out = []
        for i in ids:
            if out and out[-1][0] + out[-1][1] == i:
                out[-1][1] += 1
            else:
                out.append([int(i), 1])
        return out

    def run_plain(trace):
        """The plain per-request pipeline: no server, one composite context
        per session (32-bit counts), and every request recomputed from its
        session's member set with the plain calls -- clear, one add per run of
        consecutive member ids (resident runs read in place, overflow runs
        streamed through the staging buffers), render -- one request at a time
        in arrival order."""
        ctxs = [binding.Composite(W, H, count_bits=32, stream=stream.cuda_stream, mask_format=args.mask_format)
                for _ in range(n_sessions)]
        sets = [np.zeros(R + O, bool) for _ in range(n_sessions)]
        lat, checks = [], []
        t0 = time.perf_counter()
        try:
            for i, (t_arr, s, ids) in enumerate(trace):
                now = time.perf_counter() - t0
                if t_arr > now:
                    time.sleep(t_arr - now)
                for t in ids:
                    sets[s][t] ^= True
                members = np.flatnonzero(sets[s])
                comp = ctxs[s]
                comp.clear()
                for first, length in runs_of(members):
                    if first < R:
                        take = min(length, R - first)
                        comp.add(resident[first:first + take])
                        first, length = first + take, length - take
                    if length:
                        comp.add(overflow[first - R:first - R + length])
                if i % 25 == 0:
                    c = torch.empty((H, W), dtype=torch.int32, device=device)
                    comp.render(counts_out=c)
                    checks.append((c, members))
                else:
                    comp.render(bucket_out=outs[s][0], rgba_out=outs[s][1])
                comp.sync()
                lat.append(1e3 * (time.perf_counter() - t0 - t_arr))
                if time.perf_counter() - t0 > 300:
                    raise RuntimeError("plain serving run exceeded 300 s")
            wall = time.perf_counter() - t0 - trace[0][0]
        finally:
            for comp in ctxs:
                comp.close()
        exact = True
        for c, members in checks:
            lv = np.sort(sorted_levels[members])
            ident = len(members) - np.searchsorted(lv, ens.terrain.ravel(), side="right").reshape(H, W)
            exact &= bool(np.array_equal(c.cpu().numpy().astype(np.int64), ident))
        return {"composites_per_s": len(trace) / wall, "p50_ms": metrics.percentile(lat, 50),
                "p99_ms": metrics.percentile(lat, 99), "mean_ms": float(np.mean(lat)), "wall_s": wall,
                "checked": len(checks), "exact": exact}

    for rate in args.rates:
        trace = synth.serving_trace(5, args.requests, rate, n_sessions, R + O)
        batched = run(trace, args.max_batch, 4)
        single = run(trace, 1, 1)      # the queue alone: one request on the device at a time
        plain = run_plain(trace) if args.plain_arm else None
        print(json.dumps({"sweep": "serving", "mask_format": args.mask_format, "rate_per_s": rate,
                          "requests": len(trace), "resident": R,
                          "overflow": O, "side": W, "sessions": n_sessions, "staging_members": staging,
                          "setup_s": setup_s,
                          "toggle_members_mean": float(np.mean([len(t[2]) for t in trace])),
                          "batched": batched, "one_at_a_time": single, "plain_per_request": plain,
                          "throughput_gain": batched["composites_per_s"] / single["composites_per_s"],
                          "p99_gain": single["p99_ms"] / batched["p99_ms"],
                          "throughput_gain_vs_plain": (batched["composites_per_s"] / plain["composites_per_s"]
                                                       if plain else None),
                          "p99_gain_vs_plain": plain["p99_ms"] / batched["p99_ms"] if plain else None}),
              flush=True)


def sweep_compressed(args, torch, binding, device, stream):
    """Bit-packed masks (one bit per pixel) against byte masks on the same
    4096x4096 x 1024 ensemble: device resident (HBM bytes per member-pixel
    1/8) and streamed from pinned host memory (link bytes 1/8)."""
    import synth
    W, H, N = args.width, args.height, args.members
    P = W * H
    ens = synth.ensemble(args.seed, W, H, N)
    tdev = torch.from_numpy(ens.terrain).to(device)
    with_bytes = "bytes" in args.formats
    dev = torch.empty((N if with_bytes else 64, H, W), dtype=torch.uint8, device=device)
    packed = torch.empty((N, H, W // 8), dtype=torch.uint8, device=device)
    for m0 in range(0, N, 64):
        m1 = min(N, m0 + 64)
        part = dev[m0:m1] if with_bytes else dev[: m1 - m0]
        synth.fill_masks_torch(ens, part, range(m0, m1), terrain_t=tdev)
        packed[m0:m1] = synth.pack_masks_torch(part)
    if not with_bytes:
        del dev
        torch.cuda.empty_cache()
    peaks, _ = measured_peaks()
    out = {"sweep": "compressed", "width": W, "height": H, "members": N}
    counts = {}
    for fmt in args.formats:
        data = dev if fmt == "bytes" else packed
        with binding.Composite(W, H, stream=stream.cuda_stream, mask_format=fmt) as comp:
            def step():
                comp.clear()
                comp.add(data)
            ms = _timed(torch, stream, step, args.steps, args.warmup)
            c = np.empty((H, W), np.uint16)
            comp.render(counts_out=c)
            counts[fmt] = c
        bytes_per = 1.0 if fmt == "bytes" else 0.125
        out[f"resident_{fmt}_ms"] = ms
        out[f"resident_{fmt}_member_px_per_s"] = N * P / (ms * 1e-3)
        out[f"resident_{fmt}_read_gbs"] = (N * P * bytes_per + 4 * P) / (ms * 1e-3) / 1e9
        out[f"resident_{fmt}_frac_of_hbm"] = out[f"resident_{fmt}_read_gbs"] / peaks["hbm_gbs"]
    if len(counts) == 2:
        out["counts_identical"] = bool(np.array_equal(counts["bytes"], counts["bits"]))
    if args.no_e2e:     # resident forms only
        print(json.dumps(out), flush=True)
        return
    host_packed = torch.empty((N, H, W // 8), dtype=torch.uint8, pin_memory=True)
    host_packed.copy_(packed)
    if with_bytes:
        del dev
    torch.cuda.empty_cache()
    h_bucket = np.empty((H, W), np.uint8)
    h_rgba = np.empty((H, W, 4), np.uint8)
    for host_read in (False, True):
        with binding.Composite(W, H, stream=stream.cuda_stream, mask_format="bits", chunk_members=255,
                               staging_buffers=args.staging, host_read=host_read) as comp:
            def host_step():
                comp.clear()
                comp.add(host_packed)
                comp.render(bucket_out=h_bucket, rgba_out=h_rgba)
            for _ in range(args.warmup):
                host_step()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                host_step()
            ms = 1e3 * (time.perf_counter() - t0) / args.steps
        key = "streamed_bits_host_read" if host_read else "streamed_bits_staged"
        out[f"{key}_ms"] = ms
        out[f"{key}_member_px_per_s"] = N * P / (ms * 1e-3)
        out[f"{key}_link_gbs"] = N * P / 8 / (ms * 1e-3) / 1e9
    print(json.dumps(out), flush=True)


def sweep_render(args, torch, binding, device, stream):
    """The render step alone (counts -> overlap classes -> colours, optionally
    the class histogram) at 4096^2 and 8192^2, device outputs."""
    import synth
    for side in (4096, 8192):
        P = side * side
        m = torch.empty((16, side, side), dtype=torch.uint8, device=device)
        ens = synth.ensemble(6, side, side, 16)
        synth.fill_masks_torch(ens, m)
        bucket = torch.empty((side, side), dtype=torch.uint8, device=device)
        rgba = torch.empty((side, side, 4), dtype=torch.uint8, device=device)
        counts = torch.empty((side, side), dtype=torch.int16, device=device)
        hist = torch.empty(256, dtype=torch.int64, device=device)
        with binding.Composite(side, side, stream=stream.cuda_stream) as comp:
            comp.add(m)
            variants = {
                "bucket+rgba": (lambda: comp.render(bucket_out=bucket, rgba_out=rgba), 2 + 1 + 4),
                "counts+bucket+rgba": (lambda: comp.render(counts, bucket, rgba), 2 + 2 + 1 + 4),
                "bucket+rgba+histogram": (lambda: comp.render_histogram(hist, bucket_out=bucket, rgba_out=rgba), 2 + 1 + 4),
                "histogram only": (lambda: comp.render_histogram(hist), 2),
            }
            for name, (fn, bpp) in variants.items():
                ms = _timed(torch, stream, fn, 50, 5)
                print(json.dumps({"sweep": "render", "side": side, "outputs": name, "us": 1e3 * ms,
                                  "gbs": bpp * P / (ms * 1e-3) / 1e9}), flush=True)
            comp.sync()
        del m
        torch.cuda.empty_cache()
    sweep_render_engine(args, torch, binding, device, stream)


def sweep_render_engine(args, torch, binding, device, stream):
    """The engine's render launch alone over the batched mix's 64 plane shapes
    (bucket + RGBA device outputs into 16-bit planes), against 64 plain
    renders of the same planes: 2 + 1 + 4 bytes per pixel.  Then both again
    with a class histogram per plane (the engine zeroes the 64 histograms in
    one clear launch before its render).  Two inputs: two random members per
    plane (salt-and-pepper classes 0 / 127 / 255, the worst case for counting
    runs of equal classes) and 32 members of one terrain ensemble, each plane
    a crop of one 4096 x 4096 terrain (smooth class fields, noisy edges)."""
    import synth
    reqs = synth.batched_requests(4, args.batch_requests)
    px = sum(w * h for w, h, _ in reqs)
    side = max(max(w, h) for w, h, _ in reqs)
    ens = synth.ensemble(4, side, side, 32)
    terrain = torch.from_numpy(ens.terrain).to(device)
    peaks, _ = measured_peaks()
    gbs = lambda ms: 7 * px / (ms * 1e-3) / 1e9
    for kind in ("random2", "terrain32"):
        gen = torch.Generator(device=device)
        gen.manual_seed(8)
        eng = binding.Engine(stream=stream.cuda_stream)
        planes, outs, ctxs = [], [], []
        for w, h, _ in reqs:
            if kind == "random2":
                m = torch.randint(0, 2, (2, h, w), dtype=torch.uint8, device=device, generator=gen)
            else:
                crop = terrain[:h, :w]
                m = torch.stack([(crop < float(lv)).to(torch.uint8) for lv in ens.levels])
            p = eng.add_plane(w, h, 16)
            eng.submit([eng.op(p, m)])
            ctx = binding.Composite(w, h, stream=stream.cuda_stream, staging_buffers=1, chunk_members=1)
            ctx.add(m)                    # device masks are read in place: no staging used
            planes.append(p)
            ctxs.append(ctx)
            outs.append((torch.empty((h, w), dtype=torch.uint8, device=device),
                         torch.empty((h, w, 4), dtype=torch.uint8, device=device)))
            eng.sync()
            del m
        rops = [eng.render_op(p, None, b, c) for p, (b, c) in zip(planes, outs)]
        ms_engine = _timed(torch, stream, lambda: eng.render(rops), 50, 5)

        def plain():
            for ctx, (b, c) in zip(ctxs, outs):
                ctx.render(bucket_out=b, rgba_out=c)

        ms_plain = _timed(torch, stream, plain, 50, 5)
        hists = [torch.empty(256, dtype=torch.int64, device=device) for _ in planes]
        hrops = [eng.render_op(p, None, b, c, hg) for p, (b, c), hg in zip(planes, outs, hists)]
        ms_engine_hist = _timed(torch, stream, lambda: eng.render(hrops), 50, 5)

        def plain_hist():
            for ctx, (b, c), hg in zip(ctxs, outs, hists):
                ctx.render_histogram(hg, bucket_out=b, rgba_out=c)

        ms_plain_hist = _timed(torch, stream, plain_hist, 50, 5)
        eng.render(hrops)
        eng.sync()
        # every histogram against a count of the bucket image rendered with it
        hist_ok = all(torch.equal(hg, torch.bincount(b.flatten(), minlength=256)) for hg, (b, _) in zip(hists, outs))
        classes = int(sum((hg > 0).sum() for hg in hists)) / len(hists)
        for ctx in ctxs:
            ctx.sync()
            ctx.close()
        eng.close()
        print(json.dumps({"sweep": "render_engine", "input": kind, "planes": len(reqs), "pixels": px,
                          "mean_classes_per_plane": classes,
                          "engine_us": 1e3 * ms_engine, "engine_gbs": gbs(ms_engine),
                          "engine_frac_of_hbm": gbs(ms_engine) / peaks["hbm_gbs"],
                          "plain_us": 1e3 * ms_plain, "plain_gbs": gbs(ms_plain),
                          "engine_hist_us": 1e3 * ms_engine_hist, "engine_hist_gbs": gbs(ms_engine_hist),
                          "plain_hist_us": 1e3 * ms_plain_hist, "hist_equals_bucket_count": hist_ok}), flush=True)


def run_sweep(args):
    import torch
    from paper_2104_14667_gb300 import binding
    if not torch.cuda.is_available():
        raise SystemExit("bench.py --sweep needs a CUDA device")
    device = torch.device("cuda", 0)
    torch.cuda.set_device(device)
    stream = torch.cuda.Stream(device)
    torch.cuda.set_stream(stream)
    binding.load()
    if args.sweep == "readpath":
        sweep_readpath(args, torch, binding, device, stream)
        if not args.no_cpu_baseline:
            for mode in ("count", "mean_depth"):
                cpu_baseline_line(args, "readpath", 3, 4096, 4096, 256, mode)
    elif args.sweep == "layout":
        sweep_layout(args, torch, binding, device, stream)
    elif args.sweep == "streaming":
        sweep_streaming(args, torch, binding, device, stream, chunks=[1, 2, 4, 8, 16, 64, 128],
                        stagings=[1, 3, 4])
    elif args.sweep == "render":
        sweep_render(args, torch, binding, device, stream)
    elif args.sweep == "compressed":
        sweep_compressed(args, torch, binding, device, stream)
    elif args.sweep == "serving":
        sweep_serving(args, torch, binding, device, stream)
    elif args.sweep == "ingest":
        sweep_ingest(args, torch, binding, device, stream)
    elif args.sweep == "batched":
        sweep_batched(args, torch, binding, device, stream)
    elif args.sweep == "tiny":
        sweep_streaming(args, torch, binding, device, stream,
                        plan=[(1024, 16, c, k) for c in (16, 1, 2, 4, 8) for k in (2, 1)] +
                             [(1024, 16, 0, 2), (1024, 16, 16, 2, "host_read")])
        if not args.no_cpu_baseline:
            cpu_baseline_line(args, "tiny", 1, 1024, 1024, 16, "count")


def main():
    args = parse_args()
    if args.sweep:
        run_sweep(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
