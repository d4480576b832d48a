#!/usr/bin/env python3
"""Benchmark of the voxelization hot path on GB300.

Headline: the arbitrary-length batch (Table 4 shape), the largest workload that
fits one GPU: 4,194,304 segments with major |delta| log-uniform in [0, 4095] in
a 4096^3 volume. One step = one pass of the whole path: count + decoupled
look-back scan, the packed 64-bit list (2.07e9 voxels, 16.5 GB) and the fresh
1-bit occupancy volume (8 GiB) built by brick ownership. Inputs are resident in
HBM; the step's outputs (24.5 GB) are far larger than L2, and L2 is also
flushed (a 256 MiB write) between timed steps, outside the step's events.

Beside it, each with its own roofline: the fixed-length batch (Table 3 shape,
1M x 64 voxels + one 1023-step segment, 1024^3, list32 + fresh volume), the
4096-segment case as a launch-latency block (microseconds per call), batched
scenes against per-scene launches, the served request stream at two offered
rates, the Section 5 sweeps, the brick-major layout and the Euclidean-N variant.

Prints ONE JSON line (rank 0). ``--impl reference`` times the CPU oracle on the
host cores instead (a bounded sample of the same workload per step).
"""

from __future__ import annotations

import argparse
import hashlib
import json
import multiprocessing as mp
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "voxels/s (bit-exact) & % HBM roofline, batched vs plain launch; p99 ms"
UNIT = "voxels/s"
WORKLOAD = ("arbitrary-length batch: 4,194,304 segments, major |delta| log-uniform in [0, 4095], minors uniform "
            "in [-major, major], 4096^3 volume; packed 64-bit list + fresh 1-bit volume (8 GiB)")
WORKLOAD2 = ("fixed-length batch: 1,048,576 segments x 64 voxels + one 1023-step segment, 1024^3 volume; "
             "packed 32-bit list + fresh 1-bit volume")
WORKLOAD1 = "4096 segments, endpoints uniform in [0, 255]^3, 256^3 volume; packed 32-bit list + 1-bit volume"
L2_NOTE = "outputs (24.5 GB) far larger than L2; L2 also flushed between steps by a 256 MiB write (outside events)"
L2_FLUSH_BYTES = 256 << 20
SM_CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                   "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                   "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


def _dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def headline_config(n: int, V: int, dims, world: int) -> dict:
    """The `config` object of both arms (identical, so the two lines describe
    the same workload)."""
    return {"workload": WORKLOAD, "segments": n, "voxels_per_gpu": V, "volume": list(dims),
            "outputs": "list64 + fresh 1-bit volume", "l2": L2_NOTE,
            "parallelism": f"replicas x{world} (independent batches, no data crosses ranks)"}


def _measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except (OSError, ValueError):
        return {"hbm_gbs": 6800.0}, "fallback"


def _kernel_source_hash() -> str:
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_2009_09500_gb300", "csrc")
    for f in sorted(os.listdir(csrc)):
        if f.endswith((".cu", ".cuh")):
            with open(os.path.join(csrc, f), "rb") as fh:
                h.update(f.encode() + b"\0" + fh.read())
    return h.hexdigest()[:16]


def _recorded_field(workload_key: str, kernels, field):
    """Sum of `field` over `kernels` of one workload in the committed ncu record,
    if every entry was taken on the current kernel sources with the launch
    tuning now in force (else None)."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
    except (OSError, ValueError):
        return None
    from paper_2009_09500_gb300 import vox

    now = vox.vox_get_tuning()
    total = 0.0
    for k in kernels:
        ent = rec.get(f"{workload_key}/{k}")
        if not ent or ent.get("source_hash") != _kernel_source_hash() or field not in ent:
            return None
        if ent.get("tuning") is not None and ent["tuning"] != now:
            return None
        total += float(ent[field])
    return total


def _issue(workload_key, kernels, ms: float, sm_mhz: float, sms: int) -> dict | None:
    """Issue-rate view of a phase: warp instructions the kernels executed (ncu
    record, per launch) per second against the issue peak of 4 warp
    instructions per SM per clock at the sampled SM clock."""
    inst = _recorded_field(workload_key, kernels, "warp_instructions")
    if inst is None or not ms or not sm_mhz:
        return None
    peak = 4.0 * sms * sm_mhz * 1e6
    achieved = inst / (ms * 1e-3)
    return {"warp_instructions_per_launch": inst, "achieved_per_s": achieved, "peak_per_s": peak,
            "frac": achieved / peak, "peak_model": f"4 warp instructions/clk/SM x {sms} SMs x {sm_mhz:.0f} MHz"}


def _link_bandwidth(dev, nbytes: int) -> dict:
    """Host link bandwidth (GB/s) with plain pinned copies of `nbytes`, best of
    five, each direction."""
    import torch

    d_buf = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    out = {}
    for name, dst, src in (("d2h", h, d_buf), ("h2d", d_buf, h)):
        ts = []
        for _ in range(6):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            dst.copy_(src, non_blocking=True)
            torch.cuda.synchronize()
            ts.append(time.perf_counter() - t0)
        out[f"{name}_GBps"] = nbytes / min(ts[1:]) / 1e9
    return out


class ClockSampler:
    """nvidia-smi clock/throttle samples while the timed region runs."""

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []
        self.thread = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={SM_CLOCK_FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"], "samples": 0}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        if self.thread:
            self.thread.join(timeout=2)
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
            for nm, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------- CPU oracle
def _cpu_model() -> str:
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    return platform.processor() or platform.machine()


def _oracle_list_part(segs: np.ndarray) -> int:
    """Worker: the oracle's 64-bit list of these segments; returns its length."""
    import oracle

    return int(oracle.get().list64(segs).shape[0])


def _oracle_slab_part(segs: np.ndarray, dims, z0: int, z1: int) -> int:
    """Worker: the oracle's volume slab z in [z0, z1) of these segments."""
    import oracle

    slab = oracle.get().bitmask_zslab(segs, dims, z0, z1)
    return int(slab.shape[0])


def _oracle_init():
    import oracle

    oracle.get()


class CpuOracle:
    """The oracle, unchanged, on the host cores: one core (the oracle itself:
    list64 + volume of a segment sample in order), or `cores` spawn-started
    workers taking disjoint parts of the same computation (the list by segment
    ranges, the volume by z-slabs), which is how the oracle's own functions
    spread over k cores."""

    def __init__(self, cores: int):
        self.cores = max(1, int(cores))
        self.ex = None
        if self.cores > 1:
            from concurrent.futures import ProcessPoolExecutor

            self.ex = ProcessPoolExecutor(self.cores, mp_context=mp.get_context("spawn"), initializer=_oracle_init)
            list(self.ex.map(_oracle_init_probe, range(self.cores)))  # workers up before timing

    def run(self, segs: np.ndarray, dims, mask: np.ndarray | None = None) -> float:
        """Seconds for the list64 + volume of `segs`."""
        import oracle

        if self.ex is None:
            O = oracle.get()
            t0 = time.perf_counter()
            O.list64(segs)
            O.bitmask(segs, dims, mask)
            return time.perf_counter() - t0
        d = int(dims[2])
        slabs = self.cores
        cuts = [d * i // slabs for i in range(slabs + 1)]
        parts = np.array_split(np.arange(segs.shape[0]), self.cores)
        t0 = time.perf_counter()
        futs = [self.ex.submit(_oracle_list_part, segs[p[0]:p[-1] + 1]) for p in parts if len(p)]
        futs += [self.ex.submit(_oracle_slab_part, segs, tuple(dims), cuts[i], cuts[i + 1]) for i in range(slabs)]
        for f in futs:
            f.result()
        return time.perf_counter() - t0

    def close(self):
        if self.ex is not None:
            self.ex.shutdown(wait=True)


def _oracle_init_probe(_):
    return os.getpid()


def cpu_baseline(w, V_total: int, cores: int, max_seconds: float) -> dict:
    """The oracle on a bounded sample of the workload: whole segments from the
    front, in chunks, until about max_seconds of CPU work."""
    import oracle

    O = oracle.get()
    cpu = CpuOracle(cores)
    mask = np.zeros(O.mask_words(w.dims), dtype=np.uint32) if cores == 1 else None
    chunk = 16384 if cores == 1 else 131072
    done, vox_done, t_total = 0, 0, 0.0
    try:
        while done < w.n and t_total < max_seconds:
            part = w.segs[done:done + chunk]
            t_total += cpu.run(part, w.dims, mask)
            vox_done += O.total(part)
            done += part.shape[0]
    finally:
        cpu.close()
    how = ("the oracle itself (list64 + volume, one core)" if cores == 1 else
           f"the oracle's list64 over {cores} segment ranges and its volume over {cores} z-slabs "
           f"(oracle.bitmask_zslab) in {cores} spawn-started processes")
    return {"value": vox_done / t_total, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": _cpu_model(),
            "sample": f"first {done} of {w.n} segments ({vox_done} voxels of {V_total}), {how}, {t_total:.1f} s"}


def run_reference(args):
    rank, world, _ = _dist_env()
    if rank != 0:
        return 0
    from paper_2009_09500_gb300 import workloads
    import oracle

    w = workloads.config3()
    O = oracle.get()
    V = O.total(w.segs)
    cores = os.cpu_count() or 1
    cpu = CpuOracle(cores)
    per_step = 131072  # segments per step: a bounded sample (~6.4e7 voxels)
    times, vox_per = [], []
    try:
        for it in range(args.warmup + args.steps):
            lo = (it * per_step) % (w.n - per_step)
            part = w.segs[lo:lo + per_step]
            dt = cpu.run(part, w.dims)
            if it >= args.warmup:
                times.append(dt)
                vox_per.append(O.total(part))
    finally:
        cpu.close()
    total_t = sum(times)
    value = sum(vox_per) / total_t
    sample = (f"{per_step} consecutive segments per step (~{int(np.mean(vox_per))} voxels): the oracle's list64 over "
              f"{cores} segment ranges and its volume over {cores} z-slabs, {cores} processes")
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1000 * total_t / len(times), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "int64", "data": "synthetic",
        "config": headline_config(w.n, V, w.dims, world),
        "note": "CPU oracle (plain C, unchanged) on the host cores, each step a bounded sample of the workload",
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle", "cpu": _cpu_model(),
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def aggregate_ranks(ms_local: float, voxels_local: int, world: int, device):
    """Whole-job figures over the ranks: the slowest rank's mean step time, the
    voxels of all ranks, and value = all voxels / slowest time (weak scaling:
    every rank voxelizes its own batch; no data crosses ranks)."""
    import torch

    if world > 1:
        import torch.distributed as dist

        t = torch.tensor([ms_local], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        v = torch.tensor([voxels_local], dtype=torch.int64, device=device)
        dist.all_reduce(v, op=dist.ReduceOp.SUM)
        ms_max, total = float(t.item()), int(v.item())
    else:
        ms_max, total = float(ms_local), int(voxels_local)
    return ms_max, total, total / (ms_max / 1000.0)


def vox_tuning_list_runs() -> int:
    from paper_2009_09500_gb300 import vox

    return int(vox.vox_get_tuning()["list_runs"])


# ------------------------------------------------------------ one scene's step
class SceneBench:
    """One scene's whole step (count + scan, the list, a fresh volume by bricks)
    on resident buffers: tuned, timed eagerly phase by phase (events between
    phases) and as batching.SceneStep (the same launches captured once as a CUDA
    graph, list and volume on two streams), outputs checked equal."""

    def __init__(self, key: str, w, list_flag: int, dev, tune: bool, tuning_arg: str = ""):
        import torch

        from paper_2009_09500_gb300 import vox

        self.key, self.w, self.list_flag, self.dev = key, w, list_flag, dev
        self.elem = 8 if list_flag == vox.OUT_LIST64 else 4
        n = w.n
        self.segs = torch.from_numpy(w.segs).to(dev)
        self.status = torch.zeros(1, dtype=torch.int32, device=dev)
        ws = torch.empty(vox.vox_workspace_size_volume(n, w.dims, 0), dtype=torch.uint8, device=dev)
        self.V, self.P = vox.vox_plan(self.segs, w.dims, ws, self.status)
        del ws
        self.ws = torch.empty(vox.vox_workspace_size_volume(n, w.dims, self.P), dtype=torch.uint8, device=dev)
        self.lst = torch.empty(self.V, dtype=torch.int64 if self.elem == 8 else torch.int32, device=dev)
        self.words = vox.vox_mask_words(w.dims)
        self.mask = torch.empty(self.words, dtype=torch.int32, device=dev)
        self.flags = list_flag | vox.OUT_BITMASK | vox.OUT_FRESH
        self.tuning = None
        if tuning_arg:
            knobs = [int(x) for x in tuning_arg.split(",")] + [0]
            vox.vox_set_tuning(*knobs[:4])
            self.tuning = {"params": vox.vox_get_tuning(), "given": True}
        elif tune:
            from paper_2009_09500_gb300 import autotune

            self.tuning = autotune.get_or_tune(
                lambda: vox.vox_generate(self.segs, w.dims, self.ws, self.status, self.lst, self.mask, self.flags),
                n, self.V, w.dims, self.flags, reps=3)
        else:
            self.tuning = {"params": vox.vox_get_tuning()}

    def step(self, s, ev=None):
        from paper_2009_09500_gb300 import vox

        w = self.w
        if ev is not None:
            ev[0].record(s)
        vox.vox_count(self.segs, w.dims, self.ws, self.status, None, None, s)
        if ev is not None:
            ev[1].record(s)
        vox.vox_generate_from_scan(self.segs, w.dims, self.ws, self.status, self.lst, None, self.list_flag, s,
                                   capacity=self.V)
        if ev is not None:
            ev[2].record(s)
        vox.vox_generate_from_scan(self.segs, w.dims, self.ws, self.status, None, self.mask,
                                   vox.OUT_BITMASK | vox.OUT_FRESH, s)
        if ev is not None:
            ev[3].record(s)

    def run(self, steps: int, warmup: int, flush, stream, world: int = 1, sampler=None) -> dict:
        import torch

        from paper_2009_09500_gb300 import batching, vox

        for _ in range(warmup):
            flush.zero_()
            self.step(stream)
        torch.cuda.synchronize()
        self._check()
        evs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(4)) for _ in range(steps)]
        for k in range(steps):
            flush.zero_()
            self.step(stream, evs[k])
        torch.cuda.synchronize()
        self._check()
        graph = batching.SceneStep(self.segs, self.w.dims, self.list_flag, volume=True, device=self.dev)
        if (graph.V, graph.P) != (self.V, self.P):
            raise RuntimeError("plan mismatch")
        for _ in range(warmup):
            flush.zero_()
            graph.replay()
        gevs = [tuple(torch.cuda.Event(enable_timing=True) for _ in range(2)) for _ in range(steps)]
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        if sampler is not None:
            sampler.start()
        t0 = time.perf_counter()
        for k in range(steps):
            flush.zero_()
            gevs[k][0].record(stream)
            graph.replay()
            gevs[k][1].record(stream)
        torch.cuda.synchronize()
        wall = time.perf_counter() - t0
        if world > 1:
            torch.distributed.barrier()
        clocks = sampler.stop() if sampler is not None else None
        if int(graph.status.item()) != 0:
            raise RuntimeError(f"device status {vox.strerror(int(graph.status.item()))}")
        if not (torch.equal(graph.lst[:self.V], self.lst) and torch.equal(graph.mask, self.mask)):
            raise RuntimeError("graph step and eager step disagree")
        del graph
        torch.cuda.empty_cache()
        step_ms = [g[0].elapsed_time(g[1]) for g in gevs]
        return {"step_ms": step_ms, "eager_ms": [e[0].elapsed_time(e[3]) for e in evs],
                "count_ms": [e[0].elapsed_time(e[1]) for e in evs], "list_ms": [e[1].elapsed_time(e[2]) for e in evs],
                "vol_ms": [e[2].elapsed_time(e[3]) for e in evs], "clocks": clocks, "wall_s": wall}

    def _check(self):
        from paper_2009_09500_gb300 import vox

        st = int(self.status.item())
        if st != 0:
            raise RuntimeError(f"device status {vox.strerror(st)}")

    def rooflines(self, t: dict, sms: int, mhz) -> dict:
        """HBM rooflines of the list and volume phases (algorithmic bytes per
        launch / mean eager phase time); `roofline` = the longer phase."""
        peaks, peak_kind = _measured_peaks()
        hbm = float(peaks["hbm_gbs"])
        n = self.w.n
        kind = "k_list" if vox_tuning_list_runs() == 2 else "k_generate"
        lname = f"{kind}<list64>" if self.elem == 8 else f"{kind}<list32>"
        list_mean, vol_mean = float(np.mean(t["list_ms"])), float(np.mean(t["vol_ms"]))
        list_bytes = 24 * n + self.elem * self.V
        vol_bytes = 24 * n + 4 * self.words
        vol_kernels = ["k_scan<false>", "k_bin_scatter", "k_brick_volume", "k_generate<volume, gated>"]
        roof_list = {"bound": "hbm", "achieved": list_bytes / list_mean / 1e6, "peak": hbm, "unit": "GB/s",
                     "frac": list_bytes / list_mean / 1e6 / hbm,
                     "traffic": _recorded_field(self.key, [lname], "dram_bytes_per_launch"),
                     "kernel": f"{lname} (one launch)", "peak_kind": f"{peak_kind} HBM copy",
                     "algorithmic_bytes_per_launch": list_bytes, "ms": list_mean,
                     "bytes_model": f"24 B/segment read + {self.elem} B/voxel written",
                     "issue": _issue(self.key, [lname], list_mean, mhz, sms)}
        roof_vol = {"bound": "hbm", "achieved": vol_bytes / vol_mean / 1e6, "peak": hbm, "unit": "GB/s",
                    "frac": vol_bytes / vol_mean / 1e6 / hbm,
                    "traffic": _recorded_field(self.key, vol_kernels, "dram_bytes_per_launch"),
                    "kernel": "volume phase: k_scan<false> + k_bin_scatter + k_brick_volume (one TMA tensor store "
                              "per brick) + gated atomic fallback (exits at once); k_bin_count runs in the count phase",
                    "peak_kind": f"{peak_kind} HBM copy", "algorithmic_bytes_per_launch": vol_bytes, "ms": vol_mean,
                    "bytes_model": "24 B/segment read + the whole volume written once (w*h*d/8 bytes)",
                    "pieces": self.P, "issue": _issue(self.key, vol_kernels, vol_mean, mhz, sms)}
        return (roof_vol, roof_list) if vol_mean >= list_mean else (roof_list, roof_vol)

    def summary(self, t: dict) -> dict:
        step = t["step_ms"]
        ms = float(np.mean(step))
        return {"segments": self.w.n, "voxels": self.V, "pieces": self.P, "ms_per_step": ms,
                "voxels_per_s": self.V / ms * 1e3, "segments_per_s": self.w.n / ms * 1e3,
                "p50_ms": float(np.percentile(step, 50)), "p99_ms": float(np.percentile(step, 99)),
                "kernels_ms": {"count_scan": float(np.mean(t["count_ms"])), "list": float(np.mean(t["list_ms"])),
                               "volume": float(np.mean(t["vol_ms"]))},
                "eager_ms_per_step": float(np.mean(t["eager_ms"])), "tuning": self.tuning}

    def free(self):
        import torch

        del self.segs, self.ws, self.lst, self.mask
        torch.cuda.empty_cache()


def measure_e2e(w, list_flag: int, P: int, reps: int, dev, stream) -> dict:
    """End to end through vox_generate_host: pinned host segments in, the list
    and the fresh volume out to pinned host buffers, all inside the timed call."""
    import torch

    from paper_2009_09500_gb300 import vox

    n = w.n
    flags = list_flag | vox.OUT_BITMASK | vox.OUT_FRESH
    elem = 8 if list_flag == vox.OUT_LIST64 else 4
    h_segs = torch.from_numpy(w.segs).pin_memory()
    words = vox.vox_mask_words(w.dims)
    # the voxel count sizes the host list (device count, one synchronous call)
    d_segs = torch.from_numpy(w.segs).to(dev)
    ws = torch.empty(vox.vox_workspace_size(n), dtype=torch.uint8, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    vox.vox_count(d_segs, w.dims, ws, st, None, off)
    V = int(off[-1].item())
    del d_segs, ws, off
    h_list = torch.empty(V, dtype=torch.int64 if elem == 8 else torch.int32, pin_memory=True)
    h_mask = torch.empty(words, dtype=torch.int32, pin_memory=True)
    arena = torch.empty(vox.vox_host_arena_size_volume(n, w.dims, flags, V, P), dtype=torch.uint8, device=dev)
    vox.vox_generate_host(h_segs, w.dims, arena, h_list, h_mask, flags, stream)
    ts = []
    for _ in range(reps):
        torch.cuda.synchronize()
        ta = time.perf_counter()
        got = vox.vox_generate_host(h_segs, w.dims, arena, h_list, h_mask, flags, stream)
        ts.append(time.perf_counter() - ta)
        assert got == V
    e2e_s = float(np.median(ts))
    h2d_b, d2h_b = 24 * n, elem * V + 4 * words + 8 + 4 + 4
    del arena
    torch.cuda.empty_cache()
    link = _link_bandwidth(dev, 1 << 30)
    bound_s = h2d_b / (link["h2d_GBps"] * 1e9) + d2h_b / (link["d2h_GBps"] * 1e9)
    return {"value": V / e2e_s, "unit": UNIT, "h2d_bytes_per_step": h2d_b, "d2h_bytes_per_step": d2h_b,
            "ms": 1000 * e2e_s,
            "copy_bound": {"h2d_GBps": link["h2d_GBps"], "d2h_GBps": link["d2h_GBps"], "ms": 1000 * bound_s,
                           "frac": bound_s / e2e_s,
                           "note": "host link measured here with plain 1 GiB pinned copies; the call cannot beat its "
                                   "own bytes over it"},
            "note": f"vox_generate_host (brick-sized arena): pinned host segments in, list + fresh volume out (the "
                    f"list copy overlapping the volume kernels); median of {reps} synchronous calls"}


def measure_latency(dev, stream, reps: int = 50) -> dict:
    """The 4096-segment case: one vox_generate (count + scan + list32 + atomic
    volume) per call. Device time (events around the call) and the host's time
    from the call to its completion (synchronised), microseconds."""
    import torch

    from paper_2009_09500_gb300 import vox, workloads

    w = workloads.config1()
    segs = torch.from_numpy(w.segs).to(dev)
    ws = torch.empty(vox.vox_workspace_size(w.n), dtype=torch.uint8, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    off = torch.empty(w.n + 1, dtype=torch.int64, device=dev)
    vox.vox_count(segs, w.dims, ws, st, None, off)
    V = int(off[-1].item())
    lst = torch.empty(V, dtype=torch.int32, device=dev)
    mask = torch.zeros(vox.vox_mask_words(w.dims), dtype=torch.int32, device=dev)
    dev_us, host_us = [], []
    for i in range(reps + 5):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        a.record(stream)
        vox.vox_generate(segs, w.dims, ws, st, lst, mask, stream=stream)
        b.record(stream)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        if i >= 5:
            dev_us.append(1000 * a.elapsed_time(b))
            host_us.append(1e6 * (t1 - t0))
    if int(st.item()) != 0:
        raise RuntimeError(vox.strerror(int(st.item())))
    return {"workload": WORKLOAD1, "segments": w.n, "voxels": V,
            "device_us_p50": float(np.percentile(dev_us, 50)), "device_us_p99": float(np.percentile(dev_us, 99)),
            "host_us_p50": float(np.percentile(host_us, 50)),
            "voxels_per_s": V / float(np.percentile(dev_us, 50)) * 1e6,
            "note": "launch-latency bound: one vox_generate call (memset + count/scan + list + volume kernels), "
                    f"{reps} calls, warm caches"}


def measure_batched(steps: int, dev, tune: bool = True) -> dict:
    """Batched vs plain launches on the 256-scene workload (uneven scenes, volume
    edges 64..512, 1e3..1e5 segments each; list32 + one volume per scene):
    one vox_generate_batched sequence against one vox_generate per scene, both
    eager and both replayed from a CUDA graph. L2 is flushed between steps,
    outside the events."""
    import torch

    from paper_2009_09500_gb300 import autotune, batching, vox, workloads

    scenes = workloads.config4()
    b = batching.make_batch(scenes, device=dev)
    plain = batching.PlainScenes(b, device=dev)
    if tune:  # the launch tuning is process-wide: tune for this batch (its own workload class)
        tuning = autotune.get_or_tune(lambda: b.run(), int(b.segs.shape[0]), b.V, (512, 512, 512), b.flags | 0x100,
                                      reps=3)
    else:
        tuning = {"params": vox.vox_get_tuning()}
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    stream = torch.cuda.current_stream()

    def timed(fn, reps):
        ts = []
        for i in range(reps + 2):
            flush.zero_()
            a, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            e.record(stream)
            torch.cuda.synchronize()
            if i >= 2:
                ts.append(a.elapsed_time(e))
        return float(np.mean(ts)), float(np.percentile(ts, 99))

    reps = max(3, min(steps, 20))
    batched_eager = timed(lambda: b.run(stream), reps)
    plain_eager = timed(lambda: plain.run(stream), reps)
    g_b = batching.GraphRunner(b.run)
    batched_graph = timed(g_b.replay, reps)
    g_p = batching.GraphRunner(plain.run)
    plain_graph = timed(g_p.replay, reps)
    torch.cuda.synchronize()
    st = int(b.status.item())
    if st != 0:
        raise RuntimeError(f"device status {st}")
    V = b.V
    return {
        "workload": "256 uneven scenes: edges {64,128,256,512}, 1e3..1e5 segments each, list32 + volume per scene",
        "scenes": b.n_scenes, "segments": int(b.segs.shape[0]), "voxels": V,
        "batched_over_plain_graph": plain_graph[0] / batched_graph[0],
        "batched_graph_ms": batched_graph[0], "plain_graph_ms": plain_graph[0],
        "batched_graph_p99_ms": batched_graph[1],
        "voxels_per_s_batched_graph": V / batched_graph[0] * 1e3, "voxels_per_s_plain_graph": V / plain_graph[0] * 1e3,
        "batched_eager_ms": batched_eager[0], "plain_eager_ms": plain_eager[0],
        "batched_over_plain_eager": plain_eager[0] / batched_eager[0],
        "launches": {"batched": "one sequence: scene map, count + scan, scene bases, list, scene bricks, bin count, "
                                "slot scan, scatter, brick volume, gated atomics (10 kernels + 3 memsets)",
                     "plain": "per scene: 2-3 memsets + 7 kernels (256 scenes)"},
        "tuning": tuning["params"],
    }


# The paper's GTX 1070 Ti column (ms) of Tables 2, 3 and 4: context only (other
# hardware; its timings were taken with a profiler and include its own copies).
PAPER_E1_MS = (0.45, 0.46, 0.49, 0.51, 0.52, 0.67, 0.92, 1.52, 2.22, 3.65428571)
PAPER_E2_MS = (0.42, 0.46, 0.75, 1.44, 4.13, 10.91, 21.70, 43.85, 105.84, 218.17, 427.62)
PAPER_E3_MS = 4071.01


def measure_sweeps(dev, reps: int = 5, e2e: bool = True) -> dict:
    """The three sweeps of Section 5 (Tables 2-4) with 64-bit lists in a 2^21-edge
    volume: E1 one segment of 10^3..10^6 voxels; E2 1024 segments of equal length
    20..200 000 voxels; E3 1024 segments of pairwise different lengths totalling
    10^9 voxels. Each point times one vox_generate call (count + scan + list) on
    device buffers (L2 flushed between calls, CUDA events) and, end to end, one
    vox_generate_host call (pinned host segments in, host list out)."""
    import torch

    from paper_2009_09500_gb300 import vox, workloads

    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    flags = vox.OUT_LIST64

    def point(w, paper_ms):
        n = w.n
        segs = torch.from_numpy(w.segs).to(dev)
        ws = torch.empty(vox.vox_workspace_size(n), dtype=torch.uint8, device=dev)
        status = torch.zeros(1, dtype=torch.int32, device=dev)
        off = torch.empty(n + 1, dtype=torch.int64, device=dev)
        vox.vox_count(segs, w.dims, ws, status, None, off)
        V = int(off[-1].item())
        lst = torch.empty(V, dtype=torch.int64, device=dev)
        ts = []
        for i in range(reps + 2):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            vox.vox_generate(segs, w.dims, ws, status, lst, None, flags, stream, capacity=V)
            b.record(stream)
            torch.cuda.synchronize()
            if i >= 2:
                ts.append(a.elapsed_time(b))
        if int(status.item()) != 0:
            raise RuntimeError(f"device status {vox.strerror(int(status.item()))}")
        ms = float(np.median(ts))
        out = {"segments": n, "voxels": V, "device_ms": ms, "voxels_per_s": V / ms * 1e3,
               "paper_gtx1070ti_ms": paper_ms}
        del segs, ws, lst, off
        if e2e:
            h_segs = torch.from_numpy(w.segs).pin_memory()
            h_list = torch.empty(V, dtype=torch.int64).pin_memory()
            arena = torch.empty(vox.vox_host_arena_size(n, w.dims, flags, V), dtype=torch.uint8, device=dev)
            te = []
            for i in range(reps + 1):
                torch.cuda.synchronize()
                ta = time.perf_counter()
                got = vox.vox_generate_host(h_segs, w.dims, arena, h_list, None, flags, stream)
                if i >= 1:
                    te.append(time.perf_counter() - ta)
                assert got == V
            out.update({"e2e_ms": 1000 * float(np.median(te)), "h2d_bytes": 24 * n, "d2h_bytes": 8 * V})
            del h_list, arena
        torch.cuda.empty_cache()
        return out

    e1 = [dict(length=L, **point(workloads.sweep_single(L), p))
          for L, p in zip(workloads.E1_LENGTHS, PAPER_E1_MS)]
    e2 = [dict(length=L, **point(workloads.sweep_fixed(L), p))
          for L, p in zip(workloads.E2_LENGTHS, PAPER_E2_MS)]
    e3 = point(workloads.sweep_giga(), PAPER_E3_MS)
    return {"E1_single_segment": e1, "E2_1024_equal_length": e2, "E3_1024_arbitrary_total_1e9": e3,
            "output": "list64 (x | y << 21 | z << 42), 2^21-edge volume",
            "device_ms": "one vox_generate call (count + scan + list), median of "
                         f"{reps}, L2 flushed between calls",
            "e2e_ms": "one vox_generate_host call (pinned H2D of the segments, count, list, D2H of the "
                      "list), median, synchronous"}


def measure_serving(duration_s: float, rate_hz: float, dev) -> dict:
    """The request stream: Poisson arrivals at `rate_hz` for `duration_s`, each
    request a scene of log-uniform 1e3..1e6 segments in a 128^3..1024^3 volume,
    served by the continuous-batching loop into device-resident volumes,
    admitted by the device's free memory (live probe). Latency = completion
    (host clock, event polled) - arrival."""
    import torch

    from paper_2009_09500_gb300 import serving, vox, workloads

    stream = workloads.config5(rate_hz=rate_hz, duration_s=duration_s)
    reqs = serving.make_requests(stream, pool_size=128)
    probe = lambda: serving.gpu_free_bytes(dev)
    launcher = serving.GpuLauncher(slots=4, device=dev)
    warm = serving.make_requests(workloads.config5(seed=99, duration_s=0.01), pool_size=8)
    cap = 64 << 30
    serving.Server(launcher, budget_bytes=cap, max_inflight=4, mem_probe=probe).run(warm)
    torch.cuda.synchronize()
    srv = serving.Server(launcher, budget_bytes=cap, max_inflight=4, max_batch_requests=64, mem_probe=probe)
    st = srv.run(reqs)
    out = st.summary()
    out.update({"offered_req_per_s": rate_hz, "duration_s": duration_s, "requests": len(reqs),
                "offered_requests_per_s_measured": len(reqs) / duration_s,
                "admission": "free device memory (probe) less a 1 GiB reserve, capped at 64 GiB in flight",
                "slots": 4, "tuning": vox.vox_get_tuning()})
    return out


def measure_bricked(sb: SceneBench, stream, flush, reps: int) -> dict:
    """The brick-major volume layout (VOX_OUT_BRICKED) on the scene's volume:
    the volume phase writing one contiguous bulk copy per brick, and
    vox_unbrick back to row-major, checked equal to the row-major volume."""
    import torch

    from paper_2009_09500_gb300 import vox

    w = sb.w
    bmask = torch.empty(vox.vox_mask_words_bricked(w.dims), dtype=torch.int32, device=sb.dev)
    row = torch.empty_like(sb.mask)
    vox.vox_count(sb.segs, w.dims, sb.ws, sb.status, None, None, stream)
    tb, tu = [], []
    for i in range(reps + 2):
        flush.zero_()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        vox.vox_generate_from_scan(sb.segs, w.dims, sb.ws, sb.status, None, bmask, vox.OUT_BITMASK | vox.OUT_BRICKED,
                                   stream)
        e1.record(stream)
        vox.vox_unbrick(bmask, w.dims, row, stream)
        e2.record(stream)
        torch.cuda.synchronize()
        if i >= 2:
            tb.append(e0.elapsed_time(e1))
            tu.append(e1.elapsed_time(e2))
    if int(sb.status.item()) != 0:
        raise RuntimeError(f"device status {vox.strerror(int(sb.status.item()))}")
    if not torch.equal(row, sb.mask):
        raise RuntimeError("unbricked volume differs from the row-major volume")
    del bmask, row
    torch.cuda.empty_cache()
    return {"volume_ms": float(np.mean(tb)), "unbrick_ms": float(np.mean(tu)), "brick_shape": vox.vox_brick_shape(w.dims)[0],
            "note": "volume phase (slot scan, scatter, brick kernel) writing the brick-major layout, and vox_unbrick "
                    "back to row-major, checked equal to the row-major volume"}


def measure_euclid(w, dev, stream, flush, reps: int) -> dict:
    """The Euclidean-N variant of Eq. (1)-(2) (repeats dropped) on the scene: one
    vox_euclid_generate (sample scan, run counts, run scan, compacted list32 +
    fresh volume by bricks)."""
    import torch

    from paper_2009_09500_gb300 import vox

    n = w.n
    segs = torch.from_numpy(w.segs).to(dev)
    status = torch.zeros(1, dtype=torch.int32, device=dev)
    words = vox.vox_mask_words(w.dims)
    ews = torch.empty(vox.vox_euclid_workspace_size_volume(n, w.dims, 0), dtype=torch.uint8, device=dev)
    Vd, Vs, EP = vox.vox_euclid_plan(segs, w.dims, ews, status, with_pieces=True)
    ews = torch.empty(vox.vox_euclid_workspace_size_volume(n, w.dims, EP), dtype=torch.uint8, device=dev)
    elst = torch.empty(Vd, dtype=torch.int32, device=dev)
    emask = torch.empty(words, dtype=torch.int32, device=dev)
    te = []
    for i in range(reps + 3):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        vox.vox_euclid_generate(segs, w.dims, ews, status, elst, emask, vox.OUT_LIST32 | vox.OUT_BITMASK |
                                vox.OUT_FRESH, None, stream)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= 3:
            te.append(e0.elapsed_time(e1))
    if int(status.item()) != 0:
        raise RuntimeError(f"device status {vox.strerror(int(status.item()))}")
    ems = float(np.mean(te))
    del ews, elst, emask, segs
    torch.cuda.empty_cache()
    return {"ms": ems, "voxels": Vd, "samples": Vs, "pieces": EP, "voxels_per_s": Vd / ems * 1e3,
            "samples_per_s": Vs / ems * 1e3,
            "note": "N = int(|E - S|); one vox_euclid_generate call on the fixed-length batch: list32 (compacted, run "
                    "walk) + fresh volume (bricks); L2 flushed between calls"}


def measure_atomics(dev, stream, flush, reps: int, big: bool = True) -> dict:
    """The per-voxel atomic volume against the GPU's red.or throughput. The
    microbenchmark (vox_probe_red_or: 32-bit OR reductions at pseudo-random
    words) on a 128 MiB buffer (the fixed-length batch's 1024^3 volume, about
    L2's size) and on an 8 GiB buffer (the 4096^3 volume); then the fixed-length
    batch's volume alone by per-voxel atomics, with each thread merging its
    consecutive voxels' bits per word (VOX_VOLUME_ATOMIC) and merged across the
    warp as well (VOX_VOLUME_ATOMIC_WARP), and by bricks for comparison. The
    reductions a launch issues come from the committed ncu record (LTS red
    requests), when it matches the current kernel sources."""
    import torch

    from paper_2009_09500_gb300 import vox, workloads

    def timed(fn):
        ts = []
        for i in range(reps + 2):
            flush.zero_()
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            fn()
            b.record(stream)
            torch.cuda.synchronize()
            if i >= 2:
                ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    micro = {}
    for name, words in (("128MiB", 32 << 20), ("8GiB", 2 << 30))[:2 if big else 1]:
        buf = torch.zeros(words, dtype=torch.int32, device=dev)
        ops = vox.vox_probe_red_or_ops(1 << 28)
        ms = timed(lambda: vox.vox_probe_red_or(buf, 1 << 28, 7, stream))
        micro[name] = {"reductions": ops, "ms": ms, "reductions_per_s": ops / ms * 1e3}
        del buf
        torch.cuda.empty_cache()
    w = workloads.config2()
    segs = torch.from_numpy(w.segs).to(dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    ws0 = torch.empty(vox.vox_workspace_size_volume(w.n, w.dims, 0), dtype=torch.uint8, device=dev)
    V, P = vox.vox_plan(segs, w.dims, ws0, st)
    ws = torch.empty(vox.vox_workspace_size_volume(w.n, w.dims, P), dtype=torch.uint8, device=dev)
    del ws0
    mask = torch.zeros(vox.vox_mask_words(w.dims), dtype=torch.int32, device=dev)
    ref = None
    paths = {}
    saved = vox.vox_get_tuning()
    try:
        for name, vp, kern in (("per-lane merged", vox.VOLUME_ATOMIC, "k_generate<volume, atomic>"),
                               ("warp merged", vox.VOLUME_ATOMIC_WARP, "k_generate<volume, atomic warp>"),
                               ("bricks", vox.VOLUME_AUTO, None)):
            vox.vox_set_tuning(saved["run_len"], vp, saved["ctas_per_sm"], saved["list_runs"])
            vox.vox_count(segs, w.dims, ws, st, None, None, stream)

            def run():
                mask.zero_()
                vox.vox_generate_from_scan(segs, w.dims, ws, st, None, mask, vox.OUT_BITMASK, stream)

            ms = timed(run)
            if int(st.item()) != 0:
                raise RuntimeError(vox.strerror(int(st.item())))
            if ref is None:
                ref = mask.clone()
            elif not torch.equal(ref, mask):
                raise RuntimeError(f"{name} volume differs")
            ent = {"ms_with_clear": ms, "voxels_per_s": V / ms * 1e3}
            if kern is not None:
                red = _recorded_field("config2", [kern], "lts_red_requests")
                if red is not None:
                    rate = red / (ms * 1e-3)
                    ent.update({"lts_red_requests_per_launch": red, "reductions_per_s": rate,
                                "frac_of_probe_128MiB": rate / micro["128MiB"]["reductions_per_s"]})
            paths[name] = ent
    finally:
        vox.vox_set_tuning(saved["run_len"], saved["volume_path"], saved["ctas_per_sm"], saved["list_runs"])
    del segs, ws, mask, ref
    torch.cuda.empty_cache()
    return {"red_or_probe": micro, "volume_alone": paths, "workload": WORKLOAD2,
            "note": "volume alone after one count; times include the 128 MiB clear (OR into zeros); "
                    "L2 flushed between calls"}


def measure_phase(phase: str, n: int, edge: int, steps: int, dev, stream, flush) -> dict:
    """One phase of a log-uniform batch of n segments in an edge^3 volume (the
    headline workload's shape at a size a profiler can replay): the list64
    alone or the fresh volume alone, `steps` launches after one count, with the
    launch tuning in force (--tuning)."""
    import torch

    from paper_2009_09500_gb300 import vox, workloads

    w = workloads.config3(n=n, edge=edge)
    segs = torch.from_numpy(w.segs).to(dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = torch.empty(vox.vox_workspace_size_volume(n, w.dims, 0), dtype=torch.uint8, device=dev)
    V, P = vox.vox_plan(segs, w.dims, ws, st)
    ws = torch.empty(vox.vox_workspace_size_volume(n, w.dims, P), dtype=torch.uint8, device=dev)
    vox.vox_count(segs, w.dims, ws, st, None, None, stream)
    if phase == "list":
        out = torch.empty(V, dtype=torch.int64, device=dev)
        run = lambda: vox.vox_generate_from_scan(segs, w.dims, ws, st, out, None, vox.OUT_LIST64, stream, capacity=V)
        nbytes = 24 * n + 8 * V
    else:
        out = torch.empty(vox.vox_mask_words(w.dims), dtype=torch.int32, device=dev)
        run = lambda: vox.vox_generate_from_scan(segs, w.dims, ws, st, None, out, vox.OUT_BITMASK | vox.OUT_FRESH,
                                                 stream)
        nbytes = 24 * n + 4 * out.numel()
    ts = []
    for _ in range(steps):
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        run()
        b.record(stream)
        torch.cuda.synchronize()
        ts.append(a.elapsed_time(b))
    if int(st.item()) != 0:
        raise RuntimeError(vox.strerror(int(st.item())))
    return {"phase": phase, "segments": n, "edge": edge, "voxels": V, "pieces": P, "ms": ts,
            "algorithmic_bytes": nbytes, "tuning": vox.vox_get_tuning()}


def _section(name, fn, *a, **kw):
    """An auxiliary measurement: its result, or the error it raised (so that one
    failing side measurement does not lose the headline line)."""
    try:
        return fn(*a, **kw)
    except Exception as e:  # noqa: BLE001 - reported in the JSON line
        print(f"section {name} failed: {e!r}", file=sys.stderr, flush=True)
        return {"error": f"{type(e).__name__}: {e}"}


def run_ours(args):
    import torch

    from paper_2009_09500_gb300 import build, vox, workloads

    rank, world, local = _dist_env()
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    build.build_library()
    vox.load()
    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    if args.only == "atomics":  # one section alone (e.g. under a profiler)
        print(json.dumps({"atomic_volume": measure_atomics(dev, stream, flush, min(args.steps, 10),
                                                           big=not args.no_big_probe)}), flush=True)
        return 0
    if args.only and args.tuning:
        knobs = [int(x) for x in args.tuning.split(",")] + [0]
        vox.vox_set_tuning(*knobs[:4])
    if args.only == "config2":  # the fixed-length batch's block alone (profiler runs)
        w2 = workloads.config2()
        sb2 = SceneBench("config2", w2, vox.OUT_LIST32, dev, tune=not args.no_tune and not args.tuning,
                         tuning_arg=args.tuning)
        t2 = sb2.run(args.steps, args.warmup, flush, stream)
        print(json.dumps(sb2.summary(t2)), flush=True)
        return 0
    if args.only == "batched":  # the 256-scene batched-vs-plain block alone (profiler runs)
        print(json.dumps({"batched_vs_plain": measure_batched(args.steps, dev, tune=not args.tuning)}), flush=True)
        return 0
    if args.only == "euclid":  # the Euclidean-N variant on the fixed-length batch alone (profiler runs)
        print(json.dumps({"euclid_variant": measure_euclid(workloads.config2(), dev, stream, flush, args.steps)}),
              flush=True)
        return 0
    if args.only in ("list", "volume"):  # one phase of a smaller log-uniform batch (profiler runs)
        print(json.dumps(measure_phase(args.only, args.segments, args.edge, args.steps, dev, stream, flush)),
              flush=True)
        return 0

    # headline: each rank voxelizes its own arbitrary-length batch (weak scaling)
    w3 = workloads.config3(seed=2 + 1000 * rank)
    sb = SceneBench("config3", w3, vox.OUT_LIST64, dev, tune=not args.no_tune, tuning_arg=args.tuning)
    sampler = ClockSampler(dev.index if dev.index is not None else 0)
    t3 = sb.run(args.steps, args.warmup, flush, stream, world, sampler)
    clocks = t3["clocks"]
    mhz = (clocks or {}).get("sm_mhz") or (clocks or {}).get("sm_max_mhz")
    s3 = sb.summary(t3)
    ms_mean_max, total_voxels, value = aggregate_ranks(s3["ms_per_step"], sb.V, world, dev)
    roofline, roofline_other = sb.rooflines(t3, sms, mhz)
    main_tuning = vox.vox_get_tuning()
    bricked = None
    if not args.no_bricked and world == 1:
        bricked = _section("bricked", measure_bricked, sb, stream, flush, min(args.steps, 10))
        bricked["row_major_volume_ms"] = s3["kernels_ms"]["volume"]
    V3, P3 = sb.V, sb.P
    sb.free()
    del sb
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(w3, vox.OUT_LIST64, P3, 3, dev, stream)
        e2e["value"] = e2e["value"] * world  # every rank moves its own batch (the headline e2e: not guarded)
    # the fixed-length batch, with its own tuning and roofline
    cfg2 = None
    if not args.no_config2:
        w2 = workloads.config2(seed=1 + 1000 * rank)
        sb2 = SceneBench("config2", w2, vox.OUT_LIST32, dev, tune=not args.no_tune, tuning_arg=args.tuning)
        t2 = sb2.run(args.steps, args.warmup, flush, stream, world)
        cfg2 = sb2.summary(t2)
        cfg2["workload"] = WORKLOAD2
        cfg2["roofline"], cfg2["roofline_other"] = sb2.rooflines(t2, sms, mhz)
        sb2.free()
        del sb2
        if not args.no_euclid and world == 1:
            cfg2["euclid_variant"] = _section("euclid", measure_euclid, w2, dev, stream, flush, min(args.steps, 20))
    latency = _section("latency", measure_latency, dev, stream) if world == 1 and not args.no_latency else None
    atomics = (_section("atomics", measure_atomics, dev, stream, flush, min(args.steps, 10))
               if world == 1 and not args.no_atomics else None)
    batched = None
    if not args.no_batched and world == 1:
        batched = _section("batched", measure_batched, args.steps, dev, tune=not args.tuning)  # serving keeps its tuning
    served = None
    if not args.no_serve and world == 1:
        served = [_section("serving", measure_serving, args.serve_seconds, 2000.0, dev),
                  _section("serving", measure_serving, args.serve_seconds / 2, 6000.0, dev)]
    vox.vox_set_tuning(main_tuning["run_len"], main_tuning["volume_path"], main_tuning["ctas_per_sm"],
                       main_tuning["list_runs"])
    sweeps = None
    if not args.no_sweeps and world == 1:
        sweeps = _section("sweeps", measure_sweeps, dev)

    if rank != 0:
        return 0
    cpu = cpu_all = None
    if world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w3, V3, 1, args.cpu_seconds)
        cpu_all = cpu_baseline(w3, V3, os.cpu_count() or 1, args.cpu_seconds)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_mean_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "int32", "data": "synthetic",
        "config": headline_config(w3.n, V3, w3.dims, world),
        "launch": "batching.SceneStep: the step's launches captured once as a CUDA graph (count; list and volume on "
                  "two streams) and replayed; per-phase times from the same launches issued eagerly on one stream "
                  "with events between phases",
        "segments_per_s": w3.n * world / (ms_mean_max / 1000.0),
        "p50_ms": s3["p50_ms"], "p99_ms": s3["p99_ms"], "kernels_ms": s3["kernels_ms"],
        "eager_ms_per_step": s3["eager_ms_per_step"], "pieces": P3, "tuning": s3["tuning"],
        "roofline": roofline, "roofline_other": roofline_other, "cpu_baseline": cpu, "cpu_baseline_all_cores": cpu_all,
        "e2e": e2e, "clocks": clocks,
        "gpu_launches": 7 * args.steps,
        "gpu_launches_note": "graph-timed region, per step: k_scan<true>, k_bin_count, the list kernel (k_list with "
                             "list_runs 2, else k_generate), k_scan<false>, k_bin_scatter, k_brick_volume, "
                             "k_generate (gated volume fallback; exits at once); the eager per-phase region launches "
                             "the same 7 per step",
        "batched_vs_plain": batched, "config2_fixed_length": cfg2, "config1_latency": latency,
        "serving": served, "bricked_volume": bricked, "sweeps": sweeps, "atomic_volume": atomics,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=100)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-tune", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-sweeps", action="store_true")
    ap.add_argument("--no-euclid", action="store_true")
    ap.add_argument("--no-bricked", action="store_true")
    ap.add_argument("--no-config2", action="store_true")
    ap.add_argument("--no-latency", action="store_true")
    ap.add_argument("--no-atomics", action="store_true")
    ap.add_argument("--only", choices=["atomics", "list", "volume", "config2", "euclid", "batched"], default=None,
                    help="run one section alone and print it (list / volume: one phase of a smaller log-uniform batch)")
    ap.add_argument("--segments", type=int, default=1 << 19, help="--only list/volume: segments")
    ap.add_argument("--edge", type=int, default=2048, help="--only list/volume: volume edge")
    ap.add_argument("--no-big-probe", action="store_true", help="atomics: skip the 8 GiB red.or probe")
    ap.add_argument("--tuning", default="", help="run_len,volume_path,ctas_per_sm[,list_runs]: use this launch tuning")
    ap.add_argument("--serve-seconds", type=float, default=1.0)
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
