#!/usr/bin/env python3
"""Benchmark of the GPU LSD radix sort: one JSON line on rank 0.

Default workload (one "step" = one whole sort through isort_keys): n = 2^28
uniform uint32 keys, radix 256 (4 count-sort passes), keys only, seeded
synthetic data generated in HBM. Inputs (1 GiB) are larger than L2; before each
timed sort the keys are restored from a pristine copy and L2 is flushed by
reading a 512 MiB buffer, both outside the timed event pair.

  python bench.py [--gpus N --steps K --warmup W]   our GPU path
  python bench.py --impl reference                    the serial C oracle on host cores

Other workloads (--workload): r16 (radix 65536, 2 passes), pairs (2^27 u32 keys
+ u32 index payloads), u64 (2^26 u64 keys, 8 passes), and any of the six key
distributions via --dist.
"""
from __future__ import annotations

import argparse
import atexit
import hashlib
import json
import os
import shutil
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

PROFILE_TRAFFIC = os.path.join(ROOT, "profiles", "traffic.json")

WORKLOADS = {
    # name: (n, key_bits, val_bits, radix_bits, description)
    "u32_2p28_r256": (1 << 28, 32, 0, 8, "plain sort, 2^28 uint32 keys, radix 256 (4 passes)"),
    "u32_2p28_r65536": (1 << 28, 32, 0, 16, "plain sort, 2^28 uint32 keys, radix 65536 (2 passes)"),
    "u32_2p28_r2048": (1 << 28, 32, 0, 11, "plain sort, 2^28 uint32 keys, radix 2048 (3 passes: "
                                           "11, 11, 10 bits)"),
    "pairs_2p27": (1 << 27, 32, 32, 8, "stable pairs, 2^27 uint32 keys + uint32 index payloads"),
    "u64_2p26": (1 << 26, 64, 0, 8, "plain sort, 2^26 uint64 keys, radix 256 (8 passes)"),
    "sample_2p28": (1 << 28, 32, 0, 8, "GVR sample sort (Algorithm 3; 256 buckets, oversampling "
                                        "16) of 2^28 uint32 keys"),
    "gsd_2p28": (1 << 28, 32, 0, 8, "GSD regular-oversampling sort (Algorithm 1; p = 16, r = 4) "
                                     "of 2^28 uint32 keys"),
    "u32_128M_paper": (131_072_000, 32, 0, 8, "the paper's 128M (1M = 1,024,000) uint32 keys"),
    # n is the total over 20,000 ranges with log-uniform lengths in [1, 2^20]
    "segmented_20000": (0, 32, 0, 8, "batched segmented sort, 20,000 ranges, lengths "
                                     "log-uniform in [1, 2^20], uniform uint32 keys"),
    "short_ranges": (1 << 26, 32, 0, 8, "short ranges (32 .. 4096 keys), BTN vs OET networks"),
    "mbsp_model": (1 << 28, 32, 0, 8, "MBSP cost model calibrated on the radix-256 round, "
                                      "predicted vs measured sort times"),
    "serve_poisson": (0, 32, 32, 8, "serving loop: Poisson arrivals at 2,000 req/s, sizes "
                                    "log-uniform in [2^10, 2^24] uint32 keys, half with "
                                    "uint32 payloads, 40 GB admission budget"),
}
ALIASES = {"r16": "u32_2p28_r65536", "r11": "u32_2p28_r2048", "pairs": "pairs_2p27", "u64": "u64_2p26",
           "paper128m": "u32_128M_paper", "default": "u32_2p28_r256",
           "segmented": "segmented_20000", "serve": "serve_poisson", "networks": "short_ranges", "mbsp": "mbsp_model",
           "gvr": "sample_2p28", "gsd": "gsd_2p28"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="u32_2p28_r256")
    ap.add_argument("--dist", default="uniform")
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=12.0,
                    help="target CPU time of the oracle baseline sample")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="duration of each arm of the serving workload")
    ap.add_argument("--n", type=int, default=0,
                    help="override the key count of a plain workload (small profiling cases)")
    a = ap.parse_args()
    a.workload = ALIASES.get(a.workload, a.workload)
    if a.workload not in WORKLOADS:
        ap.error(f"unknown workload {a.workload}")
    if a.warmup < 3 and a.impl == "ours":
        ap.error("at least 3 warm-up steps")
    return a


# --------------------------------------------------------------------------- dist
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


class Replicas:
    """N independent replicas (one per GPU); a barrier and a max over ranks only."""

    def __init__(self, world, rank, local, backend):
        self.world, self.rank = world, rank
        self.pg = None
        if world > 1:
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg:
            self.pg.barrier()

    def max(self, x: float) -> float:
        if not self.pg:
            return x
        import torch
        dev = "cuda" if self.pg.get_backend() == "nccl" else "cpu"
        t = torch.tensor([x], dtype=torch.float64, device=dev)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def close(self):
        if self.pg:
            self.pg.destroy_process_group()


# --------------------------------------------------------------------------- clocks
class ClockSampler:
    """nvidia-smi clock/throttle samples every 20 ms. start() before the warm-up
    (nvidia-smi takes a while to come up), window(t0, t1) with the timed
    region's host clock, stop() summarises the samples that arrived inside the
    window (plus one sampling period); if none did, all samples since start."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    PERIOD_MS = 20

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []  # (host arrival time, csv line)
        self.t0 = self.t1 = None

    def start(self, wait_s: float = 3.0):
        cmd = ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
               "--format=csv,noheader,nounits", "-lms", str(self.PERIOD_MS)]
        if shutil.which("stdbuf"):
            cmd = ["stdbuf", "-oL"] + cmd  # one line per sample through the pipe
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, ValueError):
            self.proc = None
            return
        atexit.register(self._end)  # no sampler outlives the process, even on an error
        t_end = time.perf_counter() + wait_s
        while not self.lines and time.perf_counter() < t_end and self.proc.poll() is None:
            time.sleep(0.01)

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.perf_counter(), line.strip()))

    def _end(self):
        if self.proc and self.proc.poll() is None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def window(self, t0: float, t1: float):
        self.t0, self.t1 = t0, t1

    def stop(self):
        if not self.proc:
            return None
        if self.t1 is not None:  # let the samples of the window's end arrive
            time.sleep(max(0.0, self.t1 + 2 * self.PERIOD_MS / 1000 - time.perf_counter()))
        self._end()
        self.t.join(timeout=2)
        inside = [ln for t, ln in self.lines
                  if self.t0 is not None and self.t0 <= t <= self.t1 + self.PERIOD_MS / 1000]
        use = inside or [ln for _, ln in self.lines]
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in use:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm), "samples_in_timed_region": len(inside),
                "period_ms": self.PERIOD_MS}


# --------------------------------------------------------------------------- helpers
def measured_peak_hbm():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        v = json.load(open(p))["hbm_gbs"]
        return float(v), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


def onesweep_source_hash() -> str:
    """Hash of the radix-256 round's code: its sources with // comments and
    blank lines removed (a comment edit does not change the kernel)."""
    h = hashlib.sha256()
    for f in ("onesweep.cuh", "common.cuh"):
        for line in open(os.path.join(ROOT, "paper_1808_10292_gb300", "csrc", f)):
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def recorded_traffic(workload, variant):
    """Per-launch DRAM bytes of the dominant kernel from a committed ncu summary,
    or None if there is none for this exact kernel source and shape."""
    try:
        rec = json.load(open(PROFILE_TRAFFIC))
    except (OSError, ValueError):
        return None
    r = rec.get(workload)
    if not r or r.get("source_hash") != onesweep_source_hash() or r.get("variant") != list(variant):
        return None
    return r.get("dram_bytes_per_launch")


def cpu_cores_available() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample(n_full, key_bits, val_bits, radix_bits, dist, seed, target_s, max_sorts=None,
                  gvr=False, gsd=False):
    """Time the oracle on a bounded sample of the workload: sorts of a 2^24-key
    slice (or the whole input if smaller) until target_s seconds have passed
    (the oracle's GVR sample sort for the sample-sort workload)."""
    import inputs
    import oracle
    n = min(n_full, 1 << 24)
    k = inputs.keys(n, key_bits, dist, seed)
    v = inputs.iota(n, val_bits) if val_bits else None
    oracle.radix_sort(k[:1024], None if v is None else v[:1024], radix_bits)  # load + warm
    times = []
    t_end = time.perf_counter() + target_s
    while time.perf_counter() < t_end and (max_sorts is None or len(times) < max_sorts):
        t0 = time.perf_counter()
        if gvr:
            oracle.gvr_sort(k, v, buckets=256, oversample=16, seed=seed)
        elif gsd:
            oracle.gsd_sort(k, v, buckets=16, oversample=4)
        else:
            oracle.radix_sort(k, v, radix_bits)
        times.append(time.perf_counter() - t0)
    return n, times


# --------------------------------------------------------------------------- reference arm
def run_reference(a):
    world, rank, local = dist_env()
    if rank != 0:
        return 0
    n_full, kb, vb, rb, desc = WORKLOADS[a.workload]
    # each step: one oracle sort of a 2^24-key slice of the workload
    n, times = oracle_sample(n_full, kb, vb, rb, a.dist, a.seed, target_s=1e9,
                             max_sorts=a.steps + a.warmup, gvr=a.workload == "sample_2p28",
                             gsd=a.workload == "gsd_2p28")
    timed = times[a.warmup:]
    total = sum(timed)
    value = n * len(timed) / total
    sample = (f"{len(timed)} oracle sorts of a {n}-key slice ({a.dist}, seed {a.seed}) of the "
              f"{n_full}-key workload, 1 thread")
    line = {
        "impl": "reference",
        "metric": f"uint{kb} keys/s ({desc})",
        "value": value,
        "unit": "keys/s",
        "n_gpus": a.gpus,
        "steps": len(timed),
        "warmup": a.warmup,
        "ms_per_step": 1000 * total / len(timed),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": f"u{kb}",
        "data": "synthetic",
        "config": {"workload": a.workload, "n": n_full, "key_bits": kb, "val_bits": vb,
                   "radix_bits": rb, "dist": a.dist, "seed": a.seed, "sample_n": n},
        "cpu_baseline": {"value": value, "unit": "keys/s", "cores": 1, "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": "keys/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def run_reference_segmented(a):
    world, rank, local = dist_env()
    if rank != 0:
        return 0
    import inputs
    import oracle
    L = inputs.segment_lengths(20_000, seed=a.seed)
    off = inputs.segment_offsets(L)
    # each step: the oracle sorts the next 200 ranges of the workload
    host = inputs.keys(int(off[min(len(L), 200 * (a.steps + a.warmup))]), 32, a.dist, a.seed)
    times, keys_done = [], []
    s = 0
    for step in range(a.steps + a.warmup):
        t0 = time.perf_counter()
        k = 0
        for _ in range(200):
            if s >= len(L):
                break
            seg = host[off[s]:off[s + 1]]
            oracle.radix_sort(seg)
            k += len(seg)
            s += 1
        times.append(time.perf_counter() - t0)
        keys_done.append(k)
    t, kd = sum(times[a.warmup:]), sum(keys_done[a.warmup:])
    value = kd / t
    line = {"impl": "reference",
            "metric": "batched-segment keys/s (20,000 ranges, log-uniform lengths in [1, 2^20])",
            "value": value, "unit": "keys/s", "n_gpus": a.gpus, "steps": a.steps,
            "warmup": a.warmup, "ms_per_step": 1000 * t / a.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": {"workload": a.workload, "num_segments": 20000, "dist": a.dist,
                       "seed": a.seed},
            "cpu_baseline": {"value": value, "unit": "keys/s", "cores": 1, "kind": "oracle",
                             "sample": f"{a.steps} steps of 200 consecutive ranges each, one "
                                       f"oracle sort per range, 1 thread"},
            "e2e": {"value": value, "unit": "keys/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# --------------------------------------------------------------------------- our arm
def run_ours(a):
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    rep = Replicas(world, rank, local, "nccl")
    import inputs
    import paper_1808_10292_gb300 as isort
    from paper_1808_10292_gb300 import _lib

    n, kb, vb, rb, desc = WORKLOADS[a.workload]
    if a.n:
        n, desc = a.n, f"{desc}; n overridden to {a.n}"
    kdt = torch.uint32 if kb == 32 else torch.uint64
    pristine = inputs.device_keys(n, kb, a.dist, a.seed)
    keys = torch.empty_like(pristine)
    vals = vpr = None
    if vb:
        vpr = inputs.device_iota(n, vb)
        vals = torch.empty_like(vpr)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda").view(torch.int32)
    flush.zero_()
    stream = torch.cuda.current_stream()

    def restore():
        keys.copy_(pristine)
        if vb:
            vals.copy_(vpr)
        flush.sum()  # read-only pass over 512 MiB: evicts keys from L2 without dirty lines

    gvr = a.workload == "sample_2p28"
    gsd = a.workload == "gsd_2p28"

    def sort():
        if gvr:
            isort.sample_sort(keys, vals, buckets=256, oversample=16, seed=a.seed)
        elif gsd:
            isort.gsd_sort(keys, vals, buckets=16, oversample=4)
        elif vb:
            isort.sort_pairs(keys, vals, rb)
        else:
            isort.sort_keys(keys, rb)

    variant = None
    if rb == 8 and not gvr and not gsd:  # the kernel shape the library resolves for this sort
        r_bits, vi = isort.resolve(n, kb, vb, rb)
        variant = isort.tune_variants(kb, vb, r_bits)[vi]

    clocks = ClockSampler(local)
    clocks.start()  # streaming before the timed region begins
    # warm-up (also allocates the workspace)
    for _ in range(a.warmup):
        restore()
        sort()
    torch.cuda.synchronize()
    if isort.stream_status() != _lib.OK:
        raise RuntimeError("device error during warm-up")

    isort.debug_set(_lib.DEBUG_KERNEL_TIMING, 1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    kernel_ms = {}
    kernel_launches = 0
    rep.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    for i in range(a.steps):
        restore()
        ev[i][0].record(stream)
        sort()
        ev[i][1].record(stream)
        for name, ms in isort.kernel_times():
            kernel_ms.setdefault(name, []).append(ms)
            kernel_launches += 1
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    clocks.window(t_wall0, t_wall0 + t_wall)
    clk = clocks.stop()
    rep.barrier()
    isort.debug_set(_lib.DEBUG_KERNEL_TIMING, 0)
    if isort.stream_status() != _lib.OK:
        raise RuntimeError("device error during the timed steps")
    step_ms = [s.elapsed_time(e) for s, e in ev]
    total_s = rep.max(sum(step_ms) / 1000.0)
    value = n * a.steps * world / total_s

    # sanity: the last result is sorted (device-side check, outside timing);
    # flipping the top bit turns the unsigned order into the signed one
    sk = keys.view(torch.int64 if kb == 64 else torch.int32) ^ (-(1 << (kb - 1)))
    if not bool((sk[1:] >= sk[:-1]).all()):
        raise RuntimeError("benchmark result is not sorted")
    del sk

    # dominant kernel: the onesweep pass (radix 256) or a routing step of a
    # wide-radix round
    dom = max(kernel_ms, key=lambda k: sum(kernel_ms[k]))
    dom_ms = statistics.mean(kernel_ms[dom])
    bytes_per_key = (kb + vb) // 8
    # GVR: the split round, then the radix rounds; GSD: the radix rounds, then lg 16 merge rounds
    passes = -(-kb // rb) + (1 if gvr else 0) + (4 if gsd else 0)
    if dom in ("k_onesweep", "k_wide_high", "k_wide_low", "k_seg_onesweep", "k_gvr_split",
               "k_gsd_merge"):
        # one count-sort round: read and write every key (and payload) once
        alg_bytes = 2 * n * bytes_per_key
    else:
        alg_bytes = n * kb // 8
    peak, peak_kind = measured_peak_hbm()
    achieved = alg_bytes / (dom_ms / 1000.0) / 1e9
    traffic = recorded_traffic(a.workload, variant) if variant else None
    roofline = {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "alg_bytes_per_launch": alg_bytes,
                "avg_launch_ms": dom_ms, "launches": len(kernel_ms[dom])}
    # keys only: the order-free pass-0 round is its own kernel; same algorithmic bytes
    first = next((k for k in ("k_onesweep_first", "k_seg_onesweep_first") if k in kernel_ms), None)
    if first and dom in ("k_onesweep", "k_seg_onesweep"):
        f_ms = statistics.mean(kernel_ms[first])
        roofline["first_round"] = {"kernel": first, "avg_launch_ms": f_ms,
                                   "achieved": alg_bytes / (f_ms / 1000.0) / 1e9,
                                   "frac": alg_bytes / (f_ms / 1000.0) / 1e9 / peak,
                                   "launches": len(kernel_ms[first])}
    if "k_wide_high" in kernel_ms:
        # a wide-radix round = histogram + scans + the two routing steps (radix
        # 65536: plus its share of the one byte-histogram read per sort); its
        # algorithmic bytes are one read and one write of every key
        parts = [k for k in ("k_hist_wide", "k_scan_high", "k_bucket_hist", "k_scan_buckets", "k_scan_wide",
                             "k_wide_high", "k_wide_low") if k in kernel_ms]
        r_ms = sum(statistics.mean(kernel_ms[k]) for k in parts)
        if "k_hist" in kernel_ms:
            rounds = -(-kb // rb)
            r_ms += sum(kernel_ms["k_hist"]) / len(kernel_ms["k_wide_high"])
            parts.append(f"k_hist / {rounds}")
        rb_bytes = 2 * n * bytes_per_key
        roofline["round"] = {"kernels": " + ".join(parts), "avg_round_ms": r_ms,
                             "achieved": rb_bytes / (r_ms / 1000.0) / 1e9,
                             "frac": rb_bytes / (r_ms / 1000.0) / 1e9 / peak}
    # whole-sort roofline by the headline formula: 2 n (w_k + w_v) per executed pass
    sort_alg_bytes = 2 * n * bytes_per_key * passes
    per_kernel = {k: {"launches": len(v), "mean_ms": statistics.mean(v), "total_ms": sum(v)}
                  for k, v in kernel_ms.items()}

    e2e = None
    if not a.no_e2e:
        e2e = measure_e2e(a, n, kb, vb, rb, torch, isort, inputs, stream)

    cpu = None
    if not a.no_cpu_baseline and rank == 0 and world == 1:
        sn, times = oracle_sample(n, kb, vb, rb, a.dist, a.seed, a.cpu_seconds, gvr=gvr, gsd=gsd)
        cpu = {"value": sn * len(times) / sum(times), "unit": "keys/s", "cores": 1,
               "kind": "oracle",
               "sample": f"{len(times)} single-thread oracle sorts of a {sn}-key slice "
                         f"({a.dist}, seed {a.seed}) of the {n}-key workload; host has "
                         f"{cpu_cores_available()} cores"}

    line = {
        "metric": f"uint{kb} keys/s ({desc})",
        "value": value,
        "unit": "keys/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": 1000 * total_s / a.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": f"u{kb}" + (f"+u{vb}" if vb else ""),
        "data": "synthetic",
        "config": {"workload": a.workload, "n": n, "key_bits": kb, "val_bits": vb,
                   "radix_bits": rb, "passes": passes, "dist": a.dist, "seed": a.seed,
                   "variant": list(variant) if variant else None,
                   "l2": "inputs (1 GiB+) larger than L2; keys restored and L2 flushed by a "
                         "512 MiB read before each timed sort, outside the event pair",
                   "parallelism": "replicas" if world > 1 else "1 GPU"},
        "roofline": roofline,
        "sort_roofline": {"alg_bytes_per_sort": sort_alg_bytes,
                          "achieved_gbs": sort_alg_bytes * a.steps / total_s / 1e9,
                          "frac": sort_alg_bytes * a.steps / total_s / 1e9 / peak},
        "kernels": per_kernel,
        "gpu_launches": kernel_launches,
        "clocks": clk,
        "e2e": e2e,
        "cpu_baseline": cpu,
        "wall_s_timed_loop": t_wall,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    rep.close()
    return 0


def measure_e2e(a, n, kb, vb, rb, torch, isort, inputs, stream):
    """keys/s through the C-ABI call with HOST buffers: every step sorts the
    pinned host input into a pinned host output with isort_keys_host /
    isort_pairs_host, which copies the input to the device, sorts it and
    copies the result back on the step's stream (the sample sorts, which have
    no host-buffer entry point, copy with torch around isort_sample_sort /
    isort_gsd_sort). Measured two ways: one step at a time, and pipelined over
    three streams, so that a step's upload overlaps the earlier steps' sorts
    and downloads (the host link runs both directions at once, so the period is
    bound by one direction's copy); the pipelined figure is the line's e2e."""
    host_in = inputs.device_keys(n, kb, a.dist, a.seed).cpu().pin_memory()
    hv_in = inputs.device_iota(n, vb).cpu().pin_memory() if vb else None
    gvr = a.workload == "sample_2p28"
    gsd = a.workload == "gsd_2p28"
    host_api = not (gvr or gsd)
    steps = max(8, min(a.steps, 20))
    nbuf = 3
    streams = [torch.cuda.Stream() for _ in range(nbuf)]
    dev = [None if host_api else torch.empty(n, dtype=host_in.dtype, device="cuda")
           for _ in streams]
    dv = [torch.empty(n, dtype=hv_in.dtype, device="cuda") if vb and not host_api else None
          for _ in streams]
    host_out = [torch.empty_like(host_in).pin_memory() for _ in streams]
    hv_out = [torch.empty_like(hv_in).pin_memory() if vb else None for _ in streams]

    def step(b):
        if host_api:
            if vb:
                isort.sort_pairs_host(host_in, hv_in, host_out[b], hv_out[b], rb,
                                      stream=streams[b])
            else:
                isort.sort_keys_host(host_in, host_out[b], rb, stream=streams[b])
            return
        d, v = dev[b], dv[b]
        d.copy_(host_in, non_blocking=True)
        if vb:
            v.copy_(hv_in, non_blocking=True)
        if gvr:
            isort.sample_sort(d, v, buckets=256, oversample=16, seed=a.seed)
        else:
            isort.gsd_sort(d, v, buckets=16, oversample=4)
        if vb:
            hv_out[b].copy_(v, non_blocking=True)
        host_out[b].copy_(d, non_blocking=True)

    def timed(pipelined):
        for b in range(nbuf):  # warm-up (and workspaces of every stream)
            with torch.cuda.stream(streams[b]):
                step(b)
        torch.cuda.synchronize()
        s, e = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        s.record(stream)
        for i in range(steps):
            b = i % nbuf if pipelined else 0
            streams[b].wait_event(s) if i < nbuf else None
            with torch.cuda.stream(streams[b]):
                step(b)
        for st in streams:
            stream.wait_stream(st)
        e.record(stream)
        e.synchronize()
        return s.elapsed_time(e) / steps

    # the host link and host memory are shared with the machine's other GPUs, and
    # runs fall into a fast and a slow mode: median of five runs each
    serial_runs = [timed(False) for _ in range(5)]
    runs = [timed(True) for _ in range(5)]
    ms_serial = statistics.median(serial_runs)
    ms = statistics.median(runs)
    for b in range(nbuf):
        out = host_out[b].numpy()
        if not (out[1:] >= out[:-1]).all():
            raise RuntimeError("e2e result not sorted")
    bi = n * (kb + vb) // 8
    api = (("isort_pairs_host" if vb else "isort_keys_host") if host_api else
           ("torch copies + isort_sample_sort" if gvr else "torch copies + isort_gsd_sort"))
    return {"value": n / (ms / 1000.0), "unit": "keys/s", "h2d_bytes_per_step": bi,
            "d2h_bytes_per_step": bi, "ms_per_step": ms, "steps": steps, "api": api,
            "pipelined": "three device buffers on three streams: a step's upload overlaps "
                         "the earlier steps' sorts and downloads",
            "runs_ms_per_step": runs,
            "serial": {"value": n / (ms_serial / 1000.0), "ms_per_step": ms_serial,
                       "runs_ms_per_step": serial_runs}}


def run_ours_segmented(a):
    """Batched segmented sort vs one plain sort launch per range, same GPU."""
    import numpy as np
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    rep = Replicas(world, rank, local, "nccl")
    import inputs
    import paper_1808_10292_gb300 as isort
    from paper_1808_10292_gb300 import _lib, tune

    applied = tune.apply(32, 0)
    nseg = 20_000
    L = inputs.segment_lengths(nseg, seed=a.seed)
    off = inputs.segment_offsets(L)
    n = int(off[-1])
    pristine = inputs.device_keys(n, 32, a.dist, a.seed)
    keys = torch.empty_like(pristine)
    d_off = torch.from_numpy(off).cuda()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda").view(torch.int32)
    flush.zero_()
    stream = torch.cuda.current_stream()

    def restore():
        keys.copy_(pristine)
        flush.sum()

    clocks = ClockSampler(local)
    clocks.start()  # streaming before the timed region begins
    for _ in range(a.warmup):
        restore()
        isort.sort_segmented(keys, d_off)
    torch.cuda.synchronize()
    if isort.stream_status() != _lib.OK:
        raise RuntimeError("device error during warm-up")

    isort.debug_set(_lib.DEBUG_KERNEL_TIMING, 1)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(a.steps)]
    kernel_ms = {}
    launches = 0
    rep.barrier()
    torch.cuda.synchronize()
    t_wall0 = time.perf_counter()
    for i in range(a.steps):
        restore()
        ev[i][0].record(stream)
        isort.sort_segmented(keys, d_off)
        ev[i][1].record(stream)
        for name, ms in isort.kernel_times():
            kernel_ms.setdefault(name, []).append(ms)
            launches += 1
    torch.cuda.synchronize()
    clocks.window(t_wall0, time.perf_counter())
    clk = clocks.stop()
    rep.barrier()
    isort.debug_set(_lib.DEBUG_KERNEL_TIMING, 0)
    if isort.stream_status() != _lib.OK:
        raise RuntimeError("device error during the timed steps")
    total_s = rep.max(sum(s.elapsed_time(e) for s, e in ev) / 1000.0)
    value = n * a.steps * world / total_s

    # the same call captured once in a CUDA graph (workspace bound to the
    # capturing stream) and replayed: the whole launch sequence without host work
    gstream = torch.cuda.Stream()
    gws = torch.empty(isort.segmented_workspace_size(nseg, n, 32, 0), dtype=torch.uint8,
                      device="cuda")
    isort.set_workspace(gws, stream=gstream)
    with torch.cuda.stream(gstream):
        restore()
        isort.sort_segmented(keys, d_off)
    gstream.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gstream):
        isort.sort_segmented(keys, d_off)
    gms = []
    for _ in range(a.steps):
        restore()
        g0, g1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        g0.record(stream)
        graph.replay()
        g1.record(stream)
        g1.synchronize()
        gms.append(g0.elapsed_time(g1))
    if isort.stream_status(gstream) != _lib.OK:
        raise RuntimeError("device error in the graph replays")
    isort.set_workspace(None, stream=gstream)
    del graph, gws
    torch.cuda.empty_cache()
    graph_replay = {"value": n / (statistics.median(gms) / 1000.0), "unit": "keys/s",
                    "ms": statistics.median(gms), "replays": len(gms),
                    "how": "isort_segmented captured once in a CUDA graph, replayed per step"}

    # baseline: one plain sort per range through the public call, same GPU
    restore()
    torch.cuda.synchronize()
    s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    s0.record(stream)
    for s in range(nseg):
        if L[s] > 1:
            isort.sort_keys(keys[off[s]:off[s + 1]], 8)
    s1.record(stream)
    s1.synchronize()
    base_ms = s0.elapsed_time(s1)
    if isort.stream_status() != _lib.OK:
        raise RuntimeError("device error in the per-range baseline")
    got = keys.cpu().numpy()
    restore()
    isort.sort_segmented(keys, d_off)
    if not np.array_equal(got, keys.cpu().numpy()):
        raise RuntimeError("batched and per-range results differ")

    btn_max = (applied.get("segmented") or {}).get("btn_max", 4096)
    n_radix = int(L[L > btn_max].sum())
    dom = "k_seg_onesweep"
    dom_ms = statistics.mean(kernel_ms[dom])
    alg_bytes = 2 * n_radix * 4
    peak, peak_kind = measured_peak_hbm()
    achieved = alg_bytes / (dom_ms / 1000.0) / 1e9
    cpu = None
    if not a.no_cpu_baseline and rank == 0 and world == 1:
        import oracle
        host = pristine.cpu().numpy()
        oracle.radix_sort(host[:1024])
        done_keys, t_cpu, t_end = 0, 0.0, time.perf_counter() + a.cpu_seconds
        s = 0
        while time.perf_counter() < t_end and s < nseg:
            seg = host[off[s]:off[s + 1]]
            t0 = time.perf_counter()
            oracle.radix_sort(seg)
            t_cpu += time.perf_counter() - t0
            done_keys += len(seg)
            s += 1
        cpu = {"value": done_keys / max(t_cpu, 1e-9), "unit": "keys/s", "cores": 1,
               "kind": "oracle",
               "sample": f"the first {s} of the 20,000 ranges ({done_keys} keys), one oracle "
                         f"sort per range, 1 thread"}
    line = {
        "metric": "batched-segment keys/s (20,000 ranges, log-uniform lengths in [1, 2^20])",
        "value": value,
        "unit": "keys/s",
        "n_gpus": world,
        "steps": a.steps,
        "warmup": a.warmup,
        "ms_per_step": 1000 * total_s / a.steps,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32",
        "data": "synthetic",
        "config": {"workload": a.workload, "num_segments": nseg, "keys": n, "dist": a.dist,
                   "seed": a.seed, "tuned": applied, "radix_keys": n_radix,
                   "l2": "inputs (6 GB) larger than L2; restored and L2 flushed before each step"},
        "per_range_baseline": {"value": n / (base_ms / 1000.0), "unit": "keys/s",
                               "ms": base_ms, "calls": int((L > 1).sum()),
                               "how": "one isort_keys call per range (radix 256), same GPU"},
        "speedup_vs_per_range": (n / total_s * a.steps) / (n / (base_ms / 1000.0)),
        "graph_replay": graph_replay,
        "roofline": {"bound": "hbm", "kernel": dom, "achieved": achieved, "peak": peak,
                     "peak_kind": peak_kind, "unit": "GB/s", "frac": achieved / peak,
                     "traffic": None, "alg_bytes_per_launch": alg_bytes, "avg_launch_ms": dom_ms},
        "kernels": {k: {"launches": len(v), "mean_ms": statistics.mean(v), "total_ms": sum(v)}
                    for k, v in kernel_ms.items()},
        "gpu_launches": launches,
        "clocks": clk,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    rep.close()
    return 0


def run_ours_short_ranges(a):
    """The two short-range networks of the paper (BTN, OET) on batches of equal
    ranges: for each range length L, 2^26 / L ranges of uint32 keys sorted with
    one isort_segmented call; CUDA events per call, keys restored and L2
    flushed outside the event pair, median of the timed steps."""
    import numpy as np
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    import inputs
    import paper_1808_10292_gb300 as isort
    from paper_1808_10292_gb300 import _lib
    n = 1 << 26
    stream = torch.cuda.current_stream()
    pristine = inputs.device_keys(n, 32, a.dist, a.seed)
    keys = torch.empty_like(pristine)
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda").view(torch.int32)
    flush.zero_()
    clocks = ClockSampler(local)
    clocks.start()
    table, launches = {}, 0
    isort.debug_set(_lib.DEBUG_KERNEL_TIMING, 1)  # to count the library's launches
    t_wall0 = time.perf_counter()
    for L in (32, 128, 512, 2048, 4096):
        off = torch.arange(0, n + 1, L, dtype=torch.int64, device="cuda")
        table[L] = {}
        for net in ("btn", "oet"):
            isort.tune_segmented_network(32, 0, net)
            ms = []
            for i in range(a.warmup + a.steps):
                keys.copy_(pristine)
                flush.sum()
                s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                s0.record(stream)
                isort.sort_segmented(keys, off)
                s1.record(stream)
                s1.synchronize()
                kt = isort.kernel_times()
                if i >= a.warmup:
                    ms.append(s0.elapsed_time(s1))
                    launches += len(kt)
            if isort.stream_status() != _lib.OK:
                raise RuntimeError("device error in the short-range benchmark")
            sk = keys.view(torch.int32) ^ (-(1 << 31))
            srt = (sk.view(-1, L)[:, 1:] >= sk.view(-1, L)[:, :-1]).all().item()
            if not srt:
                raise RuntimeError(f"ranges of {L} keys not sorted ({net})")
            q = 32 if L <= 128 else 64 if L <= 512 else 256
            table[L][net] = {"keys_per_s": n / (statistics.median(ms) / 1000.0),
                             "ms": statistics.median(ms), "q_threads": q,
                             "network_steps": (q.bit_length() - 1) * q.bit_length() // 2
                             if net == "btn" else q}
    isort.tune_segmented_network(32, 0, "btn")
    isort.debug_set(_lib.DEBUG_KERNEL_TIMING, 0)
    clocks.window(t_wall0, time.perf_counter())
    clk = clocks.stop()
    tot_btn = sum(table[L]["btn"]["ms"] for L in table)
    line = {
        "metric": "short-range keys/s (equal ranges of 32..4096 uint32 keys, BTN network)",
        "value": n * len(table) / (tot_btn / 1000.0),
        "unit": "keys/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": tot_btn, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": a.workload, "keys_per_length": n, "dist": a.dist, "seed": a.seed,
                   "l2": "256 MiB of keys per call, restored and L2 flushed before each call"},
        "networks": {str(L): v for L, v in table.items()},
        "oet_over_btn_time": {str(L): table[L]["oet"]["ms"] / table[L]["btn"]["ms"]
                              for L in table},
        "gpu_launches": launches,
        "clocks": clk,
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    return 0


def run_mbsp(a):
    """The paper's MBSP accounting (paper_1808_10292_gb300/mbsp.py) on this GPU:
    g from the measured copy bandwidth, G from the measured radix-256 round of
    2^28 uint32 keys; then model vs measured whole-sort times for other widths,
    payloads and radixes, and with the paper's own g = 5G."""
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    import inputs
    import paper_1808_10292_gb300 as isort
    from paper_1808_10292_gb300 import _lib, mbsp
    stream = torch.cuda.current_stream()
    flush = torch.empty(512 << 20, dtype=torch.uint8, device="cuda").view(torch.int32)
    flush.zero_()
    isort.debug_set(_lib.DEBUG_KERNEL_TIMING, 1)
    clocks = ClockSampler(local)
    clocks.start()
    t_wall0 = time.perf_counter()
    cases = [(1 << 28, 32, 0, 8), (1 << 27, 32, 32, 8), (1 << 26, 64, 0, 8),
             (1 << 28, 32, 0, 11), (1 << 28, 32, 0, 16)]
    measured, launches = {}, 0
    for n, kb, vb, rb in cases:
        pristine = inputs.device_keys(n, kb, a.dist, a.seed)
        keys = torch.empty_like(pristine)
        vals = inputs.device_iota(n, vb) if vb else None
        ms, rounds_ms = [], []
        for i in range(a.warmup + a.steps):
            keys.copy_(pristine)
            flush.sum()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            if vb:
                isort.sort_pairs(keys, vals, rb)
            else:
                isort.sort_keys(keys, rb)
            e1.record(stream)
            e1.synchronize()
            kt = isort.kernel_times()
            if i >= a.warmup:
                ms.append(e0.elapsed_time(e1))
                # the last ordered round of the sort
                rounds_ms += [t for k, t in kt if k == "k_onesweep"][-1:]
                launches += len(kt)
        if isort.stream_status() != _lib.OK:
            raise RuntimeError("device error in the model benchmark")
        measured[(n, kb, vb, rb)] = {"sort_ms": statistics.median(ms),
                                     "round_ms": statistics.median(rounds_ms) if rounds_ms else None}
        del pristine, keys, vals
        torch.cuda.empty_cache()
    isort.debug_set(_lib.DEBUG_KERNEL_TIMING, 0)
    clocks.window(t_wall0, time.perf_counter())
    clk = clocks.stop()
    peak, peak_kind = measured_peak_hbm()
    base = measured[cases[0]]
    cal = mbsp.calibrate(peak, base["round_ms"] / 1000.0, cases[0][0])
    g, G = cal["g"], cal["G"]
    rows = []
    for (n, kb, vb, rb) in cases:
        m = measured[(n, kb, vb, rb)]["sort_ms"]
        pred = 1000 * mbsp.gpu_sort(n, kb, vb, 1 << rb, g, G)
        pred5 = 1000 * mbsp.gpu_sort(n, kb, vb, 1 << rb, g, g / 5)
        rows.append({"n": n, "key_bits": kb, "val_bits": vb, "radix": 1 << rb,
                     "measured_ms": m, "model_ms": pred, "model_error": pred / m - 1,
                     "model_g5G_ms": pred5, "model_g5G_error": pred5 / m - 1})
    line = {
        "metric": "MBSP model vs measured sort time (calibrated on the 2^28 uint32 radix-256 round)",
        "value": cases[0][0] / (base["sort_ms"] / 1000.0),
        "unit": "keys/s", "n_gpus": 1, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": base["sort_ms"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": a.workload, "dist": a.dist, "seed": a.seed,
                   "l2": "inputs larger than L2; restored and L2 flushed before each sort"},
        "calibration": {"hbm_gbs": peak, "peak_kind": peak_kind, "g_s_per_word": g,
                        "G_s_per_access": G, "g_over_G": cal["g_over_G"],
                        "shared_accesses_per_key_round": mbsp.SHARED_ACCESSES_ORDERED,
                        "onesweep_round_ms": base["round_ms"]},
        "predictions": rows,
        "gpu_launches": launches,
        "clocks": clk,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_ours_serve(a):
    """Served (continuous batching) vs sequential plain sorts on one Poisson trace;
    then both arms on a backlog (every request queued at once) for capacity."""
    import numpy as np
    import torch
    world, rank, local = dist_env()
    torch.cuda.set_device(local)
    import inputs
    import paper_1808_10292_gb300 as isort
    from paper_1808_10292_gb300 import serve, tune
    applied = tune.apply(32, 0)
    tune.apply(32, 32)
    arrivals, sizes, payload = inputs.requests(int(2000 * a.serve_seconds * 1.2) + 10, seed=a.seed)

    def make_fill(rid, n, pay):
        def fill(keys, vals, stream):
            inputs.device_keys(n, 32, "uniform", seed=a.seed,
                               stream=inputs.STREAM_REQUEST_BASE + rid, out=keys,
                               cuda_stream=stream)
            if vals is not None:
                inputs.device_iota(n, 32, out=vals, cuda_stream=stream)
        return fill

    # self-checks of the served loop: every 100th request and every request of
    # at most 2^16 keys keeps a copy of its result (taken in its done callback,
    # before its arena space is reused), verified after the run
    kept = {}

    def keep(r, keys, vals):
        if r.rid % 100 == 0 or r.n <= (1 << 16):
            kept[r.rid] = (r, keys.clone(), None if vals is None else vals.clone())
            torch.cuda.current_stream().synchronize()

    def verify():
        """Each kept result equals the same request sorted alone (plain sort,
        bit for bit, on the device); every 10th kept one also the CPU oracle."""
        import oracle
        bad = oracle_checked = 0
        for i, (rid, (r, k, v)) in enumerate(sorted(kept.items())):
            alone_k = torch.empty(r.n, dtype=torch.uint32, device="cuda")
            alone_v = torch.empty(r.n, dtype=torch.uint32, device="cuda") if r.payload else None
            make_fill(rid, r.n, r.payload)(alone_k, alone_v, torch.cuda.current_stream())
            if r.payload:
                isort.sort_pairs(alone_k, alone_v, 8)
            else:
                isort.sort_keys(alone_k, 8)
            ok = torch.equal(alone_k, k) and (v is None or torch.equal(alone_v, v))
            if ok and i % 10 == 0:
                src = inputs.keys(r.n, 32, "uniform", seed=a.seed,
                                  stream=inputs.STREAM_REQUEST_BASE + rid)
                ok = bool(np.array_equal(k.cpu().numpy(), oracle.radix_sort(src)))
                oracle_checked += 1
            bad += 0 if ok else 1
        return {"kept": len(kept), "mismatches": bad, "oracle_checked": oracle_checked,
                "how": "every 100th request and all of at most 2^16 keys: bit-exact against the "
                       "same request sorted alone on the device; every 10th of those against "
                       "the CPU oracle"}

    def arm(batching, arr, duration, done=None):
        srv = serve.SortServer(budget_bytes=40 << 30, num_streams=4, max_batch_keys=1 << 27,
                               max_batch_requests=2048, batching=batching)
        # warm-up: a few requests through the same server
        wa = np.zeros(16)
        serve.drive(srv, wa, sizes[:16], payload[:16], make_fill, duration_s=1.0)
        srv.close()
        srv = serve.SortServer(budget_bytes=40 << 30, num_streams=4, max_batch_keys=1 << 27,
                               max_batch_requests=2048, batching=batching)
        clocks = ClockSampler(local)
        clocks.start()
        l0 = isort.launch_count()
        t0 = time.perf_counter()
        reqs = serve.drive(srv, arr, sizes, payload, make_fill, duration_s=duration, done=done)
        srv.close()
        wall = time.perf_counter() - t0
        launches = isort.launch_count() - l0
        clocks.window(t0, t0 + wall)
        clk = clocks.stop()
        if srv.errors:
            raise RuntimeError(f"serving errors: {srv.errors[:3]}")
        out = serve.latency_summary(reqs)
        out.update({"batches": srv.batches, "rejected": len(srv.rejected), "wall_s": wall,
                    "gpu_launches": launches, "clocks": clk})
        del srv
        torch.cuda.empty_cache()
        return out

    served = arm(True, arrivals, a.serve_seconds)
    # a separate, untimed served run of the trace's first seconds keeps and checks
    # results (the copies would disturb the latencies of the timed run)
    arm(True, arrivals, min(5.0, a.serve_seconds), done=keep)
    served["self_check"] = verify()
    if served["self_check"]["mismatches"]:
        raise RuntimeError(f"served results differ: {served['self_check']}")
    kept.clear()
    sequential = arm(False, arrivals, a.serve_seconds)
    # capacity: a backlog of the first 4,000 requests, all queued at t = 0
    backlog = np.zeros_like(arrivals)
    cap_n = 4000
    cap_served = arm(True, backlog[:cap_n], 1.0)
    cap_seq = arm(False, backlog[:cap_n], 1.0)
    line = {
        "metric": "served keys/s and p50/p99 latency (Poisson 2,000 req/s, sizes log-uniform in "
                  "[2^10, 2^24] uint32 keys, half with uint32 payloads, 40 GB budget)",
        "value": served["keys_per_s"],
        "unit": "keys/s",
        "n_gpus": 1,
        "steps": served["requests"],
        "warmup": 16,
        "ms_per_step": served["mean_ms"],
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "u32+u32",
        "data": "synthetic",
        "config": {"workload": a.workload, "rate_per_s": 2000, "seconds": a.serve_seconds,
                   "budget_bytes": 40 << 30, "streams": 4, "max_batch_keys": 1 << 27,
                   "tuned": applied, "seed": a.seed},
        "served": served,
        "sequential_plain_sorts": sequential,
        "capacity_backlog_4000": {"served": cap_served, "sequential": cap_seq,
                                  "speedup": cap_served["keys_per_s"] / cap_seq["keys_per_s"]},
        "gpu_launches": served["gpu_launches"],
        "clocks": served["clocks"],
        "e2e": None,  # requests are generated on the device by their fill callbacks
    }
    print(json.dumps(line), flush=True)
    return 0


def main():
    a = parse()
    if a.workload == "serve_poisson":
        if a.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "the serving workload has "
                              "no CPU counterpart; the oracle arm is timed on the plain and "
                              "segmented workloads"}))
            return 0
        return run_ours_serve(a)
    if a.workload == "segmented_20000":
        if a.impl == "reference":
            return run_reference_segmented(a)
        return run_ours_segmented(a)
    if a.workload == "mbsp_model":
        if a.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "model comparison only; the "
                              "oracle arm is timed on the plain and segmented workloads"}))
            return 0
        return run_mbsp(a)
    if a.workload == "short_ranges":
        if a.impl == "reference":
            print(json.dumps({"impl": "reference", "unavailable": "network comparison only; "
                              "the oracle arm is timed on the plain and segmented workloads"}))
            return 0
        return run_ours_short_ranges(a)
    if a.impl == "reference":
        return run_reference(a)
    return run_ours(a)


if __name__ == "__main__":
    sys.exit(main())
