#!/usr/bin/env python3
"""Throughput of the single-device sort on GB300: keys GB/s sorted.

Workload (one "step"): 268,435,456 int64 keys uniform over all 2^64 bit patterns
and 268,435,456 float32 keys ~ N(0,1) with 0.1% NaN (random sign and payload)
and 0.1% -0.0; each array goes through a stable ak_sortperm (UInt32 indices) and
an in-place ak_sort, ascending -- the rank-local sort of the paper's sample sort
(Sec. IV-A) on its int64/float32 dtypes.  value = key bytes sorted per step (4
calls) / device time, in GB/s (1e9 B/s), summed over ranks.

Timing: 3+ warm-up steps; each call is bracketed by CUDA events on its stream;
before every call the keys are restored from a pristine device copy and a 256 MiB
buffer is written to flush L2 -- both outside the events.  The inputs (1-2 GiB)
are larger than L2 as well.  SM clocks are sampled with nvidia-smi during the
timed steps.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
       python bench.py --workload c1|c3|c4|c5|searchsorted|accumulate|int128   (their own lines)
Under torchrun every rank sorts its own replica of the workload on its own GPU
(the sort has no exchange step on one node here: replicas, weak scaling).
"""
from __future__ import annotations

import argparse
import ctypes
import json
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

FULL_N = 268_435_456
METRIC = "keys GB/s sorted (device-timed, 1 GB300) and % of 2×bytes/8TB/s roofline; learned vs plain"
NOMINAL_HBM_GBS = 8000.0
# ncu dram__bytes_read.sum + dram__bytes_write.sum of onesweep_pass, averaged
# over the digit-pass launches of one step of this workload at a smaller n
# (keys per array, bytes per launch).  Traffic grows in proportion to the keys,
# so it is scaled to the run's n.  None whenever the digit-pass kernel has
# changed since the counters were taken.
NCU_TRAFFIC = (67_108_864, 995_233_738)
# ncu DRAM read + write bytes of one int64 accumulate call (keys, bytes)
ACC_NCU_TRAFFIC = (268_435_456, 6_404_700_000)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=FULL_N, help="keys per array (default: the full workload)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-vs-plain comparison of the headline")
    ap.add_argument("--workload", default="c2", choices=["c2", "c1", "c3", "c4", "c5", "searchsorted", "accumulate", "int128"],
                    help="c2 (default): the headline line; the others print their own lines")
    ap.add_argument("--segments", type=int, default=65536, help="c4: number of segments")
    ap.add_argument("--tile-config", type=int, default=0, choices=range(0, 6),
                    help="c2: digit-pass tile configuration (0 = default = 1; 5 = reduce-then-scan)")
    return ap.parse_args()


def workload_config(n: int) -> dict:
    return {
        "workload": (f"{n:,} int64 uniform(all bits) + {n:,} float32 N(0,1) with 0.1% NaN and 0.1% -0.0; "
                     "ak_sortperm (stable, UInt32) + ak_sort each, ascending; plain radix path"),
        "keys_per_array": n,
        "calls_per_step": 4,
        "key_bytes_per_step": 24 * n,
        "l2": "256 MiB flush write before every call; inputs 1-2 GiB (> 129 MB L2)",
        "timing": "sum of CUDA-event intervals around each ak_* call; input restore and L2 flush excluded",
        "parallelism": "replicas (one independent sort per GPU)",
    }


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks/throttle reasons every 200 ms while running."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, target: str | None):
        self.proc = None
        self.target = target

    def start(self):
        cmd = ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.target:
            cmd += ["-i", self.target]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            out, _ = self.proc.communicate(timeout=5)
        except Exception:
            self.proc.kill()
            out, _ = self.proc.communicate()
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
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def gpu_target(torch, dev: int):
    try:
        p = torch.cuda.get_device_properties(dev)
        return f"{p.pci_domain_id:08X}:{p.pci_bus_id:02X}:{p.pci_device_id:02X}.0"
    except Exception:
        vis = os.environ.get("CUDA_VISIBLE_DEVICES", "")
        return vis.split(",")[dev] if vis else str(dev)


def _cpulist(text: str) -> set[int]:
    """CPU ids of a sysfs list such as '0-71,144-215'."""
    out = set()
    for part in text.strip().split(","):
        if part:
            a, _, b = part.partition("-")
            out.update(range(int(a), int(b or a) + 1))
    return out


def bind_to_gpu_node(torch, dev: int) -> dict:
    """Keep this process on the CPUs next to the GPU (its PCI device's local
    CPU list), so that the pinned host buffers of the end-to-end leg come from
    the memory attached to the GPU rather than another socket's.  Leaves the
    affinity alone when the list is missing or shares no CPU with it."""
    try:
        allowed = os.sched_getaffinity(0)
        p = torch.cuda.get_device_properties(dev)
        path = f"/sys/bus/pci/devices/{p.pci_domain_id:04x}:{p.pci_bus_id:02x}:{p.pci_device_id:02x}.0/local_cpulist"
        with open(path) as f:
            local = _cpulist(f.read())
        use = local & allowed
        if use and use != allowed:
            os.sched_setaffinity(0, use)
        return {"gpu_local_cpus": len(local), "allowed_cpus": len(allowed), "bound_cpus": len(use or allowed)}
    except Exception as e:  # no sysfs entry or no affinity call: measure unbound
        return {"unbound": type(e).__name__}


def onesweep_bytes(op: str, n: int, w: int, passes: int, packed: bool = False) -> list[int]:
    """Algorithmic bytes of each digit pass (the dominant kernel) of one call,
    every pass active.  packed: a sortperm of 8-byte keys whose upper-half
    passes move (upper key half, index) words of 8 bytes."""
    if op == "sort":
        return [2 * n * w] * passes
    out = []
    half = passes // 2
    for q in range(passes):
        if q == 0:
            out.append(2 * n * w + 4 * n)          # read keys, write keys + generated index
        elif packed and q == half - 1:
            out.append(n * w + 4 * n + 8 * n)      # read keys + index, write packed words
        elif packed and q == passes - 1:
            out.append(8 * n + 4 * n)              # read packed words, write the index
        elif packed and q >= half:
            out.append(16 * n)                     # packed words in and out
        elif q == passes - 1:
            out.append(n * w + 8 * n)              # read keys + perm, write perm only
        else:
            out.append(2 * n * w + 8 * n)
    return out


# ------------------------------------------------------------ output checks
# Every GB/s printed comes from a call whose output was checked on the host.
# These checks are the bench's own (numpy, no library code): the order of Julia
# isless as unsigned integers, an order-independent hash of the raw bits for the
# multiset, and the three properties that make a permutation THE stable one.

def _order_key(a: np.ndarray) -> np.ndarray:
    """Unsigned integers of a's width ordered like Julia isless: unsigned as is,
    signed with the sign bit flipped, floats negative -> all bits flipped,
    non-negative -> sign bit flipped, every NaN -> the maximum."""
    w = a.dtype.itemsize
    ut = np.dtype(f"u{w}")
    u = a.view(ut)
    if a.dtype.kind == "u":
        return u
    sign = ut.type(1 << (8 * w - 1))
    if a.dtype.kind == "i":
        return u ^ sign
    out = np.where((u & sign) != 0, ~u, u ^ sign).astype(ut)
    out[np.isnan(a)] = np.iinfo(ut).max
    return out


def _bits_hash(a: np.ndarray) -> int:
    """Sum over elements of a 64-bit mix of their raw bits (mod 2^64): equal for
    any two orderings of the same multiset."""
    z = a.view(np.dtype(f"u{a.dtype.itemsize}")).astype(np.uint64)
    with np.errstate(over="ignore"):
        z = (z ^ (z >> np.uint64(31))) * np.uint64(0x7FB5D329728EA185)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x81DADEF4BC2DD44D)
        z ^= z >> np.uint64(33)
        return int(z.sum(dtype=np.uint64))


def check_sorted(inp: np.ndarray, out: np.ndarray, desc: bool = False) -> bool:
    """out is inp's multiset, in isless order (reversed when desc)."""
    if out.shape != inp.shape:
        return False
    r = _order_key(out)
    ok = bool(np.all(r[1:] <= r[:-1])) if desc else bool(np.all(r[1:] >= r[:-1]))
    return ok and _bits_hash(inp) == _bits_hash(out)


def check_perm(inp: np.ndarray, perm: np.ndarray, desc: bool = False, sorted_out: np.ndarray | None = None) -> bool:
    """perm is the stable sortperm of inp: a permutation, listing keys in order,
    equivalent neighbours in increasing index; sorted_out (if given) = inp[perm]."""
    p = perm.astype(np.int64)
    n = inp.size
    if p.size != n or (n and (p.min() < 0 or p.max() >= n)):
        return False
    if n and not np.all(np.bincount(p, minlength=n) == 1):
        return False
    r = _order_key(inp)[p]
    if desc:
        r = ~r
    if not np.all(r[1:] >= r[:-1]):
        return False
    tie = r[1:] == r[:-1]
    if not np.all(p[1:][tie] > p[:-1][tie]):
        return False
    if sorted_out is not None:
        w = np.dtype(f"u{inp.dtype.itemsize}")
        return bool(np.array_equal(sorted_out.view(w), inp.view(w)[p]))
    return True


def time_sort(torch, ak, dev, stream, flush, host, kd, opts, op="sort", vals=None, order="ascending",
              warmup=3, steps=5, check=True):
    """Median device time of one ak_sort / ak_sortperm / ak_sort_pairs call on
    `host` keys (restored from a pristine device copy and L2 flushed before
    every call, both outside the events).  Returns (key GB/s, ms, ak_info, ok),
    ok from the host check of the last call's output."""
    unsigned = host.dtype.kind == "u"
    view = {2: np.int16, 4: np.int32, 8: np.int64}[host.itemsize] if unsigned else host.dtype
    pristine = torch.from_numpy(host.view(view)).to(dev)
    work = torch.empty_like(pristine)
    o = ak.Options()
    for k, v in (opts or {}).items():
        setattr(o, k, v)
    vp = vw = perm = None
    if op == "pairs":
        vp = torch.from_numpy(vals.view(np.int32)).to(dev)
        vw = torch.empty_like(vp)
        tb = ak.temp_bytes(ak.AK_OP_SORT_PAIRS, host.size, kd, 4, options=o)
    elif op == "sortperm":
        perm = torch.empty(host.size, dtype=torch.int32, device=dev)
        tb = ak.temp_bytes(ak.AK_OP_SORTPERM, host.size, kd, options=o)
    else:
        tb = ak.temp_bytes(ak.AK_OP_SORT, host.size, kd, options=o)
    temp = ak.workspace(tb, dev)
    lib = ak.load()
    od = ak.order_code(order)

    def restore():
        work.copy_(pristine)
        if vw is not None:
            vw.copy_(vp)

    def call():
        if op == "pairs":
            rc = lib.ak_sort_pairs(work.data_ptr(), vw.data_ptr(), 4, host.size, kd, od, temp.data_ptr(),
                                   temp.numel(), stream.cuda_stream, ctypes.byref(o))
        elif op == "sortperm":
            rc = lib.ak_sortperm(work.data_ptr(), perm.data_ptr(), host.size, kd, od, temp.data_ptr(), temp.numel(),
                                 stream.cuda_stream, ctypes.byref(o))
        else:
            rc = lib.ak_sort(work.data_ptr(), host.size, kd, od, temp.data_ptr(), temp.numel(),
                             stream.cuda_stream, ctypes.byref(o))
        if rc:
            raise ak.AkError(rc, op)

    ms = _timed(torch, stream, flush, restore, call, warmup, steps)
    info = ak.ak_last_info(temp)
    ok = None
    if check:
        desc = od == ak.AK_DESCENDING
        if op == "sortperm":
            ok = check_perm(host, perm.cpu().numpy().view(np.uint32), desc)
        else:
            out = work.cpu().numpy().view(host.dtype)
            ok = check_sorted(host, out, desc)
            if ok and op == "pairs":
                v_out = vw.cpu().numpy().view(np.uint32)
                ok = check_perm(host, v_out, desc, sorted_out=out)  # values = input index
        ok = ok and info["status"] == 0
    del pristine, work, temp, vp, vw, perm
    torch.cuda.empty_cache()
    return host.nbytes / (ms / 1e3) / 1e9, ms, info, ok


PATH_NAMES = {1: "radix", 2: "learned", 3: "block", 4: "merge"}


def cpu_oracle_rate(k64: np.ndarray, k32: np.ndarray, sample: int, threads: int) -> tuple[float, float]:
    """Oracle (threaded merge sort) on `sample` keys of each array, the same four
    calls as a step.  Returns (GB/s of keys, seconds)."""
    import oracle
    t0 = time.perf_counter()
    nbytes = 0
    for arr in (k64[:sample], k32[:sample]):
        oracle.sortperm(arr, threads=threads)                  # sortperm
        oracle.gather(arr, oracle.sortperm(arr, threads=threads))  # sort
        nbytes += 2 * arr.nbytes
    dt = time.perf_counter() - t0
    return nbytes / dt / 1e9, dt


def job_ms(local_ms, world, device=None):
    """Job time: the slowest rank's time (max over ranks; barrier-synchronised
    steps), all-reduced so every rank holds it."""
    if world <= 1:
        return float(local_ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(local_ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_gbps(world, bytes_per_rank_step, steps, total_ms):
    """Whole-job throughput: every rank's bytes over the job time (weak scaling)."""
    return world * bytes_per_rank_step * steps / (total_ms / 1e3) / 1e9


def base_line(args, world, cfg):
    return {"metric": METRIC, "unit": "GB/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64+u32 radix keys (int64, float32 inputs)", "data": "synthetic (seeded splitmix64)",
            "config": cfg}


def run_reference(args):
    """The oracle as it stands, on this host's cores, on bounded samples."""
    world, rank, _ = dist_env()
    if rank != 0:
        return
    import synth
    threads = os.cpu_count() or 1
    sample = min(args.n, 1 << 23)
    k64 = synth.uniform_i64(sample, seed=2)
    k32 = synth.normal_f32_special(sample, seed=3)
    for _ in range(args.warmup):
        cpu_oracle_rate(k64, k32, min(sample, 1 << 16), threads)
    secs = []
    for _ in range(args.steps):
        _, dt = cpu_oracle_rate(k64, k32, sample, threads)
        secs.append(dt)
    step_bytes = 24 * sample
    value = step_bytes * len(secs) / sum(secs) / 1e9
    line = base_line(args, world, workload_config(args.n))
    line.update({"impl": "reference", "value": round(value, 4), "ms_per_step": round(1e3 * sum(secs) / len(secs), 3),
                 "cpu_baseline": {"value": round(value, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
                                  "sample": f"{sample:,} int64 + {sample:,} float32 keys per step (sortperm + sort each)"},
                 "e2e": {"value": round(value, 4), "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
                 "gpu_launches": 0})
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch

    import paper_2507_16710_gb300 as ak
    import synth

    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local if world > 1 else 0)
    torch.cuda.set_device(dev)
    host_binding = bind_to_gpu_node(torch, dev.index)  # before any large host allocation
    n = args.n
    cfg = workload_config(n)

    k64 = synth.uniform_i64(n, seed=2)
    k32 = synth.normal_f32_special(n, seed=3)
    arrays = []
    for host, kd, w in ((k64, ak.AK_I64, 8), (k32, ak.AK_F32, 4)):
        pristine = torch.from_numpy(host).to(dev)
        arrays.append({"pristine": pristine, "work": torch.empty_like(pristine), "kd": kd, "w": w})
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    tb = max(ak.temp_bytes(op, n, kd, options={"path": ak.AK_PATH_RADIX, "tile_config": args.tile_config})
             for op in (ak.AK_OP_SORT, ak.AK_OP_SORTPERM) for kd in (ak.AK_I64, ak.AK_F32))
    temp = ak.workspace(tb, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream(dev)
    lib = ak.load()

    # per-pass profiling events (raw handles created by a first record)
    pass_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * ak.AK_MAX_PASSES)]
    for e in pass_ev:
        e.record(stream)
    ev_arr = (ctypes.c_void_p * len(pass_ev))(*[e.cuda_event for e in pass_ev])
    opts = ak.Options()
    opts.path = ak.AK_PATH_RADIX  # the plain radix path: the digit-pass kernel is the roofline's subject
    opts.tile_config = args.tile_config
    opts.pass_events = ctypes.cast(ev_arr, ctypes.c_void_p)
    calls = [("sortperm", 0), ("sort", 0), ("sortperm", 1), ("sort", 1)]

    radix_opts = ak.Options()
    radix_opts.path = ak.AK_PATH_RADIX
    radix_opts.tile_config = args.tile_config

    def call(op, a, with_events):
        o = ctypes.byref(opts) if with_events else ctypes.byref(radix_opts)
        if op == "sort":
            rc = lib.ak_sort(a["work"].data_ptr(), n, a["kd"], 0, temp.data_ptr(), temp.numel(),
                             stream.cuda_stream, o)
        else:
            rc = lib.ak_sortperm(a["work"].data_ptr(), perm.data_ptr(), n, a["kd"], 0, temp.data_ptr(),
                                 temp.numel(), stream.cuda_stream, o)
        if rc:
            raise ak.AkError(rc, op)

    # warm-up (also learns how many digit passes move data per call)
    passes = {}
    for _ in range(args.warmup):
        for op, i in calls:
            arrays[i]["work"].copy_(arrays[i]["pristine"])
            call(op, arrays[i], False)
            passes[(op, i)] = ak.ak_last_info(temp)["radix_passes"]
    torch.cuda.synchronize(dev)
    if world > 1:
        torch.distributed.barrier()

    call_ms = []
    per_call = {f"{op}_{'i64' if i == 0 else 'f32'}": [] for op, i in calls}
    pass_ms, pass_bytes = [], []
    sampler = ClockSampler(gpu_target(torch, dev.index))
    sampler.start()
    time.sleep(0.3)
    torch.cuda.synchronize(dev)
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        evs = []
        for op, i in calls:
            a = arrays[i]
            a["work"].copy_(a["pristine"])
            flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            call(op, a, True)
            e1.record(stream)
            torch.cuda.synchronize(dev)  # pass events are reused by the next call
            evs.append((e0, e1))
            npass = a["w"]
            packed = a["w"] == 8 and args.tile_config in (0, 1) and n <= (1 << 30)
            pb = onesweep_bytes(op, n, a["w"], npass, packed)
            for p in range(npass):
                pass_ms.append(pass_ev[2 * p].elapsed_time(pass_ev[2 * p + 1]))
                pass_bytes.append(pb[p] if passes[(op, i)] == npass else 0)
        ms = [e0.elapsed_time(e1) for e0, e1 in evs]
        for (op, i), t in zip(calls, ms):
            per_call[f"{op}_{'i64' if i == 0 else 'f32'}"].append(t)
        call_ms.append(sum(ms))
    torch.cuda.synchronize(dev)
    wall = time.perf_counter() - wall0
    clocks = sampler.stop()

    total_ms = job_ms(sum(call_ms), world, dev)
    step_bytes = 24 * n
    value = job_gbps(world, step_bytes, args.steps, total_ms)

    # dominant kernel: onesweep_pass (digit passes)
    peak, peak_kind = load_peaks()
    achieved = sum(pass_bytes) / (sum(pass_ms) / 1e3) / 1e9
    traffic = None
    if NCU_TRAFFIC is not None and args.tile_config in (0, 1):  # counters of the default configuration
        traffic = int(NCU_TRAFFIC[1] * n / NCU_TRAFFIC[0])
    # tile configuration 5: each timed pass is the upsweep count plus the chunk-ordered pass
    kname = "chunk_hist_kernel + onesweep_pass" if args.tile_config == 5 else "onesweep_pass"
    roofline = {"bound": "hbm", "kernel": kname, "achieved": round(achieved, 1), "peak": peak,
                "peak_kind": f"{peak_kind} (copy, burst)", "unit": "GB/s", "frac": round(achieved / peak, 4),
                "traffic": traffic, "launches": len(pass_ms),
                "avg_launch_ms": round(sum(pass_ms) / len(pass_ms), 4),
                "share_of_call_time": round(sum(pass_ms) / total_ms, 4) if world == 1 else None,
                "algorithmic_bytes_per_launch": int(sum(pass_bytes) / len(pass_bytes))}
    extra = {"literal_2x_key_bytes_frac_of_8TBs": round(2 * value / world / NOMINAL_HBM_GBS, 4),
             "literal_2x_key_bytes_frac_of_measured": round(2 * value / world / peak, 4),
             "per_call_ms": {k: round(statistics.median(v), 4) for k, v in per_call.items()},
             "wall_s_timed_region": round(wall, 3)}

    # the last step's outputs: sorted int64 and float32 keys, the float32 sortperm
    verified = {"i64_sort": check_sorted(k64, arrays[0]["work"].cpu().numpy()),
                "f32_sort_and_sortperm": check_perm(k32, perm.cpu().numpy().view(np.uint32),
                                                    sorted_out=arrays[1]["work"].cpu().numpy())}
    if not all(verified.values()):
        raise RuntimeError(f"output check failed: {verified}")
    extra["output_checked"] = verified

    # end to end through the public API with host buffers
    e2e = None
    if not args.no_e2e:
        extra["host_link_GBps"] = host_link_bandwidth(torch, dev)
        extra["host_binding"] = host_binding
        # the call a user makes (default options: the library's own path choice), then the
        # plain radix path the device-timed value uses
        e2e = measure_e2e(args, torch, ak, lib, dev, stream, k64, k32, None, n)
        extra["e2e_radix_path"] = measure_e2e(args, torch, ak, lib, dev, stream, k64, k32, None, n,
                                              path=ak.AK_PATH_RADIX)

    # learned-CDF buckets vs plain radix, same run, outputs checked: the int64
    # arrays (the library's own choice for them) and smooth float64 at this n
    if not args.no_learned:
        flush2 = flush
        lvp = {}
        cases = [("i64_uniform_sort", k64, ak.AK_I64, "sort"), ("i64_uniform_sortperm", k64, ak.AK_I64, "sortperm")]
        for dist in ("uniform", "normal"):
            cases.append((f"f64_{dist}_sort", synth.dist_f64(n, dist, seed=10 + synth.F64_DISTS.index(dist)),
                          ak.AK_F64, "sort"))
        del temp
        torch.cuda.empty_cache()
        for name, host, kd, op in cases:
            r = {}
            for pname, path in (("plain", ak.AK_PATH_RADIX), ("learned", ak.AK_PATH_LEARNED)):
                gbs, ms, info, ok = time_sort(torch, ak, dev, stream, flush2, host, kd, {"path": path}, op,
                                              warmup=args.warmup, steps=min(args.steps, 5))
                if not ok:
                    raise RuntimeError(f"output check failed: {name} {pname}")
                r[f"{pname}_GBps"] = round(gbs, 2)
                r[f"{pname}_ms"] = round(ms, 3)
                if pname == "learned":
                    r["learned_path_taken"] = PATH_NAMES.get(info["path"])
            r["output_checked"] = True
            r["learned_over_plain"] = round(r["learned_GBps"] / r["plain_GBps"], 3)
            lvp[name] = r
        extra["learned_vs_plain"] = lvp
        # the MLP residual on a heavy-tailed distribution that the 64 knots underfit
        # (Pareto, alpha 1.5): piecewise-linear CDF alone vs trained residual
        par = (1.0 - synth.u01_f64(44, n)) ** (-1.0 / 1.5)
        mlp = {}
        for label, steps in (("pl_only", -1), ("mlp_16_steps", 0), ("mlp_64_steps", 64)):
            gbs, ms, info, ok = time_sort(torch, ak, dev, stream, flush2, par, ak.AK_F64,
                                          {"path": ak.AK_PATH_LEARNED, "train_steps": steps}, "sort",
                                          warmup=args.warmup, steps=min(args.steps, 5))
            if not ok:
                raise RuntimeError(f"output check failed: pareto {label}")
            mlp[label] = {"GBps": round(gbs, 2), "ms": round(ms, 3), "max_bucket": info["max_bucket"],
                          "buckets": info["buckets"], "path": PATH_NAMES.get(info["path"]),
                          "loss_before": info["loss_before"], "loss_after": info["loss_after"],
                          "mlp_used": info["mlp_used"], "sample_max_pl": info["sample_max_pl"],
                          "sample_max_mlp": info["sample_max_mlp"]}
        extra["mlp_residual_pareto"] = mlp
        del par
        temp = None


    cpu = None
    if world == 1 and not args.no_cpu:
        threads = len(os.sched_getaffinity(0)) or 1
        sample = min(n, 1 << 24)
        rate, dt = cpu_oracle_rate(k64, k32, sample, threads)
        cpu = {"value": round(rate, 4), "unit": "GB/s", "cores": threads, "kind": "oracle",
               "sample": f"first {sample:,} keys of each array, sortperm + sort each (threaded merge sort), {dt:.1f} s"}

    def pass_launches(op, i):
        w = 8 if i == 0 else 4
        if op == "sortperm" and w == 8 and args.tile_config in (0, 1) and n <= (1 << 30):
            return 2 * w + w // 2  # plain and packing variant per pass, packed-word variant in the upper half
        return w * (2 if args.tile_config == 5 else 1)  # tile configuration 5: upsweep + pass
    launches_per_step = sum(3 + pass_launches(op, i) for op, i in calls)
    if rank == 0:
        line = base_line(args, world, cfg)
        line.update({"value": round(value, 3), "ms_per_step": round(total_ms / args.steps, 4),
                     "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "clocks": clocks,
                     "gpu_launches": launches_per_step * args.steps, "extra": extra})
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def host_link_bandwidth(torch, dev, nbytes=1 << 30):
    """Plain pinned-host <-> device copy bandwidth (GB/s) of nbytes each way, the
    ceiling of the e2e leg's copies on this machine."""
    h = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    d = torch.empty(nbytes, dtype=torch.uint8, device=dev)
    res = {}
    for name, (dst, src) in (("h2d", (d, h)), ("d2h", (h, d))):
        dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(3):
            dst.copy_(src, non_blocking=True)
        e1.record()
        torch.cuda.synchronize(dev)
        res[name] = round(3 * nbytes / (e0.elapsed_time(e1) / 1e3) / 1e9, 1)
    del h, d
    torch.cuda.empty_cache()
    return res


def measure_e2e(args, torch, ak, lib, dev, stream, k64, k32, temp, n, path=None):
    """Same four calls from pinned host buffers: H2D keys, sortperm, sort, D2H perm + sorted keys,
    through `path` (None: the library's own choice, as a caller's plain call gets).  Copies run
    on their own streams and the device buffers alternate between two sets by step, so that
    the next step's uploads and this step's downloads overlap the sorts (events order every
    buffer reuse).  The last step's outputs are checked on the host."""
    del temp
    opts = None
    if path is not None:
        opts = ak.Options()
        opts.path = path
    oref = ctypes.byref(opts) if opts is not None else None
    temp = ak.workspace(max(ak.temp_bytes(op, n, kd, options=opts) for op in (ak.AK_OP_SORT, ak.AK_OP_SORTPERM)
                            for kd in (ak.AK_I64, ak.AK_F32)), dev)
    hosts = [torch.from_numpy(k64).pin_memory(), torch.from_numpy(k32).pin_memory()]
    outs_k = [torch.empty_like(h).pin_memory() for h in hosts]
    outs_p = [torch.empty(n, dtype=torch.int32).pin_memory() for _ in hosts]
    # two sets of device buffers, by step parity
    dk = [[torch.empty(h.shape, dtype=h.dtype, device=dev) for h in hosts] for _ in range(2)]
    dp = [[torch.empty(n, dtype=torch.int32, device=dev) for _ in hosts] for _ in range(2)]
    kds = [ak.AK_I64, ak.AK_F32]
    up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    ev = lambda: torch.cuda.Event()  # noqa: E731
    freed = [[None, None], [None, None]]  # per set and array: its previous results have left the device
    host_out_free = [None, None]  # per array: the previous step's download to the host buffers is done
    parity = [0]

    def step():
        b = parity[0]
        parity[0] ^= 1
        loaded = []
        for i in range(2):  # both uploads queue at once on the upload stream
            with torch.cuda.stream(up):
                if freed[b][i] is not None:
                    up.wait_event(freed[b][i])
                dk[b][i].copy_(hosts[i], non_blocking=True)
                e = ev()
                e.record(up)
                loaded.append(e)
        for i in range(2):
            stream.wait_event(loaded[i])
            rc = lib.ak_sortperm(dk[b][i].data_ptr(), dp[b][i].data_ptr(), n, kds[i], 0, temp.data_ptr(),
                                 temp.numel(), stream.cuda_stream, oref)
            perm_done = ev()
            perm_done.record(stream)
            rc |= lib.ak_sort(dk[b][i].data_ptr(), n, kds[i], 0, temp.data_ptr(), temp.numel(), stream.cuda_stream,
                              oref)
            if rc:
                raise ak.AkError(rc, "e2e")
            sort_done = ev()
            sort_done.record(stream)
            with torch.cuda.stream(down):  # downloads stay in order on one stream: host buffers reused safely
                down.wait_event(perm_done)
                outs_p[i].copy_(dp[b][i], non_blocking=True)
                down.wait_event(sort_done)
                outs_k[i].copy_(dk[b][i], non_blocking=True)
                f = ev()
                f.record(down)
                freed[b][i] = f
                host_out_free[i] = f

    for _ in range(max(1, args.warmup)):
        step()
    torch.cuda.synchronize(dev)
    steps = max(1, min(args.steps, 3))
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(up)
    for _ in range(steps):
        step()
    stream.wait_event(host_out_free[0])
    stream.wait_event(host_out_free[1])
    e1.record(stream)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / steps
    h2d = sum(h.numel() * h.element_size() for h in hosts)
    d2h = h2d + 2 * 4 * n
    # the last step's results, read back to the host: each sortperm is THE stable one and the
    # sorted keys are keys[perm]
    ok = all(check_perm(src, outs_p[i].numpy().view(np.uint32), sorted_out=outs_k[i].numpy())
             for i, src in enumerate((k64, k32)))
    if not ok:
        raise RuntimeError("e2e output check failed")
    paths = {}
    for i, kd in enumerate(kds):
        dk[0][i].copy_(hosts[i], non_blocking=True)
        lib.ak_sort(dk[0][i].data_ptr(), n, kd, 0, temp.data_ptr(), temp.numel(), stream.cuda_stream, oref)
        paths["i64" if i == 0 else "f32"] = PATH_NAMES.get(ak.ak_last_info(temp)["path"])
    del dk, dp, temp
    torch.cuda.empty_cache()
    return {"value": round(24 * n / (ms / 1e3) / 1e9, 3), "unit": "GB/s", "h2d_bytes_per_step": h2d,
            "d2h_bytes_per_step": d2h, "ms_per_step": round(ms, 3), "steps": steps, "paths": paths,
            "output_checked": True, "copies": "upload / download streams overlapping the sorts"}


# ------------------------------------------------------------ other workloads
def _timed(torch, stream, flush, restore, call, warmup, steps):
    """Median device time (ms) of call(); restore() and an L2 flush run before
    every call, outside the events."""
    for _ in range(warmup):
        restore()
        call()
    ms = []
    for _ in range(steps):
        restore()
        flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        call()
        e1.record(stream)
        torch.cuda.synchronize()
        ms.append(e0.elapsed_time(e1))
    return statistics.median(ms)


def _line(args, workload, value, extra):
    line = {"metric": METRIC, "unit": "GB/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "data": "synthetic (seeded splitmix64)",
            "config": {"workload": workload}, "value": round(value, 3)}
    line.update(extra)
    print(json.dumps(line), flush=True)


def run_workload(args):
    import torch

    import paper_2507_16710_gb300 as ak
    import synth
    dev = torch.device("cuda", 0)
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    peak, _ = load_peaks()
    W, K = args.warmup, args.steps

    def sort_gbs(host, kd, opts, op="sort", vals=None, order="ascending"):
        """Key GB/s of one operation on `host` keys (device-timed; output checked)."""
        gbs, ms, info, ok = time_sort(torch, ak, dev, stream, flush, host, kd, opts, op, vals, order, W, K)
        if not ok:
            raise RuntimeError(f"output check failed: {op} {host.dtype} {opts}")
        return gbs, ms, info

    if args.workload == "c1":
        keys = synth.uniform_u32(1 << 20, seed=1)
        res = {}
        for name, opts in (("auto", None), ("radix", {"path": ak.AK_PATH_RADIX}), ("block", {"path": ak.AK_PATH_BLOCK})):
            gbs, ms, info = sort_gbs(keys, ak.AK_U32, opts)
            res[name] = {"GBps": round(gbs, 2), "ms": round(ms, 4), "path": info["path"], "output_checked": True}
        best = max(v["GBps"] for v in res.values())
        _line(args, "1,048,576 u32 uniform, ak_sort ascending (L2-resident)", best,
              {"dtype": "u32", "results": res})
    elif args.workload == "c3":
        n = args.n if args.n != FULL_N else 100_000_000
        res, tot_b, tot_l, tot_p = {}, 0, 0.0, 0.0
        for i, dist in enumerate(synth.F64_DISTS):
            keys = synth.dist_f64(n, dist, seed=10 + i)
            gp, mp, _ = sort_gbs(keys, ak.AK_F64, {"path": ak.AK_PATH_RADIX})
            gl, ml, info = sort_gbs(keys, ak.AK_F64, {"path": ak.AK_PATH_LEARNED})
            res[dist] = {"plain_GBps": round(gp, 2), "learned_GBps": round(gl, 2), "plain_ms": round(mp, 3),
                         "learned_ms": round(ml, 3), "learned_path_taken": info["path"] == ak.AK_PATH_LEARNED,
                         "overfull_frac": round(info["overfull_keys"] / n, 4),
                         "loss_before": info["loss_before"], "loss_after": info["loss_after"]}
            tot_b += keys.nbytes
            tot_l += ml
            tot_p += mp
        big = {}
        for i, dist in enumerate(("uniform", "normal") if args.n == FULL_N else ()):  # --n: that size only
            keys = synth.dist_f64(FULL_N, dist, seed=10 + synth.F64_DISTS.index(dist))
            gp, mp, _ = sort_gbs(keys, ak.AK_F64, {"path": ak.AK_PATH_RADIX})
            gl, ml, info = sort_gbs(keys, ak.AK_F64, {"path": ak.AK_PATH_LEARNED})
            big[dist] = {"plain_GBps": round(gp, 2), "learned_GBps": round(gl, 2),
                         "learned_path_taken": info["path"] == ak.AK_PATH_LEARNED}
            del keys
        value = tot_b / (tot_l / 1e3) / 1e9
        _line(args, f"{n:,} float64 x 6 distributions, ak_sort ascending: learned-CDF bucketing vs plain radix",
              value, {"dtype": "u64 radix keys (float64)", "learned_GBps_all": round(value, 3),
                      "plain_GBps_all": round(tot_b / (tot_p / 1e3) / 1e9, 3), "results": res,
                      "smooth_268M": big, "literal_2x_key_bytes_frac_of_8TBs": round(2 * value / NOMINAL_HBM_GBS, 4)})
    elif args.workload == "c4":
        off = synth.lognormal_segments(args.segments, seed=20)
        n = int(off[-1])
        keys = synth.uniform_u32(n, seed=21)
        pristine = torch.from_numpy(keys.view(np.int32)).to(dev)
        work = torch.empty_like(pristine)
        o = torch.from_numpy(off).to(dev)
        temp = ak.workspace(ak.temp_bytes(ak.AK_OP_SORT_SEGMENTED, n, ak.AK_U32, nseg=off.size - 1), dev)
        s = torch.cuda.Stream()
        work.copy_(pristine)
        ak.ak_sort_segmented(work, o, temp=temp, stream=s, unsigned=True)
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=s):
            ak.ak_sort_segmented(work, o, temp=temp, stream=s, unsigned=True)

        def restore():
            work.copy_(pristine)

        def call():
            g.replay()

        ms = _timed(torch, torch.cuda.current_stream(dev), flush, restore, call, W, K)
        gbs = keys.nbytes / (ms / 1e3) / 1e9
        # output check: every segment is its own sorted multiset ((segment, key) as one u64)
        got = work.cpu().numpy().view(np.uint32)
        seg = np.repeat(np.arange(off.size - 1, dtype=np.uint64), np.diff(off))
        comb = (seg << np.uint64(32)) | got.astype(np.uint64)
        ok = bool(np.all(comb[1:] >= comb[:-1])) and _bits_hash(got) == _bits_hash(keys)
        if not ok or ak.ak_status_check(temp) != 0:
            raise RuntimeError("segmented output check failed")
        _line(args, f"{args.segments:,} segments, lognormal lengths (median 2,048), {n:,} u32 keys, one persistent launch "
              "replayed from a CUDA graph", gbs,
              {"dtype": "u32", "ms": round(ms, 4), "keys": n, "output_checked": True,
               "roofline_2x_bytes_frac_of_measured": round(2 * gbs / peak, 4)})
    elif args.workload == "c5":
        n = args.n if args.n != FULL_N else 1 << 30
        keys = synth.zipf_mix_u32(n, seed=30, workers=os.cpu_count() or 1)
        vals = np.arange(n, dtype=np.uint32)
        gp, mp, _ = sort_gbs(keys, ak.AK_U32, {"path": ak.AK_PATH_RADIX}, op="pairs", vals=vals, order="descending")
        gl, ml, info = sort_gbs(keys, ak.AK_U32, {"path": ak.AK_PATH_LEARNED}, op="pairs", vals=vals,
                                order="descending")
        _line(args, f"{n:,} u32 keys (Zipf s=1.1 over 2^24 + uniform, 50/50) with u32 values, descending pairs: "
              "learned vs plain", max(gp, gl),
              {"dtype": "u32", "plain_GBps": round(gp, 3), "learned_GBps": round(gl, 3), "plain_ms": round(mp, 3),
               "learned_ms": round(ml, 3), "learned_path_taken": info["path"] == ak.AK_PATH_LEARNED,
               "overfull_frac": round(info["overfull_keys"] / n, 4),
               "keys_plus_values_GBps_plain": round(2 * gp, 3), "keys_plus_values_GBps_learned": round(2 * gl, 3)})
    elif args.workload == "searchsorted":
        run_searchsorted(args, torch, ak, synth, dev, stream, flush, peak)
    elif args.workload == "accumulate":
        run_accumulate(args, torch, ak, synth, dev, stream, flush, peak)
    elif args.workload == "int128":
        run_int128(args, torch, ak, synth, dev, stream, flush, peak)


def _i128_order_ok(lo: np.ndarray, hi: np.ndarray) -> bool:
    """Signed 128-bit keys (low, high words) in non-decreasing order."""
    h = hi.view(np.int64)
    return bool(np.all((h[1:] > h[:-1]) | ((h[1:] == h[:-1]) & (lo[1:] >= lo[:-1]))))


def _i128_hash(lo: np.ndarray, hi: np.ndarray) -> int:
    """Order-independent hash of a multiset of 128-bit keys."""
    with np.errstate(over="ignore"):
        z = lo ^ ((hi ^ (hi >> np.uint64(29))) * np.uint64(0xBF58476D1CE4E5B9))
        z = (z ^ (z >> np.uint64(31))) * np.uint64(0x94D049BB133111EB)
        z ^= z >> np.uint64(32)
        return int(z.sum(dtype=np.uint64))


def run_int128(args, torch, ak, synth, dev, stream, flush, peak):
    """Int128 keys (the widest type of the paper's local-sort benchmarks):
    268,435,456 signed 128-bit keys over all bit patterns (4 GiB), stable
    ak_sort in place and ak_sortperm, through the radix path (16 digit
    passes).  value = key bytes sorted per second over both calls."""
    n = args.n
    lo = synth.splitmix64(50, n)
    hi = synth.splitmix64(51, n)
    host = np.empty((n, 2), dtype=np.uint64)
    host[:, 0], host[:, 1] = lo, hi
    pristine = torch.from_numpy(host.view(np.int64)).to(dev)
    work = torch.empty_like(pristine)
    perm = torch.empty(n, dtype=torch.int32, device=dev)
    lib = ak.load()
    tb = max(ak.temp_bytes(op, n, ak.AK_I128) for op in (ak.AK_OP_SORT, ak.AK_OP_SORTPERM))
    temp = ak.workspace(tb, dev)
    pass_ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * ak.AK_MAX_PASSES)]
    for e in pass_ev:
        e.record(stream)
    opts = ak.Options()
    ev_arr = (ctypes.c_void_p * len(pass_ev))(*[e.cuda_event for e in pass_ev])
    opts.pass_events = ctypes.cast(ev_arr, ctypes.c_void_p)
    res, pass_ms, pass_bytes = {}, [], []
    for op in ("sort", "sortperm"):
        def call(op=op):
            if op == "sort":
                rc = lib.ak_sort(work.data_ptr(), n, ak.AK_I128, 0, temp.data_ptr(), temp.numel(), stream.cuda_stream,
                                 ctypes.byref(opts))
            else:
                rc = lib.ak_sortperm(pristine.data_ptr(), perm.data_ptr(), n, ak.AK_I128, 0, temp.data_ptr(),
                                     temp.numel(), stream.cuda_stream, ctypes.byref(opts))
            if rc:
                raise ak.AkError(rc, op)

        ms = _timed(torch, stream, flush, lambda: work.copy_(pristine), call, args.warmup, args.steps)
        npass = ak.ak_last_info(temp)["radix_passes"]
        pb = onesweep_bytes(op, n, 16, 16)
        for p in range(16):  # the last timed call's passes
            pass_ms.append(pass_ev[2 * p].elapsed_time(pass_ev[2 * p + 1]))
            pass_bytes.append(pb[p] if npass == 16 else 0)
        res[op] = {"ms": round(ms, 3), "GBps": round(n * 16 / (ms / 1e3) / 1e9, 2), "digit_passes": npass}
        if op == "sort":  # the last timed sort's output, before the sortperm timing restores the keys
            out = work.cpu().numpy().view(np.uint64)
            ok_sort = _i128_order_ok(out[:, 0], out[:, 1]) and _i128_hash(out[:, 0], out[:, 1]) == _i128_hash(lo, hi)
            del out
    p = perm.cpu().numpy().view(np.uint32).astype(np.int64)
    ok_perm = bool(np.all(np.bincount(p, minlength=n) == 1)) and _i128_order_ok(lo[p], hi[p])
    if not (ok_sort and ok_perm):
        raise RuntimeError(f"int128 output check failed: sort {ok_sort} sortperm {ok_perm}")
    total_ms = res["sort"]["ms"] + res["sortperm"]["ms"]
    value = 2 * n * 16 / (total_ms / 1e3) / 1e9
    achieved = sum(pass_bytes) / (sum(pass_ms) / 1e3) / 1e9
    _line(args, f"{n:,} Int128 keys over all bit patterns (4 GiB), ak_sort + ak_sortperm ascending, radix path",
          value, {"dtype": "i128", "results": res, "output_checked": True,
                  "roofline": {"bound": "hbm", "kernel": "onesweep_pass<u128>", "achieved": round(achieved, 1),
                               "peak": peak, "unit": "GB/s", "frac": round(achieved / peak, 4), "traffic": None,
                               "launches": len(pass_ms)},
                  "literal_2x_key_bytes_frac_of_measured": round(2 * value / peak, 4)})


def check_scan_i64(x, out):
    """Inclusive + of int64 keys: out[0] = x[0] and out[i] - out[i-1] = x[i],
    both in wrapping int64 arithmetic (exact)."""
    with np.errstate(over="ignore"):
        return bool(out[0] == x[0] and np.array_equal(out[1:] - out[:-1], x[1:]))


def check_scan_f64(x, out):
    """Inclusive + of float64 keys: consecutive outputs differ by the key up to
    the sum of both outputs' rounding bounds, gamma_D * sum |x_j| over each
    prefix with D = 8 + 2 ceil(n / 2^18) + 84 the depth of the scan's summation
    tree (8 keys per lane, 2^18 keys per warp range), plus an ulp of each output
    (a dropped, repeated or misplaced key moves the difference by the key)."""
    u = np.finfo(np.float64).eps / 2
    depth = 8 + 2 * -(-x.size // (32768 * 8)) + 84
    bound = (depth * u / (1 - depth * u)) * np.cumsum(np.abs(x)) + np.spacing(np.abs(out))
    ok0 = abs(out[0] - x[0]) <= bound[0]
    d = np.abs((out[1:] - out[:-1]) - x[1:])
    return bool(ok0 and np.all(d <= bound[1:] + bound[:-1]))


def run_accumulate(args, torch, ak, synth, dev, stream, flush, peak):
    """Inclusive + scan (Sec. II-B accumulate) of 268,435,456 int64 keys (2 GiB
    in, 2 GiB out; --n another size) and of as many float64 keys ~ N(0, 1).
    value = algorithmic bytes (read once, written once) per second of the
    whole scan, its three launches together (the HBM roofline's own units).
    Both outputs of the last timed call are checked on the host."""
    import oracle
    n = args.n if args.n != FULL_N else 1 << 28
    xh = synth.uniform_i64(n, seed=117)
    xf = synth.dist_f64(n, "normal", seed=118)
    lib = ak.load()
    res = {}
    checked = {}
    for name, kd, host, check in (("i64_add", ak.AK_I64, xh, check_scan_i64),
                                  ("f64_add", ak.AK_F64, xf, check_scan_f64)):
        x = torch.from_numpy(host).to(dev)
        out = torch.empty_like(x)
        temp = ak.workspace(ak.accumulate_temp_bytes(n, kd), dev)

        def call(kd=kd, temp=temp):
            rc = lib.ak_accumulate(x.data_ptr(), out.data_ptr(), n, kd, 0, 1, None, temp.data_ptr(), temp.numel(),
                                   stream.cuda_stream, None)
            if rc:
                raise ak.AkError(rc, "ak_accumulate")

        ms = _timed(torch, stream, flush, lambda: None, call, args.warmup, args.steps)
        if ak.ak_status_check(temp) != 0:
            raise RuntimeError("ak_accumulate: device status not clean")
        checked[name] = check(host, out.cpu().numpy())
        if not checked[name]:
            raise RuntimeError(f"output check failed: accumulate {name}")
        res[name] = {"ms": round(ms, 4), "GBps": round(2 * n * 8 / (ms / 1e3) / 1e9, 1)}
        del x, out, temp
    gbs = res["i64_add"]["GBps"]
    cpu = None
    if not args.no_cpu:
        sample = 1 << 26
        t0 = time.perf_counter()
        oracle.accumulate(xh[:sample], "add")
        dt = time.perf_counter() - t0
        cpu = {"value": round(2 * sample * 8 / dt / 1e9, 3), "unit": "GB/s", "cores": 1, "kind": "oracle",
               "sample": f"inclusive + over the first {sample:,} int64 keys"}
    _line(args, f"{n:,} int64 keys uniform over all bit patterns, inclusive + scan (ak_accumulate), out of place; "
                f"{n:,} float64 keys ~ N(0, 1) alongside",
          gbs, {"metric": "accumulate GB/s read + written (device-timed, 1 GB300)", "dtype": "i64",
                "results": res, "output_checked": checked,
                "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s",
                             "frac": round(gbs / peak, 4),
                             # DRAM bytes of one int64 call (reduce + carry + scan launches),
                             # scaled from the 2^28-key launch list to this n
                             "traffic": int(ACC_NCU_TRAFFIC[1] * n / ACC_NCU_TRAFFIC[0]),
                             "traffic_per": "call (3 launches; the input is read twice by design)"},
                "cpu_baseline": cpu})


def run_searchsorted(args, torch, ak, synth, dev, stream, flush, peak):
    """Batched binary search (Sec. II-B): 2^26 float64 queries against 2^27
    ascending float64 keys (1 GiB, 25% equal neighbours), once with queries
    uniform over the keys' range (independent random searches) and once with
    the queries themselves ascending.  value = queries per second over the
    first and last searches of the random queries."""
    import oracle
    n, m = 1 << 27, 1 << 26
    v = synth.ascending_f64(n, seed=40)
    xr = synth.u01_f64(92, m) * v[-1]
    xs = synth.ascending_f64(m, seed=93)
    xs *= v[-1] / xs[-1]
    tv = torch.from_numpy(v).to(dev)
    out = torch.empty(m, dtype=torch.int64, device=dev)
    lib = ak.load()
    res, ms_random = {}, 0.0
    for qname, xh in (("random", xr), ("ascending", xs)):
        tx = torch.from_numpy(xh).to(dev)
        for side in ("first", "last"):
            f = lib.ak_searchsortedfirst if side == "first" else lib.ak_searchsortedlast

            def call(f=f, tx=tx):
                rc = f(tv.data_ptr(), n, tx.data_ptr(), m, ak.AK_F64, 0, out.data_ptr(), stream.cuda_stream)
                if rc:
                    raise ak.AkError(rc, "searchsorted")

            ms = _timed(torch, stream, flush, lambda: None, call, args.warmup, args.steps)
            res[f"{qname}_{side}"] = {"ms": round(ms, 4), "Gq_per_s": round(m / (ms / 1e3) / 1e9, 3)}
            if qname == "random":
                ms_random += ms
        del tx
    value = 2 * m / (ms_random / 1e3) / 1e9
    # algorithmic bytes: each query read (8 B) and its index written (8 B)
    achieved = 2 * m * 16 / (ms_random / 1e3) / 1e9
    # ascending queries: tiles in the keys' order read v once through the
    # shared window, so the bound is HBM: keys + queries read, indices written
    ms_asc = res["ascending_first"]["ms"] + res["ascending_last"]["ms"]
    asc_gbs = 2 * (n * 8 + m * 8 + m * 8) / (ms_asc / 1e3) / 1e9
    asc = {"Gq_per_s": round(2 * m / (ms_asc / 1e3) / 1e9, 3), "achieved_GBps": round(asc_gbs, 1),
           "frac_of_measured_copy": round(asc_gbs / peak, 4),
           "bytes_per_call": "8 n (keys) + 8 m (queries) + 8 m (indices)"}
    table = 2048  # pivot keys per CTA for 8-byte keys
    steps = int(np.ceil(np.log2(n / (table + 1))))
    cpu = None
    if not args.no_cpu:
        sample = 1 << 20
        t0 = time.perf_counter()
        oracle.searchsorted(v, xr[:sample], "first")
        oracle.searchsorted(v, xr[:sample], "last")
        dt = time.perf_counter() - t0
        cpu = {"value": round(2 * sample / dt / 1e9, 5), "unit": "G queries/s", "cores": 1, "kind": "oracle",
               "sample": f"first and last of the first {sample:,} random queries against all {n:,} keys"}
    _line(args, f"{m:,} float64 queries against {n:,} ascending float64 keys (1 GiB), searchsortedfirst + "
          "searchsortedlast", value,
          {"metric": "searchsorted queries/s (device-timed, 1 GB300)", "unit": "G queries/s", "dtype": "f64",
           "results": res,
           "roofline": {"bound": "hbm", "achieved": round(achieved, 2), "peak": peak, "unit": "GB/s",
                        "frac": round(achieved / peak, 4), "traffic": None,
                        "note": f"latency bound: after the shared-memory table each query makes {steps} "
                                "dependent loads into the 1 GiB key array; bytes counted are the query "
                                "read and the index write (16 B per query)"},
           "ascending_queries": asc,
           "cpu_baseline": cpu})


def main():
    args = parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        run_reference(args)
    elif args.workload != "c2":
        run_workload(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
