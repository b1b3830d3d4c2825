#!/usr/bin/env python
"""Benchmark: work-efficient triangle-inequality K-means (KPynq) on GB300.

One step = one whole K-means job on the large anisotropic workload
(N=1,048,576 points, D=64, K=256 centroids, G=26 groups, at most 50 iterations
or tol 1e-4): restart from C0 (kmeans_reset), then kmeans_fit -- the dense
iteration 0, the filtered iterations, and the final assignment -- through the
C ABI, with X resident in HBM.  Metric: points x iterations per second.

The JSON line also carries: plain GPU Lloyd on the same GPU and inputs, the
fraction of distance evaluations the filters skipped, the roofline of the
dominant kernel (from a profiled pass that brackets every launch with CUDA
events on the library's stream), the FP64 oracle timed on the host cores, an
end-to-end number through the C ABI with host buffers, and SM clocks sampled
during the timed region.

``--impl reference`` times the FP64 CPU oracle (brute-force Lloyd) instead.
Multi-GPU (torchrun): every rank runs its own replica problem (weak scaling,
no collective on the data path); the step time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "points*iters/s (filtered K-means, exact labels)"
UNIT = "points*iters/s"
L2_BYTES = 129 * 1024 * 1024
SMS, FP32_LANES, SM_MAX_GHZ = 152, 128, 2.07
# the distance loop issues one FSUB and one FFMA per (point, centroid, dim):
# 3 flops in 2 issue slots of a FP32 lane
ALU_PEAK_TFLOPS = SMS * FP32_LANES * SM_MAX_GHZ * 1.5 / 1e3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--lloyd-steps", type=int, default=3)
    ap.add_argument("--e2e-steps", type=int, default=5)
    ap.add_argument("--profile-steps", type=int, default=3)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-forms", action="store_true",
                    help="skip the sub-records of the other workloads (high-dim 4M, batched 512, proposal 8M)")
    ap.add_argument("--form-steps", type=int, default=2, help="timed steps of each sub-record")
    ap.add_argument("--form-warmup", type=int, default=1, help="warm-up steps of each sub-record")
    ap.add_argument("--energy-seconds", type=float, default=5.0,
                    help="length of the fit loop over which the board's energy counter is read (0: skip)")
    ap.add_argument("--workload", default="aniso1m", choices=["aniso1m", "highdim4m", "batched", "gsweep", "proposal"],
                    help="aniso1m: the 1M-point anisotropic job (default line); highdim4m: 4M points, "
                         "D=128, K=1024, stored as bfloat16; batched: 512 independent problems of uneven "
                         "N, D, K fitted by one graph launch; gsweep: the 1M job at G in {1, K/20, K/10, "
                         "K/5, K} (throughput and skip fraction per G); proposal: the 8.4M-point family "
                         "(D=32, K=4096, G=410), fits with and without the learned group proposal")
    ap.add_argument("--problems", type=int, default=512, help="batched workload: number of problems")
    ap.add_argument("--grouping", default="clustered", choices=["contiguous", "clustered"],
                    help="centroid groups of the filtered fits: groups of nearby centroids (Lloyd over the "
                         "initial centroids; the default) or contiguous index ranges")
    ap.add_argument("--profile-only", action="store_true",
                    help="run only the profiled pass (every kernel launched eagerly, timed with CUDA "
                         "events) and print its breakdown: the command the ncu launch list is taken on")
    ap.add_argument("--n", type=int, default=None, help="points (default: the full workload)")
    ap.add_argument("--train-steps", type=int, default=3000,
                    help="proposal workload: Adam steps (8192 rows each) of the GPU trainer")
    ap.add_argument("--train-n", type=int, default=1 << 20,
                    help="proposal workload: points per training seed (8 seeds)")
    return ap.parse_args()


# ---------------------------------------------------------------------------
# multi-rank plumbing (timing only; the data path has no collective)
# ---------------------------------------------------------------------------
def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def aggregate(local_ms: float, local_units: float, world_size: int, backend_device=None):
    """Max step time over ranks and the units all ranks processed.  Uses
    torch.distributed when world_size > 1 (any backend)."""
    if world_size == 1:
        return local_ms, local_units
    import torch
    import torch.distributed as dist
    t = torch.tensor([local_ms], dtype=torch.float64, device=backend_device)
    u = torch.tensor([local_units], dtype=torch.float64, device=backend_device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.all_reduce(u, op=dist.ReduceOp.SUM)
    return float(t.item()), float(u.item())


def barrier(world_size: int):
    if world_size > 1:
        import torch.distributed as dist
        dist.barrier()


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str | None):
        self.gpu_id = gpu_id
        self.proc = None
        # raw samples in a scratch file (KPYNQ_CLOCKS_DIR, else the system's
        # temporary directory); the JSON line carries their summary
        d = os.environ.get("KPYNQ_CLOCKS_DIR") or tempfile.gettempdir()
        self.path = os.path.join(d, f"kpynq_clocks_{os.getpid()}_{id(self):x}.csv")

    def __enter__(self):
        os.makedirs(os.path.dirname(self.path), exist_ok=True)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200"]
        if self.gpu_id:
            cmd[1:1] = ["-i", self.gpu_id]
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.f.close()

    def summary(self) -> dict:
        if not self.proc or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, pw, reasons = [], [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            try:
                pw.append(float(f[3]))
            except ValueError:
                pass
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "samples": len(sm),
                "reasons": sorted(reasons), "power_w_mean": statistics.mean(pw) if pw else None}


def energy_mj(gpu_id: str | None) -> float | None:
    """The board's cumulative energy counter (mJ since the driver loaded):
    NVML's total-energy query (read-only), else nvidia-smi's."""
    import ctypes
    try:
        nv = ctypes.CDLL("libnvidia-ml.so.1")
        if nv.nvmlInit_v2() == 0:
            h = ctypes.c_void_p()
            rc = (nv.nvmlDeviceGetHandleByUUID(gpu_id.encode(), ctypes.byref(h)) if gpu_id
                  else nv.nvmlDeviceGetHandleByIndex_v2(0, ctypes.byref(h)))
            e = ctypes.c_ulonglong(0)
            if rc == 0 and nv.nvmlDeviceGetTotalEnergyConsumption(h, ctypes.byref(e)) == 0 and e.value > 0:
                return float(e.value)
    except (OSError, AttributeError):
        pass
    cmd = ["nvidia-smi", "--query-gpu=total_energy_consumption", "--format=csv,noheader,nounits"]
    if gpu_id:
        cmd[1:1] = ["-i", gpu_id]
    try:
        out = subprocess.run(cmd, capture_output=True, text=True, timeout=10).stdout.strip().splitlines()
        return float(out[0])
    except (OSError, ValueError, IndexError, subprocess.TimeoutExpired):
        return None


def energy_loop(run_one, units_per_call: float, seconds: float, gpu_id: str | None) -> dict | None:
    """points*iters per joule over a loop of calls lasting at least `seconds`,
    from the difference of the cumulative energy counter across the loop."""
    import torch
    torch.cuda.synchronize()
    e0 = energy_mj(gpu_id)
    if e0 is None:
        return None
    t0 = time.perf_counter()
    calls = 0
    while True:
        run_one()
        calls += 1
        if calls % 8 == 0:
            torch.cuda.synchronize()
            if time.perf_counter() - t0 >= seconds:
                break
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    e1 = energy_mj(gpu_id)
    if e1 is None or e1 <= e0:
        return None
    joules = (e1 - e0) / 1e3
    return {"value": units_per_call * calls / joules, "unit": "points*iters/J", "joules": joules,
            "seconds": dt, "calls": calls, "mean_power_w": joules / dt,
            "source": "NVML total energy consumption (cumulative board counter, read-only) across the loop"}


def energy_of(value: float, clocks: dict) -> dict | None:
    """points*iters per joule from the mean board power sampled during the timed steps."""
    w = clocks.get("power_w_mean")
    if not w:
        return None
    return {"value": value / w, "unit": "points*iters/J", "mean_power_w": w, "samples": clocks.get("samples"),
            "source": "nvidia-smi power.draw every 200 ms during the timed steps (whole board)"}


def gpu_uuid():
    try:
        import torch
        u = torch.cuda.get_device_properties(torch.cuda.current_device()).uuid
        s = str(u)
        return s if s.startswith("GPU-") else f"GPU-{s}"
    except Exception:
        return None


def measured_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6800.0), d.get("bf16_tflops", 1900.0), "measured"
    return 6800.0, 1900.0, "fallback"


# ---------------------------------------------------------------------------
# CPU baseline: the FP64 oracle on the host cores
# ---------------------------------------------------------------------------
def cpu_baseline(w, n_sample: int, iters: int) -> dict:
    import oracle
    oracle.build()
    Xs = w.X[:n_sample].astype("float64")
    dt = oracle_iterations(Xs, w.C0.astype("float64"), iters)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    return {"value": n_sample * iters / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"brute-force FP64 Lloyd (oracle O1: assign + update), first {n_sample} of {w.N} "
                      f"points, {iters} iterations, K={w.K}, D={w.D}; {dt:.2f} s wall"}


def oracle_iterations(Xs, C, iters: int) -> float:
    """Wall time of `iters` oracle Lloyd iterations (assign + update)."""
    import oracle
    t0 = time.perf_counter()
    prev = None
    for _ in range(iters):
        lab, _, _, _ = oracle.lloyd_assign(Xs, C, prev)
        C, _, _ = oracle.lloyd_update(Xs, lab, C)
        prev = lab
    return time.perf_counter() - t0


# ---------------------------------------------------------------------------
# roofline bookkeeping: algorithmic bytes / flops per launch of each kernel
# ---------------------------------------------------------------------------
def algorithmic(kind: str, w, stats: list, launches: int) -> list[tuple[str, float]]:
    """[(bound, units per launch)] from the per-iteration counters: bytes for
    "hbm", flops for "alu" (3 per point x centroid x dimension: the FSUB and
    FFMA of a direct squared distance) and for "tensor" (the BF16x3 dense
    pass: three bfloat16 products of 2 flops per point x centroid x
    dimension).  The caller keeps the bound with the larger fraction of its
    peak."""
    N, D, K, G = w.N, w.D, w.K, w.G
    Gp = (G + 3) // 4 * 4
    # the filtered iterations proper: the survivor kernel does no work in
    # iterations that switched to the dense pass (path != 0)
    filt = [s for s in stats if s["iter"] > 0 and s["path"] == 0]
    dense_fp32 = [s for s in stats if s["path"] == 1]
    dense_tc = [s for s in stats if s["path"] == 2]
    mean = lambda key, rows: sum(s[key] for s in rows) / max(1, len(rows))
    if kind == "dense_assign":
        # X read once (FP32, or its two bfloat16 halves: 4 bytes per coordinate
        # either way) and label/u/lbg/stamp plus the lb row written per point
        out = [("hbm", N * (4.0 * D + 16.0 + 4.0 * Gp))]
        if dense_fp32:  # the CUDA-core engine evaluates every distance
            out.append(("alu", 3.0 * N * K * D))
        if dense_tc:  # the tensor-core engine: three bfloat16 products per pair
            out.append(("tensor", 6.0 * N * K * D))
        return out
    if kind == "filter":
        return [("hbm", 16.0 * N + 4.0 * mean("n_survivors", filt))]
    if kind == "survivor":
        surv, scan = mean("n_survivors", filt), mean("n_scanned", filt)
        # per survivor: queue entry, label/stamp/lbg, x row, u/stamp writes;
        # per scanned point: lb row read + write, label/lbg/u/stamp writes
        b = surv * (4 + 12 + 4 * D + 8) + scan * (8 * Gp + 16)
        return [("hbm", b), ("alu", 3.0 * D * mean("n_dist", filt))]
    if kind == "apply_moves":
        return [("hbm", 4.0 * N * D + 4.0 * N)]
    if kind == "stats":
        # labels read twice, point ids and labels written and read once, X read once
        return [("hbm", 8.0 * N + 16.0 * N + 4.0 * N * D)]
    return [("hbm", 0.0)]


def source_sha(files) -> str:
    h = hashlib.sha256()
    for f in files:
        h.update(open(os.path.join(ROOT, f), "rb").read())
    return h.hexdigest()[:16]


KERNEL_SOURCES = {
    "dense_assign": ["paper_1905_09345_gb300/csrc/kp_dense_tc.cu", "paper_1905_09345_gb300/csrc/kp_tc.cuh",
                     "paper_1905_09345_gb300/csrc/kp_common.cuh"],
    "apply_moves": ["paper_1905_09345_gb300/csrc/kp_dense.cu", "paper_1905_09345_gb300/csrc/kp_common.cuh"],
    "filter": ["paper_1905_09345_gb300/csrc/kp_filter.cu", "paper_1905_09345_gb300/csrc/kp_common.cuh"],
    "survivor": ["paper_1905_09345_gb300/csrc/kp_survivor_tp.cu", "paper_1905_09345_gb300/csrc/kp_common.cuh"],
    "update": ["paper_1905_09345_gb300/csrc/kp_update.cu", "paper_1905_09345_gb300/csrc/kp_common.cuh"],
    "settle": ["paper_1905_09345_gb300/csrc/kp_settle.cu", "paper_1905_09345_gb300/csrc/kp_common.cuh"],
    "stats": ["paper_1905_09345_gb300/csrc/kp_stats.cu", "paper_1905_09345_gb300/csrc/kp_common.cuh"],
}


def ncu_traffic(kernel: str, workload: str = "aniso1m"):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of that kernel and on this workload."""
    p = os.path.join(ROOT, "profiles", "ncu_traffic.json")
    if not os.path.exists(p):
        return None
    d = json.load(open(p)).get(kernel)
    if not d or d.get("source_sha") != source_sha(KERNEL_SOURCES.get(kernel, [])):
        return None
    if d.get("workload", "aniso1m") != workload:
        return None
    return d.get("dram_bytes_per_launch")


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
# the oracle samples are sized to about the same FP64 work whatever K and D:
# 2^18 points x K=256 x D=64 per timed iteration for the cpu_baseline
ORACLE_WORK = (1 << 18) * 256 * 64


def grouping_of(args) -> int:
    """KM_GROUP_* of the filtered fits (--grouping)."""
    return 1 if getattr(args, "grouping", "clustered") == "clustered" else 0


def make_workload(args, rank: int = 0):
    """The measured job (one replica per rank: the data seed follows the rank)."""
    from paper_1905_09345_gb300 import synth
    if args.workload == "highdim4m":
        return synth.highdim_4m(N=args.n or 1 << 22, seed=3 + rank)
    return synth.anisotropic_1m(N=args.n or 1 << 20, seed=2 + rank)


def oracle_sample(w, work: int) -> int:
    return max(1024, min(w.N, work // (w.K * w.D)))


def device_points(w, dev, pinned: bool = False):
    """X as the library is handed it: FP32, or bfloat16 bit patterns for the
    workloads stored as bfloat16 (the library widens those exactly at init)."""
    import numpy as np
    import torch
    from paper_1905_09345_gb300 import synth
    if w.meta.get("storage") == "bf16":
        t = torch.from_numpy(synth.bf16_bits(w.X).view(np.int16)).view(torch.bfloat16)
    else:
        t = torch.from_numpy(w.X)
    return t.pin_memory() if pinned else t.to(dev)


# ---------------------------------------------------------------------------
# arms
# ---------------------------------------------------------------------------
def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    w = make_workload(args)
    n_sample = oracle_sample(w, ORACLE_WORK // 4)
    import oracle
    oracle.build()
    Xs = w.X[:n_sample].astype("float64")
    C0 = w.C0.astype("float64")
    for _ in range(args.warmup):
        oracle_iterations(Xs, C0, 1)
    times = [oracle_iterations(Xs, C0, 1) for _ in range(args.steps)]
    ms = 1e3 * statistics.mean(times)
    value = n_sample / (ms / 1e3)
    cores = int(os.environ.get("OMP_NUM_THREADS", os.cpu_count() or 1))
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": w.name, "N": w.N, "D": w.D, "K": w.K, "G": w.G},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"brute-force FP64 Lloyd (oracle O1): one iteration over the first "
                                       f"{n_sample} of {w.N} points per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def profiled_pass(kpynq, X, C0, w, lab, C, stream, flush, steps, grouping=0):
    """Fits launched kernel by kernel with CUDA events around every launch.
    Returns per-kind (launches, ms), the launches that did work, and the
    last fit's per-iteration statistics."""
    prof = kpynq.KMeans(X, C0, w.G, stream=stream, profile=True, grouping=grouping)
    pstats = None
    kinds = {}
    # launches that did work: the dense pass and its settle run only in dense
    # iterations, the survivor kernel only in filtered ones (the others exit
    # at once); every launch of the other kinds works
    working = {"dense_assign": 0, "settle": 0, "survivor": 0}
    for _ in range(steps):
        flush.zero_()
        prof.reset(C0)
        r = prof.fit(w.max_iter, w.tol, lab, C)
        pstats = r.stats
        paths = [s["path"] for s in r.stats] + [prof.final_stats()["path"]]
        nd = sum(1 for pa in paths if pa != kpynq.KM_PATH_FILTERED)
        working["dense_assign"] += nd
        working["settle"] += nd
        working["survivor"] += len(paths) - nd
        for k, (n, t) in prof.profile().items():
            a = kinds.setdefault(k, [0, 0.0])
            a[0] += n
            a[1] += t
    prof.close()
    return kinds, working, pstats


def breakdown_of(kinds, working):
    total = sum(t for _, t in kinds.values())
    out = {}
    for k, (n, t) in kinds.items():
        if not n:
            continue
        nw = working.get(k, n)
        out[k] = {"launches": n, "working_launches": nw, "ms_total": round(t, 4),
                  "share": round(t / total, 4) if total else None,
                  "us_per_working_launch": round(1e3 * t / nw, 3) if nw else None}
    return out


def roofline_of(w, kinds, working, pstats, breakdown, workload) -> dict:
    """The dominant kernel's achieved fraction of its roofline: algorithmic
    units per working launch over its CUDA-event time (the bound with the
    larger fraction of its measured peak is reported, the other beside it)."""
    hbm_peak, tc_peak, peak_src = measured_peaks()
    dom = max(breakdown, key=lambda k: breakdown[k]["ms_total"])
    t_l = kinds[dom][1]
    n_l = working.get(dom, kinds[dom][0])
    per_launch_s = t_l / n_l / 1e3
    roofs = []
    for bound, units_l in algorithmic(dom, w, pstats, n_l):
        if bound == "alu":
            achieved = units_l / per_launch_s / 1e12
            roofs.append({"kernel": dom, "bound": "alu", "achieved": achieved, "peak": ALU_PEAK_TFLOPS,
                          "unit": "TFLOP/s", "frac": achieved / ALU_PEAK_TFLOPS, "_units": units_l,
                          "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz x 1.5 flop/issue "
                                         "(FSUB+FFMA mix)"})
        elif bound == "tensor":
            achieved = units_l / per_launch_s / 1e12
            roofs.append({"kernel": dom, "bound": "tensor", "achieved": achieved, "peak": tc_peak,
                          "unit": "TFLOP/s", "frac": achieved / tc_peak, "_units": units_l,
                          "peak_source": f"{peak_src} bf16_tflops (burst)"})
        else:
            achieved = units_l / per_launch_s / 1e9
            roofs.append({"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm_peak, "unit": "GB/s",
                          "frac": achieved / hbm_peak, "_units": units_l, "peak_source": f"{peak_src} hbm_gbs"})
    roof = max(roofs, key=lambda r: r["frac"])
    units_l = roof.pop("_units")
    others = sorted((r for r in roofs if r is not roof), key=lambda r: -r["frac"])
    if others:
        roof["other_bound"] = {"bound": others[0]["bound"], "frac": others[0]["frac"]}
    roof["traffic"] = ncu_traffic(dom, workload)
    roof["algorithmic_per_launch"] = units_l
    roof["launch_us"] = per_launch_s * 1e6
    roof["launches_averaged"] = n_l

    return roof


def run_ours(args):
    import numpy as np
    import torch

    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    from paper_1905_09345_gb300 import kpynq
    kpynq.lib()
    w = make_workload(args, rank)  # one replica problem per rank
    dev = torch.device("cuda", local)
    X = device_points(w, dev)
    C0 = torch.from_numpy(w.C0).to(dev)
    stream = torch.cuda.current_stream(dev)
    lab = torch.empty(w.N, dtype=torch.int32, device=dev)
    C = torch.empty(w.K, w.D, dtype=torch.float32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    log = lambda *a: print(*a, file=sys.stderr, flush=True) if rank == 0 else None

    def timed_steps(km, steps, warmup, label):
        iters, times, kern, stats = [], [], 0, None
        for i in range(warmup + steps):
            flush.zero_()  # L2 flush between steps (outside the timed interval)
            k0 = km.kernel_count
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            km.reset(C0)
            r = km.fit(w.max_iter, w.tol, lab, C, with_stats=False)
            e1.record(stream)
            e1.synchronize()
            if i >= warmup:
                times.append(e0.elapsed_time(e1))
                iters.append(r.n_iter)
                kern += km.kernel_count - k0
        stats = km.stats(0, iters[-1])
        log(f"[{label}] {steps} steps: {statistics.mean(times):.3f} ms/step, iters {iters[0]}")
        return times, iters, kern, stats

    grouping = grouping_of(args)
    if args.profile_only:
        kinds, working, _ = profiled_pass(kpynq, X, C0, w, lab, C, stream, flush, args.profile_steps, grouping)
        if rank == 0:
            print(json.dumps({"profile_only": True, "config": {"workload": w.name}, "fits": args.profile_steps,
                              "kernel_breakdown": breakdown_of(kinds, working)}), flush=True)
        return

    # --- the filtered method (the measured line) ---
    km = kpynq.KMeans(X, C0, w.G, stream=stream, grouping=grouping)
    torch.cuda.synchronize()
    barrier(ws)
    with ClockSampler(gpu_uuid()) as clk:
        torch.cuda.synchronize()
        barrier(ws)
        times, iters, kern, stats = timed_steps(km, args.steps, args.warmup, "filtered")
        torch.cuda.synchronize()
        barrier(ws)
    clocks = clk.summary()  # now: later samplers of this process reuse the file
    ms = statistics.mean(times)
    units = w.N * statistics.mean(iters)
    ms_max, units_all = aggregate(ms, units, ws, dev)
    value = units_all / (ms_max / 1e3)
    n_dist = sum(s["n_dist"] for s in stats)
    skip = 1.0 - n_dist / (w.N * w.K * len(stats))

    # --- plain GPU Lloyd on the same GPU and inputs: tensor cores, FP32 ---
    lloyd = kpynq.KMeans(X, C0, w.G, algo=kpynq.KM_ALGO_LLOYD, stream=stream)
    lt, li, _, lst = timed_steps(lloyd, args.lloyd_steps, 1, "plain Lloyd (library default dense engine)")
    lloyd_value = w.N * statistics.mean(li) / (statistics.mean(lt) / 1e3)
    lloyd.close()
    lloyd_tc = any(s["path"] == kpynq.KM_PATH_DENSE_TC for s in lst)
    if lloyd_tc:
        lloyd32 = kpynq.KMeans(X, C0, w.G, algo=kpynq.KM_ALGO_LLOYD, stream=stream, dense=kpynq.KM_DENSE_FP32)
        lt32, li32, _, _ = timed_steps(lloyd32, args.lloyd_steps, 1, "plain Lloyd (FP32 CUDA cores)")
        lloyd32.close()
    else:  # the tensor-core engine does not take this shape: the default arm already is FP32
        lt32, li32 = lt, li
    lloyd32_value = w.N * statistics.mean(li32) / (statistics.mean(lt32) / 1e3)

    # --- profiled pass: CUDA events around every launch ---
    kinds, working, pstats = profiled_pass(kpynq, X, C0, w, lab, C, stream, flush, args.profile_steps, grouping)
    breakdown = breakdown_of(kinds, working)
    roof = roofline_of(w, kinds, working, pstats, breakdown, args.workload)

    # --- end to end through the C ABI with host buffers ---
    Xh = device_points(w, None, pinned=True)
    C0h = torch.from_numpy(w.C0).pin_memory()
    labh = torch.empty(w.N, dtype=torch.int32).pin_memory()
    Ch = torch.empty(w.K, w.D, dtype=torch.float32).pin_memory()
    et, ei = [], []
    for i in range(args.e2e_steps + 1):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        k2 = kpynq.KMeans(Xh, C0h, w.G, stream=stream, grouping=grouping)
        r = k2.fit(w.max_iter, w.tol, labh, Ch)
        k2.close()
        torch.cuda.synchronize()
        if i > 0:
            et.append(time.perf_counter() - t0)
            ei.append(r.n_iter)
    e2e_value = w.N * statistics.mean(ei) / statistics.mean(et)
    # energy: fits looped for at least --energy-seconds, cumulative board counter
    energy = None
    if args.energy_seconds > 0:
        def one_fit():
            km.reset(C0)
            km.fit(w.max_iter, w.tol, lab, C, with_stats=False)
        energy = energy_loop(one_fit, w.N * statistics.mean(iters), args.energy_seconds, gpu_uuid())
    if energy is None:  # no energy counter: mean sampled power over the timed steps
        energy = energy_of(value, clocks)
    fstats = km.final_stats()
    near = {"n_recheck_total": int(sum(s_["n_recheck"] for s_ in stats) + fstats["n_recheck"]),
            "n_settle_total": int(sum(s_["n_settle"] for s_ in stats) + fstats["n_settle"]),
            "per_iteration_n_recheck": [s_["n_recheck"] for s_ in stats],
            "what": "n_recheck: points whose label was settled in FP64 (the FP32 error bound could not "
                    "order their two nearest centroids); n_settle: rows the tensor-core pass sent to the "
                    "exact settle.  Labels are exact for all of them."}
    e2e = {"value": e2e_value, "unit": UNIT,
           "h2d_bytes_per_step": int(Xh.numel() * Xh.element_size() + C0h.numel() * 4),
           "d2h_bytes_per_step": int(labh.numel() * 4 + Ch.numel() * 4 + 8 + 4),
           "ms_per_step": 1e3 * statistics.mean(et),
           "includes": "context creation (allocation, H2D copy of X), graph recording, fit, D2H of outputs"}

    if rank != 0:
        km.close()
        return
    cpu = None
    if ws == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(w, oracle_sample(w, ORACLE_WORK), 3)
    forms = None
    if not args.no_forms and args.workload == "aniso1m":
        km.close()
        del X
        torch.cuda.empty_cache()
        forms = {}
        fs, fw = args.form_steps, args.form_warmup
        for name, fn in (("highdim4m", lambda: highdim_record(args, dev, fs, fw)),
                         ("batched512", lambda: batched_record(args, dev, steps=fs, warmup=fw)),
                         ("proposal8m", lambda: proposal_record(args, dev, log=log, steps=fs, warmup=fw)),
                         ("skewed1m", lambda: skewed_record(args, dev, fs, fw)),
                         ("grouping_aniso1m", lambda: grouping_record(args, dev, fs, fw))):
            t0 = time.perf_counter()
            try:
                rec = fn()
                rec.pop("_units", None)
                rec["wall_s"] = time.perf_counter() - t0
            except Exception as e:  # one form failing must not lose the main line
                rec = {"error": f"{type(e).__name__}: {e}"}
            forms[name] = rec
            torch.cuda.empty_cache()
            log(f"[form {name}] {time.perf_counter() - t0:.1f} s")
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": w.name, "N": w.N, "D": w.D, "K": w.K, "G": w.G, "max_iter": w.max_iter,
                   "tol": w.tol, "iters_per_step": statistics.mean(iters),
                   "step": "kmeans_reset + kmeans_fit (dense iteration 0, filtered iterations, final assignment)",
                   "storage": w.meta.get("storage", "f32"), "grouping": args.grouping,
                   "l2": f"flushed between steps (256 MiB write); X is {w.N * w.D * 4 >> 20} MiB > L2",
                   "parallelism": f"replicas x{ws}"},
        "clocks": clocks,
        "energy": energy,
        "near_ties": near,
        "e2e": e2e,
        "gpu_launches": kern,
        "roofline": roof,
        "cpu_baseline": cpu,
        "skip_fraction": skip,
        "plain_lloyd": {"value": lloyd_value, "ms_per_step": statistics.mean(lt), "iters": statistics.mean(li),
                        "dense": "BF16x3 tensor cores (tcgen05) + exact FP32/FP64 settle" if lloyd_tc else
                                 "FP32 CUDA cores (the tensor-core engine does not take this shape)"},
        "vs_plain_lloyd": value / lloyd_value,
        "plain_lloyd_fp32": {"value": lloyd32_value, "ms_per_step": statistics.mean(lt32),
                             "iters": statistics.mean(li32), "dense": "FP32 CUDA cores"},
        "vs_plain_lloyd_fp32": value / lloyd32_value,
        "paths": [s["path"] for s in stats],
        "filter_counts": {"n_survivors": [s["n_survivors"] for s in stats],
                          "n_scanned": [s["n_scanned"] for s in stats],
                          "n_dist": [s["n_dist"] for s in stats],
                          "what": "per iteration: points the global filter did not keep, points still "
                                  "unresolved after tightening u (then group and point filters), distances "
                                  "evaluated (K per point in a dense pass)"},
        "kernel_breakdown": breakdown,
        "forms": forms,
    }
    print(json.dumps(line), flush=True)
    if forms is None:
        km.close()
    if ws > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_batched(args):
    """512 independent problems (N ~ logU[1e3, 2e5], D in {8,32,64,128},
    K ~ logU[8,512], G = K/10, 25 iterations each) fitted by one graph launch
    of the batched form, against the same problems fitted one after another
    with single contexts, and against batched plain Lloyd.  Metric: points x
    iterations per second over the batch."""
    import torch
    ws_, rank, local = dist_env()
    torch.cuda.set_device(local)
    rec = batched_record(args, torch.device("cuda", local), seed0=1000 * rank)
    units, ms = rec.pop("_units"), rec["ms_per_step"]
    ms_max, units_all = aggregate(ms, units, ws_, torch.device("cuda", local))
    if rank != 0:
        return
    line = {"metric": "points*iters/s (batched filtered K-means, 512 problems, exact labels)",
            "value": units_all / (ms_max / 1e3), "unit": UNIT, "n_gpus": ws_, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic"}
    line.update(rec)
    line["ms_per_step"] = ms_max
    line["config"]["parallelism"] = f"replicas x{ws_}"
    print(json.dumps(line), flush=True)


def batched_record(args, dev, seed0=0, steps=None, warmup=None) -> dict:
    import tempfile
    import torch
    from paper_1905_09345_gb300 import kpynq, synth
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    t0 = time.perf_counter()
    specs = synth.batched_problems(args.problems, seed0=seed0)
    works = [synth.batched_problem(s) for s in specs]
    gen_s = time.perf_counter() - t0
    probs = [(torch.from_numpy(w.X).to(dev), torch.from_numpy(w.C0).to(dev), w.G) for w in works]
    stream = torch.cuda.current_stream(dev)
    max_iter = works[0].max_iter
    cache = os.path.join(tempfile.gettempdir(), f"kpynq_tune_{os.getpid()}.txt")
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)

    def timed_batch(b):
        def one_step():
            flush.zero_()
            b.reset()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            b.fit(max_iter, 0.0)
            e1.record(stream)
            e1.synchronize()
            return e0.elapsed_time(e1)
        for _ in range(warmup):
            one_step()
        return [one_step() for _ in range(steps)]

    t0 = time.perf_counter()
    b = kpynq.KMeansBatch(probs, stream=stream, tune_cache=cache)
    init_s = time.perf_counter() - t0
    with ClockSampler(gpu_uuid()) as clk:
        times = timed_batch(b)
    iters = [b.get(i)[1] for i in range(len(works))]
    units = sum(w.X.shape[0] * it for w, it in zip(works, iters))
    ms = statistics.mean(times)
    switches = sorted(set(round(b.switch(i), 2) for i in range(len(works))))
    tunings = [b.tuning(i) for i in range(len(works))]
    tuned = {"problems_on_fp32_engine": sum(1 for t in tunings if t[1] == kpynq.KM_DENSE_FP32),
             "survivor_claim": {str(g): sum(1 for t in tunings if t[2] == g) for g in sorted({t[2] for t in tunings})}}
    b.close()
    # batched plain Lloyd: the same problems, every distance every iteration
    bl = kpynq.KMeansBatch(probs, stream=stream, algo=kpynq.KM_ALGO_LLOYD)
    ltimes = timed_batch(bl)
    liters = [bl.get(i)[1] for i in range(len(works))]
    lunits = sum(w.X.shape[0] * it for w, it in zip(works, liters))
    bl.close()
    # the same problems, one fit after another (single contexts, graphs recorded beforehand)
    kms = [kpynq.KMeans(X, C0, G, stream=stream) for X, C0, G in probs]
    for km in kms:
        km.fit(max_iter, 0.0, with_stats=False)
    seq = []
    for _ in range(max(1, min(3, steps))):
        for km, (X, C0, G) in zip(kms, probs):
            km.reset(C0)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        for km in kms:
            km.fit(max_iter, 0.0, with_stats=False)
        torch.cuda.synchronize()
        seq.append(time.perf_counter() - t1)
    for km in kms:
        km.close()
    try:
        os.remove(cache)
    except OSError:
        pass
    value = units / (ms / 1e3)
    lvalue = lunits / (statistics.mean(ltimes) / 1e3)
    seq_value = units / statistics.mean(seq)
    return {
        "value": value, "ms_per_step": ms, "_units": units,
        "config": {"workload": f"batched{len(works)}", "problems": len(works),
                   "points": int(sum(w.X.shape[0] for w in works)), "max_iter": max_iter,
                   "step": "kmeans_batch_reset + kmeans_batch_fit (one graph launch)",
                   "l2": "flushed between steps (256 MiB write)"},
        "clocks": clk.summary(), "init_s": init_s, "generate_s": gen_s, "tuned_switches": switches,
        "tuned": tuned,
        "batched_plain_lloyd": {"value": lvalue, "ms_per_step": statistics.mean(ltimes)},
        "vs_batched_plain_lloyd": value / lvalue,
        "sequential_single_contexts": {"value": seq_value, "s_per_step": statistics.mean(seq)},
        "vs_sequential": value / seq_value,
    }


def skewed_record(args, dev, steps, warmup) -> dict:
    """The real-data-like skewed job (N=1,048,576, D=32, K=128, G=13) seeded by
    k-means++ on the GPU: the seeding's time, then the filtered method and
    plain Lloyd on the same GPU and inputs."""
    import torch
    from paper_1905_09345_gb300 import kpynq, synth
    w = synth.skewed_mixture()
    X = torch.from_numpy(w.X).to(dev)
    stream = torch.cuda.current_stream(dev)
    C0 = torch.empty(w.K, w.D, dtype=torch.float32, device=dev)
    times = []
    for i in range(warmup + steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        kpynq.kmeans_init_kmeanspp(X, w.N, w.D, w.K, w.meta["pp_u"], C0, None, stream)
        e1.record(stream)
        e1.synchronize()
        if i >= warmup:
            times.append(e0.elapsed_time(e1))
    lab = torch.empty(w.N, dtype=torch.int32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    out = {}
    for name, algo in (("filtered", kpynq.KM_ALGO_FILTERED), ("plain_lloyd", kpynq.KM_ALGO_LLOYD)):
        km = kpynq.KMeans(X, C0, w.G, stream=stream, algo=algo,
                          grouping=grouping_of(args) if algo == kpynq.KM_ALGO_FILTERED else 0)
        ft, fi = [], []
        for i in range(warmup + steps):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            km.reset(C0)
            r = km.fit(w.max_iter, w.tol, lab, with_stats=False)
            e1.record(stream)
            e1.synchronize()
            if i >= warmup:
                ft.append(e0.elapsed_time(e1))
                fi.append(r.n_iter)
        st = km.stats(0, fi[-1])
        km.close()
        ms = statistics.mean(ft)
        out[name] = {"value": w.N * statistics.mean(fi) / (ms / 1e3), "ms_per_fit": ms, "iters": fi[-1],
                     "skip_fraction": 1.0 - sum(s_["n_dist"] for s_ in st) / (w.N * w.K * len(st)),
                     "n_recheck_total": int(sum(s_["n_recheck"] for s_ in st)),
                     "paths": [s_["path"] for s_ in st]}
    return {"config": {"workload": w.name, "N": w.N, "D": w.D, "K": w.K, "G": w.G, "max_iter": w.max_iter,
                       "tol": w.tol, "init": "k-means++ on the GPU (kmeans_init_kmeanspp)", "grouping": args.grouping},
            "kmeanspp_ms": statistics.mean(times),
            "filtered": out["filtered"], "plain_lloyd": out["plain_lloyd"],
            "vs_plain_lloyd": out["filtered"]["value"] / out["plain_lloyd"]["value"]}


def grouping_record(args, dev, steps, warmup) -> dict:
    """The anisotropic 1M job (G = 26) with contiguous and with clustered
    groups (Lloyd over the initial centroids): time per fit and the fraction
    of distance evaluations skipped, with the default switch and with the
    filters alone after iteration 0."""
    import torch
    from paper_1905_09345_gb300 import kpynq
    w = make_workload(argparse.Namespace(workload="aniso1m", n=None), 0)
    X = device_points(w, dev)
    C0 = torch.from_numpy(w.C0).to(dev)
    stream = torch.cuda.current_stream(dev)
    lab = torch.empty(w.N, dtype=torch.int32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    rows = []
    for grouping, name in ((kpynq.KM_GROUP_CONTIGUOUS, "contiguous"), (kpynq.KM_GROUP_CLUSTERED, "clustered")):
        for switch in (0.0, 1.0):
            km = kpynq.KMeans(X, C0, w.G, stream=stream, dense_switch=switch, grouping=grouping)
            ng = km.groups()
            times, iters = [], []
            for i in range(warmup + steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                km.reset(C0)
                r = km.fit(w.max_iter, w.tol, lab, with_stats=False)
                e1.record(stream)
                e1.synchronize()
                if i >= warmup:
                    times.append(e0.elapsed_time(e1))
                    iters.append(r.n_iter)
            st = km.stats(0, iters[-1])
            km.close()
            later = [s_ for s_ in st if s_["iter"] > 0]
            rows.append({"grouping": name, "groups": ng, "switch": "default" if switch == 0.0 else "filters only",
                         "ms_per_fit": statistics.mean(times), "iters": iters[-1],
                         "skip_fraction": 1.0 - sum(s_["n_dist"] for s_ in st) / (w.N * w.K * len(st)),
                         "skip_fraction_iters_ge_1": 1.0 - sum(s_["n_dist"] for s_ in later) /
                         max(1, w.N * w.K * len(later))})
    return {"config": {"workload": w.name, "N": w.N, "D": w.D, "K": w.K, "G": w.G}, "rows": rows}


def highdim_record(args, dev, steps, warmup) -> dict:
    """The high-dimension job (N=4,194,304, D=128, K=1024, G=103, bfloat16
    storage, 30 iterations): the filtered method and plain Lloyd, both with
    tensor-core dense passes, on the same GPU and inputs."""
    import torch
    from paper_1905_09345_gb300 import kpynq, synth
    t0 = time.perf_counter()
    w = synth.highdim_4m()
    gen_s = time.perf_counter() - t0
    X = device_points(w, dev)
    C0 = torch.from_numpy(w.C0).to(dev)
    stream = torch.cuda.current_stream(dev)
    lab = torch.empty(w.N, dtype=torch.int32, device=dev)
    C = torch.empty(w.K, w.D, dtype=torch.float32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    out = {}
    with ClockSampler(gpu_uuid()) as clk:
        for name, algo in (("filtered", kpynq.KM_ALGO_FILTERED), ("plain_lloyd", kpynq.KM_ALGO_LLOYD)):
            # contiguous groups: on this job they beat groups of nearby centroids
            # (79.8 against 85.3 ms per fit), unlike the anisotropic 1M job
            km = kpynq.KMeans(X, C0, w.G, stream=stream, algo=algo)
            times, iters = [], []
            for i in range(warmup + steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                km.reset(C0)
                r = km.fit(w.max_iter, w.tol, lab, C, with_stats=False)
                e1.record(stream)
                e1.synchronize()
                if i >= warmup:
                    times.append(e0.elapsed_time(e1))
                    iters.append(r.n_iter)
            st = km.stats(0, iters[-1]) + [km.final_stats()]
            km.close()
            ms = statistics.mean(times)
            out[name] = {"value": w.N * statistics.mean(iters) / (ms / 1e3), "ms_per_fit": ms, "iters": iters[-1],
                         "skip_fraction": 1.0 - sum(s_["n_dist"] for s_ in st[:-1]) / (w.N * w.K * (len(st) - 1)),
                         "n_recheck_total": int(sum(s_["n_recheck"] for s_ in st)),
                         "n_settle_total": int(sum(s_["n_settle"] for s_ in st)),
                         "paths": [s_["path"] for s_ in st[:-1]]}
    kinds, working, pstats = profiled_pass(kpynq, X, C0, w, lab, C, stream, flush, 1)
    breakdown = breakdown_of(kinds, working)
    return {"config": {"workload": w.name, "N": w.N, "D": w.D, "K": w.K, "G": w.G, "max_iter": w.max_iter,
                       "storage": "bf16", "l2": "flushed between steps", "grouping": "contiguous"},
            "generate_s": gen_s, "clocks": clk.summary(),
            "filtered": out["filtered"], "plain_lloyd": out["plain_lloyd"],
            "plain_lloyd_dense": "BF16x3 tensor cores (tcgen05, streamed centroid blocks) + exact settle",
            "vs_plain_lloyd": out["filtered"]["value"] / out["plain_lloyd"]["value"],
            "roofline": roofline_of(w, kinds, working, pstats, breakdown, "highdim4m"),
            "kernel_breakdown": breakdown}


def run_gsweep(args):
    """The anisotropic job with the number of centroid groups swept (the
    method's group-filter granularity): throughput and the fraction of
    distance evaluations the filters skip, per G; the dense switch never
    fires after iteration 0 here, so that the filters alone do the work."""
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    from paper_1905_09345_gb300 import kpynq
    w = make_workload(args, rank)
    dev = torch.device("cuda", local)
    X = device_points(w, dev)
    C0 = torch.from_numpy(w.C0).to(dev)
    stream = torch.cuda.current_stream(dev)
    lab = torch.empty(w.N, dtype=torch.int32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    K = w.K
    rows = []
    with ClockSampler(gpu_uuid()) as clk:
        for G in sorted({1, max(1, K // 20), max(1, K // 10), max(1, K // 5), K}):
            for grouping, switch, label in ((0, 0.0, "default switch"), (0, 1.0, "filters only"),
                                            (1, 0.0, "clustered, default switch"),
                                            (1, 1.0, "clustered, filters only")):
                if grouping and G in (1, K):
                    continue  # one group, or one centroid per group: the same as contiguous
                km = kpynq.KMeans(X, C0, G, stream=stream, dense_switch=switch, grouping=grouping)
                times, iters, nd = [], [], 0
                for i in range(args.warmup + args.steps):
                    flush.zero_()
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    km.reset(C0)
                    r = km.fit(w.max_iter, w.tol, lab, with_stats=False)
                    e1.record(stream)
                    e1.synchronize()
                    if i >= args.warmup:
                        times.append(e0.elapsed_time(e1))
                        iters.append(r.n_iter)
                st = km.stats(0, iters[-1])
                km.close()
                nd = sum(s_["n_dist"] for s_ in st)
                ms = statistics.mean(times)
                rows.append({"G": G, "switch": label, "ms_per_fit": ms, "iters": iters[-1],
                             "points_iters_per_s": w.N * statistics.mean(iters) / (ms / 1e3),
                             "skip_fraction": 1.0 - nd / (w.N * K * len(st))})
    if rank == 0:
        best = max(rows, key=lambda r_: r_["points_iters_per_s"])
        print(json.dumps({"metric": METRIC, "value": best["points_iters_per_s"], "unit": UNIT, "n_gpus": ws,
                          "steps": args.steps, "warmup": args.warmup, "ms_per_step": best["ms_per_fit"],
                          "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                          "data": "synthetic", "config": {"workload": w.name + "_gsweep", "N": w.N, "D": w.D,
                                                          "K": K, "best_G": best["G"], "best": best["switch"]},
                          "clocks": clk.summary(), "sweep": rows}), flush=True)


def run_proposal(args):
    """The learned-proposal family (N=8,388,608, D=32, K=4096, G=410, 40
    iterations).  The network D -> 256 -> 256 -> G is trained on the GPU
    (kmeans_mlp_train: tcgen05 forward and backward, Adam) on (point, group of
    its final centroid) pairs from the library's own fits of training seeds
    1..8 of the family, then seeds iteration 0 of fits of the held-out seed 9;
    fits with and without it."""
    import numpy as np
    import torch
    ws, rank, local = dist_env()
    torch.cuda.set_device(local)
    from paper_1905_09345_gb300 import kpynq, synth
    rec = proposal_record(args, torch.device("cuda", local), log=lambda *a: print(*a, file=sys.stderr, flush=True)
                          if rank == 0 else None)
    if rank != 0:
        return
    line = {"metric": "points*iters/s (filtered K-means seeded by the learned proposal, exact labels)",
            "value": rec["with_proposal"]["points_iters_per_s"], "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": rec["with_proposal"]["ms_per_fit"], "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic"}
    line.update(rec)
    print(json.dumps(line), flush=True)


def proposal_record(args, dev, log=None, steps=None, warmup=None):
    import numpy as np
    import torch
    from paper_1905_09345_gb300 import kpynq, synth
    log = log or (lambda *a: None)
    steps = args.steps if steps is None else steps
    warmup = args.warmup if warmup is None else warmup
    stream = torch.cuda.current_stream(dev)
    N = args.n or 1 << 23
    H = 256
    n_train = args.train_n
    # training pairs: the groups of the final labels of fits on seeds 1..8
    t0 = time.perf_counter()
    Xs, labs = [], []
    for seed in range(1, 9):
        wt = synth.proposal_family(seed, N=n_train)
        Xd = torch.from_numpy(wt.X).to(dev)
        km = kpynq.KMeans(Xd, torch.from_numpy(wt.C0).to(dev), wt.G, stream=stream)
        lab = torch.empty(wt.N, dtype=torch.int32, device=dev)
        km.fit(wt.max_iter, wt.tol, lab, with_stats=False)
        km.close()
        Xs.append(Xd)
        labs.append(lab)
    G, K, D = wt.G, wt.K, wt.D
    Xtr = torch.cat(Xs)
    ytr = torch.cat(labs)
    del Xs, labs
    torch.cuda.synchronize()
    prep_s = time.perf_counter() - t0
    net = kpynq.MLP(D, H, G, seed=1, stream=stream)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    train_loss, train_acc = net.train(Xtr, ytr, K, steps=args.train_steps, batch=8192, lr=1e-3, seed=7)
    e1.record(stream)
    e1.synchronize()
    train_ms = e0.elapsed_time(e1)
    per_sample = 2.0 * 3.0 * (D * H + H * H + H * G)  # forward + backward flops per row
    train_tflops = args.train_steps * 8192 * per_sample / (train_ms / 1e3) / 1e12
    log(f"[proposal] trained {args.train_steps} steps x 8192 rows on {Xtr.shape[0]} pairs in {train_ms:.0f} ms "
        f"(loss {train_loss:.3f}, batch accuracy {train_acc:.3f})")
    params = net.get_params({k: torch.empty(shp, dtype=torch.float32, device=dev)
                             for k, shp in net.shapes().items()})
    del Xtr, ytr
    # held-out seed 9
    w = synth.proposal_family(9, N=N)
    X = torch.from_numpy(w.X).to(dev)
    C0 = torch.from_numpy(w.C0).to(dev)
    lab = torch.empty(w.N, dtype=torch.int32, device=dev)
    flush = torch.empty(2 * L2_BYTES // 4, dtype=torch.float32, device=dev)
    out = {}
    final_groups = None
    with ClockSampler(gpu_uuid()) as clk:
        for name in ("without", "with"):
            km = kpynq.KMeans(X, C0, G, stream=stream)
            if name == "with":
                km.set_proposal(params)
            times, iters = [], []
            for i in range(warmup + steps):
                flush.zero_()
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record(stream)
                km.reset(C0)
                r = km.fit(w.max_iter, w.tol, lab, with_stats=False)
                b.record(stream)
                b.synchronize()
                if i >= warmup:
                    times.append(a.elapsed_time(b))
                    iters.append(r.n_iter)
            st = km.stats(0, iters[-1])
            km.close()
            prof = kpynq.KMeans(X, C0, G, stream=stream, profile=True)
            if name == "with":
                prof.set_proposal(params)
            prof.fit(w.max_iter, w.tol, lab)
            breakdown = {k: v for k, v in prof.profile().items() if v[0]}
            prof.close()
            if name == "without":
                final_groups = (lab.to(torch.int64) * G) // K
            ms = statistics.mean(times)
            out[name] = {"ms_per_fit": ms, "iters": iters[-1],
                         "points_iters_per_s": w.N * statistics.mean(iters) / (ms / 1e3),
                         "iter0": {k: st[0][k] for k in ("path", "n_dist", "n_survivors", "n_settle", "n_recheck")},
                         "n_recheck_total": int(sum(s_["n_recheck"] for s_ in st)),
                         "skip_fraction": 1.0 - sum(s_["n_dist"] for s_ in st) / (w.N * K * len(st)),
                         "profile_ms": {k: round(v[1], 3) for k, v in breakdown.items()}}
    pred = torch.empty(w.N, dtype=torch.int32, device=dev)
    net.predict(X, pred)
    acc = float((pred.to(torch.int64) == final_groups).float().mean().item())
    net.close()
    inf_flops = 2.0 * w.N * (D * H + H * H + H * G)
    prop_ms = out["with"]["profile_ms"].get("proposal")
    rec = {"config": {"workload": w.name, "N": w.N, "D": D, "K": K, "G": G, "hidden": H,
                      "train": f"GPU (kmeans_mlp_train, tcgen05 BF16 products, FP32 Adam): {args.train_steps} "
                               f"steps x 8192 rows drawn from {8 * n_train} (point, final group) pairs of "
                               f"training seeds 1-8 ({n_train} points each), lr 1e-3",
                      "l2": "flushed between steps"},
           "clocks": clk.summary(),
           "train": {"ms": train_ms, "steps": args.train_steps, "batch": 8192, "mean_loss": train_loss,
                     "batch_accuracy": train_acc, "tflops": train_tflops, "prep_s": prep_s},
           "proposal_accuracy": acc,
           "mlp_inference": {"flops": inf_flops,
                             "proposal_kernels_ms": prop_ms,
                             "tflops_upper": (inf_flops / (prop_ms / 1e3) / 1e12) if prop_ms else None,
                             "note": "proposal_kernels_ms also holds the centroid table and the seeded bounds"},
           "with_proposal": out["with"], "without_proposal": out["without"],
           "vs_without": out["with"]["points_iters_per_s"] / out["without"]["points_iters_per_s"]}
    return rec


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "gsweep":
        run_gsweep(args)
    elif args.workload == "proposal":
        run_proposal(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
