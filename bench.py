#!/usr/bin/env python3
"""Throughput of the fused D2Q9 pseudopotential LBM step on GB300.

Workload (default): one 1024 x 4096 domain, FP32 populations with FP64
reductions, Carnahan-Starling EOS with a = 0.25, b = 4, R = 1 at T = 0.80 T_c,
gravity (rho - <rho>) g with g_y = -1e-4, liquid below y = 2048 under vapour,
seeded +-1e-3 uniform density noise across the interface, tau = 1,
sigma = 1.385. A step is one time step of the whole domain (one launch of the
fused kernel). Metric: MLUPS (million lattice-node updates per second).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

With N > 1 (torchrun, one rank per GPU) the column is cut into N slabs of rows,
one per GPU - by default a 1024 x 4096 slab per GPU of a 1024 x 4096 N column (weak
scaling; ``--slab-scaling strong`` cuts the 1024 x 4096 column itself): every step
each rank runs the fused step on its rows, sums the column's mass with the others
(NCCL all-reduce, for <rho> of Eq. Gravity_2) and swaps two ghost rows with each
neighbour (NCCL send / receive); ``--partition replicas`` runs N independent copies
instead. The time-to-steady
block splits its columns over the ranks with no exchange. The JSON line reports
the aggregate over ranks with the max-over-ranks time. ``--impl reference``
times the FP64 CPU oracle on the host cores on a bounded slice of the same
workload.
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
sys.path.insert(0, ROOT)

NX, NY = 1024, 4096
A, B, R = 0.25, 4.0, 1.0
TR = 0.80
GY = -1e-4
LIQUID_ROWS = 2048
NOISE = 1e-3
SEED = 20230130
BYTES_PER_NODE = {"fp32": 72, "fp64": 144}   # 9 populations read + 9 written
# The FP64 step is bound by GB300's FP64 pipe, not by HBM: ncu counts 57 DFMA + 54 DADD +
# 35 DMUL per node (step_kernel<double>, 1024 x 4096, tau = 1) = 203 FP64 flops per node
# (FMA = 2). Peak: 2 FP64 FMAs per SM per clock, the rate the nominal 1.25 TFLOP/s dense
# FP64 of GB300 gives for 152 SMs at 2.07 GHz (1.25e12 / (2 x 152 x 2.07e9) = 1.99).
FP64_FLOPS_PER_NODE = 203
FP64_PEAK_TFLOPS = 2 * 2 * 152 * 2.07e9 / 1e12
# With (rho - <rho>) g at g_y = -1e-4 the 2048-row vapour column accelerates freely
# (max |u| = 0.42 after 500 steps, NaN before 1000): the workload is physical only for
# its first ~500 steps. Timed runs longer than WINDOW steps restore the post-warm-up
# state every WINDOW steps (lbm_set_state from a device snapshot, inside the timing).
WINDOW = 400
KERNEL_SRC = os.path.join(ROOT, "paper_2301_12869_gb300", "csrc", "lbm_kernels.cu")
PROFILE_SUMMARY = os.path.join(ROOT, "profiles", "step_kernel_fp32_1024x4096.json")


PREROLL_CYCLES = 200_000  # ~0.1 ms at 2 GHz


def run_steps(lbm, h, nsteps, snapshot):
    """nsteps fused steps; every WINDOW steps the snapshot state is restored on the device.
    Returns the number of restores."""
    done = restores = 0
    while done < nsteps:
        n = min(WINDOW, nsteps - done)
        lbm.lbm_step(h, n)
        done += n
        if done < nsteps:
            lbm.lbm_set_state(h, snapshot)
            restores += 1
    return restores


def workload_config(precision):
    return {
        "workload": f"single liquid column {NX}x{NY} D2Q9, {precision.upper()} populations, FP64 reductions",
        "nx": NX, "ny": NY, "T_over_Tc": TR, "a": A, "b": B, "R": R, "gravity": "(rho-<rho>)g", "g_y": GY,
        "liquid_rows": LIQUID_ROWS, "noise": NOISE, "seed": SEED, "tau": 1.0, "sigma": 1.385,
        "l2": "state 302 MB (FP32) > 129 MB L2: no flush needed",
        "physical_window": f"state restored from the post-warm-up snapshot every {WINDOW} steps "
                           "(the workload goes non-physical after ~500 steps)",
    }


def kernel_source_hash():
    """sha256[:16] of the kernel source with comments and blank space removed: a profile
    stays valid across comment edits and goes stale with any change to the code."""
    import re

    with open(KERNEL_SRC) as fh:
        src = fh.read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = "\n".join(line.strip() for line in src.splitlines() if line.strip())
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as fh:
            return json.load(fh), "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def traffic_from_profile(precision):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on this kernel source."""
    if precision != "fp32" or not os.path.exists(PROFILE_SUMMARY):
        return None
    with open(PROFILE_SUMMARY) as fh:
        prof = json.load(fh)
    if prof.get("kernel_source_sha256_16") != kernel_source_hash():
        return None
    return prof.get("dram_bytes_per_launch")


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 20 ms while running."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.proc = None
        self.gpu = gpu_index

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "20"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            parts = [s.strip() for s in ln.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                mx = float(parts[1])
            except ValueError:
                continue
            for name, val in zip(names, parts[3:7]):
                if val.lower() == "active":
                    reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


class NvmlClocks:
    """SM clock and clock-event reasons of one GPU read through NVML (libnvidia-ml, ctypes)
    by a thread every ~0.2 ms between start() and stop(), so that a timed region of a
    millisecond still gets samples. Reads only; falls back to nothing if NVML is absent.
    Reason bits as NVML defines them: 0x4 sw_power_cap, 0x8 hw_slowdown,
    0x20 sw_thermal_slowdown, 0x40 hw_thermal_slowdown, 0x80 hw_power_brake_slowdown."""

    REASONS = {0x4: "sw_power_cap", 0x8: "hw_slowdown", 0x20: "sw_thermal_slowdown", 0x40: "hw_thermal_slowdown",
               0x80: "hw_power_brake_slowdown"}

    def __init__(self, torch_device, period_s=0.0002):
        import ctypes
        import threading

        self.period = period_s
        self.samples, self.max_mhz, self.err = [], None, None
        self._stop = threading.Event()
        self._thread = None
        try:
            lib = ctypes.CDLL("libnvidia-ml.so.1")
            if lib.nvmlInit_v2() != 0:
                raise RuntimeError("nvmlInit failed")
            self.lib, self.h = lib, ctypes.c_void_p()
            rc = -1
            uuid = getattr(self._props(torch_device), "uuid", None)
            if uuid is not None:
                rc = lib.nvmlDeviceGetHandleByUUID(("GPU-" + str(uuid)).encode(), ctypes.byref(self.h))
            if rc != 0:
                rc = lib.nvmlDeviceGetHandleByIndex_v2(ctypes.c_uint(torch_device), ctypes.byref(self.h))
            if rc != 0:
                raise RuntimeError("no NVML handle")
            mx = ctypes.c_uint()
            if lib.nvmlDeviceGetMaxClockInfo(self.h, 1, ctypes.byref(mx)) == 0:  # 1: NVML_CLOCK_SM
                self.max_mhz = mx.value
            self._reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
                getattr(lib, "nvmlDeviceGetCurrentClocksThrottleReasons")
        except Exception as exc:  # noqa: BLE001 - reported in the summary
            self.lib, self.err = None, str(exc)

    @staticmethod
    def _props(dev):
        import torch

        return torch.cuda.get_device_properties(dev)

    def _run(self):
        import ctypes

        clk, rsn = ctypes.c_uint(), ctypes.c_ulonglong()
        while not self._stop.is_set():
            if self.lib.nvmlDeviceGetClockInfo(self.h, 1, ctypes.byref(clk)) == 0:
                r = rsn.value if self._reasons(self.h, ctypes.byref(rsn)) == 0 else 0
                self.samples.append((time.perf_counter(), clk.value, r))
            time.sleep(self.period)

    def start(self):
        import threading

        if self.lib is not None:
            self._thread = threading.Thread(target=self._run, daemon=True)
            self._thread.start()
        return self

    def stop(self):
        if self._thread is not None:
            self._stop.set()
            self._thread.join(timeout=5)

    def summary(self, t0=None, t1=None):
        """Median SM clock and the reasons seen, over the samples taken within [t0, t1]
        (host perf_counter seconds) if given, else over all of them."""
        sel = [s for s in self.samples if (t0 is None or s[0] >= t0) and (t1 is None or s[0] <= t1)]
        if not sel:
            return {"sm_mhz": None, "sm_max_mhz": self.max_mhz, "reasons": ["unavailable"], "samples": 0,
                    "source": "nvml" if self.lib is not None else f"none ({self.err})"}
        reasons = sorted({name for _, _, r in sel for bit, name in self.REASONS.items() if r & bit})
        return {"sm_mhz": statistics.median(c for _, c, _ in sel), "sm_max_mhz": self.max_mhz, "reasons": reasons,
                "samples": len(sel), "source": f"nvml, ~{1e3 * self.period:g} ms period"}


# ---------------------------------------------------------------- CPU oracle timing
def oracle_sample_main(ny_slice, steps, warmup=1):
    """Runs in a child process: `warmup` untimed, then `steps` timed oracle steps on a
    1024 x ny_slice slice around the interface."""
    import numpy as np

    from oracle import eos
    from oracle import lbm as olbm
    from paper_2301_12869_gb300 import inputs

    _, Tc, _ = eos.critical_point(A, B, R)
    rv, rl, _ = eos.maxwell(TR * Tc, A, B, R)
    rho_full_rows = inputs.column_rho0(NX, NY, rl, rv, LIQUID_ROWS, noise_amp=NOISE, seed=SEED)
    y0 = LIQUID_ROWS - ny_slice // 2
    rho0 = np.ascontiguousarray(rho_full_rows[y0:y0 + ny_slice])
    p = olbm.Params(nx=NX, ny=ny_slice, a=A, b=B, R=R, T=TR * Tc, g=(0.0, GY), form=2)
    f = olbm.init_state(rho0)
    for _ in range(max(1, warmup)):  # warm-up (allocations)
        f = olbm.step(f, p)
    t0 = time.perf_counter()
    for _ in range(steps):
        f = olbm.step(f, p)
    dt = time.perf_counter() - t0
    print(json.dumps({"seconds": dt, "nodes": NX * ny_slice, "steps": steps}))


def time_oracle(ny_slice, steps, warmup=1):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1")
    code = f"import bench; bench.oracle_sample_main({ny_slice}, {steps}, {warmup})"
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, env=env, capture_output=True, text=True, timeout=1800)
    if out.returncode != 0:
        raise RuntimeError(out.stderr[-2000:])
    res = json.loads(out.stdout.strip().splitlines()[-1])
    return res["nodes"] * res["steps"] / res["seconds"] / 1e6, res


def _oracle_task(task):
    """One unit of the CPU baseline's process pool (runs in a spawned child, one thread):
    ("small", steps) - the 4 x 200 FP64 column; ("column", index, steps) - one column of the
    seeded batched set. Returns (node updates, seconds)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import numpy as np

    np.seterr(all="ignore")  # some columns of the set go non-physical (NaN) within the sample
    from oracle import eos
    from oracle import lbm as olbm
    from paper_2301_12869_gb300 import inputs

    _, Tc, _ = eos.critical_point(A, B, R)
    if task[0] == "small":
        rv, rl, _ = eos.maxwell(0.85 * Tc, A, B, R)
        f = olbm.init_state(inputs.column_rho0(4, 200, rl, rv, 100, width=5.0))
        p = olbm.Params(nx=4, ny=200, a=A, b=B, R=R, T=0.85 * Tc, g=(0.0, -2e-5), form=1)
        nodes = 800
    else:
        c = inputs.batched_columns(task[1] + 1, seed=SEED)[task[1]]
        T = c["Tr"] * Tc
        rv, rl, _ = eos.maxwell(T, A, B, R)
        ny = c["ny"]
        f = olbm.init_state(inputs.column_rho0(4, ny, rl, rv, max(1, int(round(c["liquid_fraction"] * ny)))))
        p = olbm.Params(nx=4, ny=ny, a=A, b=B, R=R, T=T, g=(0.0, c["gy"]), form=c["form"])
        nodes = 4 * ny
    steps = task[-1]
    t0 = time.perf_counter()
    olbm.run(f, p, steps)
    return nodes * steps, time.perf_counter() - t0


def cpu_oracle_pool(small_steps=20000, columns=64, column_steps=1000):
    """The FP64 oracle on all host cores at once (a spawned process pool, one thread per
    process, spawned before any GPU work): the 4 x 200 column in full (20 000 steps) as one
    task and `column_steps` steps of each of the first `columns` columns of the seeded
    batched set (heights 64..1024) as the others. Returns the all-core throughput, the
    single-process rates and the 4 x 200 column's time."""
    import multiprocessing as mp

    cores = os.cpu_count() or 1
    tasks = [("small", small_steps)] + [("column", i, column_steps) for i in range(columns)]
    ctx = mp.get_context("spawn")
    t0 = time.perf_counter()
    with ctx.Pool(cores) as pool:
        res = pool.map_async(_oracle_task, tasks, chunksize=1).get(timeout=600)
    wall = time.perf_counter() - t0
    col_units = sum(u for u, _ in res[1:])
    col_secs = sum(t for _, t in res[1:])
    return {
        "cores": cores, "wall_s": wall,
        "all_cores_mlups": sum(u for u, _ in res) / wall / 1e6,
        "columns_one_process_mlups": col_units / col_secs / 1e6,
        "small_column_seconds": res[0][1], "small_column_us_per_step": 1e6 * res[0][1] / small_steps,
        "sample": f"{len(tasks)} tasks on {cores} processes: the 4x200 FP64 column for {small_steps} steps "
                  f"(config 1 in full) and {column_steps} steps of each of the first {columns} columns of the "
                  "seeded batched set (config 3)",
    }


def cpu_baseline_entry(ny_slice=512, steps=60):
    mlups, res = time_oracle(ny_slice, steps)
    entry = {
        "value": mlups, "unit": "MLUPS", "cores": 1, "kind": "oracle",
        "sample": f"{steps} FP64 oracle steps on a {NX}x{ny_slice} slice of the workload around the interface "
                  f"({res['seconds']:.1f} s, numpy, 1 thread)",
    }
    try:
        entry["all_cores"] = cpu_oracle_pool()
    except Exception as exc:  # noqa: BLE001 - reported, not hidden
        entry["all_cores"] = {"error": str(exc)}
    return entry


# ---------------------------------------------------------------- distributed helpers
def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def reduce_over_ranks(torch, values, op="max"):
    """All-reduce a list of floats over ranks (max or sum); identity when not distributed."""
    import torch.distributed as dist

    if not (dist.is_available() and dist.is_initialized()):
        return list(values)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor(list(values), dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX if op == "max" else dist.ReduceOp.SUM)
    return [float(v) for v in t.cpu()]


def aggregate(local_ms, local_units, torch):
    """Whole-job throughput: all ranks' units divided by the slowest rank's time."""
    ms = reduce_over_ranks(torch, [local_ms], "max")[0]
    units = reduce_over_ranks(torch, [local_units], "sum")[0]
    return ms, units


# ---------------------------------------------------------------- end to end
def run_e2e(args, rho0, Tc, nodes, world, torch, lbm, snapshot):
    """The same metric through the public C ABI with host buffers: lbm_init from pinned
    host rho0 (host-to-device copy and the initial state inside), K steps (the same
    restores as the device-timed run), lbm_moments of rho to pinned host memory and
    lbm_reduce(MASS). The handle's device workspace is allocated once before the timed
    region (lbm_workspace_bytes, a torch buffer passed as p->workspace), as a user who
    runs many jobs allocates it once. Timed on the host clock around the synchronous
    calls."""
    pinned = torch.empty((NY, NX), dtype=torch.float64, pin_memory=True)
    pinned.copy_(torch.from_numpy(rho0))
    rho_h = torch.empty((NY, NX), dtype=torch.float64, pin_memory=True)
    pe = lbm.make_params(NX, NY, TR * Tc, args.precision, a=A, b=B, R=R, form=2, g=(0.0, GY))
    nbytes = lbm.lbm_workspace_bytes(pe)
    ws = torch.empty(nbytes + 256, dtype=torch.uint8, device="cuda")
    pe.workspace = (ws.data_ptr() + 255) // 256 * 256
    pe.workspace_bytes = nbytes
    stream = torch.cuda.current_stream().cuda_stream
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h = lbm.lbm_init(pe, pinned.numpy(), stream)
    run_steps(lbm, h, args.steps, snapshot)
    lbm.lbm_moments(h, rho_h.numpy())
    mass = lbm.lbm_reduce(h, lbm.LBM_REDUCE_MASS)[0]
    t1 = time.perf_counter()
    lbm.lbm_destroy(h)
    del ws
    ms, units = aggregate((t1 - t0) * 1e3, float(nodes) * args.steps, torch)
    return {
        "value": units / (ms / 1e3) / 1e6, "unit": "MLUPS", "h2d_bytes_per_step": 8 * nodes / args.steps,
        "d2h_bytes_per_step": (8 * nodes + 8) / args.steps, "mass": mass, "seconds": (t1 - t0),
        "what": "lbm_init from pinned host rho0 + K steps + lbm_moments(rho) to pinned host + lbm_reduce(MASS), "
                "workspace allocated before the timed region, host clock",
    }


# ---------------------------------------------------------------- FP32 against FP64 on the domain
PRECISION_STEPS = 400  # inside the workload's physical window (~500 steps)


def precision_report(lbm, rho0, Tc, steps=PRECISION_STEPS, every=100):
    """The FP32 path against the FP64 GPU run of the same workload and initial state (the
    FP64 run matches the FP64 oracle to 1e-12, tests/test_gpu_parity.py): every `every`
    steps, max |rho_32 - rho_64| over the domain, the interface height (first crossing of the
    coexistence midpoint by the x-averaged profile, LBM_REDUCE_INTERFACE_Y) and the liquid /
    vapour densities (max / min of that profile, LBM_REDUCE_RHO_LV) of both."""
    import numpy as np

    hs = {}
    for prec in ("fp32", "fp64"):
        q = lbm.make_params(NX, NY, TR * Tc, prec, a=A, b=B, R=R, form=2, g=(0.0, GY))
        hs[prec] = lbm.lbm_init(q, rho0)
    rows = []
    try:
        rho = {k: np.empty((NY, NX)) for k in hs}
        done = 0
        while done < steps:
            n = min(every, steps - done)
            for h in hs.values():
                lbm.lbm_step(h, n)
            done += n
            row = {"step": done}
            for k, h in hs.items():
                lbm.lbm_moments(h, rho[k])
                row[f"interface_{k}"] = lbm.lbm_reduce(h, lbm.LBM_REDUCE_INTERFACE_Y)[0]
                row[f"rho_l_{k}"], row[f"rho_v_{k}"] = lbm.lbm_reduce(h, lbm.LBM_REDUCE_RHO_LV)[:2]
                row[f"status_{k}"] = lbm.lbm_status(h)
            row["max_abs_drho"] = float(np.max(np.abs(rho["fp32"] - rho["fp64"])))
            row["interface_error"] = row["interface_fp32"] - row["interface_fp64"]
            row["rho_l_rel_error"] = row["rho_l_fp32"] / row["rho_l_fp64"] - 1.0
            row["rho_v_rel_error"] = row["rho_v_fp32"] / row["rho_v_fp64"] - 1.0
            rows.append(row)
    finally:
        for h in hs.values():
            lbm.lbm_destroy(h)
    return {"what": "FP32 populations (FP64 reductions) against the FP64 GPU run, same initial state",
            "steps": steps, "samples": rows,
            "max_abs_drho": max(r["max_abs_drho"] for r in rows),
            "max_abs_interface_error": max(abs(r["interface_error"]) for r in rows),
            "max_abs_rho_l_rel_error": max(abs(r["rho_l_rel_error"]) for r in rows),
            "max_abs_rho_v_rel_error": max(abs(r["rho_v_rel_error"]) for r in rows)}


# ---------------------------------------------------------------- the domain as slabs (N GPUs)
def run_slabs(args, torch, lbm, inputs, world, rank, local, rho0, Tc):
    """One liquid column cut into `world` slabs of rows, one per GPU. Weak scaling (the
    default): every rank holds a 1024 x 4096 slab of a 1024 x 4096 N column, liquid in its
    lower half; strong scaling (--slab-scaling strong): the 1024 x 4096 column itself is
    cut. Per step each rank runs the fused step on its rows (lbm_slab_step), then sums the
    column's mass over ranks (NCCL all-reduce of one double, for <rho> of Eq. Gravity_2)
    and swaps 2 ghost rows x 9 planes with each neighbour (NCCL send / receive). Returns
    (local ms, local node updates, restores, per-step bytes exchanged, end-to-end dict or
    None, status, the rank's slab, the column's rows)."""
    import numpy as np

    from paper_2301_12869_gb300 import partition

    weak = args.slab_scaling == "weak"
    ny_total = NY * world if weak else NY
    if weak and world > 1:
        rv, rl, _ = lbm.lbm_coexistence(A, B, R, TR * Tc)
        rho0 = inputs.column_rho0(NX, ny_total, rl, rv, LIQUID_ROWS * world, noise_amp=NOISE, seed=SEED)
    rho_ref = float(rho0.mean()) if args.precision == "fp32" else 0.0
    p = lbm.make_params(NX, ny_total, TR * Tc, args.precision, a=A, b=B, R=R, form=2, g=(0.0, GY), rho_ref=rho_ref)
    plan = partition.SlabPlan(ny_total, world)
    sl = plan[rank]
    if world > 1:
        import torch.distributed as dist

        comm = partition.TorchComm(dist)
    else:
        comm = partition.SingleComm()
    own = np.ascontiguousarray(rho0[sl.y0:sl.y0 + sl.ny_own])
    lat = partition.SlabLattice(p, sl, torch.from_numpy(own).cuda(), comm)
    lat.step(args.warmup)
    snap = lat.snapshot()
    stream = torch.cuda.current_stream()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    start.record(stream)
    done = restores = 0
    while done < args.steps:
        n = min(WINDOW, args.steps - done)
        lat.step(n)
        done += n
        if done < args.steps:
            lat.restore(snap)
            restores += 1
    end.record(stream)
    torch.cuda.synchronize()
    if world > 1:
        torch.distributed.barrier()
    local_ms = start.elapsed_time(end)
    status = lat.status_code()
    del lat, snap
    torch.cuda.empty_cache()
    # end to end: this rank's rows of rho0 from pinned host memory, the slab's set-up and K
    # steps, the domain's mass read back to the host
    e2e = None
    if not args.no_e2e:
        pinned = torch.empty(own.shape, dtype=torch.float64, pin_memory=True)
        pinned.copy_(torch.from_numpy(own))
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lat = partition.SlabLattice(p, sl, pinned.cuda(non_blocking=True), comm)
        lat.step(args.steps)
        mass = lat.mass + rho_ref * NX * ny_total
        t1 = time.perf_counter()
        ms_e, units_e = aggregate((t1 - t0) * 1e3, float(NX * sl.ny_own) * args.steps, torch)
        e2e = {"value": units_e / (ms_e / 1e3) / 1e6, "unit": "MLUPS",
               "h2d_bytes_per_step": 8 * NX * ny_total / args.steps,
               "d2h_bytes_per_step": 8 * world / args.steps, "mass": mass,
               "what": "each rank: its rows of rho0 from pinned host memory, slab set-up, K steps with the "
                       "exchanges, the domain mass to the host; host clock, max over ranks"}
        del lat
    halo_bytes = 2 * 2 * partition.HALO * 9 * NX * (4 if args.precision == "fp32" else 8)
    return local_ms, float(NX * sl.ny_own) * args.steps, restores, halo_bytes, e2e, status, sl, ny_total


# ---------------------------------------------------------------- batched columns
# FP32 phase of the FP32 -> FP64 runs: each column runs in FP32 to --fp32-tol, or until
# --fp32-stall checks below the FP32 floor region bring no 1 % gain, then hands over to FP64
FP32_TOL, FP32_STALL_CHECKS = 1e-8, 50
# extrapolation (lbm_batch_set_acceleration) of the FP32 -> FP64 runs: every ACCEL_CHECKS
# residual checks; the plain FP64 reference runs without it
ACCEL_CHECKS = 5


def column_set(n, seed, heights, lbm, inputs):
    """n seeded 4 x H columns of the batched generator with H in heights: descriptors and
    the concatenated tanh initial densities."""
    import numpy as np

    gen = [c for c in inputs.batched_columns(4 * n, seed=seed) if c["ny"] in heights][:n]
    _, Tc, _ = lbm.lbm_critical_point(A, B, R)
    cols, rhos = [], []
    for c in gen:
        T = c["Tr"] * Tc
        rv, rl, _ = lbm.lbm_coexistence(A, B, R, T)
        rhos.append(inputs.column_rho0(4, c["ny"], rl, rv, max(1, int(round(c["liquid_fraction"] * c["ny"])))))
        cols.append(dict(ny=c["ny"], T=T, gy=c["gy"], form=c["form"]))
    return cols, np.concatenate([r.ravel() for r in rhos])


TUNE_STEPS = 200  # steps per candidate block size of the batched kernel's autotuner


def run_to_steady(lbm, cols, rho0, cap, fp32_first, tuned=None, rest=False):
    """FP64 alone, or FP32 until each column reaches FP32_TOL or its FP32 rounding floor (no
    1 % gain in FP32_STALL_CHECKS checks) then double-float (FP32-pair) arithmetic from that
    state, to residual 1e-10 (checked every 100 steps). The populations start at the rest
    equilibrium f_eq(rho0, 0), or with rest=True at the rest state of rho0 (lbm_batch_rest_state,
    timed with the run). Each batch's block size comes from lbm_batch_autotune (its
    timing runs on a copy of the batch, outside the timed runs); the choices and timings go
    into `tuned`. Returns (device seconds, steps, residual, status, batch)."""
    import torch

    _, Tc, _ = lbm.lbm_critical_point(A, B, R)
    tuned = {} if tuned is None else tuned
    t_rest = 0.0

    def rest_state(batch):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        lbm.lbm_batch_rest_state(batch)
        return time.perf_counter() - t0

    if fp32_first:
        b32 = lbm.lbm_batch_init(lbm.make_params(4, 8, 0.8 * Tc, "fp32", a=A, b=B, R=R), cols, rho0)
        if rest:
            t_rest = rest_state(b32)
        tuned["fp32"] = lbm.lbm_batch_autotune(b32, TUNE_STEPS)
        lbm.lbm_batch_set_acceleration(b32, ACCEL_CHECKS)
        t32 = lbm.lbm_batch_run_stall(b32, FP32_TOL, cap, 100, FP32_STALL_CHECKS)
        b = lbm.lbm_batch_convert(b32, lbm.LBM_DOUBLE_FLOAT)
        lbm.lbm_batch_destroy(b32)
        tuned["dd_after_fp32"] = lbm.lbm_batch_autotune(b, TUNE_STEPS)
        lbm.lbm_batch_set_acceleration(b, ACCEL_CHECKS)
    else:
        t32 = 0.0
        b = lbm.lbm_batch_init(lbm.make_params(4, 8, 0.8 * Tc, "fp64", a=A, b=B, R=R), cols, rho0)
        if rest:
            t_rest = rest_state(b)
        tuned["fp64"] = lbm.lbm_batch_autotune(b, TUNE_STEPS)
    t64 = lbm.lbm_batch_run(b, 1e-10, cap, 100)
    st, res, status = lbm.lbm_batch_results(b, len(cols), check=False)
    return t_rest + t32 + t64, st, res, status, b


def tuned_summary(tuned):
    """{batch: {"threads": kept, "us_per_step": {candidate: us}}} of the autotuner's results."""
    return {k: {"threads": v[0], "us_per_step": {str(t): round(u, 2) for t, u in v[1].items()}}
            for k, v in tuned.items()}


def run_columns(args):
    """Time to steady state of independent liquid columns (the batched workload): seeded
    4 x H columns from the batched-column generator (T/T_c ~ U[0.70, 0.95], |g| log-uniform
    in [1e-6, 1e-4], either gravity form, liquid fraction ~ U[0.3, 0.7]) restricted to the
    heights in --column-heights, each run to max |rho_t - rho_(t-1)| <= 1e-10 (checked every
    100 steps): plain FP64 against FP32 down to its rounding floor (~1e-8; the residual is
    evaluated in FP64) followed, from that state, by FP64 or by double-float (FP32-pair)
    arithmetic. `value` is the FP32 + double-float time."""
    import numpy as np

    from paper_2301_12869_gb300 import inputs, lbm

    heights = tuple(int(h) for h in args.column_heights.split(","))
    cols, rho = column_set(args.columns, SEED, heights, lbm, inputs)
    _, Tc, _ = lbm.lbm_critical_point(A, B, R)
    nodes = rho.size
    cap = args.column_max_steps
    out = {}
    tuned = {}
    p64 = lbm.make_params(4, 8, 0.8 * Tc, "fp64", a=A, b=B, R=R)
    b64 = lbm.lbm_batch_init(p64, cols, rho)
    tuned["fp64_plain"] = lbm.lbm_batch_autotune(b64, TUNE_STEPS)
    t64 = lbm.lbm_batch_run(b64, 1e-10, cap, 100)
    st64, res64, s64 = lbm.lbm_batch_results(b64, len(cols), check=False)
    lbm.lbm_batch_destroy(b64)
    p32 = lbm.make_params(4, 8, 0.8 * Tc, "fp32", a=A, b=B, R=R)
    b32 = lbm.lbm_batch_init(p32, cols, rho)
    tuned["fp32"] = lbm.lbm_batch_autotune(b32, TUNE_STEPS)
    lbm.lbm_batch_set_acceleration(b32, ACCEL_CHECKS)
    t32 = lbm.lbm_batch_run_stall(b32, FP32_TOL, cap, 100, FP32_STALL_CHECKS)
    st32, _, _ = lbm.lbm_batch_results(b32, len(cols), check=False)
    bc = lbm.lbm_batch_convert(b32, lbm.LBM_FP64)
    bd = lbm.lbm_batch_convert(b32, lbm.LBM_DOUBLE_FLOAT)
    lbm.lbm_batch_destroy(b32)
    tuned["fp64_after_fp32"] = lbm.lbm_batch_autotune(bc, TUNE_STEPS)
    lbm.lbm_batch_set_acceleration(bc, ACCEL_CHECKS)
    tpol = lbm.lbm_batch_run(bc, 1e-10, cap, 100)
    stc, resc, sc = lbm.lbm_batch_results(bc, len(cols), check=False)
    rc_ = np.empty(nodes)
    lbm.lbm_batch_moments(bc, rho=rc_)
    lbm.lbm_batch_destroy(bc)
    # the same FP32 state finished in double-float (FP32-pair) arithmetic instead of FP64
    tuned["dd_after_fp32"] = lbm.lbm_batch_autotune(bd, TUNE_STEPS)
    lbm.lbm_batch_set_acceleration(bd, ACCEL_CHECKS)
    tdd = lbm.lbm_batch_run(bd, 1e-10, cap, 100)
    std_, resd, sd = lbm.lbm_batch_results(bd, len(cols), check=False)
    rd_ = np.empty(nodes)
    lbm.lbm_batch_moments(bd, rho=rd_)
    lbm.lbm_batch_destroy(bd)
    ok64 = (res64 <= 1e-10) & (s64 == 0)
    okc = (resc <= 1e-10) & (sc == 0)
    okd = (resd <= 1e-10) & (sd == 0)
    both = ok64 & okc
    offs = np.cumsum([0] + [4 * c["ny"] for c in cols])
    dd_vs_fp64 = np.array([np.max(np.abs(rd_[offs[i]:offs[i + 1]] - rc_[offs[i]:offs[i + 1]]))
                           for i in np.nonzero(okc & okd)[0]])
    out = {
        "metric": "time to steady state (residual 1e-10), batched columns", "unit": "s",
        "value": t32 + tdd, "higher_is_better": False, "impl": "gb300", "n_gpus": 1,
        "config": {"workload": f"{len(cols)} seeded 4xH liquid columns, H in {heights}", "nodes": nodes,
                   "max_steps": cap, "check_every": 100, "fp32_tol": FP32_TOL, "fp32_stall_checks": FP32_STALL_CHECKS,
                   "accel_checks": ACCEL_CHECKS},
        "fp64_plain": {"seconds": t64, "converged": int(ok64.sum()), "nonphysical": int((s64 != 0).sum()),
                       "node_steps_per_s": float(np.sum(st64 * [4 * c["ny"] for c in cols]) / t64)},
        "fp32_then_fp64": {"seconds": t32 + tpol, "fp32_seconds": t32, "fp64_seconds": tpol,
                           "converged": int(okc.sum()), "nonphysical": int((sc != 0).sum()),
                           "speedup_vs_fp64": t64 / (t32 + tpol)},
        "fp32_then_double_float": {"seconds": t32 + tdd, "fp32_seconds": t32, "double_float_seconds": tdd,
                                   "converged": int(okd.sum()), "nonphysical": int((sd != 0).sum()),
                                   "speedup_vs_fp64": t64 / (t32 + tdd),
                                   "max_rho_difference_vs_fp32_then_fp64": {
                                       "median": float(np.median(dd_vs_fp64)) if dd_vs_fp64.size else None,
                                       "max": float(np.max(dd_vs_fp64)) if dd_vs_fp64.size else None}},
        "speedup_vs_fp64": t64 / (t32 + tdd),
        "steps_ratio_converged": float(np.sum(stc[both]) / max(1, np.sum(st64[both]))),
        "block_threads": tuned_summary(tuned),
    }
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------- time to steady state (default line)
STEADY_HEIGHTS = (64, 128, 256, 512, 1024)
# the warm-start network of that block: trained on 16384 steady columns of another seed with
# the heights whose columns converge within the step cap
WARM_TRAIN_COLUMNS, WARM_HEIGHTS, WARM_ITERS = 16384, (64, 128), 12000


def column_stats(rho, cols, lbm):
    """Per column of a concatenated density field (4 x H columns): the x-averaged profile's
    first crossing of the coexistence midpoint at the column's T (interface height), its
    max (liquid) and min (vapour)."""
    import numpy as np

    out = np.full((len(cols), 3), np.nan)
    off = 0
    for c, col in enumerate(cols):
        n = 4 * col["ny"]
        prof = rho[off:off + n].reshape(col["ny"], 4).mean(axis=1)
        off += n
        rv, rl, _ = lbm.lbm_coexistence(A, B, R, col["T"])
        d = prof - 0.5 * (rv + rl)
        with np.errstate(all="ignore"):  # a non-physical column's profile may be NaN or huge
            k = np.nonzero(d[:-1] * d[1:] <= 0.0)[0]
        k = k[d[k] != d[k + 1]]
        if k.size:
            y = int(k[0])
            out[c, 0] = y + d[y] / (d[y] - d[y + 1])
        out[c, 1], out[c, 2] = prof.max(), prof.min()
    return out


def _path_summary(seconds, steps, res, status, col_sec, cols, ok):
    import numpy as np

    hs = np.array([c["ny"] for c in cols])
    by_h = {}
    for H in sorted(set(hs.tolist())):
        m = hs == H
        mk = m & ok
        by_h[str(H)] = {"columns": int(m.sum()), "converged": int(mk.sum()),
                        "median_steps": float(np.median(steps[mk])) if mk.any() else None,
                        "median_seconds": float(np.median(col_sec[mk])) if mk.any() else None}
    return {"makespan_s": seconds, "converged": int(ok.sum()), "columns": len(cols),
            "nonphysical": int((status != 0).sum()),
            "median_steps_converged": float(np.median(steps[ok])) if ok.any() else None,
            "median_column_seconds_converged": float(np.median(col_sec[ok])) if ok.any() else None,
            "by_height": by_h}


def _error_summary(stats, ref, rho, rho_ref, cols, mask):
    """Per-column errors of a path's densities against the FP64 run's (columns in mask)."""
    import numpy as np

    off = np.cumsum([0] + [4 * c["ny"] for c in cols])
    dmax = np.array([np.max(np.abs(rho[off[i]:off[i + 1]] - rho_ref[off[i]:off[i + 1]])) for i in range(len(cols))])
    both = mask & np.isfinite(stats[:, 0]) & np.isfinite(ref[:, 0])
    def q(v, m):
        return {"median": float(np.median(v[m])), "max": float(np.max(v[m]))} if m.any() else None
    return {"columns": int(mask.sum()), "max_abs_drho": q(dmax, mask),
            "abs_interface_error": q(np.abs(stats[:, 0] - ref[:, 0]), both),
            "rho_l_rel_error": q(np.abs(stats[:, 1] / ref[:, 1] - 1.0), mask),
            "rho_v_rel_error": q(np.abs(stats[:, 2] / ref[:, 2] - 1.0), mask)}


def time_to_steady(args, lbm, inputs, world, rank, torch):
    """Time to steady state (residual max |rho_t - rho_(t-1)| <= 1e-10, checked every 100
    steps) of the batched 4 x H columns with the heights, temperatures, gravities and forms
    of the batched workload: plain FP64 against FP32 down to its rounding floor then
    double-float (FP32-pair) arithmetic, both capped at args.steady_cap steps per phase.
    With N ranks every rank runs its share of the columns (partition.column_shares, no
    exchange); makespans are the max over ranks. Per column: the device seconds its CTA
    spent on it (lbm_batch_column_seconds) and its steps; the FP32 phase's end state and
    the final double-float state against the FP64 run's: max |drho|, interface height,
    liquid and vapour densities."""
    import numpy as np

    from paper_2301_12869_gb300 import partition

    cols_all, rho_all = column_set(args.steady_columns, SEED, STEADY_HEIGHTS, lbm, inputs)
    offs = np.cumsum([0] + [4 * c["ny"] for c in cols_all])
    share = partition.column_shares([c["ny"] for c in cols_all], world)[rank]
    cols = [cols_all[i] for i in share]
    rho = np.concatenate([rho_all[offs[i]:offs[i + 1]] for i in share])
    n, cap = len(cols), args.steady_cap
    _, Tc, _ = lbm.lbm_critical_point(A, B, R)
    tuned = {}
    # plain FP64
    b = lbm.lbm_batch_init(lbm.make_params(4, 8, 0.8 * Tc, "fp64", a=A, b=B, R=R), cols, rho)
    tuned["fp64"] = lbm.lbm_batch_autotune(b, TUNE_STEPS)
    t64 = lbm.lbm_batch_run(b, 1e-10, cap, 100)
    st64, res64, s64 = lbm.lbm_batch_results(b, n, check=False)
    sec64 = lbm.lbm_batch_column_seconds(b, n)
    rho64 = np.empty(rho.size)
    lbm.lbm_batch_moments(b, rho=rho64)
    lbm.lbm_batch_destroy(b)
    # FP32 to its floor, then double-float
    b32 = lbm.lbm_batch_init(lbm.make_params(4, 8, 0.8 * Tc, "fp32", a=A, b=B, R=R), cols, rho)
    tuned["fp32"] = lbm.lbm_batch_autotune(b32, TUNE_STEPS)
    lbm.lbm_batch_set_acceleration(b32, ACCEL_CHECKS)
    t32 = lbm.lbm_batch_run_stall(b32, FP32_TOL, cap, 100, FP32_STALL_CHECKS)
    st32, res32, s32 = lbm.lbm_batch_results(b32, n, check=False)
    rho32 = np.empty(rho.size)
    lbm.lbm_batch_moments(b32, rho=rho32)
    bd = lbm.lbm_batch_convert(b32, lbm.LBM_DOUBLE_FLOAT)
    lbm.lbm_batch_destroy(b32)
    tuned["dd_after_fp32"] = lbm.lbm_batch_autotune(bd, TUNE_STEPS)
    lbm.lbm_batch_set_acceleration(bd, ACCEL_CHECKS)
    tdd = lbm.lbm_batch_run(bd, 1e-10, cap, 100)
    stdd, resdd, sdd = lbm.lbm_batch_results(bd, n, check=False)
    secdd = lbm.lbm_batch_column_seconds(bd, n)  # FP32 + double-float phases of each column
    rhodd = np.empty(rho.size)
    lbm.lbm_batch_moments(bd, rho=rhodd)
    lbm.lbm_batch_destroy(bd)
    # FP32 then double-float from the warm start: the network (trained here, on the GPU, on the
    # steady columns of another seed) gives the profile of the columns of the heights it was
    # trained on, the tanh profile stays for the others; every column then starts from the
    # rest state of its profile (lbm_batch_rest_state). Timed: inference, rest state, both
    # phases; the training is a one-off cost, reported beside it.
    net, train = train_warm_network(lbm, inputs, torch, WARM_TRAIN_COLUMNS, WARM_HEIGHTS, cap, WARM_ITERS, 8192,
                                    SEED + 1)
    lo = np.cumsum([0] + [4 * c["ny"] for c in cols])
    sel = [i for i, c in enumerate(cols) if c["ny"] in WARM_HEIGHTS]
    rho_w = torch.from_numpy(rho).cuda()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if sel:
        sub = [cols[i] for i in sel]
        pred = torch.empty(sum(4 * c["ny"] for c in sub), dtype=torch.float64, device="cuda")
        lbm.lbm_mlp_warm_start(net, sub, 4, A, B, R, np.array([rho[lo[i]:lo[i + 1]].mean() for i in sel]), pred)
        po = 0
        for i, c in zip(sel, sub):
            rho_w[lo[i]:lo[i + 1]] = pred[po:po + 4 * c["ny"]]
            po += 4 * c["ny"]
    torch.cuda.synchronize()
    t_inf = time.perf_counter() - t0
    lbm.lbm_mlp_destroy(net)
    bw = lbm.lbm_batch_init(lbm.make_params(4, 8, 0.8 * Tc, "fp32", a=A, b=B, R=R), cols, rho_w)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbm.lbm_batch_rest_state(bw)
    t_rest = time.perf_counter() - t0
    tuned["fp32_warm"] = lbm.lbm_batch_autotune(bw, TUNE_STEPS)
    lbm.lbm_batch_set_acceleration(bw, ACCEL_CHECKS)
    tw32 = lbm.lbm_batch_run_stall(bw, FP32_TOL, cap, 100, FP32_STALL_CHECKS)
    bwd = lbm.lbm_batch_convert(bw, lbm.LBM_DOUBLE_FLOAT)
    lbm.lbm_batch_destroy(bw)
    tuned["dd_after_fp32_warm"] = lbm.lbm_batch_autotune(bwd, TUNE_STEPS)
    lbm.lbm_batch_set_acceleration(bwd, ACCEL_CHECKS)
    twdd = lbm.lbm_batch_run(bwd, 1e-10, cap, 100)
    stw, resw, sw = lbm.lbm_batch_results(bwd, n, check=False)
    secw = lbm.lbm_batch_column_seconds(bwd, n)
    rhow = np.empty(rho.size)
    lbm.lbm_batch_moments(bwd, rho=rhow)
    lbm.lbm_batch_destroy(bwd)
    local = dict(idx=share, cols=cols, t64=t64, t32=t32, tdd=tdd, st64=st64, res64=res64, s64=s64, sec64=sec64,
                 st32=st32, s32=s32, stdd=stdd, resdd=resdd, sdd=sdd, secdd=secdd,
                 tw=t_inf + t_rest + tw32 + twdd, tw32=tw32, stw=stw, resw=resw, sw=sw, secw=secw, train=train,
                 warm_columns=len(sel), t_inf=t_inf, t_rest=t_rest,
                 stats64=column_stats(rho64, cols, lbm), stats32=column_stats(rho32, cols, lbm),
                 statsdd=column_stats(rhodd, cols, lbm), statsw=column_stats(rhow, cols, lbm), tuned=tuned)
    ok64 = (res64 <= 1e-10) & (s64 == 0)
    okdd = (resdd <= 1e-10) & (sdd == 0)
    local["prec32"] = _error_summary(local["stats32"], local["stats64"], rho32, rho64, cols, ok64 & (s32 == 0))
    local["precdd"] = _error_summary(local["statsdd"], local["stats64"], rhodd, rho64, cols, ok64 & okdd)
    okw = (resw <= 1e-10) & (sw == 0)
    local["precw"] = _error_summary(local["statsw"], local["stats64"], rhow, rho64, cols, ok64 & okw)
    if world > 1:
        import torch.distributed as dist

        gathered = [None] * world
        dist.all_gather_object(gathered, {k: v for k, v in local.items()})
    else:
        gathered = [local]
    if rank != 0:
        return None
    cat = lambda k: np.concatenate([g[k] for g in gathered])  # noqa: E731
    cols_g = [c for g in gathered for c in g["cols"]]
    T64 = max(g["t64"] for g in gathered)
    T32DD = max(g["t32"] + g["tdd"] for g in gathered)
    ok64 = (cat("res64") <= 1e-10) & (cat("s64") == 0)
    okdd = (cat("resdd") <= 1e-10) & (cat("sdd") == 0)
    both = ok64 & okdd
    sec64, secdd = cat("sec64"), cat("secdd")
    TW = max(g["tw"] for g in gathered)
    okw = (cat("resw") <= 1e-10) & (cat("sw") == 0)
    secw = cat("secw")
    all3 = ok64 & okw
    out = {
        "what": "time to residual 1e-10 of batched 4xH columns: plain FP64 vs FP32 then double-float, "
                "without and with the warm start",
        "workload": f"{len(cols_g)} seeded 4xH liquid columns, H in {STEADY_HEIGHTS}, step cap {args.steady_cap} per phase",
        "ranks": world, "partition": "disjoint column sets balanced by nodes, no exchange" if world > 1 else None,
        "check_every": 100, "fp32_tol": FP32_TOL, "fp32_stall_checks": FP32_STALL_CHECKS, "accel_checks": ACCEL_CHECKS,
        "fp64_plain": _path_summary(T64, cat("st64"), cat("res64"), cat("s64"), sec64, cols_g, ok64),
        "fp32_then_double_float": _path_summary(T32DD, cat("stdd"), cat("resdd"), cat("sdd"), secdd, cols_g, okdd)
        | {"fp32_makespan_s": max(g["t32"] for g in gathered)},
        "fp32_then_double_float_warm_start": _path_summary(TW, cat("stw"), cat("resw"), cat("sw"), secw, cols_g, okw)
        | {"fp32_makespan_s": max(g["tw32"] for g in gathered), "warm_started_columns": sum(g["warm_columns"] for g in gathered),
           "start": f"network profile for H in {WARM_HEIGHTS} (tanh for the others), every column from the rest "
                    "state of its profile", "inference_s": max(g["t_inf"] for g in gathered),
           "rest_state_s": max(g["t_rest"] for g in gathered), "training (not timed)": gathered[0]["train"]},
        "makespan_speedup": T64 / T32DD,
        "makespan_speedup_warm_start": T64 / TW,
        "converged_in_plain_and_warm": int(all3.sum()),
        "median_column_speedup_warm_start": float(np.median(sec64[all3] / secw[all3])) if all3.any() else None,
        "steps_ratio_warm_start_vs_plain_fp64": float(np.sum(cat("stw")[all3]) / max(1, np.sum(cat("st64")[all3]))),
        "converged_in_both": int(both.sum()),
        "median_column_seconds_both": {"fp64_plain": float(np.median(sec64[both])) if both.any() else None,
                                       "fp32_then_double_float": float(np.median(secdd[both])) if both.any() else None},
        "median_column_speedup_both": float(np.median(sec64[both] / secdd[both])) if both.any() else None,
        "precision_vs_fp64": {"fp32_end_of_phase": gathered[0]["prec32"] if world == 1 else [g["prec32"] for g in gathered],
                              "fp32_then_double_float": gathered[0]["precdd"] if world == 1 else [g["precdd"] for g in gathered],
                              "fp32_then_double_float_warm_start": gathered[0]["precw"] if world == 1 else [g["precw"] for g in gathered]},
        "block_threads": tuned_summary(gathered[0]["tuned"]),
    }
    return out


# ---------------------------------------------------------------- thermal variant
TH_NX, TH_NY, TH_LIQUID = 512, 2048, 1024
TH_TBOT, TH_TTOP, TH_GY = 0.95, 0.80, -5e-5
# per node and step, as launched: fused step 72 B populations + 4 B T read, 12 B rho/u
# written; Heun kernel 4 B T + 12 B rho/u read, 4 B T written (FP32 storage, rho and u
# handed over as floats; FP64 storage doubles every term)
TH_BYTES_PER_NODE = {"fp32": 88 + 20, "fp64": 176 + 40}
# The heated column goes non-physical: its 1024 vapour rows weigh more than the vapour's
# saturation pressure can carry at g_y = -5e-5 (scale height of the vapour ~100 rows), so
# the vapour falls freely and the top empties (max |u| = |g| t) within ~5000 steps. Timed
# runs restore the post-warm-up populations and temperature every TH_WINDOW steps.
TH_WINDOW = 1000


def thermal_setup(precision, lbm, inputs):
    _, Tc, _ = lbm.lbm_critical_point(A, B, R)
    T_mid = TH_TBOT + (TH_TTOP - TH_TBOT) * TH_LIQUID / TH_NY  # conduction profile at the interface
    rv, rl, _ = lbm.lbm_coexistence(A, B, R, T_mid * Tc)
    rho0 = inputs.column_rho0(TH_NX, TH_NY, rl, rv, TH_LIQUID, noise_amp=NOISE, seed=SEED)
    p = lbm.make_params(TH_NX, TH_NY, T_mid * Tc, precision, a=A, b=B, R=R, form=1, g=(0.0, TH_GY), thermal=1,
                        T_bot=TH_TBOT * Tc, T_top=TH_TTOP * Tc)
    return p, rho0, Tc


_LEVELS = {}


def coexistence_midpoint(lbm, T, Tc):
    """(rho_l + rho_v)/2 of the Maxwell rule at T, interpolated from 400 temperatures."""
    import numpy as np

    if "T" not in _LEVELS:
        grid = np.linspace(0.70, 0.999, 400) * Tc
        _LEVELS["T"] = grid
        _LEVELS["mid"] = np.array([0.5 * sum(lbm.lbm_coexistence(A, B, R, t)[:2]) for t in grid])
    return np.interp(T, _LEVELS["T"], _LEVELS["mid"])


def crossing_heights(lbm, h, Tc):
    """Heights (from the bottom wall, linear interpolation of the x-averaged profiles) where
    rho crosses the level halfway between the coexistence densities at the row's mean T:
    the first is the top of the liquid at the bottom wall (the nucleation height once a
    vapour layer forms there)."""
    import numpy as np

    rho = np.empty((TH_NY, TH_NX))
    T = np.empty((TH_NY, TH_NX))
    lbm.lbm_moments(h, rho)
    lbm.lbm_get_temperature(h, T)
    rbar, Tbar = rho.mean(axis=1), T.mean(axis=1)
    d = rbar - coexistence_midpoint(lbm, Tbar, Tc)
    out = []
    for y in range(TH_NY - 1):
        if (d[y] > 0) != (d[y + 1] > 0):
            out.append(y + d[y] / (d[y] - d[y + 1]))
    return out


def run_thermal(args, torch, lbm, inputs):
    """Throughput of the thermal step (fused LBM step with T(x) in psi that also stores
    rho, u; one launch for the two Heun stages of the energy equation) on the 512 x 2048
    heated-from-below column; with
    --thermal-track, config 4 in full (FP32 and FP64, --thermal-steps steps) with the
    liquid/vapour crossing heights every --thermal-every steps."""
    import numpy as np

    p, rho0, Tc = thermal_setup(args.precision, lbm, inputs)
    nodes = TH_NX * TH_NY
    lat = lbm.Lattice(p, torch.from_numpy(rho0).cuda())
    lat.step(args.warmup)
    snap_f = torch.empty((9, TH_NY, TH_NX), dtype=torch.float64, device="cuda")
    snap_T = torch.empty((TH_NY, TH_NX), dtype=torch.float64, device="cuda")
    lbm.lbm_get_state(lat.h, snap_f)
    lbm.lbm_get_temperature(lat.h, snap_T)
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    restores = 0
    with ClockSampler(0) as clocks:
        start.record(stream)
        done = 0
        while done < args.steps:
            n = min(TH_WINDOW, args.steps - done)
            lat.step(n)
            done += n
            if done < args.steps:
                lbm.lbm_set_state(lat.h, snap_f)
                lbm.lbm_set_temperature(lat.h, snap_T)
                restores += 1
        end.record(stream)
        torch.cuda.synchronize()
    ms = start.elapsed_time(end)
    status = lat.status()
    lat.close()
    del lat
    peaks, peak_kind = measured_peaks()
    step_s = ms / 1e3 / args.steps
    bytes_step = TH_BYTES_PER_NODE[args.precision] * nodes
    line = {
        "metric": "MLUPS (thermal step)", "value": nodes * args.steps / (ms / 1e3) / 1e6, "unit": "MLUPS",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic", "impl": "gb300",
        "config": {"workload": f"thermal liquid column {TH_NX}x{TH_NY}, heated from below", "T_bot_over_Tc": TH_TBOT,
                   "T_top_over_Tc": TH_TTOP, "gravity": "rho g", "g_y": TH_GY, "liquid_rows": TH_LIQUID,
                   "c_v": p.c_v, "kappa": p.kappa, "noise": NOISE, "seed": SEED,
                   "l2": "state 151 MB (FP32) > 129 MB L2"},
        "roofline": {"bound": "hbm", "achieved": bytes_step / step_s / 1e9, "peak": peaks["hbm_gbs"], "unit": "GB/s",
                     "frac": bytes_step / step_s / 1e9 / peaks["hbm_gbs"], "traffic": None, "peak_kind": peak_kind,
                     "kernel": "whole thermal step (fused step storing rho, u; Heun: 2 launches)",
                     "bytes_per_node": TH_BYTES_PER_NODE[args.precision]},
        "gpu_launches": 2 * args.steps + restores * (9 + 1 + 1), "restores": restores,
        "physical_window": f"populations and T restored from the post-warm-up snapshot every {TH_WINDOW} steps",
        "clocks": clocks.summary(), "status": status,
    }
    if args.thermal_track:
        track = {}
        for prec in ("fp32", "fp64"):
            q, rho0, Tc = thermal_setup(prec, lbm, inputs)
            h = lbm.lbm_init(q, rho0)
            rows, t0 = [], time.perf_counter()
            done = 0
            while done < args.thermal_steps:
                n = min(args.thermal_every, args.thermal_steps - done)
                lbm.lbm_step(h, n)
                done += n
                st = lbm.lbm_status(h)
                rows.append({"step": done, "status": st, "max_u": lbm.lbm_reduce(h, lbm.LBM_REDUCE_MAX_U, check=False)[0][0],
                             "crossings": [round(c, 3) for c in crossing_heights(lbm, h, Tc)] if st == 0 else None})
                if st != 0:
                    break
            track[prec] = {"seconds": time.perf_counter() - t0, "samples": rows}
            lbm.lbm_destroy(h)
        line["track"] = track
    print(json.dumps(line), flush=True)
    return 0 if status == 0 else 2


# ---------------------------------------------------------------- learned warm start
def train_warm_network(lbm, inputs, torch, ncols, heights, cap, iters, batch, seed):
    """The warm-start network trained on the GPU (the library's tcgen05 kernels) on the
    steady profiles of `ncols` seeded columns of `heights` (another seed than any evaluated
    set), each run by the batch runner in FP32 to residual 1e-7 within `cap` steps; the
    converged columns give the rows. Returns (network handle, summary)."""
    import numpy as np

    _, Tc, _ = lbm.lbm_critical_point(A, B, R)
    cols_tr, rho_tr = column_set(ncols, seed, heights, lbm, inputs)
    b = lbm.lbm_batch_init(lbm.make_params(4, 8, 0.8 * Tc, "fp32", a=A, b=B, R=R), cols_tr, rho_tr)
    t_gen = lbm.lbm_batch_run(b, 1e-7, cap, 100)
    _, res, status = lbm.lbm_batch_results(b, len(cols_tr), check=False)
    rho_dev = torch.empty(rho_tr.size, dtype=torch.float64, device="cuda")
    lbm.lbm_batch_moments(b, rho=rho_dev)
    lbm.lbm_batch_destroy(b)
    rows = sum(c["ny"] for c in cols_tr)
    x_all = torch.empty((rows, lbm.MLP_INPUTS), dtype=torch.float32, device="cuda")
    t_all = torch.empty(rows, dtype=torch.float32, device="cuda")
    lbm.lbm_mlp_features(cols_tr, 4, A, B, R, x_all, t=t_all, rho=rho_dev)
    good = (res <= 1e-7) & (status == 0)
    row_mask = torch.from_numpy(np.repeat(good, [c["ny"] for c in cols_tr])).cuda()
    x, t = x_all[row_mask].contiguous(), t_all[row_mask].contiguous()
    del rho_dev, x_all, t_all
    h = lbm.lbm_mlp_create(lbm.mlp_initial_params(SEED), batch)
    t0 = time.perf_counter()
    losses = []
    for frac, lr in ((0.5, 1e-3), (0.3, 3e-4), (0.2, 1e-4)):
        losses.append(lbm.lbm_mlp_train(h, x, t, batch, int(frac * iters), lr, SEED + len(losses)))
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    losses = np.concatenate(losses)
    return h, {"columns": len(cols_tr), "heights": list(heights), "converged_columns": int(good.sum()),
               "rows": int(x.shape[0]), "generation_s": t_gen, "train_s": t_train, "iters": int(losses.size),
               "batch": batch, "loss_first": float(np.mean(losses[:20])), "loss_last": float(np.mean(losses[-200:]))}


def run_warmstart(args):
    """Config 5: steady columns generated by the batch runner train the warm-start network
    on the GPU; held-out seeded columns then run to residual 1e-10 from the tanh profile and
    from the network's (mass-corrected) profile, in FP64 alone and FP32 then FP64."""
    import numpy as np
    import torch

    from paper_2301_12869_gb300 import inputs, lbm

    heights = tuple(int(h) for h in args.column_heights.split(","))
    rho_c, Tc, _ = lbm.lbm_critical_point(A, B, R)
    cap = args.column_max_steps
    out = {"metric": "time to steady state (residual 1e-10), batched columns, FP32 (+ double-float finish) + warm start vs plain FP64",
           "unit": "s", "higher_is_better": False, "impl": "gb300", "n_gpus": 1}
    # ---- training data (steady profiles of the method, FP32 to its rounding floor) and training
    h, out["training"] = train_warm_network(lbm, inputs, torch, args.train_columns, heights, cap, args.mlp_iters,
                                            args.mlp_batch, SEED + 1)
    # ---- held-out columns: tanh start vs warm start
    cols, rho0 = column_set(args.columns, SEED + 2, heights, lbm, inputs)
    sizes = [4 * c["ny"] for c in cols]
    mean = np.array([blk.mean() for blk in np.split(rho0, np.cumsum(sizes)[:-1])])
    rho_ml = torch.empty(rho0.size, dtype=torch.float64, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    lbm.lbm_mlp_warm_start(h, cols, 4, A, B, R, mean, rho_ml)
    t_inf = time.perf_counter() - t0
    lbm.lbm_mlp_destroy(h)
    runs = {}
    final = {}
    for name, init, fp32_first, rest in (("fp64_tanh", rho0, False, False), ("fp64_tanh_rest", rho0, False, True),
                                         ("fp64_warm", rho_ml, False, False), ("fp64_warm_rest", rho_ml, False, True),
                                         ("fp32_dd_tanh", rho0, True, False), ("fp32_dd_tanh_rest", rho0, True, True),
                                         ("fp32_dd_warm_rest", rho_ml, True, True)):
        tuned = {}
        sec, st, res, status, bb = run_to_steady(lbm, cols, init, cap, fp32_first, tuned, rest=rest)
        final[name] = torch.empty(rho0.size, dtype=torch.float64, device="cuda")
        lbm.lbm_batch_moments(bb, rho=final[name])
        lbm.lbm_batch_destroy(bb)
        runs[name] = dict(seconds=sec + (t_inf if "warm" in name else 0.0), steps=st, ok=(res <= 1e-10) & (status == 0),
                          nonphysical=int((status != 0).sum()), block_threads=tuned_summary(tuned))
    # the bound of any density-only warm start: the converged plain-FP64 profile itself as the
    # start (populations at equilibrium with u = 0, as every start here), run to the same target
    sec, st, res, status, bb = run_to_steady(lbm, cols, final["fp64_tanh"], cap, False, {})
    lbm.lbm_batch_destroy(bb)
    runs["fp64_converged_rho"] = dict(seconds=sec, steps=st, ok=(res <= 1e-10) & (status == 0),
                                      nonphysical=int((status != 0).sum()), block_threads={})
    ok = np.logical_and.reduce([r["ok"] for r in runs.values()])
    def per_column_max(v):
        return np.array([blk.max() for blk in np.split(np.abs(v), np.cumsum(sizes)[:-1])])

    # profile error of the network's start against the converged plain-FP64 profile
    ref = final["fp64_tanh"]
    per_col = per_column_max((rho_ml - ref).cpu().numpy())
    per_col_tanh = per_column_max(rho0 - ref.cpu().numpy())
    # final profiles against the plain FP64 run: FP32 mass rounding moves the FP32 paths'
    # steady states slightly; a start that settles in another basin (a column's steady
    # state need not be unique) differs by O(0.1): counted above 1e-3
    diff = {}
    for k in final:
        d = per_column_max((final[k] - ref).cpu().numpy())[ok]
        diff[k] = {"median": float(np.median(d)), "p90": float(np.percentile(d, 90)), "max": float(d.max()),
                   "columns_over_1e-3": int(np.sum(d > 1e-3))}
    out["config"] = {"workload": f"{len(cols)} held-out seeded 4xH liquid columns, H in {heights}; network trained on "
                                 f"{out['training']['columns']} steady columns of another seed", "max_steps": cap, "check_every": 100}
    out["runs"] = {k: {"seconds": v["seconds"], "converged": int(v["ok"].sum()), "nonphysical": v["nonphysical"],
                       "steps_all_converged": int(v["steps"][ok].sum()), "block_threads": v["block_threads"]}
                   for k, v in runs.items()}
    out["columns_converged_in_all_runs"] = int(ok.sum())
    out["warm_start_inference_s"] = t_inf
    out["final_profile_difference_vs_plain_fp64"] = diff
    out["start_profile_error"] = {"network_max_abs_median": float(np.median(per_col[ok])),
                                  "tanh_max_abs_median": float(np.median(per_col_tanh[ok])),
                                  "network_max_abs_p90": float(np.percentile(per_col[ok], 90)),
                                  "tanh_max_abs_p90": float(np.percentile(per_col_tanh[ok], 90))}
    out["value"] = runs["fp32_dd_warm_rest"]["seconds"]
    out["speedup_vs_plain_fp64"] = runs["fp64_tanh"]["seconds"] / runs["fp32_dd_warm_rest"]["seconds"]

    def ratio(a, b):
        return out["runs"][a]["steps_all_converged"] / max(1, out["runs"][b]["steps_all_converged"])

    out["steps_ratios_fp64"] = {
        "warm_vs_tanh (equilibrium starts)": ratio("fp64_warm", "fp64_tanh"),
        "converged_rho_vs_tanh (equilibrium starts: the bound of any density-only start)":
            ratio("fp64_converged_rho", "fp64_tanh"),
        "tanh_rest_vs_tanh (the rest-state start alone)": ratio("fp64_tanh_rest", "fp64_tanh"),
        "warm_rest_vs_tanh_rest (the network's gain with rest-state starts)": ratio("fp64_warm_rest", "fp64_tanh_rest"),
        "warm_rest_vs_tanh (network and rest state against the plain method)": ratio("fp64_warm_rest", "fp64_tanh"),
    }
    out["steps_ratio_warm_vs_tanh_fp64"] = out["steps_ratios_fp64"]["warm_rest_vs_tanh_rest (the network's gain with rest-state starts)"]
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------- tensor-core GEMM of the network
def run_gemm(args):
    """Throughput of the warm-start network's tcgen05 GEMM (C = A B^T, bfloat16 in, FP32 out)
    on the network's own shape (a batch of rows through a 128 x 128 layer) and on a large
    square product. `tflops`: K launches enqueued back to back through lbm_mlp_gemm_enqueue,
    timed with CUDA events on their stream; `e2e_tflops`: K calls of the synchronising
    lbm_mlp_gemm (argument checks, a status word allocated, copied back and waited for)."""
    import torch

    from paper_2301_12869_gb300 import lbm

    peaks, peak_kind = measured_peaks()
    rows = []
    stream = torch.cuda.current_stream()
    for M, N, K in ((int(args.gemm_m), 128, 128), (8192, 8192, 8192)):
        A = torch.randn(M, K, device="cuda").to(torch.bfloat16).view(torch.int16)
        Bm = torch.randn(N, K, device="cuda").to(torch.bfloat16).view(torch.int16)
        C = torch.empty(M, N, device="cuda", dtype=torch.float32)
        status = torch.zeros(1, device="cuda", dtype=torch.int32)
        flops = 2.0 * M * N * K
        row = {"M": M, "N": N, "K": K, "operand_bytes": 2 * (M + N) * K + 4 * M * N}
        for key, call in (("tflops", lambda: lbm.lbm_mlp_gemm_enqueue(A, Bm, C, status, stream=stream.cuda_stream)),
                          ("e2e_tflops", lambda: lbm.lbm_mlp_gemm(A, Bm, C, stream=stream.cuda_stream))):
            for _ in range(max(args.warmup, 3)):
                call()
            torch.cuda.synchronize()
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            for _ in range(args.steps):
                call()
            t1.record(stream)
            torch.cuda.synchronize()
            ms = t0.elapsed_time(t1) / args.steps
            row[key.replace("tflops", "ms")] = ms
            row[key] = flops / (ms * 1e-3) / 1e12
        if int(status.item()) != 0:
            raise RuntimeError("a tensor-core wait timed out")
        row["frac_of_bf16_peak"] = row["tflops"] / peaks["bf16_tflops"]
        row["GB_per_s"] = row["operand_bytes"] / (row["ms"] * 1e-3) / 1e9
        rows.append(row)
    # the whole network per row in one fused kernel (lbm_mlp_predict): layers of 16 (padded
    # input) x 128, 128 x 128, 128 x 128 on the tensor cores and the 128-wide output layer
    n = int(args.gemm_m) * 16
    flops_row = 2 * (16 * 128 + 128 * 128 + 128 * 128) + 2 * 128
    hm = lbm.lbm_mlp_create(lbm.mlp_initial_params(SEED), 1024)
    g = torch.Generator(device="cuda").manual_seed(SEED)
    feats = torch.stack([0.7 + 0.25 * torch.rand(n, device="cuda", generator=g),
                         -6 + 2 * torch.rand(n, device="cuda", generator=g),
                         1.0 + torch.randint(0, 2, (n,), device="cuda", generator=g).float(),
                         0.3 + 2.2 * torch.rand(n, device="cuda", generator=g),
                         torch.rand(n, device="cuda", generator=g)], dim=1).contiguous()
    yv = torch.empty(n, device="cuda", dtype=torch.float32)
    for _ in range(max(args.warmup, 3)):
        lbm.lbm_mlp_predict(hm, feats, yv)
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        lbm.lbm_mlp_predict(hm, feats, yv)
    t1.record(stream)
    torch.cuda.synchronize()
    lbm.lbm_mlp_destroy(hm)
    ms = t0.elapsed_time(t1) / args.steps
    forward = {"rows": n, "ms": ms, "rows_per_s": n / (ms * 1e-3), "flops_per_row": flops_row,
               "tflops": n * flops_row / (ms * 1e-3) / 1e12,
               "frac_of_bf16_peak": n * flops_row / (ms * 1e-3) / 1e12 / peaks["bf16_tflops"],
               "what": "lbm_mlp_predict: the fused forward kernel (plus its status read-back) per call"}
    print(json.dumps({"metric": "tcgen05 GEMM throughput", "unit": "TFLOP/s", "impl": "gb300", "n_gpus": 1,
                      "peak": peaks["bf16_tflops"], "peak_kind": peak_kind, "hbm_peak_GB_per_s": peaks["hbm_gbs"],
                      "shapes": rows, "fused_forward": forward}), flush=True)
    return 0


# ---------------------------------------------------------------- small FP64 column
def run_small(args):
    """The plain method in FP64 on a 4 x 200 column (bounce-back walls, T = 0.85 T_c, rho g
    with g_y = -2e-5, liquid below y = 100 joined by a tanh of width 5, tau = 1): 20 000
    steps, device-timed with CUDA events. 800 nodes give 2 CTAs, so the step is bound by
    launch and pipeline latency, not by HBM: the line reports microseconds per step."""
    import torch

    from paper_2301_12869_gb300 import inputs, lbm

    nx, ny, steps = 4, 200, 20000
    _, Tc, _ = lbm.lbm_critical_point(A, B, R)
    rv, rl, _ = lbm.lbm_coexistence(A, B, R, 0.85 * Tc)
    rho0 = inputs.column_rho0(nx, ny, rl, rv, 100, width=5.0)
    p = lbm.make_params(nx, ny, 0.85 * Tc, "fp64", a=A, b=B, R=R, form=1, g=(0.0, -2e-5))
    lat = lbm.Lattice(p, torch.from_numpy(rho0).cuda())
    lat.step(max(args.warmup, 3))
    s = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    e0.record(s)
    lat.step(steps)
    e1.record(s)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1)
    mass = lat.reduce(lbm.LBM_REDUCE_MASS)[0]
    info = lbm.lbm_launch_info(lat.h)
    status = lat.status()
    lat.close()
    print(json.dumps({"metric": "us per step (4 x 200 FP64 column)", "value": 1e3 * ms / steps, "unit": "us",
                      "higher_is_better": False, "impl": "gb300", "n_gpus": 1, "steps": steps,
                      "mlups": nx * ny * steps / (ms * 1e-3) / 1e6, "dtype": "f64", "data": "synthetic",
                      "config": {"workload": "4x200 D2Q9 column, FP64, bounce-back walls", "T_over_Tc": 0.85,
                                 "gravity": "rho g", "g_y": -2e-5, "liquid_rows": 100, "tanh_width": 5.0,
                                 "launch": info},
                      "status": status, "mass": mass}), flush=True)
    return 0


# ---------------------------------------------------------------- boiling example
def run_boiling(args):
    """The paper's phase-formation example (Sec. V): a 1-D column of 101 wet nodes (h = 100,
    Zou-He walls), a = 0.5, <rho> = 1.3344 rho_c, rho g with g = 1.5e-5, T_med = 0.75 T_c,
    c_v = 5, kappa = 0.02. For each Delta T/T_c: equilibrate with the top wall at
    0.6213 T_c, lower it to T_med - Delta T/2 (lbm_set_params), and follow the rows next to
    the hot bottom wall: a vapour layer has formed once the density two nodes above the
    wall falls below the midpoint of the coexistence densities at its temperature."""
    import numpy as np

    from paper_2301_12869_gb300 import inputs, lbm

    a, ny, nx = 0.5, 101, 4
    rho_c, Tc, _ = lbm.lbm_critical_point(a, B, R)
    mean, g = 1.3344 * rho_c, -1.5e-5
    out = {"metric": "vapour layer formation at the hot wall (Sec. V example)", "impl": "gb300", "n_gpus": 1,
           "config": {"workload": "1-D thermal column, 101 wet nodes, Zou-He walls", "a": a, "mean_rho_reduced": 1.3344,
                      "g_y": g, "T_med_over_Tc": 0.75, "T_top_prerun_over_Tc": 0.6213, "c_v": 5.0, "kappa": 0.02,
                      "post_steps": args.boiling_steps, "check_every": 10000},
           "cases": []}
    cases = [(float(d), "fp64") for d in args.boiling_dT.split(",")]
    cases.append((cases[-1][0], "fp32"))
    for dT, prec in cases:
        T_bot, T_top = (0.75 + dT / 2) * Tc, (0.75 - dT / 2) * Tc
        rv, rl, _ = lbm.lbm_coexistence(a, B, R, 0.75 * Tc)
        rho0 = inputs.column_rho0(nx, ny, rl, rv, 54)
        rho0 *= mean / rho0.mean()
        p = lbm.make_params(nx, ny, 0.75 * Tc, prec, a=a, b=B, R=R, form=1, g=(0.0, g), thermal=1, T_bot=T_bot,
                            T_top=0.6213 * Tc, wall=lbm.LBM_WALL_ZOU_HE)
        h = lbm.lbm_init(p, rho0)
        t0 = time.perf_counter()
        pre, res = 0, math.inf
        tol = 1e-10 if prec == "fp64" else 1e-7
        while pre < args.boiling_prerun_cap and not res < tol:
            lbm.lbm_step(h, 49999)
            lbm.lbm_reduce(h, lbm.LBM_REDUCE_RESIDUAL)
            lbm.lbm_step(h, 1)
            res = lbm.lbm_reduce(h, lbm.LBM_REDUCE_RESIDUAL)[0]
            pre += 50000
        p.T_top = T_top
        lbm.lbm_set_params(h, p)
        rho = np.empty((ny, nx))
        T = np.empty((ny, nx))
        layer_step, samples = None, []
        for k in range(args.boiling_steps // 10000):
            lbm.lbm_step(h, 10000)
            lbm.lbm_moments(h, rho)
            lbm.lbm_get_temperature(h, T)
            Ty = T[:, 0]
            level = np.array([0.5 * sum(lbm.lbm_coexistence(a, B, R, min(t, 0.999 * Tc))[:2]) for t in Ty[:4]])
            vapour_at_wall = rho[2, 0] < level[2]
            if vapour_at_wall and layer_step is None:
                layer_step = (k + 1) * 10000
            if (k + 1) % 10 == 0 or (vapour_at_wall and len(samples) < 200):
                samples.append({"step": (k + 1) * 10000, "rho_row2": float(rho[2, 0]), "level_row2": float(level[2]),
                                "rho_max": float(rho[:, 0].max()), "argmax_y": int(np.argmax(rho[:, 0]))})
        out["cases"].append({"dT_over_Tc": dT, "precision": prec, "T_bot_over_Tc": 0.75 + dT / 2,
                             "T_top_over_Tc": 0.75 - dT / 2, "prerun_steps": pre, "prerun_residual": res,
                             "vapour_layer_step": layer_step, "status": lbm.lbm_status(h),
                             "seconds": time.perf_counter() - t0, "samples": samples[-12:]})
        lbm.lbm_destroy(h)
    print(json.dumps(out), flush=True)
    return 0


# ---------------------------------------------------------------- main
def run_reference(args, world, rank):
    if rank != 0:
        return 0
    ny_slice = args.ref_rows
    # the child process runs W untimed warm-up steps, then times K oracle steps
    mlups, res = time_oracle(ny_slice, max(1, args.steps), max(1, args.warmup))
    line = {
        "metric": "MLUPS", "value": mlups, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": res["seconds"] * 1e3 / res["steps"], "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
        # the workload of the GPU arm's line; the oracle computes it in FP64 (dtype)
        "config": workload_config(args.precision) | {"sample_rows": ny_slice},
        "cpu_baseline": {"value": mlups, "unit": "MLUPS", "cores": 1, "kind": "oracle",
                         "sample": f"{res['steps']} FP64 oracle steps on a {NX}x{ny_slice} slice around the interface"},
        "e2e": {"value": mlups, "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--partition", choices=["auto", "slabs", "replicas"], default="auto",
                    help="N > 1: the domain as slabs, one per GPU (auto) or N independent replicas; "
                         "slabs also runs at N = 1 (one slab = the whole domain)")
    ap.add_argument("--slab-scaling", choices=["weak", "strong"], default="weak",
                    help="slabs: a 1024 x 4096 slab per GPU of a 1024 x 4096 N column (weak), or the "
                         "1024 x 4096 column cut into N slabs (strong)")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end leg (profiling runs)")
    ap.add_argument("--ref-rows", type=int, default=64, help="rows of the oracle slice for --impl reference")
    ap.add_argument("--workload", choices=["domain", "columns", "thermal", "warmstart", "boiling", "gemm", "small"],
                    default="domain",
                    help="domain: the 1024 x 4096 single-domain throughput line (default); "
                         "columns: time to steady state of batched columns; "
                         "thermal: the 512 x 2048 thermal column; "
                         "small: the 4 x 200 FP64 column, 20000 steps (latency-bound)")
    ap.add_argument("--thermal-track", action="store_true")
    ap.add_argument("--thermal-steps", type=int, default=8000)
    ap.add_argument("--thermal-every", type=int, default=500)
    ap.add_argument("--columns", type=int, default=1024)
    ap.add_argument("--column-heights", default="64,128")
    ap.add_argument("--column-max-steps", type=int, default=200000)
    ap.add_argument("--train-columns", type=int, default=16384)
    ap.add_argument("--fp32-tol", type=float, default=None, help="FP32 target before the FP64 phase (default 1e-8)")
    ap.add_argument("--fp32-stall", type=int, default=None, help="stall checks of the FP32 phase (default 50)")
    ap.add_argument("--accel-checks", type=int, default=None, help="extrapolation cycle of the FP32 -> FP64 runs "
                                                                    "in residual checks (default 5; 0: off)")
    ap.add_argument("--boiling-dT", default="0.3166,0.3381,0.3382")
    ap.add_argument("--gemm-m", type=int, default=65536, help="rows of the network-shaped GEMM")
    ap.add_argument("--boiling-steps", type=int, default=1000000)
    ap.add_argument("--boiling-prerun-cap", type=int, default=4000000)
    ap.add_argument("--steady-columns", type=int, default=4096,
                    help="columns of the time-to-steady block of the default line")
    ap.add_argument("--steady-cap", type=int, default=20000, help="step cap per phase of that block")
    ap.add_argument("--no-steady", action="store_true", help="skip the time-to-steady block")
    ap.add_argument("--no-precision", action="store_true", help="skip the FP32-vs-FP64 report")
    ap.add_argument("--mlp-iters", type=int, default=6000)
    ap.add_argument("--mlp-batch", type=int, default=8192)
    args = ap.parse_args(argv)
    global FP32_TOL, FP32_STALL_CHECKS, ACCEL_CHECKS
    if args.accel_checks is not None:
        ACCEL_CHECKS = args.accel_checks
    if args.fp32_tol is not None:
        FP32_TOL = args.fp32_tol
    if args.fp32_stall is not None:
        FP32_STALL_CHECKS = args.fp32_stall
    if args.warmup < 3:
        ap.error("--warmup must be >= 3")
    world, rank, local = dist_env()

    if args.impl == "reference":
        return run_reference(args, world, rank)
    if args.workload == "columns":
        return run_columns(args) if rank == 0 else 0
    if args.workload == "warmstart":
        return run_warmstart(args) if rank == 0 else 0
    if args.workload == "boiling":
        return run_boiling(args) if rank == 0 else 0
    if args.workload == "gemm":
        return run_gemm(args) if rank == 0 else 0
    if args.workload == "small":
        return run_small(args) if rank == 0 else 0

    import numpy as np
    import torch

    from paper_2301_12869_gb300 import inputs, lbm

    if not torch.cuda.is_available():
        print(json.dumps({"error": "no CUDA device"}))
        return 1
    torch.cuda.set_device(local)
    if args.workload == "thermal":
        return run_thermal(args, torch, lbm, inputs) if rank == 0 else 0
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local))

    # cpu baseline first (child process, before heavy GPU work; spawn-safe)
    cpu_base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        try:
            cpu_base = cpu_baseline_entry()
        except Exception as exc:  # noqa: BLE001 - reported, not hidden
            cpu_base = {"value": None, "unit": "MLUPS", "cores": 1, "kind": "oracle", "sample": f"failed: {exc}"}

    rho_c, Tc, p_c = lbm.lbm_critical_point(A, B, R)
    rv, rl, _ = lbm.lbm_coexistence(A, B, R, TR * Tc)
    rho0 = inputs.column_rho0(NX, NY, rl, rv, LIQUID_ROWS, noise_amp=NOISE, seed=SEED)
    p = lbm.make_params(NX, NY, TR * Tc, args.precision, a=A, b=B, R=R, form=2, g=(0.0, GY))
    nodes = NX * NY

    use_slabs = args.partition == "slabs" or (args.partition == "auto" and world > 1)
    peaks, peak_kind = measured_peaks()
    if use_slabs:
        # ---- the column cut into slabs, one per GPU, NCCL exchanges per step; the slab loop
        # runs Python per step, so the sampler polls slowly (it competes for the interpreter)
        nvml = NvmlClocks(local, period_s=0.005).start()
        with ClockSampler(local) as smi:
            t_host0 = time.perf_counter()
            local_ms, local_units, restores, halo_bytes, e2e, status, sl, ny_total = run_slabs(
                args, torch, lbm, inputs, world, rank, local, rho0, Tc)
            t_host1 = time.perf_counter()
        nvml.stop()
        ms, units = aggregate(local_ms, local_units, torch)
        value = units / (ms / 1e3) / 1e6
        kernel_s = ms / 1e3 / args.steps  # the slowest rank's step, exchanges included
        alg_bytes = BYTES_PER_NODE[args.precision] * NX * sl.ny_own
        achieved = alg_bytes / kernel_s / 1e9
        mass = e2e["mass"] if e2e else None
        info = {"column_rows": ny_total, "slab_rows_rank0": sl.ny_own, "ghost_rows_per_side": 2,
                "exchange_bytes_per_step_per_rank": halo_bytes,
                "exchanges_per_step": "NCCL all-reduce of the FP64 mass partials (one per CTA of the largest "
                                      "slab's grid) + send/receive of 2 ghost rows x 9 planes with each neighbour"}
        scaling, parallelism = args.slab_scaling, f"y-slabs x{world}"
        launches = args.steps  # one slab step kernel per step (the exchanges are NCCL's and torch's copies)
        kernel_name = "step_kernel_ws on the rank's slab (+ exchanges, per step)"
        torch.cuda.empty_cache()
    else:
        # ---- device-resident run (value)
        lat = lbm.Lattice(p, torch.from_numpy(rho0).cuda())
        info = lbm.lbm_launch_info(lat.h)
        nvml = NvmlClocks(local).start()  # clocks from before the warm-up to the end of the timed region
        lat.step(args.warmup)
        snapshot = torch.empty((9, NY, NX), dtype=torch.float64, device="cuda")
        lbm.lbm_get_state(lat.h, snapshot)
        torch.cuda.synchronize()
        stream = torch.cuda.current_stream()
        start, end = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()
        with ClockSampler(local) as smi:
            # a ~0.1 ms spin kernel ahead of the start event: while it runs the host enqueues
            # the event and the steps, so the events bracket the K step kernels alone and not
            # the host's latency to its first launch after the synchronisation
            torch.cuda._sleep(PREROLL_CYCLES)
            t_host0 = time.perf_counter()
            start.record(stream)
            restores = run_steps(lbm, lat.h, args.steps, snapshot)
            end.record(stream)
            torch.cuda.synchronize()
            t_host1 = time.perf_counter()
        nvml.stop()
        if world > 1:
            torch.distributed.barrier()
        local_ms = start.elapsed_time(end)
        status = lat.status()
        ms, units = aggregate(local_ms, float(nodes) * args.steps, torch)
        value = units / (ms / 1e3) / 1e6
        # one fused-kernel launch per step, back to back; the restores are counted against it
        kernel_s = local_ms / 1e3 / args.steps
        alg_bytes = BYTES_PER_NODE[args.precision] * nodes
        achieved = alg_bytes / kernel_s / 1e9
        mass = lat.reduce(lbm.LBM_REDUCE_MASS)[0]
        lat.close()
        del lat
        torch.cuda.empty_cache()
        # ---- end to end through the C ABI with host buffers (init from pinned host rho0,
        #      K steps, rho and the mass read back to host)
        e2e = None
        if not args.no_e2e:
            e2e = run_e2e(args, rho0, Tc, nodes, world, torch, lbm, snapshot)
        del snapshot
        torch.cuda.empty_cache()
        scaling, parallelism = "weak", (f"replicas x{world}" if world > 1 else "single GPU")
        launches = args.steps + restores * (9 + 1)
        kernel_name = (f"step_kernel_ws<8 consumer warps, {info['stages']} stages>" if args.precision == "fp32"
                       else "step_kernel<double, 128-node bands>")
    # the metric's second half: time to steady state of the batched columns (all ranks, each
    # on its share of the columns)
    steady = None if args.no_steady else time_to_steady(args, lbm, inputs, world, rank, torch)
    precision = None
    if rank == 0 and not args.no_precision:
        precision = precision_report(lbm, rho0, Tc)
    if rank != 0:
        if world > 1:
            torch.distributed.destroy_process_group()
        return 0
    line = {
        "metric": "MLUPS", "value": value, "unit": "MLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": scaling,
        "vs_baseline": None, "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": workload_config(args.precision) | {"launch": info, "parallelism": parallelism} | (
            {"workload": f"liquid column {NX}x{ny_total} D2Q9 as {world} slabs of {NX}x{ny_total // world}, "
                         f"{args.precision.upper()} populations, FP64 reductions",
             "ny": ny_total, "liquid_rows": LIQUID_ROWS * ny_total // NY} if use_slabs else {
                "pre_roll": "a ~0.1 ms spin kernel (torch.cuda._sleep) precedes the start event, so the "
                            "events bracket the K steps without the host's first-launch latency"}),
        "roofline": ({
            "bound": "hbm", "achieved": achieved, "peak": peaks["hbm_gbs"], "unit": "GB/s",
            "frac": achieved / peaks["hbm_gbs"], "traffic": None if use_slabs else traffic_from_profile(args.precision),
            "peak_kind": peak_kind, "kernel": kernel_name, "algorithmic_bytes_per_launch": alg_bytes,
        } if args.precision == "fp32" else {
            "bound": "alu", "achieved": FP64_FLOPS_PER_NODE * alg_bytes / BYTES_PER_NODE["fp64"] / kernel_s / 1e12,
            "peak": FP64_PEAK_TFLOPS, "unit": "TFLOP/s",
            "frac": FP64_FLOPS_PER_NODE * alg_bytes / BYTES_PER_NODE["fp64"] / kernel_s / 1e12 / FP64_PEAK_TFLOPS,
            "traffic": None, "peak_kind": "derived from the nominal FP64 rate (2 FP64 FMA / SM / clock)",
            "kernel": kernel_name, "fp64_flops_per_node": FP64_FLOPS_PER_NODE,
            "hbm": {"achieved_GB_per_s": achieved, "frac_of_measured": achieved / peaks["hbm_gbs"]},
        }),
        "cpu_baseline": cpu_base,
        "e2e": e2e,
        "time_to_steady": steady,
        "precision": precision,
        "gpu_launches": launches,
        "restores": restores,
        "clocks": nvml.summary(t_host0, t_host1) | {"warmup_and_timed": nvml.summary(), "nvidia_smi": smi.summary()},
        "status": status,
        "mass": mass,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0 if status == 0 and math.isfinite(value) else 2


if __name__ == "__main__":
    sys.exit(main())
