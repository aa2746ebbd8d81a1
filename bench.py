#!/usr/bin/env python3
"""MPPI benchmark on B300: rollout-steps/s of one MPPI iteration.

Workload (the car-on-a-track configuration): dynamic bicycle car on a 1024x1024
FP32 cost-map track, K=16384 samples, T=100 steps, nu=10, lambda=1,
Sigma=diag(0.3, 0.35), R = lambda Sigma^-1, receding horizon (update + shift every
step), seeded synthetic inputs.  A step is one full MPPI iteration: noise,
rollout, cost with the importance-sampling terms, weights, update, shift.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  value = rollout-steps/s with inputs resident in HBM (CUDA
events on the controller's stream, L2 flushed between steps, outside the timed
events).  e2e = the same metric through mppi_step with host buffers (x0 H2D and
u0 D2H inside each timed step).  The plain single-controller loop on the same GPU
(unfused kernels, sync per step) is reported beside it.  With torchrun, every rank
runs its own independent controller (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import glob
import hashlib
import json
import math
import os
import statistics
import shutil
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "rollout-steps/s (K*T per MPPI iteration) and MPPI iters/s vs plain loop on same GPU; p50/p99 step latency"
UNIT = "rollout-steps/s"
SYSTEM = W.CAR
K_SAMPLES, T_STEPS, NU = 16384, 100, 10.0

# Algorithmic FP32 work of one rollout-step (one sample, one time step), counted from
# the formulas: adds, multiplies and divides, each elementary function as one op.
# Derivation in the design notes.
ALGO_FLOPS_PER_ROLLOUT_STEP = {W.CARTPOLE: 55.5, W.CAR: 127.0, W.QUAD: 936.0}
# the same with the quadrotor's nearest cylinder counted over the ~2.9 candidates of its grid
# cell that the kernels evaluate (7 flop each) instead of all 64 cylinders
SEARCHED_FLOPS_PER_ROLLOUT_STEP = {**ALGO_FLOPS_PER_ROLLOUT_STEP, W.QUAD: 936.0 - 64 * 7 + 2.9 * 7}
SMS, FP32_LANES, SM_MAX_MHZ = 148, 128, 2032.0


def fp32_peak_tflops(mhz=SM_MAX_MHZ):
    return SMS * FP32_LANES * 2 * mhz * 1e6 / 1e12


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--e2e-steps", type=int, default=1000,
                    help="timed end-to-end steps for the p50/p99 latency (after 50 untimed)")
    ap.add_argument("--plain-steps", type=int, default=1000,
                    help="timed plain-loop steps for its p50/p99 latency (after 50 untimed)")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--serving", default="256,512,1024",
                    help="concurrency levels of the serving measurement ('' to skip)")
    ap.add_argument("--serving-ticks", type=int, default=500)
    ap.add_argument("--serving-async", default="256,512,1024",
                    help="concurrency levels of the real-time closed loop over submit / reap ('' to skip)")
    ap.add_argument("--serving-async-periods", type=int, default=500,
                    help="50 Hz control periods per level of the real-time closed loop")
    ap.add_argument("--serving-heavy", default="256",
                    help="concurrency levels of the heavy-skewed serving mix ('' to skip)")
    ap.add_argument("--serving-capacity", action="store_true",
                    help="measure the largest 50 Hz concurrency of every (system, K, T) (about a minute)")
    ap.add_argument("--serving-only", action="store_true", help="run only the serving measurement")
    ap.add_argument("--no-learned", action="store_true", help="skip the learned-dynamics measurement")
    ap.add_argument("--shard-k", action="store_true",
                    help="with several ranks: one controller K-sharded over them (weak scaling) instead of "
                         "one independent controller per rank")
    ap.add_argument("--learned-only", action="store_true")
    ap.add_argument("--no-systems", action="store_true", help="skip the per-workload iteration table")
    ap.add_argument("--nu-sweep", action="store_true",
                    help="only the Sec. V-A cart-pole swing-up over exploration variance and K")
    ap.add_argument("--systems-only", action="store_true")
    ap.add_argument("--learned-train", type=int, default=10_000_000, help="training transitions")
    ap.add_argument("--learned-steps", type=int, default=6000, help="training steps")
    return ap.parse_args()


def source_hash(names=None):
    """sha256 prefix of the CUDA sources (all of csrc/, or the named files in it)."""
    h = hashlib.sha256()
    csrc = os.path.join(ROOT, "paper_1509_01149_b300", "csrc")
    paths = ([os.path.join(csrc, n) for n in names] if names else
             sorted(q for q in glob.glob(os.path.join(csrc, "*")) if os.path.isfile(q) and not q.endswith(".pyc")))
    for p in paths:
        h.update(open(p, "rb").read())
    return h.hexdigest()[:16]


# device code of each profiled kernel (a capture stays valid while these files are unchanged)
KERNEL_SOURCES = {
    "rollout_car_ws_k16384": ["rollout_ws.cuh", "rollout_body.cuh", "systems.cuh", "mppi_device.cuh",
                              "tc_common.cuh"],
}


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
_REASONS = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]


# NVML clock-event reason bits (nvml.h: nvmlClocksEventReason*)
_REASON_BITS = {"hw_slowdown": 0x8, "hw_thermal_slowdown": 0x40, "sw_thermal_slowdown": 0x20, "sw_power_cap": 0x4}


def _nvml_clock_reader(gpu_id: str | None):
    """A function returning (SM clock MHz, max SM clock MHz, clock-event reason bits) of the GPU
    from NVML's read-only queries (the Python bindings, else the driver's libnvidia-ml through
    ctypes), or None where NVML is unavailable."""
    try:
        import pynvml as nv
        nv.nvmlInit()
        h = nv.nvmlDeviceGetHandleByUUID(gpu_id) if gpu_id else nv.nvmlDeviceGetHandleByIndex(0)
        return lambda: (nv.nvmlDeviceGetClockInfo(h, nv.NVML_CLOCK_SM), nv.nvmlDeviceGetMaxClockInfo(h, nv.NVML_CLOCK_SM),
                        nv.nvmlDeviceGetCurrentClocksEventReasons(h))
    except Exception:
        pass
    try:
        import ctypes as C
        lib = C.CDLL("libnvidia-ml.so.1")
        if lib.nvmlInit_v2() != 0:
            return None
        h = C.c_void_p()
        rc = (lib.nvmlDeviceGetHandleByUUID(gpu_id.encode(), C.byref(h)) if gpu_id else
              lib.nvmlDeviceGetHandleByIndex_v2(0, C.byref(h)))
        if rc != 0:
            return None
        sm, smax, why = C.c_uint(), C.c_uint(), C.c_ulonglong()
        reasons = getattr(lib, "nvmlDeviceGetCurrentClocksEventReasons", None) or \
            lib.nvmlDeviceGetCurrentClocksThrottleReasons

        def read():
            if (lib.nvmlDeviceGetClockInfo(h, 1, C.byref(sm)) or lib.nvmlDeviceGetMaxClockInfo(h, 1, C.byref(smax))
                    or reasons(h, C.byref(why))):
                raise RuntimeError("NVML query failed")
            return sm.value, smax.value, why.value
        read()
        return read
    except Exception:
        return None


def _nvml_sample_loop(gpu_id: str, path: str, period_s: float = 0.002):
    """Sampler process: every period_s append 'unix time,SM MHz,max SM MHz,reason bits' to path
    (line-buffered) until terminated.  Run as its own process, so that the timed host loops of
    the bench never wait for this thread's interpreter lock."""
    read = _nvml_clock_reader(gpu_id or None)
    if read is None:
        return
    with open(path, "w", buffering=1) as f:
        while True:
            try:
                sm, smax, why = read()
                f.write("%.6f,%d,%d,%d\n" % (time.time(), sm, smax, why))
            except Exception:
                pass
            time.sleep(period_s)


class ClockSampler:
    """SM clocks and throttle reasons during the timed regions.  A sampler process of its own
    (NVML, read-only queries) timestamps a sample every 2 ms, so that a short timed region still
    has a record without a thread of this process competing with the timed host loops;
    nvidia-smi runs beside it every 20 ms (started ahead of the timed region, waiting for its
    first sample) and is the record where NVML is unavailable.  Only samples whose timestamps
    fall between a mark_start() and its mark_end() are kept."""

    def __init__(self, gpu_id: str | None, settle_s: float = 2.0):
        self.path = tempfile.mktemp(suffix=".csv")
        self.t0 = self.t1 = None
        self.windows = []                  # (start, end) of each timed region
        # NVML in a sampler process of its own (read-only queries, every 2 ms, timestamped);
        # the samples inside the timed windows are kept at stop()
        self.nvml_path = tempfile.mktemp(suffix=".nvml")
        try:
            self.nvml_p = subprocess.Popen(
                [sys.executable, "-c", "import sys; sys.path.insert(0, sys.argv[1]); import bench; "
                 "bench._nvml_sample_loop(sys.argv[2], sys.argv[3])", ROOT, gpu_id or "", self.nvml_path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.nvml_p = None
        q = ("timestamp,clocks.sm,clocks.max.sm,utilization.gpu,power.draw,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        cmd = ["nvidia-smi", f"--query-gpu={q}", "--format=csv,noheader,nounits", "-lms", "20"]
        if gpu_id:
            cmd += ["-i", gpu_id]
        if shutil.which("stdbuf"):
            cmd = ["stdbuf", "-oL"] + cmd     # line-buffered: no sample left in a buffer at stop()
        try:
            self.f = open(self.path, "w")
            self.p = subprocess.Popen(cmd, stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None
            return
        deadline = time.time() + settle_s
        while time.time() < deadline and os.path.getsize(self.path) == 0:
            time.sleep(0.01)
        deadline = time.time() + 4 * settle_s
        while (self.nvml_p is not None and self.nvml_p.poll() is None and time.time() < deadline and
               not (os.path.exists(self.nvml_path) and os.path.getsize(self.nvml_path) > 0)):
            time.sleep(0.01)

    def mark_start(self):
        self.t0 = time.time()

    def mark_end(self):
        self.t1 = time.time()
        self.windows.append((self.t0, self.t1))

    def _stop_nvml(self):
        """The sampler process's samples inside the timed windows."""
        if self.nvml_p is None:
            return []
        if self.t1 is not None:   # a sample stamped past the last window, or a short wait
            deadline = time.time() + 0.5
            while time.time() < deadline and self.nvml_p.poll() is None:
                time.sleep(0.01)
                try:
                    with open(self.nvml_path) as f:
                        last = f.read().splitlines()[-1:]
                    if last and float(last[0].split(",")[0]) > self.t1:
                        break
                except (OSError, ValueError, IndexError):
                    pass
        self.nvml_p.terminate()
        try:
            self.nvml_p.wait(timeout=5)
        except Exception:
            self.nvml_p.kill()
        rows = []
        try:
            with open(self.nvml_path) as f:
                for line in f:
                    try:
                        t, sm, smax, why = line.strip().split(",")
                        t, why = float(t), int(why)
                    except ValueError:
                        continue
                    if self.windows and not any(a <= t <= b for a, b in self.windows):
                        continue
                    rows.append(dict(sm=float(sm), smax=float(smax),
                                     reasons={r: bool(why & b) for r, b in _REASON_BITS.items()}))
            os.unlink(self.nvml_path)
        except OSError:
            pass
        return rows

    @staticmethod
    def _stamp(stamp: str):
        import datetime
        try:
            return datetime.datetime.strptime(stamp, "%Y/%m/%d %H:%M:%S.%f").timestamp()
        except ValueError:
            return None

    def _inside(self, stamp: str) -> bool:
        if not self.windows:
            return True
        t = self._stamp(stamp)
        return True if t is None else any(a <= t <= b for a, b in self.windows)

    def _past_end(self) -> bool:
        """True once the file holds a sample stamped after mark_end()."""
        try:
            with open(self.path) as f:
                lines = f.read().splitlines()
        except OSError:
            return False
        for line in reversed(lines):
            t = self._stamp(line.split(",")[0].strip())
            if t is not None:
                return t > self.t1
        return False

    def stop(self):
        rows = self._stop_nvml()
        smi = self._stop_smi()
        if not rows:
            return dict(smi, source="nvidia-smi")
        reasons = sorted({r for row in rows for r, on in row["reasons"].items() if on})
        return {"sm_mhz": statistics.median(r["sm"] for r in rows), "sm_max_mhz": max(r["smax"] for r in rows),
                "reasons": reasons, "samples": len(rows), "source": "nvml, every 2 ms (a sampler process)",
                "nvidia_smi": {k: smi.get(k) for k in ("sm_mhz", "reasons", "samples")}}

    def _stop_smi(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        if self.t1 is not None:   # every sample of the timed region written before the stop
            deadline = time.time() + 3.0
            while time.time() < deadline and not self._past_end():
                time.sleep(0.02)
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [s.strip() for s in line.split(",")]
            if len(parts) < 9 or not self._inside(parts[0]):
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), util=float(parts[3]),
                                 reasons={r: parts[5 + i].lower().startswith("active") for i, r in enumerate(_REASONS)}))
            except ValueError:
                continue
        os.unlink(self.path)
        busy = [r for r in rows if r["util"] > 0] or rows
        if not busy:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        reasons = sorted({r for row in busy for r, on in row["reasons"].items() if on})
        return {"sm_mhz": statistics.median(r["sm"] for r in busy), "sm_max_mhz": max(r["smax"] for r in busy),
                "reasons": reasons, "samples": len(busy)}


# ---------------------------------------------------------------------------
# the oracle on the host cores (cpu_baseline and --impl reference)
# ---------------------------------------------------------------------------
_ONE_THREAD = {v: "1" for v in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS",
                                  "NUMEXPR_NUM_THREADS", "VECLIB_MAXIMUM_THREADS")}


def _oracle_loop(seconds: float, k_sample: int, max_iters: int | None):
    from oracle import mppi as om
    from oracle import systems as osys
    cfg = W.config(SYSTEM, K=k_sample, T=T_STEPS, nu=NU)
    sysm = osys.Car(cfg["dt"], W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_H_CELL)
    U = cfg["U"].copy()
    times = []
    t_end = time.perf_counter() + seconds
    while time.perf_counter() < t_end and (max_iters is None or len(times) < max_iters):
        t0 = time.perf_counter()
        r = om.iteration_seeded(sysm, cfg["x0"], U, k_sample, cfg["lam"], cfg["nu"], cfg["Sigma"], cfg["R"],
                                0, counter=len(times))
        U = om.shift(r.U, cfg["u_init"])
        times.append(time.perf_counter() - t0)
    return times


def oracle_rate(seconds: float, k_sample: int = 1024, max_iters: int | None = None):
    """Oracle iterations of the bench workload on a bounded sample of k_sample samples
    (full horizon T), in a child process pinned to one thread (numpy/BLAS).
    Returns (rollout-steps/s, iterations, per-iteration seconds)."""
    env = dict(os.environ, **_ONE_THREAD)
    arg = json.dumps([seconds, k_sample, max_iters])
    out = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-child", arg], env=env,
                         capture_output=True, text=True, check=True)
    times = json.loads(out.stdout.strip().splitlines()[-1])
    return k_sample * T_STEPS * len(times) / sum(times), len(times), times


def reduce_max(value: float, dist=None, device=None) -> float:
    """The largest value over the ranks of the process group (float64 all-reduce), or the
    value itself without one: the timed region of a multi-rank run is the slowest rank's."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput: the units every rank processed over the slowest rank's time."""
    return units_per_rank * world / seconds


def cpu_model() -> str:
    try:
        for line in open("/proc/cpuinfo"):
            if line.startswith("model name"):
                return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_rate_all_cores(seconds: float, k_sample: int = 1024, max_procs: int = 64):
    """The same oracle loop in one single-threaded child process per host core (up to
    max_procs), all at once, each on its own k_sample-sample batch; returns the summed
    rollout-steps/s and the number of processes."""
    procs = max(1, min(os.cpu_count() or 1, max_procs))
    env = dict(os.environ, **_ONE_THREAD)
    arg = json.dumps([seconds, k_sample, None])
    ps = [subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-child", arg], env=env,
                           stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True) for _ in range(procs)]
    total = 0.0
    for p in ps:
        out, _ = p.communicate()
        times = json.loads(out.strip().splitlines()[-1])
        total += k_sample * T_STEPS * len(times) / sum(times)
    return total, procs


def oracle_errors(N, stream_handle, seed, gid, U, counter, **over):
    """The error of one headline iteration against the FP64 oracle (part of the CPU-baseline leg,
    outside every timed region): the GPU runs one iteration of the car K=16384, T=100 from the
    controls and iteration counter the timed loop reached; the oracle runs the same iteration
    (same FP32 inputs, same Philox noise).  Reports, per result, the whole iteration's error
    (path costs S~, argmin k*, normaliser eta, update dU, u0) and the weighting's own error
    (the oracle's FP64 weighting and weighted sum of the GPU's own costs and perturbations)."""
    from oracle import mppi as om
    from oracle import systems as osys
    c, cfg = make_ctrl(N, N.MPPI_IMPL_FUSED, seed=seed, gid=gid, stream_handle=stream_handle, **over)
    c.set_controls(np.asarray(U, dtype=np.float32))
    c.set_iteration(counter)
    x0 = np.asarray(cfg["x0"], dtype=np.float32)
    u0 = c.step(x0)
    d = c.get_debug()
    U_gpu = c.get_controls().astype(np.float64)
    du = c.get_noise(counter).astype(np.float64)
    c.close()
    f64 = lambda a: np.asarray(a, dtype=np.float32).astype(np.float64)
    lam, nu = float(np.float32(cfg["lam"])), float(np.float32(cfg["nu"]))
    car = osys.Car(cfg["dt"], W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_H_CELL)
    o = om.iteration_seeded(car, f64(x0), f64(U), cfg["K"], lam, nu, f64(cfg["Sigma"]), f64(cfg["R"]), seed, counter,
                            gid)
    scale = np.sqrt(cfg["nu"] * np.diag(cfg["Sigma"]))
    Sg = d["S"].astype(np.float64)
    fin = np.isfinite(o.S)
    rel = np.abs(Sg[fin] - o.S[fin]) / np.abs(o.S[fin])
    srt = np.sort(o.S[fin])
    rho, kst, eta_r, w_r = om.weights(Sg, lam)                      # the weighting of the GPU's own costs
    dU_r = np.einsum("tmk,k->tm", du, w_r)
    ess = 1.0 / float(np.sum(o.w ** 2))
    return {
        "workload": f"car K={cfg['K']} T={cfg['T']} nu={cfg['nu']} lambda={cfg['lam']}"
                    f"{'' if not over else ', R fixed at Sigma^-1'}, controls and counter {counter} of the timed loop",
        "effective_sample_size": ess,
        "S_rel_max": float(rel.max()), "S_rel_p99": float(np.percentile(rel, 99)),
        "kstar_match": bool(d["kstar"] == o.kstar), "kstar_unique": bool(srt[1] - srt[0] > 2e-4 * abs(srt[0])),
        "eta_rel_iteration": abs(d["eta"] - o.eta) / o.eta,
        "dU_err_over_scale_iteration": float(np.max(np.abs(d["dU"] - o.dU) / scale[None, :])),
        "U_err_over_scale_iteration": float(np.max(np.abs(U_gpu - o.U) / scale[None, :])),
        "u0_err_over_scale": float(np.max(np.abs(u0.astype(np.float64) - o.u0) / scale)),
        "kstar_match_on_gpu_costs": bool(d["kstar"] == kst),
        "eta_rel_reduction": abs(d["eta"] - eta_r) / eta_r,
        "dU_err_over_scale_reduction": float(np.max(np.abs(d["dU"] - dU_r) / scale[None, :])),
        "bars": {"S_rel": 1e-4, "U_over_scale": 1e-3, "kstar": "exact where the oracle's minimum is unique"},
        "note": "iteration: GPU vs the oracle's full FP64 iteration; reduction: GPU vs the oracle's FP64 weighting "
                "of the GPU's own path costs and perturbations (the error of the FP32 weights, FP32 block sums and "
                "double-FP32 cross-block sums alone)",
    }


def run_reference(args, rank, world, max_procs: int = 64):
    """The reference arm: the FP64 oracle on the host cores, one single-threaded child process
    per core (up to max_procs), each iterating its own 1024-sample batch at the full horizon,
    all at once (with 16 cores a step covers all 16384 samples).  Warm-up iterations are
    dropped; a step's time is the slowest process's; the rate sums the processes' rates."""
    if rank != 0:
        return
    k_sample = 1024
    procs = max(1, min(os.cpu_count() or 1, max_procs))
    env = dict(os.environ, **_ONE_THREAD)
    arg = json.dumps([1e9, k_sample, max(args.warmup, 1) + args.steps])
    ps = [subprocess.Popen([sys.executable, os.path.abspath(__file__), "--oracle-child", arg], env=env,
                           stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True) for _ in range(procs)]
    per_proc = []
    for p in ps:
        out, _ = p.communicate()
        per_proc.append(json.loads(out.strip().splitlines()[-1])[max(args.warmup, 1):])
    rate = sum(k_sample * T_STEPS * len(t) / sum(t) for t in per_proc)
    ms = 1e3 * statistics.mean(max(t[j] for t in per_proc) for j in range(args.steps))
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64", "data": "synthetic",
        "config": {"workload": "car on cost-map track (1024x1024 FP32 map), one MPPI iteration + shift per step",
                   "K": K_SAMPLES, "T": T_STEPS, "nu": NU, "lambda": 1.0, "sample_K": k_sample * procs,
                   "parallelism": f"{procs} single-threaded oracle processes on the host cores"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": procs, "kind": "oracle",
                         "sample": f"{procs} x {k_sample} samples (one batch per process), full horizon "
                                   f"T={T_STEPS}, per step"},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------
def make_ctrl(N, impl, seed, gid, stream_handle, **over):
    cfg = W.config(SYSTEM, **dict(dict(K=K_SAMPLES, T=T_STEPS, nu=NU, seed=seed, gid=gid), **over))
    c = N.Controller(cfg["system"], cfg["K"], cfg["T"], cfg["dt"], cfg["nu"], cfg["lam"], cfg["Sigma"], cfg["R"])
    c.set_stream(stream_handle)
    c.set_seed(seed)
    c.set_controller_id(gid)
    c.set_impl(impl)
    c.set_cost_map(W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_ORIGIN, W.MAP_H_CELL)
    c.set_controls(cfg["U"].astype(np.float32))
    c.set_u_init(cfg["u_init"].astype(np.float32))
    return c, cfg


def run_serving(levels, n_ticks, seed=0, mix=None):
    """Batched serving of a Poisson stream of controllers (by default a uniform mix of
    cart-pole / car / quadrotor, K in {512, 1024, 4096, 16384}, T in {50, 100, 150, 200};
    `mix` gives choice probabilities) at each target concurrency: prefill, autotune, then
    n_ticks receding-horizon ticks with arrivals and departures.  Per level: tick latency
    p50/p99, deadline misses, rollout-steps/s and the algorithmic FP32 rate of the rollouts
    against the FP32 peak."""
    from paper_1509_01149_b300 import _native as N
    from paper_1509_01149_b300 import serving
    out = {}
    for target in levels:
        srv = N.Server(max(2 * target, 64), max(256 << 20, target << 21))
        srv.set_env(0, N.map_blob(W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_ORIGIN, W.MAP_H_CELL))
        srv.set_env(1, N.forest_blob(W.quad_forest(0), W.QUAD_GOAL))
        loop = serving.ServingLoop(srv, W, {W.CAR: 0, W.QUAD: 1}, seed=seed + target, **(mix or {}))
        loop.prefill(target, 200.0)
        srv.autotune([r.slot for r in loop.active], [W.config(r.system)["x0"] for r in loop.active])
        flops, flops_searched = [], []
        orig_step = loop.step

        def step(rate, life, record=True, _loop=loop):
            f = sum(r.K * r.T * ALGO_FLOPS_PER_ROLLOUT_STEP[r.system] for r in _loop.active)
            fs = sum(r.K * r.T * SEARCHED_FLOPS_PER_ROLLOUT_STEP[r.system] for r in _loop.active)
            orig_step(rate, life, record)
            if record:
                flops.append(f)
                flops_searched.append(fs)
        loop.step = step
        summ = loop.run(n_ticks, target_active=target, mean_lifetime=200.0)
        info = srv.info()
        busy = sum(loop.stats.tick_ms) / 1e3
        tf = sum(flops) / busy / 1e12 if busy > 0 else None
        tfs = sum(flops_searched) / busy / 1e12 if busy > 0 else None
        summ.update({"algorithmic_tflops": tf, "fp32_frac": tf / fp32_peak_tflops() if tf else None,
                     "fp32_frac_searched": tfs / fp32_peak_tflops() if tfs else None,
                     "rollout_block": info["rollout_block"], "ctas_per_sm": info["rollout_ctas_per_sm"]})
        out[str(target)] = summ
        loop.drain()
        srv.close()
    return out


# (name, system, K, T, cost-to-go weighting, general per-step sampling covariance)
SYSTEM_CONFIGS = (("cart-pole", W.CARTPOLE, 1000, 100, 0, 0), ("car", W.CAR, 4096, 100, 0, 0),
                  ("car", W.CAR, 16384, 100, 0, 0), ("quadrotor", W.QUAD, 8192, 150, 0, 0),
                  ("car, cost-to-go weighting", W.CAR, 16384, 100, 1, 0),
                  ("quadrotor, cost-to-go weighting", W.QUAD, 8192, 150, 1, 0),
                  ("car, general sampling covariance", W.CAR, 16384, 100, 0, 1),
                  ("quadrotor, general sampling covariance", W.QUAD, 8192, 150, 0, 1))


def run_systems(steps=200, warmup=10):
    """Device-resident receding-horizon iterations (mppi_iterate_async: one graph per
    iteration) of each workload configuration: cart-pole K=1000 T=100, car K=4096 and 16384
    T=100, quadrotor K=8192 T=150, and the car and quadrotor with the per-time-step
    cost-to-go weighting and with a general per-step sampling covariance.  Per configuration: rollout-steps/s, iteration time and the
    rollout kernel's algorithmic FP32 rate against the FP32 peak (rollout timed alone)."""
    import torch

    from paper_1509_01149_b300 import _native as N
    out = []
    s = torch.cuda.Stream()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    for name, system, K, T, to_go, gen in SYSTEM_CONFIGS:
        cfg = W.config(system, K=K, T=T)
        c = N.Controller(system, K, T, cfg["dt"], cfg["nu"], cfg["lam"], cfg["Sigma"], cfg["R"])
        c.set_stream(s.cuda_stream)
        if to_go:
            c.set_weighting(N.MPPI_WEIGHT_TO_GO)
        if gen:
            c.set_sampling_covariance(W.sampling_covariances(cfg))
        if system == W.CAR:
            c.set_cost_map(W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_ORIGIN, W.MAP_H_CELL)
        elif system == W.QUAD:
            c.set_forest(W.quad_forest(0), W.QUAD_GOAL)
        c.set_controls(np.asarray(cfg["U"], np.float32))
        c.set_u_init(np.asarray(cfg["u_init"], np.float32))
        dx = torch.tensor(np.asarray(cfg["x0"], np.float32), device="cuda")
        du = torch.zeros(4, device="cuda")
        for _ in range(warmup):
            c.iterate_async(dx.data_ptr(), du.data_ptr())
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        rv = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        with torch.cuda.stream(s):
            for a, b in ev:
                flush.zero_()
                a.record(s)
                c.iterate_async(dx.data_ptr(), du.data_ptr())
                b.record(s)
            for a, b in rv:
                flush.zero_()
                a.record(s)
                c.rollout_async(dx.data_ptr())
                b.record(s)
                c.update_async(None)
                c.shift()
        torch.cuda.synchronize()
        it_ms = statistics.median(a.elapsed_time(b) for a, b in ev)
        ro_ms = statistics.median(a.elapsed_time(b) for a, b in rv)
        tf = ALGO_FLOPS_PER_ROLLOUT_STEP[system] * K * T / (ro_ms * 1e-3) / 1e12
        tfs = SEARCHED_FLOPS_PER_ROLLOUT_STEP[system] * K * T / (ro_ms * 1e-3) / 1e12
        out.append({"system": name, "K": K, "T": T, "iteration_ms": it_ms, "rollout_ms": ro_ms,
                    "rollout_steps_per_s": K * T / (it_ms * 1e-3), "iters_per_s": 1e3 / it_ms,
                    "rollout_tflops_algorithmic": tf, "fp32_frac": tf / fp32_peak_tflops(),
                    "fp32_frac_searched": tfs / fp32_peak_tflops()})
        c.close()
    return out


def cartpole_vel_plant(x, u, dt):
    """The Sec. V-A cart-pole (desired-velocity input) as the simulated plant: one explicit
    Euler step in FP64 on the host (x = p, p', theta, theta'; theta = 0 hanging down)."""
    p, v, th, om = x
    acc = 10.0 * (u - v)
    th_acc = -(3.0 / (4.0 * 0.5)) * (9.81 * np.sin(th) + acc * np.cos(th))
    return np.array([p + dt * v, v + dt * acc, th + dt * om, om + dt * th_acc])


def serving_plant(system, X, U, dt):
    """The simulated plants of the serving measurement, one control period in FP64 on the host,
    vectorised over controllers of one system (X [n][nx], U [n][m]): the force-input cart-pole
    (Euler), the dynamic bicycle car with its steering actuator and Pacejka tyres (Euler) and
    the quadrotor (RK4), the models the controllers optimise over (no collision model: a
    crashed plant keeps flying).  Non-finite results are reset by the serving loop."""
    X = np.asarray(X, dtype=np.float64).T.copy()
    U = np.asarray(U, dtype=np.float64).T
    with np.errstate(all="ignore"):
        if system == W.CARTPOLE:
            mc, mp, l, g = 1.0, 0.1, 0.5, 9.81
            _, v, th, om = X
            s, c = np.sin(th), np.cos(th)
            tmp = (U[0] + mp * l * om * om * s) / (mc + mp)
            tha = (g * s - c * tmp) / (l * (4.0 / 3.0 - mp * c * c / (mc + mp)))
            xa = tmp - mp * l * tha * c / (mc + mp)
            X = X + dt * np.stack([v, xa, om, tha])
        elif system == W.CAR:
            m, Iz, lf, lr, B, C, mu, g = 21.7, 1.12, 0.34, 0.23, 4.0, 1.8, 0.9, 9.81
            _, _, psi, vx, vy, r, de = X
            vxs = np.maximum(vx, 1.0)
            L = lf + lr
            Fyf = mu * m * g * lr / L * np.sin(C * np.arctan(B * (de - np.arctan((vy + lf * r) / vxs))))
            Fyr = mu * m * g * lf / L * np.sin(C * np.arctan(B * -np.arctan((vy - lr * r) / vxs)))
            Fx = 120.0 * U[1] - 2.0 * vx - 0.35 * vx * np.abs(vx)
            X = X + dt * np.stack([vx * np.cos(psi) - vy * np.sin(psi), vx * np.sin(psi) + vy * np.cos(psi), r,
                                   (Fx - Fyf * np.sin(de)) / m + vy * r, (Fyr + Fyf * np.cos(de)) / m - vx * r,
                                   (lf * Fyf * np.cos(de) - lr * Fyr) / Iz, (0.5 * U[0] - de) / 0.1])
        elif system == W.QUAD:
            ms, g, arm, kap, Ix, Iy, Izz = 0.5, 9.81, 0.17, 0.016, 2.3e-3, 2.3e-3, 4.0e-3
            f = U

            def deriv(x):
                ph, th, ps, wp, wq, wr = x[6], x[7], x[8], x[9], x[10], x[11]
                a = (f[0] + f[1] + f[2] + f[3]) / ms
                cph, sph, cth, sth, cps, sps = np.cos(ph), np.sin(ph), np.cos(th), np.sin(th), np.cos(ps), np.sin(ps)
                ws = wq * sph + wr * cph
                return np.stack([x[3], x[4], x[5], a * (cps * sth * cph + sps * sph), a * (sps * sth * cph - cps * sph),
                                 a * cth * cph - g, wp + ws * sth / cth, wq * cph - wr * sph, ws / cth,
                                 (arm * (f[1] - f[3]) - (Izz - Iy) * wq * wr) / Ix,
                                 (arm * (f[2] - f[0]) - (Ix - Izz) * wr * wp) / Iy,
                                 (kap * (f[0] - f[1] + f[2] - f[3]) - (Iy - Ix) * wp * wq) / Izz])
            k1 = deriv(X)
            k2 = deriv(X + 0.5 * dt * k1)
            k3 = deriv(X + 0.5 * dt * k2)
            k4 = deriv(X + dt * k3)
            X = X + dt / 6.0 * (k1 + 2 * k2 + 2 * k3 + k4)
    return X.T


def run_serving_async(levels, periods, seed=0, mix=None):
    """The real-time closed loop over the asynchronous serving interface at each target
    concurrency: controllers at 50 Hz from random phases, each request submitted from its plant's
    state and the plant advanced by the returned u0 (serving_plant), Poisson arrivals and
    departures with admission and release while ticks are on the GPU.  Per level: the latency of
    every request from submit to result (p50 / p99 / max), deadline misses and rollout-steps/s."""
    from paper_1509_01149_b300 import _native as N
    from paper_1509_01149_b300 import serving
    out = {}
    for target in levels:
        srv = N.Server(max(2 * target, 64), max(256 << 20, target << 21))
        srv.set_env(0, N.map_blob(W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_ORIGIN, W.MAP_H_CELL))
        srv.set_env(1, N.forest_blob(W.quad_forest(0), W.QUAD_GOAL))
        loop = serving.AsyncServingLoop(srv, W, {W.CAR: 0, W.QUAD: 1}, plant=serving_plant, seed=seed + target,
                                        **(mix or {}))
        summ = loop.run(periods * serving.DEADLINE_MS / 1e3, target_active=target)
        summ["periods_per_controller"] = periods
        st = srv.stats()
        summ["ticks"] = st["ticks"]
        summ["mean_requests_per_tick"] = st["completed"] / max(st["ticks"], 1)
        out[str(target)] = summ
        loop.drain()
        srv.close()
    return out


def run_nu_sweep(nus=(1.0, 10.0, 50.0, 100.0, 300.0, 1000.0, 1500.0), Ks=(100, 1000, 10000), seconds=10.0, seed=0):
    """The cart-pole swing-up of Sec. V-A in closed loop: 50 Hz receding horizon (T = 50,
    1 s), the paper's natural noise 1/sqrt(rho) = 0.01 (Sigma = 0.005 per step, also applied to
    the plant's control), R = 1, lambda = Sigma R, exploration variance nu Sigma.  Per (nu, K):
    the average running cost of the plant's state over the run and the first time the pole
    is within 0.3 rad of upright."""
    from paper_1509_01149_b300 import _native as N
    out = {}
    for nu in nus:
        for K in Ks:
            cfg = W.config(W.CARTPOLE_VEL, K=K, nu=nu)
            c = N.Controller(W.CARTPOLE_VEL, K, cfg["T"], cfg["dt"], nu, cfg["lam"], cfg["Sigma"], cfg["R"])
            c.set_seed(seed)
            c.set_controls(np.zeros((cfg["T"], 1), np.float32))
            rng = np.random.default_rng(seed + 17)
            x = np.zeros(4)
            ticks = int(round(seconds / cfg["dt"]))
            costs, up = [], None
            sd = math.sqrt(cfg["Sigma"][0, 0])
            for t in range(ticks):
                u0 = float(c.step_shift(x.astype(np.float32))[0])
                x = cartpole_vel_plant(x, u0 + sd * rng.standard_normal(), cfg["dt"])
                q = x[0] ** 2 + 500.0 * (1.0 + math.cos(x[2])) ** 2 + x[3] ** 2 + x[1] ** 2
                costs.append(q)
                if up is None and abs(math.remainder(x[2] - math.pi, 2 * math.pi)) < 0.3:
                    up = (t + 1) * cfg["dt"]
            out[f"{nu:g}/{K}"] = {"nu": nu, "K": K, "average_cost": float(np.mean(costs)), "swing_up_s": up}
            c.close()
    return out


def run_capacity(probe=(16, 64), ticks=5, cap=2048, seed=0):
    """Largest number of identical controllers of each (system, K, T) that one server steps
    within the 20 ms (50 Hz) deadline: tick time measured at two probe sizes (autotuned at the
    larger), a line t(N) = a + b N fitted, N* = (20 ms - a) / b capped at `cap`, then checked
    by running N* controllers (the worst of `ticks` ticks must meet the deadline; else N* is
    lowered by 10 % and checked again, up to three times)."""
    from paper_1509_01149_b300 import _native as N
    from paper_1509_01149_b300 import serving
    srv = N.Server(cap + 64, 6 << 30)
    srv.set_env(0, N.map_blob(W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_ORIGIN, W.MAP_H_CELL))
    srv.set_env(1, N.forest_blob(W.quad_forest(0), W.QUAD_GOAL))
    env_ids = {W.CAR: 0, W.QUAD: 1}
    out = {}

    def timed(system, K, T, n, tune=False):
        slots = []
        for i in range(n):
            slot = srv.admit(serving.default_config(system, K, T, seed * 100000 + i, srv, W, env_ids))
            if slot is None:
                break
            slots.append(slot)
        x0 = [W.config(system)["x0"]] * len(slots)
        try:
            if len(slots) < n:
                return None
            if tune:
                srv.autotune(slots, x0)
            for _ in range(2):
                srv.tick(slots, x0)
            ts = []
            for _ in range(ticks):
                t0 = time.perf_counter()
                srv.tick(slots, x0)
                ts.append(1e3 * (time.perf_counter() - t0))
            return statistics.median(ts), max(ts)
        finally:
            for s in slots:
                srv.release(s)

    for system in serving.SYSTEMS:
        for K in serving.K_CHOICES:
            for T in serving.T_CHOICES:
                pts = [(n, timed(system, K, T, n, tune=(n == probe[-1]))) for n in probe]
                (n1, r1), (n2, r2) = pts[0], pts[-1]
                b = (r2[0] - r1[0]) / (n2 - n1)
                a = r1[0] - b * n1
                est = cap if b <= 0 else int(min(cap, max(1, (serving.DEADLINE_MS - a) / b)))
                n, got = est, None
                for _ in range(4):
                    got = timed(system, K, T, n)
                    if got is not None and got[1] <= serving.DEADLINE_MS:
                        break
                    n = max(1, int(n * 0.9))
                out[f"{system}/{K}/{T}"] = {"max_controllers": n if got and got[1] <= serving.DEADLINE_MS else None,
                                           "capped": n >= cap, "tick_ms_p50": got[0] if got else None,
                                           "tick_ms_max": got[1] if got else None,
                                           "probe_ms": [[nn, r[0]] for nn, r in pts]}
    srv.close()
    return out


def run_learned(n_train=10_000_000, n_test=100_000, steps=6000, batch=8192):
    """Learned car dynamics: train on n_train analytic transitions (the GPU's analytic step
    generates the targets), test on n_test held-out ones; one-step and 100-step errors
    against the analytic model (the yardstick); MPPI rollout throughput with the network in
    BF16 and in FP8 at K=16384, T=100."""
    import torch

    from paper_1509_01149_b300 import _native as N
    out = {"n_train": n_train, "n_test": n_test, "train_steps": steps, "batch": batch}
    xs, us = W.car_transition_inputs(101, n_train)
    dx, du = torch.tensor(xs).cuda(), torch.tensor(us).cuda()
    del xs, us
    net = N.MLP(3)
    net.set_data(dx.data_ptr(), du.data_ptr(), n_train, 0.02)
    del dx, du
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    net.train(steps * 2 // 3, batch, 2e-3, seed=7)
    net.train(steps - steps * 2 // 3, batch, 5e-4, seed=8)
    torch.cuda.synchronize()
    dt_train = time.perf_counter() - t0
    # forward + backward (data and weight gradients): three products per layer
    fl = 3 * 2 * (9 * 256 + 256 * 256 + 256 * 7) * batch * steps          # the network's own
    fl_exec = 3 * 2 * (16 * 256 + 256 * 256 + 256 * 16) * batch * steps   # on the padded tiles
    out.update(train_s=dt_train, train_samples_per_s=batch * steps / dt_train, train_tflops=fl / dt_train / 1e12,
               train_tflops_executed=fl_exec / dt_train / 1e12)
    params, scale = net.get_params()
    # held-out one-step error (normalised by the per-state increment scale)
    xt, ut = W.car_transition_inputs(202, n_test)
    dxt, dut = torch.tensor(xt).cuda(), torch.tensor(ut).cuda()
    pred, true = torch.empty_like(dxt), torch.empty_like(dxt)
    net.predict(dxt.data_ptr(), dut.data_ptr(), n_test, pred.data_ptr())
    N.mppi_car_step(dxt.data_ptr(), dut.data_ptr(), n_test, 0.02, true.data_ptr())
    torch.cuda.synchronize()
    sc = torch.tensor(scale).cuda()
    one = (((pred - true) / sc) ** 2).mean(0).sqrt().cpu().numpy()
    out["one_step_rms_over_increment_scale"] = [round(float(v), 5) for v in one]
    # 100-step open-loop error: both models from the same 4096 states with the same controls
    n100 = 4096
    xa = dxt[:n100].clone()
    xb = dxt[:n100].clone()
    g = torch.Generator(device="cuda").manual_seed(3)
    sig = torch.tensor([0.3 ** 0.5, 0.35 ** 0.5], device="cuda")
    tmp = torch.empty_like(xa)
    for _ in range(100):
        u = (torch.rand(n100, 2, device="cuda", generator=g) * 2 - 1) * 3 * sig
        net.predict(xa.data_ptr(), u.data_ptr(), n100, tmp.data_ptr())
        xa.copy_(tmp)
        N.mppi_car_step(xb.data_ptr(), u.data_ptr(), n100, 0.02, tmp.data_ptr())
        torch.cuda.synchronize()
        xb.copy_(tmp)
    pos = (xa[:, :2] - xb[:, :2]).norm(dim=1)
    out["hundred_step_position_error_m"] = {"median": float(pos.median()), "p90": float(pos.quantile(0.9))}
    out["hundred_step_speed_error_mps"] = float((xa[:, 3] - xb[:, 3]).abs().median())
    net.close()
    # MPPI with the learned dynamics, BF16 and FP8
    cfg = W.config(W.CAR, K=K_SAMPLES, T=T_STEPS, nu=NU)
    for prec, name in ((0, "bf16"), (1, "fp8")):
        c = N.Controller(W.CAR_MLP, K_SAMPLES, T_STEPS, cfg["dt"], cfg["nu"], cfg["lam"], cfg["Sigma"], cfg["R"])
        c.set_cost_map(W.car_cost_map(0), W.MAP_ORIGIN, W.MAP_ORIGIN, W.MAP_H_CELL)
        c.set_env(N.mlp_blob(params, scale, prec))
        s = torch.cuda.Stream()
        c.set_stream(s.cuda_stream)
        dx0 = torch.tensor(np.asarray(cfg["x0"], np.float32)).cuda()
        for _ in range(3):
            c.step_async(dx0.data_ptr(), None)
            c.shift()
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(20)]
        with torch.cuda.stream(s):
            for e0, e1 in evs:
                e0.record(s)
                c.rollout_async(dx0.data_ptr())
                e1.record(s)
                c.update_async(None)
                c.shift()
        torch.cuda.synchronize()
        ms = statistics.mean(e0.elapsed_time(e1) for e0, e1 in evs)
        # per rollout-step: the network's algorithmic multiply-adds (9 -> 256 -> 256 -> 7) and the
        # ones the tensor core executes on the padded tiles (16 -> 256 -> 256 -> 16)
        alg = 2 * (9 * 256 + 256 * 256 + 256 * 7) * K_SAMPLES * T_STEPS / (ms * 1e-3) / 1e12
        tf = 2 * (16 * 256 + 256 * 256 + 256 * 16) * K_SAMPLES * T_STEPS / (ms * 1e-3) / 1e12
        bf16_peak, basis = bf16_peak_tflops()
        peak = bf16_peak * (2 if prec == 1 else 1)
        out[f"mppi_rollout_{name}"] = {"ms": ms, "rollout_steps_per_s": K_SAMPLES * T_STEPS / (ms * 1e-3),
                                       "tensor_tflops": tf, "algorithmic_tflops": alg, "frac_of_peak": alg / peak,
                                       "frac_of_peak_executed": tf / peak,
                                       "peak_basis": basis + (" x2 (fp8 nominal ratio)" if prec else "")}
        c.close()
    return out


def bf16_peak_tflops():
    """Dense BF16 burst peak: the measured figure of MEASURED_PEAKS.json, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            v = float(json.load(f)["bf16_tflops"])
        return v, "measured bf16 burst (%.1f TFLOP/s)" % v
    except (OSError, KeyError, ValueError, TypeError):
        return 1800.0, "fallback bf16 burst (1800 TFLOP/s)"


def load_profile(kernel_tag: str):
    """The committed ncu record of a kernel (DRAM bytes per launch, FP32 work per rollout-step
    from its instruction counters), if it was taken on the current kernel sources (same
    source hash); else None."""
    p = os.path.join(ROOT, "profiles", f"{kernel_tag}.json")
    if not os.path.exists(p):
        return None
    try:
        d = json.load(open(p))
    except Exception:
        return None
    if d.get("source_hash") != source_hash(KERNEL_SOURCES.get(kernel_tag)):
        return None
    return d


def run_sharded(args, rank, world, dev, stream, dist):
    """One controller K-sharded over the ranks (weak scaling: K_SAMPLES samples per rank, the
    controller has K_SAMPLES * world): per step each rank rolls out its shard, the ranks
    all-gather their partials (NCCL, the only collective) and every rank merges them and
    shifts.  Same timing rules as the replicated run (barrier + synchronize around the timed
    steps, L2 flushed between them outside the events, max over ranks)."""
    import torch

    from paper_1509_01149_b300 import _native as N
    from paper_1509_01149_b300 import sharded
    K_total = K_SAMPLES * world
    ctrl, cfg = make_ctrl(N, N.MPPI_IMPL_FUSED, seed=1000, gid=0, stream_handle=stream.cuda_stream, K=K_total)
    sc = sharded.ShardedController(ctrl, rank, world, dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    with torch.cuda.stream(stream):
        d_x0 = torch.tensor(cfg["x0"], dtype=torch.float32, device=dev)
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        sc.step(d_x0.data_ptr(), stream)
    torch.cuda.synchronize()
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    dist.barrier()
    torch.cuda.synchronize()
    with torch.cuda.stream(stream):
        for s in range(args.steps):
            flush.zero_()
            ev[s][0].record(stream)
            sc.step(d_x0.data_ptr(), stream)
            ev[s][1].record(stream)
    torch.cuda.synchronize()
    dist.barrier()
    total_s = reduce_max(sum(a.elapsed_time(b) for a, b in ev) / 1e3, dist, dev)
    value = K_total * T_STEPS * args.steps / total_s
    # e2e: x0 from pinned host memory, u0 back to the host, every step
    x_host = torch.tensor(cfg["x0"], dtype=torch.float32).pin_memory()
    lat = []
    for s in range(args.e2e_steps + 50):
        dist.barrier()
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            d_x0.copy_(x_host, non_blocking=True)
        u0 = sc.step(d_x0.data_ptr(), stream)
        with torch.cuda.stream(stream):
            u0_host = u0.to("cpu", non_blocking=False)
        lat.append(time.perf_counter() - t0)
    lat = lat[50:]
    e2e_total = reduce_max(sum(lat), dist, dev)
    if rank == 0:
        lat_ms = sorted(1e3 * x for x in lat)
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": "car on cost-map track, one K-sharded controller, one MPPI iteration + shift per step",
                       "K": K_total, "K_per_rank": K_SAMPLES, "T": T_STEPS, "nu": NU, "lambda": 1.0,
                       "parallelism": f"K-sharded over {world} ranks, one all-gather of (T*m + 3) doubles per rank "
                                      f"and step (NCCL)",
                       "l2": "flushed between timed steps (256 MB write, outside the timed events)"},
            "e2e": {"value": K_total * T_STEPS * len(lat) / e2e_total, "unit": UNIT,
                    "h2d_bytes_per_step": 4 * ctrl.n, "d2h_bytes_per_step": 4 * ctrl.m,
                    "p50_ms": lat_ms[len(lat_ms) // 2], "p99_ms": lat_ms[min(len(lat_ms) - 1, int(0.99 * len(lat_ms)))],
                    "latency_samples": len(lat_ms)},
            "gpu_launches": 4 * args.steps,
            "source_hash": source_hash()}), flush=True)
    dist.destroy_process_group()


def run_ours(args, rank, world, local_rank):
    import torch

    from paper_1509_01149_b300 import _native as N

    dev = torch.device("cuda", local_rank)
    torch.cuda.set_device(dev)
    levels = [int(v) for v in args.serving.split(",") if v.strip()]
    heavy_levels = [int(v) for v in args.serving_heavy.split(",") if v.strip()]
    if args.systems_only:
        print(json.dumps({"systems": run_systems()}), flush=True)
        return
    if args.nu_sweep:
        print(json.dumps({"nu_sweep": run_nu_sweep()}), flush=True)
        return
    if args.serving_only:
        from paper_1509_01149_b300.serving import HEAVY_MIX
        res = {"serving": run_serving(levels, args.serving_ticks)}
        async_levels = [int(v) for v in args.serving_async.split(",") if v.strip()]
        if async_levels:
            res["serving_async"] = run_serving_async(async_levels, args.serving_async_periods)
        if heavy_levels:
            res["serving_heavy"] = run_serving(heavy_levels, args.serving_ticks, mix=HEAVY_MIX)
        if args.serving_capacity:
            res["serving_capacity"] = run_capacity()
        print(json.dumps(res), flush=True)
        return
    if args.learned_only:
        print(json.dumps({"learned": run_learned(args.learned_train, steps=args.learned_steps)}), flush=True)
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    stream = torch.cuda.Stream(device=dev)
    if args.shard_k and world > 1:
        run_sharded(args, rank, world, dev, stream, dist)
        return
    ctrl, cfg = make_ctrl(N, N.MPPI_IMPL_FUSED, seed=1000 + rank, gid=rank, stream_handle=stream.cuda_stream)
    n, m = ctrl.n, ctrl.m
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)     # > 126 MB L2
    with torch.cuda.stream(stream):
        d_x0 = torch.tensor(cfg["x0"], dtype=torch.float32, device=dev)
        d_u0 = torch.zeros(m, dtype=torch.float32, device=dev)
    torch.cuda.synchronize()

    # clock sampling runs from before the warm-up; only the timed region's samples are kept
    try:
        gpu_uuid = str(torch.cuda.get_device_properties(dev).uuid)
        gpu_id = gpu_uuid if gpu_uuid.startswith("GPU-") else f"GPU-{gpu_uuid}"
    except Exception:
        gpu_id = None
    clocks = ClockSampler(gpu_id)
    # warm-up
    for _ in range(args.warmup):
        ctrl.iterate_async(d_x0.data_ptr(), d_u0.data_ptr())
    torch.cuda.synchronize()

    # ---- value: inputs resident, one graph launch per receding-horizon iteration ---
    ev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(args.steps)]
    barrier()
    torch.cuda.synchronize()
    clocks.mark_start()
    with torch.cuda.stream(stream):
        for s in range(args.steps):
            flush.zero_()                              # evict L2 between timed steps
            e0, e1 = ev[s]
            e0.record(stream)
            ctrl.iterate_async(d_x0.data_ptr(), d_u0.data_ptr())
            e1.record(stream)
    torch.cuda.synchronize()
    clocks.mark_end()
    barrier()
    step_ms = [e0.elapsed_time(e1) for e0, e1 in ev]
    total_s = reduce_max(sum(step_ms) / 1e3, dist, dev)
    value = whole_job_rate(K_SAMPLES * T_STEPS * args.steps, world, total_s)
    # the merge and the shift share one cluster launch while the T*m outputs fit 8 CTAs of 32
    fused_shift = T_STEPS * W.CONTROL_DIM[SYSTEM] <= 8 * 32
    launches_per_step = 2 if fused_shift else 3
    launch_note = ("per step one CUDA-graph launch of 2 kernels (rollout; merge (FP64 normaliser, double-FP32 sums) + update + shift in one "
                   "thread-block cluster)" if fused_shift else
                   "per step one CUDA-graph launch of 3 kernels (rollout, merge (FP64 normaliser, double-FP32 sums) + update, shift)")
    ms_per_step = 1e3 * total_s / args.steps
    # the dominant kernel alone (for the roofline): rollout launches between events, same stream
    n_roll = max(min(args.steps, 200), 5)
    rev = [[torch.cuda.Event(enable_timing=True) for _ in range(2)] for _ in range(n_roll)]
    with torch.cuda.stream(stream):
        for s in range(n_roll):
            flush.zero_()
            rev[s][0].record(stream)
            ctrl.rollout_async(d_x0.data_ptr())
            rev[s][1].record(stream)
            ctrl.update_async(d_u0.data_ptr())
            ctrl.shift()
    torch.cuda.synchronize()
    roll_ms = [a.elapsed_time(b) for a, b in rev]

    # ---- e2e: host buffers through mppi_step (graph), x0 H2D + u0 D2H per step ---
    e2e_steps = max(args.e2e_steps, 1)
    x_host = np.asarray(cfg["x0"], dtype=np.float32)
    lat = []
    e2e_warm = 50                                      # untimed steps before the measured ones
    for s in range(e2e_steps + e2e_warm):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        if s == e2e_warm:
            clocks.mark_start()
        t0 = time.perf_counter()
        ctrl.step_shift(x_host)
        lat.append(time.perf_counter() - t0)
    stream.synchronize()
    clocks.mark_end()
    lat = lat[e2e_warm:]
    e2e_total = reduce_max(sum(lat), dist, dev)
    e2e_value = whole_job_rate(K_SAMPLES * T_STEPS * e2e_steps, world, e2e_total)

    # ---- plain loop baseline (unfused kernels, sync per step) -----------------
    plain_steps = max(args.plain_steps, 1)
    plain_warm = 50
    pctrl, _ = make_ctrl(N, N.MPPI_IMPL_PLAIN, seed=1000 + rank, gid=rank, stream_handle=stream.cuda_stream)
    plat = []
    for s in range(plain_steps + plain_warm):
        with torch.cuda.stream(stream):
            flush.zero_()
        stream.synchronize()
        if s == plain_warm:
            clocks.mark_start()
        t0 = time.perf_counter()
        pctrl.step(x_host)
        pctrl.shift()
        plat.append(time.perf_counter() - t0)
    stream.synchronize()
    clocks.mark_end()
    clk = clocks.stop()
    clk["windows"] = "the device-resident timed steps, the e2e steps and the plain-loop steps"
    plat = plat[plain_warm:]
    plain_value = K_SAMPLES * T_STEPS * len(plat) * world / sum(plat)
    pctrl.close()

    U_end, it_end = ctrl.get_controls(), ctrl.get_iteration()     # for the oracle-error sample
    serving_res = run_serving(levels, args.serving_ticks, seed=rank) if levels else None
    from paper_1509_01149_b300.serving import HEAVY_MIX
    heavy_res = run_serving(heavy_levels, args.serving_ticks, seed=rank, mix=HEAVY_MIX) if heavy_levels else None
    async_levels = [int(v) for v in args.serving_async.split(",") if v.strip()]
    async_res = run_serving_async(async_levels, args.serving_async_periods, seed=rank) if async_levels else None
    capacity_res = run_capacity(seed=rank) if args.serving_capacity else None
    learned_res = None if args.no_learned else run_learned(args.learned_train, steps=args.learned_steps)
    systems_res = None if args.no_systems else run_systems()

    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return

    prof = load_profile("rollout_car_ws_k16384")
    formula_flops = ALGO_FLOPS_PER_ROLLOUT_STEP[SYSTEM]
    counted = prof.get("flops_per_rollout_step") if prof else None
    flops_step = counted or formula_flops
    flops = flops_step * K_SAMPLES * T_STEPS
    roll_mean_s = statistics.mean(roll_ms) / 1e3
    achieved = flops / roll_mean_s / 1e12
    peak = fp32_peak_tflops()
    traffic = prof.get("dram_bytes_per_launch") if prof else None
    cpu = None
    oracle_err = None
    if not args.no_cpu_baseline:
        oracle_err = oracle_errors(N, stream.cuda_stream, 1000 + rank, rank, U_end, it_end)
        # the same iteration with weights spread over many samples (R fixed, a larger temperature),
        # so that the normaliser and the weighted sum are exercised, not just the argmin
        oracle_err = {"headline": oracle_err,
                      "spread_weights": oracle_errors(N, stream.cuda_stream, 1000 + rank, rank, U_end, it_end,
                                                      lam=300.0, R=np.linalg.inv(np.diag([0.3, 0.35])))}
        rate1, iters, _ = oracle_rate(args.cpu_seconds, 1024)
        rate_all, procs = oracle_rate_all_cores(args.cpu_seconds, 1024)
        cpu = {"value": rate_all, "unit": UNIT, "cores": procs, "kind": "oracle",
               "sample": f"{procs} single-threaded oracle processes at once, each running ~{args.cpu_seconds:.0f} s of "
                         f"iterations on its own 1024 of the {K_SAMPLES} samples at full horizon T={T_STEPS} "
                         f"(FP64 numpy); one core alone: {iters} iterations",
               "one_core_value": rate1, "cpu_model": cpu_model(), "nproc": os.cpu_count()}
    lat_ms = sorted(1e3 * x for x in lat)
    plat_ms = sorted(1e3 * x for x in plat)

    def pct(a, q):
        return a[min(len(a) - 1, int(round(q * (len(a) - 1))))]

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": "car on cost-map track (1024x1024 FP32 map), one MPPI iteration + shift per step",
                   "K": K_SAMPLES, "T": T_STEPS, "nu": NU, "lambda": 1.0, "Sigma": [0.3, 0.35],
                   "parallelism": f"{world} independent controller(s), one per GPU",
                   "l2": "flushed between timed steps (256 MB write, outside the timed events)",
                   "x0": "fixed state, receding-horizon warm start with shift"},
        "iters_per_s": value / (K_SAMPLES * T_STEPS),
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 4 * n, "d2h_bytes_per_step": 4 * m,
                "p50_ms": pct(lat_ms, 0.5), "p99_ms": pct(lat_ms, 0.99), "steps": e2e_steps,
                "latency_samples": len(lat_ms), "untimed_warmup_steps": e2e_warm,
                "call": "mppi_step_shift (x0 copied from pinned host memory, u0 written by the update kernel "
                        "into mapped pinned memory; one graph per step, blocking until u0 is on the host)"},
        "plain_loop": {"value": plain_value, "unit": UNIT, "p50_ms": pct(plat_ms, 0.5), "p99_ms": pct(plat_ms, 0.99),
                       "steps": len(plat), "latency_samples": len(plat_ms), "untimed_warmup_steps": plain_warm,
                       "e2e_speedup": e2e_value / plain_value,
                       "what": "unfused: noise->HBM, rollout, min, normaliser, weighted-sum kernels, "
                               "sync per step, no graph"},
        "gpu_launches": launches_per_step * args.steps,
        "launch_note": launch_note,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
                     "traffic": traffic, "kernel": "k_rollout_car_ws<128> (core, noise and pose warps per 128 samples)",
                     "flops_per_rollout_step": flops_step,
                     "flops_basis": ("ncu FP32 thread-instruction counters of the kernel, 2 ffma + fadd + fmul (+ 4 ffma2 + 2 fadd2 + "
                                     "2 fmul2, packed) per rollout-step (profiles/rollout_car_ws_k16384.json)" if counted else
                                     "formula count (no counter record for the current sources)"),
                     "flops_per_rollout_step_formula": formula_flops,
                     "frac_formula": formula_flops * K_SAMPLES * T_STEPS / roll_mean_s / 1e12 / peak,
                     "rollout_ms_mean": 1e3 * roll_mean_s,
                     "peak_basis": "148 SMs x 128 FP32 lanes x 2 flop x 2032 MHz (derived, not measured)",
                     "frac_at_observed_clock": (achieved / fp32_peak_tflops(clk["sm_mhz"])) if clk.get("sm_mhz")
                     else None},
        "clocks": clk,
        "oracle_error": oracle_err,
        "cpu_baseline": cpu,
        "serving": serving_res,
        "serving_heavy": heavy_res and dict(heavy_res, mix=HEAVY_MIX),
        "serving_async": async_res,
        "serving_capacity": capacity_res,
        "systems": systems_res,
        "learned": learned_res,
        "source_hash": source_hash(),
    }
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def main():
    if len(sys.argv) == 3 and sys.argv[1] == "--oracle-child":
        seconds, k_sample, max_iters = json.loads(sys.argv[2])
        print(json.dumps(_oracle_loop(seconds, k_sample, max_iters)))
        return
    args = parse()
    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local_rank = int(os.environ.get("LOCAL_RANK", 0))
    if args.impl == "reference":
        run_reference(args, rank, world)
    else:
        run_ours(args, rank, world, local_rank)


if __name__ == "__main__":
    main()
