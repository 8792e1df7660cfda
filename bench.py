#!/usr/bin/env python3
"""Benchmark: Z-Model high-order steps on one GB300 (and replicas on N GPUs).

Workload (one "step" = one SSP-RK3 step = three derivative evaluations, each running the
geometry pass, the all-pairs Birkhoff-Rott sum, the split reduction and the vorticity/RK3
pass): the 256 x 256 periodic multi-mode interface (65,536 points; z3 = sum of 16 modes with
integer (kx, ky) in [2, 8], amplitudes N(0, 0.01), phases U[0, 2 pi) from seed 0; w = 0;
A = 0.5, g = 1, delta = 0.1 dx, dt = 1e-3) with FP32-compensated Birkhoff-Rott pair terms.
Each step evaluates 3 x 65536^2 = 1.29e10 pair interactions.

Also measured and reported beside the headline (not the headline):
  * the plain FP64 form of the same step (the comparator);
  * the low-order 1024 x 1024 FFT Riesz step (8 modes, amplitude 0.02, A = 0.7);
  * the 32 x 32 single-mode FP64 step (launch bound).

`--impl reference` times the CPU oracle (test infrastructure) on a bounded sample of the same
workload and metric, on this host's cores.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "BR G-pair-interactions/s & Z-Model steps/s vs plain FP64; serve p50/p99 ms"
UNIT = "Gpair/s"
N_SIDE = 256


def _measured_hbm_gbs(default=6795.5):
    """Copy bandwidth (read + write bytes) measured on this GPU model, from the peaks file at the
    repository root when present."""
    try:
        with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["hbm_gbs"])
    except Exception:
        return default


HBM_GBS = _measured_hbm_gbs()
FLOPS_PER_PAIR = 26  # direct-formula FP32 flops per pair interaction (FMA = 2; rsqrt on MUFU)
FP32_LANES = 128     # FP32 FMA lanes per SM (for the derived peak beside the measured one)
CONFIG = {"workload": "multimode-256x256-highorder-fp32c", "n_side": N_SIDE, "points": N_SIDE**2,
          "modes": 16, "order": "high", "precision": "fp32c",
          "pairs_per_step": 3 * N_SIDE**4, "l2": "flushed between timed steps (256 MB write)"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-extras", action="store_true", help="skip the side runs (FP64, low order, 32^2, batch, serving)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving runs")
    ap.add_argument("--serve-compare", action="store_true",
                    help="also serve both traces with the all-resident first-come-first-served policy")
    ap.add_argument("--case", nargs=3, metavar=("KIND", "SIZE", "STEPS"),
                    help="run one small fixed workload for a profiler and exit (no timing, no JSON): "
                         "KIND is low | lowdf | high32 | high32tc | high64 | batch | single")
    return ap.parse_args()


# ---------------------------------------------------------------------------------------------
# helpers
# ---------------------------------------------------------------------------------------------

class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region (every 50 ms: the headline
    region lasts ~0.1 s at 20 steps)."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.rows = []
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "50"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.rows.append([x.strip() for x in line.split(",")])

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=2)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm = [float(r[1]) for r in self.rows if len(r) > 2 and r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if len(r) > 2 and r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = set()
        for r in self.rows:
            for k, nm in enumerate(names):
                if len(r) > 5 + k and r[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": sorted(reasons),
                "samples": len(sm)}


def kernel_source_hash():
    """Of the headline kernel's sources: the kernel and the device code it shares."""
    h = hashlib.sha256()
    for f in ("zm_br32.cu", "zm_br32_common.cuh"):
        h.update(open(os.path.join(ROOT, "paper_2406_05490_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic(tiles):
    """DRAM bytes per Birkhoff-Rott launch from the committed ncu summary, if it was taken on the
    current kernel source with the same tile shape (else None)."""
    p = os.path.join(ROOT, "profiles", "br_fp32c_traffic.json")
    try:
        d = json.load(open(p))
        if d.get("source_sha256_16") == kernel_source_hash() and d.get("tile_shape") == list(tiles):
            return d.get("dram_bytes_per_launch_full_size")
    except Exception:
        pass
    return None


def fp64_inst_record():
    """FP64-pipe thread instructions per unit of work per kernel class, counted by ncu on the
    current kernel sources (profiles/fp64_pipe_instructions.json); an entry whose sources changed
    since the count is dropped (its fraction is then reported as null)."""
    p = os.path.join(ROOT, "profiles", "fp64_pipe_instructions.json")
    try:
        d = json.load(open(p))
    except Exception:
        return {}
    out = {}
    for k, e in d.get("entries", {}).items():
        h = hashlib.sha256()
        try:
            for f in e["sources"]:
                h.update(open(os.path.join(ROOT, f), "rb").read())
        except Exception:
            continue
        if h.hexdigest()[:16] == e.get("source_sha256_16"):
            if "by_side" in e:  # counts that depend on the mesh side: {side: count}
                out[k] = ({int(n): float(v["thread_inst"]) for n, v in e["by_side"].items()}, "by_side")
            else:
                out[k] = (float(e["thread_inst"]), None)
    return out


def df64_issue_record():
    """Warp instructions per point of the double-word low-order kernels by mesh side, counted by
    ncu on the current kernel sources (profiles/df64_issue_instructions.json); {} if the sources
    changed since the count (the issue fractions are then reported as null)."""
    p = os.path.join(ROOT, "profiles", "df64_issue_instructions.json")
    try:
        d = json.load(open(p))
        h = hashlib.sha256()
        for f in d["sources"]:
            h.update(open(os.path.join(ROOT, f), "rb").read())
        if h.hexdigest()[:16] != d.get("source_sha256_16"):
            return {}
        return {k: {int(n): float(v["warp_inst"]) for n, v in e["by_side"].items()}
                for k, e in d["entries"].items()}
    except Exception:
        return {}


def dist_setup(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "gb300" else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(ws, x, device=None):
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ---------------------------------------------------------------------------------------------
# CPU oracle arm
# ---------------------------------------------------------------------------------------------

def oracle_sample_rate(n_targets=1024, seed=0):
    """The oracle's Birkhoff-Rott sum on a bounded sample of the 256^2 workload: n_targets
    seeded targets against all 65,536 sources (geometry and sheet strength computed by the
    oracle on the full mesh first).  Returns (pairs/s, seconds, sample description)."""
    import numpy as np

    import oracle
    from paper_2406_05490_gb300 import inputs
    n = N_SIDE
    z, w = inputs.multi_mode(n, n_modes=16, seed=0)
    # the first stage has w = 0 (gamma = 0); a smooth non-zero w gives the same work per pair
    _, w = inputs.random_state(n, seed=1)
    m = oracle.Mesh(n, periodic=True)
    a1, a2, _, _ = oracle.geometry(m, z)
    gam = oracle.sheet_strength(w, a1, a2)
    idx = np.random.default_rng(seed).choice(n * n, n_targets, replace=False)
    t0 = time.perf_counter()
    oracle.br_velocity(z[:, idx], z, gam, 1.0 / n**2, 0.1 / n)
    dt = time.perf_counter() - t0
    pairs = n_targets * n * n
    return pairs / dt, dt, (f"{n_targets} seeded targets x all {n*n} sources of the 256^2 interface, "
                            "one Birkhoff-Rott evaluation of the oracle (serial FP64, 1 core)")


# ---- the oracle on all host cores: disjoint target slices in spawned worker processes --------------
_ORACLE_ARGS = None


def _oracle_worker_init(z, gam, weight, delta):
    global _ORACLE_ARGS
    import oracle  # noqa: F401  (loads the oracle library once per worker)
    _ORACLE_ARGS = (z, gam, weight, delta)


def _oracle_worker_slice(idx):
    import oracle
    z, gam, weight, delta = _ORACLE_ARGS
    t0 = time.perf_counter()
    oracle.br_velocity(z[:, idx], z, gam, weight, delta)
    return time.perf_counter() - t0


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


class OraclePool:
    """The unchanged oracle Birkhoff-Rott sum of the 256^2 workload, run over disjoint slices of
    seeded targets by one spawned process per host core (no fork after the GPU is in use)."""

    def __init__(self, procs=None):
        import multiprocessing as mp

        import numpy as np

        import oracle
        from paper_2406_05490_gb300 import inputs
        n = N_SIDE
        z, _ = inputs.multi_mode(n, n_modes=16, seed=0)
        _, w = inputs.random_state(n, seed=1)  # non-zero strength: the same work per pair
        m = oracle.Mesh(n, periodic=True)
        a1, a2, _, _ = oracle.geometry(m, z)
        gam = oracle.sheet_strength(w, a1, a2)
        self.n = n
        self.procs = procs or host_cores()
        self.pool = mp.get_context("spawn").Pool(self.procs, initializer=_oracle_worker_init,
                                                 initargs=(z, gam, 1.0 / n**2, 0.1 / n))
        self.pool.map(_oracle_worker_slice, [np.zeros(1, dtype=np.int64)] * self.procs)  # warm up
        self._np = np

    def rate(self, targets_per_proc, seed=0):
        """(pairs/s, wall seconds, sample description) of one evaluation for procs x
        targets_per_proc seeded targets against all sources."""
        np = self._np
        n = self.n
        total = targets_per_proc * self.procs
        idx = np.random.default_rng(seed).choice(n * n, total, replace=False)
        t0 = time.perf_counter()
        self.pool.map(_oracle_worker_slice, np.array_split(idx, self.procs))
        dt = time.perf_counter() - t0
        return total * n * n / dt, dt, (f"{total} seeded targets x all {n*n} sources of the 256^2 "
                                        f"interface, one Birkhoff-Rott evaluation of the oracle (serial "
                                        f"FP64 code) in {self.procs} processes, one per host core")

    def close(self):
        self.pool.close()
        self.pool.join()


def run_reference(args):
    ws, rank, _ = dist_setup(args)
    if rank != 0:
        return 0
    # each step: one bounded sample (256 targets per host core x 65,536 sources)
    pool = OraclePool()
    for _ in range(args.warmup):
        pool.rate(16)
    pairs, secs = 0, 0.0
    sample = ""
    for k in range(args.steps):
        r, dt, sample = pool.rate(256, seed=k)
        pairs += r * dt
        secs += dt
    pool.close()
    value = pairs / secs / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": dict(CONFIG, parallelism="replicas x1"),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
                             "sample": "per step: " + sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------------
# GPU arm
# ---------------------------------------------------------------------------------------------

def run_case(kind, size, steps):
    """A few RK3 steps of one fixed configuration through the C ABI and nothing else, so that a
    profiler (ncu -k / -s / -c) sees a short, known launch sequence:
      low SIZE STEPS      low order, FP64, SIZE^2 periodic 8-mode interface with vorticity
      lowdf SIZE STEPS    the same in double words
      high32 SIZE STEPS   high order, FP32C pair terms
      high32tc SIZE STEPS the same with the far tile pairs on the tensor cores (opt-in path)
      high64 SIZE STEPS   high order, FP64
      batch COUNT STEPS   COUNT ragged interfaces (sides 64-384), FP32C batch
      single SIZE STEPS   single mode on free edges, FP64"""
    import torch

    from paper_2406_05490_gb300 import inputs, zm
    torch.cuda.set_device(0)
    if kind == "batch":
        insts = inputs.ragged_batch(count=size, lo=64, hi=384, n_modes=4, seed=0)
        h = zm.zm_batch_create([(r.n, r.n, 1.0, 1.0, True) for r in insts], [r.atwood for r in insts],
                               delta=[0.1 / r.n for r in insts])
        for k, r in enumerate(insts):
            zm.zm_batch_set_state(h, k, r.z, inputs.random_state(r.n, seed=k)[1])
        zm.zm_batch_step(h, 1e-3, steps)
        zm.zm_batch_sync(h)
        zm.zm_batch_destroy(h)
        return 0
    if kind == "single":
        z, w = inputs.single_mode(size)
        model = zm.ZModel(size, periodic=False, atwood=0.5, g=1.0, delta=0.1 / size)
        model.set_state(z, w)
        model.step(1e-3, steps)
        model.sync()
        model.close()
        return 0
    if kind not in ("low", "lowdf", "high32", "high32tc", "high64"):
        print(run_case.__doc__)
        return 2
    order = zm.ZM_ORDER_LOW if kind in ("low", "lowdf") else zm.ZM_ORDER_HIGH
    z, _ = inputs.multi_mode(size, n_modes=8, seed=7, amp=0.02)
    _, w = inputs.random_state(size, seed=3)
    model = zm.ZModel(size, periodic=True, atwood=0.7, g=1.0, order=order,
                      fp32c=kind in ("high32", "high32tc"), df64=(kind == "lowdf"))
    if kind == "high32tc":
        zm.zm_set_far_path(model.h, zm.ZM_FAR_TENSOR)
    model.set_state(z, w)
    model.step(1e-3, steps)
    model.sync()
    model.close()
    return 0


def measured_fp32_peak(zm, reps=3):
    """The FP32 FMA rate of this GPU measured by the library's probe kernels (scalar FFMA and
    packed FP32x2 FMA chains on every SM), best of `reps` runs each, in TFLOP/s."""
    scalar = max(zm.zm_measure_peak(zm.PEAK_FP32) for _ in range(reps)) / 1e12
    packed = max(zm.zm_measure_peak(zm.PEAK_FP32X2) for _ in range(reps)) / 1e12
    return max(scalar, packed), {"scalar_ffma": scalar, "packed_ffma2": packed}

def timed_steps(model, zm, torch, steps, warmup, flush, profile=True):
    """Device time of `steps` RK3 steps (CUDA events on the context's stream, L2 flushed
    between steps, flush excluded).  Returns (ms_total, profile dict)."""
    stream = torch.cuda.current_stream()
    zm.zm_set_stream(model.h, stream.cuda_stream)
    for _ in range(warmup):
        model.step(1e-3, 1)
    torch.cuda.synchronize()
    zm.zm_set_profiling(model.h, 1 if profile else 0)
    zm.zm_reset_profile(model.h)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        model.step(1e-3, 1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    prof = zm.zm_get_profile(model.h)
    zm.zm_set_profiling(model.h, 0)
    return ms, prof


# Algorithmic HBM bytes per mesh point of each low-order kernel class and launch (8 bytes per
# value in FP64 and in double-word storage alike):
#   geometry   reads z, w (40), writes the normal and q (32);
#   fft        three passes: w -> spectrum (16 + 16), spectrum -> filtered (16 + 16), filtered,
#              normal, q -> u, Phi (48 + 32); the method's floor, one pass reading w, N, q and
#              writing u, Phi, is 80 B;
#   vorticity  reads Phi, y, u, y0 (112), writes the next stage (40).
LOW_BYTES = {"geometry": 72, "fft": 144, "vorticity": 152}
LOW_LAUNCHES_PER_EVAL = {"geometry": 1, "fft": 3, "vorticity": 1}


def bench_low_order(zm, torch, inputs, flush, nl, steps, warmup, df64, fp64_tflops=None, issue_rate=None):
    """Low-order steps on an nl^2 periodic 8-mode interface (amplitude 0.02, A = 0.7): device
    time per step, and per kernel class its time per evaluation and algorithmic HBM GB/s as a
    fraction of the measured copy bandwidth; for the FP64 path also the fraction of the FP64
    pipe it keeps busy (ncu-counted FP64 instructions per point / time / the measured FP64
    instruction rate), the roofline these kernels actually sit on."""
    zl, wl = inputs.multi_mode(nl, n_modes=8, seed=7, amp=0.02)
    ml = zm.ZModel(nl, periodic=True, atwood=0.7, g=1.0, order=zm.ZM_ORDER_LOW, df64=df64)
    ml.set_state(zl, wl)
    del zl, wl
    msl, profl = timed_steps(ml, zm, torch, steps, warmup, flush)
    ml.close()
    pts = nl * nl
    kern = {}
    for k, b in LOW_BYTES.items():
        evals = max(profl["launches"][k] // LOW_LAUNCHES_PER_EVAL[k], 1)
        t = profl["ms"][k] / evals
        gbs = b * pts / (t * 1e-3) / 1e9 if t > 0 else 0.0
        kern[k] = {"ms_per_eval": t, "alg_bytes_per_point": b, "alg_gbs": gbs, "hbm_frac": gbs / HBM_GBS}
        if df64 and issue_rate:
            inst = df64_issue_record().get(k, {}).get(nl)
            kern[k]["warp_inst_per_point"] = inst
            kern[k]["issue_frac"] = inst * pts / (t * 1e-3) / issue_rate if inst and t > 0 else None
        if not df64 and fp64_tflops:
            inst, kind = fp64_inst_record().get(k, (None, None))
            if kind == "by_side":
                inst = inst.get(nl)  # counted per mesh side; None for a side not counted
            kern[k]["fp64_inst_per_point"] = inst
            kern[k]["fp64_pipe_frac"] = (inst * pts / (t * 1e-3) / (fp64_tflops * 1e12 / 2)
                                         if inst and t > 0 else None)
    step_bytes = 3 * sum(LOW_BYTES.values()) * pts
    return {"precision": "double-word (FP32 pairs)" if df64 else "fp64", "points": pts,
            "steps": steps, "steps_per_s": steps / (msl * 1e-3), "ms_per_step": msl / steps,
            "step_alg_gbs": step_bytes / (msl / steps * 1e-3) / 1e9,
            "step_hbm_frac": step_bytes / (msl / steps * 1e-3) / 1e9 / HBM_GBS,
            "issue_basis": ("ncu-counted warp instructions per point (profiles/df64_issue_instructions.json)"
                            " x points / time / (SMs x 4 schedulers x sampled SM clock)") if df64 and issue_rate else None,
            "riesz_floor_gbs": 80 * pts / (kern["fft"]["ms_per_eval"] * 1e-3) / 1e9
            if kern["fft"]["ms_per_eval"] > 0 else 0.0,
            "kernels": kern, "hbm_peak_gbs": HBM_GBS, "hbm_peak_basis": "measured copy bandwidth",
            "fp64_pipe_basis": None if df64 else
            "FP64 instructions per point counted by ncu (profiles/fp64_pipe_instructions.json) / kernel "
            "time / (measured FP64 FMA rate / 2)"}


def bench_batched(zm, torch, inputs, flush, steps=10, warmup=2, count=64):
    """64 periodic interfaces, sides log-uniform in [64, 384] (seed 0), 4 modes, A ~ U[0.2, 0.8],
    FP32C, one graph-replayed RK3 step per timed step; beside it the same interfaces solved one at
    a time (FP32C contexts) and the plain per-instance FP64 form on a sample of them."""
    insts = inputs.ragged_batch(count=count, lo=64, hi=384, n_modes=4, seed=0)
    meshes = [(r.n, r.n, 1.0, 1.0, True) for r in insts]
    h = zm.zm_batch_create(meshes, [r.atwood for r in insts], g=1.0, delta=[0.1 / r.n for r in insts])
    stream = torch.cuda.current_stream()
    zm.zm_batch_set_stream(h, stream.cuda_stream)
    for k, r in enumerate(insts):
        zm.zm_batch_set_state(h, k, r.z, r.w)
    # autotuned tile shape and work-item size on states with vorticity, then the initial states again
    for k, r in enumerate(insts):
        zm.zm_batch_set_state(h, k, r.z, inputs.random_state(r.n, seed=k)[1])
    tiles, chunk, _ = zm.zm_batch_autotune_tiles(h)
    for k, r in enumerate(insts):
        zm.zm_batch_set_state(h, k, r.z, r.w)
    info = zm.zm_batch_info(h)
    zm.zm_batch_step(h, 1e-3, warmup)
    torch.cuda.synchronize()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    for k in range(steps):
        flush.zero_()
        ev[k][0].record(stream)
        zm.zm_batch_step(h, 1e-3, 1)
        ev[k][1].record(stream)
    torch.cuda.synchronize()
    ms = sum(a.elapsed_time(b) for a, b in ev)
    zm.zm_batch_destroy(h)
    pairs_step = 3 * info["pairs_per_eval"]
    out = {"interfaces": count, "sides": [int(r.n) for r in insts], "points": info["points"],
           "autotuned_chunk": chunk, "autotuned_tiles": list(tiles),
           "pairs_per_step": pairs_step, "work_items": info["work_items"], "ctas": info["ctas"],
           "steps": steps, "ms_per_step": ms / steps,
           "gpairs_per_s": pairs_step * steps / (ms * 1e-3) / 1e9}
    # the same interfaces one at a time (FP32C contexts, one step each, L2 flushed between)
    models = []
    for r in insts:
        m = zm.ZModel(r.n, periodic=True, atwood=r.atwood, g=1.0, delta=0.1 / r.n, fp32c=True,
                      stream=stream.cuda_stream)
        m.set_state(r.z, r.w)
        m.step(1e-3, 1)
        models.append(m)
    torch.cuda.synchronize()
    t_ms = 0.0
    for m in models:
        flush.zero_()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        m.step(1e-3, 1)
        b.record(stream)
        torch.cuda.synchronize()
        t_ms += a.elapsed_time(b)
    for m in models:
        m.close()
    out["one_at_a_time_fp32c_gpairs_per_s"] = pairs_step / (t_ms * 1e-3) / 1e9
    # plain per-instance FP64 form on a sample (the smallest, a median and the largest side)
    order = sorted(range(count), key=lambda k: insts[k].n)
    sample = [order[0], order[count // 2], order[-1]]
    f_pairs, f_ms = 0, 0.0
    for k in sample:
        r = insts[k]
        m = zm.ZModel(r.n, periodic=True, atwood=r.atwood, g=1.0, delta=0.1 / r.n, fp32c=False,
                      stream=stream.cuda_stream)
        m.set_state(r.z, r.w)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        m.step(1e-3, 1)
        b.record(stream)
        torch.cuda.synchronize()
        f_ms += a.elapsed_time(b)
        f_pairs += 3 * r.n ** 4
        m.close()
    out["fp64_per_instance_gpairs_per_s"] = f_pairs / (f_ms * 1e-3) / 1e9
    out["fp64_per_instance_sample_sides"] = [int(insts[k].n) for k in sample]
    out["speedup_vs_fp64_per_instance"] = out["gpairs_per_s"] / out["fp64_per_instance_gpairs_per_s"]
    return out


def bench_cutoff(zm, torch, inputs, n=256, cutoffs=(0.05, 0.1, 0.2, 0.4)):
    """Accuracy/performance trade-off of the cutoff sum against the exact all-pairs sum (the
    purpose the paper gives the exact solver, Sec. 3.2.1): one derivative evaluation of the
    256^2 interface with vorticity per cutoff; time of the all-pairs kernel and relative L2
    difference of u from the exact sum."""
    import numpy as np
    z, _ = inputs.multi_mode(n, n_modes=16, seed=0)
    _, w = inputs.random_state(n, seed=1)
    m = zm.ZModel(n, periodic=True, atwood=0.5, g=1.0, delta=0.1 / n, fp32c=True,
                  stream=torch.cuda.current_stream().cuda_stream)
    m.set_state(z, w)

    def one(c):
        zm.zm_set_cutoff(m.h, c)
        m.velocity(want_wdot=False)  # warm-up
        zm.zm_set_profiling(m.h, 1)
        u = m.velocity(want_wdot=False)
        p = zm.zm_get_profile(m.h)
        zm.zm_set_profiling(m.h, 0)
        return u, p["ms"]["br"] / max(p["launches"]["br"], 1)

    u_ex, t_ex = one(0.0)
    rows = []
    for c in cutoffs:
        u, t = one(c)
        rows.append({"cutoff": c, "br_ms": t, "speedup": t_ex / t,
                     "rel_l2_vs_exact": float(np.linalg.norm(u - u_ex) / np.linalg.norm(u_ex))})
    m.close()
    return {"n_side": n, "exact_br_ms": t_ex, "cutoffs": rows}


def serve_trace(zm, trace, budget, slots, dt=1e-3, policy=None, cap=0):
    """Replay a trace through the continuous-batching server; latencies from submission."""
    srv = zm.zm_server_create(budget, slots, g=1.0)
    if policy is not None:
        zm.zm_server_set_policy(srv, policy, cap)
    t0 = time.perf_counter()
    ids = []
    for r in trace:
        while time.perf_counter() - t0 < r.arrival_s:
            time.sleep(min(0.001, max(0.0, r.arrival_s - (time.perf_counter() - t0))))
        ids.append(zm.zm_server_submit(srv, r.n, r.n, r.z, r.w, r.atwood, 0.1 / r.n, dt, r.nsteps))
    lat, bad = [], 0
    for r, rid in zip(trace, ids):
        st = zm.zm_server_wait(srv, rid, 3600.0)
        st, _, _, l, _ = zm.zm_server_result(srv, rid, r.n * r.n)
        bad += st != zm.ZM_OK
        lat.append(l)
    span = time.perf_counter() - t0
    stats = zm.zm_server_get_stats(srv)
    zm.zm_server_destroy(srv)
    import numpy as np
    lat = np.array(lat)
    return {"requests": len(trace), "failed": int(bad), "p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)), "mean_ms": 1e3 * float(lat.mean()),
            "makespan_s": span, "gpairs_per_s": stats["pairs"] / span / 1e9,
            "gpu_busy_frac": stats["busy_s"] / span, "peak_resident": stats["peak_running"],
            "peak_bytes": stats["peak_bytes"], "iterations": stats["iterations"],
            "policy": "srpt" if policy == zm.ZM_SERVE_SRPT else "all",
            "pairs_per_iteration_cap": cap if policy == zm.ZM_SERVE_SRPT else None}


def fp64_sequential_trace(zm, trace, dt=1e-3):
    """The plain per-instance FP64 form as a server: one request at a time in arrival order,
    each on its own FP64 context; latency = completion - arrival."""
    import numpy as np
    t0 = time.perf_counter()
    lat, pairs = [], 0
    for r in trace:
        while time.perf_counter() - t0 < r.arrival_s:
            time.sleep(0.0005)
        m = zm.ZModel(r.n, periodic=True, atwood=r.atwood, g=1.0, delta=0.1 / r.n, fp32c=False)
        m.set_state(r.z, r.w)
        m.step(dt, r.nsteps)
        m.get_state()
        m.close()
        lat.append(time.perf_counter() - t0 - r.arrival_s)
        pairs += 3 * r.nsteps * r.n ** 4
    span = time.perf_counter() - t0
    lat = np.array(lat)
    return {"requests": len(trace), "p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)), "makespan_s": span,
            "gpairs_per_s": pairs / span / 1e9}


def fp64_service_model(zm, inputs, sides=(32, 64, 128, 192, 256), dt=1e-3):
    """Measured service time of one request in the plain per-instance FP64 form (context
    creation, state upload, one RK3 step, state download, teardown), per mesh side; fitted as
    t(n) = a + b * 3 n^4 (fixed cost plus pair interactions) for the queue model below."""
    import numpy as np
    rows = []
    for n in sides:
        z, w = inputs.multi_mode(n, n_modes=4, seed=n)
        best = None
        for _ in range(2):
            t0 = time.perf_counter()
            m = zm.ZModel(n, periodic=True, atwood=0.5, g=1.0, delta=0.1 / n, fp32c=False)
            m.set_state(z, w)
            m.step(dt, 1)
            m.get_state()
            m.close()
            t = time.perf_counter() - t0
            best = t if best is None else min(best, t)
        rows.append((n, best))
    x = np.array([3.0 * n ** 4 for n, _ in rows])
    y = np.array([t for _, t in rows])
    b, a = np.polyfit(x, y, 1)
    return {"a_s": float(max(a, 0.0)), "b_s_per_pair": float(b),
            "measured": [{"side": n, "s_per_step": t} for n, t in rows]}


def fp64_queue_model(model, trace):
    """Latencies of the plain per-instance FP64 form serving `trace` one request at a time in
    arrival order (a single FIFO server), from the measured service times: request k starts at
    max(arrival, previous completion) and takes nsteps * (a + b * 3 n^4)."""
    import numpy as np
    t, lat = 0.0, []
    for r in trace:
        t = max(t, r.arrival_s) + r.nsteps * (model["a_s"] + model["b_s_per_pair"] * 3.0 * r.n ** 4)
        lat.append(t - r.arrival_s)
    lat = np.array(lat)
    return {"requests": len(trace), "p50_ms": 1e3 * float(np.percentile(lat, 50)),
            "p99_ms": 1e3 * float(np.percentile(lat, 99)), "makespan_s": t,
            "kind": "modelled: measured FP64 per-request service times (fp64_service_model) "
                    "replayed through a FIFO queue on the same arrivals"}


SERVE_CAP = 20_000_000_000  # SRPT: pair interactions per server iteration (about 10 ms of GPU work)


def bench_serving(zm, inputs, count=256, budget=16 << 30, slots=64, compare=False):
    """Poisson arrivals at 200/s, sides log-uniform in [32, 512], 20 RK3 steps each (FP32C),
    256 requests, served shortest-remaining-work-first; then a trace of the same kind at about
    70% of the measured capacity; the plain per-instance FP64 form on that same trace (modelled
    from its measured service times: run for real it would take over an hour); and a reduced
    trace (sides [32, 96], 5 steps) served both by the server and, for real, by the plain FP64
    form.  compare=True adds the first-come-first-served all-resident policy on both traces."""
    full = inputs.poisson_trace(count=count, rate_hz=200.0, lo=32, hi=512, nsteps=20, seed=0)
    out = {"offered": serve_trace(zm, full, budget, slots, policy=zm.ZM_SERVE_SRPT, cap=SERVE_CAP)}
    out["offered"]["rate_hz"] = 200.0
    # capacity in pairs/s, measured while the GPU was saturated; the second trace's rate is set
    # from its own mean work per request (sides are heavy-tailed in work ~ n^4, so two traces'
    # means differ a lot).  The same seed draws the same sides at any rate.
    cap_pairs = out["offered"]["gpairs_per_s"] * 1e9
    probe = inputs.poisson_trace(count=count, rate_hz=1.0, lo=32, hi=512, nsteps=20, seed=1)
    mean_pairs = sum(3 * r.nsteps * r.n ** 4 for r in probe) / len(probe)
    rate70 = max(0.7 * cap_pairs / mean_pairs, 0.1)
    t70 = inputs.poisson_trace(count=count, rate_hz=rate70, lo=32, hi=512, nsteps=20, seed=1)
    out["at_70pct_capacity"] = serve_trace(zm, t70, budget, slots, policy=zm.ZM_SERVE_SRPT, cap=SERVE_CAP)
    out["at_70pct_capacity"]["rate_hz"] = rate70
    model = fp64_service_model(zm, inputs)
    out["fp64_service_time_fit"] = model
    out["fp64_per_instance_at_70pct_capacity"] = fp64_queue_model(model, t70)
    out["fp64_per_instance_offered"] = fp64_queue_model(model, full)
    if compare:
        out["offered_policy_all"] = serve_trace(zm, full, budget, slots, policy=zm.ZM_SERVE_ALL)
        out["at_70pct_capacity_policy_all"] = serve_trace(zm, t70, budget, slots, policy=zm.ZM_SERVE_ALL)
    small = inputs.poisson_trace(count=16, rate_hz=200.0, lo=32, hi=96, nsteps=5, seed=2)
    out["reduced_trace"] = {"server_fp32c": serve_trace(zm, small, budget, slots, policy=zm.ZM_SERVE_SRPT,
                                                        cap=SERVE_CAP),
                            "fp64_per_instance_sequential": fp64_sequential_trace(zm, small)}
    return out


def run_gb300(args):
    import numpy as np
    import torch
    ws, rank, local = dist_setup(args)
    torch.cuda.set_device(local)
    from paper_2406_05490_gb300 import inputs, zm
    zm.load()
    dev = torch.device("cuda", local)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 256 MB > L2

    n = N_SIDE
    N = n * n
    z0, w0 = inputs.multi_mode(n, n_modes=16, seed=rank)
    model = zm.ZModel(n, periodic=True, atwood=0.5, g=1.0, delta=0.1 / n, fp32c=True)
    model.set_state(z0, w0)
    # the autotuner times tile shapes and work-item sizes on a state with vorticity (w = 0 makes the first
    # stage's sheet strength vanish), then the interface is reset to its initial state
    model.set_state(z0, inputs.random_state(n, seed=1)[1])
    tiles, chunk = zm.zm_autotune_tiles(model.h)
    model.set_state(z0, w0)

    barrier(ws)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        ms, prof = timed_steps(model, zm, torch, args.steps, args.warmup, flush)
    barrier(ws)
    torch.cuda.synchronize()
    ms_max = allmax(ws, ms, dev)
    pairs_per_step = 3 * N * N
    value = ws * pairs_per_step * args.steps / (ms_max * 1e-3) / 1e9
    steps_per_s = args.steps / (ms_max * 1e-3)
    launches = sum(prof["launches"].values())

    # roofline of the dominant kernel (Birkhoff-Rott sum): ALU bound, FP32.  Denominator: the
    # FP32 FMA rate measured on this GPU by probe kernels; beside it the figure derived from the
    # SM count and the SM clock sampled during the timed region
    br_ms = prof["ms"]["br"] / max(prof["launches"]["br"], 1)
    achieved = FLOPS_PER_PAIR * N * N / (br_ms * 1e-3) / 1e12
    peak, peak_probes = measured_fp32_peak(zm)
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    clk_summary = clk.summary()
    clk_mhz = clk_summary["sm_mhz"] or clk_summary["sm_max_mhz"] or 2070.0
    derived = sm_count * FP32_LANES * 2 * clk_mhz * 1e6 / 1e12
    traffic = recorded_traffic(tiles)

    # end to end through the C ABI with host buffers: H2D state in, one step, D2H state out
    zh = np.ascontiguousarray(z0)
    wh = np.ascontiguousarray(w0)
    try:
        zp = torch.from_numpy(zh).pin_memory()
        wp = torch.from_numpy(wh).pin_memory()
        zo = torch.empty_like(zp).pin_memory()
        wo = torch.empty_like(wp).pin_memory()
    except Exception:
        zp, wp, zo, wo = torch.from_numpy(zh), torch.from_numpy(wh), torch.empty(3, N, dtype=torch.float64), torch.empty(2, N, dtype=torch.float64)
    e2e_model = zm.ZModel(n, periodic=True, atwood=0.5, g=1.0, delta=0.1 / n, fp32c=True)
    zm.zm_autotune_tiles(e2e_model.h)  # the same mesh: the choice above, remembered in this process
    e2e_steps = max(3, min(args.steps, 10))
    for k in range(e2e_steps + 1):
        if k == 1:
            torch.cuda.synchronize()
            t0 = time.perf_counter()
        zm.zm_set_state(e2e_model.h, zp, wp)
        zm.zm_step(e2e_model.h, 1e-3, 1)
        zm.zm_get_state(e2e_model.h, zo, wo)  # host pointers: returns after the copy
    e2e_s = time.perf_counter() - t0
    e2e_s = allmax(ws, e2e_s, dev)
    e2e_model.close()
    e2e_value = ws * pairs_per_step * e2e_steps / e2e_s / 1e9

    extras = {}
    if not args.no_extras:
        # plain FP64 comparator: the same interface, FP64 pair terms
        m64 = zm.ZModel(n, periodic=True, atwood=0.5, g=1.0, delta=0.1 / n, fp32c=False)
        # the headline's FP32C derivative against the FP64 path on the same interface with
        # vorticity (w = 0 makes the velocity vanish), per field: the accuracy side of the
        # FP32C-vs-FP64 comparison (the oracle parity itself is in the tests)
        zq, wq = z0, inputs.random_state(n, seed=1)[1]
        m32 = zm.ZModel(n, periodic=True, atwood=0.5, g=1.0, delta=0.1 / n, fp32c=True)
        u32, wd32 = m32.velocity(zq, wq)
        m32.close()
        u64, wd64 = m64.velocity(zq, wq)
        rl2 = lambda a, b: float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
        extras["fp32c_vs_fp64_rel_l2"] = {"u": rl2(u32, u64), "wdot": rl2(wd32, wd64)}
        m64.set_state(z0, w0)
        k64 = 2
        ms64, prof64 = timed_steps(m64, zm, torch, k64, 1, flush)
        m64.close()
        # its all-pairs kernel against the FP64 FMA rate measured on this GPU by a probe kernel
        br64_ms = prof64["ms"]["br"] / max(prof64["launches"]["br"], 1)
        fp64_ach = FLOPS_PER_PAIR * N * N / (br64_ms * 1e-3) / 1e12
        fp64_peak = max(zm.zm_measure_peak(zm.PEAK_FP64) for _ in range(3)) / 1e12
        br64_inst = fp64_inst_record().get("br64", (None, None))[0]
        extras["fp64_plain"] = {"gpairs_per_s": pairs_per_step * k64 / (ms64 * 1e-3) / 1e9,
                                "steps_per_s": k64 / (ms64 * 1e-3), "ms_per_step": ms64 / k64,
                                "steps": k64,
                                "roofline": {"bound": "fp64 alu", "achieved": fp64_ach, "peak": fp64_peak,
                                             "unit": "TFLOP/s", "frac": fp64_ach / fp64_peak,
                                             "peak_basis": "measured FP64 FMA probe (zm_measure_peak)",
                                             "flops_per_pair": FLOPS_PER_PAIR, "br_ms_per_launch": br64_ms,
                                             "fp64_inst_per_pair": br64_inst,
                                             "fp64_pipe_frac": (br64_inst * N * N / (br64_ms * 1e-3) /
                                                                (fp64_peak * 1e12 / 2)) if br64_inst else None,
                                             "fp64_pipe_basis": "ncu-counted FP64 instructions per pair "
                                                                "(profiles/fp64_pipe_instructions.json) x pairs / "
                                                                "time / (measured FP64 FMA rate / 2)"}}
        extras["fp32c_speedup_vs_fp64"] = value / ws / extras["fp64_plain"]["gpairs_per_s"]
        # low order (FFT Riesz velocity): 1024^2 (the low-vs-high configuration), FP64 and
        # double-word; 4096^2, the largest power-of-two side below the paper's 4864^2 mesh
        issue_rate = sm_count * 4 * clk_mhz * 1e6  # warp instructions per second at one per scheduler per clock
        extras["low_order_1024"] = bench_low_order(zm, torch, inputs, flush, 1024, 10, 3, False, fp64_peak)
        extras["low_order_1024_df64"] = bench_low_order(zm, torch, inputs, flush, 1024, 10, 3, True, issue_rate=issue_rate)
        # the high-order half of the low-vs-high configuration: the same 8-mode interface
        # (amplitude 0.02, A = 0.7) at 512^2, FP32C all-pairs sum, 10 RK3 steps
        nh = 512
        zh8, wh8 = inputs.multi_mode(nh, n_modes=8, seed=7, amp=0.02)
        mh = zm.ZModel(nh, periodic=True, atwood=0.7, g=1.0, delta=0.1 / nh, fp32c=True)
        mh.set_state(zh8, inputs.random_state(nh, seed=1)[1])
        zm.zm_autotune_tiles(mh.h)
        mh.set_state(zh8, wh8)
        kh = 10
        msh, profh = timed_steps(mh, zm, torch, kh, 2, flush)
        mh.close()
        br_h = profh["ms"]["br"] / max(profh["launches"]["br"], 1)
        extras["high_order_512_fp32c"] = {
            "steps": kh, "ms_per_step": msh / kh, "steps_per_s": kh / (msh * 1e-3),
            "gpairs_per_s": 3 * nh**4 * kh / (msh * 1e-3) / 1e9,
            "br_ms_per_launch": br_h,
            "br_frac_of_fp32_peak": FLOPS_PER_PAIR * nh**4 / (br_h * 1e-3) / 1e12 / peak,
            "peak_basis": "measured FP32 FMA probe (as the headline roofline)",
            "kernel_ms_per_step": {k: v / kh for k, v in profh["ms"].items()}}
        extras["low_order_4096"] = bench_low_order(zm, torch, inputs, flush, 4096, 3, 1, False, fp64_peak)
        extras["low_order_4096_df64"] = bench_low_order(zm, torch, inputs, flush, 4096, 5, 2, True, issue_rate=issue_rate)
        # the paper's single-GPU low-order mesh: 4864^2 = (19 x 256)^2, FP64 (radix-19 stage)
        extras["low_order_4864"] = bench_low_order(zm, torch, inputs, flush, 4864, 3, 1, False, fp64_peak)
        extras["low_order_4864_df64"] = bench_low_order(zm, torch, inputs, flush, 4864, 5, 2, True, issue_rate=issue_rate)
        # 32^2 single-mode FP64 (launch bound)
        zs, wsn = inputs.single_mode(32)
        ms_ = zm.ZModel(32, periodic=False, atwood=0.5, g=1.0, delta=0.1 / 32)
        ms_.set_state(zs, wsn)
        k1 = 10
        ms1, _ = timed_steps(ms_, zm, torch, k1, 3, flush, profile=False)
        # per-stage kernel times from a second, event-profiled run (plain launches: profiling
        # replaces the graph replay, so these add up to more than the replayed step)
        ms1p, prof1 = timed_steps(ms_, zm, torch, k1, 1, flush, profile=True)
        ms_.close()
        extras["single_mode_32_fp64"] = {"steps_per_s": k1 / (ms1 * 1e-3), "ms_per_step": ms1 / k1,
                                         "profiled_ms_per_step": ms1p / k1,
                                         "kernel_us_per_stage": {k: 1e3 * v / (3 * k1) for k, v in prof1["ms"].items()
                                                                 if prof1["launches"][k]}}
        # medium order (BR velocity moves the interface, FFT velocity drives the vorticity),
        # 256^2 periodic, FP32C pair terms
        mm = zm.ZModel(n, periodic=True, atwood=0.5, g=1.0, delta=0.1 / n, order=zm.ZM_ORDER_MEDIUM,
                       fp32c=True)
        mm.set_state(z0, w0)
        kmed = 5
        msm, profm = timed_steps(mm, zm, torch, kmed, 2, flush)
        mm.close()
        extras["medium_256_fp32c"] = {"steps_per_s": kmed / (msm * 1e-3), "ms_per_step": msm / kmed,
                                      "gpairs_per_s": pairs_per_step * kmed / (msm * 1e-3) / 1e9,
                                      "kernel_ms_per_step": {k: v / kmed for k, v in profm["ms"].items()}}
        extras["cutoff_tradeoff_256"] = bench_cutoff(zm, torch, inputs)
        extras["batched_64"] = bench_batched(zm, torch, inputs, flush)
        if not args.no_serve:
            extras["serving"] = bench_serving(zm, inputs, compare=args.serve_compare)

    # the same 256^2 all-pairs sum with its far tile pairs on the tensor cores beside the
    # CUDA cores (same work items; the headline uses the CUDA-core far path)
    if not args.no_extras:
        mc = zm.ZModel(n, periodic=True, atwood=0.5, g=1.0, delta=0.1 / n, fp32c=True,
                       stream=torch.cuda.current_stream().cuda_stream)
        mc.set_state(z0, inputs.random_state(n, seed=1)[1])
        zm.zm_set_tile_shape(mc.h, *tiles)
        paths = {}
        for name, path in (("tensor", zm.ZM_FAR_TENSOR), ("cuda", zm.ZM_FAR_CUDA)):
            zm.zm_set_far_path(mc.h, path)
            zm.zm_autotune(mc.h)
            mc.velocity(want_wdot=False)
            zm.zm_set_profiling(mc.h, 1)
            zm.zm_reset_profile(mc.h)
            for _ in range(3):
                flush.zero_()
                mc.velocity(want_wdot=False)
            p = zm.zm_get_profile(mc.h)
            zm.zm_set_profiling(mc.h, 0)
            t = p["ms"]["br"] / max(p["launches"]["br"], 1)
            paths[name] = {"br_ms_per_launch": t, "gpairs_per_s": N * N / (t * 1e-3) / 1e9}
        mc.close()
        extras["far_path_comparison_256"] = paths

    cpu = None
    if rank == 0 and ws == 1:
        rate, secs, sample = oracle_sample_rate(1024)
        pool = OraclePool()
        prate, psecs, psample = pool.rate(1024)
        pool.close()
        cpu = {"value": prate / 1e9, "unit": UNIT, "cores": pool.procs, "kind": "oracle",
               "sample": psample, "seconds": psecs,
               "serial": {"value": rate / 1e9, "cores": 1, "sample": sample, "seconds": secs}}
    model.close()
    if rank != 0:
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32+f64",
        "data": "synthetic",
        "config": dict(CONFIG, parallelism=f"replicas x{ws}", autotuned_chunk=chunk,
                       autotuned_tiles=list(tiles)),
        "steps_per_s": steps_per_s * 1.0,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic, "kernel": "br32_batch_kernel",
                     "peak_basis": "measured: FP32 FMA probe kernels on this GPU (zm_measure_peak, "
                                   "best of scalar FFMA and packed FP32x2 chains, 3 runs each)",
                     "peak_probes": peak_probes,
                     "derived_peak": derived, "derived_frac": achieved / derived,
                     "derived_basis": f"{sm_count} SMs x {FP32_LANES} FP32 lanes x 2 x {clk_mhz:.0f} MHz "
                                      "(median SM clock sampled during the timed region)",
                     "flops_per_pair": FLOPS_PER_PAIR, "br_ms_per_launch": br_ms},
        "cpu_baseline": cpu,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 5 * N * 8,
                "d2h_bytes_per_step": 5 * N * 8},
        "gpu_launches": launches,
        "kernel_ms": prof["ms"], "kernel_launches": prof["launches"],
        "clocks": clk_summary,
    }
    line.update(extras)
    print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.case:
        return run_case(args.case[0], int(args.case[1]), int(args.case[2]))
    if args.impl == "reference":
        return run_reference(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
