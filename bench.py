"""Benchmark of the binary Shan-Chen D2Q9 capillary step on one GB300.

Workload: the single large FP32 capillary, 8192 x 160 lattice, capillary
length 6144 (plates at rows 0 and 129, H = 128), liquid on x < 2560,
G = 1.4, tau_A = tau_B = 1, complete-wetting wall coupling; z(t) and the
FP64 mass sums logged every 50 steps.  A "step" is one lattice time step of
the whole hot path: the fused pull-stream + collide kernel on every node, and
on every 50th step the front reduction and the mass sums.

value     GLUPS (lattice node updates of both species per second, all nodes),
          device time of the timed steps (CUDA events on the library's stream),
          with L2 flushed between timed steps: a 256 MB buffer is written and
          another 256 MB buffer read before every step, outside the timed
          region, so the step starts with none of its data in L2 and no dirty
          flush lines left to write back inside its own time.
e2e       the same metric for the whole job through the C ABI with host
          buffers: initial fields uploaded from pinned host memory, the steps,
          the log and the final densities copied back, inside the timed region.
          The steps run back to back (CUDA graphs, no flush), as in a user's
          loop: part of a step's input is still in L2 from the step before, so
          e2e can exceed value.
roofline  the step kernel: algorithmic bytes (18 populations read + written
          per fluid node, storage precision) / its average launch time,
          against the measured HBM copy bandwidth.
cpu_baseline / --impl reference: the FP64 oracle on the host cores, one
          spawned process per core, each on its own column window of the
          workload.

Multi-GPU (torchrun): every rank advances its own replica of the workload
(independent runs, no data-path collective); the time is the maximum over
ranks and value counts the nodes of all ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "2-species D2Q9 GLUPS & HBM-peak fraction; FP32/batched vs FP64 at stated error"
WORKLOAD = ("binary Shan-Chen D2Q9 capillary 8192x160, L_cap 6144, H 128, FP32 populations, "
            "G 1.4, tau_A = tau_B = 1, complete-wetting wall, z(t) + mass log every 50 steps")
BYTES_PER_NODE = {"f64": 288, "f32": 144, "f16s": 72}
# steps of the first lbm_step call of an autotuned handle: enough for both
# passes of the tuner (up to about 120 candidates x 7 steps, then 3 rounds of
# 4 x 33)
TUNE_STEPS = 2000
KERNELS = ["register", "cp.async", "tma", "pipelined", "split", "l2-prefetch", "smem-staged", "column-pair",
           "node-tile", "bidirectional", "ring", "bidirectional-jit"]
KERNEL_NAMES = ["k_step", "k_step_async", "k_step_tma", "k_step_pf", "k_step_split", "k_step (L2 prefetch)",
                "k_step_smem", "k_step_pair", "k_step_tile", "k_step_bidir", "k_step_ring",
                "k_step_bidir (compiled for the grid)"]
# committed ncu summaries of the step kernel on this workload, by (variant, tile)
# keyed by (kernel, tile, species): species None for alpha = 4/9, m = 1, else --species
SPECIES_1_3 = (4.0 / 9.0, 0.8, 1.0, 25.0 / 9.0)
PROFILES = {
    (11, (64, 18), None, "f32"): os.path.join(ROOT, "profiles", "k_step_bidir_jit_tile64x18_f32_capillary_8192x160.txt"),
    (11, (64, 9), None, "f32"): os.path.join(ROOT, "profiles", "k_step_bidir_jit_tile64x9_f32_capillary_8192x160.txt"),
    (9, (64, 18), None, "f32"): os.path.join(ROOT, "profiles", "k_step_bidir_tile64x18_f32_capillary_8192x160.txt"),
    (9, (64, 9), None, "f32"): os.path.join(ROOT, "profiles", "k_step_bidir_tile64x9_f32_capillary_8192x160.txt"),
    (6, (64, 4), None, "f32"): os.path.join(ROOT, "profiles", "k_step_smem_tile64x4_f32_capillary_8192x160.txt"),
    (10, (128, 4), None, "f32"): os.path.join(ROOT, "profiles", "k_step_ring_depth4_f32_capillary_8192x160.txt"),
    (11, (64, 9), None, "f16s"): os.path.join(ROOT, "profiles", "k_step_bidir_jit_tile64x9_f16s_capillary_8192x160.txt"),
    (11, (64, 18), None, "f16s"): os.path.join(ROOT, "profiles",
                                               "k_step_bidir_jit_tile64x18_f16s_capillary_8192x160.txt"),
    (9, (64, 9), None, "f16s"): os.path.join(ROOT, "profiles", "k_step_bidir_tile64x9_f16s_capillary_8192x160.txt"),
    (6, (128, 4), None, "f64"): os.path.join(ROOT, "profiles", "k_step_smem_tile128x4_f64_capillary_8192x160.txt"),
    (0, (128, 4), None, "f64"): os.path.join(ROOT, "profiles",
                                             "k_step_register_tile128x4_f64_capillary_8192x160.txt"),
    (11, (64, 8), None, "f64"): os.path.join(ROOT, "profiles", "k_step_bidir_jit_tile64x8_f64_capillary_8192x160.txt"),
    (9, (64, 18), SPECIES_1_3, "f32"): os.path.join(ROOT, "profiles",
                                                    "k_step_bidir_species_tile64x18_f32_capillary_8192x160.txt"),
    (11, (64, 18), SPECIES_1_3, "f32"): os.path.join(ROOT, "profiles",
                                                     "k_step_bidir_jit_species_tile64x18_f32_capillary_8192x160.txt"),
}
KERNEL_SOURCES = [os.path.join(ROOT, "paper_0807_0602_gb300", "csrc", f)
                  for f in ("lbm_kernels.cuh", "lbm_ring.cuh", "lbm_launch.cuh", "kernels_f32.cu",
                            "kernels_gen_f32.cu", "lbm_device.h", "lbm_jit.cu")]


# (alpha_A, alpha_B, m_A, m_B) of --species, or None for alpha = 4/9, m = 1
SPECIES = None


def workload(tau_B: float = 1.0):
    import workloads as W
    c = W.config_capillary_8192x160(tau_B=tau_B)
    if SPECIES is not None:
        c["params"] = dict(c["params"], alpha=tuple(SPECIES[:2]), mass=tuple(SPECIES[2:]))
    return c


def _code(text: str) -> str:
    """Source text without its comments and blank lines: the hash follows
    the code that is compiled, not the comments around it."""
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    text = re.sub(r"//[^\n]*", "", text)
    return "\n".join(line.strip() for line in text.splitlines() if line.strip())


def kernel_hash() -> str:
    h = hashlib.sha256()
    for f in KERNEL_SOURCES:
        with open(f, encoding="utf-8") as fh:
            h.update(_code(fh.read()).encode())
    return h.hexdigest()[:16]


def read_traffic(kvar: int, tile, precision: str = "f32"):
    """DRAM bytes per step-kernel launch from the committed ncu summary of
    this kernel variant, tile and precision, or None if there is none or the
    kernel sources changed since the counters were taken."""
    key = (int(kvar), (int(tile[0]), int(tile[1])), SPECIES, precision)
    if key not in PROFILES:
        return None
    try:
        kv = {}
        with open(PROFILES[key]) as fh:
            for line in fh:
                if ":" in line:
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_hash") != kernel_hash() or kv.get("tile") != f"{tile[0]}x{tile[1]}":
            return None
        return float(kv["dram_bytes_per_launch"])
    except (OSError, KeyError, ValueError):
        return None


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as fh:
            d = json.load(fh)
        return float(d["hbm_gbs"]), "measured"
    except (OSError, KeyError, ValueError):
        return 6800.0, "fallback"


class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        try:
            import tempfile
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        reasons = sorted({n for r in rows for n, v in zip(names, r[5:9]) if v.lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def dist_setup(n_gpus: int):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        import torch
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device(f"cuda:{local}"))
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(world, value: float) -> float:
    """Largest value over the ranks (the job's time is its slowest rank's)."""
    if world <= 1:
        return value
    import torch
    import torch.distributed as dist
    dev = "cpu" if dist.get_backend() == "gloo" else "cuda"
    t = torch.tensor([value], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def shard(n_items: int, world: int, rank: int):
    """Contiguous block of independent runs owned by `rank` (no data-path
    exchange between ranks: the runs never communicate)."""
    base, extra = divmod(n_items, world)
    start = rank * base + min(rank, extra)
    return range(start, start + base + (1 if rank < extra else 0))


def ensemble_runs():
    """The uneven 512-run ensemble in the scheme's stable band, each run's wall
    coupling mapped from its target contact angle through a calibration
    table measured on the GPU (sessile droplets, 8000 steps)."""
    import workloads as W
    from paper_0807_0602_gb300 import calibrate as Cb
    runs = W.batch_uneven_capillaries_stable(512, seed=3)
    table = Cb.map_couplings(runs)
    return runs, table


def measure_batched(world: int, rank: int, stream, runs, precision: str = "f32", steps: int = 20,
                    total_steps: int = 20000):
    """The uneven ensemble: 512 independent capillaries (H ~ U{16..128},
    L_cap ~ U{256..4096}, about 1.6e8 nodes, 23 GB of FP32 populations, far
    beyond L2), advanced by one launch per step over one tile table; each
    rank takes its own block of runs.  After the timed steps the same handle
    runs on to total_steps, and every run's mass must still be finite."""
    import numpy as np
    import torch
    from paper_0807_0602_gb300.lbm import Lattice
    from paper_0807_0602_gb300._lib import LbmError
    mine = [runs[i] for i in shard(len(runs), world, rank)]
    nodes = sum(r["geom"]["nx"] * r["geom"]["ny"] for r in mine)
    with torch.cuda.stream(stream):
        lat = Lattice(mine, precision=precision, autotune=True, stream=stream)
        lat.step(TUNE_STEPS)              # autotuning on real steps
        lat.sync()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        barrier(world)
        e0.record(stream)
        lat.step(steps)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        sched = lat.schedule
        lat.step(max(0, total_steps - TUNE_STEPS - steps))
        finite, bad = 0, []
        for r in range(len(mine)):
            try:
                finite += bool(np.all(np.isfinite(lat.mass(r))))
            except LbmError:        # this run's sums are NaN or infinite
                bad.append(r)
        t_done = lat.t
        lat.close()
    ms = max_over_ranks(world, ms)
    total_nodes = nodes * world if world > 1 else nodes
    return {"value": total_nodes / (ms * 1e-3) / 1e9, "unit": "GLUPS", "runs": len(runs),
            "nodes": total_nodes, "ms_per_step": ms, "precision": precision,
            "schedule": {"tile": list(sched[:2]), "kernel": KERNELS[sched[2]]},
            "runs_per_hour_at_2e4_steps": len(runs) * 3600.0 / (ms * 1e-3 * 2e4),
            "alg_GBs": total_nodes * BYTES_PER_NODE[precision] / (ms * 1e-3) / 1e9,
            "finite_runs_after": {"steps": t_done, "finite": finite, "of": len(mine),
                                  "diverged": [dict(run=r, **{k: mine[r]["params"][k] for k in ("G", "tau_B", "G_Aw")},
                                                    H=mine[r]["geom"]["ny"] - 2,
                                                    L=mine[r]["geom"]["cap_x1"] - mine[r]["geom"]["cap_x0"])
                                               for r in bad[:20]]},
            "note": "inputs 23 GB >> L2, no flush needed; all nodes counted; the runs/hour rate is the timed "
                    "step's rate, and every run of the ensemble is still finite after the 2e4 steps it is quoted for"}


def measure_ensemble_accuracy(runs, n_runs: int = 64, steps: int = 20000, log_every: int = 250):
    """FP32 against the FP64 GPU build on the n_runs smallest runs of the
    ensemble (the 64 smallest cost 30 s of FP64; a random subset of the same
    count would cost 270 s): per run the front difference in lattice units
    and the relative difference of the prefactor of Eq. 15's viscous law,
    F(z) = mu_g L z + (mu_l - mu_g) z^2 / 2 against t, whose slope is
    gamma H cos(theta) / 6 (the Washburn prefactor of Eq. 1 is twice that
    over mu_l), fitted over t >= steps / 4 while the front is inside the
    capillary."""
    import numpy as np
    from paper_0807_0602_gb300.lbm import Lattice
    idx = sorted(range(len(runs)), key=lambda r: runs[r]["geom"]["nx"] * runs[r]["geom"]["ny"])[:n_runs]
    sub = [runs[i] for i in idx]
    logs = {}
    for prec in ("f64", "f32"):
        with Lattice(sub, precision=prec, log_every=log_every, log_capacity=steps // log_every + 2) as lat:
            lat.step(steps)
            logs[prec] = [lat.log(r) for r in range(len(sub))]

    def slope(run, lg):
        p = run["params"]
        L = run["geom"]["cap_x1"] - run["geom"]["cap_x0"]
        mu_l, mu_g = 2.04 * (p["tau_A"] - 0.5) / 3.0, 2.04 * (p["tau_B"] - 0.5) / 3.0
        t, z = lg[:, 0], lg[:, 1]
        if not np.all(np.isfinite(z[t >= steps / 4])):    # a diverged run has no prefactor
            return float("nan")
        m = (t >= steps / 4) & (z > 0) & (z < 0.9 * L)
        if m.sum() < 3:
            return float("nan")
        F = mu_g * L * z[m] + 0.5 * (mu_l - mu_g) * z[m] ** 2
        return float(np.polyfit(t[m], F, 1)[0])

    rel, dz = [], []
    for r, run in enumerate(sub):
        a, b = slope(run, logs["f64"][r]), slope(run, logs["f32"][r])
        if np.isfinite(a) and abs(a) > 1e-12 and np.isfinite(b):
            rel.append(abs(b - a) / abs(a))
        dz.append(float(np.max(np.abs(logs["f32"][r][:, 1:4] - logs["f64"][r][:, 1:4]))))   # NaN if not finite
    rel = np.array(rel)
    return {"runs": len(sub), "steps": steps, "prefactor_runs_fitted": int(len(rel)),
            "prefactor_rel_err_max": float(rel.max()) if len(rel) else None,
            "prefactor_rel_err_median": float(np.median(rel)) if len(rel) else None,
            "front_err_lu_max": float(np.nanmax(dz)), "front_err_lu_median": float(np.nanmedian(dz)),
            "runs_not_finite": int(np.sum(~np.isfinite(dz))),
            "selection": f"the {n_runs} runs with the fewest nodes of the 512-run ensemble"}


class Flush:
    """The L2 flush of the timed steps: 256 MB written (evicting the step's
    data), then another 256 MB read (so that L2 holds clean lines and no
    dirty flush line is written back inside the next timed step)."""

    def __init__(self, dev):
        import torch
        self.w = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)   # 2x L2
        self.r = torch.ones(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        self.acc = torch.empty((), dtype=torch.float32, device=dev)

    def __call__(self):
        import torch
        self.w.zero_()
        torch.sum(self.r, 0, out=self.acc)


def timed_steps(lat, stream, flush, steps: int):
    """Per-step CUDA-event durations (ms) of `steps` single steps, each after
    the L2 flush; returns (durations, index of the first step)."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    t0 = lat.t
    for a, b in ev:
        flush()
        a.record(stream)
        lat.step(1)
        b.record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], t0


def select_schedule(lat, stream, flush, steps: int = 24, log_every: int = 50):
    """The autotuner times its candidates on back-to-back steps; the timed
    steps here start after an L2 flush, where the ranking of near-equal
    finalists can differ.  Each of the tuner's finalists is timed for `steps`
    flushed steps (the logged ones left out) and the fastest is kept."""
    import statistics
    fin = lat.tuning()
    if len(fin) < 2:
        return {"finalists": [], "chosen": list(lat.schedule)}
    rows = []
    for sched, ms_b2b in fin:
        lat.schedule = sched
        lat.step(2)
        durs, t0 = timed_steps(lat, stream, flush, steps)
        kern = [d for k, d in enumerate(durs) if log_every <= 0 or (t0 + k + 1) % log_every != 0]
        rows.append({"schedule": list(sched), "kernel": KERNELS[sched[2]], "ms_back_to_back": ms_b2b,
                     "ms_flushed": statistics.median(kern)})
    best = min(rows, key=lambda r: r["ms_flushed"])
    lat.schedule = tuple(best["schedule"])
    return {"finalists": rows, "chosen": best["schedule"],
            "rule": "the tuner's finalists re-timed under this line's protocol (L2 flushed before each step); "
                    "the fastest median kept"}


def fp64_ops_per_node():
    """FP64 instructions per node of the step (DADD + DMUL + DFMA thread
    instructions, from the committed FP64 ncu summary), or None when the
    kernel sources changed since.  Every FP64 step kernel evaluates the same
    canonical arithmetic, so the count holds for each of them."""
    path = PROFILES[(6, (128, 4), None, "f64")]
    try:
        kv = {}
        with open(path) as fh:
            for line in fh:
                if ":" in line and not line.startswith("#"):
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("kernel_hash") != kernel_hash():
            return None
        return float(kv["fp64_ops_per_node"])
    except (OSError, KeyError, ValueError):
        return None


def measure_precision(stream, dev, precision: str, steps: int = 200):
    """The headline workload in another storage precision: autotuned, the
    finalists re-timed under the headline's protocol, then `steps` steps
    timed one by one after the L2 flush (log every 50 steps, logged steps
    left out of the kernel time).  Roofline against HBM; FP64 also against
    the FP64 pipe (its measured rate, lbm_selftest_fp64_rate)."""
    import ctypes
    import numpy as np
    import torch
    import workloads as W
    from paper_0807_0602_gb300 import _lib as L
    from paper_0807_0602_gb300.lbm import Lattice
    c = workload()
    g = c["geom"]
    nodes, fluid = g["nx"] * g["ny"], g["nx"] * g["ny"] - 2 * (g["cap_x1"] - g["cap_x0"])
    shift = W.fp16_shift(dict(geom=g, params=c["params"], init=c["init"])) if precision == "f16s" else (0.0, 0.0)
    with torch.cuda.stream(stream):
        lat = Lattice(dict(geom=g, params=c["params"], init=c["init"]), precision=precision, log_every=50,
                      log_capacity=4096, autotune=True, stream=stream, rho_ref=shift)
        lat.step(TUNE_STEPS)
        lat.sync()
        flush = Flush(dev)
        selection = select_schedule(lat, stream, flush)
        durs, t0 = timed_steps(lat, stream, flush, steps)
        kern = [d for k, d in enumerate(durs) if (t0 + k + 1) % 50 != 0]
        sched = lat.schedule
        finite = bool(np.all(np.isfinite(lat.mass())))
        lat.close()
    kernel_ms = statistics.mean(kern)
    peak, peak_kind = peaks()
    alg = fluid * BYTES_PER_NODE[precision]
    gbs = alg / (kernel_ms * 1e-3) / 1e9
    out = {"value": nodes * steps / (sum(durs) * 1e-3) / 1e9, "unit": "GLUPS", "steps": steps,
           "rho_ref": list(shift), "schedule": {"tile": list(sched[:2]), "kernel": KERNELS[sched[2]]},
           "schedule_selection": selection, "state_finite": finite,
           "roofline": {"bound": "hbm", "achieved": gbs, "peak": peak, "unit": "GB/s", "frac": gbs / peak,
                        "traffic": read_traffic(sched[2], sched[:2], precision), "peak_source": peak_kind,
                        "alg_bytes_per_launch": alg, "kernel_ms": kernel_ms}}
    if precision == "f64":
        rate = ctypes.c_double()
        lib = L.load()
        with torch.cuda.stream(stream):
            L.check(lib.lbm_selftest_fp64_rate(ctypes.byref(rate), ctypes.c_void_p(stream.cuda_stream)),
                    "lbm_selftest_fp64_rate")
        ops = fp64_ops_per_node()
        fp64 = {"bound": "fp64 pipe", "unit": "FP64 instructions/s",
                "peak": rate.value / 2.0, "peak_source": "measured: lbm_selftest_fp64_rate (DFMA chains, "
                                                         "2 flops each) / 2 = DFMA instructions per second",
                "ops_per_node": ops}
        if ops is not None:
            fp64["achieved"] = nodes * ops / (kernel_ms * 1e-3)
            fp64["frac"] = fp64["achieved"] / fp64["peak"]
        out["roofline_fp64"] = fp64
    return out


def measure_density_ratio(stream, dev, precision: str, steps: int = 1000):
    """The workload with the paper's 1:3 species (alpha = (4/9, 0.8),
    m = (1, 25/9)): autotuned, then `steps` steps timed one by one with CUDA
    events after the same L2 flush as the headline, log every 50 steps."""
    import numpy as np
    import torch
    from paper_0807_0602_gb300.lbm import Lattice
    c = workload()
    g = c["geom"]
    prm = dict(c["params"], alpha=SPECIES_1_3[:2], mass=SPECIES_1_3[2:])
    nodes, fluid = g["nx"] * g["ny"], g["nx"] * g["ny"] - 2 * (g["cap_x1"] - g["cap_x0"])
    with torch.cuda.stream(stream):
        lat = Lattice(dict(geom=g, params=prm, init=c["init"]), precision=precision, log_every=50,
                      log_capacity=4096, autotune=True, stream=stream)
        lat.step(TUNE_STEPS)
        lat.sync()
        flush = Flush(dev)
        selection = select_schedule(lat, stream, flush)
        durs, t0 = timed_steps(lat, stream, flush, steps)
        kern = [d for k, d in enumerate(durs) if (t0 + k + 1) % 50 != 0]
        sched = lat.schedule
        finite = bool(np.all(np.isfinite(lat.mass())))
        lat.close()
    kernel_ms = statistics.mean(kern)
    peak, _ = peaks()
    gbs = fluid * BYTES_PER_NODE[precision] / (kernel_ms * 1e-3) / 1e9
    return {"value": nodes * steps / (sum(durs) * 1e-3) / 1e9, "unit": "GLUPS", "steps": steps,
            "alpha": list(SPECIES_1_3[:2]), "mass": list(SPECIES_1_3[2:]), "kernel_ms": kernel_ms,
            "alg_GBs": gbs, "frac": gbs / peak, "schedule": {"tile": list(sched[:2]), "kernel": KERNELS[sched[2]]},
            "schedule_selection": selection, "state_finite": finite}


def measure_accuracy(steps: int = 2000):
    """The error at which the throughput is quoted: FP32 and FP16-shifted
    storage against the FP64 GPU build after `steps` steps of the workload
    at its configured G = 1.4 (FP16S offsets from workloads.fp16_shift: each
    species' density in the majority phase).  Densities: max |n - n_64| over the max of |n_64| (per species,
    worst of the two); fronts: max |z - z_64| in lattice units (bulk and both
    precursors); mass: relative difference; prefactors: the Washburn slope of
    z_bulk^2 against t and the square-root-law prefactors of z_bulk and of the
    mean precursor front against t^(1/2), least-squares fits over the logged
    z(t) for t >= steps/4, relative difference (worst run)."""
    import numpy as np
    import workloads as W
    from paper_0807_0602_gb300.lbm import Lattice

    def state(runs, precision):
        # one handle per run: a run that diverges makes its own handle's state sticky
        from paper_0807_0602_gb300._lib import LbmError
        out = []
        for run in runs:
            shift = W.fp16_shift(run) if precision == "f16s" else (0.0, 0.0)
            with Lattice(run, precision=precision, log_every=50, log_capacity=steps // 50 + 1,
                         rho_ref=shift) as lat:
                lat.step(steps)
                try:
                    out.append((*lat.densities(), lat.interface(), lat.mass(), lat.log()))
                except LbmError:
                    nan = np.full((run["geom"]["ny"], run["geom"]["nx"]), np.nan)
                    out.append((nan, nan, np.full(3, np.nan), np.full(2, np.nan), np.full((1, 6), np.nan)))
        return out

    def prefactors(log):
        t, zb, zp = log[:, 0], log[:, 1], 0.5 * (log[:, 2] + log[:, 3])
        keep = t >= steps / 4
        t, zb, zp = t[keep], zb[keep], zp[keep]
        if len(t) < 3 or not (np.all(np.isfinite(zb)) and np.all(np.isfinite(zp))):
            return (float("nan"),) * 3
        A = np.vstack([t, np.ones_like(t)]).T
        wash = np.linalg.lstsq(A, zb * zb, rcond=None)[0][0]
        A = np.vstack([np.sqrt(t), np.ones_like(t)]).T
        return wash, np.linalg.lstsq(A, zb, rcond=None)[0][0], np.linalg.lstsq(A, zp, rcond=None)[0][0]

    def compare(ref, got):
        # runs whose FP64 state stayed finite (the uneven ensemble samples parameters
        # outside the scheme's stable band: some of its runs diverge)
        ok = [i for i, r in enumerate(ref) if np.all(np.isfinite(r[0])) and np.all(np.isfinite(r[1]))]
        pairs = [(ref[i], got[i]) for i in ok]
        dn = max(float(np.max(np.abs(g[k] - r[k])) / max(float(np.max(np.abs(r[k]))), 1e-300))
                 for r, g in pairs for k in (0, 1))
        dz = max(float(np.nanmax(np.abs(np.asarray(g[2]) - np.asarray(r[2])))) for r, g in pairs)
        dm = max(float(np.max(np.abs(g[3] - r[3]) / r[3])) for r, g in pairs)
        pf = [(prefactors(r[4]), prefactors(g[4])) for r, g in pairs]
        rel = lambda a, b: float(abs(a - b) / max(abs(a), 1e-300))
        return {"density_err_scale_rel": dn, "front_err_lu": dz, "mass_rel": dm, "finite_runs": len(ok),
                "washburn_prefactor_rel": max(rel(a[0], b[0]) for a, b in pf),
                "sqrt_prefactor_bulk_rel": max(rel(a[1], b[1]) for a, b in pf),
                "sqrt_prefactor_precursor_rel": max(rel(a[2], b[2]) for a, b in pf)}

    c = workload()
    run = [dict(geom=c["geom"], params=c["params"], init=c["init"])]
    ref = state(run, "f64")
    res = {"steps": steps, "f32": compare(ref, state(run, "f32")), "f16s": compare(ref, state(run, "f16s"))}
    return res


G_STABLE = 1.0      # the stable band of the velocity-shift scheme (tau_A = tau_B = 1, G <= 1.1)


def measure_capillary_physics(steps: int = 100000, log_every: int = 500,
                              precisions=("f32", "f16s_shift0", "f16s_majority_shift")):
    """The 8192x160 capillary's physics deliverable in the stable band
    (G = 1.0, tau_A = tau_B = 1, the workload's own wall coupling G_Aw = -0.5:
    a sessile-droplet angle of 51 degrees at G = 1.0; stronger couplings
    diverge on this grid before 10^5 steps): 10^5 steps in FP64,
    FP32 and FP16S (shift 0 and the majority shift), each logging z(t) every
    log_every steps; the bulk and precursor square-root prefactors (least
    squares of z against t^(1/2) over t >= steps/10), the Washburn slope of
    z_bulk^2 against t, and the FP32 and FP16S errors against the FP64 GPU
    build (densities relative to the scale, fronts in lattice units, mass,
    prefactors)."""
    import numpy as np
    import workloads as W
    from paper_0807_0602_gb300.lbm import Lattice
    from paper_0807_0602_gb300._lib import LbmError
    c = W.config_capillary_8192x160(tau_B=1.0)
    run = dict(geom=c["geom"], params=dict(c["params"], G=G_STABLE), init=c["init"])

    def one(prec, rho_ref=(0.0, 0.0)):
        t0 = time.perf_counter()
        with Lattice(run, precision=prec, log_every=log_every, log_capacity=steps // log_every + 2,
                     rho_ref=rho_ref) as lat:
            lat.step(steps)
            try:
                out = (*lat.densities(), lat.log(), lat.mass())
            except LbmError:
                out = None
        return out, time.perf_counter() - t0

    def fits(log):
        t, zb, zp = log[:, 0], log[:, 1], 0.5 * (log[:, 2] + log[:, 3])
        m = t >= steps / 10
        if m.sum() < 3 or not (np.all(np.isfinite(zb[m])) and np.all(np.isfinite(zp[m]))):
            return None
        A = np.vstack([np.sqrt(t[m]), np.ones(m.sum())]).T
        Aw = np.vstack([t[m], np.ones(m.sum())]).T
        return dict(sqrt_bulk=float(np.linalg.lstsq(A, zb[m], rcond=None)[0][0]),
                    sqrt_precursor=float(np.linalg.lstsq(A, zp[m], rcond=None)[0][0]),
                    washburn_slope=float(np.linalg.lstsq(Aw, zb[m] ** 2, rcond=None)[0][0]),
                    z_bulk_end=float(zb[-1]), z_precursor_end=float(zp[-1]), z_bulk_start=float(zb[0]))

    ref, t64 = one("f64")
    if ref is None:
        return {"steps": steps, "f64": {"finite": False}}
    res = {"steps": steps, "G": G_STABLE, "G_Aw": run["params"]["G_Aw"], "f64": dict(fits(ref[2]) or {}, seconds=t64)}
    shift = W.fp16_shift(run)
    for key, prec, rr in (("f32", "f32", (0.0, 0.0)), ("f16s_shift0", "f16s", (0.0, 0.0)),
                          ("f16s_majority_shift", "f16s", shift)):
        if key not in precisions:
            continue
        got, secs = one(prec, rr)
        if got is None:
            res[key] = {"finite": False}
            continue
        r = {"rho_ref": list(rr), "seconds": secs}
        for k, name in ((0, "A"), (1, "B")):
            scale = float(np.abs(ref[k]).max())
            r[f"density_err_scale_rel_{name}"] = float(np.abs(got[k] - ref[k]).max() / scale)
        r["front_err_lu"] = float(np.nanmax(np.abs(got[2][:, 1:4] - ref[2][:, 1:4])))
        r["mass_rel"] = float(np.max(np.abs(got[3] - ref[3]) / ref[3]))
        f, f64 = fits(got[2]), fits(ref[2])
        if f and f64:
            for k in ("sqrt_bulk", "sqrt_precursor", "washburn_slope"):
                r[k] = f[k]
                r[k + "_rel_err"] = float(abs(f[k] - f64[k]) / abs(f64[k]))
        res[key] = r
    return res


def measure_surrogate(reps: int = 50):
    """The surrogate network's kernels (include/mlp.h): forward over 4096
    rows, one Adam training step on 512 rows, and the proposal of couplings
    for 64 target angles (1201 candidates each through one forward), timed
    with CUDA events after warm-up; random weights, seeded inputs."""
    import numpy as np
    import torch
    from paper_0807_0602_gb300.surrogate import Surrogate
    rng = np.random.Generator(np.random.PCG64(5))
    X = rng.uniform(-1, 1, size=(4096, 6))
    T = rng.uniform(-1, 1, size=(4096, 3))
    sur = Surrogate(X, T, seed=0, max_batch=4096)
    xd = torch.as_tensor(sur.xn.fwd(X), dtype=torch.float32, device="cuda")
    td = torch.as_tensor(sur.tn.fwd(T), dtype=torch.float32, device="cuda")

    def timed(fn):
        for _ in range(5):
            fn()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps
    fwd_ms = timed(lambda: sur.net.forward(xd))
    train_ms = timed(lambda: sur.net.train_step(xd[:512], td[:512], 1e-3))
    targets = np.cos(np.radians(np.linspace(0.0, 90.0, 64)))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(5):
        sur.propose(targets, (1.0, 1.0, 1.0, 32.0))
    prop_s = (time.perf_counter() - t0) / 5
    flops_fwd = 2 * 4096 * (6 * 128 + 128 * 128 * 2 + 128 * 3)
    return {"forward_rows_per_s": 4096 / (fwd_ms * 1e-3), "forward_ms_4096_rows": fwd_ms,
            "forward_GFLOPs": flops_fwd / (fwd_ms * 1e-3) / 1e9, "train_step_ms_512_rows": train_ms,
            "proposals_per_s": 64 / prop_s, "note": "bf16 mma.sync kernels; GEMMs of at most 128x128"}


def _oracle_window(args):
    """One host process: the FP64 oracle as it stands on the periodic column
    window [x0, x0 + ncols) of the workload, for `steps` steps (after `warm`
    untimed ones) or, with steps = 0, for `budget_s` seconds.  Returns (node
    updates, seconds)."""
    x0, ncols, steps, warm, budget_s, species = args
    import numpy as np
    import oracle
    import workloads as W
    global SPECIES
    SPECIES = species
    c = workload()
    g = c["geom"]
    nA, nB = W.initial_fields(c)
    if ncols >= g["nx"]:
        sub = dict(g)
    else:
        sub = dict(nx=ncols, ny=g["ny"], cap_x0=min(max(0, g["cap_x0"] - x0), ncols),
                   cap_x1=min(max(0, g["cap_x1"] - x0), ncols), y_bot=g["y_bot"], y_top=g["y_top"])
    o = oracle.OracleLattice(sub, c["params"], np.ascontiguousarray(nA[:, x0:x0 + ncols]),
                             np.ascontiguousarray(nB[:, x0:x0 + ncols]))
    o.step(warm)
    t0 = time.perf_counter()
    n = 0
    if steps:
        o.step(steps)
        n = steps
    else:
        while time.perf_counter() - t0 < budget_s:
            o.step(1)
            n += 1
    return ncols * g["ny"] * n, time.perf_counter() - t0


def _oracle_on_all_cores(ncols: int, steps: int, warm: int, budget_s: float):
    """The oracle in one process per host core (spawned, so that no process
    inherits a CUDA context), each on its own column window of the workload;
    returns (GLUPS over all processes, processes, seconds of the slowest)."""
    import multiprocessing as mp
    nproc = os.cpu_count() or 1
    nx = workload()["geom"]["nx"]
    jobs = [(((k * ncols) % max(1, nx - ncols + 1)), ncols, steps, warm, budget_s, SPECIES) for k in range(nproc)]
    with mp.get_context("spawn").Pool(nproc) as pool:
        out = pool.map(_oracle_window, jobs)
    updates = sum(u for u, _ in out)
    slowest = max(t for _, t in out)
    return updates / slowest / 1e9, nproc, slowest


def cpu_baseline(budget_s: float = 15.0):
    """The FP64 oracle as it stands on the host cores: one process per core,
    each stepping a 512-column window of the 8192x160 workload for about
    budget_s seconds (the per-process rate of one thread on the full grid is
    reported beside it)."""
    u, t = _oracle_window((0, workload()["geom"]["nx"], 0, 0, budget_s / 3, SPECIES))
    one = u / t / 1e9
    value, nproc, _ = _oracle_on_all_cores(512, 0, 1, budget_s)
    return {"value": value, "unit": "GLUPS", "cores": nproc, "kind": "oracle",
            "sample": f"FP64 oracle, {nproc} processes (one per host core), each stepping a 512x160 periodic "
                      f"window of the 8192x160 workload for {budget_s:.0f} s",
            "single_thread_full_grid": {"value": one, "unit": "GLUPS", "cores": 1}}


def run_reference(args):
    """Reference arm: the FP64 oracle on the host cores, one process per core,
    each on a window of the workload."""
    world, rank, _ = int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("RANK", "0")), 0
    if rank != 0:
        return 0
    import numpy as np
    import oracle
    import workloads as W
    c = workload()
    g = c["geom"]
    # columns per window sized so that warm-up + timed steps take about 60 s
    nA, nB = W.initial_fields(c)
    probe = oracle.OracleLattice(W.periodic_box(64, g["ny"]), c["params"], nA[:, 1024:1088], nB[:, 1024:1088])
    t0 = time.perf_counter()
    probe.step(3)
    rate = 3 * 64 * g["ny"] / (time.perf_counter() - t0)
    total = max(1, args.steps + args.warmup)
    ncols = int(max(8, min(g["nx"], rate * 60.0 / total / g["ny"])))
    # one process per host core, each on its own window (together at most the
    # whole grid once), the same steps
    ncols = min(ncols, -(-g["nx"] // (os.cpu_count() or 1)))
    value, nproc, dt = _oracle_on_all_cores(ncols, max(1, args.steps), args.warmup, 0.0)
    sample = (f"{nproc} processes (one per host core), each stepping a {ncols}x{g['ny']} " +
              ("grid (the whole workload)" if ncols == g["nx"] else "periodic window of the 8192x160 workload") +
              f" for {args.steps} steps, FP64 oracle")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt / max(1, args.steps) * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": "GLUPS", "cores": nproc, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": "GLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_profile(args):
    """Steps the workload with a fixed schedule and no graphs, for profilers."""
    import torch
    from paper_0807_0602_gb300.build import build as build_lib
    from paper_0807_0602_gb300.lbm import Lattice
    build_lib()
    c = workload()
    w, h, k, d = (int(v) for v in args.schedule.split(","))
    if args.ensemble:
        # the first runs of the uneven ensemble (a few GB, for ncu); the
        # coupling does not change the kernel's work, so it is fixed here
        import workloads as W
        runs = W.batch_uneven_capillaries_stable(512, seed=3)[:args.ensemble]
        for r in runs:
            r["params"]["G_Aw"] = -0.2
        what = runs
    else:
        # the z(t) and mass log every 50 steps as in the timed run
        what = dict(geom=c["geom"], params=c["params"], init=c["init"])
    with Lattice(what, precision=args.precision, tile=(w, h), kernel=(k, d), graph_chunk=-1,
                 log_every=0 if args.ensemble else 50, log_capacity=4096) as lat:
        lat.step(args.profile)
        lat.sync()
    torch.cuda.synchronize()
    print(json.dumps({"profile_steps": args.profile, "schedule": [w, h, k, d], "precision": args.precision,
                      "ensemble_runs": args.ensemble}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=4000)
    ap.add_argument("--warmup", type=int, default=50)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f32", choices=["f32", "f16s", "f64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-batched", action="store_true", help="skip the 512-run ensemble measurement")
    ap.add_argument("--profile", type=int, default=0,
                    help="only step the workload this many times (for ncu captures) and exit")
    ap.add_argument("--schedule", default="128,4,6,4",
                    help="tile_w,tile_h,kernel,depth used by --profile")
    ap.add_argument("--ensemble", type=int, default=0,
                    help="with --profile: step the first this many runs of the uneven ensemble instead")
    ap.add_argument("--species", default=None,
                    help="alpha_A,alpha_B,m_A,m_B: rest fractions (Eqs. 3-5) and molecular masses of the species")
    args = ap.parse_args()
    if args.species:
        global SPECIES
        SPECIES = tuple(float(v) for v in args.species.split(","))
        if len(SPECIES) != 4:
            ap.error("--species takes alpha_A,alpha_B,m_A,m_B")
    if args.impl == "reference":
        return run_reference(args)
    if args.profile:
        return run_profile(args)
    args.warmup = max(3, args.warmup)

    world, rank, local = dist_setup(args.gpus)
    import numpy as np
    import torch
    import workloads as W
    from paper_0807_0602_gb300.build import build as build_lib
    from paper_0807_0602_gb300.lbm import Lattice

    if rank == 0:
        build_lib()
    barrier(world)
    build_lib()
    torch.cuda.set_device(local)
    dev = torch.device(f"cuda:{local}")
    c = workload()
    g = c["geom"]
    nodes = g["nx"] * g["ny"]
    fluid_nodes = nodes - 2 * (g["cap_x1"] - g["cap_x0"])
    log_every = 50
    stream = torch.cuda.Stream(device=dev)
    run = dict(geom=g, params=c["params"], init=c["init"])

    with torch.cuda.stream(stream):
        lat = Lattice(run, precision=args.precision, log_every=log_every, log_capacity=4096, autotune=True,
                      stream=stream)
        lat.step(TUNE_STEPS)   # autotuning: real steps, every schedule gives the same bits
        lat.sync()
        flush = Flush(dev)
        selection = select_schedule(lat, stream, flush, log_every=log_every)
        lat.step(args.warmup)
        lat.sync()
        starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
        logged = []
        t_first = lat.t
        sampler = ClockSampler(local)
        sampler.start()
        time.sleep(0.25)
        barrier(world)
        torch.cuda.synchronize()
        for k in range(args.steps):
            flush()                                       # L2 holds no data of the step, and no dirty lines
            starts[k].record(stream)
            lat.step(1)
            ends[k].record(stream)
            logged.append((t_first + k + 1) % log_every == 0)
        torch.cuda.synchronize()
        barrier(world)
        clocks = sampler.stop()
        durs = [s.elapsed_time(e) for s, e in zip(starts, ends)]
        total_ms = sum(durs)
        kern = [d for d, lg in zip(durs, logged) if not lg]
        kernel_ms = statistics.mean(kern)
        M = lat.mass()
        finite = bool(np.all(np.isfinite(M)))
        sched = lat.schedule
        lat.close()

    total_ms = max_over_ranks(world, total_ms)
    value = world * nodes * args.steps / (total_ms * 1e-3) / 1e9
    n_logs = sum(logged)
    gpu_launches = args.steps + 5 * n_logs  # step kernel + (front scan, front final, mass rows, mass final, log advance)

    # ---- end to end through the C ABI with host buffers ----------------------
    nA0, nB0 = W.initial_fields(c)
    hA = torch.from_numpy(nA0).pin_memory()
    hB = torch.from_numpy(nB0).pin_memory()
    barrier(world)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    with torch.cuda.stream(stream):
        lat2 = Lattice(dict(geom=g, params=c["params"], init=("fields", hA.numpy(), hB.numpy())),
                       precision=args.precision, log_every=log_every, log_capacity=4096, tile=sched[:2],
                       kernel=sched[2:], stream=stream)
        lat2.step(args.steps)
        log = lat2.log()
        dA, dB = lat2.densities()
        lat2.close()
    torch.cuda.synchronize()
    e2e_s = max_over_ranks(world, time.perf_counter() - t0)
    h2d = 2 * nodes * 8
    d2h = log.nbytes + dA.nbytes + dB.nbytes
    e2e = {"value": world * nodes * args.steps / e2e_s / 1e9, "unit": "GLUPS",
           "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
           "steps": args.steps,
           "note": "host wall clock over lbm_create from pinned host fields (21 MB upload), the steps, "
                   "the log and both densities copied back; at a few tens of steps creation and the "
                   "copies dominate, at thousands the steps do"}

    ens_runs, ens_table = (None, None) if args.no_batched else ensemble_runs()
    batched = None if args.no_batched else measure_batched(world, rank, stream, ens_runs, args.precision)
    if batched is not None:
        batched["angle_table"] = ens_table
        batched["parameters"] = ("G ~ U[1.0, 1.1], tau_A = 1, tau_B ~ U[1.0, 1.5], theta ~ U[60, 105] deg mapped to "
                                 "G_Aw through the angle table (the configured G ~ U[1.2, 1.6], tau_B ~ U[0.55, 1.5] "
                                 "diverge within a few thousand steps)")
    ens_acc = (measure_ensemble_accuracy(ens_runs) if (rank == 0 and not args.no_batched) else None)
    physics = (measure_capillary_physics() if (rank == 0 and not args.no_batched) else None)
    density_ratio = (measure_density_ratio(stream, dev, args.precision)
                     if (rank == 0 and not args.no_batched and SPECIES is None) else None)
    others = ({p: measure_precision(stream, dev, p) for p in ("f16s", "f64") if p != args.precision}
              if (rank == 0 and not args.no_batched) else None)
    surrogate = measure_surrogate() if (rank == 0 and not args.no_batched) else None
    accuracy = measure_accuracy() if (rank == 0 and not args.no_batched) else None
    if rank != 0:
        return 0
    peak, peak_kind = peaks()
    alg_bytes = fluid_nodes * BYTES_PER_NODE[args.precision]
    achieved = alg_bytes / (kernel_ms * 1e-3) / 1e9
    traffic = read_traffic(sched[2], sched[:2], args.precision)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": traffic, "peak_source": peak_kind,
                "kernel": f"{KERNEL_NAMES[sched[2]]} (tile {sched[0]}x{sched[1]})",
                "alg_bytes_per_launch": alg_bytes, "kernel_ms": kernel_ms}
    line = {
        "metric": METRIC, "value": value, "unit": "GLUPS", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": args.precision, "data": "synthetic",
        "config": {"workload": WORKLOAD, "grid": [g["nx"], g["ny"]], "fluid_nodes": fluid_nodes,
                   "fluid_GLUPS": value * fluid_nodes / nodes,
                   "precision": args.precision, "tile": list(sched[:2]),
                   "step_kernel": KERNELS[sched[2]], "log_every": log_every,
                   "schedule_selection": selection,
                   "l2": "flushed between timed steps: 256 MB written, then another 256 MB read",
                   "state_finite": finite,
                   "parallelism": f"replicas x{world}",
                   "species": ({"alpha": list(SPECIES[:2]), "mass": list(SPECIES[2:])} if SPECIES
                               else {"alpha": [4 / 9, 4 / 9], "mass": [1.0, 1.0]})},
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": gpu_launches,
        "clocks": clocks,
    }
    if not args.no_batched:
        line["batched"] = batched
        if density_ratio is not None:
            line["density_ratio"] = density_ratio
        if others:
            line["precisions"] = others
        line["surrogate"] = surrogate
        line["accuracy"] = accuracy
        line["accuracy"]["ensemble_f32_vs_f64"] = ens_acc
        line["capillary_physics"] = physics
    if not args.no_cpu_baseline and world == 1:
        line["cpu_baseline"] = cpu_baseline()
    print(json.dumps(line), flush=True)
    return 0


if __name__ == "__main__":
    sys.exit(main())
