#!/usr/bin/env python
"""NEP3 molecular-dynamics throughput on GB300: atom-steps/s of velocity-Verlet NVE.

Default workload: Si diamond, 100^3 conventional cells (8,000,000 atoms), a = 5.43 A,
sigma = 0.05 A, NEP radial/angular cutoffs 5.0/4.0 A, n_max 8/4, basis 8/4, l_max 4/2/1,
50 neurons, random weights (seed 0), 300 K Maxwell-Boltzmann velocities, dt = 1 fs; the
plain FP32 form is `value`, the BF16 tensor-core network form is reported beside it, both
with their force error against the FP64 oracle on the 4096-atom subcell (cells [0, 8)^3).
The two-species PbTe workload (32^3 rocksalt cells, 262,144 atoms, 1000 steps of 2 fs) is
reported as an extra key.

One timed step = one MD step of the whole hot path (drift, neighbour rebuild when
triggered, descriptor + network + angular partial forces, force/virial gather, kick,
energy/virial reductions), replayed from the library's captured CUDA graph. Each step is
bracketed by CUDA events on the launching stream; L2 is flushed (a 256 MiB write) before
every timed step, outside the events.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]
Multi-GPU (torchrun): every rank runs an independent replica of the workload.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import re
import subprocess
import sys
import threading
import time

# more hardware work queues than the default 8, so that the serving workers' streams
# (one per concurrent job) do not share queues (read when the CUDA context is created)
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 256 << 20
METRIC = "NEP atom-steps/s on 1 GB300 (plain vs batched/BF16); p50/p99 request latency"
UNIT = "atom-steps/s"


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=20)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--workload", choices=["pbte", "si", "si_medium", "si_large"], default="si_large",
                    help="si_medium (40^3 cells, 512,000 atoms) is the profiling case of the si_large kernels")
    ap.add_argument("--pbte-steps", type=int, default=1000, help="timed steps of the extra PbTe key (0: skip)")
    ap.add_argument("--skin", type=float, default=None,
                    help="neighbour-list skin (A) of the MD workload (default: 0.3 for the Si boxes, 0.4 for PbTe, "
                         "the fastest of a sweep on each)")
    ap.add_argument("--atom-form", type=int, choices=[0, 1, 3], default=0,
                    help="FP32 per-atom kernel form (nep_tuning.atom_form; 0 = the library's default)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=8.0)
    ap.add_argument("--plain-graph", action="store_true",
                    help="capture the rebuild as ordinary kernel nodes (for kernel-level profilers)")
    ap.add_argument("--no-batch", action="store_true", help="skip the structure-batch and population forms")
    ap.add_argument("--batch-only", action="store_true", help="only the structure-batch and population forms")
    ap.add_argument("--batch-calls", type=int, default=20)
    ap.add_argument("--no-serve", action="store_true", help="skip the serving measurement")
    ap.add_argument("--serve-only", action="store_true", help="only the serving measurement")
    ap.add_argument("--serve-seconds", type=float, default=3.0, help="arrival window of each serving run")
    ap.add_argument("--serve-rate", type=float, default=2000.0, help="Poisson arrival rate (requests/s)")
    ap.add_argument("--serve-workers", type=int, default=1024, help="job slots of the serving batch")
    ap.add_argument("--serve-compact", type=int, default=8,
                    help="lazy leaving of finished jobs (nep_server_config.compact_every; 0 = at once)")
    ap.add_argument("--serve-min-chunk", type=int, default=4,
                    help="least iterations between two reads of the job states (nep_server_config.min_chunk)")
    ap.add_argument("--serve-rate2", type=float, default=0.0,
                    help="arrival rate of the second (sustained-load) serving run; 0 = half the measured FP32 capacity")
    ap.add_argument("--pop-calls", type=int, default=5)
    return ap.parse_args()


def make_workload(name: str):
    from paper_2205_10046_gb300 import workloads as W
    if name == "pbte":
        return W.pbte_rocksalt(32, seed=1)
    if name == "si":
        return W.si_diamond(3, seed=0)
    if name == "si_medium":
        return W.si_diamond(40, seed=0, n_steps=100, dt_fs=1.0)
    return W.si_diamond(100, seed=0, n_steps=100, dt_fs=1.0)


def workload_config(w, name):
    desc = {"pbte": "rocksalt PbTe 32x32x32 conventional cells, a=6.46 A, sigma=0.1 A, 300 K, dt=2 fs",
            "si": "diamond Si 3x3x3 conventional cells, a=5.43 A, sigma=0.05 A, 300 K, dt=1 fs",
            "si_medium": "diamond Si 40x40x40 conventional cells, a=5.43 A, sigma=0.05 A, 300 K, dt=1 fs",
            "si_large": "diamond Si 100x100x100 conventional cells, a=5.43 A, sigma=0.05 A, 300 K, dt=1 fs"}[name]
    m = w.model
    return {"workload": f"{w.name} ({w.n_atoms} atoms): {desc}", "n_atoms": w.n_atoms,
            "nep": f"types={m.n_types} rc={m.rc_radial}/{m.rc_angular} n_max={m.n_max_radial}/{m.n_max_angular} "
                   f"basis={m.basis_radial}/{m.basis_angular} l_max={m.l_max_3b}/{m.l_max_4b}/{m.l_max_5b} "
                   f"neurons={m.n_neuron} random weights",
            "integrator": "velocity Verlet NVE", "l2": "flushed (256 MiB write) before every timed step"}


# ----------------------------------------------------------------------------- flop model
def flop_model(m, T, nr_list, nr_valid, na_list, na_valid):
    """FP32 flops per atom of the two NEP kernels, counted from their arithmetic (FMA = 2).

    Returns (atom_kernel_flops, gather_kernel_flops). Inputs: model shape, number of types,
    mean list lengths (r < r_c + skin) and mean in-cutoff counts (r < r_c) per atom.
    """
    nR, KR, nA, KA, H = m.n_max_radial, m.basis_radial, m.n_max_angular, m.basis_angular, m.n_neuron
    NK = 24
    D = m.n_des
    entry = 12                                   # pair vector, r^2, compare
    cheb = 14 + 4 * max(KR - 1, 0)               # cutoff + Chebyshev f_k
    cheb_a = 14 + 4 * max(KA - 1, 0)
    cheb_d = 25 + 12 * max(KA - 1, 0)            # f_k and f_k'
    poly_b = 100                                 # the 24 homogeneous polynomials
    poly_g = 190                                 # their gradients
    rad_desc = nr_list * entry + nr_valid * (2 + cheb + (KR + 1)) + T * 2 * (nR + 1) * (KR + 1)
    ang_desc = na_list * entry + na_valid * (2 + cheb_a + 2 * (nA + 1) * (KA + 1) + 4 + poly_b + NK
                                             + 2 * (nA + 1) * NK)
    comps = (nA + 1) * 104
    ann = H * (4 * D + 7)
    evec = T * (KR + 1) * (2 * (nR + 1) + 1)
    dS = (nA + 1) * 137
    ang_force = na_list * entry + na_valid * (2 + cheb_d + 4 * (nA + 1) * (KA + 1)
                                              + NK * (4 * (nA + 1) + 12) + poly_b + poly_g + 50)
    atom = rad_desc + ang_desc + comps + ann + evec + dS + ang_force
    rad_force = nr_list * entry + nr_valid * (2 + 25 + 12 * max(KR - 1, 0) + 4 * (KR + 1) + 10 + 9 * 2 + 6)
    ang_gather = na_list * entry + na_valid * (6 + 18)
    gather = rad_force + ang_gather + 12
    return atom, gather


def naive_flop_model(m, nr, na):
    """The naive per-pair estimate of the method (g_n evaluated per pair for every n):
    NN_R [6 (n_R+1)(K_R+1) + 40] + NN_A [6 (n_A+1)(K_A+1) + 240 (n_A+1) + 60] + 4 N_des H + 90 (n_A+1)."""
    nR, KR, nA, KA, H = m.n_max_radial, m.basis_radial, m.n_max_angular, m.basis_angular, m.n_neuron
    return (nr * (6 * (nR + 1) * (KR + 1) + 40) + na * (6 * (nA + 1) * (KA + 1) + 240 * (nA + 1) + 60)
            + 4 * m.n_des * H + 90 * (nA + 1))


# ----------------------------------------------------------------------------- helpers
class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": mx, "reasons": [], "samples": 0}
        sm.sort()
        return {"sm_mhz": sm[len(sm) // 2], "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


def kernel_source_hash() -> str:
    """Hash of the kernel sources with comments and blank lines removed (a comment edit does
    not change the kernels the ncu counters were taken on)."""
    h = hashlib.sha1()
    for f in ("nep_kernels.cuh", "nep_internal.cuh"):
        with open(os.path.join(ROOT, "paper_2205_10046_gb300", "csrc", f)) as fh:
            for line in fh:
                code = line.split("//", 1)[0].rstrip()
                if code:
                    h.update(code.encode() + b"\n")
    return h.hexdigest()[:12]


def profiled_traffic(workload: str):
    """dram bytes per nep_atom launch from the committed ncu summary, if it was taken on the
    current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", f"nep_atom_{workload}.txt")
    if not os.path.exists(path):
        return None
    txt = open(path).read()
    m = re.search(r"kernel_source_sha1:\s*(\w+)", txt)
    b = re.search(r"dram_bytes_per_launch_full_size:\s*([0-9.eE+]+)", txt)
    if not m or not b or m.group(1) != kernel_source_hash():
        return None
    return float(b.group(1))


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class _Null:
    def __enter__(self):
        return self

    def __exit__(self, *a):
        return False


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def max_over_ranks(seconds: float, device, world: int) -> float:
    """The slowest rank's time (every rank gets it): the replicas' job ends when the last one
    does. One process: the time itself."""
    if world <= 1:
        return seconds
    import torch
    import torch.distributed as dist
    t = torch.tensor([seconds], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_rate(world: int, units_per_rank: float, seconds: float) -> float:
    """Whole-job throughput of `world` independent replicas that each processed
    `units_per_rank` units, over the slowest rank's time."""
    return world * units_per_rank / seconds


# ----------------------------------------------------------------------------- CPU oracle
def oracle_sample(w_name: str):
    """A bounded sample of the same workload for the FP64 oracle: the same lattice, model,
    seed, jitter and temperature in a small periodic box (512 atoms PbTe or Si)."""
    from paper_2205_10046_gb300 import workloads as W
    if w_name == "pbte":
        return W.pbte_rocksalt(4, seed=1), "rocksalt PbTe 4x4x4 cells (512 atoms), same model/seed/jitter/300 K"
    if w_name == "si":
        return W.si_diamond(3, seed=0), "diamond Si 3x3x3 cells (216 atoms), same model/seed/jitter/300 K"
    return (W.si_diamond(4, seed=0, n_steps=100, dt_fs=1.0),
            "diamond Si 4x4x4 cells (512 atoms), same model/seed/jitter/300 K")


def cpu_model() -> str:
    """The host CPU's model name (lscpu, else /proc/cpuinfo, else the platform string)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    try:
        for line in open("/proc/cpuinfo"):
            if line.lower().startswith("model name"):
                return line.split(":", 1)[1].strip()
    except Exception:
        pass
    import platform
    return platform.processor() or platform.machine()


def _oracle_md_rate(s, seconds, n_threads):
    """atom-steps/s of the oracle's velocity Verlet on sample s, run for about `seconds`."""
    import oracle
    t0 = time.perf_counter()
    oracle.md(s.model, s.pos, s.vel, s.types, s.box, 1, s.dt_fs, n_threads=n_threads)  # 2 force evaluations
    per_eval = (time.perf_counter() - t0) / 2.0
    steps = max(1, int(seconds / per_eval) - 1)
    t0 = time.perf_counter()
    oracle.md(s.model, s.pos, s.vel, s.types, s.box, steps, s.dt_fs, n_threads=n_threads)
    el = time.perf_counter() - t0
    return s.n_atoms * steps / el, steps, el


def oracle_tiny_run():
    """The tiny configuration as stated, on the oracle: the 216-atom Si diamond box (3x3x3
    cells), one energy/force/virial evaluation, then 100 velocity-Verlet NVE steps of 1 fs, on
    all host cores."""
    import oracle
    from paper_2205_10046_gb300 import workloads as W
    w = W.si_diamond(3, seed=0)
    t0 = time.perf_counter()
    oracle.compute(w.model, w.pos, w.types, w.box)
    t1 = time.perf_counter()
    oracle.md(w.model, w.pos, w.vel, w.types, w.box, 100, w.dt_fs)
    t2 = time.perf_counter()
    return {"workload": f"{w.name} ({w.n_atoms} atoms): one evaluation, then 100 NVE steps of {w.dt_fs} fs",
            "evaluation_s": t1 - t0, "md_s": t2 - t1, "value": w.n_atoms * 100 / (t2 - t1), "unit": UNIT,
            "cores": oracle.max_threads()}


def cpu_baseline(w_name: str, seconds: float):
    """The oracle as it stands, on the host cores: all threads (the reported value) and one
    thread, on a bounded periodic sample of the workload; and the tiny configuration's own run."""
    import oracle
    s, desc = oracle_sample(w_name)
    value, steps, el = _oracle_md_rate(s, seconds, 0)
    one, steps1, el1 = _oracle_md_rate(s, max(2.0, seconds / 2), 1)
    return {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
            "sample": f"{desc}; {steps} velocity-Verlet steps (+1 initial force evaluation) in {el:.1f} s, "
                      f"FP64, OpenMP over atoms",
            "single_thread": {"value": one, "unit": UNIT, "cores": 1,
                              "sample": f"same sample, {steps1} steps in {el1:.1f} s on one thread"},
            "tiny_configuration": oracle_tiny_run(),
            "cpu_model": cpu_model()}


def subcell_reference(w, w_name):
    """FP64 oracle energies and forces of the error sample: for the 8,000,000-atom box the 4096
    atoms of conventional cells [0, 8)^3 (for PbTe the 512 atoms of cells [0, 4)^3), cut out
    with every atom within 2 r_c^R as an open cluster; the small Si box is evaluated whole.
    Returns (indices in the workload, U [n], F [n, 3], description, seconds)."""
    import numpy as np
    import oracle
    from paper_2205_10046_gb300 import workloads as W
    t0 = time.perf_counter()
    if w_name == "si":
        U, F, _ = oracle.compute(w.model, w.pos, w.types, w.box)
        sel, desc = np.arange(w.n_atoms), "the whole periodic box"
    else:
        reps, cells = {"si_large": (100, 8), "si_medium": (40, 8), "pbte": (32, 4)}[w_name]
        cpos, ctypes, cbox, inner, sel = W.subcell_cluster(w, reps, cells)
        U, F, _ = oracle.compute(w.model, cpos, ctypes, cbox, sel=inner)
        desc = (f"{sel.shape[0]} atoms of conventional cells [0,{cells})^3, cut out with every atom within "
                f"2 r_c^R ({cpos.shape[0]} atoms) as an open cluster, step-0 positions")
    return sel, U, F, desc, time.perf_counter() - t0


def _labels_chunk(args):
    """Oracle energies per atom, forces and virials of a chunk of structures (one thread)."""
    import numpy as np
    import oracle
    model, parts = args
    out = []
    for pos, types, box in parts:
        U, F, Wv = oracle.compute(model, pos, types, box, n_threads=1)
        out.append((U.sum() / pos.shape[0], F, oracle.virial6(Wv.sum(0))[0] / pos.shape[0]))
    return out


def population_labels(model, batch):
    """FP64 oracle labels (energy per atom, forces, six virial components per atom) of every
    structure of `batch`, one structure per task over a spawned process pool on all host cores.
    Returns (e [S], F [N, 3], w [S, 6], seconds, processes)."""
    import multiprocessing as mp
    import numpy as np
    import oracle
    oracle.build()
    nproc = max(1, os.cpu_count() or 1)
    parts = [batch.structure(s) for s in range(batch.n_struct)]
    order = np.argsort([-p[0].shape[0] for p in parts], kind="stable")  # largest first
    chunks = [[parts[k] for k in order[c::nproc * 4]] for c in range(nproc * 4)]
    t0 = time.perf_counter()
    with mp.get_context("spawn").Pool(nproc) as pool:
        res = pool.map(_labels_chunk, [(model, c) for c in chunks])
    secs = time.perf_counter() - t0
    e = np.zeros(batch.n_struct)
    w = np.zeros((batch.n_struct, 6))
    F = np.zeros((batch.n_atoms, 3))
    for c, r in enumerate(res):
        for k, (ek, Fk, wk) in zip(order[c::nproc * 4], r):
            a0, a1 = int(batch.offsets[k]), int(batch.offsets[k + 1])
            e[k], w[k], F[a0:a1] = ek, wk, Fk
    return e, F, w, secs, nproc


def form_errors(step0, ref):
    """Force and energy error of each form's step-0 evaluation against the oracle sample."""
    import numpy as np
    sel, U, F, desc, secs = ref
    out = {"sample": desc, "oracle_seconds": secs, "f_rms_eV_per_A": float(np.sqrt(np.mean(F ** 2)))}
    for key, (Fg, Ug) in step0.items():
        d = Fg - F
        out[key] = {"force_rmse_eV_per_A": float(np.sqrt(np.mean(d ** 2))),
                    "force_rmse_meV_per_A": 1e3 * float(np.sqrt(np.mean(d ** 2))),
                    "force_relative_rms": float(np.linalg.norm(d) / max(np.linalg.norm(F), 1e-30)),
                    "energy_error_eV_per_atom": float(abs(Ug.sum() - U.sum()) / U.shape[0]),
                    "site_energy_max_abs_error_eV": float(np.abs(Ug - U).max())}
    return out


def run_reference(args):
    """The oracle timed as it stands on the host cores: one velocity-Verlet run of K steps on
    a bounded sample of the workload (the largest 2^3/3^3/4^3-cell box whose run is estimated
    to finish in about 90 s)."""
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import oracle
    from paper_2205_10046_gb300 import workloads as W
    oracle.build()
    w = make_workload(args.workload)
    maker = (lambda r: W.pbte_rocksalt(r, seed=1)) if args.workload == "pbte" else (lambda r: W.si_diamond(r, seed=0))
    probe = maker(2)
    t0 = time.perf_counter()
    oracle.md(probe.model, probe.pos, probe.vel, probe.types, probe.box, 1, probe.dt_fs)
    per_atom_eval = (time.perf_counter() - t0) / (2 * probe.n_atoms)
    reps = 2
    for r in (3, 4):
        if per_atom_eval * maker(r).n_atoms * (args.steps + args.warmup + 2) < 90.0:
            reps = r
    s = maker(reps)
    pos, vel = s.pos, s.vel
    if args.warmup:
        pos, vel, _, _ = oracle.md(s.model, pos, vel, s.types, s.box, args.warmup, s.dt_fs)
    t0 = time.perf_counter()
    oracle.md(s.model, pos, vel, s.types, s.box, args.steps, s.dt_fs)
    total = time.perf_counter() - t0
    value = s.n_atoms * args.steps / total
    desc = f"{s.name} ({s.n_atoms} atoms), same model/seed/jitter/300 K as the GPU workload"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * total / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(w, args.workload),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": oracle.max_threads(), "kind": "oracle",
                             "sample": f"{desc}; {args.steps} FP64 velocity-Verlet steps in one oracle call"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ----------------------------------------------------------------------------- batched forms
BATCH_SKIN = 0.01  # single-point evaluations rebuild their lists on every call: no skin needed


def _events_timed(fn, calls, warmup, stream, flush):
    """Per-call device time (CUDA events on `stream`, L2 flushed before each call outside the
    events) and host wall time of `calls` calls after `warmup` untimed ones."""
    import torch
    for _ in range(warmup):
        fn()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    dev_ms, wall = [], 0.0
    for c in range(calls):
        flush.fill_(c)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ev0.record(stream)
        fn()
        ev1.record(stream)
        ev1.synchronize()
        wall += time.perf_counter() - t0
        dev_ms.append(ev0.elapsed_time(ev1))
    return sum(dev_ms) / 1e3, wall


def run_batch_forms(args, dev, stream, flush, peak, oracle_labels=True):
    """The structure batch (4096 structures of 8-512 atoms in one evaluation) and the
    population evaluation (64 candidate vectors on a fixed 1024-structure subset against FP64
    oracle labels), FP32 and BF16, with the autotuner's launch shapes."""
    import numpy as np
    import torch
    from paper_2205_10046_gb300 import nep
    from paper_2205_10046_gb300 import workloads as W

    b = W.batch_structures(4096, seed=3)
    model = W.mixed_model(0)
    h = nep.NEP(model, skin=BATCH_SKIN)
    N, S = b.n_atoms, b.n_struct
    p = torch.tensor(b.pos, device=dev)
    t = torch.tensor(b.types, device=dev)
    f64 = dict(dtype=torch.float64, device=dev)
    E = torch.empty(S, **f64)
    F = torch.empty((N, 3), **f64)
    Wv = torch.empty((S, 9), **f64)
    call = lambda: nep.nep_compute_batch(h.h, b.offsets, p, t, b.boxes, None, E, F, None, Wv)
    names = ["neighbor_rebuild", "nep_atom", "nep_gather", "finalize"]
    out = {}
    for prec, key in FORMS:
        nep.nep_set_precision(h.h, prec)
        tune = nep.nep_autotune(h.h, b.offsets, p, t, b.boxes, 0)
        dev_s, wall = _events_timed(call, args.batch_calls, 3, stream, flush)
        nep.nep_set_profiling(h.h, True)  # one eager call with per-kernel events
        call()
        kt = nep.nep_kernel_times(h.h)
        nep.nep_set_profiling(h.h, False)
        st = nep.nep_get_stats(h.h)
        atom_f, gather_f = flop_model(model, model.n_types, st["mean_radial"], st["mean_radial_in_rc"],
                                      st["mean_angular"], st["mean_angular_in_rc"])
        out[key] = {
            "value": N * args.batch_calls / dev_s, "unit": "atom-evaluations/s",
            "structures_per_s": S * args.batch_calls / dev_s, "ms_per_call": 1e3 * dev_s / args.batch_calls,
            "wall_ms_per_call": 1e3 * wall / args.batch_calls,
            "kernel_ms": {k: kt.get(k, 0.0) for k in names},
            "atom_kernel_roofline": {"bound": "alu", "achieved": atom_f * N / (kt["nep_atom"] / 1e3) / 1e12,
                                     "peak": peak, "unit": "TFLOP/s",
                                     "frac": atom_f * N / (kt["nep_atom"] / 1e3) / 1e12 / peak,
                                     "flops_per_atom": atom_f},
            "tuning": {k: tune[k] for k in ("atom_block", "gather_block", "n_tried", "best_ms", "default_ms")},
            "neighbours": {"radial_list": st["mean_radial"], "angular_list": st["mean_angular"]},
        }
    out["workload"] = (f"{S} structures, {N} atoms: atom counts U[8,512], FCC/BCC/diamond with +-10% shear, "
                       f"1-3 of 3 species, sigma 0.1 A; NEP rc 5.5/4.0 n_max 8/4 basis 8/4 l_max 4/2/1 "
                       f"40 neurons (seed 0); lists r_c + {BATCH_SKIN} A rebuilt every call")
    out["path"] = ("nep_compute_batch (graph replay: copy-in, neighbour build, atom + gather kernels, "
                   "per-structure sums, status read)")
    out["gpu_launches_per_call"] = nep.nep_get_stats(h.h)["batch_graph_kernels"]
    out["l2"] = "flushed (256 MiB write) before every timed call"

    # population: 64 candidates on the first 1024 structures, against FP64 oracle labels of
    # the seed-0 model (computed on the host cores before the timed calls)
    sub = b.subset(range(1024))
    Ns = sub.n_atoms
    ps = torch.tensor(sub.pos, device=dev)
    ts = torch.tensor(sub.types, device=dev)
    f64 = dict(dtype=torch.float64, device=dev)
    if oracle_labels:
        e_l, f_l, w_l, label_s, label_procs = population_labels(model, sub)
        label_desc = (f"FP64 oracle energies/forces/virials of the seed-0 model on the 1024 structures "
                      f"({Ns} atoms), {label_s:.1f} s on {label_procs} host processes")
    else:  # --no-cpu-baseline: labels from the FP32 batch path (the cost does not depend on them)
        nep.nep_set_precision(h.h, 0)
        nep.nep_set_tuning(h.h, 0, 0, 0)
        Es = torch.empty(1024, **f64)
        Fs = torch.empty((Ns, 3), **f64)
        Ws = torch.empty((1024, 9), **f64)
        nep.nep_compute_batch(h.h, sub.offsets, ps, ts, sub.boxes, None, Es, Fs, None, Ws)
        torch.cuda.synchronize()
        cnt = np.diff(sub.offsets).astype(np.float64)
        e_l, f_l = Es.cpu().numpy() / cnt, Fs.cpu().numpy()
        w9 = Ws.cpu().numpy() / cnt[:, None]
        w_l = np.stack([w9[:, 0], w9[:, 1], w9[:, 2], 0.5 * (w9[:, 3] + w9[:, 6]), 0.5 * (w9[:, 5] + w9[:, 8]),
                        0.5 * (w9[:, 4] + w9[:, 7])], 1)
        label_desc = "FP32 batch path of the seed-0 model (no oracle run requested)"
    e_tar = torch.tensor(e_l, **f64)
    Fs = torch.tensor(f_l, **f64)
    w_tar = torch.tensor(np.ascontiguousarray(w_l), **f64)
    P = 64
    z = torch.tensor(np.stack([W.mixed_model(100 + k).to_vector() for k in range(P)]), device=dev)
    lam = (1.0, 1.0, 0.1, 0.0, 0.0)
    pop = {}
    for prec, key in FORMS:
        nep.nep_set_precision(h.h, prec)
        tune = nep.nep_autotune(h.h, sub.offsets, ps, ts, sub.boxes, P)
        loss = torch.empty((P, 6), **f64)
        fn = lambda: nep.nep_eval_population(h.h, z, sub.offsets, ps, ts, sub.boxes, e_tar, Fs, w_tar, lam, loss)
        dev_s, wall = _events_timed(fn, args.pop_calls, 1, stream, flush)
        l = loss.cpu().numpy()
        pop[key] = {
            "value": P * Ns * args.pop_calls / dev_s, "unit": "member-atom-evaluations/s",
            "candidates_per_s": P * args.pop_calls / dev_s, "ms_per_call": 1e3 * dev_s / args.pop_calls,
            "wall_ms_per_call": 1e3 * wall / args.pop_calls,
            "tuning": {k: tune[k] for k in ("members_per_launch", "atom_block", "gather_block", "n_tried",
                                            "best_ms", "default_ms")},
            "loss_min_median": [float(l[:, 0].min()), float(np.median(l[:, 0]))],
        }
    pop["workload"] = (f"{P} random candidate vectors (seeds 100..{100 + P - 1}) on 1024 structures "
                       f"({Ns} atoms) of the batch; Eq. loss with lambda_e = lambda_f = 1, lambda_v = 0.1")
    pop["targets"] = label_desc
    if oracle_labels:
        pop["cpu_baseline"] = {"value": Ns / label_s, "unit": "atom-evaluations/s", "cores": label_procs,
                               "kind": "oracle", "sample": label_desc}
    h.close()
    return out, pop


# ----------------------------------------------------------------------------- serving
SERVE_BUDGET = 40 << 30  # bytes of device workspace admitted at once
SERVE_SKIN = 0.4         # neighbour-list skin (A) of the serving batch


def serve_requests(rate, seconds, seed, pool):
    """Poisson arrivals: (arrival time, structure index in the pool, kind, steps)."""
    import numpy as np
    rng = np.random.default_rng(seed)
    t, out = 0.0, []
    while True:
        t += rng.exponential(1.0 / rate)
        if t >= seconds:
            return out
        u = rng.uniform()
        kind, steps = (0, 0) if u < 0.5 else ((1, 50) if u < 0.8 else (2, int(rng.integers(10, 1001))))
        out.append((t, int(rng.integers(0, len(pool))), kind, steps))


def serve_pool(n_pool, seed):
    """Structures of 32-20,000 atoms (log-uniform), 1-3 species, FCC/BCC/diamond, +-10% shear,
    sigma 0.1 A, with 300 K velocities for the NVE jobs."""
    import numpy as np
    from paper_2205_10046_gb300 import workloads as W
    rng = np.random.default_rng(seed)
    m = W.mixed_model(0)
    pool = []
    for k in range(n_pool):
        n = int(np.exp(rng.uniform(np.log(32), np.log(20000))))
        pos, types, box = W.random_structure(200000 + k, n)
        vel = W.maxwell_boltzmann(m.mass[types], 300.0, 300000 + k)
        pool.append((pos, types, box, vel))
    return pool


def serve_sample(pool, reqs):
    """Requests whose served results are checked against the oracle: the first 12 single
    points on structures of at most 2500 atoms and the first 3 NVE jobs of at most 50 steps on
    at most 400 atoms."""
    sp, nve = [], []
    for q, (t, k, kind, steps) in enumerate(reqs):
        n = pool[k][0].shape[0]
        if kind == 0 and n <= 2500 and len(sp) < 12:
            sp.append(q)
        elif kind == 2 and n <= 400 and steps <= 50 and len(nve) < 3:
            nve.append(q)
    return set(sp + nve)


def serve_run(model, pool, reqs, precision, workers, sample=(), compact_every=0, min_chunk=0):
    """Submit the requests at their arrival times; collect every result (with the final
    arrays of the requests in `sample`)."""
    import numpy as np
    from paper_2205_10046_gb300 import nep
    srv = nep.Server(model, memory_budget=SERVE_BUDGET, workers=workers, precision=precision, skin=SERVE_SKIN,
                     compact_every=compact_every, min_chunk=min_chunk)
    done = {}
    offered = 0.0
    lag = []
    kinds, req_of, kept = {}, {}, {}
    lock = threading.Lock()

    def collector():
        while len(done) < len(reqs):
            r = srv.wait(0.5)
            if r is not None:
                with lock:  # the submitting thread has recorded this job
                    q = req_of.get(r["id"])
                if q in sample and r["status"] == 0:
                    kept[q] = (r["energy"], *srv.arrays(r["id"]))
                else:
                    srv.drop(r["id"])
                done[r["id"]] = r

    th = threading.Thread(target=collector)
    th.start()
    t0 = time.perf_counter()
    for q, (t, k, kind, steps) in enumerate(reqs):
        delay = t - (time.perf_counter() - t0)
        if delay > 0:
            time.sleep(delay)
        lag.append(max(0.0, -delay))
        pos, types, box, vel = pool[k]
        with lock:
            jid = srv.submit(kind, pos, types, box, n_steps=steps, dt_fs=1.0, fmax=0.0,
                             vel=vel if kind == 2 else None)
            kinds[jid] = kind
            req_of[jid] = q
        offered += pos.shape[0] * (1 if kind == 0 else steps + 2)
    th.join()
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    res = list(done.values())
    lat = np.array([r["t_done"] - r["t_submit"] for r in res])
    wait = np.array([r["t_start"] - r["t_submit"] for r in res])
    t_first = min(r["t_start"] for r in res)
    t_last = max(r["t_done"] for r in res)
    pct = lambda a, q: float(np.percentile(a, q)) * 1e3 if a.size else None
    by_kind = {}
    for kind, name in ((0, "single_point"), (1, "fire_50"), (2, "nve")):
        lk = np.array([r["t_done"] - r["t_submit"] for r in res if kinds.get(r["id"]) == kind])
        by_kind[name] = {"n": int(lk.size), "p50_ms": pct(lk, 50), "p99_ms": pct(lk, 99)}
    return {
        "requests": len(reqs), "completed": int(st["completed"]), "failed": int(st["failed"]),
        "latency_ms": {"p50": pct(lat, 50), "p90": pct(lat, 90), "p99": pct(lat, 99), "max": pct(lat, 100)},
        "queue_wait_ms": {"p50": pct(wait, 50), "p99": pct(wait, 99)},
        "by_kind": by_kind,
        "throughput_atom_evaluations_per_s": st["atom_evaluations"] / (t_last - t_first),
        "offered_atom_evaluations_per_s": offered / reqs[-1][0],
        "service_seconds": t_last - t_first, "wall_seconds": wall,
        "peak_bytes_reserved": int(st["peak_bytes_reserved"]),
        "submit_lag_ms_p99": float(np.percentile(lag, 99)) * 1e3,
        "errors": sorted({r["message"] for r in res if r["status"] != 0})[:3],
        "scheduler": {"iterations": int(st["iterations"]), "relayouts": int(st["relayouts"]),
                      "builds": int(st["builds"]),
                      "relayout_s": st["relayout_seconds"], "iteration_s": st["step_seconds"],
                      "fetch_s": st["fetch_seconds"]},
    }, kept


def serving_errors(model, pool, reqs, kept_by_form):
    """Force and energy errors of the sampled served results against the FP64 oracle: single
    points at the submitted positions, NVE jobs after the oracle's own velocity Verlet of the
    same steps (dt 1 fs) from the submitted positions and velocities."""
    import numpy as np
    import oracle
    t0 = time.perf_counter()
    refs = {}
    qs = sorted(set().union(*[set(k) for k in kept_by_form.values()]))
    for q in qs:
        t, k, kind, steps = reqs[q]
        pos, types, box, vel = pool[k]
        if kind == 0:
            U, F, _ = oracle.compute(model, pos, types, box)
            refs[q] = (U.sum(), pos, F)
        else:
            p1, v1, th, F = oracle.md(model, pos, vel, types, box, steps, 1.0)
            refs[q] = (th[-1, 0], p1, F)
    out = {"sample": f"{sum(1 for q in qs if reqs[q][2] == 0)} single points (<= 2500 atoms) and "
                     f"{sum(1 for q in qs if reqs[q][2] == 2)} NVE jobs (<= 400 atoms, <= 50 steps) of the "
                     f"2000 req/s stream; NVE against the oracle's velocity Verlet from the same start",
           "oracle_seconds": time.perf_counter() - t0}
    for key, kept in kept_by_form.items():
        d2, f2, de, n_at, dx = 0.0, 0.0, [], 0, 0.0
        for q, (E, pos_g, F_g, _) in kept.items():
            E_ref, pos_ref, F_ref = refs[q]
            d2 += float(np.sum((F_g - F_ref) ** 2))
            f2 += float(np.sum(F_ref ** 2))
            n_at += F_ref.shape[0]
            de.append(abs(E - E_ref) / F_ref.shape[0])
            box = pool[reqs[q][1]][2]
            ds = (pos_g - pos_ref) @ np.linalg.inv(box)
            dx = max(dx, float(np.abs((ds - np.round(ds)) @ box).max()))
        out[key] = {"jobs": len(kept), "force_rmse_meV_per_A": 1e3 * float(np.sqrt(d2 / max(3 * n_at, 1))),
                    "force_relative_rms": float(np.sqrt(d2 / max(f2, 1e-300))),
                    "energy_error_eV_per_atom_max": float(max(de)) if de else None,
                    "position_error_A_max": dx}
    return out


def run_serving(args):
    """Config-4 serving: Poisson arrivals of single-point (50%), 50-step FIRE (30%) and NVE
    (20%, 10-1000 steps of 1 fs) jobs on 32-20,000-atom structures, 40 GB admission budget,
    FP32 and BF16 forms; then both forms again at half the measured FP32 capacity. Returns
    (report, the sampled results of the full-rate runs for the oracle check)."""
    from paper_2205_10046_gb300 import workloads as W
    model = W.mixed_model(0)
    pool = serve_pool(256, 4)
    reqs = serve_requests(args.serve_rate, args.serve_seconds, 5, pool)
    sample = serve_sample(pool, reqs)
    out = {"workload": (f"Poisson {args.serve_rate:.0f} req/s for {args.serve_seconds:.0f} s ({len(reqs)} requests); "
                        f"structures drawn from a pool of 256 (32-20,000 atoms, log-uniform, FCC/BCC/diamond, "
                        f"1-3 of 3 species); 50% single point, 30% 50-step FIRE, 20% NVE U{{10..1000}} steps "
                        f"of 1 fs; NEP rc 5.5/4.0 n_max 8/4 40 neurons; one batch of up to {args.serve_workers} jobs (iteration-level batching), "
                        f"{SERVE_BUDGET >> 30} GB admission budget, compact_every {args.serve_compact}, "
                        f"min_chunk {args.serve_min_chunk}"),
           "latency": "submission (arrival) to result on the host, server clock"}
    kept = {}
    for prec, key in ((0, "fp32"), (1, "bf16")):
        out[key], kept[key] = serve_run(model, pool, reqs, prec, args.serve_workers, sample, args.serve_compact,
                                        args.serve_min_chunk)
    # a load the server sustains: half the FP32 capacity measured above (or a given rate)
    cap = out["fp32"]["throughput_atom_evaluations_per_s"]
    work = out["fp32"]["offered_atom_evaluations_per_s"] / args.serve_rate  # per request
    rate2 = args.serve_rate2 if args.serve_rate2 > 0 else max(10.0, 0.5 * cap / work)
    reqs2 = serve_requests(rate2, args.serve_seconds, 6, pool)
    out["half_capacity"] = {"rate_req_per_s": rate2, "requests": len(reqs2)}
    for prec, key in ((0, "fp32"), (1, "bf16")):
        out["half_capacity"][key], _ = serve_run(model, pool, reqs2, prec, args.serve_workers,
                                                 compact_every=args.serve_compact, min_chunk=args.serve_min_chunk)
    return out, (model, pool, reqs, kept)


# ----------------------------------------------------------------------------- GPU arm
KERNELS = ["md_drift", "neighbor_rebuild", "nep_atom", "nep_gather", "finalize"]
FORMS = ((0, "fp32"), (1, "bf16"), (2, "bf16_split"))
NETWORK = {1: "descriptor->hidden and hidden->dU/dq as BF16 tcgen05 GEMMs, FP32 accumulate",
           2: "as bf16, each operand split into two BF16 terms (hi + lo), products hi.hi + lo.hi + hi.lo"}


def timed_md(nep, h, dt, steps, warmup, stream, flush, world, sampler=None):
    """Warm up, then time `steps` MD steps one graph replay at a time (L2 flushed before
    each, outside the events). Returns (seconds, per-kernel ms totals, rebuilds)."""
    import torch
    nep.md_run(h.h, max(warmup, 3), dt, 1, None)
    torch.cuda.synchronize()
    ktime = {k: 0.0 for k in KERNELS}
    step_ms = []
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    if world > 1:
        import torch.distributed as dist
        dist.barrier()
    torch.cuda.synchronize()
    r0 = nep.nep_get_stats(h.h)["n_rebuilds"]
    ctx = sampler if sampler is not None else _Null()
    with ctx:
        for s in range(steps):
            flush.fill_(s)
            ev0.record(stream)
            nep.md_run_async(h.h, 1, dt, 1, None, stream.cuda_stream)
            ev1.record(stream)
            kt = nep.nep_kernel_times(h.h)  # synchronises on this step's last kernel
            ev1.synchronize()
            step_ms.append(ev0.elapsed_time(ev1))
            for k in KERNELS:
                ktime[k] += kt.get(k, 0.0)
            if (s + 1) % 100 == 0:
                nep.md_status(h.h, stream.cuda_stream)  # list health, outside the timed events
    nep.md_status(h.h)
    torch.cuda.synchronize()
    tot = max_over_ranks(sum(step_ms) / 1e3, flush.device, world)
    return tot, ktime, nep.nep_get_stats(h.h)["n_rebuilds"] - r0


def atom_roofline(w, stats, atom_ms, peak, peak_basis, traffic=None):
    atom_f, gather_f = flop_model(w.model, w.model.n_types, stats["mean_radial"], stats["mean_radial_in_rc"],
                                  stats["mean_angular"], stats["mean_angular_in_rc"])
    achieved = atom_f * w.n_atoms / (atom_ms / 1e3) / 1e12
    return {"kernel": "nep_atom", "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": achieved / peak, "traffic": traffic, "flops_per_atom": atom_f, "peak_basis": peak_basis}, gather_f


def md_forms(nep, w, name, skin, steps, warmup, stream, flush, world, clk=None, step0_sel=None,
             plain_graph=False, atom_form=0):
    """Every network form of the MD workload w on one handle: optional step-0 evaluations
    (forces and site energies of the atoms step0_sel, for the error against the oracle), then
    `steps` timed MD steps per form from the same start state. Returns (handle, results)."""
    import torch
    dev = flush.device
    h = nep.NEP(w.model, skin=skin)
    nep.nep_set_tuning(h.h, 0, 0, 0, atom_form)
    pos_d = torch.tensor(w.pos, device=dev)
    types_d = torch.tensor(w.types, device=dev)
    vel_d = torch.tensor(w.vel, device=dev)
    step0 = {}
    if step0_sel is not None:
        sel_d = torch.tensor(step0_sel, device=dev, dtype=torch.int64)
        for prec, key in FORMS:
            nep.nep_set_precision(h.h, prec)
            r = h.compute(pos_d, types_d, w.box)
            step0[key] = (r["F"][sel_d].cpu().numpy(), r["U"][sel_d].cpu().numpy())
            del r
        torch.cuda.synchronize()
    nep.nep_set_profiling(h.h, True)
    nep.nep_set_graph_conditional(h.h, not plain_graph)
    res = {}
    for prec, key in FORMS:
        nep.nep_set_precision(h.h, prec)
        nep.md_init(h.h, pos_d, types_d, w.box, vel_d)
        tot, ktime, rebuilds = timed_md(nep, h, w.dt_fs, steps, warmup, stream, flush, world,
                                        clk if prec == 0 else None)
        res[key] = {"seconds": tot, "ktime": ktime, "rebuilds": rebuilds, "stats": nep.nep_get_stats(h.h),
                    "atom_form": nep.nep_get_tuning(h.h)["atom_form"]}
    nep.nep_set_precision(h.h, 0)
    del pos_d, types_d, vel_d
    return h, res, step0


# MD steps of the configuration's own run, by workload (the 8,000,000-atom box: 100 NVE steps)
CONFIG_STEPS = {"si_large": 100}


def config_run(nep, h, w, steps, stream, flush, world):
    """The configuration's own MD run in every network form: md_init from the initial state,
    then `steps` steps in one md_run_async call (no warm-up), timed with CUDA events on the
    launching stream (L2 flushed once before). Leaves the handle in the FP32 form."""
    import torch
    dev = flush.device
    pos_d, types_d, vel_d = (torch.tensor(a, device=dev) for a in (w.pos, w.types, w.vel))
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    out = {"steps": steps, "from": "md_init of the initial state, no warm-up, one md_run_async call"}
    for prec, key in FORMS:
        nep.nep_set_precision(h.h, prec)
        nep.md_init(h.h, pos_d, types_d, w.box, vel_d)
        r0 = nep.nep_get_stats(h.h)["n_rebuilds"]
        flush.fill_(prec)
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()
        ev0.record(stream)
        nep.md_run_async(h.h, steps, w.dt_fs, steps, None, stream.cuda_stream)
        ev1.record(stream)
        ev1.synchronize()
        nep.md_status(h.h)
        sec = max_over_ranks(ev0.elapsed_time(ev1) / 1e3, dev, world)
        out[key] = {"value": replica_rate(world, w.n_atoms * steps, sec), "unit": UNIT, "ms_per_step": 1e3 * sec / steps,
                    "rebuilds": nep.nep_get_stats(h.h)["n_rebuilds"] - r0}
    nep.nep_set_precision(h.h, 0)
    return out


def run_gb300(args):
    import numpy as np
    import torch
    from paper_2205_10046_gb300 import nep
    from paper_2205_10046_gb300 import workloads as W

    rank, world, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())
    import __graft_entry__ as ge
    if rank == 0 or world == 1:
        ge.build()
    if world > 1:
        dist.barrier()
    nep.load()

    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.int32, device=dev)
    props = torch.cuda.get_device_properties(dev)
    fp32_peak_2070 = props.multi_processor_count * 128 * 2 * 2070e6 / 1e12
    if args.serve_only:
        clk = ClockSampler(torch.cuda.current_device() if world == 1 else local)
        with clk:
            sv, sv_sample = run_serving(args)
        if rank == 0:
            if not args.no_cpu_baseline:
                sv["force_error_vs_fp64_oracle"] = serving_errors(*sv_sample)
            print(json.dumps({"serving": sv, "clocks": clk.summary()}), flush=True)
        return 0
    if args.batch_only:
        clk = ClockSampler(torch.cuda.current_device() if world == 1 else local)
        with clk:
            bf, pf = run_batch_forms(args, dev, stream, flush, fp32_peak_2070,
                                     oracle_labels=not args.no_cpu_baseline and world == 1)
        if rank == 0:
            print(json.dumps({"batch_form": bf, "population": pf, "clocks": clk.summary()}), flush=True)
        return 0

    w = make_workload(args.workload)
    N = w.n_atoms
    if args.workload == "si_large":
        err_sel = W.subcell_cluster(w, 100, 8)[4]
    elif args.workload == "pbte":
        err_sel = W.subcell_cluster(w, 32, 4)[4]
    elif args.workload == "si_medium":
        err_sel = W.subcell_cluster(w, 40, 8)[4]
    else:
        err_sel = np.arange(N)
    clk = ClockSampler(torch.cuda.current_device() if world == 1 else local)
    h, md, step0 = md_forms(nep, w, args.workload, args.skin, args.steps, args.warmup, stream, flush, world, clk,
                            err_sel, args.plain_graph, args.atom_form)
    stats = md["fp32"]["stats"]
    total_s, ktime, timed_rebuilds = md["fp32"]["seconds"], md["fp32"]["ktime"], md["fp32"]["rebuilds"]
    nep.nep_set_profiling(h.h, False)
    crun = config_run(nep, h, w, CONFIG_STEPS[args.workload], stream, flush, world) \
        if args.workload in CONFIG_STEPS else None

    # end-to-end through the host-pointer entry points: upload from page-locked host memory,
    # run, read the state back into page-locked host memory
    thermo_every = min(100, args.steps)
    th = torch.zeros((max(1, args.steps // thermo_every), 4), dtype=torch.float64, device=dev)
    pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).pin_memory().numpy()
    pos_h, types_h, vel_h = pin(w.pos, np.float64), pin(w.types, np.int32), pin(w.vel, np.float64)
    out_h = [torch.empty((N, 3), dtype=torch.float64).pin_memory().numpy() for _ in range(3)]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    nep.md_init_host(h.h, pos_h, types_h, w.box, vel_h)
    nep.md_run_async(h.h, args.steps, w.dt_fs, thermo_every, th, stream.cuda_stream)
    nep.md_status(h.h)
    th_host = th.cpu()
    p_out, v_out, f_out = nep.md_get_state_host(h.h, N, *out_h)
    e2e_s = max_over_ranks(time.perf_counter() - t0, dev, world)
    h2d = N * (24 + 4 + 24) + 72
    d2h = N * 72 + th_host.numel() * 8
    etot = (th_host[:, 0] + th_host[:, 1]).numpy()
    h.close()
    del p_out, v_out, f_out

    # the two-species workload as an extra key, with its own fixed step count
    pbte = None
    if args.pbte_steps > 0 and args.workload != "pbte":
        wp = W.pbte_rocksalt(32, seed=1)
        hp, mp, _ = md_forms(nep, wp, "pbte", args.pbte_skin, args.pbte_steps, 20, stream, flush, world,
                             atom_form=args.atom_form)
        hp.close()
        pbte = {"workload": workload_config(wp, "pbte")["workload"], "steps": args.pbte_steps, "warmup": 20,
                "neighbour_skin_A": args.pbte_skin}
        for key in mp:
            r = mp[key]
            rl, _ = atom_roofline(wp, r["stats"], r["ktime"]["nep_atom"] / args.pbte_steps, fp32_peak_2070,
                                  "152 SMs x 128 FP32 lanes x 2 x 2070 MHz")
            pbte[key] = {"value": world * wp.n_atoms * args.pbte_steps / r["seconds"], "unit": UNIT,
                         "ms_per_step": 1e3 * r["seconds"] / args.pbte_steps,
                         "kernel_ms_per_step": {k: v / args.pbte_steps for k, v in r["ktime"].items()},
                         "atom_kernel_frac_of_fp32_peak": rl["frac"], "rebuilds": r["rebuilds"]}
        del wp

    batch_forms = None
    if not args.no_batch:
        with ClockSampler(torch.cuda.current_device() if world == 1 else local) as bclk:
            batch_forms = run_batch_forms(args, dev, stream, flush, fp32_peak_2070,
                                          oracle_labels=not args.no_cpu_baseline and world == 1)
        batch_forms[0]["clocks"] = bclk.summary()
    serving = None
    if not args.no_serve and world == 1:
        with ClockSampler(torch.cuda.current_device()) as sclk:
            serving, serving_sample = run_serving(args)
        serving["clocks"] = sclk.summary()
    if rank == 0:
        clocks = clk.summary()
        sm_max = clocks.get("sm_max_mhz") or 2070.0
        peak = props.multi_processor_count * 128 * 2 * sm_max * 1e6 / 1e12  # FP32 FMA lanes
        basis = f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 x {sm_max:.0f} MHz"
        roof, gather_f = atom_roofline(w, stats, ktime["nep_atom"] / args.steps, peak, basis,
                                       profiled_traffic(args.workload))
        value = replica_rate(world, N * args.steps, total_s)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": dict(workload_config(w, args.workload), parallelism=f"replicas x{world}",
                           neighbour_skin_A=args.skin, atom_form=md["fp32"]["atom_form"]),
            "roofline": roof,
            "kernel_ms_per_step": {k: v / args.steps for k, v in ktime.items()},
            "gather_roofline": {"achieved": gather_f * N / (ktime["nep_gather"] / args.steps / 1e3) / 1e12,
                                "unit": "TFLOP/s", "flops_per_atom": gather_f},
            "e2e": {"value": world * N * args.steps / e2e_s, "unit": UNIT,
                    "h2d_bytes_per_step": h2d / args.steps, "d2h_bytes_per_step": d2h / args.steps,
                    "path": f"md_init_host + md_run_async + md_status + md_get_state_host, page-locked host "
                            f"buffers (thermo every {thermo_every})"},
            "gpu_launches": int(stats["graph_kernels"]) * args.steps + int(stats["rebuild_kernels"]) * timed_rebuilds,
            "clocks": clocks,
            "neighbours": {"radial_list": stats["mean_radial"], "radial_in_rc": stats["mean_radial_in_rc"],
                           "angular_list": stats["mean_angular"], "angular_in_rc": stats["mean_angular_in_rc"],
                           "rebuilds_in_timed_steps": timed_rebuilds},
            "energy_drift_ev_per_atom": float((etot.max() - etot.min()) / N) if etot.size > 1 else None,
            "naive_flops_per_atom_step": naive_flop_model(w.model, stats["mean_radial_in_rc"],
                                                            stats["mean_angular_in_rc"]),
        }
        for prec, key in FORMS[1:]:
            r = md[key]
            rl, _ = atom_roofline(w, r["stats"], r["ktime"]["nep_atom"] / args.steps, peak, basis)
            line[f"{key}_form"] = {
                "value": world * N * args.steps / r["seconds"], "unit": UNIT,
                "ms_per_step": 1e3 * r["seconds"] / args.steps,
                "kernel_ms_per_step": {k: v / args.steps for k, v in r["ktime"].items()},
                "atom_kernel_ms": r["ktime"]["nep_atom"] / args.steps,
                "atom_kernel_frac_of_fp32_peak": rl["frac"],
                "network": NETWORK[prec]}
        if crun is not None:
            line["config_run"] = crun
        if pbte is not None:
            line["pbte"] = pbte
        if batch_forms is not None:
            line["batch_form"], line["population"] = batch_forms
        if serving is not None:
            line["serving"] = serving
        if not args.no_cpu_baseline and world == 1:
            line["cpu_baseline"] = cpu_baseline(args.workload, args.cpu_seconds)
            ref = subcell_reference(w, args.workload)
            line["force_error_vs_fp64_oracle"] = form_errors(step0, ref)
            if serving is not None:
                serving["force_error_vs_fp64_oracle"] = serving_errors(*serving_sample)
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()
    return 0


SKIN_DEFAULT = {"si_large": 0.3, "si_medium": 0.3, "si": 0.4, "pbte": 0.4}


def main():
    args = parse_args()
    args.pbte_skin = args.skin if args.skin is not None else SKIN_DEFAULT["pbte"]
    if args.skin is None:
        args.skin = SKIN_DEFAULT[args.workload]
    if args.impl == "reference":
        return run_reference(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
