#!/usr/bin/env python
"""Benchmark of the multispecies glioblastoma step on GB300.

Metric: voxel-steps/s = N^3 * steps / time for steps of the operator-split model (Section 3 of
the paper: transport, Crank-Nicolson diffusion, reactions, screened elasticity) on the 256^3
synthetic brain, through the library's C ABI.  Prints one JSON line (rank 0).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed]
  python bench.py --impl reference ...   # the CPU oracle on the host cores, same metric

With N > 1 (torchrun), every rank runs an independent replica of the workload (the workload
has no exchange step between replicas); the time is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "voxel-steps/s at 256^3 (mixed FP32 vs plain FP64, same GPU); adjoint/forward time"
UNIT = "voxel-steps/s"
PRECONDS = {"jacobi": 0, "spectral": 1, "scaled": 2}
FIELDS = ("p", "i", "n", "g", "w", "f", "o", "l", "bg", "ux", "uy", "uz", "vx", "vy", "vz")

# Algorithmic traffic and arithmetic of the elasticity operator kernel, per voxel and launch.
# FP64 path: reads p (3 comps), face coefficients (lambda+2mu)/h^2 and mu/h^2 (3 + 3), Jacobi
# diagonal (3), node mu and lambda (2); writes q (3): 17 FP64 arrays; 123 FP64 flops.
# Mixed path with Jacobi (the CG p-update fused into the operator kernel): reads r, D^{-1},
# p_old (3 each) and node mu, lambda, eta and writes p_new and q (3 each): 18 FP32 arrays.
# With a spectral preconditioner the p-update is fused into the preconditioner's last pass,
# so the operator kernel reads p (3) and mu, lambda, eta and writes q (3): 9 FP32 arrays.
ELAS_MATVEC_BYTES_PER_VOXEL = {("fp64", "jacobi"): 17 * 8, ("fp64", "spectral"): 17 * 8,
                               ("fp64", "scaled"): 17 * 8,
                               ("mixed", "jacobi"): 18 * 4, ("mixed", "spectral"): 9 * 4,
                               ("mixed", "scaled"): 9 * 4}
ELAS_MATVEC_FLOPS_PER_VOXEL = 123


def mixed_kernel_bytes(n, precond):
    """Algorithmic bytes per voxel of one launch of each kernel of the mixed multispecies step
    (every array element the kernel must read or write once; neighbour re-reads are free).
    FP64 arrays 8 B, FP32 arrays 4 B, (hi, lo) FP32 pairs 8 B; W is the half spectrum of the
    three components, n/2 + 1 complex FP32 modes per row of n voxels."""
    W = 3 * 8 * (n // 2 + 1) / n
    s = 12 if precond == "scaled" else 0        # the scaled preconditioner's s (3 comps)
    return {
        "k_diff_faces": 80,          # g, w, f in; 3 faces, rho, 3 face pairs out
        "k_diff_diag": 40,           # 3 faces in; diagonal and its inverse out
        "k_to_f32": 120,             # FP32 copies of the 10 fields the transport gathers
        "k_divergence": 32,          # v (3) in, div v out
        "k_sl32": 96,                # 3 interleaved float4 inputs gathered, 6 FP64 fields out
        "k_sl32_pack": 120,          # v (3), 6 species in (FP64); 3 interleaved float4 out
        "k_lame_df": 116,            # p, i, n, g, w, f, bg in; mu, lam, eta (FP64 and FP32),
                                     # mu, lam and p + n pairs out
        "k_df_pack3": 48,            # 3 FP64 in, 3 pairs out
        "k_cn_ir_residual_df": 76,   # 3 face pairs, D^-1; per field (i, l): x pair, rhs pair, r, e
        "k_cn32_pupdate": 28,        # D^-1, r and p (2 fields) in, p out
        "k_cn32_matvec": 44,         # 3 FP32 faces, z, previous p (2 fields) in; p, q out
        "k_cn32_update": 52,         # D^-1, e, r, p, q (2 fields) in, e, r out
        "k_cn_ir_correct": 56,       # x (FP64), e in; x, x pair out (2 fields)
        "k_cn32_neumann": 32,        # r (2 fields), 3 FP32 faces, D^-1 in; z (2 fields) out
        "k_diff_node_df": 40,        # g, w, f in; K pair, rho out
        "k_diff_faces_df": 48,       # K pairs in; 3 face pairs, 3 FP32 faces, D^-1 out
        "k_ox_prep": 56,             # oxygen, double-FP32: 3 face pairs, o in; d, D^-1, x pairs out
        "k_ox_init": 56,             # 3 face pairs, x, D^-1 in; r, p out
        "k_ox_matvec": 48,           # 3 face pairs, d, p in; q out
        "k_ox_update": 56,           # x, p, r, q, D^-1 in; x, r out
        "k_ox_pupdate": 32,          # D^-1, r, p in; p out
        "k_ox_finish": 16,           # x pair in, o out
        "k_cn_init": 56,             # oxygen, FP64: 3 faces, D^-1, x in; r, p out
        "k_cn_matvec": 48,           # 3 faces, diagonal, p in; q out
        "k_cn_update": 56,           # D^-1, x, r, p, q in; x, r out
        "k_cn_pupdate": 32,          # D^-1, r, p in; p out
        "k_react": 128,              # 9 FP64 in, 7 out
        "k_lame": 80,                # 7 species in; mu, lambda, eta out
        "k_elas_coef_df": 128,       # mu, lambda, p + n pairs, eta in; F, G, diagonal, b pairs out
        "k_elas32_coef": 48,         # u (3) in; u pairs out
        "k_elas_extrapolate": 144,   # u, v, v^{n-1} in; u, du, u pairs out
        "k_spec_mean": 24,           # mu, lambda, eta in
        "k_elas_ir_residual_df": 160,  # u, F, G, diagonal, b pairs (3 each), mu, lambda pairs
        #                                in; r, e (FP32) out
        "k_spec_x_fwd": 12 + s + W,  # r (and s) in, half spectrum out
        "k_spec_y_fwd": 2 * W,       # half spectrum in and out
        "k_spec_y_inv": 2 * W,
        "k_spec_zr": 2 * W,
        "k_spec_z": 2 * W,
        "k_spec_x_inv_p": W + s + 24,  # half spectrum (and s), p_old in; p out
        "k_elas32_matvec_spec": 36,  # p (3), mu, lambda, eta in; q (3) out
        "k_spec_update_xfwd": 72 + s + W,  # e, p, r, q in; e, r out (3 each); spectrum out
        "k_elas_ir_correct": 132,    # u, du, e in; u, du, u pairs out
        "k_elas_ir_finish": 96,      # du, v in; v, v^{n-1} out
    }


# DRAM traffic per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture
# of a single kernel, per voxel, with the hash of the source it was measured on: reported
# only while the kernel's source (its .cu file and the shared headers) is unchanged.
MEASURED_TRAFFIC = {   # 256^3 mixed step, profiles/launches_mixed_spectral_256.md
    "k_spec_update_xfwd": {"bytes_per_voxel": 85.6, "sha": "d59493db2c07f8d9"},
    "k_elas32_matvec_spec": {"bytes_per_voxel": 32.2, "sha": "7ec7d47f12615f35"},
    "k_spec_x_inv_p": {"bytes_per_voxel": 42.6, "sha": "d59493db2c07f8d9"},
    "k_spec_y_fwd": {"bytes_per_voxel": 19.9, "sha": "d59493db2c07f8d9"},
    "k_spec_y_inv": {"bytes_per_voxel": 19.4, "sha": "d59493db2c07f8d9"},
    "k_spec_zr": {"bytes_per_voxel": 20.4, "sha": "d59493db2c07f8d9"},
    "k_cn32_neumann": {"bytes_per_voxel": 32.6, "sha": "7336241f68141960"},
    "k_cn32_matvec": {"bytes_per_voxel": 40.4, "sha": "7336241f68141960"},
    "k_cn32_update": {"bytes_per_voxel": 45.3, "sha": "7336241f68141960"},
    "k_cn_ir_residual_df": {"bytes_per_voxel": 75.9, "sha": "7336241f68141960"},
    "k_elas_ir_residual_df": {"bytes_per_voxel": 166.7, "sha": "7ec7d47f12615f35"},
    "k_ox_matvec": {"bytes_per_voxel": 48.0, "sha": "63e5600d8107b556"},
    "k_ox_update": {"bytes_per_voxel": 53.7, "sha": "63e5600d8107b556"},
    "k_ox_pupdate": {"bytes_per_voxel": 28.8, "sha": "63e5600d8107b556"},
    "k_sl32": {"bytes_per_voxel": 97.5, "sha": "7ec7d47f12615f35"},
    "k_sl32_pack": {"bytes_per_voxel": 118.4, "sha": "7ec7d47f12615f35"},
    "k_elas_coef_df": {"bytes_per_voxel": 126.4, "sha": "eb3281616b3713f0"},
    "k_react": {"bytes_per_voxel": 125.2, "sha": "8ca213d5b6f3fcea"},
    "k_lame_df": {"bytes_per_voxel": 113.0, "sha": "8ca213d5b6f3fcea"},
}
KERNEL_SOURCE = {
    "k_spec_update_xfwd": "tg_spectral.cu", "k_elas32_matvec_spec": "tg_mixed.cu",
    "k_spec_x_inv_p": "tg_spectral.cu", "k_spec_y_fwd": "tg_spectral.cu",
    "k_spec_y_inv": "tg_spectral.cu", "k_spec_zr": "tg_spectral.cu",
    "k_cn32_neumann": "tg_cn_mixed.cu", "k_cn32_matvec": "tg_cn_mixed.cu",
    "k_cn32_update": "tg_cn_mixed.cu", "k_cn_ir_residual_df": "tg_cn_mixed.cu",
    "k_elas_ir_residual_df": "tg_mixed.cu", "k_ox_matvec": "tg_cn_ox.cu",
    "k_ox_update": "tg_cn_ox.cu", "k_ox_pupdate": "tg_cn_ox.cu", "k_sl32": "tg_mixed.cu",
    "k_sl32_pack": "tg_mixed.cu", "k_elas_coef_df": "tg_elasticity.cu",
    "k_react": "tg_reaction.cu", "k_lame_df": "tg_reaction.cu"}


def kernel_source_sha(kernel):
    import hashlib
    csrc = os.path.join(ROOT, "paper_1810_05370_gb300", "csrc")
    h = hashlib.sha256()
    for f in (KERNEL_SOURCE.get(kernel), "tg_internal.cuh", "tg_tiles.cuh", "tg_fpconv.cuh"):
        if f is None:
            return None
        with open(os.path.join(csrc, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def measured_traffic(kernel, n):
    m = MEASURED_TRAFFIC.get(kernel)
    if m is None or m["sha"] != kernel_source_sha(kernel):
        return None
    return m["bytes_per_voxel"] * n ** 3


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--dt", type=float, default=0.01)
    ap.add_argument("--precision", choices=("fp64", "mixed"), default="mixed")
    ap.add_argument("--precond", choices=("scaled", "spectral", "jacobi"), default="scaled",
                    help="elasticity preconditioner: Section 3's spectral one, that one between "
                         "diagonal scalings (scaled), or Jacobi")
    ap.add_argument("--no-compare", action="store_true",
                    help="skip timing the other precision on the same GPU")
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-adjoint", action="store_true")
    ap.add_argument("--adjoint-n", type=int, default=128)
    ap.add_argument("--adjoint-steps", type=int, default=50)
    ap.add_argument("--adjoint-checkpoint", type=int, default=10)
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-single", action="store_true",
                    help="skip the single-species model (Eq. e:rd) line")
    ap.add_argument("--batch-sims", type=int, default=64)
    ap.add_argument("--batch-threads", type=int, default=0,
                    help="host threads of the concurrent batch (0: up to 8)")
    ap.add_argument("--batch-steps", type=int, default=50)
    ap.add_argument("--batch-seq-steps", type=int, default=5,
                    help="timed steps per simulation of the sequential mixed comparison")
    ap.add_argument("--batch-seq-steps-fp64", type=int, default=2)
    ap.add_argument("--cpu-sample-n", type=int, default=256,
                    help="grid of the all-core oracle timing (init untimed)")
    ap.add_argument("--cpu-sample-steps", type=int, default=1)
    ap.add_argument("--cpu-single-n", type=int, default=64,
                    help="grid of the one-thread oracle timing")
    ap.add_argument("--ref-n", type=int, default=128,
                    help="grid of each step of the reference arm (the oracle)")
    ap.add_argument("--oracle-child", type=int, nargs=4, default=None,
                    metavar=("N", "STEPS", "WARMUP", "PRECOND"), help=argparse.SUPPRESS)
    return ap.parse_args()


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


# GB300 FP64 peak: not in the measured-peaks file.  Derived from the FP64 issue rate of the
# SM (2 DFMA per clock) and the maximum SM clock; a probe of independent FMA chains reaches
# 95 % of it.
FP64_PEAK_TFLOPS = 1.26


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ("hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap")
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 9:
                    continue
                try:
                    sm.append(float(parts[1]))
                    smax.append(float(parts[2]))
                except ValueError:
                    continue
                for nm, val in zip(names, parts[5:9]):
                    if val.lower() == "active":
                        reasons.add(nm)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def job_rate(ms_local, units_per_rank, world, dist=None, device=None):
    """Whole-job throughput of `world` replicas (one per GPU, no data-path collective): every
    rank's units over the slowest rank's time.  Returns (max ms, units per second)."""
    ms = ms_local
    if dist is not None:
        import torch
        t = torch.tensor([ms], dtype=torch.float64, device=device)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        ms = float(t.item())
    return ms, world * units_per_rank / (ms * 1e-3)


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def oracle_child(a):
    """--oracle-child: init (untimed) and `steps` timed oracle steps on the n^3 synthetic
    brain in this process (OMP_NUM_THREADS set by the parent); prints one JSON line."""
    from oracle import Oracle
    from synth import initial_state, workload_params
    n, steps, warm, precond = a.oracle_child
    O = Oracle()
    P = workload_params(precond_elas=precond)
    st = initial_state(n, seed=0)
    t0 = time.perf_counter()
    O.init(n, P, st)
    t_init = time.perf_counter() - t0
    for _ in range(warm):
        O.step(n, P, 0.01, st)
    its = []
    t0 = time.perf_counter()
    for _ in range(steps):
        its.append(O.step(n, P, 0.01, st))
    secs = time.perf_counter() - t0
    print(json.dumps({"n": n, "steps": steps, "secs": secs, "init_secs": t_init,
                      "value": n ** 3 * steps / secs,
                      "threads": int(os.environ.get("OMP_NUM_THREADS", "0")),
                      "it_elas": [s["it_elas"] for s in its],
                      "it_diff": [s["it_diff"] for s in its]}), flush=True)


def oracle_sample(n, steps, warm_steps=0, precond=0, threads=None):
    """Time the CPU oracle on `steps` steps of an n^3 synthetic brain (init and warm-up steps
    untimed) in a child process with `threads` OpenMP threads (default: every core this
    process may run on)."""
    cores = len(os.sched_getaffinity(0))
    threads = cores if threads is None else threads
    env = dict(os.environ, OMP_NUM_THREADS=str(threads))
    r = subprocess.run([sys.executable, os.path.abspath(__file__), "--oracle-child", str(n),
                        str(steps), str(warm_steps), str(precond)], env=env,
                       capture_output=True, text=True, check=True)
    return json.loads(r.stdout.strip().splitlines()[-1])


def run_reference(args, world, rank):
    """The reference arm: the CPU oracle (the paper has no code; the oracle is the plain FP64
    statement of the same step) on the host cores, rank 0 only."""
    if rank != 0:
        return
    n = args.ref_n
    o = oracle_sample(n, args.steps, warm_steps=args.warmup, precond=PRECONDS[args.precond])
    value, secs = o["value"], o["secs"]
    sample = (f"CPU oracle, {n}^3 synthetic brain per step (same generator and parameters as "
              f"the {args.n}^3 workload, {args.precond} elasticity preconditioner), init and "
              f"{args.warmup} warm-up steps untimed, {args.steps} timed steps, "
              f"{o['threads']} OpenMP threads; elasticity and diffusion CG iterations grow with "
              f"N, so the per-voxel rate at {args.n}^3 is lower")
    out = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": 0,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": f"{args.n}^3 synthetic brain, multispecies step, dt {args.dt}",
                   "grid": args.n, "precision": args.precision,
                   "elasticity_preconditioner": args.precond, "sample_grid": n},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": o["threads"], "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(out), flush=True)


def run_batch(args, dev):
    """64 simulations of uneven grids (64/96/128^3, rho ~ U[5,15], k_scale ~ U[0.5,2]) stepped
    as one batch for the workload's steps, in both batch forms: persistent (cooperative
    solvers, replayed step graph, autotuned tiles) and concurrent (each member on the
    single-simulation path with its best elasticity preconditioner -- the scaled spectral one
    where the grid allows it -- on its own stream, host threads driving them); against the
    same simulations run one after another through the single-simulation path, mixed and
    FP64, timed on a sample of steps per simulation after one untimed step."""
    import torch
    from paper_1810_05370_gb300 import Simulation
    from paper_1810_05370_gb300.batch import Batch
    from paper_1810_05370_gb300 import _tg
    from synth import batch_workload, initial_state
    spec = batch_workload(args.batch_sims)
    states = [initial_state(n, seed) for n, _, seed in spec]
    bt = Batch([(n, P, st) for (n, P, _), st in zip(spec, states)], device=dev)
    tune = bt.autotune(args.dt)
    bt.step(args.dt, 1)                                   # warm-up (captures the step graph)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    stats = bt.step(args.dt, args.batch_steps)
    torch.cuda.synchronize(dev)
    t_batch = time.perf_counter() - t0
    voxels = bt.voxels
    bt.close()
    del bt
    torch.cuda.empty_cache()

    def best_precond(n, P):
        for pc in (PRECONDS["scaled"], PRECONDS["jacobi"]):
            if _tg.tg_workspace_bytes(_tg.make_grid(n), _tg.make_params(dict(P, precond_elas=pc)),
                                      _tg.TG_MIXED) > 0:
                return pc
        return PRECONDS["jacobi"]

    # the concurrent batch: every member on the single-simulation path with its best
    # preconditioner, on its own stream, host threads driving them
    cb = Batch([(n, dict(P, precond_elas=best_precond(n, P)), st)
                for (n, P, _), st in zip(spec, states)], device=dev, concurrent=True,
               threads=args.batch_threads)
    cb.step(args.dt, 1)                                   # warm-up
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    cstats = cb.step(args.dt, args.batch_steps)
    torch.cuda.synchronize(dev)
    t_conc = time.perf_counter() - t0
    cb.close()
    del cb
    torch.cuda.empty_cache()

    seq = {}
    for prec, k in (("mixed", args.batch_seq_steps), ("fp64", args.batch_seq_steps_fp64)):
        t_seq, vs = 0.0, 0
        for (n, P, _), st in zip(spec, states):
            Pb = dict(P, precond_elas=best_precond(n, P))
            sim = Simulation(n, Pb, st, precision=prec, device=dev)
            sim.step(args.dt)                             # untimed first step
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            sim.step(args.dt, k)
            torch.cuda.synchronize(dev)
            t_seq += time.perf_counter() - t0
            vs += n ** 3 * k
            sim.close()
        torch.cuda.empty_cache()
        seq[prec] = {"voxel_steps_per_s": vs / t_seq, "steps_per_sim": k, "seconds": t_seq}
    vs = voxels * args.batch_steps
    return {"sims": len(spec), "voxels": voxels, "steps": args.batch_steps, "precision": "mixed",
            "concurrent": {"voxel_steps_per_s": vs / t_conc, "seconds": t_conc,
                           "threads": args.batch_threads or min(len(spec), 8),
                           "speedup_over_sequential_mixed":
                               (vs / t_conc) / seq["mixed"]["voxel_steps_per_s"],
                           "inner_iterations": cstats["it_elas_total"],
                           "launches": cstats["launches"]},
            "voxel_steps_per_s": vs / t_batch, "seconds": t_batch,
            "sequential_best_path": seq,
            "speedup_over_sequential_mixed": (vs / t_batch) / seq["mixed"]["voxel_steps_per_s"],
            "graph": stats["graph"], "tile_depth": stats["tile_depth"],
            "coop_blocks": stats["coop_blocks"], "inner_iterations": stats["it_elas_total"],
            "launches": stats["launches"],
            "autotune": {"best_zc": tune["best_zc"], "best_blocks": tune["best_blocks"],
                         "candidates": tune["candidates"]}}


def main():
    args = parse()
    if args.oracle_child:
        oracle_child(args)
        return
    world, rank, local = dist_setup(args)
    if args.impl == "reference":
        run_reference(args, world, rank)
        return
    import numpy as np
    import torch
    from paper_1810_05370_gb300 import Simulation
    from synth import initial_state, workload_params

    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    dev = torch.device("cuda", local)
    n = args.n
    V = n ** 3
    P = workload_params(precond_elas=PRECONDS[args.precond])
    st0 = initial_state(n, seed=0)
    sim = Simulation(n, P, st0, precision=args.precision, device=dev)
    stream = sim.stream
    ws_bytes = sim.workspace.numel()

    def barrier():
        torch.cuda.synchronize(dev)
        if dist is not None:
            dist.barrier()

    # ---------------------------------------------------------------- device-resident timing
    def time_steps(sim, clocks=None):
        for _ in range(args.warmup):
            sim.step(args.dt)
        sim.set_timing(True)
        barrier()
        if clocks is not None:
            clocks.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(sim.stream)
        agg = {"launches": 0, "t_mv": 0.0, "n_mv": 0, "t_up": 0.0, "n_up": 0, "it_elas": [],
               "it_elas_outer": [], "it_diff": [], "phase_ms": [0.0, 0.0, 0.0, 0.0]}
        for _ in range(args.steps):
            s = sim.step(args.dt)
            agg["launches"] += s["launches"]
            agg["t_mv"] += s["t_elas_matvec_ms"]
            agg["n_mv"] += s["n_elas_matvec"]
            agg["t_up"] += s["t_spec_update_ms"]
            agg["n_up"] += s["n_spec_update"]
            agg["it_elas"].append(s["it_elas"])
            agg["it_elas_outer"].append(s["it_elas_outer"])
            agg["it_diff"].append(s["it_diff"])
            for q in range(4):
                agg["phase_ms"][q] += s["t_phase_ms"][q] / args.steps
        e1.record(sim.stream)
        barrier()
        agg["clocks"] = clocks.stop() if clocks is not None else None
        agg["kernels"] = sim.kernel_times()
        sim.set_timing(False)
        agg["ms"], agg["value"] = job_rate(e0.elapsed_time(e1), V * args.steps, world, dist, dev)
        return agg

    clocks = Clocks(local)
    agg = time_steps(sim, clocks)
    clk = agg["clocks"]
    ms_max = agg["ms"]
    value = agg["value"]

    # ---------------------------------------------------------------- roofline of the top kernel
    peaks, peak_src = load_peaks()

    def roofline(agg, precision):
        """The dominant kernel's roofline and one row per timed kernel (CUDA events on the
        launching stream, launches that did work only)."""
        if precision == "fp64":
            avg_ms = agg["t_mv"] / max(agg["n_mv"], 1)
            gbs = ELAS_MATVEC_BYTES_PER_VOXEL[(precision, args.precond)] * V / (avg_ms * 1e-3) / 1e9
            tfl = ELAS_MATVEC_FLOPS_PER_VOXEL * V / (avg_ms * 1e-3) / 1e12
            r64 = {"kernel": "k_elas_matvec (FP64 19-point Navier-Lame operator + <p, Ap>)",
                   "bound": "alu", "achieved": tfl, "peak": FP64_PEAK_TFLOPS,
                   "unit": "TFLOP/s", "frac": tfl / FP64_PEAK_TFLOPS, "traffic": None,
                   "peak_source": "derived FP64 roof (152 SMs x 2 DFMA/clk x 2.07 GHz)",
                   "hbm_gbs": gbs, "avg_launch_ms": avg_ms, "launches_timed": agg["n_mv"],
                   "share_of_step": agg["t_mv"] / agg["ms"] if agg["ms"] > 0 else None}
            return r64, [r64]
        table = mixed_kernel_bytes(args.n, args.precond)
        rows = []
        for name, (ms, launches) in agg["kernels"].items():
            bpv = table.get(name)
            avg = ms / max(launches, 1)
            row = {"kernel": name, "launches_per_step": launches / args.steps,
                   "avg_launch_ms": avg, "ms_per_step": ms / args.steps,
                   "share_of_step": ms / agg["ms"] if agg["ms"] > 0 else None,
                   "bytes_per_voxel": bpv}
            if bpv is not None and avg > 0:
                gbs = bpv * V / (avg * 1e-3) / 1e9
                traffic = measured_traffic(name, args.n)
                row.update({"bound": "hbm", "achieved": gbs, "peak": peaks["hbm_gbs"],
                            "unit": "GB/s", "frac": gbs / peaks["hbm_gbs"], "traffic": traffic,
                            "traffic_per_voxel": traffic / V if traffic else None})
            rows.append(row)
        rows.sort(key=lambda r: -r["ms_per_step"])
        top = next(r for r in rows if r["bytes_per_voxel"] is not None)
        roof = {k: top.get(k) for k in ("bound", "achieved", "peak", "unit", "frac", "traffic")}
        roof.update({"kernel": top["kernel"], "bytes_per_voxel": top["bytes_per_voxel"],
                     "traffic_per_voxel": top.get("traffic_per_voxel"),
                     "peak_source": f"{peak_src} HBM copy bandwidth",
                     "avg_launch_ms": top["avg_launch_ms"],
                     "launches_timed": int(round(top["launches_per_step"] * args.steps)),
                     "share_of_step": top["share_of_step"]})
        return roof, rows

    roof, roof_all = roofline(agg, args.precision)

    # ---------------------------------------------------------------- end to end (host buffers)
    e2e = None
    if not args.no_e2e:
        host = {k: torch.empty(sim.shape, dtype=torch.float64, pin_memory=True) for k in FIELDS}
        for k in FIELDS:
            host[k].copy_(sim.state[k])
        nbytes = sum(h.numel() * 8 for h in host.values())
        barrier()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            # the state up from pinned host memory, one step, the new state down: the
            # library overlaps the copies with the step's phases (tg_step_host)
            sim.step_host(host, host, args.dt)
        barrier()
        _, e2e_rate = job_rate(1e3 * (time.perf_counter() - t0), V * args.steps, world, dist, dev)
        e2e = {"value": e2e_rate, "unit": UNIT,
               "h2d_bytes_per_step": nbytes, "d2h_bytes_per_step": nbytes}

    # ---------------------------------------------------------------- the other precision
    other = None
    if not args.no_compare:
        sim.close()
        torch.cuda.empty_cache()
        oprec = "fp64" if args.precision == "mixed" else "mixed"
        sim_o = Simulation(n, P, st0, precision=oprec, device=dev)
        ag_o = time_steps(sim_o)
        other = {"precision": oprec, "value": ag_o["value"], "unit": UNIT,
                 "ms_per_step": ag_o["ms"] / args.steps, "phase_ms_per_step": ag_o["phase_ms"],
                 "solver": {"it_elas_per_step": ag_o["it_elas"],
                            "it_elas_outer_per_step": ag_o["it_elas_outer"],
                            "it_diff_per_step": ag_o["it_diff"]},
                 "roofline": roofline(ag_o, oprec)[0], "gpu_launches": ag_o["launches"]}
        sim_o.close()
        sim = None

    # ---------------------------------------------------------------- gradient cost (rank 0)
    adjoint = None
    if rank == 0 and world == 1 and not args.no_adjoint:
        from paper_1810_05370_gb300.rollout import Rollout
        an, asteps = args.adjoint_n, args.adjoint_steps
        ast0 = initial_state(an, seed=0)
        ce = args.adjoint_checkpoint
        # untimed: a rollout of one checkpoint segment loads the adjoint's kernels (first use)
        wu = Rollout(an, P, ast0, ce, args.dt, checkpoint_every=ce)
        wu.gradient(wu.forward())
        wu.close()
        del wu
        # two rounds, the second kept: the first on a freshly started GPU has measured up to
        # 25 % slower for the gradient pass; simulations and rollouts are created (u^0 solve,
        # workspace) before each clock starts
        for _ in range(2):
            sim_f = Simulation(an, P, ast0, precision="fp64", device=dev)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            sim_f.step(args.dt, nsteps=asteps)
            torch.cuda.synchronize(dev)
            t_fwd = time.perf_counter() - t0
            sim_f.close()
            ro = Rollout(an, P, ast0, asteps, args.dt, checkpoint_every=ce)
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            p_final = ro.forward()
            vol = (2 * np.pi / an) ** 3
            g = ro.gradient(vol * (p_final - 1.05 * p_final))
            torch.cuda.synchronize(dev)
            t_grad = time.perf_counter() - t0
            ro.close()
            del ro
        adjoint = {"grid": an, "steps": asteps, "checkpoint_every": args.adjoint_checkpoint,
                   "precision": "fp64", "forward_s": t_fwd,
                   "forward_recompute_adjoint_s": t_grad,
                   "adjoint_over_forward": t_grad / t_fwd,
                   "gradient": [float(x) for x in g],
                   "note": "init (u^0 solve) outside both clocks; kernels loaded by an untimed "
                           "rollout first; second of two rounds; misfit against 1.05 p_N"}
        torch.cuda.empty_cache()

    # ---------------------------------------------------------------- batched workload (rank 0)
    # ---------------------------------------------------------------- single-species model
    single = None
    if rank == 0 and world == 1 and not args.no_single:
        from synth import initial_state_single
        Ps = workload_params(precond_elas=PRECONDS[args.precond], model=1)
        sim_s = Simulation(n, Ps, initial_state_single(n, seed=0), precision=args.precision,
                           device=dev)
        ag_s = time_steps(sim_s)
        single = {"model": "single species (Eq. e:rd)", "precision": args.precision,
                  "value": ag_s["value"], "unit": UNIT, "ms_per_step": ag_s["ms"] / args.steps,
                  "solver": {"it_elas_per_step": ag_s["it_elas"],
                             "it_diff_per_step": ag_s["it_diff"]},
                  "gpu_launches": ag_s["launches"]}
        sim_s.close()
        torch.cuda.empty_cache()

    batch = None
    if rank == 0 and world == 1 and not args.no_batch:
        batch = run_batch(args, dev)
        torch.cuda.empty_cache()

    # ---------------------------------------------------------------- CPU baseline (rank 0)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        pc = PRECONDS[args.precond]
        o_all = oracle_sample(args.cpu_sample_n, args.cpu_sample_steps, precond=pc)
        o_one = oracle_sample(args.cpu_single_n, 2, precond=pc, threads=1)
        cpu = {"value": o_all["value"], "unit": UNIT, "cores": o_all["threads"],
               "kind": "oracle",
               "sample": f"{args.cpu_sample_n}^3 synthetic brain (the workload), "
                         f"{args.precond} elasticity preconditioner, init untimed "
                         f"({o_all['init_secs']:.1f} s), {args.cpu_sample_steps} timed step(s) "
                         f"({o_all['secs']:.1f} s), {o_all['threads']} OpenMP threads",
               "solver": {"it_elas": o_all["it_elas"], "it_diff": o_all["it_diff"]},
               "single_thread": {"value": o_one["value"], "unit": UNIT, "cores": 1,
                                 "sample": f"{args.cpu_single_n}^3, init untimed, 2 timed steps "
                                           f"({o_one['secs']:.1f} s), 1 thread"}}

    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if args.precision == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": f"{n}^3 synthetic brain (nested ellipsoids, seed 0), "
                                   f"multispecies step dt {args.dt}, CG rtol 1e-8, "
                                   f"{args.precision} path",
                       "grid": n, "precision": args.precision,
                       "elasticity_preconditioner": args.precond,
                       "l2": "inputs larger than L2 (15 state arrays + workspace, "
                             f"{(15 * V * 8 + ws_bytes) / 1e9:.1f} GB)",
                       "parallelism": f"replicas x{world}"},
            "phase_ms_per_step": dict(zip(("S0-S1 transport", "S2 diffusion", "S3-S5 reactions",
                                           "S6-S7 elasticity"), agg["phase_ms"])),
            "solver": {"it_elas_per_step": agg["it_elas"],
                       "it_elas_outer_per_step": agg["it_elas_outer"],
                       "it_diff_per_step": agg["it_diff"]},
            "roofline": roof,
            "roofline_kernels": roof_all,
            "kernel_ms_per_step": sum(r["ms_per_step"] for r in roof_all)
            if args.precision == "mixed" else None,
            "compare": other,
            "adjoint": adjoint,
            "single_species": single,
            "batch": batch,
            "mixed_over_fp64": (None if other is None else
                                (value / other["value"] if args.precision == "mixed"
                                 else other["value"] / value)),
            "cpu_baseline": cpu,
            "e2e": e2e,
            "clocks": clk,
            "gpu_launches": agg["launches"],
        }
        print(json.dumps(out), flush=True)
    if sim is not None:
        sim.close()
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
