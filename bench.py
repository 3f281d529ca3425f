#!/usr/bin/env python
"""Benchmark of the spin-polarized XL-BOMD hot path on GB300.

Metric: MD steps/s (and Krylov response ranks/s) of the 1024-atom
iron-like cell (8x8x8 bcc, 9216 orbitals x 2 spins, Krylov rank 8) in the
mixed-precision form (fp16 tensor-core products with the split fp32
residual, fp32 accumulation; fp64 for mu, the Krylov least squares, forces
and energies).

One step = one xlbomd_step: half kick, drift, n update with dissipation,
H build, Fermi-operator expansion with the common-mu Newton search,
Mulliken charges, forces, the rank-8 Krylov kernel (8 density-matrix
responses) and the second half kick.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Multi-GPU: replicas only (each rank advances its own independent cell, no
collective); value = total steps of all ranks / max-over-ranks time.
--impl reference times the FP64 CPU oracle on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "MD steps/s and Krylov response ranks/s at 1024 atoms; % tensor-core peak"
UNIT = "steps/s"


def metric_for(w):
    if w.n_atoms == 1024:
        return METRIC
    return f"MD steps/s and Krylov response ranks/s at {w.n_atoms} atoms; % tensor-core peak"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="fe1024")
    ap.add_argument("--precision", default="fp16", choices=["fp16", "bf16", "fp64"])
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-sample-steps", type=int, default=1)
    return ap.parse_args()


# ---------------------------------------------------------------------------
class ClockSampler:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.lines = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                mx.append(float(parts[1]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[4:8]):
                if val.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return d, "measured"
    return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


def kernel_source_hash(path: str) -> str:
    """Hash of a CUDA source with comments and whitespace removed, so that only
    code changes invalidate counters taken on it."""
    import hashlib
    import re
    src = open(path).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    src = re.sub(r"//[^\n]*", "", src)
    src = re.sub(r"\s+", "", src)
    return hashlib.sha256(src.encode()).hexdigest()[:16]


def traffic_record():
    """ncu DRAM traffic of the tensor-core GEMM per launch, if a capture of the
    current kernel code exists (profiles/tc_gemm_traffic.json holds the code
    hash it was taken on)."""
    path = os.path.join(ROOT, "profiles", "tc_gemm_traffic.json")
    src = os.path.join(ROOT, "paper_2303_03529_gb300", "csrc", "mixed.cu")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        rec = json.load(f)
    if rec.get("source_sha") != kernel_source_hash(src):
        return None
    return rec


# ---------------------------------------------------------------------------
def init_dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def max_over_ranks(x: float) -> float:
    """Maximum of a per-rank scalar (timings) over all ranks; identity when
    torch.distributed is not initialized.  Works with nccl (CUDA tensor) and
    gloo (CPU tensor)."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return float(x)
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(steps_per_rank: int, world: int, max_seconds: float) -> float:
    """Whole-job steps/s of independent replicas: all ranks' steps over the
    slowest rank's time (weak scaling, no exchange between replicas)."""
    return world * steps_per_rank / max_seconds


def prepare_state(sxl, w, precision, local):
    """Initial MD state: SCF from n = 0 with the Krylov kernel mixer and
    K0 = -I (outside the timed region), all history slots = n*."""
    import numpy as np
    import torch
    p = w.params
    ctx = sxl.Context(p, w.n_atoms, w.cell, precision, scf_keep_k0=1)
    n0 = np.zeros(2 * w.n_atoms)
    t0 = time.time()
    n_star, iters, rms = ctx.scf(w.R, n0, tol=1e-5, max_iter=40)
    t_scf = time.time() - t0
    _, mu = ctx.density(w.R, n_star)
    nh = torch.stack([n_star] * (p.kmax + 1)).contiguous()
    ctx.set_state(w.R, w.V, nh, mu)
    return ctx, dict(scf_iters=iters, scf_rms=rms, scf_s=round(t_scf, 2))


def run_ours(args):
    import numpy as np
    import torch
    from paper_2303_03529_gb300 import build as _build
    from paper_2303_03529_gb300 import sxl, workload

    ws, rank, local = init_dist()
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", init_method="env://")
    torch.cuda.set_device(local)
    if rank == 0:
        _build.build()
    if ws > 1:
        torch.distributed.barrier()
    w = workload.WORKLOADS[args.workload]()
    ctx, setup = prepare_state(sxl, w, args.precision, local)
    stream = ctx.stream

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    # warm-up (untimed)
    for _ in range(args.warmup):
        ctx.step(1, stats=False)
    ctx.timers(reset=True)

    # device-resident timed region
    ctx.enable_gemm_timing(True)
    sampler = ClockSampler(local)
    sampler.start()
    launches0 = ctx.info()["launches"]
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    ev0.record(stream)
    for _ in range(args.steps):
        ctx.step(1, stats=False)
    ev1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier()
    clocks = sampler.stop()
    ms = ev0.elapsed_time(ev1)
    launches = int(ctx.info()["launches"] - launches0)
    tm = ctx.timers(reset=True)
    ctx.enable_gemm_timing(False)
    ms = max_over_ranks(ms)
    ms_step = ms / args.steps
    value = replica_throughput(args.steps, ws, ms / 1e3)
    ranks_per_s = tm["ranks"] / (tm["krylov_ms"] / 1e3) if tm["krylov_ms"] > 0 else None

    # end to end through the public API with host buffers: every step uploads
    # the full MD state (R, V, n history, F, Kf) from pinned host memory and
    # downloads the advanced state (the step's result)
    e2e = None
    if not args.no_e2e:
        nat, n2, K1 = w.n_atoms, 2 * w.n_atoms, w.params.kmax + 1
        pin = lambda *s: torch.empty(*s, dtype=torch.float64).pin_memory()
        hR, hV, hN = pin(nat, 3), pin(nat, 3), pin(K1, n2)
        hF, hK = pin(nat, 3), pin(n2)
        mu = ctx.get_state_host(hR, hV, hN)
        ctx.get_derived_host(hF, hK)
        h2d = 8 * (hR.numel() + hV.numel() + hN.numel() + hF.numel() + hK.numel())
        d2h = h2d
        barrier()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(args.steps):
            ctx.set_state_host(hR, hV, hN, mu)
            ctx.set_derived_host(hF, hK)
            ctx.step(1, stats=False)
            mu = ctx.get_state_host(hR, hV, hN)
            ctx.get_derived_host(hF, hK)
        torch.cuda.synchronize()
        t_e2e = time.perf_counter() - t0
        t_e2e = max_over_ranks(t_e2e)
        e2e = {"value": round(replica_throughput(args.steps, ws, t_e2e), 6), "unit": UNIT,
               "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}
        # one step with the full statistics (energies incl. entropy), untimed
        st = ctx.step(1, stats=True)
        e2e["after_stats"] = {"Etot_eV": float(st[0][0]), "T_K": float(st[0][1]),
                              "rms_residual": float(st[0][2]), "mu_eV": float(st[0][3])}

    if rank != 0:
        return
    peaks, src = measured_peaks()
    peak = peaks.get("bf16_tflops_sustained", peaks.get("bf16_tflops"))
    roof = None
    if tm["tc_launches"] > 0:
        avg_ms = tm["tc_ms"] / tm["tc_launches"]
        alg_per_launch = tm["tc_alg_flops"] / tm["tc_launches"]
        achieved = alg_per_launch / (avg_ms / 1e3) / 1e12
        trec = traffic_record()
        roof = {"bound": "tensor", "achieved": round(achieved, 2), "peak": peak,
                "unit": "TFLOP/s", "frac": round(achieved / peak, 4),
                "traffic": trec["bytes_per_launch"] if trec else None,
                "kernel": "k_tc_gemm (tcgen05 kind::f16, split hi/lo operands)",
                "peak_source": f"{src} bf16_tflops_sustained (fp16 dense rate = bf16)",
                "launches": int(tm["tc_launches"]), "avg_launch_ms": round(avg_ms, 4),
                "share_of_step": round(tm["tc_ms"] / ms, 4),
                "fp32_equiv_tflops": round(tm["tc_fp32_flops"] / tm["tc_launches"] /
                                           (avg_ms / 1e3) / 1e12, 2),
                "mma_issued_tflops": round(tm["tc_mma_flops"] / tm["tc_launches"] /
                                           (avg_ms / 1e3) / 1e12, 2)}
    cpu = None
    if not args.no_cpu_baseline and ws == 1:
        cpu = cpu_baseline(w, args.cpu_sample_steps)
    line = {
        "metric": metric_for(w), "value": round(value, 6), "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_step, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": {"fp16": "f16x2-split/f32acc+f64", "bf16": "bf16x2-split/f32acc+f64",
                  "fp64": "f64"}[args.precision],
        "data": "synthetic (seeded bcc iron-like cell, Maxwell 300 K velocities)",
        "config": {"workload": w.name, "n_atoms": w.n_atoms, "orbitals": w.n_orb,
                   "krylov_rank": w.params.krylov_rank, "dt_fs": w.params.dt_fs,
                   "precision": args.precision, "parallelism": f"replicas x{ws}",
                   "l2": "inputs larger than L2 (each chain matrix 2 x 9216^2 x 4 B = 680 MB)",
                   "k0": "-I (scaled delta kernel)", "init": setup},
        "krylov_ranks_per_s": round(ranks_per_s, 4) if ranks_per_s else None,
        "phase_ms_per_step": {"density": round(tm["density_ms"] / args.steps, 2),
                              "forces": round(tm["forces_ms"] / args.steps, 2),
                              "krylov": round(tm["krylov_ms"] / args.steps, 2)},
        "gpu_launches": launches,
        "clocks": clocks,
        "roofline": roof,
        "e2e": e2e,
        "cpu_baseline": cpu,
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------
class OracleSampler:
    """Times the FP64 CPU oracle on parts of one MD step of the workload and
    scales to a full step by operation counts.

    A full oracle step does 2 dense eigendecompositions (one per spin) and
    2 (m + 1) first-order product pairs (C^T dh C and the diagonal of
    C dD' C^T; m Krylov directions plus density matrix and forces), so
    t_step = 2 t_eigh + 2 (m + 1) t_pair.  The eigendecomposition of H_up is
    timed once (setup); each sample() times one product pair on the
    workload's own eigenvectors."""

    def __init__(self, w):
        import numpy as np
        from oracle import model, electronic
        self.w, self.np, self.electronic = w, np, electronic
        p = w.params
        H0 = model.build_h0(w.R, w.cell, p)
        G = model.gamma_matrix(w.R, w.cell, p)
        n = np.zeros(2 * w.n_atoms)
        Hu, _ = model.hamiltonians(H0, n, G, p)
        t0 = time.perf_counter()
        self.ch = electronic.SpinChannel(Hu)
        self.t_eigh = time.perf_counter() - t0
        self.dh = np.repeat(G @ np.ones(w.n_atoms), 9)
        self.F = electronic.fermi_divided_differences(self.ch.eps, float(np.median(self.ch.eps)),
                                                      1.0 / p.kT)

    def sample(self):
        """Times one product pair; returns (steps/s estimate, t_pair)."""
        C = self.ch.C
        t0 = time.perf_counter()
        dHp = C.T @ (self.dh[:, None] * C)
        dD = C @ (self.F * dHp) @ C.T
        _ = self.np.diag(dD)
        t_pair = time.perf_counter() - t0
        m = self.w.params.krylov_rank
        return 1.0 / (2 * self.t_eigh + 2 * (m + 1) * t_pair), t_pair

    def describe(self, t_pair):
        m = self.w.params.krylov_rank
        return (f"oracle on {self.w.name}: 1 eigh of H_up ({self.t_eigh:.1f} s) + 1 response "
                f"product pair ({t_pair:.1f} s); full step = 2 eigh + 2(m+1) pairs, m={m}")


def blas_threads():
    try:
        from threadpoolctl import threadpool_info
        info = threadpool_info()
        return max(d.get("num_threads", 1) for d in info) if info else os.cpu_count()
    except Exception:
        return int(os.environ.get("OPENBLAS_NUM_THREADS", os.cpu_count() or 1))


def cpu_baseline(w, nsteps=1):
    smp = OracleSampler(w)
    best = None
    for _ in range(max(1, nsteps)):
        v, tp = smp.sample()
        best = (v, tp) if best is None or v > best[0] else best
    return {"value": round(best[0], 8), "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
            "sample": smp.describe(best[1])}


def run_reference(args):
    ws, rank, local = init_dist()
    if rank != 0:
        return
    from paper_2303_03529_gb300 import workload
    w = workload.WORKLOADS[args.workload]()
    t_start = time.perf_counter()
    smp = OracleSampler(w)            # includes the one timed eigendecomposition
    for _ in range(args.warmup):
        smp.sample()
    vals, tps = [], []
    for _ in range(args.steps):
        v, tp = smp.sample()
        vals.append(v)
        tps.append(tp)
    wall = time.perf_counter() - t_start
    value = statistics.median(vals)
    cpu = {"value": round(value, 8), "unit": UNIT, "cores": blas_threads(), "kind": "oracle",
           "sample": "per step: " + smp.describe(statistics.median(tps))}
    line = {"metric": metric_for(w), "value": round(value, 8), "unit": UNIT, "n_gpus": ws,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 / value, 1), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded bcc iron-like cell)",
            "config": {"workload": w.name, "n_atoms": w.n_atoms, "orbitals": w.n_orb,
                       "krylov_rank": w.params.krylov_rank, "wall_s": round(wall, 1)},
            "impl": "reference", "cpu_baseline": cpu,
            "e2e": {"value": round(value, 8), "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
