#!/usr/bin/env python
"""Benchmark of the RSGDF hot path on GB300.

One step = the whole path for one cell: j2c with its Cholesky factors, then j3c
(SR lattice sums, G = 0 correction, pair and aux Fourier transforms, LR
contraction, Bloch-phase contractions) for every k pair of the mesh and every
aux function.  Default workload: FCC two-atom cell a = 6.74 Bohr, k-mesh 2x2x2
(64 k pairs), 30 Cartesian AO and 90 aux functions, eps = 1e-8, G box 7^3 with
omega from the LR cutoff, FP64 throughout.  Synthetic seeded inputs (the
paper's basis sets are not available).

Metric: SR shell-triple lattice terms (aux shell, AO shell pair, l, d) per
second of the whole step; the j3c build time is ms_per_step.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun every rank runs its own copy of the step on its GPU (weak
scaling, no collective on the data path); rank 0 prints one JSON line.
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
sys.path.insert(0, ROOT)

METRIC = "j3c build s and shell-triple integrals/s per k-mesh; learned+mixed vs plain FP64 at 1e-8"
UNIT = "shell-triple lattice terms/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kmesh", default="2,2,2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--precision", default="fp64", choices=["fp64", "mixed"])
    return ap.parse_args()


def workload(kmesh):
    from paper_2102_02989_gb300 import inputs
    p = inputs.config2(tuple(kmesh))
    return p


def describe(p, omega, gmesh):
    return {"workload": "FCC a=6.74 Bohr 2-atom cell, k-mesh %dx%dx%d (%d k pairs), %d AO / %d aux Cartesian "
                        "functions, 3s2p1d AO per atom, ETB aux s8p5d2f1 per atom, eps_screen=eps_lr=%g, "
                        "G box %dx%dx%d, omega=%.6f; j2c+Cholesky+j3c(SR+G0+LR) FP64"
                        % (*p.kmesh, p.nk * p.nk, p.ao.nfunc, p.aux.nfunc, p.eps_sr, *gmesh, omega),
            "k_mesh": list(p.kmesh), "n_kpairs": p.nk * p.nk, "n_ao": p.ao.nfunc, "n_aux": p.aux.nfunc,
            "eps": p.eps_sr, "gmesh": list(gmesh), "omega": omega,
            "l2": "flushed between timed steps (256 MiB device write, untimed)"}


class Clocks:
    """nvidia-smi samples during the timed region."""

    def __init__(self):
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.p = subprocess.Popen(["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits",
                                       "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self, gpu_index=0):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        self.f.seek(0)
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in self.f.read().splitlines():
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9 or parts[0] != str(gpu_index):
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.f.name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def oracle_sample(p, omega, gmesh, shells):
    """The oracle on a bounded sample of the workload: every k pair, aux shells
    ``shells``, SR + G0 + LR.  Returns (terms, seconds, threads)."""
    import oracle
    oracle.build()
    kp = [(i, j) for i in range(p.nk) for j in range(p.nk)]
    t0 = time.perf_counter()
    _, cnt = oracle.j3c(p.a, p.kmesh, p.ao, p.aux, omega, kp, eps_sr=p.eps_sr, eps_lr=p.eps_lr,
                        gmesh=gmesh, shells=shells, return_counts=True)
    dt = time.perf_counter() - t0
    return cnt["terms"], dt, oracle.num_threads()


def run_reference(args, rank, world):
    """The oracle as it stands, timed on the host cores (rank 0 only)."""
    if rank != 0:
        return
    from paper_2102_02989_gb300 import inputs  # noqa: F401
    kmesh = [int(x) for x in args.kmesh.split(",")]
    p = workload(kmesh)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from rules_ref import omega_for
    omega = omega_for(p.a, p.gmesh, p.eps_lr, p.kmesh)
    gmesh = p.gmesh
    shells = (0, 4)   # s shells 0..3 of the first atom: a few seconds per step
    for _ in range(args.warmup):
        oracle_sample(p, omega, gmesh, shells)
    times, terms, th = [], 0, 1
    for _ in range(args.steps):
        n, dt, th = oracle_sample(p, omega, gmesh, shells)
        times.append(dt)
        terms += n
    tot = sum(times)
    val = terms / tot
    sample = ("aux shells [0,4) of %d (the first four s shells) x all %d k pairs, SR+G0+LR per step"
              % (p.aux.nshell, p.nk * p.nk))
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": describe(p, omega, gmesh),
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": th, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }), flush=True)


def main():
    args = parse()
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import numpy as np
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    from paper_2102_02989_gb300 import rsgdf
    rsgdf.load()
    kmesh = [int(x) for x in args.kmesh.split(",")]
    p = workload(kmesh)
    omega, gmesh = rsgdf.rsgdf_params(p.a, p.kmesh, gmesh=p.gmesh, eps_lr=p.eps_lr)
    kp = np.array([(i, j) for i in range(p.nk) for j in range(p.nk)], dtype=np.int32)
    kl = list(range(p.nk))
    opt = dict(omega=omega, gmesh=gmesh, eps_screen=p.eps_sr, eps_lr=p.eps_lr,
               precision=rsgdf.RSGDF_MIXED if args.precision == "mixed" else rsgdf.RSGDF_FP64)
    V = torch.zeros((len(kp), p.aux.nfunc, p.ao.nfunc, p.ao.nfunc), dtype=torch.complex128, device=dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step():
        J, L, info = rsgdf.rsgdf_j2c(p.a, p.kmesh, p.aux, kl, **opt)
        s2 = rsgdf.rsgdf_last_stats()
        rsgdf.rsgdf_j3c(p.a, p.kmesh, p.ao, p.aux, kp, out=V, **opt)
        s3 = rsgdf.rsgdf_last_stats()
        return (J, L, info), s2, s3

    peak_fp64 = rsgdf.rsgdf_probe_fp64()
    for _ in range(max(args.warmup, 0)):
        step()
    torch.cuda.synchronize()
    clocks = Clocks()
    clocks.start()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    stats = []
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    for i in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        ev[i][0].record()
        out, s2, s3 = step()
        ev[i][1].record()
        torch.cuda.synchronize()
        stats.append((s2, s3))
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop(gpu_index=local)
    times = [a.elapsed_time(b) for a, b in ev]
    tot_ms = sum(times)
    # end to end through the public API: host inputs (uploaded by the call) and
    # a device-to-host read of every result into pinned memory
    hV = torch.empty(V.shape, dtype=V.dtype, pin_memory=True)
    h2d = sum(np.asarray(x).nbytes for b in (p.ao, p.aux) for x in (b.l, b.nprim, b.prim_off, b.center, b.exps, b.coeffs))
    h2d = 2 * h2d + kp.nbytes + 4 * len(kl)
    e2e_ms = []
    for i in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        (J, L, info), _, _ = step()
        hV.copy_(V, non_blocking=True)
        hJ = J.to("cpu", non_blocking=True)
        hL = L.to("cpu", non_blocking=True)
        hi = info.to("cpu", non_blocking=True)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    d2h = V.numel() * 16 + J.numel() * 16 + L.numel() * 16 + info.numel() * 4
    terms = sum(s3["sr_terms"] + s2["sr_terms"] for s2, s3 in stats)
    # max over ranks of the timed region; units summed over ranks
    tmax, ttot, e2e_max = tot_ms, terms, sum(e2e_ms)
    if dist:
        t = torch.tensor([tot_ms, sum(e2e_ms)], dtype=torch.float64, device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        n = torch.tensor([float(terms)], dtype=torch.float64, device=dev)
        dist.all_reduce(n, op=dist.ReduceOp.SUM)
        tmax, e2e_max, ttot = float(t[0]), float(t[1]), float(n[0])
    value = ttot / (tmax * 1e-3)
    e2e_val = ttot / (e2e_max * 1e-3)
    # roofline of the dominant phase (device times measured by the library's events)
    ph = {}
    for key, fl in (("sr_ms", "sr_flops"), ("aft_ms", None), ("lr_gemm_ms", "lr_flops"), ("phase_ms", None),
                    ("other_ms", None)):
        ms = sum(s3[key] + s2[key] for s2, s3 in stats) / args.steps
        flops = (sum(s3[fl] + s2[fl] for s2, s3 in stats) / args.steps) if fl else None
        ph[key] = {"ms": ms, "tflops": (flops / (ms * 1e-3) / 1e12) if (fl and ms > 0) else None}
    dom = max(ph, key=lambda k: ph[k]["ms"])
    names = {"sr_ms": "k_sr3c (SR lattice-sum kernels)", "aft_ms": "k_aft (pair Fourier transforms)",
             "lr_gemm_ms": "k_zgemm_tn (LR contraction)", "phase_ms": "k_phase1/k_phase2", "other_ms": "other"}
    ach = ph[dom]["tflops"]
    roof = {"kernel": names[dom], "bound": "alu", "achieved": ach, "peak": peak_fp64, "unit": "TFLOP/s",
            "frac": (ach / peak_fp64) if ach else None, "traffic": None,
            "peak_source": "measured live: rsgdf_probe_fp64 (FP64 FMA chains on every SM)",
            "achieved_note": "algorithmic FP64 flops of the phase / its device time (CUDA events on the call's stream)"}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64" if args.precision == "fp64" else "f64+tf32x3/f32",
        "data": "synthetic", "config": dict(describe(p, omega, gmesh), precision=args.precision),
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": e2e_max / args.steps},
        "gpu_launches": int(sum(s2["n_launch"] + s3["n_launch"] for s2, s3 in stats)),
        "clocks": clk, "roofline": roof,
        "phases_ms_per_step": {k: v["ms"] for k, v in ph.items()},
        "phases_tflops": {k: v["tflops"] for k, v in ph.items()},
        "sr_terms_per_step": int(terms / args.steps), "sr_integrals_per_step": int(stats[0][1]["sr_integrals"]),
        "sr_primitive_terms_per_step": int(sum(s3["sr_prim_terms"] + s2["sr_prim_terms"] for s2, s3 in stats) / args.steps),
        "j3c_sr_by_L": {"terms": stats[-1][1]["sr_terms_by_L"], "ms": [round(x, 3) for x in stats[-1][1]["sr_ms_by_L"]]},
        "j3c_build_ms": statistics.median([s3["sr_ms"] + s3["aft_ms"] + s3["lr_gemm_ms"] + s3["phase_ms"] +
                                           s3["other_ms"] for _, s3 in stats]),
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        shells = (0, 16)
        n, dt, th = oracle_sample(p, omega, gmesh, shells)
        line["cpu_baseline"] = {"value": n / dt, "unit": UNIT, "cores": th, "kind": "oracle",
                                "sample": "aux shells [0,16) (all aux functions of the first atom, half the "
                                          "workload) x all %d k pairs, SR+G0+LR, %.1f s" % (p.nk * p.nk, dt)}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
