#!/usr/bin/env python
"""Benchmark of the RSGDF hot path on GB300.

One step = the whole path for one cell: j2c with its Cholesky factors, then j3c
(SR lattice sums, G = 0 correction, pair and aux Fourier transforms, LR
contraction, Bloch-phase contractions) for every k pair of the mesh and every
aux function.  Default workload: FCC two-atom cell a = 6.74 Bohr, k-mesh 2x2x2
(64 k pairs), 30 Cartesian AO and 90 aux functions, eps = 1e-8, G box 7^3 with
omega from the LR cutoff.  Synthetic seeded inputs (the paper's basis sets are
not available).

Paths (--path): learned-mixed (default: learned screening of SR work items,
FP64 SR lattice sums, split-TF32 tensor-core LR contraction, FP32 phase
contractions), mixed, fp64.  Plain FP64 is always timed beside it on the same
workload, and the line reports the speedup and the error against it (max |dV|
and the first-order HF-energy proxy).

Metric: SR shell-triple lattice terms (aux shell, AO shell pair, l, d) of the
workload under the bound screening, per second of the whole step: the same
numerator for every path, so terms the learned screen skips count as speed.
The j3c build time is ms_per_step.  Besides the headline line: the same cell
on the 3x3x3 and 4x4x4 meshes (both paths) and the 32-cell batched workload
(graph replay with autotuned SR tiles vs one call per cell).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--path learned-mixed|mixed|fp64] [--quick] [--no-cpu-baseline]

Under torchrun the step is partitioned with no collective on the data path:
rank r computes j3c for its contiguous aux-shell range (rows P of V,
shard.aux_shell_shards) and j2c for its round-robin share of the k points;
units (bound-screened SR terms) are summed over ranks and the time is the
maximum over ranks; rank 0 prints one JSON line.  Extra sections (other
meshes, the batch, the rocksalt chunk, the tuned box, the DF consumers, the
compact/diffuse split) each run under a guard that records a failure in the
line instead of losing it.
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
DTYPES = {"fp64": "f64", "mixed": "f64 SR / tf32x3 LR / f32 phases",
          "learned-mixed": "f64 SR / tf32x3 LR / f32 phases, f16 screen network"}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--kmesh", default="2,2,2")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--path", default="learned-mixed", choices=["learned-mixed", "mixed", "fp64"])
    ap.add_argument("--quick", action="store_true", help="skip the per-k-mesh and batched measurements")
    return ap.parse_args()


def workload(kmesh):
    from paper_2102_02989_gb300 import inputs
    p = inputs.config2(tuple(kmesh))
    return p


def describe(p, omega, gmesh):
    return {"workload": "FCC a=6.74 Bohr 2-atom cell, k-mesh %dx%dx%d (%d k pairs), %d AO / %d aux Cartesian "
                        "functions, 3s2p1d AO per atom, ETB aux s8p5d2f1 per atom, eps_screen=eps_lr=%g, "
                        "G box %dx%dx%d, omega=%.6f; j2c+Cholesky+j3c(SR+G0+LR)"
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


def df_oracle_sample(J, V, D, kp, kmesh, ao_l, aux_l):
    """The DF and spherical oracles (numpy) on the same tensors as the GPU:
    metric transforms (automatic route), fit, J/K, and the Cartesian -> spherical
    transform of V.  Returns {step: seconds} and the threads numpy may use."""
    from oracle import dfjk, sph
    out = {}
    t0 = time.perf_counter()
    T, _, _, _ = dfjk.metric_transforms(J, "auto", rel=1e-6)
    out["metric_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    B = dfjk.fit(T, V, kp, kmesh)
    out["fit_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    dfjk.jk(B, kp, kmesh, D)
    out["jk_s"] = time.perf_counter() - t0
    t0 = time.perf_counter()
    sph.j3c(V, ao_l, aux_l)
    out["cart2sph_s"] = time.perf_counter() - t0
    return out, os.cpu_count()


# The oracle sample both arms time: every aux shell of the first atom (s8 p5 d2 f1,
# every angular-momentum class of the workload, half of its aux functions) x
# every k pair, SR + G0 + LR.  The one-core figure uses one shell per class.
ORACLE_SHELLS = (0, 16)
ORACLE_SHELL_1CORE = 10   # the first atom's p shell of exponent 0.8, the middle of its p shells


def oracle_1core_sample(p, omega, gmesh):
    """The oracle on one host core: one aux shell (ORACLE_SHELL_1CORE, a
    p shell from the middle of the exponent range; one shell already takes
    about 20 s on one core, most of it the reciprocal-space part over 64
    k pairs), every k pair."""
    import oracle
    oracle.build()
    s = ORACLE_SHELL_1CORE
    kp = [(i, j) for i in range(p.nk) for j in range(p.nk)]
    nth = oracle.num_threads()
    oracle.set_num_threads(1)
    try:
        t0 = time.perf_counter()
        _, cnt = oracle.j3c(p.a, p.kmesh, p.ao, p.aux, omega, kp, eps_sr=p.eps_sr, eps_lr=p.eps_lr,
                            gmesh=gmesh, shells=(s, s + 1), return_counts=True)
        dt = time.perf_counter() - t0
    finally:
        oracle.set_num_threads(nth)
    return {"value": cnt["terms"] / dt, "unit": UNIT, "cores": 1, "kind": "oracle", "seconds": dt,
            "terms": int(cnt["terms"]),
            "sample": "aux shell %d (l=%d, exponent %g) x all %d k pairs, SR+G0+LR"
                      % (s, int(p.aux.l[s]), float(p.aux.exps[p.aux.prim_off[s]]), p.nk * p.nk)}


def run_reference(args, rank, world):
    """The oracle as it stands, timed on the host cores (rank 0 only; the other
    ranks of a torchrun launch exit without work).  Each step is the bounded
    sample ORACLE_SHELLS of the headline workload, the same sample as the
    cpu_baseline leg of the GPU arm; after the timed steps, one run of
    oracle_1core_sample gives the single-core figure."""
    if rank != 0:
        return
    kmesh = [int(x) for x in args.kmesh.split(",")]
    p = workload(kmesh)
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    from rules_ref import omega_for
    omega = omega_for(p.a, p.gmesh, p.eps_lr, p.kmesh)
    gmesh = p.gmesh
    for _ in range(args.warmup):
        oracle_sample(p, omega, gmesh, ORACLE_SHELLS)
    times, terms, th = [], 0, 1
    for _ in range(args.steps):
        n, dt, th = oracle_sample(p, omega, gmesh, ORACLE_SHELLS)
        times.append(dt)
        terms += n
    tot = sum(times)
    val = terms / tot
    sample = ("aux shells [%d,%d) of %d (every aux shell of the first atom: s8 p5 d2 f1) x all %d k pairs, "
              "SR+G0+LR per step" % (ORACLE_SHELLS[0], ORACLE_SHELLS[1], p.aux.nshell, p.nk * p.nk))
    line = {
        "impl": "reference", "metric": METRIC, "value": val, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": dict(describe(p, omega, gmesh), path=args.path),
        "cpu_baseline": {"value": val, "unit": UNIT, "cores": th, "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    guarded(line, "cpu_baseline_1core", lambda: oracle_1core_sample(p, omega, gmesh))
    print(json.dumps(line), flush=True)


def guarded(line, key, fn):
    """line[key] = fn(), or {"error": ...} if fn raises: a failing extra section
    is recorded and never costs the headline line."""
    t0 = time.perf_counter()
    try:
        out = fn()
    except Exception as e:   # noqa: BLE001 -- recorded in the line
        out = {"error": repr(e)[:400]}
    if out is not None:
        if isinstance(out, dict):
            out.setdefault("section_s", round(time.perf_counter() - t0, 2))
        line[key] = out


def train_network(rsgdf, screening, inputs):
    """Learned screen: trained on the SR items of the cubic 2-atom Gamma cell
    and of an FCC cell with another draw of the basis (not the timed one)."""
    p1 = inputs.config1()
    _, gm1 = rsgdf.rsgdf_params(p1.a, p1.kmesh, omega=p1.omega, eps_lr=p1.eps_lr)
    pt = inputs.config2(seed_offset=12)
    wt, gmt = rsgdf.rsgdf_params(pt.a, pt.kmesh, gmesh=pt.gmesh, eps_lr=pt.eps_lr)
    t0 = time.perf_counter()
    X, t = screening.items_dataset([(p1.a, p1.kmesh, p1.ao, p1.aux, p1.omega, gm1, p1.eps_lr),
                                    (pt.a, pt.kmesh, pt.ao, pt.aux, wt, gmt, pt.eps_lr)], eps_screen=1e-8)
    m, info = screening.train_screen(X, t, seed=0, eps_screen=1e-8)
    info["train_s"] = time.perf_counter() - t0
    info["data"] = ("SR items of the cubic a=4.0 2-atom Gamma cell and of the FCC a=6.74 cell with another "
                    "basis draw (seed offset 12), eps 1e-8")
    return m, info


def setup_dist(world, local):
    import torch
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    return dist, dev


def sr_flops_table():
    """Per-class FP64 flops of one SR term (one primitive combination at one
    lattice translation), as counted by the oracle's instrumented evaluation
    and stored beside the golden fixtures; None if the table is absent."""
    path = os.path.join(ROOT, "tests", "golden", "sr_flops_by_L.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def measured_traffic(kernel_key):
    """DRAM bytes per step of a kernel from the committed ncu summary, if the
    summary was taken on the current kernel source (its sha256 recorded in
    the summary); None otherwise."""
    import hashlib
    import glob
    src = os.path.join(ROOT, "paper_2102_02989_gb300", "csrc", "k_sr.cu")
    sha = hashlib.sha256(open(src, "rb").read()).hexdigest()[:16]
    for f in sorted(glob.glob(os.path.join(ROOT, "profiles", "*.md"))):
        for ln in open(f):
            if ln.startswith("bench-traffic:"):
                try:
                    rec = json.loads(ln.split(":", 1)[1])
                except ValueError:
                    continue
                if rec.get("kernel") == kernel_key and rec.get("k_sr_sha16") == sha:
                    return rec
    return None


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
    dist, dev = setup_dist(world, local)
    from paper_2102_02989_gb300 import hfproxy, inputs, rsgdf, screening, shard
    rsgdf.load()
    kmesh = [int(x) for x in args.kmesh.split(",")]
    p = workload(kmesh)
    omega, gmesh = rsgdf.rsgdf_params(p.a, p.kmesh, gmesh=p.gmesh, eps_lr=p.eps_lr)
    base = dict(omega=omega, gmesh=gmesh, eps_screen=p.eps_sr, eps_lr=p.eps_lr)
    mlp, train_info = (None, None)
    if args.path == "learned-mixed":
        mlp, train_info = train_network(rsgdf, screening, inputs)
    paths = {"fp64": dict(base, precision=rsgdf.RSGDF_FP64),
             "mixed": dict(base, precision=rsgdf.RSGDF_MIXED),
             "learned-mixed": dict(base, precision=rsgdf.RSGDF_MIXED, screening=rsgdf.RSGDF_SCREEN_LEARNED,
                                   mlp=mlp.h if mlp else None)}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    # this rank's share of the step: a contiguous aux-shell range of j3c
    # (rows P of V) and a round-robin share of the k points of j2c; one rank
    # holds the whole step
    shells = shard.aux_shell_shards(p.aux, world, cost=shard.planner_costs(p.a, p.kmesh, p.ao, p.aux, **base)
                                    if world > 1 else None)[rank]
    klist = list(range(rank, p.nk, world))

    def make(prob, opt, shells=None, klist=None):
        kp = np.array([(i, j) for i in range(prob.nk) for j in range(prob.nk)], dtype=np.int32)
        kl = list(range(prob.nk)) if klist is None else list(klist)
        s0, s1 = shells if shells is not None else (0, prob.aux.nshell)
        nP = shard.aux_func_offset(prob.aux, s1) - shard.aux_func_offset(prob.aux, s0)
        V = torch.zeros((len(kp), nP, prob.ao.nfunc, prob.ao.nfunc), dtype=torch.complex128, device=dev)
        empty = {"sr_terms": 0, "n_launch": 0}
        # j2c statistics are the same every step: read them once here, so that
        # no stream synchronisation sits between the two calls of a step (the
        # host planning of j3c overlaps the device work of j2c, as for any caller)
        if kl:
            rsgdf.rsgdf_j2c(prob.a, prob.kmesh, prob.aux, kl, **opt)
            s2 = rsgdf.rsgdf_last_stats()
        else:
            s2 = None

        def step():
            J2 = rsgdf.rsgdf_j2c(prob.a, prob.kmesh, prob.aux, kl, **opt) if kl else (None, None, None)
            if s1 > s0:
                rsgdf.rsgdf_j3c(prob.a, prob.kmesh, prob.ao, prob.aux, kp, shells=(s0, s1), out=V, **opt)
                s3 = rsgdf.rsgdf_last_stats()
            else:
                s3 = None
            return J2, _stats0(s2), _stats0(s3)
        return step, V, kp

    def timed(step, nsteps, nwarm, rng="timed_step"):
        for _ in range(max(nwarm, 0)):
            step()
        torch.cuda.synchronize()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(nsteps)]
        stats = []
        out = None
        for i in range(nsteps):
            flush.zero_()
            torch.cuda.synchronize()
            torch.cuda.nvtx.range_push(rng)   # launch lists: ncu --nvtx --nvtx-include timed_step/
            ev[i][0].record()
            out, s2, s3 = step()
            ev[i][1].record()
            torch.cuda.nvtx.range_pop()
            torch.cuda.synchronize()
            stats.append((s2, s3))
        return [a.elapsed_time(b) for a, b in ev], stats, out

    peak_fp64 = rsgdf.rsgdf_probe_fp64()
    step, V, kp = make(p, paths[args.path], shells, klist)
    ref_step, Vref, _ = make(p, paths["fp64"], shells, klist)
    clocks = Clocks()
    clocks.start()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    times, stats, (J, L, info) = timed(step, args.steps, args.warmup)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop(gpu_index=local)
    tot_ms = sum(times)
    # plain FP64 on the same workload: the comparison and the work count
    ref_times, ref_stats, _ = (timed(ref_step, args.steps, args.warmup, "fp64_step") if args.path != "fp64"
                               else (times, stats, None))
    work = sum(s3["sr_terms"] + s2["sr_terms"] for s2, s3 in ref_stats) / len(ref_stats)   # bound-screened terms
    own_terms = sum(s3["sr_terms"] + s2["sr_terms"] for s2, s3 in stats) / len(stats)
    # end to end through the public API: host inputs (uploaded by the call) and
    # a device-to-host read of every result into pinned memory
    hV = torch.empty(V.shape, dtype=V.dtype, pin_memory=True)
    h2d = sum(np.asarray(x).nbytes for b in (p.ao, p.aux) for x in (b.l, b.nprim, b.prim_off, b.center, b.exps, b.coeffs))
    h2d = 2 * h2d + kp.nbytes + 4 * len(klist)
    e2e_ms = []
    d2h = 0
    for i in range(args.steps):
        flush.zero_()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        (J, L, info), _, _ = step()
        hV.copy_(V, non_blocking=True)
        hres = [x.to("cpu", non_blocking=True) for x in (J, L, info) if x is not None]
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
        d2h = V.numel() * 16 + sum(x.numel() * x.element_size() for x in hres)
    # max over ranks of the timed region; units summed over ranks
    (tmax, e2e_max), ttot = shard.reduce_timing(dist, [tot_ms, sum(e2e_ms)], work * args.steps, device=dev)
    value = ttot / (tmax * 1e-3)
    e2e_val = ttot / (e2e_max * 1e-3)
    ref_ms = sum(ref_times) / len(ref_times)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": tmax / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[args.path], "data": "synthetic",
        "config": dict(describe(p, omega, gmesh), path=args.path,
                       parallelism="aux-shell shards of j3c, k-point shards of j2c, %d rank(s)" % world,
                       rank0_shard={"aux_shells": list(shells), "j2c_k": klist}),
        "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": int(h2d), "d2h_bytes_per_step": int(d2h),
                "ms_per_step": e2e_max / args.steps},
        "gpu_launches": int(sum(s2["n_launch"] + s3["n_launch"] for s2, s3 in stats)),
        "clocks": clk,
        "vs_plain_fp64": {"fp64_ms_per_step": ref_ms, "fp64_value": work / (ref_ms * 1e-3),
                          "speedup": ref_ms / (tmax / args.steps)},
        "sr_terms_per_step": {"bound_screened": int(work), "computed": int(own_terms),
                              "prim_terms_evaluated": int(sum(sum(s2.get("sr_prim_terms_by_L", [])) +
                                                              sum(s3.get("sr_prim_terms_by_L", []))
                                                              for s2, s3 in stats) / len(stats)),
                              "prim_terms_dropped_by_combination_bound": int(
                                  sum(s2.get("sr_prim_terms_skipped", 0) + s3.get("sr_prim_terms_skipped", 0)
                                      for s2, s3 in stats) / len(stats))},
    }
    guarded(line, "roofline", lambda: roofline(stats, args, peak_fp64))
    line["phases_ms_per_step"] = line["roofline"].pop("phases_ms", None)
    line["phases_tflops"] = line["roofline"].pop("phases_tflops", None)
    last3 = stats[-1][1]
    line.update({
        "sr_items_pruned_per_step": int(last3.get("sr_items_pruned", 0)),
        "sr_items_per_step": int(last3.get("sr_items", 0)),
        "j3c_sr_by_L": {"terms": last3.get("sr_terms_by_L"), "prim_terms": last3.get("sr_prim_terms_by_L"),
                        "ms": [round(x, 3) for x in last3.get("sr_ms_by_L", [])]},
        "j3c_build_ms": statistics.median([s3["sr_ms"] + s3["aft_ms"] + s3["lr_gemm_ms"] + s3["phase_ms"] +
                                           s3["other_ms"] for _, s3 in stats]),
    })
    if train_info:
        line["learned_screen"] = {k: (round(v, 4) if isinstance(v, float) else v) for k, v in train_info.items()}

    # accuracy against plain FP64 on the same GPU: max |dV| and the HF-energy proxy
    def accuracy():
        ref_step()
        step()
        torch.cuda.synchronize()
        hv, hr = V.cpu().numpy(), Vref.cpu().numpy()
        acc = {"max_abs_vs_fp64": float(np.max(np.abs(hv - hr))), "max_abs_fp64": float(np.max(np.abs(hr)))}
        if world == 1:
            acc.update({"hf_proxy_" + k: v for k, v in
                        hfproxy.energy_error(hv, hr, kp, p.kmesh, J.cpu().numpy()).items()})
            acc["hf_proxy_note"] = ("first-order HF energy change per cell, Hartree; metric inverted on "
                                    "eigenvalues > 1e-6 of the largest")
        return acc
    guarded(line, "accuracy", accuracy)
    if isinstance(line.get("accuracy"), dict):
        line["vs_plain_fp64"].update(line.pop("accuracy"))
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        def cpu_leg():
            n, dt, th = oracle_sample(p, omega, gmesh, ORACLE_SHELLS)
            return {"value": n / dt, "unit": UNIT, "cores": th, "kind": "oracle",
                    "sample": "aux shells [%d,%d) (every aux shell of the first atom: s8 p5 d2 f1, half the aux "
                              "functions) x all %d k pairs, SR+G0+LR, %.1f s"
                              % (ORACLE_SHELLS[0], ORACLE_SHELLS[1], p.nk * p.nk, dt)}
        guarded(line, "cpu_baseline", cpu_leg)
    if rank == 0 and not args.quick:
        del hV
        guarded(line, "per_kmesh", lambda: per_kmesh(rsgdf, inputs, paths, make, timed, np))
        guarded(line, "batch", lambda: batch_bench(rsgdf, inputs, np, torch))
        if paths["learned-mixed"].get("mlp") is not None:
            guarded(line, "rocksalt_chunk", lambda: rocksalt_bench(rsgdf, inputs, paths, np, torch))
            guarded(line, "auto_omega", lambda: auto_omega_bench(rsgdf, p, paths, make, timed, np))
        guarded(line, "df_consumers", lambda: df_bench(rsgdf, hfproxy, inputs, paths, make, np, torch, peak_fp64,
                                                        cpu_baseline=world == 1 and not args.no_cpu_baseline))
        guarded(line, "split_route", lambda: split_bench(rsgdf, inputs, torch))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist:
        dist.destroy_process_group()


def _stats0(s):
    """Library statistics of a call, or zeros for a call this rank did not make."""
    if s is not None:
        return s
    return {"sr_terms": 0, "sr_integrals": 0, "sr_flops": 0, "aft_units": 0, "lr_flops": 0, "n_launch": 0,
            "sr_ms": 0.0, "aft_ms": 0.0, "lr_gemm_ms": 0.0, "phase_ms": 0.0, "other_ms": 0.0,
            "sr_terms_by_L": [0] * 10, "sr_prim_terms": 0, "sr_items": 0, "sr_items_pruned": 0,
            "sr_ms_by_L": [0.0] * 10, "sr_prim_terms_by_L": [0] * 10, "sr_prim_terms_skipped": 0}


PHASE_NAMES = {"sr_ms": "k_sr3c (SR lattice-sum kernels, all class launches of one step)",
               "aft_ms": "k_aft (pair Fourier transforms)", "lr_gemm_ms": "LR contraction GEMM",
               "phase_ms": "k_phase1/k_phase2", "other_ms": "other"}


def roofline(stats, args, peak_fp64):
    """Roofline of the dominant phase.  Device times are the library's CUDA
    events on the call's stream; the SR flop numerator is the oracle-counted
    per-class table (flops per primitive-combination term) times the
    primitive-combination terms the kernels evaluated, per class."""
    nsteps = len(stats)
    ph = {}
    for key in ("sr_ms", "aft_ms", "lr_gemm_ms", "phase_ms", "other_ms"):
        ph[key] = sum(s3[key] + s2[key] for s2, s3 in stats) / nsteps
    table = sr_flops_table()
    sr_flops = None
    if table is not None:
        fl = table["flops_per_term_by_L"]
        sr_flops = sum(sum(n * fl[L] for L, n in enumerate(s2.get("sr_prim_terms_by_L", [])) if n) +
                       sum(n * fl[L] for L, n in enumerate(s3.get("sr_prim_terms_by_L", [])) if n)
                       for s2, s3 in stats) / nsteps
    lr_flops = sum(s3["lr_flops"] + s2["lr_flops"] for s2, s3 in stats) / nsteps
    tflops = {"sr_ms": (sr_flops / (ph["sr_ms"] * 1e-3) / 1e12) if (sr_flops and ph["sr_ms"] > 0) else None,
              "lr_gemm_ms": (lr_flops / (ph["lr_gemm_ms"] * 1e-3) / 1e12) if ph["lr_gemm_ms"] > 0 else None}
    dom = max(ph, key=lambda k: ph[k])
    ach = tflops.get(dom)
    tr = measured_traffic("k_sr3c") if dom == "sr_ms" else None
    traffic = None
    if tr is not None and tr.get("workload_kmesh") == [int(x) for x in args.kmesh.split(",")] and \
            tr.get("path") == args.path:
        traffic = tr["bytes_per_step"]
    return {"kernel": PHASE_NAMES[dom], "bound": "alu", "achieved": ach, "peak": peak_fp64, "unit": "TFLOP/s",
            "frac": (ach / peak_fp64) if ach else None, "traffic": traffic,
            "traffic_unit": "DRAM bytes per step of the phase (all its launches), from the committed ncu summary "
                            "of the current kernel source; null when none matches",
            "peak_source": "measured live: rsgdf_probe_fp64 (independent FP64 FMA chains on every SM)",
            "achieved_note": "oracle-counted FP64 flops per SR term (tests/golden/sr_flops_by_L.json) x "
                             "primitive-combination terms evaluated, per class L / the phase's device time "
                             "(CUDA events on the call's stream)",
            "flops_per_step": sr_flops if dom == "sr_ms" else lr_flops,
            "phases_tflops": tflops, "phases_ms": ph}


def per_kmesh(rsgdf, inputs, paths, make, timed, np):
    """The same cell on the 3x3x3 and 4x4x4 meshes: both paths, 2 steps each."""
    out = {}
    for km in ((3, 3, 3), (4, 4, 4)):
        p = inputs.config2(km)
        w, gm = rsgdf.rsgdf_params(p.a, p.kmesh, gmesh=p.gmesh, eps_lr=p.eps_lr)
        res = {}
        Vs = {}
        for name in ("fp64", "learned-mixed"):
            opt = dict(paths[name], omega=w, gmesh=gm)
            if name == "learned-mixed" and opt.get("mlp") is None:
                continue
            step, V, _ = make(p, opt)
            t, st, _ = timed(step, 2, 1, "kmesh_step")
            ms = sum(t) / len(t)
            res[name] = {"ms_per_step": ms, "sr_terms": int(st[-1][1]["sr_terms"] + st[-1][0]["sr_terms"])}
            Vs[name] = V
        if "learned-mixed" in Vs:
            d = (Vs["learned-mixed"] - Vs["fp64"]).abs().max().item()
            res["max_abs_vs_fp64"] = d
            res["speedup"] = res["fp64"]["ms_per_step"] / res["learned-mixed"]["ms_per_step"]
            res["value_learned_mixed"] = res["fp64"]["sr_terms"] / (res["learned-mixed"]["ms_per_step"] * 1e-3)
        res["value_fp64"] = res["fp64"]["sr_terms"] / (res["fp64"]["ms_per_step"] * 1e-3)
        del Vs
        out["%dx%dx%d" % km] = res
    return out


def df_bench(rsgdf, hfproxy, inputs, paths, make, np, torch, peak_fp64, cpu_baseline=True):
    """Density-fitting consumers after the step: the fitting transforms of the
    j2c metrics (automatic Cholesky / eigen choice), the fit B = T V over every
    k pair and the fitted Coulomb and exchange matrices of a synthetic
    closed-shell density, each timed alone (CUDA events, median of 3 after one
    warm-up), on the headline cell at 2x2x2 and 4x4x4.  The energies from the
    GPU J/K (eigen route, as the host proxy) are checked against the host's
    FP64 HF-energy proxy of the same tensors."""
    def ev(f, reps=3):
        f()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            f()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    out = {}
    for km in ((2, 2, 2), (4, 4, 4)):
        prob = inputs.config2(km)
        w, gm = rsgdf.rsgdf_params(prob.a, prob.kmesh, gmesh=prob.gmesh, eps_lr=prob.eps_lr)
        step, V, kp = make(prob, dict(paths["fp64"], omega=w, gmesh=gm))
        (J, _, _), _, _ = step()
        nao, naux = V.shape[-1], V.shape[1]
        D = torch.from_numpy(hfproxy.densities(prob.kmesh, nao, max(1, nao // 4))).to(V.device)
        res, keep = {}, {}

        def metric(method):
            keep["m"] = rsgdf.rsgdf_df_metric(J, method, 1e-6)
        res["metric_ms"] = ev(lambda: metric(rsgdf.RSGDF_FIT_AUTO))
        info = keep["m"][3].cpu().numpy()
        res["routes"] = {"cholesky": int(np.sum(info == 0)), "eigen": int(np.sum(info >= 1)),
                         "max_sweeps": int(info.max())}
        metric(rsgdf.RSGDF_FIT_EIGEN)
        T = keep["m"][0]
        B = torch.empty_like(V)
        res["fit_ms"] = ev(lambda: rsgdf.rsgdf_df_fit(prob.a, prob.kmesh, T, V, kp, out=B))
        res["jk_ms"] = ev(lambda: keep.update(jk=rsgdf.rsgdf_df_jk(prob.a, prob.kmesh, B, kp, D)))
        fit_fl = 8.0 * naux * naux * nao * nao * len(kp)
        jk_fl = 2 * 8.0 * naux * nao ** 3 * len(kp)
        res["fit_tflops"] = fit_fl / (res["fit_ms"] * 1e-3) / 1e12
        res["jk_tflops"] = jk_fl / (res["jk_ms"] * 1e-3) / 1e12
        res["fp64_peak_tflops"] = peak_fp64
        Jm, Km = (x.cpu().numpy() for x in keep["jk"])
        Dh = D.cpu().numpy()
        ej = float(np.real(sum(np.trace(Dh[k] @ Jm[k]) for k in range(prob.nk)))) / (2 * prob.nk)
        ek = -float(np.real(sum(np.trace(Dh[k] @ Km[k]) for k in range(prob.nk)))) / (4 * prob.nk)
        hj, hk = hfproxy.energies(V.cpu().numpy(), kp, prob.kmesh, hfproxy.fit_transforms(J.cpu().numpy(), 1e-6), Dh)
        res.update({"E_J": ej, "E_K": ek, "dE_J_vs_host": abs(ej - hj), "dE_K_vs_host": abs(ek - hk)})
        # Cartesian -> spherical transform of the whole j3c tensor (HBM-bound gather)
        Vs = rsgdf.rsgdf_cart2sph_j3c(prob.ao, prob.aux, V)
        res["cart2sph_ms"] = ev(lambda: rsgdf.rsgdf_cart2sph_j3c(prob.ao, prob.aux, V))
        nbytes = V.numel() * 16 + Vs.numel() * 16
        res["cart2sph_gbs"] = nbytes / (res["cart2sph_ms"] * 1e-3) / 1e9
        res["cart2sph_bytes"] = int(nbytes)
        peaks = os.path.join(ROOT, "MEASURED_PEAKS.json")
        if os.path.exists(peaks):
            res["cart2sph_frac_of_measured_hbm"] = res["cart2sph_gbs"] / json.load(open(peaks))["hbm_gbs"]
        del Vs
        if cpu_baseline and km == (2, 2, 2):
            try:
                t, cores = df_oracle_sample(J.cpu().numpy(), V.cpu().numpy(), Dh, kp, prob.kmesh, prob.ao.l,
                                            prob.aux.l)
                res["cpu_baseline"] = {"kind": "oracle", "cores": cores, "unit": "s",
                                       "sample": "the same tensors, numpy FP64 (LAPACK eigh, matmul)", **t}
            except Exception as e:   # recorded, so that a failure here does not cost the headline line
                res["cpu_baseline"] = {"error": repr(e)[:300]}
        out["%dx%dx%d" % km] = res
        del V, B, J, keep
        torch.cuda.empty_cache()
    out["note"] = ("FP64 throughout; fit and J/K are complex GEMMs on the FP64 pipe (flops 8 naux^2 nao^2 and "
                   "16 naux nao^3 per k pair); metric = Cholesky + triangular inverse, Jacobi where it fails")
    return out


def split_bench(rsgdf, inputs, torch):
    """j3c (every k pair and aux shell) of the headline cell at 2x2x2 on the
    11^3 box (omega 0.691, the box the tuner picks for the mixed path): the
    plain range-separated route against the compact/diffuse split route
    (alpha_cut = omega^2/2), FP64 and mixed, CUDA events around the whole
    call, median of 3 after one warm-up; the planner's SR work of both."""
    from paper_2102_02989_gb300 import cdsplit
    p = inputs.config2((2, 2, 2))
    gm = (11, 11, 11)
    w, _ = rsgdf.rsgdf_params(p.a, p.kmesh, gmesh=gm, eps_lr=p.eps_lr)
    kp = inputs.kpairs_all(p.nk)
    opt = dict(omega=w, gmesh=gm, eps_screen=p.eps_sr, eps_lr=p.eps_lr)
    ac = 0.5 * w * w
    out = {}

    def ev(f, reps=3):
        f()
        torch.cuda.synchronize()
        ts = []
        for _ in range(reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            f()
            b.record()
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        return statistics.median(ts)

    res = {"workload": "FCC a=6.74 2-atom cell, 2x2x2, all 64 k pairs, j3c only, eps 1e-8",
           "gmesh": list(gm), "omega": w, "alpha_cut": ac,
           "sr_candidate_terms_plain_split_rs": list(
               rsgdf.rsgdf_sr_items_split(p.a, p.kmesh, p.ao, p.aux, ac, **opt)["terms"])}
    for name, prec in (("fp64", rsgdf.RSGDF_FP64), ("mixed", rsgdf.RSGDF_MIXED)):
        try:
            o = dict(opt, precision=prec)
            r = {"plain_ms": ev(lambda: out.update(plain=rsgdf.rsgdf_j3c(p.a, p.kmesh, p.ao, p.aux, kp, **o))),
                 "split_ms": ev(lambda: out.update(split=cdsplit.j3c_split(p.a, p.kmesh, p.ao, p.aux, kp,
                                                                             alpha_cut=ac, **o)))}
            r["speedup"] = r["plain_ms"] / r["split_ms"]
            r["max_abs_split_vs_plain"] = (out["split"] - out["plain"]).abs().max().item()
            res[name] = r
        except Exception as e:   # recorded per precision
            res[name] = {"error": repr(e)[:300]}
        out.clear()
    return res


def auto_omega_bench(rsgdf, p, paths, make, timed, np):
    """The same cell and mesh with the G box (hence omega) chosen per path by
    timing the candidates 5^3..13^3 (tuning.tune_gmesh), then the whole step
    (j2c + j3c) on the chosen box, learned+mixed and plain FP64."""
    from paper_2102_02989_gb300 import tuning
    kp = np.array([(i, j) for i in range(p.nk) for j in range(p.nk)], dtype=np.int32)
    res = {}
    Vs = {}
    for name in ("learned-mixed", "fp64"):
        opt = {k: v for k, v in paths[name].items() if k not in ("omega", "gmesh")}
        gm, w, times = tuning.tune_gmesh(p.a, p.kmesh, p.ao, p.aux, kp, candidates=(5, 7, 9, 11, 13), reps=1, **opt)
        step, V, _ = make(p, dict(opt, omega=w, gmesh=gm))
        t, st, _ = timed(step, 3, 1, "auto_step")
        res[name] = {"gmesh": list(gm), "omega": w, "ms_per_step": statistics.median(t),
                     "j3c_ms_by_box": {str(n): round(ms, 2) for n, (_, ms) in times.items()}}
        Vs[name] = V
    res["speedup"] = res["fp64"]["ms_per_step"] / res["learned-mixed"]["ms_per_step"]
    res["max_abs_vs_fp64"] = (Vs["learned-mixed"] - Vs["fp64"]).abs().max().item()
    res["note"] = ("the range-separated sum is omega-independent; each path runs on the box that is fastest for it, "
                   "same cell, mesh and eps as the headline")
    return res


def rocksalt_bench(rsgdf, inputs, paths, np, torch):
    """The network applied to the 8-atom rocksalt cell (a = 8.0, 4x4x4 mesh,
    120 AO, 360 aux): j3c of the first atom's 16 aux shells on the 64 diagonal
    k pairs, learned+mixed vs plain FP64 (one warm-up, median of 3)."""
    p = inputs.config5()
    w, gm = rsgdf.rsgdf_params(p.a, p.kmesh, gmesh=p.gmesh, eps_lr=p.eps_lr)
    kp = inputs.kpairs_diag(p.nk)
    sh = (0, 16)
    res = {}
    outs = {}
    for name in ("fp64", "learned-mixed"):
        opt = dict(paths[name], omega=w, gmesh=gm)
        out = None
        times = []
        for rep in range(4):
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = rsgdf.rsgdf_j3c(p.a, p.kmesh, p.ao, p.aux, kp, shells=sh, out=out, **opt)
            e1.record()
            torch.cuda.synchronize()
            st = rsgdf.rsgdf_last_stats()
            if rep:
                times.append(e0.elapsed_time(e1))
        res[name] = {"ms": statistics.median(times), "sr_ms": st["sr_ms"], "sr_terms": int(st["sr_terms"]),
                     "sr_items": int(st["sr_items"]), "sr_items_pruned": int(st["sr_items_pruned"]),
                     "sr_prim_terms": int(sum(st.get("sr_prim_terms_by_L", [])))}
        outs[name] = out
    res["speedup"] = res["fp64"]["ms"] / res["learned-mixed"]["ms"]
    res["sr_speedup"] = res["fp64"]["sr_ms"] / res["learned-mixed"]["sr_ms"]
    res["max_abs_vs_fp64"] = (outs["learned-mixed"] - outs["fp64"]).abs().max().item()
    res["workload"] = ("rocksalt a=8.0 8-atom cell, 4x4x4, aux shells [0,16) (45 of 360 aux functions), 64 diagonal "
                       "k pairs, eps 1e-8, G box 7^3, omega %.4f; network trained on other cells" % w)
    return res


def batch_bench(rsgdf, inputs, np, torch):
    """32 heterogeneous cells, diagonal k pairs, FP64: batched handle with
    graph + autotuned SR tiles vs the same cells one call at a time."""
    cells = inputs.config4()
    probs = [(c.a, c.kmesh, c.ao, c.aux) for c in cells]
    kps = [inputs.kpairs_diag(c.nk) for c in cells]
    opt = dict(gmesh=(7, 7, 7), eps_screen=1e-8, eps_lr=1e-8)
    s = torch.cuda.Stream()
    t0 = time.perf_counter()
    b = rsgdf.Batch(probs, kps, flags=rsgdf.RSGDF_BATCH_GRAPH | rsgdf.RSGDF_BATCH_AUTOTUNE, stream=s, **opt)
    outs = b.outputs()
    b.run(outs, stream=s)     # autotune + capture
    s.synchronize()
    setup_s = time.perf_counter() - t0
    st = rsgdf.rsgdf_last_stats()
    times = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(s)
        b.run(outs, stream=s)
        e1.record(s)
        s.synchronize()
        times.append(e0.elapsed_time(e1))
    tiles = b.tiles()
    b.close()
    # the same cells, one library call each (plans included, as a user would call)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    terms = 0
    with torch.cuda.stream(s):
        for c, kp, o in zip(cells, kps, outs):
            rsgdf.rsgdf_j3c(c.a, c.kmesh, c.ao, c.aux, kp, out=o, stream=s, **opt)
            terms += rsgdf.rsgdf_last_stats()["sr_terms"]
    s.synchronize()
    seq_ms = 1e3 * (time.perf_counter() - t0)
    ms = statistics.median(times)
    return {"workload": "32 cells: 1-8 atoms, cubic/FCC a in [5,10] Bohr, random AO shells l<=3, ETB aux ~3x, "
                        "k-meshes 1^3-3^3, diagonal k pairs, eps 1e-8, G box 7^3, FP64",
            "graph_replay_ms": ms, "value": terms / (ms * 1e-3), "unit": UNIT,
            "sequential_calls_ms": seq_ms, "speedup_vs_sequential": seq_ms / ms,
            "create_tune_capture_s": setup_s, "sr_items": int(st["sr_items"]), "launches_per_run": int(st["n_launch"]),
            "sr_tiles": tiles}


if __name__ == "__main__":
    main()
