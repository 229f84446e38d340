"""Automatic choice of the G box, hence of omega, for a j3c problem.

The range-separation parameter trades SR work (the real-space lattice sums
shrink roughly as omega^-3) against LR work (the plane waves grow as the box
volume).  The paper tunes the plane-wave count by hand so that the two parts
balance; this module does it by measurement: it times the library's own j3c
on each candidate odd box n^3 (omega from the LR cutoff for that box) and
keeps the fastest.  Every candidate computes the same integrals up to the
screening thresholds (the sum is omega-independent), so the choice changes the
cost only.  Host orchestration; all work runs in the library.
"""
from __future__ import annotations

import statistics


def tune_gmesh(a, kmesh, ao, aux, kpairs, candidates=(5, 7, 9, 11, 13), reps=2, shells=None, stream=None,
               **opt):
    """Time rsgdf_j3c on each box n^3 in ``candidates`` (one warm-up, median
    of ``reps``) and return (best gmesh, best omega, {n: (omega, ms)}).
    ``opt`` are the other j3c options (eps_screen, eps_lr, precision, ...);
    omega and gmesh are set per candidate."""
    import torch
    from . import rsgdf
    opt = {k: v for k, v in opt.items() if k not in ("omega", "gmesh")}
    times = {}
    out = None
    for n in candidates:
        gm = (n, n, n)
        try:
            w, _ = rsgdf.rsgdf_params(a, kmesh, gmesh=gm, eps_lr=opt.get("eps_lr", 1e-8))
        except rsgdf.RsgdfError:
            continue   # box too small for this k mesh
        ts = []
        for r in range(reps + 1):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            out = rsgdf.rsgdf_j3c(a, kmesh, ao, aux, kpairs, shells=shells, out=out, gmesh=gm, stream=stream, **opt)
            e1.record()
            torch.cuda.synchronize()
            if r:
                ts.append(e0.elapsed_time(e1))
        times[n] = (w, statistics.median(ts))
    if not times:
        raise ValueError("no candidate box is usable for this k mesh")
    best = min(times, key=lambda n: times[n][1])
    return (best, best, best), times[best][0], times
