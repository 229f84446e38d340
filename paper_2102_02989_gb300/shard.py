"""Partitioning of the RSGDF work over ranks (one GPU each), with no exchange
on the data path: aux-shell ranges of one j3c (rows P of V are independent:
each needs the full lattice sums and G sum for its own aux functions only),
or the cells of a batch.  Host logic only; every rank then calls the library
on its own shard, and a consumer that wants the whole tensor gathers it.
"""
from __future__ import annotations

import numpy as np


def _shell_cost(aux, s):
    """Relative cost of one aux shell in j3c: Cartesian functions x primitives."""
    l = int(aux.l[s])
    return (l + 1) * (l + 2) // 2 * int(aux.nprim[s]) * (1 + l)


def aux_shell_shards(aux, nranks):
    """Contiguous aux-shell ranges [(s0, s1)] per rank, balanced by cost; every
    shell belongs to exactly one range; a range may be empty when there are
    more ranks than shells."""
    ns = len(aux.l)
    cost = np.array([_shell_cost(aux, s) for s in range(ns)], dtype=np.float64)
    cum = np.concatenate([[0.0], np.cumsum(cost)])
    cuts = [0]
    for r in range(1, nranks):
        cuts.append(int(np.searchsorted(cum, cum[-1] * r / nranks, side="left")))
    cuts.append(ns)
    cuts = [min(max(c, cuts[i - 1] if i else 0), ns) for i, c in enumerate(cuts)]
    return [(cuts[r], cuts[r + 1]) for r in range(nranks)]


def aux_func_offset(aux, s):
    """First aux function of shell s."""
    return int(sum((int(l) + 1) * (int(l) + 2) // 2 for l in aux.l[:s]))


def cell_shards(cells, nranks):
    """Cells of a batch per rank (longest-processing-time greedy on a cost
    estimate n_aux n_ao^2 N_k); returns lists of cell indices."""
    cost = [float(c.aux.nfunc) * c.ao.nfunc ** 2 * int(np.prod(c.kmesh)) for c in cells]
    order = sorted(range(len(cells)), key=lambda i: -cost[i])
    load = [0.0] * nranks
    out = [[] for _ in range(nranks)]
    for i in order:
        r = int(np.argmin(load))
        out[r].append(i)
        load[r] += cost[i]
    return [sorted(o) for o in out]


def reduce_timing(dist, times_ms, units, device=None):
    """Whole-job figures of a timed region: the time is the maximum over
    ranks, the units the sum.  Returns (max_ms_per_entry list, total units)."""
    import torch
    if dist is None:
        return list(times_ms), float(units)
    t = torch.tensor(list(times_ms), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    n = torch.tensor([float(units)], dtype=torch.float64, device=device)
    dist.all_reduce(n, op=dist.ReduceOp.SUM)
    return [float(x) for x in t.cpu()], float(n.item())
