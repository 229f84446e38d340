"""Partitioning of the RSGDF work over ranks (one GPU each).  The integrals
need no exchange on the data path: aux-shell ranges of one j3c (rows P of V
are independent: each needs the full lattice sums and G sum for its own aux
functions only), or the cells of a batch.  The fitted J/K matrices of a
pair-sharded B do have one: the fitted density rho sums over every diagonal
pair before J can be formed, and K^{k1} sums over every k2 (df_jk_sharded).
Host logic only; every rank calls the library on its own shard.
"""
from __future__ import annotations

import numpy as np


def _shell_cost(aux, s):
    """Relative cost of one aux shell in j3c without a plan: Cartesian
    functions x primitives x (1 + l)."""
    l = int(aux.l[s])
    return (l + 1) * (l + 2) // 2 * int(aux.nprim[s]) * (1 + l)


def planner_costs(a, kmesh, ao, aux, **opt):
    """Per aux shell, the SR work the library's host planner assigns it: its
    screened work items (aux shell, AO shell pair, d) times its Cartesian
    functions and primitives.  Host planning only (no device work)."""
    from . import rsgdf
    cost = []
    for s in range(len(aux.l)):
        n = rsgdf.rsgdf_sr_items(a, kmesh, ao, aux, shells=(s, s + 1), features=False, **opt)[0]
        l = int(aux.l[s])
        cost.append(max(1, n) * (l + 1) * (l + 2) // 2 * int(aux.nprim[s]))
    return np.array(cost, dtype=np.float64)


def aux_shell_shards(aux, nranks, cost=None):
    """Contiguous aux-shell ranges [(s0, s1)] per rank, balanced by cost (per
    shell, e.g. planner_costs; default _shell_cost); every shell belongs to
    exactly one range; a range may be empty when there are more ranks than
    shells."""
    ns = len(aux.l)
    if cost is None:
        cost = np.array([_shell_cost(aux, s) for s in range(ns)], dtype=np.float64)
    cost = np.asarray(cost, dtype=np.float64)
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


def pair_shards(npair, nranks):
    """k-pair indices per rank for the DF fit and J/K (equal counts to within
    one, round robin, so diagonal pairs spread over the ranks); every pair
    belongs to exactly one rank."""
    return [list(range(r, npair, nranks)) for r in range(nranks)]


def _sum_over_ranks(dist, x):
    import torch
    if x is None:
        return None
    r = torch.view_as_real(x) if x.is_complex() else x
    dist.all_reduce(r, op=dist.ReduceOp.SUM)
    return x


def df_jk_sharded(dist, rho_fn, jk_fn):
    """Fitted J and K over k pairs split across ranks.  rho_fn() gives this
    rank's fitted density (its diagonal pairs), jk_fn(rho) this rank's J/K
    contributions given the total density; the exchange is one sum of rho
    (naux numbers) before J and one sum of J and K (Nk nao^2 each) after.
    With dist None the local results are returned unchanged."""
    rho = rho_fn()
    if dist is not None:
        rho = _sum_over_ranks(dist, rho)
    J, K = jk_fn(rho)
    if dist is not None:
        J = _sum_over_ranks(dist, J)
        K = _sum_over_ranks(dist, K)
    return J, K
