"""Two pieces of the SR kernel's work split, emulated on the CPU.

1. Lanes over BvK cells: a chunk's translations are sorted by cell; cell b with
   n_b translations gets k_b = ceil(n_b / R) of the Lg lanes of a combination
   group, R the fewest rounds with sum_b ceil(n_b / R) <= Lg (a binary search
   over R); lane j of cell b takes translations b_start + j, + k_b, ...  Every
   translation must be taken exactly once, no lane more than R times, and R
   must be minimal.
2. Candidate radius from the screening windows: the exact test keeps a
   translation at distance Rc <= Rc_cut only if win[min(floor(Rc / DR), nwin - 1)]
   admits the pair's R12.  With wlast the last window that admits it, the
   candidates need only reach (wlast + 1) DR, unless wlast is the open-ended
   last window (then Rc_cut).  Every distance the full test keeps must lie
   within that radius."""
import math

import numpy as np


def lane_split(counts, lanes):
    nz = sum(1 for c in counts if c > 0)
    if nz > lanes:
        return None
    lo, hi = 1, max(counts)
    while lo < hi:
        mid = (lo + hi) // 2
        if sum((c + mid - 1) // mid for c in counts) <= lanes:
            hi = mid
        else:
            lo = mid + 1
    R = lo
    k = [(c + R - 1) // R for c in counts]
    start = np.concatenate([[0], np.cumsum(counts)])
    taken = np.zeros(int(start[-1]), int)
    per_lane = []
    ls = 0
    for b, kb in enumerate(k):
        for j in range(kb):
            idx = list(range(int(start[b]) + j, int(start[b + 1]), kb))
            taken[idx] += 1
            per_lane.append(len(idx))
        ls += kb
    assert ls <= lanes
    return R, taken, per_lane


def test_lane_split_covers_every_translation_once():
    rng = np.random.default_rng(3)
    for _ in range(3000):
        nb = int(rng.integers(1, 17))
        counts = [int(x) for x in rng.poisson(rng.uniform(0.3, 30), size=nb)]
        if sum(counts) == 0:
            continue
        for lanes in (32, 16, 8):
            out = lane_split(counts, lanes)
            if out is None:
                assert sum(1 for c in counts if c > 0) > lanes
                continue
            R, taken, per_lane = out
            assert np.all(taken == 1)
            assert max(per_lane) <= R
            if R > 1:   # one round fewer would need more lanes
                assert sum((c + R - 2) // (R - 1) for c in counts) > lanes


def kernel_radius(win, R12, rc_cut, dr):
    nwin = len(win)
    wlast = -1
    for w in range(nwin - 1, -1, -1):
        if R12 <= win[w]:
            wlast = w
            break
    if wlast < 0:
        return None
    return rc_cut if wlast == nwin - 1 else min(rc_cut, (wlast + 1) * dr)


def test_window_radius_keeps_every_accepted_translation():
    rng = np.random.default_rng(4)
    dr = 1.0
    for _ in range(4000):
        rc_cut = float(rng.uniform(0.5, 30.0))
        nwin = int(math.floor(rc_cut / dr)) + 1
        if rng.random() < 0.2:
            win = [1e300]                                   # a triple without windows
            nwin = 1
        else:
            win = list(rng.uniform(0.0, 12.0, size=nwin))  # not monotone in general
        R12 = float(rng.uniform(0.0, 12.0))
        rad = kernel_radius(win, R12, rc_cut, dr)
        for rc in rng.uniform(0.0, rc_cut, size=64):
            w = min(int(math.floor(rc / dr)), nwin - 1)
            if R12 <= win[w]:
                assert rad is not None and rc <= rad, (win, R12, rc_cut, rc, rad)
