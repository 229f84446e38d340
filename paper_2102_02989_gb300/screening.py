"""Learned screening driver: training data from the FP64 SR kernels'
magnitude mode, training with the library's kernels, margin calibration and
use in j3c.  Host orchestration only; every numerical step runs in the CUDA
library (features, magnitudes, forward, backward, Adam, masking).

Model: the network learns the correction to the s-type estimate carried as
feature ``BASE`` (log10 of the SR integral of the nearest term, exact for s
shells) times the image sum of the diffuse s-type kernel within the
screening radius.  Targets and that estimate are clamped to the decision window
[k - 5, k + 1] around the keep level k = log10(eps) - ``drop``: outside it
only the side of the cut matters.
Item magnitudes are not a smooth function of the features (symmetric images
cancel for odd angular momentum, to a depth set by rounding and truncation),
so the network is fitted to an upper expectile (tau = 0.99) of the targets
rather than their mean.  Screening prediction = clamp(est) + network(x).

Policy: the library skips an item when its prediction plus the margin is
below cut = log10(eps) - 1 and, as a guard against extrapolation, the
estimate itself plus its own calibrated margin for the item's class
L = lP + lmu + lnu (the guard, the largest cut - estimate over all training
items of that class with magnitude >= eps 10^-drop, plus ``safety``) is
below the cut too; a class with training items but fewer than ``min_class``
at that level takes the largest calibrated guard (a guard calibrated on a
handful of items says little), and a class absent from the training data is
never skipped.  The margin is calibrated on held-out items that
must be kept (magnitude >= eps 10^-drop; many skipped items can land in one
output element, so the per-item budget sits well below eps): the largest
shortfall cut - prediction among them plus ``safety`` decades (zero if
negative), so no held-out item of that magnitude or more is skipped.
"""
from __future__ import annotations

import numpy as np

from . import rsgdf


def items_dataset(problems, eps_screen=1e-8):
    """Features and log10 magnitudes of every SR work item of the problems
    (each a (cell a, kmesh, ao, aux, omega, gmesh, eps_lr) tuple)."""
    import torch
    Xs, ts = [], []
    for (a, km, ao, aux, omega, gmesh, eps_lr) in problems:
        n, feat, mag = rsgdf.rsgdf_sr_items(a, km, ao, aux, features=True, magnitudes=True, omega=omega, gmesh=gmesh,
                                            eps_screen=eps_screen, eps_lr=eps_lr)
        if n:
            Xs.append(feat)
            ts.append(mag)
    torch.cuda.synchronize()
    return torch.cat(Xs), torch.cat(ts)


BASE = 8


def train_screen(X, t, epochs=40, batch=2048, lr=2e-3, tau=0.99, seed=0, holdout=0.2, safety=0.5, eps_screen=1e-8,
                 drop=2.0, min_class=50):
    """Train the network on (X, t) and calibrate its margin on a held-out part."""
    import torch
    # data preparation and calibration statistics on host copies (torch only moves memory)
    Xh = X.cpu().numpy()
    traw = t.cpu().numpy()
    le = float(np.log10(eps_screen))
    k = le - drop
    lo, hi = k - 5.0, k + 1.0
    th = np.clip(traw, lo, hi).astype(np.float32)
    base = np.clip(Xh[:, BASE], lo, hi).astype(np.float32)
    n = Xh.shape[0]
    perm = np.random.default_rng(seed).permutation(n)
    nh = max(1, int(holdout * n))
    hv, tr = perm[:nh], perm[nh:]
    mean = Xh[tr].astype(np.float64).mean(0).astype(np.float32)
    std = (Xh[tr].astype(np.float64).std(0) + 1e-3).astype(np.float32)
    dev = X.device
    Xt = torch.tensor(Xh[tr], device=dev)
    tt = torch.tensor(th[tr] - base[tr], device=dev)
    Xv = torch.tensor(Xh[hv], device=dev)
    from .mlp_init import init_params
    m = rsgdf.Mlp(init_params(Xh.shape[1], seed), mean, std)
    cut = le - 1.0
    # guard: the physical estimate alone, calibrated on every item (it has no
    # fitted parameters): no item of magnitude >= k may have est + guard < cut
    # per class L = lP + lmu + lnu; a class without training items is never skipped
    keep_all = traw >= k
    Lc = np.rint(Xh[:, 0] + Xh[:, 1] + Xh[:, 2]).astype(int)
    guard = np.full(10, np.inf, np.float32)
    calibrated = []
    for L in range(10):
        kk = keep_all & (Lc == L)
        if kk.sum() >= min_class:
            guard[L] = float((cut - Xh[kk, BASE]).max()) + safety
            calibrated.append(guard[L])
    # a class seen in training with too few items at the keep level takes the
    # most conservative calibrated guard; a class never seen is never skipped (inf)
    for L in range(10):
        if not np.isfinite(guard[L]) and (Lc == L).any() and calibrated:
            guard[L] = max(calibrated)
    m.set_base(BASE, lo, hi, guard)
    loss = m.train(Xt, tt, epochs=epochs, batch=batch, lr=lr, tau=tau, seed=seed)
    pv = m.forward(Xv).cpu().numpy() + base[hv]
    keep = traw[hv] >= k
    short = float((cut - pv[keep]).max()) if keep.any() else -np.inf
    margin = max(0.0, short + safety)
    m.set_margin(margin)
    allowed = Xh[hv, BASE] + guard[Lc[hv]] < cut
    r = th[hv] - pv
    return m, {"train_loss": loss, "holdout_rmse": float(np.sqrt(np.mean(r * r))), "max_shortfall": short,
               "margin": margin, "guard": [round(float(g), 3) if np.isfinite(g) else None for g in guard], "holdout_pruned": float(np.mean((pv + margin < cut) & allowed)),
               "holdout_ideal": float(np.mean(traw[hv] < k)), "n_train": int(n - nh), "n_holdout": int(nh)}
