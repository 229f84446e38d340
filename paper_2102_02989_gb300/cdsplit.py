"""j3c with the compact/diffuse split (Fig. 1 of the paper, Eq. VPmunu_FT).

Both bases are cut at alpha_cut into compact and diffuse sub-shells
(rsgdf_split_basis).  On the split bases the library computes
  * the range-separated route with the SR sums and the G = 0 term restricted to
    (C|cc) and (C|cd) (rsgdf_j3c with split_alpha = alpha_cut), and
  * the plain-kernel reciprocal sum on the same G box (rsgdf_j3c_lr with the
    plain kernel), which the other four types converge on,
and rsgdf_split_combine takes each block from its route and sums the
sub-functions back into the parent functions.  Default alpha_cut = omega^2/2:
a pair of diffuse primitives then has exponent sum <= omega^2, so its transform
has decayed to eps at the edge of the long-range box.  Host orchestration
only; every step runs in the library.
"""
from __future__ import annotations

from types import SimpleNamespace

import numpy as np


def split_bases(ao, aux, alpha_cut):
    from . import rsgdf
    out = []
    for b in (ao, aux):
        d = rsgdf.rsgdf_split_basis(b, alpha_cut)
        out.append(SimpleNamespace(l=d["l"], nprim=d["nprim"], prim_off=d["prim_off"], center=d["center"],
                                   exps=d["exps"], coeffs=d["coeffs"]))
    return out


def j3c_split(a, kmesh, ao, aux, kpairs, alpha_cut=None, stream=None, **opt):
    """V[pair][P][mu][nu] over every aux shell by the split route."""
    import torch
    from . import rsgdf
    if alpha_cut is None:
        w, _ = rsgdf.rsgdf_params(a, kmesh, omega=opt.get("omega"), gmesh=opt.get("gmesh"),
                                  eps_lr=opt.get("eps_lr", 1e-8))
        alpha_cut = 0.5 * w * w
    opt = {k: v for k, v in opt.items() if k not in ("split_alpha", "kernel")}
    sa, sx = split_bases(ao, aux, alpha_cut)
    v_rs = rsgdf.rsgdf_j3c(a, kmesh, sa, sx, kpairs, split_alpha=alpha_cut, stream=stream, **opt)
    v_g = torch.zeros_like(v_rs)
    rsgdf.rsgdf_j3c_lr(a, kmesh, sa, sx, kpairs, out=v_g, kernel=rsgdf.RSGDF_KERNEL_PLAIN, stream=stream, **opt)
    out = rsgdf.rsgdf_split_combine(ao, aux, alpha_cut, v_rs, v_g, stream=stream)
    del v_rs, v_g
    return out
