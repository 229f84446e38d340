"""Test-side restatement of the G-mesh / omega coupling rule (a reading of the
paper's parameter discussion; the paper picks N_PW by hand).  The G box must
contain the sphere |G + k12| <= G_cut for every k12 folded to [-1/2, 1/2) in
fractional coordinates, with G_cut = 2 omega sqrt(-ln eps_lr) the radius beyond
which the kernel factor e^{-q^2/4 omega^2} drops below eps_lr."""
import math

import numpy as np


def gmesh_for(a, omega, eps, kmesh):
    gc = 2 * omega * math.sqrt(-math.log(eps))
    out = []
    for i in range(3):
        la = float(np.linalg.norm(a[i]))
        sh = 0.5 if kmesh[i] > 1 else 0.0
        out.append(2 * math.ceil(gc * la / (2 * math.pi) + sh) + 1)
    return tuple(out)


def omega_for(a, gmesh, eps, kmesh):
    cov = min(2 * math.pi * ((gmesh[i] - 1) / 2 - (0.5 if kmesh[i] > 1 else 0.0)) / float(np.linalg.norm(a[i]))
              for i in range(3))
    return cov / (2 * math.sqrt(-math.log(eps)))


def gmesh_box(a, qmax, kmesh):
    """a box containing |G + k12| <= qmax (route R2)"""
    return tuple(2 * math.ceil(qmax * float(np.linalg.norm(a[i])) / (2 * math.pi) + (0.5 if kmesh[i] > 1 else 0.0)) + 1
                 for i in range(3))
