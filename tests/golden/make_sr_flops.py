"""Writes ``sr_flops_by_L.json``: the FP64 flops of one SR primitive term per
total angular momentum L = lP + lmu + lnu (0..9), as tallied by the oracle's
instrumented operation counter while it evaluates the erfc-kernel integral
(Eq. VPmunu_SR through the auxiliary function G_n and the McMurchie-Davidson
Hermite integrals R_tuv).  The per-term work depends on the class only
through L (checked for every split in tests/test_oracle_flops.py).

The measured roofline of the SR lattice-sum kernels takes its numerator from
this table: flops(L) x the primitive-combination terms evaluated per class.

    python tests/golden/make_sr_flops.py
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402

LTOT = 9


def split(L):
    """One (lP, lmu, lnu) with lP, lmu, lnu <= 3 summing to L."""
    lc = min(L, 3)
    la = min(L - lc, 3)
    return lc, la, L - lc - la


def table():
    counts = [oracle.sr_term_op_counts(*split(L)) for L in range(LTOT + 1)]
    return {
        "flops_per_term_by_L": [oracle.sr_term_flops(*split(L)) for L in range(LTOT + 1)],
        "counts_by_L": counts,
        "boys_convention": {"base_flops": oracle.BOYS_BASE_FLOPS, "step_flops": oracle.BOYS_STEP_FLOPS},
        "unit": "FP64 flops per SR term (one primitive combination at one lattice translation), an FMA "
                "counting 2; the per-term part only: separation and T, two Boys evaluations (by the "
                "convention), the erfc combination, the Hermite seeds and recursion",
        "source": "oracle/rsgdf_oracle.c instrumented counter (or_flops_begin/or_flops_end) via "
                  "oracle.sr_term_op_counts",
    }


if __name__ == "__main__":
    with open(os.path.join(HERE, "sr_flops_by_L.json"), "w") as f:
        json.dump(table(), f, indent=1)
        f.write("\n")
