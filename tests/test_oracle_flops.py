"""Pins of the oracle's instrumented operation counter, the numerator of the
SR kernels' measured roofline (flops per SR primitive term, per class L).

The Hermite recursion count is checked against a closed form derived
independently of the oracle's loops: R^n_{tuv} with s = t + u + v >= 1 and
n = 0..L - s is one multiply when its leading nonzero index is 1 and three
operations (multiply, multiply, add) when it is 2 or more; of the C(s+2, 2)
index triples of level s, exactly s + 1 (s >= 2) or 3 (s = 1) lead with a 1
(t = 1 with any u + v = s - 1; t = 0, u = 1, v = s - 1; and for s = 1 also
(0, 0, 1)).  The worked value for L = 2 is 18: level 1 gives 3 triples x 2
orders x 1, level 2 gives 3 x 1 + 3 x 3."""
import json
import os
from math import comb

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))


def hermite_closed_form(L):
    total = 0
    for s in range(1, L + 1):
        lead1 = 3 if s == 1 else s + 1
        lead2 = comb(s + 2, 2) - lead1
        total += (L - s + 1) * (lead1 * 1 + lead2 * 3)
    return total


def test_hermite_count_closed_form(orc):
    assert hermite_closed_form(2) == 18
    for L in range(10):
        lc = min(L, 3)
        la = min(L - lc, 3)
        c = orc.sr_term_op_counts(lc, la, L - lc - la)
        assert c["hermite"] == hermite_closed_form(L), L


def test_counts_depend_on_class_only_through_L(orc):
    for L in range(10):
        ref = None
        for lc in range(4):
            for la in range(4):
                lb = L - lc - la
                if not 0 <= lb <= 3:
                    continue
                c = orc.sr_term_op_counts(lc, la, lb)
                ref = ref or c
                assert c == ref, (lc, la, lb)


def test_two_boys_evaluations_of_order_L(orc):
    # the erfc auxiliary function F_n(T) - s^{n+1/2} F_n(sT) needs exactly two
    # Boys evaluations of orders 0..L per term, and one G_n per order
    for L in range(10):
        c = orc.sr_term_op_counts(min(L, 3), min(max(L - 3, 0), 3), max(L - 6, 0))
        assert c["boys_calls"] == 2 and c["boys_orders"] == 2 * L
        assert c["seed"] == L + 1


def test_counts_do_not_depend_on_geometry(orc):
    a = orc.sr_term_op_counts(2, 1, 1, omega=0.3, T=0.01)
    b = orc.sr_term_op_counts(2, 1, 1, omega=0.9, T=45.0)
    assert a == b


def test_golden_table_is_the_oracle_count(orc):
    import sys
    sys.path.insert(0, os.path.join(HERE, "golden"))
    import make_sr_flops
    with open(os.path.join(HERE, "golden", "sr_flops_by_L.json")) as f:
        stored = json.load(f)
    fresh = make_sr_flops.table()
    assert stored["flops_per_term_by_L"] == fresh["flops_per_term_by_L"]
    assert stored["counts_by_L"] == fresh["counts_by_L"]
    # flops grow strictly with L (more Hermite integrals and Boys orders)
    fl = stored["flops_per_term_by_L"]
    assert all(fl[i] < fl[i + 1] for i in range(len(fl) - 1))


if __name__ == "__main__":
    pytest.main([__file__, "-q"])
