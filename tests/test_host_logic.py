"""Host-side rules that are not integrals: k-difference counting (Table S1) and
the omega / G-mesh coupling."""
import numpy as np
import pytest

from rules_ref import gmesh_for, omega_for


@pytest.mark.parametrize("n,count", [(1, 1), (2, 14), (3, 63), (4, 172), (5, 365)])
def test_table_s1_unique_k12_counts(n, count):
    """Table S1 prints N_k12 = 1, 14, 63, 172, 365 for N_k = 1^3..5^3: the raw
    differences k2 - k1 of an N^3 mesh (not folded by G), identified with their
    inverses."""
    ks = np.array([(i, j, k) for i in range(n) for j in range(n) for k in range(n)])
    diffs = {tuple(b - a) for a in ks for b in ks}
    canon = {max(d, tuple(-x for x in d)) for d in diffs}
    assert len(canon) == count
    assert count == ((2 * n - 1) ** 3 + 1) // 2


def test_omega_gmesh_rule_roundtrip():
    a = 0.5 * 6.74 * np.array([[0, 1, 1], [1, 0, 1], [1, 1, 0.0]])
    for km in ((1, 1, 1), (2, 2, 2), (4, 4, 4)):
        for eps in (1e-8, 1e-10):
            w = omega_for(a, (7, 7, 7), eps, km)
            assert gmesh_for(a, w * (1 - 1e-12), eps, km) == (7, 7, 7)
            assert gmesh_for(a, w * 1.05, eps, km)[0] > 7
