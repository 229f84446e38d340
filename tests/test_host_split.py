"""Host-side compact/diffuse split (rsgdf_split_basis, rsgdf_sr_items_split;
no device work): the library's split equals the oracle's (oracle/split.py, an
independent restatement: sub-shell structure, kinds, parents and weights), and
the planner's count of range-separated work equals the sum, over compact aux
sub-shells, of the items with every AO sub-shell pair minus those with pairs of
diffuse sub-shells only."""
import numpy as np
import pytest

from oracle import split
from paper_2102_02989_gb300 import inputs

A = 4.0 * np.eye(3)
C1, C2 = np.zeros(3), np.array([1.7, 2.1, 1.9])
KM = (2, 1, 1)
W = 0.9


@pytest.fixture(scope="module")
def rs():
    from paper_2102_02989_gb300 import rsgdf
    rsgdf.load()
    return rsgdf


def _bases():
    ao = inputs.make_basis([(0, C1, [3.0, 0.3], [0.6, 0.5]), (1, C1, [0.25], [1.0]), (0, C2, [12.0], [1.0]),
                            (0, C2, [0.7], [1.0]), (1, C1, [0.75], [1.0]), (1, C2, [2.2, 0.35], [0.7, 0.4]),
                            (2, C2, [4.0, 1.1, 0.2], [0.3, 0.5, 0.4])])
    aux = inputs.make_basis([(0, C1, [25.0], [1.0]), (0, C1, [0.3], [1.0]), (1, C2, [0.5], [1.0]),
                             (2, C2, [0.2], [1.0]), (2, C1, [1.2, 0.25], [1.0, 0.6])])
    return ao, aux


def _as_basis(d, keep=None):
    keep = range(len(d["l"])) if keep is None else keep
    shells = []
    for s in keep:
        o, n = int(d["prim_off"][s]), int(d["nprim"][s])
        shells.append((int(d["l"][s]), d["center"][s], list(d["exps"][o:o + n]), list(d["coeffs"][o:o + n])))
    return inputs.make_basis(shells)


@pytest.mark.parametrize("acut", [0.405, 1.0, 0.1])
def test_split_matches_the_oracle(rs, orc, acut):
    for b in _bases():
        got = rs.rsgdf_split_basis(b, acut)
        sb, R, kind = split.split_basis(b, acut)
        assert list(got["l"]) == list(sb.l) and list(got["nprim"]) == list(sb.nprim)
        assert np.array_equal(got["exps"], sb.exps) and np.array_equal(got["coeffs"], sb.coeffs)
        nc = lambda l: (int(l) + 1) * (int(l) + 2) // 2
        f0 = np.concatenate([[0], np.cumsum([nc(l) for l in sb.l])]).astype(int)
        for s in range(len(sb.l)):
            assert "cd"[got["kind"][s]] == kind[f0[s]]
            parent_f = int(np.nonzero(R[:, f0[s]])[0][0])
            pf0 = np.concatenate([[0], np.cumsum([nc(l) for l in b.l])]).astype(int)
            assert pf0[got["parent"][s]] == parent_f
            assert abs(got["weight"][s] - R[parent_f, f0[s]]) < 1e-13 * abs(R[parent_f, f0[s]])


def test_range_separated_work_count_is_additive(rs):
    ao, aux = _bases()
    acut = 0.405
    opt = dict(omega=W, gmesh=(9, 9, 9), eps_screen=1e-8, eps_lr=1e-8)
    r = rs.rsgdf_split_basis(ao, acut), rs.rsgdf_split_basis(aux, acut)
    sa, sx = _as_basis(r[0]), _as_basis(r[1])
    dd = _as_basis(r[0], [s for s in range(len(r[0]["l"])) if r[0]["kind"][s] == 1])
    got = rs.rsgdf_sr_items_split(A, KM, ao, aux, acut, **opt)
    items = lambda a, x, sh=None: rs.rsgdf_sr_items(A, KM, a, x, shells=sh, features=False, **opt)[0]
    assert got["items"][0] == items(ao, aux)
    assert got["items"][1] == items(sa, sx)
    want = sum(items(sa, sx, (s, s + 1)) - items(dd, sx, (s, s + 1))
               for s in range(len(r[1]["l"])) if r[1]["kind"][s] == 0)
    assert got["items"][2] == want
    assert got["terms"][2] < got["terms"][1]
