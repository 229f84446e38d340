"""Host-only pieces of bench.py: a static check that every name a function
uses is defined, the guard that keeps a failing extra section from costing
the headline line, the roofline arithmetic on synthetic statistics, and the
DF/spherical oracle timing leg on tensors shaped like the GPU's."""
import builtins
import os
import symtable

import numpy as np

from paper_2102_02989_gb300 import inputs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def undefined_names(path):
    """(function, name) pairs for names a function reads that are bound in no
    enclosing scope, at module level, or among the builtins."""
    src = open(path).read()
    top = symtable.symtable(src, path, "exec")
    module = {s.get_name() for s in top.get_symbols() if s.is_assigned() or s.is_imported()}
    module |= {c.get_name() for c in top.get_children()}
    bad = []

    def walk(t):
        for ch in t.get_children():
            if ch.get_type() == "function":
                for s in ch.get_symbols():
                    n = s.get_name()
                    if s.is_referenced() and s.is_global() and n not in module and not hasattr(builtins, n):
                        bad.append((ch.get_name(), n))
            walk(ch)
    walk(top)
    return bad


def test_bench_uses_no_undefined_name():
    assert undefined_names(os.path.join(ROOT, "bench.py")) == []


def test_static_check_catches_an_undefined_name(tmp_path):
    f = tmp_path / "m.py"
    f.write_text("def f(x):\n    if cpu_baseline:\n        return x\n    return len(x)\n")
    assert undefined_names(str(f)) == [("f", "cpu_baseline")]


def test_guard_records_a_failing_section():
    import bench
    line = {"value": 1.0}

    def bad():
        raise NameError("name 'cpu_baseline' is not defined")
    bench.guarded(line, "extra", bad)
    bench.guarded(line, "ok", lambda: {"x": 1})
    assert line["value"] == 1.0 and "NameError" in line["extra"]["error"]
    assert line["ok"]["x"] == 1


def test_roofline_numerator_from_the_oracle_table():
    import argparse
    import bench
    table = bench.sr_flops_table()
    fl = table["flops_per_term_by_L"]
    z = bench._stats0(None)
    s3 = dict(z, sr_ms=2.0, aft_ms=0.5, lr_gemm_ms=0.25, phase_ms=0.25, other_ms=0.1, lr_flops=10 ** 9,
              sr_prim_terms_by_L=[0, 0, 10 ** 6, 0, 0, 2 * 10 ** 6, 0, 0, 0, 0])
    s2 = dict(z, sr_ms=1.0, sr_prim_terms_by_L=[10 ** 6] + [0] * 9)
    args = argparse.Namespace(kmesh="2,2,2", path="learned-mixed")
    r = bench.roofline([(s2, s3), (s2, s3)], args, peak_fp64=1.25)
    want = (10 ** 6 * fl[2] + 2 * 10 ** 6 * fl[5] + 10 ** 6 * fl[0]) / 3e-3 / 1e12
    assert r["bound"] == "alu" and r["kernel"].startswith("k_sr3c")
    assert abs(r["achieved"] - want) < 1e-12 and abs(r["frac"] - want / 1.25) < 1e-12
    assert r["phases_ms"]["sr_ms"] == 3.0


def test_df_oracle_sample_reports_every_step():
    import bench
    p = inputs.tiny(kmesh=(2, 1, 1), lmax_ao=2, lmax_aux=3, natm=1)
    J, V, D = inputs.df_synthetic((2, 1, 1), naux=p.aux.nfunc, nao=p.ao.nfunc, nocc=2, cond=1e-4, seed=5)
    kp = inputs.kpairs_all(2)
    t, cores = bench.df_oracle_sample(J, V, D, kp, (2, 1, 1), p.ao.l, p.aux.l)
    assert set(t) == {"metric_s", "fit_s", "jk_s", "cart2sph_s"}
    assert all(v >= 0.0 for v in t.values()) and cores >= 1
