"""Host-only pieces of bench.py: the DF/spherical oracle timing leg runs on
tensors shaped like the GPU's (numpy, no device) and reports every step."""
import numpy as np

from paper_2102_02989_gb300 import inputs


def test_df_oracle_sample_reports_every_step():
    import bench
    p = inputs.tiny(kmesh=(2, 1, 1), lmax_ao=2, lmax_aux=3, natm=1)
    J, V, D = inputs.df_synthetic((2, 1, 1), naux=p.aux.nfunc, nao=p.ao.nfunc, nocc=2, cond=1e-4, seed=5)
    kp = inputs.kpairs_all(2)
    t, cores = bench.df_oracle_sample(J, V, D, kp, (2, 1, 1), p.ao.l, p.aux.l)
    assert set(t) == {"metric_s", "fit_s", "jk_s", "cart2sph_s"}
    assert all(v >= 0.0 for v in t.values()) and cores >= 1
