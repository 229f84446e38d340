"""The multi-rank path on CPU (gloo, world size 2): the aux-shell shards of a
j3c computed independently per rank (here by the oracle, the library's GPU
calls take the same shell ranges) and gathered equal the whole tensor; the
batch partition covers every cell once; the timing reduction takes the
maximum time and the summed units over ranks."""
import numpy as np
import pytest

from paper_2102_02989_gb300 import inputs, shard


def _worker(rank, world, init_file, q):
    import torch.distributed as dist
    import oracle
    # file rendezvous: no port to race for
    dist.init_process_group("gloo", init_method="file://" + init_file, rank=rank, world_size=world)
    p = inputs.tiny(kmesh=(2, 1, 1), lmax_ao=1, lmax_aux=2, natm=2, seed=4)
    kp = inputs.kpairs_all(2)
    s0, s1 = shard.aux_shell_shards(p.aux, world)[rank]
    part, terms = None, 0
    if s1 > s0:
        part, cnt = oracle.j3c(p.a, p.kmesh, p.ao, p.aux, 0.9, kp, eps_sr=1e-12, eps_lr=1e-12, gmesh=(9, 9, 9),
                               shells=(s0, s1), return_counts=True)
        terms = cnt["terms"]
    got = [None] * world
    dist.all_gather_object(got, (s0, s1, part))
    # timing reduction: rank r took 10 + r ms and processed 100 + r units
    tm, units = shard.reduce_timing(dist, [10.0 + rank, 1.0], 100 + rank)
    # the bench's units: SR lattice terms of each rank's shard, summed over ranks
    _, terms_all = shard.reduce_timing(dist, [1.0], terms)
    dist.barrier()
    dist.destroy_process_group()
    if rank == 0:
        q.put((got, tm, units, terms_all))


@pytest.fixture(scope="module")
def orc_built():
    import oracle
    oracle.build()
    return oracle


def test_aux_shards_gather_to_the_whole(orc_built, tmp_path):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    init_file = str(tmp_path / "rendezvous")
    procs = [ctx.Process(target=_worker, args=(r, 2, init_file, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    got, tm, units, terms_all = q.get(timeout=600)
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    p = inputs.tiny(kmesh=(2, 1, 1), lmax_ao=1, lmax_aux=2, natm=2, seed=4)
    kp = inputs.kpairs_all(2)
    full, cnt = orc_built.j3c(p.a, p.kmesh, p.ao, p.aux, 0.9, kp, eps_sr=1e-12, eps_lr=1e-12, gmesh=(9, 9, 9),
                              return_counts=True)
    # the shards' units add up to the whole problem's
    assert terms_all == cnt["terms"] > 0
    parts = sorted(got, key=lambda x: x[0])
    assert parts[0][0] == 0 and parts[-1][1] == len(p.aux.l)
    cat = np.concatenate([x[2] for x in parts if x[2] is not None], axis=1)
    assert cat.shape == full.shape
    assert np.max(np.abs(cat - full)) < 1e-13
    assert tm == [11.0, 1.0] and units == 201.0


def test_shard_partitions():
    p = inputs.config2()
    for n in (1, 2, 3, 8, 40):
        sh = shard.aux_shell_shards(p.aux, n)
        assert len(sh) == n and sh[0][0] == 0 and sh[-1][1] == len(p.aux.l)
        assert all(a[1] == b[0] for a, b in zip(sh, sh[1:]))
        assert all(s0 <= s1 for s0, s1 in sh)
    cells = inputs.config4()
    for n in (1, 2, 4, 8):
        cs = shard.cell_shards(cells, n)
        assert sorted(i for c in cs for i in c) == list(range(len(cells)))
    assert shard.aux_func_offset(p.aux, len(p.aux.l)) == p.aux.nfunc


def _df_worker(rank, world, init_file, q):
    import torch
    import torch.distributed as dist
    from oracle import dfjk
    dist.init_process_group("gloo", init_method="file://" + init_file, rank=rank, world_size=world)
    kmesh = (3, 1, 1)
    J, V, D = inputs.df_synthetic(kmesh, naux=10, nao=4, nocc=2, cond=1e-4, seed=70)
    kp = inputs.kpairs_all(3)
    mine = shard.pair_shards(len(kp), world)[rank]
    T, _, _, _ = dfjk.metric_transforms(J, "auto", rel=1e-10)
    B = dfjk.fit(T, V[mine], kp[mine], kmesh)          # this rank's pairs only

    def rho_fn():
        return torch.from_numpy(dfjk.jk(B, kp[mine], kmesh, D)[2].copy())

    def jk_fn(rho):
        Jm, Km, _ = dfjk.jk(B, kp[mine], kmesh, D, rho=rho.numpy())
        return torch.from_numpy(Jm), torch.from_numpy(Km)
    Jt, Kt = shard.df_jk_sharded(dist, rho_fn, jk_fn)
    dist.barrier()
    dist.destroy_process_group()
    if rank == 0:
        q.put((Jt.numpy(), Kt.numpy()))


def test_df_jk_over_pair_shards_equals_the_whole(orc_built, tmp_path):
    """J/K from pairs split over two ranks (one sum of rho, one of J and K)
    equal J/K from every pair in one process."""
    import torch.multiprocessing as mp
    from oracle import dfjk
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    init_file = str(tmp_path / "rendezvous_df")
    procs = [ctx.Process(target=_df_worker, args=(r, 2, init_file, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    Jt, Kt = q.get(timeout=600)
    for pr in procs:
        pr.join(timeout=120)
        assert pr.exitcode == 0
    kmesh = (3, 1, 1)
    J, V, D = inputs.df_synthetic(kmesh, naux=10, nao=4, nocc=2, cond=1e-4, seed=70)
    kp = inputs.kpairs_all(3)
    T, _, _, _ = dfjk.metric_transforms(J, "auto", rel=1e-10)
    Jo, Ko, _ = dfjk.jk(dfjk.fit(T, V, kp, kmesh), kp, kmesh, D)
    assert np.max(np.abs(Jt - Jo)) < 1e-12 * np.max(np.abs(Jo))
    assert np.max(np.abs(Kt - Ko)) < 1e-12 * np.max(np.abs(Ko))


def test_pair_shards_cover_every_pair_once():
    for npair, world in [(1, 2), (64, 3), (4096, 8), (5, 8)]:
        sh = shard.pair_shards(npair, world)
        flat = sorted(i for s in sh for i in s)
        assert flat == list(range(npair))
        assert max(len(s) for s in sh) - min(len(s) for s in sh) <= 1


def test_j2c_k_shards_cover_the_mesh():
    """The bench's j2c partition: round-robin k points, each exactly once."""
    for nk in (1, 8, 27, 64):
        for world in (1, 2, 3, 8):
            ks = [k for r in range(world) for k in range(r, nk, world)]
            assert sorted(ks) == list(range(nk))
