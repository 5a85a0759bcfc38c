"""Sharding the subgraph solves over ranks: the native LPT planner (sedacs_shard_lpt, host only)
and the exchange a sharded step needs, modelled with the FP64 oracle on two gloo ranks (CPU).

The planner is checked against what fixes it: Graham's bound 4/3 - 1/(3m) against the optimum by
brute force on small instances, its tie rules, its loads, and on the 9,000-atom water subgraphs.
The exchange model: each rank solves its LPT share of the subgraphs; every bisection step on mu
sums the ranks' collected counts (Eq. 2 over all subgraphs); the charges and band energy of the
owned cores are summed over ranks.  The result must equal the single-process oracle's.
"""
import itertools
import math
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _lpt(cost, m):
    from paper_2606_03140_gb300 import sedacs as S

    return S.sedacs_shard_lpt(np.asarray(cost, dtype=np.float64), m)


def test_lpt_within_graham_bound_of_brute_force_optimum():
    rng = np.random.default_rng(11)
    for trial in range(60):
        m = int(rng.integers(2, 4))
        k = int(rng.integers(1, 9))
        cost = rng.integers(1, 40, size=k).astype(np.float64) ** 3
        owner, load = _lpt(cost, m)
        assert owner.shape == (k,) and np.all((owner >= 0) & (owner < m))
        assert np.allclose(load, [cost[owner == r].sum() for r in range(m)], rtol=0, atol=0)
        best = min(max(sum(cost[i] for i in range(k) if a[i] == r) for r in range(m))
                   for a in itertools.product(range(m), repeat=k))
        assert best <= load.max() <= (4.0 / 3.0 - 1.0 / (3 * m)) * best * (1 + 1e-12), (cost, m)


def test_lpt_order_and_ties():
    # equal costs: ascending index, each to the least-loaded rank, ties to the lowest rank
    owner, load = _lpt([1.0] * 7, 3)
    assert list(owner) == [0, 1, 2, 0, 1, 2, 0] and list(load) == [3.0, 2.0, 2.0]
    # descending cost first: 5 -> r0, 4 -> r1, 3 -> r1 (4 < 5), 3 -> r0 ... loads 5+3, 4+3
    owner, load = _lpt([3.0, 5.0, 3.0, 4.0], 2)
    assert list(owner) == [1, 0, 0, 1] and list(load) == [8.0, 7.0]
    owner, load = _lpt([2.0, 1.0], 1)
    assert list(owner) == [0, 0] and list(load) == [3.0]
    owner, load = _lpt([], 4)
    assert owner.shape == (0,) and list(load) == [0.0] * 4


@pytest.mark.parametrize("cost,m", [([1.0, -1.0], 2), ([1.0, float("nan")], 2), ([1.0], 0)])
def test_lpt_rejects_bad_input(cost, m):
    from paper_2606_03140_gb300 import sedacs as S

    with pytest.raises(S.SedacsError):
        _lpt(cost, m)


def test_lpt_on_the_water9000_subgraphs():
    """Costs n_i^3 of the 281 subgraphs of the 9,000-atom box (distance graph, RCB cores of ~32
    atoms, one-hop halos): the largest rank load stays within 2 % of the mean up to 8 ranks (the
    paper reports an imbalance of 1.37 for its own assignment)."""
    from oracle import graph as og
    from paper_2606_03140_gb300 import inputs as I

    s = I.workload("water9000")
    m = I.default_model()
    rp, col = og.build_graph(s.R, s.box, 3.0)
    cores = og.rcb_partition(s.R, s.box, 32)
    halos = og.halos(rp, col, cores)
    norb = np.asarray(m.n_orb)[s.species]
    n = np.array([norb[c].sum() + norb[h].sum() for c, h in zip(cores, halos)], dtype=np.float64)
    for ranks in (2, 4, 8):
        owner, load = _lpt(n ** 3, ranks)
        assert load.max() / load.mean() < 1.02, (ranks, load.max() / load.mean())
        assert abs(load.sum() - np.sum(n ** 3)) <= 1e-9 * np.sum(n ** 3)


# ---- the exchange of a sharded step, modelled with the oracle on two gloo ranks -----------------

def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as sk:
        sk.bind(("127.0.0.1", 0))
        return sk.getsockname()[1]


def _system():
    from oracle import ewald
    from oracle import graph as og
    from paper_2606_03140_gb300 import inputs as I

    s = I.small_water_box(100, 14.5, seed=21)
    m = I.default_model()
    n = I.random_charges(s.n_atoms, 5, 0.05)
    rp, col = og.build_graph(s.R, s.box, 3.0)
    cores = og.rcb_partition(s.R, s.box, 12)
    halos = og.halos(rp, col, cores)
    V = ewald.coulomb_potential(s.R, s.species, m.hubbard_u, s.box, n)
    return s, m, n, cores, halos, V


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist

    from oracle import KB_HA
    from oracle import density as odn
    from paper_2606_03140_gb300 import sedacs as S

    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        s, m, n, cores, halos, V = _system()
        norb = np.asarray(m.n_orb)[s.species]
        size = np.array([norb[c].sum() + norb[h].sum() for c, h in zip(cores, halos)], dtype=np.float64)
        owner, _ = S.sedacs_shard_lpt(size ** 3, world)
        mine = [i for i in range(len(cores)) if owner[i] == rank]
        atoms = [np.concatenate([cores[i], halos[i]]).astype(np.int64) for i in mine]
        subs = odn.subgraph_setup_all(atoms, [len(cores[i]) for i in mine], s.R, s.species, s.box, m, V)
        beta = 1.0 / (KB_HA * 300.0)
        n_e = float(np.sum(np.asarray(m.z_val)[s.species]))

        def allsum(x):
            t = torch.tensor(np.atleast_1d(np.asarray(x, dtype=np.float64)))
            dist.all_reduce(t, op=dist.ReduceOp.SUM)
            return t.numpy()

        # Eq. 2 over all subgraphs: one allreduce of the local collected count per bisection step
        eps = [sg.eps for sg in subs]
        w = [sg.w for sg in subs]
        # the oracle's bracket [min eps - 1, max eps + 1] over all subgraphs
        bounds = np.array([min((float(e.min()) for e in eps), default=math.inf),
                           -max((float(e.max()) for e in eps), default=-math.inf)])
        t = torch.tensor(bounds)
        dist.all_reduce(t, op=dist.ReduceOp.MIN)
        lo, hi = float(t[0]) - 1.0, -float(t[1]) + 1.0
        mu = 0.5 * (lo + hi)
        for _ in range(400):
            mu = 0.5 * (lo + hi)
            nel = float(allsum(odn.collected_count(eps, w, mu, beta))[0])
            if abs(nel - n_e) < 1e-11 or hi - lo < 1e-15:
                break
            if nel < n_e:
                lo = mu
            else:
                hi = mu
        res = odn.density(s.R, s.species, s.box, m, n, [cores[i] for i in mine], [halos[i] for i in mine],
                          mu=mu, V=V)
        q = allsum(res.q)
        eb = float(allsum(res.e_band)[0])
        out[rank] = (mu, q, eb, len(mine))
    finally:
        dist.destroy_process_group()


def test_sharded_step_exchange_matches_single_process_oracle():
    mp = pytest.importorskip("torch.multiprocessing")
    from oracle import density as odn

    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:       # no fork of a threaded test process
        out = mgr.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    s, m, n, cores, halos, V = _system()
    ref = odn.density(s.R, s.species, s.box, m, n, cores, halos, V=V)
    (mu0, q0, eb0, k0), (mu1, q1, eb1, k1) = res[0], res[1]
    assert k0 > 0 and k1 > 0 and k0 + k1 == len(cores)
    assert mu0 == mu1 and np.array_equal(q0, q1) and eb0 == eb1       # every rank holds the same result
    assert abs(mu0 - ref.mu) < 1e-12
    assert np.max(np.abs(q0 - ref.q)) < 1e-10
    assert abs(eb0 - ref.e_band) < 1e-9
