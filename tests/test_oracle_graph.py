"""Pins of the oracle's graph, partition and halo logic."""
import itertools
import math
import os

import numpy as np

from oracle import graph
from paper_2606_03140_gb300 import inputs as I

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _load_fig1():
    box = r_graph = None
    atoms, cores, halos = [], {}, {}
    for line in open(os.path.join(GOLD, "fig1_two_waters.txt")):
        t = line.split()
        if not t or t[0].startswith("#"):
            continue
        if t[0] == "box":
            box = np.array([float(x) for x in t[1:4]])
        elif t[0] == "r_graph":
            r_graph = float(t[1])
        elif t[0] == "atom":
            atoms.append((int(t[2]), [float(x) for x in t[3:6]]))
        elif t[0] == "core":
            cores[int(t[1])] = [int(x) - 1 for x in t[2:]]
        elif t[0] == "halo":
            halos[int(t[1])] = [int(x) - 1 for x in t[2:]]
    sp = np.array([a[0] for a in atoms], dtype=np.int32)
    R = np.array([a[1] for a in atoms])
    return sp, R, box, r_graph, cores, halos


def test_fig1_worked_example():
    """Paper Fig. 1: cores {1,2,3} and {4,5,6}; halos {4,5} and {3}."""
    sp, R, box, rg, cores_ref, halos_ref = _load_fig1()
    rp, col = graph.build_graph(R, box, rg)
    cores = graph.rcb_partition(R, box, 3)
    assert [list(c) for c in cores] == [cores_ref[1], cores_ref[2]]
    hal = graph.halos(rp, col, cores)
    assert [list(h) for h in hal] == [halos_ref[1], halos_ref[2]]


def _brute_edges(R, box, rg):
    N = len(R)
    E = set()
    for i, j in itertools.product(range(N), range(N)):
        if i == j:
            continue
        d = [R[j][k] - R[i][k] for k in range(3)]
        d = [d[k] - box[k] * round(d[k] / box[k]) for k in range(3)]
        if math.sqrt(sum(x * x for x in d)) < rg:
            E.add((i, j))
    return E


def test_graph_against_brute_force_with_density_edges():
    s = I.small_water_box(8, 7.0, seed=11)
    rp, col = graph.build_graph(s.R, s.box, 2.6)
    E = {(i, int(col[p])) for i in range(s.n_atoms) for p in range(rp[i], rp[i + 1])}
    assert E == _brute_edges(s.R, s.box, 2.6)
    # CSR invariants: symmetric, sorted, no self loops
    for i in range(s.n_atoms):
        c = col[rp[i]:rp[i + 1]]
        assert np.all(np.diff(c) > 0) and i not in c
    # density edges: one directed entry above tau adds both directions
    ptr = np.array([0, 1] + [1] * (s.n_atoms - 1), dtype=np.int64)
    gd = (ptr, np.array([20], dtype=np.int32), np.array([5e-3]))
    rp2, col2 = graph.build_graph(s.R, s.box, 2.6, gd, 1e-3)
    E2 = {(i, int(col2[p])) for i in range(s.n_atoms) for p in range(rp2[i], rp2[i + 1])}
    assert E2 == E | {(0, 20), (20, 0)}
    gd_low = (ptr, np.array([20], dtype=np.int32), np.array([1e-3]))   # not above tau
    rp3, col3 = graph.build_graph(s.R, s.box, 2.6, gd_low, 1e-3)
    assert np.array_equal(col3, col) and np.array_equal(rp3, rp)


def test_rcb_sizes_and_cover():
    s = I.workload("water96")
    for cs in (12, 7, 32, 96):
        cores = graph.rcb_partition(s.R, s.box, cs)
        P = max(1, round(96 / cs))
        assert len(cores) == P
        allat = np.sort(np.concatenate(cores))
        assert np.array_equal(allat, np.arange(96))
        sizes = [len(c) for c in cores]
        assert max(sizes) - min(sizes) <= 1 + 96 // P // 8 + 1


def test_rcb_split_rule_brute_force():
    # first split: widest axis, sort by (coordinate, index), first floor(N*floor(P/2)/P)
    rng = np.random.default_rng(5)
    R = rng.uniform(0, 10, size=(23, 3))
    R[:, 1] *= 2.0                           # y is the widest axis
    R[3, 1] = R[7, 1]                        # a tie broken by atom index
    box = np.array([30.0, 30.0, 30.0])
    cores = graph.rcb_partition(R, box, 23 / 3)
    w = R - box * np.floor(R / box)
    order = sorted(range(23), key=lambda a: (w[a, 1], a))
    left = sorted(order[:(23 * 1) // 3])
    assert list(cores[0]) == left


def test_halo_brute_force():
    s = I.workload("water96")
    rp, col = graph.build_graph(s.R, s.box, 3.0)
    cores = graph.rcb_partition(s.R, s.box, 12)
    hal = graph.halos(rp, col, cores)
    E = _brute_edges(s.R, s.box, 3.0)
    for c, h in zip(cores, hal):
        ref = sorted({j for (i, j) in E if i in set(c)} - set(c))
        assert list(h) == ref


def test_graph_keep_is_union_of_kept_and_rule_edges():
    """SCF graphs keep the edges they had: the graph built with keep= is the set union of the
    kept graph's edges and the rule's own edges (brute force on a small box)."""
    s = I.small_water_box(8, 7.0, seed=12)
    N = s.n_atoms
    rp1, c1 = graph.build_graph(s.R, s.box, 2.2)              # a sparser graph to keep
    shifted = s.R + 0.3 * np.random.default_rng(3).standard_normal(s.R.shape)
    rp2, c2 = graph.build_graph(shifted, s.box, 3.0)          # the rule's edges at another geometry
    rpu, cu = graph.build_graph(shifted, s.box, 3.0, keep=(rp1, c1))
    for i in range(N):
        want = set(c1[rp1[i]:rp1[i + 1]].tolist()) | set(c2[rp2[i]:rp2[i + 1]].tolist())
        got = cu[rpu[i]:rpu[i + 1]].tolist()
        assert got == sorted(want)
    # symmetric
    edges = {(i, int(j)) for i in range(N) for j in cu[rpu[i]:rpu[i + 1]]}
    assert all((j, i) in edges for i, j in edges)


# ---- weighted two-hop graph adaptation (Sec. "Dynamic Graph Adaption", Eq. "Graph_Adaptation") ----

def _gd_of_first_density(s, core_size, seed=3):
    from oracle import density as odn
    from paper_2606_03140_gb300 import inputs as I

    m = I.default_model()
    n = I.random_charges(s.n_atoms, seed, 0.05)
    rp, col = graph.build_graph(s.R, s.box, 3.0)
    cores = graph.rcb_partition(s.R, s.box, core_size)
    r0 = odn.density(s.R, s.species, s.box, m, n, cores, graph.halos(rp, col, cores))
    return m, n, cores, r0


def test_two_hop_products_and_graph_against_dense_matrices():
    """P = G^N G^D and the thresholded, symmetrised graph against dense matrices built by
    brute force: G^N from every pair's minimum-image distance, G^D from the CSR."""
    from paper_2606_03140_gb300 import inputs as I

    s = I.workload("water96")
    _, _, _, r0 = _gd_of_first_density(s, 12)
    alpha, tau = 0.7, 1e-3
    N = s.n_atoms
    rn2 = graph.two_hop_rn2(alpha, tau)
    GN = np.zeros((N, N))
    for i in range(N):
        r2 = graph.min_image_r2(s.R, s.box, i, np.arange(N))
        keep = r2 < rn2
        GN[i, keep] = np.exp(-alpha * r2[keep])
        GN[i, i] = 1.0
    ptr, col, val = r0.gd
    GD = np.zeros((N, N))
    for i in range(N):
        np.add.at(GD[i], col[ptr[i]:ptr[i + 1]], val[ptr[i]:ptr[i + 1]])
    P = GN @ GD
    rows = graph.two_hop_products(s.R, s.box, r0.gd, alpha, tau)
    for i in range(N):
        for j, v in rows[i].items():
            assert abs(v - P[i, j]) <= 1e-13 * max(1.0, abs(P[i, j]))
        assert np.count_nonzero(P[i]) == len(rows[i])
    E = (P > tau) | (P > tau).T
    np.fill_diagonal(E, False)
    rp, cl, amb = graph.build_graph_two_hop(s.R, s.box, r0.gd, alpha, tau)
    assert amb == []
    for i in range(N):
        assert list(cl[rp[i]:rp[i + 1]]) == list(np.nonzero(E[i])[0])
    # every |D| edge above tau is kept (G^N_II = 1), and the rule reaches two hops beyond it
    rp1, cl1 = graph.build_graph(s.R, s.box, 0.0, r0.gd, tau)
    for i in range(N):
        assert set(cl1[rp1[i]:rp1[i + 1]]) <= set(cl[rp[i]:rp[i + 1]])
    assert len(cl) > len(cl1)


def test_two_hop_threshold_controls_accuracy():
    """Sec. "Accuracy Control via Graph Thresholding": with the two-hop graph the band energy and
    the charges approach the single-partition reference as tau falls (monotone, power law)."""
    from oracle import density as odn
    from paper_2606_03140_gb300 import inputs as I

    s = I.small_water_box(60, 13.0, seed=41)
    m, n, cores, r0 = _gd_of_first_density(s, 12, seed=5)
    full_c, full_h = odn.full_partition(s.n_atoms)
    ref = odn.density(s.R, s.species, s.box, m, n, full_c, full_h)
    errs = []
    taus = (3e-2, 1e-2, 3e-3, 1e-3)
    for tau in taus:
        rp, cl, _ = graph.build_graph_two_hop(s.R, s.box, r0.gd, 0.7, tau)
        res = odn.density(s.R, s.species, s.box, m, n, cores, graph.halos(rp, cl, cores))
        errs.append((abs(res.e_band - ref.e_band) / s.n_atoms, float(np.max(np.abs(res.q - ref.q)))))
    e = np.array(errs)
    assert np.all(np.diff(e[:, 0]) < 0) and np.all(np.diff(e[:, 1]) < 0), e
    slope = np.polyfit(np.log(taus), np.log(e[:, 1]), 1)[0]
    assert slope > 0.3, (slope, e)


# ---- core refinement for the 128-orbital tiles ------------------------------------------------

def _refine_case():
    from paper_2606_03140_gb300 import inputs as I

    s = I.small_water_box(300, 21.0, seed=17)
    rp, col = graph.build_graph(s.R, s.box, 3.5)
    cores = graph.rcb_partition(s.R, s.box, 24)
    norb = np.where(s.species == 0, 1, 4)
    return s, rp, col, cores, norb


def test_refine_score_orders_by_padded_tiles_then_size():
    """The score ranks subgraphs by their padded cube cost T^3 (T = 128-orbital tiles) first, and
    within one T by size, so that a move that drops a subgraph below a tile boundary always wins."""
    prev = None
    for n in range(1, 18 * 128 + 1):
        t = (n + 127) // 128
        sc = graph.refine_score(n)
        assert sc // 128000 == t ** 3, n
        if prev is not None:
            assert sc > prev, n
        prev = sc
    # at the boundaries: 128 orbitals fill one tile, 129 need 2 x 2 x 2
    assert graph.refine_score(128) < 2 * 128000 < graph.refine_score(129)


def test_refine_cores_valid_cover_and_score_does_not_rise():
    s, rp, col, cores, norb = _refine_case()
    new, before, after = graph.refine_cores(rp, col, cores, norb, rounds=50, min_core=12)
    assert after <= before
    allat = np.concatenate(new)
    assert np.array_equal(np.sort(allat), np.arange(s.n_atoms))
    assert all(len(c) >= 12 for c in new) and len(new) == len(cores)
    assert all(np.all(np.diff(c) > 0) for c in new)


def test_refine_cores_ends_at_a_local_optimum_brute_force():
    """After convergence no single core-atom move that the rule may make lowers the score."""
    s, rp, col, cores, norb = _refine_case()
    new, before, after = graph.refine_cores(rp, col, cores, norb, rounds=200, min_core=12)
    N = s.n_atoms
    core_of = np.empty(N, dtype=np.int64)
    for c, at in enumerate(new):
        core_of[at] = c

    def orbs(mem):
        halo = set()
        for a in mem:
            for b in col[rp[a]:rp[a + 1]]:
                if int(b) not in mem:
                    halo.add(int(b))
        return int(sum(norb[a] for a in mem) + sum(norb[b] for b in halo))

    mems = [set(int(a) for a in c) for c in new]
    n = [orbs(m) for m in mems]
    assert sum(graph.refine_score(x) for x in n) == after
    for c, m in enumerate(mems):
        if -(-n[c] // 128) == -(-max(n[c] - 48, 1) // 128) or len(m) <= 12:
            continue
        for a in sorted(m):
            for d in sorted({int(core_of[b]) for b in col[rp[a]:rp[a + 1]] if core_of[b] != c}):
                nc = orbs(m - {a})
                nd = orbs(mems[d] | {a})
                delta = (graph.refine_score(nc) + graph.refine_score(nd) - graph.refine_score(n[c])
                         - graph.refine_score(n[d]))
                assert delta >= 0, (c, a, d, delta)
