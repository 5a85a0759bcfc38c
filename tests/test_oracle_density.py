"""Pins of the oracle's subgraph solve, chemical potential, charges, energy and forces."""
import math

import numpy as np
import pytest

from oracle import KB_HA

from oracle import density as dn
from oracle import dynamics as dyn
from oracle import graph
from paper_2606_03140_gb300 import inputs as I


@pytest.fixture(scope="module")
def w96():
    return I.workload("water96"), I.default_model(), I.random_charges(96, 3, 0.05)


@pytest.fixture(scope="module")
def full96(w96):
    s, m, n = w96
    cores, hal = dn.full_partition(96)
    return dn.density(s.R, s.species, s.box, m, n, cores, hal)


def test_inverse_square_root_overlap(full96):
    sg = full96.subs[0]
    assert np.max(np.abs(sg.Z @ sg.S @ sg.Z - np.eye(sg.S.shape[0]))) < 1e-13


def test_full_limit_idempotency_trace_neutrality(full96):
    sg = full96.subs[0]
    D, S = sg.D_rows, sg.S
    assert np.max(np.abs(D @ S @ D - 2 * D)) < 1e-12
    assert abs(np.trace(D @ S) - 256.0) < 1e-10
    assert abs(full96.q.sum()) < 1e-10
    # [h~, P] = 0 for the orthogonalised projector
    P = 0.5 * np.linalg.solve(sg.Z, np.linalg.solve(sg.Z, D.T).T)
    Ht = sg.Z @ sg.H @ sg.Z
    assert np.max(np.abs(Ht @ P - P @ Ht)) < 1e-11


def test_mu_full_limit_in_gap_and_count(full96):
    """Eq. 2 in the full limit: N(mu) = N_e and mu lies in the HOMO-LUMO gap."""
    e = np.concatenate([sg.eps for sg in full96.subs])
    occ = np.sort(e)[127], np.sort(e)[128]
    assert occ[0] < full96.mu < occ[1]
    assert abs(full96.n_electrons - 256.0) < 1e-9


@pytest.fixture(scope="module")
def trunc96(w96):
    s, m, n = w96
    cores = graph.rcb_partition(s.R, s.box, 12)
    r0 = dn.density(s.R, s.species, s.box, m, n, cores, graph.halos(*graph.build_graph(s.R, s.box, 3.0), cores))
    rp, col = graph.build_graph(s.R, s.box, 3.0, r0.gd, 1e-3)
    return dn.density(s.R, s.species, s.box, m, n, cores, graph.halos(rp, col, cores)), cores, (rp, col)


def test_mu_truncated_graph_brute_force_scan(trunc96):
    """Eq. 2 on a truncated graph: a brute-force scan of the collected Fermi count (explicit
    loops over states) crosses N_e in the grid cell that holds mu, and the charges sum to
    neutrality although the T -> 0 count at mu misses N_e."""
    r, _, _ = trunc96
    beta = 1.0 / (KB_HA * 300.0)
    states = [(float(e), float(w)) for sg in r.subs for e, w in zip(sg.eps, sg.w)]

    def count(mu):
        tot = 0.0
        for e, w in states:
            x = beta * (e - mu)
            tot += 2.0 * w * (1.0 / (1.0 + math.exp(x)) if x < 700 else 0.0)
        return tot

    grid = np.linspace(r.mu - 0.02, r.mu + 0.02, 81)
    c = np.array([count(g) for g in grid])
    assert np.all(np.diff(c) >= -1e-12)
    k = int(np.searchsorted(c, 256.0))
    assert 0 < k < len(grid) and grid[k - 1] <= r.mu <= grid[k]
    assert abs(count(r.mu) - 256.0) < 1e-9
    assert abs(r.q.sum()) < 1e-9
    assert abs(r.t0_miss) > 1e-6          # the truncation miss the Fermi tails absorb


def test_density_graph_block_maxima_explicit_loop(trunc96):
    """G^D_IJ = max |D_mu nu| over the orbital block of core atom I and subgraph atom J."""
    r, _, _ = trunc96
    ptr, col, val = r.gd
    for sg in r.subs[:3]:
        for a in range(sg.n_core):
            I_ = int(sg.atoms[a])
            got = dict(zip(col[ptr[I_]:ptr[I_ + 1]].tolist(), val[ptr[I_]:ptr[I_ + 1]].tolist()))
            for b, J in enumerate(sg.atoms):
                best = 0.0
                for mu_ in range(int(sg.off[a]), int(sg.off[a + 1])):
                    for nu in range(int(sg.off[b]), int(sg.off[b + 1])):
                        best = max(best, abs(float(sg.D_rows[mu_, nu])))
                assert got[int(J)] == best


def test_entropy_free_energy_identity():
    """Per level: f eps - T s = -kT ln(1 + exp(-beta (eps - mu))) + mu f (grand potential
    plus mu N), with s = -k_B [f ln f + (1 - f) ln(1 - f)]; s(1/2) = k_B ln 2."""
    beta = 1.0 / (KB_HA * 300.0)
    mu = -0.31
    eps = np.array([-0.35, -0.32, -0.311, -0.31, -0.305, -0.2, 0.4])
    f = dn.fermi(eps - mu, beta)
    lhs = f * eps - dn.entropy_density(f) / beta
    rhs = -np.logaddexp(0.0, -beta * (eps - mu)) / beta + mu * f
    assert np.max(np.abs(lhs - rhs)) < 1e-15
    assert abs(dn.entropy_density(np.array([0.5]))[0] - math.log(2.0)) < 1e-15
    assert dn.entropy_density(np.array([0.0, 1.0])).tolist() == [0.0, 0.0]


def test_sp2_noise_floor_stop_rule():
    """SP2 stop rules: the idempotency tolerance, and the finite-precision rule of Kruchinina,
    Rudberg and Rubensson (2016): stop at the first step k >= 4 whose error t_k has not fallen
    below t_{k-2} once t_{k-2} < 1e-4 n."""
    # clean gap: stops on the tolerance, result is the step function
    x = np.array([0.05, 0.3, 0.45, 0.55, 0.7, 0.95])
    occ, k = dn.sp2_mu_occupations(x, 0.5, 6, tol=1e-9)
    assert np.allclose(occ, [0, 0, 0, 1, 1, 1], atol=1e-8) and k < 30
    # a level sitting at the image of mu never converges: the error stays at 1/4 per level
    # (never below 1e-4 n), so only kmax stops it
    occ, k = dn.sp2_mu_occupations(np.array([0.2, 0.5, 0.8]), 0.5, 3, tol=1e-9, kmax=25)
    assert k == 25
    # the same stuck level among 4999 levels that converge: the error stalls near the stuck
    # level's share, below 1e-4 n = 0.5, so the floor rule ends the recursion long before kmax
    # with every other level converged
    far = np.concatenate([np.linspace(0.0, 0.3, 2500), np.linspace(0.7, 1.0, 2499)])
    x = np.concatenate([far, [0.5]])
    occ, k = dn.sp2_mu_occupations(x, 0.5, x.shape[0], tol=1e-12, kmax=60)
    assert 4 <= k < 30
    assert np.max(np.minimum(occ[:-1], 1.0 - occ[:-1])) < 1e-6
    assert 0.05 < occ[-1] < 0.95


def test_halo_everything_equals_full(w96, full96):
    s, m, n = w96
    cores = graph.rcb_partition(s.R, s.box, 12)
    hal = [np.setdiff1d(np.arange(96), c).astype(np.int32) for c in cores]
    r = dn.density(s.R, s.species, s.box, m, n, cores, hal)
    assert np.max(np.abs(r.q - full96.q)) < 1e-10
    assert abs(r.e_band - full96.e_band) < 1e-9


def test_sp2_polynomial_equals_fermi_in_gap(w96, full96):
    s, m, n = w96
    cores, hal = dn.full_partition(96)
    e = np.sort(full96.subs[0].eps)
    mid = 0.5 * (e[127] + e[128])            # any mu inside the gap gives the same Fermi density
    r = dn.density(s.R, s.species, s.box, m, n, cores, hal, mode="sp2", mu=mid)
    assert np.max(np.abs(r.q - full96.q)) < 1e-9
    x, k = dn.sp2_mu_occupations(np.array([0.0, 0.2, 0.45, 0.55, 0.8, 1.0]), 0.5, 6)
    assert np.allclose(x, [0, 0, 0, 1, 1, 1], atol=1e-6) and k < 60


def test_charges_converge_with_threshold(w96, full96):
    """Sec. "Accuracy Control via Graph Thresholding": error falls as tau falls."""
    s, m, n = w96
    cores = graph.rcb_partition(s.R, s.box, 12)
    cores_f, hal_f = dn.full_partition(96)
    prev = dn.density(s.R, s.species, s.box, m, n, cores, graph.halos(*graph.build_graph(s.R, s.box, 3.0), cores))
    errs = []
    for tau in (1e-2, 1e-3, 1e-4):
        rp, col = graph.build_graph(s.R, s.box, 3.0, full96.gd, tau)
        r = dn.density(s.R, s.species, s.box, m, n, cores, graph.halos(rp, col, cores))
        errs.append(np.max(np.abs(r.q - full96.q)))
    assert errs[0] > errs[1] > errs[2]
    assert errs[2] < 1e-4


def test_forces_equal_finite_difference_of_shadow_energy(w96, full96):
    s, m, n = w96
    cores, hal = dn.full_partition(96)
    F = dn.forces(full96, n, s.R, s.species, s.box, m)

    def U(R):
        r = dn.density(R, s.species, s.box, m, n, cores, hal)
        return dn.shadow_energy(r, n, R, s.species, s.box, m)["total"]

    h = 1e-4
    for A, c in [(0, 0), (1, 2), (50, 1), (95, 0)]:
        Rp = s.R.copy(); Rp[A, c] += h
        Rm = s.R.copy(); Rm[A, c] -= h
        assert abs(F[A, c] + (U(Rp) - U(Rm)) / (2 * h)) < 1e-6
    assert np.max(np.abs(F.sum(axis=0))) < 1e-9      # no net force


def test_subset_rows_equal_full_rows(w96, trunc96):
    """The row-restricted forms of forces, Coulomb potential and gradient, and repulsion give the
    full computation's rows for the chosen atoms."""
    s, m, n = w96
    r, _, _ = trunc96
    pick = np.array([0, 5, 41, 77, 95])
    F = dn.forces(r, n, s.R, s.species, s.box, m)
    Fs = dn.forces(r, n, s.R, s.species, s.box, m, atoms=pick)
    assert np.max(np.abs(Fs[pick] - F[pick])) < 1e-13
    assert np.all(Fs[np.setdiff1d(np.arange(96), pick)] == 0.0)
    from oracle import ewald
    V = ewald.coulomb_potential(s.R, s.species, m.hubbard_u, s.box, n)
    Vs = ewald.coulomb_potential(s.R, s.species, m.hubbard_u, s.box, n, rows=pick)
    assert np.max(np.abs(Vs[pick] - V[pick])) < 1e-13
