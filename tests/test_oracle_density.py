"""Pins of the oracle's subgraph solve, chemical potential, charges, energy and forces."""
import numpy as np
import pytest

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


def test_mu_in_gap_brute_force_grid(full96):
    e = np.concatenate([sg.eps for sg in full96.subs])
    w = np.concatenate([sg.w for sg in full96.subs])
    grid = np.linspace(e.min(), e.max(), 20001)
    n0 = np.array([2 * np.sum(w[e < g]) for g in grid])
    ok = grid[np.abs(n0 - 256.0) < 0.5]
    assert ok.min() <= full96.mu <= ok.max()
    assert abs(full96.mu - 0.5 * (ok.min() + ok.max())) < 2 * (grid[1] - grid[0])


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
    r = dn.density(s.R, s.species, s.box, m, n, cores, hal, mode="sp2", mu=full96.mu)
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
