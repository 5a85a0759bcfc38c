"""Pins of the oracle's plain-C cyclic Jacobi eigensolver and of the subgraph solve built on it.

Each check is fixed by mathematics independent of the code: closed-form spectra (2 x 2, the
tridiagonal Toeplitz matrix), a spectrum planted by an orthogonal similarity, the eigen-equation
and orthonormality, and agreement with the LAPACK route of the same subgraph solve.
"""
import math

import numpy as np
import pytest

from oracle import cjacobi as J
from oracle import density as odn
from oracle import ewald
from oracle import graph as og
from paper_2606_03140_gb300 import inputs as I


def test_two_by_two_closed_form():
    a, b, d = 0.7, -0.3, -1.1
    w, v, _ = J.eigh(np.array([[a, b], [b, d]]))
    m, r = 0.5 * (a + d), math.hypot(0.5 * (a - d), b)
    assert abs(w[0] - (m - r)) < 1e-15 and abs(w[1] - (m + r)) < 1e-15
    for k in range(2):
        x = v[:, k]
        assert abs((a - w[k]) * x[0] + b * x[1]) < 1e-15 and abs(np.linalg.norm(x) - 1) < 1e-15


def test_tridiagonal_toeplitz_spectrum_and_vectors():
    n, a, b = 37, 0.25, -0.8
    A = np.diag(np.full(n, a)) + np.diag(np.full(n - 1, b), 1) + np.diag(np.full(n - 1, b), -1)
    w, v, _ = J.eigh(A)
    k = np.arange(1, n + 1)
    exact = np.sort(a + 2 * b * np.cos(k * np.pi / (n + 1)))
    assert np.max(np.abs(w - exact)) < 1e-14
    # eigenvector of a + 2 b cos(k pi / (n+1)) is sin(j k pi / (n+1)), j = 1..n (up to sign)
    j = np.arange(1, n + 1)
    for col in range(n):
        kk = int(np.argmin(np.abs(a + 2 * b * np.cos(k * np.pi / (n + 1)) - w[col]))) + 1
        u = np.sin(j * kk * np.pi / (n + 1))
        u /= np.linalg.norm(u)
        assert abs(abs(u @ v[:, col]) - 1.0) < 1e-12


def test_planted_spectrum():
    rng = np.random.default_rng(5)
    n = 48
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.sort(rng.uniform(-3, 3, n))
    A = (Q * lam) @ Q.T
    w, v, sweeps = J.eigh(A)
    assert np.max(np.abs(w - lam)) < 1e-13
    assert np.max(np.abs(np.abs(np.sum(v * Q, axis=0)) - 1.0)) < 1e-9
    assert 3 <= sweeps <= 15


def test_degenerate_eigenspace_projector():
    rng = np.random.default_rng(6)
    n = 20
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.array([-1.0] * 5 + [0.5] * 7 + list(np.linspace(1, 2, 8)))
    A = (Q * lam) @ Q.T
    w, v, _ = J.eigh(A)
    assert np.max(np.abs(w - np.sort(lam))) < 1e-13
    P = v[:, :5] @ v[:, :5].T
    assert np.max(np.abs(P - Q[:, :5] @ Q[:, :5].T)) < 1e-12


def test_eigen_equation_orthonormal_and_edges():
    rng = np.random.default_rng(7)
    A = rng.standard_normal((60, 60))
    A = A + A.T
    w, v, _ = J.eigh(A)
    assert np.max(np.abs(A @ v - v * w)) < 1e-12 * np.abs(w).max()
    assert np.max(np.abs(v.T @ v - np.eye(60))) < 1e-13
    assert np.all(np.diff(w) >= 0)
    w0, v0, s0 = J.eigh(np.zeros((0, 0)))
    assert w0.shape == (0,) and s0 == 0
    w1, v1, s1 = J.eigh(np.array([[-2.5]]))
    assert w1[0] == -2.5 and v1[0, 0] == 1.0 and s1 == 0
    wd, vd, sd = J.eigh(np.diag([3.0, -1.0, 2.0]))
    assert sd == 0 and list(wd) == [-1.0, 2.0, 3.0] and np.array_equal(np.abs(vd), np.eye(3)[:, [1, 2, 0]])


def test_indefinite_overlap_is_an_error():
    s = np.array([[1.0, 2.0], [2.0, 1.0]])
    with pytest.raises(RuntimeError):
        J.subgraph_eig(np.eye(2), s, 1)


def _water96():
    s = I.workload("water96")
    m = I.default_model()
    n = I.random_charges(s.n_atoms, 3, 0.05)
    rp, col = og.build_graph(s.R, s.box, 3.0)
    cores = og.rcb_partition(s.R, s.box, 12)
    return s, m, n, cores, og.halos(rp, col, cores)


def test_subgraph_solve_matches_lapack_route():
    s, m, n, cores, halos = _water96()
    V = ewald.coulomb_potential(s.R, s.species, m.hubbard_u, s.box, n)
    atoms = [np.concatenate([c, h]).astype(np.int64) for c, h in zip(cores, halos)]
    jac = odn.subgraph_setup_all(atoms, [len(c) for c in cores], s.R, s.species, s.box, m, V, eig="jacobi")
    lap = odn.subgraph_setup_all(atoms, [len(c) for c in cores], s.R, s.species, s.box, m, V, eig="lapack")
    for a, b in zip(jac, lap):
        k = len(a.eps)
        assert np.max(np.abs(a.eps - b.eps)) < 1e-12
        assert np.max(np.abs(a.Z @ a.S @ a.Z - np.eye(k))) < 1e-12
        assert np.max(np.abs(a.Z - b.Z)) < 1e-12
        # the core weights of one state depend on the basis chosen inside a degenerate
        # eigenspace; their sums over each eigenspace do not
        assert abs(a.w.sum() - b.w.sum()) < 1e-11
        Ht = a.Z @ a.H @ a.Z
        assert np.max(np.abs(Ht @ a.X - a.X * a.eps)) < 1e-12
        assert np.max(np.abs(a.C - a.Z @ a.X)) < 1e-13
    one = odn.subgraph_setup(atoms[3], len(cores[3]), s.R, s.species, s.box, m, V, eig="jacobi")
    assert np.array_equal(one.eps, jac[3].eps) and np.array_equal(one.C, jac[3].C)


def test_density_jacobi_equals_lapack():
    s, m, n, cores, halos = _water96()
    a = odn.density(s.R, s.species, s.box, m, n, cores, halos, eig="jacobi")
    b = odn.density(s.R, s.species, s.box, m, n, cores, halos, eig="lapack")
    assert abs(a.mu - b.mu) < 1e-11
    assert np.max(np.abs(a.q - b.q)) < 1e-11
    assert abs(a.e_band - b.e_band) < 1e-10


def test_collected_count_in_c_equals_plain_sum_and_bisection_meets_the_count():
    rng = np.random.default_rng(12)
    eps = [np.sort(rng.uniform(-1.2, 0.4, k)) for k in (7, 11, 5)]
    w = [rng.uniform(0.0, 1.0, len(e)) for e in eps]
    beta = 1.0 / (3.166811563e-6 * 3000.0)
    for mu in (-0.6, -0.1, 0.05):
        plain = 2.0 * sum(float(np.sum(wi / (1.0 + np.exp(beta * (ei - mu))))) for ei, wi in zip(eps, w))
        assert abs(J.collected_count(eps, w, mu, beta) - plain) < 1e-12
    n_e = 0.8 * 2.0 * sum(float(x.sum()) for x in w)
    mu = J.solve_mu(eps, w, n_e, beta)
    assert abs(J.collected_count(eps, w, mu, beta) - n_e) < 1e-9
    assert min(float(e.min()) for e in eps) - 1.0 < mu < max(float(e.max()) for e in eps) + 1.0
    with pytest.raises(ValueError):
        J.solve_mu([np.zeros(0)], [np.zeros(0)], 1.0, beta)
