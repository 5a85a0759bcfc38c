"""Pins of the oracle's preconditioner network: finite-difference gradient, linearity, K0 limit."""
import numpy as np

from oracle import gnn, graph
from paper_2606_03140_gb300 import inputs as I


def _setup():
    s = I.small_water_box(6, 7.5, seed=41)
    rp, col = graph.build_graph(s.R, s.box, 3.0)
    edges = gnn.edges_from_csr(rp, col, s.R, s.box)
    return s, edges


def test_gradient_matches_finite_difference():
    s, edges = _setup()
    rng = np.random.default_rng(2)
    p = gnn.init_params(7) * 5.0
    y = rng.standard_normal(s.n_atoms)
    gu = rng.standard_normal(s.n_atoms)
    g = gnn.backward(p, y, s.species, edges, 0.5, gu)
    h = 1e-6
    idx = rng.choice(len(p), size=40, replace=False)
    idx = np.concatenate([idx, [0, 200, len(p) - 1]])       # embedding, a filter weight, output
    for k in idx:
        pp = p.copy(); pp[k] += h
        pm = p.copy(); pm[k] -= h
        fd = (gnn.forward(pp, y, s.species, edges, 0.5) @ gu - gnn.forward(pm, y, s.species, edges, 0.5) @ gu) / (2 * h)
        assert abs(fd - g[k]) < 1e-6 * max(1.0, abs(fd))


def test_network_is_linear_in_the_residual_and_reduces_to_k0():
    s, edges = _setup()
    rng = np.random.default_rng(3)
    p = gnn.init_params(1) * 3.0
    y1, y2 = rng.standard_normal(s.n_atoms), rng.standard_normal(s.n_atoms)
    u = gnn.forward(p, 2.0 * y1 - 0.5 * y2, s.species, edges, 0.5)
    assert np.allclose(u, 2.0 * gnn.forward(p, y1, s.species, edges, 0.5) - 0.5 * gnn.forward(p, y2, s.species, edges, 0.5),
                       atol=1e-12)
    assert np.allclose(gnn.forward(np.zeros_like(p), y1, s.species, edges, 0.5), -0.5 * y1)


def test_training_step_reduces_loss():
    s, edges = _setup()
    rng = np.random.default_rng(4)
    p = gnn.init_params(5)
    X = rng.standard_normal((3, s.n_atoms))
    V = -0.8 * X + 0.1 * np.roll(X, 1, axis=1)
    L0, G = gnn.loss_and_grad(p, X, V, s.species, edges, 0.5)
    L1, _ = gnn.loss_and_grad(p - 1e-3 * G / np.linalg.norm(G), X, V, s.species, edges, 0.5)
    assert L1 < L0
