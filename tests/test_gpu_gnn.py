"""Learned preconditioner on the GPU: forward and parameter gradients against the FP64 oracle
network (same weights, same graph), training on Krylov response pairs, and the gain over K0."""
import numpy as np
import pytest

from oracle import gnn as ognn
from oracle import graph as og
from paper_2606_03140_gb300 import inputs as I

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_2606_03140_gb300 import sedacs
    return sedacs


def _ctx(S, s, kernel=1):
    prm = S.sedacs_default_params(core_size=12, precision=1, kernel=kernel, krylov_rank=4, krylov_tol=1e-6)
    ctx = S.sedacs_create(s.species, s.box, I.default_model(), prm)
    R = np.ascontiguousarray(s.R)
    S.sedacs_graph_build(ctx, R)
    S.sedacs_partition(ctx, R)
    return ctx, R


def test_forward_and_gradient_match_oracle(S):
    s = I.workload("water96")
    ctx, R = _ctx(S, s)
    try:
        rp, col = og.build_graph(s.R, s.box, 3.0)
        edges = ognn.edges_from_csr(rp, col, s.R, s.box)
        p = ognn.init_params(11) * 4.0
        S.sedacs_gnn_set_params(ctx, p)
        assert np.allclose(S.sedacs_gnn_get_params(ctx), p, rtol=1e-6, atol=1e-7)
        rng = np.random.default_rng(1)
        y = rng.standard_normal(96)
        gu = rng.standard_normal(96)
        u = S.sedacs_gnn_apply(ctx, y)
        u_ref = ognn.forward(p, y, s.species, edges, 0.5)
        assert np.max(np.abs(u - u_ref)) < 1e-4 * np.max(np.abs(u_ref))
        g = S.sedacs_gnn_param_grad(ctx, y, gu)
        g_ref = ognn.backward(p, y, s.species, edges, 0.5, gu)
        assert np.max(np.abs(g - g_ref)) < 1e-3 * np.max(np.abs(g_ref))
    finally:
        S.sedacs_destroy(ctx)


def test_training_on_krylov_pairs_beats_k0(S):
    s = I.workload("water96")
    ctx, R = _ctx(S, s)
    try:
        n = np.zeros(96)
        mu, q, _, _ = S.sedacs_subgraph_density(ctx, R, n)
        S.sedacs_gnn_init(ctx, 3)
        S.sedacs_gnn_collect(ctx, True, 256)
        rng = np.random.default_rng(7)
        for _ in range(24):                       # Krylov responses of random residuals -> pairs
            S.sedacs_kernel_apply(ctx, rng.standard_normal(96) * 0.02)
        S.sedacs_gnn_collect(ctx, False)
        # held-out pairs: fresh Krylov vectors through the response directly
        X, V = [], []
        for _ in range(6):
            v = rng.standard_normal(96)
            v /= np.linalg.norm(v)
            X.append(S.sedacs_charge_response(ctx, v) - v)   # J v
            V.append(v)
        X, V = np.array(X), np.array(V)
        def err(apply):
            return float(np.mean([np.linalg.norm(apply(x) - v) / np.linalg.norm(v) for x, v in zip(X, V)]))
        e_k0 = err(lambda x: -0.5 * x)
        l0, l1 = S.sedacs_gnn_train(ctx, epochs=300, lr=2e-3)
        assert l1 < 0.5 * l0
        e_nn = err(lambda x: S.sedacs_gnn_apply(ctx, x))
        assert e_nn < 0.7 * e_k0, (e_nn, e_k0)
    finally:
        S.sedacs_destroy(ctx)
