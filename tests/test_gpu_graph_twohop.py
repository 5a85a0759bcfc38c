"""The weighted two-hop graph adaptation (Sec. "Dynamic Graph Adaption", Eq. "Graph_Adaptation")
through the C ABI against the oracle.

G^N_IK = exp(-alpha R_IK^2) on the pairs with R^2 < ln(2/tau)/alpha, G^N_II = 1, P = G^N G^D with
the oracle's atom-condensed density graph G^D of a first density; edge when P_IJ or P_JI exceeds
tau.  The graph is integer output decided by FP64 sums that both sides take in the same order;
only the exponentials differ (CUDA's exp and numpy's, each within 1-2 ulp), so the CSR must be
bit-exact except for pairs whose deciding product lies within 1e-12 tau of tau (none occur here).
A density on that graph then matches the oracle's as on the distance/|D| graph.
"""
import numpy as np
import pytest

from oracle import density as odn
from oracle import graph as og
from paper_2606_03140_gb300 import inputs as I

pytestmark = pytest.mark.gpu

ALPHA, TAU = 0.7, 1e-3


def _first_density(s, core_size):
    m = I.default_model()
    n = I.random_charges(s.n_atoms, 3, 0.05)
    rp, col = og.build_graph(s.R, s.box, 3.0)
    cores = og.rcb_partition(s.R, s.box, core_size)
    r0 = odn.density(s.R, s.species, s.box, m, n, cores, og.halos(rp, col, cores))
    return m, n, cores, r0


@pytest.mark.parametrize("which", ["water96", "water3000"])
def test_two_hop_graph_bit_exact(which):
    from paper_2606_03140_gb300 import sedacs as S

    s = I.workload("water96") if which == "water96" else I.small_water_box(1000, 31.0, seed=33)
    core = 12 if which == "water96" else 32
    m, n, cores, r0 = _first_density(s, core)
    rp_ref, col_ref, amb = og.build_graph_two_hop(s.R, s.box, r0.gd, ALPHA, TAU)
    prm = S.sedacs_default_params(core_size=core, graph_rule=1, graph_alpha=ALPHA, tau=TAU)
    ctx = S.sedacs_create(s.species, s.box, m, prm)
    try:
        R = np.ascontiguousarray(s.R)
        S.sedacs_graph_build(ctx, R)                      # first build: the distance rule
        nnz = S.sedacs_graph_build(ctx, R, gd=r0.gd)      # then the two-hop rule
        rp, col = S.sedacs_graph_get(ctx, s.n_atoms, nnz)
    finally:
        S.sedacs_destroy(ctx)
    print(f"[parity] {which} two-hop graph: {len(col)} edges (oracle {len(col_ref)}), ambiguous pairs {len(amb)}")
    if not amb:
        assert np.array_equal(rp, rp_ref) and np.array_equal(col, col_ref)
    else:
        got = {(i, int(j)) for i in range(s.n_atoms) for j in col[rp[i]:rp[i + 1]]}
        ref = {(i, int(j)) for i in range(s.n_atoms) for j in col_ref[rp_ref[i]:rp_ref[i + 1]]}
        diff = {(min(a, b), max(a, b)) for a, b in got ^ ref}
        assert diff <= set(amb)


@pytest.mark.parametrize("precision,tol", [(0, 1e-8), (1, 2e-5)])
def test_density_on_two_hop_graph(precision, tol):
    from paper_2606_03140_gb300 import sedacs as S

    s = I.workload("water96")
    m, n, cores, r0 = _first_density(s, 12)
    rp, col, _ = og.build_graph_two_hop(s.R, s.box, r0.gd, ALPHA, TAU)
    ref = odn.density(s.R, s.species, s.box, m, n, cores, og.halos(rp, col, cores))
    prm = S.sedacs_default_params(core_size=12, precision=precision, graph_rule=1, graph_alpha=ALPHA, tau=TAU)
    ctx = S.sedacs_create(s.species, s.box, m, prm)
    try:
        R = np.ascontiguousarray(s.R)
        S.sedacs_graph_build(ctx, R)
        S.sedacs_partition(ctx, R)
        S.sedacs_graph_build(ctx, R, gd=r0.gd)
        mu, q, eb, _ = S.sedacs_subgraph_density(ctx, R, np.ascontiguousarray(n))
    finally:
        S.sedacs_destroy(ctx)
    dq = float(np.max(np.abs(q - ref.q)))
    print(f"[parity] water96 density on the two-hop graph, form {precision}: max|dq| {dq:.2e} e, "
          f"|dmu| {abs(mu - ref.mu):.2e} Ha")
    assert dq < tol
