"""Core refinement for the 128-orbital tiles through the C ABI against the oracle.

The refinement is integer work on the graph and the cores (greedy single-atom moves decided by an
integer score of the padded cube cost), so cores, halos and both scores must be bit-exact.  The
subgraph solves then run on the refined cores and give the oracle's density on them.
"""
import numpy as np
import pytest

from oracle import density as odn
from oracle import graph as og
from paper_2606_03140_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _cores_from(sp, sa, nc):
    return [np.sort(sa[sp[i]:sp[i] + nc[i]]) for i in range(len(nc))]


@pytest.mark.parametrize("which,core", [("water96", 12), ("water3000", 32)])
def test_refine_cores_bit_exact(which, core):
    from paper_2606_03140_gb300 import sedacs as S

    s = I.workload("water96") if which == "water96" else I.small_water_box(1000, 31.0, seed=33)
    m = I.default_model()
    norb = np.asarray(m.n_orb)[s.species]
    prm = S.sedacs_default_params(core_size=core)
    ctx = S.sedacs_create(s.species, s.box, m, prm)
    try:
        R = np.ascontiguousarray(s.R)
        nnz = S.sedacs_graph_build(ctx, R)
        S.sedacs_partition(ctx, R)
        rp, col = S.sedacs_graph_get(ctx, s.n_atoms, nnz)
        cores0 = _cores_from(*S.sedacs_parts_get(ctx))
        b, a = S.sedacs_refine_cores(ctx, 4, 16 if core >= 32 else 4)
        sp, sa, nc = S.sedacs_parts_get(ctx)
    finally:
        S.sedacs_destroy(ctx)
    ref, rb, ra = og.refine_cores(rp, col, cores0, norb, rounds=4, min_core=16 if core >= 32 else 4)
    got = _cores_from(sp, sa, nc)
    print(f"[parity] {which} refine: score {b} -> {a} (oracle {rb} -> {ra}), {len(got)} cores")
    assert (b, a) == (rb, ra)
    assert len(got) == len(ref) and all(np.array_equal(x, y) for x, y in zip(got, ref))
    halos = og.halos(rp, col, ref)
    for i in range(len(ref)):
        assert np.array_equal(np.sort(sa[sp[i] + nc[i]:sp[i + 1]]), np.sort(halos[i]))


def test_refine_needs_graph_and_cores():
    from paper_2606_03140_gb300 import sedacs as S

    s = I.workload("water96")
    ctx = S.sedacs_create(s.species, s.box, I.default_model(), S.sedacs_default_params(core_size=12))
    try:
        with pytest.raises(RuntimeError):
            S.sedacs_refine_cores(ctx)
    finally:
        S.sedacs_destroy(ctx)


def test_density_on_refined_cores():
    from paper_2606_03140_gb300 import sedacs as S

    s = I.small_water_box(1000, 31.0, seed=33)
    m = I.default_model()
    n = I.random_charges(s.n_atoms, 3, 0.05)
    prm = S.sedacs_default_params(core_size=32, precision=0)
    ctx = S.sedacs_create(s.species, s.box, m, prm)
    try:
        R = np.ascontiguousarray(s.R)
        nnz = S.sedacs_graph_build(ctx, R)
        S.sedacs_partition(ctx, R)
        S.sedacs_refine_cores(ctx)
        rp, col = S.sedacs_graph_get(ctx, s.n_atoms, nnz)
        cores = _cores_from(*S.sedacs_parts_get(ctx))
        mu, q, _, _ = S.sedacs_subgraph_density(ctx, R, np.ascontiguousarray(n))
    finally:
        S.sedacs_destroy(ctx)
    r0 = odn.density(s.R, s.species, s.box, m, n, cores, og.halos(rp, col, cores))
    dq = float(np.max(np.abs(q - r0.q)))
    print(f"[parity] water3000 density on refined cores (FP64): max |dq| {dq:.2e} e, |dmu| {abs(mu - r0.mu):.2e} Ha")
    assert dq < 1e-8
