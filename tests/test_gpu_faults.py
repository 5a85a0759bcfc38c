"""Failure reporting through the C ABI, made on the host side or by a bounded wait (no GPU fault).

* A NaN in a host-given input (one dynamical charge) propagates through the Coulomb potential
  into every subgraph's Hamiltonian; the collected count comes back non-finite and the call
  returns SEDACS_ENUMERIC.  The context stays usable: the next call with valid charges matches
  a fresh context.  (NaN is not given in the positions: the cell lists index by them.)
* A device wait that nothing completes gives up after its cycle limit and the call returns
  SEDACS_ETIMEOUT (sedacs_selftest_wait: the same bit every bounded wait of the library raises);
  the context stays usable.
* An SCC cut off after two iterations from zero charges returns SEDACS_ENOCONV.
* Invalid cores given by the host are refused with SEDACS_EINVAL and leave the context's cores as
  they were.
"""
import numpy as np
import pytest

from paper_2606_03140_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _ctx(S, precision=1):
    s = I.workload("water96")
    m = I.default_model()
    ctx = S.sedacs_create(s.species, s.box, m, S.sedacs_default_params(core_size=12, precision=precision))
    R = np.ascontiguousarray(s.R)
    S.sedacs_graph_build(ctx, R)
    S.sedacs_partition(ctx, R)
    return s, ctx, R


@pytest.mark.parametrize("precision", [0, 1])
def test_nan_charge_reports_enumeric_and_context_recovers(precision):
    from paper_2606_03140_gb300 import sedacs as S

    s, ctx, R = _ctx(S, precision)
    try:
        n = np.ascontiguousarray(I.random_charges(96, 3, 0.05))
        bad = n.copy()
        bad[17] = np.nan
        with pytest.raises(S.SedacsError) as ei:
            S.sedacs_subgraph_density(ctx, R, bad)
        assert ei.value.status == 6                      # SEDACS_ENUMERIC
        mu, q, _, _ = S.sedacs_subgraph_density(ctx, R, n)
    finally:
        S.sedacs_destroy(ctx)
    s2, ref, R2 = _ctx(S, precision)
    try:
        mu2, q2, _, _ = S.sedacs_subgraph_density(ref, R2, n)
    finally:
        S.sedacs_destroy(ref)
    assert np.all(np.isfinite(q))
    assert np.max(np.abs(q - q2)) < (1e-12 if precision == 0 else 1e-6)


def test_bounded_wait_reports_etimeout_and_context_recovers():
    from paper_2606_03140_gb300 import sedacs as S

    s, ctx, R = _ctx(S)
    try:
        assert S.sedacs_selftest_wait(ctx, 20000) == 5    # SEDACS_ETIMEOUT after ~20 ms
        assert S.sedacs_selftest_wait(ctx, 0) == 1        # SEDACS_EINVAL: limit out of range
        mu, q, _, _ = S.sedacs_subgraph_density(ctx, R, np.zeros(96))
        assert np.all(np.isfinite(q))
    finally:
        S.sedacs_destroy(ctx)


def test_scc_cut_short_reports_enoconv():
    from paper_2606_03140_gb300 import sedacs as S

    s, ctx, R = _ctx(S)
    try:
        n = np.zeros(96)
        mu, resid, it, ok = S.sedacs_scc_step(ctx, R, n, max_iter=2)
    finally:
        S.sedacs_destroy(ctx)
    assert not ok and it == 2 and resid > 1e-3


def test_invalid_cores_are_refused_and_context_recovers():
    """Cores that leave an atom out, repeat one, hold no atom or outnumber the atoms are refused
    with SEDACS_EINVAL before anything reaches the device; the context keeps its cores."""
    from paper_2606_03140_gb300 import sedacs as S

    s, ctx, R = _ctx(S)
    try:
        sp, sa, nc = S.sedacs_parts_get(ctx)
        good = [sa[sp[i]:sp[i] + nc[i]].copy() for i in range(len(nc))]
        n = np.ascontiguousarray(I.random_charges(96, 3, 0.05))
        mu0, q0, _, _ = S.sedacs_subgraph_density(ctx, R, n)
        bad_sets = [
            [good[0][1:]] + good[1:],                                   # an atom left out
            [np.concatenate([good[0], good[1][:1]])] + good[1:],        # an atom in two cores
            good + [np.zeros(0, np.int32)],                             # an empty core
            [np.array([a], np.int32) for a in range(96)] + [np.array([0], np.int32)],  # 97 cores
        ]
        for cores in bad_sets:
            with pytest.raises(S.SedacsError) as ei:
                S.sedacs_set_cores(ctx, cores)
            assert ei.value.status == 1                                 # SEDACS_EINVAL
        sp1, sa1, nc1 = S.sedacs_parts_get(ctx)
        assert np.array_equal(sp1, sp) and np.array_equal(sa1, sa) and np.array_equal(nc1, nc)
        mu1, q1, _, _ = S.sedacs_subgraph_density(ctx, R, n)
        # the second solve may start mu from the first one's, so equal up to the solve's tolerance
        assert abs(mu1 - mu0) < 1e-8 and np.max(np.abs(q1 - q0)) < 1e-6
    finally:
        S.sedacs_destroy(ctx)
