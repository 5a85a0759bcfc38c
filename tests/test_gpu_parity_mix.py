"""Parity on the 9,999-atom methanol/water mixture (1:1, 0.9 g/cm3) in the mixed form: graph,
cores and halos bit for bit on the whole system, charges of sampled subgraphs (C/O sp and H s
orbitals) within the 1e-5 e bound, at zero trial charges and one chemical potential in a clean
window of the sampled spectra, given to both sides (Fermi occupations at 300 K; the oracle solves
the sampled subgraphs one by one, through its LAPACK eigensolver route)."""
import numpy as np
import pytest

from oracle import density as odn
from oracle import graph as og
from paper_2606_03140_gb300 import inputs as I

pytestmark = pytest.mark.gpu

PICK = [0, 101, 202, 311]


def test_mixture_graph_and_sampled_charges():
    from paper_2606_03140_gb300 import sedacs as S

    s = I.workload("mix9999")
    m = I.default_model()
    rp_o, col_o = og.build_graph(s.R, s.box, 3.0)
    cores = og.rcb_partition(s.R, s.box, 32)
    hal = og.halos(rp_o, col_o, cores)
    res0 = odn.density(s.R, s.species, s.box, m, np.zeros(s.n_atoms), [cores[i] for i in PICK],
                       [hal[i] for i in PICK], mu=-0.1, V=np.zeros(s.n_atoms), eig="lapack")
    e = np.sort(np.concatenate([sg.eps[sg.w > 1e-6] for sg in res0.subs]))
    e = e[(e > -0.35) & (e < 0.05)]
    k = int(np.argmax(np.diff(e)))
    mu = 0.5 * (e[k] + e[k + 1])
    assert e[k + 1] - e[k] > 0.05
    ref = odn.density(s.R, s.species, s.box, m, np.zeros(s.n_atoms), [cores[i] for i in PICK],
                      [hal[i] for i in PICK], mu=mu, V=np.zeros(s.n_atoms), eig="lapack")
    R = np.ascontiguousarray(s.R)
    ctx = S.sedacs_create(s.species, s.box, m, S.sedacs_default_params(core_size=32, precision=1, mu_given=1))
    try:
        nnz = S.sedacs_graph_build(ctx, R)
        rp, col = S.sedacs_graph_get(ctx, s.n_atoms, nnz)
        assert np.array_equal(rp, rp_o) and np.array_equal(col, col_o)
        S.sedacs_partition(ctx, R)
        sp, sa, nc = S.sedacs_parts_get(ctx)
        for i in PICK:
            assert np.array_equal(sa[sp[i]:sp[i] + nc[i]], cores[i])
            assert np.array_equal(sa[sp[i] + nc[i]:sp[i + 1]], hal[i])
        mu_g, q, eb, it = S.sedacs_subgraph_density(ctx, R, np.zeros(s.n_atoms), mu=mu, n_parts=len(nc))
    finally:
        S.sedacs_destroy(ctx)
    atoms = np.concatenate([cores[i] for i in PICK])
    print(f"[parity] mix9999 form 1, sampled subgraphs: max|dq| = {np.max(np.abs(q[atoms] - ref.q[atoms])):.3e} e")
    assert np.max(np.abs(q[atoms] - ref.q[atoms])) < 1e-5
