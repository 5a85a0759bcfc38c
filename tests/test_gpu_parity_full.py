"""Parity at the full size of the benchmark workload (9,000-atom water box), in the
configuration bench.py times (cores ~32 atoms, precision 1: SP2 squares in two fp16 planes, the
other products three-way split bf16, on tcgen05).

The oracle cannot solve every subgraph of every step in seconds, so it recomputes sampled
subgraphs one by one: with zero trial charges (no Coulomb shift) on the distance graph,
whose cores and halos the oracle builds itself, and at one explicit chemical potential in
the gap given to both sides.  Graph / cores / halos are compared bit for bit on the whole
system; charges of the sampled cores within the 1e-5 e bound.
"""
import numpy as np
import pytest

from oracle import density as odn
from oracle import graph as og
from paper_2606_03140_gb300 import inputs as I

pytestmark = pytest.mark.gpu

PICK = [0, 97, 180, 280]


def _clean_mu(subs):
    """Middle of the widest interval in [-0.35, 0.05] Ha free of sampled states with core weight > 1e-6."""
    e = np.sort(np.concatenate([sg.eps[sg.w > 1e-6] for sg in subs]))
    e = e[(e > -0.35) & (e < 0.05)]
    k = int(np.argmax(np.diff(e)))
    return 0.5 * (e[k] + e[k + 1]), e[k + 1] - e[k]


@pytest.fixture(scope="module")
def full():
    from paper_2606_03140_gb300 import sedacs as S

    s = I.workload("water9000")
    m = I.default_model()
    rp_o, col_o = og.build_graph(s.R, s.box, 3.0)
    cores = og.rcb_partition(s.R, s.box, 32)
    hal = og.halos(rp_o, col_o, cores)
    res0 = odn.density(s.R, s.species, s.box, m, np.zeros(s.n_atoms), [cores[i] for i in PICK],
                       [hal[i] for i in PICK], mu=-0.13, V=np.zeros(s.n_atoms))
    MU, width = _clean_mu(res0.subs)
    R = np.ascontiguousarray(s.R)
    ctx = S.sedacs_create(s.species, s.box, m, S.sedacs_default_params(core_size=32, precision=1))
    nnz = S.sedacs_graph_build(ctx, R)
    rp, col = S.sedacs_graph_get(ctx, s.n_atoms, nnz)
    S.sedacs_partition(ctx, R)
    sp, sa, nc = S.sedacs_parts_get(ctx)
    n = np.zeros(s.n_atoms)
    mu, q, eb, iters = S.sedacs_subgraph_density(ctx, R, n, mu=MU, n_parts=len(nc))
    F = S.sedacs_forces(ctx, s.n_atoms)
    S.sedacs_destroy(ctx)
    ref = odn.density(s.R, s.species, s.box, m, np.zeros(s.n_atoms), [cores[i] for i in PICK],
                      [hal[i] for i in PICK], mu=MU, V=np.zeros(s.n_atoms))
    return dict(s=s, m=m, rp=rp, col=col, sp=sp, sa=sa, nc=nc, q=q, iters=iters, F=F, ref=ref, mu=MU,
                width=width, cores=cores)


def test_graph_cores_halos_bit_exact_full_size(full):
    s = full["s"]
    rp, col = og.build_graph(s.R, s.box, 3.0)
    assert np.array_equal(rp, full["rp"]) and np.array_equal(col, full["col"])
    cores = og.rcb_partition(s.R, s.box, 32)
    hal = og.halos(rp, col, cores)
    sp, sa, nc = full["sp"], full["sa"], full["nc"]
    assert len(cores) == len(nc) == 281
    for i in range(len(cores)):
        assert np.array_equal(sa[sp[i]:sp[i] + nc[i]], cores[i])
        assert np.array_equal(sa[sp[i] + nc[i]:sp[i + 1]], hal[i])


def test_sampled_subgraph_charges_full_size(full):
    res = full["ref"]
    assert full["width"] > 0.05                      # mu sits in a clean window of the sampled spectra
    atoms = np.concatenate([full["cores"][i] for i in PICK])
    err = np.max(np.abs(full["q"][atoms] - res.q[atoms]))
    print(f"[parity] water9000 form 1, sampled subgraphs: max|dq| = {err:.3e} e")
    assert err < 1e-5, err
    assert np.all(np.isfinite(full["F"]))
