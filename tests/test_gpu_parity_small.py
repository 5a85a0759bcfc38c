"""GPU parity against the FP64 oracle on the 96-atom water box (32 H2O, 9.86 A), every stage.

All calls go through the C ABI.  Each side solves Eq. 2 for its own chemical potential (Fermi
occupations at 300 K).  Tolerances: bit-exact for graph / partition / halos; FP64 plain form
~1e-9; FP32-class forms (1: recursion products in two fp16 planes, 4: in three bf16 planes)
2e-5 e on charges (measured 7e-6 - 1.0e-5: levels within a few kT of mu respond to the ~1e-7 Ha
level noise of FP32 accumulation with beta f (1 - f)); mixed BF16 form 3e-4 e; energies 1e-5
Ha/atom.  The T -> 0 SP2 recursion (Te = 0) is checked at a chemical potential in the clean gap
above the occupied band, where the 300 K Fermi occupations are steps, against the 1e-5 e bound.
"""
import numpy as np
import pytest

from oracle import density as odn
from oracle import dynamics as odyn
from oracle import ewald as oew
from oracle import graph as og
from paper_2606_03140_gb300 import inputs as I

pytestmark = pytest.mark.gpu

# precisions 1 (SP2 squares in two fp16 planes, 22 bits) and 4 (three bf16 planes, 24 bits;
# other products three-way bf16 in both, FP32 accumulation) are held to the 1e-5 e bound of the
# mixed-vs-plain comparison; precision 2 (two-way bf16 SP2 squares, 16 bits) is a diagnostic
# form whose error (~1e-4 e) is bounded here, not claimed to meet 1e-5.
PREC = {0: dict(q=1e-8, V=1e-9, hs=1e-12, Z=1e-9, F=1e-7, e=1e-8, mu=1e-8, rsp=3e-5, kry=1e-4),
        1: dict(q=2e-5, V=1e-6, hs=1e-6, Z=1e-5, F=2e-5, e=1e-5, mu=5e-5, rsp=3e-2, kry=5e-2),
        2: dict(q=3e-4, V=1e-6, hs=1e-6, Z=1e-5, F=5e-4, e=1e-4, mu=5e-3, rsp=1.0, kry=1.0)}
PREC[4] = PREC[1]


@pytest.fixture(scope="module")
def S():
    from paper_2606_03140_gb300 import sedacs
    return sedacs


@pytest.fixture(scope="module")
def sysdata():
    s = I.workload("water96")
    m = I.default_model()
    n = I.random_charges(96, 3, 0.05)
    rp, col = og.build_graph(s.R, s.box, 3.0)
    cores = og.rcb_partition(s.R, s.box, 12)
    ref0 = odn.density(s.R, s.species, s.box, m, n, cores, og.halos(rp, col, cores))
    rp2, col2 = og.build_graph(s.R, s.box, 3.0, ref0.gd, 1e-3)
    hal2 = og.halos(rp2, col2, cores)
    ref = odn.density(s.R, s.species, s.box, m, n, cores, hal2)
    return dict(s=s, m=m, n=n, rp=rp, col=col, cores=cores, ref0=ref0, rp2=rp2, col2=col2, hal2=hal2, ref=ref)


def make_ctx(S, d, precision):
    prm = S.sedacs_default_params(core_size=12, precision=precision)
    return S.sedacs_create(d["s"].species, d["s"].box, d["m"], prm)


def test_graph_partition_halos_bit_exact(S, sysdata):
    d = sysdata
    s = d["s"]
    R = np.ascontiguousarray(s.R)
    ctx = make_ctx(S, d, 1)
    try:
        nnz = S.sedacs_graph_build(ctx, R)
        rp, col = S.sedacs_graph_get(ctx, 96, nnz)
        assert np.array_equal(rp, d["rp"]) and np.array_equal(col, d["col"])
        S.sedacs_partition(ctx, R)
        sp, sa, nc = S.sedacs_parts_get(ctx)
        hal = og.halos(d["rp"], d["col"], d["cores"])
        for i, (c, h) in enumerate(zip(d["cores"], hal)):
            assert list(sa[sp[i]:sp[i] + nc[i]]) == list(c)
            assert list(sa[sp[i] + nc[i]:sp[i + 1]]) == list(h)
        # graph with the oracle's density graph as input
        nnz2 = S.sedacs_graph_build(ctx, R, gd=d["ref0"].gd)
        rp2, col2 = S.sedacs_graph_get(ctx, 96, nnz2)
        assert np.array_equal(rp2, d["rp2"]) and np.array_equal(col2, d["col2"])
        sp, sa, nc = S.sedacs_parts_get(ctx)
        for i, h in enumerate(d["hal2"]):
            assert list(sa[sp[i] + nc[i]:sp[i + 1]]) == list(h)
    finally:
        S.sedacs_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1])
def test_coulomb_potential(S, sysdata, precision):
    d = sysdata
    s = d["s"]
    ctx = make_ctx(S, d, precision)
    try:
        V = S.sedacs_coulomb_potential(ctx, np.ascontiguousarray(s.R), d["n"])
    finally:
        S.sedacs_destroy(ctx)
    Vref = oew.coulomb_potential(s.R, s.species, d["m"].hubbard_u, s.box, d["n"])
    assert np.max(np.abs(V - Vref)) < PREC[precision]["V"]


@pytest.mark.parametrize("precision", [0, 1, 4, 2])
def test_density_stages_and_charges(S, sysdata, precision):
    d = sysdata
    s = d["s"]
    R = np.ascontiguousarray(s.R)
    tol = PREC[precision]
    ctx = make_ctx(S, d, precision)
    try:
        S.sedacs_graph_build(ctx, R, gd=d["ref0"].gd)
        S.sedacs_partition(ctx, R)
        mu, q, eb, iters = S.sedacs_subgraph_density(ctx, R, d["n"], n_parts=8)
        ref = d["ref"]
        for i, sg in enumerate(ref.subs[:2]):
            h = S.sedacs_subgraph_matrix(ctx, i, 0)
            sm = S.sedacs_subgraph_matrix(ctx, i, 1)
            Z = S.sedacs_subgraph_matrix(ctx, i, 2)
            assert np.max(np.abs(h - sg.H)) < tol["hs"], "h"
            assert np.max(np.abs(sm - sg.S)) < tol["hs"], "s"
            assert np.max(np.abs(Z - sg.Z)) < tol["Z"], "Z"
        # mu of Eq. 2 solved by each side, charges, band energy
        info = S.sedacs_density_info(ctx)
        print(f"[parity] water96 form {precision}: mu {mu:.10f} vs {ref.mu:.10f} (|dmu| {abs(mu - ref.mu):.2e} Ha), "
              f"count - N_e {info['count_err']:.2e}, dN/dmu {info['dn_dmu']:.3e}, passes {info['passes']}, "
              f"doublings {info['doublings']}; oracle T->0 miss {ref.t0_miss:.3e} e, in-gap weight "
              f"{ref.in_gap_weight:.3f}")
        assert abs(mu - ref.mu) < tol["mu"]
        assert abs(info["count_err"]) < (1e-9 if precision == 0 else 1e-4)
        dq = np.max(np.abs(q - ref.q))
        print(f"[parity] water96 form {precision}: max|dq| = {dq:.3e} e")
        assert dq < tol["q"], f"charges differ by {dq}"
        assert abs(eb - ref.e_band) / 96 < tol["e"]
        assert np.all(iters == info["doublings"]) and info["doublings"] > 0
        # forces
        F = S.sedacs_forces(ctx, 96)
        Fref = odn.forces(ref, d["n"], s.R, s.species, s.box, d["m"])
        print(f"[parity] water96 form {precision}: max|dF| = {np.max(np.abs(F - Fref)):.3e} Ha/A")
        assert np.max(np.abs(F - Fref)) < tol["F"], f"forces differ by {np.max(np.abs(F - Fref))}"
        e = S.sedacs_energy(ctx)
        eref = odn.shadow_energy(ref, d["n"], s.R, s.species, s.box, d["m"])
        print(f"[parity] water96 form {precision}: |dE|/atom = {abs(e[3] - eref['total']) / 96:.3e} Ha")
        assert abs(e[3] - eref["total"]) / 96 < tol["e"]
        # density graph
        gp, gc, gv = S.sedacs_density_graph_get(ctx, 96)
        for I_ in (0, 17, 95):
            a = dict(zip(gc[gp[I_]:gp[I_ + 1]], gv[gp[I_]:gp[I_ + 1]]))
            b = dict(zip(ref.gd[1][ref.gd[0][I_]:ref.gd[0][I_ + 1]], ref.gd[2][ref.gd[0][I_]:ref.gd[0][I_ + 1]]))
            assert set(a) == set(b)
            # single elements of D carry the recursion's accumulated FP32 rounding (~1e-4 here) that
            # the charges, sums dominated by the diagonal, largely do not
            assert max(abs(a[k] - b[k]) for k in a) < {0: 1e-8, 1: 3e-4, 4: 3e-4, 2: 3e-3}[precision]
    finally:
        S.sedacs_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1, 4])
def test_t0_sp2_at_given_mu(S, sysdata, precision):
    """Te = 0: the mu-branch SP2 recursion at a chemical potential in the clean gap above the
    occupied band equals the 300 K Fermi density there (every level > 40 kT away)."""
    d = sysdata
    s = d["s"]
    R = np.ascontiguousarray(s.R)
    ref = d["ref"]
    e = np.concatenate([sg.eps for sg in ref.subs])
    top = np.max(e[e < ref.mu])
    bot = np.min(e[e > top + 0.05])
    mu_gap = 0.5 * (top + bot)
    ref_gap = odn.density(s.R, s.species, s.box, d["m"], d["n"], d["cores"], d["hal2"], mu=mu_gap)
    prm = S.sedacs_default_params(core_size=12, precision=precision, Te=0.0)
    ctx = S.sedacs_create(s.species, s.box, d["m"], prm)
    try:
        S.sedacs_graph_build(ctx, R, gd=d["ref0"].gd)
        S.sedacs_partition(ctx, R)
        with pytest.raises(S.SedacsError):
            S.sedacs_subgraph_density(ctx, R, d["n"])            # Te = 0 needs a given mu
        mu, q, eb, iters = S.sedacs_subgraph_density(ctx, R, d["n"], mu=mu_gap, n_parts=8)
    finally:
        S.sedacs_destroy(ctx)
    dq = np.max(np.abs(q - ref_gap.q))
    print(f"[parity] water96 T->0 SP2 form {precision} at mu {mu_gap:.4f} (gap {bot - top:.3f} Ha): max|dq| = {dq:.3e} e")
    assert mu == mu_gap and dq < (1e-8 if precision == 0 else 1e-5)
    assert np.all(iters > 0) and np.all(iters < 60)


@pytest.mark.parametrize("precision", [0, 1, 4])
def test_charge_response_and_krylov_kernel(S, sysdata, precision):
    """Canonical charge response (Fermi divided differences + the mu shift that keeps N_e) and the
    rank-4 Krylov kernel K f against the oracle's, on the same residual f = q - n (the oracle's)."""
    d = sysdata
    s = d["s"]
    R = np.ascontiguousarray(s.R)
    tol = PREC[precision]
    ctx = make_ctx(S, d, precision)
    try:
        S.sedacs_graph_build(ctx, R, gd=d["ref0"].gd)
        S.sedacs_partition(ctx, R)
        mu, q, eb, _ = S.sedacs_subgraph_density(ctx, R, d["n"])
        v = I.random_charges(96, 11, 1.0)
        dq = S.sedacs_charge_response(ctx, v)
        dq_ref = odyn.charge_response(d["ref"], v, s.R, s.species, s.box, d["m"])
        rel = np.max(np.abs(dq - dq_ref)) / np.max(np.abs(dq_ref))
        print(f"[parity] water96 form {precision}: response rel. error {rel:.2e}, sum {dq.sum():.1e}")
        assert rel < tol["rsp"], rel
        assert abs(dq.sum()) < 1e-6
        # Krylov kernel at full rank 4 on both sides
        f = np.ascontiguousarray(d["ref"].q - d["n"])
        S.sedacs_set_params(ctx, S.sedacs_default_params(core_size=12, precision=precision, kernel=1,
                                                          krylov_rank=4, krylov_tol=1e-14))
        S.sedacs_subgraph_density(ctx, R, d["n"])
        u, rank = S.sedacs_kernel_apply(ctx, f)
        u_ref, rank_ref = odyn.low_rank_kernel(s.R, s.species, s.box, d["m"], d["ref"], f, 0.5, 4, tol=1e-14)
        relk = np.max(np.abs(u - u_ref)) / np.max(np.abs(u_ref))
        print(f"[parity] water96 form {precision}: Krylov K f rank {rank}/{rank_ref}, rel. error {relk:.2e}")
        assert rank == rank_ref == 4 and relk < tol["kry"], relk
    finally:
        S.sedacs_destroy(ctx)
