"""GPU parity against the FP64 oracle on the 96-atom water box (32 H2O, 9.86 A), every stage.

All calls go through the C ABI.  Tolerances: bit-exact for graph / partition / halos;
FP64 plain form ~1e-9; FP32-class forms (1: two-plane fp16 SP2, 4: three-plane bf16 SP2)
1e-5 e on charges; mixed BF16 form 3e-4 e;
energies 1e-5 Ha/atom (the stated accuracy targets of the mixed / plain comparison).
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
PREC = {0: dict(q=1e-8, V=1e-9, hs=1e-12, Z=1e-9, F=1e-7, e=1e-8),
        1: dict(q=1e-5, V=1e-6, hs=1e-6, Z=1e-5, F=1e-5, e=1e-5),
        2: dict(q=3e-4, V=1e-6, hs=1e-6, Z=1e-5, F=5e-4, e=1e-4)}
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
        # mu in the same gap, charges, band energy
        eps = np.concatenate([sg.eps for sg in ref.subs])
        w = np.concatenate([sg.w for sg in ref.subs])
        mu_o, eh, el = odn.solve_mu([sg.eps for sg in ref.subs], [sg.w for sg in ref.subs], 256.0)
        assert eh < mu < el
        dq = np.max(np.abs(q - ref.q))
        print(f"[parity] water96 form {precision}: max|dq| = {dq:.3e} e")
        assert dq < tol["q"], f"charges differ by {dq}"
        assert abs(eb - ref.e_band) / 96 < tol["e"]
        assert np.all(iters > 0) and np.all(iters < 60)
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
            assert max(abs(a[k] - b[k]) for k in a) < max(tol["q"], 1e-6)
    finally:
        S.sedacs_destroy(ctx)


@pytest.mark.parametrize("precision", [0, 1, 4])
def test_charge_response_and_krylov_kernel(S, sysdata, precision):
    d = sysdata
    s = d["s"]
    R = np.ascontiguousarray(s.R)
    ctx = make_ctx(S, d, precision)
    try:
        S.sedacs_graph_build(ctx, R, gd=d["ref0"].gd)
        S.sedacs_partition(ctx, R)
        mu, q, eb, _ = S.sedacs_subgraph_density(ctx, R, d["n"])
        v = I.random_charges(96, 11, 1.0)
        dq = S.sedacs_charge_response(ctx, v)
        dq_ref = odyn.charge_response(d["ref"], v, s.R, s.species, s.box, d["m"])
        rel = np.max(np.abs(dq - dq_ref)) / np.max(np.abs(dq_ref))
        assert rel < (1e-6 if precision == 0 else 1e-3), rel
    finally:
        S.sedacs_destroy(ctx)
