"""The finite-temperature path at 10,000 K (the paper's hot-electron runs, Sec. "Dynamic Graph
Adaption") through the C ABI against the oracle, 96-atom water box.

At Te = 10,000 K (kT = 0.032 Ha) the Fermi tails cover many levels: the recursion starts at
2^n Te with n ~ 5, mu of Eq. 2 sits where dN/dmu is large, and the electronic entropy term
-Te S of the shadow energy is no longer negligible.  Charges, mu, band and total (free) energy
and forces are compared with each side solving Eq. 2; the FP32-class form is held to the same
bounds as at 300 K (its level noise of ~1e-7 Ha moves occupations by beta f (1 - f) x 1e-7,
smaller here).
"""
import numpy as np
import pytest

from oracle import density as odn
from oracle import graph as og
from paper_2606_03140_gb300 import inputs as I

pytestmark = pytest.mark.gpu

TE = 10000.0
TOL = {0: dict(q=1e-8, mu=1e-8, e=1e-8, F=1e-7), 1: dict(q=2e-5, mu=5e-5, e=1e-5, F=2e-5)}


@pytest.fixture(scope="module")
def hot():
    s = I.workload("water96")
    m = I.default_model()
    n = I.random_charges(96, 3, 0.05)
    rp, col = og.build_graph(s.R, s.box, 3.0)
    cores = og.rcb_partition(s.R, s.box, 12)
    r0 = odn.density(s.R, s.species, s.box, m, n, cores, og.halos(rp, col, cores), Te=TE)
    rp2, col2 = og.build_graph(s.R, s.box, 3.0, r0.gd, 1e-3)
    ref = odn.density(s.R, s.species, s.box, m, n, cores, og.halos(rp2, col2, cores), Te=TE)
    return s, m, n, r0, ref


@pytest.mark.parametrize("precision", [0, 1])
def test_density_energy_forces_at_10000K(hot, precision):
    from paper_2606_03140_gb300 import sedacs as S

    s, m, n, r0, ref = hot
    tol = TOL[precision]
    prm = S.sedacs_default_params(core_size=12, precision=precision, Te=TE)
    ctx = S.sedacs_create(s.species, s.box, m, prm)
    try:
        R = np.ascontiguousarray(s.R)
        S.sedacs_graph_build(ctx, R)
        S.sedacs_partition(ctx, R)
        S.sedacs_graph_build(ctx, R, gd=r0.gd)
        mu, q, eb, _ = S.sedacs_subgraph_density(ctx, R, np.ascontiguousarray(n))
        info = S.sedacs_density_info(ctx)
        F = S.sedacs_forces(ctx, 96)
        e = S.sedacs_energy(ctx)
    finally:
        S.sedacs_destroy(ctx)
    eref = odn.shadow_energy(ref, n, s.R, s.species, s.box, m)
    Fref = odn.forces(ref, n, s.R, s.species, s.box, m)
    dq = float(np.max(np.abs(q - ref.q)))
    dF = float(np.max(np.abs(F - Fref)))
    dE = abs(e[3] - eref["total"]) / 96
    print(f"[parity] water96 at 10,000 K, form {precision}: |dmu| {abs(mu - ref.mu):.2e} Ha, max|dq| {dq:.2e} e, "
          f"|dE_free|/atom {dE:.2e} Ha (-TS {eref['ts_entropy'] / 96:.2e} Ha/atom), max|dF| {dF:.2e} Ha/A, "
          f"doublings {info['doublings']}, passes {info['passes']}")
    assert abs(mu - ref.mu) < tol["mu"]
    assert dq < tol["q"] and dF < tol["F"] and dE < tol["e"]
    assert abs(eb - ref.e_band) / 96 < tol["e"]
