"""Parity at the full size of the benchmark workload (9,000-atom water box), in the launch
configuration bench.py times (cores ~32 atoms, precision 1: Fermi-recursion products in two
fp16 planes, the other products three-way split bf16, on tcgen05; Te = 300 K).

Seeded nonzero trial charges with the periodic Coulomb potential.  The density graph is built
from the oracle's first density (on the distance graph's halos) and given to both sides, so
graph, cores and halos are compared bit for bit on the whole system.  Each side solves Eq. 2 for
its own chemical potential over all 281 subgraphs.  Compared: the charges of every atom, mu, the
collected electron count, the band and Coulomb energies of the whole system, and the forces on
the atoms of four sampled cores (the oracle evaluates the rows of those atoms only).

With these seeded trial charges mu lies inside a band (dN/dmu ~ 1,900 e/Ha, 76 levels within
2 kT).  Two effects of FP32-class arithmetic are tested apart:

* at the oracle's mu (mu passed as given), every atom's charge: FP32 accumulation in the
  recursion's products (which span the whole ~1 Ha spectrum) leaves ~1e-7 Ha of level noise, which
  moves an occupation near mu by beta f (1 - f) x 1e-7 ~ 3e-5; held to 1e-4 e per atom and 5e-6 e
  RMS.  The collected count then carries a systematic offset of ~1e-7 e per atom (measured
  1.0e-3 to 1.7e-3 e over the 9,000 atoms for two seeds; hydrogen -6e-7 e on average), held to
  4e-3 e.
* mu solved by each side (Eq. 2): the count offset becomes a mu offset of offset / (dN/dmu), at
  most 4e-3 / 1,900 ~ 2.1e-6 Ha, which moves the atoms holding a level within kT of mu by up to
  beta / 4 x 2.1e-6 ~ 5.5e-4 e; so mu is held to 2.5e-6 Ha, those atoms to 6e-4 e and the RMS
  over all atoms to 1e-5 e.

The oracle's subgraph eigensolves take its LAPACK route here (562 solves of ~500 orbitals; the
plain-C Jacobi route agrees with it to ~1e-13 on the eigenvalues and 1e-11 e on the charges, and
would take minutes at this size).

The plain FP64 form is held to 5e-9 e on every atom: its recursion's inverse polynomial (degree 15,
fit error 8.2e-13) errs by that much at each doubling, and a level at mu carries the error of the
first doubling amplified by 2^n (n = 11 here), ~1.7e-9 in its occupation.
"""
import numpy as np
import pytest

from oracle import density as odn
from oracle import ewald as oew
from oracle import graph as og
from paper_2606_03140_gb300 import inputs as I

pytestmark = pytest.mark.gpu

PICK = [0, 97, 180, 280]


@pytest.fixture(scope="module")
def full():
    from paper_2606_03140_gb300 import sedacs as S

    s = I.workload("water9000")
    m = I.default_model()
    N = s.n_atoms
    n = I.random_charges(N, 7, 0.05)
    V = oew.coulomb_potential(s.R, s.species, m.hubbard_u, s.box, n)
    rp0, col0 = og.build_graph(s.R, s.box, 3.0)
    cores = og.rcb_partition(s.R, s.box, 32)
    r0 = odn.density(s.R, s.species, s.box, m, n, cores, og.halos(rp0, col0, cores), V=V, eig="lapack")
    rp1, col1 = og.build_graph(s.R, s.box, 3.0, r0.gd, 1e-3)
    hal1 = og.halos(rp1, col1, cores)
    ref = odn.density(s.R, s.species, s.box, m, n, cores, hal1, V=V, eig="lapack")
    atoms = np.concatenate([cores[i] for i in PICK])
    Fref = odn.forces(ref, n, s.R, s.species, s.box, m, atoms=atoms)
    R = np.ascontiguousarray(s.R)
    ctx = S.sedacs_create(s.species, s.box, m, S.sedacs_default_params(core_size=32, precision=1))
    try:
        nnz = S.sedacs_graph_build(ctx, R)
        g0 = S.sedacs_graph_get(ctx, N, nnz)
        S.sedacs_partition(ctx, R)
        nnz = S.sedacs_graph_build(ctx, R, gd=r0.gd)
        g1 = S.sedacs_graph_get(ctx, N, nnz)
        sp, sa, nc = S.sedacs_parts_get(ctx)
        mu, q, eb, iters = S.sedacs_subgraph_density(ctx, R, n, n_parts=len(nc))
        info = S.sedacs_density_info(ctx)
        F = S.sedacs_forces(ctx, N)
        e = S.sedacs_energy(ctx)
        # the same context at the oracle's mu, taken as given
        prm = S.sedacs_default_params(core_size=32, precision=1, mu_given=1)
        S.sedacs_set_params(ctx, prm)
        _, q_at, _, _ = S.sedacs_subgraph_density(ctx, R, n, mu=float(ref.mu))
        info_at = S.sedacs_density_info(ctx)
    finally:
        S.sedacs_destroy(ctx)
    # the plain FP64 form on the same graph
    ctx = S.sedacs_create(s.species, s.box, m, S.sedacs_default_params(core_size=32, precision=0))
    try:
        S.sedacs_graph_build(ctx, R)
        S.sedacs_partition(ctx, R)
        S.sedacs_graph_build(ctx, R, gd=r0.gd)
        mu64, q64, eb64, _ = S.sedacs_subgraph_density(ctx, R, n)
        F64 = S.sedacs_forces(ctx, N)
    finally:
        S.sedacs_destroy(ctx)
    return dict(s=s, m=m, n=n, V=V, g0=g0, g1=g1, rp0=rp0, col0=col0, rp1=rp1, col1=col1, cores=cores,
                hal1=hal1, sp=sp, sa=sa, nc=nc, mu=mu, q=q, eb=eb, info=info, F=F, e=e, ref=ref, atoms=atoms,
                Fref=Fref, mu64=mu64, q64=q64, eb64=eb64, F64=F64, q_at=q_at, info_at=info_at)


def test_graph_cores_halos_bit_exact_full_size(full):
    assert np.array_equal(full["g0"][0], full["rp0"]) and np.array_equal(full["g0"][1], full["col0"])
    assert np.array_equal(full["g1"][0], full["rp1"]) and np.array_equal(full["g1"][1], full["col1"])
    sp, sa, nc = full["sp"], full["sa"], full["nc"]
    cores, hal = full["cores"], full["hal1"]
    assert len(cores) == len(nc) == 281
    for i in range(len(cores)):
        assert np.array_equal(sa[sp[i]:sp[i] + nc[i]], cores[i])
        assert np.array_equal(sa[sp[i] + nc[i]:sp[i + 1]], hal[i])


def test_charges_at_oracle_mu_full_size(full):
    ref = full["ref"]
    dq = full["q_at"] - ref.q
    off = full["info_at"]["count_err"]
    print(f"[parity] water9000 form 1 at the oracle's mu: max|dq| {np.max(np.abs(dq)):.3e} e, RMS "
          f"{np.sqrt(np.mean(dq ** 2)):.2e} e, count offset {off:+.3e} e ({off / len(dq):+.1e} e per atom)")
    assert np.max(np.abs(dq)) < 1e-4
    assert np.sqrt(np.mean(dq ** 2)) < 5e-6
    assert abs(off) < 4e-3
    assert abs(float(np.sum(dq)) - off) < 1e-6


def test_mu_count_charges_energies_full_size(full):
    ref, info = full["ref"], full["info"]
    N = full["s"].n_atoms
    dq = np.max(np.abs(full["q"] - ref.q))
    print(f"[parity] water9000 form 1: mu {full['mu']:.9f} vs {ref.mu:.9f} (|dmu| {abs(full['mu'] - ref.mu):.2e} Ha), "
          f"count - N_e {info['count_err']:.2e} e, dN/dmu {info['dn_dmu']:.1f} e/Ha, passes {info['passes']}, "
          f"doublings {info['doublings']}; oracle T->0 miss {ref.t0_miss:.3f} e, in-gap weight "
          f"{ref.in_gap_weight:.2f}; max|dq| over all {N} atoms = {dq:.3e} e, RMS "
          f"{np.sqrt(np.mean((full['q'] - ref.q) ** 2)):.2e} e, atoms above 1e-5 e: "
          f"{int(np.sum(np.abs(full['q'] - ref.q) > 1e-5))}")
    assert dq < 6e-4, dq
    assert np.sqrt(np.mean((full["q"] - ref.q) ** 2)) < 1e-5
    assert abs(full["mu"] - ref.mu) < 2.5e-6
    assert abs(info["count_err"]) < 1e-3
    assert abs(full["q"].sum()) < 1e-3
    deb = abs(full["eb"] - ref.e_band) / N
    ecoul_ref = float(np.dot(ref.q - 0.5 * full["n"], full["V"]))
    dec = abs(full["e"][1] - ecoul_ref) / N
    print(f"[parity] water9000 form 1: |dE_band|/atom = {deb:.2e} Ha, |dE_coul|/atom = {dec:.2e} Ha")
    assert deb < 1e-5 and dec < 1e-5


def test_sampled_forces_full_size(full):
    a = full["atoms"]
    dF = np.max(np.abs(full["F"][a] - full["Fref"][a]))
    print(f"[parity] water9000 form 1: max|dF| on {len(a)} atoms of sampled cores = {dF:.3e} Ha/A")
    assert dF < 2e-4, dF
    assert np.all(np.isfinite(full["F"]))


def test_plain_fp64_form_full_size(full):
    ref = full["ref"]
    a = full["atoms"]
    dq = np.max(np.abs(full["q64"] - ref.q))
    dF = np.max(np.abs(full["F64"][a] - full["Fref"][a]))
    print(f"[parity] water9000 FP64 form: |dmu| {abs(full['mu64'] - ref.mu):.2e} Ha, max|dq| {dq:.2e} e, "
          f"|dE_band|/atom {abs(full['eb64'] - ref.e_band) / len(ref.q):.2e} Ha, max|dF| (sampled) {dF:.2e} Ha/A")
    assert dq < 5e-9 and dF < 1e-8 and abs(full["mu64"] - ref.mu) < 1e-9
