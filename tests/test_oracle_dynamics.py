"""Pins of the oracle's SCC, response, Krylov kernel and XL-BOMD integrator."""
import numpy as np
import pytest

from oracle import density as dn
from oracle import dynamics as dyn
from oracle import graph
from paper_2606_03140_gb300 import inputs as I


@pytest.fixture(scope="module")
def tiny():
    s = I.small_water_box(4, 6.5, seed=21)
    return s, I.default_model(), dyn.GraphParams(r_graph=3.0, tau=1e-3, core_size=3)


def test_scc_fixed_point_independent_of_mixer(tiny):
    s, m, gp = tiny
    n1, r1, it1, _ = dyn.scc(s.R, s.species, s.box, m, gp, tol=1e-9)
    n2, r2, it2, _ = dyn.scc(s.R, s.species, s.box, m, gp, tol=1e-9, krylov_rank=4)
    n3, _, _, _ = dyn.scc(s.R, s.species, s.box, m, gp, tol=1e-9, alpha=0.4, n0=np.full(12, 0.01))
    assert np.max(np.abs(n1 - n2)) < 1e-8 and np.max(np.abs(n1 - n3)) < 1e-8
    assert it2 < it1


def test_charge_response_equals_finite_difference(tiny):
    s, m, gp = tiny
    n = I.random_charges(12, 4, 0.03)
    cores = graph.rcb_partition(s.R, s.box, 3)
    _, _, hal = dyn.graph_and_halos(s.R, s.box, gp, cores, None)
    r0 = dn.density(s.R, s.species, s.box, m, n, cores, hal)
    v = I.random_charges(12, 5, 1.0)
    e = 1e-4
    # at fixed mu
    dq = dyn.charge_response(r0, v, s.R, s.species, s.box, m, canonical=False)
    qp = dn.density(s.R, s.species, s.box, m, n + e * v, cores, hal, mu=r0.mu).q
    qm = dn.density(s.R, s.species, s.box, m, n - e * v, cores, hal, mu=r0.mu).q
    assert np.max(np.abs(dq - (qp - qm) / (2 * e))) < 1e-7
    # canonical: mu solved again from Eq. 2 on both sides of the difference
    dqc = dyn.charge_response(r0, v, s.R, s.species, s.box, m)
    qp = dn.density(s.R, s.species, s.box, m, n + e * v, cores, hal).q
    qm = dn.density(s.R, s.species, s.box, m, n - e * v, cores, hal).q
    assert np.max(np.abs(dqc - (qp - qm) / (2 * e))) < 1e-7
    assert abs(dqc.sum()) < 1e-10


def test_full_rank_krylov_equals_dense_inverse_jacobian(tiny):
    s, m, gp = tiny
    cores = graph.rcb_partition(s.R, s.box, 3)
    n = I.random_charges(12, 6, 0.03)
    _, _, hal = dyn.graph_and_halos(s.R, s.box, gp, cores, None)
    r0 = dn.density(s.R, s.species, s.box, m, n, cores, hal)
    J = np.zeros((12, 12))
    e = 1e-5
    for j in range(12):
        ej = np.zeros(12); ej[j] = e
        qp = dn.density(s.R, s.species, s.box, m, n + ej, cores, hal).q
        qm = dn.density(s.R, s.species, s.box, m, n - ej, cores, hal).q
        J[:, j] = (qp - qm) / (2 * e)
    J -= np.eye(12)
    f = r0.q - n
    u, rank = dyn.low_rank_kernel(s.R, s.species, s.box, m, r0, f, 0.5, 12, tol=1e-13)
    assert np.max(np.abs(u - np.linalg.solve(J, f))) < 1e-6 * np.max(np.abs(np.linalg.solve(J, f)))


def test_xlbomd_energy_fluctuation_scales_dt2(tiny):
    """Sec. "Dynamic Graph Adaption": amplitude ~x4 per doubling of dt, no drift."""
    s, m, gp = tiny
    v = I.maxwell_boltzmann(s.species, 300.0, 9, m)
    amp = []
    for dt in (0.4, 0.2):
        o = dyn.xlbomd(s.R, v, s.species, s.box, m, gp, int(round(12.0 / dt)), dt)
        E = o["energies"][:, 2]
        amp.append(E.max() - E.min())
    assert 2.5 < amp[0] / amp[1] < 6.5
