"""Pins of the oracle's model layer (SK blocks, Ewald) against closed forms and invariants."""
import math

import numpy as np
import pytest

from oracle import BOHR_A, ewald, sk
from paper_2606_03140_gb300 import inputs as I


def test_sk_gradient_matches_finite_difference():
    m = I.SKModel()
    rng = np.random.default_rng(1)
    d = rng.uniform(-3, 3, size=(6, 3))
    d[0] = [0.5, 5.4, 0.3]                       # inside the switching region
    si = np.array([2, 2, 0, 1, 0, 2])
    sj = np.array([0, 2, 0, 2, 1, 1])
    for scale in (1.0, m.overlap_scale):
        B, dB = sk.pair_blocks(m, si, sj, d, scale=scale, with_grad=True)
        h = 1e-6
        for c in range(3):
            dp = d.copy(); dp[:, c] += h
            dm = d.copy(); dm[:, c] -= h
            fd = (sk.pair_blocks(m, si, sj, dp, scale=scale) - sk.pair_blocks(m, si, sj, dm, scale=scale)) / (2 * h)
            assert np.max(np.abs(fd - dB[:, c])) < 1e-8


def test_sk_block_transpose_symmetry():
    # H[i,j](d) = H[j,i](-d)^T : the global matrix is symmetric
    m = I.SKModel()
    d = np.array([[1.1, -0.4, 0.7]])
    Bij = sk.pair_blocks(m, np.array([2]), np.array([1]), d)
    Bji = sk.pair_blocks(m, np.array([1]), np.array([2]), -d)
    assert np.max(np.abs(Bij[0] - Bji[0].T)) < 1e-15


def test_h2_dimer_closed_form():
    # two s orbitals: generalised eigenvalues (eps +- V) / (1 +- s)
    m = I.SKModel()
    r = 1.3
    R = np.array([[5.0, 5.0, 5.0], [5.0 + r, 5.0, 5.0]])
    H, S, _, _ = sk.hs_blocks_for_atoms(np.arange(2), R, np.array([0, 0]), np.array([30.0] * 3), m)
    v = m.v0[0][0][0] * math.exp(-r / m.decay)
    s = m.overlap_scale * v
    eps = m.eps_s[0]
    from scipy.linalg import eigh
    ev = eigh(H, S, eigvals_only=True)
    ref = sorted([(eps + v) / (1 + s), (eps - v) / (1 - s)])
    assert np.allclose(ev, ref, atol=1e-14)


def test_rotation_invariance_of_molecule_spectrum():
    m = I.SKModel()
    sp, pos = I._methanol_template()
    box = np.array([40.0] * 3)
    R0 = pos + 20.0
    rng = np.random.default_rng(3)
    Q = I._random_rotation(rng)
    R1 = (pos @ Q.T) + 20.0
    from scipy.linalg import eigh
    e = []
    for R in (R0, R1):
        H, S, _, _ = sk.hs_blocks_for_atoms(np.arange(len(sp)), R, sp, box, m)
        assert np.max(np.abs(H - H.T)) == 0.0
        e.append(eigh(H, S, eigvals_only=True))
    assert np.max(np.abs(e[0] - e[1])) < 1e-13


def test_ewald_eta_independence_and_symmetry():
    m = I.SKModel()
    s = I.workload("water96")
    g1 = ewald.gamma_matrix(s.R, s.species, m.hubbard_u, s.box)
    g2 = ewald.gamma_matrix(s.R, s.species, m.hubbard_u, s.box, eta=0.2)
    assert np.max(np.abs(g1 - g1.T)) < 1e-14
    assert np.max(np.abs(g1 - g2)) < 1e-10


def test_ewald_nacl_madelung():
    a0 = BOHR_A                       # nearest-neighbour distance 1 bohr
    pos, q = [], []
    for i in range(2):
        for j in range(2):
            for k in range(2):
                pos.append([i * a0, j * a0, k * a0])
                q.append((-1.0) ** (i + j + k))
    pos, q = np.array(pos), np.array(q)
    U = (1e3, 1e3, 1e3)               # point-charge limit; remove the on-site U q term
    V = ewald.coulomb_potential(pos, np.full(8, 2), U, np.array([2 * a0] * 3), q)
    mad = -(V - 1e3 * q) / q
    assert np.allclose(mad, 1.747564594633, atol=1e-9)


def test_gaussian_self_and_pair_in_large_box():
    # gamma_II(0) = U_I and gamma_IJ -> erf(a r)/r, both shifted by the cubic-box
    # point-charge self term -2.837297/L of the neutralising background
    from scipy.special import erf
    m = I.SKModel()
    L = 120.0
    R = np.array([[0.0, 0.0, 0.0], [3.0, 0.0, 0.0]])
    g = ewald.gamma_matrix(R, np.array([2, 0]), m.hubbard_u, np.array([L] * 3))
    shift = -2.837297479 / (L / BOHR_A)
    a = 1.0 / math.sqrt(2 * ((1 / (math.sqrt(math.pi) * 0.5)) ** 2 + (1 / (math.sqrt(math.pi) * 0.4)) ** 2))
    r = 3.0 / BOHR_A
    assert abs(g[0, 0] - (0.5 + shift)) < 5e-5
    assert abs(g[1, 1] - (0.4 + shift)) < 5e-5
    assert abs(g[0, 1] - (erf(a * r) / r + shift)) < 5e-5


def test_ewald_gradient_finite_difference():
    m = I.SKModel()
    s = I.workload("water96")
    n = I.random_charges(96, 1)
    a = n + 0.01
    G = ewald.coulomb_gradient(s.R, s.species, m.hubbard_u, s.box, a, n)
    h = 1e-4
    for A, c in [(0, 0), (5, 1), (40, 2)]:
        Rp = s.R.copy(); Rp[A, c] += h
        Rm = s.R.copy(); Rm[A, c] -= h
        fd = (a @ ewald.coulomb_potential(Rp, s.species, m.hubbard_u, s.box, n)
              - a @ ewald.coulomb_potential(Rm, s.species, m.hubbard_u, s.box, n)) / (2 * h)
        assert abs(fd - G[A, c]) < 1e-8


def _dimer_model():
    # distinct constants per bond type and, for sp sigma, per ordered element pair (s on i, p on j),
    # so that a swapped pp sigma / pp pi, a swapped s-on-i / s-on-j constant or a flipped sign all show
    v0 = [[[0.0] * 4 for _ in range(3)] for _ in range(3)]
    for i in range(3):
        for j in range(3):
            v0[i][j] = [-1.1 - 0.05 * (i + j), 1.3 + 0.2 * i + 0.05 * j, 1.7 + 0.03 * (i + j), -0.45 - 0.02 * (i + j)]
    return I.SKModel(v0=tuple(tuple(tuple(x) for x in row) for row in v0))


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_aligned_dimer_closed_form_blocks(axis):
    """Slater-Koster table for a pair on a Cartesian axis (Slater & Koster 1954): with the
    bond along +e_a (atom 1 - atom 0), H[s0, s1] = V_ss, H[s0, p_a1] = +V_sp(s on 0),
    H[p_a0, s1] = -V_sp(s on 1), H[p_a0, p_a1] = V_pp sigma, H[p_b0, p_b1] = V_pp pi (b != a),
    every other entry of the block zero; S the same with the overlap scale."""
    m = _dimer_model()
    r = 1.9
    sp = np.array([2, 1])          # O at R0, C at R1
    R = np.array([[7.0, 7.0, 7.0], [7.0, 7.0, 7.0]])
    R[1, axis] += r
    H, S, norb, off = sk.hs_blocks_for_atoms(np.arange(2), R, sp, np.array([30.0] * 3), m)
    g = math.exp(-r / m.decay)
    for M, scale in ((H, 1.0), (S, m.overlap_scale)):
        v = lambda a, b, X: scale * m.v0[a][b][X] * g
        blk = M[0:4, 4:8]
        ref = np.zeros((4, 4))
        ref[0, 0] = v(2, 1, 0)
        ref[0, 1 + axis] = v(2, 1, 1)          # s on O (atom 0), p on C
        ref[1 + axis, 0] = -v(1, 2, 1)         # s on C (atom 1), p on O
        for b in range(3):
            ref[1 + b, 1 + b] = v(2, 1, 2) if b == axis else v(2, 1, 3)
        assert np.max(np.abs(blk - ref)) < 1e-14
        assert np.max(np.abs(M[4:8, 0:4] - ref.T)) < 1e-14
    # on-site diagonal and unit overlap diagonal
    assert np.allclose(np.diag(H), [m.eps_s[2]] + [m.eps_p[2]] * 3 + [m.eps_s[1]] + [m.eps_p[1]] * 3, atol=0)
    assert np.allclose(np.diag(S), 1.0, atol=0)
    # reversing the bond direction flips only the s-p entries
    R2 = R.copy()
    R2[1, axis] -= 2 * r
    H2, _, _, _ = sk.hs_blocks_for_atoms(np.arange(2), R2, sp, np.array([30.0] * 3), m)
    flip = np.ones((4, 4))
    flip[0, 1:] = -1.0
    flip[1:, 0] = -1.0
    assert np.max(np.abs(H2[0:4, 4:8] - flip * H[0:4, 4:8])) < 1e-14
