"""Periodic Gaussian-gamma Coulomb interaction by Ewald summation (FP64 oracle).

Test infrastructure only (see ``oracle/__init__``).

SCC-DFTB couples net Mulliken charges through a screened Coulomb interaction
that decays as 1/|R_I - R_J| at long range and is screened at short range, with
the on-site value set by the Hubbard U (SI Sec. "Implementation with SCC-DFTB
theory").  The synthetic model uses Gaussian charge clouds of width
sigma_I = 1 / (sqrt(pi) U_I):

    gamma_IJ(r) = erf(a_IJ r) / r,  a_IJ = 1 / sqrt(2 (sigma_I^2 + sigma_J^2)),
    gamma_II(0) = U_I.

The periodic matrix sums gamma over all images.  Writing erf(a r)/r = 1/r -
erfc(a r)/r and summing 1/r by Ewald's method (with a neutralising background):

    gamma_IJ = sum_L' [erfc(eta d) - erfc(a_IJ d)] / d                 (d = |R_J - R_I + L|)
             + (4 pi / V) sum_{k != 0} exp(-k^2 / 4 eta^2) / k^2 cos(k . (R_J - R_I))
             - pi / (eta^2 V)
             + delta_IJ (U_I - 2 eta / sqrt(pi))

(the primed sum omits d = 0).  Internal units bohr / Hartree; positions come in
Angstrom.  Pinned by tests against: eta independence, gamma_II(0) = U_I for an
isolated Gaussian in a large box, the NaCl Madelung constant 1.747565 in the
point-charge limit, and a finite-difference gradient.
"""
from __future__ import annotations

import math

import numpy as np
from scipy.special import erfc

from . import BOHR_A


def ewald_parameters(box_bohr: np.ndarray, rc_bohr: float | None = None, tol: float = 1e-12):
    """Splitting eta, real-space cutoff and reciprocal cutoff for relative accuracy ~tol."""
    x = math.sqrt(-math.log(tol))          # exp(-x^2) ~ tol
    if rc_bohr is None:
        rc_bohr = 10.0 / BOHR_A
    eta = (x + 0.3) / rc_bohr              # erfc(eta rc) ~ tol
    kmax = 2.0 * eta * x                   # exp(-k^2 / 4 eta^2) ~ tol
    return eta, rc_bohr, kmax


def _kvectors(box_bohr: np.ndarray, kmax: float):
    """Half-space reciprocal vectors 0 < |k| <= kmax (one of each +-k pair)."""
    nmax = [int(math.floor(kmax * L / (2 * math.pi))) for L in box_bohr]
    g = [np.arange(-n, n + 1) for n in nmax]
    ii, jj, kk = np.meshgrid(*g, indexing="ij")
    m = np.stack([ii.ravel(), jj.ravel(), kk.ravel()], axis=1)
    # half space: first nonzero component positive
    half = (m[:, 0] > 0) | ((m[:, 0] == 0) & (m[:, 1] > 0)) | ((m[:, 0] == 0) & (m[:, 1] == 0) & (m[:, 2] > 0))
    m = m[half]
    k = m * (2 * math.pi / box_bohr)[None, :]
    k2 = np.sum(k * k, axis=1)
    keep = k2 <= kmax * kmax
    return k[keep], k2[keep]


def _a_matrix(species_i, species_j, hubbard_u):
    u = np.asarray(hubbard_u, dtype=np.float64)
    sig_i = 1.0 / (math.sqrt(math.pi) * u[species_i])
    sig_j = 1.0 / (math.sqrt(math.pi) * u[species_j])
    return 1.0 / np.sqrt(2.0 * (sig_i[:, None] ** 2 + sig_j[None, :] ** 2))


def coulomb_potential(R_A, species, hubbard_u, box_A, b, eta=None, rc_bohr=None, chunk=256, rows=None):
    """V = gamma @ b (b shape [N] or [N, m]); Hartree per unit charge.  Plain Ewald sums.

    rows: evaluate V only at these atoms (the other entries stay 0); the sums run over every atom."""
    R = np.asarray(R_A, dtype=np.float64) / BOHR_A
    box = np.asarray(box_A, dtype=np.float64) / BOHR_A
    b = np.asarray(b, dtype=np.float64)
    vec = b.ndim == 1
    B = b[:, None] if vec else b
    N = R.shape[0]
    e0, rc, kmax = ewald_parameters(box, rc_bohr)
    if eta is None:
        eta = e0
    else:
        rc = (math.sqrt(-math.log(1e-12)) + 0.3) / eta
        kmax = 2.0 * eta * math.sqrt(-math.log(1e-12))
    vol = float(np.prod(box))
    u = np.asarray(hubbard_u, dtype=np.float64)
    V = np.zeros_like(B)
    rows = np.arange(N) if rows is None else np.asarray(rows, dtype=np.int64)
    # real space, every image within rc (I = J, L = 0 excluded)
    nimg = [int(math.floor((rc + 0.5 * L) / L)) for L in box]
    shifts = np.array([[i, j, k] for i in range(-nimg[0], nimg[0] + 1)
                       for j in range(-nimg[1], nimg[1] + 1)
                       for k in range(-nimg[2], nimg[2] + 1)], dtype=np.float64) * box
    for s in range(0, rows.shape[0], chunk):
        I = rows[s:s + chunk]
        a = _a_matrix(species[I], species, u)
        d0 = R[None, :, :] - R[I, None, :]
        d0 -= box * np.round(d0 / box)
        phi = np.zeros((I.shape[0], N))
        for L in shifts:
            d = np.sqrt(np.sum((d0 + L) ** 2, axis=2))
            ok = (d < rc) & (d > 0.0)
            dd = np.where(ok, d, 1.0)
            phi += np.where(ok, (erfc(eta * dd) - erfc(a * dd)) / dd, 0.0)
        V[I] += phi @ B
    # reciprocal space (+-k pairs: factor 2)
    k, k2 = _kvectors(box, kmax)
    w = 2.0 * (4.0 * math.pi / vol) * np.exp(-k2 / (4.0 * eta * eta)) / k2
    for s in range(0, k.shape[0], 2048):
        kk = k[s:s + 2048]
        ph = R @ kk.T                                   # [N, nk]
        c, sn = np.cos(ph), np.sin(ph)
        Sc = c.T @ B                                    # [nk, m]  Re S(k)
        Ss = sn.T @ B                                   # [nk, m]  Im S(k)
        ww = w[s:s + 2048][:, None]
        V[rows] += c[rows] @ (ww * Sc) + sn[rows] @ (ww * Ss)
    # background and self terms
    V[rows] += -math.pi / (eta * eta * vol) * B.sum(axis=0)[None, :]
    V[rows] += (u[species[rows]] - 2.0 * eta / math.sqrt(math.pi))[:, None] * B[rows]
    return V[:, 0] if vec else V


def gamma_matrix(R_A, species, hubbard_u, box_A, eta=None):
    """Dense periodic gamma (N x N), Hartree; column J = potential of a unit charge on J."""
    N = R_A.shape[0]
    return coulomb_potential(R_A, species, hubbard_u, box_A, np.eye(N), eta=eta)


def coulomb_gradient(R_A, species, hubbard_u, box_A, a_vec, b_vec, chunk=256, rows=None):
    """d/dR_A of E = sum_IJ a_I gamma_IJ b_J for every atom A (or the atoms in rows), in Hartree / Angstrom.

    Real space: dE/dR_A = -sum_{J,L'} (a_A b_J + a_J b_A) phi'(d) d_hat, d = R_J - R_A + L;
    reciprocal: (4 pi / V) sum_k w(k) k [a_A Im(S_b e^{-ik.R_A}) + b_A Im(S_a e^{-ik.R_A})].
    """
    R = np.asarray(R_A, dtype=np.float64) / BOHR_A
    box = np.asarray(box_A, dtype=np.float64) / BOHR_A
    a_vec = np.asarray(a_vec, dtype=np.float64)
    b_vec = np.asarray(b_vec, dtype=np.float64)
    N = R.shape[0]
    eta, rc, kmax = ewald_parameters(box)
    vol = float(np.prod(box))
    u = np.asarray(hubbard_u, dtype=np.float64)
    G = np.zeros((N, 3))
    rows = np.arange(N) if rows is None else np.asarray(rows, dtype=np.int64)
    nimg = [int(math.floor((rc + 0.5 * L) / L)) for L in box]
    shifts = np.array([[i, j, k] for i in range(-nimg[0], nimg[0] + 1)
                       for j in range(-nimg[1], nimg[1] + 1)
                       for k in range(-nimg[2], nimg[2] + 1)], dtype=np.float64) * box
    sq = 2.0 / math.sqrt(math.pi)
    for s in range(0, rows.shape[0], chunk):
        I = rows[s:s + chunk]
        a = _a_matrix(species[I], species, u)
        coef = a_vec[I, None] * b_vec[None, :] + a_vec[None, :] * b_vec[I, None]
        d0 = R[None, :, :] - R[I, None, :]
        d0 -= box * np.round(d0 / box)
        for L in shifts:
            dv = d0 + L
            d = np.sqrt(np.sum(dv * dv, axis=2))
            ok = (d < rc) & (d > 0.0)
            dd = np.where(ok, d, 1.0)
            dphi = (-sq * eta * np.exp(-(eta * dd) ** 2) + sq * a * np.exp(-(a * dd) ** 2)) / dd \
                - (erfc(eta * dd) - erfc(a * dd)) / (dd * dd)
            fac = np.where(ok, coef * dphi / dd, 0.0)     # times d vector gives phi' d_hat
            G[I] -= np.einsum("ij,ijk->ik", fac, dv)
    k, k2 = _kvectors(box, kmax)
    w = 2.0 * (4.0 * math.pi / vol) * np.exp(-k2 / (4.0 * eta * eta)) / k2
    for s in range(0, k.shape[0], 2048):
        kk = k[s:s + 2048]
        ph = R @ kk.T
        c, sn = np.cos(ph), np.sin(ph)
        Sa_re, Sa_im = c.T @ a_vec, sn.T @ a_vec
        Sb_re, Sb_im = c.T @ b_vec, sn.T @ b_vec
        # Im(S e^{-ik.R_A}) = S_im cos - S_re sin
        imb = c * Sb_im[None, :] - sn * Sb_re[None, :]
        ima = c * Sa_im[None, :] - sn * Sa_re[None, :]
        ww = w[s:s + 2048]
        G[rows] += (a_vec[rows, None] * imb[rows] + b_vec[rows, None] * ima[rows]) @ (ww[:, None] * kk)
    return G / BOHR_A
