"""Slater-Koster sp blocks of the synthetic SCC tight-binding model (FP64 oracle).

Test infrastructure only (see ``oracle/__init__``).

The paper's electronic-structure engine is SCC-DFTB with Slater-Koster tabulated
Hamiltonian and overlap elements in a minimal basis (SI Sec. "Implementation
with SCC-DFTB theory").  Its LATTE parameters are not available, so the model is
the synthetic sp model given as input data (``inputs.SKModel``):

    V_X(r) = V0_X exp(-r/decay) sw(r),  X in {ss sigma, sp sigma, pp sigma, pp pi}

with the Slater-Koster direction-cosine table (Slater & Koster 1954):

    H[s_i, s_j]     = V_ss
    H[s_i, p_a,j]   =  l_a V_sp
    H[p_a,i, s_j]   = -l_a V_sp
    H[p_a,i, p_b,j] =  l_a l_b (V_pps - V_ppp) + delta_ab V_ppp

where l = (R_j - R_i)/|R_j - R_i|.  S uses the same table with every V0 scaled
by ``overlap_scale``; S has unit diagonal.  Orbital order per atom: s, px, py, pz.
Lengths in Angstrom, energies in Hartree.  Pinned by tests against: a finite-
difference derivative, H = H^T, rotation invariance of a molecule's spectrum,
and the isolated-dimer ss case (a 2x2 closed form).
"""
from __future__ import annotations

import numpy as np


def switch(r: np.ndarray, r_on: float, r_off: float) -> tuple[np.ndarray, np.ndarray]:
    """Quintic switch sw(r) = 1 - 10t^3 + 15t^4 - 6t^5, t = (r-r_on)/(r_off-r_on); and d sw/dr."""
    w = r_off - r_on
    t = np.clip((r - r_on) / w, 0.0, 1.0)
    sw = 1.0 - 10.0 * t**3 + 15.0 * t**4 - 6.0 * t**5
    dsw = (-30.0 * t**2 + 60.0 * t**3 - 30.0 * t**4) / w
    inside = (r > r_on) & (r < r_off)
    dsw = np.where(inside, dsw, 0.0)
    return sw, dsw


def radial(model, si: np.ndarray, sj: np.ndarray, r: np.ndarray, scale: float = 1.0):
    """Radial functions f[P, 4] (ss, sp(s on i), ps(s on j), ppsig, pppi folded) and df/dr.

    Returns f, df with columns (ss, sp_ij, sp_ji, pps, ppp): sp_ij is V_sp with the s
    orbital on atom i; sp_ji with the s orbital on atom j.
    """
    v0 = model.v0_array() * scale
    sw, dsw = switch(r, model.r_on, model.r_off)
    e = np.exp(-r / model.decay)
    g = e * sw
    dg = e * (dsw - sw / model.decay)
    cols = [v0[si, sj, 0], v0[si, sj, 1], v0[sj, si, 1], v0[si, sj, 2], v0[si, sj, 3]]
    f = np.stack([c * g for c in cols], axis=1)
    df = np.stack([c * dg for c in cols], axis=1)
    return f, df


def pair_blocks(model, si, sj, d, scale: float = 1.0, with_grad: bool = False):
    """4x4 SK blocks for pairs (i, j) at displacement d = R_j - R_i (Angstrom).

    Returns B[P,4,4] and, if requested, dB[P,3,4,4] = dB/dd_c (derivative with
    respect to the displacement vector; dB/dR_i = -dB/dd, dB/dR_j = +dB/dd).
    Rows/columns past an atom's orbital count are meaningless and must be sliced
    away by the caller (H carries only the s orbital).
    """
    d = np.atleast_2d(np.asarray(d, dtype=np.float64))
    si = np.atleast_1d(si)
    sj = np.atleast_1d(sj)
    r = np.sqrt(np.sum(d * d, axis=1))
    lvec = d / r[:, None]
    f, df = radial(model, si, sj, r, scale)
    fss, fsp, fps, fsig, fpi = (f[:, k] for k in range(5))
    P = d.shape[0]
    B = np.zeros((P, 4, 4))
    B[:, 0, 0] = fss
    for a in range(3):
        B[:, 0, 1 + a] = lvec[:, a] * fsp
        B[:, 1 + a, 0] = -lvec[:, a] * fps
        for b in range(3):
            B[:, 1 + a, 1 + b] = lvec[:, a] * lvec[:, b] * (fsig - fpi) + (fpi if a == b else 0.0)
    if not with_grad:
        return B
    dss, dsp, dps, dsig, dpi = (df[:, k] for k in range(5))
    dB = np.zeros((P, 3, 4, 4))
    eye = np.eye(3)
    for c in range(3):
        # dl_a/dd_c = (delta_ac - l_a l_c) / r ; dr/dd_c = l_c
        dl = (eye[:, c][None, :] - lvec * lvec[:, c:c + 1]) / r[:, None]     # [P,3] over a
        lc = lvec[:, c]
        dB[:, c, 0, 0] = dss * lc
        for a in range(3):
            dB[:, c, 0, 1 + a] = dl[:, a] * fsp + lvec[:, a] * dsp * lc
            dB[:, c, 1 + a, 0] = -(dl[:, a] * fps + lvec[:, a] * dps * lc)
            for b in range(3):
                val = (dl[:, a] * lvec[:, b] + lvec[:, a] * dl[:, b]) * (fsig - fpi) \
                    + lvec[:, a] * lvec[:, b] * (dsig - dpi) * lc
                if a == b:
                    val = val + dpi * lc
                dB[:, c, 1 + a, 1 + b] = val
    return B, dB


def image_shifts(box: np.ndarray, r_cut: float) -> np.ndarray:
    """Lattice vectors k*box (k integer per axis) that can bring a minimum-image pair within r_cut."""
    nimg = [int(np.floor((r_cut + 0.5 * L) / L)) for L in box]
    ks = np.array([[i, j, k] for i in range(-nimg[0], nimg[0] + 1)
                   for j in range(-nimg[1], nimg[1] + 1)
                   for k in range(-nimg[2], nimg[2] + 1)], dtype=np.float64)
    return ks * box[None, :]


def orbital_layout(species: np.ndarray, model) -> tuple[np.ndarray, np.ndarray]:
    """Per-atom orbital counts and offsets (atom order, orbitals s, px, py, pz)."""
    norb = np.asarray(model.n_orb, dtype=np.int64)[species]
    off = np.concatenate([[0], np.cumsum(norb)])
    return norb, off


def hs_blocks_for_atoms(atoms: np.ndarray, R: np.ndarray, species: np.ndarray, box: np.ndarray, model):
    """Principal submatrices H0[g,g], S[g,g] of the periodic (Gamma-point) model over atom list g.

    Element (I,J) sums the SK block over every periodic image with |d + L| < r_off
    (I = J: images L != 0 only, plus the on-site diagonal).  This is the principal
    submatrix of the global matrices (paper Sec. "Matrix Functions on a Graph").
    """
    atoms = np.asarray(atoms, dtype=np.int64)
    sp = species[atoms]
    norb, off = orbital_layout(sp, model)
    na = atoms.shape[0]
    H4 = np.zeros((na, na, 4, 4))
    S4 = np.zeros((na, na, 4, 4))
    shifts = image_shifts(box, model.r_off)
    ii, jj = np.meshgrid(np.arange(na), np.arange(na), indexing="ij")
    ii = ii.ravel()
    jj = jj.ravel()
    d0 = R[atoms[jj]] - R[atoms[ii]]
    d0 = d0 - box * np.round(d0 / box)
    same = ii == jj
    for L in shifts:
        d = d0 + L
        r2 = np.sum(d * d, axis=1)
        keep = (r2 < model.r_off**2) & ~(same & (np.sum(L * L) == 0.0))
        if not np.any(keep):
            continue
        k_i, k_j, dk = ii[keep], jj[keep], d[keep]
        np.add.at(H4, (k_i, k_j), pair_blocks(model, sp[k_i], sp[k_j], dk))
        np.add.at(S4, (k_i, k_j), pair_blocks(model, sp[k_i], sp[k_j], dk, scale=model.overlap_scale))
    eps_s = np.asarray(model.eps_s)
    eps_p = np.asarray(model.eps_p)
    idx = np.arange(na)
    H4[idx, idx, 0, 0] += eps_s[sp]
    for k in range(1, 4):
        H4[idx, idx, k, k] += eps_p[sp]
    for k in range(4):
        S4[idx, idx, k, k] += 1.0
    mask = (np.arange(4)[None, :] < norb[:, None]).ravel()
    H = H4.transpose(0, 2, 1, 3).reshape(4 * na, 4 * na)[np.ix_(mask, mask)]
    S = S4.transpose(0, 2, 1, 3).reshape(4 * na, 4 * na)[np.ix_(mask, mask)]
    return H, S, norb, off
