"""Subgraph electronic structure, global chemical potential and collected observables (FP64 oracle).

Test infrastructure only (see ``oracle/__init__``).

What is computed, in the paper's order:

1. Coulomb potential of the trial charges n: V = gamma n (SCC-DFTB, SI Sec. D), and
   the n-dependent Hamiltonian H[n] = H0 + 1/2 (S V + V S), V diagonal per atom
   (the linearised shadow functional, Eq. "Shadow_Energy" and below).
2. For every core+halo subgraph g_i the principal submatrices h = H[n][g,g],
   s = S[g,g] (Sec. "Matrix Functions on a Graph", Eq. 1).
3. Change to an orthonormal basis with Z = s^(-1/2) (the paper assumes S = I for
   simplicity and points to the change of basis, Sec. "Density Matrix Evaluation on
   Partitioned Graphs"); h~ = Z h Z.
4. The Fermi operator D = [exp(beta (h~ - mu I)) + I]^(-1) (Eq. 2) through the
   eigen-decomposition of h~ (the paper allows direct diagonalisation, Sec. "Density
   Matrix Evaluation on Partitioned Graphs"); spin factor 2, closed shell.  Steps 3-4
   run in plain C by cyclic Jacobi rotations (``cjacobi``, default) or through
   numpy.linalg.eigh (``eig="lapack"``).
5. One chemical potential mu for the whole system with Tr[D S] = N_e (Eq. 2, with the
   trace read as the collected count): N(mu) = 2 sum_i sum_k w_ik f(eps_ik - mu) = N_e,
   w_ik the core Mulliken weight of state k of subgraph i, f the Fermi function at Te
   (``solve_mu``, bisection).  The graph truncation leaves the T -> 0 count at mid-gap
   off N_e; the finite-temperature rule absorbs that miss in the Fermi tails of the
   states nearest to mu (for the water boxes: mu sits ~9 kT above the flat lone-pair
   band).  ``t0_miss`` reports the T -> 0 count at mu minus N_e, ``in_gap_weight`` the
   core weight of states within 0.05 Ha of mu.
6. Collection of the core rows (Eq. 3 / SI Eq. A): D_c = 2 Z C f C^T Z and the
   energy-weighted W_c = 2 Z C (f eps) C^T Z, restricted to core orbitals.
7. Net Mulliken charges dq_I = sum_{mu in I} sum_nu D_mu,nu S_nu,mu - Z_I
   (SI Sec. D), band energy Tr[D H0], shadow energy
   U = Tr[D H0] + 1/2 (2 dq - n)^T gamma n + E_rep, and forces
   F = -[Tr(D dH[n]) - Tr(W dS) + (dq - n/2)^T dgamma n + dE_rep] at fixed n (Eq. NEQ).
8. Atom-condensed density graph G^D_IJ = max over the (I,J) block of |D| (Sec.
   "Dynamic Graph Adaption").
9. Electronic entropy of the collected Fermi occupations,
   S_e = -2 k_B sum_ik w_ik [f ln f + (1 - f) ln(1 - f)]; the free-energy term -T S_e is
   reported beside the shadow energy (``ts_entropy``), not inside its ``total``.

Pinned by tests: Z s Z = I; idempotency D S D = 2 D and Tr(D S) = N_e in the full
(single partition) limit; subgraph result equal to full diagonalisation when every
halo is the whole system; charge neutrality; mu against a brute-force scan of the
collected count on a truncated graph; G^D against an explicit loop over the full core
rows; forces equal to a central finite difference of U in the full limit.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

from . import BOHR_A, KB_HA, cjacobi, ewald, sk


def fermi(x: np.ndarray, beta: float) -> np.ndarray:
    """1 / (1 + exp(beta x)) evaluated with exp of -|beta x| only."""
    e = np.exp(-np.abs(beta * x))
    return np.where(x > 0, e / (1.0 + e), 1.0 / (1.0 + e))


def sp2_mu_occupations(x: np.ndarray, y: float, n_real: int, tol: float = 1e-9, kmax: int = 60):
    """mu-branch SP2 polynomial applied to scaled eigenvalues x of one subgraph.

    The recursion (Fermi-operator expansion by recursive projection, Sec. "Density
    Matrix Evaluation on Partitioned Graphs", refs. Niklasson 2002 / Finkelstein 2021)
    with the branch set by the image y of the chemical potential: y >= 1/2 -> x <- x^2,
    y <- y^2; else x <- 2x - x^2, y <- 2y - y^2.  At step k the idempotency error
    t_k = sum x(1-x) of the current iterate is taken and the update is applied.  The
    recursion stops after the first step with t_k < tol * n_real, or -- the parameterless
    rule of Kruchinina, Rudberg and Rubensson (2016) for finite precision -- after the
    first step k >= 4 with t_{k-2} < 1e-4 n_real and t_k >= t_{k-2}, or after kmax steps.
    Returns (occupations, number of steps).
    """
    x = np.array(x, dtype=np.float64)
    it = 0
    hist = []
    for it in range(1, kmax + 1):
        t = float(np.sum(x - x * x))
        hist.append(t)
        if y >= 0.5:
            x = x * x
            y = y * y
        else:
            x = 2.0 * x - x * x
            y = 2.0 * y - y * y
        floor_hit = it >= 4 and hist[-3] < 1e-4 * n_real and t >= hist[-3]
        if t < tol * n_real or floor_hit:
            break
    return x, it


def gershgorin(a: np.ndarray) -> tuple[float, float]:
    """Spectral bounds of a symmetric matrix from Gershgorin discs."""
    r = np.sum(np.abs(a), axis=1) - np.abs(np.diag(a))
    return float(np.min(np.diag(a) - r)), float(np.max(np.diag(a) + r))


@dataclass
class SubgraphSolution:
    atoms: np.ndarray           # subgraph atom list (core first)
    n_core: int                 # number of core atoms
    norb: np.ndarray            # orbitals per subgraph atom
    off: np.ndarray             # orbital offsets
    H0: np.ndarray
    H: np.ndarray
    S: np.ndarray
    Z: np.ndarray
    eps: np.ndarray             # eigenvalues of h~
    C: np.ndarray               # AO coefficients Z X
    X: np.ndarray               # eigenvectors of h~
    w: np.ndarray               # core weights
    occ: np.ndarray | None = None
    D_rows: np.ndarray | None = None   # core rows of D  [n_core_orb, n]
    W_rows: np.ndarray | None = None
    sp2_steps: int = 0
    bounds: tuple = (0.0, 0.0)


@dataclass
class DensityResult:
    mu: float
    q: np.ndarray                # net Mulliken charges dq (electron excess), per atom
    e_band: float
    n_electrons: float
    V: np.ndarray                # Coulomb potential used (Ha per e)
    subs: list = field(default_factory=list)
    gd: tuple | None = None      # (ptr, col, val) atom-condensed density graph
    in_gap_weight: float = 0.0   # sum of core weights of states within +-0.05 Ha of mu
    t0_miss: float = 0.0         # T -> 0 collected count at mu minus N_e (graph truncation)
    entropy: float = 0.0         # S_e / k_B of the collected occupations (spin factor 2)
    Te: float = 300.0


# Eigensolver of the subgraph solves: "jacobi" is the plain-C cyclic Jacobi method of
# ``oracle/csrc/jacobi.c`` (Z, h~, eigenpairs and core weights in C, subgraphs spread over the host
# threads); "lapack" is numpy.linalg.eigh with the same steps in numpy.  The two agree to ~1e-13 on
# the eigenvalues (tests/test_oracle_jacobi.py).
EIG = "jacobi"


def subgraph_blocks(atoms, R, species, box, model, V):
    """h = H[n] and s = S restricted to one subgraph's orbitals, with H0, orbitals per atom and
    orbital offsets: H[n] = H0 + 1/2 (S V + V S), V diagonal per atom."""
    H0, S, norb, off = sk.hs_blocks_for_atoms(atoms, R, species, box, model)
    vorb = np.repeat(V[atoms], norb)
    H = H0 + 0.5 * S * (vorb[:, None] + vorb[None, :])
    return H0, H, S, norb, off


def _solution(atoms, n_core, blocks, Z, eps, X, Cc, w):
    H0, H, S, norb, off = blocks
    Ht = Z @ H @ Z
    Ht = 0.5 * (Ht + Ht.T)
    return SubgraphSolution(atoms=np.asarray(atoms), n_core=int(n_core), norb=norb, off=off,
                            H0=H0, H=H, S=S, Z=Z, eps=eps, C=Cc, X=X, w=w, bounds=gershgorin(Ht))


def _eig_lapack(H, S, nco):
    lam, U = np.linalg.eigh(S)
    Z = (U * (1.0 / np.sqrt(lam))[None, :]) @ U.T
    Ht = Z @ H @ Z
    Ht = 0.5 * (Ht + Ht.T)
    eps, X = np.linalg.eigh(Ht)
    Cc = Z @ X
    SC = S @ Cc
    w = np.sum(Cc[:nco, :] * SC[:nco, :], axis=0)
    return Z, eps, X, Cc, w


def subgraph_setup(atoms, n_core, R, species, box, model, V, eig: str | None = None):
    """h, s, Z = s^-1/2, eigenpairs of h~ = Z h Z, and core weights of one subgraph."""
    blocks = subgraph_blocks(atoms, R, species, box, model, V)
    _, H, S, _, off = blocks
    nco = int(off[n_core])
    if (eig or EIG) == "jacobi":
        sol = cjacobi.subgraph_eig(H, S, nco)
    else:
        sol = _eig_lapack(H, S, nco)
    return _solution(atoms, n_core, blocks, *sol)


def subgraph_setup_all(atom_lists, n_cores, R, species, box, model, V, eig: str | None = None):
    """subgraph_setup over many subgraphs (the Jacobi route solves them on the host threads)."""
    blocks = [subgraph_blocks(a, R, species, box, model, V) for a in atom_lists]
    if (eig or EIG) == "jacobi":
        sols = cjacobi.subgraph_eig_batch([(b[1], b[2], int(b[4][nc])) for b, nc in zip(blocks, n_cores)])
    else:
        sols = [_eig_lapack(b[1], b[2], int(b[4][nc])) for b, nc in zip(blocks, n_cores)]
    return [_solution(a, nc, b, *sol) for a, nc, b, sol in zip(atom_lists, n_cores, blocks, sols)]


def collected_count(eps_list, w_list, mu: float, beta: float) -> float:
    """N(mu) = 2 sum_i sum_k w_ik f(eps_ik - mu) at inverse temperature beta (Eq. 2)."""
    return 2.0 * sum(float(np.dot(w, fermi(np.asarray(e) - mu, beta))) for e, w in zip(eps_list, w_list))


def solve_mu(eps_list, w_list, n_e: float, beta: float) -> float:
    """Global chemical potential of Eq. 2: bisection on N(mu) = N_e.

    N(mu) is non-decreasing in mu (core weights of the collected states are positive up
    to the truncation; the test keeps the bracket).  Start [min eps - 1, max eps + 1];
    stop when |N - N_e| < 1e-11 or the interval is narrower than 1e-15 Ha; return the
    midpoint.  The bisection runs in plain C (``oracle/csrc/mu.c``); ``collected_count`` above
    is the same count in numpy, which the tests scan against it.
    """
    return cjacobi.solve_mu(eps_list, w_list, n_e, beta)


def entropy_density(f: np.ndarray) -> np.ndarray:
    """-[f ln f + (1 - f) ln(1 - f)] with 0 ln 0 = 0."""
    f = np.asarray(f, dtype=np.float64)
    out = np.zeros_like(f)
    m = (f > 0.0) & (f < 1.0)
    g = f[m]
    out[m] = -(g * np.log(g) + (1.0 - g) * np.log1p(-g))
    return out


def density(R, species, box, model, n, cores, halo_lists, Te: float = 300.0, mu: float | None = None,
            mode: str = "fermi", sp2_tol: float = 1e-9, V: np.ndarray | None = None,
            eig: str | None = None) -> DensityResult:
    """Graph-partitioned density at trial charges n: charges, band energy, mu, core rows of D and W.

    mode "fermi": Fermi occupations at Te (default), mu from Eq. 2 (``solve_mu``) unless
    given; "sp2": the mu-branch SP2 polynomial of ``sp2_mu_occupations`` on every eigenvalue
    (same function as the T -> 0 GPU recursion), with Gershgorin bounds of h~, at a given mu.
    """
    R = np.asarray(R, dtype=np.float64)
    species = np.asarray(species)
    if V is None:
        V = ewald.coulomb_potential(R, species, model.hubbard_u, box, n)
    atom_lists = [np.concatenate([core, halo]).astype(np.int64) for core, halo in zip(cores, halo_lists)]
    subs = subgraph_setup_all(atom_lists, [len(c) for c in cores], R, species, box, model, V, eig=eig)
    n_e = float(np.sum(np.asarray(model.z_val)[species]))
    if mode == "sp2" and mu is None:
        raise ValueError("the T -> 0 SP2 occupations take a given chemical potential")
    if mode == "fermi" and not Te > 0.0:
        raise ValueError("Fermi occupations need Te > 0")
    beta = 1.0 / (KB_HA * Te) if Te > 0.0 else math.inf

    def occ_for(mu_):
        out = []
        for sg in subs:
            if mode == "fermi":
                out.append(fermi(sg.eps - mu_, beta))
            else:
                lo, hi = sg.bounds
                x = (hi - sg.eps) / (hi - lo)
                y = (hi - mu_) / (hi - lo)
                occ, steps = sp2_mu_occupations(x, y, len(sg.eps), tol=sp2_tol)
                sg.sp2_steps = steps
                out.append(occ)
        return out

    if mu is None:
        mu = solve_mu([sg.eps for sg in subs], [sg.w for sg in subs], n_e, beta)
    occs = occ_for(mu)
    q = np.zeros(R.shape[0])
    e_band = 0.0
    nel = 0.0
    gap_w = 0.0
    t0 = 0.0
    ent = 0.0
    z = np.asarray(model.z_val)
    gd_rows = {}
    for sg, f in zip(subs, occs):
        sg.occ = f
        nco = int(sg.off[sg.n_core])
        Cc = sg.C
        sg.D_rows = 2.0 * (Cc[:nco, :] * f[None, :]) @ Cc.T
        sg.W_rows = 2.0 * (Cc[:nco, :] * (f * sg.eps)[None, :]) @ Cc.T
        pop = np.sum(sg.D_rows * sg.S[:, :nco].T, axis=1)      # (D S)_mu,mu over core rows
        eb = np.sum(sg.D_rows * sg.H0[:, :nco].T, axis=1)
        e_band += float(np.sum(eb))
        for a in range(sg.n_core):
            I = int(sg.atoms[a])
            q[I] = float(np.sum(pop[sg.off[a]:sg.off[a + 1]])) - z[species[I]]
            nel += float(np.sum(pop[sg.off[a]:sg.off[a + 1]]))
            # atom-condensed |D| block maxima of this core atom's rows
            row = np.abs(sg.D_rows[sg.off[a]:sg.off[a + 1], :])
            vals = np.array([np.max(row[:, sg.off[b]:sg.off[b + 1]]) for b in range(len(sg.atoms))])
            gd_rows[I] = (sg.atoms.astype(np.int32), vals)
        gap_w += float(np.sum(sg.w[np.abs(sg.eps - mu) < 0.05]))
        t0 += 2.0 * float(np.sum(sg.w[sg.eps < mu]))
        ent += 2.0 * float(np.dot(sg.w, entropy_density(f)))
    N = R.shape[0]
    ptr = np.zeros(N + 1, dtype=np.int64)
    cols, vals = [], []
    for I in range(N):
        c, v = gd_rows.get(I, (np.zeros(0, np.int32), np.zeros(0)))
        order = np.argsort(c, kind="stable")
        cols.append(c[order])
        vals.append(v[order])
        ptr[I + 1] = ptr[I] + len(c)
    gd = (ptr, np.concatenate(cols).astype(np.int32), np.concatenate(vals))
    return DensityResult(mu=float(mu), q=q, e_band=e_band, n_electrons=nel, V=V, subs=subs, gd=gd,
                         in_gap_weight=gap_w, t0_miss=t0 - n_e, entropy=ent, Te=Te)


def repulsion(R, species, box, model, with_grad: bool = False, rows=None):
    """E_rep = 1/2 sum_{I,J,L}' A_IJ exp(-r/rep_decay) sw(r) over pairs within r_off (Ha, Ha/A).

    rows: sum only the terms of these atoms (energy: their halves of the pair terms; gradient:
    their rows, which are complete)."""
    R = np.asarray(R, dtype=np.float64)
    A = model.rep_array()
    N = R.shape[0]
    E = 0.0
    G = np.zeros((N, 3))
    if not np.any(A):
        return (E, G) if with_grad else E
    shifts = sk.image_shifts(box, model.r_off)
    for i in (range(N) if rows is None else [int(x) for x in rows]):
        d0 = R - R[i]
        d0 = d0 - box * np.round(d0 / box)
        for L in shifts:
            d = d0 + L
            r = np.sqrt(np.sum(d * d, axis=1))
            ok = (r < model.r_off) & (r > 0.0)
            rr = np.where(ok, r, 1.0)
            sw, dsw = sk.switch(rr, model.r_on, model.r_off)
            amp = A[species[i], species]
            ex = np.exp(-rr / model.rep_decay)
            e = np.where(ok, amp * ex * sw, 0.0)
            de = np.where(ok, amp * ex * (dsw - sw / model.rep_decay), 0.0)
            E += 0.5 * float(np.sum(e))
            # d/dR_i of e(|R_j - R_i + L|) = -de * d_hat ; both orderings give a factor 2 * 1/2
            G[i] -= np.sum((de / rr)[:, None] * d, axis=0)
    return (E, G) if with_grad else E


def shadow_energy(res: DensityResult, n, R, species, box, model) -> dict:
    """U = Tr[D H0] + 1/2 (2 dq - n)^T gamma n + E_rep  (Eq. "Shadow_Energy" with SCC-DFTB).

    ``ts_entropy`` = -T S_e of the collected Fermi occupations, the electronic free-energy
    term at finite Te; it is reported beside ``total`` and not added to it."""
    e_coul = float(np.dot(res.q - 0.5 * np.asarray(n), res.V))
    e_rep = repulsion(R, species, box, model)
    return {"band": res.e_band, "coulomb": e_coul, "repulsion": e_rep,
            "total": res.e_band + e_coul + e_rep, "ts_entropy": -KB_HA * res.Te * res.entropy}


def forces(res: DensityResult, n, R, species, box, model, atoms=None) -> np.ndarray:
    """F = -[Tr(D dH[n]) - Tr(W dS) + (dq - n/2)^T dgamma n + dE_rep] in Ha/A at fixed n (Eq. NEQ).

    atoms: compute only the rows of these atoms (every pair term that touches one of them is
    kept, the others skipped; the other rows are returned as 0).

    The trace runs over the collected (core-row) D and W: for every subgraph, every
    core atom A and every subgraph atom B (each periodic image within r_off), the
    block gradient g = sum_{mu in A, nu in B} [D dH0 + 1/2 (V_A + V_B) D dS - W dS]_mu,nu
    taken with respect to d = R_B - R_A + L is added to dU/dR_B and subtracted from dU/dR_A.
    """
    R = np.asarray(R, dtype=np.float64)
    N = R.shape[0]
    dU = np.zeros((N, 3))
    V = res.V
    want = np.ones(N, dtype=bool) if atoms is None else np.isin(np.arange(N), atoms)
    shifts = sk.image_shifts(box, model.r_off)
    for sg in res.subs:
        sg_atoms = sg.atoms
        if not np.any(want[sg_atoms]):
            continue
        sp = species[sg_atoms]
        for a in range(sg.n_core):
            A = int(sg_atoms[a])
            ra = slice(sg.off[a], sg.off[a + 1])
            na = int(sg.norb[a])
            d0 = R[sg_atoms] - R[A]
            d0 = d0 - box * np.round(d0 / box)
            for L in shifts:
                d = d0 + L
                r2 = np.sum(d * d, axis=1)
                bs = np.nonzero((r2 < model.r_off**2) & (r2 > 0.0) & (want[A] | want[sg_atoms]))[0]
                if bs.shape[0] == 0:
                    continue
                _, dH = sk.pair_blocks(model, np.full(bs.shape[0], sp[a]), sp[bs], d[bs], with_grad=True)
                _, dS = sk.pair_blocks(model, np.full(bs.shape[0], sp[a]), sp[bs], d[bs],
                                       scale=model.overlap_scale, with_grad=True)
                for p, b in enumerate(bs):
                    nb = int(sg.norb[b])
                    rb = slice(sg.off[b], sg.off[b + 1])
                    Dblk = sg.D_rows[ra, rb]
                    Wblk = sg.W_rows[ra, rb]
                    vab = 0.5 * (V[A] + V[int(sg_atoms[b])])
                    g = np.einsum("mn,cmn->c", Dblk, dH[p, :, :na, :nb]) \
                        + vab * np.einsum("mn,cmn->c", Dblk, dS[p, :, :na, :nb]) \
                        - np.einsum("mn,cmn->c", Wblk, dS[p, :, :na, :nb])
                    dU[A] -= g
                    dU[int(sg_atoms[b])] += g
    n = np.asarray(n, dtype=np.float64)
    rows = None if atoms is None else np.asarray(atoms, dtype=np.int64)
    dU += ewald.coulomb_gradient(R, species, model.hubbard_u, box, res.q - 0.5 * n, n, rows=rows)
    _, grep = repulsion(R, species, box, model, with_grad=True, rows=rows)
    dU += grep
    out = -dU
    if atoms is not None:
        out[~want] = 0.0
    return out


def full_partition(N: int):
    """Single subgraph holding every atom as core (the full-diagonalisation limit)."""
    return [np.arange(N, dtype=np.int32)], [np.zeros(0, dtype=np.int32)]
