"""SCC optimisation, XL-BOMD shadow dynamics and the low-rank Krylov kernel (FP64 oracle).

Test infrastructure only (see ``oracle/__init__``).

* SCC (Sec. "Determining the Subgraphs"): charges n are iterated to the fixed point
  n = q[n] by linear mixing n <- n + alpha (q[n] - n); the graph is rebuilt from the
  previous step's density (distance cutoff + |D| threshold) at every iteration and
  the cores stay fixed.  Converged when max |q - n| <= tol.
* Kernel-accelerated quasi-Newton SCC (SI Sec. C): n <- n - (K0 J)^-1 K0 (q - n) with
  the rank-m approximation of (K0 J)^-1.
* Response (SI Sec. B, Eq. "dfdv"): J v = dq/dn v - v, from first-order perturbation
  theory on every subgraph at the Fermi occupations of Te (sum over state pairs with the
  divided differences (f_j - f_k)/(eps_j - eps_k), -beta f (1 - f) for equal levels), and
  with the canonical shift of mu that keeps the collected electron count fixed.
* Low-rank kernel (SI Sec. B, Eqs. "PreKernel", "LowRankEEOM"): v_j an orthonormalised
  preconditioned Krylov basis starting at K0 f, f_vj = K0 J v_j, O_ij = f_vi . f_vj,
  M = O^-1, K f ~ sum_ij v_i M_ij f_vj^T K0 f; stops at rank m or when the relative
  residual of the projected equation falls below tol.
* XL-BOMD (Eqs. NEQ / HW): velocity Verlet for the nuclei with forces at fixed n, and
  n_{t+1} = 2 n_t - n_{t-1} - kappa K(q[n_t] - n_t) + alpha sum_k c_k n_{t-k} with the
  dissipation coefficients of the paper's integrator reference (Niklasson et al. 2009,
  K = 5: kappa = 1.82, alpha = 0.018, c = (-6, 14, -8, -3, 4, -1)).

Pinned by tests: the SCC fixed point is independent of the mixer; full-rank Krylov equals
the dense J^-1 (finite-difference Jacobian) on a tiny box; responses equal a central finite
difference at fixed mu and, canonical, with mu solved again; energy fluctuation of the
dynamics scales with dt^2 and shows no drift.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import KB_HA
from . import density as dn
from . import ewald, graph

XL_KAPPA = 1.82
XL_ALPHA = 0.018
XL_C = (-6.0, 14.0, -8.0, -3.0, 4.0, -1.0)
ACC_HA_A_AMU = 0.2625499639      # (Ha/A)/amu in A/fs^2  (1 Ha / (1 amu A^2 fs^-2))


@dataclass
class GraphParams:
    r_graph: float = 3.0      # A
    tau: float = 1e-3
    core_size: int = 12


def graph_and_halos(R, box, gp: GraphParams, cores, gd, keep=None):
    row_ptr, col = graph.build_graph(R, box, gp.r_graph, gd, gp.tau, keep)
    return row_ptr, col, graph.halos(row_ptr, col, cores)


def scc(R, species, box, model, gp: GraphParams, n0=None, max_iter: int = 300, tol: float = 1e-8,
        alpha: float = 0.2, cores=None, gd=None, krylov_rank: int = 0, c_k0: float = 0.5):
    """Self-consistent charges.  Returns (n, density result, iterations, residual history).

    Each iteration rebuilds the graph from the latest density graph; from the second iteration on
    the new graph also keeps every edge of the previous one."""
    N = R.shape[0]
    if cores is None:
        cores = graph.rcb_partition(R, box, gp.core_size)
    n = np.zeros(N) if n0 is None else np.array(n0, dtype=np.float64)
    hist = []
    res = None
    it = 0
    prev = None
    for it in range(1, max_iter + 1):
        # from the second iteration on the graph keeps the edges it had (SCF iterations add edges
        # and do not remove them, Sec. "Determining the Subgraphs"), so halos only grow
        rp, col, hal = graph_and_halos(R, box, gp, cores, gd, prev)
        prev = (rp, col)
        res = dn.density(R, species, box, model, n, cores, hal)
        f = res.q - n
        r = float(np.max(np.abs(f)))
        hist.append(r)
        if r <= tol:
            break
        if krylov_rank > 0 and r < 0.1:
            u, _ = low_rank_kernel(R, species, box, model, res, f, c_k0, krylov_rank, tol=1e-2)
            n = n - u                       # n - (K0 J)^-1 K0 f
        else:
            n = n + alpha * f
        gd = res.gd
    return n, res, it, hist


def divided_differences(eps: np.ndarray, f: np.ndarray, beta: float) -> np.ndarray:
    """F[j, k] = (f_j - f_k) / (eps_j - eps_k), and -beta f_j (1 - f_j) where the levels coincide."""
    de = eps[:, None] - eps[None, :]
    df = f[:, None] - f[None, :]
    close = np.abs(de) < 1e-12
    safe = np.where(close, 1.0, de)
    deriv = -beta * 0.5 * ((f * (1.0 - f))[:, None] + (f * (1.0 - f))[None, :])
    return np.where(close, deriv, df / safe)


def charge_response(res: dn.DensityResult, v, R, species, box, model, canonical: bool = True):
    """dq/dn v on fixed subgraphs (first-order perturbation, sum over state pairs).

    dV = gamma v, dh = 1/2 (s dV + dV s) on every subgraph, dh~ = Z dh Z; in the eigenbasis
    dP_jk = F[j, k] (x_j^T dh~ x_k) with the divided differences of the Fermi function at
    Te; dD_c = 2 Z_c dP Z.  canonical: add dmu * dq/dmu with dq/dmu from
    dP/dmu = X diag(beta f (1 - f)) X^T, dmu chosen so that sum dq = 0 (fixed electron count)."""
    dV = ewald.coulomb_potential(R, species, model.hubbard_u, box, v)
    beta = 1.0 / (KB_HA * res.Te)
    dq = np.zeros(R.shape[0])
    dqmu = np.zeros(R.shape[0])
    for sg in res.subs:
        vorb = np.repeat(dV[sg.atoms], sg.norb)
        dh = 0.5 * sg.S * (vorb[:, None] + vorb[None, :])
        X = sg.X                                   # eigenvectors of h~ (C = Z X)
        dht = X.T @ (sg.Z @ dh @ sg.Z) @ X         # perturbation in the eigenbasis
        dP = X @ (divided_differences(sg.eps, sg.occ, beta) * dht) @ X.T
        dPmu = (X * (beta * sg.occ * (1.0 - sg.occ))[None, :]) @ X.T
        nco = int(sg.off[sg.n_core])
        for P_, out in ((dP, dq), (dPmu, dqmu)):
            dD = 2.0 * sg.Z @ P_ @ sg.Z
            pop = np.sum(dD[:nco, :] * sg.S[:, :nco].T, axis=1)
            for a in range(sg.n_core):
                out[int(sg.atoms[a])] = float(np.sum(pop[sg.off[a]:sg.off[a + 1]]))
    if canonical:
        s_mu = float(np.sum(dqmu))
        if s_mu > 0.0:
            dq = dq - (float(np.sum(dq)) / s_mu) * dqmu
    return dq


def low_rank_kernel(R, species, box, model, res, f, c_k0: float, m_max: int, tol: float = 1e-2):
    """(K0 J)^-1 K0 f by the preconditioned rank-m Krylov approximation; K0 = -c I.

    Returns (u, rank used).  u approximates J^-1 f = K f.
    """
    k0f = -c_k0 * f
    vs, fvs = [], []
    vec = k0f.copy()
    u = k0f.copy()
    for j in range(m_max):
        for v in vs:                               # modified Gram-Schmidt
            vec = vec - np.dot(v, vec) * v
        nrm = np.linalg.norm(vec)
        if nrm < 1e-14:
            break
        v = vec / nrm
        jv = charge_response(res, v, R, species, box, model) - v
        fv = -c_k0 * jv                            # K0 J v
        vs.append(v)
        fvs.append(fv)
        F = np.stack(fvs, axis=1)
        Vm = np.stack(vs, axis=1)
        O = F.T @ F
        M = np.linalg.inv(O)
        coef = M @ (F.T @ k0f)
        u = Vm @ coef
        resid = np.linalg.norm(F @ coef - k0f) / np.linalg.norm(k0f)
        if resid < tol:
            break
        vec = fv.copy()
    return u, len(vs)


def xlbomd(R, Vel, species, box, model, gp: GraphParams, n_steps: int, dt_fs: float,
           n0=None, cores=None, c_k0: float = 0.5, krylov_rank: int = 0, gd=None, scc_tol=1e-8):
    """Shadow XL-BOMD NVE trajectory.  Returns dict with energies [steps+1, 3] (kin, pot, total) in Ha."""
    R = np.array(R, dtype=np.float64)
    Vel = np.array(Vel, dtype=np.float64)
    mass = np.asarray(model.mass)[species]
    if cores is None:
        cores = graph.rcb_partition(R, box, gp.core_size)
    if n0 is None:
        n0, res, _, _ = scc(R, species, box, model, gp, cores=cores, gd=gd, tol=scc_tol)
        gd = res.gd
    n = np.array(n0, dtype=np.float64)
    hist = [n.copy() for _ in range(len(XL_C))]      # n_t, n_{t-1}, ..., n_{t-5}
    _, _, hal = graph_and_halos(R, box, gp, cores, gd)
    res = dn.density(R, species, box, model, n, cores, hal)
    F = dn.forces(res, n, R, species, box, model)
    out = []

    def energies(res_, n_, Vel_):
        kin = 0.5 * float(np.sum(mass[:, None] * Vel_ * Vel_)) / ACC_HA_A_AMU
        pot = dn.shadow_energy(res_, n_, R, species, box, model)["total"]
        return (kin, pot, kin + pot)

    out.append(energies(res, n, Vel))
    for _ in range(n_steps):
        f = res.q - n
        if krylov_rank > 0:
            u, _ = low_rank_kernel(R, species, box, model, res, f, c_k0, krylov_rank)
        else:
            u = -c_k0 * f
        Vel = Vel + 0.5 * dt_fs * ACC_HA_A_AMU * F / mass[:, None]
        R = R + dt_fs * Vel
        n_new = 2.0 * hist[0] - hist[1] - XL_KAPPA * u \
            + XL_ALPHA * sum(c * h for c, h in zip(XL_C, hist))
        hist = [n_new] + hist[:-1]
        n = n_new
        gd = res.gd
        _, _, hal = graph_and_halos(R, box, gp, cores, gd)
        res = dn.density(R, species, box, model, n, cores, hal)
        F = dn.forces(res, n, R, species, box, model)
        Vel = Vel + 0.5 * dt_fs * ACC_HA_A_AMU * F / mass[:, None]
        out.append(energies(res, n, Vel))
    return {"energies": np.asarray(out), "R": R, "V": Vel, "n": n, "res": res}
