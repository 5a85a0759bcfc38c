"""Atom graph, core partition and halos (FP64 / integer oracle).

Test infrastructure only (see ``oracle/__init__``).

* Graph (paper Sec. "Determining the Subgraphs", Fig. 1a/e; SI Sec. A): an atom
  pair (I, J), I != J, is an edge when its minimum-image distance is below the
  cutoff r_G, or when the atom-condensed density graph of the previous step
  exceeds the threshold tau in either direction (symmetrisation, Sec. "Dynamic
  Graph Adaption").  G^D_IJ is the largest |D_mu nu| over the orbital block of
  atoms I and J.  The distance test is r^2 < r_G^2 with
  r^2 = (dx*dx + dy*dy) + dz*dz and dx = (x_J - x_I) - L * rint((x_J - x_I) / L),
  every operation a separately rounded IEEE double operation (no fused
  multiply-add), so the integer result is reproducible bit for bit.
* Cores (Fig. 1b): non-overlapping parts by recursive coordinate bisection of the
  wrapped positions w = x - L * floor(x / L): a part of c atoms that must hold p
  cores splits along its widest axis (first axis on ties) after sorting by
  (w_axis, atom index); the first floor(c * floor(p/2) / p) atoms take floor(p/2)
  cores.  The number of cores is max(1, round(N / core_size)).  The paper uses a
  METIS community detection here; RCB is the deterministic stand-in.
* Halo (Fig. 1c): the graph neighbours of the core atoms that are not core atoms.
  Subgraph order: core atoms ascending, then halo atoms ascending.
* Core refinement for the 128-orbital tiles of the subgraph solves (a reading of the paper's
  remark that the cost of a subgraph grows with the cube of its size, Sec. "Scalability"): single
  core atoms move to an adjacent core while that lowers the integer score
  sum over cores of 128000 T^3 + (n - 128 (T - 1)) (T^3 - (T - 1)^3), T = ceil(n / 128), n the
  orbitals of core + halo: the padded cost T^3 plus a small pull of n toward the boundary below.
  Cores whose n is more than 48 orbitals above that boundary are not touched, cores keep at least
  min_core atoms; cores are visited in order, their atoms ascending, targets ascending, the best
  strict improvement taken.  Deterministic, integer arithmetic throughout.
* Weighted two-hop adaptation (Sec. "Dynamic Graph Adaption", Eqs. "neigh_mat" and
  "Graph_Adaptation"): G^N_IK = exp(-alpha R_IK^2) on the neighbour list, G^N_II = 1;
  P = G^N G^D with G^D in the row form the collection produces (each atom's row from
  the subgraph it is core of); edge (I, J), I != J, when P_IJ > tau or P_JI > tau
  (each subgraph's product thresholded, then collected and symmetrised).  The
  neighbour list holds the pairs with exp(-alpha R^2) >= tau / 2 (R^2 < ln(2/tau) /
  alpha): a two-hop path through a longer pair weighs less than tau, since G^D <= 2.
  P_IJ is summed over K in ascending order, each term w * v rounded and then added.

Pinned by tests against brute force on tiny inputs (edge sets, partition sizes,
halo sets recomputed by explicit loops) and by the bit-exact CSR invariants.
"""
from __future__ import annotations

import numpy as np


def min_image_r2(R: np.ndarray, box: np.ndarray, i: int, js: np.ndarray) -> np.ndarray:
    """Squared minimum-image distances from atom i to atoms js, evaluated without FMA."""
    d = R[js] - R[i]
    d = d - box * np.rint(d / box)
    return (d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1]) + d[:, 2] * d[:, 2]


def build_graph(R: np.ndarray, box: np.ndarray, r_graph: float, gd=None, tau: float = 0.0, keep=None):
    """Symmetric CSR (row_ptr int64, col int32, columns ascending) of the atom graph.

    gd: optional previous atom-condensed density graph as (ptr, col, val) CSR over
    atoms (rows need not be symmetric); an entry with val > tau adds edge (I, J)
    and (J, I).
    keep: optional previous graph (row_ptr, col) whose edges are all kept (during the
    initial SCF, edges are added and not removed: Sec. "Determining the Subgraphs").
    """
    R = np.asarray(R, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    N = R.shape[0]
    rg2 = r_graph * r_graph
    adj = [set() for _ in range(N)]
    allj = np.arange(N)
    for i in range(N):
        r2 = min_image_r2(R, box, i, allj)
        nb = np.nonzero(r2 < rg2)[0]
        for j in nb:
            if j != i:
                adj[i].add(int(j))
    if gd is not None:
        ptr, col, val = gd
        for i in range(N):
            for p in range(int(ptr[i]), int(ptr[i + 1])):
                j = int(col[p])
                if j != i and val[p] > tau:
                    adj[i].add(j)
                    adj[j].add(i)
    if keep is not None:
        kp, kc = keep
        for i in range(N):
            for p in range(int(kp[i]), int(kp[i + 1])):
                adj[i].add(int(kc[p]))
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    cols = []
    for i in range(N):
        c = sorted(adj[i])
        cols.extend(c)
        row_ptr[i + 1] = row_ptr[i] + len(c)
    return row_ptr, np.asarray(cols, dtype=np.int32)


def wrap(R: np.ndarray, box: np.ndarray) -> np.ndarray:
    """w = x - L * floor(x / L), separately rounded operations."""
    return R - box * np.floor(R / box)


def rcb_partition(R: np.ndarray, box: np.ndarray, core_size: int) -> list[np.ndarray]:
    """Core atom lists (each ascending) in depth-first order of the bisection tree."""
    R = np.asarray(R, dtype=np.float64)
    N = R.shape[0]
    n_parts = max(1, int(round(N / core_size)))
    w = wrap(R, np.asarray(box, dtype=np.float64))
    out: list[np.ndarray] = []

    def rec(atoms: np.ndarray, p: int):
        if p == 1:
            out.append(np.sort(atoms).astype(np.int32))
            return
        ext = [float(np.max(w[atoms, a]) - np.min(w[atoms, a])) for a in range(3)]
        axis = 0
        for a in (1, 2):
            if ext[a] > ext[axis]:
                axis = a
        order = np.lexsort((atoms, w[atoms, axis]))      # key: coordinate, then index
        srt = atoms[order]
        pl = p // 2
        m = (atoms.shape[0] * pl) // p
        rec(srt[:m], pl)
        rec(srt[m:], p - pl)

    rec(np.arange(N, dtype=np.int64), n_parts)
    return out


def halos(row_ptr: np.ndarray, col: np.ndarray, cores: list[np.ndarray]) -> list[np.ndarray]:
    """One-hop halo of every core: graph neighbours of core atoms outside the core, ascending."""
    res = []
    for core in cores:
        cs = set(int(a) for a in core)
        h = set()
        for a in core:
            for p in range(int(row_ptr[a]), int(row_ptr[a + 1])):
                j = int(col[p])
                if j not in cs:
                    h.add(j)
        res.append(np.asarray(sorted(h), dtype=np.int32))
    return res


def subgraphs(cores, halo_lists):
    """Atom lists of every core+halo subgraph (core ascending, then halo ascending)."""
    return [np.concatenate([c, h]).astype(np.int64) for c, h in zip(cores, halo_lists)]


def two_hop_rn2(alpha: float, tau: float) -> float:
    """Squared neighbour-list radius of the weighted two-hop rule: exp(-alpha R^2) >= tau / 2."""
    return float(np.log(2.0 / tau) / alpha)


def two_hop_products(R: np.ndarray, box: np.ndarray, gd, alpha: float, tau: float):
    """Rows of P = G^N G^D: a list over atoms I of dicts {J: P_IJ} (every J reached)."""
    R = np.asarray(R, dtype=np.float64)
    box = np.asarray(box, dtype=np.float64)
    N = R.shape[0]
    rn2 = two_hop_rn2(alpha, tau)
    ptr, col, val = gd
    allj = np.arange(N)
    rows = []
    for i in range(N):
        r2 = min_image_r2(R, box, i, allj)
        ks = [int(k) for k in np.nonzero(r2 < rn2)[0]]          # ascending, i itself included
        acc = {}
        for k in ks:
            w = 1.0 if k == i else float(np.exp(-alpha * r2[k]))
            for p in range(int(ptr[k]), int(ptr[k + 1])):
                j = int(col[p])
                acc[j] = acc.get(j, 0.0) + w * float(val[p])
        rows.append(acc)
    return rows


def build_graph_two_hop(R: np.ndarray, box: np.ndarray, gd, alpha: float, tau: float, keep=None):
    """Symmetric CSR of G_tau = (G^N G^D + G^D G^N)|_tau, read as P = G^N G^D thresholded and
    symmetrised: edge (I, J), I != J, when P_IJ > tau or P_JI > tau; keep as in build_graph.
    Returns (row_ptr, col, ambiguous): ambiguous lists the pairs whose deciding products lie
    within 1e-12 tau of tau (where another rounding of exp may decide the other way)."""
    N = np.asarray(R).shape[0]
    rows = two_hop_products(R, box, gd, alpha, tau)
    adj = [set() for _ in range(N)]
    amb = set()
    for i in range(N):
        for j, v in rows[i].items():
            if j == i:
                continue
            if abs(v - tau) <= 1e-12 * tau:
                amb.add((min(i, j), max(i, j)))
            if v > tau:
                adj[i].add(j)
                adj[j].add(i)
    if keep is not None:
        kp, kc = keep
        for i in range(N):
            for p in range(int(kp[i]), int(kp[i + 1])):
                adj[i].add(int(kc[p]))
    row_ptr = np.zeros(N + 1, dtype=np.int64)
    cols = []
    for i in range(N):
        c = sorted(adj[i])
        cols.extend(c)
        row_ptr[i + 1] = row_ptr[i] + len(c)
    return row_ptr, np.asarray(cols, dtype=np.int32), sorted(amb)


def refine_score(n: int) -> int:
    """Integer score of a subgraph of n orbitals (padded cost T^3 with T = ceil(n / 128), in units
    of 128^3 times 128000, plus the distance of n above the boundary below)."""
    t = -(-int(n) // 128)
    return 128000 * t ** 3 + (int(n) - 128 * (t - 1)) * (t ** 3 - (t - 1) ** 3)


def refine_cores(row_ptr, col, cores, norb, rounds: int = 4, min_core: int = 16):
    """Greedy refinement of the cores (see the module notes).  Returns (cores, score before, after);
    each core ascending."""
    N = len(row_ptr) - 1
    nbr = [np.asarray(col[row_ptr[i]:row_ptr[i + 1]], dtype=np.int64) for i in range(N)]
    core_of = np.empty(N, dtype=np.int64)
    members = []
    for c, at in enumerate(cores):
        core_of[np.asarray(at)] = c
        members.append(set(int(a) for a in at))
    norb = np.asarray(norb, dtype=np.int64)

    def orbs(c):
        mem = members[c]
        halo = set()
        for a in mem:
            for b in nbr[a]:
                if int(b) not in mem:
                    halo.add(int(b))
        return int(sum(norb[a] for a in mem) + sum(norb[b] for b in halo))

    n = [orbs(c) for c in range(len(members))]
    before = sum(refine_score(x) for x in n)
    for _ in range(rounds):
        moves = 0
        for c in range(len(members)):
            if -(-n[c] // 128) == -(-max(n[c] - 48, 1) // 128):
                continue
            for a in sorted(members[c]):
                if len(members[c]) <= min_core:
                    break
                targets = sorted({int(core_of[b]) for b in nbr[a] if core_of[b] != c})
                best = None
                for d in targets:
                    members[c].discard(a)
                    members[d].add(a)
                    nc, nd = orbs(c), orbs(d)
                    members[d].discard(a)
                    members[c].add(a)
                    delta = refine_score(nc) + refine_score(nd) - refine_score(n[c]) - refine_score(n[d])
                    if delta < 0 and (best is None or delta < best[0]):
                        best = (delta, d, nc, nd)
                if best is not None:
                    _, d, nc, nd = best
                    members[c].discard(a)
                    members[d].add(a)
                    core_of[a] = d
                    n[c], n[d] = nc, nd
                    moves += 1
        if moves == 0:
            break
    after = sum(refine_score(x) for x in n)
    return [np.asarray(sorted(m), dtype=np.int32) for m in members], before, after
