"""Message-passing preconditioner network: forward and backward (FP64 oracle).

Test infrastructure only (see ``oracle/__init__``).

The kernel K = J^-1 of the electronic equation of motion (Eq. HW, SI Eq. "Jacobian") is
approximated by K_NN(y) = -c y + G(y), where G is a message-passing network on the atom
graph that is linear in the residual vector y (the paper mentions data-driven acceleration
as an extension; the network form is this project's reading):

    h0_i      = y_i e[s_i]                                    (e: species embedding, 3 x 64)
    a^l_i     = sum_{j in N(i)} phi_l(r_ij) * h^l_j           (channel-wise radial filter)
    h^{l+1}_i = h^l_i + A_l a^l_i + B_l h^l_i                 (l = 0, 1, 2; A_l, B_l 64 x 64)
    G(y)_i    = w . h^3_i
    phi_l(r)  = sum_b C_l[b] exp(-((r - m_b)/sig)^2) fc(r),   m_b = linspace(0.8, 6.0, 8) A,
                sig = 0.7 A, fc(r) = (cos(pi r / 6.0) + 1)/2 for r < 6 A, else 0.

Training minimises the mean over pairs (x, v) of |K_NN(x) - v|^2 with x = J v.  Parameters are
a flat vector in the order e, then for each layer C_l (8 x 64), A_l, B_l, then w.
Pinned by tests: the gradient equals a central finite difference; linearity in y; with all
weights zero the network is K0 = -c I.
"""
from __future__ import annotations

import numpy as np

WIDTH = 64
NBASIS = 8
NLAYER = 3
R_CUT = 6.0
SIG = 0.7
CENTERS = np.linspace(0.8, 6.0, NBASIS)


def n_params() -> int:
    return 3 * WIDTH + NLAYER * (NBASIS * WIDTH + 2 * WIDTH * WIDTH) + WIDTH


def unpack(p: np.ndarray) -> dict:
    p = np.asarray(p, dtype=np.float64)
    o = 0
    out = {"e": p[o:o + 3 * WIDTH].reshape(3, WIDTH)}
    o += 3 * WIDTH
    out["C"], out["A"], out["B"] = [], [], []
    for _ in range(NLAYER):
        out["C"].append(p[o:o + NBASIS * WIDTH].reshape(NBASIS, WIDTH)); o += NBASIS * WIDTH
        out["A"].append(p[o:o + WIDTH * WIDTH].reshape(WIDTH, WIDTH)); o += WIDTH * WIDTH
        out["B"].append(p[o:o + WIDTH * WIDTH].reshape(WIDTH, WIDTH)); o += WIDTH * WIDTH
    out["w"] = p[o:o + WIDTH]
    return out


def pack(d: dict) -> np.ndarray:
    parts = [d["e"].ravel()]
    for l in range(NLAYER):
        parts += [d["C"][l].ravel(), d["A"][l].ravel(), d["B"][l].ravel()]
    parts.append(d["w"].ravel())
    return np.concatenate(parts)


def init_params(seed: int) -> np.ndarray:
    """Seeded initial weights (normal, scaled by 1/sqrt(fan-in); small output layer)."""
    rng = np.random.default_rng(seed)
    d = {"e": rng.standard_normal((3, WIDTH)) * 0.1,
         "C": [rng.standard_normal((NBASIS, WIDTH)) * 0.1 for _ in range(NLAYER)],
         "A": [rng.standard_normal((WIDTH, WIDTH)) / np.sqrt(WIDTH) * 0.1 for _ in range(NLAYER)],
         "B": [rng.standard_normal((WIDTH, WIDTH)) / np.sqrt(WIDTH) * 0.1 for _ in range(NLAYER)],
         "w": rng.standard_normal(WIDTH) * 0.01}
    return pack(d)


def edge_basis(r: np.ndarray) -> np.ndarray:
    """Radial basis [E, NBASIS] with the cosine cutoff."""
    fc = np.where(r < R_CUT, 0.5 * (np.cos(np.pi * r / R_CUT) + 1.0), 0.0)
    return np.exp(-((r[:, None] - CENTERS[None, :]) / SIG) ** 2) * fc[:, None]


def edges_from_csr(row_ptr, col, R, box):
    """(i, j, r_ij) for every directed CSR edge, minimum-image distance in Angstrom."""
    rows = np.repeat(np.arange(len(row_ptr) - 1), np.diff(row_ptr))
    d = R[col] - R[rows]
    d = d - box * np.round(d / box)
    return rows, np.asarray(col, dtype=np.int64), np.sqrt(np.sum(d * d, axis=1))


def forward(p, y, species, edges, c_k0: float, keep: bool = False):
    """K_NN(y) = -c y + G(y).  edges = (i, j, r)."""
    d = unpack(p)
    i, j, r = edges
    bas = edge_basis(r)
    h = y[:, None] * d["e"][species]
    hs, as_ = [h], []
    for l in range(NLAYER):
        phi = bas @ d["C"][l]                                   # [E, 64]
        a = np.zeros_like(h)
        np.add.at(a, i, phi * h[j])
        h = h + a @ d["A"][l].T + h @ d["B"][l].T
        as_.append(a)
        hs.append(h)
    u = -c_k0 * y + h @ d["w"]
    if keep:
        return u, {"hs": hs, "as": as_, "bas": bas}
    return u


def backward(p, y, species, edges, c_k0: float, gu):
    """Gradient of sum_i gu_i K_NN(y)_i with respect to the flat parameter vector."""
    d = unpack(p)
    i, j, r = edges
    _, cache = forward(p, y, species, edges, c_k0, keep=True)
    hs, as_, bas = cache["hs"], cache["as"], cache["bas"]
    g = {"e": np.zeros_like(d["e"]), "C": [None] * NLAYER, "A": [None] * NLAYER, "B": [None] * NLAYER}
    g["w"] = hs[-1].T @ gu
    gh = gu[:, None] * d["w"][None, :]
    for l in reversed(range(NLAYER)):
        h, a = hs[l], as_[l]
        g["A"][l] = gh.T @ a
        g["B"][l] = gh.T @ h
        ga = gh @ d["A"][l]
        phi = bas @ d["C"][l]
        # d/dphi of sum_i ga_i . sum_j phi_ij h_j  ->  per edge ga_i * h_j
        gphi = ga[i] * h[j]
        g["C"][l] = bas.T @ gphi
        gprev = gh + gh @ d["B"][l]
        np.add.at(gprev, j, phi * ga[i])                       # transpose of the aggregation
        gh = gprev
    # h0 = y e[s]
    for sp in range(3):
        m = species == sp
        g["e"][sp] = (y[m][:, None] * gh[m]).sum(axis=0)
    return pack(g)


def loss_and_grad(p, X, V, species, edges, c_k0: float):
    """Mean over pairs of |K_NN(x) - v|^2 and its gradient."""
    L = 0.0
    G = np.zeros_like(p)
    for x, v in zip(X, V):
        res = forward(p, x, species, edges, c_k0) - v
        L += float(res @ res)
        G += backward(p, x, species, edges, c_k0, 2.0 * res)
    return L / len(X), G / len(X)
