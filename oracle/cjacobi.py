"""ctypes access to the plain-C parts of the oracle: the cyclic Jacobi eigensolver and subgraph
solve (``oracle/csrc/jacobi.c``) and the bisection for mu on the collected count
(``oracle/csrc/mu.c``).

Test infrastructure only (see ``oracle/__init__``).  The library is compiled with gcc (no vendor
or CUDA code, no -march flags, IEEE arithmetic) into ``oracle/_build/`` by the package build step,
or here on first use when it is missing or older than its sources.

Pinned by tests: the 2 x 2 closed form; the eigenvalues a + 2 b cos(k pi / (n + 1)) of the
tridiagonal Toeplitz matrix; a spectrum planted by an orthogonal similarity; eigenvectors
orthonormal and A V = V diag(w); the subgraph solve against the LAPACK route of
``density.subgraph_setup`` (eigenvalues, Z s Z = I, core weights) on water subgraphs; mu in the
gap with the exact count in the full limit and against a brute-force scan of the count on a
truncated graph (``tests/test_oracle_density.py``); the count against a plain sum.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
SRCS = [os.path.join(_HERE, "csrc", f) for f in ("jacobi.c", "mu.c")]
LIB = os.path.join(_HERE, "_build", "liboracle.so")
_lib = None


def compile_lib(force: bool = False) -> str:
    """gcc -O2 -fopenmp shared library from the C sources (rebuilt when a source is newer)."""
    if force or not os.path.exists(LIB) or any(os.path.getmtime(LIB) < os.path.getmtime(f) for f in SRCS):
        os.makedirs(os.path.dirname(LIB), exist_ok=True)
        tmp = LIB + f".{os.getpid()}.tmp"
        subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-o", tmp, *SRCS, "-lm"], check=True)
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(compile_lib())
        P = C.c_void_p
        lib.oracle_jacobi_eigh.argtypes = [C.c_int, P, P, P, P]
        lib.oracle_jacobi_eigh.restype = C.c_int
        lib.oracle_subgraph_eig.argtypes = [C.c_int, C.c_int, P, P, P, P, P, P, P]
        lib.oracle_subgraph_eig.restype = C.c_int
        lib.oracle_subgraph_eig_batch.argtypes = [C.c_int, P, P, P, P, P, P, P, P, P, P, P, P]
        lib.oracle_subgraph_eig_batch.restype = C.c_int
        lib.oracle_collected_count.argtypes = [C.c_int64, P, P, C.c_double, C.c_double]
        lib.oracle_collected_count.restype = C.c_double
        lib.oracle_solve_mu.argtypes = [C.c_int64, P, P, C.c_double, C.c_double, P]
        lib.oracle_solve_mu.restype = C.c_int
        _lib = lib
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(C.c_void_p)


def eigh(a: np.ndarray):
    """Eigenvalues (ascending) and eigenvectors (columns) of a symmetric matrix; also the sweep
    count.  Raises on no convergence."""
    lib = _load()
    a = np.array(a, dtype=np.float64, order="C", copy=True)
    n = a.shape[0]
    v = np.zeros((n, n))
    w = np.zeros(n)
    work = np.zeros(n * n + n)
    st = lib.oracle_jacobi_eigh(n, _p(a), _p(v), _p(w), _p(work))
    if st < 0:
        raise RuntimeError(f"Jacobi eigensolver failed ({st})")
    return w, v, st


def subgraph_eig(h: np.ndarray, s: np.ndarray, n_core_orb: int):
    """Z = s^-1/2, eigenpairs of h~ = Z h Z and core weights of one subgraph: (Z, eps, X, C, w)."""
    lib = _load()
    h = np.ascontiguousarray(h, dtype=np.float64)
    s = np.ascontiguousarray(s, dtype=np.float64)
    n = h.shape[0]
    z = np.zeros((n, n))
    x = np.zeros((n, n))
    cst = np.zeros((n, n))
    eps = np.zeros(n)
    w = np.zeros(n)
    st = lib.oracle_subgraph_eig(n, int(n_core_orb), _p(h), _p(s), _p(z), _p(eps), _p(x), _p(cst), _p(w))
    if st != 0:
        raise RuntimeError(f"subgraph solve failed ({st})")
    return z, eps, x, cst, w


def subgraph_eig_batch(blocks):
    """subgraph_eig over a list of (h, s, n_core_orb), spread over the host's threads."""
    lib = _load()
    k = len(blocks)
    n = np.array([b[0].shape[0] for b in blocks], dtype=np.int32)
    nco = np.array([int(b[2]) for b in blocks], dtype=np.int32)
    sq = np.zeros(k + 1, dtype=np.int64)
    sq[1:] = np.cumsum(n.astype(np.int64) ** 2)
    vo = np.zeros(k + 1, dtype=np.int64)
    vo[1:] = np.cumsum(n)
    H = np.concatenate([np.ascontiguousarray(b[0], dtype=np.float64).ravel() for b in blocks]) if k else np.zeros(1)
    S = np.concatenate([np.ascontiguousarray(b[1], dtype=np.float64).ravel() for b in blocks]) if k else np.zeros(1)
    Z = np.zeros_like(H)
    X = np.zeros_like(H)
    Cs = np.zeros_like(H)
    E = np.zeros(max(int(vo[-1]), 1))
    W = np.zeros_like(E)
    status = np.zeros(max(k, 1), dtype=np.int32)
    st = lib.oracle_subgraph_eig_batch(k, _p(n), _p(nco), _p(sq), _p(vo), _p(H), _p(S), _p(Z), _p(E), _p(X),
                                       _p(Cs), _p(W), _p(status))
    if st != 0:
        raise RuntimeError(f"subgraph solve failed ({st})")
    out = []
    for i in range(k):
        m = int(n[i])
        a, b = int(sq[i]), int(sq[i + 1])
        out.append((Z[a:b].reshape(m, m), E[vo[i]:vo[i + 1]].copy(), X[a:b].reshape(m, m), Cs[a:b].reshape(m, m),
                    W[vo[i]:vo[i + 1]].copy()))
    return out


def _flat(eps_list, w_list):
    e = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in eps_list]))
    w = np.ascontiguousarray(np.concatenate([np.asarray(x, dtype=np.float64).ravel() for x in w_list]))
    if e.shape != w.shape:
        raise ValueError("one core weight per state")
    return e, w


def collected_count(eps_list, w_list, mu: float, beta: float) -> float:
    """N(mu) = 2 sum_i sum_k w_ik f(eps_ik - mu) (Eq. 2), summed in C in state order."""
    e, w = _flat(eps_list, w_list)
    return float(_load().oracle_collected_count(len(e), _p(e), _p(w), float(mu), float(beta)))


def solve_mu(eps_list, w_list, n_e: float, beta: float) -> float:
    """mu of Eq. 2 by bisection in C (bracket [min eps - 1, max eps + 1], |N - N_e| < 1e-11 or a
    bracket narrower than 1e-15 Ha)."""
    e, w = _flat(eps_list, w_list)
    mu = C.c_double()
    st = _load().oracle_solve_mu(len(e), _p(e), _p(w), float(n_e), float(beta), C.byref(mu))
    if st < 0:
        raise ValueError("mu bisection needs at least one state and finite inputs")
    return mu.value
