"""Thin ctypes binding of libsedacs.so (the C ABI in include/sedacs.h).

Argument marshalling only: every step of the method runs in the CUDA library.  Functions
carry the names of the C entry points.  Array arguments are numpy arrays (host I/O) or
torch CUDA tensors (after ``sedacs_set_device_io``).  Importing this module fails loudly
when the shared library is missing; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsedacs.so")

STATUS = {0: "SEDACS_OK", 1: "SEDACS_EINVAL", 2: "SEDACS_ENOMEM", 3: "SEDACS_ECUDA", 4: "SEDACS_ENOCONV",
          5: "SEDACS_ETIMEOUT", 6: "SEDACS_ENUMERIC", 7: "SEDACS_EPRECISION", 8: "SEDACS_ECAPACITY",
          9: "SEDACS_EIO"}


class SedacsError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class sedacs_model(C.Structure):
    _fields_ = [("n_orb", C.c_int32 * 3), ("eps_s", C.c_double * 3), ("eps_p", C.c_double * 3),
                ("hubbard_u", C.c_double * 3), ("z_val", C.c_double * 3), ("mass", C.c_double * 3),
                ("v0", C.c_double * 36), ("decay", C.c_double), ("overlap_scale", C.c_double),
                ("r_on", C.c_double), ("r_off", C.c_double), ("rep_a", C.c_double * 9), ("rep_decay", C.c_double)]


class sedacs_params(C.Structure):
    _fields_ = [("r_graph", C.c_double), ("tau", C.c_double), ("core_size", C.c_int32), ("precision", C.c_int32),
                ("kernel", C.c_int32), ("krylov_rank", C.c_int32), ("krylov_tol", C.c_double),
                ("c_k0", C.c_double), ("scc_tol", C.c_double), ("scc_alpha", C.c_double),
                ("sp2_tol", C.c_double), ("sp2_kmax", C.c_int32), ("ns_iters", C.c_int32),
                ("ewald_tol", C.c_double), ("judge_every", C.c_int32), ("judge_tol", C.c_double),
                ("Te", C.c_double), ("mu_given", C.c_int32), ("fermi_lin", C.c_double),
                ("graph_rule", C.c_int32), ("graph_alpha", C.c_double)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libsedacs.so is not built ({LIB_PATH}); run paper_2606_03140_gb300/build.py")
    lib = C.CDLL(LIB_PATH)
    P, I32, I64, D = C.c_void_p, C.c_int32, C.c_int64, C.c_double
    sig = {
        "sedacs_default_params": (None, [P]),
        "sedacs_create": (I32, [I32, P, P, P, P, P]),
        "sedacs_destroy": (None, [P]),
        "sedacs_last_error": (C.c_char_p, [P]),
        "sedacs_set_device_io": (I32, [P, I32, P]),
        "sedacs_graph_build": (I32, [P, P, P, P, P, I64, I32, P]),
        "sedacs_graph_get": (I32, [P, P, P]),
        "sedacs_partition": (I32, [P, P, P]),
        "sedacs_set_cores": (I32, [P, I32, P, P]),
        "sedacs_update_halos": (I32, [P]),
        "sedacs_parts_sizes": (I32, [P, P, P]),
        "sedacs_parts_get": (I32, [P, P, P, P]),
        "sedacs_coulomb_potential": (I32, [P, P, P, P]),
        "sedacs_subgraph_density": (I32, [P, P, P, P, P, P, P]),
        "sedacs_energy": (I32, [P, P]),
        "sedacs_forces": (I32, [P, P]),
        "sedacs_density_graph_size": (I32, [P, P]),
        "sedacs_density_graph_get": (I32, [P, P, P, P]),
        "sedacs_subgraph_matrix": (I32, [P, I32, I32, P, P, P]),
        "sedacs_charge_response": (I32, [P, P, P]),
        "sedacs_kernel_apply": (I32, [P, P, P, P]),
        "sedacs_scc_step": (I32, [P, P, P, I32, P, P, P]),
        "sedacs_xlbomd_init": (I32, [P, P, P, P, D]),
        "sedacs_xlbomd_step": (I32, [P, P, P, I32, D, P, P]),
        "sedacs_phase_times": (I32, [P, P, P]),
        "sedacs_reset_counters": (I32, [P]),
        "sedacs_kernel_stats": (I32, [P, I32, P, P, P]),
        "sedacs_kernel_stats_fp16": (I32, [P, P, P, P, P]),
        "sedacs_checkpoint_save": (I32, [P, C.c_char_p]),
        "sedacs_selftest_wait": (I32, [P, I32]),
        "sedacs_refine_cores": (I32, [P, I32, I32, P, P]),
        "sedacs_shard_lpt": (I32, [I32, P, I32, P, P]),
        "sedacs_checkpoint_load": (I32, [P, C.c_char_p]),
        "sedacs_set_params": (I32, [P, P]),
        "sedacs_graph_build_noalloc": (I32, [P, I32, P, D, P, P, I64, P, P]),
        "sedacs_gnn_num_params": (I32, []),
        "sedacs_gnn_init": (I32, [P, C.c_uint64]),
        "sedacs_gnn_set_params": (I32, [P, P]),
        "sedacs_gnn_get_params": (I32, [P, P, I32]),
        "sedacs_gnn_apply": (I32, [P, P, P]),
        "sedacs_gnn_param_grad": (I32, [P, P, P, P]),
        "sedacs_gnn_collect": (I32, [P, I32, I32]),
        "sedacs_gnn_train": (I32, [P, P, P, I32, I32, D, P, P]),
        "sedacs_kernel_judge": (I32, [P, P, P]),
        "sedacs_density_info": (I32, [P, P, I32]),
        "sedacs_charges": (I32, [P, P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_lib = _load()
EXPORTED = (
    "sedacs_default_params", "sedacs_create", "sedacs_destroy", "sedacs_last_error", "sedacs_set_device_io",
    "sedacs_graph_build", "sedacs_graph_get", "sedacs_partition", "sedacs_set_cores", "sedacs_update_halos",
    "sedacs_parts_sizes", "sedacs_parts_get", "sedacs_coulomb_potential", "sedacs_subgraph_density",
    "sedacs_energy", "sedacs_forces", "sedacs_density_graph_size", "sedacs_density_graph_get",
    "sedacs_subgraph_matrix", "sedacs_charge_response", "sedacs_kernel_apply", "sedacs_scc_step",
    "sedacs_xlbomd_init", "sedacs_xlbomd_step", "sedacs_phase_times", "sedacs_reset_counters",
    "sedacs_kernel_stats", "sedacs_set_params", "sedacs_graph_build_noalloc", "sedacs_gnn_num_params",
    "sedacs_gnn_init", "sedacs_gnn_set_params", "sedacs_gnn_get_params", "sedacs_gnn_apply", "sedacs_gnn_param_grad",
    "sedacs_gnn_collect", "sedacs_gnn_train", "sedacs_kernel_judge", "sedacs_density_info", "sedacs_charges",
    "sedacs_kernel_stats_fp16", "sedacs_checkpoint_save", "sedacs_checkpoint_load", "sedacs_selftest_wait",
    "sedacs_refine_cores", "sedacs_shard_lpt",
)


def _ptr(x):
    """Pointer of a numpy array (host) or torch tensor (device); None -> NULL."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags["C_CONTIGUOUS"], "arrays must be C-contiguous"
        return x.ctypes.data_as(C.c_void_p)
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous(), "tensors must be contiguous"
        return C.c_void_p(x.data_ptr())
    if isinstance(x, C._SimpleCData) or isinstance(x, C.Array):
        return C.cast(C.pointer(x), C.c_void_p)
    raise TypeError(f"unsupported array type {type(x)}")


def _check(ctx, st):
    if st != 0:
        msg = _lib.sedacs_last_error(ctx) if ctx else b""
        raise SedacsError(st, (msg or b"").decode())


def model_struct(model) -> sedacs_model:
    """sedacs_model from an inputs.SKModel."""
    m = sedacs_model()
    m.n_orb[:] = list(model.n_orb)
    m.eps_s[:] = list(model.eps_s)
    m.eps_p[:] = list(model.eps_p)
    m.hubbard_u[:] = list(model.hubbard_u)
    m.z_val[:] = list(model.z_val)
    m.mass[:] = list(model.mass)
    m.v0[:] = list(np.asarray(model.v0, dtype=np.float64).ravel())
    m.decay, m.overlap_scale, m.r_on, m.r_off = model.decay, model.overlap_scale, model.r_on, model.r_off
    m.rep_a[:] = list(np.asarray(model.rep_a, dtype=np.float64).ravel())
    m.rep_decay = model.rep_decay
    return m


def sedacs_default_params(**overrides) -> sedacs_params:
    p = sedacs_params()
    _lib.sedacs_default_params(C.byref(p))
    for k, v in overrides.items():
        setattr(p, k, v)
    return p


def sedacs_create(species, box, model, params) -> C.c_void_p:
    sp = np.ascontiguousarray(species, dtype=np.int32)
    bx = np.ascontiguousarray(box, dtype=np.float64)
    m = model_struct(model) if not isinstance(model, sedacs_model) else model
    out = C.c_void_p()
    _check(None, _lib.sedacs_create(len(sp), _ptr(sp), _ptr(bx), C.byref(m), C.byref(params), C.byref(out)))
    return out


def sedacs_destroy(ctx):
    _lib.sedacs_destroy(ctx)


def sedacs_set_params(ctx, params):
    _check(ctx, _lib.sedacs_set_params(ctx, C.byref(params)))


def sedacs_set_device_io(ctx, on: bool, stream: int = 0):
    _check(ctx, _lib.sedacs_set_device_io(ctx, 1 if on else 0, C.c_void_p(stream)))


def sedacs_graph_build(ctx, R, gd=None, use_prev_D=False) -> int:
    nnz = C.c_int64()
    if gd is not None:
        ptr, col, val = (np.ascontiguousarray(gd[0], np.int64), np.ascontiguousarray(gd[1], np.int32),
                         np.ascontiguousarray(gd[2], np.float64))
        _check(ctx, _lib.sedacs_graph_build(ctx, _ptr(R), _ptr(ptr), _ptr(col), _ptr(val), len(col), 0,
                                            C.byref(nnz)))
    else:
        _check(ctx, _lib.sedacs_graph_build(ctx, _ptr(R), None, None, None, 0, 1 if use_prev_D else 0,
                                            C.byref(nnz)))
    return nnz.value


def sedacs_graph_get(ctx, n_atoms: int, nnz: int):
    rp = np.zeros(n_atoms + 1, np.int64)
    col = np.zeros(max(nnz, 1), np.int32)
    _check(ctx, _lib.sedacs_graph_get(ctx, _ptr(rp), _ptr(col)))
    return rp, col[:nnz]


def sedacs_partition(ctx, R) -> int:
    n = C.c_int32()
    _check(ctx, _lib.sedacs_partition(ctx, _ptr(R), C.byref(n)))
    return n.value


def sedacs_set_cores(ctx, cores):
    ptr = np.zeros(len(cores) + 1, np.int64)
    ptr[1:] = np.cumsum([len(c) for c in cores])
    allc = np.ascontiguousarray(np.concatenate(cores), np.int32)
    _check(ctx, _lib.sedacs_set_cores(ctx, len(cores), _ptr(ptr), _ptr(allc)))


def sedacs_update_halos(ctx):
    _check(ctx, _lib.sedacs_update_halos(ctx))


def sedacs_parts_get(ctx):
    n = C.c_int32()
    tot = C.c_int64()
    _check(ctx, _lib.sedacs_parts_sizes(ctx, C.byref(n), C.byref(tot)))
    sp = np.zeros(n.value + 1, np.int64)
    sa = np.zeros(max(tot.value, 1), np.int32)
    nc = np.zeros(n.value, np.int32)
    _check(ctx, _lib.sedacs_parts_get(ctx, _ptr(sp), _ptr(sa), _ptr(nc)))
    return sp, sa[:tot.value], nc


def sedacs_coulomb_potential(ctx, R, b, V=None):
    out = np.zeros(len(b)) if V is None else V
    _check(ctx, _lib.sedacs_coulomb_potential(ctx, _ptr(R), _ptr(b), _ptr(out)))
    return out


def sedacs_subgraph_density(ctx, R, n, mu=float("nan"), q=None, n_parts=None):
    muc = C.c_double(mu)
    qo = np.zeros(len(n)) if q is None else q
    eb = C.c_double()
    it = np.zeros(n_parts, np.int32) if n_parts else None
    _check(ctx, _lib.sedacs_subgraph_density(ctx, _ptr(R), _ptr(n), C.byref(muc), _ptr(qo), C.byref(eb),
                                             _ptr(it) if it is not None else None))
    return muc.value, qo, eb.value, it


def sedacs_charges(ctx, n_atoms: int, q=None):
    out = np.zeros(n_atoms) if q is None else q
    _check(ctx, _lib.sedacs_charges(ctx, _ptr(out)))
    return out


def sedacs_energy(ctx):
    e = np.zeros(4)
    _check(ctx, _lib.sedacs_energy(ctx, _ptr(e)))
    return e


def sedacs_forces(ctx, n_atoms: int, F=None):
    out = np.zeros((n_atoms, 3)) if F is None else F
    _check(ctx, _lib.sedacs_forces(ctx, _ptr(out)))
    return out


def sedacs_density_graph_get(ctx, n_atoms: int):
    nnz = C.c_int64()
    _check(ctx, _lib.sedacs_density_graph_size(ctx, C.byref(nnz)))
    ptr = np.zeros(n_atoms + 1, np.int64)
    col = np.zeros(max(nnz.value, 1), np.int32)
    val = np.zeros(max(nnz.value, 1))
    _check(ctx, _lib.sedacs_density_graph_get(ctx, _ptr(ptr), _ptr(col), _ptr(val)))
    return ptr, col[:nnz.value], val[:nnz.value]


def sedacs_subgraph_matrix(ctx, part: int, which: int):
    n = C.c_int32()
    nc = C.c_int32()
    _check(ctx, _lib.sedacs_subgraph_matrix(ctx, part, which, None, C.byref(n), C.byref(nc)))
    rows = nc.value if which >= 4 else n.value
    out = np.zeros((rows, n.value))
    _check(ctx, _lib.sedacs_subgraph_matrix(ctx, part, which, _ptr(out), C.byref(n), C.byref(nc)))
    return out


def sedacs_charge_response(ctx, v, dq=None):
    out = np.zeros(len(v)) if dq is None else dq
    _check(ctx, _lib.sedacs_charge_response(ctx, _ptr(v), _ptr(out)))
    return out


def sedacs_kernel_apply(ctx, f, u=None):
    out = np.zeros(len(f)) if u is None else u
    r = C.c_int32()
    _check(ctx, _lib.sedacs_kernel_apply(ctx, _ptr(f), _ptr(out), C.byref(r)))
    return out, r.value


def sedacs_scc_step(ctx, R, n, max_iter: int = 200, mu: float = float("nan")):
    """n is updated in place; returns (mu, residual, iterations)."""
    muc = C.c_double(mu)
    res = C.c_double()
    it = C.c_int32()
    st = _lib.sedacs_scc_step(ctx, _ptr(R), _ptr(n), max_iter, C.byref(muc), C.byref(res), C.byref(it))
    if st not in (0, 4):
        _check(ctx, st)
    return muc.value, res.value, it.value, st == 0


def sedacs_xlbomd_init(ctx, R, V, n0, mu: float):
    _check(ctx, _lib.sedacs_xlbomd_init(ctx, _ptr(R), _ptr(V), _ptr(n0), mu))


def sedacs_xlbomd_step(ctx, R, V, nsteps: int, dt_fs: float, energies=None, n_out=None):
    """R, V are updated in place; returns energies [nsteps, 3]."""
    e = np.zeros((nsteps, 3)) if energies is None else energies
    _check(ctx, _lib.sedacs_xlbomd_step(ctx, _ptr(R), _ptr(V), nsteps, dt_fs, _ptr(e), _ptr(n_out)))
    return e


def sedacs_phase_times(ctx):
    t = np.zeros(8)
    n = C.c_int64()
    _check(ctx, _lib.sedacs_phase_times(ctx, _ptr(t), C.byref(n)))
    return t, n.value


def sedacs_reset_counters(ctx):
    _check(ctx, _lib.sedacs_reset_counters(ctx))


def sedacs_density_info(ctx) -> dict:
    """Diagnostics of the last density call (Te > 0)."""
    v = np.zeros(6 + 3 * 16)
    _check(ctx, _lib.sedacs_density_info(ctx, _ptr(v), len(v)))
    npass = int(v[3])
    return {"count_err": float(v[0]), "dn_dmu": float(v[1]), "dmu_linear": float(v[2]),
            "passes": npass, "doublings": int(v[4]), "reentries": int(v[5]),
            "history": [tuple(float(x) for x in v[6 + 3 * k:9 + 3 * k]) for k in range(min(npass, 16))]}


def sedacs_kernel_stats(ctx, on: bool = True):
    """(Fermi-operator product ms, launches, algorithmic flops: n^3 per symmetric product) since the last reset."""
    ms = C.c_double()
    nl = C.c_int64()
    fl = C.c_double()
    _check(ctx, _lib.sedacs_kernel_stats(ctx, 1 if on else 0, C.byref(ms), C.byref(nl), C.byref(fl)))
    return ms.value, nl.value, fl.value


def sedacs_kernel_stats_fp16(ctx):
    """(ms, launches, flops, algorithmic bytes) of the two-plane fp16 products since the last reset."""
    ms = C.c_double()
    nl = C.c_int64()
    fl = C.c_double()
    by = C.c_double()
    _check(ctx, _lib.sedacs_kernel_stats_fp16(ctx, C.byref(ms), C.byref(nl), C.byref(fl), C.byref(by)))
    return ms.value, nl.value, fl.value, by.value


def sedacs_refine_cores(ctx, rounds: int = 4, min_core: int = 16) -> tuple[int, int]:
    """Refine the cores for the 128-orbital tiles; returns (score before, score after)."""
    b = C.c_int64()
    a = C.c_int64()
    _check(ctx, _lib.sedacs_refine_cores(ctx, int(rounds), int(min_core), C.byref(b), C.byref(a)))
    return b.value, a.value


def sedacs_shard_lpt(cost, n_ranks: int):
    """LPT assignment of subgraphs (costs) to ranks: (owner per subgraph, load per rank)."""
    c = np.ascontiguousarray(cost, dtype=np.float64)
    owner = np.zeros(max(len(c), 1), np.int32)
    load = np.zeros(max(int(n_ranks), 1), np.float64)
    _check(None, _lib.sedacs_shard_lpt(len(c), _ptr(c), int(n_ranks), _ptr(owner), _ptr(load)))
    return owner[:len(c)], load[:int(n_ranks)]


def sedacs_selftest_wait(ctx, limit_us: int) -> int:
    """Run the bounded-wait self-test; returns the status (SEDACS_ETIMEOUT = 5 expected)."""
    return int(_lib.sedacs_selftest_wait(ctx, int(limit_us)))


def sedacs_checkpoint_save(ctx, path: str):
    """Write the XL-BOMD state of ctx to the file path."""
    _check(ctx, _lib.sedacs_checkpoint_save(ctx, str(path).encode()))


def sedacs_checkpoint_load(ctx, path: str):
    """Restore the XL-BOMD state written by sedacs_checkpoint_save into ctx (same atoms and parameters)."""
    _check(ctx, _lib.sedacs_checkpoint_load(ctx, str(path).encode()))


def sedacs_graph_build_noalloc(R_dev, box, r_graph: float, row_ptr_dev, col_dev, stream: int = 0) -> tuple[int, int]:
    """Distance graph into caller-owned device tensors, without any device allocation.

    R_dev float64 [N, 3], row_ptr_dev int64 [N+1], col_dev int32 [capacity] (torch CUDA tensors).
    Returns (status, nnz); status SEDACS_ECAPACITY (8) means col_dev is too small for nnz edges.
    """
    bx = np.ascontiguousarray(box, dtype=np.float64)
    nnz = C.c_int64()
    st = _lib.sedacs_graph_build_noalloc(_ptr(R_dev), int(R_dev.shape[0]), _ptr(bx), float(r_graph),
                                         _ptr(row_ptr_dev), _ptr(col_dev), int(col_dev.numel()), C.byref(nnz),
                                         C.c_void_p(stream))
    if st not in (0, 8):
        _check(None, st)
    return st, nnz.value


def sedacs_gnn_num_params() -> int:
    return int(_lib.sedacs_gnn_num_params())


def sedacs_gnn_init(ctx, seed: int):
    _check(ctx, _lib.sedacs_gnn_init(ctx, C.c_uint64(seed)))


def sedacs_gnn_set_params(ctx, p):
    p = np.ascontiguousarray(p, dtype=np.float64)
    _check(ctx, _lib.sedacs_gnn_set_params(ctx, _ptr(p)))


def sedacs_gnn_get_params(ctx, grad: bool = False):
    out = np.zeros(sedacs_gnn_num_params())
    _check(ctx, _lib.sedacs_gnn_get_params(ctx, _ptr(out), 1 if grad else 0))
    return out


def sedacs_gnn_apply(ctx, y):
    y = np.ascontiguousarray(y, dtype=np.float64)
    u = np.zeros_like(y)
    _check(ctx, _lib.sedacs_gnn_apply(ctx, _ptr(y), _ptr(u)))
    return u


def sedacs_gnn_param_grad(ctx, y, gu):
    y = np.ascontiguousarray(y, dtype=np.float64)
    gu = np.ascontiguousarray(gu, dtype=np.float64)
    g = np.zeros(sedacs_gnn_num_params())
    _check(ctx, _lib.sedacs_gnn_param_grad(ctx, _ptr(y), _ptr(gu), _ptr(g)))
    return g


def sedacs_gnn_collect(ctx, on: bool, capacity: int = 256):
    _check(ctx, _lib.sedacs_gnn_collect(ctx, 1 if on else 0, capacity))


def sedacs_gnn_train(ctx, X=None, V=None, epochs: int = 100, lr: float = 1e-3):
    l0 = C.c_double()
    l1 = C.c_double()
    if X is not None:
        X = np.ascontiguousarray(X, dtype=np.float64)
        V = np.ascontiguousarray(V, dtype=np.float64)
        _check(ctx, _lib.sedacs_gnn_train(ctx, _ptr(X), _ptr(V), X.shape[0], epochs, lr, C.byref(l0), C.byref(l1)))
    else:
        _check(ctx, _lib.sedacs_gnn_train(ctx, None, None, 0, epochs, lr, C.byref(l0), C.byref(l1)))
    return l0.value, l1.value


def sedacs_kernel_judge(ctx):
    e = C.c_double()
    n = C.c_int32()
    _check(ctx, _lib.sedacs_kernel_judge(ctx, C.byref(e), C.byref(n)))
    return e.value, n.value
