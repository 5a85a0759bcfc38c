"""Run drivers on top of the C ABI: the SCC ground state an XL-BOMD run starts from.

Used by bench.py and by the trajectory tool (python -m paper_2606_03140_gb300.md).  Argument
marshalling and orchestration only: every step runs in the library's kernels.
"""
from __future__ import annotations

import numpy as np

from . import inputs as I
from . import sedacs as S


class NoGroundState(RuntimeError):
    """The SCC did not reach the ground state."""


# K0 = -c I for the dynamics: at 300 K mu sits at a band edge and atoms holding a level within
# a few kT of mu respond to a charge change with dq/dn of order -100, so the scaled-delta kernel
# must stay small for the charge integrator (kappa c |dq/dn - 1| <= 4) to remain stable; c = 0.5
# diverges within ~30 steps of the 9,000-atom box, 0.05 and 0.01 are stable over 100 steps.
MD_C_K0 = 0.05


def ground_state(workload: str, precision: int, seed_v: int = 20260703, quick: bool = False,
                 core_size: int = 32, refine: bool = False):
    """SCC ground state (mu from Eq. 2 at 300 K) and Maxwell-Boltzmann velocities at 300 K.

    Returns (system, model, ctx, R, V, n, info) with ctx ready for sedacs_xlbomd_init (kernel
    K0).  The ground state comes from the kernel-accelerated quasi-Newton SCC (SI Sec. C, rank-4
    Krylov) in the three-plane bf16 form (precision 4, 24-bit products); a context of the
    requested form (FP64 plain, or form 1) then receives its charges, mu and density graph, so
    all forms start from the same state.
    quick=True starts from zero charges (same per-step work, no SCC).
    refine=True refines the recursive-bisection cores for the 128-orbital tiles of the subgraph
    solves (sedacs_refine_cores) after each partition."""
    s = I.workload(workload)
    model = I.default_model()
    R = np.ascontiguousarray(s.R.copy())
    n = np.zeros(s.n_atoms)
    V = np.ascontiguousarray(I.maxwell_boltzmann(s.species, 300.0, seed_v, model))
    scc_precision = 4 if precision in (0, 1) else precision
    prm = S.sedacs_default_params(core_size=core_size, precision=scc_precision,
                                  scc_tol=2e-5, kernel=1, krylov_rank=4)
    ctx = S.sedacs_create(s.species, s.box, model, prm)
    S.sedacs_graph_build(ctx, R)
    S.sedacs_partition(ctx, R)
    if refine:
        S.sedacs_refine_cores(ctx)
    it = it2 = 0
    res2 = None
    if quick:
        mu, _, _, _ = S.sedacs_subgraph_density(ctx, R, n)
        S.sedacs_graph_build(ctx, R, use_prev_D=True)
    else:
        mu, res2, it, ok = S.sedacs_scc_step(ctx, R, n, max_iter=60)
        if not ok:
            S.sedacs_destroy(ctx)
            raise NoGroundState(f"{workload}: SCC ground state not reached (max residual {res2})")
    if precision != scc_precision:
        gd = S.sedacs_density_graph_get(ctx, s.n_atoms)
        S.sedacs_destroy(ctx)
        prm = S.sedacs_default_params(core_size=core_size, precision=precision)
        ctx = S.sedacs_create(s.species, s.box, model, prm)
        S.sedacs_graph_build(ctx, R, gd=gd)
        S.sedacs_partition(ctx, R)
        if refine:
            S.sedacs_refine_cores(ctx)
    # dynamics with the scaled-delta kernel K0 = -c I (SI Sec. B)
    prm.kernel = 0
    prm.c_k0 = MD_C_K0
    S.sedacs_set_params(ctx, prm)
    S.sedacs_xlbomd_init(ctx, R, V, n, mu)
    return s, model, ctx, R, V, n, {"scc_iters": it, "scc_resid": res2, "mu": mu}
