"""Checkpoint round trip of the XL-BOMD state through the C ABI (96-atom water box).

Three steps, save, four more steps; then a fresh context with the same parameters loads the file
and runs the same four steps.  The resumed trajectory must reproduce the continued one: positions,
velocities, dynamical charges and energies.  The force scatter adds pair reactions with FP64
atomics, whose order may differ between runs, so the bound is the run-to-run level (1e-10
relative), and the test reports whether the resume was bit-identical.  A file written for another
precision form is refused (SEDACS_EINVAL), a truncated file too (SEDACS_EIO).
"""
import os

import numpy as np
import pytest

from oracle import density as odn
from oracle import graph as og
from paper_2606_03140_gb300 import inputs as I

pytestmark = pytest.mark.gpu


def _start(S, s, m, precision):
    prm = S.sedacs_default_params(core_size=12, precision=precision, c_k0=0.05)
    ctx = S.sedacs_create(s.species, s.box, m, prm)
    R = np.ascontiguousarray(s.R.copy())
    n0 = np.ascontiguousarray(I.random_charges(96, 5, 0.02))
    rp, col = og.build_graph(s.R, s.box, 3.0)
    cores = og.rcb_partition(s.R, s.box, 12)
    r0 = odn.density(s.R, s.species, s.box, m, n0, cores, og.halos(rp, col, cores))
    S.sedacs_graph_build(ctx, R)
    S.sedacs_partition(ctx, R)
    S.sedacs_graph_build(ctx, R, gd=r0.gd)
    mu, _, _, _ = S.sedacs_subgraph_density(ctx, R, n0)
    V = np.ascontiguousarray(I.maxwell_boltzmann(s.species, 300.0, 9, m))
    S.sedacs_xlbomd_init(ctx, R, V, n0, mu)
    return prm, ctx, R, V


@pytest.mark.parametrize("precision", [0, 1])
def test_checkpoint_round_trip(tmp_path, precision):
    from paper_2606_03140_gb300 import sedacs as S

    s = I.workload("water96")
    m = I.default_model()
    path = os.path.join(tmp_path, "md.ck")
    prm, ctx, R, V = _start(S, s, m, precision)
    try:
        S.sedacs_xlbomd_step(ctx, R, V, 3, 0.25)
        S.sedacs_checkpoint_save(ctx, path)
        na = np.zeros(96)
        Ea = S.sedacs_xlbomd_step(ctx, R, V, 4, 0.25, n_out=na)
        Ra, Va = R.copy(), V.copy()
    finally:
        S.sedacs_destroy(ctx)
    ctx = S.sedacs_create(s.species, s.box, m, prm)
    try:
        S.sedacs_checkpoint_load(ctx, path)
        Rb = np.zeros_like(Ra)
        Vb = np.zeros_like(Va)
        nb = np.zeros(96)
        Eb = S.sedacs_xlbomd_step(ctx, Rb, Vb, 4, 0.25, n_out=nb)
    finally:
        S.sedacs_destroy(ctx)
    dR, dV, dn, dE = (float(np.max(np.abs(a - b))) for a, b in ((Ra, Rb), (Va, Vb), (na, nb), (Ea, Eb)))
    exact = dR == 0.0 and dV == 0.0 and dn == 0.0 and dE == 0.0
    print(f"[parity] water96 checkpoint round trip, form {precision}: max|dR| {dR:.1e} A, |dV| {dV:.1e}, "
          f"|dn| {dn:.1e} e, |dE| {dE:.1e} Ha, bit-identical: {exact}")
    assert dR <= 1e-10 and dV <= 1e-10 and dn <= 1e-10 and dE <= 1e-10 * np.max(np.abs(Ea))


def test_checkpoint_refuses_other_form_and_truncated_file(tmp_path):
    from paper_2606_03140_gb300 import sedacs as S

    s = I.workload("water96")
    m = I.default_model()
    path = os.path.join(tmp_path, "md.ck")
    prm, ctx, R, V = _start(S, s, m, 0)
    try:
        S.sedacs_xlbomd_step(ctx, R, V, 1, 0.25)
        S.sedacs_checkpoint_save(ctx, path)
    finally:
        S.sedacs_destroy(ctx)
    other = S.sedacs_create(s.species, s.box, m, S.sedacs_default_params(core_size=12, precision=1))
    try:
        with pytest.raises(S.SedacsError):
            S.sedacs_checkpoint_load(other, path)
    finally:
        S.sedacs_destroy(other)
    with open(path, "rb") as f:
        data = f.read()
    cut = os.path.join(tmp_path, "cut.ck")
    with open(cut, "wb") as f:
        f.write(data[: len(data) // 2])
    ctx = S.sedacs_create(s.species, s.box, m, prm)
    try:
        with pytest.raises(S.SedacsError):
            S.sedacs_checkpoint_load(ctx, cut)
    finally:
        S.sedacs_destroy(ctx)
