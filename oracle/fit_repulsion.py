"""Fit the repulsive pair amplitudes of the synthetic model once (writes oracle/repulsion_fit.json).

Test infrastructure only (see ``oracle/__init__``).  The paper's SCC-DFTB energy has a
repulsive pair term (SI Sec. D) whose parameters are not available; the synthetic
model's A_ZZ' exp(-r / 0.3 A) sw(r) amplitudes are chosen so that an isolated
molecule at its input geometry feels no force:

* water: A_OH and A_HH solve the in-plane force balance of H2O at the SCC charges;
* methanol: A_CH and A_CO by least squares with A_OH, A_HH fixed;
* A_OO = A_OH and A_CC = A_CH (pairs that occur only between molecules).

Run:  python -m oracle.fit_repulsion
"""
from __future__ import annotations

import json
import os

import numpy as np

from paper_2606_03140_gb300 import inputs as inp

from . import density as dn
from . import dynamics as dyn
from . import sk


def _isolated(kind: str):
    sp, pos = (inp._water_template() if kind == "water" else inp._methanol_template())
    box = np.array([60.0, 60.0, 60.0])
    return sp, pos - pos.mean(axis=0) + 30.0, box


def _pair_force_basis(R, sp, box, model, pairs):
    """Force per unit amplitude of each repulsive pair type (columns), flattened."""
    cols = []
    for (a, b) in pairs:
        rep = np.zeros((3, 3))
        rep[a, b] = rep[b, a] = 1.0
        m = inp.SKModel(rep_a=tuple(tuple(r) for r in rep))
        _, g = dn.repulsion(R, sp, box, m, with_grad=True)
        cols.append(-g.ravel())
    return np.stack(cols, axis=1)


def electronic_force(R, sp, box, model):
    gp = dyn.GraphParams(r_graph=3.0, tau=1e-3, core_size=len(sp))
    cores, halos = dn.full_partition(len(sp))
    n, res, _, _ = dyn.scc(R, sp, box, model, gp, cores=cores, tol=1e-10)
    return dn.forces(res, n, R, sp, box, model).ravel()


def main():
    base = inp.SKModel()
    H, C, O = inp.H, inp.C, inp.O
    sp, R, box = _isolated("water")
    fe = electronic_force(R, sp, box, base)
    B = _pair_force_basis(R, sp, box, base, [(O, H), (H, H)])
    a_oh, a_hh = np.linalg.lstsq(B, -fe, rcond=None)[0]
    sp2, R2, box2 = _isolated("methanol")
    fe2 = electronic_force(R2, sp2, box2, base)
    B2 = _pair_force_basis(R2, sp2, box2, base, [(O, H), (H, H), (C, H), (C, O)])
    rhs = -fe2 - B2[:, :2] @ np.array([a_oh, a_hh])
    a_ch, a_co = np.linalg.lstsq(B2[:, 2:], rhs, rcond=None)[0]
    fit = {"A": {"O-H": a_oh, "H-H": a_hh, "C-H": a_ch, "C-O": a_co, "O-O": a_oh, "C-C": a_ch},
           "note": "amplitudes in Hartree of A exp(-r/0.3 A) sw(r); written by oracle/fit_repulsion.py"}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "repulsion_fit.json")
    with open(path, "w") as fh:
        json.dump(fit, fh, indent=1)
    print(json.dumps(fit, indent=1))
    m = inp.default_model()
    for kind in ("water", "methanol"):
        s_, R_, b_ = _isolated(kind)
        f = electronic_force(R_, s_, b_, m)
        print(kind, "residual max |F| (Ha/A):", float(np.max(np.abs(f))))


if __name__ == "__main__":
    main()
