"""XL-BOMD trajectories on one GPU: energy conservation and the charge-response kernel.

    python -m paper_2606_03140_gb300.md --workload water9000 --steps 2000 --kernel 2 --out run.json

Kernel 0 is K0 = -c I.  Kernel 1 is the rank-m Krylov kernel from first-order SP2 responses
(SI Sec. B).  Kernel 2 is the learned message-passing preconditioner: it is trained on the GPU
on the (J v, v) pairs that the Krylov kernel generates during the first --train-steps steps,
then judged every 20 steps against the Krylov kernel, falling back to it above a relative
error of 0.1.  The run starts from the SCC ground state (paper_2606_03140_gb300.runs) and
reports:
- the drift of the total shadow energy (linear fit after --skip steps, Ha per atom per ps);
- its RMS fluctuation about that fit;
- the SCC iterations from a perturbed start, with the kernel of the run and, for kernel 2, with
  the Krylov kernel for comparison;
- the wall time per step.
With --jsonl the run also writes one JSON object per MD step (energies, and at the end of every
chunk of steps the chemical potential, the Fermi evaluations and the electron-count error of that
step's density).  With --checkpoint and --checkpoint-every it saves the XL-BOMD state
(sedacs_checkpoint_save) every that many steps; --resume continues from such a file instead of
computing a ground state (kernels 0 and 1; the SCC comparison from a perturbed start is skipped).
Argument marshalling and orchestration only: every step runs in the library's kernels.
"""
from __future__ import annotations

import argparse
import json
import time

import numpy as np

from . import inputs as I
from . import runs
from . import sedacs as S


def _params(precision: int, kernel: int, rank: int, scc_tol: float = 2e-5, md: bool = False):
    """Context parameters; md=True takes the dynamics' K0 constant (runs.MD_C_K0), else the
    SCC's default."""
    extra = {"c_k0": runs.MD_C_K0} if md else {}
    return S.sedacs_default_params(core_size=32, precision=precision, kernel=kernel, krylov_rank=rank,
                                   scc_tol=scc_tol, **extra)


def step_records(E, first_step: int, dt_fs: float, info: dict | None = None) -> list[dict]:
    """Per-step metric records of one chunk of steps: energies [m, 3] (kinetic, shadow potential,
    total; Ha); the density diagnostics `info` (sedacs_density_info of the chunk's last step)
    go on the last record."""
    out = []
    for i, (ek, ep, et) in enumerate(np.asarray(E, dtype=np.float64)):
        k = first_step + i + 1
        out.append({"step": k, "t_fs": k * dt_fs, "e_kin_ha": float(ek), "e_pot_ha": float(ep),
                    "e_tot_ha": float(et)})
    if info is not None and out:
        mu = info["history"][-1][0] + info["dmu_linear"] if info.get("history") else None
        out[-1].update({"mu_ha": mu, "fermi_evaluations": info["passes"], "count_err_e": info["count_err"]})
    return out


def _md(ctx, R, V, steps: int, dt: float, chunk: int = 50, first_step: int = 0, jsonl=None, ck_path=None,
        ck_every: int = 0):
    E = np.zeros((steps, 3))
    k = 0
    while k < steps:
        m = min(chunk, steps - k)
        if ck_every > 0:
            m = min(m, ck_every - (first_step + k) % ck_every)
        e = np.zeros((m, 3))
        S.sedacs_xlbomd_step(ctx, R, V, m, dt, e)
        E[k:k + m] = e
        if jsonl is not None:
            for rec in step_records(e, first_step + k, dt, S.sedacs_density_info(ctx)):
                jsonl.write(json.dumps(rec) + "\n")
            jsonl.flush()
        k += m
        if ck_path and ck_every > 0 and (first_step + k) % ck_every == 0:
            S.sedacs_checkpoint_save(ctx, ck_path)
    return E


def _scc_iterations(s, model, R0, n0, gd, mu0, precision, kernel, rank, gnn_params, perturb, seed=5):
    """Iterations of the SCC (to max |q - n| <= 2e-5 e, the ground-state tolerance) from the
    ground-state charges plus seeded noise of RMS `perturb`, on the ground state's density graph
    and chemical potential."""
    ctx = S.sedacs_create(s.species, s.box, model, _params(precision, kernel, rank))
    try:
        if gnn_params is not None:
            S.sedacs_gnn_set_params(ctx, gnn_params)
        R = np.ascontiguousarray(R0.copy())
        S.sedacs_graph_build(ctx, R, gd=gd)
        S.sedacs_partition(ctx, R)
        n = np.ascontiguousarray(n0 + perturb * np.random.default_rng(seed).standard_normal(len(n0)))
        n -= (n.sum() - n0.sum()) / len(n)          # keep the total charge
        t0 = time.perf_counter()
        mu, res, it, ok = S.sedacs_scc_step(ctx, R, n, max_iter=100, mu=mu0)
        return {"iterations": int(it), "converged": bool(ok), "residual": float(res),
                "seconds": time.perf_counter() - t0}
    finally:
        S.sedacs_destroy(ctx)


def _energy_stats(E, n_atoms: int, dt_fs: float, skip: int):
    t = np.arange(len(E)) * dt_fs / 1000.0                 # ps
    y = E[skip:, 2]
    tt = t[skip:]
    slope, icpt = np.polyfit(tt, y, 1)
    resid = y - (slope * tt + icpt)
    return {"drift_ha_per_atom_ps": float(slope / n_atoms), "fluct_rms_ha_per_atom": float(resid.std() / n_atoms),
            "fit_window_ps": [float(tt[0]), float(tt[-1])], "e_total_first_last": [float(E[0, 2]), float(E[-1, 2])],
            "e_kin_first_last": [float(E[0, 0]), float(E[-1, 0])]}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workload", default="water9000")
    ap.add_argument("--precision", type=int, default=1, choices=[0, 1, 2, 3, 4],
                    help="0 plain FP64; 1 FP32-class (SP2 squares in two fp16 planes, other products "
                         "three-way bf16); 4 FP32-class three-way bf16 throughout; 2, 3 diagnostics")
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--dt", type=float, default=0.25, help="fs")
    ap.add_argument("--kernel", type=int, default=0, choices=[0, 1, 2])
    ap.add_argument("--krylov-rank", type=int, default=4)
    ap.add_argument("--train-steps", type=int, default=200)
    ap.add_argument("--epochs", type=int, default=300)
    ap.add_argument("--lr", type=float, default=2e-3)
    ap.add_argument("--skip", type=int, default=400, help="steps left out of the drift fit (relaxation)")
    ap.add_argument("--scc-perturb", type=float, default=0.02, help="RMS charge noise of the SCC start (e)")
    ap.add_argument("--out", default=None)
    ap.add_argument("--jsonl", default=None, help="per-step metrics, one JSON object per line")
    ap.add_argument("--checkpoint", default=None, help="checkpoint file, written every --checkpoint-every steps")
    ap.add_argument("--checkpoint-every", type=int, default=0)
    ap.add_argument("--resume", default=None, help="continue from a checkpoint file (kernels 0 and 1)")
    ap.add_argument("--first-step", type=int, default=0,
                    help="number of the first step of this run (metrics and checkpoint cadence; for a resume)")
    args = ap.parse_args(argv)
    if args.resume and args.kernel == 2:
        ap.error("--resume continues kernels 0 and 1 only (the network's parameters are not in the file)")
    if args.checkpoint_every < 0 or (args.checkpoint_every > 0 and not args.checkpoint):
        ap.error("--checkpoint-every needs --checkpoint and a step count >= 1")

    if args.resume:
        s = I.workload(args.workload)
        model = I.default_model()
        prm = _params(args.precision, args.kernel, args.krylov_rank, md=True)
        ctx = S.sedacs_create(s.species, s.box, model, prm)
        S.sedacs_checkpoint_load(ctx, args.resume)
        R = np.zeros((s.n_atoms, 3))
        V = np.zeros((s.n_atoms, 3))
        info = {"resumed_from": args.resume}
    else:
        s, model, ctx, R, V, n0, info = runs.ground_state(args.workload, args.precision)
        R0 = R.copy()
        n0 = n0.copy()
        gd0 = S.sedacs_density_graph_get(ctx, s.n_atoms)
    N = s.n_atoms
    jsonl = open(args.jsonl, "a") if args.jsonl else None
    mdkw = {"jsonl": jsonl, "ck_path": args.checkpoint, "ck_every": args.checkpoint_every}
    s0 = args.first_step
    out = {"workload": args.workload, "n_atoms": N, "precision": args.precision, "kernel": args.kernel,
           "steps": args.steps, "dt_fs": args.dt, "ground_state": info}
    gnn = None
    try:
        t_md = 0.0
        if args.kernel == 2:
            # Krylov steps that also collect the training pairs of the network
            S.sedacs_set_params(ctx, _params(args.precision, 1, args.krylov_rank, md=True))
            S.sedacs_gnn_init(ctx, 3)
            S.sedacs_gnn_collect(ctx, True, min(1024, 4 * args.krylov_rank * args.train_steps))
            t0 = time.perf_counter()
            E1 = _md(ctx, R, V, args.train_steps, args.dt, first_step=s0, **mdkw)
            t_md += time.perf_counter() - t0
            S.sedacs_gnn_collect(ctx, False)
            t0 = time.perf_counter()
            l0, l1 = S.sedacs_gnn_train(ctx, epochs=args.epochs, lr=args.lr)
            out["training"] = {"loss_first": l0, "loss_last": l1, "seconds": time.perf_counter() - t0}
            gnn = S.sedacs_gnn_get_params(ctx)
            S.sedacs_set_params(ctx, _params(args.precision, 2, args.krylov_rank, md=True))
            t0 = time.perf_counter()
            E2 = _md(ctx, R, V, args.steps - args.train_steps, args.dt, first_step=s0 + args.train_steps, **mdkw)
            t_md += time.perf_counter() - t0
            E = np.concatenate([E1, E2])
            err, fallbacks = S.sedacs_kernel_judge(ctx)
            out["judge"] = {"last_relative_error": err, "fallbacks": fallbacks}
        else:
            if not args.resume:
                S.sedacs_set_params(ctx, _params(args.precision, args.kernel, args.krylov_rank, md=True))
            t0 = time.perf_counter()
            E = _md(ctx, R, V, args.steps, args.dt, first_step=s0, **mdkw)
            t_md += time.perf_counter() - t0
        out["ms_per_step"] = 1e3 * t_md / args.steps
        out["energy"] = _energy_stats(E, N, args.dt, min(args.skip, args.steps // 2))
        out["e_total_every_10"] = E[::10, 2].tolist()
    finally:
        S.sedacs_destroy(ctx)
        if jsonl is not None:
            jsonl.close()
    scc = {}
    if args.resume:
        pass
    elif args.kernel == 2:
        mu0 = info["mu"]
        scc["learned"] = _scc_iterations(s, model, R0, n0, gd0, mu0, args.precision, 2, args.krylov_rank, gnn,
                                         args.scc_perturb)
        scc["krylov"] = _scc_iterations(s, model, R0, n0, gd0, mu0, args.precision, 1, args.krylov_rank, None,
                                        args.scc_perturb)
    else:
        mu0 = info["mu"]
        scc[["k0", "krylov"][args.kernel]] = _scc_iterations(s, model, R0, n0, gd0, mu0, args.precision,
                                                             args.kernel, args.krylov_rank, None, args.scc_perturb)
    out["scc_from_perturbed_start"] = scc
    txt = json.dumps(out)
    if args.out:
        with open(args.out, "w") as f:
            f.write(txt)
    print(json.dumps({k: v for k, v in out.items() if k != "e_total_every_10"}))


if __name__ == "__main__":
    main()
