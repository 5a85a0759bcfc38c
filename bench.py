"""Benchmark: atoms x QMD-steps/s of graph-partitioned shadow XL-BOMD on one GB300.

Workload: the 9,000-atom water box (3,000 H2O, 44.8 A, seeded synthetic geometry, synthetic
sp SCC-TB model) -- cores of ~32 atoms, halos from the distance + |D| > 1e-3 graph,
Maxwell-Boltzmann velocities at 300 K, dt = 0.25 fs.  A step is one full QMD step: graph
rebuild from the previous density, halos, Coulomb (Ewald), H/S gather, S^-1/2, h~, the Fermi
operator at 300 K (tanh-doubling recursion on tcgen05) with mu solved from Eq. 2, core rows,
charges, energies, forces, kernel K(q - n), charge and Verlet updates.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--precision 1] [--workload water9000]

`value` times K steps with inputs resident on the device (device I/O through the C ABI);
`e2e` times K steps through the same public call with host arrays (H2D of R, V and D2H of
R, V and the energies inside the timed region).  N > 1 runs independent replicas, one per
rank (weak scaling); the engine itself is single-GPU.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=40)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", type=int, default=1, choices=[0, 1, 2, 3, 4],
                    help="0 plain FP64; 1 FP32-class (Fermi-recursion products in two fp16 planes, other "
                         "products three-way bf16); 4 FP32-class three-way bf16 throughout; 2, 3 diagnostics")
    ap.add_argument("--workload", default="water9000")
    ap.add_argument("--dt", type=float, default=0.25)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 sub-record")
    ap.add_argument("--no-frames", action="store_true", help="skip the oracle check of sampled frames")
    ap.add_argument("--refine-cores", action="store_true",
                    help="refine the recursive-bisection cores for the 128-orbital tiles (sedacs_refine_cores); "
                         "off by default: measured slower over the MD, as the density graph follows the cores")
    ap.add_argument("--profile-case", action="store_true",
                    help="small ncu case: 3,000-atom water box, two densities, the second inside NVTX range 'second'")
    ap.add_argument("--quick-setup", action="store_true",
                    help="start the dynamics from zero charges instead of the SCC ground state "
                         "(same per-step work; used to time the slow plain FP64 form)")
    return ap.parse_args()


METRIC = "atoms*QMD-steps/s at |dq|<=1e-5 e vs FP64 oracle (mixed vs plain, one GB300)"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) per launch of the Fermi-recursion
# product kernel (tc_gemm_persistent<2, true>) on the benchmarked 9,000-atom workload: the mean over
# its 136 launches in the NVTX range 'timed' of `bench.py --no-plain --no-frames --no-cpu-baseline
# --steps 2 --warmup 1` (one ncu pass, so the full workload could be captured); reported only while
# the kernel source is the one the counters were taken on, and on the cores the capture used (the
# recursive-bisection cores, not refined: refinement changes the subgraph sizes).
FERMI_TRAFFIC = {"kernel_sha1": "f1e27abead4ca70ebedad479f3f8cb922699ee59", "precision": 1,
                 "workload": "water9000", "core_refine": False, "bytes_per_launch": 998.1e6}


def strip_comments(src: str) -> str:
    """C/C++ source without comments and blank lines (string literals kept)."""
    out, i, n = [], 0, len(src)
    while i < n:
        c = src[i]
        if c == '"':
            j = i + 1
            while j < n and src[j] != '"':
                j += 2 if src[j] == "\\" else 1
            out.append(src[i:j + 1])
            i = j + 1
        elif src.startswith("//", i):
            while i < n and src[i] != "\n":
                i += 1
        elif src.startswith("/*", i):
            j = src.find("*/", i + 2)
            i = n if j < 0 else j + 2
        else:
            out.append(c)
            i += 1
    return "\n".join(line.rstrip() for line in "".join(out).splitlines() if line.strip())


def kernel_sha1() -> str:
    """sha1 of the GEMM kernel's source (dense_gemm.cu, dense.cuh, common.cuh), comments stripped."""
    import hashlib
    h = hashlib.sha1()
    for f in ("dense_gemm.cu", "dense.cuh", "common.cuh"):
        with open(os.path.join(ROOT, "paper_2606_03140_gb300", "csrc", f), encoding="utf-8") as fh:
            h.update(strip_comments(fh.read()).encode())
    return h.hexdigest()


UNIT = "atom-steps/s"


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        """Start sampling every 100 ms and wait (up to 3 s) for the first sample."""
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.idx), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
            t0 = time.time()
            while not self.lines and time.time() - t0 < 3.0:
                time.sleep(0.01)
        except Exception:
            self.proc = None
        self.t_mark = time.time()

    def mark(self):
        """Samples from now on belong to the timed region."""
        self.t_mark = time.time()

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append((time.time(), line.strip()))

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        return self.summarise(self.lines, self.t_mark)

    @staticmethod
    def summarise(lines, t_mark: float) -> dict:
        """Median SM clock, maximum clock and the throttle reasons seen active, over the
        (time, csv line) samples taken at or after t_mark."""
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for t, ln in lines:
            if t < t_mark:
                continue
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for k, nm in enumerate(names):
                if f[5 + k].lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group(backend="nccl" if os.environ.get("BENCH_BACKEND", "nccl") == "nccl" else "gloo")
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, x: float) -> float:
    """Maximum of x over the ranks (the slowest replica sets the job's time)."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([x], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def setup_system(S, I, workload: str, precision: int, seed_v: int = 20260703, quick: bool = False,
                 refine: bool = False):
    """SCC ground state and velocities, context ready for XL-BOMD (paper_2606_03140_gb300.runs)."""
    from paper_2606_03140_gb300 import runs

    try:
        return runs.ground_state(workload, precision, seed_v=seed_v, quick=quick, refine=refine)
    except runs.NoGroundState as e:
        # XL-BOMD starts from the SCC ground state; timing dynamics from an unconverged start
        # would time charge oscillations, not the method
        raise SystemExit(f"{e}; it is not an MD benchmark")


def frame_check(parts, R, n, q, mu, picks, model, species, box):
    """Charges of sampled subgraphs at one frame, recomputed by the FP64 oracle from the GPU's
    positions R, charges n, chemical potential mu and subgraph lists of that frame (parts, as
    sedacs_parts_get returned them right after the frame's step; the Coulomb potential only at
    the sampled atoms, its sums over every atom).  Returns max |q_gpu - q_oracle| there."""
    from oracle import density as odn
    from oracle import ewald as oew

    sp, sa, nc = parts
    cores = [sa[sp[i]:sp[i] + nc[i]] for i in picks]
    halos = [sa[sp[i] + nc[i]:sp[i + 1]] for i in picks]
    atoms = np.unique(np.concatenate([sa[sp[i]:sp[i + 1]] for i in picks]))
    V = oew.coulomb_potential(R, species, model.hubbard_u, box, n, rows=atoms)
    ref = odn.density(R, species, box, model, n, cores, halos, mu=mu, V=V, eig="lapack")
    a = np.concatenate(cores)
    d = np.abs(q[a] - ref.q[a])
    return float(np.max(d)), float(np.sqrt(np.mean(d ** 2))), int(np.sum(d > 1e-5)), int(d.shape[0])


def run_plain(args, S, model, s, R0, V0, n0, mu0, gd, cores, steps: int = 2):
    """The plain FP64 form from the same ground state: charges at the start (against the mixed
    form's) and the device-timed step."""
    import torch

    N = s.n_atoms
    prm = S.sedacs_default_params(core_size=32, precision=0)
    ctx = S.sedacs_create(s.species, s.box, model, prm)
    try:
        R = np.ascontiguousarray(R0.copy())
        V = np.ascontiguousarray(V0.copy())
        S.sedacs_graph_build(ctx, R, gd=gd)
        S.sedacs_partition(ctx, R)
        if args.refine_cores:
            S.sedacs_set_cores(ctx, cores)      # the mixed form's cores, so both forms share subgraphs
        S.sedacs_xlbomd_init(ctx, R, V, np.ascontiguousarray(n0), mu0)
        q0 = S.sedacs_charges(ctx, N)
        S.sedacs_xlbomd_step(ctx, R, V, 1, args.dt)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        S.sedacs_xlbomd_step(ctx, R, V, steps, args.dt)
        torch.cuda.synchronize()
        dt = (time.perf_counter() - t0) / steps
    finally:
        S.sedacs_destroy(ctx)
    return q0, dt


def run_ours(args, world, rank, local):
    import torch

    torch.cuda.set_device(local)
    from paper_2606_03140_gb300 import inputs as I
    from paper_2606_03140_gb300 import sedacs as S

    s, model, ctx, R, V, n, info = setup_system(S, I, args.workload, args.precision, quick=args.quick_setup,
                                                refine=args.refine_cores)
    N = s.n_atoms
    R0, V0, n0, mu0 = R.copy(), V.copy(), n.copy(), info["mu"]
    q_start = S.sedacs_charges(ctx, N)
    gd0 = S.sedacs_density_graph_get(ctx, N)
    sp0, sa0, nc0 = S.sedacs_parts_get(ctx)
    cores0 = [sa0[sp0[i]:sp0[i] + nc0[i]].copy() for i in range(len(nc0))]
    # warm-up (host I/O)
    S.sedacs_xlbomd_step(ctx, R, V, args.warmup, args.dt)
    # ---- device-resident timed region -------------------------------------------------
    stream = torch.cuda.current_stream()
    Rd = torch.from_numpy(R).cuda()
    Vd = torch.from_numpy(V).cuda()
    Ed = torch.zeros((args.steps, 3), dtype=torch.float64, device="cuda")
    S.sedacs_set_device_io(ctx, True, stream.cuda_stream)
    S.sedacs_reset_counters(ctx)
    clk = ClockSampler(local)
    clk.start()
    barrier(world)
    torch.cuda.synchronize()
    clk.mark()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(stream)
    S.sedacs_xlbomd_step(ctx, Rd, Vd, args.steps, args.dt, Ed)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    barrier(world)
    clocks = clk.stop()
    ms = e0.elapsed_time(e1)
    ms = allmax(world, ms)
    phases, launches = S.sedacs_phase_times(ctx)
    S.sedacs_set_device_io(ctx, False, 0)
    E = Ed.cpu().numpy()
    # ---- end to end through the public call with host buffers ----------------------------
    # (frames of this run are kept for the oracle check: positions, charges, density, mu)
    Rh = Rd.cpu().numpy().copy()
    Vh = Vd.cpu().numpy().copy()
    Eh = np.zeros((1, 3))
    nh = np.zeros(N)
    keep = sorted({0, args.steps // 2, args.steps - 1})
    frames, evals = [], []
    torch.cuda.synchronize()
    barrier(world)
    t_e2e = 0.0
    for k in range(args.steps):
        t0 = time.perf_counter()
        S.sedacs_xlbomd_step(ctx, Rh, Vh, 1, args.dt, Eh, nh)
        t_e2e += time.perf_counter() - t0
        dinf = S.sedacs_density_info(ctx)
        evals.append((dinf["passes"], dinf["reentries"]))
        if k in keep and rank == 0 and not args.no_frames:
            mu_k = dinf["history"][-1][0] + dinf["dmu_linear"]
            frames.append((k, Rh.copy(), nh.copy(), S.sedacs_charges(ctx, N), mu_k, S.sedacs_parts_get(ctx)))
    torch.cuda.synchronize()
    t_e2e = allmax(world, t_e2e)
    # roofline of the Fermi-operator products from a separate pass with per-launch CUDA events
    # (kept out of the timed region: the events read back after every density)
    S.sedacs_kernel_stats(ctx, True)
    S.sedacs_reset_counters(ctx)
    S.sedacs_kernel_stats(ctx, True)
    S.sedacs_xlbomd_step(ctx, Rh, Vh, 4, args.dt)
    k_ms, k_launch, k_flops = S.sedacs_kernel_stats(ctx, False)
    f16_ms, f16_launch, f16_flops, f16_bytes = S.sedacs_kernel_stats_fp16(ctx)
    ph4, _ = S.sedacs_phase_times(ctx)
    # oracle check of sampled subgraphs at the kept frames
    acc = None
    if frames:
        picks = [0, 97, 180, 280]
        nsub = S.sedacs_parts_get(ctx)[2].shape[0]
        picks = [p for p in picks if p < nsub]
        t0 = time.perf_counter()
        res = [frame_check(pf, Rf, nf, qf, muf, picks, model, s.species, s.box) for (_, Rf, nf, qf, muf, pf) in frames]
        errs = [r[0] for r in res]
        acc = {"max_dq_vs_oracle": max(errs), "rms_dq_vs_oracle": float(np.sqrt(np.mean([r[1] ** 2 for r in res]))),
               "atoms_above_1e-5": sum(r[2] for r in res), "atoms_checked": sum(r[3] for r in res),
               "per_frame": {str(k): r[0] for (k, *_), r in zip(frames, res)},
               "sampled_subgraphs": picks, "oracle_seconds": round(time.perf_counter() - t0, 1),
               "how": "FP64 oracle on the sampled subgraphs from the GPU's positions, charges n, mu and subgraph "
                      "lists at steps " + ",".join(str(f[0]) for f in frames) + " of the e2e trajectory"}
    S.sedacs_destroy(ctx)
    value = world * N * args.steps / (ms / 1e3)
    e2e = world * N * args.steps / t_e2e
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    bf16 = peaks.get("bf16_tflops_sustained", 1700.0)
    peak_src = "of measured" if "bf16_tflops_sustained" in peaks else "of fallback"
    split = {1: 3, 2: 3, 3: 1, 4: 6}.get(args.precision, 6)
    hbm = peaks.get("hbm_gbs", 6800.0)
    hbm_src = "of measured" if "hbm_gbs" in peaks else "of fallback"
    traffic = None
    if FERMI_TRAFFIC and kernel_sha1() == FERMI_TRAFFIC["kernel_sha1"] and args.precision == FERMI_TRAFFIC["precision"] \
            and args.workload == FERMI_TRAFFIC["workload"] and args.refine_cores == FERMI_TRAFFIC["core_refine"]:
        traffic = FERMI_TRAFFIC["bytes_per_launch"]
    if args.precision == 1 and f16_ms > 0:
        # the dominant kernel: the products in two fp16 planes.  Roofline: its algorithmic bytes
        # (operands once, FP32 addends, output planes and master, over the upper triangles) against
        # the measured HBM copy bandwidth, and its algorithmic flops (n^3 per symmetric product) x 3
        # tensor-core products against the measured bf16 rate; the larger fraction is the bound
        bw = f16_bytes / (f16_ms / 1e3) / 1e9
        tf = f16_flops / (f16_ms / 1e3) / 1e12
        f_bw, f_tf = bw / hbm, tf * split / bf16
        kname = "tc_gemm_persistent<2,F16> (Fermi-recursion products, two-plane fp16 on tcgen05)"
        if f_bw >= f_tf:
            bound, achieved, peak, unit = "hbm", bw, hbm, "GB/s"
        else:
            bound, achieved, peak, unit = "tensor", tf, bf16, "TFLOP/s"
        roof = {"kernel": kname, "bound": bound, "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": traffic,
                "traffic_unit": "bytes per launch (DRAM read + write, ncu)",
                "algorithmic_bytes_per_launch": f16_bytes / f16_launch,
                "hbm": {"achieved_gbs": bw, "peak_gbs": hbm, "frac": f_bw, "peak_note": f"STREAM copy {hbm_src}"},
                "tensor": {"achieved_tflops": tf, "peak_tflops": bf16, "frac": tf / bf16,
                           "frac_with_split_products": f_tf, "split_products": split,
                           "peak_note": f"dense bf16 sustained {peak_src} (fp16 runs at the bf16 rate); the FP32-class "
                                        f"product costs {split} tensor-core products"},
                "launches": f16_launch, "kernel_ms": f16_ms,
                "work_note": "bytes: per launch, over the upper triangle of every subgraph (n (n+1)/2 elements), operands "
                             "read once (4 B an element in two fp16 planes; once when A = B), each FP32 addend (4 B), "
                             "output planes (4 B, 6 B in three bf16 planes), FP32 master (4 B) unless planes-only, second "
                             "output (4 B); flops: n^3 per symmetric product",
                "all_fermi_products": {"launches": k_launch, "kernel_ms": k_ms,
                                       "tflops_algorithmic": (k_flops / (k_ms / 1e3)) / 1e12 if k_ms > 0 else None}}
    else:
        # algorithmic work: a symmetric product of two n x n matrices (upper triangle) = n^3 flops
        achieved = (k_flops / (k_ms / 1e3)) / 1e12 if k_ms > 0 else None
        if args.precision == 0:
            kname, bound, peak = "f64_gemm_kernel (Fermi-recursion products, FP64 CUDA cores)", "alu", 1.25
            peak_note = "nominal FP64 1.25 TF/s (no measured FP64 peak)"
        else:
            kname = "tc_gemm_persistent (Fermi-recursion products, split bf16 on tcgen05)"
            bound, peak = "tensor", bf16
            peak_note = (f"measured sustained dense bf16 {bf16} TF/s {peak_src}; the FP32-class product costs {split} "
                         f"tensor-core products, counted as work of the kernel, not of the method")
        roof = {"kernel": kname, "bound": bound, "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                "traffic_unit": "bytes per launch (DRAM read + write, ncu)",
                "split_products": split,
                "tensor_frac_with_split_products": (achieved * split / peak) if achieved else None,
                "peak_note": peak_note, "launches": k_launch, "kernel_ms": k_ms,
                "work_note": "flops = sum over launches of sum_i n_i^3 (one symmetric product per subgraph, upper "
                             "triangle, n_i the orbital count)"}
    plain = None
    if not args.no_plain and args.precision != 0 and rank == 0:
        q64, t64 = run_plain(args, S, model, s, R0, V0, n0, mu0, gd0, cores0)
        dq_mp = float(np.max(np.abs(q64 - q_start)))
        plain = {"precision": 0, "ms_per_step": 1e3 * t64, "value": N / t64, "unit": UNIT,
                 "mixed_vs_plain_max_dq": dq_mp,
                 "mixed_vs_plain_rms_dq": float(np.sqrt(np.mean((q64 - q_start) ** 2))),
                 "how": "same SCC ground state handed to an FP64 context; charges of its first density against the "
                        "mixed form's; step time from 2 steps with host I/O (FP64 GEMMs on the CUDA cores)",
                 "speedup_mixed_over_plain": (value / world) / (N / t64)}
    drift = float(E[-1, 2] - E[0, 2])
    names = ["graph+halos", "coulomb", "gather", "Z+h~", "fermi(mu solve)", "collect", "forces", "kernel+update"]
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None,
        "dtype": {1: "f32-class (Fermi products: 2-plane fp16 on tcgen05; other products 3-way bf16) / f64 sums",
                  4: "f32 (3-way split bf16 on tcgen05) / f64 sums", 2: "bf16x2 split / f64 sums",
                  3: "bf16 / f64 sums", 0: "f64"}[args.precision],
        "data": "synthetic (seeded water box, synthetic sp SCC-TB model)",
        "config": {"workload": f"{args.workload}: {N} atoms, cores~32, tau 1e-3, r_graph 3 A, XL-BOMD NVE 300 K, "
                               f"Te 300 K, dt {args.dt} fs",
                   "precision": args.precision, "parallelism": f"replicas x{world}",
                   "cores": "recursive bisection" + (", refined for 128-orbital tiles" if args.refine_cores else ""),
                   "l2": "working set (per-subgraph arena, several GB) far exceeds the 129 MB L2; no flush needed",
                   "scc_iters_setup": info["scc_iters"], "scc_resid_setup": info["scc_resid"], "mu": info["mu"],
                   "kernel": "K0 = -0.05 I (paper_2606_03140_gb300.runs.MD_C_K0)"},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 2 * 3 * N * 8,
                "d2h_bytes_per_step": 2 * 3 * N * 8 + 3 * 8 + N * 8},
        "gpu_launches": int(launches),
        "phase_ms_per_step": {k: round(float(v) / args.steps, 3) for k, v in zip(names, phases)},
        "mu_solve": {"fermi_evaluations_per_step": float(np.mean([e[0] for e in evals])) if evals else None,
                     "of_which_stage_shifts": float(np.mean([e[1] for e in evals])) if evals else None},
        "accuracy": acc, "plain_fp64": plain,
        "energy_drift_ha": drift, "energy_fluct_ha": float(E[:, 2].max() - E[:, 2].min()),
        "clocks": clocks, "roofline": roof,
        "rooflines_other": phase_rooflines(ph4, 4, k_ms, bf16, peak_src, args.precision),
    }


def phase_rooflines(ph, steps, fermi_ms, bf16, peak_src, precision):
    """Per-phase times of the kernel-statistics pass, per step (the phases hold several kernels each;
    the Fermi phase minus its product kernels is the mu-solve bookkeeping: counts, core rows)."""
    names = ["graph+halos", "coulomb", "gather", "Z+h~", "fermi", "collect", "forces", "kernel+update"]
    out = {k: {"ms_per_step": round(float(v) / steps, 3)} for k, v in zip(names, ph)}
    out["fermi"]["product_kernels_ms_per_step"] = round(fermi_ms / steps, 3)
    return out


class OracleStep:
    """The FP64 oracle, as it stands, on the host cores, on a bounded sample of the workload.

    A QMD step of the oracle = graph + RCB cores + halos on the full box, the Coulomb potential
    and its gradient on the full box, and the subgraph solve (S^-1/2, eigh, Fermi occupations,
    core rows, charges) of every subgraph.  The Ewald potential is timed once on the full box
    and counted twice (potential + gradient); each step times the graph on the full box and the
    solve of `sample` randomly drawn subgraphs, scaled to all subgraphs.  The oracle's
    subgraph forces are not included (the sample is an underestimate of its step time)."""

    def __init__(self, workload: str, sample: int):
        from oracle import ewald as oew
        from paper_2606_03140_gb300 import inputs as I

        self.s = I.workload(workload)
        self.m = I.default_model()
        self.n = I.random_charges(self.s.n_atoms, 3, 0.05)
        self.sample = sample
        t0 = time.perf_counter()
        self.V = oew.coulomb_potential(self.s.R, self.s.species, self.m.hubbard_u, self.s.box, self.n)
        self.t_ew = time.perf_counter() - t0
        self.rng = np.random.default_rng(5)

    def step(self) -> dict:
        from oracle import density as odn
        from oracle import graph as og

        s = self.s
        t0 = time.perf_counter()
        rp, col = og.build_graph(s.R, s.box, 3.0)
        cores = og.rcb_partition(s.R, s.box, 32)
        hal = og.halos(rp, col, cores)
        t_graph = time.perf_counter() - t0
        pick = self.rng.choice(len(cores), size=min(self.sample, len(cores)), replace=False)
        t0 = time.perf_counter()
        odn.density(s.R, s.species, s.box, self.m, self.n, [cores[i] for i in pick], [hal[i] for i in pick], V=self.V,
                    eig="lapack")
        t_sub = time.perf_counter() - t0
        t_step = t_graph + 2.0 * self.t_ew + t_sub * len(cores) / len(pick)
        return {"t_step": t_step, "t_graph": t_graph, "t_sub": t_sub, "P": len(cores), "picked": len(pick)}


def _threads() -> int:
    try:
        import threadpoolctl
        info = threadpoolctl.threadpool_info()
        return int(max(p["num_threads"] for p in info)) if info else 1
    except Exception:
        return int(os.cpu_count() or 1)


def cpu_baseline(args, sample: int = 8, steps: int = 1):
    ors = OracleStep(args.workload, sample)
    recs = [ors.step() for _ in range(steps)]
    t = float(np.median([r["t_step"] for r in recs]))
    r = recs[0]
    return {"value": ors.s.n_atoms / t, "unit": UNIT, "cores": _threads(), "kind": "oracle",
            "sample": (f"EXTRAPOLATED: full-box graph+RCB+halos ({r['t_graph']:.1f}s), full-box Ewald potential "
                       f"({ors.t_ew:.1f}s, counted x2 for potential+gradient), {r['picked']} of {r['P']} subgraphs "
                       f"solved ({r['t_sub']:.1f}s) and scaled to all; subgraph forces not included (an "
                       f"underestimate of the oracle's step)"),
            "extrapolated": True, "seconds_per_step": t}


def run_reference(args, world, rank):
    if rank != 0:
        return None
    ors = OracleStep(args.workload, 4)
    for _ in range(args.warmup):
        ors.step()
    recs = [ors.step() for _ in range(args.steps)]
    t = float(np.median([r["t_step"] for r in recs]))
    v = ors.s.n_atoms / t
    cb = {"value": v, "unit": UNIT, "cores": _threads(), "kind": "oracle",
          "sample": f"EXTRAPOLATED per step: full-box graph + {recs[0]['picked']} sampled subgraph solves scaled to "
                    f"{recs[0]['P']}, plus 2 x full-box Ewald potential timed once ({ors.t_ew:.1f}s); forces "
                    f"not included", "extrapolated": True}
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "implementation": "FP64 oracle (numpy/scipy, subgraph eigensolves by its LAPACK route) on host cores",
                       "extrapolated": "each step's time is a bounded sample scaled to the full step (see cpu_baseline)"},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def profile_case(args):
    """Small case for kernel captures: 3,000-atom water box (1,000 H2O, 31 A), distance graph,
    RCB cores, one density (mu solved), graph rebuilt from it, a second density (warm-started mu)
    inside NVTX range 'second'."""
    import torch

    from paper_2606_03140_gb300 import inputs as I
    from paper_2606_03140_gb300 import sedacs as S

    s = I.small_water_box(1000, 31.0, seed=33)
    R = np.ascontiguousarray(s.R)
    ctx = S.sedacs_create(s.species, s.box, I.default_model(),
                          S.sedacs_default_params(core_size=32, precision=args.precision))
    S.sedacs_graph_build(ctx, R)
    P = S.sedacs_partition(ctx, R)
    n = np.zeros(s.n_atoms)
    mu, _, _, _ = S.sedacs_subgraph_density(ctx, R, n, n_parts=P)
    S.sedacs_graph_build(ctx, R, use_prev_D=True)
    torch.cuda.nvtx.range_push("second")
    _, q, _, it = S.sedacs_subgraph_density(ctx, R, n, mu=mu, n_parts=P)
    torch.cuda.nvtx.range_pop()
    info = S.sedacs_density_info(ctx)
    S.sedacs_destroy(ctx)
    print(json.dumps({"profile_case": "water3000", "subgraphs": P, "doublings": info["doublings"],
                      "fermi_evaluations": info["passes"]}))


def main():
    args = parse()
    if args.profile_case:
        profile_case(args)
        return
    world, rank, local = dist_init()
    if args.impl == "reference":
        out = run_reference(args, world, rank)
        if out is not None:
            print(json.dumps(out))
        return
    out = run_ours(args, world, rank, local)
    if rank == 0:
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(args)
        print(json.dumps(out))


if __name__ == "__main__":
    main()
