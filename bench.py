"""Benchmark: atoms x QMD-steps/s of graph-partitioned shadow XL-BOMD on one GB300.

Workload: the 9,000-atom water box (3,000 H2O, 44.8 A, seeded synthetic geometry, synthetic
sp SCC-TB model) -- cores of ~32 atoms, halos from the distance + |D| > 1e-3 graph,
Maxwell-Boltzmann velocities at 300 K, dt = 0.25 fs.  A step is one full QMD step: graph
rebuild from the previous density, halos, Coulomb (Ewald), H/S gather, S^-1/2, h~, SP2 Fermi
operator, core rows, charges, energies, forces, kernel K(q - n), charge and Verlet updates.

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
                    help="0 plain FP64; 1 FP32-class (SP2 squares in two fp16 planes, other products "
                         "three-way bf16); 4 FP32-class three-way bf16 throughout; 2, 3 diagnostics")
    ap.add_argument("--workload", default="water9000")
    ap.add_argument("--dt", type=float, default=0.25)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", action="store_true",
                    help="small ncu case: 3,000-atom water box, two densities, the second inside NVTX range 'second'")
    ap.add_argument("--quick-setup", action="store_true",
                    help="start the dynamics from zero charges instead of the SCC ground state "
                         "(same per-step work; used to time the slow plain FP64 form)")
    return ap.parse_args()


METRIC = "atoms*QMD-steps/s at |dq|<=1e-5 e vs FP64 oracle (mixed vs plain, one GB300)"

# DRAM traffic (dram__bytes_read.sum + dram__bytes_write.sum) of the SP2 square kernel, averaged
# over the SP2 launches of 2 timed steps of the 9,000-atom water workload in the mixed form (one
# ncu capture, profiles/tc_gemm_sp2_traffic_water9000.md).  Reported only while the kernel
# source is the one the counters were taken on.
SP2_TRAFFIC = {"bytes_per_launch": 182.9e6, "workload": "water9000", "precision": 1,
               "kernel_sha1": "5b91c84eede22b3ba5e372166adf3648e1512de0"}


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
    """sha1 of the SP2 kernel's source (dense_gemm.cu, dense.cuh, common.cuh), comments stripped."""
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


def setup_system(S, I, workload: str, precision: int, seed_v: int = 20260703, quick: bool = False):
    """SCC ground state and velocities, context ready for XL-BOMD (paper_2606_03140_gb300.runs)."""
    from paper_2606_03140_gb300 import runs

    try:
        return runs.ground_state(workload, precision, seed_v=seed_v, quick=quick)
    except runs.NoGroundState as e:
        # XL-BOMD starts from the SCC ground state; timing dynamics from an unconverged start
        # would time charge oscillations, not the method
        raise SystemExit(f"{e}; it is not an MD benchmark")


def run_ours(args, world, rank, local):
    import torch

    torch.cuda.set_device(local)
    from paper_2606_03140_gb300 import inputs as I
    from paper_2606_03140_gb300 import sedacs as S

    s, model, ctx, R, V, n, info = setup_system(S, I, args.workload, args.precision, quick=args.quick_setup)
    N = s.n_atoms
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
    Rh = Rd.cpu().numpy().copy()
    Vh = Vd.cpu().numpy().copy()
    Eh = np.zeros((1, 3))
    torch.cuda.synchronize()
    barrier(world)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        S.sedacs_xlbomd_step(ctx, Rh, Vh, 1, args.dt, Eh)
    torch.cuda.synchronize()
    t_e2e = allmax(world, time.perf_counter() - t0)
    # roofline of the SP2 square kernel from a separate pass with per-launch CUDA events (kept
    # out of the timed region: the events and the per-density readback of the step counts
    # would slow it down)
    S.sedacs_kernel_stats(ctx, True)
    S.sedacs_xlbomd_step(ctx, Rh, Vh, 4, args.dt)
    k_ms, k_launch, k_pairs = S.sedacs_kernel_stats(ctx, False)
    S.sedacs_destroy(ctx)
    value = world * N * args.steps / (ms / 1e3)
    e2e = world * N * args.steps / t_e2e
    # roofline of the dominant kernel (SP2 squares on tcgen05): algorithmic FLOPs = 2 n^3 per
    # symmetric square (n^3 multiply-add pairs); one FP32-class product = 3 fp16 tensor-core products
    # (two-plane fp16 form 1) or 6 bf16 products (three-plane form 4); fp16 and bf16 run at one rate
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    bf16 = peaks.get("bf16_tflops_sustained", 1700.0)
    nsplit_products = {1: 3, 2: 3, 3: 1, 4: 6}.get(args.precision, 6)
    achieved = (2.0 * k_pairs / max(k_launch, 1)) / (k_ms / max(k_launch, 1) / 1e3) / 1e12 if k_ms > 0 else None
    peak = bf16 / nsplit_products
    kname = ("tc_gemm_persistent (SP2 square, " + ("two-plane fp16" if args.precision == 1 else "split-bf16")
             + " tcgen05)")
    bound = "tensor"
    peak_note = f"measured sustained bf16 {bf16} TF/s (= fp16 rate) / {nsplit_products} split products (of measured)"
    if args.precision == 0:
        # FP64 form: the SIMT FP64 GEMM on the CUDA cores; no measured FP64 peak, the nominal
        # 1.25 TFLOP/s of the part (algorithmic flops count the full square, the kernel computes
        # the upper tiles, so the fraction can exceed 1)
        kname, bound, peak = "f64_gemm_kernel (SP2 square, FP64 CUDA cores)", "alu", 1.25
        peak_note = "nominal FP64 1.25 TF/s (no measured FP64 peak)"
    roof = {"kernel": kname, "bound": bound,
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
            "frac": (achieved / peak) if achieved else None,
            "traffic": (SP2_TRAFFIC["bytes_per_launch"]
                        if (kernel_sha1() == SP2_TRAFFIC["kernel_sha1"] and args.workload == SP2_TRAFFIC["workload"]
                            and args.precision == SP2_TRAFFIC["precision"]) else None),
            "traffic_unit": "bytes per launch (DRAM read + write, ncu, average over the SP2 launches)",
            "peak_note": peak_note,
            "launches": k_launch, "kernel_ms": k_ms}
    drift = float(E[-1, 2] - E[0, 2])
    return {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": {1: "f32-class (SP2: 2-plane fp16 on tcgen05; other products 3-way bf16) / "
                                          "f64 sums",
                                       4: "f32 (3-way split bf16 on tcgen05) / f64 sums", 2: "bf16x2 split / f64 sums",
                                       3: "bf16 / f64 sums", 0: "f64"}[args.precision],
        "data": "synthetic (seeded water box, synthetic sp SCC-TB model)",
        "config": {"workload": f"{args.workload}: {N} atoms, cores~32, tau 1e-3, r_graph 3 A, XL-BOMD NVE 300 K, dt {args.dt} fs",
                   "precision": args.precision, "parallelism": f"replicas x{world}",
                   "l2": "working set (per-subgraph arena, several GB) far exceeds the 129 MB L2; no flush needed",
                   "scc_iters_setup": info["scc_iters"], "scc_resid_setup": info["scc_resid"], "mu": info["mu"],
                   "kernel": "K0 = -0.5 I"},
        "e2e": {"value": e2e, "unit": UNIT, "h2d_bytes_per_step": 2 * 3 * N * 8,
                "d2h_bytes_per_step": 2 * 3 * N * 8 + 3 * 8},
        "gpu_launches": int(launches),
        "phase_ms_per_step": {k: round(float(v) / args.steps, 3) for k, v in zip(
            ["graph+halos", "coulomb", "gather", "Z+h~", "sp2", "collect", "forces", "kernel+update"], phases)},
        "energy_drift_ha": drift, "energy_fluct_ha": float(E[:, 2].max() - E[:, 2].min()),
        "clocks": clocks, "roofline": roof,
    }


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
        odn.density(s.R, s.species, s.box, self.m, self.n, [cores[i] for i in pick], [hal[i] for i in pick], V=self.V)
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
            "sample": (f"full-box graph+RCB+halos ({r['t_graph']:.1f}s), full-box Ewald potential ({ors.t_ew:.1f}s, "
                       f"counted x2 for potential+gradient), {r['picked']} of {r['P']} subgraphs solved "
                       f"({r['t_sub']:.1f}s) and scaled to all; subgraph forces not included"),
            "seconds_per_step": t}


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
          "sample": f"per step: full-box graph + {recs[0]['picked']} sampled subgraph solves scaled to {recs[0]['P']}, "
                    f"plus 2 x full-box Ewald potential timed once ({ors.t_ew:.1f}s)"}
    return {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * t, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": args.workload, "implementation": "FP64 oracle (numpy/scipy) on host cores"},
            "cpu_baseline": cb, "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def profile_case(args):
    """Small case for kernel captures: 3,000-atom water box (1,000 H2O, 31 A), distance graph,
    RCB cores, one density, graph rebuilt from it, a second density inside NVTX range 'second'."""
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
    S.sedacs_subgraph_density(ctx, R, n, mu=-0.13, n_parts=P)
    S.sedacs_graph_build(ctx, R, use_prev_D=True)
    torch.cuda.nvtx.range_push("second")
    _, q, _, it = S.sedacs_subgraph_density(ctx, R, n, mu=-0.13, n_parts=P)
    torch.cuda.nvtx.range_pop()
    S.sedacs_destroy(ctx)
    print(json.dumps({"profile_case": "water3000", "subgraphs": P, "sp2_steps_mean": float(it.mean())}))


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
