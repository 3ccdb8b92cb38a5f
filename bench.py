"""Benchmark: leverage scores of a dense tall-skinny matrix on GB300.

Workload (one "step" = one pass of the whole sketching hot path):
  A: 4,000,000 x 256 float32 (4.1 GB), A_ij = z_ij * 10^u_j, z ~ N(0,1),
     u_j ~ U(-3, 3);  CountSketch r = 65,536;  Gaussian k = 512 (BF16 tensor
     stage, FP32 accumulation; the two stages as separate kernels unless
     --fused-sketch);  FP64 R of the 512 x 256 sketch;  row norms
     ell_i = ||A_i R^-1||^2.
  metric: A-bytes per second through lsk_leverage_scores ("A GB/s sketched
  and scored"); the input (4.1 GB) is larger than L2, so no flush is needed.

Prints ONE JSON line (rank 0).  --impl reference times the FP64 CPU oracle
on a bounded row sample of the same workload instead (no GPU work).
"""
import argparse
import json
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads  # noqa: E402

N_ROWS, D, R_SKETCH, K_GAUSS, SEED, DATA_SEED = 4_000_000, 256, 65_536, 512, 2, 2
METRIC = "A GB/s sketched+scored (leverage scores, dense 4M x 256 FP32)"


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 1900.0, 2070.0, "fallback"


# ------------------------------------------------------------------ clocks --
class ClockSampler:
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self, t0, t1):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                frac = float("0." + parts[0].split(".")[1]) if "." in parts[0] else 0.0
                rows.append((ts + frac, float(parts[2]), float(parts[3]), parts[6:10]))
            except Exception:
                continue
        os.unlink(self.path)
        inside = [r for r in rows if t0 - 0.15 <= r[0] <= t1 + 0.15]
        use = inside if inside else rows[-3:]
        if not use:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in use for i, v in enumerate(r[3]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median([r[1] for r in use])), "sm_max_mhz": max(r[2] for r in use),
                "reasons": reasons, "samples": len(use), "samples_in_timed_region": len(inside)}


# ------------------------------------------------------------------ oracle --
def oracle_sample(n_sample):
    """Time the FP64 oracle's leverage pipeline on the first n_sample rows."""
    from oracle import gaussian as oga
    from oracle import leverage as olev
    A = workloads.dense_colscaled(n=n_sample, d=D, seed=DATA_SEED)
    t = time.perf_counter()
    olev.leverage_scores_dense(A, R_SKETCH, K_GAUSS, SEED, oga.PREC_BF16)
    dt = time.perf_counter() - t
    return A.nbytes, dt


ORACLE_THREADING = ("FP64 numpy oracle: the BLAS products (G S A, the QR, A R^-1) on every host core, "
                    "the CountSketch scatter and the row sums single-threaded")


def cpu_baseline_leg(n2):
    """The oracle on two row samples of the workload (n2 / 4 and n2 rows): the
    rate on the larger one (the same sample the reference arm times), and a
    fit t(n) = fixed + per_row * n -- the fixed part is the Gaussian stage
    (k r d FP64 flops) and the QR, the per-row part the scatter and the row
    norms -- extrapolated to the full workload."""
    n1 = max(1024, n2 // 4)
    b1, t1 = oracle_sample(n1)
    b2, t2 = oracle_sample(n2)
    per_row = max((t2 - t1) / (n2 - n1), 0.0)
    fixed = max(t2 - per_row * n2, 0.0)
    full = fixed + per_row * N_ROWS
    return {"value": b2 / t2 / 1e9, "unit": "GB/s", "cores": cores(), "kind": "oracle",
            "sample": f"first {n2} rows of the workload (r={R_SKETCH}, k={K_GAUSS}), one run, {t2:.1f} s "
                      f"(and {n1} rows, {t1:.1f} s, for the fit); {ORACLE_THREADING}",
            "fit": {"fixed_s": fixed, "per_row_us": per_row * 1e6,
                    "full_workload_s": full, "full_workload_GB/s": N_ROWS * D * 4 / full / 1e9}}


def max_over_ranks(x):
    """The largest x over all ranks (x itself when torch.distributed is not
    initialised): the job takes as long as its slowest rank."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()) or dist.get_world_size() == 1:
        return x
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(bytes_per_rank, world, ms):
    """GB/s of the whole job: every rank processes bytes_per_rank (its block,
    weak scaling), in the time of the slowest rank (ms)."""
    return world * bytes_per_rank / (ms * 1e-3) / 1e9


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_s = args.ref_rows
    for _ in range(args.warmup):
        oracle_sample(n_s)
    times, nbytes = [], 0
    for _ in range(args.steps):
        nbytes, dt = oracle_sample(n_s)
        times.append(dt)
    tot = sum(times)
    value = nbytes * len(times) / tot / 1e9
    sample = (f"first {n_s} rows of the {N_ROWS} x {D} workload per step (r={R_SKETCH}, k={K_GAUSS}); "
              f"{ORACLE_THREADING}")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * tot / len(times),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic", "config": workload_config(args, int(os.environ.get("WORLD_SIZE", "1"))),
        "cpu_baseline": {"value": value, "unit": "GB/s", "cores": cores(), "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "GB/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


def workload_config(args, world=1):
    cfg = {"workload": "dense_colscaled_leverage", "n": N_ROWS, "d": D, "r": R_SKETCH, "k": K_GAUSS,
           "prec": args.prec, "input_bytes": N_ROWS * D * 4, "l2_policy": "input 4.1 GB > L2 (no flush)",
           "parallelism": "single" if world == 1 else f"rows{world}"}
    if world > 1:
        cfg["partition"] = (f"one {world * N_ROWS} x {D} matrix split by rows, {N_ROWS} rows per GPU; one sum "
                            f"all-reduce of the {K_GAUSS} x {D} partial sketches per step (NCCL)")
    return cfg


# ---------------------------------------------------------------- GPU path --
def main():
    global N_ROWS
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="tf32", choices=["fp32", "tf32", "bf16"],
                    help="tf32: BF16 Gaussian stage + TF32 row norms (the workload's own recipe); "
                         "bf16: BF16x3 row norms; fp32: CUDA-core FP32")
    ap.add_argument("--ref-rows", type=int, default=262_144,
                    help="rows of the workload the reference arm's oracle runs per step")
    ap.add_argument("--cpu-rows", type=int, default=262_144,
                    help="rows of the larger oracle sample of the cpu_baseline leg (the smaller is a quarter)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true")
    ap.add_argument("--rows", type=int, default=N_ROWS, help="rows of A (smaller for profiling)")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--batch-problems", type=int, default=512)
    ap.add_argument("--serve-requests", type=int, default=2000)
    ap.add_argument("--no-gram", action="store_true", help="skip the A^T A leg")
    ap.add_argument("--no-jl", action="store_true", help="skip the Alg. 15 right-projection leg")
    ap.add_argument("--no-configs", action="store_true",
                    help="skip the dense 20,000 x 50 and CSR 1M x 200 legs")
    ap.add_argument("--no-next", action="store_true",
                    help="skip the sketch-and-solve (Alg. 11) and csrjlt (Alg. 4) legs")
    ap.add_argument("--jl-m", type=int, default=64, help="columns of the right JL projection Pi")
    ap.add_argument("--fused-sketch", type=int, default=1, choices=[0, 1, 2],
                    help="BF16 sketch: 0 the two stages, 1 the fused kernel (lsk_count_gauss) where the shape "
                         "favours it (default), 2 the fused kernel wherever it applies")
    ap.add_argument("--no-sketch-stage", action="store_true",
                    help="skip the leg that times the fused sketch against the two stages")
    ap.add_argument("--gram-only", action="store_true",
                    help="time only lsk_gram_prec (BF16x3 and FP32) on the workload's A (for profiling)")
    args = ap.parse_args()
    N_ROWS = args.rows
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)

    from paper_2203_02798_gb300 import build as lskbuild
    lskbuild.build()
    import paper_2203_02798_gb300 as lsk

    hbm, bf16_peak, sm_max, peak_kind = peaks()
    # inputs: pinned host copy (for e2e) and the device copy
    # With N > 1 GPUs rank g holds rows [g n, (g + 1) n) of one (N n) x d
    # matrix (its own draws: data seed DATA_SEED + g) and the step is the
    # row-partitioned path: partial sketch, one all-reduce, R, local scores.
    A_host = torch.empty((N_ROWS, D), dtype=torch.float32, pin_memory=True)
    workloads.dense_colscaled(n=N_ROWS, d=D, seed=DATA_SEED + rank, out=A_host.numpy())
    A = A_host.cuda()
    ell = torch.empty(N_ROWS, dtype=torch.float32, device="cuda")
    ctx = lsk.context()
    st = torch.cuda.current_stream()
    lsk.set_fused_sketch(args.fused_sketch)
    from paper_2203_02798_gb300 import sharded

    def step(prec):
        if world == 1:
            lsk.leverage_scores(A, R_SKETCH, K_GAUSS, SEED, prec, out=ell, ctx=ctx)
        else:
            sharded.leverage_scores_sharded(A, rank * N_ROWS, R_SKETCH, K_GAUSS, SEED, prec, out=ell, ctx=ctx)

    def gram_leg(steps):
        """A^T A of the workload's A (csrrk), BF16x3 on tensor cores and FP32 SIMT,
        with the relative Frobenius error of each against an FP64 product."""
        C = torch.empty((D, D), dtype=torch.float32, device="cuda")
        ref = A.double().T @ A.double()
        out = {}
        for prec in ("bf16", "fp32"):
            lsk.gram(A, C=C, prec=prec, ctx=ctx)
            ctx.sync()
            gms, _, _ = timed(lambda: lsk.gram(A, C=C, prec=prec, ctx=ctx), steps)
            gms /= steps
            err = float(torch.linalg.norm(C.double() - ref) / torch.linalg.norm(ref))
            gbs = N_ROWS * D * 4 / (gms * 1e-3) / 1e9
            out[prec] = {"ms": gms, "GB/s": gbs, "rel_fro_err": err,
                         "algorithmic_bytes": N_ROWS * D * 4, "frac_of_measured_hbm": gbs / hbm}
            if prec == "bf16":
                # BF16x3 products of the upper triangle: 3 n d (d + 1) flops
                tf = 3 * N_ROWS * D * (D + 1) / (gms * 1e-3) / 1e12
                out[prec].update({"TFLOP/s": tf, "frac_of_measured_bf16": tf / bf16_peak,
                                  "traffic": measured_traffic("gram_tc", N_ROWS)})
        del ref
        return out

    def jl_leg(steps):
        """Alg. 15 with the d x m right projection Pi on the same workload:
        ||A_i R^-1 Pi||^2, timed like the main step, with the spread of the
        estimates around ||A_i R^-1||^2 (expected sqrt(2/m))."""
        m = args.jl_m
        out_jl = torch.empty_like(ell)
        run = lambda: lsk.leverage_scores_jl(A, R_SKETCH, K_GAUSS, m, SEED, args.prec, out=out_jl, ctx=ctx)
        for _ in range(2):
            run()
        ctx.sync()
        jms, _, _ = timed(run, steps)
        jms /= steps
        step(args.prec)
        ctx.sync()
        ratio = (out_jl.double() / ell.double().clamp_min(1e-30))
        return {"m": m, "ms": jms, "GB/s": whole_job_rate(N_ROWS * D * 4, world, jms),
                "ratio_mean": float(ratio.mean()), "ratio_std": float(ratio.std()),
                "expected_std": (2.0 / m) ** 0.5}

    def sketch_stage_leg(steps):
        """G (S A) of the workload (r = 65,536, k = 512, BF16 mode): the fused
        kernel (S A kept on chip, Alg. 3's blocking) against lsk_cs_sketch +
        lsk_gauss_sketch, ms per call, and their relative difference."""
        GSA = torch.empty((K_GAUSS, D), dtype=torch.float32, device="cuda")
        GSA2 = torch.empty_like(GSA)
        SA = torch.empty((R_SKETCH, D), dtype=torch.float32, device="cuda")
        runs = {"fused": lambda: lsk.count_gauss(A, R_SKETCH, K_GAUSS, SEED, out=GSA, ctx=ctx),
                "two_stage": lambda: lsk.gauss_sketch(lsk.cs_sketch(A, R_SKETCH, SEED, out=SA, ctx=ctx),
                                                      K_GAUSS, SEED, "bf16", out=GSA2, ctx=ctx)}
        out = {}
        for name, fn in runs.items():
            fn()
            ctx.sync()
            sms, _, _ = timed(fn, steps)
            sms /= steps
            out[name] = {"ms": sms, "GB/s": whole_job_rate(N_ROWS * D * 4, world, sms)}
        out["rel_diff"] = float(torch.linalg.norm((GSA - GSA2).double()) / torch.linalg.norm(GSA2.double()))
        out["workload"] = "dense 4M x 256, r = 65,536, k = 512"
        del SA
        return out

    def next_legs(steps):
        """Sketch-and-solve (Alg. 11) on the workload's A with a synthetic b, and
        the Gaussian CSR sketch (Alg. 4) of the 1,000,000 x 200 CSR workload
        (p = 0.01, m = 2 d = 400): ms per call and the rate of the main input."""
        out = {}
        g = torch.Generator(device="cuda").manual_seed(DATA_SEED)
        b = torch.randn(N_ROWS, dtype=torch.float64, device="cuda", generator=g)
        x = torch.empty(D, dtype=torch.float64, device="cuda")
        run = lambda: lsk.sketch_solve(A, b, R_SKETCH, K_GAUSS, SEED, args.prec, out=x, ctx=ctx)
        run()
        ctx.sync()
        ms, _, _ = timed(run, steps)
        ms /= steps
        out["sketch_solve"] = {"ms": ms, "GB/s": whole_job_rate(N_ROWS * D * 4 + N_ROWS * 8, world, ms),
                               "workload": "dense 4M x 256 + b, r = 65,536, k = 512"}
        V, J, I = workloads.csr_bernoulli(1_000_000, 200, 0.01, seed=1)
        Acsr = lsk.csr_from_numpy(V, J, I, 200)
        C = torch.empty((400, 200), dtype=torch.float32, device="cuda")
        runj = lambda: lsk.csrjlt(Acsr, 400, SEED, "fp32", out=C, ctx=ctx)
        runj()
        ctx.sync()
        jms, _, _ = timed(runj, steps)
        jms /= steps
        out["csrjlt"] = {"ms": jms, "gaussians_per_s": 400 * 1_000_000 / (jms * 1e-3),
                         "nnz": int(len(V)), "workload": "CSR 1M x 200, p = 0.01, m = 400"}
        del Acsr, V, J, I
        # column subset selection (Alg. 9) of 64 columns and the scores on them
        # (Alg. 16 sketched, Alg. 14 exact) on the workload's A
        c = 64
        runs = {"column_select": lambda: lsk.column_select(A, R_SKETCH, K_GAUSS, SEED, c, args.prec, ctx=ctx),
                "hrn_approx": lambda: lsk.leverage_scores_hrn(A, R_SKETCH, K_GAUSS, SEED, c, exact=False,
                                                              prec=args.prec, out=ell, ctx=ctx),
                "hrn_exact": lambda: lsk.leverage_scores_hrn(A, R_SKETCH, K_GAUSS, SEED, c, exact=True,
                                                             prec=args.prec, out=ell, ctx=ctx),
                "leverage_exact": lambda: lsk.leverage_scores_exact(A, args.prec, out=ell, ctx=ctx),
                "lsq_gram": lambda: lsk.least_squares_gram(A, bvec, refine=2, out=x, ctx=ctx)}
        bvec = torch.randn(N_ROWS, dtype=torch.float64, device="cuda", generator=g)
        for name, fn in runs.items():
            fn()
            ctx.sync()
            cms, _, _ = timed(fn, steps)
            cms /= steps
            out[name] = {"ms": cms, "GB/s": whole_job_rate(N_ROWS * D * 4, world, cms),
                         "workload": "dense 4M x 256" + (f", r = 65,536, k = 512, c = {c}"
                                                         if name in ("column_select", "hrn_approx", "hrn_exact")
                                                         else "")}
        del b, bvec
        return out

    def configs_leg(steps):
        """The two smaller workloads the path is specified on, each one step =
        the whole leverage-score path, with the A^T A of the same A, per-kernel
        CUDA-event times and each kernel's fraction of the measured HBM
        bandwidth on its algorithmic bytes (the CountSketch pass: A once + the
        S A write; the row norms: A once + the scores; the Gram: A once):
          dense 20,000 x 50 (FP64 input cast to FP32 once; rows 0-4 x 100),
              r = 2,500, k = 100, FP32 and BF16 stages;
          CSR 1,000,000 x 200, each entry kept with p = 0.01 (~2M nnz), r = 40,000,
              k = 400, FP32 throughout."""
        out = {}

        def run_case(name, Ac, r, k, prec, a_bytes, kernel_bytes):
            ellc = torch.empty(Ac.n if isinstance(Ac, lsk.CSR) else Ac.shape[0], dtype=torch.float32, device="cuda")
            fn = lambda: lsk.leverage_scores(Ac, r, k, SEED, prec, out=ellc, ctx=ctx)
            for _ in range(3):
                fn()
            ctx.sync()
            gfn = lambda: lsk.gram(Ac, prec="fp32", ctx=ctx)
            ms, _, _ = timed(fn, steps)
            gms, _, _ = timed(gfn, steps)
            # the per-kernel record: the same calls again with CUDA events
            # around every launch (the Gram's kernels join it)
            ctx.profile(True)
            ctx.profile_reset()
            timed(fn, steps)
            timed(gfn, steps)
            ctx.profile(False)
            ctx.sync()
            ms /= steps
            gms /= steps
            kern = {}
            for kn, (launches, tot) in ctx.profile_totals().items():
                per = tot / max(launches, 1)
                e = {"launches_per_step": launches / steps, "ms_per_launch": per}
                if kn in kernel_bytes:
                    e["algorithmic_bytes"] = kernel_bytes[kn]
                    e["GB/s"] = kernel_bytes[kn] / (per * 1e-3) / 1e9
                    e["frac_of_measured_hbm"] = e["GB/s"] / hbm
                kern[kn] = e
            out[name] = {"ms_per_step": ms, "value": a_bytes / (ms * 1e-3) / 1e9, "unit": "GB/s of A",
                         "prec": prec, "kernels": kern,
                         "gram_fp32": {"ms": gms, "GB/s": a_bytes / (gms * 1e-3) / 1e9}}

        A1 = torch.from_numpy(workloads.dense_outliers().astype(np.float32)).cuda()
        n1, d1 = A1.shape
        b1 = n1 * d1 * 4
        for prec in ("fp32", "bf16"):
            run_case(f"dense_outliers_20000x50_{prec}", A1, 2500, 100, prec, b1,
                     {"cs_dense_gather": b1 + 4 * 2500 * d1, "rownorm_dense_simt": b1 + 4 * n1,
                      "rownorm_dense_tc": b1 + 4 * n1})
        V, J, I = workloads.csr_bernoulli(1_000_000, 200, 0.01, seed=1)
        A2 = lsk.csr_from_numpy(V, J, I, 200)
        nnz, n2 = int(len(V)), 1_000_000
        b2 = 8 * nnz + 8 * (n2 + 1)
        run_case("csr_1Mx200_p0.01_fp32", A2, 40_000, 400, "fp32", b2,
                 {"cs_csr_gather": b2 + 4 * 40_000 * 200, "rownorm_csr": b2 + 4 * n2, "gram_csr": b2})
        out["csr_1Mx200_p0.01_fp32"]["nnz"] = nnz
        del A1, A2, V, J, I
        return out

    def barrier():
        if world > 1:
            dist.barrier()

    def timed(fn, steps):
        barrier()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        t0 = time.time()
        e0.record(st)
        for _ in range(steps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        t1 = time.time()
        barrier()
        ms = max_over_ranks(e0.elapsed_time(e1))
        return ms, t0, t1

    if args.gram_only:
        g = gram_leg(args.steps)
        if rank == 0:
            print(json.dumps({"gram": g, "config": workload_config(args, world)}))
        return

    for _ in range(max(3, args.warmup)):
        step(args.prec)
    ctx.sync()

    # main timed region (clocks sampled; no per-kernel events, which would add
    # an event record around every launch)
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(0.3)
    ms, t0, t1 = timed(lambda: step(args.prec), args.steps)
    clk = clocks.stop(t0, t1)
    ctx.sync()
    # the per-kernel record: the same steps again with CUDA events around
    # every launch, on the launching stream
    ctx.profile(True)
    ctx.profile_reset()
    timed(lambda: step(args.prec), args.steps)
    ctx.profile(False)
    ctx.sync()
    kern = ctx.profile_totals()
    ms_step = ms / args.steps
    a_bytes = N_ROWS * D * 4
    value = whole_job_rate(a_bytes, world, ms_step)

    # roofline of the dominant kernel
    top = max(kern.items(), key=lambda kv: kv[1][1]) if kern else ("none", (1, 0.0))
    name, (launches, tot_ms) = top
    per_launch_ms = tot_ms / max(launches, 1)
    algo = algorithmic_work(name)
    if algo["bound"] == "hbm":
        achieved = algo["bytes"] / (per_launch_ms * 1e-3) / 1e9
        peak, unit = hbm, "GB/s"
    elif algo["bound"] == "tensor":
        achieved = algo["flops"] / (per_launch_ms * 1e-3) / 1e12
        peak, unit = bf16_peak, "TFLOP/s"
    else:
        achieved = algo["flops"] / (per_launch_ms * 1e-3) / 1e12
        peak, unit = 152 * 128 * 2 * sm_max * 1e6 / 1e12, "TFLOP/s"
    roofline = {"kernel": name, "bound": algo["bound"], "achieved": achieved, "peak": peak, "unit": unit,
                "frac": achieved / peak, "traffic": measured_traffic(name, N_ROWS), "peak_source": peak_kind if algo["bound"] != "alu"
                else "152 SMs x 128 FP32 lanes x 2 x max SM clock", "per_launch_ms": per_launch_ms,
                "algorithmic": algo["bytes"] if algo["bound"] == "hbm" else algo["flops"]}
    kernels = {k: {"launches_per_step": v[0] / args.steps, "ms_per_step": v[1] / args.steps,
                   "share": v[1] / max(sum(x[1] for x in kern.values()), 1e-9)} for k, v in kern.items()}
    gpu_launches = int(sum(v[0] for v in kern.values()))

    # end to end through the public API with host buffers
    ell_host = torch.empty(N_ROWS, dtype=torch.float32, pin_memory=True)

    # N = 1: lsk.leverage_scores_host (the copy of row block c + 1 overlaps the
    # CountSketch of block c); N > 1: the copy, then the row-partitioned step
    def e2e_step():
        if world == 1:
            lsk.leverage_scores_host(A_host, R_SKETCH, K_GAUSS, SEED, args.prec, out_host=ell_host, A_dev=A,
                                     ctx=ctx)
        else:
            A.copy_(A_host, non_blocking=True)
            step(args.prec)
            ell_host.copy_(ell, non_blocking=True)

    e2e_steps = max(3, min(args.steps, 20))
    e2e_step()
    ems, _, _ = timed(e2e_step, e2e_steps)
    ems /= e2e_steps
    # the copy alone (the floor of any end-to-end step on this host link)
    cms, _, _ = timed(lambda: A.copy_(A_host, non_blocking=True), e2e_steps)
    cms /= e2e_steps
    e2e = {"value": whole_job_rate(a_bytes, world, ems), "unit": "GB/s", "ms_per_step": ems,
           "h2d_bytes_per_step": a_bytes, "d2h_bytes_per_step": N_ROWS * 4,
           "copy_only_ms": cms, "copy_only_GB/s": a_bytes / (cms * 1e-3) / 1e9,
           "overlapped": world == 1}

    # the same step with the other tensor-core row-norm arithmetic (BF16x3
    # against TF32), for comparison
    other = None
    if args.prec in ("tf32", "bf16") and world == 1:
        op = "bf16" if args.prec == "tf32" else "tf32"
        for _ in range(2):
            step(op)
        oms, _, _ = timed(lambda: step(op), max(3, args.steps // 5))
        oms /= max(3, args.steps // 5)
        other = {"prec": op, "value": whole_job_rate(a_bytes, world, oms), "unit": "GB/s", "ms_per_step": oms}

    # the plain FP32 single-problem path on the same GPU
    plain = None
    if not args.no_plain and args.prec != "fp32" and world == 1:
        for _ in range(2):
            step("fp32")
        pms, _, _ = timed(lambda: step("fp32"), max(3, args.steps // 5))
        pms /= max(3, args.steps // 5)
        plain = {"value": whole_job_rate(a_bytes, world, pms), "unit": "GB/s", "ms_per_step": pms}

    # the other legs time single-GPU calls: rank 0's GPU alone, and only at N = 1
    solo = world == 1
    gram = None if args.no_gram or not solo else gram_leg(max(3, args.steps // 5))
    jl = None if args.no_jl or not solo else jl_leg(max(3, args.steps // 5))
    sstage = None if args.no_sketch_stage or not solo else sketch_stage_leg(max(3, args.steps // 5))
    nxt = None if args.no_next or not solo else next_legs(max(3, args.steps // 5))
    small = None if args.no_configs or not solo else configs_leg(max(5, args.steps // 2))
    batched = None if args.no_batch or not solo else run_batched(args, lsk, torch, ctx, plain)
    served = None if args.no_serve or not solo else run_served(args, lsk, torch)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline_leg(args.cpu_rows)

    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "GB/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": {"tf32": "bf16+tf32+fp32+f64", "bf16": "bf16+fp32+f64"}.get(args.prec, "f32+f64"),
            "data": "synthetic", "config": workload_config(args, world),
            "hbm_frac_of_step": (a_bytes * 2 + 4 * N_ROWS) / (ms_step * 1e-3) / 1e9 / hbm,
            "roofline": roofline, "kernels": kernels, "gpu_launches": gpu_launches,
            "other_prec": other, "plain_fp32": plain, "gram": gram, "jl": jl, "sketch_stage": sstage, "next": nxt, "configs": small,
            "batched": batched, "served": served, "e2e": e2e, "clocks": clk,
            "cpu_baseline": cpu,
        }))
    if world > 1:
        dist.destroy_process_group()


def run_batched(args, lsk, torch, ctx, plain):
    """512 independent problems (n log-uniform 1e4..1e6, d in {32..256}, half
    CSR), r = d^2, k = 2d, BF16 stages, one batch call (CUDA graph)."""
    specs = workloads.batch_specs(args.batch_problems, seed=3)
    probs, a_bytes = [], 0
    for sp in specs:
        if sp["kind"] == "dense":
            A = workloads.batch_problem_torch(sp)
            a_bytes += A.numel() * 4
        else:
            V, J, I = workloads.batch_problem_torch(sp)
            A = lsk.CSR(V, J, I, sp["n"], sp["d"])
            a_bytes += V.numel() * 8 + I.numel() * 8
        probs.append((A, sp["r"], sp["k"], sp["sketch_seed"]))
    outs = lsk.batch_leverage_scores(probs, prec="bf16", autotune=True, ctx=ctx)
    ctx.sync()
    streams = lsk.batch_streams(probs, prec="bf16", ctx=ctx)
    _, schedule = lsk.batch_schedule(probs, prec="bf16", ctx=ctx)
    lsk.batch_leverage_scores(probs, prec="bf16", graph=True, outs=outs, ctx=ctx)   # capture
    ctx.sync()
    reps = 3
    st = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        lsk.batch_leverage_scores(probs, prec="bf16", graph=True, outs=outs, ctx=ctx)
    e1.record(st)
    torch.cuda.synchronize()
    ctx.sync()
    ms = e0.elapsed_time(e1) / reps
    value = a_bytes / (ms * 1e-3) / 1e9
    out = {"workload": "batch_512_leverage", "problems": len(probs), "input_bytes": a_bytes,
           "ms_per_batch": ms, "value": value, "unit": "GB/s", "streams": streams, "schedule": schedule,
           "graph": True,
           "vs_plain_fp32_single": (value / plain["value"]) if plain else None}
    del probs, outs
    torch.cuda.empty_cache()
    return out


def run_served(args, lsk, torch):
    """Poisson arrivals (200 req/s) of sketch-and-precondition least-squares
    requests drawn from the batch size distribution; continuous batching."""
    from paper_2203_02798_gb300.serve import Request, Server, latency_summary
    specs = workloads.batch_specs(512, seed=3)
    pool_specs = specs[:24] + specs[256:280]
    pool = []
    for sp in pool_specs:
        if sp["kind"] == "dense":
            A = workloads.batch_problem_torch(sp)
            mv = (lambda x, A=A: (A @ x.float()).double())
        else:
            V, J, I = workloads.batch_problem_torch(sp)
            A = lsk.CSR(V, J, I, sp["n"], sp["d"])
            rows = torch.repeat_interleave(torch.arange(sp["n"], device="cuda"), I[1:] - I[:-1])
            mv = (lambda x, V=V, J=J, rows=rows, n=sp["n"]: torch.zeros(n, dtype=torch.float64, device="cuda")
                  .index_add_(0, rows, V.double() * x[J.long()]))
        pool.append((sp, A, mv))
    arrivals = workloads.poisson_arrivals(200.0, args.serve_requests, seed=4)
    rng = np.random.default_rng(4)
    server = Server(slots=8)
    reqs = []
    for i, t in enumerate(arrivals):
        sp, A, mv = pool[int(rng.integers(len(pool)))]
        _, b = workloads.lsq_rhs_torch(mv, sp["n"], sp["d"], seed=10_000 + i)
        reqs.append(Request(i, float(t), Server.footprint(sp["n"], sp["d"], r=sp["r"], k=sp["k"]),
                            {"A": A, "b": b, "opts": {"r": sp["r"], "k": sp["k"], "seed": sp["sketch_seed"]}}))
    torch.cuda.synchronize()
    # warm-up: one request per slot outside the trace
    for s in range(server.slots):
        p = reqs[s].payload
        server.solve(s, p["A"], p["b"], **p["opts"])
    done, rejected = server.run(reqs, hbm_budget=150 * 10**9)
    summ = latency_summary(done, slots=server.slots)
    etas = [c.result[1]["eta"] for c in done if c.error is None]
    errors = sorted({c.error for c in done if c.error is not None})
    summ.update({"workload": "served_lsq_poisson200", "requests": len(reqs), "rejected": len(rejected),
                 "slots": server.slots, "pool_problems": len(pool),
                 "converged": int(sum(e <= 1e-10 for e in etas)), "max_eta": float(max(etas)) if etas else None,
                 "error_samples": errors[:3]})
    server.close()
    del pool, reqs
    torch.cuda.empty_cache()
    return summ


# DRAM traffic of one launch, from an ncu capture of a smaller case of the same
# kernel (profiles/dram_traffic_<kernel>.txt: the capture's rows and
# dram__bytes_read.sum + dram__bytes_write.sum, and a digest of the sources the
# kernel is built from).  Scaled to the bench's rows (traffic grows with rows:
# A is streamed once); reported as null once the sources differ from the
# captured ones.
def source_digest(paths):
    import hashlib
    h = hashlib.sha256()
    for rel in paths:
        with open(os.path.join(ROOT, rel), "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def measured_traffic(kernel, rows):
    path = os.path.join(ROOT, "profiles", f"dram_traffic_{kernel}.txt")
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                line = line.strip()
                if line and not line.startswith("#"):
                    key, _, val = line.partition(" ")
                    kv[key] = val.strip()
        if source_digest(kv["sources"].split()) != kv["sha256"]:
            return None
        return float(kv["dram_bytes"]) * rows / float(kv["rows"])
    except (OSError, KeyError, ValueError):
        return None


def algorithmic_work(kernel):
    """Algorithmic bytes / flops of one launch of `kernel` on this workload."""
    n, d, r, k = N_ROWS, D, R_SKETCH, K_GAUSS
    a_bytes = n * d * 4
    table = {
        "cs_dense_gather": {"bound": "hbm", "bytes": a_bytes + 4 * r * d},
        "rownorm_dense_simt": {"bound": "alu", "flops": n * d * (d + 1)},
        "rownorm_dense_tf32": {"bound": "hbm", "bytes": a_bytes + 4 * n, "flops": n * d * (d + 1)},
        "rownorm_dense_tc": {"bound": "hbm", "bytes": a_bytes + 4 * n,
                             "flops": 3 * n * d * (d + 1)},
        "gauss_simt": {"bound": "alu", "flops": 2 * k * r * d},
        "gauss_tc": {"bound": "tensor", "flops": 2 * 2 * k * r * d},
        "count_gauss": {"bound": "hbm", "bytes": a_bytes + 4 * n},
    }
    return table.get(kernel, {"bound": "hbm", "bytes": a_bytes})


if __name__ == "__main__":
    main()
