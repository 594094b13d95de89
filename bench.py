"""Benchmark: N=25600 complex R-matrix solve, FP32+IR vs FP64, on GB300.

One step = the whole hot path on one coupled-channel system already resident
in HBM: assemble C and Phi (G1), blocked LU (G2-G4), triangular solves with
FP64 structured-residual refinement until the residual stagnates (G6-G8), then
R and U (G9-G10).  Default workload: nch=256 x nlag=100 (N=25600), 256
right-hand sides, E=10 MeV, seed 11592 (the FP32+IR configuration); the
complex128 path on the same system is timed once beside it and the two U's
compared.  The matrix (5.2 GB complex64 / 10.5 GB complex128) is far larger
than L2, so no flush is needed between steps.

  value     algorithmic TFLOP/s of the FP32+IR step: (8/3 N^3 + 8 N^2 nrhs) / t
  e2e       same, through the C ABI from pinned host buffers: V host->device,
            full step, R and U device->host, all inside the timed region
  roofline  the trailing-update kernel: algorithmic flops of its launches over
            their CUDA-event time, against the tensor peak it runs on
  cpu_baseline  the CPU oracle on a bounded sample (N=1600 of the same family)

--impl reference times the CPU oracle (the reference arm of this build).
Multi-GPU (torchrun): every rank solves its own system (replicas, weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED = os.path.join(ROOT, "MEASURED_PEAKS.json")
FALLBACK_PEAKS = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}
TF32_PER_BF16 = 0.5          # nominal dense tf32 : bf16 tensor rate on GB300 (1.1 : 2.25 PF)
DTYPES = {1: "c64 factor with 3xTF32 tensor updates / f64 refinement",
          4: "c64 factor with 1xFP16 (scaled) tensor updates / f64 GMRES-IR",
          2: "c64 factor with FP32 CUDA-core updates / f64 refinement",
          3: "c64 factor with 3xFP16 (scaled split) tensor updates / f64 refinement",
          0: "c128 throughout (FP64 tensor-instruction GEMMs, FP64 refinement)"}


def peaks():
    try:
        with open(MEASURED) as f:
            return json.load(f), "measured"
    except Exception:
        return dict(FALLBACK_PEAKS), "fallback"


def max_over_ranks(ms, dist, device):
    """The job's time: the slowest rank's (all-reduce MAX; identity on one rank)."""
    if dist is None:
        return ms
    import torch
    t = torch.tensor([float(ms)], device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world, flops_per_step, ms):
    """Whole-job TFLOP/s of `world` replicas, each doing flops_per_step per step."""
    return world * flops_per_step / (ms * 1e-3) / 1e12


def paired_update_bytes(N, nb, plane_bytes):
    """Algorithmic bytes of each tensor-core factor update launch with paired panels:
    C read + write (16 B per complex64 element) plus the operand planes (4 per
    operand, plane_bytes per element in total)."""
    out, k0 = [], 0
    while k0 < N:
        ja = min(nb, N - k0)
        ra = N - k0 - ja
        if ra <= 0:
            break
        if ra <= nb:
            out.append(16.0 * ra * ra + plane_bytes * ja * 2 * ra)
            k0 += ja
            continue
        jb, far = nb, N - k0 - ja - nb
        out.append(16.0 * ra * jb + plane_bytes * ja * (ra + jb))     # columns of b
        out.append(16.0 * jb * far + plane_bytes * ja * (jb + far))   # rows of b
        out.append(16.0 * far * far + plane_bytes * (ja + jb) * 2 * far)
        k0 += ja + jb
    return out


def lu_flops(N, nrhs):
    return 8.0 / 3.0 * N ** 3 + 8.0 * N ** 2 * nrhs


FP64_NOMINAL_TFLOPS = 1.25   # GB300 FP64 (no measured FP64 peak in MEASURED_PEAKS.json)


def profile_ratio(name):
    """DRAM bytes per algorithmic byte of one captured launch, from the summary's
    `dram_per_algorithmic_byte:` line under profiles/ (None if absent)."""
    try:
        with open(os.path.join(ROOT, "profiles", name)) as f:
            for line in f:
                if line.startswith("dram_per_algorithmic_byte:"):
                    return float(line.split(":")[1].split()[0])
    except OSError:
        pass
    return None


def truth_errors(W, results):
    """max|delta|/max|truth| of X, R, U over the stored samples of the oracle's
    N = 25600 truth (tests/golden/truth_config3_W*_n25600.txt)."""
    sys.path.insert(0, os.path.join(ROOT, "tests", "golden"))
    try:
        from make_truth_n25600 import load_truth, sampled_relerr, truth_file
        if not os.path.exists(truth_file(W)):
            return None
        t = load_truth(W)
    except Exception as e:  # the stored samples are optional context
        return {"unavailable": str(e)}
    out = {"source": os.path.relpath(truth_file(W), ROOT)}
    for key, (X, R, U) in results.items():
        if X is None:
            continue
        out[key] = {"X": sampled_relerr(X, t, "X"), "R": sampled_relerr(R, t, "R"),
                    "U": sampled_relerr(U, t, "U")}
    return out


def stage_rooflines(stats, N, nch, nb, iters, pk, src):
    """Where the rest of the step goes: per-class algorithmic work over CUDA-event time."""
    out = {}
    ms, n = stats.get("panel_ms"), stats.get("panel_launches")
    if ms and ms > 0:
        out["panel"] = {"bound": "latency", "ms": ms, "launches": n,
                        "us_per_column": ms * 1e3 / N,
                        "hbm_gbs": 16.0 * N * N / 2 / (ms * 1e-3) / 1e9,
                        "note": "one grid-wide pivot search per column; bytes = each panel read "
                                "and written once (8 N^2 in total), far below the HBM roof; with "
                                "the factorisation's look-ahead part of this time runs beside the "
                                "far updates (32-column sub-panels, counted as launches here)"}
    solves = 1 + int(iters)
    ms = stats.get("solve_tc_ms")
    if ms and ms > 0:
        fl = solves * 8.0 * nch * N * (N - nb)
        peak = pk["bf16_tflops_sustained"] / 3.0
        out["solve_tc"] = {"bound": "tensor", "ms": ms, "launches": stats.get("solve_tc_launches"),
                           "achieved_tflops": fl / (ms * 1e-3) / 1e12, "peak": peak,
                           "frac": fl / (ms * 1e-3) / 1e12 / peak,
                           "flops": "%d solves x 8 nrhs N (N - nb) (off-diagonal block updates)" % solves}
    ms = stats.get("apply_inv_ms")
    if ms and ms > 0:
        out["apply_inv"] = {"bound": "latency", "ms": ms, "launches": stats.get("apply_inv_launches"),
                            "us_per_launch": ms * 1e3 / max(1.0, stats.get("apply_inv_launches") or 1),
                            "note": "one diagonal block x nrhs per launch (solves and the factor's U12)"}
    ms, n = stats.get("resid_ms"), stats.get("resid_launches")
    if ms and ms > 0 and n:
        nlag = N // nch
        fl = n * (4.0 * nlag * nlag * nch * nch + 8.0 * nch * nch * nlag * nch)
        out["fp64_residual"] = {"bound": "fp64", "ms": ms, "evaluations": n,
                                "achieved_tflops": fl / (ms * 1e-3) / 1e12,
                                "peak": FP64_NOMINAL_TFLOPS,
                                "frac": fl / (ms * 1e-3) / 1e12 / FP64_NOMINAL_TFLOPS,
                                "peak_source": "nominal GB300 FP64 (no measured FP64 peak)",
                                "note": "FP64-accurate products; from nch >= 32 they run as "
                                        "exact integer-digit products on the FP16 tensor cores "
                                        "(a frac above 1 is that arithmetic, not FP64 units)"}
    return out


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms during the timed region."""

    def __init__(self, index):
        self.index, self.samples, self.proc = index, [], None

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 7:
                self.samples.append(parts)

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.samples:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(s[0]) for s in self.samples if s[0].replace(".", "").isdigit()]
        mx = [float(s[1]) for s in self.samples if s[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for s in self.samples for k in range(4) if s[3 + k].strip() == "Active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.samples)}


# ---------------------------------------------------------------------------
def workload(args):
    import cc_problems as cp
    if args.small:
        return cp.config3(16), "config3 nch=16 nlag=100 N=1600 E=10 MeV seed 11592"
    return cp.config3(256), "config3 nch=256 nlag=100 N=25600 E=10 MeV seed 11592"


class Runner:
    """One system on one GPU through the C ABI (device-resident buffers)."""

    def __init__(self, p, precision, device, method=0, lookahead=1, residual=0, solve_block=0,
                 factor=0, factor_lookahead=1, la_panel_ctas=0, la_min_rows=0, solve_groups=0,
                 la_both_rows=0, tc_bn=0):
        import torch

        import cc_problems as cp
        import paper_2512_11590_gb300 as g
        self.g, self.p, self.torch = g, p, torch
        self.stream = torch.cuda.current_stream()
        self.ctx = g.rmat_create(device, self.stream.cuda_stream)
        g.rmat_set_param(self.ctx, g.RMAT_PARAM_METHOD, method)
        g.rmat_set_param(self.ctx, g.RMAT_PARAM_SOLVE_LOOKAHEAD, lookahead)
        g.rmat_set_param(self.ctx, g.RMAT_PARAM_RESIDUAL, residual)
        g.rmat_set_param(self.ctx, g.RMAT_PARAM_SOLVE_BLOCK, solve_block)
        g.rmat_set_param(self.ctx, g.RMAT_PARAM_FACTOR, factor)
        g.rmat_set_param(self.ctx, g.RMAT_PARAM_FACTOR_LOOKAHEAD, factor_lookahead)
        g.rmat_set_param(self.ctx, g.RMAT_PARAM_LA_PANEL_CTAS, la_panel_ctas)
        g.rmat_set_param(self.ctx, g.RMAT_PARAM_LA_MIN_ROWS, la_min_rows)
        g.rmat_set_param(self.ctx, g.RMAT_PARAM_SOLVE_GROUPS, solve_groups)
        g.rmat_set_param(self.ctx, g.RMAT_PARAM_LA_BOTH_ROWS, la_both_rows)
        g.rmat_set_param(self.ctx, g.RMAT_PARAM_TC_BN, tc_bn)
        m = g.rmat_mesh(p.nlag, p.a)
        self.V_host = cp.potential_at(p, m["r"]).ravel()
        self.Vd = torch.from_numpy(self.V_host).cuda()
        self.prob, self._keep = g.make_problem_struct(p.nch, p.nlag, p.a, p.hm, p.l, p.thresh,
                                                      precision, zz=p.zz)
        self.precision = precision
        self.nopen = int(np.sum(p.E - p.thresh > 0))
        self.X = torch.zeros((p.nch, p.N), dtype=torch.complex128, device="cuda")
        self.R = torch.zeros(p.nch * p.nch, dtype=torch.complex128, device="cuda")
        self.U = torch.zeros(max(1, self.nopen) ** 2, dtype=torch.complex128, device="cuda")
        self.last = None

    def step(self, Vptr=None):
        g, p = self.g, self.p
        g.rmat_assemble(self.ctx, self.prob, p.E, Vptr or self.Vd.data_ptr())
        g.rmat_factor(self.ctx, want_info=False)
        st, it, rel = g.rmat_solve(self.ctx, self.X.data_ptr(), p.N, max_refine=30, tol=1e-13)
        g.rmat_collision(self.ctx, self.R.data_ptr(), self.U.data_ptr())
        self.last = {"status": st, "iters": it, "rel_resid": rel,
                     "history": [float("%.3g" % h) for h in g.rmat_refine_history(self.ctx)]}

    def XR_host(self):
        """X (N x nrhs) and R (nch x nch) of the last step, host complex128."""
        self.torch.cuda.synchronize()
        return self.X.cpu().numpy().T, self.R.cpu().numpy().reshape(self.p.nch, self.p.nch).T

    def U_host(self):
        n = self.nopen
        return self.U.cpu().numpy()[:n * n].reshape(n, n).T

    def close(self):
        self.g.rmat_destroy(self.ctx)


def time_steps(runner, K, W, sync_all):
    torch = runner.torch
    g = runner.g
    for _ in range(W):
        runner.step()
    g.rmat_set_param(runner.ctx, g.RMAT_PARAM_TIMING, 1)
    runner.step()                               # one timed-instrumented step for the roofline
    torch.cuda.synchronize()
    g.rmat_reset_counters(runner.ctx)
    runner.step()
    torch.cuda.synchronize()
    stats = g.rmat_get_stats(runner.ctx)
    g.rmat_set_param(runner.ctx, g.RMAT_PARAM_TIMING, 0)
    g.rmat_reset_counters(runner.ctx)
    sync_all()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(K + 1)]
    ev[0].record(runner.stream)
    for k in range(K):
        runner.step()
        ev[k + 1].record(runner.stream)
    torch.cuda.synchronize()
    sync_all()
    launches = g.rmat_get_stats(runner.ctx)["launches"]
    per = [ev[k].elapsed_time(ev[k + 1]) for k in range(K)]
    stats["ms_steps"] = {"best": min(per), "median": float(np.median(per)), "all": per}
    return ev[0].elapsed_time(ev[K]) / K, stats, launches


def time_e2e(runner, K):
    """Same step from pinned host buffers: V H2D + step + R, U D2H, per step."""
    torch = runner.torch
    Vh = torch.from_numpy(runner.V_host).pin_memory()
    Rh = torch.empty(runner.R.numel(), dtype=torch.complex128).pin_memory()
    Uh = torch.empty(runner.U.numel(), dtype=torch.complex128).pin_memory()
    Vd = torch.empty_like(runner.Vd)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(runner.stream)
    for _ in range(K):
        Vd.copy_(Vh, non_blocking=True)
        runner.step(Vd.data_ptr())
        Rh.copy_(runner.R, non_blocking=True)
        Uh.copy_(runner.U, non_blocking=True)
    e1.record(runner.stream)
    torch.cuda.synchronize()
    h2d = Vh.numel() * 16
    d2h = (Rh.numel() + Uh.numel()) * 16
    return e0.elapsed_time(e1) / K, h2d, d2h


def _oracle_job(nch):
    """One oracle solve of the config-3 family at nch x nlag=100 (worker process)."""
    import cc_problems as cp
    from oracle import oracle_solve
    t0 = time.perf_counter()
    oracle_solve(cp.config3(nch), refine_steps=3)
    return time.perf_counter() - t0


def oracle_pool(cores):
    """Spawned worker processes for the oracle, one BLAS thread each (the oracle's
    elementwise NumPy work runs on one core per process)."""
    import multiprocessing as mp
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["OMP_NUM_THREADS"] = "1"
    return mp.get_context("spawn").Pool(cores)


def oracle_round(pool, cores, nch):
    """`cores` independent oracle solves at once; returns (TFLOP/s of the round, wall s)."""
    import cc_problems as cp
    p = cp.config3(nch)
    t0 = time.perf_counter()
    pool.map(_oracle_job, [nch] * cores)
    wall = time.perf_counter() - t0
    return cores * lu_flops(p.N, p.nch) / wall / 1e12, wall


def host_cores():
    return len(os.sched_getaffinity(0))


def cpu_baseline(nch=8):
    """The CPU oracle (as it stands) on all host cores: one process per core, each
    solving one system of the same family at N = nch*100 (a bounded sample of the
    N = 25600 workload; LU + 3 double-double refinement steps + R + U)."""
    cores = host_cores()
    with oracle_pool(cores) as pool:
        pool.map(_oracle_job, [2] * cores)        # start-up and imports outside the sample
        val, wall = oracle_round(pool, cores, nch)
    return {"value": val, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
            "sample": f"{cores} concurrent oracle solves (one per core) of config3 nch={nch} "
                      f"nlag=100 (N={nch * 100}, {nch} rhs): LU + 3 double-double refinement "
                      f"steps + R + U; {wall:.1f} s wall"}


def reference_main(args):
    """The reference arm: the CPU oracle on the host cores, each step one round of
    concurrent oracle solves (one per core) at N = 400 of the workload's family."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    nch = 4
    cores = host_cores()
    with oracle_pool(cores) as pool:
        for _ in range(args.warmup):
            oracle_round(pool, cores, nch)
        t0 = time.perf_counter()
        for _ in range(args.steps):
            oracle_round(pool, cores, nch)
        dt = (time.perf_counter() - t0) / args.steps
    import cc_problems as cp
    p = cp.config3(nch)
    val = cores * lu_flops(p.N, p.nch) / dt / 1e12
    sample = (f"per step {cores} concurrent oracle solves (one per core) of config3 nch={nch} "
              f"nlag=100 (N={p.N}, {nch} rhs): LU + 3 double-double refinement steps + R + U")
    line = {"impl": "reference", "metric": "N=25600 complex solve time & TFLOP/s: FP32+IR vs FP64 "
            "at equal U error", "value": val, "unit": "TFLOP/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": dt * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": f"config3 nch={nch} nlag=100 N={p.N} E=10 MeV seed 11592 "
                                   f"(bounded CPU sample of the N=25600 workload's family)",
                       "sample": sample},
            "cpu_baseline": {"value": val, "unit": "TFLOP/s", "cores": cores, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": val, "unit": "TFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


def profile_step(nch, precision, warm=True, method=0, factor=0):
    """Launch sequence for ncu: the warm-up step uses the SIMT precision, so the
    first tensor-core launch of the run is the first trailing update at N = nch*100."""
    import torch

    import cc_problems as cp
    import paper_2512_11590_gb300 as g
    torch.cuda.set_device(0)
    if warm:
        w = Runner(cp.config3(16), g.RMAT_C64_SIMT_IR, 0)
        w.step()
        w.close()
    run = Runner(cp.config3(nch), precision, 0, method, factor=factor)
    run.step()
    torch.cuda.synchronize()
    print("profile step", nch, run.last)
    run.close()
    return 0


def batch_main(args):
    """Config 4: 512 independent systems of uneven size (N = 80 .. 6400) through
    the batch driver (tuned plan + CUDA graph), against a loop of single-system
    calls on the same inputs.  Prints one JSON line (systems/s)."""
    print(json.dumps(batch_run(args, args.batch, args.steps, args.warmup, args.precision)))
    return 0


def batch_run(args, nsys, steps, warmup, precision):
    import torch

    import cc_problems as cp
    import paper_2512_11590_gb300 as g
    torch.cuda.set_device(0)
    probs = cp.batch_problems(nsys)
    prec = {"tf32": g.RMAT_C64_3XTF32_IR, "f16": g.RMAT_C64_3XF16_IR,
            "simt": g.RMAT_C64_SIMT_IR, "c128": g.RMAT_C128}[precision]
    stream = torch.cuda.Stream()                 # capturable stream for the batch's CUDA graph
    ctx = g.rmat_create(0, stream.cuda_stream)
    Vs, structs, keep = [], [], []
    for p in probs:
        m = g.rmat_mesh(p.nlag, p.a)
        Vs.append(torch.from_numpy(cp.potential_at(p, m["r"]).ravel()).cuda())
        s, k = g.make_problem_struct(p.nch, p.nlag, p.a, p.hm, p.l, p.thresh, prec, zz=p.zz)
        structs.append(s)
        keep.append(k)
    b = g.rmat_batch_create(ctx, structs, [p.E for p in probs], [v.data_ptr() for v in Vs],
                            max_refine=args.batch_refine, tol=1e-13)
    nopen = g.rmat_batch_nopen(b, len(probs))
    Us = [torch.zeros(max(1, n) ** 2, dtype=torch.complex128, device="cuda") for n in nopen]
    Uptr = [u.data_ptr() for u in Us]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if prec == g.RMAT_C128:   # the default plan (16 lanes, every system whose panels fit a cluster)
        lanes, split = 16, 8192
        g.rmat_batch_set(b, g.RMAT_BATCH_LANES, lanes)
        g.rmat_batch_set(b, g.RMAT_BATCH_SPLIT_N, split)
    else:
        # the autotuner's cache: plans tuned on GB300 ship with the package (a copy, so
        # that new entries do not touch it); a workload without an entry is timed here
        if "RMAT_TUNE_CACHE" not in os.environ:
            import shutil
            import tempfile
            tmp = os.path.join(tempfile.mkdtemp(prefix="rmat_tune_"), "plans.jsonl")
            shutil.copy(os.path.join(ROOT, "paper_2512_11590_gb300", "tuned_plans.jsonl"), tmp)
            os.environ["RMAT_TUNE_CACHE"] = tmp
        lanes, split = g.rmat_batch_tune(b, Uptr)
    tune_s = time.perf_counter() - t0
    for _ in range(warmup):
        g.rmat_batch_run(b, Uptr)
    torch.cuda.synchronize()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    with ClockSampler(0) as clk:
        e0.record(stream)
        for _ in range(steps):
            st, it = g.rmat_batch_run(b, Uptr)
        e1.record(stream)
        torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / steps
    info = g.rmat_batch_info(b)
    Ub = [u.cpu().numpy() for u in Us]
    g.rmat_batch_destroy(b)
    # the same systems one at a time through the single-system calls
    Xs = [torch.zeros((p.nch, p.N), dtype=torch.complex128, device="cuda") for p in probs]
    Ul = [torch.zeros_like(u) for u in Us]

    def loop():
        for p, s, v, X, U in zip(probs, structs, Vs, Xs, Ul):
            g.rmat_assemble(ctx, s, p.E, v.data_ptr())
            g.rmat_factor(ctx, want_info=False)
            g.rmat_solve(ctx, X.data_ptr(), p.N, max_refine=30, tol=1e-13)
            g.rmat_collision(ctx, 0, U.data_ptr())
    loop()
    torch.cuda.synchronize()
    e0.record(stream)
    loop()
    e1.record(stream)
    torch.cuda.synchronize()
    ms_loop = e0.elapsed_time(e1)
    diff = max(float(np.max(np.abs(u - w.cpu().numpy())) / max(1e-300, np.max(np.abs(w.cpu().numpy()))))
               for u, w, n in zip(Ub, Ul, nopen) if n > 0)
    g.rmat_destroy(ctx)
    Ns = np.array([p.N for p in probs])
    flops = float(sum(lu_flops(p.N, p.nch) for p in probs))
    line = {"metric": "batched systems/s (config 4: %d uneven systems)" % len(probs),
            "value": len(probs) / (ms * 1e-3), "unit": "systems/s", "n_gpus": 1,
            "steps": steps, "warmup": warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES.get(prec, "c128"),
            "data": "synthetic",
            "config": {"workload": "config4 batch_problems(%d) seed 11593, N %d..%d, median %d"
                       % (len(probs), Ns.min(), Ns.max(), int(np.median(Ns))),
                       "lanes": lanes, "split_n": split, "graph": info.get("graph"),
                       "plan": {k: info.get(k) for k in ("small_systems", "small_n", "nb_lane",
                                                         "nb_serial", "tc_bn_lane")},
                       "tune_s": tune_s, "tune_cache": os.environ.get("RMAT_TUNE_CACHE"),
                       "max_refine": args.batch_refine},
            "tflops": flops / (ms * 1e-3) / 1e12,
            "loop": {"ms_per_step": ms_loop, "systems_per_s": len(probs) / (ms_loop * 1e-3),
                     "speedup_batch_over_loop": ms_loop / ms, "u_rel_diff_batch_vs_loop": diff},
            "statuses": {str(k): int(v) for k, v in zip(*np.unique(st, return_counts=True))},
            "refine_steps_max": int(max(it)), "clocks": clk.summary()}
    return line


def solve_once(p, precision, device=0, warm=False, energies=None, method=0, refine=0):
    """One assembled system through the C ABI on a non-default stream: wall times of
    assemble+factor+solve+collision per energy, refinement info, U per energy."""
    import torch

    import cc_problems as cp
    import paper_2512_11590_gb300 as g
    stream = torch.cuda.Stream()
    ctx = g.rmat_create(device, stream.cuda_stream)
    g.rmat_set_param(ctx, g.RMAT_PARAM_METHOD, method)
    g.rmat_set_param(ctx, g.RMAT_PARAM_REFINE, refine)
    m = g.rmat_mesh(p.nlag, p.a)
    Vd = torch.from_numpy(cp.potential_at(p, m["r"]).ravel()).cuda()
    prob, keep = g.make_problem_struct(p.nch, p.nlag, p.a, p.hm, p.l, p.thresh, precision,
                                       zz=p.zz)
    X = torch.zeros((p.nch, p.N), dtype=torch.complex128, device="cuda")
    R = torch.zeros(p.nch * p.nch, dtype=torch.complex128, device="cuda")
    Es = list(energies) if energies else [p.E]
    out = []
    for k, E in enumerate(([Es[0]] if warm else []) + Es):
        nopen = int(np.sum(E - p.thresh > 0))
        U = torch.zeros(max(1, nopen) ** 2, dtype=torch.complex128, device="cuda")
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.rmat_assemble(ctx, prob, E, Vd.data_ptr())
        g.rmat_factor(ctx, want_info=False)
        st, it, rel = g.rmat_solve(ctx, X.data_ptr(), p.N, max_refine=30, tol=1e-13)
        g.rmat_collision(ctx, R.data_ptr(), U.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        if warm and k == 0:
            continue
        out.append({"E": E, "ms": e0.elapsed_time(e1), "status": st, "iters": it, "rel_resid": rel,
                    "inner": g.rmat_get_stats(ctx).get("gmres_inner", 0),
                    "U": U.cpu().numpy()[:nopen * nopen].reshape(nopen, nopen).T})
    g.rmat_destroy(ctx)
    return out


def sweep_main(args):
    """Config 2 sweep N in {1600, 6400, 12800, 25600} and config 3b (W = -1): the
    complex128 path against FP32+IR (split FP16) on the same systems."""
    import torch

    import cc_problems as cp
    import paper_2512_11590_gb300 as g
    torch.cuda.set_device(0)
    rows = []
    cases = [("config2", cp.config2(n)) for n in (16, 64, 128, 256)] + [("config3b", cp.config3(256, W=-1.0))]
    def rd(a, b):
        return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
    for name, p in cases:
        lo = solve_once(p, g.RMAT_C64_3XF16_IR, warm=True)[0]
        wb = solve_once(p, g.RMAT_C64_3XF16_IR, warm=True, method=1)[0]
        gm = solve_once(p, g.RMAT_C64_3XF16_IR, warm=True, refine=20)[0]
        fl = lu_flops(p.N, p.nch)
        row = {"case": name, "N": p.N, "nrhs": p.nch,
               "fp32ir_ms": lo["ms"], "fp32ir_tflops": fl / (lo["ms"] * 1e-3) / 1e12,
               "fp32ir_iters": lo["iters"], "fp32ir_rel_resid": lo["rel_resid"],
               "woodbury_ms": wb["ms"], "woodbury_iters": wb["iters"],
               "woodbury_rel_resid": wb["rel_resid"], "u_rel_diff_woodbury_vs_direct": rd(wb["U"], lo["U"]),
               "gmres_ir_ms": gm["ms"], "gmres_ir_outer": gm["iters"], "gmres_ir_inner": gm["inner"],
               "gmres_ir_rel_resid": gm["rel_resid"], "u_rel_diff_gmres_vs_direct": rd(gm["U"], lo["U"])}
        if not args.no_fp64:
            hi = solve_once(p, g.RMAT_C128, warm=p.N <= 6400)[0]
            row.update({"fp64_ms": hi["ms"], "fp64_tflops": fl / (hi["ms"] * 1e-3) / 1e12,
                        "fp64_iters": hi["iters"], "speedup": hi["ms"] / lo["ms"],
                        "u_rel_diff": rd(lo["U"], hi["U"]), "u_rel_diff_woodbury": rd(wb["U"], hi["U"])})
        rows.append(row)
        print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"metric": "config 2 sweep + config 3b: FP32+IR vs FP64 (complex128) per system",
                      "unit": "ms", "rows": rows, "data": "synthetic"}))
    return 0


def propagate_main(args):
    """R-matrix propagation: a charged alpha + 208Pb-like system (nch = 64, E = 30 MeV)
    carried to a = 40 fm over 4 sectors of nlag = 100 (N = 6400 each) against one
    system of nlag = 400 on (0, 40) (N = 25600), split-FP16 factors, FP64 refinement."""
    import torch

    import cc_problems as cp
    import paper_2512_11590_gb300 as g
    torch.cuda.set_device(0)
    prec = g.RMAT_C64_3XF16_IR
    a, ns, nlag = 40.0, 4, 100
    radii = [a * s / ns for s in range(ns + 1)]
    p = cp.charged_problem(26, 64, nlag, 30.0, a=a)
    stream = torch.cuda.current_stream()
    ctx = g.rmat_create(0, stream.cuda_stream)
    Vs = []
    for s in range(ns):
        r = (g.rmat_mesh(nlag, radii[1])["r"] if s == 0
             else g.rmat_sector_mesh(nlag, radii[s], radii[s + 1])["r"])
        Vs.append(torch.from_numpy(cp.potential_at(p, r).ravel()).cuda())
    prob, keep = g.make_problem_struct(p.nch, nlag, a, p.hm, p.l, p.thresh, prec, zz=p.zz)
    no = int(np.sum(p.E - p.thresh > 0))
    U = torch.zeros(no * no, dtype=torch.complex128, device="cuda")
    times = []
    for k in range(args.warmup + args.steps):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        st, _ = g.rmat_propagate(ctx, prob, p.E, radii, [v.data_ptr() for v in Vs], 30, 1e-13,
                                 0, U.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        if k >= args.warmup:
            times.append(e0.elapsed_time(e1))
    Up = U.cpu().numpy().reshape(no, no).T
    g.rmat_set_param(ctx, g.RMAT_PARAM_PROP_CONCURRENT, 0)   # sectors one after the other
    seq = []
    for k in range(2):
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        g.rmat_propagate(ctx, prob, p.E, radii, [v.data_ptr() for v in Vs], 30, 1e-13, 0,
                         U.data_ptr())
        e1.record(stream)
        torch.cuda.synchronize()
        seq.append(e0.elapsed_time(e1))
    g.rmat_destroy(ctx)
    p1 = cp.charged_problem(26, 64, 4 * nlag, 30.0, a=a)
    one = solve_once(p1, prec, warm=True)[0]
    rd = float(np.max(np.abs(Up - one["U"])) / np.max(np.abs(one["U"])))
    print(json.dumps({"metric": "R-matrix propagation: 4 sectors of N=6400 vs one system of N=25600 "
                                "to a = 40 fm (charged, nch = 64)",
                      "unit": "ms", "propagation_ms": float(np.median(times)),
                      "propagation_sequential_ms": float(seq[-1]),
                      "single_system_ms": one["ms"], "single_system_iters": one["iters"],
                      "speedup": one["ms"] / float(np.median(times)), "u_rel_diff": rd,
                      "sectors": ns, "nlag_per_sector": nlag, "status": st, "data": "synthetic"}))
    return 0


def cpu_lapack_main(args):
    """Host-core context (the paper's Type 1 and Type 2 on the CPU): SciPy LAPACK
    complex128 LU + solve (zgetrf/zgetrs) and complex64 LU (cgetrf) + FP64
    refinement on the config-2 systems at N = 1600 and 6400, threads as the BLAS
    build provides them.  The matrix is assembled densely from the library's host
    mesh tables (no GPU)."""
    import time

    import scipy.linalg as sl

    import cc_problems as cp
    import paper_2512_11590_gb300 as g
    rows = []
    for nch in (16, 64):
        p = cp.config2(nch)
        m = g.rmat_mesh(p.nlag, p.a)
        V = cp.potential_at(p, m["r"])
        n, L = p.N, p.nlag
        l = np.asarray(p.l, dtype=np.float64)
        C = np.zeros((n, n), dtype=np.complex128)
        for al in range(p.nch):
            blk = slice(al * L, (al + 1) * L)
            C[blk, blk] = p.hm * m["T0"]
            C[blk, blk] += np.diag(p.hm * l[al] * (l[al] + 1) / m["r"] ** 2 + p.thresh[al] - p.E)
            for be in range(p.nch):
                C[al * L + np.arange(L), be * L + np.arange(L)] += V[be, al, :]
        B = np.zeros((n, p.nch), dtype=np.complex128)
        for al in range(p.nch):
            B[al * L:(al + 1) * L, al] = m["f_a"]
        t0 = time.perf_counter()
        X64 = sl.lu_solve(sl.lu_factor(C, check_finite=False), B, check_finite=False)
        t1 = time.perf_counter()
        lu32 = sl.lu_factor(C.astype(np.complex64), check_finite=False)
        X = sl.lu_solve(lu32, B.astype(np.complex64), check_finite=False).astype(np.complex128)
        for _ in range(8):
            r = B - C @ X
            if np.abs(r).max() / np.abs(B).max() < 1e-13:
                break
            X += sl.lu_solve(lu32, r.astype(np.complex64), check_finite=False)
        t2 = time.perf_counter()
        rows.append({"N": n, "nrhs": p.nch, "zgesv_s": t1 - t0, "cgetrf_ir_s": t2 - t1,
                     "x_rel_diff": float(np.abs(X - X64).max() / np.abs(X64).max())})
        print(json.dumps(rows[-1]), flush=True)
    print(json.dumps({"metric": "host-core LAPACK context (Type 1 / Type 2 analogues)",
                      "cores": len(os.sched_getaffinity(0)), "rows": rows, "data": "synthetic"}))
    return 0


def config5_main(args):
    """Config 5: N = 51200 (nch = 512, nlag = 100), 512 right-hand sides, an energy sweep
    of 8 points reusing the assembly buffers (FP32+IR), and one energy in complex128 for
    the U error."""
    import torch

    import cc_problems as cp
    import paper_2512_11590_gb300 as g
    torch.cuda.set_device(0)
    p = cp.config5(cp.CONFIG5_ENERGIES[0])
    sweep = solve_once(p, g.RMAT_C64_3XF16_IR, warm=True, energies=cp.CONFIG5_ENERGIES)
    fl = lu_flops(p.N, p.nch)
    line = {"metric": "config 5: N=51200 energy sweep (8 energies), FP32+IR", "unit": "ms",
            "N": p.N, "nrhs": p.nch, "data": "synthetic",
            "energies": [{"E": r["E"], "ms": r["ms"], "tflops": fl / (r["ms"] * 1e-3) / 1e12,
                          "iters": r["iters"], "rel_resid": r["rel_resid"], "status": r["status"]}
                         for r in sweep],
            "total_ms": sum(r["ms"] for r in sweep)}
    if not args.no_fp64:
        hi = solve_once(p, g.RMAT_C128, warm=False)[0]
        lo = sweep[0]
        line["fp64_first_energy"] = {
            "ms": hi["ms"], "tflops": fl / (hi["ms"] * 1e-3) / 1e12, "iters": hi["iters"],
            "u_rel_diff_fp32ir_vs_fp64": float(np.max(np.abs(lo["U"] - hi["U"])) /
                                               np.max(np.abs(hi["U"]))),
            "speedup_fp32ir_over_fp64": hi["ms"] / lo["ms"]}
    print(json.dumps(line))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f16", choices=["f16", "f16x1", "tf32", "simt", "c128"],
                    help="c128 only with --batch")
    ap.add_argument("--small", action="store_true", help="N=1600 instead of N=25600")
    ap.add_argument("--no-fp64", action="store_true", help="skip the complex128 comparison")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-tf32", action="store_true", help="skip the 3xTF32 comparison leg")
    ap.add_argument("--factor", default="lu", choices=["lu", "ldlt"],
                    help="main line's factorisation: LU with partial pivoting or LDL^T")
    ap.add_argument("--no-ldlt", action="store_true", help="skip the LDL^T comparison leg")
    ap.add_argument("--residual", default="auto", choices=["auto", "fp64mma", "tensor", "tensor-all"],
                    help="products of the FP64 residual (RMAT_PARAM_RESIDUAL 0..3)")
    ap.add_argument("--solve-block", type=int, default=0, choices=[0, 128, 256],
                    help="rows per tensor-path solve step (RMAT_PARAM_SOLVE_BLOCK; 0 = 256)")
    ap.add_argument("--refine", type=int, default=0,
                    help="GMRES-IR inner steps per correction (RMAT_PARAM_REFINE; 0 classical)")
    ap.add_argument("--no-batch", action="store_true",
                    help="skip the config-4 batch leg (512 systems) of the default line")
    ap.add_argument("--method", default="direct", choices=["direct", "woodbury"],
                    help="factor M itself or the Woodbury-kinetic Schur matrix S")
    ap.add_argument("--no-woodbury", action="store_true",
                    help="skip the Woodbury-kinetic comparison leg")
    ap.add_argument("--solve-lookahead", type=int, default=1, choices=[1, 2],
                    help="RMAT_PARAM_SOLVE_LOOKAHEAD mode (2: next rows in the diagonal step)")
    ap.add_argument("--no-lookahead", action="store_true",
                    help="tensor-path solves without look-ahead (bitwise reproducible)")
    ap.add_argument("--factor-lookahead", type=int, default=1, choices=[0, 1, 2],
                    help="RMAT_PARAM_FACTOR_LOOKAHEAD: 0 one far update at a time, 1 panels "
                         "beside the far update, 2 the look-ahead order on one stream")
    ap.add_argument("--la-panel-ctas", type=int, default=0,
                    help="CTAs of a look-ahead sub-panel (RMAT_PARAM_LA_PANEL_CTAS; 0 = every SM)")
    ap.add_argument("--solve-groups", type=int, default=0, choices=[0, 1, 2],
                    help="concurrent column groups of the tensor-path solves (0 = default, 1)")
    ap.add_argument("--la-min-rows", type=int, default=0,
                    help="smallest far block that looks ahead (RMAT_PARAM_LA_MIN_ROWS; 0 = 6144)")
    ap.add_argument("--la-both-rows", type=int, default=0,
                    help="smallest far block with both next panels beside its update "
                         "(RMAT_PARAM_LA_BOTH_ROWS; 0 = 20480)")
    ap.add_argument("--tc-bn", type=int, default=0, choices=[0, 128, 256],
                    help="tile width of the factor's tensor-core updates (RMAT_PARAM_TC_BN)")
    ap.add_argument("--profile-step", action="store_true",
                    help="for ncu: one untimed SIMT warm-up step at N=1600, then one FP32+IR "
                         "tensor step at N = nch*100; no timing, no JSON")
    ap.add_argument("--nch", type=int, default=256, help="channels of the --profile-step system")
    ap.add_argument("--no-warm", action="store_true", help="--profile-step without the warm-up step")
    ap.add_argument("--batch", type=int, default=0,
                    help="time the batch driver on this many config-4 systems instead")
    ap.add_argument("--sweep", action="store_true",
                    help="config 2 sweep (N=1600..25600) and config 3b, FP32+IR vs complex128")
    ap.add_argument("--cpu-lapack", action="store_true",
                    help="host-core SciPy LAPACK context at N = 1600 and 6400 (no GPU)")
    ap.add_argument("--propagate", action="store_true",
                    help="R-matrix propagation over 4 sectors vs one system (charged, a = 40 fm)")
    ap.add_argument("--config5", action="store_true",
                    help="config 5: N=51200, 8-energy FP32+IR sweep (+ one complex128 energy)")
    ap.add_argument("--batch-refine", type=int, default=10,
                    help="refinement-step budget of the batch (stopping decided on the device)")
    args = ap.parse_args()
    if args.warmup < 3:
        print("warmup must be >= 3", file=sys.stderr)
        return 2
    if args.impl == "reference":
        return reference_main(args)
    if args.profile_step:
        import paper_2512_11590_gb300 as g
        return profile_step(args.nch, {"tf32": g.RMAT_C64_3XTF32_IR, "f16": g.RMAT_C64_3XF16_IR,
                                       "simt": g.RMAT_C64_SIMT_IR}[args.precision],
                            warm=not args.no_warm, method=1 if args.method == "woodbury" else 0,
                            factor=1 if args.factor == "ldlt" else 0)
    if args.batch:
        return batch_main(args)
    if args.precision == "c128":
        print("--precision c128 is for --batch (the main line times FP32+IR)", file=sys.stderr)
        return 2
    if args.precision == "f16x1" and args.refine == 0:
        print("--precision f16x1 needs --refine m (GMRES-IR)", file=sys.stderr)
        return 2
    if args.sweep:
        return sweep_main(args)
    if args.config5:
        return config5_main(args)
    if args.propagate:
        return propagate_main(args)
    if args.cpu_lapack:
        return cpu_lapack_main(args)

    import torch
    import paper_2512_11590_gb300 as g
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)

    def sync_all():
        torch.cuda.synchronize()
        if dist is not None:
            dist.barrier()

    p, desc = workload(args)
    prec = {"tf32": g.RMAT_C64_3XTF32_IR, "f16": g.RMAT_C64_3XF16_IR,
            "f16x1": g.RMAT_C64_1XF16_IR, "simt": g.RMAT_C64_SIMT_IR}[args.precision]
    method = 1 if args.method == "woodbury" else 0
    resid = {"auto": 0, "fp64mma": 1, "tensor": 2, "tensor-all": 3}[args.residual]
    factor = 1 if args.factor == "ldlt" else 0
    run = Runner(p, prec, local, method, 0 if args.no_lookahead else args.solve_lookahead, resid, args.solve_block,
                 factor, args.factor_lookahead, args.la_panel_ctas,
                 args.la_min_rows, args.solve_groups, args.la_both_rows, args.tc_bn)
    g.rmat_set_param(run.ctx, g.RMAT_PARAM_REFINE, args.refine)
    with ClockSampler(local) as clk:
        ms, stats, launches = time_steps(run, args.steps, args.warmup, sync_all)
    ms = max_over_ranks(ms, dist, "cuda")
    flops = lu_flops(p.N, p.nch)
    value = replica_throughput(world, flops, ms)
    sync_all()
    e2e_ms, h2d, d2h = time_e2e(run, max(1, min(args.steps, 3)))
    e2e_ms = max_over_ranks(e2e_ms, dist, "cuda")
    U32 = run.U_host()
    X32, R32 = run.XR_host()
    ir = dict(run.last)
    run.close()

    fp64, fp64_arrays = None, (None, None, None)
    if not args.no_fp64:
        r64 = Runner(p, g.RMAT_C128, local, residual=resid)
        r64.step()                                  # warm-up (module load, buffers)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(r64.stream)
        r64.step()
        e1.record(r64.stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        U64 = r64.U_host()
        X64, R64 = r64.XR_host()

        def rd(a, b):
            return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
        fp64_arrays = (X64, R64, U64)
        fp64 = {"ms_per_step": ms64, "tflops": flops / (ms64 * 1e-3) / 1e12,
                "refine": dict(r64.last),
                "u_rel_diff_fp32ir_vs_fp64": rd(U32, U64),
                "r_rel_diff_fp32ir_vs_fp64": rd(R32, R64),
                "x_rel_diff_fp32ir_vs_fp64": rd(X32, X64),
                "speedup_fp32ir_over_fp64": ms64 / ms}
        r64.close()

    serial = None
    if factor == 0 and method == 0 and args.factor_lookahead != 0:
        # the same step without the factorisation's look-ahead: the trailing update
        # then runs alone on every SM (its kernel-only roofline) and the panels in order
        rs = Runner(p, prec, local, method, 0 if args.no_lookahead else args.solve_lookahead, resid,
                    args.solve_block, factor, 0, 0, 0, args.solve_groups, 0, args.tc_bn)
        rs.step()
        g.rmat_set_param(rs.ctx, g.RMAT_PARAM_TIMING, 1)
        g.rmat_reset_counters(rs.ctx)
        rs.step()
        torch.cuda.synchronize()
        st_s = g.rmat_get_stats(rs.ctx)
        g.rmat_set_param(rs.ctx, g.RMAT_PARAM_TIMING, 0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ks = max(1, min(args.steps, 3))
        e0.record(rs.stream)
        for _ in range(ks):
            rs.step()
        e1.record(rs.stream)
        torch.cuda.synchronize()
        mss = max_over_ranks(e0.elapsed_time(e1) / ks, dist, "cuda")
        serial = {"factor_lookahead": 0, "ms_per_step": mss, "steps": ks,
                  "value": replica_throughput(world, flops, mss), "refine": dict(rs.last),
                  "stage_ms": {k: st_s[k] for k in ("factor_ms", "solve_ms", "refine_ms")},
                  "panel_ms": [st_s.get("panel_ms"), st_s.get("panel_launches")],
                  "trailing_update": {"kernel_ms_per_step": st_s["tu_ms"],
                                      "launches": st_s["tu_launches"],
                                      "achieved_tflops": st_s["tu_flops"] / (st_s["tu_ms"] * 1e-3) / 1e12
                                      if st_s["tu_ms"] > 0 else None}}
        rs.close()

    other = None
    if not args.no_woodbury:
        # the other factored matrix (Woodbury-kinetic S vs M) on the same workload
        rw = Runner(p, prec, local, 1 - method, 0 if args.no_lookahead else args.solve_lookahead, resid)
        for _ in range(2):
            rw.step()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(rw.stream)
        for _ in range(args.steps):
            rw.step()
        e1.record(rw.stream)
        torch.cuda.synchronize()
        msw = max_over_ranks(e0.elapsed_time(e1) / args.steps, dist, "cuda")
        Uw = rw.U_host()

        def rdw(a, b):
            return float(np.max(np.abs(a - b)) / np.max(np.abs(b)))
        other = {"method": "direct" if method else "woodbury", "ms_per_step": msw,
                 "value": replica_throughput(world, flops, msw), "refine": dict(rw.last),
                 "u_rel_diff_vs_main": rdw(Uw, U32)}
        if fp64 is not None:
            other["u_rel_diff_vs_fp64"] = rdw(Uw, U64)
        rw.close()

    pk, src = peaks()
    tf32 = None
    if prec == g.RMAT_C64_3XF16_IR and not args.no_tf32:
        # the FP32-class 3xTF32 split on the same system (the FP32 factorisation of the method)
        rt = Runner(p, g.RMAT_C64_3XTF32_IR, local, residual=resid)
        rt.step()
        g.rmat_set_param(rt.ctx, g.RMAT_PARAM_TIMING, 1)
        g.rmat_reset_counters(rt.ctx)
        rt.step()
        torch.cuda.synchronize()
        st_t = g.rmat_get_stats(rt.ctx)
        g.rmat_set_param(rt.ctx, g.RMAT_PARAM_TIMING, 0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        kt = max(1, min(args.steps, 3))
        e0.record(rt.stream)
        for _ in range(kt):
            rt.step()
        e1.record(rt.stream)
        torch.cuda.synchronize()
        mst = max_over_ranks(e0.elapsed_time(e1) / kt, dist, "cuda")
        Ut = rt.U_host()
        Xt, Rt = rt.XR_host()
        tpk = pk["bf16_tflops_sustained"] * TF32_PER_BF16 / 3.0
        ach = st_t["tu_flops"] / (st_t["tu_ms"] * 1e-3) / 1e12 if st_t["tu_ms"] > 0 else None
        tf32 = {"precision": DTYPES[g.RMAT_C64_3XTF32_IR], "ms_per_step": mst, "steps": kt,
                "value": replica_throughput(world, flops, mst), "unit": "TFLOP/s",
                "refine": dict(rt.last),
                "u_rel_diff_vs_main": float(np.max(np.abs(Ut - U32)) / np.max(np.abs(U32))),
                "roofline": {"kernel": "trailing update C22 -= L21 U12 (kind::tf32, 3 products)",
                             "bound": "tensor", "achieved": ach, "peak": tpk, "unit": "TFLOP/s",
                             "frac": ach / tpk if ach else None,
                             "peak_source": "bf16 sustained (%s) x 0.5 (tf32/bf16 nominal) / 3 "
                                            "(tf32 split products per fp32 product)" % src,
                             "kernel_ms_per_step": st_t["tu_ms"], "launches": st_t["tu_launches"]}}
        tf32_arrays = (Xt, Rt, Ut)
        rt.close()
    else:
        tf32_arrays = (None, None, None)
    ldlt, ldlt_arrays = None, (None, None, None)
    if prec == g.RMAT_C64_3XF16_IR and factor == 0 and method == 0 and not args.no_ldlt:
        # the complex-symmetric LDL^T (no pivot panel, half the update) on the same system
        rl = Runner(p, prec, local, residual=resid, solve_block=args.solve_block, factor=1)
        rl.step()
        g.rmat_set_param(rl.ctx, g.RMAT_PARAM_TIMING, 1)
        g.rmat_reset_counters(rl.ctx)
        rl.step()
        torch.cuda.synchronize()
        st_l = g.rmat_get_stats(rl.ctx)
        g.rmat_set_param(rl.ctx, g.RMAT_PARAM_TIMING, 0)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        kl = max(1, min(args.steps, 3))
        e0.record(rl.stream)
        for _ in range(kl):
            rl.step()
        e1.record(rl.stream)
        torch.cuda.synchronize()
        msl = max_over_ranks(e0.elapsed_time(e1) / kl, dist, "cuda")
        Ul = rl.U_host()
        Xl, Rl = rl.XR_host()
        lpk = pk["bf16_tflops_sustained"] / 3.0
        lach = st_l["tu_flops"] / (st_l["tu_ms"] * 1e-3) / 1e12 if st_l["tu_ms"] > 0 else None
        ldlt = {"factor": "complex-symmetric LDL^T without pivoting (C = C^T), 3xFP16 updates "
                          "on the tiles on or above the diagonal",
                "ms_per_step": msl, "steps": kl,
                "value_lu_flop_count": replica_throughput(world, flops, msl), "unit": "TFLOP/s",
                "value_note": "LU's flop count (8N^3/3 + 8N^2 nrhs) over this time: the LDL^T "
                              "does about half the factor flops",
                "speedup_vs_main": ms / msl,
                "refine": dict(rl.last), "ldlt_lmax": st_l.get("ldlt_lmax"),
                "stage_ms": {k: st_l[k] for k in ("assemble_ms", "factor_ms", "solve_ms",
                                                   "refine_ms", "collision_ms")},
                "diag_block_ms": [st_l.get("panel_ms"), st_l.get("panel_launches")],
                "u_rel_diff_vs_main": float(np.max(np.abs(Ul - U32)) / np.max(np.abs(U32))),
                "roofline": {"kernel": "symmetric trailing update (upper tiles) C22 -= L21 U12",
                             "bound": "tensor", "achieved": lach, "peak": lpk, "unit": "TFLOP/s",
                             "frac": lach / lpk if lach else None,
                             "peak_source": "bf16 sustained (%s) / 3 (fp16 split products per "
                                            "fp32 product)" % src,
                             "flops": "8 K M (M + 128) / 2 per launch (upper triangle and the "
                                      "diagonal blocks' lower halves)",
                             "kernel_ms_per_step": st_l["tu_ms"],
                             "launches": st_l["tu_launches"]}}
        ldlt_arrays = (Xl, Rl, Ul)
        rl.close()
    tu_ms, tu_flops, tu_n = stats["tu_ms"], stats["tu_flops"], stats["tu_launches"]
    if prec == g.RMAT_C64_3XTF32_IR:
        # each complex product = 4 real GEMMs x 3 tf32 split products: 12 tensor GEMMs
        peak = pk["bf16_tflops_sustained"] * TF32_PER_BF16 / 3.0
        bound, unit, pname = "tensor", "TFLOP/s", ("bf16 sustained (%s) x 0.5 (tf32/bf16 nominal) / 3 "
                                                    "(tf32 split products per fp32 product)" % src)
    elif prec in (g.RMAT_C64_3XF16_IR, g.RMAT_C64_1XF16_IR):
        # 4 real GEMMs x 3 (or 1) fp16 split products; fp16 and bf16 share the tensor rate
        npr = 3.0 if prec == g.RMAT_C64_3XF16_IR else 1.0
        peak = pk["bf16_tflops_sustained"] / npr
        bound, unit, pname = "tensor", "TFLOP/s", ("bf16 sustained (%s) / %d (fp16 split products "
                                                    "per fp32 product; fp16 rate = bf16 rate)"
                                                    % (src, npr))
    else:
        peak = 152 * 128 * 2 * 2070e6 / 1e12
        bound, unit, pname = "alu", "TFLOP/s", "FP32 FMA: 152 SMs x 128 lanes x 2 flop x 2070 MHz"
    achieved = tu_flops / (tu_ms * 1e-3) / 1e12 if tu_ms and tu_ms > 0 else None
    compute_peak = peak
    traffic, tsrc = None, None
    nbk = int(stats["nb"])
    rests = [p.N - (k + 1) * nbk for k in range(p.N // nbk) if p.N - (k + 1) * nbk > 0]
    if prec == g.RMAT_C64_3XF16_IR:
        # the fp16 update is bound by C22's read-modify-write in HBM (8-byte complex64,
        # read + written per update) more than by the tensor pipe; report it against HBM.
        # Paired updates (default): per pair one narrow update of the next panel's
        # columns, one of its rows, and one K = 2 nb update of the far block.
        # Report the roof the kernel is nearest to (the larger fraction).
        alg = paired_update_bytes(p.N, nbk, 8.0)
        gbs = sum(alg) / (tu_ms * 1e-3) / 1e9 if tu_ms and tu_ms > 0 else None
        if gbs and achieved and gbs / pk["hbm_gbs"] > achieved / peak:
            pname = "STREAM copy (%s); tensor view: %.1f of %.1f TFLOP/s (bf16 sustained / 3)" % (
                src, achieved, peak)
            achieved, peak, bound, unit = gbs, pk["hbm_gbs"], "hbm", "GB/s"
        else:
            pname = ("bf16 sustained (%s) / 3 (fp16 split products per fp32 product; fp16 rate = "
                     "bf16 rate); HBM view: %.0f of %.0f GB/s algorithmic" % (src, gbs or 0.0,
                                                                               pk["hbm_gbs"]))
        # DRAM bytes per launch: the ncu capture of the first K = 256 paired update at
        # N = 6400 (the bench's N = 25600 launches are too large to capture), its DRAM
        # bytes per algorithmic byte scaled to this run's average launch
        ratio = profile_ratio("trailing_update_pair_f16_n6400.md")
        if ratio:
            traffic = ratio * (sum(alg) / len(alg))
            tsrc = ("scaled: ncu dram__bytes_read+write per algorithmic byte (%.3f) of the first "
                    "paired update at N=6400 (profiles/trailing_update_pair_f16_n6400.md) x this "
                    "run's average algorithmic bytes per launch" % ratio)
    if prec == g.RMAT_C64_3XTF32_IR:
        alg = [r * r * 16.0 + 2 * r * nbk * 16.0 for r in rests]
        ratio = profile_ratio("trailing_update_tc_n6400.md")
        if ratio:
            traffic = ratio * (sum(alg) / len(alg))
            tsrc = ("scaled: ncu dram__bytes_read+write per algorithmic byte (%.3f) of the first "
                    "update at N=6400 (profiles/trailing_update_tc_n6400.md) x this run's "
                    "average algorithmic bytes per launch" % ratio)
    if serial is not None and serial["trailing_update"]["achieved_tflops"]:
        serial["trailing_update"]["peak"] = compute_peak
        serial["trailing_update"]["frac"] = (serial["trailing_update"]["achieved_tflops"]
                                             / compute_peak)
        serial["trailing_update"]["note"] = ("the trailing update alone on every SM; in the main "
                                             "line the far part shares the SMs with the next panels")
    W = getattr(p, "W", -10.0)
    errs = None if p.N != 25600 else truth_errors(W, {"fp32ir": (X32, R32, U32), "fp64": fp64_arrays,
                                                      "tf32": tf32_arrays, "ldlt": ldlt_arrays})
    line = {
        "metric": "N=25600 complex solve time & TFLOP/s: FP32+IR vs FP64 at equal U error",
        "value": value, "unit": "TFLOP/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": DTYPES[prec],
        "data": "synthetic",
        "config": {"workload": desc, "precision": args.precision, "nrhs": p.nch,
                   "factor": {"lu": "LU with partial pivoting", "ldlt": "LDL^T"}[args.factor],
                   "method": args.method, "residual": args.residual,
                   "solve_block": args.solve_block or 256,
                   "solve_lookahead": 0 if args.no_lookahead else args.solve_lookahead,
                   "factor_lookahead": args.factor_lookahead,
                   "la_panel_ctas": args.la_panel_ctas or "all SMs",
                   "la_min_rows": args.la_min_rows or 6144,
                   "la_both_rows": args.la_both_rows or 20480,
                   "tc_bn": args.tc_bn or 256,
                   "solve_groups": args.solve_groups or 1,
                   "refinement": ir, "l2": "inputs larger than L2 (C is %.1f GB)" % (p.N * p.N * 8 / 1e9),
                   "lu_block": stats["nb"], "panel_ctas": stats["panel_ctas"],
                   "ms_per_step_best_median": [stats["ms_steps"]["best"],
                                               stats["ms_steps"]["median"]],
                   "stage_ms": {k: stats[k] for k in ("assemble_ms", "factor_ms", "solve_ms",
                                                       "refine_ms", "collision_ms")},
                   "kernel_ms": {k: [stats.get(k + "_ms"), stats.get(k + "_launches")]
                                 for k in ("panel", "apply_inv", "solve_tc", "resid")}},
        "fp64_path": fp64,
        "no_factor_lookahead": serial,
        "tf32_path": tf32,
        "ldlt_path": ldlt,
        "error_vs_truth": errs,
        "stages_roofline": stage_rooflines(stats, p.N, p.nch, int(stats["nb"]), ir["iters"], pk, src),
        "other_method": other,
        "e2e": {"value": replica_throughput(world, flops, e2e_ms), "unit": "TFLOP/s",
                "ms_per_step": e2e_ms, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": int(launches),
        "paper_context": {
            "hardware": "RTX 3090 (sm_86, CUDA 11.5) + 2x Xeon Gold 6248R (48 cores)",
            "n25600_type4_fp32_cusolver_s": 3.554, "n25600_type4_error": 8e-10,
            "n25600_hybrid_fp32_factor_plus_2_host_ir_s": 9.85, "n25600_hybrid_error": 6e-16,
            "n25600_type1_zgesv_cpu_s": 52.098, "n25600_legacy_zgetri_cpu_s": 144.948,
            "paper_speedups": "about 15x over its CPU direct solver and about 41x over the "
                              "legacy code at N=25600 (Type 4 vs Type 1 / Ref.)",
            "note": "other hardware and workloads: context only, not a ratio target"},
        "roofline": {"kernel": "trailing update C22 -= L21 U12 (with the factorisation's "
                               "look-ahead its far part runs beside the next panels)",
                     "bound": bound,
                     "achieved": achieved, "peak": peak, "peak_source": pname, "unit": unit,
                     "frac": (achieved / peak) if achieved else None, "traffic": traffic,
                     "traffic_source": tsrc,
                     "launches": tu_n, "kernel_ms_per_step": tu_ms,
                     "share_of_step": (tu_ms / ms) if tu_ms and tu_ms > 0 else None},
        "clocks": clk.summary(),
    }
    if world == 1 and not args.no_batch and not args.small:
        # config 4 (512 uneven systems) through the tuned batch driver, 3 timed runs
        bl = batch_run(args, 512, 3, 3, "f16")
        line["batch"] = {k: bl[k] for k in ("metric", "value", "unit", "ms_per_step", "tflops",
                                             "loop", "statuses", "refine_steps_max", "config")}
    if rank == 0:
        if world == 1 and not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline()
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
