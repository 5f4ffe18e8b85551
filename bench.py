"""Benchmark of the FMPBEM/PBEM hot path on the sonic-crystal barrier workload.

Workload: 3 x 20 rigid capped cylinders (r = 0.15 m, h = 3.0 m, square lattice
0.4 m), 1,200 flat triangles per cell, N = 72,000 dofs, plane wave at 30 deg
azimuth, frequencies 100..1000 Hz in 10 steps.  The cells are too tall for
the cell-as-box multipole expansion, so the library builds the PBEM form:
195 dense offset blocks, FFT over the padded 5 x 40 cell grid, circulant
products inside GMRES.

One step = one frequency of the sweep: operator build (collocation quadrature
of every offset block, FFT of the first block column), plane-wave right-hand
side, GMRES to relative residual 1e-8 (restart 1000, i.e. unrestarted on this
workload).  value = solves/s over K
steps timed with CUDA events; e2e = the same through the public API with host
buffers and the surface pressure copied back.  Under torchrun each rank runs
its own frequencies (replicas, weak scaling) and the slowest rank's time
counts.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
import argparse
import dataclasses
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from workloads import WORKLOADS, random_complex_vectors, SPEED_OF_SOUND  # noqa: E402

WORKLOAD = "sonic_crystal_3x20"
TOL = 1e-8
RESTART = 1000          # the 3x20 crystal near its Bragg frequency needs long Krylov bases (no frequency
                        # needs more than about 550 iterations, so this is unrestarted GMRES in 1.2 GB)
SHORT_RESTART = 200     # FMM workloads converge in < 100 iterations; a shorter basis saves memory
MAXIT = 3000
METRIC = "GMRES solves/s (operator build + solve, tol 1e-8) at N=72,000"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--profile-case", default=None,
                    choices=["product", "build", "near", "batch", "batch_full", "solve_bf16", "gmres", "barrier",
                             "admittance", "fmm2"],
                    help="small case for kernel captures: product/build = 3x8 cylinders (1.8 GB spectrum) at "
                         "500 Hz; near = 32x32 sphere array FMM; batch = 8x8x4 cube lattice, 64 RHS, BF16; gmres = 320 "
                         "Arnoldi steps of the full crystal at 300 Hz")
    ap.add_argument("--serving", type=int, default=0,
                    help="run only the serving study on the first N requests of the seeded stream (FP64, MIXED, "
                         "and the 10 Hz-snapped cache variant)")
    ap.add_argument("--only-headline", action="store_true",
                    help="skip the FMM, mixed-precision, serving and batching sections")
    ap.add_argument("--no-overlap", action="store_true",
                    help="run each step's operator build and solve back to back instead of building the next "
                         "step's operator on a second stream during the current solve")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def frequency_index(step, world, rank, nf):
    """Frequency of a step on a rank: the ranks of a replica run interleave the
    sweep, so N ranks cover N different frequencies per step (weak scaling)."""
    return (step * world + rank) % nf


def reduce_max_ms(ms, world, device="cpu"):
    """Slowest rank's time (the job's time) via an all-reduce MAX."""
    if world <= 1:
        return ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def config_block(w, extra=None):
    cfg = {
        "workload": "sonic_crystal_3x20: 3x20 rigid capped cylinders r=0.15 h=3.0, lattice 0.4 m, "
                    "1200 tri/cell, N=72000, PBEM form (195 offset blocks, P=5x40), 10 freqs 100-1000 Hz",
        "N": 72000,
        "frequencies_hz": [round(k * SPEED_OF_SOUND / (2 * math.pi), 3) for k in w.wavenumbers],
        "gmres": {"tol": TOL, "restart": RESTART, "maxit": MAXIT, "x0": 0},
        "l2": "inputs larger than L2: the 4.6 GB spectrum is streamed by every product",
    }
    if extra:
        cfg.update(extra)
    return cfg


# ------------------------------------------------------------ clock probe --

class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
              "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
              "clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-lms", "200",
                 "-i", str(index)], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons, power = [], [], set(), []
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 7:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
                power.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[3:7]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "power_w_max": max(power) if power else None, "samples": len(sm), "reasons": sorted(reasons)}


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except (OSError, ValueError):
        return {}


# ---------------------------------------------------------------- our arm --

class StepPipeline:
    """Runs steps (operator build, right-hand side, solve) so that the build of
    step i + 1 overlaps the solve of step i: the builds run on a low-priority
    stream from a second host thread (the library is thread-safe across
    operators, and ctypes releases the GIL during its calls), the solves on a
    high-priority stream from this thread.  The quadrature of a build is
    bound by FP32 issue while the solve's products are bound by HBM, so the
    two share the GPU well.  Every step still builds its own operator and
    solves it; run(first, count) builds step `first` alone and solves the last
    step alone, so a run of K steps holds exactly K builds and K solves."""

    def __init__(self, torch, make_op, solve_op, overlap=True):
        from concurrent.futures import ThreadPoolExecutor
        self.torch = torch
        self.make_op, self.solve_op, self.overlap = make_op, solve_op, overlap
        self.solve_stream = torch.cuda.Stream(priority=-1) if overlap else torch.cuda.current_stream()
        self.build_stream = torch.cuda.Stream(priority=0) if overlap else self.solve_stream
        self.pool = ThreadPoolExecutor(1) if overlap else None

    def _build(self, i):
        with self.torch.cuda.stream(self.build_stream):
            return self.make_op(i)

    def run(self, first, count, on_result):
        if count <= 0:
            return
        nxt = self.pool.submit(self._build, first) if self.overlap else None
        for i in range(first, first + count):
            op = nxt.result() if self.overlap else self._build(i)
            if self.overlap and i + 1 < first + count:
                nxt = self.pool.submit(self._build, i + 1)
            with self.torch.cuda.stream(self.solve_stream):
                res = self.solve_op(i, op)
            on_result(i, res)
            op.close()   # synchronises the device: the next build has finished too


def run_ours(args):
    import torch
    import paper_2201_12050_gb300 as gb

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    w = WORKLOADS[WORKLOAD]
    v, t = w.mesh()
    ks = w.wavenumbers
    d = w.directions
    nf = len(ks)

    def make_op(i):
        return gb.Operator(v, t, w.counts, w.lattice, ks[frequency_index(i, world, rank, nf)])

    def solve_op(i, op):
        b = op.rhs_plane_wave(d)
        return op.solve(b, tol=TOL, restart=RESTART, maxit=MAXIT, raise_on_noconv=False)

    pipe = StepPipeline(torch, make_op, solve_op, overlap=not args.no_overlap)

    def barrier():
        if world > 1:
            import torch.distributed as dist
            dist.barrier()
        torch.cuda.synchronize()

    pipe.run(0, args.warmup, lambda i, res: None)
    barrier()
    clocks = ClockSampler(local)
    gb.profile_reset()
    gb.profile_enable(True)
    launches0 = gb.kernel_launches()
    stream = torch.cuda.current_stream()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e0.record(stream)
    iters, relres, conv, sols, iters_by_freq = [], [], [], {}, {}

    def record(i, res):
        p, info = res
        iters.append(info[0]["iters"])
        iters_by_freq[frequency_index(i, world, rank, nf)] = info[0]["iters"]
        relres.append(info[0]["relres_true"])
        conv.append(info[0]["converged"])
        sols[frequency_index(i, world, rank, nf)] = p

    pipe.run(args.warmup, args.steps, record)
    torch.cuda.synchronize()
    e1.record(stream)
    barrier()
    gb.profile_enable(False)
    ms = e0.elapsed_time(e1)
    launches = gb.kernel_launches() - launches0
    prof = gb.profile_summary()
    clk = clocks.stop()
    ms = reduce_max_ms(ms, world, "cuda")
    value = args.steps * world / (ms / 1e3)

    # product throughput on one operator (100 Hz), and the block-product roofline
    op = gb.Operator(v, t, w.counts, w.lattice, ks[0])
    info_op = op.info
    x = torch.as_tensor(random_complex_vectors(w.rhs_seed, 1, op.N), device="cuda")
    y = torch.empty_like(x)
    for _ in range(3):
        op.matvec(x, out=y)
    torch.cuda.synchronize()
    gb.profile_reset()
    gb.profile_enable(True)
    nmv = 20
    m0, m1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    m0.record(stream)
    for _ in range(nmv):
        op.matvec(x, out=y)
    m1.record(stream)
    torch.cuda.synchronize()
    gb.profile_enable(False)
    mv_ms = m0.elapsed_time(m1) / nmv
    mv_prof = gb.profile_summary()
    B, F = info_op["B"], info_op["F"]
    spec_bytes = F * B * B * 16
    bp_launches, bp_ms = mv_prof.get("block_product", (nmv, float("nan")))
    bp_bytes = spec_bytes + 2 * F * B * 16           # spectrum once + X in + Y out, per launch
    peaks = measured_peaks()
    hbm_peak = peaks.get("hbm_gbs") or 6800.0
    bp_gbs = bp_bytes / (bp_ms / bp_launches / 1e3) / 1e9

    # e2e through the public API: host mesh in, host pressure out, wall clock
    e2e_steps = max(2, min(args.steps, 4))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    h2d = d2h = 0

    def fetch(i, res):
        nonlocal h2d, d2h
        p, info = res
        ph = p.cpu()
        h2d += v.nbytes + t.nbytes + d.nbytes
        d2h += ph.numel() * 16

    pipe.run(0, e2e_steps, fetch)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    e2e = {"value": e2e_steps * world / e2e_s, "unit": "solves/s", "h2d_bytes_per_step": h2d // e2e_steps,
           "d2h_bytes_per_step": d2h // e2e_steps}

    # dominant kernel of the timed steps
    dom = max(prof.items(), key=lambda kv: kv[1][1])
    total_prof = sum(v_[1] for v_ in prof.values())
    roof = dominant_roofline(dom, prof, w, v, t, args.steps, hbm_peak, peaks, bp_gbs, bp_ms / bp_launches, B, F)

    sections = rank == 0 and not args.only_headline
    fmm = fmm_section(gb, torch, stream) if sections else None
    serving = serving_section(gb) if sections else None
    batching = batching_section(gb, torch, stream) if sections else None
    admittance = admittance_section(gb, torch, stream, w, v, t) if sections else None
    halfspace = halfspace_section(gb, torch, stream) if sections else None
    fmm2 = fmm2_section(gb, torch, stream) if sections else None
    quad9 = _guarded(quad9_section, gb, torch, stream) if sections else None
    c0 = _guarded(config0_section, gb, torch, stream) if sections else None
    config0, p_c0 = (c0 if isinstance(c0, tuple) else (c0, None))
    mixed = (mixed_section(gb, torch, stream, args, w, v, t, sols, ms / args.steps, world, rank)
             if not args.only_headline else None)

    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "ff48 (float-float pairs of FP32, 48-bit significand) with FP64 control", "data": "synthetic",
        "config": config_block(w, {"parallelism": f"replicas{world}" if world > 1 else "single"}),
        "pipeline": ("build of step i+1 overlapped with the solve of step i (second stream and host thread); "
                     "K steps = K builds + K solves" if not args.no_overlap else "steps back to back"),
        "e2e": e2e, "gpu_launches": launches, "clocks": clk, "roofline": roof,
        "matvec": {"value": 1e3 / mv_ms, "unit": "matvecs/s", "ms": mv_ms,
                   "block_product": {"bytes_per_launch": bp_bytes, "ms_per_launch": bp_ms / bp_launches,
                                     "achieved_gbs": bp_gbs, "peak_gbs": hbm_peak,
                                     "frac": bp_gbs / hbm_peak, "peak_source": "measured hbm_gbs" if peaks.get("hbm_gbs") else "fallback"},
                   "kernels_ms_per_matvec": {k_: v_[1] / nmv for k_, v_ in mv_prof.items()}},
        "gmres": {"iters": iters, "relres_true_max": max(relres), "all_converged": all(conv)},
        "kernels_share": {k_: round(v_[1] / total_prof, 4) for k_, v_ in sorted(prof.items(), key=lambda kv: -kv[1][1])},
        "operator": {"form": info_op["form_name"], "B": B, "P": info_op["P"], "F": F,
                     "bytes_device": info_op["bytes_device"]},
        "fmm_workload": fmm,
        "mixed": mixed,
        "serving": serving,
        "batching": batching,
        "admittance": admittance,
        "halfspace": halfspace,
        "fmm2": fmm2,
        "quad9": quad9,
        "config0": config0,
    }
    if rank == 0 and world == 1:
        out["cpu_baseline"] = cpu_baseline(w, v, t, iters_by_freq)
        if p_c0 is not None:
            config0["cpu_baseline"] = _guarded(config0_dense_baseline, p_c0)
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def _guarded(section, *args):
    """Runs a section; an exception is recorded in its place instead of
    ending the run."""
    try:
        return section(*args)
    except Exception as e:  # noqa: BLE001
        return {"error": f"{type(e).__name__}: {e}"}


def _near_pairs(M):
    """Target/source cell pairs of the 3^d near stencil on an M grid."""
    pairs = 0
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (M[2] == 1 and dz) or (M[1] == 1 and dy):
                    continue
                pairs += max(0, M[0] - abs(dx)) * max(0, M[1] - abs(dy)) * max(0, M[2] - abs(dz))
    return pairs


def _tc_rows(m):
    return (2 * m + 127) // 128 * 128


def _tc_depth(k):
    return (2 * k + 63) // 64 * 64


def batching_section(gb, torch, stream, freq_index=3, n_t=12):
    """Batched right-hand sides on the 3-D cube lattice: 16 x 16 x 4 rigid cubes
    (432 triangles each, N = 442,368), FMM form, the 64 spherical-Fibonacci
    incidence directions solved as one 64-RHS GMRES(30) at one frequency of the
    200-1600 Hz sweep (the full workload repeats this for 8 frequencies).

    The batched forms run on the tensor cores: the BF16 operator (near field,
    P2M, L2P and the per-frequency M2L products as BF16 x BF16 -> FP32 tcgen05
    GEMMs) solved to 1e-3, and the MIXED operator (the same BF16 products in
    the inner GMRES, float-float outer residuals) solved to 1e-5.  The FP32 and
    FP64 (float-float) 64-RHS products are timed beside them; a 64-RHS FP64
    solve is not run (about 466 x 0.62 s)."""
    w = WORKLOADS["cube_lattice_16x16x4"]
    v, t = w.mesh()
    k = w.wavenumbers[freq_index]
    ev = lambda: torch.cuda.Event(enable_timing=True)
    R = len(w.directions)
    n = len(t)
    peaks = measured_peaks()

    def build(prec):
        torch.cuda.synchronize()
        b0, b1 = ev(), ev()
        b0.record(stream)
        op = gb.Operator(v, t, w.counts, w.lattice, k, form=gb.FORM_FMM, n_t=n_t, precision=prec)
        b1.record(stream)
        torch.cuda.synchronize()
        return op, b0.elapsed_time(b1)

    def products(op, b, reps):
        y = torch.empty_like(b)
        op.matvec(b, out=y)
        torch.cuda.synchronize()
        gb.profile_reset()
        gb.profile_enable(True)
        m0, m1 = ev(), ev()
        m0.record(stream)
        for _ in range(reps):
            op.matvec(b, out=y)
        m1.record(stream)
        torch.cuda.synchronize()
        gb.profile_enable(False)
        return m0.elapsed_time(m1) / reps, {k_: v_[1] / reps for k_, v_ in gb.profile_summary().items()}, \
            {k_: v_ for k_, v_ in gb.profile_summary().items()}

    def solve(op, b, **kw):
        s0, s1 = ev(), ev()
        torch.cuda.synchronize()
        s0.record(stream)
        p, info = op.solve(b, raise_on_noconv=False, **kw)
        s1.record(stream)
        torch.cuda.synchronize()
        op.check()
        return s0.elapsed_time(s1), p, info

    out = {"workload": f"cube_lattice_16x16x4: N={16 * 16 * 4 * n}, FMM form n_t={n_t}, {R} RHS at "
                       f"{k * SPEED_OF_SOUND / (2 * math.pi):.0f} Hz, GMRES(30)"}
    # BF16 tensor-core operator
    op, build_ms = build(gb.BF16)
    B = op.info["B"]
    b = op.rhs_plane_wave(w.directions)
    mv_ms, kern, raw = products(op, b, 3)
    nc = int(np.prod(w.counts))
    pairs = _near_pairs(w.counts)
    near_alg = 8.0 * pairs * n * n * R                       # complex MACs of the near field x 8
    issued = 2.0 * (_tc_rows(n) * _tc_depth(n) * 27 + _tc_rows(B) * _tc_depth(n) + _tc_rows(n) * _tc_depth(B)) * nc * R
    tc_launches, tc_ms = raw.get("tc_gemm", (3, float("nan")))
    bp_launches, bp_ms = raw.get("tc_block_product", (3, float("nan")))
    F = op.info["F"]
    bp_issued = 2.0 * _tc_rows(B) * _tc_depth(B) * F * max(R, 32)
    s_ms, pb, info = solve(op, b, tol=1e-3, restart=30, maxit=2000)
    bf16_peak = peaks.get("bf16_tflops") or 1900.0
    out["bf16"] = {"build_ms": build_ms, "matvec_64rhs_ms": mv_ms, "rhs_products_per_s": R * 1e3 / mv_ms,
                   "matvec_kernels_ms": kern,
                   "tc_gemm": {"ms_per_matvec": tc_ms / 3, "launches_per_matvec": tc_launches / 3, "issued_tflops":
                               issued / (tc_ms / 3 / 1e3) / 1e12, "near_algorithmic_tflops":
                               near_alg / (tc_ms / 3 / 1e3) / 1e12, "peak_bf16_tflops": bf16_peak,
                               "frac_issued": issued / (tc_ms / 3 / 1e3) / 1e12 / bf16_peak,
                               "peak_source": "measured bf16_tflops" if peaks.get("bf16_tflops") else "fallback"},
                   "tc_block_product": {"ms_per_matvec": bp_ms / 3,
                                        "issued_tflops": bp_issued / (bp_ms / 3 / 1e3) / 1e12,
                                        "spectrum_bytes": 2 * F * _tc_rows(B) * _tc_depth(B)},
                   "solve_tol1e-3": {"ms": s_ms, "solves_per_s_incl_build": R * 1e3 / (s_ms + build_ms),
                                     "iters_max": max(i["iters"] for i in info),
                                     "relres_true_max": max(i["relres_true"] for i in info)},
                   "operator_bytes": op.info["bytes_device"],
                   "tc_tiles_chosen": [{k_: e[k_] for k_ in ("m", "k", "columns", "offsets", "rows_per_cta",
                                                              "columns_per_cta", "ms")}
                                       for e in gb.tuning_summary()
                                       if e.get("kernel") == "tc_gemm" and e["columns"] == nc * R],
                   "dft_plans_chosen": [e for e in gb.tuning_summary() if e.get("kernel") == "dft"]}
    op.close()
    # MIXED: BF16 inner products, float-float outer residuals
    op, build_ms = build(gb.MIXED)
    s_ms, pm, info = solve(op, b, tol=1e-5, restart=30, maxit=3000, inner_tol=1e-2)
    out["mixed"] = {"build_ms": build_ms, "solve_tol1e-5": {
        "ms": s_ms, "solves_per_s_incl_build": R * 1e3 / (s_ms + build_ms),
        "iters_max": max(i["iters"] for i in info), "refinements_max": max(i["refinements"] for i in info),
        "relres_true_max": max(i["relres_true"] for i in info)}, "operator_bytes": op.info["bytes_device"]}
    out["bf16"]["solve_tol1e-3"]["rel_err_vs_mixed_solution"] = float(
        torch.linalg.vector_norm(pb - pm) / torch.linalg.vector_norm(pm))
    op.close()
    # FP32 and FP64 (float-float) products of the same 64 right-hand sides
    for name, prec, reps in (("fp32", gb.FP32, 2), ("fp64", gb.FP64, 1)):
        op, build_ms = build(prec)
        mv_ms, kern, _ = products(op, b, reps)
        out[name] = {"build_ms": build_ms, "matvec_64rhs_ms": mv_ms, "matvec_kernels_ms": kern}
        op.close()
    out["speedup_bf16_product_vs_fp64"] = out["fp64"]["matvec_64rhs_ms"] / out["bf16"]["matvec_64rhs_ms"]
    out["frequency_batch"] = _guarded(frequency_batch, gb, torch, stream, w, v, t, n_t)
    # a smaller case (8 x 8 x 4 cells, 8 directions per frequency), where one
    # operator's products do not fill the GPU on their own
    small = dataclasses.replace(w, counts=(8, 8, 4), directions=w.directions[:8])
    out["frequency_batch_small"] = _guarded(frequency_batch, gb, torch, stream, small, v, t, n_t)
    return out


def frequency_batch(gb, torch, stream, w, v, t, n_t, tol=1e-2, restart=30, maxit=300):
    """The whole batching workload: the workload's frequencies x directions
    (8 x 64 = 512 systems on the 16 x 16 x 4 lattice) with BF16 tensor-core
    operators, solved as one GMRES run per frequency, one after the other, and
    as one fmpb_solve_batch (one product sequence per iteration over the
    operators: near field, P2M, DFT passes, M2L and L2P each one launch;
    operators whose systems have all converged drop out).
    Tolerance 1e-2: BF16 products round their input vectors, which leaves the
    true residual of these systems at 5e-3..3e-2, and tighter tolerances make
    GMRES stagnate at that level for some frequencies."""
    ev = lambda: torch.cuda.Event(enable_timing=True)
    ks = list(w.wavenumbers)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    ops = [gb.Operator(v, t, w.counts, w.lattice, k, form=gb.FORM_FMM, n_t=n_t, precision=gb.BF16) for k in ks]
    torch.cuda.synchronize()
    build_s = time.perf_counter() - t0
    bs = torch.stack([op.rhs_plane_wave(w.directions) for op in ops])
    R = bs.shape[1]
    res = {"grid": list(w.counts), "rhs_per_frequency": R, "systems": len(ops) * R, "frequencies_hz": [round(k * SPEED_OF_SOUND / (2 * math.pi), 1) for k in ks],
           "tol": tol, "restart": restart, "maxit": maxit, "builds_s": build_s}
    # one after the other
    s0, s1 = ev(), ev()
    s0.record(stream)
    seq, seq_info = [], []
    for o, op in enumerate(ops):
        p, info = op.solve(bs[o], tol=tol, restart=restart, maxit=maxit, raise_on_noconv=False)
        seq.append(p)
        seq_info.append(info)
    s1.record(stream)
    torch.cuda.synchronize()
    seq_ms = s0.elapsed_time(s1)
    # the batched products' first launches tune their tile shapes (as the
    # single products' did in the section before): two untimed iterations
    gb.solve_batch(ops, bs, tol=tol, restart=2, maxit=2, raise_on_noconv=False)
    torch.cuda.synchronize()
    # one batched solve
    b0, b1 = ev(), ev()
    b0.record(stream)
    pb, binfo = gb.solve_batch(ops, bs, tol=tol, restart=restart, maxit=maxit, raise_on_noconv=False)
    b1.record(stream)
    torch.cuda.synchronize()
    bat_ms = b0.elapsed_time(b1)
    res["sequential"] = {"ms": seq_ms, "solves_per_s": len(ops) * R * 1e3 / seq_ms,
                         "iters_max_per_frequency": [max(i["iters"] for i in inf) for inf in seq_info],
                         "converged": sum(i["converged"] for inf in seq_info for i in inf)}
    res["batched"] = {"ms": bat_ms, "solves_per_s": len(ops) * R * 1e3 / bat_ms,
                      "iters_max_per_frequency": [max(i["iters"] for i in inf) for inf in binfo],
                      "relres_true_max_per_frequency": [max(i["relres_true"] for i in inf) for inf in binfo],
                      "converged": sum(i["converged"] for inf in binfo for i in inf)}
    res["batched_vs_sequential_rel_diff_per_frequency"] = [
        float(torch.linalg.vector_norm(pb[o] - seq[o]) / torch.linalg.vector_norm(seq[o])) for o in range(len(ops))]
    res["speedup_batched_vs_sequential"] = seq_ms / bat_ms
    res["tc_tiles_chosen_batched"] = [{k_: e[k_] for k_ in ("m", "k", "columns", "offsets", "rows_per_cta",
                                                         "columns_per_cta", "ms")}
                                      for e in gb.tuning_summary() if e.get("kernel") == "tc_gemm" and e.get("batched")]
    for op in ops:
        op.close()
    # each frequency's batched solution against the FP64 (float-float) operator
    res64 = []
    for o, k in enumerate(ks):
        op64 = gb.Operator(v, t, w.counts, w.lattice, k, form=gb.FORM_FMM, n_t=n_t)
        res64.append(float((torch.linalg.vector_norm(op64.matvec(pb[o]) - bs[o], dim=1) /
                            torch.linalg.vector_norm(bs[o], dim=1)).max()))
        op64.close()
    res["batched"]["relres_fp64_operator_max_per_frequency"] = res64
    return res


def run_serving(gb, reqs, precision, snap_hz=None, tol=TOL):
    """Replays requests of the seeded serving stream at their arrival times
    through the serving runtime (both cells; the AUTO form and the library's
    truncation rule, as a caller without tuning would submit them) and
    summarises latency, queueing and service times, cache use and HBM.
    snap_hz: frequencies rounded to this grid (the cache variant)."""
    from workloads import icosphere, capped_cylinder
    cells = {"sphere": icosphere(2, 0.2), "cylinder": capped_cylinder(0.15, 3.0, 20, 29)}
    t0 = time.perf_counter()
    with gb.Server(max_batch_rhs=64, precision=precision, tol=tol, restart=SHORT_RESTART, maxit=MAXIT) as srv:
        tickets = []
        base = reqs[0]["t"]
        for r in reqs:
            delay = (r["t"] - base) - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            k = r["k"]
            if snap_hz:
                f = max(snap_hz, round(r["freq_hz"] / snap_hz) * snap_hz)
                k = 2.0 * math.pi * f / SPEED_OF_SOUND
            v, t = cells[r["cell"]]
            tickets.append(srv.submit(v, t, r["counts"], r["lattice"], k, r["dirs"], form=gb.FORM_AUTO, n_t=0))
        results = [srv.wait(tk)[0] for tk in tickets]
        st = srv.stats()
    wall = time.perf_counter() - t0
    ok = [x for x in results if x["status_name"] == "FMPB_OK"]
    pct = lambda a, q: float(np.percentile(a, q)) if len(a) else None
    queue = [x["queue_ms"] for x in ok]
    service = [x["build_ms"] + x["solve_ms"] for x in ok]
    span = reqs[-1]["t"] - base
    return {"requests": len(reqs), "cells": {c: sum(1 for r in reqs if r["cell"] == c) for c in cells},
            "offered_req_per_s": (len(reqs) - 1) / span if span > 0 else None,
            "achieved_solves_per_s": len(ok) / wall, "wall_s": wall,
            "latency_p50_ms": st["p50_ms"], "latency_p99_ms": st["p99_ms"], "latency_mean_ms": st["mean_ms"],
            "queue_p50_ms": pct(queue, 50), "queue_p99_ms": pct(queue, 99),
            "service_p50_ms": pct(service, 50), "service_p99_ms": pct(service, 99),
            "build_mean_ms": float(np.mean([x["build_ms"] for x in ok])) if ok else None,
            "solve_mean_ms": float(np.mean([x["solve_ms"] for x in ok])) if ok else None,
            "completed": st["completed"], "failed": st["failed"], "batches": st["batches"],
            "cache_hits": st["cache_hits"], "hbm_high_water_bytes": st["hbm_high_water"],
            "iters_max": max((x["iters_max"] for x in results), default=None),
            "relres_true_max": max((x["relres_true_max"] for x in ok), default=None),
            "failures": [dict({k_: x.get(k_) for k_ in ("status_name", "iters_max", "relres_true_max")},
                              cell=r["cell"], counts=list(r["counts"]), freq_hz=round(r["freq_hz"], 1))
                         for r, x in zip(reqs, results) if x["status_name"] != "FMPB_OK"]}


def serving_section(gb, n_sample=24):
    """The serving runtime on the first n_sample sphere-cell requests of the
    seeded stream (Poisson arrivals at 50 req/s, grids 4x4..64x8, 100-2000 Hz,
    1-16 plane waves) at their arrival times, plain FP64 operators, and the
    same requests with MIXED operators (BF16 tensor-core inner products,
    float-float outer residuals, the same 1e-8 tolerance) in "mixed": a bounded
    sample for the default run.  The study with both cells (the capped
    cylinders take the PBEM form with spectra up to 44 GB), plain FP64 beside
    MIXED and the 10 Hz-snapped cache variant is `--serving N`."""
    from workloads import serving_stream
    reqs = [r for r in serving_stream(400) if r["cell"] == "sphere"][:n_sample]
    out = run_serving(gb, reqs, gb.FP64)
    out["sample"] = f"first {n_sample} sphere-cell requests of the seeded 50 req/s stream, FP64"
    out["mixed"] = _guarded(run_serving, gb, reqs, gb.MIXED)
    return out


def run_serving_study(args):
    """`--serving N`: the first N sphere-cell requests of the seeded stream
    replayed three times through the serving runtime at their arrival times:
    plain FP64 operators, MIXED operators (BF16 tensor-core inner products,
    float-float outer residuals, the same 1e-8 tolerance), and FP64 with
    frequencies snapped to a 10 Hz grid (the cache variant); then the first
    12 requests of both cells (the capped cylinders take the PBEM form with
    spectra up to 44 GB) in FP64 and MIXED.  Prints one JSON line."""
    import torch
    import paper_2201_12050_gb300 as gb
    from workloads import serving_stream
    torch.cuda.set_device(0)
    stream = serving_stream(max(4 * args.serving, 24))
    spheres = [r for r in stream if r["cell"] == "sphere"][:args.serving]
    out = {"serving_study": f"first {len(spheres)} sphere-cell requests of the seeded 50 req/s stream",
           "fp64": run_serving(gb, spheres, gb.FP64)}
    out["mixed"] = _guarded(run_serving, gb, spheres, gb.MIXED)
    out["fp64_snapped_10hz"] = _guarded(run_serving, gb, spheres, gb.FP64, 10.0)
    both = stream[:12]
    out["both_cells_first_12"] = {"fp64": _guarded(run_serving, gb, both, gb.FP64),
                                  "mixed": _guarded(run_serving, gb, both, gb.MIXED)}
    print(json.dumps(out))


def mixed_section(gb, torch, stream, args, w, v, t, sols, fp64_ms_per_step, world, rank):
    """The same frequency steps solved at equal accuracy by the plain FP64
    operator and by the FP32-spectrum operator (both to relative residual
    1e-5, about 1e-4 solution error on this crystal), plus the MIXED operator
    (FP32 + float-float spectra, GMRES-IR to the headline 1e-8).  Errors are
    relative L2 against the FP64 solution of the same step at 1e-8 (which is
    itself checked against the FP64 oracle by the parity tests)."""
    ks, d, nf = w.wavenumbers, w.directions, len(w.wavenumbers)
    out = {}
    for name, prec, tol in (("fp64_tol1e-5", gb.FP64, 1e-5), ("fp32_tol1e-5", gb.FP32, 1e-5),
                            ("mixed_ir_tol1e-8", gb.MIXED, TOL)):
        errs, iters, refs = [], [], []
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)

        def make_op(i, prec=prec):
            return gb.Operator(v, t, w.counts, w.lattice, ks[frequency_index(i, world, rank, nf)], precision=prec)

        def solve_op(i, op, tol=tol):
            b = op.rhs_plane_wave(d)
            return op.solve(b, tol=tol, restart=RESTART, maxit=MAXIT, raise_on_noconv=False, inner_tol=1e-4)

        def record(i, res):
            p, info = res
            ref = sols[frequency_index(i, world, rank, nf)]
            errs.append(float(torch.linalg.vector_norm(p - ref) / torch.linalg.vector_norm(ref)))
            iters.append(info[0]["iters"])
            refs.append(info[0]["refinements"])

        pipe = StepPipeline(torch, make_op, solve_op, overlap=not args.no_overlap)
        torch.cuda.synchronize()
        e0.record(stream)
        pipe.run(args.warmup, args.steps, record)
        torch.cuda.synchronize()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / args.steps
        out[name] = {"solves_per_s": world * 1e3 / ms, "ms_per_step": ms, "speedup_vs_fp64": fp64_ms_per_step / ms,
                     "max_rel_err_vs_fp64_solution": max(errs), "iters": iters, "refinements": refs}
    return out


def fmm_section(gb, torch, stream):
    """FMPBEM form on the 32 x 32 sphere array (N = 327,680, n_t = 8, k = 4):
    operator build, product (near field + P2M + circulant M2L + L2P) and a
    plane-wave GMRES solve, each timed with CUDA events, with per-kernel
    times from the library's telemetry."""
    w = WORKLOADS["sphere_array_32x32"]
    v, t = w.mesh()
    k = w.wavenumbers[0]
    ev = lambda: torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    gb.profile_reset()
    gb.profile_enable(True)
    b0, b1 = ev(), ev()
    b0.record(stream)
    op = gb.Operator(v, t, w.counts, w.lattice, k, form=gb.FORM_FMM, n_t=w.n_t)
    b1.record(stream)
    torch.cuda.synchronize()
    gb.profile_enable(False)
    build_ms = b0.elapsed_time(b1)
    build_prof = gb.profile_summary()
    x = torch.as_tensor(random_complex_vectors(w.rhs_seed, 1, op.N), device="cuda")
    y = torch.empty_like(x)
    for _ in range(3):
        op.matvec(x, out=y)
    torch.cuda.synchronize()
    gb.profile_reset()
    gb.profile_enable(True)
    n = 10
    m0, m1 = ev(), ev()
    m0.record(stream)
    for _ in range(n):
        op.matvec(x, out=y)
    m1.record(stream)
    torch.cuda.synchronize()
    gb.profile_enable(False)
    mv_ms = m0.elapsed_time(m1) / n
    prof = gb.profile_summary()
    near_launches, near_ms = prof.get("near_apply", (n, float("nan")))
    near_macs = 0
    M = w.counts
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                near_macs += max(0, M[0] - abs(dx)) * max(0, M[1] - abs(dy)) * max(0, M[2] - abs(dz))
    near_macs *= len(t) * len(t)
    near_tflops = 8.0 * near_macs / (near_ms / near_launches / 1e3) / 1e12
    b = op.rhs_plane_wave(w.directions)
    s0, s1 = ev(), ev()
    s0.record(stream)
    p, info = op.solve(b, tol=TOL, restart=SHORT_RESTART, maxit=MAXIT, raise_on_noconv=False)
    s1.record(stream)
    torch.cuda.synchronize()
    solve_ms = s0.elapsed_time(s1)
    out = {"workload": "sphere_array_32x32: 32x32 rigid spheres r=0.2, lattice 0.6 m, 320 tri/cell, N=327680, "
                       "FMPBEM form n_t=8 (B=81, P=63x63), k=4",
           "build_ms": build_ms, "build_kernels_ms": {k_: v_[1] for k_, v_ in build_prof.items()},
           "matvec_ms": mv_ms, "matvecs_per_s": 1e3 / mv_ms,
           "matvec_kernels_ms": {k_: v_[1] / n for k_, v_ in prof.items()},
           "near_apply": {"complex_macs": near_macs, "fp64_equiv_tflops": near_tflops},
           "solve": {"ms": solve_ms, "iters": info[0]["iters"], "relres_true": info[0]["relres_true"],
                     "solves_per_s_incl_build": 1e3 / (solve_ms + build_ms)},
           "operator_bytes": op.info["bytes_device"]}
    out["precision"] = precision_section(gb, torch, stream, w, v, t, k, op, x, y, p, solve_ms, build_ms)
    op.close()
    return out


def admittance_section(gb, torch, stream, w, v, t, beta=0.4 + 0.2j, freq_index=3):
    """The headline sonic crystal with an absorbing surface of uniform
    normalised admittance beta (Eq. (admittance)) against the rigid one at the
    same frequency: operator build (the quadrature kernels now also integrate
    G and dG/dn_x), the product, and a plane-wave solve to 1e-8."""
    ev = lambda: torch.cuda.Event(enable_timing=True)
    k = w.wavenumbers[freq_index]
    out = {"workload": f"{WORKLOAD} at k = {k:.4f}, beta = {beta}", "beta": [beta.real, beta.imag]}
    x = torch.as_tensor(random_complex_vectors(w.rhs_seed, 1, len(t) * int(np.prod(w.counts))), device="cuda")
    pts = quadrature_points(w, v, t)
    for name, b in (("rigid", 0.0), ("admittance", beta)):
        torch.cuda.synchronize()
        gb.profile_reset()
        gb.profile_enable(True)
        b0, b1 = ev(), ev()
        b0.record(stream)
        op = gb.Operator(v, t, w.counts, w.lattice, k, beta=b)
        b1.record(stream)
        torch.cuda.synchronize()
        gb.profile_enable(False)
        build_ms = b0.elapsed_time(b1)
        bprof = gb.profile_summary()
        y = op.matvec(x)
        torch.cuda.synchronize()
        m0, m1 = ev(), ev()
        m0.record(stream)
        for _ in range(10):
            op.matvec(x, out=y)
        m1.record(stream)
        rhs = op.rhs_plane_wave(w.directions)
        s0, s1 = ev(), ev()
        s0.record(stream)
        p, info = op.solve(rhs, tol=TOL, restart=RESTART, maxit=MAXIT, raise_on_noconv=False)
        s1.record(stream)
        torch.cuda.synchronize()
        quad = "build_blocks_adm" if b else "build_blocks"
        qms = bprof.get(quad, (1, float("nan")))[1]
        out[name] = {"build_ms": build_ms, "build_kernels_ms": {k_: v_[1] for k_, v_ in bprof.items()},
                     "quadrature_points_per_s": pts / (qms / 1e3),
                     "matvec_ms": m0.elapsed_time(m1) / 10, "solve_ms": s0.elapsed_time(s1),
                     "iters": info[0]["iters"], "relres_true": info[0]["relres_true"],
                     "converged": info[0]["converged"],
                     "solves_per_s_incl_build": 1e3 / (build_ms + s0.elapsed_time(s1))}
        op.close()
    r, a = out["rigid"], out["admittance"]
    out["quadrature_kernel_time_ratio"] = (a["build_kernels_ms"].get("build_blocks_adm", float("nan"))
                                           / r["build_kernels_ms"].get("build_blocks", float("nan")))
    return out


def fmm2_section(gb, torch, stream, n_t_near=6):
    """FMPBEM2 (Sec. 3.3) against the single-level FMM form on large unit
    cells: 5 x 10 spheres of 5,120 triangles (N = 256,000, n_t = 8, k = 4).
    The FMM form stores 9 exact near blocks of 5,120 x 5,120; FMPBEM2 keeps
    only the entries of leaf pairs that are not well separated and runs the
    rest of the near field as a multilevel FMM (n_t,near = 6).  Build,
    product, plane-wave solve to 1e-8, device bytes, and the differences of
    the FMPBEM2 product and solution from the FMM form's."""
    w = WORKLOADS["sphere_array_5x10_fine"]
    v, t = w.mesh()
    k = w.wavenumbers[0]
    ev = lambda: torch.cuda.Event(enable_timing=True)
    out = {"workload": w.notes}
    x = torch.as_tensor(random_complex_vectors(w.rhs_seed, 1, len(t) * int(np.prod(w.counts))), device="cuda")
    res = {}
    for name, form in (("fmm", gb.FORM_FMM), ("fmm2", gb.FORM_FMM2)):
        torch.cuda.synchronize()
        gb.profile_reset()
        gb.profile_enable(True)
        b0, b1 = ev(), ev()
        b0.record(stream)
        op = gb.Operator(v, t, w.counts, w.lattice, k, form=form, n_t=w.n_t, n_t_near=n_t_near)
        b1.record(stream)
        torch.cuda.synchronize()
        gb.profile_enable(False)
        build_ms = b0.elapsed_time(b1)
        bprof = gb.profile_summary()
        y = op.matvec(x)
        torch.cuda.synchronize()
        gb.profile_reset()
        gb.profile_enable(True)
        m0, m1 = ev(), ev()
        m0.record(stream)
        for _ in range(5):
            op.matvec(x, out=y)
        m1.record(stream)
        torch.cuda.synchronize()
        gb.profile_enable(False)
        mprof = gb.profile_summary()
        rhs = op.rhs_plane_wave(w.directions)
        s0, s1 = ev(), ev()
        s0.record(stream)
        p, info = op.solve(rhs, tol=TOL, restart=SHORT_RESTART, maxit=MAXIT, raise_on_noconv=False)
        s1.record(stream)
        torch.cuda.synchronize()
        res[name] = (y.clone(), p)
        out[name] = {"build_ms": build_ms, "build_kernels_ms": {k_: v_[1] for k_, v_ in bprof.items()},
                     "matvec_ms": m0.elapsed_time(m1) / 5,
                     "matvec_kernels_ms": {k_: v_[1] / 5 for k_, v_ in mprof.items()},
                     "solve_ms": s0.elapsed_time(s1), "iters": info[0]["iters"],
                     "relres_true": info[0]["relres_true"], "converged": info[0]["converged"],
                     "operator_bytes": op.info["bytes_device"], "near_levels": op.info["near_levels"],
                     "n_m2l_near": op.info["n_m2l_near"], "n_p2p_near": op.info["n_p2p_near"]}
        op.close()
    rel = lambda a, b: float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    out["fmm2_vs_fmm_product_rel_diff"] = rel(res["fmm2"][0], res["fmm"][0])
    out["fmm2_vs_fmm_solution_rel_diff"] = rel(res["fmm2"][1], res["fmm"][1])
    return out


def quad9_section(gb, torch, stream, freq_index=1):
    """The paper's first scattering example on its own element family: 5 x 5
    rigid spheres (r = 0.1 m, lattice 0.35 m), each of 600 nine-node
    quadratic quadrilaterals with one pressure per element (N = 15,000), at
    500 Hz, PBEM form in FP64: operator build (the class-rule point tables,
    the regular entries of the 81 offset blocks, the singular self terms with
    the hypersingular finite part, the FFT), the product, and a plane-wave
    solve to 1e-8."""
    w = WORKLOADS["sphere_array_5x5_q9"]
    nodes, el = w.mesh()
    k = w.wavenumbers[freq_index]
    ev = lambda: torch.cuda.Event(enable_timing=True)
    out = {"workload": w.notes, "k": k, "frequency_hz": k * SPEED_OF_SOUND / (2 * np.pi)}
    torch.cuda.synchronize()
    gb.profile_reset()
    gb.profile_enable(True)
    b0, b1 = ev(), ev()
    b0.record(stream)
    op = gb.Operator(nodes, el, w.counts, w.lattice, k, form=gb.FORM_PBEM)
    b1.record(stream)
    torch.cuda.synchronize()
    gb.profile_enable(False)
    bprof = gb.profile_summary()
    x = torch.as_tensor(random_complex_vectors(w.rhs_seed, 1, op.N), device="cuda")
    y = op.matvec(x)
    torch.cuda.synchronize()
    m0, m1 = ev(), ev()
    m0.record(stream)
    for _ in range(10):
        op.matvec(x, out=y)
    m1.record(stream)
    rhs = op.rhs_plane_wave(w.directions)
    s0, s1 = ev(), ev()
    s0.record(stream)
    p, info = op.solve(rhs, tol=TOL, restart=SHORT_RESTART, maxit=MAXIT, raise_on_noconv=False)
    s1.record(stream)
    torch.cuda.synchronize()
    pts = quad9_points(w, nodes, el)
    qms = sum(bprof.get(name, (0, 0.0))[1] for name in ("q9_blocks", "q9_near"))
    out.update({"element": op.info["element"], "n": op.info["n"], "N": op.N, "form": op.info["form_name"],
                "build_ms": b0.elapsed_time(b1), "build_kernels_ms": {k_: v_[1] for k_, v_ in bprof.items()},
                "regular_quadrature_points": pts, "regular_points_per_s": pts / (qms / 1e3) if qms else None,
                "matvec_ms": m0.elapsed_time(m1) / 10, "solve_ms": s0.elapsed_time(s1),
                "iters": info[0]["iters"], "relres_true": info[0]["relres_true"], "converged": info[0]["converged"],
                "operator_bytes": op.info["bytes_device"]})
    out["solves_per_s_incl_build"] = 1e3 / (out["build_ms"] + out["solve_ms"])
    op.close()
    # the FMM form at the paper's n_t = 4 for this example, and its solution's
    # distance from the PBEM form's
    torch.cuda.synchronize()
    gb.profile_reset()
    gb.profile_enable(True)
    b0, b1 = ev(), ev()
    b0.record(stream)
    opf = gb.Operator(nodes, el, w.counts, w.lattice, k, form=gb.FORM_FMM, n_t=4)
    b1.record(stream)
    torch.cuda.synchronize()
    gb.profile_enable(False)
    fprof = gb.profile_summary()
    yf = opf.matvec(x)
    torch.cuda.synchronize()
    m0, m1 = ev(), ev()
    m0.record(stream)
    for _ in range(10):
        opf.matvec(x, out=yf)
    m1.record(stream)
    s0, s1 = ev(), ev()
    s0.record(stream)
    pf, finfo = opf.solve(opf.rhs_plane_wave(w.directions), tol=TOL, restart=SHORT_RESTART, maxit=MAXIT,
                          raise_on_noconv=False)
    s1.record(stream)
    torch.cuda.synchronize()
    out["fmm_nt4"] = {"build_ms": b0.elapsed_time(b1), "build_kernels_ms": {k_: v_[1] for k_, v_ in fprof.items()},
                      "matvec_ms": m0.elapsed_time(m1) / 10, "solve_ms": s0.elapsed_time(s1),
                      "iters": finfo[0]["iters"], "converged": finfo[0]["converged"],
                      "solution_rel_diff_from_pbem": float(torch.linalg.vector_norm(pf - p)
                                                           / torch.linalg.vector_norm(p)),
                      "operator_bytes": opf.info["bytes_device"]}
    opf.close()
    out["paper_context"] = {"note": "the paper's timings for this example, on its own (CPU) hardware",
                            "pbem_assembly_s": 19.4, "pbem_matvec_s": 0.018,
                            "fmpbem_nt4_assembly_s": 2.4, "fmpbem_nt4_matvec_s": 0.030,
                            "fmpbem_vs_pbem_rel_error_at_500hz": "< 1e-4"}
    return out


def quad9_points(w, nodes, el):
    """Regular quadrature points of one nine-node PBEM build: pairs per class
    (distance to the source centre against its longest corner chord) x rule
    size (16, 64, 256)."""
    Y = np.asarray(nodes, dtype=float)[np.asarray(el)]
    cen = Y[:, 4]
    c = Y[:, [0, 2, 8, 6]]
    h = np.max(np.linalg.norm(c - np.roll(c, 1, axis=1), axis=2), axis=1)
    L = np.asarray(w.lattice, dtype=float)
    total = 0
    M = w.counts
    for dz in range(1 - M[2], M[2]):
        for dy in range(1 - M[1], M[1]):
            for dx in range(1 - M[0], M[0]):
                sh = -(np.array([dx, dy, dz], dtype=float) @ L)
                d = np.linalg.norm(cen[:, None, :] - (cen[None, :, :] + sh), axis=2)
                far = d >= 4.0 * (1 + 1e-9) * h[None, :]
                near = ~far & (d >= 1.5 * (1 + 1e-9) * h[None, :])
                very = ~far & ~near
                if dx == 0 and dy == 0 and dz == 0:
                    very &= ~np.eye(len(el), dtype=bool)
                total += 16 * int(far.sum()) + 64 * int(near.sum()) + 256 * int(very.sum())
    return total


def halfspace_section(gb, torch, stream, freq_indices=(1, 3)):
    """The cylinder sound barrier of the paper's barrier study on a sound-hard
    ground (Sec. 2.3, Sec. 3.4): 3 x 25 x 5 cells, N = 126,000, the image part
    block Hankel along z, two monopoles.  FMM form (n_t = 10) at 200 Hz and at
    the first Bragg frequency 428.75 Hz, with the insertion loss over 3200
    observation points; PBEM form (two spectra, 8 GB) at 200 Hz, and the
    relative difference of the two solutions (the FMM truncation error on
    this workload)."""
    w = WORKLOADS["barrier_cylinders_3x25x5"]
    v, t = w.mesh()
    ev = lambda: torch.cuda.Event(enable_timing=True)
    inc = [("monopole", pos, amp) for pos, amp in w.monopoles]
    out = {"workload": w.notes + "; monopoles " + str(list(w.monopoles))}
    sols = {}
    for form, fi in [("fmm", freq_indices[0]), ("fmm", freq_indices[1]), ("pbem", freq_indices[0])]:
        k = w.wavenumbers[fi]
        torch.cuda.synchronize()
        gb.profile_reset()
        gb.profile_enable(True)
        b0, b1 = ev(), ev()
        b0.record(stream)
        op = gb.Operator(v, t, w.counts, w.lattice, k, form=gb.FORM_FMM if form == "fmm" else gb.FORM_PBEM,
                         n_t=w.n_t, plane=w.plane)
        b1.record(stream)
        torch.cuda.synchronize()
        gb.profile_enable(False)
        build_ms = b0.elapsed_time(b1)
        bprof = gb.profile_summary()
        x = torch.as_tensor(random_complex_vectors(w.rhs_seed, 1, op.N), device="cuda")
        y = op.matvec(x)
        torch.cuda.synchronize()
        gb.profile_reset()
        gb.profile_enable(True)
        m0, m1 = ev(), ev()
        m0.record(stream)
        for _ in range(10):
            op.matvec(x, out=y)
        m1.record(stream)
        torch.cuda.synchronize()
        gb.profile_enable(False)
        mprof = gb.profile_summary()
        rhs = op.rhs_incident(inc)
        s0, s1 = ev(), ev()
        s0.record(stream)
        p, info = op.solve(rhs, tol=TOL, restart=SHORT_RESTART, maxit=MAXIT, raise_on_noconv=False)
        s1.record(stream)
        torch.cuda.synchronize()
        solve_ms = s0.elapsed_time(s1)
        sols[(form, fi)] = p
        il = il_ms = None
        if form == "fmm":
            # Eq. (insertionloss) over 40 x 80 = 3200 points behind the barrier, 1 m above the ground
            gx, gy = np.meshgrid(np.linspace(2.0, 6.0, 40), np.linspace(0.0, 9.6, 80), indexing="ij")
            obs = np.column_stack([gx.ravel(), gy.ravel(), np.full(gx.size, 0.8)])
            i0, i1 = ev(), ev()
            i0.record(stream)
            il = op.insertion_loss(p, inc, obs)
            i1.record(stream)
            torch.cuda.synchronize()
            il_ms = i0.elapsed_time(i1)
        out[f"{form}_{w.wavenumbers[fi] * SPEED_OF_SOUND / (2 * np.pi):.2f}Hz"] = {
            "insertion_loss_db": il, "insertion_loss_ms": il_ms,
            "k": k, "build_ms": build_ms, "build_kernels_ms": {k_: v_[1] for k_, v_ in bprof.items()},
            "matvec_ms": m0.elapsed_time(m1) / 10,
            "matvec_kernels_ms": {k_: v_[1] / 10 for k_, v_ in mprof.items()},
            "solve_ms": solve_ms, "iters": [i["iters"] for i in info],
            "relres_true": [i["relres_true"] for i in info], "converged": all(i["converged"] for i in info),
            "solves_per_s_incl_build": len(inc) * 1e3 / (build_ms + solve_ms),
            "operator_bytes": op.info["bytes_device"], "n_near_image": op.info["n_near_image"]}
        op.close()
    a, b = sols[("fmm", freq_indices[0])], sols[("pbem", freq_indices[0])]
    out["fmm_vs_pbem_solution_rel_diff"] = float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    return out


def precision_section(gb, torch, stream, w, v, t, k, op64, x, y64, p64, fp64_solve_ms, fp64_build_ms):
    """The 32 x 32 sphere array in every precision of the library, against the
    FP64 (float-float) operator, whose products match the FP64 oracle to 1e-12:
    FP32 (near field, P2M, L2P and M2L spectrum in complex FP32), BF16 (all of
    them as BF16 x BF16 -> FP32 tensor-core GEMMs) and MIXED (GMRES-IR: BF16
    inner solves, float-float outer residuals).  Products at 1 and 16
    right-hand sides; solves of the +x plane wave, errors relative (L2) to the
    FP64 solution at 1e-8."""
    ev = lambda: torch.cuda.Event(enable_timing=True)
    rel = lambda a, b: float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))
    x16 = torch.as_tensor(random_complex_vectors(w.rhs_seed + 1, 16, op64.N), device="cuda")
    y16 = op64.matvec(x16)

    def timed(fn, reps):
        fn()
        torch.cuda.synchronize()
        a, c = ev(), ev()
        a.record(stream)
        for _ in range(reps):
            r = fn()
        c.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(c) / reps, r

    out = {"fp64": {"matvec_ms_R1": timed(lambda: op64.matvec(x), 5)[0],
                    "matvec_ms_R16": timed(lambda: op64.matvec(x16), 3)[0],
                    "solve_tol1e-8": {"ms": fp64_solve_ms, "solves_per_s_incl_build":
                                      1e3 / (fp64_solve_ms + fp64_build_ms)}}}
    b = op64.rhs_plane_wave(w.directions)
    for name, prec, tol, inner in (("fp32", gb.FP32, 1e-5, 0.0), ("bf16", gb.BF16, 1e-3, 0.0),
                                   ("mixed", gb.MIXED, 1e-8, 1e-2)):
        torch.cuda.synchronize()
        b0, b1 = ev(), ev()
        b0.record(stream)
        op = gb.Operator(v, t, w.counts, w.lattice, k, form=gb.FORM_FMM, n_t=w.n_t, precision=prec)
        b1.record(stream)
        torch.cuda.synchronize()
        build_ms = b0.elapsed_time(b1)
        r = {"build_ms": build_ms}
        if prec != gb.MIXED:
            ms1, y1 = timed(lambda: op.matvec(x), 5)
            ms16, yy = timed(lambda: op.matvec(x16), 3)
            r.update({"matvec_ms_R1": ms1, "matvec_ms_R16": ms16, "product_rel_err_vs_fp64": max(rel(y1, y64),
                                                                                                   rel(yy, y16))})
        op.solve(b, tol=tol, restart=SHORT_RESTART, maxit=MAXIT, raise_on_noconv=False, inner_tol=inner)
        ms, (p, info) = timed(lambda: op.solve(b, tol=tol, restart=SHORT_RESTART, maxit=MAXIT, raise_on_noconv=False,
                                               inner_tol=inner), 2)
        op.check()
        r[f"solve_tol{tol:.0e}"] = {"ms": ms, "solves_per_s_incl_build": 1e3 / (ms + build_ms),
                                   "iters": info[0]["iters"], "refinements": info[0]["refinements"],
                                   "relres_true": info[0]["relres_true"], "rel_err_vs_fp64_solution": rel(p, p64),
                                   "speedup_vs_fp64_solve": (fp64_solve_ms + fp64_build_ms) / (ms + build_ms)}
        out[name] = r
        op.close()
    return out


QUAD_POINTS = {0: 9, 1: 64, 2: 256}
FLOPS_PER_POINT = 80      # FP64-equivalent operations of one kernel evaluation (D and H at one point)


def quadrature_points(w, v, t):
    """Quadrature points evaluated by one PBEM build: pairs per class x rule size."""
    from workloads.meshes import capped_cylinder  # noqa: F401  (mesh already given)
    verts = np.asarray(v, dtype=float)
    tri = verts[np.asarray(t)]
    cen = tri.mean(axis=1)
    h = np.max(np.linalg.norm(tri - np.roll(tri, 1, axis=1), axis=2), axis=1)
    M = w.counts
    L = np.asarray(w.lattice, dtype=float)
    total = 0
    for dz in range(1 - M[2], M[2]):
        for dy in range(1 - M[1], M[1]):
            for dx in range(1 - M[0], M[0]):
                sh = -np.array([dx, dy, dz], dtype=float) @ L
                dist = np.linalg.norm(cen[:, None, :] - (cen[None, :, :] + sh), axis=2)
                r = dist / h[None, :]
                far = r >= 4.0 * (1 + 1e-9)
                near = (~far) & (r >= 1.5 * (1 + 1e-9))
                vnear = ~(far | near)
                if dx == 0 and dy == 0 and dz == 0:
                    vnear[np.arange(len(t)), np.arange(len(t))] = False
                total += 9 * far.sum() + 64 * near.sum() + 256 * vnear.sum()
    return int(total)


# DRAM bytes per frequency of the float-float block product with B = 1200 and
# one right-hand side, measured with ncu (see dominant_roofline)
BP_TRAFFIC_SHAPE = (1200, 1)
BP_TRAFFIC_PER_FREQUENCY = (1729498624 + 3911424) / 75


def dominant_roofline(dom, prof, w, v, t, steps, hbm_peak, peaks, bp_gbs, bp_ms_per_launch, B=0, F=0):
    name, (launches, total_ms) = dom
    per_launch_s = total_ms / launches / 1e3
    if name == "build_blocks":
        pts = quadrature_points(w, v, t)
        flops = pts * FLOPS_PER_POINT
        achieved = flops / per_launch_s / 1e12
        peak = 1.25      # FP64 FLOP/s of GB300 (nominal table; FMA-chain probe measured 1.2)
        return {"kernel": name, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak, "traffic": None, "launches": launches,
                "ms_per_launch": per_launch_s * 1e3, "work_per_launch": {"quadrature_points": pts,
                                                                         "fp64_flops": flops},
                "peak_source": "nominal FP64 rate (no measured FP64 peak in MEASURED_PEAKS.json)"}
    if name == "block_product":
        # achieved from the product loop on one operator (the timed steps
        # overlap the next build, which shares the SMs with these launches);
        # traffic: DRAM bytes per frequency of k_block_product_ff<1,1> from an
        # ncu capture of `--profile-case product` (B = 1200, one right-hand
        # side, 75 frequencies: 1,729,498,624 read + 3,911,424 written), scaled
        # by the frequencies of a launch (every frequency streams its own block)
        traffic = (BP_TRAFFIC_PER_FREQUENCY * F if (B, len(w.directions)) == BP_TRAFFIC_SHAPE else None)
        return {"kernel": name, "bound": "hbm", "achieved": bp_gbs, "peak": hbm_peak, "unit": "GB/s",
                "frac": bp_gbs / hbm_peak, "traffic": traffic, "launches": launches,
                "ms_per_launch": bp_ms_per_launch, "ms_per_launch_in_timed_steps": per_launch_s * 1e3,
                "peak_source": "measured hbm_gbs"}
    return {"kernel": name, "bound": "unmodelled", "launches": launches, "ms_per_launch": per_launch_s * 1e3,
            "achieved": None, "peak": None, "unit": None, "frac": None, "traffic": None}


# --------------------------------------------------- CPU oracle baseline --
# The oracle as it stands, timed on the host cores in whole units and scaled
# to one solve of the workload:
#   * quadrature rows: every entry of one target row in all 195 offset blocks
#     (oracle.bem.dh_block), rows spread over the cell, split across a
#     spawn-started process pool with one single-threaded worker per core;
#   * one full-size explicit block-Toeplitz product y_c = sum_c' T_{c-c'} p_c'
#     (oracle.bem.toeplitz_matvec) over 195 distinct dense 1200 x 1200 blocks
#     (4.49 GB, streamed from DRAM as a solve would), with the BLAS threads of
#     the host;
#   * seconds per solve = 1200 x seconds per row + (iterations + 2) x seconds
#     per product (the initial residual and the true residual add two), with
#     the GMRES(1000) iteration count of that frequency to 1e-8.
# The blocks of the product are seeded random values of the same shape (an
# exact build of all 195 blocks takes the oracle many minutes on the host);
# the time of a dense product does not depend on the values.

# GMRES(1000) iterations to relative residual 1e-8 of each frequency of the
# sweep (100 ... 1000 Hz), as this bench's solves measure them; an iteration
# count is a property of the linear system and the tolerance, which the
# oracle's GMRES on the same system would need as well.  The GPU arm reports
# its live counts beside its own number.
SWEEP_ITERS = [455, 275, 435, 267, 296, 405, 320, 94, 168, 532]

_ROW_CACHE = {}


def _row_worker(job):
    """Worker of the row pool: the entries of rows `rows` of every offset
    block at wavenumber k.  Returns the worker's own seconds."""
    k, rows = job
    from oracle import bem
    if "cell" not in _ROW_CACHE:
        w = WORKLOADS[WORKLOAD]
        v, t = w.mesh()
        _ROW_CACHE["cell"] = bem.CellMesh(v, t)
        _ROW_CACHE["w"] = w
    cell, w = _ROW_CACHE["cell"], _ROW_CACHE["w"]
    n = cell.n
    rows = np.asarray(rows, dtype=int)

    class Rows:
        centroid = cell.centroid[rows]
        normal = cell.normal[rows]

    Rows.n = len(rows)
    L = np.asarray(w.lattice, dtype=float)
    t0 = time.perf_counter()
    for delta in bem.all_offsets(w.counts):
        shift = -np.asarray(delta, dtype=float) @ L
        selfp = None
        if not any(delta):
            selfp = np.zeros((len(rows), n), dtype=bool)
            selfp[np.arange(len(rows)), rows] = True
        bem.dh_block(Rows, cell.v + shift, k, self_pairs=selfp)
    return time.perf_counter() - t0


def _blas_threads():
    try:
        from threadpoolctl import threadpool_info
        return int(max((i.get("num_threads", 1) for i in threadpool_info()), default=1))
    except Exception:
        return None


class OracleTimer:
    """Times the oracle's units on the host (see above).  The process pool is
    started with spawn, so it is safe after CUDA calls in this process."""

    def __init__(self, w, v, t):
        import multiprocessing as mp
        from oracle import bem
        self.w, self.bem = w, bem
        self.n = len(t)
        self.workers = os.cpu_count() or 1
        old = os.environ.get("OMP_NUM_THREADS")
        os.environ["OMP_NUM_THREADS"] = "1"      # one core per worker
        try:
            self.pool = mp.get_context("spawn").Pool(self.workers)
        finally:
            if old is None:
                del os.environ["OMP_NUM_THREADS"]
            else:
                os.environ["OMP_NUM_THREADS"] = old
        self.pool.map(_row_worker, [(w.wavenumbers[0], [0])] * self.workers)     # imports, mesh
        n = self.n
        rng = np.random.default_rng(w.rhs_seed + 7)
        base = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
        offs = bem.all_offsets(w.counts)
        phase = np.exp(1j * rng.uniform(0, 2 * np.pi, len(offs)))
        self.blocks = {d_: base * phase[i] for i, d_ in enumerate(offs)}     # 195 distinct arrays
        self.x = random_complex_vectors(w.rhs_seed, 1, n * int(np.prod(w.counts)))

    def rows(self, k, n_rows):
        """Wall seconds of n_rows rows (spread over the cell) across the pool."""
        rows = np.linspace(0, self.n - 1, n_rows).astype(int)
        jobs = [(k, rows[i::self.workers].tolist()) for i in range(self.workers) if len(rows[i::self.workers])]
        t0 = time.perf_counter()
        self.pool.map(_row_worker, jobs, chunksize=1)
        return time.perf_counter() - t0

    def product(self):
        t0 = time.perf_counter()
        self.bem.toeplitz_matvec(self.blocks, self.w.counts, self.x)
        return time.perf_counter() - t0

    def step(self, k, iters, n_rows):
        """One sample: n_rows rows and one product.  Returns (sample seconds,
        extrapolated seconds per solve, seconds per row, seconds per product)."""
        tr = self.rows(k, n_rows)
        tp = self.product()
        per_row = tr / n_rows
        return tr + tp, self.n * per_row + (iters + 2) * tp, per_row, tp

    def close(self):
        self.pool.close()
        self.pool.join()

    def cores(self):
        return {"row_workers": self.workers, "blas_threads_product": _blas_threads()}


def _rows_per_sample(workers, minimum=48):
    """Rows per sample: three per worker, at least `minimum` (a run of K
    samples times K times as many rows)."""
    return max(minimum, 3 * workers)


def cpu_baseline(w, v, t, iters_by_freq):
    """The oracle on the host, whole units measured, for the GPU arm's line:
    rows and products timed once per sweep frequency that the GPU ran, with
    that frequency's live iteration count."""
    ot = OracleTimer(w, v, t)
    try:
        n_rows = _rows_per_sample(ot.workers)
        total_sample = total_solve = 0.0
        per_rows, per_mvs = [], []
        for fi, it in sorted(iters_by_freq.items())[:2]:
            s, full, pr, pm = ot.step(w.wavenumbers[fi], it, n_rows)
            total_sample += s
            total_solve += full
            per_rows.append(pr)
            per_mvs.append(pm)
        nfreq = min(2, len(iters_by_freq))
        mean_iters = float(np.mean(list(iters_by_freq.values())))
        sec_per_solve = ot.n * float(np.mean(per_rows)) + (mean_iters + 2) * float(np.mean(per_mvs))
        return {"value": 1.0 / sec_per_solve, "unit": "solves/s", "cores": ot.workers, "kind": "oracle",
                "cores_detail": ot.cores(),
                "sample": f"{nfreq} frequencies x ({n_rows} of 1200 quadrature rows of all 195 offset blocks "
                          f"across {ot.workers} single-threaded processes + 1 full-size explicit block-Toeplitz "
                          f"product over 195 distinct 1200x1200 blocks); per solve = 1200 rows + "
                          f"(mean live GMRES iterations {mean_iters:.1f} + 2) products; sample took "
                          f"{total_sample:.1f} s",
                "seconds_per_quadrature_row": float(np.mean(per_rows)),
                "seconds_per_product": float(np.mean(per_mvs)),
                "seconds_per_solve": sec_per_solve}
    finally:
        ot.close()


def config0_section(gb, torch, stream, reps=20):
    """The 1 x 4 row of rigid spheres (N = 1,280, k = 2, unit plane wave along
    +x; the plain method, i.e. the PBEM form, FP64 class, GMRES to 1e-8):
    operator build + right-hand side + solve on the GPU, timed over `reps`
    repetitions after one untimed run.  Returns the section and the last
    solution (host), which the oracle's dense solve is compared with."""
    w = WORKLOADS["sphere_row_4"]
    v, t = w.mesh()
    k = w.wavenumbers[0]

    def one():
        op = gb.Operator(v, t, w.counts, w.lattice, k, form=gb.FORM_PBEM)
        b = op.rhs_plane_wave(w.directions)
        p, info = op.solve(b, tol=TOL)
        op.close()
        return p, info

    one()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        p, info = one()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / reps
    return {"workload": "sphere_row_4: 1x4 rigid spheres r=0.2 m, lattice 1.0 m, 320 tri/cell, N=1280, k=2, "
                        "plane wave +x, PBEM form, GMRES tol 1e-8",
            "ms_per_solve_incl_build": ms, "solves_per_s": 1e3 / ms, "reps": reps,
            "iters": info[0]["iters"], "relres_true": info[0]["relres_true"]}, p.cpu().numpy()[0]


def config0_dense_baseline(p_gpu):
    """The oracle's whole solve of the same system on the host, measured end
    to end: assembly of the 1,280 x 1,280 collocation matrix (vectorised
    numpy, one process), the right-hand side, and the LAPACK solve (numpy's
    default thread count); plus the relative distance of the GPU solution."""
    from oracle import bem, solve as osolve
    w = WORKLOADS["sphere_row_4"]
    v, t = w.mesh()
    k = w.wavenumbers[0]
    t0 = time.perf_counter()
    A = bem.dense_matrix(v, t, w.lattice, w.counts, k)
    t1 = time.perf_counter()
    b = bem.plane_wave_rhs(bem.CellMesh(v, t), w.lattice, w.counts, k, w.directions[0])
    p = osolve.dense_solve(A, b)
    t2 = time.perf_counter()
    return {"value": 1.0 / (t2 - t0), "unit": "solves/s", "kind": "oracle", "cores": 1,
            "cores_detail": "assembly in one process (vectorised numpy); the LAPACK solve with numpy's default "
                            f"thread count on {os.cpu_count()} host cores",
            "sample": "the whole dense solve of the 1x4 sphere row, measured once",
            "seconds_assembly": t1 - t0, "seconds_rhs_and_solve": t2 - t1, "seconds_total": t2 - t0,
            "gpu_solution_rel_diff": float(np.linalg.norm(p_gpu - p) / np.linalg.norm(p))}


def run_reference(args):
    rank, world, local = dist_env()
    if rank != 0:
        return
    w = WORKLOADS[WORKLOAD]
    v, t = w.mesh()
    ot = OracleTimer(w, v, t)
    n_rows = _rows_per_sample(ot.workers)
    try:
        for i in range(args.warmup):
            ot.rows(w.wavenumbers[i % len(w.wavenumbers)], ot.workers)
        t0 = time.perf_counter()
        tot_solve, per_rows, per_mvs = 0.0, [], []
        for i in range(args.steps):
            fi = i % len(w.wavenumbers)
            _, full, pr, pm = ot.step(w.wavenumbers[fi], SWEEP_ITERS[fi], n_rows)
            tot_solve += full
            per_rows.append(pr)
            per_mvs.append(pm)
        wall = time.perf_counter() - t0
    finally:
        ot.close()
    value = args.steps / tot_solve
    out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": wall / args.steps * 1e3, "higher_is_better": True,
           "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
           "config": config_block(w, {"parallelism": "single"}),
           "pipeline": "oracle on the host cores: whole units timed per step, scaled to one solve "
                       "(see cpu_baseline.sample)",
           "cpu_baseline": {"value": value, "unit": "solves/s", "cores": ot.workers, "kind": "oracle",
                            "cores_detail": ot.cores(),
                            "sample": f"per step (one sweep frequency): {n_rows} of 1200 quadrature rows of all "
                                      f"195 offset blocks across {ot.workers} single-threaded processes + 1 "
                                      f"full-size explicit block-Toeplitz product over 195 distinct 1200x1200 "
                                      f"blocks; value = steps / sum over steps of (1200 x s/row + (GMRES "
                                      f"iterations of that frequency + 2) x s/product); ms_per_step is the "
                                      f"sample's own wall time",
                            "seconds_per_quadrature_row": float(np.mean(per_rows)),
                            "seconds_per_product": float(np.mean(per_mvs)),
                            "seconds_per_solve": tot_solve / args.steps,
                            "iterations_per_frequency": SWEEP_ITERS},
           "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


def run_profile_case(args):
    """Small cases for kernel captures (inputs larger than L2, a few GB at most):
    product/build: 3 x 8 cylinders at 500 Hz (PBEM, spectrum 1.84 GB), one build
    and 4 products; near: the 32 x 32 sphere array (FMM form), one build and 3
    products; batch: 8 x 8 x 4 cubes, BF16 (tensor-core) FMM operator, 3 products
    of 64 right-hand sides (batch_full: the 16 x 16 x 4 lattice, about 4 GB);
    solve_bf16: the 8 x 8 x 4 BF16 operator's 64-RHS solve, 60 iterations on
    the FP32 Krylov basis; barrier: the half-space cylinder barrier (FMM form,
    block Hankel image part), one build and 3 products; fmm2: the 5 x 10 fine
    spheres in the FMPBEM2 form, one build and 3 products; admittance: the 3 x 8
    cylinders at 500 Hz with beta = 0.4 + 0.2i, one build.  Prints one JSON
    line."""
    import torch
    import paper_2201_12050_gb300 as gb
    if args.profile_case == "gmres":
        # full-size crystal at 300 Hz, 320 Arnoldi steps: the basis (up to 370 MB) exceeds L2
        w = WORKLOADS[WORKLOAD]
        v, t = w.mesh()
        op = gb.Operator(v, t, w.counts, w.lattice, w.wavenumbers[2])
        b = op.rhs_plane_wave(w.directions)
        p, info = op.solve(b, tol=TOL, restart=RESTART, maxit=320, raise_on_noconv=False)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "gmres", "N": op.N, "iters": info[0]["iters"],
                          "relres_est": info[0]["relres_est"]}))
        return
    if args.profile_case == "barrier":
        w2 = WORKLOADS["barrier_cylinders_3x25x5"]
        v2, t2 = w2.mesh()
        op = gb.Operator(v2, t2, w2.counts, w2.lattice, w2.wavenumbers[3], n_t=w2.n_t, plane=w2.plane)
        x = torch.as_tensor(random_complex_vectors(w2.rhs_seed, 1, op.N), device="cuda")
        y = torch.empty_like(x)
        for _ in range(3):
            op.matvec(x, out=y)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "barrier", "N": op.N, "form": op.info["form_name"], "B": op.info["B"],
                          "F": op.info["F"], "n_near_image": op.info["n_near_image"],
                          "y_norm": float(torch.linalg.vector_norm(y))}))
        return
    if args.profile_case == "fmm2":
        w2 = WORKLOADS["sphere_array_5x10_fine"]
        v2, t2 = w2.mesh()
        op = gb.Operator(v2, t2, w2.counts, w2.lattice, w2.wavenumbers[0], form=gb.FORM_FMM2, n_t=w2.n_t,
                         n_t_near=6)
        x = torch.as_tensor(random_complex_vectors(w2.rhs_seed, 1, op.N), device="cuda")
        y = torch.empty_like(x)
        for _ in range(3):
            op.matvec(x, out=y)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "fmm2", "N": op.N, "near_levels": op.info["near_levels"],
                          "n_m2l_near": op.info["n_m2l_near"], "n_p2p_near": op.info["n_p2p_near"],
                          "y_norm": float(torch.linalg.vector_norm(y))}))
        return
    if args.profile_case == "admittance":
        w = WORKLOADS[WORKLOAD]
        v, t = w.mesh()
        op = gb.Operator(v, t, (3, 8, 1), w.lattice, 2 * math.pi * 500.0 / SPEED_OF_SOUND, beta=0.4 + 0.2j)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": "admittance", "N": op.N, "F": op.info["F"]}))
        return
    if args.profile_case == "solve_bf16":
        # 8 x 8 x 4 cubes, BF16 operator, 64 right-hand sides, GMRES(30) toward
        # 1e-3 for 60 iterations on the FP32 Krylov basis (1.76 GB)
        w2 = WORKLOADS["cube_lattice_16x16x4"]
        v2, t2 = w2.mesh()
        op = gb.Operator(v2, t2, (8, 8, 4), w2.lattice, w2.wavenumbers[3], form=gb.FORM_FMM, n_t=12,
                         precision=gb.BF16)
        b = op.rhs_plane_wave(w2.directions)
        p, info = op.solve(b, tol=1e-3, restart=30, maxit=60, raise_on_noconv=False)
        print(json.dumps({"profile_case": args.profile_case, "N": op.N, "R": b.shape[0],
                          "iters": max(i["iters"] for i in info)}))
        return
    if args.profile_case in ("near", "batch", "batch_full"):
        if args.profile_case == "near":
            w2 = WORKLOADS["sphere_array_32x32"]
            v2, t2 = w2.mesh()
            op = gb.Operator(v2, t2, w2.counts, w2.lattice, w2.wavenumbers[0], form=gb.FORM_FMM, n_t=w2.n_t)
            x = torch.as_tensor(random_complex_vectors(w2.rhs_seed, 1, op.N), device="cuda")
        else:
            w2 = WORKLOADS["cube_lattice_16x16x4"]
            v2, t2 = w2.mesh()
            counts = w2.counts if args.profile_case == "batch_full" else (8, 8, 4)
            op = gb.Operator(v2, t2, counts, w2.lattice, w2.wavenumbers[3], form=gb.FORM_FMM, n_t=12,
                             precision=gb.BF16)
            x = op.rhs_plane_wave(w2.directions)
        y = torch.empty_like(x)
        for _ in range(3):
            op.matvec(x, out=y)
        torch.cuda.synchronize()
        print(json.dumps({"profile_case": args.profile_case, "N": op.N, "R": x.shape[0], "B": op.info["B"],
                          "F": op.info["F"], "y_norm": float(torch.linalg.vector_norm(y))}))
        return
    w = WORKLOADS[WORKLOAD]
    v, t = w.mesh()
    k = 2 * math.pi * 500.0 / SPEED_OF_SOUND
    t0 = time.perf_counter()
    op = gb.Operator(v, t, (3, 8, 1), w.lattice, k)
    build_s = time.perf_counter() - t0
    x = torch.as_tensor(random_complex_vectors(w.rhs_seed, 1, op.N), device="cuda")
    y = torch.empty_like(x)
    for _ in range(4):
        op.matvec(x, out=y)
    torch.cuda.synchronize()
    print(json.dumps({"profile_case": args.profile_case, "N": op.N, "F": op.info["F"], "B": op.info["B"],
                      "build_s": build_s, "y_norm": float(torch.linalg.vector_norm(y))}))


if __name__ == "__main__":
    a = parse()
    if a.serving:
        run_serving_study(a)
    elif a.profile_case:
        run_profile_case(a)
    elif a.impl == "reference":
        run_reference(a)
    else:
        run_ours(a)
