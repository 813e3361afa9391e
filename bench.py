"""Online solves/s of the method of polarized traces on one GB300 (or N replicas).

A step is one online solve (Algorithm 2: interface right-hand side by local
solves, flexible GMRES to the relative residual 1e-7 with the Gauss-Seidel
sweep preconditioner, volume reconstruction) of one batch of synthetic point
sources with the offline data (local factors, interface Green's matrices)
already resident in HBM.  Prints one JSON line.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--precision fp64|mixed] [--impl ours|reference]

Multi-GPU: sources are independent right-hand sides, so N ranks run N
replicas (each builds its own offline data and solves its own batch); no
collective is on the data path, the ranks only meet at the timing barriers.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

METRIC = "solves/s at rel. residual 1e-7 (online GMRES), chosen form vs plain FP64, 1 GB300"
PEAKS_FALLBACK = {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}
# FP64 issue rate: 2 FMA per clock per SM (measured with a dependent-free FMA loop),
# 152 SMs, 2070 MHz maximum SM clock, 2 flops per FMA.
FP64_PEAK_TFLOPS = 2 * 152 * 2.070e9 * 2 / 1e12


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        with open(p) as fh:
            d = json.load(fh)
        return d, "measured"
    return PEAKS_FALLBACK, "fallback"


class ClockSampler:
    """nvidia-smi clock / throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, smax, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax = float(parts[2])
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": smax, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_setup(gpus: int):
    """Rank / world from torchrun; gloo for the timing barriers (no data collective)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("gloo")
        pg = dist
    return rank, world, local, pg


def barrier(pg):
    if pg is not None:
        pg.barrier()


def max_over_ranks(pg, v: float) -> float:
    if pg is None:
        return v
    import torch

    t = torch.tensor([v], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.MAX)
    return float(t.item())


def sum_over_ranks(pg, v: float) -> float:
    if pg is None:
        return v
    import torch

    t = torch.tensor([v], dtype=torch.float64)
    pg.all_reduce(t, op=pg.ReduceOp.SUM)
    return float(t.item())


def sources_for(wl: W.Workload, count: int) -> np.ndarray:
    """The workload's sources, repeated (shifted one node right each time) to fill a batch."""
    pos = list(wl.sources)
    out = []
    k = 0
    while len(out) < count:
        p, q = pos[k % len(pos)]
        out.append((min(wl.nx, p + k // len(pos)), q))
        k += 1
    return W.point_sources(wl.nt, wl.Nz, wl.npml, wl.h, out)


def cpu_baseline(wl: W.Workload, sample_solves: int, c: np.ndarray, omega: float):
    """The oracle's plain definition of the solve (global sparse LU, Section 2.1) on the host cores:
    factorization once (excluded, like the GPU offline phase), then back-substitutions timed."""
    from oracle import discretization as D
    from oracle import solver as S

    prob = D.make_problem(c, wl.npml, wl.h, omega)
    t0 = time.perf_counter()
    lu = S.global_factor(prob)
    t_fact = time.perf_counter() - t0
    f = sources_for(wl, sample_solves)
    t0 = time.perf_counter()
    for s in range(sample_solves):
        lu.solve(f[s].reshape(-1))
    dt = time.perf_counter() - t0
    return {"value": sample_solves / dt, "unit": "solves/s", "cores": 1, "kind": "oracle",
            "sample": f"{sample_solves} back-substitutions with the global SuperLU factorization of the same "
                      f"{wl.name} problem (factorization {t_fact:.1f} s excluded; SciPy SuperLU is single-threaded)"}


def batched_section(args, dev, pg, pk):
    """The batched form on the layered 1023 x 2047 workload (L = 32, 256 sources along the
    top row): tensor-core block products (PT_MIXED_TC), source-batched FP32 local solves,
    FP64 flexible GMRES with double-float restarts; against the plain FP64 form solving
    the same sources one at a time."""
    import torch

    from paper_1410_5910_gb300 import PT_FP64, PT_MIXED_TC, PolarTrace, default_pml_strength

    wl = W.LAYERED_1023x2047
    S = args.batched_sources
    c = wl.c_ext()
    om = wl.omega(c)
    pmlC = default_pml_strength(float(c.max()))
    c_dev = torch.from_numpy(c).to(dev)
    f = torch.from_numpy(sources_for(wl, S)).to(dev)
    stream = torch.cuda.current_stream(dev)
    t0 = time.perf_counter()
    tc = PolarTrace(wl.nx, wl.nz, wl.npml, wl.L, wl.h, om, c_dev, pml_C=pmlC, precision=PT_MIXED_TC, max_sources=S,
                    max_krylov=40)
    torch.cuda.synchronize(dev)
    t_off = time.perf_counter() - t0
    u = torch.empty_like(f)
    for _ in range(args.warmup):
        _, _, its, rel = tc.solve(f, tol=wl.tol, u=u, want_traces=False)
    steps = max(2, args.batched_steps)
    barrier(pg)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        e0.record(stream)
        for _ in range(steps):
            _, _, its, rel = tc.solve(f, tol=wl.tol, u=u, want_traces=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    barrier(pg)
    ms = max_over_ranks(pg, e0.elapsed_time(e1) / steps)
    cycles, _ = tc.last_solve_cycles()
    launches, _ = tc.last_solve_stats()
    vres = tc.volume_residual(f, u)
    # tensor-pipe roofline of the three-pass matvec: executed MMA flops / time
    x = torch.randn((S, tc.T4, tc.nt), dtype=torch.complex128, device=dev)
    for _ in range(3):
        tc.apply("matvec", x, working=True)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(5)]
    for a_, b_ in ev:
        a_.record(stream)
        tc.apply("matvec", x, working=True)
        b_.record(stream)
    torch.cuda.synchronize(dev)
    t_mv = statistics.mean(a_.elapsed_time(b_) for a_, b_ in ev) / 1e3
    nblocks = 16 * (wl.L - 2) + 8
    cplx_flops = 8.0 * nblocks * wl.nt * wl.nt * S
    peak = pk.get("bf16_tflops")  # a kernel timed alone: the burst figure
    roof_tc = {"kernel": "tc_apply_kernel (tcgen05 FP16 x FP16 -> FP32, three hi/lo passes)", "bound": "tensor",
               "achieved": 3 * cplx_flops / t_mv / 1e12, "peak": peak, "unit": "TFLOP/s", "frac": None,
               "traffic": None, "complex_tflops": cplx_flops / t_mv / 1e12, "launch_ms": t_mv * 1e3,
               "peak_source": "measured bf16 dense burst (FP16 runs at the same rate)"}
    roof_tc["frac"] = roof_tc["achieved"] / roof_tc["peak"] if peak else None
    del tc, x, u
    torch.cuda.empty_cache()
    out = {"workload": wl.name, "sources_per_step": S, "tol": wl.tol, "value": S / (ms / 1e3),
           "unit": "solves/s", "ms_per_step": ms, "steps": steps, "gmres_iterations_max": max(its),
           "gmres_iterations_min": min(its), "restart_cycles": cycles, "true_relres_max": max(rel),
           "volume_residual_max": max(vres), "offline_s": t_off, "gpu_launches_per_step": launches,
           "clocks": clk.summary(), "roofline_tc_matvec": roof_tc,
           "form": "tensor-core block products (FP16 hi/lo, FP32 accumulation), FP32 source-batched local "
                   "solves, FP64 flexible GMRES with double-float restarts"}
    if not args.no_plain:
        t0 = time.perf_counter()
        p64 = PolarTrace(wl.nx, wl.nz, wl.npml, wl.L, wl.h, om, c_dev, pml_C=pmlC, precision=PT_FP64,
                         max_sources=1, max_krylov=40)
        torch.cuda.synchronize(dev)
        t_off64 = time.perf_counter() - t0
        f1 = f[:1].contiguous()
        u1 = torch.empty_like(f1)
        for _ in range(2):
            p64.solve(f1, tol=wl.tol, u=u1, want_traces=False)
        torch.cuda.synchronize(dev)
        e0.record(stream)
        for _ in range(3):
            _, _, its64, _ = p64.solve(f1, tol=wl.tol, u=u1, want_traces=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        ms64 = e0.elapsed_time(e1) / 3
        out["plain_fp64"] = {"value": 1e3 / ms64, "unit": "solves/s", "ms_per_solve": ms64,
                             "gmres_iterations": its64, "offline_s": t_off64, "sources_per_solve": 1}
        del p64
        torch.cuda.empty_cache()
    return out


def uneven_section(args, dev, pg):
    """Uneven batch: independent problems of the GRF family with different sizes, layer counts and source
    counts (mixed form with FP16 preconditioner blocks: the concurrent instances take the per-step sweeps,
    whose bytes the FP16 copies halve), solved one instance after another and concurrently (pt_solve_many,
    one stream per instance).  Offline phases excluded."""
    import torch

    from paper_1410_5910_gb300 import PT_MIXED_FP32, PT_OPT_PRECOND_FP16, PolarTrace, default_pml_strength, solve_many

    cases = W.uneven_batch(count=args.uneven_count, nmin=255, nmax=args.uneven_nmax, Lmin=8, Lmax=16)
    solvers, fs = [], []
    t0 = time.perf_counter()
    for wl in cases:
        c = wl.c_ext()
        om = wl.omega(c)
        sv = PolarTrace(wl.nx, wl.nz, wl.npml, wl.L, wl.h, om, torch.from_numpy(c).to(dev),
                        pml_C=default_pml_strength(float(c.max())), precision=PT_MIXED_FP32,
                        max_sources=len(wl.sources), max_krylov=40, stream=torch.cuda.Stream(dev))
        sv.set_option(PT_OPT_PRECOND_FP16, 1)
        solvers.append(sv)
        fs.append(torch.from_numpy(wl.f()).to(dev))
    torch.cuda.synchronize(dev)
    t_off = time.perf_counter() - t0
    nsol = sum(f.shape[0] for f in fs)

    def sequential():
        for sv, f in zip(solvers, fs):
            sv.solve(f, tol=1e-7, want_traces=False)
        torch.cuda.synchronize(dev)

    def concurrent():
        return solve_many(solvers, fs, tol=1e-7)

    out = {"instances": len(cases), "sources": nsol, "offline_s": t_off,
           "n_range": [min(w.nx for w in cases), max(w.nx for w in cases)],
           "L_range": [min(w.L for w in cases), max(w.L for w in cases)],
           "form": "mixed with FP16 preconditioner blocks, one stream and one host thread per instance"}
    for name, fn in (("sequential", sequential), ("concurrent", concurrent)):
        fn()
        barrier(pg)
        t0 = time.perf_counter()
        for _ in range(args.uneven_steps):
            r = fn()
        dt = max_over_ranks(pg, (time.perf_counter() - t0) / args.uneven_steps)
        out[name] = {"value": nsol / dt, "unit": "solves/s", "ms_per_batch": dt * 1e3}
        if name == "concurrent":
            out["gmres_iterations_max"] = max(max(i) for i in r[1])
            out["true_relres_max"] = max(max(x) for x in r[2])
    out["value"] = out["concurrent"]["value"]
    del solvers, fs
    torch.cuda.empty_cache()
    return out


def run_reference(args, wl, rank, world, pg):
    """--impl reference: the CPU oracle timed on the host cores, rank 0 only."""
    if rank != 0:
        return
    c = wl.c_ext()
    om = wl.omega(c)
    from oracle import discretization as D
    from oracle import solver as S

    prob = D.make_problem(c, wl.npml, wl.h, om)
    lu = S.global_factor(prob)
    f = sources_for(wl, args.sources)
    for _ in range(args.warmup):
        for s in range(args.sources):
            lu.solve(f[s].reshape(-1))
    t0 = time.perf_counter()
    for _ in range(args.steps):
        for s in range(args.sources):
            lu.solve(f[s].reshape(-1))
    dt = time.perf_counter() - t0
    value = args.steps * args.sources / dt
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": wl.name, "sources_per_step": args.sources},
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": 1, "kind": "oracle",
                             "sample": f"{args.sources} back-substitution(s) per step with the global SuperLU "
                                       "factorization (factorization excluded)"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=W.GRF_511x1023.name, choices=sorted(W.WORKLOADS))
    ap.add_argument("--precision", default="mixed", choices=["fp64", "mixed", "tc"])
    ap.add_argument("--sources", type=int, default=1, help="sources per step (batch)")
    ap.add_argument("--tol", type=float, default=None)
    ap.add_argument("--cpu-sample", type=int, default=20, help="oracle back-substitutions in cpu_baseline")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 comparison")
    ap.add_argument("--no-plr", action="store_true", help="skip the partitioned low-rank variants")
    ap.add_argument("--plr-eps", type=float, default=1e-9)
    ap.add_argument("--plr-rmax", type=int, default=24)
    ap.add_argument("--no-batched", action="store_true", help="skip the batched tensor-core form (256 sources)")
    ap.add_argument("--batched-sources", type=int, default=256)
    ap.add_argument("--batched-steps", type=int, default=3)
    ap.add_argument("--no-uneven", action="store_true", help="skip the uneven batch of independent problems")
    ap.add_argument("--uneven-count", type=int, default=16)
    ap.add_argument("--uneven-nmax", type=int, default=511)
    ap.add_argument("--uneven-steps", type=int, default=2)
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    wl = W.WORKLOADS[args.workload]
    rank, world, local, pg = dist_setup(args.gpus)

    if args.impl == "reference":
        run_reference(args, wl, rank, world, pg)
        return

    import torch

    from paper_1410_5910_gb300 import (PT_FP64, PT_MIXED_FP32, PT_MIXED_TC, PolarTrace, default_pml_strength,
                                       layer_partition)

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    tol = args.tol if args.tol is not None else wl.tol
    c = wl.c_ext()
    om = wl.omega(c)
    pmlC = default_pml_strength(float(c.max()))
    c_dev = torch.from_numpy(c).to(dev)
    S = args.sources
    f_host = sources_for(wl, S)
    f_dev = torch.from_numpy(f_host).to(dev)
    stream = torch.cuda.current_stream(dev)

    def make(prec, plr=False):
        t0 = time.perf_counter()
        s = PolarTrace(wl.nx, wl.nz, wl.npml, wl.L, wl.h, om, c_dev, pml_C=pmlC, precision=prec, max_sources=S,
                       max_krylov=40, plr=plr, plr_eps=args.plr_eps, plr_rmax=args.plr_rmax)
        torch.cuda.synchronize(dev)
        return s, time.perf_counter() - t0

    def time_solves(solver, steps, warmup):
        u = torch.empty_like(f_dev)
        its = None
        for _ in range(warmup):
            _, _, its, rel = solver.solve(f_dev, tol=tol, u=u, want_traces=False)
        barrier(pg)
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            e0.record(stream)
            for _ in range(steps):
                _, _, its, rel = solver.solve(f_dev, tol=tol, u=u, want_traces=False)
            e1.record(stream)
            torch.cuda.synchronize(dev)
        barrier(pg)
        ms = e0.elapsed_time(e1)
        return ms / steps, its, rel, u, clk.summary()

    chosen_prec = {"fp64": PT_FP64, "mixed": PT_MIXED_FP32, "tc": PT_MIXED_TC}[args.precision]
    solver, t_off = make(chosen_prec)
    ms_local, its, rel, u, clocks = time_solves(solver, args.steps, args.warmup)
    launches, _ = solver.last_solve_stats()
    ms = max_over_ranks(pg, ms_local)
    total_solves = sum_over_ranks(pg, float(S))  # per step, all ranks
    value = total_solves / (ms / 1e3)

    # plain FP64 form on the same workload, and the volume difference of the chosen form against it
    extra = {}
    plain = None
    fp64_solver = solver
    if not args.no_plain and chosen_prec != PT_FP64:
        fp64_solver, t_off64 = make(PT_FP64)
        ms64, its64, rel64, u64, _ = time_solves(fp64_solver, max(2, args.steps // 2), 3)
        diff = float(torch.linalg.vector_norm(u - u64) / torch.linalg.vector_norm(u64))
        plain = {"value": total_solves / (max_over_ranks(pg, ms64) / 1e3),
                 "ms_per_step": ms64, "gmres_iterations": its64, "true_relres": rel64, "offline_s": t_off64}
        extra["volume_rel_diff_vs_fp64"] = diff

    # partitioned low-rank blocks (Algorithm 5, eps and r_max of the workload), FP64 and mixed
    plr_results = {}
    if not args.no_plr:
        for name, prec in (("plr_fp64", PT_FP64), ("plr_mixed", PT_MIXED_FP32)):
            ps, t_offp = make(prec, plr=True)
            msp, itsp, relp, up, _ = time_solves(ps, max(2, args.steps // 2), 3)
            stored, leaves = ps.plr_stats()
            dense_entries = (16 * (wl.L - 2) + 8) * wl.nt * wl.nt
            plr_results[name] = {
                "value": total_solves / (max_over_ranks(pg, msp) / 1e3), "ms_per_step": msp,
                "gmres_iterations": itsp, "true_relres": relp, "offline_s": t_offp, "leaves": leaves,
                "compression": dense_entries / stored,
                "volume_rel_diff_vs_chosen": float(torch.linalg.vector_norm(up - u) / torch.linalg.vector_norm(u))}
            del ps
            torch.cuda.empty_cache()

    # ---- roofline of the dominant kernel of the chosen form ----
    pk, pk_kind = peaks()
    L_ = wl.L
    nt = wl.nt
    nb = [int(v) for v in np.diff(np.asarray(layer_partition(wl.nx, wl.nz, wl.npml, L_)))]
    nloc = [n_ + (wl.npml if l_ > 0 else 0) + (wl.npml if l_ < L_ - 1 else 0) for l_, n_ in enumerate(nb)]
    roof_ls = None
    if chosen_prec == PT_MIXED_FP32:
        # (1) the double-float matvec P M x of the GMRES iterations and restart residuals (the largest share
        #     of a solve): one pt_apply call = the input conversion + apply_lowp_kernel<2>, timed live
        nblocks = 16 * (L_ - 2) + 8
        xm = torch.randn((S, solver.T4, solver.nt), dtype=torch.complex128, device=dev)
        for _ in range(3):
            solver.apply("matvec", xm, working=True)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
        for a_, b_ in ev:
            a_.record(stream)
            solver.apply("matvec", xm, working=True)
            b_.record(stream)
        torch.cuda.synchronize(dev)
        t_df = statistics.mean(a_.elapsed_time(b_) for a_, b_ in ev) / 1e3
        # algorithmic bytes: hi and lo complex64 copies of every block entry, the FP64 input and output
        alg_df = nblocks * nt * nt * 16 + 2 * S * solver.T4 * nt * 16
        roof = {"kernel": "apply_lowp_kernel<2> (double-float P M x, with its input conversion)", "bound": "hbm",
                "achieved": alg_df / t_df / 1e9, "peak": pk.get("hbm_gbs"), "unit": "GB/s", "frac": None,
                # DRAM traffic of the same kernel on the 255 x 511, L = 8 layered case (ncu): 1.03 x its
                # algorithmic bytes; it grows with the block bytes, so it is scaled
                "traffic": 1.03 * alg_df, "algorithmic_bytes": alg_df, "launch_ms": t_df * 1e3,
                "traffic_source": "scaled from the ncu capture of the layered-255x511-L8 case"}
        roof["frac"] = roof["achieved"] / roof["peak"]
        # (2) the chunked local solves of the reconstruction (every layer, K_v chunks of n_t / K_v columns,
        #     two passes and the boundary propagation), timed live as the difference of solves with and
        #     without the volume output
        u_tmp = torch.empty_like(f_dev)
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2)]
        t_with, t_without = [], []
        for _ in range(5):
            ev[0][0].record(stream)
            solver.solve(f_dev, tol=tol, u=u_tmp, want_traces=False)
            ev[0][1].record(stream)
            ev[1][0].record(stream)
            solver.solve(f_dev, tol=tol, want_u=False, want_traces=False)
            ev[1][1].record(stream)
            torch.cuda.synchronize(dev)
            t_with.append(ev[0][0].elapsed_time(ev[0][1]))
            t_without.append(ev[1][0].elapsed_time(ev[1][1]))
        t_launch = (statistics.median(t_with) - statistics.median(t_without)) / 1e3
        # chunks per layer as the library chooses them: at least 16 columns, about one CTA per SM
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        kv = max(1, min(max(1, min(64, nt // 16)), sms // L_))
        # algorithmic bytes: Sinv (complex64) of every column read by the forward and the backward
        # substitution of both passes, the transfer matrices of the propagation, couplings, stored
        # iterates, the volume output and the trace forcing
        sinv = sum(4 * nt * n_ * n_ * 8 for n_ in nloc)
        trans = sum(3 * (kv - 1) * n_ * n_ * 8 for n_ in nloc)
        coef = sum(2 * 2 * nt * n_ * 8 for n_ in nloc)
        ystore = sum(2 * 2 * nt * n_ * 8 for n_ in nloc)
        vol = wl.Nz * nt * 16 + 4 * (L_ - 1) * nt * 16
        alg = (sinv + trans + coef + ystore + vol) * S
        steps = 2 * 2 * -(-nt // kv)
        roof_ls = {"kernel": "layer_solve_chunk_kernel<1, 1|3> + chunk_propagate_kernel (FP32 local solves chunked "
                             "along x, reconstruction)", "bound": "hbm", "achieved": alg / t_launch / 1e9,
                   "peak": pk.get("hbm_gbs"), "unit": "GB/s", "frac": None, "traffic": None, "algorithmic_bytes": alg,
                   "launch_ms": t_launch * 1e3, "chunks_per_layer": kv,
                   "latency_bound": f"{steps} dependent column steps in two passes ({kv} chunks per layer) "
                                    f"plus {2 * (kv - 1)} propagation products",
                   "achieved_gflops": 8.0 * sum(n_ * n_ for n_ in nloc) * 2 * 2 * nt * S / t_launch / 1e9}
        roof_ls["frac"] = roof_ls["achieved"] / roof_ls["peak"]
    else:
        roof = None
    # the interface-system matvec with FP64 blocks (the plain form's GEMV), one launch
    x = torch.randn((S, fp64_solver.T4, fp64_solver.nt), dtype=torch.complex128, device=dev)
    for _ in range(3):
        fp64_solver.matvec(x)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(10)]
    for a_, b_ in ev:
        a_.record(stream)
        fp64_solver.matvec(x)
        b_.record(stream)
    torch.cuda.synchronize(dev)
    t_mv = statistics.mean(a_.elapsed_time(b_) for a_, b_ in ev) / 1e3
    nblocks = 16 * (L_ - 2) + 8
    flops = 8.0 * nblocks * nt * nt * S
    roof64 = {"kernel": "apply_kernel<double2> (interface-system matvec P M x, FP64 blocks)", "bound": "alu",
              "achieved": flops / t_mv / 1e12, "peak": round(FP64_PEAK_TFLOPS, 3), "unit": "TFLOP/s",
              "frac": None, "traffic": None, "peak_source": "FP64 2 FMA/clk/SM x 152 SMs x 2.07 GHz",
              "algorithmic_bytes": nblocks * nt * nt * 16 + 2 * 4 * (L_ - 1) * nt * 16 * S,
              "achieved_hbm_gbs": (nblocks * nt * nt * 16) / t_mv / 1e9, "launch_ms": t_mv * 1e3}
    roof64["frac"] = roof64["achieved"] / roof64["peak"]
    if roof is None:
        roof = roof64

    # ---- end to end through the host-buffer entry point (pinned memory) ----
    f_pin = torch.from_numpy(f_host).pin_memory()
    u_pin = torch.empty_like(f_pin).pin_memory()
    scratch = torch.empty(solver.host_scratch_bytes(), dtype=torch.uint8, device=dev)
    for _ in range(2):
        solver.solve_host(f_pin, u_pin, tol=tol, scratch=scratch)
    barrier(pg)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        solver.solve_host(f_pin, u_pin, tol=tol, scratch=scratch)
    dt = max_over_ranks(pg, time.perf_counter() - t0)
    e2e = {"value": total_solves * args.steps / dt, "unit": "solves/s",
           "h2d_bytes_per_step": int(f_pin.numel() * 16), "d2h_bytes_per_step": int(u_pin.numel() * 16)}

    batched = None
    if not args.no_batched:
        del solver, fp64_solver, scratch
        torch.cuda.empty_cache()
        batched = batched_section(args, dev, pg, pk)
    uneven = None
    if not args.no_uneven:
        torch.cuda.empty_cache()
        uneven = uneven_section(args, dev, pg)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(wl, args.cpu_sample, c, om)

    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None,
            "dtype": {PT_FP64: "f64", PT_MIXED_FP32: "f64+f32", PT_MIXED_TC: "f64+f32+f16"}[chosen_prec],
            "data": "synthetic",
            "config": {"workload": wl.name, "nx": wl.nx, "nz": wl.nz, "npml": wl.npml, "L": wl.L,
                       "medium": wl.medium, "omega": om, "sources_per_step": S, "tol": tol,
                       "form": {PT_FP64: "plain FP64", PT_MIXED_FP32: "mixed: FP32 preconditioner, double-float "
                                "matvec and local solves, FP64 FGMRES",
                                PT_MIXED_TC: "tensor-core block products, FP32 batched local solves, FP64 "
                                "FGMRES with double-float restarts"}[chosen_prec],
                       "blocks": "dense", "parallelism": f"replicas x{world}",
                       "l2": f"interface blocks {16 * L_ * nt * nt * 16 / 1e9:.2f} GB stream from HBM each "
                             "iteration (> 129 MB L2); no flush needed"},
            "gmres_iterations": its, "true_relres": rel, "offline_s": t_off,
            "roofline": roof, "roofline_local_solve": roof_ls, "roofline_fp64_matvec": roof64, "peaks_source": pk_kind, "clocks": clocks,
            "e2e": e2e,
            "gpu_launches": int(launches * args.steps), "cpu_baseline": cpu,
        }
        if plain is not None:
            line["plain_fp64"] = plain
        if batched is not None:
            line["batched"] = batched
        if uneven is not None:
            line["uneven"] = uneven
        line.update(plr_results)
        line.update(extra)
        print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
