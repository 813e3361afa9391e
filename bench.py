"""Online solves/s of the method of polarized traces on one GB300 (or N replicas).

A step is one online solve (Algorithm 2: interface right-hand side by local
solves, flexible GMRES to the relative residual 1e-7 with the Gauss-Seidel
sweep preconditioner, volume reconstruction) of one batch of synthetic point
sources with the offline data (local factors, interface Green's matrices)
already resident in HBM.  Prints one JSON line.

The top-level line is the largest workload, layered 1023 x 2047 + 20 PML,
L = 32, 256 sources along the first physical row, in the chosen form
(tensor-core block products, source-batched local solves, FP64 flexible GMRES
with double-float restarts).  Secondary records: the plain FP64 form on the
same workload, the 511 x 1023 GRF workload (mixed, FP64, and both with
partitioned low-rank blocks), the 128 x 128 constant-medium workload (FP64,
tol 1e-10), and an uneven batch of independent problems.  Every record
carries the relative L2 error of its volume field against the CPU oracle's
global sparse direct solve, on sampled sources.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

The CPU oracle runs in a helper process started (spawn) before the first GPU
call: it factors each workload's global operator while the GPU is measured,
solves the sampled sources for the error checks, and after the GPU timings
times the CPU baselines on all host cores.

Multi-GPU: sources are independent right-hand sides, so N ranks run N
replicas (each builds its own offline data and solves its own batch); no
collective is on the data path, the ranks only meet at the timing barriers.
"""
from __future__ import annotations

import argparse
import multiprocessing as mp
import json
import os

# The CPU oracle (helper process, its forked workers, the reference arm) runs one BLAS thread per
# process: its parallelism is one process per core, and unpinned BLAS thread pools in 16 processes
# oversubscribe the host and slow the GPU's host-driven loop measured meanwhile.  Set before numpy
# is first imported (spawned and forked children inherit it).
for _v in ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS"):
    os.environ.setdefault(_v, "1")
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




# ---- inputs -------------------------------------------------------------------
def batch_positions(wl: W.Workload, count: int) -> list:
    """The workload's source positions, repeated (shifted one node right each time) to fill a batch."""
    pos = list(wl.sources)
    out = []
    k = 0
    while len(out) < count:
        p, q = pos[k % len(pos)]
        out.append((min(wl.nx, p + k // len(pos)), q))
        k += 1
    return out


def point_source_tensor(wl: W.Workload, positions, device=None, pin: bool = False):
    """The batch of discrete point sources of ``workloads.point_sources`` built in place in a torch tensor
    (a dense host copy of the 256-source batch would take 9 GB)."""
    import torch

    t = torch.zeros((len(positions), wl.Nz, wl.nt), dtype=torch.complex128, device=device, pin_memory=pin)
    rows, cols, val = W.point_source_entries(wl.npml, wl.h, positions)
    t[torch.arange(len(positions)), torch.as_tensor(rows), torch.as_tensor(cols)] = val
    return t


# ---- the CPU oracle leg (cpu_baseline and the reference fields of the error checks) ----------
# This helper process is the only part of the default run that executes oracle/: it is spawned
# before the first GPU call and never touches CUDA.  Phase 1 (while the GPU is measured): the
# global sparse LU of every requested workload (Section 2.1, the plain definition of the
# discrete solution), the reference fields of the sampled sources, and the offline phase of the
# oracle's polarized-traces solver for CPU leg (i).  Phase 2 (after the GPU timings, on request):
# leg (ii), back-substitutions of a source subset with the global factorization on every host
# core (workers forked from this process share the factors), and leg (i), the oracle's
# polarized-traces online solve (Algorithm 2, one warm-up, median of five).
_HELPER_LU = None


def _backsub_worker(task):
    """Forked from the helper: back-substitute the given sources with the inherited factorization."""
    name, positions = task
    wl = W.WORKLOADS[name]
    f = W.point_sources(wl.nt, wl.Nz, wl.npml, wl.h, positions)
    t0 = time.perf_counter()
    for s in range(len(positions)):
        _HELPER_LU.solve(f[s].reshape(-1))
    return time.perf_counter() - t0


def _oracle_helper(conn, jobs: list, tmpdir: str, backsub: dict, online: dict):
    global _HELPER_LU
    from oracle import discretization as D
    from oracle import solver as S

    pool, lu_keep = None, None
    ncores = os.cpu_count() or 1
    try:
        os.nice(5)  # below the GPU-driving bench process while both run
    except OSError:
        pass
    try:
        for job in jobs:
            wl = W.WORKLOADS[job["workload"]]
            c = wl.c_ext()
            prob = D.make_problem(c, wl.npml, wl.h, wl.omega(c))
            t0 = time.perf_counter()
            lu = S.global_factor(prob)
            t_fact = time.perf_counter() - t0
            pos = job["positions"]
            F = W.point_sources(wl.nt, wl.Nz, wl.npml, wl.h, pos).reshape(len(pos), -1).T.copy()
            t0 = time.perf_counter()
            U = lu.solve(F)
            t_sol = time.perf_counter() - t0
            path = os.path.join(tmpdir, wl.name + ".npy")
            np.save(path, np.ascontiguousarray(U.T).reshape(len(pos), wl.Nz, wl.nt))
            del U, F
            conn.send(("ref", wl.name, path, t_fact, t_sol))
            if backsub and backsub["workload"] == wl.name:
                # workers forked now, before any multi-threaded BLAS call of this process
                _HELPER_LU = lu
                lu_keep = lu
                pool = mp.get_context("fork").Pool(ncores)
                backsub["t_factor"] = t_fact
            del lu
        off = None
        if online:
            wl = W.WORKLOADS[online["workload"]]
            c = wl.c_ext()
            prob = D.make_problem(c, wl.npml, wl.h, wl.omega(c))
            t0 = time.perf_counter()
            off = S.precompute(prob, wl.L)
            online["t_offline"] = time.perf_counter() - t0
        conn.send(("ready",))
        if conn.recv() != "go":
            return
        out = {}
        if pool is not None:
            pos = backsub["positions"]
            chunks = [(backsub["workload"], pos[i::ncores]) for i in range(min(ncores, len(pos)))]
            pool.map(_backsub_worker, [(backsub["workload"], pos[:1])] * len(chunks))  # warm-up
            t0 = time.perf_counter()
            busy = pool.map(_backsub_worker, chunks)
            wall = time.perf_counter() - t0
            out["backsub"] = {"value": len(pos) / wall, "unit": "solves/s", "cores": len(chunks),
                              "host_cores": ncores, "wall_s": wall, "busy_s": sum(busy),
                              "t_factor_s": backsub["t_factor"], "sources": len(pos)}
            pool.close()
            pool.join()
        _HELPER_LU = None
        del lu_keep
        if off is not None:
            wl = W.WORKLOADS[online["workload"]]
            f = wl.f()[0]
            S.online_solve(off, f, tol=wl.tol)
            times, its = [], None
            for _ in range(online.get("repeats", 5)):
                t0 = time.perf_counter()
                r = S.online_solve(off, f, tol=wl.tol)
                times.append(time.perf_counter() - t0)
                its = r.iterations
            med = statistics.median(times)
            out["online"] = {"value": 1.0 / med, "unit": "solves/s", "median_s": med, "repeats": len(times),
                             "gmres_iterations": its, "true_relres": float(r.true_relres),
                             "t_offline_s": online["t_offline"], "host_cores": ncores, "cores": 1,
                             "blas_threads": os.environ.get("OPENBLAS_NUM_THREADS", "library default")}
        conn.send(("timed", out))
    except Exception as exc:  # reported in the bench line, never fatal for the GPU measurement
        conn.send(("error", repr(exc)))


class OracleLeg:
    """Parent side of the helper process."""

    def __init__(self, jobs, backsub=None, online=None):
        import tempfile

        self.tmp = tempfile.mkdtemp(prefix="pt_oracle_")
        self.refs, self.error, self.timed = {}, None, None
        self.ready = False
        ctx = mp.get_context("spawn")
        self.conn, child = ctx.Pipe()
        # not a daemon: it forks the back-substitution workers; close() ends it
        self.proc = ctx.Process(target=_oracle_helper, args=(child, jobs, self.tmp, backsub or {}, online or {}))
        self.proc.start()

    def _pump(self, until):
        while not until():
            if not self.proc.is_alive() and not self.conn.poll():
                self.error = self.error or f"oracle helper exited ({self.proc.exitcode})"
                return
            if not self.conn.poll(1.0):
                continue
            msg = self.conn.recv()
            if msg[0] == "ref":
                self.refs[msg[1]] = {"path": msg[2], "t_factor_s": msg[3], "t_solve_s": msg[4]}
            elif msg[0] == "ready":
                self.ready = True
            elif msg[0] == "timed":
                self.timed = msg[1]
            elif msg[0] == "error":
                self.error = msg[1]
                return

    def ref(self, name):
        """Reference fields (sampled sources, FP64, the global sparse direct solve) of a workload."""
        self._pump(lambda: name in self.refs or self.error is not None)
        if name not in self.refs:
            return None
        return np.load(self.refs[name]["path"], mmap_mode="r")

    def run_timed(self):
        self._pump(lambda: self.ready or self.error is not None)
        if self.error is not None:
            return None
        self.conn.send("go")
        self._pump(lambda: self.timed is not None or self.error is not None)
        return self.timed

    def close(self):
        import shutil

        try:
            if self.proc.is_alive():
                self.conn.send("stop")
        except (BrokenPipeError, OSError):
            pass
        self.proc.join(timeout=10)
        if self.proc.is_alive():
            self.proc.kill()
        shutil.rmtree(self.tmp, ignore_errors=True)


def field_errors(u_gpu: np.ndarray, u_ref: np.ndarray, wl: W.Workload) -> dict:
    """Relative L2 errors of volume fields against the oracle's: over the physical region and over the
    whole extended grid; maxima over the sampled sources."""
    p = wl.npml
    phys, full = [], []
    for a, b in zip(u_gpu, u_ref):
        b = np.asarray(b)
        phys.append(float(np.linalg.norm(a[p:p + wl.nz, p:p + wl.nx] - b[p:p + wl.nz, p:p + wl.nx])
                          / np.linalg.norm(b[p:p + wl.nz, p:p + wl.nx])))
        full.append(float(np.linalg.norm(a - b) / np.linalg.norm(b)))
    return {"max": max(phys), "max_full_grid": max(full), "per_source": phys, "sources": len(phys),
            "norm": "relative L2 over the physical region (PML excluded); max_full_grid over the extended grid",
            "reference": "oracle global sparse LU solve (SuperLU, FP64)"}


# ---- GPU measurement helpers ------------------------------------------------------
def timed_solves(solver, f, u, steps: int, warmup: int, tol: float, dev, pg, stream):
    """W untimed solves, then K solves between CUDA events on the solver's stream, clocks sampled."""
    import torch

    its = rel = None
    for _ in range(warmup):
        _, _, its, rel = solver.solve(f, tol=tol, u=u, want_traces=False)
    barrier(pg)
    torch.cuda.synchronize(dev)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(dev.index) as clk:
        e0.record(stream)
        for _ in range(steps):
            _, _, its, rel = solver.solve(f, tol=tol, u=u, want_traces=False)
        e1.record(stream)
        torch.cuda.synchronize(dev)
    barrier(pg)
    return max_over_ranks(pg, e0.elapsed_time(e1) / steps), its, rel, clk.summary()


def time_apply(solver, which: str, x, stream, reps: int = 5, working: bool = True) -> float:
    """Mean seconds of one pt_apply call (one operator over all sources), CUDA events on the stream."""
    import torch

    for _ in range(2):
        solver.apply(which, x, working=working)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        a.record(stream)
        solver.apply(which, x, working=working)
        b.record(stream)
    torch.cuda.synchronize()
    return statistics.mean(a.elapsed_time(b) for a, b in ev) / 1e3


def gather_fields(u, idx) -> np.ndarray:
    import torch

    return u[torch.as_tensor(idx, device=u.device)].cpu().numpy()


def errors_vs_oracle(oracle, wl, u_host: np.ndarray, ref_idx=None):
    """Field errors of the given sampled fields against the oracle's reference fields of ``wl``."""
    if oracle is None:
        return None
    ref = oracle.ref(wl.name)
    if ref is None:
        return {"unavailable": oracle.error or "no reference"}
    if ref_idx is not None:
        ref = ref[ref_idx]
    return field_errors(u_host, ref, wl)


def make_solver(wl, c, c_dev, prec, S, dev, plr=False, plr_eps=1e-9, plr_rmax=24, max_krylov=40):
    """Offline phase (Algorithm 1) of one form on the GPU; returns (solver, seconds)."""
    import torch

    from paper_1410_5910_gb300 import PolarTrace, default_pml_strength

    t0 = time.perf_counter()
    sv = PolarTrace(wl.nx, wl.nz, wl.npml, wl.L, wl.h, wl.omega(c), c_dev, pml_C=default_pml_strength(float(c.max())),
                    precision=prec, max_sources=S, max_krylov=max_krylov, plr=plr, plr_eps=plr_eps,
                    plr_rmax=plr_rmax)
    torch.cuda.synchronize(dev)
    return sv, time.perf_counter() - t0


ORACLE_SAMPLE = (0, 85, 170, 255)  # sources of the 256-source batch compared with the oracle


def headline_section(args, dev, pg, pk, oracle, world):
    """The chosen form on the largest workload: layered 1023 x 2047, L = 32, 256 sources per step."""
    import torch

    from paper_1410_5910_gb300 import PT_MIXED_TC

    wl = W.WORKLOADS[args.workload]
    S = args.sources
    pos = batch_positions(wl, S)
    c = wl.c_ext()
    c_dev = torch.from_numpy(c).to(dev)
    f = point_source_tensor(wl, pos, device=dev)
    stream = torch.cuda.current_stream(dev)
    tc, t_off = make_solver(wl, c, c_dev, PT_MIXED_TC, S, dev)
    u = torch.empty_like(f)
    ms, its, rel, clocks = timed_solves(tc, f, u, args.steps, args.warmup, wl.tol, dev, pg, stream)
    launches, _ = tc.last_solve_stats()
    cycles, _ = tc.last_solve_cycles()
    vres = tc.volume_residual(f, u)
    sample = [i for i in ORACLE_SAMPLE if i < S]
    err = errors_vs_oracle(oracle, wl, gather_fields(u, sample)) if world == 1 else None
    out = {"value": sum_over_ranks(pg, float(S)) / (ms / 1e3), "ms_per_step": ms, "omega": wl.omega(c),
           "gmres_iterations_max": max(its),
           "gmres_iterations_min": min(its), "restart_cycles": cycles, "true_relres_max": max(rel),
           "volume_residual_max": max(vres), "offline_s": t_off, "launches_per_step": launches, "clocks": clocks,
           "volume_rel_err_vs_oracle": err, "oracle_sample_sources": sample}

    # ---- kernel rooflines, timed live on the solver's stream ----
    nblocks_mv = 16 * (wl.L - 2) + 8
    nblocks_it = 48 * wl.L - 80
    x = torch.randn((S, tc.T4, tc.nt), dtype=torch.complex128, device=dev)
    t_mv = time_apply(tc, "matvec", x, stream)  # three FP16 hi/lo passes, the GMRES matvec
    t_rs = time_apply(tc, "restart", x, stream)  # double-float P M, the explicit residual of a restart
    t_dinv = time_apply(tc, "Dinv", x, stream)   # one FP16 pass, 31 sweep steps
    t_R = time_apply(tc, "R", x, stream)         # one FP16 pass
    # the reconstruction: solves with and without the volume output
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2)]
    t_with, t_without = [], []
    for _ in range(2):
        ev[0][0].record(stream)
        tc.solve(f, tol=wl.tol, u=u, want_traces=False)
        ev[0][1].record(stream)
        ev[1][0].record(stream)
        tc.solve(f, tol=wl.tol, want_u=False, want_traces=False)
        ev[1][1].record(stream)
        torch.cuda.synchronize(dev)
        t_with.append(ev[0][0].elapsed_time(ev[0][1]))
        t_without.append(ev[1][0].elapsed_time(ev[1][1]))
    out["time_split_ms"] = {"matvec_3pass": t_mv * 1e3, "Dinv": t_dinv * 1e3, "R": t_R * 1e3,
                            "restart_product": t_rs * 1e3,
                            "reconstruction": statistics.median(t_with) - statistics.median(t_without),
                            "note": "one call each over all sources; a GMRES iteration is one matvec and n_it = 2 "
                                    "sweeps D^-1 with one R between them"}
    cplx_mv = 8.0 * nblocks_mv * wl.nt * wl.nt * S
    peak_tc = pk.get("bf16_tflops")
    roof_tc = {"kernel": "tc_apply_kernel (tcgen05 FP16 x FP16 -> FP32, GMRES matvec, three hi/lo passes)",
               "bound": "tensor", "achieved": cplx_mv / t_mv / 1e12, "peak": peak_tc, "unit": "TFLOP/s",
               "frac": cplx_mv / t_mv / 1e12 / peak_tc if peak_tc else None, "traffic": None,
               "algorithmic_flops": cplx_mv, "executed_tflops": 3 * cplx_mv / t_mv / 1e12, "launch_ms": t_mv * 1e3,
               "flops_per_unit": "8 n_t^2 real flops per block term and source (one pass of the complex product)",
               "peak_source": "measured bf16 dense burst (FP16 runs at the same rate)"}
    # split products of the restart residual: 15 slice pairs, each a full real-concatenated product
    roof_rs = {"kernel": "oz_apply_kernel (restart residual P M x by split products: five 7-bit FP16 slices per "
                         "operand, 15 slice pairs, exact FP32 accumulation per 512-long K segment)",
               "bound": "tensor", "achieved": 15 * cplx_mv / t_rs / 1e12, "peak": peak_tc, "unit": "TFLOP/s",
               "frac": 15 * cplx_mv / t_rs / 1e12 / peak_tc if peak_tc else None, "traffic": None,
               "launch_ms": t_rs * 1e3, "complex_tflops": cplx_mv / t_rs / 1e12,
               "flops_per_unit": "15 x 8 n_t^2 executed FP16 MMA flops per block term and source",
               "peak_source": "measured bf16 dense burst (FP16 runs at the same rate)"}
    cplx_dinv = 8.0 * (16 * (wl.L - 2) + 8) / 2 * wl.nt * wl.nt * S
    roof_dinv = {"kernel": "tc_apply_kernel, one D^-1 (31 sweep steps, one FP16 pass)", "bound": "tensor",
                 "achieved": cplx_dinv / t_dinv / 1e12, "peak": peak_tc, "unit": "TFLOP/s",
                 "frac": cplx_dinv / t_dinv / 1e12 / peak_tc if peak_tc else None, "launch_ms": t_dinv * 1e3}
    out["roofline_tc_matvec"], out["roofline_restart"], out["roofline_tc_dinv"] = roof_tc, roof_rs, roof_dinv
    out["iteration_flops"] = 8.0 * nblocks_it * wl.nt * wl.nt * S
    del x

    # ---- end to end through the host-buffer entry point (pinned memory, copies inside) ----
    del f
    f_pin = point_source_tensor(wl, pos, pin=True)
    u_pin = torch.empty_like(f_pin).pin_memory()
    scratch = torch.empty(tc.host_scratch_bytes(), dtype=torch.uint8, device=dev)
    tc.solve_host(f_pin, u_pin, tol=wl.tol, scratch=scratch)
    e2e_steps = max(2, args.steps // 4)
    barrier(pg)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        tc.solve_host(f_pin, u_pin, tol=wl.tol, scratch=scratch)
    dt = max_over_ranks(pg, time.perf_counter() - t0)
    out["e2e"] = {"value": sum_over_ranks(pg, float(S)) * e2e_steps / dt, "unit": "solves/s",
                  "h2d_bytes_per_step": int(f_pin.numel() * 16), "d2h_bytes_per_step": int(u_pin.numel() * 16),
                  "steps": e2e_steps}
    del tc, u, scratch, f_pin, u_pin
    torch.cuda.empty_cache()

    # ---- the plain FP64 form on the same workload, one source per solve (the paper's setting) ----
    if not args.no_plain:
        from paper_1410_5910_gb300 import PT_FP64

        p64, t_off64 = make_solver(wl, c, c_dev, PT_FP64, 1, dev)
        f1 = point_source_tensor(wl, pos[:1], device=dev)
        u1 = torch.empty_like(f1)
        ms64, its64, rel64, _ = timed_solves(p64, f1, u1, 3, 2, wl.tol, dev, pg, stream)
        out["plain_fp64"] = {"value": 1e3 / ms64 * world, "unit": "solves/s", "ms_per_solve": ms64,
                             "gmres_iterations": its64, "true_relres": rel64, "offline_s": t_off64,
                             "sources_per_solve": 1,
                             "volume_rel_err_vs_oracle": errors_vs_oracle(oracle, wl, u1.cpu().numpy(), [0])
                             if world == 1 else None}
        del p64, f1, u1
        torch.cuda.empty_cache()
    return out


def grf_section(args, dev, pg, pk, oracle, world):
    """The 511 x 1023 GRF workload, one source (511 x 1023 + 20 PML, L = 16): the mixed form, the plain
    FP64 form and both with partitioned low-rank blocks (Algorithm 5, eps 1e-9 relative, r_max 24)."""
    import torch

    from paper_1410_5910_gb300 import PT_FP64, PT_MIXED_FP32, layer_partition

    wl = W.GRF_511x1023
    c = wl.c_ext()
    c_dev = torch.from_numpy(c).to(dev)
    f = point_source_tensor(wl, wl.sources, device=dev)
    stream = torch.cuda.current_stream(dev)
    steps = max(3, args.steps // 2)
    out = {"workload": wl.name, "sources_per_solve": 1, "tol": wl.tol}
    forms = [("mixed", PT_MIXED_FP32, False), ("plain_fp64", PT_FP64, False)]
    if not args.no_plr:
        forms += [("plr_fp64", PT_FP64, True), ("plr_mixed", PT_MIXED_FP32, True)]
    for name, prec, plr in forms:
        sv, t_off = make_solver(wl, c, c_dev, prec, 1, dev, plr=plr, plr_eps=args.plr_eps, plr_rmax=args.plr_rmax)
        u = torch.empty_like(f)
        ms, its, rel, clocks = timed_solves(sv, f, u, steps, 3, wl.tol, dev, pg, stream)
        launches, _ = sv.last_solve_stats()
        rec = {"value": world * 1e3 / ms, "unit": "solves/s", "ms_per_solve": ms, "gmres_iterations": its,
               "true_relres": rel, "offline_s": t_off, "launches_per_solve": launches, "clocks": clocks,
               "volume_rel_err_vs_oracle": errors_vs_oracle(oracle, wl, u.cpu().numpy()) if world == 1 else None}
        if plr:
            stored, leaves = sv.plr_stats()
            rec["leaves"] = leaves
            rec["compression"] = (16 * (wl.L - 2) + 8) * wl.nt * wl.nt / stored
        nblocks = 16 * (wl.L - 2) + 8
        x = torch.randn((1, sv.T4, sv.nt), dtype=torch.complex128, device=dev)
        if name == "mixed":
            t_df = time_apply(sv, "matvec", x, stream, reps=10)
            alg = nblocks * wl.nt * wl.nt * 16 + 2 * sv.T4 * wl.nt * 16
            rec["roofline_df_matvec"] = {
                "kernel": "apply_lowp_kernel<2> (double-float P M x, with its input conversion)", "bound": "hbm",
                "achieved": alg / t_df / 1e9, "peak": pk.get("hbm_gbs"), "unit": "GB/s",
                "frac": alg / t_df / 1e9 / pk.get("hbm_gbs"), "traffic": None, "algorithmic_bytes": alg,
                "launch_ms": t_df * 1e3,
                "bytes_per_unit": "hi and lo complex64 copies of every block entry (16 B) plus the FP64 in/out vectors"}
            # chunked reconstruction: solves with and without the volume output
            ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(2)]
            t_with, t_without = [], []
            for _ in range(5):
                ev[0][0].record(stream)
                sv.solve(f, tol=wl.tol, u=u, want_traces=False)
                ev[0][1].record(stream)
                ev[1][0].record(stream)
                sv.solve(f, tol=wl.tol, want_u=False, want_traces=False)
                ev[1][1].record(stream)
                torch.cuda.synchronize(dev)
                t_with.append(ev[0][0].elapsed_time(ev[0][1]))
                t_without.append(ev[1][0].elapsed_time(ev[1][1]))
            t_rec = (statistics.median(t_with) - statistics.median(t_without)) / 1e3
            nb = [int(v) for v in np.diff(np.asarray(layer_partition(wl.nx, wl.nz, wl.npml, wl.L)))]
            nloc = [n_ + (wl.npml if l_ > 0 else 0) + (wl.npml if l_ < wl.L - 1 else 0) for l_, n_ in enumerate(nb)]
            sms = torch.cuda.get_device_properties(dev).multi_processor_count
            kv = max(1, min(max(1, min(64, wl.nt // 16)), sms // wl.L))
            alg_rec = (sum(4 * wl.nt * n_ * n_ * 8 for n_ in nloc) + sum(3 * (kv - 1) * n_ * n_ * 8 for n_ in nloc)
                       + sum(8 * wl.nt * n_ * 8 for n_ in nloc) + wl.Nz * wl.nt * 16 + 4 * (wl.L - 1) * wl.nt * 16)
            rec["roofline_reconstruction"] = {
                "kernel": "layer_solve_chunk_kernel<1, 1|3> + chunk_propagate_kernel (FP32 local solves chunked "
                          "along x)", "bound": "hbm", "achieved": alg_rec / t_rec / 1e9, "peak": pk.get("hbm_gbs"),
                "unit": "GB/s", "frac": alg_rec / t_rec / 1e9 / pk.get("hbm_gbs"), "traffic": None,
                "algorithmic_bytes": alg_rec, "launch_ms": t_rec * 1e3, "chunks_per_layer": kv}
        elif name == "plain_fp64":
            t_mv = time_apply(sv, "matvec", x, stream, reps=10, working=False)
            flops = 8.0 * nblocks * wl.nt * wl.nt
            rec["roofline_fp64_matvec"] = {
                "kernel": "apply_kernel<double2> (P M x, FP64 blocks)", "bound": "alu",
                "achieved": flops / t_mv / 1e12, "peak": round(FP64_PEAK_TFLOPS, 3), "unit": "TFLOP/s",
                "frac": flops / t_mv / 1e12 / FP64_PEAK_TFLOPS, "traffic": None, "launch_ms": t_mv * 1e3,
                "achieved_hbm_gbs": nblocks * wl.nt * wl.nt * 16 / t_mv / 1e9,
                "peak_source": "FP64 2 FMA/clk/SM x 152 SMs x 2.07 GHz"}
        elif name.startswith("plr"):
            t_pa = time_apply(sv, "matvec", x, stream, reps=10)
            rec["roofline_plr_matvec"] = {
                "kernel": "plr_project_kernel + plr_expand_kernel (P M x with compressed blocks)", "bound": "hbm",
                "achieved": stored * 16 / t_pa / 1e9, "peak": pk.get("hbm_gbs"),
                "unit": "GB/s", "frac": stored * 16 / t_pa / 1e9 / pk.get("hbm_gbs"),
                "traffic": None, "launch_ms": t_pa * 1e3,
                "bytes_per_unit": "compressed entries of every block (all are in P M) x 16 B: the working matvec keeps FP64 leaves"}
        out[name] = rec
        del sv, u, x
        torch.cuda.empty_cache()
    out["speedup_mixed_vs_plain_fp64"] = out["mixed"]["value"] / out["plain_fp64"]["value"]
    return out


def constant_section(args, dev, pg, oracle, world):
    """128 x 128 + 10 PML, constant medium, L = 4, one centred source, FP64, GMRES tolerance 1e-10."""
    import torch

    from paper_1410_5910_gb300 import PT_FP64

    wl = W.CONSTANT_128
    c = wl.c_ext()
    c_dev = torch.from_numpy(c).to(dev)
    f = point_source_tensor(wl, wl.sources, device=dev)
    sv, t_off = make_solver(wl, c, c_dev, PT_FP64, 1, dev)
    u = torch.empty_like(f)
    ms, its, rel, _ = timed_solves(sv, f, u, max(5, args.steps), 3, wl.tol, dev, pg, torch.cuda.current_stream(dev))
    out = {"workload": wl.name, "form": "plain FP64", "value": world * 1e3 / ms, "unit": "solves/s",
           "ms_per_solve": ms, "gmres_iterations": its, "true_relres": rel, "tol": wl.tol, "offline_s": t_off,
           "volume_rel_err_vs_oracle": errors_vs_oracle(oracle, wl, u.cpu().numpy()) if world == 1 else None}
    del sv
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




# ---- experiments (not part of the default run; one JSON line each) -----------------------------
def _grf_case(nx: int, nz: int, L: int, ppw: float, seed: int = 7) -> W.Workload:
    return W.Workload(f"grf-{nx}x{nz}-L{L}-ppw{ppw:.1f}", nx, nz, 20, L, ppw, "grf", seed, ((nx // 2 + 1, 10),),
                      1e-7)


def experiment_hf_sweep(args, dev):
    """The paper's two frequency regimes (Section 7 tables) on the GRF family: omega ~ n (fixed points per
    wavelength) and omega ~ sqrt(n) (points per wavelength growing like sqrt(n)), n_x x n_z with n_z ~ 4 n_x,
    layered along z.  Per case: GMRES iterations and time per solve and per iteration (mixed form, one source
    near the top, tol 1e-7), FP64 iterations, and the partitioned low-rank storage of the blocks
    (eps = 1e-9 / L, r_max = ceil(sqrt(n_t)), Section 5.1) for the compression-scaling fit."""
    import math

    import torch

    from paper_1410_5910_gb300 import PT_FP64, PT_MIXED_FP32

    sizes = [(127, 511, (8, 16)), (255, 1023, (16, 32)), (511, 2047, (32,))]
    out = []
    stream = torch.cuda.current_stream(dev)
    for regime in ("omega~n", "omega~sqrt(n)"):
        for nx, nz, Ls in sizes:
            ppw = 10.0 if regime == "omega~n" else 10.0 * math.sqrt(nx / 127.0)
            for L in Ls:
                wl = _grf_case(nx, nz, L, ppw)
                c = wl.c_ext()
                c_dev = torch.from_numpy(c).to(dev)
                f = point_source_tensor(wl, wl.sources, device=dev)
                rec = {"regime": regime, "nx": nx, "nz": nz, "N": nx * nz, "L": L, "ppw": ppw, "omega": wl.omega(c)}
                sv, t_off = make_solver(wl, c, c_dev, PT_MIXED_FP32, 1, dev)
                u = torch.empty_like(f)
                ms, its, rel, _ = timed_solves(sv, f, u, 3, 3, wl.tol, dev, None, stream)
                rec.update({"mixed_ms_per_solve": ms, "mixed_iterations": its[0], "mixed_ms_per_iteration": ms / its[0],
                            "true_relres": rel[0], "offline_s": t_off})
                del sv
                rmax = int(math.ceil(math.sqrt(wl.nt)))
                sp, _ = make_solver(wl, c, c_dev, PT_FP64, 1, dev, plr=True, plr_eps=1e-9 / L, plr_rmax=min(31, rmax))
                ms64, its64, _, _ = timed_solves(sp, f, u, 2, 1, wl.tol, dev, None, stream)
                stored, leaves = sp.plr_stats()
                dense = (16 * (L - 2) + 8) * wl.nt * wl.nt
                rec.update({"plr_fp64_iterations": its64[0], "plr_fp64_ms_per_solve": ms64, "plr_stored_entries": stored,
                            "plr_leaves": leaves, "plr_compression": dense / stored, "plr_rmax": min(31, rmax)})
                del sp, f, u, c_dev
                torch.cuda.empty_cache()
                out.append(rec)
                print(json.dumps(rec), flush=True)
    # compression scaling: stored entries of one interior layer's blocks against N, per regime
    fits = {}
    for regime in ("omega~n", "omega~sqrt(n)"):
        pts = [(r["N"], r["plr_stored_entries"] / (16 * (r["L"] - 2) + 8)) for r in out
               if r["regime"] == regime and r["L"] == max(x["L"] for x in out if x["nx"] == r["nx"])]
        if len(pts) >= 2:
            xs, ys = np.log([p[0] for p in pts]), np.log([p[1] for p in pts])
            fits[regime] = float(np.polyfit(xs, ys, 1)[0])
    print(json.dumps({"experiment": "hf-sweep", "cases": len(out), "compression_exponent_per_block_vs_N": fits,
                      "note": "stored entries per block ~ N^p; dense blocks scale as N (n_t^2)"}), flush=True)


def experiment_gs_vs_gmres(args, dev):
    """Gauss-Seidel iteration as the solver (Algorithm 3) against flexible GMRES preconditioned by it
    (Algorithm 4, n_it = 1, 2, 3), FP64 form, on the GRF 511 x 1023 (L = 16) and layered 255 x 511 (L = 8)
    workloads, tol 1e-7: iterations and time per solve (Section 4.2 compares the two)."""
    import torch

    from paper_1410_5910_gb300 import PT_FP64

    stream = torch.cuda.current_stream(dev)
    for wl in (W.GRF_511x1023, W.LAYERED_255x511):
        c = wl.c_ext()
        c_dev = torch.from_numpy(c).to(dev)
        f = point_source_tensor(wl, wl.sources[:1], device=dev)
        rec = {"experiment": "gs-vs-gmres", "workload": wl.name}
        for n_it in (1, 2, 3):
            from paper_1410_5910_gb300 import PolarTrace, default_pml_strength

            sv = PolarTrace(wl.nx, wl.nz, wl.npml, wl.L, wl.h, wl.omega(c), c_dev,
                            pml_C=default_pml_strength(float(c.max())), precision=PT_FP64, gs_iters=n_it)
            u = torch.empty_like(f)
            ms, its, rel, _ = timed_solves(sv, f, u, 3, 2, 1e-7, dev, None, stream)
            rec[f"gmres_n_it{n_it}"] = {"iterations": its[0], "ms_per_solve": ms, "true_relres": rel[0]}
            if n_it == 2:
                for _ in range(2):
                    sv.solve_gs(f, tol=1e-7, max_it=500, allow_not_converged=True)
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                _, _, gits, grel = sv.solve_gs(f, tol=1e-7, max_it=500, allow_not_converged=True)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                rec["gauss_seidel"] = {"iterations": gits[0], "ms_per_solve": e0.elapsed_time(e1),
                                       "true_relres": grel[0], "converged": gits[0] < 500,
                                       "stop": "relative change of the iterate <= 1e-7 (Algorithm 3)"}
            del sv
            torch.cuda.empty_cache()
        print(json.dumps(rec), flush=True)


def top_config(args, world: int, omega: float) -> dict:
    """The ``config`` of the top-level line (both arms)."""
    wl = W.WORKLOADS[args.workload]
    return {"workload": wl.name, "nx": wl.nx, "nz": wl.nz, "npml": wl.npml, "L": wl.L, "medium": wl.medium,
            "omega": omega, "sources_per_step": args.sources, "tol": wl.tol,
            "form": "tensor-core block products (FP16 hi/lo, FP32 accumulation), FP32 source-batched local "
                    "solves, FP64 flexible GMRES with double-float restart residuals",
            "blocks": "dense", "parallelism": f"replicas x{world}",
            "l2": f"interface blocks {16 * wl.L * wl.nt * wl.nt * 16 / 1e9:.1f} GB and their FP16 copies "
                  "stream from HBM each iteration (> 129 MB L2); no flush needed"}


def run_reference(args, rank):
    """--impl reference: the CPU oracle on the top-level workload, on the host cores, rank 0 only.  The
    oracle's plain definition of the solve (the global sparse LU of Section 2.1, factorization excluded
    like the GPU offline phase); a step back-substitutes one source per host core in parallel (workers
    forked from this process, which never touches CUDA, share the factors)."""
    global _HELPER_LU
    if rank != 0:
        return
    from oracle import discretization as D
    from oracle import solver as S

    wl = W.WORKLOADS[args.workload]
    c = wl.c_ext()
    prob = D.make_problem(c, wl.npml, wl.h, wl.omega(c))
    t0 = time.perf_counter()
    _HELPER_LU = S.global_factor(prob)
    t_fact = time.perf_counter() - t0
    ncores = os.cpu_count() or 1
    pos = batch_positions(wl, args.sources)
    per_step = min(ncores, len(pos))
    with mp.get_context("fork").Pool(per_step) as pool:
        def step(k):
            chunk = [(wl.name, [pos[(k * per_step + i) % len(pos)]]) for i in range(per_step)]
            pool.map(_backsub_worker, chunk)

        for k in range(args.warmup):
            step(k)
        t0 = time.perf_counter()
        for k in range(args.steps):
            step(args.warmup + k)
        dt = time.perf_counter() - t0
    value = args.steps * per_step / dt
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": top_config(args, 1, wl.omega(c)), "sample_sources_per_step": per_step,
            "cpu_baseline": {"value": value, "unit": "solves/s", "cores": per_step, "kind": "oracle",
                             "sample": f"{per_step} back-substitutions per step (one per host core, in parallel) "
                                       f"with the global SuperLU factorization of the {wl.name} operator "
                                       f"(factorization {t_fact:.1f} s excluded)"},
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=W.LAYERED_1023x2047.name, choices=sorted(W.WORKLOADS),
                    help="workload of the top-level line (default: the largest one)")
    ap.add_argument("--sources", type=int, default=256, help="sources per step of the top-level workload")
    ap.add_argument("--cpu-sources", type=int, default=16, help="sources of the timed CPU back-substitution leg")
    ap.add_argument("--no-cpu-baseline", action="store_true", help="no oracle helper (no CPU legs, no oracle errors)")
    ap.add_argument("--no-online-leg", action="store_true", help="skip CPU leg (i), the oracle's online solve")
    ap.add_argument("--no-plain", action="store_true", help="skip the plain FP64 form on the top-level workload")
    ap.add_argument("--no-grf", action="store_true", help="skip the 511 x 1023 GRF records")
    ap.add_argument("--no-plr", action="store_true", help="skip the partitioned low-rank records")
    ap.add_argument("--no-constant", action="store_true", help="skip the 128 x 128 constant-medium record")
    ap.add_argument("--plr-eps", type=float, default=1e-9)
    ap.add_argument("--plr-rmax", type=int, default=24)
    ap.add_argument("--no-uneven", action="store_true", help="skip the uneven batch of independent problems")
    ap.add_argument("--uneven-count", type=int, default=16)
    ap.add_argument("--uneven-nmax", type=int, default=511)
    ap.add_argument("--uneven-steps", type=int, default=2)
    ap.add_argument("--experiment", default=None, choices=["hf-sweep", "gs-vs-gmres"],
                    help="run one experiment instead of the benchmark (prints one JSON line per case)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    rank, world, local, pg = dist_setup(args.gpus)
    if args.experiment is not None:
        import torch

        torch.cuda.set_device(local)
        dev = torch.device("cuda", local)
        {"hf-sweep": experiment_hf_sweep, "gs-vs-gmres": experiment_gs_vs_gmres}[args.experiment](args, dev)
        return

    if args.impl == "reference":
        run_reference(args, rank)
        return

    # the oracle helper starts (spawn) before the first GPU call
    oracle = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        top = W.WORKLOADS[args.workload]
        pos = batch_positions(top, args.sources)
        jobs = [{"workload": top.name, "positions": [pos[i] for i in ORACLE_SAMPLE if i < args.sources]}]
        # (a record on the top-level workload compares its first source with the first sampled one)
        if not args.no_grf and top.name != W.GRF_511x1023.name:
            jobs.append({"workload": W.GRF_511x1023.name, "positions": list(W.GRF_511x1023.sources)})
        if not args.no_constant and top.name != W.CONSTANT_128.name:
            jobs.append({"workload": W.CONSTANT_128.name, "positions": list(W.CONSTANT_128.sources)})
        backsub = {"workload": top.name, "positions": pos[:args.cpu_sources]}
        online = None if (args.no_online_leg or args.no_grf) else {"workload": W.GRF_511x1023.name, "repeats": 5}
        oracle = OracleLeg(jobs, backsub, online)

    import torch

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pk, pk_kind = peaks()
    try:
        head = headline_section(args, dev, pg, pk, oracle, world)
        grf = None if args.no_grf else grf_section(args, dev, pg, pk, oracle, world)
        const = None if args.no_constant else constant_section(args, dev, pg, oracle, world)
        uneven = None if args.no_uneven else uneven_section(args, dev, pg)
        timed = oracle.run_timed() if oracle is not None else None
    finally:
        if oracle is not None:
            oracle.close()

    if rank != 0:
        return
    wl = W.WORKLOADS[args.workload]
    cpu = None
    if timed and "backsub" in timed:
        b = timed["backsub"]
        cpu = {"value": b["value"], "unit": "solves/s", "cores": b["cores"], "kind": "oracle",
               "host_cores": b["host_cores"],
               "sample": f"{b['sources']} sources of the {wl.name} batch, back-substituted with the global SuperLU "
                         f"factorization of the same operator, one worker process per core in parallel "
                         f"(factorization {b['t_factor_s']:.1f} s excluded); the oracle's plain definition of the "
                         "solve (Section 2.1)"}
    line = {
        "metric": METRIC, "value": head["value"], "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": head["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64+f32+f16", "data": "synthetic",
        "config": top_config(args, world, head["omega"]),
        "gmres_iterations_max": head["gmres_iterations_max"], "gmres_iterations_min": head["gmres_iterations_min"],
        "true_relres_max": head["true_relres_max"], "restart_cycles": head["restart_cycles"],
        "volume_rel_err_vs_oracle": head["volume_rel_err_vs_oracle"],
        "volume_residual_max": head["volume_residual_max"], "offline_s": head["offline_s"],
        "roofline": head["roofline_tc_matvec"], "roofline_restart": head["roofline_restart"],
        "roofline_tc_dinv": head["roofline_tc_dinv"], "time_split_ms": head["time_split_ms"],
        "peaks_source": pk_kind, "clocks": head["clocks"],
        "e2e": head["e2e"], "gpu_launches": int(head["launches_per_step"] * args.steps), "cpu_baseline": cpu,
    }
    if "plain_fp64" in head:
        line["plain_fp64"] = head["plain_fp64"]
        line["speedup_vs_plain_fp64"] = head["value"] / head["plain_fp64"]["value"]
    if timed and "online" in timed:
        line["cpu_baseline_online"] = dict(timed["online"], kind="oracle", workload=W.GRF_511x1023.name,
                                           sample="the oracle's polarized-traces online solve (Algorithm 2, "
                                                  "flexible GMRES, n_it = 2), one warm-up then the median of "
                                                  "the repeats; its offline phase excluded")
    if oracle is not None and oracle.error:
        line["oracle_error"] = oracle.error
    if oracle is not None:
        line["oracle_reference_timing"] = {k: {"t_factor_s": v["t_factor_s"], "t_solve_s": v["t_solve_s"]}
                                           for k, v in oracle.refs.items()}
    if grf is not None:
        line["grf_511x1023"] = grf
    if const is not None:
        line["constant_128"] = const
    if uneven is not None:
        line["uneven"] = uneven
    print(json.dumps(line), flush=True)


if __name__ == "__main__":
    main()
