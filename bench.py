"""Benchmark: shifted solutions/sec to a 1e-8 FP64 residual (mixed + batched
vs plain FP64) on the Wilson-Dirac-style 24^3x32 lattice (5,308,416 unknowns,
10 kappa shifts x 12 Z2 right-hand sides, gauge links stored in bfloat16,
GMRES-DR(80,40) for the first right-hand side, batched GMRES(m_p)-Proj(40)-Sh
for the others), plus the roofline of the dominant kernel and short
measurements of the other workloads (Wilson 8^4 and 16^4, the batch of 64
convection-diffusion problems).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--config C]

One step = one complete multi-shift solve (every shift of every right-hand
side to a true FP64 relative residual <= 1e-8, checked inside the library)
with the operator and right-hand sides resident in HBM.  L2 is flushed
(a 512 MB write) before every timed step.  With N > 1 (torchrun) every rank
solves its own replica of the workload (the solver does not shard); the
value is the aggregate over ranks.  Prints one JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
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

CONFIG_ID = 4
METRIC = "shifted solutions/sec to 1e-8 FP64 residual, mixed+batched vs plain FP64; matvec HBM GB/s"
UNIT = "solutions/s"

# Matvecs of the complete complex128 solve of a workload too large for a complete
# oracle run on the host (first right-hand side, extra right-hand side and Proj
# columns), as counted by the library's FP64 path, which repeats the oracle's
# algorithm cycle for cycle.  Used only to scale the oracle's timed Arnoldi steps
# (bounded samples) to a whole solve.
FP64_SOLVE_MVPS = {3: 2580, 4: 4360}

# DRAM traffic of the dominant kernel from one ncu capture (dram__bytes_read.sum +
# dram__bytes_write.sum over the algorithmic bytes of the same launch), valid for the
# kernel source it was measured on (sha256 prefix of the file); reported as null once
# that file changes.
NCU_TRAFFIC = {"dcgs2_update_c64": {"ratio": 0.996, "sha16": "915cf905142f8a03",
                                    "profile": "dcgs2_update_wilson16x16x16x16"}}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=CONFIG_ID)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-scale", action="store_true", help="skip the large-lattice kernel measurements")
    ap.add_argument("--no-others", action="store_true", help="skip the short runs of the other workloads")
    ap.add_argument("--only-timed", action="store_true",
                    help="only the warm-up and timed mixed solves (no side legs): the launch-list profiling entry "
                         "point; the first timed solve is the NVTX range 'timed_solve'")
    ap.add_argument("--kernels-only", metavar="LATTICE", default=None,
                    help="only the large-lattice kernel measurements of one lattice (16x16x16x16 or 24x24x24x32), "
                         "default launch shapes (no autotuning): the profiling entry point")
    ap.add_argument("--links", choices=["c64", "bf16"], default=None,
                    help="with --kernels-only: link storage (default: the lattice's own)")
    ap.add_argument("--arnoldi-form", choices=["tuned", "launches", "sweep"], default="tuned",
                    help="Arnoldi form of the short-vector cycles: chosen by the autotuner (default), or pinned "
                         "(profiling runs pin the form the plain run chose: serialised launches under ncu "
                         "would bias the tuner)")
    ap.add_argument("--matvec-only", action="store_true",
                    help="with --kernels-only: the matvecs alone (same as --part matvec)")
    ap.add_argument("--part", choices=["all", "arnoldi", "matvec", "projection"], default="all",
                    help="with --kernels-only: only the Arnoldi steps, the matvecs, or the shared-basis projection "
                         "(tensor-core dot and residual update)")
    ap.add_argument("--shape", default=None, metavar="FORM,THREADS,COLINNER",
                    help="with --kernels-only: the multi-column matvec's launch shape (default: the library's)")
    return ap.parse_args()


def max_over_ranks(x, world):
    """Largest value of x over the ranks of the default process group (x itself
    when world == 1): the job's time is its slowest replica's.  The tensor lives
    where the backend needs it (CUDA for NCCL, host for gloo)."""
    if world <= 1:
        return float(x)
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, units_per_replica, seconds_max):
    """Whole-job rate: every rank solves its own replica (weak scaling), so the job
    processes world * units in the slowest rank's time."""
    return world * units_per_replica / seconds_max


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        return {}


# the profiling recipe's stated fallback when no measured peaks are on the box
FALLBACK_HBM_GBS = 6800.0


def hbm_peak():
    """(HBM GB/s denominator, "measured" | "fallback")."""
    v = peaks().get("hbm_gbs")
    return (float(v), "measured") if v else (FALLBACK_HBM_GBS, "fallback")


def workload(cid):
    p = W.config(cid)
    return p, {
        "workload": f"{p.name} Wilson-Dirac-style, n={p.n}, {len(p.sigma)} kappa shifts, "
                    f"{p.B.shape[1]} rhs, GMRES-DR({p.m},{p.k}), m_proj={p.m_proj}",
        "config_id": cid,
        "lattice": "x".join(map(str, p.op[1])) if p.op[0] == "wilson" else None,
        "n": p.n, "ns": len(p.sigma), "nrhs": int(p.B.shape[1]), "m": p.m, "k": p.k, "m_proj": p.m_proj,
        "tol": 1e-8, "prec": "c64 inner + FP64 refinement", "links": p.extra.get("links", "c64"),
        "l2": "flushed before every timed step (512 MB write)",
    }


BATCH_WORKLOAD = "64 convection-diffusion CSR problems, sides 32-256, 4 shifts each, GMRES-DR(30,10), one batched solve"


# ------------------------------------------------------------- clock sampling

class Clocks:
    """nvidia-smi samples during the timed region."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except FileNotFoundError:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------- the oracle (reference arm, CPU baseline)

def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def oracle_operator(p):
    from oracle import CSROperator, WilsonOperator
    if p.op[0] == "wilson":
        return WilsonOperator(p.op[1], p.op[3], p.op[2])
    return CSROperator(*p.op[1:])


def oracle_solve(p, A=None):
    """The oracle (complex128, numpy/scipy) solving every shift of every rhs."""
    from oracle import solve_all_rhs
    A = A or oracle_operator(p)
    t = time.perf_counter()
    out = solve_all_rhs(A.matvec, p.B, p.sigma, p.m, p.k, p.m_proj, p.tol, p.extra_tol, max_mvps=20000)
    return time.perf_counter() - t, out


class ArnoldiSample:
    """A bounded sample of the oracle on a workload too large for a complete run:
    one oracle Arnoldi step (matvec + classical Gram-Schmidt twice) at the average
    basis size m/2 of a GMRES-DR(m, k) cycle, on random orthonormal basis vectors
    of the workload's length.  A whole solve is estimated as that step's time times
    the solve's matvec count (the small dense steps left out)."""

    def __init__(self, p):
        from oracle import arnoldi_cgs2_step
        self.step = arnoldi_cgs2_step
        self.A = oracle_operator(p)
        self.j = p.m // 2
        g = np.random.default_rng(0)
        self.V = np.zeros((p.n, self.j + 2), dtype=np.complex128)
        for q in range(self.j + 1):
            v = g.standard_normal(p.n) + 1j * g.standard_normal(p.n)
            self.V[:, q] = v / np.linalg.norm(v)
        self.H = np.zeros((self.j + 2, self.j + 1), dtype=np.complex128)

    def time_step(self):
        t = time.perf_counter()
        self.step(self.A.matvec, self.V, self.H, self.j)
        return time.perf_counter() - t


def cpu_baseline(p, solve_mvps=None):
    """The oracle on the host cores.  Small workloads (up to 10^5 unknowns x rhs): one
    complete solve.  Larger ones: two timed oracle Arnoldi steps (ArnoldiSample) scaled
    to the matvec count of the whole solve (``solve_mvps``, the FP64 GPU run's, which
    follows the same algorithm)."""
    sols = len(p.sigma) * p.B.shape[1]
    if p.n * p.B.shape[1] <= 100000 or not solve_mvps:
        dt, out = oracle_solve(p)
        return {"value": sols / dt, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                "sample": f"one complete oracle solve of the workload ({sols} shifted solutions, "
                          f"{out['mvps_rhs1']} mvps for rhs 1) in {dt:.2f} s, numpy/BLAS threads = cores"}
    s = ArnoldiSample(p)
    dt = min(s.time_step() for _ in range(2))
    est = dt * solve_mvps
    return {"value": sols / est, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": f"estimated: the oracle's Arnoldi step (matvec + CGS2) at j = {s.j} of GMRES-DR({p.m},{p.k}) "
                      f"took {dt:.2f} s (best of 2), scaled to the {solve_mvps} matvecs of the whole FP64 solve "
                      f"({sols} shifted solutions), numpy/BLAS threads = cores"}


def run_reference(args):
    """The reference arm: the oracle as it stands, on the host cores.  Each step is
    one complete oracle solve where that takes seconds (Wilson 8^4); one oracle
    GMRES-DR-Sh solve of one problem of the batch, in batch order (the batch of 64);
    else one oracle Arnoldi step scaled to the whole solve's matvec count
    (ArnoldiSample, FP64_SOLVE_MVPS)."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.config == 5:
        from oracle import CSROperator, gmres_dr_sh
        probs = W.config(5)
        cfg = {"workload": BATCH_WORKLOAD, "config_id": 5}
        state = {"q": 0}

        def step():
            q = probs[state["q"] % len(probs)]
            state["q"] += 1
            A = CSROperator(*q.op[1:])
            t0 = time.perf_counter()
            gmres_dr_sh(A.matvec, q.B[:, 0], q.sigma, q.m, q.k, 1e-8)
            return time.perf_counter() - t0, len(q.sigma)
        sample = "each step the oracle's GMRES-DR(30,10)-Sh on one problem of the batch, in batch order"
    else:
        p, cfg = workload(args.config)
        sols = len(p.sigma) * p.B.shape[1]
        if p.n * p.B.shape[1] <= 100000:
            A = oracle_operator(p)

            def step():
                return oracle_solve(p, A)[0], sols
            sample = "each step one complete oracle solve of the workload"
        else:
            s = ArnoldiSample(p)
            mv = FP64_SOLVE_MVPS[args.config]

            def step():  # a whole solve estimated from one timed Arnoldi step
                return s.time_step() * mv, sols
            sample = (f"each step one oracle Arnoldi step (matvec + CGS2) at j = {s.j} of GMRES-DR({p.m},{p.k}), "
                      f"its time scaled to the {mv} matvecs of the whole complex128 solve")
    for _ in range(args.warmup):
        step()
    secs, units = 0.0, 0
    for _ in range(args.steps):
        dt, u = step()
        secs += dt
        units += u
    value = units / secs
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": sample + ", numpy/BLAS threads = cores"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def timed_solves(g, ctx, stream, flush, call, steps, warm, check, nvtx=None):
    """warm untimed calls, then `steps` calls each bracketed by CUDA events on the
    library stream after an L2 flush; returns (ms list, last report).  With nvtx,
    the first timed call is the NVTX range of that name (for ncu's --nvtx-include)."""
    import torch
    rep = None
    for _ in range(warm):
        check(*call())
    ms = []
    for q in range(steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        if nvtx and q == 0:
            torch.cuda.nvtx.range_push(nvtx)
        out = call()
        if nvtx and q == 0:
            torch.cuda.nvtx.range_pop()
        e1.record(stream)
        e1.synchronize()
        check(*out)
        rep = out[1]
        ms.append(e0.elapsed_time(e1))
    return ms, rep


def wilson_params(g, p, prec, extra_flags=0):
    if prec == g.GDR_PREC_FP64:  # the plain FP64 solve: complex128, right-hand sides one by one, no graphs
        flags = g.GDR_FLAG_SEQUENTIAL | g.GDR_FLAG_NO_GRAPH | g.GDR_FLAG_AUTOTUNE
    else:
        flags = g.GDR_FLAG_AUTOTUNE
    return g.gdr_params_default(m=p.m, k=p.k, m_proj=p.m_proj, tol=p.tol, extra_tol=p.extra_tol, prec=prec,
                                flags=flags | extra_flags)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.config == 5:
        main_batch(args)
        return
    import torch
    import __graft_entry__
    if args.kernels_only:
        __graft_entry__.build()
        import paper_0707_0502_gb300 as g
        stream = torch.cuda.Stream()
        ctx = g.gdr_create(0, stream)
        part = "matvec" if args.matvec_only else args.part
        shape = tuple(int(v) for v in args.shape.split(",")) if args.shape else None
        out = kernels_at_scale(g, ctx, stream, only=args.kernels_only, link_store=args.links, tune=False,
                               parts=("arnoldi", "matvec", "projection") if part == "all" else (part,), shape=shape)
        print(json.dumps({"kernels_at_scale": out}), flush=True)
        g.gdr_destroy(ctx)
        return
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    __graft_entry__.build()
    import paper_0707_0502_gb300 as g

    p, cfg = workload(args.config)
    ns, nrhs = len(p.sigma), p.B.shape[1]
    sols = ns * nrhs
    stream = torch.cuda.Stream()
    ctx = g.gdr_create(local, stream)
    store = g.GDR_LINK_BF16 if p.extra.get("links") == "bf16" else g.GDR_LINK_C64
    with torch.cuda.stream(stream):
        op = g.make_operator(ctx, p, store=store)
        B = torch.as_tensor(np.ascontiguousarray(p.B.T), device="cuda")
        X = torch.zeros((nrhs, ns, p.n), dtype=torch.complex128, device="cuda")
        flush = torch.empty(512 * 2**20, dtype=torch.uint8, device="cuda")
    stream.synchronize()
    # launch shapes: the first-stage matvec and Arnoldi form tuned here (reported), every
    # other stage's by GDR_FLAG_AUTOTUNE in the first (untimed) warm-up solve of each leg
    tune = g.gdr_autotune(ctx, op, g.GDR_PREC_MIXED, 1, p.m if args.arnoldi_form == "tuned" else 0)
    form_flag = g.GDR_FLAG_NO_SWEEP if args.arnoldi_form == "launches" else 0
    mixed = wilson_params(g, p, g.GDR_PREC_MIXED, form_flag)

    def solve(params, Bx=B, Xx=X):
        st, rep, _ = g.gdr_solve_multishift(ctx, op, p.sigma, Bx, Xx, params)
        return st, rep

    def check(st, rep):
        assert st == g.GDR_OK and rep["max_relres"] <= p.tol, (st, rep)

    # ---- timed region: mixed + batched path
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    ms, rep = timed_solves(g, ctx, stream, flush, lambda: solve(mixed), args.steps, args.warmup, check,
                           nvtx="timed_solve")
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_s = sum(ms) / 1e3
    t_max = max_over_ranks(total_s, world)
    if world > 1:
        dist.barrier()
    value = job_throughput(world, sols * args.steps, t_max)
    launches = rep["kernel_launches"]
    if args.only_timed:
        if rank == 0:
            print(json.dumps({"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
                              "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "config": cfg,
                              "clocks": clk, "gpu_launches": launches * args.steps,
                              "solve": rep, "note": "--only-timed: side legs skipped"}), flush=True)
        g.gdr_destroy(ctx)
        return
    big = p.n * nrhs > 10**7  # one solve takes seconds: fewer repetitions of the side legs

    # ---- plain FP64 GPU path (same algorithm, complex128, rhs sequential, no graphs); its
    #      matvec shape tuned here, so the timed solves need no warm-up
    g.gdr_autotune(ctx, op, g.GDR_PREC_FP64, 1, 0)
    plain = wilson_params(g, p, g.GDR_PREC_FP64)
    ms64, rep64 = timed_solves(g, ctx, stream, flush, lambda: solve(plain), 1 if big else min(args.steps, 5),
                               0 if big else 1, check)
    fp64_value = sols * len(ms64) / (sum(ms64) / 1e3)

    # ---- the mixed solve with every small dense step in FP64 (no FP32 eigensolve or FP32 least squares)
    dense64 = wilson_params(g, p, g.GDR_PREC_MIXED, form_flag | g.GDR_FLAG_FP64_DENSE)
    msd, repd = timed_solves(g, ctx, stream, flush, lambda: solve(dense64), 2 if big else min(args.steps, 5),
                             1, check)

    # ---- end to end through the C ABI with host buffers (copies inside)
    Bh = torch.as_tensor(np.ascontiguousarray(p.B.T)).pin_memory()
    Xh = torch.zeros((nrhs, ns, p.n), dtype=torch.complex128).pin_memory()
    host_params = wilson_params(g, p, g.GDR_PREC_MIXED, form_flag | g.GDR_FLAG_HOST_PTRS)
    e2e_ms = []
    nwarm, nstep = 1, (3 if big else min(args.steps, 5))
    for i in range(nwarm + nstep):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        stream.synchronize()
        t0 = time.perf_counter()
        st, r2, _ = g.gdr_solve_multishift(ctx, op, p.sigma, Bh.numpy(), Xh.numpy(), host_params)
        t1 = time.perf_counter()
        check(st, r2)
        if i >= nwarm:
            e2e_ms.append((t1 - t0) * 1e3)
    e2e_value = job_throughput(world, sols * len(e2e_ms), max_over_ranks(sum(e2e_ms) / 1e3, world))

    # ---- dominant kernel roofline (per-kernel CUDA events on the library stream)
    roof, ktable = kernel_roofline(g, ctx, p, lambda: solve(mixed))
    g.gdr_op_destroy(op)
    del B, X
    torch.cuda.empty_cache()
    scale = kernels_at_scale(g, ctx, stream) if not args.no_scale else None
    others = other_workloads(g, ctx, stream, flush, [c for c in (2, 3, 5) if c != args.config]) \
        if not args.no_others and world == 1 else None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic", "config": cfg,
        "clocks": clk, "gpu_launches": launches * args.steps,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(p.B.nbytes),
                "d2h_bytes_per_step": int(nrhs * ns * p.n * 16)},
        "fp64_plain": {"value": fp64_value, "unit": UNIT, "ms_per_step": sum(ms64) / len(ms64),
                       "steps": len(ms64), "speedup_mixed_over_fp64": value / world / fp64_value,
                       "mvps_total": rep64["mvps_rhs1"] + rep64["mvps_extra"] + rep64["mvps_proj"]},
        "fp64_dense": {"value": sols * len(msd) / (sum(msd) / 1e3), "unit": UNIT,
                       "ms_per_step": sum(msd) / len(msd), "steps": len(msd),
                       "what": "the same mixed solve with the harmonic-Ritz eigensolve and every reduced least "
                               "squares in FP64 (GDR_FLAG_FP64_DENSE)",
                       "t_rhs1_ms": repd["t_rhs1_ms"], "t_proj_ms": repd["t_proj_ms"],
                       "t_refine_ms": repd["t_refine_ms"]},
        "solve": {k: rep[k] for k in ("mvps_rhs1", "cycles_rhs1", "mvps_extra", "mvps_proj", "mvps_refine",
                                      "refine_passes", "pairs_cleaned", "max_relres", "t_total_ms", "t_rhs1_ms",
                                      "t_proj_ms", "t_refine_ms", "host_syncs", "kernel_launches")},
        "roofline": roof,
        "kernels": ktable,
        "autotune": {"stage": "rhs1 matvec (1 column) and Arnoldi form", "arnoldi_form": args.arnoldi_form,
                     **tune},
    }
    if scale is not None:
        line["kernels_at_scale"] = scale
    if others is not None:
        line["other_workloads"] = others
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(p, line["fp64_plain"]["mvps_total"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.gdr_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()


def batch_setup(g, ctx, stream):
    import torch
    probs = W.config(5)
    ntot = sum(q.n for q in probs)
    ns = len(probs[0].sigma)
    with torch.cuda.stream(stream):
        op = g.make_batch_operator(ctx, probs)
        Bh = np.concatenate([q.B[:, 0] for q in probs])
        B = torch.as_tensor(Bh, device="cuda")
        X = torch.zeros(ntot * ns, dtype=torch.complex128, device="cuda")
    stream.synchronize()
    sig = np.stack([q.sigma for q in probs])
    return probs, op, Bh, B, X, sig


def batch_params(g, p0, prec, extra=0):
    flags = g.GDR_FLAG_AUTOTUNE | (g.GDR_FLAG_NO_GRAPH if prec == g.GDR_PREC_FP64 else 0) | extra
    return g.gdr_params_default(m=p0.m, k=p0.k, m_proj=p0.m_proj, tol=1e-8, prec=prec, flags=flags)


def batch_check(g):
    def check(st, rep, per):
        assert st == g.GDR_OK and (per == 0).all() and rep["max_relres"] <= 1e-8, (st, rep)
    return check


def main_batch(args):
    """The batch of 64 independent convection-diffusion problems (sides 32..256, 4
    shifts each) in one batched GMRES-DR(30,10)-Sh solve (gdr_solve_batch), mixed
    precision against the plain FP64 batch; one step = one solve of the whole batch."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_0707_0502_gb300 as g
    world = int(os.environ.get("WORLD_SIZE", "1"))
    stream = torch.cuda.Stream()
    ctx = g.gdr_create(0, stream)
    probs, op, Bh, B, X, sig = batch_setup(g, ctx, stream)
    nprob, ns = len(probs), len(probs[0].sigma)
    ntot = sum(q.n for q in probs)
    sols = nprob * ns
    p0 = probs[0]
    flush = torch.empty(512 * 2**20, dtype=torch.uint8, device="cuda")
    tune = g.gdr_autotune(ctx, op, g.GDR_PREC_MIXED, nprob, p0.m)
    mixed = batch_params(g, p0, g.GDR_PREC_MIXED)
    plain = batch_params(g, p0, g.GDR_PREC_FP64)
    check = batch_check(g)
    clocks = Clocks(0)
    clocks.start()
    ms, rep = timed_solves(g, ctx, stream, flush, lambda: g.gdr_solve_batch(ctx, op, sig, B, X, mixed),
                           args.steps, args.warmup, check)
    clk = clocks.stop()
    value = job_throughput(world, sols * args.steps, sum(ms) / 1e3)
    ms64, _ = timed_solves(g, ctx, stream, flush, lambda: g.gdr_solve_batch(ctx, op, sig, B, X, plain),
                           max(1, min(args.steps, 3)), 1, check)
    fp64_value = sols * len(ms64) / (sum(ms64) / 1e3)
    Bp = torch.as_tensor(Bh).pin_memory()
    Xp = torch.zeros(ntot * ns, dtype=torch.complex128).pin_memory()
    hostp = batch_params(g, p0, g.GDR_PREC_MIXED, g.GDR_FLAG_HOST_PTRS)
    e2e_ms = []
    for i in range(min(args.warmup, 2) + min(args.steps, 3)):
        stream.synchronize()
        t0 = time.perf_counter()
        g.gdr_solve_batch(ctx, op, sig, Bp.numpy(), Xp.numpy(), hostp)
        if i >= min(args.warmup, 2):
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    roof, ktable = kernel_roofline(g, ctx, p0, lambda: g.gdr_solve_batch(ctx, op, sig, B, X, mixed))
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(ms) / len(ms), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic",
        "config": {"workload": f"{BATCH_WORKLOAD} ({ntot} unknowns)", "config_id": 5,
                   "l2": "flushed before every timed step (512 MB write)"},
        "clocks": clk, "gpu_launches": rep["kernel_launches"] * args.steps,
        "e2e": {"value": sols * len(e2e_ms) / (sum(e2e_ms) / 1e3), "unit": UNIT,
                "h2d_bytes_per_step": int(Bh.nbytes), "d2h_bytes_per_step": int(ntot * ns * 16)},
        "fp64_plain": {"value": fp64_value, "unit": UNIT, "ms_per_step": sum(ms64) / len(ms64),
                       "speedup_mixed_over_fp64": value / world / fp64_value},
        "solve": {k: rep[k] for k in ("mvps_rhs1", "cycles_rhs1", "mvps_refine", "refine_passes", "max_relres",
                                      "t_total_ms", "kernel_launches")},
        "roofline": roof, "kernels": ktable, "autotune": tune,
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = batch_cpu_baseline(probs)
    print(json.dumps(line), flush=True)
    g.gdr_op_destroy(op)
    g.gdr_destroy(ctx)


def batch_cpu_baseline(probs, budget_s=15.0):
    """The oracle on the first problems of the batch (in batch order) for about budget_s."""
    from oracle import CSROperator, gmres_dr_sh
    t, done, names = 0.0, 0, []
    for q in probs:
        A = CSROperator(*q.op[1:])
        t0 = time.perf_counter()
        gmres_dr_sh(A.matvec, q.B[:, 0], q.sigma, q.m, q.k, 1e-8)
        t += time.perf_counter() - t0
        done += 1
        names.append(q.n)
        if t > budget_s:
            break
    return {"value": done * len(probs[0].sigma) / t, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": f"oracle GMRES-DR({probs[0].m},{probs[0].k})-Sh of the first {done} problems of the batch "
                      f"(n = {names}), {t:.1f} s, numpy/BLAS threads = cores"}


def other_workloads(g, ctx, stream, flush, cids, steps=3):
    """Short runs of the other workloads on the same context (their own operators):
    the mixed solve (one warm-up, `steps` timed) and the plain FP64 solve (one timed),
    inputs resident in HBM, L2 flushed before each timed solve."""
    import torch
    out = {}
    for cid in cids:
        if cid == 5:
            probs, op, Bh, B, X, sig = batch_setup(g, ctx, stream)
            p0 = probs[0]
            sols = len(probs) * len(p0.sigma)
            g.gdr_autotune(ctx, op, g.GDR_PREC_MIXED, len(probs), p0.m)
            check = batch_check(g)
            mixed, plain = batch_params(g, p0, g.GDR_PREC_MIXED), batch_params(g, p0, g.GDR_PREC_FP64)
            ms, rep = timed_solves(g, ctx, stream, flush, lambda: g.gdr_solve_batch(ctx, op, sig, B, X, mixed),
                                   steps, 1, check)
            ms64, rep64 = timed_solves(g, ctx, stream, flush, lambda: g.gdr_solve_batch(ctx, op, sig, B, X, plain),
                                       1, 1, check)
            desc = BATCH_WORKLOAD
        else:
            p, cfg = workload(cid)
            sols = len(p.sigma) * p.B.shape[1]
            store = g.GDR_LINK_BF16 if p.extra.get("links") == "bf16" else g.GDR_LINK_C64
            with torch.cuda.stream(stream):
                op = g.make_operator(ctx, p, store=store)
                B = torch.as_tensor(np.ascontiguousarray(p.B.T), device="cuda")
                X = torch.zeros((p.B.shape[1], len(p.sigma), p.n), dtype=torch.complex128, device="cuda")
            stream.synchronize()
            g.gdr_autotune(ctx, op, g.GDR_PREC_MIXED, 1, p.m)

            def check(st, rep, p=p):
                assert st == g.GDR_OK and rep["max_relres"] <= p.tol, (st, rep)

            def call(params, p=p, op=op, B=B, X=X):
                st, rep, _ = g.gdr_solve_multishift(ctx, op, p.sigma, B, X, params)
                return st, rep
            mixed, plain = wilson_params(g, p, g.GDR_PREC_MIXED), wilson_params(g, p, g.GDR_PREC_FP64)
            ms, rep = timed_solves(g, ctx, stream, flush, lambda: call(mixed), steps, 1, check)
            ms64, rep64 = timed_solves(g, ctx, stream, flush, lambda: call(plain), 1, 1, check)
            desc = cfg["workload"]
        v, v64 = sols * len(ms) / (sum(ms) / 1e3), sols * len(ms64) / (sum(ms64) / 1e3)
        out[str(cid)] = {"workload": desc, "value": v, "unit": UNIT, "ms_per_step": sum(ms) / len(ms),
                         "steps": len(ms), "fp64_plain_value": v64, "speedup_mixed_over_fp64": v / v64,
                         "max_relres": rep["max_relres"], "mvps_refine": rep["mvps_refine"],
                         "fp64_mvps_total": rep64["mvps_rhs1"] + rep64.get("mvps_extra", 0) + rep64.get("mvps_proj", 0)}
        g.gdr_op_destroy(op)
        del B, X
        torch.cuda.empty_cache()
    return out


# FP64 flops of one launch of a dense kernel (complex multiply-add = 8 real flops),
# textbook counts for dense Householder QR (2mn^2 - 2n^3/3 real -> x4 complex),
# Hessenberg reduction (10/3 m^3 -> x4), explicit Q (4/3 m^3 -> x4) and the shifted
# QR sweeps with Schur vectors (20 m^3 -> x4).
def dense_flops(name, m, k, ns, ncol):
    qr = 4.0 * (4.0 / 3.0) * m**3
    if name == "dense_ls_harmonic_ritz":
        return ncol * (qr + qr + 4 * (10 / 3) * m**3 + 4 * (4 / 3) * m**3 + 4 * 20 * m**3)
    if name == "dense_ls":
        return ncol * qr
    if name == "dense_shifts_restart":
        return ncol * ((ns - 1) * qr + 8.0 * (m + 1) * m * k)
    if name == "dense_projection":  # the formed operators applied: (ns + 1) (k+1)^2 complex FMA
        return ncol * 8.0 * (ns + 1) * (k + 1) ** 2
    if name == "dense_projection_setup":  # per CTA: normal equations, 2 Gauss-Jordan, 3 products
        return ncol * 8.0 * (k * k * (k + 1) + 3.0 * k**3 + 3.0 * k * (k + 1) ** 2)
    return 0.0


KERNEL_SOURCES = {"dcgs2_update_c64": "krylov.cu", "dcgs2_dot_c64": "krylov.cu",
                  "wilson_matvec_c64_bf16links": "ops.cu", "wilson_matvec_c64": "ops.cu"}


def traffic_for(name, bytes_per_launch):
    """ncu DRAM bytes of one launch of `name`: the captured ratio to the algorithmic
    bytes times this launch's algorithmic bytes, while the kernel's source file is
    the one the capture ran (else None)."""
    rec = NCU_TRAFFIC.get(name)
    src = KERNEL_SOURCES.get(name)
    if not rec or not src:
        return None, "no ncu capture of this kernel's current source"
    path = os.path.join(ROOT, "paper_0707_0502_gb300", "csrc", src)
    sha = hashlib.sha256(open(path, "rb").read()).hexdigest()[:16]
    if sha != rec["sha16"]:
        return None, f"{src} changed since the ncu capture"
    return rec["ratio"] * bytes_per_launch, f"ncu {rec['profile']}: DRAM bytes / algorithmic bytes = {rec['ratio']}"


def kernel_roofline(g, ctx, p, solve):
    """One extra solve of the workload with per-kernel CUDA events (graphs off):
    every kernel's launches, time and algorithmic bytes; the roofline of the one
    with the largest total time."""
    pk = peaks()
    hbm, hbm_src = hbm_peak()
    sm_mhz = pk.get("sm_max_mhz", 2070.0)
    g.gdr_profile(ctx, True)
    solve()
    prof = g.gdr_profile_report(ctx)
    g.gdr_profile(ctx, False)
    total = sum(v["ms"] for v in prof.values())
    table = {}
    for name, v in prof.items():
        e = {"launches": v["launches"], "ms": round(v["ms"], 4), "share": round(v["ms"] / total, 4)}
        if v["bytes"] > 0:
            e["GBs"] = round(v["bytes"] / (v["ms"] / 1e3) / 1e9, 1)
        table[name] = e
    dom = max(prof, key=lambda k: prof[k]["ms"])
    v = prof[dom]
    per_launch_s = v["ms"] / 1e3 / v["launches"]
    if v["bytes"] > 0:
        achieved = v["bytes"] / v["launches"] / per_launch_s / 1e9
        bpl = v["bytes"] / v["launches"]
        traffic, tnote = traffic_for(dom, bpl)
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic, "bytes_per_launch": bpl,
                "note": f"peak = HBM copy bandwidth (of {hbm_src}); traffic: " + tnote}
    else:
        ns = len(p.sigma)
        flops = dense_flops(dom, p.m, p.k, ns, 1)
        # one CTA per problem on one SM: 4 SMSPs x 32 lanes x 2 flops per 64 cycles
        # (one FP64 warp-instruction occupies its SMSP for 64 cycles on GB300)
        peak = 4 * 32 * 2 / 64.0 * sm_mhz * 1e6 / 1e9
        achieved = flops / per_launch_s / 1e9
        roof = {"kernel": dom, "bound": "alu", "achieved": achieved, "peak": peak, "unit": "GFLOP/s",
                "frac": achieved / peak, "traffic": None, "flops_per_launch": flops,
                "note": "FP64 single-CTA kernel: peak = one SM's FP64 rate (2 FMA/clk) at sm_max_mhz; "
                        "flops from the textbook counts of bench.dense_flops"}
    roof["us_per_launch"] = per_launch_s * 1e6
    roof["share_of_solve"] = v["ms"] / total
    return roof, table


def kernels_at_scale(g, ctx, stream, only=None, link_store=None, tune=True, parts=("arnoldi", "matvec", "projection"),
                     shape=None):
    """The HBM-bound kernels on the two large lattices of the workload family
    (Wilson 16^4, complex64 links; 24^3x32, bf16 links), each profiled alone: the
    last steps of an m-step complex64 Arnoldi cycle (steps m-3..m-1 and the
    finalising pass, m = 60 / 80, the form the solves run), the single-column
    matvec and the multi-column matvec of the Proj / refinement stages (8 / 12
    columns) in the launch shape the autotuner chose (its time and the default
    shape's reported beside), and the projection over a kept basis shared by the
    120 columns of a refinement batch (k + 1 = 41 vectors: the dot c = V^H r and
    the residual update r += V t, on the tensor cores).  Inputs far larger than
    L2.  Per kernel: microseconds per launch, GB/s and fraction of the HBM
    peak."""
    step = "arnoldi" in parts
    import torch
    hbm, hbm_src = hbm_peak()
    out = {}
    for cid, dims, eps, store, m, ncol in [(3, (16, 16, 16, 16), 0.4, g.GDR_LINK_C64, 60, 8),
                                           (4, (24, 24, 24, 32), 0.5, g.GDR_LINK_BF16, 80, 12)]:
        if only is not None and only != "x".join(map(str, dims)):
            continue
        if link_store is not None:
            store = g.GDR_LINK_BF16 if link_store == "bf16" else g.GDR_LINK_C64
        links = W.su3_links(dims, eps, W.rng(cid, 0))
        n = 12 * int(np.prod(dims))
        with torch.cuda.stream(stream):
            op = g.gdr_op_wilson(ctx, dims, torch.as_tensor(links).cuda(), 0.0, store)
            gen = torch.Generator(device="cuda").manual_seed(cid)
            X = torch.randn((ncol, n), dtype=torch.complex64, device="cuda", generator=gen)
            Y = torch.empty_like(X)
            if step:
                V = torch.zeros((m + 1, n), dtype=torch.complex64, device="cuda")
                V[0] = torch.randn(n, dtype=torch.complex64, device="cuda", generator=gen)
                V[0] /= V[0].abs().square().sum().sqrt()
                Hb = torch.zeros((m, m + 1), dtype=torch.complex128, device="cuda")
        stream.synchronize()
        if step:  # an orthonormal basis: one complete cycle from V[0]
            g.gdr_arnoldi_cycle(ctx, op, g.GDR_PREC_MIXED, V, 0, m, Hb)
        del links
        tuned = {"1": g.gdr_autotune(ctx, op, g.GDR_PREC_MIXED, 1),
                 str(ncol): g.gdr_autotune(ctx, op, g.GDR_PREC_MIXED, ncol)} if tune else None

        def profiled(call, reps=5):
            for _ in range(2):  # warm-up
                call()
            g.gdr_profile(ctx, True)
            for _ in range(reps):
                call()
            prof = g.gdr_profile_report(ctx)
            g.gdr_profile(ctx, False)
            tab = {}
            for name, v in prof.items():
                if v["bytes"] <= 0:
                    continue
                us = v["ms"] / v["launches"] * 1e3
                gbs = v["bytes"] / (v["ms"] / 1e3) / 1e9
                tab[name] = {"launches": v["launches"], "us_per_launch": round(us, 1), "GBs": round(gbs, 1),
                             "frac_of_hbm": round(gbs / hbm, 3), "hbm_peak": hbm_src}
            return tab

        res = {}
        if step:  # Gram-Schmidt passes and single-column matvecs of the cycle's last steps
            res[f"arnoldi_steps_j{m - 3}_to_{m - 1}"] = profiled(
                lambda: g.gdr_arnoldi_cycle(ctx, op, g.GDR_PREC_MIXED, V, m - 3, m, Hb), reps=3)
        X1, Y1 = X[:1], Y[:1]
        if "matvec" in parts:
            if shape is not None:
                g.gdr_op_set_shape(op, g.GDR_PREC_MIXED, ncol, *shape)
            res["matvec_1col"] = profiled(lambda: g.gdr_op_apply(ctx, op, g.GDR_PREC_MIXED, np.zeros(1), X1, Y1))
            res[f"matvec_{ncol}col"] = profiled(
                lambda: g.gdr_op_apply(ctx, op, g.GDR_PREC_MIXED, np.zeros(ncol), X, Y))
            # the FP64 true-residual matvec: one right-hand side's shifts as complex128 columns
            nf = min(10, ncol)
            with torch.cuda.stream(stream):
                X64 = X[:nf].to(torch.complex128)
                Y64 = torch.empty_like(X64)
            stream.synchronize()
            res[f"matvec_fp64_{nf}col"] = profiled(
                lambda: g.gdr_op_apply(ctx, op, g.GDR_PREC_FP64, np.zeros(nf), X64, Y64), reps=3)
            del X64, Y64
        if "projection" in parts:  # the refinement batch's shared-basis projection
            nvp, ncp = 41, 120
            with torch.cuda.stream(stream):
                gen2 = torch.Generator(device="cuda").manual_seed(cid + 100)
                Vp = torch.randn((nvp, n), dtype=torch.complex64, device="cuda", generator=gen2)
                Rp = torch.randn((ncp, n), dtype=torch.complex64, device="cuda", generator=gen2)
                Tp = 1e-3 * torch.randn((ncp, nvp), dtype=torch.complex128, device="cuda", generator=gen2)
                Cp = torch.zeros((ncp, nvp), dtype=torch.complex128, device="cuda")
            stream.synchronize()

            def proj():
                g.gdr_basis_dot(ctx, g.GDR_PREC_MIXED, n, nvp, Vp, ncp, Rp, n, Cp)
                g.gdr_basis_residual_update(ctx, g.GDR_PREC_MIXED, n, nvp, Vp, ncp, Tp, Rp, n)
            res[f"projection_{nvp}x{ncp}col"] = profiled(proj)
            del Vp, Rp, Tp, Cp
        entry = {"n": n, "links": "bf16" if store == g.GDR_LINK_BF16 else "c64", "kernels": res,
                 "matvec_autotune": tuned}
        if tuned:  # the tuner's back-to-back timing of the chosen shape (no per-launch events)
            sl = 2 if store == g.GDR_LINK_BF16 else 4
            entry["matvec_back_to_back"] = {}
            for c, t in tuned.items():
                byt = n // 12 * (4 * 18 * sl + int(c) * 12 * 8 * 2)
                gbs = byt / (t["mv_ms"] * 1e-3) / 1e9
                entry["matvec_back_to_back"][c + "col"] = {"us_per_launch": round(t["mv_ms"] * 1e3, 1),
                                                           "GBs": round(gbs, 1),
                                                           "frac_of_hbm": round(gbs / hbm, 3)}
        out["x".join(map(str, dims))] = entry
        g.gdr_op_destroy(op)
        del X, Y, X1, Y1
        if step:
            del V, Hb
        torch.cuda.empty_cache()
    return out


if __name__ == "__main__":
    main()
