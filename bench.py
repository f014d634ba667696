"""Benchmark: shifted solutions/sec to a 1e-8 FP64 residual (mixed + batched
vs plain FP64) on the Wilson-Dirac-style 8^4 lattice (49,152 unknowns,
6 kappa shifts, GMRES-DR(40,20)), plus the roofline of the dominant kernel.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one complete multi-shift solve (every shift of every right-hand
side to a true FP64 relative residual <= 1e-8, checked inside the library)
with the operator and right-hand sides resident in HBM.  L2 is flushed
(a 512 MB write) before every timed step.  With N > 1 (torchrun) every rank
solves its own replica of the workload (the solver does not shard); the
value is the aggregate over ranks.  Prints one JSON line on rank 0.
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

CONFIG_ID = 2
METRIC = "shifted solutions/sec to 1e-8 FP64 residual, mixed+batched vs plain FP64; matvec HBM GB/s"
UNIT = "solutions/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=60)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", type=int, default=CONFIG_ID)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-scale", action="store_true", help="skip the large-lattice kernel measurements")
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
                    help="with --kernels-only: the matvecs alone (no Arnoldi-step basis on the device)")
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


# ------------------------------------------------------------- reference arm

def oracle_solve(p):
    """The oracle (complex128, numpy/scipy) solving every shift of every rhs."""
    from oracle import CSROperator, WilsonOperator, solve_all_rhs
    if p.op[0] == "wilson":
        A = WilsonOperator(p.op[1], p.op[3], p.op[2])
    else:
        A = CSROperator(*p.op[1:])
    t = time.perf_counter()
    out = solve_all_rhs(A.matvec, p.B, p.sigma, p.m, p.k, p.m_proj, p.tol, p.extra_tol, max_mvps=20000)
    return time.perf_counter() - t, out


def cpu_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count()


def cpu_baseline(p, solve_mvps=None):
    """The oracle on the host cores.  Small workloads (up to 10^5 unknowns x rhs): one
    complete solve.  Larger ones (configurations 3, 4): a bounded sample -- three timed
    oracle Arnoldi steps (matvec + CGS2) at the cycle's average basis size m/2 -- scaled
    to the matvec count of the whole solve (``solve_mvps``, the FP64 GPU run's, which
    follows the same algorithm); the small dense steps are left out of the estimate."""
    sols = len(p.sigma) * p.B.shape[1]
    if p.n * p.B.shape[1] <= 100000 or not solve_mvps:
        dt, out = oracle_solve(p)
        return {"value": sols / dt, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                "sample": f"one complete oracle solve of the workload ({sols} shifted solutions, "
                          f"{out['mvps_rhs1']} mvps for rhs 1) in {dt:.2f} s, numpy/BLAS threads = cores"}
    from oracle import WilsonOperator, arnoldi_cgs2_step
    A = WilsonOperator(p.op[1], p.op[3], p.op[2])
    j = p.m // 2  # the average basis size of a cycle
    g = np.random.default_rng(0)
    V = np.zeros((p.n, j + 2), dtype=np.complex128)
    for q in range(j + 1):
        v = g.standard_normal(p.n) + 1j * g.standard_normal(p.n)
        V[:, q] = v / np.linalg.norm(v)
    Hs = np.zeros((j + 2, j + 1), dtype=np.complex128)
    t = time.perf_counter()
    for _ in range(3):
        arnoldi_cgs2_step(A.matvec, V, Hs, j)
    dt = (time.perf_counter() - t) / 3
    est = dt * solve_mvps
    return {"value": sols / est, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
            "sample": f"estimated: the oracle's Arnoldi step (matvec + CGS2) at j = {j} of GMRES-DR({p.m},{p.k}) took "
                      f"{dt:.2f} s (mean of 3), scaled to the {solve_mvps} matvecs of the whole FP64 solve "
                      f"({sols} shifted solutions), numpy/BLAS threads = cores"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    if args.config == 5:  # the oracle on every problem of the batch, one after the other
        from oracle import CSROperator, gmres_dr_sh
        probs = W.config(5)
        cfg = {"workload": "64 convection-diffusion CSR problems, sides 32-256, 4 shifts each, GMRES-DR(30,10)",
               "config_id": 5}

        def batch_solve():
            t0 = time.perf_counter()
            for q in probs:
                gmres_dr_sh(CSROperator(*q.op[1:]).matvec, q.B[:, 0], q.sigma, q.m, q.k, 1e-8)
            return time.perf_counter() - t0, None
        solve, sols = batch_solve, sum(len(q.sigma) for q in probs)
    else:
        p, cfg = workload(args.config)
        solve, sols = (lambda: oracle_solve(p)), len(p.sigma) * p.B.shape[1]
    times = []
    for _ in range(args.warmup):
        solve()
    for _ in range(args.steps):
        dt, _ = solve()
        times.append(dt)
    value = sols * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": cfg,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                             "sample": "each step one complete oracle solve of the workload"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ our arm

def main_batch(args):
    """Configuration 5: 64 independent convection-diffusion problems (sides 32..256,
    4 shifts each) in one batched GMRES-DR(30,10)-Sh solve (gdr_solve_batch), mixed
    precision against the plain FP64 batch; one step = one solve of the whole batch."""
    import torch
    import __graft_entry__
    __graft_entry__.build()
    import paper_0707_0502_gb300 as g
    world = int(os.environ.get("WORLD_SIZE", "1"))
    probs = W.config(5)
    nprob, ns = len(probs), len(probs[0].sigma)
    ntot = sum(p.n for p in probs)
    sols = nprob * ns
    p0 = probs[0]
    stream = torch.cuda.Stream()
    ctx = g.gdr_create(0, stream)
    with torch.cuda.stream(stream):
        op = g.make_batch_operator(ctx, probs)
        Bh = np.concatenate([p.B[:, 0] for p in probs])
        B = torch.as_tensor(Bh, device="cuda")
        X = torch.zeros(ntot * ns, dtype=torch.complex128, device="cuda")
        flush = torch.empty(512 * 2**20, dtype=torch.uint8, device="cuda")
    stream.synchronize()
    sig = np.stack([p.sigma for p in probs])
    tune = g.gdr_autotune(ctx, op, g.GDR_PREC_MIXED, nprob, p0.m)
    mixed = g.gdr_params_default(m=p0.m, k=p0.k, m_proj=p0.m_proj, tol=1e-8, prec=g.GDR_PREC_MIXED,
                                 flags=g.GDR_FLAG_AUTOTUNE)
    plain = g.gdr_params_default(m=p0.m, k=p0.k, m_proj=p0.m_proj, tol=1e-8, prec=g.GDR_PREC_FP64,
                                 flags=g.GDR_FLAG_NO_GRAPH | g.GDR_FLAG_AUTOTUNE)

    def timed(params, steps, warm, Bx=B, Xx=X):
        for _ in range(warm):
            g.gdr_solve_batch(ctx, op, sig, Bx, Xx, params)
        ms, reps = [], []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, rep, per = g.gdr_solve_batch(ctx, op, sig, Bx, Xx, params)
            e1.record(stream)
            e1.synchronize()
            assert st == g.GDR_OK and (per == 0).all() and rep["max_relres"] <= 1e-8, (st, rep)
            ms.append(e0.elapsed_time(e1))
            reps.append(rep)
        return ms, reps

    clocks = Clocks(0)
    clocks.start()
    ms, reps = timed(mixed, args.steps, args.warmup)
    clk = clocks.stop()
    value = job_throughput(world, sols * args.steps, sum(ms) / 1e3)
    ms64, reps64 = timed(plain, max(1, min(args.steps, 3)), 1)
    fp64_value = sols * len(ms64) / (sum(ms64) / 1e3)
    Bp = torch.as_tensor(Bh).pin_memory()
    Xp = torch.zeros(ntot * ns, dtype=torch.complex128).pin_memory()
    hostp = g.gdr_params_default(m=p0.m, k=p0.k, m_proj=p0.m_proj, tol=1e-8, prec=g.GDR_PREC_MIXED,
                                 flags=g.GDR_FLAG_HOST_PTRS)
    e2e_ms = []
    for i in range(min(args.warmup, 2) + min(args.steps, 3)):
        stream.synchronize()
        t0 = time.perf_counter()
        st, _, _ = g.gdr_solve_batch(ctx, op, sig, Bp.numpy(), Xp.numpy(), hostp)
        if i >= min(args.warmup, 2):
            e2e_ms.append((time.perf_counter() - t0) * 1e3)
    roof, ktable = kernel_roofline(g, ctx, op, p0, mixed, stream, B, X, 5,
                                   solve=lambda: g.gdr_solve_batch(ctx, op, sig, B, X, mixed))
    rep = reps[-1]
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": sum(ms) / len(ms), "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic",
        "config": {"workload": f"64 convection-diffusion CSR problems, sides 32-256 ({ntot} unknowns), 4 shifts "
                               f"each, GMRES-DR({p0.m},{p0.k}), one batched solve", "config_id": 5,
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
        from oracle import CSROperator, gmres_dr_sh
        t, done, names = 0.0, 0, []
        for p in probs:  # a bounded sample: problems in batch order until ~15 s
            A = CSROperator(*p.op[1:])
            t0 = time.perf_counter()
            gmres_dr_sh(A.matvec, p.B[:, 0], p.sigma, p.m, p.k, 1e-8)
            t += time.perf_counter() - t0
            done += 1
            names.append(p.n)
            if t > 15.0:
                break
        line["cpu_baseline"] = {"value": done * ns / t, "unit": UNIT, "cores": cpu_cores(), "kind": "oracle",
                                "sample": f"oracle GMRES-DR({p0.m},{p0.k})-Sh of the first {done} problems of the "
                                          f"batch (n = {names}), {t:.1f} s, numpy/BLAS threads = cores"}
    print(json.dumps(line), flush=True)
    g.gdr_op_destroy(op)
    g.gdr_destroy(ctx)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.config == 5:
        main_batch(args)
        return
    if args.kernels_only:
        import torch
        import __graft_entry__
        __graft_entry__.build()
        import paper_0707_0502_gb300 as g
        stream = torch.cuda.Stream()
        ctx = g.gdr_create(0, stream)
        out = kernels_at_scale(g, ctx, stream, only=args.kernels_only, link_store=args.links, tune=False,
                               step=not args.matvec_only)
        print(json.dumps({"kernels_at_scale": out}), flush=True)
        g.gdr_destroy(ctx)
        return
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    import __graft_entry__
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
    mixed = g.gdr_params_default(m=p.m, k=p.k, m_proj=p.m_proj, tol=p.tol, extra_tol=p.extra_tol,
                                 prec=g.GDR_PREC_MIXED,
                                 flags=g.GDR_FLAG_AUTOTUNE | form_flag)  # inner_tol: automatic
    plain = g.gdr_params_default(m=p.m, k=p.k, m_proj=p.m_proj, tol=p.tol, extra_tol=p.extra_tol,
                                 prec=g.GDR_PREC_FP64,
                                 flags=g.GDR_FLAG_SEQUENTIAL | g.GDR_FLAG_NO_GRAPH | g.GDR_FLAG_AUTOTUNE)

    def timed(params, steps, warm, Bx=B, Xx=X):
        reps = []
        for _ in range(warm):
            st, rep, _ = g.gdr_solve_multishift(ctx, op, p.sigma, Bx, Xx, params)
            assert st == g.GDR_OK, (st, rep)
        ms = []
        for _ in range(steps):
            with torch.cuda.stream(stream):
                flush.fill_(1)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            st, rep, _ = g.gdr_solve_multishift(ctx, op, p.sigma, Bx, Xx, params)
            e1.record(stream)
            e1.synchronize()
            assert st == g.GDR_OK and rep["max_relres"] <= p.tol, (st, rep)
            ms.append(e0.elapsed_time(e1))
            reps.append(rep)
        return ms, reps

    # ---- timed region: mixed + batched path
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    ms, reps = timed(mixed, args.steps, args.warmup)
    torch.cuda.synchronize()
    clk = clocks.stop()
    total_s = sum(ms) / 1e3
    t_max = max_over_ranks(total_s, world)
    if world > 1:
        dist.barrier()
    value = job_throughput(world, sols * args.steps, t_max)
    rep = reps[-1]
    launches = rep["kernel_launches"]

    # ---- plain FP64 GPU path (same algorithm, complex128, rhs sequential, no graphs)
    ms64, reps64 = timed(plain, max(1, min(args.steps, 5)), 1)
    fp64_value = sols * len(ms64) / (sum(ms64) / 1e3)

    # ---- end to end through the C ABI with host buffers (copies inside)
    Bh = torch.as_tensor(np.ascontiguousarray(p.B.T)).pin_memory()
    Xh = torch.zeros((nrhs, ns, p.n), dtype=torch.complex128).pin_memory()
    host_params = g.gdr_params_default(m=p.m, k=p.k, m_proj=p.m_proj, tol=p.tol, extra_tol=p.extra_tol,
                                       prec=g.GDR_PREC_MIXED, flags=g.GDR_FLAG_HOST_PTRS)
    e2e_ms = []
    for i in range(min(args.warmup, 3) + min(args.steps, 5)):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        stream.synchronize()
        t0 = time.perf_counter()
        st, r2, _ = g.gdr_solve_multishift(ctx, op, p.sigma, Bh.numpy(), Xh.numpy(), host_params)
        t1 = time.perf_counter()
        assert st == g.GDR_OK
        if i >= min(args.warmup, 3):
            e2e_ms.append((t1 - t0) * 1e3)
    e2e_value = job_throughput(world, sols * len(e2e_ms), max_over_ranks(sum(e2e_ms) / 1e3, world))

    # ---- dominant kernel roofline (per-kernel CUDA events on the library stream)
    roof, ktable = kernel_roofline(g, ctx, op, p, mixed, stream, B, X, args.config)
    scale = kernels_at_scale(g, ctx, stream) if not args.no_scale else None

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "c64+f64", "data": "synthetic", "config": cfg,
        "clocks": clk, "gpu_launches": launches * args.steps,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": int(p.B.nbytes),
                "d2h_bytes_per_step": int(nrhs * ns * p.n * 16)},
        "fp64_plain": {"value": fp64_value, "unit": UNIT, "ms_per_step": sum(ms64) / len(ms64),
                       "speedup_mixed_over_fp64": value / world / fp64_value,
                       "mvps_rhs1": reps64[-1]["mvps_rhs1"]},
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
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        r64 = reps64[-1]
        line["cpu_baseline"] = cpu_baseline(p, r64["mvps_rhs1"] + r64["mvps_extra"] + r64["mvps_proj"])
    if rank == 0:
        print(json.dumps(line), flush=True)
    g.gdr_op_destroy(op)
    g.gdr_destroy(ctx)
    if world > 1:
        dist.destroy_process_group()


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


# DRAM bytes per launch of a dominant kernel, from one ncu capture of this bench's own
# launches on the default workload (profiles/gs_update_dot_wilson8x8x8x8.md: average over
# the 200 launches of one solve; ncu flushes the caches before each captured launch, so
# this is the cold-cache traffic).  Reset when the kernel changes.
NCU_TRAFFIC = {(CONFIG_ID, "gs_update_dot_c64"): 10243110}


def kernel_roofline(g, ctx, op, p, params, stream, B, X, cid=CONFIG_ID, solve=None):
    """One extra solve of the workload with per-kernel CUDA events (graphs off):
    every kernel's launches, time and algorithmic bytes; the roofline of the one
    with the largest total time."""
    import torch
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    sm_mhz = peaks.get("sm_max_mhz", 2070.0)
    g.gdr_profile(ctx, True)
    if solve is not None:
        solve()
    else:
        g.gdr_solve_multishift(ctx, op, p.sigma, B, X, params)
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
        traffic = NCU_TRAFFIC.get((cid, dom))
        roof = {"kernel": dom, "bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "traffic": traffic,
                "bytes_per_launch": v["bytes"] / v["launches"],
                "note": "peak = MEASURED_PEAKS.json hbm_gbs (of measured)"
                        + ("; traffic: ncu dram__bytes_read.sum + dram__bytes_write.sum per launch, cold caches"
                           if traffic is not None else "")}
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


def kernels_at_scale(g, ctx, stream, only=None, link_store=None, tune=True, step=True):
    """The HBM-bound kernels on the two large lattices of the workload family
    (Wilson 16^4, c64 links; 24^3x32, bf16 links), each profiled alone: one
    Arnoldi step at the last column of the basis (j = m - 1, m = 60 / 80), the
    single-column matvec and the multi-column matvec of the refinement / Proj
    stages (8 / 12 columns), the matvecs in the launch shape the autotuner chose
    (its time and the default shape's reported beside).  Inputs far larger than
    L2.  Per kernel: microseconds per launch, GB/s and fraction of measured HBM
    peak."""
    import torch
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
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
                V = torch.randn((m + 1, n), dtype=torch.complex64, device="cuda", generator=gen)
                V /= V.norm(dim=1, keepdim=True)
                hcol = torch.zeros(m + 1, dtype=torch.complex128, device="cuda")
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
                             "frac_of_measured_hbm": round(gbs / hbm, 3)}
            return tab

        res = {}
        if step:  # Gram-Schmidt kernels and the single-column matvec of one Arnoldi step
            res[f"arnoldi_step_j{m - 1}"] = profiled(
                lambda: g.gdr_arnoldi_step(ctx, op, g.GDR_PREC_MIXED, V, m - 1, hcol))
        X1, Y1 = X[:1], Y[:1]
        res["matvec_1col"] = profiled(lambda: g.gdr_op_apply(ctx, op, g.GDR_PREC_MIXED, np.zeros(1), X1, Y1))
        res[f"matvec_{ncol}col"] = profiled(
            lambda: g.gdr_op_apply(ctx, op, g.GDR_PREC_MIXED, np.zeros(ncol), X, Y))
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
                                                           "frac_of_measured_hbm": round(gbs / hbm, 3)}
        out["x".join(map(str, dims))] = entry
        g.gdr_op_destroy(op)
        del X, Y, X1, Y1
        if step:
            del V, hcol
        torch.cuda.empty_cache()
    return out


if __name__ == "__main__":
    main()
