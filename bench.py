#!/usr/bin/env python
"""Benchmark: ms per SP2 purification with error control on GB300.

One step = one full SP2 purification (hybrid, Algorithm 5) of the 3D-lattice
Fock matrix, n = 16384 (4096 sites x 4 functions, decay 0.8, gap 0.1 enforced
by an eigenvector shift), leaf blocks 64, eps = 1e-5: every hot-path stage
(leaf norms, Algorithm 3 tau search, Algorithm 2 task planning, leaf
products with the fused SP2 epilogue, truncation) runs inside it, on the GPU.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--form fp64|mixed|auto]
    python bench.py --impl reference      # the CPU oracle arm
    python bench.py --protocol            # the paper's two-squares experiment

--protocol runs the experiment of the paper's Section 5 on a converged density
matrix D (this path's own purification of the same Fock matrix): for each
tolerance delta and each of truncmul (Algorithm 1's multiply-then-truncate),
SpAMM (Algorithm 4) and hybrid (Algorithm 5), X1 = approximate square of D,
X2 = approximate square of X1 at the same delta; the second square is timed
(T_mul, T_trunc, T_SpAMM, T_CSE as in Fig. 1), the block fill of X1, of the
product before truncation and of X2 is reported (Fig. 2), and ||X2 - X1^2||_F
against the exact float64 square of X1 (Fig. 3). One JSON line per (variant,
delta).

Prints one JSON line (rank 0). Timing: CUDA events on the library's stream,
barrier + synchronize on both sides of the K timed steps; inputs (2.1 GB per
matrix) are larger than L2, so no flush is needed between steps.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "ms per SpAMM product & per purification at ||E||_F<delta, mixed vs FP64 form"
WORKLOAD = ("SP2 purification (hybrid, Algorithm 5) of a 3D-lattice Fock matrix, n=16384 "
            "(4096 sites x 4 functions, decay 0.8, gap 0.1 by eigenvector shift), leaf 64, "
            "eps 1e-5")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="auto", choices=["auto", "fp64", "mixed"])
    ap.add_argument("--n", type=int, default=16384)
    ap.add_argument("--bs", type=int, default=64)
    ap.add_argument("--eps", type=float, default=1e-5)
    ap.add_argument("--n-iter", type=int, default=60)
    ap.add_argument("--variant", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--sample-n", type=int, default=2048)
    ap.add_argument("--protocol", action="store_true",
                    help="run the two-squares experiment instead of the purification bench")
    ap.add_argument("--deltas", default="1e-2,1e-4,1e-6,1e-8")
    ap.add_argument("--bound", default="alg3", choices=["alg3", "flat", "spectral"],
                    help="error bound of the tau searches (Algorithm 3, the flat bound, or the "
                         "spectral-norm bound; the last only with --protocol)")
    ap.add_argument("--tau-start", type=float, default=None,
                    help="first tau candidate (default: the paper's list, 1)")
    ap.add_argument("--tau-ratio", type=float, default=None,
                    help="ratio of successive tau candidates (default: the paper's list, 0.9)")
    ap.add_argument("--input-cache", default=None,
                    help="npz file holding the generated input (written when absent)")
    return check_args(ap, ap.parse_args(argv))


def check_args(ap, args):
    if args.bound == "spectral" and not args.protocol:
        ap.error("--bound spectral certifies the spectral norm of one product; the purification "
                 "keeps a Frobenius guarantee, so use it with --protocol")
    if (args.tau_start is None) != (args.tau_ratio is None):
        args.tau_start = 1.0 if args.tau_start is None else args.tau_start
        args.tau_ratio = 0.9 if args.tau_ratio is None else args.tau_ratio
    return args


def tau_table_config(args):
    """The candidate list of this run for the JSON line (None: the paper's list)."""
    if args.tau_start is None:
        return None
    return {"start": args.tau_start, "ratio": args.tau_ratio, "length": 350}


# --------------------------------------------------------------- inputs

def make_problem(n, use_gpu_eigh, cache=None):
    import numpy as np

    import synth
    if cache and os.path.exists(cache):
        z = np.load(cache)
        P = synth.FockProblem(z["F"], int(z["n_occ"]), float(z["homo"]), float(z["lumo"]), 0.8, "eig")
        P.occupied = z["occupied"]
        P.eigvals = z["eigvals"]
        return P
    eigh = None
    if use_gpu_eigh:
        import torch

        def eigh(F):
            t = torch.from_numpy(F).cuda()
            w, v = torch.linalg.eigh(t)
            out = (w.cpu().numpy(), v.cpu().numpy())
            del t, w, v
            torch.cuda.empty_cache()
            return out
    P = synth.lattice_fock(n, seed=synth.SEED_BASE + 1, decay=0.8, gap=0.1, gap_mode="eig",
                           eigh=eigh, keep_vectors=True)
    if cache:
        np.savez(cache, F=P.F, n_occ=P.n_occ, homo=P.homo, lumo=P.lumo, occupied=P.occupied,
                 eigvals=P.eigvals)
    return P


# -------------------------------------------------------------- clocks

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id: str):
        self.rows = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200", "-i", gpu_id], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                text=True)
        except OSError:
            return
        self.th = threading.Thread(target=self._read, daemon=True)
        self.th.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
        rows = self.rows
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        mx = [num(r[2]) for r in rows if num(r[2]) is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows),
                "power_w_max": max((num(r[3]) or 0.0) for r in rows)}


# ------------------------------------------------------------ baseline

def oracle_sample(X0, n_s, delta, bs):
    """Time the CPU oracle's spamm(X, X, delta) on the leading n_s x n_s
    principal block of X_0 (one thread)."""
    import numpy as np

    import oracle
    oracle.build()
    Xs = np.ascontiguousarray(X0[:n_s, :n_s])
    t0 = time.perf_counter()
    r = oracle.spamm_delta(Xs, Xs, delta, bs)
    dt = time.perf_counter() - t0
    return dt, r.products


def x0_of(F, lmin, lmax):
    import numpy as np
    n = F.shape[0]
    X = -F / (lmax - lmin)
    X[np.diag_indices(n)] += lmax / (lmax - lmin)
    return X


def gershgorin_np(F):
    import numpy as np
    d = np.diag(F)
    r = np.sum(np.abs(F), axis=1) - np.abs(d)
    return float(np.min(d - r)), float(np.max(d + r))


def scalar_sp2_steps(F_eigs, n_occ, eps, n_iter, lmin, lmax):
    """SP2 (trace-rule branches) run on the eigenvalues of F in exact arithmetic:
    the number of multiplies a purification performs until the stop rule."""
    import numpy as np
    x = (lmax - F_eigs) / (lmax - lmin)
    for it in range(1, n_iter + 1):
        c = x * x
        idem = float(np.sqrt(np.sum((c - x) ** 2)))
        if 2.0 * idem < 0.5 * eps:
            return it
        x = c if x.sum() > n_occ else 2 * x - c
    return n_iter


# ------------------------------------------------------- rank aggregation

def max_over_ranks(vals, dist=None, device="cpu"):
    """Element-wise maximum over the ranks (every rank times its own replicas)."""
    if dist is None or not dist.is_initialized():
        return list(vals)
    import torch
    t = torch.tensor(list(vals), dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.tolist()


def per_purification(sums_ms, world, steps):
    """Whole-job ms per purification: the slowest rank's time over all purifications
    of all ranks (replicas: each rank purifies its own copy, no data exchange)."""
    units = world * steps
    return [v / units for v in sums_ms]


# ---------------------------------------------------------------- arms

def run_reference(args, rank, world):
    """The oracle arm: the CPU oracle as it stands, on a bounded sample."""
    if rank != 0:
        return 0
    import numpy as np
    P = make_problem(args.n, use_gpu_eigh=False, cache=args.input_cache)
    lmin, lmax = gershgorin_np(P.F)
    X0 = x0_of(P.F, lmin, lmax)
    width = lmax - lmin
    gap = (P.lumo - P.homo) / width
    delta1 = args.eps / (2 * math.sqrt(2) * args.n_iter) * gap * 0.5
    iters = scalar_sp2_steps(P.eigvals, P.n_occ, args.eps, args.n_iter, lmin, lmax)
    nb = -(-args.n // args.bs)
    per_step = []
    prods = 0
    for _ in range(args.warmup + args.steps):
        dt, prods = oracle_sample(X0, args.sample_n, delta1, args.bs)
        per_step.append(dt)
    timed = per_step[args.warmup:]
    per_product = statistics.mean(timed) / max(1, prods)
    # S2 iterates are numerically dense: nb^3 leaf products per multiply
    value_ms = per_product * nb ** 3 * iters * 1e3
    sample = (f"oracle spamm(X0_s, X0_s, delta_1/2) on the leading {args.sample_n}x{args.sample_n} "
              f"principal block of X0 (bs {args.bs}, {prods} leaf products, "
              f"{statistics.mean(timed):.2f} s), scaled by nb^3={nb ** 3} products per multiply x "
              f"{iters} multiplies (exact-arithmetic SP2 on F's spectrum)")
    line = {"impl": "reference", "metric": METRIC, "value": value_ms, "unit": "ms",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": value_ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": args.n, "bs": args.bs, "eps": args.eps,
                       "variant": args.variant},
            "cpu_baseline": {"value": value_ms, "unit": "ms", "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value_ms, "unit": "ms", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_ours(args, rank, world):
    import numpy as np
    import torch

    import paper_2005_10680_gb300 as sp

    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    P = make_problem(args.n, use_gpu_eigh=True, cache=args.input_cache)
    n, bs = args.n, args.bs
    F_host = torch.from_numpy(P.F).pin_memory()
    D_host = torch.empty((n, n), dtype=torch.float64).pin_memory()
    stream = torch.cuda.Stream()
    ctx = sp.Context(local, stream=stream)
    ctx.set_bound(args.bound)
    if tau_table_config(args):
        ctx.set_tau_table(args.tau_start, args.tau_ratio)
    form = args.form
    if form == "auto":
        form = "mixed" if ctx.supports("mixed", bs) else "fp64"

    def step():
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        F = ctx.from_dense(F_host, bs=bs)                      # H2D of the step's input
        e[1].record(stream)
        D, rep = ctx.purify(F, P.n_occ, args.eps, args.n_iter, P.homo, P.lumo,
                            variant=args.variant, prec=form, strict=False)
        e[2].record(stream)
        D.to_host(D_host)                                      # D2H of the step's result
        e[3].record(stream)
        return e, rep, D

    for _ in range(args.warmup):
        e, rep, D = step()
        del D
    torch.cuda.synchronize()
    gpu_id = "0"
    try:
        gpu_id = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = ctx.launches()
    clocks = ClockSampler(gpu_id)
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    t_start.record(stream)
    evs, reps = [], []
    D = None
    for _ in range(args.steps):
        e, rep, D = step()
        evs.append(e)
        reps.append(rep)
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist is not None:
        dist.barrier()
    launches = ctx.launches() - launches0
    total_ms = t_start.elapsed_time(t_end)
    dev_ms = [e[1].elapsed_time(e[2]) for e in evs]
    e2e_ms = [e[0].elapsed_time(e[3]) for e in evs]
    sum_dev, sum_e2e, total_ms = max_over_ranks([sum(dev_ms), sum(e2e_ms), total_ms], dist, "cuda")
    value, e2e = per_purification([sum_dev, sum_e2e], world, args.steps)

    # correctness of the last step against the eigendecomposition (not timed)
    Dt = D_host.cuda()
    Vo = torch.from_numpy(P.occupied).cuda()
    Dt -= Vo @ Vo.T
    d_err = float(torch.linalg.norm(Dt))
    del Dt, Vo

    # roofline of the dominant kernel (leaf products), from the library's CUDA events on
    # the stream the kernel runs on: arithmetic the kernel issued / its time
    kept = sum(r["kept_total"] for r in reps)
    formed = sum(r["formed_total"] for r in reps)
    pipe = sum(r["pipe_flops_total"] for r in reps)
    gemm_ms = sum(r["ms_phase"][3] for r in reps)
    n_mult = sum(r["iters"] + (1 if r["converged"] else 0) for r in reps)
    if form == "fp64":
        # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (GB300's nominal 1.25 TFLOP/s FP64)
        roof = {"bound": "alu", "kernel": "k_gemm_fp64", "peak": 1.26, "unit": "TFLOP/s",
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
                "algorithmic": "2*bs^3 flop per formed leaf product"}
    else:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
        roof = {"bound": "tensor", "kernel": "k_gemm_tile", "peak": peaks["bf16_tflops_sustained"],
                "unit": "TFLOP/s", "peak_source": "MEASURED_PEAKS.json bf16_tflops_sustained (measured)",
                "algorithmic": "2*128*128*64 flop per (p,q) bf16 slice pair of a 128x128 tile task (4 MMAs of 128x128x16)"}
    achieved = pipe / (gemm_ms * 1e-3) / 1e12 if gemm_ms > 0 else 0.0
    roof.update({"achieved": achieved, "frac": achieved / roof["peak"], "traffic": None})
    useful_tflops = 2.0 * bs ** 3 * kept / (gemm_ms * 1e-3) / 1e12 if gemm_ms > 0 else 0.0
    rep0 = reps[-1]
    spamm_ms = (sum(r["ms_phase"][1] + r["ms_phase"][2] + r["ms_phase"][3] for r in reps) /
                max(1, n_mult))
    line = {"metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if form == "fp64" else "bf16 slices (f32 accumulate) -> f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "n": n, "bs": bs, "eps": args.eps,
                       "variant": args.variant, "form": form, "bound": args.bound,
                       **({"tau_table": tau_table_config(args)} if tau_table_config(args) else {}),
                       "l2": "inputs larger than L2 (2.1 GB per matrix), no flush",
                       "parallelism": f"replicas x{world}"},
            "spamm_ms": spamm_ms,
            "iters": rep0["iters"], "converged": rep0["converged"],
            "step_slice_levels": rep0["step_lmax"],
            "check": {"d_minus_exact_fro": d_err, "eps": args.eps},
            "phase_ms": {"cse": sum(r["ms_phase"][1] for r in reps) / args.steps,
                         "plan": sum(r["ms_phase"][2] for r in reps) / args.steps,
                         "leaf_products": gemm_ms / args.steps,
                         "truncation": sum(r["ms_phase"][4] for r in reps) / args.steps},
            "kept_products_per_step": kept / args.steps,
            "formed_products_per_step": formed / args.steps,
            "useful_tflops_f64_equivalent": useful_tflops,
            "roofline": roof,
            "e2e": {"value": e2e, "unit": "ms", "h2d_bytes_per_step": n * n * 8,
                    "d2h_bytes_per_step": n * n * 8},
            "clocks": clk, "gpu_launches": launches}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        lmin, lmax = rep0["lmin"], rep0["lmax"]
        X0 = x0_of(P.F, lmin, lmax)
        gap = (P.lumo - P.homo) / (lmax - lmin)
        delta1 = args.eps / (2 * math.sqrt(2) * args.n_iter) * gap * 0.5
        dt, prods = oracle_sample(X0, args.sample_n, delta1, bs)
        per_product = dt / max(1, prods)
        cpu_ms = per_product * (kept / args.steps) * 1e3   # the oracle forms every kept product
        line["cpu_baseline"] = {
            "value": cpu_ms, "unit": "ms", "cores": 1, "kind": "oracle",
            "sample": (f"oracle spamm(X0_s, X0_s, delta_1/2) on the leading {args.sample_n}x"
                       f"{args.sample_n} principal block of X0 (bs {bs}): {prods} leaf products "
                       f"in {dt:.2f} s, scaled by the {kept / args.steps:.0f} leaf products of one "
                       f"GPU purification")}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ---------------------------------------------------- two-squares protocol

PROTOCOL_VARIANTS = (("truncmul", 1), ("spamm", 4), ("hybrid", 5))


def approx_square(ctx, X, delta, variant, prec):
    """One approximate square X^2 with ||error||_F < delta by Algorithm 1's
    multiply + truncation (variant 1), SpAMM (4) or SpAMM at delta/2 plus
    truncation at delta/2 (5). Returns the product and the phase times (ms)
    and block counts of this square."""
    if variant == 1:
        Y, rep = ctx.sp2_step(X, 0, 0.0, 0.0, prec=prec)
    else:
        Y, rep = ctx.sp2_step(X, 0, delta if variant == 4 else 0.5 * delta, prec=prec)
    ms = rep["ms"]
    out = {"t_mul_ms": ms[6] if variant == 1 else 0.0,
           "t_spamm_ms": 0.0 if variant == 1 else ms[6] - ms[1],
           "t_cse_ms": 0.0 if variant == 1 else ms[1],
           "t_trunc_ms": 0.0, "nnzb_product": Y.nnzb, "tau": rep["tau"],
           "tau_index": rep["tau_index"], "cse_evals": rep["cse_evals"],
           "bound": rep["bound"], "bound_round": rep["bound_round"]}
    if variant in (1, 5):
        tr = ctx.truncate(Y, delta if variant == 1 else 0.5 * delta)
        out["t_trunc_ms"] = tr["ms"][4]
    out["nnzb_out"] = Y.nnzb
    return Y, out


def fro_diff(A, B):
    """||A - B||_F of two device matrices, read back densely (a check, not a step of
    the path)."""
    import torch
    a, b = A.to_torch(), B.to_torch()
    d = float(torch.linalg.norm(a - b))
    del a, b
    return d


def norm2_diff(A, B):
    """||A - B||_2 of two symmetric device matrices: the largest absolute eigenvalue of
    the difference, read back densely (a check, not a step of the path)."""
    import torch
    a, b = A.to_torch(), B.to_torch()
    a -= b
    del b
    a += a.T.clone()                      # exactly symmetric for the eigensolver
    a *= 0.5
    w = torch.linalg.eigvalsh(a)
    del a
    return float(w.abs().max())


def square_twice(ctx, D, delta, variant, prec, spectral=False):
    """The paper's protocol for one (variant, delta): square D, square the result
    again at the same delta, time the second square and check it against the exact
    float64 square of its input (in the spectral norm too when that is the norm
    the searches certify)."""
    X1, _ = approx_square(ctx, D, delta, variant, prec)
    X2, out = approx_square(ctx, X1, delta, variant, prec)
    exact, _ = ctx.sp2_step(X1, 0, 0.0, 0.0, prec="fp64")
    err = fro_diff(X2, exact)
    nb2 = D.nb * D.nb
    out.update({"nnz_pct": {"X_in": 100.0 * X1.nnzb / nb2,
                            "product": 100.0 * out.pop("nnzb_product") / nb2,
                            "X_out": 100.0 * out.pop("nnzb_out") / nb2},
                "err": err, "err_over_delta": err / delta})
    if spectral:
        err2 = norm2_diff(X2, exact)
        out.update({"err_2": err2, "err_2_over_delta": err2 / delta})
    return out


def run_protocol(args):
    import torch

    import paper_2005_10680_gb300 as sp
    torch.cuda.set_device(0)
    P = make_problem(args.n, use_gpu_eigh=True, cache=args.input_cache)
    stream = torch.cuda.Stream()
    ctx = sp.Context(0, stream=stream)
    fastest = "mixed" if ctx.supports("mixed", args.bs) else "fp64"
    F = ctx.from_dense(torch.from_numpy(P.F), bs=args.bs)
    D, rep = ctx.purify(F, P.n_occ, args.eps, args.n_iter, P.homo, P.lumo,
                        variant=args.variant, prec=fastest, strict=False)
    del F
    ctx.set_bound(args.bound)
    if tau_table_config(args):
        ctx.set_tau_table(args.tau_start, args.tau_ratio)
    forms = [args.form] if args.form != "auto" else sorted({fastest, "fp64"})
    for form in forms:
        for delta in [float(x) for x in args.deltas.split(",")]:
            for name, v in PROTOCOL_VARIANTS:
                out = square_twice(ctx, D, delta, v, form, spectral=args.bound == "spectral")
                line = {"protocol": "two squares of a converged D", "variant": name,
                        "algorithm": v, "delta": delta, "form": form, "bound_kind": args.bound,
                        "tau_table": tau_table_config(args) or "paper",
                        "n": args.n, "bs": args.bs,
                        "D": f"SP2 purification (Algorithm {args.variant}, {fastest}) of the "
                             f"bench's Fock matrix, eps {args.eps}, {rep['iters']} iterations"}
                line.update(out)
                print(json.dumps(line), flush=True)
    return 0


def main():
    args = parse()
    if args.protocol:
        return run_protocol(args)
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    return run_ours(args, rank, world)


if __name__ == "__main__":
    sys.exit(main())
