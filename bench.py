#!/usr/bin/env python
"""Benchmark: ms per SP2 purification (and per SpAMM product) with error control on GB300.

Workload: the large configuration, n = 262144. F is the 3D-lattice Fock matrix of
65536 sites (a 64 x 32 x 32 box in Morton order) x 4 functions, decay rate 4.0 with a
hard cutoff at 6 lattice units (3.3 % of the 64 x 64 leaf blocks stored, 18 GB), gap
0.1 by the Gershgorin-certified staggered onsite shift. One step = one full SP2
purification (hybrid, Algorithm 5) to eps = 1e-5 in the mixed form: every hot-path
stage (leaf norms, the Algorithm 3 tau search over the live node triples, the task
planning, operand slicing, leaf products with the fused SP2 epilogue, truncation)
runs inside it, on the GPU.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--form fp64|mixed|auto]
    python bench.py --impl reference      # the CPU oracle arm
    python bench.py --protocol            # the paper's two-squares experiment

After the timed steps, once each (not part of `value`): one SpAMM product X_0 X_0 at
delta = 1e-7 with the tau search in both forms (the configuration's SpAMM half), the
same purification in the float64 form (and the sampled difference of the two D), the
n = 2048 banded SpAMM product (delta = 1e-6, float64, leaf 32), and the n = 16384
dense-lattice purification measured in the earlier configuration.

--protocol runs the experiment of the paper's Section 5 on a converged density
matrix D (this path's own purification of a sparse lattice Fock matrix, n = 65536 by
default): for each tolerance delta and each of truncmul (Algorithm 1's
multiply-then-truncate), SpAMM (Algorithm 4) and hybrid (Algorithm 5), X1 =
approximate square of D, X2 = approximate square of X1 at the same delta; the second
square is timed (T_mul, T_trunc, T_SpAMM, T_CSE as in Fig. 1), the block fill of X1,
of the product before truncation and of X2 is reported (Fig. 2), and ||X2 - X1^2||_F
against the exact float64 square of X1 (Fig. 3). One JSON line per (variant, delta).

Prints one JSON line (rank 0). Timing: CUDA events on the library's stream, barrier
+ synchronize on both sides of the K timed steps; the matrices (18 GB each) are far
larger than L2, so no flush is needed between steps.
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


def workload_name(args):
    return (f"SP2 purification (hybrid, Algorithm 5) of a block-sparse 3D-lattice Fock matrix, "
            f"n={args.n} ({args.n // 4} sites x 4 functions, decay {args.decay}, cutoff "
            f"{args.cutoff}, gap 0.1 by staggered onsite shift), leaf {args.bs}, eps {args.eps}; "
            f"SpAMM X0*X0 with tau search at delta {args.spamm_delta}")


S2_WORKLOAD = ("SP2 purification (hybrid, Algorithm 5) of a dense 3D-lattice Fock matrix, "
               "n=16384 (decay 0.8, gap 0.1 by eigenvector shift), leaf 64, eps 1e-5")


def parse(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--form", default="auto", choices=["auto", "fp64", "mixed"])
    ap.add_argument("--n", type=int, default=262144)
    ap.add_argument("--bs", type=int, default=64)
    ap.add_argument("--decay", type=float, default=4.0)
    ap.add_argument("--cutoff", type=float, default=6.0)
    ap.add_argument("--eps", type=float, default=1e-5)
    ap.add_argument("--n-iter", type=int, default=60)
    ap.add_argument("--variant", type=int, default=5)
    ap.add_argument("--spamm-delta", type=float, default=1e-7)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the one-off measurements after the timed steps")
    ap.add_argument("--cores", type=int, default=0,
                    help="host cores for the CPU baselines (default: all)")
    ap.add_argument("--sample-n", type=int, default=2048,
                    help="side of each principal block the CPU oracle multiplies")
    ap.add_argument("--protocol", action="store_true",
                    help="run the two-squares experiment instead of the purification bench")
    ap.add_argument("--protocol-n", type=int, default=65536)
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


def config_of(args, form=None, world=1):
    """The `config` of both arms' JSON lines (identical keys and values)."""
    cfg = {"workload": workload_name(args), "n": args.n, "bs": args.bs, "decay": args.decay,
           "cutoff": args.cutoff, "eps": args.eps, "variant": args.variant,
           "spamm_delta": args.spamm_delta, "bound": args.bound,
           "l2": "inputs larger than L2 (18 GB per matrix), no flush",
           "parallelism": f"replicas x{world}"}
    if tau_table_config(args):
        cfg["tau_table"] = tau_table_config(args)
    return cfg


# --------------------------------------------------------------- inputs

def make_lattice(args, n=None):
    """The block-sparse lattice Fock matrix (block list; no dense form)."""
    import numpy as np

    import synth
    n = n or args.n
    cache = args.input_cache if n == args.n else None
    if cache and os.path.exists(cache):
        z = np.load(cache)
        return synth.BlockFockProblem(n, args.bs, z["brow"], z["bcol"], z["tiles"],
                                      int(z["n_occ"]), float(z["homo"]), float(z["lumo"]),
                                      args.decay, args.cutoff)
    B = synth.lattice_fock_blocks(n, seed=synth.SEED_BASE + 4, decay=args.decay,
                                  cutoff=args.cutoff, bs=args.bs)
    if cache:
        np.savez(cache, brow=B.brow, bcol=B.bcol, tiles=B.tiles, n_occ=B.n_occ, homo=B.homo,
                 lumo=B.lumo)
    return B


def gershgorin_blocks(B):
    """Gershgorin bounds of a block-listed symmetric matrix (host, input set-up)."""
    import numpy as np
    bs = B.bs
    R = np.zeros(B.n)
    d = np.zeros(B.n)
    rs = np.abs(B.tiles).sum(axis=2)                       # (nnzb, bs) row sums
    diag_t = np.nonzero(B.brow == B.bcol)[0]
    for t in diag_t:
        dd = np.diag(B.tiles[t])
        d[B.brow[t] * bs:(B.brow[t] + 1) * bs] = dd
        rs[t] -= np.abs(dd)
    np.add.at(R.reshape(-1, bs), B.brow, rs)
    return float((d - R).min()), float((d + R).max())


def x0_tiles(B, lmin, lmax):
    """X_0 = (lmax I - F) / (lmax - lmin) on F's block pattern."""
    import numpy as np
    w = lmax - lmin
    T = B.tiles * (-1.0 / w)
    for t in np.nonzero(B.brow == B.bcol)[0]:
        T[t][np.diag_indices(B.bs)] += lmax / w
    return T


def make_dense_problem(n, use_gpu_eigh):
    """The dense lattice Fock matrix of the n = 16384 configuration (decay 0.8, gap by an
    eigenvector shift), with its occupied eigenvectors for the exact D."""
    import synth
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
    return synth.lattice_fock(n, seed=synth.SEED_BASE + 1, decay=0.8, gap=0.1, gap_mode="eig",
                              eigh=eigh, keep_vectors=True)


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


# ------------------------------------------------------------ baselines

def _oracle_sample(job):
    """One bounded sample of the CPU oracle, in a worker process (one thread):
    spamm(X_s, X_s, delta) with the tau search on a principal block X_s of X_0."""
    import numpy as np

    import oracle
    Xs, delta, bs = job
    oracle.build()
    t0 = time.perf_counter()
    r = oracle.spamm_delta(Xs, Xs, delta, bs)
    dt = time.perf_counter() - t0
    nb = Xs.shape[0] // bs
    P = (np.abs(Xs).reshape(nb, bs, nb, bs).sum(axis=(1, 3)) > 0).astype(np.float64)
    cand = float(np.sum(P.sum(axis=0) * P.sum(axis=1)))
    return dt, int(r.products), cand


def principal_block(B, T, row0, n_s):
    """The dense principal block X[row0 : row0 + n_s, row0 : row0 + n_s] of a block list."""
    import numpy as np
    bs = B.bs
    b0, b1 = row0 // bs, (row0 + n_s) // bs
    sel = np.nonzero((B.brow >= b0) & (B.brow < b1) & (B.bcol >= b0) & (B.bcol < b1))[0]
    X = np.zeros((n_s, n_s))
    for t in sel:
        i, j = int(B.brow[t]) - b0, int(B.bcol[t]) - b0
        X[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] = T[t]
    return X


def host_cores(args):
    return args.cores if args.cores > 0 else (os.cpu_count() or 1)


def cpu_oracle_rate(B, T, delta, cores, n_s):
    """Products per second of the CPU oracle on `cores` host cores: one process per core
    (spawned, one thread each), each multiplying its own principal block of X_0 (blocks
    spread along the diagonal). Returns (rate, wall seconds, products, candidate
    products of the samples, samples)."""
    import multiprocessing as mp
    count = max(1, cores)
    stride = max(n_s, (B.n - n_s) // max(1, count - 1) // B.bs * B.bs)
    jobs = [(principal_block(B, T, min(q * stride, B.n - n_s), n_s), delta, B.bs)
            for q in range(count)]
    env = {"OMP_NUM_THREADS": "1", "OPENBLAS_NUM_THREADS": "1", "MKL_NUM_THREADS": "1"}
    old = {k: os.environ.get(k) for k in env}
    os.environ.update(env)
    try:
        with mp.get_context("spawn").Pool(count) as pool:
            pool.map(_oracle_sample, jobs[:1])            # start-up (import, build check)
            t0 = time.perf_counter()
            res = pool.map(_oracle_sample, jobs)
            wall = time.perf_counter() - t0
    finally:
        for k, v in old.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    prods = sum(r[1] for r in res)
    cand = sum(r[2] for r in res)
    return prods / wall, wall, prods, cand, count


def cpu_blas_rate(T, cores, batch=4096, reps=3):
    """Products per second of 64 x 64 float64 leaf products by a host BLAS batch GEMM
    (torch.bmm on the CPU, `cores` threads), on stored tiles of X_0 taken in pairs."""
    import numpy as np
    import torch
    torch.set_num_threads(cores)
    g = np.random.default_rng(5)
    ia = g.integers(0, len(T), batch)
    ib = g.integers(0, len(T), batch)
    A = torch.from_numpy(np.ascontiguousarray(T[ia]))
    Bm = torch.from_numpy(np.ascontiguousarray(T[ib]))
    torch.bmm(A, Bm)
    t0 = time.perf_counter()
    for _ in range(reps):
        torch.bmm(A, Bm)
    dt = (time.perf_counter() - t0) / reps
    return batch / dt


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


# ---------------------------------------------------------------- peaks

def load_peaks():
    """MEASURED_PEAKS.json when present (peaks measured on this GPU model: a copy and
    a bf16 GEMM), else fixed fallback figures."""
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        p = json.load(open(path))
        return {"hbm_gbs": float(p["hbm_gbs"]), "bf16": float(p["bf16_tflops"]),
                "bf16_sustained": float(p["bf16_tflops_sustained"]), "source": "of measured"}
    return {"hbm_gbs": 6800.0, "bf16": 1900.0, "bf16_sustained": 1700.0, "source": "of fallback"}


# ----------------------------------------------------------- schedules

def first_step_delta(B, lmin, lmax, eps, n_iter, trace_x0):
    """delta_1 of the hybrid purification (the same scalar schedule the library follows:
    bounds h, l of X_0 widened by X_0's truncation, mapped by the first SP2 branch)."""
    w = lmax - lmin
    l = (lmax - B.homo) / w
    h = (lmax - B.lumo) / w
    budget = eps / (2.0 * math.sqrt(2.0) * n_iter)
    d0 = budget * (l - h)
    h, l = h + d0, l - d0
    if trace_x0 > B.n_occ:
        hn, ln = h * h, l * l
    else:
        hn, ln = 2 * h - h * h, 2 * l - l * l
    return budget * (ln - hn)


def oracle_multiplies(args, n_small=1024):
    """Multiplies of the oracle's own purification (Algorithm 5, the workload's eps and
    generator settings) of a small instance of the generator (n = 1024: 256 sites)."""
    import oracle
    import synth
    Bs = synth.lattice_fock_blocks(n_small, seed=synth.SEED_BASE + 4, decay=args.decay,
                                   cutoff=args.cutoff, bs=args.bs)
    r = oracle.purify(Bs.to_dense(), Bs.n_occ, args.eps, args.n_iter, Bs.homo, Bs.lumo,
                      variant=args.variant, bs=args.bs)
    return r.iters + (1 if r.converged else 0)


def x0_trace(B, lmin, lmax):
    import numpy as np
    w = lmax - lmin
    d = np.concatenate([np.diag(B.tiles[t]) for t in np.nonzero(B.brow == B.bcol)[0]])
    return float(np.sum((lmax - d) / w))


def candidate_products(B):
    """Leaf triples (i, k, j) with X_ik and X_kj stored: sum_k (column count)(row count)."""
    import numpy as np
    nb = B.n // B.bs
    rc = np.bincount(B.brow, minlength=nb).astype(np.float64)
    cc = np.bincount(B.bcol, minlength=nb).astype(np.float64)
    return float(np.sum(rc * cc))


# ---------------------------------------------------------------- arms

def run_reference(args, rank, world):
    """The oracle arm: the CPU oracle as it stands, timed on the host cores on bounded
    samples of the same workload (one process per core, each multiplying its own
    principal block of X_0 at the first step's SpAMM tolerance)."""
    if rank != 0:
        return 0
    import numpy as np
    B = make_lattice(args)
    lmin, lmax = gershgorin_blocks(B)
    T = x0_tiles(B, lmin, lmax)
    tr0 = x0_trace(B, lmin, lmax)
    delta1 = first_step_delta(B, lmin, lmax, args.eps, args.n_iter, tr0)
    cores = host_cores(args)
    mults = oracle_multiplies(args)
    cand = candidate_products(B)
    per_step = []
    for _ in range(args.warmup + args.steps):
        rate, wall, prods, scand, count = cpu_oracle_rate(B, T, 0.5 * delta1, cores,
                                                          args.sample_n)
        per_step.append((rate, wall, prods, scand))
    timed = per_step[args.warmup:]
    rate = sum(r[2] for r in timed) / sum(r[1] for r in timed)
    kept_frac = sum(r[2] for r in timed) / max(1.0, sum(r[3] for r in timed))
    # the oracle forms every kept product; per purification: the multiplies of the SP2
    # map on the certified spectral bounds, each with the candidates of X_0^2 times the
    # kept fraction of the samples
    products = mults * cand * kept_frac
    value_ms = products / rate * 1e3
    sample = (f"{cores} processes (one per core), each the oracle's spamm(X_s, X_s, delta_1/2) "
              f"with its tau search on its own {args.sample_n}x{args.sample_n} principal block of "
              f"X_0 ({timed[-1][2]} leaf products in {timed[-1][1]:.2f} s per step); extrapolated "
              f"to {mults} multiplies (the oracle's own purification of the n=1024 instance of "
              f"the same generator) x {cand:.3g} candidate products of X_0^2 x the samples' "
              f"kept fraction {kept_frac:.3f}")
    line = {"impl": "reference", "metric": METRIC, "value": value_ms, "unit": "ms",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": value_ms, "higher_is_better": False, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": config_of(args, world=world),
            "cpu_baseline": {"value": value_ms, "unit": "ms", "cores": cores, "kind": "oracle",
                             "sample": sample, "extrapolated": True,
                             "products_per_s": rate},
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
    t_gen = time.perf_counter()
    B = make_lattice(args)
    t_gen = time.perf_counter() - t_gen
    n, bs = args.n, args.bs
    F_tiles = torch.from_numpy(B.tiles).pin_memory()        # the step's input, pinned host
    stream = torch.cuda.Stream()
    ctx = sp.Context(local, stream=stream)
    ctx.set_bound(args.bound)
    if tau_table_config(args):
        ctx.set_tau_table(args.tau_start, args.tau_ratio)
    form = args.form
    if form == "auto":
        form = "mixed" if ctx.supports("mixed", bs) else "fp64"

    def step(d_buf):
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        F = ctx.from_blocks(n, bs, B.brow, B.bcol, F_tiles)    # H2D of the step's input
        e[1].record(stream)
        D, rep = ctx.purify(F, B.n_occ, args.eps, args.n_iter, B.homo, B.lumo,
                            variant=args.variant, prec=form, strict=False)
        e[2].record(stream)
        nnzb_d = D.nnzb
        if d_buf is not None:
            D.to_blocks(d_buf)                                  # D2H of the step's result
        e[3].record(stream)
        del F
        return e, rep, D, nnzb_d

    D = None
    nnzb_max = 0
    for _ in range(args.warmup):
        D = None
        e, rep, D, nd = step(None)
        nnzb_max = max(nnzb_max, nd)
    torch.cuda.synchronize()
    cap = int(max(nnzb_max, len(B.brow)) * 1.5) + 16    # D's blocks (warm-up: the largest seen)
    d_buf = torch.empty(cap * bs * bs, dtype=torch.float64).pin_memory()
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
    evs, reps, d_bytes = [], [], []
    for _ in range(args.steps):
        D = None
        e, rep, D, nd = step(d_buf)
        evs.append(e)
        reps.append(rep)
        d_bytes.append(nd * bs * bs * 8)
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
    rep0 = reps[-1]
    line = {"metric": METRIC, "value": value, "unit": "ms", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": False, "scaling": "weak", "vs_baseline": None,
            "dtype": "f64" if form == "fp64" else "bf16 slices (f32 accumulate) -> f64",
            "data": "synthetic", "config": dict(config_of(args, world=world), form=form)}
    line.update(purification_summary(args, B, reps, rep0, form))
    line["e2e"] = {"value": e2e, "unit": "ms",
                   "h2d_bytes_per_step": int(B.tiles.nbytes + 8 * len(B.brow)),
                   "d2h_bytes_per_step": int(max(d_bytes)) + 8 * int(max(d_bytes)) // (bs * bs * 8)}
    line["clocks"] = clk
    line["gpu_launches"] = launches
    line["input_generation_s"] = round(t_gen, 1)
    del F_tiles, d_buf
    T0 = None
    if rank == 0 and world == 1 and not (args.no_extras and args.no_cpu_baseline):
        T0 = x0_tiles(B, rep0["lmin"], rep0["lmax"])
    if rank == 0 and world == 1 and not args.no_extras:
        line["extras"] = run_extras(args, ctx, B, T0, D, form)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line.update(cpu_baselines(args, B, T0, reps, rep0))
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


# DRAM bytes of the leaf-product kernel per issued slice-pair flop: one ncu capture of
# both passes of the third SP2 product of the n = 65536 lattice (levels 6..9: 39.29 +
# 4.55 GB read + written, levels 2..5: 13.47 + 9.03 GB; 66.34 GB), over that run's
# average pipe flops per product (796.7 TFLOP/s x 387.9 ms / 13 products = 2.377e13)
GEMM_DRAM_BYTES_PER_PIPE_FLOP = 66.34e9 / 2.377e13


def purification_summary(args, B, reps, rep0, form):
    """The roofline of the dominant kernel, the phase split, the step logs and the
    checks of one bench configuration's purifications."""
    bs = args.bs
    K = len(reps)
    kept = sum(r["kept_total"] for r in reps)
    formed = sum(r["formed_total"] for r in reps)
    pipe = sum(r["pipe_flops_total"] for r in reps)
    cand = sum(r["cand_total"] for r in reps)
    gemm_ms = sum(r["ms_phase"][3] for r in reps)
    n_mult = sum(r["iters"] + (1 if r["converged"] else 0) for r in reps)
    peaks = load_peaks()
    if form == "fp64":
        # 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz (GB300's nominal 1.26 TFLOP/s FP64)
        roof = {"bound": "alu", "kernel": "k_gemm_fp64", "peak": 1.26, "unit": "TFLOP/s",
                "peak_source": "derived: 152 SMs x 2 FP64 FMA/clk x 2 flop x 2.07 GHz",
                "algorithmic": "2*bs^3 flop per formed leaf product"}
    else:
        roof = {"bound": "tensor", "kernel": "k_gemm_tile", "peak": peaks["bf16_sustained"],
                "unit": "TFLOP/s",
                "peak_source": f"bf16 sustained {peaks['source']} (timed inside a long step)",
                "algorithmic": "2*128*128*64 flop per (p,q) bf16 slice pair of a 128x128 tile "
                               "task (4 MMAs of 128x128x16)"}
    achieved = pipe / (gemm_ms * 1e-3) / 1e12 if gemm_ms > 0 else 0.0
    traffic = None
    if form != "fp64":
        # DRAM bytes of the leaf-product kernel per issued slice-pair flop, from one
        # ncu capture of both passes of an SP2 product of the n = 65536 lattice; the
        # bytes are the pair tiles copied, so they grow with the pairs formed, and the
        # figure is scaled to this run's average launch by its pipe flops
        passes = lambda L: 1 + (L >= 6) + (L >= 10)
        launches = sum(sum(passes(L) for L in r["step_lmax"]) + passes(r["step_lmax"][-1])
                       for r in reps if r["step_lmax"])
        if launches and GEMM_DRAM_BYTES_PER_PIPE_FLOP is not None:
            traffic = GEMM_DRAM_BYTES_PER_PIPE_FLOP * pipe / launches
    roof.update({"achieved": achieved, "frac": achieved / roof["peak"], "traffic": traffic,
                 "traffic_unit": "bytes per launch (average launch)"})
    nb2 = (B.n // bs) ** 2
    phase = lambda q: sum(r["ms_phase"][q] for r in reps) / K
    return {
        "spamm_ms": sum(r["ms_phase"][1] + r["ms_phase"][2] + r["ms_phase"][3] + r["ms_phase"][5]
                        for r in reps) / max(1, n_mult),
        "iters": rep0["iters"], "converged": rep0["converged"],
        "step_slice_levels": rep0["step_lmax"],
        "step_fill_pct": [round(100.0 * z / nb2, 3) for z in rep0["nnzb"]],
        "input_fill_pct": round(100.0 * len(B.brow) / nb2, 3),
        "check": {"trace_minus_n_occ": rep0["trace"] - B.n_occ, "idem_estimate": rep0["idem"],
                  "eps": args.eps, "converged": rep0["converged"]},
        "phase_ms": {"cse": phase(1), "plan": phase(2), "leaf_products": phase(3),
                     "truncation": phase(4), "split": phase(5)},
        "candidates_per_step": cand / K,
        "kept_products_per_step": kept / K,
        "formed_products_per_step": formed / K,
        "useful_tflops_f64_equivalent": (2.0 * bs ** 3 * kept / (gemm_ms * 1e-3) / 1e12
                                         if gemm_ms > 0 else 0.0),
        "roofline": roof,
    }


def sampled_diff(A, Bm, nb, rng, count=48):
    """max over sampled blocks of ||A_ij - B_ij||_F: blocks stored in A plus random
    ones near the diagonal (a check, not a step of the path)."""
    import numpy as np
    brow, bcol, _ = A.to_blocks()
    pick = rng.integers(0, len(brow), count // 2)
    qi = list(brow[pick]) + list(rng.integers(0, nb, count // 2))
    qj = list(bcol[pick]) + [min(nb - 1, max(0, int(i) + int(d)))
                             for i, d in zip(qi[count // 2:], rng.integers(-8, 9, count // 2))]
    qi = np.array(qi, dtype=np.int32)
    qj = np.array(qj, dtype=np.int32)
    ta, _ = A.get_blocks(qi, qj)
    tb, _ = Bm.get_blocks(qi, qj)
    return float(max(np.linalg.norm(ta[q] - tb[q]) for q in range(len(qi))))


def timed_call(fn, reps=2):
    """Run fn() reps times (the first warms the search hints and the pools); return the
    last result and its wall time in ms."""
    out = None
    ms = 0.0
    for _ in range(reps):
        out = None
        t0 = time.perf_counter()
        out = fn()
        ms = (time.perf_counter() - t0) * 1e3
    return out, ms


def run_extras(args, ctx, B, T0, D_main, form):
    """One-off measurements after the timed steps (each also timed by the library's
    CUDA events, which the report carries)."""
    import numpy as np
    import torch

    import synth
    out = {}
    bs = args.bs
    nb = B.n // bs
    # the configuration's SpAMM half: X_0 X_0 with the tau search at delta, both forms
    X0 = ctx.from_blocks(B.n, bs, B.brow, B.bcol, T0)
    out["spamm_x0"] = {"delta": args.spamm_delta}
    for prec in ("mixed", "fp64"):
        (C, rep), wall = timed_call(lambda: ctx.multiply(X0, X0, args.spamm_delta, prec=prec))
        out["spamm_x0"][prec] = {"ms": rep["ms"][6], "wall_ms": wall, "tau": rep["tau"],
                                 "tau_index": rep["tau_index"], "bound": rep["bound"],
                                 "bound_round": rep["bound_round"], "lmax": rep["lmax"],
                                 "candidates": rep["candidates"], "kept": rep["kept"],
                                 "formed": rep["formed"], "nnzb_out": rep["nnzb_out"],
                                 "phase_ms": {"split": rep["ms"][5], "cse": rep["ms"][1],
                                              "plan": rep["ms"][2], "leaf_products": rep["ms"][3]}}
        del C
    del X0
    # the same purification in the float64 form, and how far its D is from the mixed one
    F = ctx.from_blocks(B.n, bs, B.brow, B.bcol, B.tiles)
    D64, r64 = ctx.purify(F, B.n_occ, args.eps, args.n_iter, B.homo, B.lumo,
                          variant=args.variant, prec="fp64", strict=False)
    del F
    diff = sampled_diff(D_main, D64, nb, np.random.default_rng(7))
    out["fp64_form"] = {"ms_per_purification": r64["ms_total"], "iters": r64["iters"],
                        "converged": r64["converged"],
                        "trace_minus_n_occ": r64["trace"] - B.n_occ,
                        "phase_ms": {"cse": r64["ms_phase"][1], "plan": r64["ms_phase"][2],
                                     "leaf_products": r64["ms_phase"][3],
                                     "truncation": r64["ms_phase"][4]},
                        "max_sampled_block_diff_vs_" + form: diff,
                        "diff_bound": 2 * args.eps}
    del D64
    # the single SpAMM product of the n = 2048 banded configuration (float64, leaf 32)
    Xb = synth.banded_decay(2048, synth.SEED_BASE + 0, length=40.0, drop=1e-12)
    Gb = ctx.from_dense(Xb, bs=32)
    (C, rep), wall = timed_call(lambda: ctx.multiply(Gb, Gb, 1e-6, prec="fp64"), reps=3)
    out["spamm_n2048_bs32"] = {"ms": rep["ms"][6], "wall_ms": wall, "tau": rep["tau"],
                               "bound": rep["bound"], "kept": rep["kept"],
                               "err_vs_dense": float(np.linalg.norm(C.to_numpy() - Xb @ Xb))}
    del C, Gb
    # the n = 16384 dense lattice purification (the configuration measured before)
    P = make_dense_problem(16384, use_gpu_eigh=True)
    Fd = ctx.from_dense(torch.from_numpy(P.F), bs=64)
    Dd, rd = ctx.purify(Fd, P.n_occ, args.eps, args.n_iter, P.homo, P.lumo,
                        variant=args.variant, prec=form, strict=False)
    del Fd
    Dt = Dd.to_torch()
    Vo = torch.from_numpy(P.occupied).cuda()
    Dt -= Vo @ Vo.T
    out["dense_n16384"] = {"workload": S2_WORKLOAD, "form": form,
                           "ms_per_purification": rd["ms_total"], "iters": rd["iters"],
                           "d_minus_exact_fro": float(torch.linalg.norm(Dt))}
    del Dt, Vo, Dd
    torch.cuda.empty_cache()
    return out


def cpu_baselines(args, B, T0, reps, rep0):
    """The CPU oracle on all host cores and a host-BLAS leaf-product rate, each scaled to
    one purification of the workload by the GPU run's own product counts."""
    cores = host_cores(args)
    kept = sum(r["kept_total"] for r in reps) / len(reps)
    cand = sum(r["cand_total"] for r in reps) / len(reps)
    delta1 = rep0["deltas"][0] if rep0["deltas"] else args.spamm_delta
    rate, wall, prods, scand, count = cpu_oracle_rate(B, T0, 0.5 * delta1, cores, args.sample_n)
    blas = cpu_blas_rate(T0, cores)
    return {
        "cpu_baseline": {
            "value": kept / rate * 1e3, "unit": "ms", "cores": count, "kind": "oracle",
            "extrapolated": True, "products_per_s": rate,
            "sample": (f"{count} processes (one per core), each the oracle's spamm(X_s, X_s, "
                       f"delta_1/2) with its tau search on its own {args.sample_n}x"
                       f"{args.sample_n} principal block of X_0: {prods} leaf products in "
                       f"{wall:.2f} s; scaled by the {kept:.4g} leaf products one purification "
                       f"keeps")},
        "cpu_blas": {
            "value": cand / blas * 1e3, "unit": "ms", "cores": cores,
            "kind": "host BLAS truncmul leaf products (torch.bmm float64, 64x64)",
            "products_per_s": blas,
            "sample": (f"4096 leaf products of stored X_0 tiles per batch; scaled by the "
                       f"{cand:.4g} candidate products of one purification (truncmul forms "
                       f"all of them)")},
    }


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
        out["removed_sq"] = tr["removed_sq"]
    out["nnzb_out"] = Y.nnzb
    return Y, out


def fro_diff(A, B):
    """||A - B||_F of two device matrices, read back densely (a check, not a step of
    the path)."""
    import torch
    a, b = A.to_torch(), B.to_torch()
    a -= b
    del b
    d = float(torch.linalg.norm(a))
    del a
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
                            "X_out": 100.0 * out.pop("nnzb_out") / nb2,
                            "exact_square": 100.0 * exact.nnzb / nb2},
                "err": err, "err_over_delta": err / delta})
    if spectral:
        err2 = norm2_diff(X2, exact)
        out.update({"err_2": err2, "err_2_over_delta": err2 / delta})
    return out


def run_protocol(args):
    import torch

    import paper_2005_10680_gb300 as sp
    torch.cuda.set_device(0)
    B = make_lattice(args, n=args.protocol_n)
    stream = torch.cuda.Stream()
    ctx = sp.Context(0, stream=stream)
    fastest = "mixed" if ctx.supports("mixed", args.bs) else "fp64"
    F = ctx.from_blocks(B.n, args.bs, B.brow, B.bcol, B.tiles)
    D, rep = ctx.purify(F, B.n_occ, args.eps, args.n_iter, B.homo, B.lumo,
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
                        "n": B.n, "bs": args.bs, "decay": args.decay, "cutoff": args.cutoff,
                        "D": f"SP2 purification (Algorithm {args.variant}, {fastest}) of the "
                             f"block-sparse lattice Fock matrix (n {B.n}, decay {args.decay}, "
                             f"cutoff {args.cutoff}), eps {args.eps}, {rep['iters']} iterations"}
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
