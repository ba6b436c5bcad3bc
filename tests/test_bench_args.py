"""bench.py's options on the CPU: the default run keeps the paper's candidate list and
Algorithm 3, the spectral bound is accepted only for the two-squares protocol (the
purification keeps a Frobenius guarantee), and a tuned list is recorded in the
JSON line's config."""
import pytest

import bench


def test_defaults_are_the_papers():
    args = bench.parse([])
    assert args.bound == "alg3" and bench.tau_table_config(args) is None
    assert args.n == 262144 and args.bs == 64 and args.eps == 1e-5 and args.spamm_delta == 1e-7


def test_spectral_bound_only_with_the_protocol():
    with pytest.raises(SystemExit):
        bench.parse(["--bound", "spectral"])
    args = bench.parse(["--protocol", "--bound", "spectral"])
    assert args.bound == "spectral"


def test_tuned_list_options():
    args = bench.parse(["--tau-start", "8"])
    assert bench.tau_table_config(args) == {"start": 8.0, "ratio": 0.9, "length": 350}
    args = bench.parse(["--tau-ratio", "0.95"])
    assert bench.tau_table_config(args) == {"start": 1.0, "ratio": 0.95, "length": 350}


def test_reference_arm_line_on_a_small_case():
    """The oracle arm's JSON line (run on the CPU, rank 0): impl, the arm's metric and
    unit, a cpu_baseline describing the sample, and an e2e entry with no copies."""
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    flags = ["--n", "4096", "--sample-n", "1024", "--cores", "2", "--steps", "1", "--warmup", "0"]
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference",
                          *flags], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads(out.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["metric"] == bench.METRIC
    assert line["unit"] == "ms" and line["higher_is_better"] is False and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 2
    # the same config as the GPU arm's line for the same flags
    assert line["config"] == bench.config_of(bench.parse(flags))
    assert line["cpu_baseline"]["value"] == line["value"] and line["cpu_baseline"]["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": "ms", "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}


def test_purification_summary_roofline_on_a_synthetic_report():
    """The roofline block of the JSON line from purification reports (no GPU): the
    achieved rate is the issued pipe flops over the leaf-product phase, the traffic
    is the per-flop DRAM figure spread over the kernel launches (one per slice-level
    pass: 6..9, 10..L and 2..5), and every phase is averaged over the purifications."""
    import types
    args = bench.parse(["--n", "4096", "--steps", "2"])
    B = types.SimpleNamespace(n=4096, brow=[0] * 100, n_occ=2048)
    rep = {"kept_total": 10, "formed_total": 8, "pipe_flops_total": 4.0e12, "cand_total": 20,
           "ms_phase": [0.0, 5.0, 3.0, 2000.0, 1.0, 7.0, 2016.0, 0.0], "iters": 3,
           "converged": 1, "step_lmax": [10, 9, 5], "nnzb": [100, 90, 80], "trace": 2048.0,
           "idem": 1e-7, "deltas": [1e-8]}
    out = bench.purification_summary(args, B, [rep, dict(rep)], rep, "mixed")
    roof = out["roofline"]
    assert roof["achieved"] == pytest.approx(4.0e12 * 2 / 4.0 / 1e12)   # 2 TFLOP/s
    assert roof["frac"] == pytest.approx(roof["achieved"] / roof["peak"])
    assert out["phase_ms"]["leaf_products"] == 2000.0 and out["phase_ms"]["cse"] == 5.0
    if bench.GEMM_DRAM_BYTES_PER_PIPE_FLOP is None:
        assert roof["traffic"] is None
    else:
        # passes: L = 10 -> 3, 9 -> 2, 5 -> 1, plus the converging multiply at L = 5 -> 1
        assert roof["traffic"] == pytest.approx(
            bench.GEMM_DRAM_BYTES_PER_PIPE_FLOP * 8.0e12 / (2 * 7))
    f64 = bench.purification_summary(args, B, [rep], rep, "fp64")
    assert f64["roofline"]["bound"] == "alu" and f64["roofline"]["traffic"] is None
