"""bench.py's options on the CPU: the default run keeps the paper's candidate list and
Algorithm 3, the spectral bound is accepted only for the two-squares protocol (the
purification keeps a Frobenius guarantee), and a tuned list is recorded in the
JSON line's config."""
import pytest

import bench


def test_defaults_are_the_papers():
    args = bench.parse([])
    assert args.bound == "alg3" and bench.tau_table_config(args) is None
    assert args.n == 16384 and args.bs == 64 and args.eps == 1e-5


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
