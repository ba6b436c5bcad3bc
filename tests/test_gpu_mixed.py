"""Mixed form (bf16 tensor-core slices, exact f32 accumulation, charged
slicing error) against the oracle and the float64 form, through the C ABI.

Bars: the certified bound covers the true error (||C - AB||_F <= bound, with
the slicing charge included); ||C - AB||_F < delta when delta is given; the
result agrees with the float64 oracle well inside the bound; products of
integer matrices come out bit-exact; SP2 steps stay exactly symmetric; the
purification reaches ||D - D~||_F < eps."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def gctx():
    import paper_2005_10680_gb300 as sp
    ctx = sp.Context(0)
    if not ctx.supports("mixed", 64):
        pytest.fail("mixed-precision leaf products are not available on this device")
    return ctx


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


@pytest.mark.parametrize("n,seed", [(128, 1), (320, 2), (1000, 3)])
def test_integer_products_are_exact(gctx, n, seed):
    g = synth.rng(seed)
    A = g.integers(-100, 101, size=(n, n)).astype(np.float64)
    B = g.integers(-100, 101, size=(n, n)).astype(np.float64)
    C, rep = gctx.multiply_tau(gctx.from_dense(A, 64), gctx.from_dense(B, 64), 0.0, prec="mixed")
    assert rep["lmax"] == 10
    np.testing.assert_array_equal(C.to_numpy(), A @ B)


@pytest.mark.parametrize("n,kind,seed", [(256, "band", 4), (448, "rand", 5), (1000, "lattice", 6)])
def test_mixed_tau_within_bound_and_close_to_oracle(gctx, orc, n, kind, seed):
    if kind == "band":
        A = synth.banded_decay(n, seed, length=n / 10.0)
        B = A
    elif kind == "rand":
        A = synth.random_decaying(n, seed, length=n / 12.0)
        B = synth.random_decaying(n, seed + 1, length=n / 9.0)
    else:
        A = synth.lattice_fock(n, seed=seed, gap_mode="stagger").F / 100.0
        B = A
    GA, GB = gctx.from_dense(A, 64), gctx.from_dense(B, 64)
    taus = orc.tau_table()
    # float64 rounding of the reference products themselves is not part of the
    # certified bound (neither the paper nor the float64 form charges it): allow
    # u * ||A||_F ||B||_F * sqrt(n) for it
    fp64_noise = 1.12e-16 * np.linalg.norm(A) * np.linalg.norm(B) * np.sqrt(n)
    for k in (40, 120, 349):
        tau = float(taus[k])
        C, rep = gctx.multiply_tau(GA, GB, tau, prec="mixed")
        Cf, repf = gctx.multiply_tau(GA, GB, tau, prec="fp64")
        ref, _ = orc.spamm(A, B, tau, 64)
        c = C.to_numpy()
        err = np.linalg.norm(c - A @ B)
        assert err <= rep["bound"] + fp64_noise
        # the mixed form forms every stored product of a 2 x 2 block tile once one of
        # them reaches tau, so it skips a subset of what the float64 form (and the
        # oracle) skip: both lie within their bounds of A B
        both = rep["bound"] + repf["bound"] + 2 * fp64_noise
        assert np.linalg.norm(c - Cf.to_numpy()) <= both
        assert np.linalg.norm(c - ref) <= both
        assert rep["kept"] == repf["kept"]
        assert rep["formed"] >= repf["formed"]
        # the charge-only bound (everything formed) is the bound's floor
        assert rep["bound"] >= rep["bound_round"] > 0


@pytest.mark.parametrize("n,delta", [(512, 1e-6), (768, 1e-9), (1024, 1e-11)])
def test_mixed_delta_certified(gctx, orc, n, delta):
    X = synth.banded_decay(n, 77, length=n / 8.0, drop=1e-14)
    X *= 10.0 / np.linalg.norm(X)          # ||X||_F = 10: float64 noise of X X stays << delta
    fp64_noise = 1.12e-16 * 100.0 * np.sqrt(n)
    G = gctx.from_dense(X, 64)
    C, rep = gctx.multiply(G, G, delta, prec="mixed")
    exact = X @ X
    c = C.to_numpy()
    assert rep["bound"] < delta
    assert np.linalg.norm(c - exact) < delta + fp64_noise
    assert rep["lmax"] >= 2
    Cf, repf = gctx.multiply(G, G, delta, prec="fp64")
    # the mixed form forms whole 2 x 2 tiles and charges its slicing, so it may need a
    # few table entries more (or many fewer) than the float64 form
    assert rep["tau_index"] <= repf["tau_index"] + 8


@pytest.mark.parametrize("branch", [0, 1])
def test_mixed_sp2_step_symmetric(gctx, orc, branch):
    P = synth.lattice_fock(640, seed=21, gap_mode="eig")
    lmin, lmax = orc.gershgorin(P.F)
    X = (lmax * np.eye(640) - P.F) / (lmax - lmin)
    G = gctx.from_dense(X, 64)
    Xn, rep = gctx.sp2_step(G, branch, delta=1e-10, prec="mixed")
    got = Xn.to_numpy()
    np.testing.assert_array_equal(got, got.T)
    want = X @ X if branch == 0 else 2 * X - X @ X
    assert np.linalg.norm(got - want) < 1e-10
    assert rep["bound"] < 1e-10


@pytest.mark.parametrize("variant,gap_mode,n", [(5, "eig", 512), (4, "stagger", 640), (1, "eig", 384)])
def test_mixed_purify_matches_eigendecomposition(gctx, orc, variant, gap_mode, n):
    P = synth.lattice_fock(n, seed=8, gap_mode=gap_mode)
    eps = 1e-5
    D, rep = gctx.purify(gctx.from_dense(P.F, 64), P.n_occ, eps, 60, P.homo, P.lumo,
                         variant=variant, prec="mixed")
    Dx = orc.exact_density(P.F, P.n_occ)
    got = D.to_numpy()
    assert rep["converged"]
    assert np.linalg.norm(got - Dx) < eps
    np.testing.assert_array_equal(got, got.T)
    Df, repf = gctx.purify(gctx.from_dense(P.F, 64), P.n_occ, eps, 60, P.homo, P.lumo,
                           variant=variant, prec="fp64")
    assert abs(rep["iters"] - repf["iters"]) <= 1
    assert np.linalg.norm(got - Df.to_numpy()) < eps


def test_eleventh_level_when_ten_cannot_certify(gctx, orc):
    # delta just above the level-10 charge: level 10 no longer fits in half of delta,
    # so the search forms level 11 (second pass) and still certifies delta
    n = 1024
    P = synth.lattice_fock(n, seed=41, gap_mode="stagger")
    lmin, lmax = orc.gershgorin(P.F)
    X = (lmax * np.eye(n) - P.F) / (lmax - lmin)
    G = gctx.from_dense(X, 64)
    C10, r10 = gctx.multiply_tau(G, G, 0.0, prec="mixed")
    assert r10["lmax"] == 10 and r10["bound_round"] > 0
    delta = 1.2 * r10["bound_round"]
    C, rep = gctx.sp2_step(G, 0, delta=delta, prec="mixed")
    assert rep["lmax"] == 11
    assert rep["bound_round"] < 0.1 * r10["bound_round"]
    assert rep["bound"] < delta
    # both products are integers rounded once or twice to float64 at the end: each
    # is within its bound of X X, up to two roundings of the output
    c10 = C10.to_numpy()
    out_round = 2.3e-16 * np.linalg.norm(c10)
    assert np.linalg.norm(C.to_numpy() - c10) <= rep["bound"] + r10["bound"] + 2 * out_round


@pytest.mark.parametrize("n", [50, 100, 130])
def test_mixed_small_and_ragged_grids(gctx, n):
    # one, two and three leaf blocks per side (the last one ragged): pair and tile
    # halves beyond the grid are empty
    g = synth.rng(n)
    A = g.integers(-50, 51, size=(n, n)).astype(np.float64)
    B = g.integers(-50, 51, size=(n, n)).astype(np.float64)
    C, rep = gctx.multiply_tau(gctx.from_dense(A, 64), gctx.from_dense(B, 64), 0.0, prec="mixed")
    np.testing.assert_array_equal(C.to_numpy(), A @ B)
    X = synth.banded_decay(n, n, length=n / 6.0)
    Y, yrep = gctx.sp2_step(gctx.from_dense(X, 64), 1, delta=1e-9, prec="mixed")
    y = Y.to_numpy()
    np.testing.assert_array_equal(y, y.T)
    noise = 1.12e-16 * np.linalg.norm(X) ** 2 * np.sqrt(n)
    assert np.linalg.norm(y - (2 * X - X @ X)) <= yrep["bound"] + noise
    assert yrep["bound"] < 1e-9


def test_mixed_zero_and_everything_skipped(gctx):
    n = 200
    Z = gctx.from_dense(np.zeros((n, n)), 64)
    C, rep = gctx.multiply(Z, Z, 1e-8, prec="mixed")
    assert rep["nnzb_out"] == 0 and rep["bound"] == 0.0 and not C.to_numpy().any()
    X = synth.banded_decay(n, 11, length=10.0)
    G = gctx.from_dense(X, 64)
    # tau above every norm product: nothing is formed; the 2X - X^2 branch keeps 2X
    C, rep = gctx.sp2_step(G, 1, tau=1e6, prec="mixed")
    assert rep["formed"] == 0
    np.testing.assert_array_equal(C.to_numpy(), 2 * X)
