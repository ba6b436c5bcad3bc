"""Pins for the mixed form's arithmetic model (oracle/mixed_ref.py), on the CPU.

The mixed form is this implementation's own way of forming leaf products: exact
fixed-point digit slices multiplied on the tensor cores, with the digits it leaves
out charged inside the Algorithm 3 bound. These tests tie its model to exact
arithmetic (Python integers and fractions): the rounding to fixed point, the
balanced digits, the bound on one level's sum that keeps the f32 accumulators
exact, and the charge that must bound the error of every product formed to a
level L. Mutated charges (a dropped term, an index off by one) must fail."""
import itertools
import math
from fractions import Fraction

import numpy as np
import pytest

from oracle import mixed_ref as mr


def _round_half_away(q: Fraction) -> int:
    a = abs(q)
    v = math.floor(a + Fraction(1, 2))
    return v if q >= 0 else -v


def _awkward(rng, n):
    """Entries that exercise the rounding: halfway cases, powers of two, subnormals,
    negative values, an all-zero row and a row of wide dynamic range."""
    X = rng.standard_normal((n, n))
    X[0, :] = 0.0
    X[1, :3] = [1.0, -0.5, 2.0 ** -70]
    X[2, :] = np.ldexp(rng.standard_normal(n), rng.integers(-60, 5, n))
    X[3, :4] = [5e-324, -1e-310, 3.0, -2.0 ** 40]
    # halfway cases: the row exponent is 0, so the unit is 2^-63 and 2^-63 + 2^-64 is
    # one and a half units
    X[4, :] = 0.0
    X[4, :3] = [0.75, 2.0 ** -63 + 2.0 ** -64, -(2.0 ** -63 + 2.0 ** -64)]
    return X


def test_fixed_point_is_exact_rounding():
    rng = np.random.default_rng(11)
    X = _awkward(rng, 12)
    e = mr.exponents(X, axis=1)
    V, r = mr.fixed_point(X, e)
    for i, j in itertools.product(range(X.shape[0]), range(X.shape[1])):
        x = Fraction(float(X[i, j]))
        amax = max(abs(Fraction(float(v))) for v in X[i])
        # the exponent: max |X[i, :]| < 2^e (0 for a zero row), and the least such e
        if amax:
            assert amax < Fraction(2) ** int(e[i]) and amax >= Fraction(2) ** (int(e[i]) - 1)
        else:
            assert e[i] == 0
        q = x * Fraction(2) ** (63 - int(e[i]))
        assert int(V[i, j]) == _round_half_away(q), (i, j)
        assert Fraction(float(r[i, j])) == q - int(V[i, j]), (i, j)
        # the row maximum scales exactly to at most (2^53 - 1) 2^10, so the rounding
        # of any entry stays at or below it: the digit recurrence cannot overflow
        assert abs(int(V[i, j])) <= 2 ** 63 - 2 ** 10


def test_halfway_rounds_away_from_zero():
    X = np.zeros((1, 3))
    X[0] = [0.75, 2.0 ** -63 + 2.0 ** -64, -(2.0 ** -63 + 2.0 ** -64)]
    e = mr.exponents(X, axis=1)
    assert e[0] == 0
    V, r = mr.fixed_point(X, e)
    assert V[0, 1] == 2 and V[0, 2] == -2          # 1.5 units -> 2, -1.5 -> -2
    assert r[0, 1] == -0.5 and r[0, 2] == 0.5


def test_digits_reconstruct_and_stay_in_range():
    import torch
    rng = np.random.default_rng(12)
    vmax = 2 ** 63 - 2 ** 10           # largest |V| the fixed-point rounding produces
    V = np.concatenate([rng.integers(-vmax, vmax, 4000, dtype=np.int64, endpoint=True),
                        np.array([0, 1, -1, 63, 64, -64, -65, 2 ** 62, -(2 ** 62),
                                  vmax, -vmax], dtype=np.int64)])
    d = mr.digits(V)
    for t in range(V.size):
        assert sum(int(d[p, t]) * 128 ** (mr.S - 1 - p) for p in range(mr.S)) == int(V[t])
    # digits 2..9 in [-64, 63] make the representation unique (V mod 128^k fixes them)
    assert d[1:].min() >= -64 and d[1:].max() <= 63
    assert np.abs(d[0]).max() <= 128
    # every digit is exact in bf16
    bf = torch.from_numpy(d.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(bf, d.astype(np.float64))


def test_slices_and_tails_add_up():
    rng = np.random.default_rng(13)
    X = _awkward(rng, 16)
    for by_rows in (True, False):
        Sx = mr.Sliced(X, by_rows)
        e = Sx.e
        for i, j in itertools.product(range(16), range(16)):
            x = Fraction(float(X[i, j]))
            ee = int(e[i] if by_rows else e[j])
            parts = [Fraction(int(Sx.d[p - 1, i, j])) * Fraction(2) ** (ee - 7 * p)
                     for p in range(1, mr.S + 1)]
            for p in range(0, mr.S + 1):
                exact_tail = x - sum(parts[:p], Fraction(0))
                got = Fraction(float(Sx.tail(p)[i, j]))
                # the tail is formed in float64 from an exact integer residue
                assert abs(got - exact_tail) <= abs(exact_tail) * Fraction(1, 2 ** 52), (p, i, j)
            # the last tail is the rounding to fixed point alone: at most half a unit
            assert abs(x - sum(parts, Fraction(0))) <= Fraction(2) ** (ee - 64)


def _level_max(L: int) -> int:
    """max over digits within their ranges of |sum_{p+q=L} d_p d_q| summed over K = 64."""
    mx = [128] + [64] * (mr.S - 1)
    s = sum(mx[p - 1] * mx[L - p - 1] for p in range(1, mr.S + 1) if 1 <= L - p <= mr.S)
    return 64 * s


@pytest.mark.parametrize("L", range(2, 2 * mr.S + 1))
def test_one_level_sum_bound_keeps_f32_exact(L):
    cap = 2 ** 18 * max(L + 1, 4)
    assert _level_max(L) <= cap
    # a window of w leaf products per f32 accumulator, for a pass whose top level is hi
    for hi in range(max(L, 4), 2 * mr.S + 1):
        w = (2 ** 24 - 1) // (2 ** 18 * max(hi + 1, 4))
        assert w >= 1
        assert w * _level_max(L) <= 2 ** 24 - 1
    # the worst case is reached: all digits at their extremes
    dA = np.array([128] + [64] * (mr.S - 1), dtype=np.int64)
    dB = np.array([128] + [64] * (mr.S - 1), dtype=np.int64)
    g = sum(int(dA[p - 1] * dB[L - p - 1]) for p in range(1, mr.S + 1) if 1 <= L - p <= mr.S)
    assert 64 * g == _level_max(L)


def _case(kind, rng, n=128):
    if kind == "normal":
        return rng.standard_normal((n, n)), rng.standard_normal((n, n))
    if kind == "decay":
        i = np.arange(n)
        D = np.exp(-np.abs(i[:, None] - i[None, :]) / 6.0)
        return D * rng.standard_normal((n, n)), D.T * rng.standard_normal((n, n))
    if kind == "wide_rows":
        A = rng.standard_normal((n, n)) * np.ldexp(1.0, rng.integers(-40, 40, n))[:, None]
        B = rng.standard_normal((n, n)) * np.ldexp(1.0, rng.integers(-40, 40, n))[None, :]
        A[5, :] = 0.0
        B[:, 7] = 0.0
        return A, B
    if kind == "wide_entries":
        A = np.ldexp(rng.standard_normal((n, n)), rng.integers(-30, 1, (n, n)))
        B = np.ldexp(rng.standard_normal((n, n)), rng.integers(-30, 1, (n, n)))
        return A, B
    if kind == "a_exact":      # A is its first slice: small integers, every tail zero
        return rng.integers(-100, 101, (n, n)).astype(np.float64), rng.standard_normal((n, n))
    if kind == "b_exact":
        return rng.standard_normal((n, n)), rng.integers(-100, 101, (n, n)).astype(np.float64)
    raise ValueError(kind)


KINDS = ["normal", "decay", "wide_rows", "wide_entries", "a_exact", "b_exact"]
LEVELS = [2, 3, 4, 5, 6, 8, 10, 11, 12, 14]
BS = 64


def _charged_errors(A, B, charge_fn):
    """(error, charge) of every block triple (I, K, J) and level in LEVELS, each
    product's error measured exactly; slices use whole-row (column) exponents."""
    SA, SB = mr.Sliced(A, True), mr.Sliced(B, False)
    nb = A.shape[0] // BS
    out = []
    for I, K, J in itertools.product(range(nb), repeat=3):
        rI, rK, rJ = (slice(x * BS, (x + 1) * BS) for x in (I, K, J))
        P, k = mr.exact_product(A[rI, rK], B[rK, rJ])
        snA, tnA = SA.slice_norms(rI, rK), SA.tail_norms(rI, rK)
        tnB = SB.tail_norms(rK, rJ)
        nB = float(np.linalg.norm(B[rK, rJ]))
        for L in LEVELS:
            G, s = mr.level_sum(SA, SB, L, rI, rK, rJ)
            out.append((mr.diff_norm(G, s, P, k), charge_fn(snA, tnA, tnB, nB, L), L))
    return out


@pytest.mark.parametrize("kind", KINDS)
def test_charge_bounds_every_formed_product(kind):
    rng = np.random.default_rng(100 + KINDS.index(kind))
    A, B = _case(kind, rng)
    for err, c, L in _charged_errors(A, B, mr.charge):
        # tail norms carry a float64 rounding of 2^-52 relative; nothing else is inexact
        assert err <= c * (1 + 1e-12), (kind, L, err, c)


@pytest.mark.parametrize("kind", ["a_exact", "b_exact"])
def test_charge_with_an_exact_operand(kind):
    """An operand of small integers is its own first slice: its slices past the first
    and all its tails vanish, and the charge reduces to one product of norms."""
    rng = np.random.default_rng(100 + KINDS.index(kind))
    A, B = _case(kind, rng)
    SA, SB = mr.Sliced(A, True), mr.Sliced(B, False)
    r = slice(0, BS)
    snA, tnA, tnB = SA.slice_norms(r, r), SA.tail_norms(r, r), SB.tail_norms(r, r)
    snB = SB.slice_norms(r, r)
    nB = float(np.linalg.norm(B[r, r]))
    for L in LEVELS:
        m = min(L - 1, mr.S)
        if kind == "a_exact":
            assert np.all(tnA[1:] == 0) and np.all(snA[1:] == 0)
            assert mr.charge(snA, tnA, tnB, nB, L) == pytest.approx(snA[0] * tnB[m], rel=1e-15)
        else:
            assert np.all(tnB[1:] == 0) and np.all(snB[1:] == 0)
            assert mr.charge(snA, tnA, tnB, nB, L) == pytest.approx(tnA[m] * nB, rel=1e-15)


def test_charge_is_not_vacuous():
    rng = np.random.default_rng(7)
    A, B = _case("normal", rng)
    ratios = [err / c for err, c, L in _charged_errors(A, B, mr.charge) if c > 0]
    # Frobenius submultiplicativity over K = 64 is loose by about sqrt(64); a charge
    # orders of magnitude above the error would make the level choice wasteful
    assert min(ratios) > 1e-3 and max(ratios) <= 1.0


def _mut_no_tail(snA, tnA, tnB, nB, L):
    m = min(L - 1, mr.S)
    return float(sum(snA[p - 1] * tnB[min(L - p, mr.S)] for p in range(1, m + 1)))


def _mut_b_index(snA, tnA, tnB, nB, L):
    m = min(L - 1, mr.S)
    return float(tnA[m] * nB + sum(snA[p - 1] * tnB[min(L - p + 1, mr.S)] for p in range(1, m + 1)))


def _mut_a_index(snA, tnA, tnB, nB, L):
    m = min(L - 1, mr.S)
    return float(tnA[min(m + 1, mr.S)] * nB + sum(snA[p - 1] * tnB[min(L - p, mr.S)]
                                                  for p in range(1, m + 1)))


def _mut_no_min(snA, tnA, tnB, nB, L):
    # forgets that B has only 9 digits: past level 10 the first slice of A is charged
    # nothing for B's rounding
    m = min(L - 1, mr.S)
    return float(tnA[m] * nB + sum(snA[p - 1] * (tnB[L - p] if L - p <= mr.S else 0.0)
                                   for p in range(1, m + 1)))


@pytest.mark.parametrize("mutant,kind", [(_mut_no_tail, "b_exact"), (_mut_b_index, "a_exact"),
                                         (_mut_a_index, "b_exact"), (_mut_no_min, "a_exact")])
def test_mutated_charges_fail(mutant, kind):
    rng = np.random.default_rng(100 + KINDS.index(kind))
    A, B = _case(kind, rng)
    violated = [(L, err, c) for err, c, L in _charged_errors(A, B, mutant) if err > c * (1 + 1e-12)]
    assert violated, mutant.__name__


# ------------------------------------------------ inputs of the GPU level check

def test_alg3_recursion_matches_the_oracle(orc):
    """The recursion tests/levels_case.py applies to leaf charges is Algorithm 3: on
    float64 leaves (p if p < tau, else 0) it reproduces the oracle's CSE."""
    import levels_case
    g = np.random.default_rng(3)
    n = 256
    A = g.standard_normal((n, n)) * np.exp(-np.abs(np.subtract.outer(np.arange(n), np.arange(n))) / 40)
    B = A.T.copy()
    nA, nB = orc.block_norms(A, 64), orc.block_norms(B, 64)
    p = nA[:, :, None] * nB[None, :, :]
    taus = np.array([0.0, np.median(p), p.max() * 1.01, 1e9])
    want = orc.cse(A, B, 64, taus)
    for t, w in zip(taus, want):
        leaf = np.where(p < t, p, 0.0)
        assert levels_case.alg3(leaf) == pytest.approx(w, rel=1e-12, abs=0.0)


@pytest.mark.parametrize("case", __import__("levels_case").CASES)
def test_level_cases_separate_levels(case):
    """Each GPU level case fixes exactly one level (checked inside build), and the
    results one level up or down differ from the expected one by far more than the
    rounding tolerance, so a level set off by one cannot pass."""
    import levels_case
    c = levels_case.build(*case)
    assert c.charge_lo <= c.charge_hi <= c.delta / 2
    assert c.neighbours.min() > 0.9, c.neighbours
