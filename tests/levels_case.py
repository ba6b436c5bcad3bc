"""Inputs for checking the mixed form's level products against the exact model.

A case is a dense product (A B, or X X for a symmetric SP2 step) whose every
leaf-norm product is above the largest tau candidate (1), so no product is ever
skipped, and a tolerance delta that makes exactly one slice level L* the fewest
whose charge fits in delta / 2. The charge of a level is Algorithm 3 applied to
per-triple charges (every product formed): between its value with exact tails and
its value with the tails' upper bounds, a bracket much narrower than the factor
of about 128 between neighbouring levels. The expected result is the exact
level-L* product rounded once (2X - X^2 for the second SP2 branch).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

import synth
from oracle import mixed_ref as mr

BS = 64
LMIN, LMAX = 4, 10          # the level search's range below the last level (11)


def alg3(leaf: np.ndarray) -> float:
    """Algorithm 3's recursion over leaf values leaf[i, k, j] (nb a power of two):
    E = sqrt(sum over the 2 x 2 result quadrants of (E(A_i0, B_0j) + E(A_i1, B_1j))^2)."""
    def rec(i0, k0, j0, size):
        if size == 1:
            return float(leaf[i0, k0, j0])
        h = size // 2
        e = 0.0
        for a in (0, 1):
            for b in (0, 1):
                s = rec(i0 + a * h, k0, j0 + b * h, h) + rec(i0 + a * h, k0 + h, j0 + b * h, h)
                e += s * s
        return math.sqrt(e)
    nb = leaf.shape[0]
    assert nb & (nb - 1) == 0
    return rec(0, 0, 0, nb)


def mirrored(c: np.ndarray) -> np.ndarray:
    """Leaf charges of a symmetric SP2 step: the blocks below the diagonal 2 x 2 tiles
    are written as transposes of blocks (j, i), so triple (i, k, j) is charged the
    product (j, k, i) when (i >> 1) > (j >> 1)."""
    nb = c.shape[0]
    out = c.copy()
    for i in range(nb):
        for j in range(nb):
            if (i >> 1) > (j >> 1):
                out[i, :, j] = c[j, :, i]
    return out


@dataclass
class Case:
    kind: str                 # "plain", "sp2_0" (X^2) or "sp2_1" (2X - X^2)
    A: np.ndarray
    B: np.ndarray             # == A for the SP2 kinds
    delta: float
    level: int                # L*
    charge_lo: float          # bracket of the level-L* charge (Algorithm 3 bound, tau = 0)
    charge_hi: float
    expected: np.ndarray      # the exact level-L* result, rounded once
    tol: np.ndarray           # per-entry bound on the float64 rounding of the kernel's sums
    neighbours: np.ndarray    # share of entries where the result at L* -+ 1 differs from the
                              # expected one by more than 10 tol


def build(kind: str, n: int, seed: int, level: int) -> Case:
    g = synth.rng(seed)
    if kind == "plain":
        A = g.standard_normal((n, n))
        B = g.standard_normal((n, n))
    else:
        M = g.standard_normal((n, n))
        A = (M + M.T) / math.sqrt(2.0)
        B = A
    levels = list(range(LMIN, LMAX + 1))
    ce = mr.triple_charges(A, B, BS, levels)
    cb = mr.triple_charges(A, B, BS, levels, bound_tails=True)
    if kind != "plain":
        ce = {L: mirrored(v) for L, v in ce.items()}
        cb = {L: mirrored(v) for L, v in cb.items()}
    lo = {L: alg3(ce[L]) for L in levels}
    hi = {L: alg3(cb[L]) * (1 + 2.0 ** -10) for L in levels}   # the kernel inflates by 2^-12
    # delta / 2 sits between the level-L* charge and the lowest charge below L*
    top = max(hi[L] for L in levels if L >= level)
    if level > LMIN:
        bottom = min(lo[L] for L in levels if L < level)
        assert top < bottom, (top, bottom)
        half = math.sqrt(top * bottom)
    else:
        half = 4.0 * top
    SA, SB = mr.Sliced(A, True), mr.Sliced(B, False)
    prods = {L: mr.level_product(SA, SB, L) for L in (level - 1, level, level + 1)}
    e, f = SA.e, SB.e
    scale = np.ldexp(1.0, (e[:, None] + f[None, :]).astype(np.int64))
    # every pass sum and every partial is at most about n 2^(e_i + f_j); the kernel rounds
    # each of at most three pass sums and two additions once, the model once
    tol = 16 * 2.0 ** -53 * n * scale
    if kind == "sp2_1":
        expected = {L: 2.0 * A - v for L, v in prods.items()}
        tol = tol + 8 * 2.0 ** -53 * np.abs(2.0 * A)
    else:
        expected = prods
    neighbours = np.array([np.mean(np.abs(expected[L] - expected[level]) > 10 * tol)
                           for L in (level - 1, level + 1)])
    return Case(kind, A, B, 2.0 * half, level, lo[level], hi[level], expected[level], tol,
                neighbours)


CASES = [("plain", 256, 41, 4), ("plain", 256, 42, 5), ("plain", 256, 43, 6),
         ("plain", 200, 44, 6), ("sp2_0", 256, 45, 4), ("sp2_0", 256, 46, 6),
         ("sp2_1", 256, 47, 5)]
