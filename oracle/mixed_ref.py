"""CPU reference for the mixed form's slicing and its error charge.

TEST INFRASTRUCTURE ONLY: imported by tests, never by the product path.

The mixed form is this implementation's own leaf-product arithmetic, not the
paper's: it multiplies float64 leaf blocks through exact fixed-point digit slices
and charges the digits it leaves out inside the Algorithm 3 bound, so that the
bound of Section 3 still covers the whole error of the product. This module
writes that arithmetic out by its definition, with numpy int64 digits and Python
integers for the exact sums:

* exponents: row r of the left operand gets e_r with max_c |A[r,c]| < 2^e_r
  (0 for an all-zero row); the right operand gets column exponents f_c;
* V = x 2^(63 - e), rounded half away from zero, formed from the float64
  mantissa and exponent in integer arithmetic;
* balanced digits from the bottom: d = ((V + 64) mod 128) - 64, V <- (V - d)/128,
  eight times, then d_1 = V, so x = sum_{p=1..9} d_p 2^(e - 7p) + T_9 with
  |T_9| <= 2^(e - 64);
* the level-L product sum_{p+q <= L} A_p B_q, every digit product summed
  exactly, rounded to float64 once and scaled by 2^(e_i + f_j - 7 L_top);
* the charge of a product formed to level L, with m = min(L - 1, 9),
      sum_{p <= m} ||A_p|| ||B - sum_{q <= min(L - p, 9)} B_q|| + ||A - sum_{p <= m} A_p|| ||B||,
  which bounds ||AB - sum_{p+q <= L} A_p B_q||_F by the triangle inequality and
  the submultiplicativity of the Frobenius norm.
"""
from __future__ import annotations

import numpy as np

S = 9          # digits per entry
W = 7          # bits per digit


def exponents(X: np.ndarray, axis: int) -> np.ndarray:
    """e with max |X| < 2^e along rows (axis = 1) or columns (axis = 0); 0 if all zero."""
    m = np.abs(X).max(axis=axis)
    e = np.frexp(m)[1].astype(np.int64)
    e[m == 0] = 0
    return e


def _scaled_parts(X: np.ndarray, e_rows: np.ndarray):
    """x 2^(63 - e_r) = M 2^sh with M a non-negative integer below 2^53 (sign apart)."""
    mant, ex = np.frexp(X)
    M = np.rint(np.abs(mant) * 2.0 ** 53).astype(np.int64)
    sh = ex.astype(np.int64) - 53 + 63 - e_rows[:, None]
    return M, sh


def fixed_point(X: np.ndarray, e_rows: np.ndarray):
    """V = round(x 2^(63 - e_r)) per entry (half away from zero), exactly, and the
    rounding remainder r = x 2^(63 - e_r) - V in [-1/2, 1/2] (float64, exact)."""
    M, sh = _scaled_parts(X, e_rows)
    V = np.zeros_like(M)
    r = np.zeros(X.shape)
    up = sh >= 0
    V[up] = M[up] << sh[up]
    dn = (~up) & (sh > -63)
    s = -sh[dn]
    Vd = (M[dn] + (np.int64(1) << (s - 1))) >> s
    V[dn] = Vd
    # remainder M 2^-s - Vd: (M - Vd 2^s) is an exact integer of at most 53 bits
    r[dn] = np.ldexp((M[dn] - (Vd << s)).astype(np.float64), -s)
    far = (~up) & (sh <= -63)
    r[far] = np.ldexp(M[far].astype(np.float64), sh[far])
    neg = X < 0
    V[neg] = -V[neg]
    r[neg] = -r[neg]
    return V, r


def digits(V: np.ndarray) -> np.ndarray:
    """Balanced base-128 digits d[0..8] (d[0] the most significant, i.e. d_1) of V."""
    d = np.zeros((S,) + V.shape, dtype=np.int64)
    rem = V.copy()
    for p in range(S - 1, 0, -1):
        d[p] = ((rem + 64) & 127) - 64
        rem = (rem - d[p]) >> W
    d[0] = rem
    return d


class Sliced:
    """Digits d[p, r, c] of an operand in units 2^(e_r - 7(p+1)) (rows) or
    2^(f_c - 7(p+1)) (columns), the exponents, and the rounding remainders."""

    def __init__(self, X: np.ndarray, by_rows: bool):
        X = np.asarray(X, dtype=np.float64)
        self.by_rows = by_rows
        if by_rows:
            self.e = exponents(X, axis=1)
            V, r = fixed_point(X, self.e)
            self.d, self.r = digits(V), r
        else:
            self.e = exponents(X, axis=0)
            V, r = fixed_point(np.ascontiguousarray(X.T), self.e)
            self.d = np.ascontiguousarray(np.transpose(digits(V), (0, 2, 1)))
            self.r = np.ascontiguousarray(r.T)

    def _scale(self, p: int, rows, cols):
        """2^(e - 7p) broadcast over the (rows, cols) window, for digit p = 1..9."""
        if self.by_rows:
            return np.ldexp(1.0, (self.e[rows] - W * p))[:, None]
        return np.ldexp(1.0, (self.e[cols] - W * p))[None, :]

    def part(self, p: int, rows=slice(None), cols=slice(None)) -> np.ndarray:
        """X_p on a window: d_p 2^(e - 7p) (exact in float64)."""
        return self.d[p - 1][rows, cols] * self._scale(p, rows, cols)

    def tail(self, p: int, rows=slice(None), cols=slice(None)) -> np.ndarray:
        """T_p = X - sum_{q <= p} X_q on a window (p = 0..9), in float64."""
        dw = self.d[:, rows, cols]
        # integer residue after digit p, in units of 2^(e - 63): sum_{q > p} d_q 128^(9 - q)
        R = np.zeros(dw.shape[1:], dtype=np.int64)
        for q in range(p + 1, S + 1):
            R = R + dw[q - 1] * (np.int64(1) << (W * (S - q)))
        unit = self._scale(S, rows, cols)
        return (R.astype(np.float64) + self.r[rows, cols]) * unit

    def tail_bound_norms(self, rows=slice(None), cols=slice(None)) -> np.ndarray:
        """Upper bounds of tn[p] (p = 0..9): sqrt(sum (|R_p| + h)^2) in units of
        2^(e - 63), with R_p the integer residue after digit p and h = 1/2 where the
        rounding to fixed point was inexact, 0 where it was exact; >= ||T_p||_F since
        |R_p + r| <= |R_p| + |r| and |r| <= h."""
        dw = self.d[:, rows, cols]
        h = np.where(self.r[rows, cols] != 0.0, 0.5, 0.0)
        unit = self._scale(S, rows, cols)
        out = []
        for p in range(0, S + 1):
            R = np.zeros(dw.shape[1:], dtype=np.int64)
            for q in range(p + 1, S + 1):
                R = R + dw[q - 1] * (np.int64(1) << (W * (S - q)))
            out.append(np.linalg.norm((np.abs(R).astype(np.float64) + h) * unit))
        return np.array(out)

    def slice_norms(self, rows=slice(None), cols=slice(None)) -> np.ndarray:
        """sn[p - 1] = ||X_p||_F on a window, p = 1..9."""
        return np.array([np.linalg.norm(self.part(p, rows, cols)) for p in range(1, S + 1)])

    def tail_norms(self, rows=slice(None), cols=slice(None)) -> np.ndarray:
        """tn[p] = ||T_p||_F on a window, p = 0..9 (tn[0] = ||X||_F)."""
        return np.array([np.linalg.norm(self.tail(p, rows, cols)) for p in range(0, S + 1)])


def level_product(SA: Sliced, SB: Sliced, L: int, rows=slice(None), ks=slice(None),
                  cols=slice(None)) -> np.ndarray:
    """sum_{p+q <= L} A_p B_q over the window A[rows, ks] B[ks, cols], every digit
    product summed exactly (Python integers) and rounded to float64 once."""
    assert SA.by_rows and not SB.by_rows
    e = SA.e[rows]
    f = SB.e[cols]
    levels = {}
    for p in range(1, S + 1):
        for q in range(1, S + 1):
            if p + q <= L:
                g = SA.d[p - 1][rows, ks] @ SB.d[q - 1][ks, cols]
                levels[p + q] = levels.get(p + q, 0) + g
    shape = (len(e), len(f))
    out = np.zeros(shape)
    if not levels:
        return out
    top = max(levels)
    total = np.zeros(shape, dtype=object)
    for lv, g in levels.items():
        total = total + g.astype(object) * (1 << (W * (top - lv)))
    for i in range(shape[0]):
        for j in range(shape[1]):
            v = int(total[i, j])
            out[i, j] = np.ldexp(float(v), int(e[i] + f[j] - W * top)) if v else 0.0
    return out


def charge(snA: np.ndarray, tnA: np.ndarray, tnB: np.ndarray, norm_b: float, L: int) -> float:
    """Bound on ||AB - sum_{p+q <= L} A_p B_q||_F from slice norms snA[p - 1] and tail
    norms tnA[p], tnB[q] (index = digits kept), for L >= 2."""
    m = min(L - 1, S)
    c = tnA[m] * norm_b
    for p in range(1, m + 1):
        c += snA[p - 1] * tnB[min(L - p, S)]
    return float(c)


def triple_charges(A: np.ndarray, B: np.ndarray, bs: int, levels, bound_tails: bool = False):
    """charge(L) of every leaf triple (i, k, j) of A B on bs x bs blocks, slices cut with
    whole-row (A) and whole-column (B) exponents: {L: array[nb, nb, nb]} indexed
    [i, k, j]. bound_tails: use the tail upper bounds instead of the exact tails."""
    n = A.shape[0]
    nb = -(-n // bs)
    SA, SB = Sliced(A, True), Sliced(B, False)
    win = [slice(x * bs, min((x + 1) * bs, n)) for x in range(nb)]
    tail = (lambda Sx, r, c: Sx.tail_bound_norms(r, c)) if bound_tails else \
           (lambda Sx, r, c: Sx.tail_norms(r, c))
    snA = {(i, k): SA.slice_norms(win[i], win[k]) for i in range(nb) for k in range(nb)}
    tnA = {(i, k): tail(SA, win[i], win[k]) for i in range(nb) for k in range(nb)}
    tnB = {(k, j): tail(SB, win[k], win[j]) for k in range(nb) for j in range(nb)}
    nB = {(k, j): float(np.linalg.norm(B[win[k], win[j]])) for k in range(nb) for j in range(nb)}
    out = {}
    for L in levels:
        c = np.zeros((nb, nb, nb))
        for i in range(nb):
            for k in range(nb):
                for j in range(nb):
                    c[i, k, j] = charge(snA[i, k], tnA[i, k], tnB[k, j], nB[k, j], L)
        out[L] = c
    return out


def to_int(X: np.ndarray):
    """X = I 2^k exactly: an object array of Python integers and one exponent k."""
    X = np.asarray(X, dtype=np.float64)
    mant, ex = np.frexp(X)
    M = np.rint(mant * 2.0 ** 53).astype(np.int64)     # signed, exact
    sh = ex.astype(np.int64) - 53
    nz = M != 0
    k = int(sh[nz].min()) if nz.any() else 0
    out = np.empty(X.shape, dtype=object)
    for idx in np.ndindex(X.shape):
        out[idx] = int(M[idx]) << int(sh[idx] - k) if M[idx] else 0
    return out, k


def exact_product(A: np.ndarray, B: np.ndarray):
    """AB exactly: (object array of integers P, exponent k) with AB = P 2^k."""
    IA, ka = to_int(A)
    IB, kb = to_int(B)
    return IA.dot(IB), ka + kb


def level_sum(SA: Sliced, SB: Sliced, L: int, rows=slice(None), ks=slice(None),
              cols=slice(None)):
    """sum_{p+q <= L} A_p B_q on a window, exactly: (object array G, per-entry exponent
    array s) with entry (i, j) = G[i, j] 2^s[i, j]."""
    assert SA.by_rows and not SB.by_rows
    e = SA.e[rows]
    f = SB.e[cols]
    G = np.zeros((len(e), len(f)), dtype=object)
    top = max(2, min(L, 2 * S))
    for p in range(1, S + 1):
        for q in range(1, S + 1):
            if p + q <= L:
                g = SA.d[p - 1][rows, ks] @ SB.d[q - 1][ks, cols]
                G = G + g.astype(object) * (1 << (W * (top - p - q)))
    s = e[:, None] + f[None, :] - W * top
    return G, s


def diff_norm(G: np.ndarray, s: np.ndarray, P: np.ndarray, k: int) -> float:
    """||G 2^s - P 2^k||_F, every entry's difference formed exactly before rounding."""
    acc = 0.0
    for idx in np.ndindex(G.shape):
        si = int(s[idx])
        t = min(si, k)
        v = int(G[idx]) * (1 << (si - t)) - int(P[idx]) * (1 << (k - t))
        if v == 0:
            continue
        nb = abs(v).bit_length()
        if nb > 900:                                   # keep float() in range
            v >>= nb - 900
            t += nb - 900
        acc += np.ldexp(float(v), t) ** 2
    return float(np.sqrt(acc))
