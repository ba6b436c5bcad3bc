"""CPU oracle for SpAMM with error control and SP2 purification.

TEST INFRASTRUCTURE ONLY: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(``paper_2005_10680_gb300``) never imports, links or runs it, and this package
never imports the product path.

What lives where:

* ``oracle.c`` (built into ``_build/liboracle.so`` with gcc) -- the tau table,
  the quadtree of Eq. 2, Algorithm 2 (SpAMM), Algorithm 3 (CSE), the one-level
  (flat) bound, the tau selection rule, the dense product and leaf norms.
* this file -- ctypes wrappers, block truncation with ||E||_F < delta (the
  unit rule below), and the SP2 purification driver in the three variants of
  Algorithms 1, 4 and 5.
* ``mixed_ref.py`` -- the mixed form's arithmetic written out exactly: the
  fixed-point rounding, the balanced base-128 digits, level products summed in
  Python integers, and the charge that bounds a product formed to level L.

Readings where the paper is silent (each one is a choice, not the paper's):

* Truncation works on leaf blocks. For a symmetric matrix the unit is the
  pair {X_ij, X_ji} (weight ||X_ij||^2 + ||X_ji||^2) or a diagonal block
  (weight ||X_ii||^2). Units are sorted by (weight, i*nb + j) and the longest
  prefix whose running float64 sum is below delta^2 is removed, so
  ||E||_F < delta.
* f_i are the SP2 polynomials: X^2 when tr(X) > n_occ, else 2X - X^2.
* X_0 = (lmax I - F) / (lmax - lmin) with Gershgorin bounds unless given.
* Eigenvalue bounds h (top of the unoccupied group) and l (bottom of the
  occupied group) follow h <- f(h) + delta_i, l <- f(l) - delta_i (Weyl's
  inequality, ||E||_2 <= ||E||_F).  delta_i = eps * (l' - h') / (2 sqrt(2) n_iter)
  with l', h' the mapped bounds before the error of step i, so that the
  accumulated subspace error sum_i sqrt(2) delta_i / gap_i stays below eps/2.
* Stop when 2 (||C - X||_F + bound(C)) < eps / 2 with C the approximate
  square formed in the current step; the current X is returned (its distance
  to the nearest projector is at most 2 ||X^2 - X||_F).
* n_occ = 0 and n_occ = n give D = 0 and D = I directly (no step): the gap
  bounds of the step tolerances have no occupied (unoccupied) group to follow.

Parity: pinned by tests/test_oracle_*.py; see the header of oracle.c.
"""
from __future__ import annotations

import ctypes
import dataclasses
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
N_TAU = 350

_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.c with gcc (no fused multiply-add contraction)."""
    src = os.path.join(_HERE, "oracle.c")
    if (not force and os.path.exists(_SO)
            and os.path.getmtime(_SO) >= os.path.getmtime(src)):
        return _SO
    os.makedirs(_BUILD, exist_ok=True)
    tmp = _SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-shared",
                           "-fPIC", "-o", tmp, src, "-lm"])
    os.replace(tmp, _SO)
    return _SO


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        pd = ctypes.POINTER(ctypes.c_double)
        _lib.or_tau_table.argtypes = [i32, pd]
        _lib.or_spamm.argtypes = [i64, i64, pd, i64, pd, i64, d, pd, i64]
        _lib.or_spamm.restype = i64
        _lib.or_cse.argtypes = [i64, i64, pd, i64, pd, i64, pd, i32, pd]
        _lib.or_flat_bound.argtypes = [i64, i64, pd, i64, pd, i64, pd, i32, pd]
        _lib.or_tau_table_scaled.argtypes = [i32, d, d, pd]
        _lib.or_spectral_norm_bound.argtypes = [i64, pd]
        _lib.or_spectral_norm_bound.restype = d
        _lib.or_spectral_bound.argtypes = [i64, i64, pd, i64, pd, i64, pd, i32, pd]
        _lib.or_select_tau.argtypes = [pd, i32, d]
        _lib.or_select_tau.restype = i32
        _lib.or_dense_gemm.argtypes = [i64, pd, pd, pd]
        _lib.or_block_norms.argtypes = [i64, i64, pd, i64, pd]
    return _lib


def _p(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(a, dtype=np.float64)


# ----------------------------------------------------------- primitives

def tau_table(N: int = N_TAU) -> np.ndarray:
    """tau_1 = 1, tau_i = 0.9 tau_{i-1} (experiment section)."""
    out = np.zeros(N)
    lib().or_tau_table(N, _p(out))
    return out


def spamm(A, B, tau: float, bs: int):
    """Algorithm 2: returns (C, number of lowest-level products formed)."""
    A, B = _f64(A), _f64(B)
    n = A.shape[0]
    C = np.zeros((n, n))
    cnt = lib().or_spamm(n, bs, _p(A), n, _p(B), n, float(tau), _p(C), n)
    return C, int(cnt)


def cse(A, B, bs: int, taus=None) -> np.ndarray:
    """Algorithm 3: error bound for every tau candidate."""
    A, B = _f64(A), _f64(B)
    taus = tau_table() if taus is None else _f64(taus)
    n = A.shape[0]
    err = np.zeros(len(taus))
    lib().or_cse(n, bs, _p(A), n, _p(B), n, _p(taus), len(taus), _p(err))
    return err


def flat_bound(A, B, bs: int, taus=None) -> np.ndarray:
    """One-level bound sqrt(sum_ij (sum_k p_ikj [p_ikj < tau])^2) for every tau."""
    A, B = _f64(A), _f64(B)
    taus = tau_table() if taus is None else _f64(taus)
    n = A.shape[0]
    err = np.zeros(len(taus))
    lib().or_flat_bound(n, bs, _p(A), n, _p(B), n, _p(taus), len(taus), _p(err))
    return err


def tau_table_scaled(N: int, start: float, ratio: float) -> np.ndarray:
    """tau_1 = start, tau_i = ratio tau_{i-1} (repeated multiplication)."""
    out = np.zeros(N)
    lib().or_tau_table_scaled(N, float(start), float(ratio), _p(out))
    return out


def spectral_norm_bound(M) -> float:
    """min(||M||_F, sqrt(||M||_1 ||M||_inf)) for a square M: an upper bound on ||M||_2."""
    M = _f64(M)
    assert M.ndim == 2 and M.shape[0] == M.shape[1]
    return float(lib().or_spectral_norm_bound(M.shape[0], _p(M)))


def spectral_bound(A, B, bs: int, taus=None) -> np.ndarray:
    """Bound on ||SpAMM(A, B, tau) - AB||_2 for every tau: spectral_norm_bound of
    M_ij = sum_k p_ikj [p_ikj < tau]."""
    A, B = _f64(A), _f64(B)
    taus = tau_table() if taus is None else _f64(taus)
    n = A.shape[0]
    err = np.zeros(len(taus))
    lib().or_spectral_bound(n, bs, _p(A), n, _p(B), n, _p(taus), len(taus), _p(err))
    return err


def select_tau(errors, delta: float) -> int:
    """Index of the largest bound still below delta, or -1 (exact product)."""
    errors = _f64(errors)
    return int(lib().or_select_tau(_p(errors), len(errors), float(delta)))


def dense_gemm(A, B) -> np.ndarray:
    A, B = _f64(A), _f64(B)
    n = A.shape[0]
    C = np.zeros((n, n))
    lib().or_dense_gemm(n, _p(A), _p(B), _p(C))
    return C


def block_norms(X, bs: int) -> np.ndarray:
    X = _f64(X)
    n = X.shape[0]
    nb = -(-n // bs)
    out = np.zeros((nb, nb))
    lib().or_block_norms(n, bs, _p(X), n, _p(out))
    return out


@dataclasses.dataclass
class SpammResult:
    C: np.ndarray
    tau: float          # 0.0 means the exact product was formed
    k: int              # selected 0-based index into the tau table, -1 if none
    bound: float        # CSE bound for the chosen tau (0 for the exact product)
    products: int       # lowest-level products formed


def spamm_delta(A, B, delta: float, bs: int, taus=None) -> SpammResult:
    """spamm(A, B, delta): CSE sweep, tau selection, then Algorithm 2."""
    taus = tau_table() if taus is None else _f64(taus)
    err = cse(A, B, bs, taus)
    k = select_tau(err, delta)
    tau = float(taus[k]) if k >= 0 else 0.0
    bound = float(err[k]) if k >= 0 else 0.0
    C, cnt = spamm(A, B, tau, bs)
    return SpammResult(C, tau, k, bound, cnt)


# ------------------------------------------------------------ truncation

@dataclasses.dataclass
class TruncResult:
    X: np.ndarray
    removed_sq: float     # running float64 sum of removed weights (||E||_F^2)
    removed_units: int


def truncate(X, delta: float, bs: int, symmetric: bool = True) -> TruncResult:
    """Remove the largest set of smallest leaf-block units with ||E||_F < delta."""
    X = np.array(X, dtype=np.float64, copy=True)
    n = X.shape[0]
    nb = -(-n // bs)
    nrm = block_norms(X, bs)
    present = nrm > 0.0
    keys, weights, members = [], [], []
    for i in range(nb):
        for j in range(nb):
            if symmetric and j < i:
                continue
            if symmetric and i != j:
                if not (present[i, j] or present[j, i]):
                    continue
                w = nrm[i, j] ** 2 + nrm[j, i] ** 2
                mem = ((i, j), (j, i))
            else:
                if not present[i, j]:
                    continue
                w = nrm[i, j] ** 2
                mem = ((i, j),)
            keys.append(i * nb + j)
            weights.append(w)
            members.append(mem)
    if not weights:
        return TruncResult(X, 0.0, 0)
    weights = np.array(weights)
    order = np.lexsort((np.array(keys), weights))      # by weight, then key
    run = np.cumsum(weights[order])                     # sequential float64 sum
    m = int(np.count_nonzero(run < delta * delta))
    for u in order[:m]:
        for (bi, bj) in members[u]:
            X[bi * bs:(bi + 1) * bs, bj * bs:(bj + 1) * bs] = 0.0
    return TruncResult(X, float(run[m - 1]) if m else 0.0, m)


# ------------------------------------------------------------------ SP2

def gershgorin(F) -> tuple[float, float]:
    F = _f64(F)
    d = np.diag(F)
    r = np.sum(np.abs(F), axis=1) - np.abs(d)
    return float(np.min(d - r)), float(np.max(d + r))


@dataclasses.dataclass
class PurifyResult:
    D: np.ndarray
    iters: int
    converged: bool
    branches: list
    deltas: list
    taus: list
    traces: list
    idem: list
    # propagated eigenvalue bounds of the iterate: entry 0 for X_0 (after its
    # truncation), entry i after accepted step i; the unoccupied eigenvalues of
    # X_i are <= hs[i] and the occupied ones >= ls[i]
    hs: list = dataclasses.field(default_factory=list)
    ls: list = dataclasses.field(default_factory=list)
    iterates: list = None        # X_0, X_1, ... when asked for


def purify(F, n_occ: int, eps: float, n_iter: int, homo: float, lumo: float,
           variant: int = 5, bs: int = 64, lmin=None, lmax=None, keep_iterates: bool = False,
           perturb=None) -> PurifyResult:
    """SP2 purification with error control: Algorithm 1 (variant=1, truncmul),
    Algorithm 4 (variant=4, SpAMM only) or Algorithm 5 (variant=5, hybrid).

    keep_iterates: also return every iterate X_0, X_1, ... (res.iterates).
    perturb: a test hook, callable (X, delta) -> E with ||E||_F <= delta. When given,
    every step's error (Algorithm 1's E_i, and X_0's truncation) is E instead of
    what truncation or SpAMM would make: the products are exact and E is added,
    so a test can put the largest error the step tolerance allows where it does
    the most harm."""
    F = _f64(F)
    n = F.shape[0]
    if n_occ in (0, n):
        # Eq. 1 with the chemical potential outside the spectrum: D = 0 or I exactly
        D = np.eye(n) if n_occ == n else np.zeros((n, n))
        return PurifyResult(D, 0, True, [], [], [], [], [])
    if lmin is None or lmax is None:
        lmin, lmax = gershgorin(F)
    width = lmax - lmin
    X = (lmax * np.eye(n) - F) / width
    l = (lmax - homo) / width       # occupied eigenvalues of X_0 are >= l
    h = (lmax - lumo) / width       # unoccupied eigenvalues of X_0 are <= h
    budget = eps / (2.0 * math.sqrt(2.0) * n_iter)
    res = PurifyResult(None, 0, False, [], [], [], [], [])
    if variant in (1, 5):
        d0 = budget * (l - h)
        X = X + perturb(X, d0) if perturb else truncate(X, d0, bs).X
        h, l = h + d0, l - d0
    res.hs.append(h)
    res.ls.append(l)
    if keep_iterates:
        res.iterates = [X]
    for it in range(1, n_iter + 1):
        tr = float(np.trace(X))
        sq = tr > n_occ
        if sq:
            hn, ln = h * h, l * l
        else:
            hn, ln = 2 * h - h * h, 2 * l - l * l
        delta = budget * (ln - hn)
        if variant == 1 or perturb:
            C = X @ X
            bound, tau = 0.0, 0.0
        else:
            r = spamm_delta(X, X, delta if variant == 4 else 0.5 * delta, bs)
            C, bound, tau = r.C, r.bound, r.tau
        idem = float(np.linalg.norm(C - X)) + bound
        res.traces.append(tr)
        res.idem.append(idem)
        if 2.0 * idem < 0.5 * eps:
            res.converged = True
            break
        Xn = C if sq else 2.0 * X - C
        if perturb:
            Xn = Xn + perturb(Xn, delta)
        elif variant == 1:
            Xn = truncate(Xn, delta, bs).X
        elif variant == 5:
            Xn = truncate(Xn, 0.5 * delta, bs).X
        h, l = hn + delta, ln - delta
        res.branches.append("sq" if sq else "dbl")
        res.deltas.append(delta)
        res.taus.append(tau)
        res.iters = it
        res.hs.append(h)
        res.ls.append(l)
        if keep_iterates:
            res.iterates.append(Xn)
        X = Xn
    res.D = X
    return res


def exact_density(F, n_occ: int) -> np.ndarray:
    """Eq. 1: D = theta(mu I - F) with mu in the gap, by eigendecomposition."""
    w, v = np.linalg.eigh(_f64(F))
    vo = v[:, :n_occ]
    return vo @ vo.T
