"""Plant plausible mistakes in a copy of the oracle (on the CPU) and check
that the pins reject every one of them: a dropped term, a wrong index, a
transposed operand, a non-strict comparison, a wrong square, a wrong table."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import synth

SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle", "oracle.c")

MUTANTS = {
    "cse_no_square": ("errors[k] += s * s;", "errors[k] += s;"),
    "cse_wrong_b_index": ("cse_rec(cx, A->child[i][1], B->child[1][j], E2);",
                          "cse_rec(cx, A->child[i][1], B->child[j][1], E2);"),
    "cse_drop_second": ("double s = E1[k] + E2[k];", "double s = E1[k];"),
    "cse_non_strict": ("if (nab < cx->tau[k]) errors[k] = nab;", "if (nab <= cx->tau[k]) errors[k] = nab;"),
    "spamm_transposed_b": ("double* T0 = spamm_rec(cx, A->child[i][0], B->child[0][j]);",
                           "double* T0 = spamm_rec(cx, A->child[i][0], B->child[j][0]);"),
    "spamm_drop_t1": ("double t1 = T1 ? T1[r * h + c] : 0.0;", "double t1 = 0.0;"),
    "spamm_non_strict": ("if (A->norm * B->norm < cx->tau) return NULL;",
                         "if (A->norm * B->norm <= cx->tau) return NULL;"),
    "leaf_transposed": ("entry(cx->B, B->r0 + k, B->c0 + j)", "entry(cx->B, B->r0 + j, B->c0 + k)"),
    "tau_table": ("tau[i] = 0.9 * tau[i - 1];", "tau[i] = 0.9 * tau[i - 1] * (1.0 - 1e-9);"),
    "norm_no_sqrt": ("q->norm = sqrt(ss);", "q->norm = ss;"),
    "flat_no_square": ("total += sum * sum;", "total += sum;"),
    "flat_non_strict": ("if (p < tau[t]) sum += p;", "if (p <= tau[t]) sum += p;"),
    "flat_no_sqrt": ("errors[t] = sqrt(total);", "errors[t] = total;"),
    "flat_transposed_b": ("double p = na[i * nb + k] * nbn[k * nb + j];",
                          "double p = na[i * nb + k] * nbn[j * nb + k];"),
    "spectral_rows_only": ("double fro = sqrt(fro2), sch = sqrt(rmax * cmax);",
                           "double fro = sqrt(fro2), sch = sqrt(rmax * rmax);"),
    "spectral_no_sqrt": ("double fro = sqrt(fro2), sch = sqrt(rmax * cmax);",
                         "double fro = sqrt(fro2), sch = rmax * cmax;"),
    "spectral_max_not_min": ("return sch < fro ? sch : fro;", "return sch < fro ? fro : sch;"),
    "spectral_non_strict": ("if (pk < tau[t]) sum += pk;", "if (pk <= tau[t]) sum += pk;"),
    "spectral_transposed_b": ("double pk = na[i * nb + k] * nbn[k * nb + j];",
                              "double pk = na[i * nb + k] * nbn[j * nb + k];"),
    "tau_scaled_fixed_ratio": ("for (int i = 1; i < N; ++i) tau[i] = ratio * tau[i - 1];",
                               "for (int i = 1; i < N; ++i) tau[i] = 0.9 * tau[i - 1];"),
}


def _build(tmp_path, name, old, new):
    src = open(SRC).read()
    assert src.count(old) == 1, name
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-ffp-contract=off", "-shared", "-fPIC", "-o", str(so), str(path), "-lm"])
    lib = ctypes.CDLL(str(so))
    d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
    pd = ctypes.POINTER(ctypes.c_double)
    lib.or_tau_table.argtypes = [i32, pd]
    lib.or_spamm.argtypes = [i64, i64, pd, i64, pd, i64, d, pd, i64]
    lib.or_spamm.restype = i64
    lib.or_cse.argtypes = [i64, i64, pd, i64, pd, i64, pd, i32, pd]
    lib.or_flat_bound.argtypes = [i64, i64, pd, i64, pd, i64, pd, i32, pd]
    lib.or_tau_table_scaled.argtypes = [i32, d, d, pd]
    lib.or_spectral_norm_bound.argtypes = [i64, pd]
    lib.or_spectral_norm_bound.restype = d
    lib.or_spectral_bound.argtypes = [i64, i64, pd, i64, pd, i64, pd, i32, pd]
    return lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _pins_hold(lib) -> bool:
    """A compact replay of the oracle pins; False as soon as one fails."""
    tau = np.zeros(350)
    lib.or_tau_table(350, _p(tau))
    if not np.allclose(tau, 0.9 ** np.arange(350), rtol=1e-13, atol=0):
        return False

    def spamm(A, B, t, bs):
        A, B = np.ascontiguousarray(A), np.ascontiguousarray(B)
        C = np.zeros_like(A)
        lib.or_spamm(A.shape[0], bs, _p(A), A.shape[0], _p(B), A.shape[0], t, _p(C), A.shape[0])
        return C

    def cse(A, B, bs, taus):
        A, B, taus = np.ascontiguousarray(A), np.ascontiguousarray(B), np.ascontiguousarray(taus, dtype=float)
        e = np.zeros(len(taus))
        lib.or_cse(A.shape[0], bs, _p(A), A.shape[0], _p(B), A.shape[0], _p(taus), len(taus), _p(e))
        return e

    def flat(A, B, bs, taus):
        A, B, taus = np.ascontiguousarray(A), np.ascontiguousarray(B), np.ascontiguousarray(taus, dtype=float)
        e = np.zeros(len(taus))
        lib.or_flat_bound(A.shape[0], bs, _p(A), A.shape[0], _p(B), A.shape[0], _p(taus), len(taus), _p(e))
        return e

    def spectral(A, B, bs, taus):
        A, B, taus = np.ascontiguousarray(A), np.ascontiguousarray(B), np.ascontiguousarray(taus, dtype=float)
        e = np.zeros(len(taus))
        lib.or_spectral_bound(A.shape[0], bs, _p(A), A.shape[0], _p(B), A.shape[0], _p(taus), len(taus), _p(e))
        return e

    def snb(M):
        M = np.ascontiguousarray(M, dtype=float)
        return lib.or_spectral_norm_bound(M.shape[0], _p(M))

    ts = np.zeros(6)
    lib.or_tau_table_scaled(6, 64.0, 0.97, _p(ts))
    if not np.allclose(ts, 64.0 * 0.97 ** np.arange(6), rtol=1e-14, atol=0):
        return False
    # spectral norm bound: closed forms (a column of ones, a permutation, a diagonal)
    col = np.zeros((8, 8))
    col[:, 0] = 1.0
    if abs(snb(col) - np.sqrt(8.0)) > 1e-14 or abs(snb(np.eye(8)[::-1]) - 1.0) > 1e-15:
        return False
    if abs(snb(np.diag([3.0, 1.0, 2.0])) - 3.0) > 1e-15 or snb(np.zeros((3, 3))) != 0.0:
        return False
    # a column of ones as the skipped product: ||E||_2 = sqrt(8)
    if abs(spectral(col, np.eye(8), 1, [2.0])[0] - np.sqrt(8.0)) > 1e-14:
        return False
    J8 = np.ones((8, 8))
    if spectral(J8, J8, 1, [1.0])[0] != 0.0:      # products equal to tau are kept
        return False
    A = np.array([[1.0, 2.0], [3.0, 4.0]])
    B = np.array([[5.0, 6.0], [7.0, 8.0]])
    if not np.array_equal(spamm(A, B, 15.5, 1), np.array([[0.0, 16.0], [28.0, 50.0]])):
        return False
    if abs(cse(A, B, 1, [15.5])[0] ** 2 - 622.0) > 1e-12:
        return False
    I = np.eye(4)
    if not np.array_equal(spamm(I, I, 1.0, 1), I) or cse(I, I, 1, [1.0])[0] != 0.0:
        return False
    if abs(cse(I, I, 1, [2.0])[0] - 2.0) > 1e-14:
        return False
    J = np.ones((8, 8))
    if abs(cse(J, J, 1, [2.0])[0] - 64.0) > 1e-12:
        return False
    # flat bound: closed forms, equal to Algorithm 3 at one level (2 x 2 leaves)
    if abs(flat(J, J, 1, [2.0])[0] - 64.0) > 1e-12 or abs(flat(I, I, 1, [2.0])[0] - 2.0) > 1e-14:
        return False
    if flat(J, J, 1, [1.0])[0] != 0.0:          # products equal to tau are kept
        return False
    g = synth.rng(21)
    A8, B8 = g.standard_normal((8, 8)), g.standard_normal((8, 8))
    t8 = np.array([0.5, 2.0, 8.0, 1e9])
    if not np.allclose(flat(A8, B8, 4, t8), cse(A8, B8, 4, t8), rtol=1e-14, atol=0):
        return False
    for seed in (1, 2):
        X = synth.random_decaying(48, seed, length=3.0)
        Y = synth.random_decaying(48, seed + 7, length=5.0).T.copy()
        if np.linalg.norm(spamm(X, Y, 0.0, 8) - X @ Y) > 1e-12 * np.linalg.norm(X @ Y):
            return False
        b = cse(X, Y, 8, tau)
        f = flat(X, Y, 8, tau)
        for k in range(0, 350, 25):
            err = np.linalg.norm(X @ Y - spamm(X, Y, tau[k], 8))
            if err > b[k] * (1 + 1e-12) + 1e-13 or err > f[k] * (1 + 1e-12) + 1e-13:
                return False
        if np.any(f > b * (1 + 1e-13)):
            return False
        sp = spectral(X, Y, 8, tau)
        if np.any(sp > f * (1 + 1e-13)) or np.any(np.diff(sp) > 0):
            return False
        for k in range(0, 350, 25):
            err2 = np.linalg.norm(X @ Y - spamm(X, Y, tau[k], 8), 2)
            if err2 > sp[k] * (1 + 1e-12) + 1e-13:
                return False
    return True


def test_unmutated_oracle_passes_replay(tmp_path):
    lib = _build(tmp_path, "clean", "q->norm = sqrt(ss);", "q->norm = sqrt(ss);")
    assert _pins_hold(lib)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, name):
    old, new = MUTANTS[name]
    assert not _pins_hold(_build(tmp_path, name, old, new))
