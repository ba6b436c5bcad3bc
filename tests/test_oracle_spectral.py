"""Pins for the oracle's spectral-norm error control and its tuned candidate list.

The conclusion leaves error control in other norms, and a candidate list with a
different length and starting value, to future work. The oracle's spectral bound
is min(||M||_F, sqrt(||M||_1 ||M||_inf)) of M_ij = sum_k p_ikj [p_ikj < tau]; these
tests tie it to closed forms, to the exact spectral norm of the error (SVD) and
to the Frobenius one-level bound it may never exceed."""
import numpy as np
import pytest

import synth


def test_scaled_table_closed_form(orc):
    t = orc.tau_table_scaled(350, 1.0, 0.9)
    assert np.array_equal(t, orc.tau_table())              # the paper's list, bit for bit
    t = orc.tau_table_scaled(200, 64.0, 0.97)
    assert t[0] == 64.0
    np.testing.assert_allclose(t, 64.0 * 0.97 ** np.arange(200), rtol=1e-13, atol=0)
    assert np.all(np.diff(t) < 0)


@pytest.mark.parametrize("nb", [1, 2, 7, 16])
def test_norm_bound_closed_forms(orc, nb):
    g = np.random.default_rng(nb)
    d = g.uniform(0.1, 2.0, nb)
    assert orc.spectral_norm_bound(np.diag(d)) == pytest.approx(d.max(), rel=1e-15)
    P = np.eye(nb)[g.permutation(nb)]
    assert orc.spectral_norm_bound(P) == pytest.approx(1.0, rel=1e-15)
    assert orc.spectral_norm_bound(np.ones((nb, nb))) == pytest.approx(nb, rel=1e-15)
    # rank one u v^T (u, v >= 0): ||.||_2 = ||.||_F = |u| |v|
    u, v = g.uniform(0, 1, nb), g.uniform(0, 1, nb)
    R = np.outer(u, v)
    assert orc.spectral_norm_bound(R) == pytest.approx(np.linalg.norm(u) * np.linalg.norm(v),
                                                       rel=1e-14)
    C = np.zeros((nb, nb))
    C[:, nb // 2] = 1.0                                     # one column: sqrt(nb), exactly
    assert orc.spectral_norm_bound(C) == pytest.approx(np.sqrt(nb), rel=1e-15)
    assert orc.spectral_norm_bound(np.zeros((nb, nb))) == 0.0


@pytest.mark.parametrize("seed", range(6))
def test_norm_bound_between_spectral_and_frobenius(orc, seed):
    g = np.random.default_rng(seed)
    nb = int(g.integers(2, 40))
    M = np.abs(g.standard_normal((nb, nb))) * (g.uniform(size=(nb, nb)) < g.uniform(0.05, 1.0))
    b = orc.spectral_norm_bound(M)
    assert np.linalg.norm(M, 2) <= b * (1 + 1e-14)
    assert b <= np.linalg.norm(M) * (1 + 1e-15)
    # non-decreasing in every entry
    M2 = M + np.abs(g.standard_normal((nb, nb))) * (g.uniform(size=(nb, nb)) < 0.2)
    assert orc.spectral_norm_bound(M2) >= b


def _inputs(kind, n, seed):
    g = synth.rng(seed)
    if kind == "decay":
        return (synth.random_decaying(n, seed, length=4.0),
                synth.random_decaying(n, seed + 1, length=6.0).T.copy())
    if kind == "symmetric":
        X = synth.random_decaying(n, seed, length=5.0, symmetric=True)
        return X, X
    if kind == "sparse":
        A = g.standard_normal((n, n)) * (g.uniform(size=(n, n)) < 0.1)
        B = g.standard_normal((n, n)) * (g.uniform(size=(n, n)) < 0.1)
        return A, B
    raise ValueError(kind)


@pytest.mark.parametrize("kind,n,bs", [("decay", 96, 8), ("decay", 256, 8), ("symmetric", 100, 16),
                                       ("symmetric", 256, 8), ("sparse", 64, 8)])
def test_bound_covers_spectral_error(orc, kind, n, bs):
    A, B = _inputs(kind, n, 5)
    taus = orc.tau_table()
    sp = orc.spectral_bound(A, B, bs, taus)
    fl = orc.flat_bound(A, B, bs, taus)
    assert np.all(np.diff(sp) <= 0)                         # non-increasing along the table
    assert np.all(sp <= fl * (1 + 1e-15))                   # never above the Frobenius bound
    AB = A @ B
    for k in range(0, 350, 7):
        E = orc.spamm(A, B, taus[k], bs)[0] - AB
        assert np.linalg.norm(E, 2) <= sp[k] * (1 + 1e-12) + 1e-14, (kind, k)
    if n >= 256:
        # on a wide grid of decaying blocks M is banded, and the spectral bound is
        # well below the Frobenius one for some candidates
        assert np.any(sp < 0.7 * fl)


def test_block_diagonal_closed_form(orc):
    """Block-diagonal operands have only (i, i, i) triples: with every product skipped
    M is diagonal and the bound is max_i ||A_ii||_F ||B_ii||_F."""
    g = np.random.default_rng(3)
    n, bs = 64, 16
    A, B = np.zeros((n, n)), np.zeros((n, n))
    for i in range(n // bs):
        s = slice(i * bs, (i + 1) * bs)
        A[s, s] = g.standard_normal((bs, bs))
        B[s, s] = g.standard_normal((bs, bs))
    na, nbn = orc.block_norms(A, bs), orc.block_norms(B, bs)
    want = max(na[i, i] * nbn[i, i] for i in range(n // bs))
    assert orc.spectral_bound(A, B, bs, [1e30])[0] == pytest.approx(want, rel=1e-14)
    assert orc.flat_bound(A, B, bs, [1e30])[0] > 1.5 * want


def test_worked_example(orc):
    """Eqs. 4-7 with scalar leaves: at tau = 15.5 the skipped products are 5, 14
    (C_00), 6 (C_01) and 15 (C_10), so M = [[19, 6], [15, 0]]: the Schur factor
    sqrt(25 * 34) exceeds ||M||_F = sqrt(622), which is the bound, and the true
    error E = -M has ||E||_2 below it."""
    A = np.array([[1.0, 2.0], [3.0, 4.0]])
    B = np.array([[5.0, 6.0], [7.0, 8.0]])
    b = orc.spectral_bound(A, B, 1, [15.5])[0]
    assert b == pytest.approx(np.sqrt(622.0), rel=1e-15)
    E = orc.spamm(A, B, 15.5, 1)[0] - A @ B
    np.testing.assert_array_equal(-E, [[19.0, 6.0], [15.0, 0.0]])
    assert np.linalg.norm(E, 2) < b
