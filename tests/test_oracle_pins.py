"""Pins for the CPU oracle: each test ties the oracle to something other than
itself -- values worked out from the paper's worked example (Eqs. 4-7), closed
forms, textbook definitions (the dense product, the eigendecomposition of
Eq. 1), brute force on small inputs, and invariants that a dropped term, a
wrong sign or index, or a transposed operand would break."""
import itertools
import math
import os

import numpy as np
import pytest

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            key, *rest = line.split()
            vals[key] = [float(x) for x in rest]
    return vals


def _np_block_norms(X, bs):
    n = X.shape[0]
    nb = -(-n // bs)
    out = np.zeros((nb, nb))
    for i in range(nb):
        for j in range(nb):
            out[i, j] = np.linalg.norm(X[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs])
    return out


def _flat_spamm(A, B, tau, bs):
    """Brute force: sum of A_ik B_kj over leaf triples with ||A_ik|| ||B_kj|| >= tau."""
    n = A.shape[0]
    nb = -(-n // bs)
    na, nbn = _np_block_norms(A, bs), _np_block_norms(B, bs)
    C = np.zeros((n, n))
    kept = 0
    for i in range(nb):
        for j in range(nb):
            for k in range(nb):
                if na[i, k] == 0 or nbn[k, j] == 0:
                    continue
                if na[i, k] * nbn[k, j] < tau:
                    continue
                kept += 1
                C[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] += (
                    A[i * bs:(i + 1) * bs, k * bs:(k + 1) * bs] @ B[k * bs:(k + 1) * bs, j * bs:(j + 1) * bs])
    return C, kept, na, nbn


# ------------------------------------------------------------------ tau

def test_tau_table_closed_form(orc):
    t = orc.tau_table(350)
    assert t[0] == 1.0 and t[1] == 0.9
    k = np.arange(350)
    np.testing.assert_allclose(t, 0.9 ** k, rtol=1e-13)
    assert np.all(np.diff(t) < 0)
    # "logarithmically equally spaced values between 1 and 1e-16"
    assert 0.5e-16 < t[-1] < 2e-16


# --------------------------------------------------------- worked example

def test_worked_example_eqs_4_to_7(orc):
    g = _golden("worked_example_eq4_7.txt")
    A = np.array(g["A"]).reshape(2, 2)
    B = np.array(g["B"]).reshape(2, 2)
    np.testing.assert_array_equal(orc.spamm(A, B, 0.0, 1)[0], np.array(g["C_exact"]).reshape(2, 2))
    # Eq. 5-7: the paper's skip set, written out on the 2x2 product
    Ct = np.array([[0.0, A[0, 0] * B[0, 1] + A[0, 1] * B[1, 1]],
                   [A[1, 0] * B[0, 0] + A[1, 1] * B[1, 0], A[1, 0] * B[0, 1]]])
    E = A @ B - Ct
    assert np.sum(E * E) == g["eq5_skip_error_sq"][0]
    tau = g["tau"][0]
    C, cnt = orc.spamm(A, B, tau, 1)
    np.testing.assert_array_equal(C, np.array(g["C_tau"]).reshape(2, 2))
    assert cnt == 4
    E = A @ B - C
    assert np.sum(E * E) == g["err_tau_sq"][0]
    b = orc.cse(A, B, 1, [tau, 1e9, 1.0])
    assert b[0] ** 2 == pytest.approx(g["cse_tau_sq"][0], rel=1e-15)
    # everything skipped, all entries positive: the bound equals ||A B||_F
    assert b[1] ** 2 == pytest.approx(sum(x * x for x in g["C_exact"]), rel=1e-15)
    assert b[2] == 0.0


def test_worked_example_sign_overestimate(orc):
    g = _golden("worked_example_eq4_7.txt")
    A = np.array(g["A"]).reshape(2, 2)
    B = np.array(g["B"]).reshape(2, 2)
    A[0, 1] = g["sign_A"][0]
    C, _ = orc.spamm(A, B, 15.5, 1)
    E = A @ B - C
    assert abs(E[0, 0]) == g["sign_true_C00_error"][0]
    b = orc.cse(A, B, 1, [15.5])[0]
    # bound = sqrt(19^2 + 6^2 + 15^2) >= true error
    assert b ** 2 == pytest.approx(g["sign_bound_C00_term"][0] ** 2 + 6.0 ** 2 + 15.0 ** 2, rel=1e-15)
    assert b >= np.linalg.norm(E)


# ----------------------------------------------------------- Algorithm 2

@pytest.mark.parametrize("n,bs", [(8, 1), (64, 8), (100, 16), (96, 32), (257, 32)])
def test_spamm_tau0_is_dense_product(orc, n, bs):
    A = synth.random_decaying(n, 11, length=5.0)
    B = synth.random_decaying(n, 12, length=9.0)
    C, _ = orc.spamm(A, B, 0.0, bs)
    ref = A @ B
    assert np.linalg.norm(C - ref) <= 1e-13 * np.linalg.norm(ref)
    D = orc.dense_gemm(A, B)
    assert np.linalg.norm(D - ref) <= 1e-13 * np.linalg.norm(ref)


def test_spamm_tau_above_norm_product_is_zero(orc):
    A = synth.random_decaying(64, 3)
    B = synth.random_decaying(64, 4)
    tau = np.linalg.norm(A) * np.linalg.norm(B) * 1.0001
    C, cnt = orc.spamm(A, B, tau, 8)
    assert cnt == 0 and not C.any()


def test_spamm_block_diagonal_closed_form(orc):
    g = synth.rng(5)
    bs, nb = 8, 8
    A = np.zeros((bs * nb,) * 2)
    B = np.zeros_like(A)
    scales = np.logspace(-4, 1, nb)
    for i in range(nb):
        A[i * bs:(i + 1) * bs, i * bs:(i + 1) * bs] = scales[i] * g.standard_normal((bs, bs))
        B[i * bs:(i + 1) * bs, i * bs:(i + 1) * bs] = g.standard_normal((bs, bs))
    tau = 1e-2
    C, cnt = orc.spamm(A, B, tau, bs)
    expect = np.zeros_like(A)
    kept = 0
    for i in range(nb):
        a = A[i * bs:(i + 1) * bs, i * bs:(i + 1) * bs]
        b = B[i * bs:(i + 1) * bs, i * bs:(i + 1) * bs]
        if np.linalg.norm(a) * np.linalg.norm(b) >= tau:
            expect[i * bs:(i + 1) * bs, i * bs:(i + 1) * bs] = a @ b
            kept += 1
    assert cnt == kept and 0 < kept < nb
    np.testing.assert_allclose(C, expect, rtol=1e-13, atol=1e-300)


@pytest.mark.parametrize("n,bs,seed", [(64, 8, 1), (96, 16, 2), (120, 16, 3)])
def test_spamm_skip_set_is_flat_leaf_rule(orc, n, bs, seed):
    A = synth.random_decaying(n, seed, length=4.0)
    B = synth.random_decaying(n, seed + 100, length=7.0)
    taus = orc.tau_table()
    for tau in taus[[20, 40, 60, 90]]:
        C, cnt = orc.spamm(A, B, tau, bs)
        Cf, kept, na, nbn = _flat_spamm(A, B, tau, bs)
        p = np.einsum("ik,kj->ikj", na, nbn)
        assert not np.any(np.abs(p - tau) <= 1e-12 * tau), "borderline triple: pick another tau"
        assert cnt == kept
        assert np.linalg.norm(C - Cf) <= 1e-13 * max(1e-300, np.linalg.norm(Cf))


# ----------------------------------------------------------- Algorithm 3

@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_cse_identity_closed_form(orc, L):
    n = 2 ** L
    I = np.eye(n)
    b = orc.cse(I, I, 1, [2.0, 0.5])
    # every leaf triple (i,i,i) has norm product 1 and is skipped at tau = 2:
    # the bound is ||I I||_F = sqrt(n) exactly; at tau = 0.5 nothing is skipped.
    assert b[0] == pytest.approx(math.sqrt(n), rel=1e-15)
    assert b[1] == 0.0


def test_skip_rule_is_strict(orc):
    # Algorithm 2 skips only when ||A|| ||B|| < tau; Algorithm 3 counts an error only then
    I = np.eye(4)
    C, cnt = orc.spamm(I, I, 1.0, 1)
    np.testing.assert_array_equal(C, I)
    assert cnt == 4
    assert orc.cse(I, I, 1, [1.0])[0] == 0.0


@pytest.mark.parametrize("L", [1, 2, 3, 4])
def test_cse_all_ones_closed_form(orc, L):
    n = 2 ** L
    J = np.ones((n, n))
    b = orc.cse(J, J, 1, [2.0])
    # each level multiplies the bound by 4: bound = 4^L = n^2 = ||J J||_F
    assert b[0] == pytest.approx(4.0 ** L, rel=1e-14)
    assert b[0] == pytest.approx(np.linalg.norm(J @ J), rel=1e-14)


def test_cse_one_level_equals_flat_sum(orc):
    g = synth.rng(9)
    bs = 4
    A = g.standard_normal((8, 8))
    B = g.standard_normal((8, 8))
    na, nbn = _np_block_norms(A, bs), _np_block_norms(B, bs)
    taus = np.sort(np.concatenate([(na[:, :, None] * nbn[None, :, :]).ravel() * 1.0000001, [0.0]]))[::-1]
    b = orc.cse(A, B, bs, taus)
    for t, v in zip(taus, b):
        flat = 0.0
        for i in range(2):
            for j in range(2):
                s = sum(na[i, k] * nbn[k, j] for k in range(2) if na[i, k] * nbn[k, j] < t)
                flat += s * s
        assert v == pytest.approx(math.sqrt(flat), rel=1e-14, abs=0)


@pytest.mark.parametrize("n,bs,seed", [(32, 4, 1), (48, 8, 2), (64, 8, 3), (50, 4, 4), (64, 16, 5)])
def test_cse_bounds_true_error_for_every_tau(orc, n, bs, seed):
    A = synth.random_decaying(n, seed, length=3.0)
    B = synth.random_decaying(n, seed + 7, length=5.0)
    if seed % 2:
        B = B.T.copy()
    taus = orc.tau_table()
    b = orc.cse(A, B, bs, taus)
    AB = A @ B
    for k in range(0, 350, 7):
        C, _ = orc.spamm(A, B, taus[k], bs)
        err = np.linalg.norm(AB - C)
        assert err <= b[k] * (1 + 1e-12) + 1e-14 * np.linalg.norm(AB)
    assert np.all(np.diff(b) <= 0.0)                       # non-increasing in k
    assert b[0] <= np.linalg.norm(A) * np.linalg.norm(B) * (1 + 1e-14)


def test_select_tau_rule(orc):
    taus = orc.tau_table()
    A = synth.random_decaying(64, 21, length=4.0)
    b = orc.cse(A, A, 8, taus)
    for delta in [1e-1, 1e-3, 1e-6, 1e-9]:
        k = orc.select_tau(b, delta)
        assert k >= 0
        assert b[k] < delta and (k == 0 or b[k - 1] >= delta)
        r = orc.spamm_delta(A, A, delta, 8)
        assert r.k == k and r.tau == taus[k]
        assert np.linalg.norm(A @ A - r.C) < delta
    assert orc.select_tau(np.array([5.0, 4.0, 3.0]), 1.0) == -1


# ------------------------------------------------------------ truncation

@pytest.mark.parametrize("seed", range(6))
def test_truncate_brute_force(orc, seed):
    g = synth.rng(100 + seed)
    bs, nb = 2, 4
    n = bs * nb
    X = g.standard_normal((n, n)) * np.exp(g.uniform(-6, 0, size=(n, n)))
    X = 0.5 * (X + X.T)
    nrm = _np_block_norms(X, bs)
    w = [(nrm[i, j] ** 2 + (nrm[j, i] ** 2 if i != j else 0.0)) for i in range(nb) for j in range(i, nb)]
    delta = math.sqrt(np.sort(w)[: 2 + seed % 5].sum()) * 1.0000001
    r = orc.truncate(X, delta, bs)
    E = X - r.X
    assert np.linalg.norm(E) < delta
    # maximal count: no set with one more unit stays below delta^2
    m = r.removed_units
    best = min(sum(c) for c in itertools.combinations(w, m + 1)) if m + 1 <= len(w) else np.inf
    assert best >= delta * delta
    # the removed units are a minimal-sum choice among sets of that size
    assert r.removed_sq == pytest.approx(min(sum(c) for c in itertools.combinations(w, m)) if m else 0.0, rel=1e-12)
    assert np.allclose(r.X, r.X.T)


def test_block_norms_definition(orc):
    X = synth.random_decaying(70, 8)
    np.testing.assert_allclose(orc.block_norms(X, 16), _np_block_norms(X, 16), rtol=1e-14)


# ------------------------------------------------------------------ SP2

@pytest.mark.parametrize("variant", [1, 4, 5])
def test_sp2_diagonal_is_heaviside(orc, variant):
    g = synth.rng(31)
    n, n_occ = 64, 20
    f = np.sort(g.uniform(-2, 2, size=n))
    f[n_occ:] += 0.3                       # gap >= 0.3 between f[n_occ-1] and f[n_occ]
    perm = g.permutation(n)
    F = np.diag(f[perm])
    D = np.diag((perm < n_occ).astype(float))     # Eq. 1 with mu in the gap
    r = orc.purify(F, n_occ, 1e-5, 80, homo=f[n_occ - 1], lumo=f[n_occ], variant=variant, bs=8)
    assert r.converged
    assert np.linalg.norm(r.D - D) < 1e-5
    assert np.count_nonzero(r.D - np.diag(np.diag(r.D))) == 0


def test_sp2_two_by_two_closed_form(orc):
    F = np.array([[0.3, -0.4], [-0.4, -0.5]])
    ev = 0.5 * (0.3 - 0.5) + np.array([-1, 1]) * math.sqrt((0.4) ** 2 + 0.4 ** 2)
    v0 = np.array([0.4, 0.3 - ev[0]])            # (F - ev0 I) v = 0, first row gives this
    v0 /= np.linalg.norm(v0)
    D = np.outer(v0, v0)
    r = orc.purify(F, 1, 1e-6, 80, homo=ev[0], lumo=ev[1], variant=4, bs=1)
    assert r.converged
    assert np.linalg.norm(r.D - D) < 1e-6


@pytest.mark.parametrize("variant,gap_mode", [(1, "eig"), (4, "eig"), (5, "eig"), (5, "stagger")])
def test_sp2_lattice_matches_eigendecomposition(orc, variant, gap_mode):
    P = synth.lattice_fock(256, seed=7, gap_mode=gap_mode)
    r = orc.purify(P.F, P.n_occ, 1e-5, 60, P.homo, P.lumo, variant=variant, bs=32)
    D = orc.exact_density(P.F, P.n_occ)
    assert r.converged
    assert np.linalg.norm(r.D - D) < 1e-5
    assert abs(np.trace(r.D) - P.n_occ) < 1e-5
    assert np.linalg.norm(r.D @ r.D - r.D) < 1e-5
    # every per-step tolerance and the branch rule are what the driver says
    assert all(d > 0 for d in r.deltas)


# ------------------------------------------------------------ flat bound

def test_flat_bound_equals_algorithm3_at_one_level(orc):
    # a 2 x 2 leaf grid is a single level of Algorithm 3, where its recursion is
    # exactly the flat formula
    g = synth.rng(21)
    A = g.standard_normal((8, 8))
    B = g.standard_normal((8, 8))
    taus = np.array([0.0, 0.5, 1.0, 2.0, 4.0, 8.0, 16.0, 1e9])
    np.testing.assert_allclose(orc.flat_bound(A, B, 4, taus), orc.cse(A, B, 4, taus),
                               rtol=1e-14, atol=0)


def test_flat_bound_closed_forms(orc):
    n = 16
    J = np.ones((n, n))
    I = np.eye(n)
    # everything skipped (tau above every leaf product, bs = 1): J J has all
    # entries n, so the bound is sqrt(n^2 n^2) = n^2 = ||J J||_F; I I keeps only
    # the diagonal triples, sqrt(n) = ||I||_F
    assert orc.flat_bound(J, J, 1, [2.0])[0] == pytest.approx(n * n, rel=1e-15)
    assert orc.flat_bound(I, I, 1, [2.0])[0] == pytest.approx(np.sqrt(n), rel=1e-15)
    # nothing skipped at tau = 0
    assert orc.flat_bound(J, J, 1, [0.0])[0] == 0.0


@pytest.mark.parametrize("n,bs,seed", [(32, 4, 1), (48, 8, 2), (64, 8, 3), (50, 4, 4)])
def test_flat_bound_between_true_error_and_algorithm3(orc, n, bs, seed):
    A = synth.random_decaying(n, seed, length=3.0)
    B = synth.random_decaying(n, seed + 7, length=4.0)
    taus = orc.tau_table()[::7]
    flat = orc.flat_bound(A, B, bs, taus)
    alg3 = orc.cse(A, B, bs, taus)
    exact = A @ B
    # Minkowski: the one-level sum never exceeds the hierarchical one
    assert np.all(flat <= alg3 * (1 + 1e-13))
    for t, f in zip(taus, flat):
        C, _ = orc.spamm(A, B, float(t), bs)
        assert np.linalg.norm(C - exact) <= f * (1 + 1e-12) + 1e-14
    # non-increasing along the table
    assert np.all(np.diff(flat) <= 0)


@pytest.mark.parametrize("n,bs", [(64, 16), (100, 32)])
def test_purify_degenerate_occupations(orc, n, bs):
    """Eq. 1 with nothing occupied gives D = 0 and with everything occupied D = I;
    the eigendecomposition agrees, and no SP2 step is taken."""
    P = synth.lattice_fock(n, seed=5, gap_mode="stagger")
    for n_occ, want in ((0, np.zeros((n, n))), (n, np.eye(n))):
        r = orc.purify(P.F, n_occ, 1e-5, 30, P.homo, P.lumo, bs=bs)
        assert r.converged and r.iters == 0
        np.testing.assert_array_equal(r.D, want)
        np.testing.assert_allclose(orc.exact_density(P.F, n_occ), want, atol=1e-12)
