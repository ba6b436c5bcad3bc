"""The flat (one-level) bound: the GPU value equals the oracle's
sqrt(sum_ij (sum_k p_ikj [p_ikj < tau])^2), never exceeds Algorithm 3's bound,
still bounds the true error, and so certifies a tau at least as large."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _flat(NA, NB, tau):
    P = NA[:, :, None] * NB[None, :, :]          # p_ikj, axes (i, k, j)
    S = np.where(P < tau, P, 0.0).sum(axis=1)    # sum over k
    return float(np.sqrt((S ** 2).sum()))


@pytest.mark.parametrize("n,seed", [(448, 3), (1000, 4)])
def test_flat_bound_formula_and_order(orc, n, seed):
    import paper_2005_10680_gb300 as sp
    A = synth.random_decaying(n, seed, length=n / 12.0)
    B = synth.random_decaying(n, seed + 1, length=n / 9.0)
    ctx = sp.Context(0)
    GA, GB = ctx.from_dense(A, 64), ctx.from_dense(B, 64)
    taus = orc.tau_table()[::25]
    e3 = ctx.cse(GA, GB, taus)
    ctx.set_bound("flat")
    ef = ctx.cse(GA, GB, taus)
    np.testing.assert_allclose(ef, orc.flat_bound(A, B, 64, taus), rtol=1e-12, atol=0)
    NA, NB = GA.block_norms(), GB.block_norms()
    want = np.array([_flat(NA, NB, t) for t in taus])
    np.testing.assert_allclose(ef, want, rtol=1e-12, atol=0)
    assert np.all(ef <= e3 * (1 + 1e-12))
    # still an upper bound on the true error of the SpAMM product (float64 rounding of
    # the products themselves is not part of any bound: u ||A||_F ||B||_F sqrt(n))
    fp64_noise = 1.12e-16 * np.linalg.norm(A) * np.linalg.norm(B) * np.sqrt(n)
    for k in (40, 120, 200):
        tau = float(orc.tau_table()[k])
        C, rep = ctx.multiply_tau(GA, GB, tau)
        assert np.linalg.norm(C.to_numpy() - A @ B) <= rep["bound"] + fp64_noise


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_flat_bound_search_certifies_a_larger_tau(orc, prec):
    import paper_2005_10680_gb300 as sp
    n = 768
    P = synth.lattice_fock(n, seed=14, gap_mode="stagger")
    lmin, lmax = orc.gershgorin(P.F)
    X = (lmax * np.eye(n) - P.F) / (lmax - lmin)
    fp64_noise = 1.12e-16 * np.linalg.norm(X) ** 2 * np.sqrt(n)
    exact = X @ X
    for delta in (1e-3, 1e-6, 1e-9):
        c3 = sp.Context(0)
        Y3, r3 = c3.sp2_step(c3.from_dense(X, 64), 0, delta=delta, prec=prec)
        cf = sp.Context(0)
        cf.set_bound("flat")
        Yf, rf = cf.sp2_step(cf.from_dense(X, 64), 0, delta=delta, prec=prec)
        assert rf["bound"] < delta
        assert np.linalg.norm(Yf.to_numpy() - exact) <= rf["bound"] + fp64_noise
        if r3["tau_index"] >= 0 and rf["tau_index"] >= 0 and prec == "fp64":
            assert rf["tau_index"] <= r3["tau_index"]
            assert rf["kept"] <= r3["kept"]
