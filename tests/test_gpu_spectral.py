"""Spectral-norm error control and a tuned tau list (the conclusion's future work)
on the GPU, through the C ABI, against the oracle.

Bars: the spectral bound equals the oracle's min(||M||_F, sqrt(||M||_1 ||M||_inf))
and the same formula on the GPU's own leaf norms within 1e-12, never exceeds the
flat bound, and bounds the true spectral error; searches with it certify
||E||_2 < delta in both leaf forms and select the oracle's candidate; the
purification drivers refuse it. A tuned list selects the oracle's candidate from
the same list, every worker of a batched purification uses it, and bad lists are
refused."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def _spec(NA, NB, tau):
    P = NA[:, :, None] * NB[None, :, :]          # p_ikj, axes (i, k, j)
    M = np.where(P < tau, P, 0.0).sum(axis=1)    # sum over k
    return min(float(np.sqrt((M ** 2).sum())), float(np.sqrt(M.sum(0).max() * M.sum(1).max())))


def _x0(orc, n, seed):
    P = synth.lattice_fock(n, seed=seed, gap_mode="stagger")
    lmin, lmax = orc.gershgorin(P.F)
    return P, (lmax * np.eye(n) - P.F) / (lmax - lmin)


@pytest.mark.parametrize("n,seed,bs", [(448, 3, 64), (1000, 4, 64), (640, 5, 32)])
def test_spectral_bound_formula_and_order(orc, n, seed, bs):
    import paper_2005_10680_gb300 as sp
    A = synth.random_decaying(n, seed, length=n / 12.0)
    B = synth.random_decaying(n, seed + 1, length=n / 9.0)
    ctx = sp.Context(0)
    GA, GB = ctx.from_dense(A, bs), ctx.from_dense(B, bs)
    taus = orc.tau_table()[::25]
    ctx.set_bound("flat")
    ef = ctx.cse(GA, GB, taus)
    ctx.set_bound("spectral")
    es = ctx.cse(GA, GB, taus)
    np.testing.assert_allclose(es, orc.spectral_bound(A, B, bs, taus), rtol=1e-12, atol=0)
    NA, NB = GA.block_norms(), GB.block_norms()
    np.testing.assert_allclose(es, [_spec(NA, NB, t) for t in taus], rtol=1e-12, atol=0)
    assert np.all(es <= ef)                      # the same Frobenius sum, then a minimum
    fp64_noise = 1.12e-16 * np.linalg.norm(A) * np.linalg.norm(B) * np.sqrt(n)
    for k in (40, 120, 200):
        C, rep = ctx.multiply_tau(GA, GB, float(orc.tau_table()[k]))
        assert np.linalg.norm(C.to_numpy() - A @ B, 2) <= rep["bound"] + fp64_noise


def test_spectral_search_selects_the_oracle_candidate(orc):
    import paper_2005_10680_gb300 as sp
    n = 640
    A = synth.random_decaying(n, 8, length=20.0)
    B = synth.random_decaying(n, 9, length=30.0)
    ctx = sp.Context(0)
    ctx.set_bound("spectral")
    GA, GB = ctx.from_dense(A, 64), ctx.from_dense(B, 64)
    e = orc.spectral_bound(A, B, 64, orc.tau_table())
    fp64_noise = 1.12e-16 * np.linalg.norm(A) * np.linalg.norm(B) * np.sqrt(n)
    for delta in (1e-1, 1e-4, 1e-7):
        C, rep = ctx.multiply(GA, GB, delta)
        k = orc.select_tau(e, delta)
        if rep["tau_index"] != k:                # only a tie at delta may move the choice
            assert k >= 0 and rep["tau_index"] >= 0
            assert min(abs(e[k] - delta), abs(e[rep["tau_index"]] - delta)) <= 1e-10 * delta
        assert rep["bound"] < delta
        assert np.linalg.norm(C.to_numpy() - A @ B, 2) <= rep["bound"] + fp64_noise


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_spectral_sp2_step_certifies_the_spectral_norm(orc, prec):
    import paper_2005_10680_gb300 as sp
    n = 768
    _, X = _x0(orc, n, 14)
    exact = X @ X
    fp64_noise = 1.12e-16 * np.linalg.norm(X) ** 2 * np.sqrt(n)
    for delta in (1e-3, 1e-6, 1e-9):
        cs = sp.Context(0)
        cs.set_bound("spectral")
        Ys, rs = cs.sp2_step(cs.from_dense(X, 64), 0, delta=delta, prec=prec)
        assert rs["bound"] < delta
        assert np.linalg.norm(Ys.to_numpy() - exact, 2) <= rs["bound"] + fp64_noise
        if prec == "fp64":
            cf = sp.Context(0)
            cf.set_bound("flat")
            _, rf = cf.sp2_step(cf.from_dense(X, 64), 0, delta=delta, prec=prec)
            if rs["tau_index"] >= 0 and rf["tau_index"] >= 0:
                assert rs["tau_index"] <= rf["tau_index"]     # never a smaller tau
                assert rs["kept"] <= rf["kept"]


def test_purification_refuses_the_spectral_bound(orc):
    import paper_2005_10680_gb300 as sp
    P, _ = _x0(orc, 256, 3)
    ctx = sp.Context(0)
    ctx.set_bound("spectral")
    F = ctx.from_dense(P.F, 64)
    with pytest.raises(sp.SpammError) as ei:
        ctx.purify(F, P.n_occ, 1e-5, 60, P.homo, P.lumo)
    assert ei.value.status == 1
    with pytest.raises(sp.SpammError) as ei:
        ctx.purify_batched([F], [P.n_occ], 1e-5, 60, [P.homo], [P.lumo])
    assert ei.value.status == 1


def test_tuned_tau_table(orc):
    import paper_2005_10680_gb300 as sp
    n = 640
    A = synth.random_decaying(n, 11, length=20.0)
    B = synth.random_decaying(n, 12, length=30.0)
    ctx = sp.Context(0)
    GA, GB = ctx.from_dense(A, 64), ctx.from_dense(B, 64)
    fp64_noise = 1.12e-16 * np.linalg.norm(A) * np.linalg.norm(B) * np.sqrt(n)
    for start, ratio in ((8.0, 0.95), (1.0, 0.9), (1e3, 0.8)):
        ctx.set_tau_table(start, ratio)
        table = orc.tau_table_scaled(350, start, ratio)
        e = orc.cse(A, B, 64, table)
        for delta in (1e-2, 1e-5):
            C, rep = ctx.multiply(GA, GB, delta)
            k = orc.select_tau(e, delta)
            if rep["tau_index"] != k:            # only a tie at delta may move the choice
                assert k >= 0 and rep["tau_index"] >= 0
                assert min(abs(e[k] - delta), abs(e[rep["tau_index"]] - delta)) <= 1e-12 * delta
            if rep["tau_index"] >= 0:
                assert rep["tau"] == table[rep["tau_index"]]
            assert rep["bound"] < delta
            assert np.linalg.norm(C.to_numpy() - A @ B) <= rep["bound"] + fp64_noise
    assert np.array_equal(orc.tau_table_scaled(350, 1.0, 0.9), orc.tau_table())
    for bad in ((0.0, 0.9), (np.inf, 0.9), (np.nan, 0.9), (1.0, 1.0), (1.0, 0.0), (1e-300, 0.5)):
        with pytest.raises(sp.SpammError) as ei:
            ctx.set_tau_table(*bad)
        assert ei.value.status == 1


def test_batched_workers_use_the_tuned_table(orc):
    import paper_2005_10680_gb300 as sp
    ctx = sp.Context(0)
    ctx.set_tau_table(16.0, 0.95)
    probs = [synth.lattice_fock(n, seed=200 + n, gap_mode="stagger") for n in (256, 320)]
    Fs = [ctx.from_dense(P.F, 64) for P in probs]
    out = ctx.purify_batched(Fs, [P.n_occ for P in probs], 1e-5, 60,
                             [P.homo for P in probs], [P.lumo for P in probs], workers=2)
    for P, F, (D, rep) in zip(probs, Fs, out):
        assert rep["status"] == 0 and rep["converged"]
        Ds, reps = ctx.purify(F, P.n_occ, 1e-5, 60, P.homo, P.lumo)
        np.testing.assert_array_equal(D.to_numpy(), Ds.to_numpy())
        assert np.linalg.norm(D.to_numpy() - orc.exact_density(P.F, P.n_occ)) < 1e-5
