"""Block-sparse inputs: the planners and Algorithm 3 walk only stored pairs (row lists
and the live node triples of the recursion), and must give what the oracle gives.

Inputs are the lattice Fock matrix with a hard distance cutoff (19-44 % block fill at
the sizes here), its X_0 map, and patterns built to empty whole branches of the
recursion. Bars as for dense inputs: Algorithm 3 vectors and products within 1e-12
relative of the oracle, the same tau index (unless the bound at the boundary ties
delta), kept sets equal up to triples within 1e-12 of tau, and ||C - AB||_F < delta."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

REL = 1e-12


@pytest.fixture(scope="module")
def gctx():
    import paper_2005_10680_gb300 as sp
    return sp.Context(0)


def _rel(a, b):
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def _x0(B):
    """X_0 = (lmax I - F) / (lmax - lmin) of a block lattice, dense, with F's pattern
    plus the diagonal."""
    import oracle
    F = B.to_dense()
    lmin, lmax = oracle.gershgorin(F)
    return (lmax * np.eye(B.n) - F) / (lmax - lmin)


CASES = [  # n, bs, cutoff, seed: fill 19 %, 29 %, 32 %
    (2048, 32, 1.5, 1),
    (2048, 32, 3.0, 3),
    (2048, 64, 1.5, 2),
]


def _pattern(X, bs):
    nb = -(-X.shape[0] // bs)
    pad = np.zeros((nb * bs, nb * bs))
    pad[:X.shape[0], :X.shape[1]] = X
    return np.abs(pad).reshape(nb, bs, nb, bs).sum(axis=(1, 3)) > 0


@pytest.mark.parametrize("n,bs,cutoff,seed", CASES + [(4096, 64, 2.0, 4), (4096, 64, 4.0, 5)])
def test_sparse_cse_matches_oracle(gctx, orc, n, bs, cutoff, seed):
    B = synth.lattice_fock_blocks(n, seed=seed, bs=bs, cutoff=cutoff)
    X = _x0(B)
    taus = orc.tau_table()
    ref = orc.cse(X, X, bs, taus)
    GX = gctx.from_dense(X, bs)
    got = gctx.cse(GX, GX, taus)
    np.testing.assert_allclose(got, ref, rtol=REL, atol=0)
    assert 0.1 < _pattern(X, bs).mean() < 0.5


@pytest.mark.parametrize("n,bs,cutoff,seed", CASES)
def test_sparse_multiply_matches_oracle(gctx, orc, n, bs, cutoff, seed):
    B = synth.lattice_fock_blocks(n, seed=seed, bs=bs, cutoff=cutoff)
    X = _x0(B)
    GX = gctx.from_dense(X, bs)
    for delta in (1e-4, 1e-8):
        r = orc.spamm_delta(X, X, delta, bs)
        C, rep = gctx.multiply(GX, GX, delta)
        if rep["tau_index"] != r.k:
            errs = orc.cse(X, X, bs)
            kk = min(rep["tau_index"], r.k)
            assert abs(errs[kk] - delta) <= REL * delta
        else:
            assert rep["tau"] == r.tau
            assert rep["bound"] == pytest.approx(r.bound, rel=REL, abs=0)
            assert _rel(C.to_numpy(), r.C) <= REL
        # candidates are the stored pairs only
        P = _pattern(X, bs).astype(np.int64)
        assert rep["candidates"] == int((P.sum(axis=0) * P.sum(axis=1)).sum())
        assert np.linalg.norm(C.to_numpy() - X @ X) < delta
        assert rep["bound"] < delta


@pytest.mark.parametrize("n,bs,cutoff,seed", CASES[:2])
def test_sparse_multiply_tau_kept_set(gctx, orc, n, bs, cutoff, seed):
    B = synth.lattice_fock_blocks(n, seed=seed + 10, bs=bs, cutoff=cutoff)
    X = _x0(B)
    Y = X[::-1, ::-1].copy()          # another pattern for the right operand
    GX, GY = gctx.from_dense(X, bs), gctx.from_dense(Y, bs)
    na, nbn = orc.block_norms(X, bs), orc.block_norms(Y, bs)
    p = na[:, :, None] * nbn[None, :, :]
    both = (na > 0)[:, :, None] & (nbn > 0)[None, :, :]
    taus = orc.tau_table()
    for k in (0, 80, 160, 240):
        tau = float(taus[k])
        C, rep = gctx.multiply_tau(GX, GY, tau)
        ref, cnt = orc.spamm(X, Y, tau, bs)
        keep = both & ~(p < tau)
        border = int(np.count_nonzero(both & (np.abs(p - tau) <= REL * tau)))
        assert cnt == int(keep.sum())
        assert abs(rep["kept"] - cnt) <= border
        assert _rel(C.to_numpy(), ref) <= REL
        if border == 0:
            np.testing.assert_array_equal(C.block_map(), keep.any(axis=1))


@pytest.mark.parametrize("branch", [0, 1])
@pytest.mark.parametrize("prec,n,cutoff", [("fp64", 2048, 1.5), ("mixed", 2048, 1.5),
                                           ("mixed", 4096, 1.5)])
def test_sparse_sp2_step(gctx, orc, prec, n, cutoff, branch):
    B = synth.lattice_fock_blocks(n, seed=31, bs=64, cutoff=cutoff)
    X = _x0(B)
    G = gctx.from_dense(X, 64)
    delta = 1e-9
    Xn, rep = gctx.sp2_step(G, branch, delta=delta, prec=prec)
    C = X @ X
    want = C if branch == 0 else 2 * X - C
    got = Xn.to_numpy()
    np.testing.assert_array_equal(got, got.T)
    noise = 1.12e-16 * np.linalg.norm(X) ** 2 * np.sqrt(n)
    assert rep["bound"] < delta
    assert np.linalg.norm(got - want) <= rep["bound"] + noise
    if prec == "fp64":
        r = orc.spamm_delta(X, X, delta, 64)
        if rep["tau_index"] == r.k:
            ref = r.C if branch == 0 else 2 * X - r.C
            assert _rel(got, ref) <= REL


@pytest.mark.parametrize("bound", ["flat", "spectral"])
def test_sparse_flat_and_spectral_match_oracle(orc, bound):
    import paper_2005_10680_gb300 as sp
    B = synth.lattice_fock_blocks(2048, seed=41, bs=32, cutoff=2.0)
    X = _x0(B)
    Y = synth.lattice_fock_blocks(2048, seed=42, bs=32, cutoff=1.5).to_dense()
    ctx = sp.Context(0)
    ctx.set_bound(bound)
    taus = orc.tau_table()[::7]
    got = ctx.cse(ctx.from_dense(X, 32), ctx.from_dense(Y, 32), taus)
    ref = (orc.flat_bound if bound == "flat" else orc.spectral_bound)(X, Y, 32, taus)
    np.testing.assert_allclose(got, ref, rtol=REL, atol=0)


def test_disjoint_patterns_and_empty_branches(gctx, orc):
    """A stored only in block columns [0, nb/2), B only in block rows [nb/2, nb): both
    are non-zero, the root triple of the recursion is live, but no triple below it is,
    and A B = 0. A second pair keeps one quadrant of candidates only."""
    n, bs = 1024, 32
    g = synth.rng(77)
    A = np.zeros((n, n))
    A[:, : n // 2] = g.standard_normal((n, n // 2))
    B = np.zeros((n, n))
    B[n // 2:, :] = g.standard_normal((n // 2, n))
    GA, GB = gctx.from_dense(A, bs), gctx.from_dense(B, bs)
    taus = orc.tau_table()[::50]
    assert not gctx.cse(GA, GB, taus).any()
    C, rep = gctx.multiply(GA, GB, 1e-6)
    assert rep["candidates"] == 0 and rep["nnzb_out"] == 0 and rep["bound"] == 0.0
    assert not C.to_numpy().any()
    # B stored in the first half of its rows only: one K half of the cube is live
    B2 = np.zeros((n, n))
    B2[: n // 2, n // 4: n // 2] = g.standard_normal((n // 2, n // 4))
    GB2 = gctx.from_dense(B2, bs)
    np.testing.assert_allclose(gctx.cse(GA, GB2, taus), orc.cse(A, B2, bs, taus), rtol=REL,
                               atol=0)
    r = orc.spamm_delta(A, B2, 1e-3, bs)
    C2, rep2 = gctx.multiply(GA, GB2, 1e-3)
    assert rep2["tau_index"] == r.k
    assert _rel(C2.to_numpy(), r.C) <= REL
