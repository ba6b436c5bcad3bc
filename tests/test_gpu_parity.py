"""GPU path vs the CPU oracle, through the C ABI, on seeded synthetic inputs.

Bars (FP64 form): leaf norms and Algorithm 3 bounds within 1e-12 relative;
the kept leaf-product set identical except for triples whose norm product is
within 1e-12 relative of tau; products within 1e-12 relative Frobenius of the
oracle; ||C - AB||_F < delta; truncation removing the same blocks except at a
unit whose running sum is within 1e-12 of delta^2; purification with the same
branch sequence (unless a trace ties n_occ) and ||D - D~||_F < eps."""
import math

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


def _flat_kept(orc, A, B, tau, bs):
    na, nbn = orc.block_norms(A, bs), orc.block_norms(B, bs)
    pa, pb = na > 0, nbn > 0
    p = na[:, :, None] * nbn[None, :, :]
    both = pa[:, :, None] & pb[None, :, :]
    keep = both & ~(p < tau)
    kept = int(np.count_nonzero(keep))
    border = int(np.count_nonzero(both & (np.abs(p - tau) <= REL * tau)))
    return kept, border, keep.any(axis=1)


CASES = [  # n, bs, kind, seed
    (64, 32, "band", 1),
    (200, 32, "rand", 2),        # ragged tail: 200 = 6*32 + 8
    (512, 64, "band", 3),
    (300, 64, "rand", 4),
    (640, 128, "band", 5),
    (1000, 32, "lattice", 6),
]


def _input(kind, n, seed):
    if kind == "band":
        return synth.banded_decay(n, seed, length=n / 16.0)
    if kind == "rand":
        return synth.random_decaying(n, seed, length=n / 20.0)
    P = synth.lattice_fock(n, seed=seed, gap_mode="stagger")
    return P.F / 100.0


# ---------------------------------------------------------------- storage

@pytest.mark.parametrize("n,bs,kind,seed", CASES)
def test_store_roundtrip_and_norms(gctx, orc, n, bs, kind, seed):
    X = _input(kind, n, seed)
    M = gctx.from_dense(X, bs=bs)
    np.testing.assert_array_equal(M.to_numpy(), X)
    nrm = M.block_norms()
    ref = orc.block_norms(X, bs)
    np.testing.assert_allclose(nrm, ref, rtol=REL, atol=0)
    assert M.nnzb == int(np.count_nonzero(ref > 0))


def test_store_drop_and_empty(gctx):
    X = synth.banded_decay(256, 9, length=4.0, drop=0.0)
    M = gctx.from_dense(X, bs=32, drop=1e-3)
    Y = X.copy()
    Y[np.abs(Y) < 1e-3] = 0.0
    np.testing.assert_array_equal(M.to_numpy(), Y)
    Z = gctx.from_dense(np.zeros((100, 100)), bs=32)
    assert Z.nnzb == 0
    assert not Z.to_numpy().any()


# ------------------------------------------------------------ Algorithm 3

@pytest.mark.parametrize("n,bs,kind,seed", CASES[:5])
def test_cse_matches_oracle(gctx, orc, n, bs, kind, seed):
    A = _input(kind, n, seed)
    B = _input(kind, n, seed + 50).T.copy()
    taus = orc.tau_table()
    ref = orc.cse(A, B, bs, taus)
    got = gctx.cse(gctx.from_dense(A, bs), gctx.from_dense(B, bs), taus)
    np.testing.assert_allclose(got, ref, rtol=REL, atol=0)


# ------------------------------------------------------------ Algorithm 2

@pytest.mark.parametrize("n,bs,kind,seed", CASES)
def test_multiply_tau_matches_oracle(gctx, orc, n, bs, kind, seed):
    A = _input(kind, n, seed)
    B = _input(kind, n, seed + 1)
    GA, GB = gctx.from_dense(A, bs), gctx.from_dense(B, bs)
    taus = orc.tau_table()
    for k in (0, 30, 60, 120, 349):
        tau = float(taus[k])
        C, rep = gctx.multiply_tau(GA, GB, tau)
        ref, cnt = orc.spamm(A, B, tau, bs)
        kept, border, pattern = _flat_kept(orc, A, B, tau, bs)
        assert cnt == kept
        assert abs(rep["kept"] - kept) <= border
        assert _rel(C.to_numpy(), ref) <= REL
        if border == 0:
            # output blocks are exactly those with a kept product (no fill-in)
            np.testing.assert_array_equal(C.block_map(), pattern)


def test_multiply_exact_and_everything_skipped(gctx, orc):
    A = synth.random_decaying(320, 3, length=12.0)
    GA = gctx.from_dense(A, 64)
    C, rep = gctx.multiply_tau(GA, GA, 0.0)
    assert _rel(C.to_numpy(), A @ A) <= 1e-13
    big = np.linalg.norm(A) ** 2 * 2
    C, rep = gctx.multiply_tau(GA, GA, big)
    assert rep["kept"] == 0 and rep["nnzb_out"] == 0 and not C.to_numpy().any()
    Z = gctx.from_dense(np.zeros((320, 320)), 64)
    C, rep = gctx.multiply(Z, GA, 1e-6)
    assert rep["nnzb_out"] == 0 and rep["bound"] == 0.0


@pytest.mark.parametrize("n,bs,kind,seed,delta", [
    (64, 32, "band", 11, 1e-3), (256, 32, "band", 12, 1e-6), (384, 64, "rand", 13, 1e-4),
    (512, 128, "band", 14, 1e-8), (1000, 32, "lattice", 15, 1e-7)])
def test_multiply_delta_matches_oracle(gctx, orc, n, bs, kind, seed, delta):
    A = _input(kind, n, seed)
    B = A if kind != "rand" else _input(kind, n, seed + 1)
    r = orc.spamm_delta(A, B, delta, bs)
    C, rep = gctx.multiply(gctx.from_dense(A, bs), gctx.from_dense(B, bs), delta)
    errs = orc.cse(A, B, bs)
    if rep["tau_index"] != r.k:
        # only when the bound at the boundary candidate ties delta
        kk = min(rep["tau_index"], r.k)
        assert abs(errs[kk] - delta) <= REL * delta
    else:
        assert rep["tau"] == r.tau
        assert rep["bound"] == pytest.approx(r.bound, rel=REL, abs=0)
        assert _rel(C.to_numpy(), r.C) <= REL
    exact = A @ B
    assert np.linalg.norm(C.to_numpy() - exact) < delta
    assert rep["bound"] < delta


@pytest.mark.slow
def test_multiply_banded_n2048_bs32_delta1e6(gctx, orc):
    """The n = 2048, bs = 32, delta = 1e-6 banded-decay product, end to end."""
    X = synth.banded_decay(2048, synth.SEED_BASE + 0, length=40.0, drop=1e-12)
    r = orc.spamm_delta(X, X, 1e-6, 32)
    C, rep = gctx.multiply(gctx.from_dense(X, 32), gctx.from_dense(X, 32), 1e-6)
    assert rep["tau_index"] == r.k
    assert _rel(C.to_numpy(), r.C) <= REL
    assert np.linalg.norm(C.to_numpy() - X @ X) < 1e-6


# --------------------------------------------------------------- truncation

@pytest.mark.parametrize("n,bs,seed,frac", [(256, 32, 1, 0.3), (500, 32, 2, 0.9),
                                            (512, 64, 3, 0.5), (768, 128, 4, 0.7)])
def test_truncate_matches_oracle(gctx, orc, n, bs, seed, frac):
    X = synth.banded_decay(n, seed, length=n / 12.0)
    nrm = orc.block_norms(X, bs)
    delta = math.sqrt(np.sort((nrm ** 2).ravel())[: int(frac * nrm.size)].sum()) + 1e-300
    ref = orc.truncate(X, delta, bs)
    G = gctx.from_dense(X, bs)
    rep = gctx.truncate(G, delta)
    got = G.to_numpy()
    diff = np.argwhere(orc.block_norms(got - ref.X, bs) > 0)
    assert len(diff) <= 2  # at most the one boundary unit (two blocks)
    if len(diff):
        assert abs(ref.removed_sq - delta * delta) <= REL * delta * delta * 10
    assert np.linalg.norm(X - got) < delta
    assert rep["removed_sq"] < delta * delta


def test_truncate_nonsymmetric_and_nothing(gctx, orc):
    X = synth.random_decaying(300, 7, length=10.0)
    G = gctx.from_dense(X, 32)
    rep = gctx.truncate(G, 1e-300, symmetric=False)
    assert rep["removed_blocks"] == 0
    np.testing.assert_array_equal(G.to_numpy(), X)
    nrm = orc.block_norms(X, 32)
    delta = math.sqrt(np.sort((nrm ** 2).ravel())[:40].sum()) * 1.0000001
    ref = orc.truncate(X, delta, 32, symmetric=False)
    rep = gctx.truncate(G, delta, symmetric=False)
    np.testing.assert_array_equal(G.to_numpy(), ref.X)


# ---------------------------------------------------------------- SP2 step

@pytest.mark.parametrize("branch", [0, 1])
def test_sp2_step_matches_oracle(gctx, orc, branch):
    P = synth.lattice_fock(512, seed=21, gap_mode="stagger")
    lmin, lmax = orc.gershgorin(P.F)
    X = (lmax * np.eye(512) - P.F) / (lmax - lmin)
    G = gctx.from_dense(X, 64)
    tau = 1e-9
    Xn, rep = gctx.sp2_step(G, branch, tau=tau)
    C, cnt = orc.spamm(X, X, tau, 64)
    want = C if branch == 0 else 2 * X - C
    got = Xn.to_numpy()
    assert _rel(got, want) <= REL
    # symmetric X: only blocks i <= j are formed and mirrored, so the result is exactly symmetric
    np.testing.assert_array_equal(got, got.T)
    kept, border, _ = _flat_kept(orc, X, X, tau, 64)
    assert cnt == kept and abs(rep["kept"] - kept) <= border
    nb = 512 // 64
    assert rep["formed"] < rep["kept"] and rep["formed"] >= rep["kept"] // 2
    assert rep["idem"] == pytest.approx(np.linalg.norm(C - X), rel=1e-10)
    assert rep["trace_out"] == pytest.approx(np.trace(want), rel=1e-12)


# ------------------------------------------------------------- purification

@pytest.mark.parametrize("variant,gap_mode,n,bs", [
    (1, "eig", 256, 32), (4, "eig", 256, 32), (5, "eig", 256, 32), (5, "stagger", 512, 64),
    (4, "stagger", 384, 128)])
def test_purify_matches_oracle_and_eigendecomposition(gctx, orc, variant, gap_mode, n, bs):
    P = synth.lattice_fock(n, seed=7, gap_mode=gap_mode)
    eps = 1e-5
    ref = orc.purify(P.F, P.n_occ, eps, 60, P.homo, P.lumo, variant=variant, bs=bs)
    D, rep = gctx.purify(gctx.from_dense(P.F, bs), P.n_occ, eps, 60, P.homo, P.lumo,
                         variant=variant)
    Dx = orc.exact_density(P.F, P.n_occ)
    got = D.to_numpy()
    assert rep["converged"] and ref.converged
    assert np.linalg.norm(got - Dx) < eps
    assert abs(np.trace(got) - P.n_occ) < eps
    branches = ["sq" if b == 0 else "dbl" for b in rep["branches"]]
    if branches != ref.branches:
        # a branch may only differ where the trace ties n_occ
        k = next(i for i, (a, b) in enumerate(zip(branches, ref.branches)) if a != b)
        assert abs(ref.traces[k] - P.n_occ) <= 1e-10 * n
    else:
        assert rep["iters"] == ref.iters
        np.testing.assert_allclose(rep["deltas"], ref.deltas, rtol=1e-12)
        assert np.linalg.norm(got - ref.D) <= 1e-7


@pytest.mark.parametrize("n,bs", [(300, 64), (256, 32), (520, 128)])
def test_from_blocks_roundtrip(gctx, orc, n, bs):
    g = synth.rng(n + bs)
    X = synth.random_decaying(n, n, length=n / 10.0)
    nb = -(-n // bs)
    # a sparse block list in shuffled order; entries of the boundary blocks beyond n
    # are given as garbage and must come back as zeros
    pad = np.zeros((nb * bs, nb * bs))
    pad[:n, :n] = X
    keep = [(i, j) for i in range(nb) for j in range(nb) if (i + 2 * j) % 3 != 1]
    order = g.permutation(len(keep))
    brow = np.array([keep[t][0] for t in order], dtype=np.int32)
    bcol = np.array([keep[t][1] for t in order], dtype=np.int32)
    tiles = np.stack([pad[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] for i, j in zip(brow, bcol)])
    outside = np.zeros_like(tiles, dtype=bool)
    for t, (i, j) in enumerate(zip(brow, bcol)):
        rows = np.arange(bs) + i * bs >= n
        cols = np.arange(bs) + j * bs >= n
        outside[t] = rows[:, None] | cols[None, :]
    tiles = np.where(outside, 7.0, tiles)
    M = gctx.from_blocks(n, bs, brow, bcol, tiles)
    want = np.zeros((n, n))
    for i, j in keep:
        want[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs] = pad[i * bs:(i + 1) * bs, j * bs:(j + 1) * bs][
            :max(0, min(bs, n - i * bs)), :max(0, min(bs, n - j * bs))]
    np.testing.assert_array_equal(M.to_numpy(), want)
    np.testing.assert_allclose(M.block_norms(), orc.block_norms(want, bs), rtol=1e-14, atol=0)
    assert M.nnzb == len(keep)


def test_from_blocks_rejects_bad_lists(gctx):
    import paper_2005_10680_gb300 as sp
    t = np.zeros((2, 32, 32))
    with pytest.raises(sp.SpammError):
        gctx.from_blocks(64, 32, [0, 0], [1, 1], t)       # the same block twice
    with pytest.raises(sp.SpammError):
        gctx.from_blocks(64, 32, [0, 2], [0, 0], t)       # outside the 2 x 2 block grid
    E = gctx.from_blocks(64, 32, [], [], np.zeros((0, 32, 32)))
    assert E.nnzb == 0 and not E.to_numpy().any()


@pytest.mark.parametrize("bad", [np.nan, np.inf, -np.inf, 1e300])
def test_constructors_reject_non_finite_entries(gctx, bad):
    """NaN or infinite entries, or entries whose squares overflow, make the leaf norms
    that Algorithm 3 and the truncation compare meaningless: both constructors
    refuse them with SPAMM_EINVAL, including in a block that holds nothing else."""
    import paper_2005_10680_gb300 as sp
    A = np.zeros((100, 100))
    A[3, 5] = 1.0
    A[70, 90] = bad                      # block (1, 1) holds only this entry
    for drop in (0.0, 1e-3):
        with pytest.raises(sp.SpammError) as ei:
            gctx.from_dense(A, 64, drop=drop)
        assert ei.value.status == 1
    t = np.zeros((2, 64, 64))
    t[0, 0, 0] = 2.0
    t[1, 6, 26] = bad                    # entry (70, 90) of block (1, 1)
    with pytest.raises(sp.SpammError) as ei:
        gctx.from_blocks(100, 64, [0, 1], [0, 1], t)
    assert ei.value.status == 1
    # outside the matrix (n = 100) the entry is zeroed before the norms: accepted
    t[1, 6, 26] = 0.0
    t[1, 50, 50] = bad
    M = gctx.from_blocks(100, 64, [0, 1], [0, 1], t)
    assert np.isfinite(M.to_numpy()).all()
