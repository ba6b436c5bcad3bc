"""spamm_mat_to_blocks, the inverse of spamm_mat_from_blocks, and
spamm_mat_get_blocks against the dense export: matrices built from an unordered
block list (ragged edge included), SP2 products, and the same products after
truncation removed blocks."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

BS = 64


def _assemble(n, brow, bcol, tiles):
    nb = -(-n // BS)
    X = np.zeros((nb * BS, nb * BS))
    for t in range(len(brow)):
        i, j = int(brow[t]), int(bcol[t])
        X[i * BS:(i + 1) * BS, j * BS:(j + 1) * BS] = tiles[t]
    return X


@pytest.mark.parametrize("n", [200, 256])
def test_blocks_round_trip(n):
    import paper_2005_10680_gb300 as sp
    ctx = sp.Context(0)
    g = synth.rng(77 + n)
    nb = -(-n // BS)
    pick = [(i, j) for i in range(nb) for j in range(nb) if i == j or g.uniform() < 0.4]
    order = g.permutation(len(pick))                      # listed out of order
    brow = np.array([pick[t][0] for t in order], dtype=np.int32)
    bcol = np.array([pick[t][1] for t in order], dtype=np.int32)
    tiles = g.standard_normal((len(pick), BS, BS))
    M = ctx.from_blocks(n, BS, brow, bcol, tiles)
    r, c, T = M.to_blocks()
    rank = np.lexsort((bcol, brow))                       # row-major block order
    np.testing.assert_array_equal(r, brow[rank])
    np.testing.assert_array_equal(c, bcol[rank])
    want = _assemble(n, brow, bcol, tiles)
    want[n:, :] = 0.0                                     # entries outside n x n are zero
    want[:, n:] = 0.0
    got = _assemble(n, r, c, T)
    np.testing.assert_array_equal(got, want)
    np.testing.assert_array_equal(got[:n, :n], M.to_numpy())
    # selected blocks, stored and absent, the ragged corner among them
    qi = np.array([nb - 1, 0] + [int(x) for x in g.integers(0, nb, 6)], dtype=np.int32)
    qj = np.array([nb - 1, nb - 1] + [int(x) for x in g.integers(0, nb, 6)], dtype=np.int32)
    Q, present = M.get_blocks(qi, qj)
    stored = M.block_map()
    for t in range(len(qi)):
        i, j = int(qi[t]), int(qj[t])
        assert present[t] == stored[i, j]
        np.testing.assert_array_equal(Q[t], want[i * BS:(i + 1) * BS, j * BS:(j + 1) * BS])
    with pytest.raises(sp.SpammError) as ei:
        M.get_blocks([nb], [0])
    assert ei.value.status == 1
    E = ctx.from_blocks(n, BS, [], [], np.zeros((0, BS, BS)))
    r, c, T = E.to_blocks()
    assert len(r) == len(c) == len(T) == 0


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_blocks_of_products_and_truncated_products(prec):
    import paper_2005_10680_gb300 as sp
    n = 448
    ctx = sp.Context(0)
    X = synth.banded_decay(n, 5, length=8.0)
    C, _ = ctx.sp2_step(ctx.from_dense(X, BS), 0, delta=1e-6, prec=prec)
    r, c, T = C.to_blocks()
    assert len(r) == C.nnzb
    assert np.all(np.diff(r.astype(np.int64) * C.nb + c) > 0)
    np.testing.assert_array_equal(_assemble(n, r, c, T)[:n, :n], C.to_numpy())
    stored = C.block_map()
    assert stored.sum() == len(r) and stored[r, c].all()
    rep = ctx.truncate(C, 1e-3)
    assert rep["removed_blocks"] > 0
    r2, c2, T2 = C.to_blocks()
    assert len(r2) == C.nnzb == len(r) - rep["removed_blocks"]
    np.testing.assert_array_equal(_assemble(n, r2, c2, T2)[:n, :n], C.to_numpy())
