"""The bench workload's size, in the bench's launch configuration: one SP2 step
X0^2 at n = 16384 (3D-lattice Fock, leaf 64), mixed and float64 forms. The oracle
cannot form a 16384^3 product in test time, so sampled output blocks are checked
one by one against float64 row-block x column-block products, and the sampled
error must stay within the step's certified bound."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

N = 16384
BS = 64


@pytest.fixture(scope="module")
def x0(orc):
    P = synth.lattice_fock(N, seed=synth.SEED_BASE + 1, gap_mode="stagger")
    lmin, lmax = orc.gershgorin(P.F)
    X = -P.F / (lmax - lmin)
    X[np.diag_indices(N)] += lmax / (lmax - lmin)
    return X


@pytest.mark.parametrize("prec,delta", [("mixed", 1e-10), ("mixed", 1e-6), ("fp64", 1e-8)])
def test_sp2_step_full_size_sampled_blocks(x0, prec, delta):
    import paper_2005_10680_gb300 as sp
    ctx = sp.Context(0)
    G = ctx.from_dense(x0, BS)
    Y, rep = ctx.sp2_step(G, 0, delta=delta, prec=prec)
    assert rep["bound"] < delta
    y = Y.to_numpy()
    nb = N // BS
    g = np.random.default_rng(5)
    picks = {(0, 0), (nb - 1, nb - 1), (0, nb - 1), (nb - 1, 0), (1, 0), (nb // 2, nb // 2 + 1)}
    while len(picks) < 24:
        picks.add((int(g.integers(nb)), int(g.integers(nb))))
    err2 = 0.0
    noise = 0.0
    for i, j in sorted(picks):
        rows = x0[i * BS:(i + 1) * BS, :]
        cols = x0[:, j * BS:(j + 1) * BS]
        ref = rows @ cols
        blk = y[i * BS:(i + 1) * BS, j * BS:(j + 1) * BS]
        err2 += float(np.sum((blk - ref) ** 2))
        noise += 1.12e-16 * np.linalg.norm(rows) * np.linalg.norm(cols) * np.sqrt(N)
        # symmetric step: the block below the diagonal is the exact transpose
        np.testing.assert_array_equal(y[j * BS:(j + 1) * BS, i * BS:(i + 1) * BS], blk.T)
    assert np.sqrt(err2) <= rep["bound"] + noise
    assert abs(rep["trace_out"] - float(np.trace(y))) <= 1e-9 * abs(rep["trace_out"])
