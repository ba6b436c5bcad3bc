"""Degenerate occupations through the C ABI: n_occ = 0 gives D = 0 and n_occ = n gives
D = I exactly (Eq. 1 with the chemical potential outside the spectrum), without an
SP2 step, in both leaf forms, for a ragged size, through the single and the batched
entry points."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_degenerate_occupations(orc, prec):
    import paper_2005_10680_gb300 as sp
    ctx = sp.Context(0)
    n = 200
    P = synth.lattice_fock(n, seed=8, gap_mode="stagger")
    F = ctx.from_dense(P.F, 64)
    zero, eye = np.zeros((n, n)), np.eye(n)
    for n_occ, want, blocks in ((0, zero, 0), (n, eye, 4)):
        D, rep = ctx.purify(F, n_occ, 1e-5, 30, P.homo, P.lumo, prec=prec)
        assert rep["converged"] and rep["iters"] == 0
        assert rep["trace"] == n_occ and rep["idem"] == 0.0
        assert D.nnzb == blocks
        np.testing.assert_array_equal(D.to_numpy(), want)
    Q = synth.lattice_fock(256, seed=9, gap_mode="stagger")       # an ordinary problem beside them
    G = ctx.from_dense(Q.F, 64)
    out = ctx.purify_batched([F, F, G], [0, n, Q.n_occ], 1e-5, 60, [P.homo, P.homo, Q.homo],
                             [P.lumo, P.lumo, Q.lumo], prec=prec, workers=2)
    np.testing.assert_array_equal(out[0][0].to_numpy(), zero)
    np.testing.assert_array_equal(out[1][0].to_numpy(), eye)
    assert out[2][1]["status"] == 0 and out[2][1]["converged"]
    assert np.linalg.norm(out[2][0].to_numpy() - orc.exact_density(Q.F, Q.n_occ)) < 1e-5
