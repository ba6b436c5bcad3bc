"""Batched purification (independent problems of different sizes purified
concurrently, one host worker and CUDA stream each) against the single-problem
entry point and the eigendecomposition of Eq. 1."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_batched_equals_single_and_eigendecomposition(orc, prec):
    import paper_2005_10680_gb300 as sp
    ctx = sp.Context(0)
    sizes = [256, 448, 640, 320, 512, 192]
    g = synth.rng(55)
    probs = [synth.lattice_fock(n, seed=100 + i, decay=float(g.uniform(0.5, 1.2)),
                                gap_mode="stagger") for i, n in enumerate(sizes)]
    Fs = [ctx.from_dense(P.F, 64) for P in probs]
    out = ctx.purify_batched(Fs, [P.n_occ for P in probs], 1e-5, 60,
                             [P.homo for P in probs], [P.lumo for P in probs], prec=prec,
                             workers=3)
    for P, F, (D, rep) in zip(probs, Fs, out):
        assert rep["status"] == 0 and rep["converged"]
        Ds, reps = ctx.purify(F, P.n_occ, 1e-5, 60, P.homo, P.lumo, prec=prec)
        got = D.to_numpy()
        np.testing.assert_array_equal(got, Ds.to_numpy())
        assert rep["iters"] == reps["iters"]
        assert np.linalg.norm(got - orc.exact_density(P.F, P.n_occ)) < 1e-5


def test_batched_empty_and_bad_arguments():
    import paper_2005_10680_gb300 as sp
    ctx = sp.Context(0)
    assert ctx.purify_batched([], [], 1e-5, 60, [], []) == []
    with pytest.raises(sp.SpammError):
        ctx.purify_batched([ctx.from_dense(np.eye(64), 64)], [10], 1e-5, 60, [2.0], [1.0])
