"""The paper's two-squares experiment (Section 5) on a small converged D: every
variant keeps ||X2 - X1^2||_F below delta, and the SpAMM product never holds
more blocks than the exact product that truncmul truncates."""
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_two_squares_error_below_delta(prec):
    import bench
    import paper_2005_10680_gb300 as sp
    ctx = sp.Context(0)
    P = synth.lattice_fock(1024, seed=31, gap_mode="eig")
    D, rep = ctx.purify(ctx.from_dense(P.F, 64), P.n_occ, 1e-6, 60, P.homo, P.lumo,
                        variant=5, prec=prec)
    assert rep["converged"]
    for delta in (1e-3, 1e-6):
        res = {name: bench.square_twice(ctx, D, delta, v, prec)
               for name, v in bench.PROTOCOL_VARIANTS}
        for name, r in res.items():
            # float64 rounding of the exact check square: ||D||_F^2 = n_occ, n = 1024
            assert r["err"] < delta + 1.12e-16 * P.n_occ * 32, (name, r)
            assert r["nnz_pct"]["X_out"] <= r["nnz_pct"]["product"]
        assert res["spamm"]["nnz_pct"]["product"] <= res["truncmul"]["nnz_pct"]["product"]
        assert res["truncmul"]["t_cse_ms"] == 0.0 and res["spamm"]["t_trunc_ms"] == 0.0
