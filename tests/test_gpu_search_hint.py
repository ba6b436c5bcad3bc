"""The tau and slice-level searches start from the previous selection made on the
same context; they must select exactly what a search from scratch selects."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_hinted_search_matches_fresh_search(orc, prec):
    import paper_2005_10680_gb300 as sp
    n = 768
    P = synth.lattice_fock(n, seed=12, gap_mode="stagger")
    lmin, lmax = orc.gershgorin(P.F)
    X = (lmax * np.eye(n) - P.F) / (lmax - lmin)
    deltas = [1e-4, 1e-10, 1e-5, 2e-6, 1e-12, 3e-3, 1e-8, 1e-8]
    hinted = sp.Context(0)
    G = hinted.from_dense(X, 64)
    for d in deltas:
        _, rh = hinted.sp2_step(G, 0, delta=d, prec=prec)
        fresh = sp.Context(0)
        _, rf = fresh.sp2_step(fresh.from_dense(X, 64), 0, delta=d, prec=prec)
        assert rh["tau_index"] == rf["tau_index"], (d, rh["tau_index"], rf["tau_index"])
        assert rh["lmax"] == rf["lmax"], (d, rh["lmax"], rf["lmax"])
        assert rh["bound"] == rf["bound"] and rh["kept"] == rf["kept"]
        taus = orc.tau_table()
        assert rh["bound"] < d
        if rh["tau_index"] > 0:
            # the next larger tau of the table does not certify delta
            _, rprev = fresh.sp2_step(fresh.from_dense(X, 64), 0, tau=float(taus[rh["tau_index"] - 1]),
                                      prec=prec)
            if prec == "fp64":
                assert rprev["bound"] >= d
