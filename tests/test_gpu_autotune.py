"""Autotuner: chooses the fastest measured candidate, answers repeated keys from
its cache, and its choice is a configuration that runs."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu


def test_autotune_picks_fastest_and_caches(orc):
    import paper_2005_10680_gb300 as sp
    ctx = sp.Context(0)
    P = synth.lattice_fock(1024, seed=77, gap_mode="stagger")
    lmin, lmax = orc.gershgorin(P.F)
    X0 = (lmax * np.eye(1024) - P.F) / (lmax - lmin)
    G = ctx.from_dense(X0, 64)
    r = ctx.autotune(G, 1e-8)
    assert not r["cached"]
    times = {k: v for k, v in r["ms"].items() if v >= 0}
    assert len(times) == 4
    best = min(times, key=times.get)
    assert (r["prec"], r["bs"]) == (best.split("_")[0], int(best.split("bs")[1]))
    r2 = ctx.autotune(G, 1e-8)
    assert r2["cached"] and r2["bs"] == r["bs"] and r2["prec"] == r["prec"]
    r3 = ctx.autotune(G, 1e-8, allow_mixed=False)
    assert r3["prec"] == "fp64" and r3["ms"]["mixed_bs64"] < 0
    Xb = ctx.from_dense(X0, r["bs"])
    Y, rep = ctx.sp2_step(Xb, 0, delta=1e-8, prec=r["prec"])
    assert np.linalg.norm(Y.to_numpy() - X0 @ X0) < 1e-8
