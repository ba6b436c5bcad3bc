"""Failure paths, made on the host: a device allocation refused by the library's
injection hook (at many points of a call), and a purification stopped by n_iter.

After a refused allocation an entry point must return SPAMM_ENOMEM with the
injected message, and the same context must then give exactly the result of a
clean call. A purification that reaches n_iter before its stop rule returns
SPAMM_ENOTCONV with D and its report filled, alone and in a batch."""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

ENOMEM, ENOTCONV = 2, 5
AFTER = [0, 1, 2, 3, 5, 8, 13, 21, 34, 55, 89, 144, 233]


@pytest.fixture
def lib():
    import paper_2005_10680_gb300 as sp
    lib = sp.load_library()
    yield lib
    lib.spamm_debug_fail_alloc(-1)


def _x0(n, cutoff, seed):
    import oracle
    B = synth.lattice_fock_blocks(n, seed=seed, bs=64, cutoff=cutoff)
    F = B.to_dense()
    lmin, lmax = oracle.gershgorin(F)
    return (lmax * np.eye(n) - F) / (lmax - lmin)


def _injected(lib, call):
    """Run call() with failures armed at every point of AFTER; return how many calls
    were refused (the others had fewer allocations than the armed one)."""
    import paper_2005_10680_gb300 as sp
    refused = 0
    for after in AFTER:
        lib.spamm_debug_fail_alloc(after)
        try:
            call()
        except sp.SpammError as e:
            assert e.status == ENOMEM, e
            assert b"injected" in lib.spamm_last_error()
            refused += 1
        finally:
            lib.spamm_debug_fail_alloc(-1)
    return refused


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_refused_allocations_in_a_product_leave_the_context_usable(lib, prec):
    import paper_2005_10680_gb300 as sp
    ctx = sp.Context(0)
    X = _x0(2048, 1.5, 51)
    G = ctx.from_dense(X, 64)
    C, rep = ctx.sp2_step(G, 0, delta=1e-8, prec=prec)
    ref = C.to_numpy()
    del C
    refused = _injected(lib, lambda: ctx.sp2_step(G, 0, delta=1e-8, prec=prec))
    assert refused >= 8
    C, rep2 = ctx.sp2_step(G, 0, delta=1e-8, prec=prec)
    np.testing.assert_array_equal(C.to_numpy(), ref)
    assert rep2["tau_index"] == rep["tau_index"]
    # the plain product and the truncation after refusals, too
    P0, _ = ctx.multiply(G, G, 1e-8, prec=prec)
    assert _injected(lib, lambda: ctx.multiply(G, G, 1e-8, prec=prec)) >= 8
    P1, _ = ctx.multiply(G, G, 1e-8, prec=prec)
    np.testing.assert_array_equal(P1.to_numpy(), P0.to_numpy())
    T0 = ctx.from_dense(X, 64)
    ctx.truncate(T0, 1e-6)
    T1 = ctx.from_dense(X, 64)
    assert _injected(lib, lambda: ctx.truncate(T1, 1e-6)) >= 1
    np.testing.assert_array_equal(T1.to_numpy(), T0.to_numpy())


def test_refused_allocations_in_a_purification(lib):
    import paper_2005_10680_gb300 as sp
    P = synth.lattice_fock(256, seed=17, gap_mode="eig")
    ctx = sp.Context(0)
    F = ctx.from_dense(P.F, 32)
    D0, r0 = ctx.purify(F, P.n_occ, 1e-5, 60, P.homo, P.lumo)
    ref = D0.to_numpy()
    refused = 0
    for after in (0, 7, 40, 150, 400, 900):
        lib.spamm_debug_fail_alloc(after)
        try:
            ctx.purify(F, P.n_occ, 1e-5, 60, P.homo, P.lumo)
        except sp.SpammError as e:
            assert e.status == ENOMEM
            refused += 1
        finally:
            lib.spamm_debug_fail_alloc(-1)
    assert refused >= 5
    D1, r1 = ctx.purify(F, P.n_occ, 1e-5, 60, P.homo, P.lumo)
    np.testing.assert_array_equal(D1.to_numpy(), ref)
    assert r1["iters"] == r0["iters"]


def test_not_converged_single_and_batched():
    import paper_2005_10680_gb300 as sp
    P = synth.lattice_fock(256, seed=18, gap_mode="eig")
    Q = synth.lattice_fock(384, seed=19, gap_mode="stagger")
    ctx = sp.Context(0)
    F, G = ctx.from_dense(P.F, 32), ctx.from_dense(Q.F, 64)
    D, rep = ctx.purify(F, P.n_occ, 1e-5, 3, P.homo, P.lumo, strict=False)
    assert rep["status"] == ENOTCONV and rep["iters"] == 3 and not rep["converged"]
    assert D.n == 256 and D.nnzb > 0
    assert abs(rep["trace"] - np.trace(D.to_numpy())) <= 1e-9 * 256
    with pytest.raises(sp.SpammError) as ei:
        ctx.purify(F, P.n_occ, 1e-5, 3, P.homo, P.lumo)
    assert ei.value.status == ENOTCONV
    out = ctx.purify_batched([F, G], [P.n_occ, Q.n_occ], 1e-5, 3, [P.homo, Q.homo],
                             [P.lumo, Q.lumo], workers=2)
    for Dq, r in out:
        assert r["status"] == ENOTCONV and r["iters"] == 3 and not r["converged"]
        assert Dq.nnzb > 0
    # with room to converge the same calls succeed
    out = ctx.purify_batched([F, G], [P.n_occ, Q.n_occ], 1e-5, 60, [P.homo, Q.homo],
                             [P.lumo, Q.lumo], workers=2)
    assert all(r["status"] == 0 and r["converged"] for _, r in out)
