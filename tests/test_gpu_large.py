"""The full-size configurations, opt-in (``pytest tests -m gpu --run-large``): each
needs a GB300 to itself for minutes and tens of GB of device and host memory.

* n = 262144 lattice at 3.25 % block fill (5.5e5 leaf blocks, 18 GB): one certified
  SP2 step X_0^2 at delta = 1e-7 in both leaf forms, sampled output blocks against
  float64 block products on the CPU; then the mixed purification to eps = 1e-5.
* n = 65536 lattice, dense (34 GB per matrix): the mixed purification (the float64
  form would take hours at ~1.25 TFLOP/s).
* 96 independent purifications, n from 1024 to 16384, decay U(0.5, 1.2), batched,
  in the mixed form.

Where no exact density matrix can be formed, the purification is checked by its
own invariants: convergence of the stop rule, the trace n_occ, idempotency."""
import numpy as np
import pytest

import synth

pytestmark = [pytest.mark.gpu, pytest.mark.large]

BS = 64


def _gershgorin(B):
    n = B.n
    R, d = np.zeros(n), np.zeros(n)
    for t in range(len(B.brow)):
        I, J = int(B.brow[t]), int(B.bcol[t])
        a = np.abs(B.tiles[t]).sum(axis=1)
        if I == J:
            dd = np.diag(B.tiles[t])
            d[I * BS:(I + 1) * BS] = dd
            a = a - np.abs(dd)
        R[I * BS:(I + 1) * BS] += a
    return float((d - R).min()), float((d + R).max())


def _x0_tiles(B):
    """X_0 = (lmax I - F) / (lmax - lmin) on F's block pattern (every diagonal block is
    stored)."""
    lmin, lmax = _gershgorin(B)
    w = lmax - lmin
    T = B.tiles * (-1.0 / w)
    for t in np.nonzero(B.brow == B.bcol)[0]:
        T[t][np.diag_indices(BS)] += lmax / w
    return T


@pytest.fixture(scope="module")
def lattice_262144():
    # the bench's input: decay 4.0, cutoff 6 (3.25 % block fill), seed of the fifth
    # configuration
    return synth.lattice_fock_blocks(262144, seed=synth.SEED_BASE + 4, decay=4.0, cutoff=6.0)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_sp2_step_n262144(lattice_262144, prec):
    import paper_2005_10680_gb300 as sp
    B = lattice_262144
    T = _x0_tiles(B)
    ctx = sp.Context(0)
    X = ctx.from_blocks(B.n, BS, B.brow, B.bcol, T)
    delta = 1e-7
    C, rep = ctx.sp2_step(X, 0, delta=delta, prec=prec)
    assert rep["bound"] < delta
    slot = {(int(i), int(j)): t for t, (i, j) in enumerate(zip(B.brow, B.bcol))}
    cols = {}
    for (i, k), t in slot.items():
        cols.setdefault(i, []).append((k, t))
    norm = np.linalg.norm(T.reshape(len(T), -1), axis=1)
    g = synth.rng(262144)
    nb = B.n // BS
    near = [(int(B.brow[t]), int(B.bcol[t])) for t in g.integers(0, len(B.brow), 12)]
    far = [(int(i), int(j)) for i, j in zip(g.integers(0, nb, 12), g.integers(0, nb, 12))]
    qi = np.array([p[0] for p in near + far], dtype=np.int32)
    qj = np.array([p[1] for p in near + far], dtype=np.int32)
    got, present = C.get_blocks(qi, qj)
    tau = rep["tau"]
    fp64_noise = 1.12e-16 * np.sqrt(B.n) * float(np.sqrt((norm ** 2).sum())) ** 2
    for q in range(len(qi)):
        i, j = int(qi[q]), int(qj[q])
        full = np.zeros((BS, BS))
        kept = np.zeros((BS, BS))
        kept_scale = 0.0
        tie = False
        for k, ta in cols.get(i, []):
            tb = slot.get((k, j))
            if tb is None:
                continue
            prod = T[ta] @ T[tb]
            full += prod
            p = norm[ta] * norm[tb]
            tie |= abs(p - tau) <= 1e-10 * tau
            if p >= tau:
                kept += prod
                kept_scale += p
        # every block of the error is within the certified bound of the whole error
        assert np.linalg.norm(got[q] - full) <= rep["bound"] + fp64_noise
        if prec == "fp64" and not tie:
            # the float64 form forms exactly the products with p >= tau (up to the
            # rounding of sums of a few hundred products)
            assert np.linalg.norm(got[q] - kept) <= 1e-13 * kept_scale
        if not present[q]:
            assert not got[q].any()
    # the symmetric step writes C_ji = C_ij^T
    gt, _ = C.get_blocks(qj, qi)
    np.testing.assert_array_equal(gt, np.transpose(got, (0, 2, 1)))


def test_purification_n262144_mixed(lattice_262144):
    import paper_2005_10680_gb300 as sp
    B = lattice_262144
    ctx = sp.Context(0)
    F = ctx.from_blocks(B.n, BS, B.brow, B.bcol, B.tiles)
    eps = 1e-5
    D, rep = ctx.purify(F, B.n_occ, eps, 60, B.homo, B.lumo, prec="mixed")
    assert rep["converged"]
    assert rep["idem"] < eps
    assert abs(rep["trace"] - B.n_occ) < np.sqrt(B.n) * eps


def test_purification_n65536_mixed():
    import paper_2005_10680_gb300 as sp
    B = synth.lattice_fock_blocks(65536, decay=0.8, cutoff=1e9)     # dense, the 0.8 recipe
    ctx = sp.Context(0)
    F = ctx.from_blocks(B.n, BS, B.brow, B.bcol, B.tiles)
    del B.tiles
    eps = 1e-5
    D, rep = ctx.purify(F, B.n_occ, eps, 60, B.homo, B.lumo, prec="mixed")
    print(f"n=65536 dense lattice, mixed: {rep['ms_total']:.0f} ms, {rep['iters']} steps, "
          f"slice levels {rep['step_lmax']}, idem {rep['idem']:.3g}, "
          f"trace - n_occ {rep['trace'] - B.n_occ:.3g}")
    assert rep["converged"]
    assert rep["idem"] < eps
    assert abs(rep["trace"] - B.n_occ) < np.sqrt(B.n) * eps


def test_batched_96_mixed(orc):
    import concurrent.futures

    import paper_2005_10680_gb300 as sp
    g = synth.rng(96)
    sizes = [4 * int(x) for x in g.integers(256, 4097, 96)]
    decays = g.uniform(0.5, 1.2, 96)
    # the inputs are built by host threads (numpy releases the interpreter lock in its
    # array operations), before the first GPU call
    with concurrent.futures.ThreadPoolExecutor(8) as ex:
        probs = list(ex.map(lambda q: synth.lattice_fock(sizes[q], seed=1000 + q,
                                                         decay=float(decays[q]),
                                                         gap_mode="stagger"), range(96)))
    ctx = sp.Context(0)
    Fs = [ctx.from_dense(P.F, BS) for P in probs]
    eps = 1e-5
    import time
    t0 = time.perf_counter()
    out = ctx.purify_batched(Fs, [P.n_occ for P in probs], eps, 60, [P.homo for P in probs],
                             [P.lumo for P in probs], prec="mixed", workers=8)
    wall = time.perf_counter() - t0
    # the batch against the problems' own purification times (each worker's events)
    print(f"batched 96: {wall * 1e3:.0f} ms for the batch, sum of single purifications "
          f"{sum(r['ms_total'] for _, r in out):.0f} ms, n from {min(sizes)} to {max(sizes)}")
    for P, (D, rep) in zip(probs, out):
        assert rep["status"] == 0 and rep["converged"]
        assert rep["idem"] < eps
        assert abs(rep["trace"] - P.n_occ) < np.sqrt(len(P.F)) * eps
        if len(P.F) <= 2048:
            assert np.linalg.norm(D.to_numpy() - orc.exact_density(P.F, P.n_occ)) < eps
