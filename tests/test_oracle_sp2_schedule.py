"""Pins of the oracle's purification schedule against the mathematics, not itself.

The paper asks that every step's error E_i stay below a tolerance delta_i chosen so
that the result is within eps of the exact D (Algorithm 1, and the delta_i
requirement of the method's introduction), and leaves the choice of delta_i to its
references. The oracle's reading: propagate bounds h (unoccupied group) and l
(occupied group) of the iterate's spectrum through the scalar SP2 maps, widened by
delta_i each step (Weyl's inequality with ||E||_2 <= ||E||_F); take delta_i = eps
(l' - h') / (2 sqrt(2) n_iter) from the mapped gap l' - h', so that the subspace
error sum_i sqrt(2) delta_i / gap_i stays below eps / 2; stop when
2 (||C - X||_F + bound) < eps / 2. Checked here:

* the propagated bounds contain the true spectrum of every iterate (eigendecomposition
  of X_i), on diagonal and lattice matrices, in all three variants;
* sum_i sqrt(2) delta_i / gap_i <= eps / 2 with the true gaps of f_i(X_{i-1}), with
  n_iter barely above the steps taken, so that a budget off by sqrt(2) would fail;
* with every step error replaced by the worst one its tolerance allows (delta_i in
  Frobenius norm, coupling the HOMO and LUMO eigenvectors with one sign, so the
  subspace rotations add up) the result still lies within eps of D, and within 100x
  of it: the slack of the schedule is measured;
* the stop rule is strict: a step whose 2 ||X^2 - X||_F equals eps / 2 exactly does
  not stop;
* mutants of the driver (the sqrt(2) dropped, h - delta for h + delta, the iteration
  count in place of n_iter, <= in the stop rule) each fail one of the checks above.
"""
import math
import os
import sys
import types

import numpy as np
import pytest

import synth

ORACLE_SRC = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "oracle",
                          "__init__.py")


def _diag_problem(n=64, seed=5):
    g = synth.rng(seed)
    w = np.sort(g.uniform(-1.0, 1.0, n))
    n_occ = n // 2
    w[n_occ:] += 0.3                      # a gap of at least 0.3 at n_occ
    q = np.linalg.qr(g.standard_normal((n, n)))[0]
    return np.diag(w), q @ np.diag(w) @ q.T, n_occ, float(w[n_occ - 1]), float(w[n_occ])


def _lattice(n=256, seed=8, gap_mode="eig"):
    P = synth.lattice_fock(n, seed=seed, gap_mode=gap_mode)
    return P.F, P.n_occ, P.homo, P.lumo


def bounds_contain_spectrum(orc, F, n_occ, homo, lumo, variant, bs, eps=1e-5, n_iter=60):
    r = orc.purify(F, n_occ, eps, n_iter, homo, lumo, variant=variant, bs=bs, keep_iterates=True)
    n = F.shape[0]
    assert len(r.iterates) == len(r.hs) == len(r.ls) == r.iters + 1
    for X, h, l in zip(r.iterates, r.hs, r.ls):
        w = np.linalg.eigvalsh(0.5 * (X + X.T))
        if not (w[n - n_occ - 1] <= h and w[n - n_occ] >= l):
            return False
    return r.converged


def budget_sum(orc, F, n_occ, homo, lumo, variant, bs, eps, n_iter):
    """sum_i sqrt(2) delta_i / gap_i with gap_i the true gap of f_i(X_{i-1})."""
    r = orc.purify(F, n_occ, eps, n_iter, homo, lumo, variant=variant, bs=bs, keep_iterates=True)
    n = F.shape[0]
    total = 0.0
    for i, delta in enumerate(r.deltas):
        w = np.linalg.eigvalsh(0.5 * (r.iterates[i] + r.iterates[i].T))
        fw = w * w if r.branches[i] == "sq" else 2.0 * w - w * w
        gap = fw[n - n_occ:].min() - fw[: n - n_occ].max()
        total += math.sqrt(2.0) * delta / gap
    return total, r


def tight_budget_sum(orc, F, n_occ, homo, lumo, variant, bs, eps):
    """The budget sum with n_iter just above the steps the purification needs."""
    r60 = orc.purify(F, n_occ, eps, 60, homo, lumo, variant=variant, bs=bs)
    assert r60.converged
    for n_iter in range(r60.iters + 1, r60.iters + 5):
        total, r = budget_sum(orc, F, n_occ, homo, lumo, variant, bs, eps, n_iter)
        if r.converged:
            return total, r, n_iter
    raise AssertionError("no n_iter near the step count converges")


def stop_tie_iters(orc, variant):
    """F = diag(t, 1), spectral bounds [0, 1]: X_0 = diag(1 - t, 0) and the first
    step's ||X^2 - X||_F = t - t^2 exactly; with eps = 4 (t - t^2), 2 idem equals
    eps / 2, which must not stop. The next step (2X - X^2 = diag(1 - t^2, 0)) stops."""
    t = 2.0 ** -20
    F = np.diag([t, 1.0])
    eps = 4.0 * (t - t * t)
    r = orc.purify(F, 1, eps, 60, t, 1.0, variant=variant, bs=64, lmin=0.0, lmax=1.0)
    return r.iters, r.converged, r.D


# ------------------------------------------------------------------ pins

@pytest.mark.parametrize("variant", [1, 4, 5])
def test_bounds_contain_spectrum_diagonal(orc, variant):
    Fd, Fq, n_occ, homo, lumo = _diag_problem()
    for F in (Fd, Fq):
        assert bounds_contain_spectrum(orc, F, n_occ, homo, lumo, variant, bs=16)


@pytest.mark.parametrize("variant,gap_mode", [(1, "eig"), (4, "eig"), (5, "eig"), (5, "stagger")])
def test_bounds_contain_spectrum_lattice(orc, variant, gap_mode):
    F, n_occ, homo, lumo = _lattice(gap_mode=gap_mode)
    assert bounds_contain_spectrum(orc, F, n_occ, homo, lumo, variant, bs=32)


@pytest.mark.parametrize("variant", [1, 5])
def test_budget_with_true_gaps(orc, variant):
    F, n_occ, homo, lumo = _lattice()
    eps = 1e-5
    total, r, n_iter = tight_budget_sum(orc, F, n_occ, homo, lumo, variant, 32, eps)
    assert total <= 0.5 * eps
    # the sum is the designed sqrt(2) * budget per step, up to the true gaps being a
    # little wider than the propagated ones: it sits just below eps / 2 * iters / n_iter
    assert total >= 0.99 * 0.5 * eps * r.iters / n_iter


def _worst_perturbation(F, n_occ):
    """E = c (u w^T + w u^T) with u, w the eigenvectors of F at the HOMO and LUMO:
    it couples the two closest states across the gap, always with the same sign, so
    the rotations of the occupied subspace add up; ||E||_F = sqrt(2) c = 0.999 delta."""
    w, v = np.linalg.eigh(F)
    u, x = v[:, n_occ - 1], v[:, n_occ]
    M = np.outer(u, x) + np.outer(x, u)

    def perturb(X, delta):
        return (0.999 * delta / math.sqrt(2.0)) * M
    return perturb


@pytest.mark.parametrize("variant", [1, 4])
def test_worst_case_step_errors_stay_within_eps(orc, variant):
    F, n_occ, homo, lumo = _lattice()
    eps = 1e-5
    r = orc.purify(F, n_occ, eps, 60, homo, lumo, variant=variant, bs=32,
                   perturb=_worst_perturbation(F, n_occ))
    assert r.converged
    err = np.linalg.norm(r.D - orc.exact_density(F, n_occ))
    assert err < eps
    assert err > eps / 100.0


@pytest.mark.parametrize("variant", [1, 4, 5])
def test_stop_rule_is_strict(orc, variant):
    t = 2.0 ** -20
    iters, converged, D = stop_tie_iters(orc, variant)
    assert converged and iters == 1
    np.testing.assert_array_equal(D, np.diag([1.0 - t * t, 0.0]))


# --------------------------------------------------------------- mutants

MUTANTS = {
    "budget_without_sqrt2": ("budget = eps / (2.0 * math.sqrt(2.0) * n_iter)",
                             "budget = eps / (2.0 * n_iter)"),
    "h_minus_delta": ("h, l = hn + delta, ln - delta", "h, l = hn - delta, ln - delta"),
    "iteration_count_for_n_iter": ("delta = budget * (ln - hn)",
                                   "delta = eps / (2.0 * math.sqrt(2.0) * it) * (ln - hn)"),
    "stop_rule_not_strict": ("if 2.0 * idem < 0.5 * eps:", "if 2.0 * idem <= 0.5 * eps:"),
}


def _mutant(orc, old, new):
    src = open(ORACLE_SRC).read()
    assert src.count(old) == 1, old
    name = "oracle_mutant"
    mod = types.ModuleType(name)
    mod.__file__ = ORACLE_SRC            # the same compiled oracle.c underneath
    sys.modules[name] = mod              # dataclasses look their module up while defining
    try:
        exec(compile(src.replace(old, new), ORACLE_SRC, "exec"), mod.__dict__)
    finally:
        del sys.modules[name]
    return mod


def _pins_hold(m) -> bool:
    """A compact replay of the pins above on a mutated driver."""
    Fd, Fq, n_occ, homo, lumo = _diag_problem()
    F, no, ho, lu = _lattice()
    try:
        if not bounds_contain_spectrum(m, Fq, n_occ, homo, lumo, 4, bs=16):
            return False
        if not bounds_contain_spectrum(m, F, no, ho, lu, 5, bs=32):
            return False
        total, r, n_iter = tight_budget_sum(m, F, no, ho, lu, 5, 32, 1e-5)
        if total > 0.5e-5:
            return False
        iters, converged, _ = stop_tie_iters(m, 1)
        if not (converged and iters == 1):
            return False
    except AssertionError:
        return False
    return True


def test_pins_hold_for_the_oracle(orc):
    assert _pins_hold(orc)


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_rejected(orc, name):
    old, new = MUTANTS[name]
    assert not _pins_hold(_mutant(orc, old, new)), name
