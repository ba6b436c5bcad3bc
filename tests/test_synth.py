"""The synthetic inputs follow their stated recipe: symmetry, decay, sign pattern,
the enforced gap at n_occ, and reproducibility from the seed."""
import numpy as np
import pytest

import synth


def test_banded_decay_recipe():
    n, L = 300, 40.0
    X = synth.banded_decay(n, seed=3, length=L, drop=1e-12)
    np.testing.assert_array_equal(X, X.T)
    i = np.arange(n)
    d = np.abs(i[:, None] - i[None, :])
    env = np.exp(-d / L)
    nz = X != 0
    # |X_ij| = u exp(-|i-j|/L) with u in [0.5, 1); the sign is (-1)^(i+j)
    assert np.all(np.abs(X[nz]) <= env[nz] * (1 + 1e-15))
    assert np.all(np.abs(X[nz]) >= 0.5 * env[nz] * (1 - 1e-15))
    sign = np.where(((i[:, None] + i[None, :]) & 1) == 0, 1.0, -1.0)
    assert np.all(np.sign(X[nz]) == sign[nz])
    # entries below the drop level are zero, the others are kept
    assert np.all(np.abs(X[nz]) >= 1e-12)
    assert np.all(0.5 * env[~nz] < 1e-12)
    np.testing.assert_array_equal(X, synth.banded_decay(n, seed=3, length=L, drop=1e-12))


@pytest.mark.parametrize("gap_mode", ["eig", "stagger"])
def test_lattice_fock_gap_and_symmetry(gap_mode):
    n = 384
    P = synth.lattice_fock(n, seed=5, gap_mode=gap_mode)
    F = P.F
    np.testing.assert_array_equal(F, F.T)
    assert P.n_occ == n // 2
    w = np.linalg.eigvalsh(F)
    # the stated bounds hold and leave the requested gap at n_occ
    assert w[P.n_occ - 1] <= P.homo + 1e-10
    assert w[P.n_occ] >= P.lumo - 1e-10
    assert w[P.n_occ] - w[P.n_occ - 1] >= 0.1 - 1e-9
    # the eigenvector shift keeps a safety slack of 1e-9 max|lambda| on each bound
    assert P.lumo - P.homo >= 0.1 - 2e-9 * np.abs(w).max() - 1e-12
    np.testing.assert_array_equal(F, synth.lattice_fock(n, seed=5, gap_mode=gap_mode).F)


def test_lattice_fock_off_diagonal_decay():
    # before any shift the off-diagonal entries are -exp(-a d) (1 + 0.1 g): with
    # gap_mode="stagger" only the diagonal moves, so the off-diagonal envelope is
    # that of the distance between the sites of the two basis functions
    n, a = 256, 0.8
    P = synth.lattice_fock(n, seed=9, decay=a, gap_mode="stagger", jitter=0.0)
    sites = synth._morton_points(n // 4).astype(np.float64)
    pos = np.repeat(sites, 4, axis=0)
    d = np.linalg.norm(pos[:, None, :] - pos[None, :, :], axis=2)
    off = ~np.eye(n, dtype=bool)
    g_abs = np.abs(P.F[off] / -np.exp(-a * d[off]) - 1.0) / 0.1
    # 1 + 0.1 g with g standard normal: |g| below 10 for every entry of this draw
    assert np.all(np.isfinite(g_abs)) and g_abs.max() < 10.0
