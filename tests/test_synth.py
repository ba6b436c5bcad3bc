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


def _ratio_stats(F, centres, decay):
    d = np.sqrt(((centres[:, None, :] - centres[None, :, :]) ** 2).sum(axis=-1))
    off = ~np.eye(len(F), dtype=bool)
    r = -F[off] / np.exp(-decay * d[off])
    return float(r.mean()), float(r.std())


def test_block_lattice_matches_the_dense_recipe():
    """Without a cutoff the block generator draws the dense generator's distribution:
    -F_ij / exp(-a d_ij) = 1 + 0.1 (g_ij + g_ji) / 2, mean 1 and deviation 0.1 / sqrt(2)."""
    n, a = 512, 0.8
    B = synth.lattice_fock_blocks(n, seed=4, decay=a, cutoff=1e9)
    assert B.fill == 1.0
    X = B.to_dense()
    np.testing.assert_array_equal(X, X.T)
    mean, std = _ratio_stats(X, B.centres, a)
    assert abs(mean - 1.0) < 0.005 and abs(std - 0.1 / np.sqrt(2)) < 0.005
    D = synth.lattice_fock(n, seed=4, decay=a, gap_mode="stagger")
    mean_d, std_d = _ratio_stats(D.F, D.centres, a)
    assert abs(mean_d - 1.0) < 0.005 and abs(std_d - 0.1 / np.sqrt(2)) < 0.005


@pytest.mark.parametrize("n,cutoff", [(2048, 2.5), (4096, 3.0)])
def test_block_lattice_cutoff_pattern_and_gap(n, cutoff):
    B = synth.lattice_fock_blocks(n, seed=6, cutoff=cutoff)
    X = B.to_dense()
    np.testing.assert_array_equal(X, X.T)
    d = np.sqrt(((B.centres[:, None, :] - B.centres[None, :, :]) ** 2).sum(axis=-1))
    off = ~np.eye(n, dtype=bool)
    assert np.all(X[off & (d > cutoff)] == 0.0)              # hard cutoff
    assert np.all(X[off & (d <= cutoff)] != 0.0)
    assert np.all(np.abs(X[off]) <= np.exp(-B.decay * d[off]) * 1.6)
    # a block is stored exactly when it holds a pair of sites within the cutoff
    nb = n // 64
    dblk = d.reshape(nb, 64, nb, 64).min(axis=(1, 3))
    stored = np.zeros((nb, nb), dtype=bool)
    stored[B.brow, B.bcol] = True
    np.testing.assert_array_equal(stored, dblk <= cutoff)
    assert np.all(np.diff(B.brow.astype(np.int64) * nb + B.bcol) > 0)   # row-major order
    # the staggered shift certifies the gap at n_occ (Gershgorin): eigenvalues agree
    w = np.linalg.eigvalsh(X)
    assert w[B.n_occ - 1] <= B.homo and w[B.n_occ] >= B.lumo and B.lumo - B.homo >= 0.1 - 1e-12
    # the pattern alone is the same and the stream does not depend on the caller
    Q = synth.lattice_fock_blocks(n, seed=6, cutoff=cutoff, pattern_only=True)
    np.testing.assert_array_equal(Q.brow, B.brow)
    np.testing.assert_array_equal(Q.bcol, B.bcol)
    np.testing.assert_array_equal(synth.lattice_fock_blocks(n, seed=6, cutoff=cutoff).tiles, B.tiles)


def test_large_lattice_block_fill():
    """n = 262144 (65536 sites in a 64 x 32 x 32 box) at the default cutoff 6: about 3 %
    of the 4096 x 4096 leaf blocks, about 5.5e5 tiles (18 GB of float64)."""
    Q = synth.lattice_fock_blocks(262144, pattern_only=True)
    assert 0.02 <= Q.fill <= 0.05
    assert np.ptp(Q.centres, axis=0).round().tolist() == [63.0, 31.0, 31.0]
