"""Seeded synthetic inputs for SpAMM and SP2 purification.

This module only builds input matrices. It holds none of the method's
arithmetic (no norms, no products, no thresholds, no purification), so both
the CUDA path and the CPU oracle can take their inputs from here.

Workloads (the paper's water-cluster density matrix is not available, so
these decaying, symmetric, block-sparse matrices stand in for it):

* ``banded_decay``  -- X_ij = (-1)^(i+j) u_ij exp(-|i-j|/L), u ~ U(0.5, 1),
  mirrored, entries below ``drop`` set to zero.
* ``lattice_fock``  -- a Fock-like matrix over basis functions centred on a
  jittered cubic lattice: F_ij = -exp(-a d_ij) (1 + 0.1 g_ij) off the
  diagonal, F_ii ~ U(-0.5, 0.5), symmetrised, with a HOMO-LUMO gap enforced
  at n_occ = n/2 either by an eigenvector-based shift (``gap_mode="eig"``) or
  by a Gershgorin-certified staggered onsite shift (``gap_mode="stagger"``).

Seeds use numpy's PCG64. All matrices are float64 and row-major.
"""
from __future__ import annotations

import dataclasses

import numpy as np

SEED_BASE = 2005_10680


def rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def banded_decay(n: int, seed: int = SEED_BASE, length: float = 40.0,
                 drop: float = 1e-12) -> np.ndarray:
    """Symmetric matrix with exponentially decaying, sign-alternating entries."""
    g = rng(seed)
    u = g.uniform(0.5, 1.0, size=(n, n))
    i = np.arange(n)
    dist = np.abs(i[:, None] - i[None, :]).astype(np.float64)
    sign = np.where(((i[:, None] + i[None, :]) & 1) == 0, 1.0, -1.0)
    x = sign * u * np.exp(-dist / length)
    x = np.triu(x)
    x = x + np.triu(x, 1).T
    x[np.abs(x) < drop] = 0.0
    return np.ascontiguousarray(x)


def _morton_points(count: int) -> np.ndarray:
    """First ``count`` integer points of the 3-D lattice in Morton (Z) order."""
    bits = max(1, int(np.ceil(np.log2(max(2, count)) / 3.0)) + 1)
    side = 1 << bits
    code = np.arange(side ** 3, dtype=np.int64)
    xyz = np.zeros((side ** 3, 3), dtype=np.int64)
    for b in range(bits):
        for axis in range(3):
            xyz[:, axis] |= ((code >> (3 * b + axis)) & 1) << b
    return xyz[:count]


@dataclasses.dataclass
class FockProblem:
    F: np.ndarray        # (n, n) float64 symmetric
    n_occ: int           # number of occupied states
    homo: float          # upper bound on the n_occ-th smallest eigenvalue
    lumo: float          # lower bound on the (n_occ+1)-th smallest eigenvalue
    decay: float
    gap_mode: str
    occupied: np.ndarray = None   # occupied eigenvectors (gap_mode="eig", keep_vectors=True)
    eigvals: np.ndarray = None    # spectrum of F after the shift (gap_mode="eig")


def lattice_fock(n: int, seed: int = SEED_BASE, decay: float = 0.8,
                 gap: float = 0.1, gap_mode: str = "eig", jitter: float = 0.1,
                 funcs_per_site: int = 4, drop: float = 0.0, eigh=None,
                 keep_vectors: bool = False) -> FockProblem:
    """Fock-like matrix on a jittered cubic lattice (basis in Morton order of sites).

    ``eigh`` (optional) replaces numpy.linalg.eigh for the eigenvector-based
    gap shift, e.g. a GPU eigensolver for large n; it must return ascending
    eigenvalues and orthonormal eigenvectors as numpy arrays.
    """
    if n % funcs_per_site:
        raise ValueError("n must be a multiple of funcs_per_site")
    g = rng(seed)
    sites = n // funcs_per_site
    pts = _morton_points(sites).astype(np.float64)
    pts = pts + g.uniform(-jitter, jitter, size=pts.shape)
    centre = np.repeat(pts, funcs_per_site, axis=0)
    F = np.zeros((n, n))
    for ax in range(3):                      # squared distances, one axis at a time
        c = centre[:, ax]
        dif = c[:, None] - c[None, :]
        dif *= dif
        F += dif
        del dif
    np.sqrt(F, out=F)
    F *= -decay
    np.exp(F, out=F)
    noise = g.standard_normal(size=(n, n))
    noise *= 0.1
    noise += 1.0
    F *= noise
    F *= -1.0
    del noise
    F += F.T.copy()
    F *= 0.5
    np.fill_diagonal(F, g.uniform(-0.5, 0.5, size=n))
    if drop > 0:
        F[np.abs(F) < drop] = 0.0
    n_occ = n // 2
    vo = None
    if gap_mode == "eig":
        w, v = (eigh or np.linalg.eigh)(F)
        natural = w[n_occ] - w[n_occ - 1]
        s = max(0.0, gap - natural)
        vo = v[:, :n_occ]
        if s > 0.0:
            F += s * np.eye(n)
            F -= s * (vo @ vo.T)
            F += F.T.copy()
            F *= 0.5
        homo = float(w[n_occ - 1])
        lumo = float(w[n_occ] + s)
        # eigenvector roundoff moves eigenvalues by ~1e-13 * |F|; keep the bounds safe
        slack = 1e-9 * float(np.abs(w).max())
        homo += slack
        lumo -= slack
        del v
    elif gap_mode == "stagger":
        # functions 0,1 of each site go down by s, functions 2,3 go up by s;
        # Gershgorin discs of the two groups are then disjoint with a gap >= gap.
        R = float(np.max(np.sum(np.abs(F), axis=1) - np.abs(np.diag(F))))
        s = R + 0.5 + 0.5 * gap
        low = (np.arange(n) % funcs_per_site) < funcs_per_site // 2
        F[np.diag_indices(n)] += np.where(low, -s, s)
        homo = 0.5 - s + R
        lumo = -0.5 + s - R
    else:
        raise ValueError(gap_mode)
    P = FockProblem(np.ascontiguousarray(F), n_occ, homo, lumo, decay, gap_mode)
    if gap_mode == "eig":
        P.eigvals = np.concatenate([w[:n_occ], w[n_occ:] + s])
    if keep_vectors:
        P.occupied = vo
    return P


def random_decaying(n: int, seed: int, length: float = 6.0, symmetric: bool = False,
                    drop: float = 0.0) -> np.ndarray:
    """Non-symmetric (unless asked) random matrix with decay away from the diagonal."""
    g = rng(seed)
    i = np.arange(n)
    x = g.standard_normal((n, n)) * np.exp(-np.abs(i[:, None] - i[None, :]) / length)
    if symmetric:
        x = np.triu(x) + np.triu(x, 1).T
    if drop > 0:
        x[np.abs(x) < drop] = 0.0
    return np.ascontiguousarray(x)
