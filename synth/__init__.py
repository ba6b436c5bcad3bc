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
* ``lattice_fock_blocks`` -- the same matrix with a hard distance cutoff, built
  as a list of leaf blocks without a dense form (the n = 262144 configuration).

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
    centres: np.ndarray = None    # (n, 3) basis-function centres


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
    P.centres = centre
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


@dataclasses.dataclass
class BlockFockProblem:
    n: int
    bs: int
    brow: np.ndarray     # (nnzb,) int32 block rows
    bcol: np.ndarray     # (nnzb,) int32 block columns
    tiles: np.ndarray    # (nnzb, bs, bs) float64, row-major tiles (None for pattern_only)
    n_occ: int
    homo: float
    lumo: float
    decay: float
    cutoff: float
    centres: np.ndarray = None   # (n, 3) basis-function centres (the site of each function)

    @property
    def fill(self) -> float:
        nb = self.n // self.bs
        return len(self.brow) / float(nb * nb)

    def to_dense(self) -> np.ndarray:
        X = np.zeros((self.n, self.n))
        for t in range(len(self.brow)):
            i, j = int(self.brow[t]), int(self.bcol[t])
            X[i * self.bs:(i + 1) * self.bs, j * self.bs:(j + 1) * self.bs] = self.tiles[t]
        return X


def lattice_fock_blocks(n: int, seed: int = SEED_BASE, decay: float = 2.5, cutoff: float = 6.0,
                        bs: int = 64, gap: float = 0.1, jitter: float = 0.1,
                        funcs_per_site: int = 4, pattern_only: bool = False) -> BlockFockProblem:
    """The lattice Fock matrix of ``lattice_fock`` built block by block, for sizes whose
    dense form does not fit in memory (n = 262144 is 550 GB dense).

    Sites and jitter as in ``lattice_fock`` (Morton order, so a leaf block is a compact
    brick of bs / funcs_per_site sites). Off the diagonal F_ij = -exp(-a d_ij)(1 + 0.1 h_ij)
    for d_ij <= cutoff and 0 beyond (a hard cutoff gives the block-sparse pattern;
    cutoff 6 at a = 2.5 drops entries below 3.1e-7), with h_ij = (g_ij + g_ji) / 2,
    g ~ N(0, 1), as the symmetrised dense generator has; F_ii ~ U(-0.5, 0.5). The gap
    at n_occ = n / 2 is enforced by the staggered onsite shift (Gershgorin-certified,
    ``gap_mode="stagger"`` of ``lattice_fock``). Only blocks holding a pair of sites
    within the cutoff are stored, both triangles, in row-major block order.

    Random numbers come from one stream per block row I (seeded by (seed, I)) for the
    blocks (I, J), J >= I, in increasing J, so the result does not depend on how the
    work is split. ``pattern_only`` returns the block pattern without tiles.
    """
    if n % bs or bs % funcs_per_site:
        raise ValueError("n must be a multiple of bs, and bs of funcs_per_site")
    g = rng(seed)
    sites = n // funcs_per_site
    spb = bs // funcs_per_site
    nb = n // bs
    pts = _morton_points(sites).astype(np.float64)
    pts = pts + g.uniform(-jitter, jitter, size=pts.shape)
    onsite = g.uniform(-0.5, 0.5, size=n)
    P = pts.reshape(nb, spb, 3)
    lo, hi = P.min(axis=1), P.max(axis=1)
    # block pairs whose bounding boxes come within the cutoff, then the exact test
    pairs = []
    for I in range(nb):
        gapv = np.maximum(0.0, np.maximum(lo[I:] - hi[I], lo[I] - hi[I:]))
        cand = I + np.nonzero(np.sqrt((gapv ** 2).sum(axis=1)) <= cutoff)[0]
        d = np.sqrt(((P[I][None, :, None, :] - P[cand][:, None, :, :]) ** 2).sum(axis=-1))
        keep = cand[d.reshape(len(cand), -1).min(axis=1) <= cutoff]
        pairs.append(keep)
    rows = [[] for _ in range(nb)]
    for I in range(nb):
        for J in pairs[I]:
            rows[I].append(int(J))
            if J != I:
                rows[int(J)].append(I)
    for r in rows:
        r.sort()
    brow = np.array([I for I in range(nb) for _ in rows[I]], dtype=np.int32)
    bcol = np.array([J for I in range(nb) for J in rows[I]], dtype=np.int32)
    centres = np.repeat(pts, funcs_per_site, axis=0)
    if pattern_only:
        return BlockFockProblem(n, bs, brow, bcol, None, n // 2, 0.0, 0.0, decay, cutoff, centres)
    start = np.zeros(nb + 1, dtype=np.int64)
    start[1:] = np.cumsum([len(r) for r in rows])

    def slot(I, J):
        return int(start[I] + np.searchsorted(rows[I], J))

    T = np.empty((len(brow), bs, bs))
    for I in range(nb):
        gi = rng_pair(seed, I)
        ci = np.repeat(P[I], funcs_per_site, axis=0)                  # (bs, 3) centres
        for J in pairs[I]:
            J = int(J)
            cj = np.repeat(P[J], funcs_per_site, axis=0)
            d = np.sqrt(((ci[:, None, :] - cj[None, :, :]) ** 2).sum(axis=-1))
            g1 = gi.standard_normal((bs, bs))                          # g_ij, i in I, j in J
            g2 = gi.standard_normal((bs, bs)) if J != I else g1.T      # g_ji, stored as (i, j)
            t = -np.exp(-decay * d) * (1.0 + 0.1 * 0.5 * (g1 + g2))
            t[d > cutoff] = 0.0
            if J == I:
                t = 0.5 * (t + t.T)                                    # exactly symmetric
                t[np.diag_indices(bs)] = onsite[I * bs:(I + 1) * bs]
            T[slot(I, J)] = t
            if J != I:
                T[slot(J, I)] = t.T
    # staggered onsite shift: functions 0, 1 of each site down by s, 2, 3 up by s
    R = np.zeros(n)
    for t in range(len(brow)):
        I, J = int(brow[t]), int(bcol[t])
        a = np.abs(T[t]).sum(axis=1)
        if I == J:
            a = a - np.abs(np.diag(T[t]))
        R[I * bs:(I + 1) * bs] += a
    Rm = float(R.max())
    s = Rm + 0.5 + 0.5 * gap
    low = (np.arange(n) % funcs_per_site) < funcs_per_site // 2
    shift = np.where(low, -s, s)
    for I in range(nb):
        T[slot(I, I)][np.diag_indices(bs)] += shift[I * bs:(I + 1) * bs]
    return BlockFockProblem(n, bs, brow, bcol, T, n // 2, 0.5 - s + Rm, -0.5 + s - Rm,
                            decay, cutoff, centres)


def rng_pair(seed: int, index: int) -> np.random.Generator:
    """Stream of one block row: PCG64 seeded by the pair (seed, index)."""
    return np.random.Generator(np.random.PCG64([seed, index]))
