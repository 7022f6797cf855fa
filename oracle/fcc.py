"""FP64 CPU oracle of the DRTS step on the close-packed sphere partition of
Section 3 of arXiv:1611.08536 (face-centred cubic packing of equal spheres).

TEST INFRASTRUCTURE ONLY: the test suite may import this module; the product
(the CUDA library and its binding) never does and shares no code with it.
Plain numpy/scipy in FP64, small problems only.

What it computes (section and equation of the paper per step):
  * sites X_i (Section 3): centres of touching spheres of radius dr, so that
    nearest neighbours are s = 2 dr apart;
  * for source state (i, n) of medium k, in one step of path L_k (Eq. 9-12):
      - unscattered share e^{-mu_s L} e^{-mu_a L} spread over the sites
        closer than s to B = X_i + L S_n with weights (s - d) / sum (Eq. 18),
        kept in direction n;
      - scattered share G_k[n][m] (1 - e^{-mu_s L}) e^{-mu_a L} spread over
        the sites closer than s to the segment A_m B, A_m = X_i + L S_m, with
        weights (s - d) / sum (Eq. 19), into direction m; for m = n the
        segment is the point B (the w0 + w1 case of Eq. 21);
  * the matrix A of Eq. 23 collects these; the step is Eq. 26,
    x(t+1) = A x(t) + s(t), x(0) = 0.

Readings where the paper is silent (the cubic-grid oracle's R1 and R7 carry
over: strict "closer than s" decided with squared distances < (1 - 1e-9) s^2,
and the discrete Henyey-Greenstein table normalised per incoming direction):
  * F1 sites: integer triples (i, j, k) with i + j + k even, times
    a = s / sqrt(2); box 0 <= i < nx, 0 <= j < ny, 0 <= k < nz with nx even;
    site index v = ((k ny + j) nx + i) // 2, state index v * n_dirs + d.
  * F2 directions: the 12 unit vectors towards the nearest neighbours,
    (dx, dy, dz) / sqrt(2) with two nonzero components, dz slowest and dx
    fastest.  The paper uses 86 Lebedev points; their table is not carried
    here, so any unit-vector set may be passed instead.
  * F3 time step: dt = s / c_max, so medium k moves light
    L_k = s n_min / n_k <= s per step.
  * F4 boundary: open.  A target site outside the box receives nothing (the
    mass leaves the medium); there is no interface folding, so all media
    share one refractive index (the Section 4.2 outline is given for the
    voxel grid).

Parity status: pinned in tests/test_oracle_fcc.py (closed-form targets and
weights of Eq. 18/19 for lattice directions, Eq. 24 column sums, symmetry
under the 48 rotations and reflections of the cube, ballistic translation,
pure absorption decay, uniform scattering for g = 0, ledger closure and
dense matrix powers on a small box against a loop-literal transcription).
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

MARGIN = 1.0 - 1e-9          # strict "closer than s" on squared distances


def neighbour_offsets() -> np.ndarray:
    """The 12 nearest-neighbour offsets of the FCC lattice in units of a
    (two nonzero components of +-1), dz slowest, dx fastest (reading F2)."""
    out = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dx != 0) + (dy != 0) + (dz != 0) == 2:
                    out.append((dx, dy, dz))
    return np.array(out, dtype=np.int64)


def directions() -> np.ndarray:
    """Unit vectors S_n of the 12 nearest-neighbour directions."""
    return neighbour_offsets().astype(np.float64) / math.sqrt(2.0)


def hg_table(g: float, dirs: np.ndarray) -> np.ndarray:
    """Discrete Henyey-Greenstein phase function: G[n][m] proportional to
    p(S_n . S_m) = (1 - g^2) / (1 + g^2 - 2 g mu)^(3/2), each row normalised
    to 1 (Section 5's HG scattering; reading R7)."""
    mu = dirs @ dirs.T
    p = (1.0 - g * g) / (1.0 + g * g - 2.0 * g * mu) ** 1.5
    return p / p.sum(axis=1, keepdims=True)


def _segment_distance(X: np.ndarray, A: np.ndarray, B: np.ndarray) -> np.ndarray:
    """Distance of each row of X to the segment from A to B."""
    d = B - A
    dd = float(d @ d)
    if dd == 0.0:
        return np.sqrt(((X - B) ** 2).sum(axis=1))
    t = np.clip((X - A) @ d / dd, 0.0, 1.0)
    P = A + t[:, None] * d
    return np.sqrt(((X - P) ** 2).sum(axis=1))


def _candidate_sites(reach: float) -> np.ndarray:
    """Lattice offsets (units of a, even coordinate sum) within `reach`."""
    r = int(math.ceil(reach)) + 1
    g = np.arange(-r, r + 1)
    X = np.stack(np.meshgrid(g, g, g, indexing="ij"), axis=-1).reshape(-1, 3)
    X = X[(X.sum(axis=1) % 2) == 0]
    return X[np.sqrt((X.astype(np.float64) ** 2).sum(axis=1)) < reach + 1e-9]


def _spread(Xf: np.ndarray, dist: np.ndarray, s: float):
    """Weights (s - d) / sum over the sites strictly closer than s (Eq. 18/19)."""
    keep = dist * dist < s * s * MARGIN
    w = np.where(keep, s - dist, 0.0)
    tot = w.sum()
    return keep, (w / tot if tot > 0.0 else w)


def stencil(mu_s: float, mu_a: float, g: float, L_over_s: float, s_mm: float,
            dirs: np.ndarray | None = None) -> dict:
    """Transitions of one source state of a medium, for every source
    direction n: {(n, (ox, oy, oz), m): value}, offsets in units of a.
    Unscattered part (Eq. 18) plus scattered part (Eq. 19), summed per
    target (Eq. 20-21).  L_over_s = L_k / s (reading F3); s_mm = 2 dr."""
    if dirs is None:
        dirs = directions()
    nd = len(dirs)
    s = math.sqrt(2.0)                      # neighbour distance in units of a
    L = L_over_s * s
    Lmm = L_over_s * s_mm
    keep_un = math.exp(-mu_s * Lmm) * math.exp(-mu_a * Lmm)          # Eq. 9
    keep_sc = (1.0 - math.exp(-mu_s * Lmm)) * math.exp(-mu_a * Lmm)  # Eq. 10
    G = hg_table(g, dirs)
    X = _candidate_sites(L + s)
    Xf = X.astype(np.float64)
    out: dict = {}

    def add(n, m, keep, w, share):
        for x, wx in zip(X[keep], w[keep]):
            key = (n, (int(x[0]), int(x[1]), int(x[2])), m)
            out[key] = out.get(key, 0.0) + share * wx

    for n in range(nd):
        B = L * dirs[n]
        # unscattered population around B (Eq. 11, 18)
        keep, w = _spread(Xf, np.sqrt(((Xf - B) ** 2).sum(axis=1)), s)
        if keep_un > 0.0:
            add(n, n, keep, w, keep_un)
        # scattered population along A_m B (Eq. 12, 19)
        if keep_sc > 0.0:
            for m in range(nd):
                A = L * dirs[m]
                keep, w = _spread(Xf, _segment_distance(Xf, A, B), s)
                add(n, m, keep, w, G[n, m] * keep_sc)
    return out


@dataclass
class FccProblem:
    shape: tuple            # (nx, ny, nz) of the integer box; nx even
    s_mm: float             # nearest-neighbour distance 2 dr in mm
    media: list             # [(mu_s, mu_a, g, n)], one refractive index
    medium: np.ndarray      # u8 per site, site index order (reading F1)

    @property
    def n_sites(self) -> int:
        nx, ny, nz = self.shape
        return nx * ny * nz // 2


def site_coords(shape) -> np.ndarray:
    """Integer coordinates of every site in site-index order (reading F1)."""
    nx, ny, nz = shape
    if nx % 2:
        raise ValueError("nx must be even")
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    C = np.stack([i.ravel(), j.ravel(), k.ravel()], axis=1)
    return C[(C.sum(axis=1) % 2) == 0]


def site_index(shape, c) -> int:
    nx, ny, nz = shape
    i, j, k = c
    return ((k * ny + j) * nx + i) // 2


def assemble(prob: FccProblem, dirs: np.ndarray | None = None):
    """The matrix A of Eq. 23 on the FCC box as scipy CSR (rows = target
    states, columns = source states), and the exit fraction of every column
    (mass whose target site lies outside the box; reading F4)."""
    if dirs is None:
        dirs = directions()
    nd = len(dirs)
    n_ref = {m[3] for m in prob.media}
    if len(n_ref) != 1:
        raise ValueError("one refractive index for all media (no interface folding)")
    nx, ny, nz = prob.shape
    C = site_coords(prob.shape)
    nsites = len(C)
    rows, cols, vals = [], [], []
    exit_frac = np.zeros(nsites * nd)
    for k, (mu_s, mu_a, g, _n) in enumerate(prob.media):
        src = np.flatnonzero(prob.medium == k)
        if src.size == 0:
            continue
        W = stencil(mu_s, mu_a, g, 1.0, prob.s_mm, dirs)   # one index: L_k = s
        for (n, off, m), w in W.items():
            T = C[src] + np.array(off)
            inside = ((T[:, 0] >= 0) & (T[:, 0] < nx) & (T[:, 1] >= 0) & (T[:, 1] < ny)
                      & (T[:, 2] >= 0) & (T[:, 2] < nz))
            tv = ((T[inside, 2] * ny + T[inside, 1]) * nx + T[inside, 0]) // 2
            rows.append(tv * nd + m)
            cols.append(src[inside] * nd + n)
            vals.append(np.full(int(inside.sum()), w))
            np.add.at(exit_frac, src[~inside] * nd + n, w)
    n = nsites * nd
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n)).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A, exit_frac


def absorb_fraction(prob: FccProblem) -> np.ndarray:
    """Absorbed share 1 - e^{-mu_a L} of every state per step (Eq. 9-10)."""
    nd = len(directions())
    mu_a = np.array([m[1] for m in prob.media])[prob.medium]
    return np.repeat(1.0 - np.exp(-mu_a * prob.s_mm), nd)


def run(A, n_steps: int, states, weights, profile, t0: int = 0,
        absorb=None, exit_frac=None):
    """Eq. 26 from x(0) = 0: x(t+1) = A x(t) + s(t) with
    s(t) = sum_e weights[e] P(t) e_{states[e]}, P(t) = profile[t - t0].
    Returns x(n_steps) and the FP64 ledger (state mass, injected, absorbed,
    exited), absorbed and exited summed over x(0) .. x(n_steps - 1)."""
    n = A.shape[0]
    x = np.zeros(n)
    injected = absorbed = exited = 0.0
    for t in range(n_steps):
        if absorb is not None:
            absorbed += float(absorb @ x)
        if exit_frac is not None:
            exited += float(exit_frac @ x)
        y = A @ x
        if t0 <= t < t0 + len(profile):
            for st, w in zip(states, weights):
                y[st] += w * profile[t - t0]
                injected += w * profile[t - t0]
        x = y
    return x, np.array([x.sum(), injected, absorbed, exited])
