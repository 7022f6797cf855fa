"""A third, loop-literal transcription of Eq. 18-21 and the Section 4.2 edge and
interface readings, producing the dense system matrix A of Eq. 23 for tiny
grids.  It is written target by target (for each source state, for each
candidate target voxel and direction) with no stencil tables and no CSR, so
that a mistake in the oracle's table or scatter logic shows up as a mismatch.

Used only by the tests (dense brute force on 4^3 grids).
"""
from __future__ import annotations

import math

import numpy as np

NDIR = 26


def _dirs():
    out = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if dx or dy or dz:
                    out.append((dx, dy, dz))
    return out


DIRS = _dirs()


def _unit(v):
    n = math.sqrt(v[0] ** 2 + v[1] ** 2 + v[2] ** 2)
    return (v[0] / n, v[1] / n, v[2] / n)


def _dist_point_segment(p, a, b):
    # closest point of segment a-b to p, parametrised a + t (b - a)
    ab = [b[c] - a[c] for c in range(3)]
    L2 = sum(x * x for x in ab)
    if L2 == 0.0:
        t = 0.0
    else:
        t = sum((p[c] - a[c]) * ab[c] for c in range(3)) / L2
        t = min(1.0, max(0.0, t))
    return math.sqrt(sum((a[c] + t * ab[c] - p[c]) ** 2 for c in range(3)))


def _fresnel(c, n1, n2):
    if n1 == n2:
        return 0.0
    s = n1 / n2 * math.sqrt(max(0.0, 1.0 - c * c))
    if s >= 1.0:
        return 1.0
    ct = math.sqrt(1.0 - s * s)
    rs = (n1 * c - n2 * ct) / (n1 * c + n2 * ct)
    rp = (n1 * ct - n2 * c) / (n1 * ct + n2 * c)
    return (rs * rs + rp * rp) / 2.0


def dense_matrix(prob):
    """Dense A (states x states) for a problem from ``inputs``."""
    nx, ny, nz = prob.shape
    N = (nx, ny, nz)
    mov = np.asarray(prob.medium_of_voxel).reshape(nz, ny, nx)
    media = prob.media
    nmin = min(m[3] for m in media)
    ns = nx * ny * nz * NDIR
    A = np.zeros((ns, ns))
    units = [_unit(v) for v in DIRS]

    def sidx(x, y, z, d):
        return ((z * ny + y) * nx + x) * NDIR + d

    def nref(p):
        return media[mov[p[2], p[1], p[0]]][3]

    for z in range(nz):
        for y in range(ny):
            for x in range(nx):
                k = mov[z, y, x]
                mu_s, mu_a, g, nk = media[k]
                lam = nmin / nk
                L = lam * prob.voxel_mm
                keep = math.exp(-mu_s * L)
                surv = math.exp(-mu_a * L)
                for n in range(NDIR):
                    Sn = units[n]
                    # Henyey-Greenstein over the 26 directions, normalised
                    ph = []
                    for m in range(NDIR):
                        mu = sum(Sn[c] * units[m][c] for c in range(3))
                        ph.append((1 - g * g) / (1 + g * g - 2 * g * mu) ** 1.5)
                    tot = sum(ph)
                    B = tuple(lam * Sn[c] for c in range(3))
                    for m in range(NDIR):
                        Am = tuple(lam * units[m][c] for c in range(3))
                        # candidate targets: every lattice offset within one voxel
                        cand = []
                        for oz in (-1, 0, 1):
                            for oy in (-1, 0, 1):
                                for ox in (-1, 0, 1):
                                    cand.append((ox, oy, oz))
                        w1 = {}
                        if keep < 1.0:
                            dsum = 0.0
                            for o in cand:
                                dd = _dist_point_segment(o, Am, B)
                                if dd * dd < 1 - 1e-9:
                                    w1[o] = 1 - dd
                                    dsum += 1 - dd
                            for o in w1:
                                w1[o] = w1[o] / dsum * (ph[m] / tot) * (1 - keep) * surv
                        w0 = {}
                        if m == n and keep > 0.0:
                            dsum = 0.0
                            for o in cand:
                                dd = math.sqrt(sum((o[c] - B[c]) ** 2 for c in range(3)))
                                if dd * dd < 1 - 1e-9:
                                    w0[o] = 1 - dd
                                    dsum += 1 - dd
                            for o in w0:
                                w0[o] = w0[o] / dsum * keep * surv
                        for o in set(w0) | set(w1):
                            w = w0.get(o, 0.0) + w1.get(o, 0.0)
                            t = [x + o[0], y + o[1], z + o[2]]
                            dv = list(DIRS[m])
                            ghost = False
                            for a in range(3):
                                if 0 <= t[a] < N[a]:
                                    continue
                                ghost = True
                                if prob.boundary == 1:
                                    R = 1.0
                                elif prob.boundary == 0:
                                    R = 0.0
                                else:
                                    R = _fresnel(abs(units[m][a]), nk, prob.n_outside)
                                w *= R
                                t[a] = 0 if t[a] < 0 else N[a] - 1
                                dv[a] = -dv[a]
                            if w == 0.0:
                                continue
                            col = sidx(x, y, z, n)
                            if not ghost and o != (0, 0, 0) and nref(t) != nk:
                                # interface normal: first offset axis whose
                                # axis-neighbour changes index, else first offset axis
                                axis = None
                                for a in range(3):
                                    if o[a] != 0:
                                        nb = [x, y, z]
                                        nb[a] += o[a]
                                        if nref(nb) != nk:
                                            axis = a
                                            break
                                if axis is None:
                                    axis = next(a for a in range(3) if o[a] != 0)
                                if dv[axis] * o[axis] > 0:
                                    R = _fresnel(abs(units[m][axis]), nk, nref(t))
                                    tr = list(t)
                                    tr[axis] = (x, y, z)[axis]
                                    dr = list(dv)
                                    dr[axis] = -dr[axis]
                                    if w * R > 0:
                                        A[sidx(*tr, DIRS.index(tuple(dr))), col] += w * R
                                    w *= 1 - R
                            if w > 0:
                                A[sidx(*t, DIRS.index(tuple(dv))), col] += w
    return A
