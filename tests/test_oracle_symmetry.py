"""Symmetry pins of the voxel-grid oracle's edge and interface folding
(Section 4.2, readings R4-R6), where the paper prints no numbers.

A homogeneous cube looks the same after any rotation or reflection of the
cube, so its matrix A (Eq. 23) must commute with the 48 permutations of
states those symmetries induce (voxel mapped, lattice direction mapped):
the folding of mass at the edges (mirror, open, Fresnel) depends only on
the geometry.  The order in which out-of-range axes are folded only decides
which face an exiting share is attributed to, not A.  A medium layered along
z keeps the 8 symmetries of the square in x and y, interfaces included."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from paper_1611_08536_gb300 import inputs as I


def _directions():
    out = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dx, dy, dz) != (0, 0, 0):
                    out.append((dx, dy, dz))
    return np.array(out)


def _signed_permutations(fix_z=False):
    for perm in itertools.permutations(range(3)):
        if fix_z and perm[2] != 2:
            continue
        for signs in itertools.product((1, -1), repeat=3):
            if fix_z and signs[2] != 1:
                continue
            P = np.zeros((3, 3), dtype=np.int64)
            for r in range(3):
                P[r, perm[r]] = signs[r]
            yield P


def _state_permutation(shape, P):
    nx, ny, nz = shape
    N = np.array(shape)
    dirs = _directions()
    dindex = {tuple(v): i for i, v in enumerate(dirs)}
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    C = np.stack([x.ravel(), y.ravel(), z.ravel()], axis=1)           # voxel order
    # map about the box centre: c' = P (c - (N-1)/2) + (N'-1)/2 (integers)
    Np = np.abs(P) @ N
    Cp = (P @ (2 * C.T - (N - 1)[:, None]) + (Np - 1)[:, None]) // 2
    vp = (Cp[2] * Np[1] + Cp[1]) * Np[0] + Cp[0]
    dmap = np.array([dindex[tuple(P @ v)] for v in dirs])
    return (vp[:, None] * 26 + dmap[None, :]).ravel()


def _matrix(oracle_mod, prob):
    c = oracle_mod.assemble(prob)
    return sp.csr_matrix((c.val, c.col, c.row_ptr), shape=(c.n_rows, c.n_rows))


def _check_invariant(A, perm):
    n = A.shape[0]
    Pm = sp.csr_matrix((np.ones(n), (perm, np.arange(n))), shape=(n, n))
    B = (Pm @ A @ Pm.T).tocsr()
    B.sort_indices()
    A = A.tocsr()
    A.sort_indices()
    assert np.array_equal(A.indptr, B.indptr) and np.array_equal(A.indices, B.indices)
    assert np.allclose(A.data, B.data, rtol=1e-13, atol=0)


@pytest.mark.parametrize("boundary", [I.FRESNEL, I.MIRROR, I.OPEN])
def test_homogeneous_cube_has_the_48_symmetries(oracle_mod, boundary):
    n = 5
    prob = I.Problem((n, n, n), 0.1, [(10.0, 0.05, 0.9, 1.4)], np.zeros((n, n, n), np.uint8), 1.0,
                     boundary, I.FP64, 1, I.FACE_PZ, 1, 1, "cube5")
    A = _matrix(oracle_mod, prob)
    groups = list(_signed_permutations())
    assert len(groups) == 48
    for P in groups:
        _check_invariant(A, _state_permutation(prob.shape, P))


def test_quadrature_kernel_keeps_the_48_symmetries(oracle_mod):
    """The quadrature shares are equal within each class of directions the
    cube's symmetries permute, so the weighted kernel keeps all 48."""
    n = 4
    prob = I.Problem((n, n, n), 0.1, [(10.0, 0.05, 0.8, 1.4)], np.zeros((n, n, n), np.uint8), 1.0,
                     I.FRESNEL, I.FP64, 1, I.FACE_PZ, 1, 1, "cube4_quadrature",
                     direction_weights=I.HG_QUADRATURE)
    A = _matrix(oracle_mod, prob)
    for P in _signed_permutations():
        _check_invariant(A, _state_permutation(prob.shape, P))


@pytest.mark.parametrize("boundary", [I.FRESNEL, I.MIRROR])
def test_layered_medium_has_the_square_symmetries(oracle_mod, boundary):
    nxy, nz = 4, 7
    mov = np.zeros((nz, nxy, nxy), np.uint8)
    mov[2:4] = 1
    mov[4:] = 2
    media = [(20.0, 0.02, 0.9, 1.45), (10.0, 0.005, 0.85, 1.44), (5.0, 0.01, 0.9, 1.37)]
    prob = I.Problem((nxy, nxy, nz), 0.1, media, mov, 1.0, boundary, I.FP64, 1, I.FACE_PZ, 1, 1,
                     "layers")
    A = _matrix(oracle_mod, prob)
    groups = list(_signed_permutations(fix_z=True))
    assert len(groups) == 8
    for P in groups:
        _check_invariant(A, _state_permutation(prob.shape, P))


def test_a_non_symmetric_medium_is_detected(oracle_mod):
    """The check is not vacuous: one inclusion off the centre breaks the
    x reflection."""
    n = 5
    mov = np.zeros((n, n, n), np.uint8)
    mov[2, 2, 0] = 1
    prob = I.Problem((n, n, n), 0.1, [(10.0, 0.05, 0.9, 1.4), (3.0, 0.5, 0.7, 1.4)], mov, 1.0,
                     I.MIRROR, I.FP64, 1, I.FACE_PZ, 1, 1, "off-centre")
    A = _matrix(oracle_mod, prob)
    P = np.diag([-1, 1, 1])
    with pytest.raises(AssertionError):
        _check_invariant(A, _state_permutation(prob.shape, P))
