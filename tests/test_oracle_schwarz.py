"""Pins of the additive Schwarz / ILU(0) preconditioner of the oracle (Sec. 5.2, eq. (AS); Sec. 6).

Fixed other than by the oracle itself: the defining property of ILU(0) (the
product of its factors equals the matrix on the matrix's pattern), the
textbook IKJ elimination with the fill pattern restricted (an independent
implementation), the exact LU of a tridiagonal matrix (one subdomain of a
column), point Jacobi (single-cell blocks without overlap), and symmetry and
positivity of the additive operator.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from oracle import discretization as disc
from oracle import schwarz
from paper_2112_05051_gb300 import synth

SOIL = synth.Soil()


def _aux(grid, seed=1):
    rng = np.random.default_rng(seed)
    p = rng.uniform(-60, -20, grid.n)
    ks = synth.ks_field(grid, seed, 1.0, (3.0, 3.0, 2.0))
    return disc.aux_matrix(grid, SOIL, synth.infiltration_bc(), synth.KMEAN_ARITH, p, 1.0, ks)


def _ilu0_ikj(Md):
    """Textbook ILU(0) (IKJ variant), dense storage, updates only on the pattern of Md."""
    A = Md.copy()
    n = A.shape[0]
    pat = Md != 0
    for i in range(1, n):
        for k in range(i):
            if not pat[i, k]:
                continue
            A[i, k] /= A[k, k]
            for j in range(k + 1, n):
                if pat[i, j]:
                    A[i, j] -= A[i, k] * A[k, j]
    L = np.tril(A, -1) + np.eye(n)
    U = np.triu(A)
    return L, U


def test_ilu0_factors_reproduce_the_matrix_on_its_pattern_and_match_ikj():
    grid = synth.Grid(5, 4, 6)
    M = _aux(grid)
    for cells, shape in schwarz.subdomains((grid.nx, grid.ny, grid.nz), 3, 1):
        Mt = M[cells][:, cells].tocsr()
        D = schwarz.ilu0_diagonal(Mt)
        Md = Mt.toarray()
        Lt = np.tril(Md, -1) / D[None, :] + np.eye(len(D))   # L = I + L_A D^-1
        Ut = np.triu(Md, 1) + np.diag(D)                     # U = D + U_A
        LU = Lt @ Ut
        pat = Md != 0
        np.testing.assert_allclose(LU[pat], Md[pat], rtol=1e-12, atol=1e-12 * np.abs(Md).max())
        L2, U2 = _ilu0_ikj(Md)
        np.testing.assert_allclose(np.diag(U2), D, rtol=1e-12)
        r = np.random.default_rng(3).standard_normal(len(D))
        np.testing.assert_allclose(schwarz.ilu0_solve(Mt, D, r), np.linalg.solve(L2 @ U2, r), rtol=1e-9, atol=1e-12)


def test_one_subdomain_of_a_column_is_the_exact_solve():
    grid = synth.Grid(1, 1, 30)
    M = _aux(grid, 4)
    pre = schwarz.AS(M, (1, 1, 30), block=30, overlap=1)
    r = np.random.default_rng(5).standard_normal(grid.n)
    np.testing.assert_allclose(pre.apply(r), np.linalg.solve(M.toarray(), r), rtol=1e-10)


def test_single_cell_blocks_without_overlap_are_point_jacobi():
    grid = synth.Grid(4, 3, 5)
    M = _aux(grid, 6)
    pre = schwarz.AS(M, (4, 3, 5), block=1, overlap=0)
    r = np.random.default_rng(7).standard_normal(grid.n)
    np.testing.assert_allclose(pre.apply(r), r / M.diagonal(), rtol=1e-14)


def test_additive_operator_is_symmetric_positive_and_covers_overlaps():
    grid = synth.Grid(7, 6, 5)
    M = _aux(grid, 8)
    pre = schwarz.AS(M, (7, 6, 5), block=3, overlap=1)
    n = grid.n
    B = np.column_stack([pre.apply(e) for e in np.eye(n)])
    np.testing.assert_allclose(B, B.T, rtol=1e-10, atol=1e-14 * np.abs(B).max())
    assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0
    # every cell lies in at least one subdomain, corner cells of interior boxes in up to 8
    cover = np.zeros(n, dtype=int)
    for cells, _ in schwarz.subdomains((7, 6, 5), 3, 1):
        cover[cells] += 1
    assert cover.min() >= 1 and cover.max() == 8


def test_pins_catch_an_ilu0_without_its_diagonal_correction(monkeypatch):
    def bad(Mt):
        return np.asarray(sp.csr_matrix(Mt).diagonal(), dtype=float)
    monkeypatch.setattr(schwarz, "ilu0_diagonal", bad)
    with pytest.raises(AssertionError):
        test_ilu0_factors_reproduce_the_matrix_on_its_pattern_and_match_ikj()
