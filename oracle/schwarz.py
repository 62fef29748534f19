"""One-level additive Schwarz preconditioner with ILU(0) subdomain solves, FP64 (oracle; test infrastructure).

The paper's AS preconditioner (Sec. 5.2, eq. (AS); set up as in Sec. 6): the
index space is split into subsets Omega_t, possibly overlapping; with R_t the
restriction to Omega_t and M_t = R_t M R_t^T the principal submatrix,

    M_AS^{-1} = sum_t R_t^T M_t^{-1} R_t,

where M_t^{-1} is applied through an incomplete LU factorisation with no fill-in
(ILU(0)), and the subdomains overlap by one layer of mesh points in each
direction.  On one GPU the subdomains are boxes of the grid, not processes:

  * the cells are tiled by boxes of `block` cells per side (the last box of each
    direction takes the remainder); subdomain t is box t grown by `overlap`
    layers in every direction, clipped to the grid;
  * M is the diffusion matrix A_aux (7-point, symmetric);
  * ILU(0) in the lexicographic order of the subdomain (i fastest, then j, then
    k).  For a 7-point matrix two distinct neighbours of a cell are never
    neighbours of each other, so elimination never updates an off-diagonal
    entry: L = I + L_A D^{-1}, U = D + U_A with L_A, U_A the strictly lower and
    upper parts of M_t and D_c = m_cc - sum over lower neighbours k of
    m_ck m_kc / D_k;
  * the solve (D + L_A) t = r forward, then y = t - D^{-1} U_A y backward;
  * the contributions of the subdomains covering a cell are summed (plain
    additive Schwarz, symmetric for a symmetric M).
"""
import numpy as np
import scipy.sparse as sp


def subdomains(grid, block, overlap):
    """List of (cells, local shape) per subdomain: cells in local lexicographic order."""
    nx, ny, nz = grid
    out = []
    for k0 in range(0, nz, block):
        for j0 in range(0, ny, block):
            for i0 in range(0, nx, block):
                i1, j1, k1 = min(i0 + block, nx), min(j0 + block, ny), min(k0 + block, nz)
                a0, a1 = max(0, i0 - overlap), min(nx, i1 + overlap)
                b0, b1 = max(0, j0 - overlap), min(ny, j1 + overlap)
                c0, c1 = max(0, k0 - overlap), min(nz, k1 + overlap)
                kk, jj, ii = np.meshgrid(np.arange(c0, c1), np.arange(b0, b1), np.arange(a0, a1), indexing="ij")
                cells = (ii + nx * (jj + ny * kk)).ravel()
                out.append((cells, (a1 - a0, b1 - b0, c1 - c0)))
    return out


def ilu0_diagonal(Mt):
    """D of the ILU(0) of a 7-point submatrix, in its row order (lower = earlier rows)."""
    Mt = sp.csr_matrix(Mt)
    n = Mt.shape[0]
    D = np.zeros(n)
    for c in range(n):
        lo, hi = Mt.indptr[c], Mt.indptr[c + 1]
        cols, vals = Mt.indices[lo:hi], Mt.data[lo:hi]
        d = vals[cols == c].sum()
        for k, v in zip(cols, vals):
            if k < c:
                d -= v * Mt[k, c] / D[k]
        D[c] = d
    return D


class AS:
    def __init__(self, M, grid, block=8, overlap=1):
        self.M = sp.csr_matrix(M)
        self.parts = []
        for cells, shape in subdomains(grid, block, overlap):
            Mt = self.M[cells][:, cells].tocsr()
            self.parts.append((cells, Mt, ilu0_diagonal(Mt)))

    def apply(self, r):
        z = np.zeros_like(np.asarray(r, dtype=np.float64))
        for cells, Mt, D in self.parts:
            z[cells] += ilu0_solve(Mt, D, r[cells])
        return z


def ilu0_solve(Mt, D, r):
    """(D + L) D^{-1} (D + U) y = r for the ILU(0) factors of Mt."""
    n = len(D)
    t = np.zeros(n)
    for c in range(n):  # (D + L) t = r
        lo, hi = Mt.indptr[c], Mt.indptr[c + 1]
        s = r[c]
        for k, v in zip(Mt.indices[lo:hi], Mt.data[lo:hi]):
            if k < c:
                s -= v * t[k]
        t[c] = s / D[c]
    y = np.zeros(n)
    for c in range(n - 1, -1, -1):  # y = t - D^{-1} U y
        lo, hi = Mt.indptr[c], Mt.indptr[c + 1]
        s = 0.0
        for k, v in zip(Mt.indices[lo:hi], Mt.data[lo:hi]):
            if k > c:
                s += v * y[k]
        y[c] = t[c] - s / D[c]
    return y
