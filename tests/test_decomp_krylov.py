"""The split grid's Krylov drivers (`decomp.fcg`, `decomp.fgmres`) against the
oracle's FCG and FGMRES, on the CPU.

The drivers only order calls to the blocks' contexts (J x on the block's own
cells, interface couplings times the neighbours' x after an exchange, the
block's preconditioner, dots and axpbys) and carry the scalars.  Here each
block's context is a small numpy-backed stand-in over the rows of a seeded SPD
matrix, the preconditioner is each block's exact solve (block Jacobi: decoupled,
as each block's own V-cycle is), and the exchange hands every block its
neighbours' vectors.  The same system solved by the oracle with the same
block-diagonal preconditioner must take the same iterations and give the same x.
"""
import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import krylov
from paper_2112_05051_gb300 import decomp

torch = pytest.importorskip("torch")


def _spd(n, seed):
    """7-point-like SPD matrix on an n-cell line of 3D-ish couplings: a shifted
    graph Laplacian with random positive weights (diagonally dominant)."""
    rng = np.random.default_rng(seed)
    rows, cols, vals = [], [], []
    for off in (1, 4, 16):
        w = rng.uniform(0.5, 2.0, n - off)
        rows += list(range(n - off)) + list(range(off, n))
        cols += list(range(off, n)) + list(range(n - off))
        vals += list(-w) + list(-w)
    A = sp.csr_matrix((vals, (rows, cols)), shape=(n, n))
    d = -np.asarray(A.sum(axis=1)).ravel() + rng.uniform(1e-3, 1e-1, n)
    return (A + sp.diags(d)).tocsr()


class _Ctx:
    """The vector calls a split-grid driver makes on one block's context."""

    def __init__(self, A, lo, hi):
        self.Abb = A[lo:hi, lo:hi].tocsc()
        self.lu = spla.splu(self.Abb)

    def jacobian_apply(self, x, y):
        y.copy_(torch.from_numpy(self.Abb @ x.numpy()))

    def vcycle(self, r, z):
        z.copy_(torch.from_numpy(self.lu.solve(r.numpy())))

    def dot(self, x, y):
        return float(np.dot(x.numpy(), y.numpy()))

    def axpby(self, a, x, b, y):
        if b == 0.0:
            y.copy_(a * x)
        else:
            y.copy_(a * x + b * y)


class _Problem:
    def __init__(self, A, bounds, r):
        self.A, self.bounds, self.rank = A, bounds, r
        self.ctx = _Ctx(A, bounds[r], bounds[r + 1])

    def couple(self, which, y):
        lo, hi = self.bounds[self.rank], self.bounds[self.rank + 1]

        def apply(s, ghosts):  # the neighbour's x times this block's couplings to it
            Ars = self.A[lo:hi, self.bounds[s]:self.bounds[s + 1]]
            y.add_(torch.from_numpy(Ars @ ghosts.numpy()))
        return apply


class _Comm:
    """Every block receives every other block's field (a neighbour with no
    couplings adds zeros); sums in block order, as LocalComm does."""

    def __init__(self, problems):
        self.problems = problems

    def exchange(self, fields, applies):
        for r, ap in enumerate(applies):
            for s, f in enumerate(fields):
                if s != r:
                    ap(s, f)

    def sum(self, values):
        return float(sum(values))

    def max(self, values):
        return float(max(values))


def _split(A, nblocks):
    n = A.shape[0]
    bounds = [round(i * n / nblocks) for i in range(nblocks + 1)]
    probs = [_Problem(A, bounds, r) for r in range(nblocks)]
    prec_parts = [spla.splu(A[bounds[r]:bounds[r + 1], bounds[r]:bounds[r + 1]].tocsc()) for r in range(nblocks)]

    def prec(v):  # the same block-diagonal preconditioner on the whole vector
        return np.concatenate([lu.solve(v[bounds[r]:bounds[r + 1]]) for r, lu in enumerate(prec_parts)])
    return bounds, probs, prec


@pytest.mark.parametrize("nblocks", [1, 2, 3])
@pytest.mark.parametrize("kind,m", [("fcg", 0), ("fgmres", 4), ("fgmres", 30)])
def test_split_krylov_drivers_match_the_oracle(nblocks, kind, m):
    n = 240
    A = _spd(n, 11 + nblocks)
    b = np.random.default_rng(5).standard_normal(n)
    bounds, probs, prec = _split(A, nblocks)
    bs = [torch.from_numpy(b[bounds[r]:bounds[r + 1]].copy()) for r in range(nblocks)]
    eta, maxit = 1e-10, 300
    if kind == "fcg":
        xs, its, ok, why = decomp.fcg(probs, _Comm(probs), bs, eta, maxit)
        xo, its_o, ok_o, _ = krylov.fcg(lambda v: A @ v, prec, b, eta, maxit)
    else:
        xs, its, ok, why = decomp.fgmres(probs, _Comm(probs), bs, eta, maxit, m)
        xo, its_o, ok_o, _ = krylov.fgmres(lambda v: A @ v, prec, b, eta, maxit, m)
    x = np.concatenate([v.numpy() for v in xs])
    assert ok and ok_o and why is None
    assert abs(its - its_o) <= 1  # sums in another order may move the stop by one
    assert np.linalg.norm(b - A @ x) <= eta * np.linalg.norm(b) * (1 + 1e-6)
    assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)
    if nblocks == 1:
        assert its == 1  # one block: the preconditioner is the exact inverse
    elif kind == "fgmres" and m == 4:
        assert its > 2 * m  # restarts from the true residual were taken


def test_split_fgmres_restarts_and_second_pass_without_a_preconditioner():
    # with the identity in place of the block solves, FGMRES(5) needs many restarts
    # on this ill-conditioned system and the DGKS second pass fires
    n = 200
    A = _spd(n, 3)
    b = np.random.default_rng(8).standard_normal(n)
    bounds, probs, _ = _split(A, 2)
    dots = [0]
    for q in probs:
        q.ctx.vcycle = lambda r, z: z.copy_(r)
        plain = q.ctx.dot

        def counted(x, y, plain=plain):
            dots[0] += 1
            return plain(x, y)
        q.ctx.dot = counted
    bs = [torch.from_numpy(b[bounds[r]:bounds[r + 1]].copy()) for r in range(2)]
    m = 5
    xs, its, ok, why = decomp.fgmres(probs, _Comm(probs), bs, 1e-8, 2000, m)
    xo, its_o, ok_o, _ = krylov.fgmres(lambda v: A @ v, lambda v: v.copy(), b, 1e-8, 2000, m)
    x = np.concatenate([v.numpy() for v in xs])
    assert ok == ok_o
    assert its > 20 and abs(its - its_o) <= max(2, its_o // 50)
    # dots per block without any second pass: ||b||, one ||r|| per restart, and
    # ||w||^2, j + 1 projections and ||w'||^2 in iteration j of a cycle
    cycles = -(-its // m)
    single = cycles + sum(j + 3 for c in range(cycles) for j in range(min(m, its - c * m)))
    assert dots[0] // 2 > single  # the second pass ran
    if ok:
        assert np.linalg.norm(b - A @ x) <= 1e-8 * np.linalg.norm(b) * (1 + 1e-6)


def test_split_krylov_zero_rhs_and_maxit():
    A = _spd(60, 2)
    bounds, probs, _ = _split(A, 2)
    zeros = [torch.zeros(bounds[r + 1] - bounds[r], dtype=torch.float64) for r in range(2)]
    for solve in (lambda b: decomp.fcg(probs, _Comm(probs), b, 1e-10, 50),
                  lambda b: decomp.fgmres(probs, _Comm(probs), b, 1e-10, 50, 5)):
        xs, its, ok, why = solve(zeros)
        assert (its, ok, why) == (0, True, None) and all(float(v.abs().max()) == 0.0 for v in xs)
    b = np.random.default_rng(1).standard_normal(60)
    bs = [torch.from_numpy(b[bounds[r]:bounds[r + 1]].copy()) for r in range(2)]
    for q in probs:
        q.ctx.vcycle = lambda r, z: z.copy_(r)
    xs, its, ok, why = decomp.fgmres(probs, _Comm(probs), bs, 1e-14, 3, 2)
    assert (its, ok, why) == (3, False, "maxit")
    xs, its, ok, why = decomp.fcg(probs, _Comm(probs), bs, 1e-14, 3)
    assert (its, ok, why) == (3, False, "maxit")


def test_split_fgmres_breakdown_keeps_the_columns_before_it():
    # a preconditioner that returns zero makes J z = 0: the column's rotation is
    # undefined, and FGMRES stops with the columns it has instead of dividing by 0
    A = _spd(80, 6)
    b = np.random.default_rng(2).standard_normal(80)
    bounds, probs, _ = _split(A, 2)
    bs = [torch.from_numpy(b[bounds[r]:bounds[r + 1]].copy()) for r in range(2)]
    for q in probs:
        q.ctx.vcycle = lambda r, z: z.zero_()
    xs, its, ok, why = decomp.fgmres(probs, _Comm(probs), bs, 1e-10, 50, 10)
    assert (its, ok, why) == (0, False, "breakdown") and all(float(v.abs().max()) == 0.0 for v in xs)
    calls = [0]
    for q in probs:  # three good columns (identity), then zeros
        def prec(r, z, calls=calls):
            calls[0] += 1
            return z.copy_(r) if calls[0] <= 2 * 3 else z.zero_()
        q.ctx.vcycle = prec
    xs, its, ok, why = decomp.fgmres(probs, _Comm(probs), bs, 1e-10, 50, 10)
    assert (its, ok, why) == (3, False, "breakdown")
    x = np.concatenate([v.numpy() for v in xs])
    xo, its_o, _, hist = krylov.fgmres(lambda v: A @ v, lambda v: v.copy(), b, 1e-10, 3, 10)
    assert its_o == 3
    np.testing.assert_allclose(x, xo, rtol=0, atol=1e-12 * np.abs(xo).max())  # the 3-column minimiser
    assert np.linalg.norm(b - A @ x) < np.linalg.norm(b)
