"""The split grid's Krylov drivers on real ranks (torch.distributed, gloo, CPU).

One block per rank: `decomp.fcg` and `decomp.fgmres` with `DistComm` (halo
exchanges of x inside J x by point-to-point messages, dots gathered and summed
in rank order), over stand-in block contexts on a seeded 7-point SPD matrix
(each block's rows, its couplings across each interface face to the
neighbour's cells, an exact block solve as its preconditioner).  Every rank's
x and iteration count must equal, bit for bit, those of the same blocks driven
in one process (`LocalComm`), and the assembled x must be the oracle's solution
of the whole system with the same block-diagonal preconditioner.

The split Newton step (`decomp.newton_step`: halo exchange of p before every
residual and Jacobian, norms, round-off scales and slopes summed over the
ranks) runs the same way on a monotone nonlinear stand-in of the backward-Euler
residual: each rank's p and counts equal the one-process step's bit for bit,
and the assembled p is the whole system's Newton solution.
"""
import os
import socket

import numpy as np
import pytest
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from paper_2112_05051_gb300 import decomp, synth

torch = pytest.importorskip("torch")

DIMS = (9, 7, 4)
ETA, MAXIT, RESTART = 1e-10, 300, 6


def _system():
    """The whole grid's SPD matrix (face weights in [0.5, 2], a positive diagonal
    shift), its cell index array (nz, ny, nx) and a right-hand side."""
    grid = synth.Grid(*DIMS)
    nz, ny, nx = grid.shape
    rng = np.random.default_rng(21)
    idx = np.arange(grid.n).reshape(grid.shape)
    diag = rng.uniform(1e-3, 1e-1, grid.n)
    rows, cols, vals = [], [], []
    for a, b in ((idx[:, :, :-1], idx[:, :, 1:]), (idx[:, :-1, :], idx[:, 1:, :]), (idx[:-1], idx[1:])):
        w = rng.uniform(0.5, 2.0, a.size)
        rows += [a.ravel(), b.ravel()]
        cols += [b.ravel(), a.ravel()]
        vals += [-w, -w]
        np.add.at(diag, a.ravel(), w)
        np.add.at(diag, b.ravel(), w)
    rows.append(idx.ravel())
    cols.append(idx.ravel())
    vals.append(diag)
    A = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(grid.n, grid.n))
    return grid, A, idx, rng.standard_normal(grid.n)


class _BlockCtx:
    """The calls a split-grid driver makes on a block's context, over the whole
    matrix's rows of the block (cells in the block's own order)."""

    def __init__(self, A, idx, b):
        self.g = idx[:, b.j0:b.j1, b.i0:b.i1].ravel()  # whole-grid index of each block cell
        self.Abb = A[self.g][:, self.g].tocsc()
        self.lu = spla.splu(self.Abb)
        l3 = np.arange(self.g.size).reshape(idx.shape[0], b.j1 - b.j0, b.i1 - b.i0)
        self.face = {}
        for f in range(4):
            if b.nbr[f] >= 0:  # face cells (face layout) and their couplings to the ghosts
                lc = [l3[:, :, 0], l3[:, :, -1], l3[:, 0, :], l3[:, -1, :]][f].reshape(-1)
                gc = np.ascontiguousarray(decomp.ghost_plane(idx, b, f)).reshape(-1)
                self.face[f] = (torch.from_numpy(lc), torch.from_numpy(np.asarray(A[self.g[lc], gc]).ravel()))

    def jacobian_apply(self, x, y):
        y.copy_(torch.from_numpy(self.Abb @ x.numpy()))

    def face_apply(self, f, which, ghosts, y):
        lc, c = self.face[f]
        y.index_add_(0, lc, c * ghosts)

    def pack_face(self, f, field, out):
        out.copy_(field[self.face[f][0]])

    def vcycle(self, r, z):
        z.copy_(torch.from_numpy(self.lu.solve(r.numpy())))

    def dot(self, x, y):
        return float(np.dot(x.numpy(), y.numpy()))

    def axpby(self, a, x, b, y):
        y.copy_(a * x if b == 0.0 else a * x + b * y)


def _problem(A, idx, blocks, r):
    """A BlockProblem (its own pack, couple and exchange methods) over a stand-in context."""
    q = object.__new__(decomp.BlockProblem)
    q.block = blocks[r]
    q.ctx = _BlockCtx(A, idx, q.block)
    q.halo = decomp.Halo(blocks, r)
    q.buffers = {f: (torch.empty(len(lc), dtype=torch.float64), torch.empty(len(lc), dtype=torch.float64))
                 for f, (lc, _) in q.ctx.face.items()}
    return q


def _solve(probs, comm, bs):
    out = {}
    for kind in ("fcg", "fgmres"):
        if kind == "fcg":
            xs, its, ok, why = decomp.fcg(probs, comm, bs, ETA, MAXIT)
        else:
            xs, its, ok, why = decomp.fgmres(probs, comm, bs, ETA, MAXIT, RESTART)
        out[kind] = ([x.numpy().copy() for x in xs], its, ok)
    return out


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, px, py, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        grid, A, idx, b = _system()
        blocks = decomp.partition(grid, px, py)
        q = _problem(A, idx, blocks, rank)
        res = _solve([q], decomp.DistComm(dist, q, "cpu"), [torch.from_numpy(b[q.ctx.g].copy())])
        np.savez(os.path.join(out_dir, "rank%d.npz" % rank),
                 **{k + "_x": v[0][0] for k, v in res.items()},
                 **{k + "_its": np.array([v[1], v[2]]) for k, v in res.items()})
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("px,py", [(2, 1), (2, 2)])
def test_split_krylov_on_gloo_ranks_equals_one_process_and_the_oracle(px, py, tmp_path):
    import torch.multiprocessing as mp
    from oracle import krylov
    world = px * py
    mp.spawn(_rank, args=(world, _free_port(), px, py, str(tmp_path)), nprocs=world, join=True)
    grid, A, idx, b = _system()
    blocks = decomp.partition(grid, px, py)
    probs = [_problem(A, idx, blocks, r) for r in range(world)]
    local = _solve(probs, decomp.LocalComm(probs), [torch.from_numpy(b[q.ctx.g].copy()) for q in probs])
    parts = [np.load(tmp_path / ("rank%d.npz" % r)) for r in range(world)]
    for kind in ("fcg", "fgmres"):
        xs, its, ok = local[kind]
        assert ok and its > (2 * RESTART if kind == "fgmres" else 3)  # FGMRES restarts across the ranks
        for r, d in enumerate(parts):  # the ranks' run is the one-process run, bit for bit
            assert list(d[kind + "_its"]) == [its, 1]
            np.testing.assert_array_equal(d[kind + "_x"], xs[r])
        x = np.empty(grid.n)
        for q, xr in zip(probs, xs):
            x[q.ctx.g] = xr
        lus = [(q.ctx.g, q.ctx.lu) for q in probs]

        def prec(v):  # the blocks' solves on the whole vector
            z = np.empty_like(v)
            for g, lu in lus:
                z[g] = lu.solve(v[g])
            return z
        if kind == "fcg":
            xo, its_o, ok_o, _ = krylov.fcg(lambda v: A @ v, prec, b, ETA, MAXIT)
        else:
            xo, its_o, ok_o, _ = krylov.fgmres(lambda v: A @ v, prec, b, ETA, MAXIT, RESTART)
        assert ok_o and abs(its - its_o) <= 1
        assert np.linalg.norm(b - A @ x) <= ETA * np.linalg.norm(b) * (1 + 1e-6)
        assert np.linalg.norm(x - xo) <= 1e-8 * np.linalg.norm(xo)


# ---------------------------------------------------------------- the split Newton step

class _NonlinearCtx(_BlockCtx):
    """A backward-Euler-like step of the block's rows: Phi(p) = (s(p) - s_old) / dt
    + A p - rhs with s(p) = p + p^3 / 10 (monotone), the neighbours' p entering as
    ghosts through the interface couplings; J = diag(s'(p)) / dt + A_bb; the
    preconditioner is the exact solve with J (factored at setup and refresh)."""

    def __init__(self, A, idx, b, rhs):
        super().__init__(A, idx, b)
        self.A_bb = self.Abb.tocsr()
        self.absA = abs(self.A_bb)
        self.rhs = rhs[self.g]
        self.ghosts = {}

    def saturation(self, p, s):
        s.copy_(p + p ** 3 / 10)

    def set_face_values(self, f, ghosts):
        self.ghosts[f] = ghosts.numpy().copy()

    def residual3(self, p, s_old, dt, F):
        pn, so = p.numpy(), s_old.numpy()
        ap, mag = self.A_bb @ pn, self.absA @ np.abs(pn)
        for f, (lc, c) in self.face.items():
            np.add.at(ap, lc.numpy(), c.numpy() * self.ghosts[f])
            np.add.at(mag, lc.numpy(), np.abs(c.numpy() * self.ghosts[f]))
        s = pn + pn ** 3 / 10
        Fn = (s - so) / dt + ap - self.rhs
        F.copy_(torch.from_numpy(Fn))
        mag += (np.abs(s) + np.abs(so)) / dt + np.abs(self.rhs)
        return float(np.linalg.norm(Fn)), float(np.abs(Fn).max()), float(np.linalg.norm(mag))

    def jacobian(self, p, dt):
        pn = p.numpy()
        self.Abb = (sp.diags((1.0 + 0.3 * pn ** 2) / dt) + self.A_bb).tocsc()

    def amg_setup(self, opts):
        self.lu = spla.splu(self.Abb)

    def amg_update(self, policy):
        self.lu = spla.splu(self.Abb)


def _nonlinear_problem(A, idx, blocks, r, rhs):
    q = _problem(A, idx, blocks, r)
    q.ctx = _NonlinearCtx(A, idx, q.block, rhs)
    return q


def _newton_opts(kind):
    from types import SimpleNamespace
    from paper_2112_05051_gb300 import richards as rb
    k = rb.KRYLOV_FGMRES if kind == "fgmres" else rb.KRYLOV_FCG
    return SimpleNamespace(rtol=1e-10, atol=1e-30, max_newton=30, armijo_c=1e-4, lambda_min=1e-8, amg=None,
                           krylov=SimpleNamespace(kind=k, eta=1e-8, maxit=200, restart=RESTART))


DT = 0.5


def _step(probs, comm, kind):
    p = [torch.zeros(q.ctx.g.size, dtype=torch.float64) for q in probs]
    ok, its, lin, why = decomp.newton_step(probs, comm, p, DT, _newton_opts(kind))
    return [v.numpy().copy() for v in p], its, lin, ok, why


def _newton_rank(rank, world, port, px, py, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        grid, A, idx, b = _system()
        blocks = decomp.partition(grid, px, py)
        q = _nonlinear_problem(A, idx, blocks, rank, 8.0 * b)
        out = {}
        for kind in ("fcg", "fgmres"):
            p, its, lin, ok, why = _step([q], decomp.DistComm(dist, q, "cpu"), kind)
            out[kind + "_p"] = p[0]
            out[kind + "_its"] = np.array([its, lin, int(ok)])
        np.savez(os.path.join(out_dir, "newton%d.npz" % rank), **out)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("px,py", [(2, 1), (2, 2)])
def test_split_newton_step_on_gloo_ranks_equals_one_process_and_solves_the_whole_system(px, py, tmp_path):
    import torch.multiprocessing as mp
    world = px * py
    mp.spawn(_newton_rank, args=(world, _free_port(), px, py, str(tmp_path)), nprocs=world, join=True)
    grid, A, idx, b = _system()
    rhs = 8.0 * b
    blocks = decomp.partition(grid, px, py)
    parts = [np.load(tmp_path / ("newton%d.npz" % r)) for r in range(world)]
    # the whole system's solution by Newton with direct solves
    pw = np.zeros(grid.n)
    phi = lambda p: (p + p ** 3 / 10) / DT + A @ p - rhs
    for _ in range(50):
        F = phi(pw)
        if np.linalg.norm(F) <= 1e-14 * np.linalg.norm(rhs):
            break
        pw = pw - spla.spsolve((sp.diags((1.0 + 0.3 * pw ** 2) / DT) + A).tocsc(), F)
    assert np.abs(pw).max() > 1.0  # the cubic term matters
    for kind in ("fcg", "fgmres"):
        probs = [_nonlinear_problem(A, idx, blocks, r, rhs) for r in range(world)]
        p, its, lin, ok, why = _step(probs, decomp.LocalComm(probs), kind)
        assert ok, why
        assert its >= 3 and lin > its
        for r, d in enumerate(parts):  # the ranks' step is the one-process step, bit for bit
            assert list(d[kind + "_its"]) == [its, lin, 1]
            np.testing.assert_array_equal(d[kind + "_p"], p[r])
        x = np.empty(grid.n)
        for q, pr in zip(probs, p):
            x[q.ctx.g] = pr
        assert np.linalg.norm(phi(x)) <= 1e-10 * np.linalg.norm(phi(np.zeros(grid.n))) * (1 + 1e-6)
        assert np.abs(x - pw).max() <= 1e-9 * np.abs(pw).max()
