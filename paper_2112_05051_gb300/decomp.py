"""Slab decomposition of the grid (Sec. 5.1): 2D x-y blocks with full z-columns.

The paper distributes the domain over processes by a block decomposition in
the horizontal plane, every process owning whole vertical columns, and
exchanges a one-cell halo before each residual evaluation.  Here each block is a
grid of its own (`rich_create`), with the spacing of the whole grid, whose faces
towards a neighbouring block are `RICH_BC_INTERFACE` faces: the ghost behind
such a face is the neighbour's boundary cell, with the neighbour's K_s (known
from the input) and the neighbour's current pressure (refreshed by a halo
exchange before every residual).  Faces on the boundary of the whole grid keep
its boundary condition, per-cell values sliced to the block.  With that, a
block's residual and its rows of J and A_aux are those of the whole grid.

The exchange packs the cells next to each interface face with the library's
face-pack kernel and hands them to the neighbour: between ranks through
`torch.distributed` point-to-point messages (one rank per block), or, for
blocks held by one process, by copies between their buffers.
"""
import dataclasses
from typing import List, Tuple

FACES = 6  # x-, x+, y-, y+, z-, z+


@dataclasses.dataclass(frozen=True)
class Block:
    rank: int
    i0: int  # cells [i0, i1) x [j0, j1) x all k of the whole grid
    i1: int
    j0: int
    j1: int
    nbr: Tuple[int, int, int, int, int, int]  # neighbour rank behind each face, -1 on the grid boundary


def _split(n, parts):
    base, extra = divmod(n, parts)
    edges = [0]
    for q in range(parts):
        edges.append(edges[-1] + base + (1 if q < extra else 0))
    return edges


def partition(grid, px, py) -> List[Block]:
    """px x py blocks of nearly equal size (the first n % p parts one cell wider);
    rank = bx + px * by."""
    if px < 1 or py < 1 or px > grid.nx or py > grid.ny:
        raise ValueError("a %d x %d split of a %d x %d grid" % (px, py, grid.nx, grid.ny))
    ex, ey = _split(grid.nx, px), _split(grid.ny, py)
    out = []
    for by in range(py):
        for bx in range(px):
            r = bx + px * by
            nbr = (r - 1 if bx > 0 else -1, r + 1 if bx < px - 1 else -1,
                   r - px if by > 0 else -1, r + px if by < py - 1 else -1, -1, -1)
            out.append(Block(r, ex[bx], ex[bx + 1], ey[by], ey[by + 1], nbr))
    return out


def sub_grid(grid, b):
    """The block as a grid of its own, carrying the whole grid's spacing explicitly
    (its own box's l / (n + 1) need not reproduce h to the last bit)."""
    from paper_2112_05051_gb300 import synth
    hx, hy, hz = grid.h
    nx, ny = b.i1 - b.i0, b.j1 - b.j0
    return synth.Grid(nx, ny, grid.nz, hx * (nx + 1), hy * (ny + 1), grid.lz, spacing=(hx, hy, hz))


def face_cells(grid, f):
    """Cells of face f of a grid: ny nz on x faces, nx nz on y faces, nx ny on z faces."""
    axis = f >> 1
    return grid.ny * grid.nz if axis == 0 else (grid.nx * grid.nz if axis == 1 else grid.nx * grid.ny)


def cell_block(a3, b):
    """The block's cells of a whole-grid array of shape (nz, ny, nx)."""
    return a3[:, b.j0:b.j1, b.i0:b.i1]


def _face_slice(a2, f, b):
    """The block's part of a whole-grid per-cell face array (flat face layout)."""
    axis = f >> 1
    return a2[:, b.j0:b.j1] if axis == 0 else (a2[:, b.i0:b.i1] if axis == 1 else a2[b.j0:b.j1, b.i0:b.i1])


def ghost_plane(a3, b, f):
    """The whole-grid cells behind interface face f of block b, in the face layout
    (x faces: j + ny k, y faces: i + nx k): the ghosts of that face."""
    if f == 0:
        return a3[:, b.j0:b.j1, b.i0 - 1]
    if f == 1:
        return a3[:, b.j0:b.j1, b.i1]
    if f == 2:
        return a3[:, b.j0 - 1, b.i0:b.i1]
    if f == 3:
        return a3[:, b.j1, b.i0:b.i1]
    raise ValueError("blocks have no interface on the z faces")


@dataclasses.dataclass(frozen=True)
class BlockBC:
    """Boundary conditions of a block: the whole grid's on its outer faces (per-cell
    values sliced), interface faces towards its neighbours."""
    kind: Tuple[int, int, int, int, int, int]
    value: Tuple[float, float, float, float, float, float]
    fields: Tuple
    ghost_ks: Tuple

    def field(self, f):
        return self.fields[f]

    def ghost_ks_field(self, f):
        return self.ghost_ks[f]


def block_bc(grid, bc, b, ks=None):
    """BlockBC of block b: whole-grid bc on the outer faces; on interface faces a
    placeholder ghost pressure (set by the first exchange) and the ghost K_s
    (ks: whole-grid K_s, flat in cell order, or None for a constant K_s)."""
    import numpy as np
    from paper_2112_05051_gb300 import richards as rb
    sg = sub_grid(grid, b)
    k3 = None if ks is None else np.asarray(ks, dtype=np.float64).reshape(grid.shape)
    shapes = [(grid.nz, grid.ny), (grid.nz, grid.ny), (grid.nz, grid.nx), (grid.nz, grid.nx),
              (grid.ny, grid.nx), (grid.ny, grid.nx)]
    kind, value, fields, gks = [], [], [], []
    for f in range(FACES):
        if b.nbr[f] >= 0:
            kind.append(rb.BC_INTERFACE)
            value.append(0.0)
            fields.append(np.zeros(face_cells(sg, f)))
            gks.append(None if k3 is None else np.ascontiguousarray(ghost_plane(k3, b, f)).ravel())
        else:
            kind.append(bc.kind[f])
            value.append(bc.value[f])
            fld = bc.field(f) if hasattr(bc, "field") else None
            if fld is not None:
                fld = np.ascontiguousarray(_face_slice(np.asarray(fld).reshape(shapes[f]), f, b)).ravel()
            fields.append(fld)
            gks.append(None)
    return BlockBC(tuple(kind), tuple(value), tuple(fields), tuple(gks))


class Halo:
    """Halo exchange of one cell field between the blocks of a partition.

    ``pack(f, out)`` must write the cells of the local field next to face f into
    ``out`` (the face layout); ``apply(f, ghosts)`` receives the neighbour's cells
    behind face f.  The neighbour behind face f packs its opposite face f ^ 1, and
    the two index their face arrays the same way (a tensor-product partition: the
    blocks on either side of an x interface share their j range, of a y interface
    their i range).
    """

    def __init__(self, blocks, rank):
        self.blocks = blocks
        self.block = blocks[rank]

    def exchange(self, dist, pack, apply, buffers):
        """Point-to-point exchange with the neighbour ranks (torch.distributed):
        buffers[f] = (send, recv) tensors of face f's size on the backend's device."""
        reqs = []
        for f in range(FACES):
            r = self.block.nbr[f]
            if r < 0:
                continue
            send, recv = buffers[f]
            pack(f, send)
            reqs.append(dist.isend(send, r, tag=f))       # my face f is the neighbour's face f ^ 1
            reqs.append(dist.irecv(recv, r, tag=f ^ 1))
        for q in reqs:
            q.wait()
        for f in range(FACES):
            if self.block.nbr[f] >= 0:
                apply(f, buffers[f][1])


def exchange_local(blocks, packs, applies, buffers):
    """The same exchange for blocks held by one process: packs[r](f, out) and
    applies[r](f, ghosts) of every block, buffers[r][f] = (send, recv)."""
    for b in blocks:
        for f in range(FACES):
            if b.nbr[f] >= 0:
                packs[b.rank](f, buffers[b.rank][f][0])
    for b in blocks:
        for f in range(FACES):
            r = b.nbr[f]
            if r >= 0:
                recv = buffers[b.rank][f][1]
                recv.copy_(buffers[r][f ^ 1][0])
                applies[b.rank](f, recv)


class BlockProblem:
    """One block of a partition as a context of its own, with the halo exchange of
    its pressure before each residual.

    grid, soil, bc, kmean, ks: the whole problem (ks flat in cell order or None);
    blocks, rank: the partition and this block.  Cell arrays of the block are in
    its own order (i fastest over its nx, then j over its ny, then k).
    """

    def __init__(self, grid, soil, bc, kmean, ks, blocks, rank, precision=0):
        import numpy as np
        import torch
        from paper_2112_05051_gb300 import richards as rb
        self.block = blocks[rank]
        self.grid = sub_grid(grid, self.block)
        ks_b = None
        if ks is not None:
            ks_b = np.ascontiguousarray(cell_block(np.asarray(ks).reshape(grid.shape), self.block)).ravel()
        self.ctx = rb.Context(self.grid, soil, block_bc(grid, bc, self.block, ks), kmean, ks_b, precision=precision)
        self.halo = Halo(blocks, rank)
        self.buffers = {}
        for f in range(FACES):
            if self.block.nbr[f] >= 0:
                m = face_cells(self.grid, f)
                self.buffers[f] = (torch.empty(m, dtype=torch.float64, device="cuda"),
                                   torch.empty(m, dtype=torch.float64, device="cuda"))

    def pack(self, field):
        return lambda f, out: self.ctx.pack_face(f, field, out)

    def apply(self, f, ghosts):
        self.ctx.set_face_values(f, ghosts)

    def exchange(self, dist, p):
        """Ghost pressures from the neighbour ranks (one rank per block)."""
        self.halo.exchange(dist, self.pack(p), self.apply, self.buffers)

    def couple(self, which, y):
        """The apply of a halo exchange of x that adds the block's interface couplings
        in J (which = 0) or A_aux (which = 1) times the neighbour's x to y."""
        return lambda f, ghosts: self.ctx.face_apply(f, which, ghosts, y)

    def apply_J(self, dist, x, y):
        """y = J x of the split grid, this block's rows (one rank per block)."""
        self.ctx.jacobian_apply(x, y)
        self.halo.exchange(dist, self.pack(x), self.couple(0, y), self.buffers)

    def residual(self, p, s_old, dt, F):
        """Phi of the block (after an exchange); returns (sum of Phi^2, max |Phi|,
        sum of m^2), the pieces of the whole grid's norms and of its round-off
        scale ||m||_2 (m: the magnitudes of the terms summed into Phi per cell)."""
        n2, ninf, nm = self.ctx.residual3(p, s_old, dt, F)
        return n2 * n2, ninf, nm * nm

    def close(self):
        self.ctx.close()


def exchange_blocks(problems, fields, applies=None):
    """Halo exchange of one field among blocks held by this process
    (problems[r], fields[r]: block r and its cell field; applies[r](f, ghosts):
    what block r does with the neighbour's cells behind face f, by default they
    become the ghost pressures of its interface faces)."""
    exchange_local([q.block for q in problems], [q.pack(x) for q, x in zip(problems, fields)],
                   applies or [q.apply for q in problems], [q.buffers for q in problems])


def apply_J_blocks(problems, xs, ys):
    """ys[r] = J x of the split grid on block r, for blocks held by this process."""
    for q, x, y in zip(problems, xs, ys):
        q.ctx.jacobian_apply(x, y)
    exchange_blocks(problems, xs, [q.couple(0, y) for q, y in zip(problems, ys)])


def combine_norms(parts):
    """(||Phi||_2, ||Phi||_inf) of the whole grid from the blocks' (sum of squares, max)."""
    import math
    return math.sqrt(sum(p[0] for p in parts)), max(p[1] for p in parts)


# ---------------------------------------------------------------- the split grid's solve

class LocalComm:
    """All blocks of the split grid in this process (one device): halo exchanges
    are copies, sums run over the blocks in rank order."""

    def __init__(self, problems):
        self.problems = problems

    def exchange(self, fields, applies=None):
        exchange_blocks(self.problems, fields, applies)

    def sum(self, values):
        return float(sum(values))

    def max(self, values):
        return float(max(values))


class DistComm:
    """One block per rank (torch.distributed, a device per rank): halo exchanges are
    point-to-point messages, sums gather every rank's value and add them in rank
    order with Python's compensated float sum (the same result on every rank,
    whatever the backend's reduction order; LocalComm sums the same way)."""

    def __init__(self, dist, problem, device):
        self.dist, self.problems, self.device = dist, [problem], device

    def exchange(self, fields, applies=None):
        q = self.problems[0]
        q.halo.exchange(self.dist, q.pack(fields[0]), (applies or [q.apply])[0], q.buffers)

    def _gather(self, v):
        import torch
        t = torch.tensor([float(v)], dtype=torch.float64, device=self.device)
        out = [torch.empty_like(t) for _ in range(self.dist.get_world_size())]
        self.dist.all_gather(out, t)
        return [float(o.item()) for o in out]

    def sum(self, values):
        return float(sum(self._gather(values[0])))

    def max(self, values):
        return float(max(self._gather(values[0])))


def dot(problems, comm, xs, ys):
    return comm.sum([q.ctx.dot(x, y) for q, x, y in zip(problems, xs, ys)])


def apply_J(problems, comm, xs, ys):
    """ys = J xs of the split grid: each block's stencil SpMV, then its interface
    couplings times the neighbours' x after a halo exchange of x."""
    for q, x, y in zip(problems, xs, ys):
        q.ctx.jacobian_apply(x, y)
    comm.exchange(xs, [q.couple(0, y) for q, y in zip(problems, ys)])


def fcg(problems, comm, b, eta, maxit):
    """Flexible CG (Notay, truncation 1) for J x = b on the split grid, right-
    preconditioned by each block's own V-cycle on its own hierarchy (decoupled
    aggregation, Sec. 5.1-5.2).  Returns (x, iterations, converged, reason)."""
    import math
    import torch
    new = lambda: [torch.empty_like(v) for v in b]
    x = [torch.zeros_like(v) for v in b]
    r, z, p, qv, qprev = new(), new(), new(), new(), new()
    for q, rr, bb in zip(problems, r, b):
        q.ctx.axpby(1.0, bb, 0.0, rr)
    bn = math.sqrt(dot(problems, comm, b, b))
    if not bn > 0:
        return x, 0, True, None
    target, best, pq_prev = eta * bn, bn, None
    for it in range(1, maxit + 1):
        for q, rr, zz in zip(problems, r, z):
            q.ctx.vcycle(rr, zz)
        if it == 1:
            for q, zz, pp in zip(problems, z, p):
                q.ctx.axpby(1.0, zz, 0.0, pp)
        else:
            beta = dot(problems, comm, z, qprev) / pq_prev
            for q, zz, pp in zip(problems, z, p):
                q.ctx.axpby(1.0, zz, -beta, pp)
        apply_J(problems, comm, p, qv)
        pq = dot(problems, comm, p, qv)
        if not pq > 0:
            return x, it, False, "curvature"
        alpha = dot(problems, comm, p, r) / pq
        for q, pp, qq, xx, rr in zip(problems, p, qv, x, r):
            q.ctx.axpby(alpha, pp, 1.0, xx)
            q.ctx.axpby(-alpha, qq, 1.0, rr)
        rn = math.sqrt(dot(problems, comm, r, r))
        if rn <= target:
            return x, it, True, None
        if rn > 10.0 * best:
            return x, it, False, "growth"
        best = min(best, rn)
        qv, qprev, pq_prev = qprev, qv, pq
    return x, maxit, False, "maxit"


def newton_step(problems, comm, p, dt, opts):
    """One backward-Euler step (Sec. 3) of the split grid: inexact Newton with the
    Armijo line search, the halo of p exchanged before every residual and Jacobian,
    the correction solved by `fcg`, or `fgmres` when opts.krylov.kind asks for it,
    with each block's own hierarchy (set up at the first iteration, refreshed at
    the next ones), norms and slopes summed over the blocks.  p: the blocks' pressures (updated in place); opts: rich_newton_opts
    (its rtol, atol, max_newton, armijo_c, lambda_min, krylov eta / maxit and amg
    settings).  Converged when ||Phi|| <= max(rtol ||Phi_0||, atol, eps ||m||_2), the
    same test as the library's step, its round-off floor from the blocks' summed
    m^2.  Returns (converged, newton iterations, linear iterations, reason)."""
    import math
    import torch
    from paper_2112_05051_gb300 import richards as rb
    new = lambda: [torch.empty_like(v) for v in p]
    s_old, F, Ft, trial, rhs, Jd = new(), new(), new(), new(), new(), new()
    for q, pp, so in zip(problems, p, s_old):
        q.ctx.saturation(pp, so)

    eps = 2.220446049250313e-16

    def phi(pp, out):  # (||Phi||_2, its round-off floor)
        comm.exchange(pp)
        parts = [q.residual(x, so, dt, f) for q, x, so, f in zip(problems, pp, s_old, out)]
        return math.sqrt(comm.sum([a for a, _, _ in parts])), eps * math.sqrt(comm.sum([c for _, _, c in parts]))

    fn, floor = phi(p, F)
    if not math.isfinite(fn):
        return False, 0, 0, "nonfinite"
    tol = max(opts.rtol * fn, opts.atol)
    lin = 0
    for it in range(opts.max_newton + 1):
        if fn <= max(tol, floor):
            return True, it, lin, None
        if it == opts.max_newton:
            return False, it, lin, "newton"
        for q, pp in zip(problems, p):  # the ghosts hold the halo of this p (its residual came last)
            q.ctx.jacobian(pp, dt)
            if it == 0:
                q.ctx.amg_setup(opts.amg)
            else:
                q.ctx.amg_update(rb.AMG_REFRESH)
        for q, f, r in zip(problems, F, rhs):
            q.ctx.axpby(-1.0, f, 0.0, r)
        if opts.krylov.kind == rb.KRYLOV_FGMRES:
            d, its, ok, why = fgmres(problems, comm, rhs, opts.krylov.eta, opts.krylov.maxit, opts.krylov.restart)
        else:
            d, its, ok, why = fcg(problems, comm, rhs, opts.krylov.eta, opts.krylov.maxit)
        lin += its
        if not ok:
            return False, it, lin, "linear (%s)" % why
        apply_J(problems, comm, d, Jd)
        slope = dot(problems, comm, F, Jd)
        if not slope < 0:
            return False, it, lin, "line search (no descent)"
        f0, lam = 0.5 * fn * fn, 1.0
        while True:
            for q, pp, dd, tt in zip(problems, p, d, trial):
                q.ctx.axpby(1.0, pp, 0.0, tt)
                q.ctx.axpby(lam, dd, 1.0, tt)
            ft, floor_t = phi(trial, Ft)
            f_t = 0.5 * ft * ft
            if not math.isfinite(f_t):
                return False, it, lin, "nonfinite"
            if f_t <= f0 + opts.armijo_c * lam * slope:
                break
            lq = -slope * lam * lam / (2.0 * (f_t - f0 - slope * lam))
            lam = min(max(lq, 0.1 * lam), 0.5 * lam)
            if lam < opts.lambda_min:
                comm.exchange(p)  # the ghosts back to the accepted p
                return False, it, lin, "line search"
        for q, pp, tt in zip(problems, p, trial):
            q.ctx.axpby(1.0, tt, 0.0, pp)
        F, Ft = Ft, F
        fn, floor = ft, floor_t


def fgmres(problems, comm, b, eta, maxit, m):
    """Flexible GMRES(m) for J x = b on the split grid, right-preconditioned by each
    block's own V-cycle: classical Gram-Schmidt with a second pass when
    ||w'||^2 < ||w||^2 / 2 (DGKS), Givens rotations, restarts every m iterations
    from the true residual.  Returns (x, iterations, converged, reason); a column
    whose rotation is undefined (J z = 0: both its entries vanish) ends the solve
    with the columns before it and the reason "breakdown"."""
    import math
    import torch
    new = lambda: [torch.empty_like(v) for v in b]
    x = [torch.zeros_like(v) for v in b]
    r, w, jx = new(), new(), new()
    for q, rr, bb in zip(problems, r, b):
        q.ctx.axpby(1.0, bb, 0.0, rr)
    beta = math.sqrt(dot(problems, comm, r, r))
    if not beta > 0:
        return x, 0, True, None
    target, its = eta * beta, 0
    V = [new() for _ in range(m + 1)]  # the basis and the preconditioned directions, reused by every cycle
    Z = [new() for _ in range(m)]
    while True:
        H = [[0.0] * m for _ in range(m + 1)]
        cs, sn, g = [0.0] * m, [0.0] * m, [0.0] * (m + 1)
        g[0] = beta
        for q, rr, v in zip(problems, r, V[0]):
            q.ctx.axpby(1.0 / beta, rr, 0.0, v)
        jdone, conv, broke = 0, False, False
        for j in range(m):
            for q, v, z in zip(problems, V[j], Z[j]):
                q.ctx.vcycle(v, z)
            apply_J(problems, comm, Z[j], w)
            wn2 = dot(problems, comm, w, w)
            h1 = [dot(problems, comm, V[i], w) for i in range(j + 1)]
            for i in range(j + 1):
                for q, vi, ww in zip(problems, V[i], w):
                    q.ctx.axpby(-h1[i], vi, 1.0, ww)
            wp2 = dot(problems, comm, w, w)
            if wp2 < 0.5 * wn2:  # DGKS: a second pass
                h2 = [dot(problems, comm, V[i], w) for i in range(j + 1)]
                for i in range(j + 1):
                    for q, vi, ww in zip(problems, V[i], w):
                        q.ctx.axpby(-h2[i], vi, 1.0, ww)
                    h1[i] += h2[i]
                wp2 = dot(problems, comm, w, w)
            hn = math.sqrt(max(wp2, 0.0))
            for i in range(j + 1):
                H[i][j] = h1[i]
            H[j + 1][j] = hn
            if hn > 0:
                for q, ww, v in zip(problems, w, V[j + 1]):
                    q.ctx.axpby(1.0 / hn, ww, 0.0, v)
            for i in range(j):
                t = cs[i] * H[i][j] + sn[i] * H[i + 1][j]
                H[i + 1][j] = -sn[i] * H[i][j] + cs[i] * H[i + 1][j]
                H[i][j] = t
            den = math.hypot(H[j][j], H[j + 1][j])
            if not den > 0:
                broke = True
                break
            cs[j], sn[j] = H[j][j] / den, H[j + 1][j] / den
            H[j][j], H[j + 1][j] = den, 0.0
            g[j + 1], g[j] = -sn[j] * g[j], cs[j] * g[j]
            its += 1
            jdone = j + 1
            if abs(g[j + 1]) <= target or hn == 0.0:
                conv = True
                break
            if its >= maxit:
                break
        y = [0.0] * jdone
        for i in range(jdone - 1, -1, -1):
            y[i] = (g[i] - sum(H[i][k] * y[k] for k in range(i + 1, jdone))) / H[i][i]
        for i in range(jdone):
            for q, zz, xx in zip(problems, Z[i], x):
                q.ctx.axpby(y[i], zz, 1.0, xx)
        if conv:
            return x, its, True, None
        if broke:
            return x, its, False, "breakdown"
        if its >= maxit:
            return x, its, False, "maxit"
        apply_J(problems, comm, x, jx)  # restart from the true residual
        for q, bb, jj, rr in zip(problems, b, jx, r):
            q.ctx.axpby(1.0, bb, 0.0, rr)
            q.ctx.axpby(-1.0, jj, 1.0, rr)
        beta = math.sqrt(dot(problems, comm, r, r))
        if beta <= target:
            return x, its, True, None
