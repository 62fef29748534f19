"""Smoothed-aggregation AMG with MIS-2 aggregation and an l1-Jacobi V-cycle (oracle; test infrastructure).

The paper's preconditioner (Sec. 5.2) is a symmetric V-cycle (eq. (Vcycle))
over Galerkin coarse matrices M_{l+1} = P_l^T M_l P_l built by decoupled
smoothed aggregation (DSVMB, Vanek-Mandel-Brezina) from the diffusion-only
matrix, with an l1-Jacobi smoother.  The paper names these pieces without
formulas; the oracle fixes them as follows (each reading is listed in the
design notes):

  strength     j != i is strong for i iff a_ij^2 >= theta_l^2 |a_ii a_jj|,
               symmetrised (strong if either direction is); theta_l =
               theta 2^-l on level l (theta = 0.08).  A constant threshold
               leaves most couplings of the smoothed-aggregation coarse
               operators weak, the aggregates there shrink to 1-3 nodes and
               the operator complexity explodes (about 27 at 40^3); halving
               it per level keeps it near 3.
  priority     key(i) = (top 30 bits of splitmix64(seed ^ i)) << 32 | i;
               splitmix64 is the published SplitMix64 finaliser (Steele, Lea
               and Flood 2014).  Larger key wins; keys are distinct.
  MIS-2        synchronous rounds over tuples (state, key) with state
               OUT=0 < UNDECIDED=1 < IN=2: m = max over the closed 2-hop
               neighbourhood (two 1-hop max passes of the previous round's
               tuples); an undecided node whose m is its own tuple turns IN,
               an undecided node whose m belongs to an IN node turns OUT.
  aggregates   roots = IN nodes numbered by increasing index; pass 1: a
               non-root with a strong root neighbour joins the one with the
               largest key; pass 2: a remaining node joins the aggregate of
               the pass-1 neighbour whose root has the largest key.
               Isolated nodes (no strong neighbour) start OUT of MIS-2.
               pass 3: an isolated node whose row is not diagonally dominant
               (a_ii < 2 sum_{j!=i} |a_ij|) joins the aggregate of its
               aggregated matrix neighbour j with the largest
               (fp32(|a_ij|), key(j)); the others (dominant rows, e.g. cells
               under a Dirichlet face) join no aggregate, their P_tent row is
               empty and the smoother alone resolves them.  On high-contrast
               fields a low-conductivity cell between cells that carry much
               larger couplings elsewhere has only weak couplings by the
               symmetric measure, yet its row sums to about zero (its error is
               the average of its neighbours'); left out of the coarse space,
               it costs the V-cycle most of its contraction.
  prolongator  P = (I - omega D^-1 A) P_tent, P_tent[i, agg(i)] = 1,
               omega = 4 / (3 rho), rho = max_i sum_j |a_ij| / |a_ii|;
               structural pattern, no dropping.  Only the first
               smooth_levels levels smooth P (default: all); deeper levels
               use P = P_tent, which keeps the coarsest operators sparse.
  coarse       A_c = R (A P) with R = P^T, structural pattern.  Coarsening
               stops when a level has fewer than coarse_max unknowns, the
               size ratio exceeds 0.8, or max_levels is reached; the last
               level is solved by dense Cholesky, or, when coarsening stalled
               above DENSE_MAX unknowns, by COARSE_SWEEPS l1-Jacobi sweeps.
  smoother     l1-Jacobi x <- x + D_l1^-1 (b - A x), D_l1,ii = sum_j |a_ij|.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

STATE_OUT, STATE_UNDECIDED, STATE_IN = 0, 1, 2
_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)
_LOW32 = np.uint64(0xFFFFFFFF)


def splitmix64(x):
    """SplitMix64 output function applied to counter values x (uint64, wraps mod 2^64)."""
    z = np.asarray(x, dtype=np.uint64) + _GOLDEN
    z = (z ^ (z >> np.uint64(30))) * _M1
    z = (z ^ (z >> np.uint64(27))) * _M2
    return z ^ (z >> np.uint64(31))


def priority_keys(n, seed):
    """Distinct 62-bit keys: (top 30 bits of splitmix64(seed ^ i)) << 32 | i."""
    idx = np.arange(n, dtype=np.uint64)
    pi = splitmix64(np.uint64(seed) ^ idx)
    return ((pi >> np.uint64(34)) << np.uint64(32)) | idx


def _pattern(rows, cols, n):
    m = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    m.sum_duplicates()
    m.sort_indices()
    m.data[:] = 1.0
    return m


def strength(A, theta):
    """Symmetrised strength pattern (no diagonal) of a square CSR matrix."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    cols = A.indices
    d = A.diagonal()
    strong = (cols != rows) & (A.data * A.data >= theta * theta * np.abs(d[rows] * d[cols]))
    r, c = rows[strong], cols[strong]
    return _pattern(np.concatenate([r, c]), np.concatenate([c, r]), n)


def _closed(S):
    n = S.shape[0]
    return _pattern(np.concatenate([np.repeat(np.arange(n), np.diff(S.indptr)), np.arange(n)]),
                    np.concatenate([S.indices, np.arange(n)]), n)


def _max_closed(Sc, v):
    """m[i] = max of v over the closed neighbourhood of i (every row holds i itself)."""
    return np.maximum.reduceat(v[Sc.indices], Sc.indptr[:-1])


def mis2(S, keys):
    """Distance-2 maximal independent set by synchronous rounds; returns (state, rounds).

    Isolated nodes (no strong neighbour) are OUT from the start.
    """
    Sc = _closed(S)
    n = S.shape[0]
    state = np.full(n, STATE_UNDECIDED, dtype=np.uint64)
    state[np.diff(S.indptr) == 0] = STATE_OUT
    rounds = 0
    while np.any(state == STATE_UNDECIDED):
        t = (state << np.uint64(62)) | keys
        m = _max_closed(Sc, _max_closed(Sc, t))
        und = state == STATE_UNDECIDED
        new_in = und & (m == t)
        new_out = und & ((m >> np.uint64(62)) == STATE_IN)
        state[new_in] = STATE_IN
        state[new_out] = STATE_OUT
        rounds += 1
    return state, rounds


def aggregate(S, state, keys, A=None):
    """Aggregate index per node (int64, -1 for nodes left out) and number of aggregates.

    With the matrix A given, pass 3 places the isolated nodes whose row is not
    diagonally dominant (module docstring); without it every isolated node is
    left out."""
    Sc = _closed(S)
    n = S.shape[0]
    isolated = np.diff(S.indptr) == 0
    roots = state == STATE_IN
    agg_id = np.cumsum(roots) - 1
    agg = np.full(n, -1, dtype=np.int64)
    agg[roots] = agg_id[roots]
    # pass 1: strong root neighbour with the largest key
    rootval = np.where(roots, keys + np.uint64(1), np.uint64(0))
    best = _max_closed(Sc, rootval)
    pass1 = (~roots) & (best > 0)
    agg[pass1] = agg_id[((best[pass1] - np.uint64(1)) & _LOW32).astype(np.int64)]
    # pass 2: neighbour assigned in pass 1 whose root has the largest key
    root_of_agg = np.flatnonzero(roots)
    val2 = np.zeros(n, dtype=np.uint64)
    val2[pass1] = keys[root_of_agg[agg[pass1]]] + np.uint64(1)
    rest = agg < 0
    best2 = _max_closed(Sc, val2)
    take = rest & (best2 > 0)
    agg[take] = agg_id[((best2[take] - np.uint64(1)) & _LOW32).astype(np.int64)]
    if np.any((agg < 0) & ~isolated):
        raise RuntimeError("aggregation left nodes unassigned")
    if A is not None:
        agg = join_isolated(A, agg, keys)
    return agg, int(roots.sum())


def join_isolated(A, agg, keys):
    """Pass 3: every node left out (agg = -1) whose row is not diagonally dominant,
    a_ii < 2 sum_{j != i} |a_ij|, joins the aggregate of the neighbour j with
    agg(j) >= 0 that has the largest (fp32(|a_ij|), key(j)); one synchronous pass
    over the aggregates of passes 1-2.  Rounding |a_ij| to FP32 keeps couplings that
    are equal in exact arithmetic equal whatever the order their FP64 values were
    summed in, so the key decides between them."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    out = agg.copy()
    d = A.diagonal()
    for i in np.flatnonzero(agg < 0):
        lo, hi = A.indptr[i], A.indptr[i + 1]
        cols = A.indices[lo:hi]
        vals = A.data[lo:hi]
        off = cols != i
        if not np.any(off) or not abs(d[i]) < 2.0 * np.sum(np.abs(vals[off])):
            continue
        best = None
        for j, v in zip(cols[off], vals[off]):
            if agg[j] < 0:
                continue
            cand = (np.float32(abs(v)), int(keys[j]))
            if best is None or cand > best[0]:
                best = (cand, j)
        if best is not None:
            out[i] = agg[best[1]]
    return out


def spgemm(A, B):
    """C = A B with the structural pattern of the product (entries that cancel to 0 are kept).

    scipy's product drops entries whose sum is exactly zero, so the pattern is
    taken from the product of the all-ones pattern matrices and the values
    from the numeric product.
    """
    A = sp.csr_matrix(A)
    B = sp.csr_matrix(B)
    onesA = sp.csr_matrix((np.ones_like(A.data), A.indices, A.indptr), shape=A.shape)
    onesB = sp.csr_matrix((np.ones_like(B.data), B.indices, B.indptr), shape=B.shape)
    pat = (onesA @ onesB).tocsr()
    pat.sort_indices()
    num = (A @ B).tocsr()
    num.sort_indices()
    ncol = np.int64(pat.shape[1])
    kp = np.repeat(np.arange(pat.shape[0], dtype=np.int64), np.diff(pat.indptr)) * ncol + pat.indices
    kn = np.repeat(np.arange(num.shape[0], dtype=np.int64), np.diff(num.indptr)) * ncol + num.indices
    vals = np.zeros(len(kp))
    vals[np.searchsorted(kp, kn)] = num.data
    return sp.csr_matrix((vals, pat.indices.copy(), pat.indptr.copy()), shape=pat.shape)


def transpose(P):
    R = sp.csr_matrix(P.T)
    R.sort_indices()
    return R


def tentative_prolongator(agg, nc):
    """P_tent[i, agg(i)] = 1; rows of isolated nodes (agg = -1) are empty."""
    n = len(agg)
    has = agg >= 0
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(has, out=indptr[1:])
    return sp.csr_matrix((np.ones(int(has.sum())), agg[has].astype(np.int64), indptr), shape=(n, nc))


def smoothed_prolongator(A, Pt):
    """P = (I - omega D^-1 A) P_tent with omega = 4/(3 ||D^-1 A||_inf)."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    d = A.diagonal()
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    rho = np.max(np.bincount(rows, weights=np.abs(A.data), minlength=n) / np.abs(d))
    omega = 4.0 / (3.0 * rho)
    vals = -omega * A.data / d[rows]
    vals = vals + (A.indices == rows)
    Smat = sp.csr_matrix((vals, A.indices.copy(), A.indptr.copy()), shape=A.shape)
    return spgemm(Smat, Pt), omega


def l1_diagonal(A):
    A = sp.csr_matrix(A)
    rows = np.repeat(np.arange(A.shape[0]), np.diff(A.indptr))
    return np.bincount(rows, weights=np.abs(A.data), minlength=A.shape[0])


# ---------------------------------------------------------------- matching aggregation
# The paper's second coarsening (SMATCH, Sec. 5.2, with aggregates of at most 8
# dofs in its runs) is coupled aggregation by weighted graph matching, named
# without formulas.  The oracle fixes it as follows:
#   weights   for the smooth vector of ones, the compatible weight of the edge
#             {i, j} is w_ij = 1 - (a_ij + a_ji) / (a_ii + a_jj), taken over the
#             negative couplings (a_ij + a_ji < 0) and rounded to FP32, so that
#             rounding-order differences of the FP64 matrices cannot reorder two
#             equal weights.  Edges are ordered by weight (larger first), then by
#             (min(i, j), max(i, j)) (smaller first): a strict total order.
#   matching  locally dominant: in synchronous rounds every unmatched node
#             proposes to its best unmatched neighbour, mutual proposals are
#             matched; rounds repeat while a proposal exists.  With a strict
#             total order this equals the sequential greedy matching (edges by
#             decreasing order, kept when both ends are free).
#   pairs     each matched pair, and each unmatched node alone, becomes a node
#             of the pair graph, numbered by its smallest member; the pair
#             graph's matrix is P_p^T A P_p with P_p the 0/1 pairing.
#   aggregates  log2(max_size) pairing passes (3 for aggregates of at most 8),
#             composed; the prolongator then follows the smoothed-aggregation
#             rule of the MIS-2 path.

def matching_weights(A):
    """Per stored entry: the FP32 compatible weight, or -inf where {i, j} is no edge."""
    A = sp.csr_matrix(A)
    A.sort_indices()
    n = A.shape[0]
    At = sp.csr_matrix(A.T)
    At.sort_indices()
    if not (np.array_equal(At.indptr, A.indptr) and np.array_equal(At.indices, A.indices)):
        raise ValueError("matching needs a structurally symmetric matrix")
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    cols = A.indices
    d = A.diagonal()
    s = A.data + At.data  # a_ij + a_ji, the same value seen from i and from j
    edge = (cols != rows) & (s < 0)
    w = np.full(len(cols), -np.inf, dtype=np.float32)
    w[edge] = (1.0 - s[edge] / (d[rows[edge]] + d[cols[edge]])).astype(np.float32)
    return rows, cols, w


def match(A):
    """Locally dominant matching in synchronous rounds; returns (mate, rounds), mate = -1 if unmatched."""
    rows, cols, w = matching_weights(A)
    n = A.shape[0]
    lo = np.minimum(rows, cols)
    hi = np.maximum(rows, cols)
    mate = np.full(n, -1, dtype=np.int64)
    rounds = 0
    while True:
        ok = np.isfinite(w) & (mate[rows] < 0) & (mate[cols] < 0)
        if not np.any(ok):
            break
        r, c, ww, l, h = rows[ok], cols[ok], w[ok], lo[ok], hi[ok]
        order = np.lexsort((h, l, -ww.astype(np.float64), r))  # by row, then best edge first
        first = np.ones(len(order), dtype=bool)
        first[1:] = r[order][1:] != r[order][:-1]
        cand = np.full(n, -1, dtype=np.int64)
        cand[r[order][first]] = c[order][first]
        i = np.flatnonzero(cand >= 0)
        mutual = i[cand[cand[i]] == i]
        mate[mutual] = cand[mutual]
        rounds += 1
    return mate, rounds


def greedy_matching(A):
    """Sequential greedy matching in the same edge order (the pin of match())."""
    rows, cols, w = matching_weights(A)
    n = A.shape[0]
    keep = np.isfinite(w) & (rows < cols)
    r, c, ww = rows[keep], cols[keep], w[keep]
    mate = np.full(n, -1, dtype=np.int64)
    for e in np.lexsort((c, r, -ww.astype(np.float64))):
        if mate[r[e]] < 0 and mate[c[e]] < 0:
            mate[r[e]] = c[e]
            mate[c[e]] = r[e]
    return mate


def pair_ids(mate):
    """Pair-graph node of every node (pairs and singletons numbered by their smallest member)."""
    n = len(mate)
    idx = np.arange(n)
    first = (mate < 0) | (idx < mate)
    ids = np.cumsum(first) - 1
    rep = np.where(mate < 0, idx, np.minimum(idx, mate))
    return ids[rep].astype(np.int64), int(first.sum())


def matching_aggregate(A, max_size=8):
    """Aggregates of at most max_size nodes by log2(max_size) pairing passes; (agg, nc, rounds)."""
    passes = int(np.floor(np.log2(max_size)))
    n = A.shape[0]
    agg = np.arange(n, dtype=np.int64)
    nc = n
    Ak = sp.csr_matrix(A)
    rounds = 0
    for _ in range(passes):
        mate, r = match(Ak)
        rounds += r
        ids, nk = pair_ids(mate)
        Pp = tentative_prolongator(ids, nk)
        Ak = spgemm(transpose(Pp), spgemm(Ak, Pp))
        agg = ids[agg]
        nc = nk
    return agg, nc, rounds


DENSE_MAX = 8192
COARSE_SWEEPS = 8


class Level:
    def __init__(self, A):
        self.A = sp.csr_matrix(A)
        self.dl1 = l1_diagonal(self.A)
        self.P = None
        self.R = None
        self.agg = None
        self.S = None
        self.mis_rounds = 0


class Hierarchy:
    def __init__(self, levels, chol):
        self.levels = levels
        self.chol = chol  # lower Cholesky factor of the coarsest matrix
        self.smoother = "l1jacobi"
        self.grid = None        # (nx, ny, nz) of level 0, for the hybrid GS blocks there
        self.hgs_seg = 16
        self.hgs_block = 16

    @property
    def sizes(self):
        return [lv.A.shape[0] for lv in self.levels]

    def operator_complexity(self):
        return sum(lv.A.nnz for lv in self.levels) / self.levels[0].A.nnz


def setup(A, theta=0.08, seed=1, coarse_max=2000, max_levels=10, max_ratio=0.8, smooth_levels=10,
          aggregation="mis2", max_agg_size=8, isolated_join=True, smoother="l1jacobi", grid=None,
          hgs_seg=16, hgs_block=16):
    """Build the hierarchy from a symmetric positive definite CSR matrix.

    aggregation: "mis2" (strength graph + MIS-2 roots) or "matching"
    (compatible weighted matching, aggregates of at most max_agg_size).
    isolated_join: pass 3 of the MIS-2 aggregation (module docstring).
    smoother: "l1jacobi" or "hgs" (hybrid Gauss-Seidel, hybrid_blocks and
    hybrid_gs_sweep; grid = (nx, ny, nz) of the finest level).
    """
    levels = [Level(A)]
    while True:
        lv = levels[-1]
        n = lv.A.shape[0]
        if n < coarse_max or len(levels) >= max_levels:
            break
        if aggregation == "matching":
            S = None
            agg, nc, rounds = matching_aggregate(lv.A, max_agg_size)
        else:
            S = strength(lv.A, theta * 0.5 ** (len(levels) - 1))
            keys = priority_keys(n, seed)
            state, rounds = mis2(S, keys)
            agg, nc = aggregate(S, state, keys, lv.A if isolated_join else None)
        if nc > max_ratio * n:
            break
        Pt = tentative_prolongator(agg, nc)
        P = smoothed_prolongator(lv.A, Pt)[0] if len(levels) - 1 < smooth_levels else Pt
        R = transpose(P)
        Ac = spgemm(R, spgemm(lv.A, P))
        lv.S, lv.agg, lv.P, lv.R, lv.mis_rounds = S, agg, P, R, rounds
        levels.append(Level(Ac))
    h = Hierarchy(levels, _coarse_factor(levels[-1].A))
    h.smoother, h.grid, h.hgs_seg, h.hgs_block = smoother, grid, hgs_seg, hgs_block
    return h


def _coarse_factor(A):
    if A.shape[0] > DENSE_MAX:
        return None  # stalled coarsening: the coarsest level is smoothed, not factored
    return np.linalg.cholesky(A.toarray())


def update_fine(h, A):
    """Replace the finest matrix (and its l1 diagonal); P, R and coarse levels stay frozen.

    This is the paper's reuse scheme (Sec. 6, experimental setup): the
    hierarchy is built once and later Jacobians only update the smoother.
    """
    lv = h.levels[0]
    lv.A = sp.csr_matrix(A)
    lv.dl1 = l1_diagonal(lv.A)
    if len(h.levels) == 1:
        h.chol = _coarse_factor(lv.A)


def refresh(h, A):
    """Keep aggregates, P and R; recompute every coarse matrix A_{l+1} = R_l A_l P_l from the new A.

    The integer part of the setup (strength, MIS-2, aggregates) and all
    sparsity patterns are reused; only values change.
    """
    h.levels[0].A = sp.csr_matrix(A)
    h.levels[0].dl1 = l1_diagonal(h.levels[0].A)
    for l in range(len(h.levels) - 1):
        lv = h.levels[l]
        Ac = spgemm(lv.R, spgemm(lv.A, lv.P))
        h.levels[l + 1].A = Ac
        h.levels[l + 1].dl1 = l1_diagonal(Ac)
    h.chol = _coarse_factor(h.levels[-1].A)


# ---------------------------------------------------------------- hybrid Gauss-Seidel smoother
# The paper's AMG smoother (Sec. 5.2 and the setup of Sec. 6) is one sweep of
# "hybrid" backward/forward Gauss-Seidel as pre/post-smoother: Gauss-Seidel
# within the block of unknowns one process owns, Jacobi between blocks.  Here a
# block is what one GPU thread (or lane group) owns:
#   level 0 (the 7-point grid): a segment of hgs_seg consecutive cells of one
#           vertical column, (i, j, k0 .. k0 + hgs_seg - 1), k0 a multiple of hgs_seg;
#   coarser levels: hgs_block consecutive rows.
# Inside a block the unknowns are visited in increasing (forward) or decreasing
# (backward) index order and use the values already updated in this sweep;
# unknowns of other blocks enter with their values from before the sweep.  The
# scaling is the l1 form of hybrid Gauss-Seidel (Baker, Falgout, Kolev, Yang,
# "Multigrid smoothers for ultraparallel computing", SIAM J. Sci. Comput. 2011):
# a_ii + sum over couplings to other blocks of |a_ij|, which makes every sweep
# convergent for SPD matrices whatever the blocks.  With pre = backward and post =
# forward sweeps the V-cycle stays a symmetric operator.

def hybrid_blocks(n, level, grid=None, seg=16, block=16):
    """(block id, position inside the block) of every node of a level."""
    idx = np.arange(n, dtype=np.int64)
    if level == 0 and grid is not None:
        nx, ny, nz = grid
        plane = nx * ny
        k = idx // plane
        return (idx % plane) + plane * (k // seg), k % seg
    return idx // block, idx % block


def hybrid_gs_sweep(A, b, x, block_id, pos, forward):
    """One hybrid Gauss-Seidel sweep from x (x = None: from zero); returns the new x."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    rows = np.repeat(np.arange(n), np.diff(A.indptr))
    same = block_id[rows] == block_id[A.indices]
    A_in = sp.csr_matrix((np.where(same, A.data, 0.0), A.indices, A.indptr), shape=A.shape)
    A_off = sp.csr_matrix((np.where(same, 0.0, A.data), A.indices, A.indptr), shape=A.shape)
    d = A.diagonal() + np.bincount(rows, weights=np.where(same, 0.0, np.abs(A.data)), minlength=n)
    x_old = np.zeros(n) if x is None else np.asarray(x, dtype=np.float64)
    x_new = x_old.copy()
    positions = range(int(pos.max()) + 1) if n else range(0)
    for t in (positions if forward else reversed(positions)):
        R = np.flatnonzero(pos == t)
        r = b[R] - A_in[R] @ x_new - A_off[R] @ x_old
        x_new[R] = x_new[R] + r / d[R]
    return x_new


def _smooth(h, level, b, x, forward):
    lv = h.levels[level]
    if h.smoother == "hgs":
        bid, pos = hybrid_blocks(lv.A.shape[0], level, h.grid, h.hgs_seg, h.hgs_block)
        return hybrid_gs_sweep(lv.A, b, x, bid, pos, forward)
    if x is None:
        return b / lv.dl1
    return x + (b - lv.A @ x) / lv.dl1


def vcycle(h, b, nu1=1, nu2=1, level=0):
    """One symmetric V-cycle x = B b, zero initial guess (eq. (Vcycle)).

    Pre-smoothing: nu1 l1-Jacobi sweeps, or nu1 backward hybrid Gauss-Seidel
    sweeps; post-smoothing: nu2 sweeps (forward for hybrid Gauss-Seidel)."""
    lv = h.levels[level]
    if level == len(h.levels) - 1:
        if h.chol is not None:
            return sla.cho_solve((h.chol, True), b)
        x = np.zeros_like(b)
        for _ in range(COARSE_SWEEPS):
            x = x + (b - lv.A @ x) / lv.dl1
        return x
    x = None
    for _ in range(nu1):
        x = _smooth(h, level, b, x, forward=False)
    if x is None:
        x = np.zeros_like(b)
    r = b - lv.A @ x
    xc = vcycle(h, lv.R @ r, nu1, nu2, level + 1)
    x = x + lv.P @ xc
    for _ in range(nu2):
        x = _smooth(h, level, b, x, forward=True)
    return x
