"""Pins of the oracle's AMG, Krylov and Newton pieces against brute force, textbook identities and invariants."""
import itertools

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import amg, krylov, newton
from oracle import constitutive as cst
from oracle import discretization as disc
from paper_2112_05051_gb300 import synth

SOIL = synth.Soil()


# ---------------------------------------------------------------- priority generator

def _golden(name):
    import os
    path = os.path.join(os.path.dirname(__file__), "golden", name)
    return [ln.split() for ln in open(path) if ln.strip() and not ln.startswith("#")]


def test_splitmix64_published_vectors():
    # SplitMix64 started from state 0 (Steele, Lea, Flood 2014; Vigna's reference
    # generator): the first outputs are the finaliser at 1x and 2x the golden gamma.
    rows = _golden("splitmix64.txt")
    assert len(rows) == 2
    for x, out in rows:
        assert int(amg.splitmix64(np.uint64(int(x, 16)))) == int(out, 16)
    k = amg.priority_keys(1000, 5)
    assert len(np.unique(k)) == 1000
    assert np.all((k & np.uint64(0xFFFFFFFF)) == np.arange(1000, dtype=np.uint64))


# ---------------------------------------------------------------- MIS-2 and aggregation

def _random_graph(n, p, seed):
    rng = np.random.default_rng(seed)
    m = np.triu(rng.random((n, n)) < p, 1)
    m = m | m.T
    return sp.csr_matrix(m.astype(float))


def _greedy_mis2(S, keys):
    """Sequential greedy distance-2 independent set in decreasing key order (brute force).

    Isolated nodes (no neighbour) are left out, as the aggregation excludes them.
    """
    n = S.shape[0]
    A = (S.toarray() != 0)
    A2 = A | (A.astype(int) @ A.astype(int) > 0)
    np.fill_diagonal(A2, False)
    chosen = np.zeros(n, bool)
    blocked = ~A.any(axis=1)
    for i in sorted(range(n), key=lambda v: int(keys[v]), reverse=True):
        if not blocked[i]:
            chosen[i] = True
            blocked |= A2[i]
            blocked[i] = True
    return chosen


def _grid_graph(nx, ny, nz):
    grid = synth.Grid(nx, ny, nz)
    st = np.zeros((grid.n, 7))
    st[:, 0] = 6.0
    st[:, 1:] = -1.0
    A = disc._stencil_to_csr(grid, st)
    return amg.strength(A, 0.08)


@pytest.mark.parametrize("case", ["rand40", "rand120", "rand200", "grid"])
@pytest.mark.parametrize("seed", [1, 2, 3])
def test_mis2_equals_sequential_greedy(case, seed):
    if case == "grid":
        S = _grid_graph(6, 5, 4)
    else:
        n = int(case[4:])
        S = _random_graph(n, 4.0 / n, seed)
    keys = amg.priority_keys(S.shape[0], seed)
    state, rounds = amg.mis2(S, keys)
    np.testing.assert_array_equal(state == amg.STATE_IN, _greedy_mis2(S, keys))
    assert np.all(state != amg.STATE_UNDECIDED)


def _bfs_dist(A, src):
    n = A.shape[0]
    dist = np.full(n, -1)
    dist[src] = 0
    frontier = [src]
    while frontier:
        nxt = []
        for u in frontier:
            for v in A.indices[A.indptr[u]:A.indptr[u + 1]]:
                if dist[v] < 0:
                    dist[v] = dist[u] + 1
                    nxt.append(v)
        frontier = nxt
    return dist


@pytest.mark.parametrize("case", ["rand150", "grid"])
def test_aggregates_are_partition_with_radius_two(case):
    S = _grid_graph(7, 6, 5) if case == "grid" else _random_graph(150, 0.03, 9)
    keys = amg.priority_keys(S.shape[0], 4)
    state, _ = amg.mis2(S, keys)
    agg, nc = amg.aggregate(S, state, keys)
    roots = np.flatnonzero(state == amg.STATE_IN)
    isolated = np.diff(S.indptr) == 0
    assert nc == len(roots)
    assert np.all(agg[isolated] == -1) and np.all(agg[~isolated] >= 0)
    assert set(agg[~isolated].tolist()) == set(range(nc))
    np.testing.assert_array_equal(agg[roots], np.arange(nc))  # numbered by root index
    for a, r in enumerate(roots):
        members = np.flatnonzero(agg == a)
        sub = S[members][:, members]
        d = _bfs_dist(sp.csr_matrix(sub), int(np.flatnonzero(members == r)[0]))
        assert np.all(d >= 0) and d.max() <= 2          # connected, radius <= 2 from its root
        dfull = _bfs_dist(S, r)
        others = np.setdiff1d(roots, [r])
        assert np.all((dfull[others] < 0) | (dfull[others] >= 3))  # roots pairwise >= 3 apart


# ---------------------------------------------------------------- sparse products and the hierarchy

def test_structural_spgemm_keeps_cancelled_entries():
    A = sp.csr_matrix(np.array([[1.0, 1.0], [0.0, 2.0]]))
    B = sp.csr_matrix(np.array([[1.0, 3.0], [-1.0, 1.0]]))
    C = amg.spgemm(A, B)
    np.testing.assert_array_equal(C.toarray(), A.toarray() @ B.toarray())
    assert C.nnz == 4  # C[0,0] = 1 - 1 = 0 is kept in the pattern
    rng = np.random.default_rng(0)
    for _ in range(5):
        A = sp.random(30, 20, 0.2, random_state=rng, format="csr")
        B = sp.random(20, 25, 0.2, random_state=rng, format="csr")
        C = amg.spgemm(A, B)
        np.testing.assert_allclose(C.toarray(), A.toarray() @ B.toarray(), rtol=1e-14, atol=1e-15)
        pat = (np.abs(A.toarray()) > 0).astype(int) @ (np.abs(B.toarray()) > 0).astype(int) > 0
        assert C.nnz == pat.sum()


def _aux(grid, seed=1, dt=1.0, kmean=synth.KMEAN_ARITH, het=True):
    rng = np.random.default_rng(seed)
    p = rng.uniform(-60, -20, grid.n)
    ks = synth.ks_field(grid, seed, 1.0, (3.0, 3.0, 2.0)) if het else None
    return disc.aux_matrix(grid, SOIL, synth.infiltration_bc(), kmean, p, dt, ks)


def test_prolongator_and_galerkin_product_against_dense_algebra():
    grid = synth.Grid(8, 7, 6)
    A = _aux(grid)
    S = amg.strength(A, 0.08)
    keys = amg.priority_keys(grid.n, 3)
    state, _ = amg.mis2(S, keys)
    agg, nc = amg.aggregate(S, state, keys)
    Pt = amg.tentative_prolongator(agg, nc)
    P, omega = amg.smoothed_prolongator(A, Pt)
    Ad = A.toarray()
    D = np.diag(Ad)
    rho = np.max(np.abs(Ad).sum(1) / np.abs(D))
    assert omega == pytest.approx(4.0 / (3.0 * rho), rel=1e-15)
    Pd = (np.eye(grid.n) - omega * Ad / D[:, None]) @ Pt.toarray()
    np.testing.assert_allclose(P.toarray(), Pd, rtol=1e-13, atol=1e-15)
    Ac = amg.spgemm(amg.transpose(P), amg.spgemm(A, P))
    # Galerkin identity x_c^T A_c y_c = (P x_c)^T A (P y_c)
    rng = np.random.default_rng(5)
    for _ in range(3):
        x, y = rng.standard_normal(nc), rng.standard_normal(nc)
        assert x @ (Ac @ y) == pytest.approx((P @ x) @ (A @ (P @ y)), rel=1e-12)
    Acd = Ac.toarray()
    assert np.abs(Acd - Acd.T).max() <= 1e-13 * np.abs(Acd).max()
    np.linalg.cholesky(Acd)


def test_hierarchy_coarsens_and_vcycle_is_symmetric_positive_contraction():
    grid = synth.Grid(8, 8, 8)
    A = _aux(grid, 2, dt=0.5)
    h = amg.setup(A, theta=0.08, seed=1, coarse_max=100)
    assert len(h.levels) >= 2 and h.sizes[-1] < 100
    assert all(b < a for a, b in zip(h.sizes, h.sizes[1:]))
    n = grid.n
    for nu in (1, 2):
        B = np.column_stack([amg.vcycle(h, e, nu, nu) for e in np.eye(n)])
        assert np.abs(B - B.T).max() <= 1e-12 * np.abs(B).max()      # symmetric V-cycle
        assert np.linalg.eigvalsh(0.5 * (B + B.T)).min() > 0          # SPD
        rho = np.abs(np.linalg.eigvals(np.eye(n) - B @ A.toarray())).max()
        assert rho < 1.0                                             # convergent
    # single-level hierarchy = exact dense solve
    h1 = amg.setup(A, coarse_max=10 ** 6)
    b = np.arange(n, dtype=float)
    np.testing.assert_allclose(A @ amg.vcycle(h1, b), b, rtol=0, atol=1e-10 * np.abs(b).max())


def test_refresh_equals_galerkin_products_of_new_matrix():
    grid = synth.Grid(8, 8, 6)
    A1 = _aux(grid, 3)
    A2 = _aux(grid, 4)
    h = amg.setup(A1, coarse_max=50)
    amg.refresh(h, A2)
    for l in range(len(h.levels) - 1):
        lv = h.levels[l]
        Pd = lv.P.toarray()
        np.testing.assert_allclose(h.levels[l + 1].A.toarray(), Pd.T @ lv.A.toarray() @ Pd, rtol=1e-12,
                                   atol=1e-12 * np.abs(lv.A.data).max())


# ---------------------------------------------------------------- Krylov

def test_fgmres_full_space_is_exact_solve_and_monotone():
    rng = np.random.default_rng(3)
    n = 27
    M = np.eye(n) * 4 + rng.standard_normal((n, n)) * 0.5
    b = rng.standard_normal(n)
    x, its, ok, hist = krylov.fgmres(lambda v: M @ v, lambda v: v, b, 1e-13, 200, n)
    np.testing.assert_allclose(x, np.linalg.solve(M, b), rtol=1e-11, atol=1e-12)
    assert ok and its <= n
    assert all(b2 <= b1 * (1 + 1e-12) for b1, b2 in zip(hist, hist[1:]))
    # restarted with a varying (flexible) preconditioner still converges
    D = np.diag(M)
    k = itertools.count()
    prec = lambda v: v / D * (1.0 + 0.1 * (next(k) % 3))
    x, its, ok, _ = krylov.fgmres(lambda v: M @ v, prec, b, 1e-10, 500, 5)
    assert ok and np.linalg.norm(M @ x - b) <= 1e-10 * np.linalg.norm(b) * 1.01


def test_fgmres_stall_stops_a_stagnating_restart_cycle():
    # The cyclic shift S e_i = e_{i+1 mod n} with b = e_1: the Krylov space K_m(S, b)
    # is spanned by e_2..e_{m+1} after the first vector, all orthogonal to b, so
    # restarted GMRES(m) with m < n makes no progress at all (complete stagnation):
    # the residual stays ||b|| and x stays 0.
    n, m = 8, 3
    S = np.roll(np.eye(n), 1, axis=0)
    b = np.zeros(n)
    b[0] = 1.0
    x, its, ok, hist = krylov.fgmres(lambda v: S @ v, lambda v: v, b, 1e-10, 30, m)
    assert not ok and its == 30 and np.abs(x).max() < 1e-14
    np.testing.assert_allclose(hist, 1.0, atol=1e-14)
    x, its, ok, _ = krylov.fgmres(lambda v: S @ v, lambda v: v, b, 1e-10, 30, m, stall=0.01)
    assert not ok and its == m and np.abs(x).max() < 1e-14  # one cycle, then it gives up
    # a cycle that does reduce the residual by more than the fraction keeps going
    rng = np.random.default_rng(9)
    M = np.eye(30) * 4 + rng.standard_normal((30, 30)) * 0.5
    c = rng.standard_normal(30)
    ref = krylov.fgmres(lambda v: M @ v, lambda v: v, c, 1e-10, 300, 5)
    got = krylov.fgmres(lambda v: M @ v, lambda v: v, c, 1e-10, 300, 5, stall=0.05)
    assert ref[2] and got[2] and ref[1] == got[1]
    np.testing.assert_array_equal(ref[0], got[0])
    # a stall fraction the cycles cannot meet: stops after the first restart
    got = krylov.fgmres(lambda v: M @ v, lambda v: v, c, 1e-10, 300, 5, stall=0.999999)
    assert not got[2] and got[1] == 5


def test_fcg_unpreconditioned_iterates_minimise_energy_error_on_krylov_space():
    # With B = I on an SPD matrix, FCG is CG: x_k minimises the A-norm error over K_k(A, b).
    rng = np.random.default_rng(4)
    n = 40
    Q = np.linalg.qr(rng.standard_normal((n, n)))[0]
    A = Q @ np.diag(np.linspace(1, 20, n)) @ Q.T
    b = rng.standard_normal(n)
    for k in range(1, 6):
        xk, its, _, _ = krylov.fcg(lambda v: A @ v, lambda v: v, b, 1e-300, k)
        Kb = np.column_stack([np.linalg.matrix_power(A, j) @ b for j in range(k)])
        V = np.linalg.qr(Kb)[0]
        xopt = V @ np.linalg.solve(V.T @ A @ V, V.T @ b)
        np.testing.assert_allclose(xk, xopt, rtol=1e-9, atol=1e-12)
    x, its, ok, _ = krylov.fcg(lambda v: A @ v, lambda v: v, b, 1e-12, 200)
    assert ok
    np.testing.assert_allclose(x, np.linalg.solve(A, b), rtol=1e-10)


# ---------------------------------------------------------------- Newton-Armijo

def test_hydrostatic_state_needs_no_newton_iteration():
    grid = synth.Grid(4, 4, 6)
    hz = grid.h[2]
    z = (np.arange(grid.nz) + 1) * hz
    p = np.broadcast_to((-12.0 - z)[:, None, None], grid.shape).ravel().copy()
    bc = synth.BC(kind=(0, 0, 0, 0, 0, 1), value=(0, 0, 0, 0, 0, -12.0 - (grid.nz + 1) * hz))
    prob = newton.Problem(grid, SOIL, bc, synth.KMEAN_ARITH)
    # a converged state: the initial residual is round-off, so use an absolute tolerance
    p1, st = newton.step(prob, p, 1.0, newton.NewtonOptions(rtol=0.0, atol=1e-12))
    assert st.newton_its == 0 and st.converged
    np.testing.assert_array_equal(p1, p)


@pytest.mark.parametrize("kmean", [synth.KMEAN_ARITH, synth.KMEAN_UPSTREAM, synth.KMEAN_HARMONIC])
def test_newton_step_converges_quadratically_and_conserves_mass(kmean):
    grid = synth.Grid(6, 6, 8)
    ks = synth.ks_field(grid, 1, 1.0, (3.0, 3.0, 2.0))
    bc = synth.infiltration_bc()
    prob = newton.Problem(grid, SOIL, bc, kmean, ks)
    # a milder initial jump than the workloads' (-61.5 under a -20.7 top): with the
    # harmonic mean a 40 cm jump across one cell makes the boundary rows of J
    # indefinite and the diffusion-only preconditioner needs hundreds of iterations
    p0 = np.full(grid.n, -25.0)
    opt = newton.NewtonOptions(krylov="fgmres", eta=1e-12, rtol=1e-12, coarse_max=50)
    p1, st = newton.step(prob, p0, 5.0, opt)
    assert st.converged
    F = prob.residual(p1, cst.saturation(p0, SOIL), 5.0)
    assert np.linalg.norm(F) <= 1e-12 * st.res0 * 1.0001
    r = st.res_hist
    # local quadratic convergence once the full step is taken
    full = [i for i, lam in enumerate(st.lambdas) if lam == 1.0]
    ratios = [r[i + 1] / r[i] ** 2 for i in full if r[i] < 1e-2 * r[0] and r[i + 1] > 1e-14 * r[0]]
    assert all(q < 1e3 for q in ratios)
    # mass balance: storage change = inflow through the Dirichlet top face, up to ||Phi||_1.
    # The top-face flux is isolated as Phi(p1) minus Phi(p1) with that face closed.
    s0 = cst.saturation(p0, SOIL)
    closed = disc.residual(grid, SOIL, synth.all_noflux_bc(), kmean, p1, s0, 5.0, ks)
    top_flux = (F - closed).sum()
    storage = SOIL.rho_phi * (cst.saturation(p1, SOIL) - s0).sum() / 5.0
    assert storage > 0 and top_flux < 0   # wetting from the top
    assert abs(storage + top_flux) <= np.abs(F).sum() + 1e-12 * storage


def test_converged_pressure_is_independent_of_solver_choices():
    grid = synth.Grid(6, 5, 7)
    bc = synth.infiltration_bc()
    p0 = np.full(grid.n, synth.P_INITIAL)
    res = []
    for kry, pol, nu in (("fcg", "refresh", 1), ("fgmres", "setup_once", 2), ("fgmres", "rebuild_step", 1)):
        prob = newton.Problem(grid, SOIL, bc, synth.KMEAN_UPSTREAM)
        opt = newton.NewtonOptions(krylov=kry, amg_policy=pol, nu1=nu, nu2=nu, coarse_max=40, rtol=1e-10)
        p = p0
        for dt in (1.0, 2.0):
            p, st = newton.step(prob, p, dt, opt)
            assert st.converged
        res.append(p)
    for q in res[1:]:
        np.testing.assert_allclose(q, res[0], rtol=1e-8)


# ---------------------------------------------------------------- matching aggregation

def _random_spd_graph(n, p, seed, levels=4):
    """Symmetric M-matrix on a random graph with few distinct coupling values (many tied weights)."""
    rng = np.random.default_rng(seed)
    m = np.triu(rng.random((n, n)) < p, 1)
    vals = -rng.integers(1, levels + 1, size=(n, n)).astype(float)
    off = np.where(m, vals, 0.0)
    off = off + off.T
    d = -off.sum(axis=1) + 1.0
    return sp.csr_matrix(off + np.diag(d))


def test_compatible_weight_of_a_two_node_laplacian():
    # w = 1 - (a_12 + a_21)/(a_11 + a_22) = 1 - (-2)/4 = 1.5 for [[2, -1], [-1, 2]]
    rows, cols, w = amg.matching_weights(sp.csr_matrix(np.array([[2.0, -1.0], [-1.0, 2.0]])))
    off = rows != cols
    assert np.all(w[off] == np.float32(1.5)) and np.all(np.isneginf(w[~off]))
    # positive couplings are not edges
    _, _, w2 = amg.matching_weights(sp.csr_matrix(np.array([[2.0, 0.5], [0.5, 2.0]])))
    assert np.all(np.isneginf(w2))


@pytest.mark.parametrize("seed", [1, 2, 3, 4])
@pytest.mark.parametrize("n,p", [(30, 0.15), (80, 0.05), (150, 0.03)])
def test_locally_dominant_matching_equals_sequential_greedy(n, p, seed):
    A = _random_spd_graph(n, p, seed)
    mate, rounds = amg.match(A)
    assert np.array_equal(mate, amg.greedy_matching(A))
    # a valid, maximal matching of the negative couplings
    m = np.flatnonzero(mate >= 0)
    assert np.all(mate[mate[m]] == m) and np.all(mate[m] != m)
    D = A.toarray()
    assert np.all(D[m, mate[m]] < 0)
    free = mate < 0
    assert not np.any((D[np.ix_(free, free)] < 0) & ~np.eye(int(free.sum()), dtype=bool))


def test_matching_on_the_grid_laplacian_pairs_every_node_along_x():
    # equal weights everywhere: ties go to the smallest index pair, so the greedy
    # order pairs (0,1), (2,3), ... along x on an even grid
    grid = synth.Grid(6, 4, 3)
    st = np.zeros((grid.n, 7))
    st[:, 0] = 6.0
    st[:, 1:] = -1.0
    A = disc._stencil_to_csr(grid, st)
    mate, _ = amg.match(A)
    idx = np.arange(grid.n)
    assert np.array_equal(mate, idx ^ 1)


@pytest.mark.parametrize("max_size", [2, 4, 8])
def test_matching_aggregates_partition_with_bounded_size(max_size):
    grid = synth.Grid(14, 12, 10)
    ks = synth.ks_field(grid, 5, 1.0, (4.0, 4.0, 2.0))
    A = disc.aux_matrix(grid, SOIL, synth.infiltration_bc(), 0, np.full(grid.n, -40.0), 1.0, ks)
    agg, nc, rounds = amg.matching_aggregate(A, max_size)
    assert agg.min() == 0 and agg.max() == nc - 1
    sizes = np.bincount(agg, minlength=nc)
    assert sizes.min() >= 1 and sizes.max() <= max_size
    assert nc < grid.n / (0.6 * max_size)  # most nodes are matched at every pass
    # every aggregate is connected through negative couplings
    G = (A < 0).astype(int)
    for a in np.unique(agg)[:200]:
        nodes = np.flatnonzero(agg == a)
        if len(nodes) > 1:
            sub = G[nodes][:, nodes]
            ncomp, _ = sp.csgraph.connected_components(sub, directed=False)
            assert ncomp == 1


def test_matching_hierarchy_gives_a_convergent_vcycle():
    grid = synth.Grid(20, 18, 16)
    ks = synth.ks_field(grid, 7, 1.5, (4.0, 4.0, 2.0))
    A = disc.aux_matrix(grid, SOIL, synth.infiltration_bc(), 1, np.full(grid.n, -50.0), 1.0, ks)
    h = amg.setup(A, 0.08, 1, 100, smooth_levels=2, aggregation="matching")
    assert len(h.levels) >= 3
    b = np.random.default_rng(2).standard_normal(grid.n)
    x, its, ok, _ = krylov.fgmres(lambda v: A @ v, lambda v: amg.vcycle(h, v), b, 1e-10, 100, 30)
    assert ok and its < 40


# ---------------------------------------------------------------- the pins catch planted mistakes

def test_pins_catch_an_mis2_that_takes_the_smallest_key(monkeypatch):
    monkeypatch.setattr(amg, "_max_closed", lambda Sc, v: np.minimum.reduceat(v[Sc.indices], Sc.indptr[:-1]))
    with pytest.raises(AssertionError):
        test_mis2_equals_sequential_greedy("rand40", 1)


def test_pins_catch_an_unsymmetrised_compatible_weight(monkeypatch):
    def bad(A):
        A = sp.csr_matrix(A)
        n = A.shape[0]
        rows = np.repeat(np.arange(n), np.diff(A.indptr))
        cols = A.indices
        d = A.diagonal()
        edge = (cols != rows) & (A.data < 0)
        w = np.full(len(cols), -np.inf, dtype=np.float32)
        w[edge] = (1.0 - A.data[edge] / (d[rows[edge]] + d[cols[edge]])).astype(np.float32)  # a_ij only
        return rows, cols, w
    monkeypatch.setattr(amg, "matching_weights", bad)
    with pytest.raises(AssertionError):
        test_compatible_weight_of_a_two_node_laplacian()


def test_pins_catch_a_wrong_smoothing_weight(monkeypatch):
    orig = amg.smoothed_prolongator

    def bad(A, Pt):  # omega = 2 / (3 rho) instead of 4 / (3 rho)
        A = sp.csr_matrix(A)
        n = A.shape[0]
        d = A.diagonal()
        rows = np.repeat(np.arange(n), np.diff(A.indptr))
        rho = np.max(np.bincount(rows, weights=np.abs(A.data), minlength=n) / np.abs(d))
        omega = 2.0 / (3.0 * rho)
        vals = -omega * A.data / d[rows] + (A.indices == rows)
        return amg.spgemm(sp.csr_matrix((vals, A.indices.copy(), A.indptr.copy()), shape=A.shape), Pt), omega
    monkeypatch.setattr(amg, "smoothed_prolongator", bad)
    with pytest.raises(AssertionError):
        test_prolongator_and_galerkin_product_against_dense_algebra()


def test_pins_catch_a_vcycle_without_post_smoothing(monkeypatch):
    orig = amg.vcycle
    monkeypatch.setattr(amg, "vcycle", lambda h, b, nu1=1, nu2=1, level=0: orig(h, b, nu1, 0, level))
    with pytest.raises(AssertionError):
        test_hierarchy_coarsens_and_vcycle_is_symmetric_positive_contraction()


# ---------------------------------------------------------------- hybrid Gauss-Seidel smoother (Sec. 5.2, Sec. 6)

def _hgs_loop(A, b, x, block_id, pos, forward):
    """The definition, one unknown at a time: blocks in any order, inside a block by
    position, new values inside the block, values from before the sweep outside."""
    A = sp.csr_matrix(A)
    n = A.shape[0]
    x0 = np.zeros(n) if x is None else np.array(x, dtype=float)
    x1 = x0.copy()
    for blk in np.unique(block_id):
        members = np.flatnonzero(block_id == blk)
        members = members[np.argsort(pos[members])]
        if not forward:
            members = members[::-1]
        for i in members:
            s, d = b[i], 0.0
            for e in range(A.indptr[i], A.indptr[i + 1]):
                j, a = A.indices[e], A.data[e]
                if j == i:
                    d += a
                if block_id[j] == block_id[i]:
                    s -= a * x1[j]
                else:
                    s -= a * x0[j]
                    d += abs(a)
            x1[i] = x1[i] + s / d
    return x1


def test_hybrid_gs_with_one_block_is_textbook_gauss_seidel():
    import scipy.sparse.linalg as spla
    A = _aux(synth.Grid(6, 5, 4))
    n = A.shape[0]
    rng = np.random.default_rng(3)
    b, x = rng.standard_normal(n), rng.standard_normal(n)
    one = np.zeros(n, dtype=np.int64)
    pos = np.arange(n)
    fwd = amg.hybrid_gs_sweep(A, b, x, one, pos, True)
    L = sp.tril(A, 0, format="csr")
    np.testing.assert_allclose(fwd, x + spla.spsolve_triangular(L, b - A @ x, lower=True), rtol=1e-12, atol=1e-12)
    bwd = amg.hybrid_gs_sweep(A, b, x, one, pos, False)
    U = sp.triu(A, 0, format="csr")
    np.testing.assert_allclose(bwd, x + spla.spsolve_triangular(U, b - A @ x, lower=False), rtol=1e-12, atol=1e-12)


def test_hybrid_gs_with_singleton_blocks_is_l1_jacobi():
    A = _aux(synth.Grid(5, 5, 5))
    n = A.shape[0]
    rng = np.random.default_rng(4)
    b, x = rng.standard_normal(n), rng.standard_normal(n)
    y = amg.hybrid_gs_sweep(A, b, x, np.arange(n), np.zeros(n, dtype=np.int64), True)
    np.testing.assert_allclose(y, x + (b - A @ x) / amg.l1_diagonal(A), rtol=1e-13)


@pytest.mark.parametrize("forward", [True, False])
def test_hybrid_gs_sweep_equals_its_one_unknown_at_a_time_definition(forward):
    grid = synth.Grid(5, 4, 7)
    A = _aux(grid)
    rng = np.random.default_rng(8)
    b, x = rng.standard_normal(grid.n), rng.standard_normal(grid.n)
    for level, seg in ((0, 3), (1, 5)):  # column segments of 3 cells; blocks of 5 rows
        bid, pos = amg.hybrid_blocks(grid.n, level, (grid.nx, grid.ny, grid.nz), seg=seg, block=seg)
        np.testing.assert_allclose(amg.hybrid_gs_sweep(A, b, x, bid, pos, forward),
                                   _hgs_loop(A, b, x, bid, pos, forward), rtol=1e-12, atol=1e-14)
        np.testing.assert_allclose(amg.hybrid_gs_sweep(A, b, None, bid, pos, forward),
                                   _hgs_loop(A, b, None, bid, pos, forward), rtol=1e-12, atol=1e-14)
    # column segments: a block is (i, j) fixed, k in [k0, k0 + seg)
    bid, pos = amg.hybrid_blocks(grid.n, 0, (grid.nx, grid.ny, grid.nz), seg=3)
    c = np.arange(grid.n)
    assert np.all(pos == (c // (grid.nx * grid.ny)) % 3)
    assert len(np.unique(bid)) == grid.nx * grid.ny * 3


def _hgs_hierarchy(grid, A, seg=4, block=6):
    return amg.setup(A, coarse_max=40, smoother="hgs", grid=(grid.nx, grid.ny, grid.nz), hgs_seg=seg,
                     hgs_block=block)


def test_hybrid_gs_vcycle_is_symmetric_positive_and_beats_l1_jacobi():
    grid = synth.Grid(14, 12, 16)
    A = _aux(grid)
    h = _hgs_hierarchy(grid, A)
    assert len(h.levels) >= 3
    n = grid.n
    rng = np.random.default_rng(1)
    x, y = rng.standard_normal(n), rng.standard_normal(n)
    assert abs(x @ amg.vcycle(h, y) - y @ amg.vcycle(h, x)) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(y) * 10
    assert y @ amg.vcycle(h, y) > 0
    b = rng.standard_normal(n)
    _, its_g, ok_g, _ = krylov.fcg(lambda v: A @ v, lambda v: amg.vcycle(h, v), b, 1e-10, 200)
    hj = amg.setup(A, coarse_max=40)
    _, its_j, ok_j, _ = krylov.fcg(lambda v: A @ v, lambda v: amg.vcycle(hj, v), b, 1e-10, 200)
    assert ok_g and ok_j and its_g < its_j


def test_pins_catch_a_forward_pre_smoother(monkeypatch):
    orig = amg._smooth
    monkeypatch.setattr(amg, "_smooth", lambda h, level, b, x, forward: orig(h, level, b, x, True))
    with pytest.raises(AssertionError):
        test_hybrid_gs_vcycle_is_symmetric_positive_and_beats_l1_jacobi()


def test_fcg_stall_window():
    # CG on an SPD matrix with eigenvalues spread over [1, 1e4] and no preconditioner
    # reduces the residual slowly; a stall fraction a 30-iteration window cannot meet
    # stops it at iteration 30 with reason "stall", and the iterate is the plain
    # run's iterate 30 (the test only ends the loop).
    rng = np.random.default_rng(12)
    n = 200
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    M = (Q * np.logspace(0, 4, n)) @ Q.T
    b = rng.standard_normal(n)
    ref30 = krylov.fcg(lambda v: M @ v, lambda v: v, b, 1e-14, 30)
    info = {}
    x, its, ok, hist = krylov.fcg(lambda v: M @ v, lambda v: v, b, 1e-14, 500, info=info, stall=0.999)
    assert not ok and its == 30 and info["reason"] == "stall" and hist[30] > 1e-3 * hist[0]
    np.testing.assert_array_equal(x, ref30[0])
    info = {}
    x2, its2, ok2, _ = krylov.fcg(lambda v: M @ v, lambda v: v, b, 1e-14, 500, info=info, stall=0.0)
    assert its2 > 30
