"""GPU parity of the AMG hierarchy, V-cycle, Krylov solves and the Newton step against the FP64 oracle.

Bars: aggregates, level sizes and sparsity patterns bit-exact; FP64 matrix
values normwise 1e-10; FP64 V-cycle output normwise 1e-10; pressure after a
converged step 1e-8 relative.  MIXED precision: the V-cycle is compared at
FP32 level (normwise 1e-4) and the converged pressure still to 1e-8 (the
Newton residual and outer Krylov are FP64).
"""
import numpy as np
import pytest

from oracle import amg, newton
from oracle import constitutive as cst
from oracle import discretization as disc
from paper_2112_05051_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SOIL = synth.Soil()


def _rb():
    from paper_2112_05051_gb300 import richards as rb
    rb.load()
    return rb


def _nrel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


def _problem(dims, seed, kmean=0, het=True, dt=1.0, bc=None):
    grid = synth.Grid(*dims)
    rng = np.random.default_rng(seed)
    # a smooth wetting front below the top face plus small noise (a state the
    # Newton iteration meets); independent random heads per cell make J far
    # from symmetric and FCG inapplicable
    z = (np.arange(grid.nz) + 1.0) / (grid.nz + 1)
    front = -61.5 + 40.8 * np.exp(-(1.0 - z) / 0.2)
    p = np.broadcast_to(front[:, None, None], grid.shape).ravel() + rng.uniform(-0.5, 0.5, grid.n)
    ks = synth.ks_field(grid, seed, 1.0, (3.0, 3.0, 2.0)) if het else None
    bc = bc or synth.infiltration_bc()
    return grid, p, ks, bc, dt, kmean


def _setup_both(grid, p, ks, bc, dt, kmean, coarse_max, seed=7, prec=0, lists=1, aggregation=0, smooth_levels=10):
    rb = _rb()
    ctx = rb.Context(grid, SOIL, bc, kmean, ks, precision=prec)
    pd = torch.tensor(p, device="cuda")
    ctx.jacobian(pd, dt)
    info = ctx.amg_setup(rb.default_amg_opts(seed=seed, coarse_max=coarse_max, product_lists=lists,
                                             aggregation=aggregation, smooth_levels=smooth_levels))
    A = disc.aux_matrix(grid, SOIL, bc, kmean, p, dt, ks)
    h = amg.setup(A, 0.08, seed, coarse_max, smooth_levels=smooth_levels,
                  aggregation="matching" if aggregation else "mis2")
    return ctx, info, h


def _compare_hierarchy(ctx, info, h):
    assert info.levels == len(h.levels)
    for l, lv in enumerate(h.levels):
        assert info.n[l] == lv.A.shape[0]
        agg, rp, col, val = ctx.export_level(l, info)
        np.testing.assert_array_equal(rp, lv.A.indptr)
        np.testing.assert_array_equal(col, lv.A.indices)
        assert _nrel(val, lv.A.data) <= 1e-10
        if l < info.levels - 1:
            np.testing.assert_array_equal(agg, lv.agg)
            prp, pcol, pval = ctx.export_prolongator(l, info)
            np.testing.assert_array_equal(prp, lv.P.indptr)
            np.testing.assert_array_equal(pcol, lv.P.indices)
            assert _nrel(pval, lv.P.data) <= 1e-10
            assert info.mis_rounds[l] == lv.mis_rounds


@pytest.mark.parametrize("dims,coarse_max,kmean", [((10, 9, 8), 60, 0), ((24, 24, 24), 300, 1),
                                                    ((33, 17, 9), 150, 2), ((1, 1, 50), 5, 0),
                                                    ((40, 40, 40), 2000, 1)])
def test_hierarchy_bit_exact(dims, coarse_max, kmean):
    grid, p, ks, bc, dt, _ = _problem(dims, 3, kmean)
    ctx, info, h = _setup_both(grid, p, ks, bc, dt, kmean, coarse_max)
    _compare_hierarchy(ctx, info, h)
    assert info.operator_complexity == pytest.approx(h.operator_complexity(), rel=1e-12)
    ctx.close()


@pytest.mark.parametrize("join", [1, 0])
def test_hierarchy_with_isolated_nodes_from_extreme_heterogeneity(join):
    # log10 Ks with std 2 spans ~16 decades: many cells have no strong coupling.
    # join=1 (pass 3): those whose row is not diagonally dominant join the aggregate of
    # their strongest aggregated neighbour; the dominant rows under the Dirichlet top
    # (and, with join=0, all of them) stay out of every aggregate (empty P_tent rows)
    rb = _rb()
    grid = synth.Grid(26, 24, 22)
    ks = synth.ks_field(grid, 4, 2.0, (4.0, 4.0, 2.0))
    p = np.full(grid.n, -40.0)
    bc = synth.infiltration_bc()
    ctx = rb.Context(grid, SOIL, bc, 0, ks)
    ctx.jacobian(torch.tensor(p, device="cuda"), 10.0)
    info = ctx.amg_setup(rb.default_amg_opts(seed=4, coarse_max=200, isolated_join=join))
    A = disc.aux_matrix(grid, SOIL, bc, 0, p, 10.0, ks)
    h = amg.setup(A, 0.08, 4, 200, isolated_join=bool(join))
    assert np.any(h.levels[0].agg < 0)
    if join:
        h0 = amg.setup(A, 0.08, 4, 200, isolated_join=False)
        assert np.sum(h.levels[0].agg < 0) < np.sum(h0.levels[0].agg < 0)
    _compare_hierarchy(ctx, info, h)
    r = np.random.default_rng(3).standard_normal(grid.n)
    z = torch.empty(grid.n, dtype=torch.float64, device="cuda")
    ctx.vcycle(torch.tensor(r, device="cuda"), z)
    assert _nrel(z.cpu().numpy(), amg.vcycle(h, r)) <= 1e-10
    ctx.close()


def test_stalled_coarsening_smooths_the_coarsest_level():
    # a single 9600-unknown level exceeds the dense limit: the coarse "solve" is
    # l1-Jacobi sweeps on both sides
    rb = _rb()
    grid, p, ks, bc, dt, kmean = _problem((24, 20, 20), 9, 0)
    ctx = rb.Context(grid, SOIL, bc, kmean, ks)
    ctx.jacobian(torch.tensor(p, device="cuda"), dt)
    info = ctx.amg_setup(rb.default_amg_opts(seed=2, max_levels=1))
    assert info.levels == 1 and info.n[0] > amg.DENSE_MAX
    h = amg.setup(disc.aux_matrix(grid, SOIL, bc, kmean, p, dt, ks), 0.08, 2, 2000, max_levels=1)
    assert h.chol is None
    r = np.random.default_rng(8).standard_normal(grid.n)
    z = torch.empty(grid.n, dtype=torch.float64, device="cuda")
    ctx.vcycle(torch.tensor(r, device="cuda"), z)
    assert _nrel(z.cpu().numpy(), amg.vcycle(h, r)) <= 1e-10
    ctx.close()


def test_hierarchy_with_unsmoothed_deep_levels():
    rb = _rb()
    grid, p, ks, bc, dt, _ = _problem((30, 28, 26), 6, 1)
    ctx = rb.Context(grid, SOIL, bc, 1, ks)
    ctx.jacobian(torch.tensor(p, device="cuda"), dt)
    info = ctx.amg_setup(rb.default_amg_opts(seed=5, coarse_max=100, smooth_levels=1))
    h = amg.setup(disc.aux_matrix(grid, SOIL, bc, 1, p, dt, ks), 0.08, 5, 100, smooth_levels=1)
    _compare_hierarchy(ctx, info, h)
    assert info.levels >= 3
    ctx.close()


@pytest.mark.parametrize("nu", [1, 2])
def test_vcycle_parity_fp64_and_mixed(nu):
    rb = _rb()
    grid, p, ks, bc, dt, kmean = _problem((20, 18, 16), 5, 1)
    r = np.random.default_rng(2).standard_normal(grid.n)
    A = disc.aux_matrix(grid, SOIL, bc, kmean, p, dt, ks)
    h = amg.setup(A, 0.08, 7, 200)
    zref = amg.vcycle(h, r, nu, nu)
    for prec, tol in ((0, 1e-10), (1, 1e-4)):
        ctx = rb.Context(grid, SOIL, bc, kmean, ks, precision=prec)
        ctx.jacobian(torch.tensor(p, device="cuda"), dt)
        ctx.amg_setup(rb.default_amg_opts(seed=7, coarse_max=200, nu1=nu, nu2=nu))
        z = torch.empty(grid.n, dtype=torch.float64, device="cuda")
        ctx.vcycle(torch.tensor(r, device="cuda"), z)
        assert _nrel(z.cpu().numpy(), zref) <= tol
        ctx.close()


@pytest.mark.parametrize("layout", ["csr", "sell", "sell8", "sell2", "sellp", "auto"])
def test_vcycle_parity_per_row_layout_after_refresh(layout):
    """The coarse-level row operations on CSR, on the SELL-C-sigma copies (P_0 with
    84k rows, R_0 and A_1 with a few thousand; ragged last slices and windows), and
    as the autotuner picks: one V-cycle after the setup and after a Galerkin refresh
    (the copies of A are refilled), FP64 and MIXED, against the oracle."""
    rb = _rb()
    lay = {"csr": rb.LAYOUT_CSR, "sell": rb.LAYOUT_SELL, "sell8": rb.LAYOUT_SELL8, "sell2": rb.LAYOUT_SELL2,
           "sellp": rb.LAYOUT_SELLP, "auto": rb.LAYOUT_AUTO}[layout]
    grid, p, ks, bc, dt, kmean = _problem((48, 44, 40), 9, 1)
    p2 = p + np.random.default_rng(6).uniform(0, 10, grid.n)
    r = np.random.default_rng(3).standard_normal(grid.n)
    h = amg.setup(disc.aux_matrix(grid, SOIL, bc, kmean, p, dt, ks), 0.08, 5, 100)
    z1 = amg.vcycle(h, r, 2, 2)
    amg.refresh(h, disc.aux_matrix(grid, SOIL, bc, kmean, p2, dt, ks))
    z2 = amg.vcycle(h, r, 2, 2)
    for prec, tol in ((0, 1e-10), (1, 1e-4)):
        ctx = rb.Context(grid, SOIL, bc, kmean, ks, precision=prec)
        ctx.jacobian(torch.tensor(p, device="cuda"), dt)
        info = ctx.amg_setup(rb.default_amg_opts(seed=5, coarse_max=100, nu1=2, nu2=2, csr_layout=lay))
        assert info.levels >= 3 and info.n[1] >= 2048  # A_1 has a SELL copy
        z = torch.empty(grid.n, dtype=torch.float64, device="cuda")
        ctx.vcycle(torch.tensor(r, device="cuda"), z)
        assert _nrel(z.cpu().numpy(), z1) <= tol
        ctx.jacobian(torch.tensor(p2, device="cuda"), dt)
        ctx.amg_update(rb.AMG_REFRESH)
        ctx.vcycle(torch.tensor(r, device="cuda"), z)
        assert _nrel(z.cpu().numpy(), z2) <= tol
        ctx.close()
    if layout == "auto":  # SELL copies were offered to the tuner
        assert any(e[4] == 1 for e in rb.autotune_table())


@pytest.mark.parametrize("prec", [0, 1])
@pytest.mark.parametrize("layout", ["auto", "sell"])
def test_vcycle_graph_replays_are_bit_identical_to_direct_launches(prec, layout):
    """rich_amg_opts.graph: the first V-cycle launches directly, the second is
    captured, the later ones replay the graph.  On one hierarchy the three give
    the same result bit for bit; two contexts, graph on and off, agree bit for bit
    (a setup is deterministic: rows of the symbolic Galerkin product that took
    the hash kernel are re-summed in the product lists' order), before and after
    a Galerkin refresh, with the same kernel count."""
    rb = _rb()
    lay = {"auto": rb.LAYOUT_AUTO, "sell": rb.LAYOUT_SELL}[layout]
    grid, p, ks, bc, dt, kmean = _problem((40, 36, 32), 9, 1)
    p2 = p + np.random.default_rng(6).uniform(0, 10, grid.n)
    rs = [torch.tensor(np.random.default_rng(20 + k).standard_normal(grid.n), device="cuda") for k in range(4)]
    out, launches = {}, {}
    for graph in (0, 1):
        ctx = rb.Context(grid, SOIL, bc, kmean, ks, precision=prec)
        ctx.jacobian(torch.tensor(p, device="cuda"), dt)
        ctx.amg_setup(rb.default_amg_opts(seed=5, coarse_max=100, nu1=2, nu2=2, csr_layout=lay, graph=graph))
        z = torch.empty(grid.n, dtype=torch.float64, device="cuda")
        first = []
        for _ in range(3):  # graph = 1: direct, captured and replayed, replayed
            ctx.vcycle(rs[0], z)
            first.append(z.cpu().numpy())
        for a in first[1:]:
            np.testing.assert_array_equal(a, first[0])
        out[("setup", graph)] = first[0]
        ctx.jacobian(torch.tensor(p2, device="cuda"), dt)
        ctx.amg_update(rb.AMG_REFRESH)
        torch.cuda.synchronize()
        l0 = ctx_launches(rb)
        zs = []
        for r in rs:
            ctx.vcycle(r, z)
            zs.append(z.cpu().numpy())
        out[graph], launches[graph] = zs, ctx_launches(rb) - l0
        ctx.close()
    np.testing.assert_array_equal(out[("setup", 0)], out[("setup", 1)])
    for a, b in zip(out[0], out[1]):
        np.testing.assert_array_equal(a, b)
    assert launches[0] == launches[1] > 0


@pytest.mark.parametrize("prec", [0, 1])
def test_fcg_iteration_graphs_are_bit_identical_to_direct_launches(prec):
    """FCG's iterations from the second on replay a graph per parity of the
    iteration (rich_amg_opts.graph): a solve and a Newton step with graphs on and
    off agree bit for bit, iterations and results."""
    rb = _rb()
    grid, p, ks, bc, dt, kmean = _problem((24, 22, 20), 4, 1)
    b = torch.tensor(np.random.default_rng(8).standard_normal(grid.n), device="cuda")
    res = {}
    for graph in (0, 1):
        ctx = rb.Context(grid, SOIL, bc, kmean, ks, precision=prec)
        ctx.jacobian(torch.tensor(p, device="cuda"), dt)
        ctx.amg_setup(rb.default_amg_opts(seed=3, coarse_max=100, graph=graph))
        x = torch.empty_like(b)
        xs, its = [], []
        for _ in range(2):  # the second solve replays what the first captured
            s, st = ctx.krylov_solve(b, x, kind=rb.KRYLOV_FCG, eta=1e-10, maxit=300)
            xs.append(x.cpu().numpy())
            its.append(st.iterations)
        ctx.close()
        ctx = rb.Context(grid, SOIL, synth.infiltration_bc(), synth.KMEAN_ARITH, synth.ks_field(grid, 2, 0.5),
                         precision=prec)
        pd = torch.tensor(np.full(grid.n, synth.P_INITIAL), device="cuda")
        st = ctx.step(pd, 0.5, rb.default_newton_opts(kind=rb.KRYLOV_FCG, seed=3, coarse_max=100, graph=graph))
        ctx.close()
        res[graph] = (xs, its, pd.cpu().numpy(), st.newton_its, st.linear_its)
    assert res[0][1] == res[1][1] and res[0][1][0] > 2
    for a, c in zip(res[0][0], res[1][0]):
        np.testing.assert_array_equal(a, c)
    np.testing.assert_array_equal(res[0][2], res[1][2])
    assert res[0][3:] == res[1][3:]


def ctx_launches(rb):
    import ctypes
    v = ctypes.c_longlong()
    rb.load().rich_kernel_launches(ctypes.byref(v))
    return v.value


@pytest.mark.parametrize("lists", [1, 0])
@pytest.mark.parametrize("dims,coarse_max", [((18, 16, 14), 150), ((40, 36, 32), 2000)])
def test_refresh_matches_oracle_galerkin_refresh(dims, coarse_max, lists):
    # lists=1: summed product lists; lists=0: the searching kernels (the larger
    # grid has coarse rows with > 64 and > 1024 products: warp and block kernels)
    rb = _rb()
    grid, p, ks, bc, dt, kmean = _problem(dims, 8, 0)
    p2 = p + np.random.default_rng(4).uniform(0, 15, grid.n)
    ctx, info, h = _setup_both(grid, p, ks, bc, dt, kmean, coarse_max, lists=lists)
    for k in range(2):  # the second refresh reuses the lists the first one built
        pk = p2 + 3.0 * k
        ctx.jacobian(torch.tensor(pk, device="cuda"), 2.0 * dt)
        ctx.amg_update(rb.AMG_REFRESH)
        amg.refresh(h, disc.aux_matrix(grid, SOIL, bc, kmean, pk, 2.0 * dt, ks))
        _compare_hierarchy(ctx, info, h)
    r = np.random.default_rng(1).standard_normal(grid.n)
    z = torch.empty(grid.n, dtype=torch.float64, device="cuda")
    ctx.vcycle(torch.tensor(r, device="cuda"), z)
    assert _nrel(z.cpu().numpy(), amg.vcycle(h, r)) <= 1e-10
    ctx.close()


@pytest.mark.parametrize("dims,coarse_max", [((18, 16, 14), 150), ((40, 36, 32), 2000)])
@pytest.mark.parametrize("lists", [1, 0])
def test_mixed_precision_refresh_runs_galerkin_in_fp32(dims, coarse_max, lists):
    # MIXED: the refreshed coarse operators are FP32 products of the FP32 fine
    # matrix and prolongators; they agree with the FP64 oracle to FP32 rounding
    rb = _rb()
    grid, p, ks, bc, dt, kmean = _problem(dims, 8, 0)
    p2 = p + np.random.default_rng(4).uniform(0, 15, grid.n)
    ctx, info, h = _setup_both(grid, p, ks, bc, dt, kmean, coarse_max, prec=1, lists=lists)
    ctx.jacobian(torch.tensor(p2, device="cuda"), 2.0 * dt)
    ctx.amg_update(rb.AMG_REFRESH)
    amg.refresh(h, disc.aux_matrix(grid, SOIL, bc, kmean, p2, 2.0 * dt, ks))
    for l, lv in enumerate(h.levels):
        _, rp, col, val = ctx.export_level(l, info)
        np.testing.assert_array_equal(rp, lv.A.indptr)
        np.testing.assert_array_equal(col, lv.A.indices)
        assert _nrel(val, lv.A.data) <= (1e-10 if l == 0 else 1e-5)
    r = np.random.default_rng(1).standard_normal(grid.n)
    z = torch.empty(grid.n, dtype=torch.float64, device="cuda")
    ctx.vcycle(torch.tensor(r, device="cuda"), z)
    assert _nrel(z.cpu().numpy(), amg.vcycle(h, r)) <= 1e-4
    ctx.close()


@pytest.mark.parametrize("kind", ["fcg", "fgmres"])
def test_krylov_solution_parity(kind):
    rb = _rb()
    grid, p, ks, bc, dt, kmean = _problem((16, 14, 12), 11, 1)
    ctx, info, h = _setup_both(grid, p, ks, bc, dt, kmean, 100)
    b = np.random.default_rng(3).standard_normal(grid.n)
    x = torch.empty(grid.n, dtype=torch.float64, device="cuda")
    k = rb.KRYLOV_FCG if kind == "fcg" else rb.KRYLOV_FGMRES
    # J of the same p, on the GPU context (rich_jacobian was called in _setup_both)
    s, st = ctx.krylov_solve(torch.tensor(b, device="cuda"), x, kind=k, restart=10, eta=1e-11, maxit=400)
    J = disc.jacobian(grid, SOIL, bc, kmean, p, dt, ks)
    from oracle import krylov
    prec = lambda v: amg.vcycle(h, v)
    if kind == "fcg":
        xr, its, ok, _ = krylov.fcg(lambda v: J @ v, prec, b, 1e-11, 400)
    else:
        xr, its, ok, _ = krylov.fgmres(lambda v: J @ v, prec, b, 1e-11, 400, 10)
    assert ok and st.converged
    assert abs(st.iterations - its) <= 1
    xg = x.cpu().numpy()
    assert np.linalg.norm(J @ xg - b) <= 1e-11 * np.linalg.norm(b) * 1.0001
    assert _nrel(xg, xr) <= 1e-8
    ctx.close()


@pytest.mark.parametrize("kind", ["fgmres", "fcg"])
def test_krylov_stall_option_matches_oracle(kind):
    """krylov.stall: a fraction that an FGMRES(4) restart cycle, or a window of 30
    FCG iterations, cannot meet ends the solve there (RICH_ENOTCONV_LIN) with the
    oracle's iterate and count; a small fraction changes nothing."""
    rb = _rb()
    grid, p, ks, bc, dt, kmean = _problem((16, 14, 12), 11, 1)
    ctx, info, h = _setup_both(grid, p, ks, bc, dt, kmean, 100)
    b = np.random.default_rng(3).standard_normal(grid.n)
    J = disc.jacobian(grid, SOIL, bc, kmean, p, dt, ks)
    from oracle import krylov
    prec = lambda v: amg.vcycle(h, v)
    lin = {name: code for code, name in rb.ERRORS.items()}["RICH_ENOTCONV_LIN"]
    eta = 1e-11 if kind == "fgmres" else 1e-13
    k = rb.KRYLOV_FGMRES if kind == "fgmres" else rb.KRYLOV_FCG
    for stall, ok_expected in ((0.999999, False), (0.01, True)):
        x = torch.empty(grid.n, dtype=torch.float64, device="cuda")
        s, st = ctx.krylov_solve(torch.tensor(b, device="cuda"), x, kind=k, restart=4, eta=eta, maxit=400,
                                 check_status=False, stall=stall)
        if kind == "fgmres":
            xr, its, ok, _ = krylov.fgmres(lambda v: J @ v, prec, b, eta, 400, 4, stall=stall)
        else:
            xr, its, ok, _ = krylov.fcg(lambda v: J @ v, prec, b, eta, 400, stall=stall)
        assert ok == ok_expected and (s == 0) == ok and bool(st.converged) == ok
        if not ok:  # stopped at the end of a cycle (FGMRES(4)) or a 30-iteration window (FCG)
            assert s == lin and st.iterations == its and its % (4 if kind == "fgmres" else 30) == 0
        else:
            assert abs(st.iterations - its) <= 1
        assert _nrel(x.cpu().numpy(), xr) <= 1e-8
    ctx.close()


def test_fgmres_long_restart_cycle_matches_oracle():
    """FGMRES(63), the largest restart, with a weak preconditioner (one 9600-unknown
    level: eight l1-Jacobi sweeps), so that a cycle runs past j = 57 where the
    Hessenberg columns h1 and h2 fill the device scalar slots up to 62 and 126."""
    rb = _rb()
    grid, p, ks, bc, dt, kmean = _problem((24, 20, 20), 9, 0)
    ctx = rb.Context(grid, SOIL, bc, kmean, ks)
    ctx.jacobian(torch.tensor(p, device="cuda"), dt)
    ctx.amg_setup(rb.default_amg_opts(seed=2, max_levels=1))
    h = amg.setup(disc.aux_matrix(grid, SOIL, bc, kmean, p, dt, ks), 0.08, 2, 2000, max_levels=1)
    b = np.random.default_rng(5).standard_normal(grid.n)
    x = torch.empty(grid.n, dtype=torch.float64, device="cuda")
    s, st = ctx.krylov_solve(torch.tensor(b, device="cuda"), x, kind=rb.KRYLOV_FGMRES, restart=63, eta=1e-12,
                             maxit=300)
    J = disc.jacobian(grid, SOIL, bc, kmean, p, dt, ks)
    from oracle import krylov
    xr, its, ok, _ = krylov.fgmres(lambda v: J @ v, lambda v: amg.vcycle(h, v), b, 1e-12, 300, 63)
    assert ok and st.converged and its >= 60  # the first cycle reaches j >= 59
    assert abs(st.iterations - its) <= 1
    xg = x.cpu().numpy()
    assert np.linalg.norm(J @ xg - b) <= 1e-12 * np.linalg.norm(b) * 1.0001
    assert _nrel(xg, xr) <= 1e-8
    ctx.close()


def _run_steps(workload, n, steps, prec=0, policy=0, opts_kw=None):
    rb = _rb()
    w = synth.WORKLOADS[workload]
    grid, soil, bc, ks, p0, dts = synth.workload_inputs(w, n)
    kw = dict(kind=rb.KRYLOV_FGMRES if w.krylov == "fgmres" else rb.KRYLOV_FCG, restart=max(w.restart, 1),
              nu1=w.nu, nu2=w.nu, seed=w.amg_seed, coarse_max=w.coarse_max, amg_policy=policy,
              smooth_levels=w.smooth_levels)
    kw.update(opts_kw or {})
    opts = rb.default_newton_opts(**kw)
    ctx = rb.Context(grid, soil, bc, w.kmean, ks, precision=prec)
    pd = torch.tensor(p0, device="cuda")
    gstats = []
    for dt in dts[:steps]:
        gstats.append(ctx.step(pd, dt, opts))
    pol = {0: "refresh", 1: "setup_once", 2: "rebuild_step"}[policy]
    prob = newton.Problem(grid, soil, bc, w.kmean, ks)
    oopt = newton.NewtonOptions(krylov=w.krylov, restart=max(w.restart, 1), nu1=w.nu, nu2=w.nu,
                                amg_seed=w.amg_seed, coarse_max=w.coarse_max, amg_policy=pol,
                                smooth_levels=w.smooth_levels)
    for k, v in (opts_kw or {}).items():
        if k == "coarse_max":
            oopt.coarse_max = v
    p = p0
    ostats = []
    for dt in dts[:steps]:
        p, st = newton.step(prob, p, dt, oopt)
        ostats.append(st)
    ctx_p = pd.cpu().numpy()
    ctx.close()
    return ctx_p, p, gstats, ostats


@pytest.mark.parametrize("policy", [0, 1, 2])
def test_step_parity_richards16(policy):
    pg, po, gs, os_ = _run_steps("richards16_fp64", None, 5, policy=policy)
    np.testing.assert_allclose(pg, po, rtol=1e-8)
    for g, o in zip(gs, os_):
        assert g.converged and o.converged
        assert g.newton_its == o.newton_its


@pytest.mark.parametrize("dims,kind", [((1, 1, 30), "fcg"), ((1, 1, 1), "fcg"), ((3, 1, 1), "fgmres"),
                                       ((1, 2, 17), "fgmres")])
def test_step_parity_on_degenerate_grids(dims, kind):
    """One column, one cell, one row: a one-level hierarchy (its dense inverse is
    the whole preconditioner, the V-cycle graph a single GEMV) and columns with
    faces on both sides in x and y; three steps against the oracle."""
    rb = _rb()
    grid = synth.Grid(*dims, 30.0, 30.0, 30.0)
    bc = synth.infiltration_bc()
    ks = synth.ks_field(grid, 5, 0.5)
    p0 = np.full(grid.n, synth.P_INITIAL)
    k = rb.KRYLOV_FCG if kind == "fcg" else rb.KRYLOV_FGMRES
    opts = rb.default_newton_opts(kind=k, seed=2, coarse_max=100)
    ctx = rb.Context(grid, SOIL, bc, synth.KMEAN_UPSTREAM, ks)
    pd = torch.tensor(p0, device="cuda")
    prob = newton.Problem(grid, SOIL, bc, synth.KMEAN_UPSTREAM, ks)
    po = p0.copy()
    for dt in (0.5, 1.0, 2.0):
        st = ctx.step(pd, dt, opts)
        po, ost = newton.step(prob, po, dt, newton.NewtonOptions(krylov=kind, amg_seed=2, coarse_max=100))
        assert st.converged and ost.converged and st.newton_its == ost.newton_its
    assert _nrel(pd.cpu().numpy(), po) <= 1e-8
    ctx.close()


def test_step_parity_richards128_shape_at_32():
    # the 128^3 workload's settings (upstream mean, FGMRES(30), V(2,2), dt ramp) on a 32^3 grid
    pg, po, gs, os_ = _run_steps("richards128_fp64", 32, 4)
    np.testing.assert_allclose(pg, po, rtol=1e-8)
    for g, o in zip(gs, os_):
        assert g.newton_its == o.newton_its


def test_step_parity_paper_infiltration_small():
    # the paper's Sec. 6 problem (Dirichlet box, p = 0 square on top, upstream mean,
    # GMRES(10)) on a 32 x 32 x 4 grid of the 64 x 64 x 1 box
    pg, po, gs, os_ = _run_steps("paper_infiltration", 32, 3)
    np.testing.assert_allclose(pg, po, rtol=1e-8)
    for g, o in zip(gs, os_):
        assert g.converged and o.converged and g.newton_its == o.newton_its


@pytest.mark.parametrize("workload,n,steps", [("richards512_mixed", 24, 1), ("richards16_fp64", None, 5)])
def test_step_mixed_precision_matches_fp64_oracle(workload, n, steps):
    # FP32 hierarchy and V-cycle, FP64 residual/Jacobian/outer Krylov: the converged
    # pressure is the FP64 oracle's to the Newton tolerance.
    pg, po, gs, os_ = _run_steps(workload, n, steps, prec=1)
    np.testing.assert_allclose(pg, po, rtol=1e-8)


# ---------------------------------------------------------------- matching aggregation (SMATCH-style)

@pytest.mark.parametrize("dims,coarse_max,kmean,het", [((24, 24, 24), 300, 1, False), ((20, 18, 16), 150, 0, True),
                                                         ((33, 17, 9), 100, 2, True), ((40, 36, 32), 2000, 1, True)])
def test_matching_hierarchy_bit_exact(dims, coarse_max, kmean, het):
    grid, p, ks, bc, dt, _ = _problem(dims, 4, kmean, het=het)
    ctx, info, h = _setup_both(grid, p, ks, bc, dt, kmean, coarse_max, aggregation=1, smooth_levels=2)
    assert info.levels == len(h.levels) >= 2
    _compare_hierarchy(ctx, info, h)
    r = np.random.default_rng(5).standard_normal(grid.n)
    z = torch.empty(grid.n, dtype=torch.float64, device="cuda")
    ctx.vcycle(torch.tensor(r, device="cuda"), z)
    assert _nrel(z.cpu().numpy(), amg.vcycle(h, r)) <= 1e-10
    # the refresh reuses the matching aggregates
    rb = _rb()
    p2 = p + np.random.default_rng(6).uniform(0, 10, grid.n)
    ctx.jacobian(torch.tensor(p2, device="cuda"), dt)
    ctx.amg_update(rb.AMG_REFRESH)
    amg.refresh(h, disc.aux_matrix(grid, SOIL, bc, kmean, p2, dt, ks))
    _compare_hierarchy(ctx, info, h)
    ctx.close()


def test_matching_newton_step_matches_oracle():
    rb = _rb()
    w = synth.WORKLOADS["richards16_fp64"]
    grid, soil, bc, ks, p0, dts = synth.workload_inputs(w)
    ks = synth.ks_field(grid, 9, 1.0, (4.0, 4.0, 2.0))
    opts = rb.default_newton_opts(kind=rb.KRYLOV_FCG, nu1=1, nu2=1, seed=1, smooth_levels=2, coarse_max=200,
                                  aggregation=rb.AGG_MATCHING)
    ctx = rb.Context(grid, soil, bc, 0, ks)
    pd = torch.tensor(p0, device="cuda")
    po = p0.copy()
    prob = newton.Problem(grid, soil, bc, 0, ks)
    oopt = newton.NewtonOptions(krylov="fcg", nu1=1, nu2=1, amg_seed=1, smooth_levels=2, coarse_max=200,
                                aggregation="matching")
    for m in range(2):
        st = ctx.step(pd, dts[m], opts)
        po, ost = newton.step(prob, po, dts[m], oopt)
        assert st.converged and ost.converged
    assert _nrel(pd.cpu().numpy(), po) <= 1e-8
    ctx.close()


# ---------------------------------------------------------------- hybrid Gauss-Seidel smoother

@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
@pytest.mark.parametrize("dims,seg,block", [((18, 16, 20), 16, 16), ((33, 17, 9), 4, 5), ((12, 11, 40), 7, 16)])
def test_hybrid_gs_vcycle_parity(prec, tol, dims, seg, block):
    rb = _rb()
    grid, p, ks, bc, dt, kmean = _problem(dims, 12, 0)
    ctx = rb.Context(grid, SOIL, bc, kmean, ks, precision=prec)
    ctx.jacobian(torch.tensor(p, device="cuda"), dt)
    info = ctx.amg_setup(rb.default_amg_opts(seed=3, coarse_max=150, smoother=rb.SMOOTH_HYBRID_GS, hgs_seg=seg,
                                             hgs_block=block))
    A = disc.aux_matrix(grid, SOIL, bc, kmean, p, dt, ks)
    h = amg.setup(A, 0.08, 3, 150, smoother="hgs", grid=(grid.nx, grid.ny, grid.nz), hgs_seg=seg, hgs_block=block)
    assert info.levels == len(h.levels) >= 3
    r = np.random.default_rng(2).standard_normal(grid.n)
    z = torch.empty(grid.n, dtype=torch.float64, device="cuda")
    ctx.vcycle(torch.tensor(r, device="cuda"), z)
    assert _nrel(z.cpu().numpy(), amg.vcycle(h, r)) <= tol
    ctx.close()


@pytest.mark.parametrize("workload,n,steps,prec", [("richards16_fp64", None, 3, 0), ("richards512_mixed", 24, 1, 1)])
def test_hybrid_gs_newton_steps_match_oracle(workload, n, steps, prec):
    rb = _rb()
    w = synth.WORKLOADS[workload]
    grid, soil, bc, ks, p0, dts = synth.workload_inputs(w, n)
    opts = rb.default_newton_opts(kind=rb.KRYLOV_FCG, seed=w.amg_seed, coarse_max=200, smooth_levels=w.smooth_levels,
                                  smoother=rb.SMOOTH_HYBRID_GS)
    ctx = rb.Context(grid, soil, bc, w.kmean, ks, precision=prec)
    pd = torch.tensor(p0, device="cuda")
    prob = newton.Problem(grid, soil, bc, w.kmean, ks)
    oopt = newton.NewtonOptions(krylov="fcg", amg_seed=w.amg_seed, coarse_max=200, smooth_levels=w.smooth_levels,
                                smoother="hgs")
    po = p0
    for m in range(steps):
        st = ctx.step(pd, dts[m], opts)
        po, ost = newton.step(prob, po, dts[m], oopt)
        assert st.converged and ost.converged
        if prec == 0:
            assert st.newton_its == ost.newton_its and abs(st.linear_its - ost.linear_its) <= st.newton_its
    assert _nrel(pd.cpu().numpy(), po) <= 1e-8
    ctx.close()


# ---------------------------------------------------------------- additive Schwarz / ILU(0)

@pytest.mark.parametrize("prec,tol", [(0, 1e-10), (1, 1e-4)])
@pytest.mark.parametrize("dims,block,overlap", [((18, 16, 20), 8, 1), ((33, 17, 9), 4, 1), ((7, 5, 11), 3, 2),
                                                ((12, 12, 12), 12, 0)])
def test_additive_schwarz_apply_parity(prec, tol, dims, block, overlap):
    from oracle import schwarz
    rb = _rb()
    grid, p, ks, bc, dt, kmean = _problem(dims, 13, 1)
    ctx = rb.Context(grid, SOIL, bc, kmean, ks, precision=prec)
    ctx.jacobian(torch.tensor(p, device="cuda"), dt)
    ctx.amg_setup(rb.default_amg_opts(precond=rb.PRECOND_AS, as_block=block, as_overlap=overlap))
    A = disc.aux_matrix(grid, SOIL, bc, kmean, p, dt, ks)
    pre = schwarz.AS(A, (grid.nx, grid.ny, grid.nz), block, overlap)
    r = np.random.default_rng(4).standard_normal(grid.n)
    z = torch.empty(grid.n, dtype=torch.float64, device="cuda")
    ctx.vcycle(torch.tensor(r, device="cuda"), z)
    assert _nrel(z.cpu().numpy(), pre.apply(r)) <= tol
    ctx.close()


def test_additive_schwarz_newton_step_matches_oracle():
    rb = _rb()
    grid = synth.Grid(10, 9, 8)
    ks = synth.ks_field(grid, 3, 1.0, (4.0, 4.0, 2.0))
    bc = synth.infiltration_bc()
    p0 = np.full(grid.n, synth.P_INITIAL)
    opts = rb.default_newton_opts(kind=rb.KRYLOV_FGMRES, restart=30, precond=rb.PRECOND_AS, as_block=4)
    ctx = rb.Context(grid, SOIL, bc, synth.KMEAN_UPSTREAM, ks)
    pd = torch.tensor(p0, device="cuda")
    st = ctx.step(pd, 1.0, opts)
    po, ost = newton.step(newton.Problem(grid, SOIL, bc, synth.KMEAN_UPSTREAM, ks), p0, 1.0,
                          newton.NewtonOptions(krylov="fgmres", precond="as", as_block=4))
    assert st.converged and ost.converged and st.newton_its == ost.newton_its
    assert abs(st.linear_its - ost.linear_its) <= st.newton_its
    assert _nrel(pd.cpu().numpy(), po) <= 1e-8
    ctx.close()
