"""Pins of the oracle's Newton control and of the paper's spectral theory (CPU only).

What fixes these parts other than the oracle itself:
  * the line search (Sec. 3): the accepted step satisfies the Armijo inequality,
    every rejected step violates it, and each new trial is the minimiser of the
    quadratic that interpolates f(0), f'(0) and the rejected f(lam), clamped to
    [0.1, 0.5] lam -- the minimiser is found here from the interpolation
    conditions and the stationarity of the quadratic, not from the oracle's
    closed form; one hand-computed backtrack on arctan checks the numbers;
  * the convergence floor eps ||m||: 40-digit evaluations of Phi on the same
    FP64 inputs show that eps ||m|| bounds the FP64 evaluation error of Phi and
    is within a small factor of it on generic states; on a 16^3 run the floor
    changes no step that converges without it and rescues the step where the
    plain relative test can only fail;
  * the eigenvalue distribution of h^2 J (Theorems (eigenvaluedistributionwith
    arithmeticmean), (spectraldistribution_jacobians_3D_arithmetic_mean) and
    (spectraldescription)): the sorted eigenvalues approach the sorted samples of
    the symbol C s'(p(x)) + K(p(x)) sum_d (2 - 2 cos theta_d) with C = h^2/dt, the
    discrepancy shrinking like 1/n, while symbols with a wrong constant do not;
  * time-step control: the substep schedule against hand-written schedules, and
    the harmonic-mean infiltration that fails even with exact Newton corrections
    and converges once the step is cut.
"""
import math

import numpy as np
import pytest
import scipy.sparse as sp

from oracle import amg
from oracle import constitutive as cst
from oracle import discretization as disc
from oracle import krylov
from oracle import newton
from paper_2112_05051_gb300 import synth

SOIL = synth.Soil()


# ---------------------------------------------------------------- line search (Sec. 3)

def _quadratic_minimiser(f0, g, lam, f_lam):
    """Minimiser of the quadratic q with q(0) = f0, q'(0) = g, q(lam) = f_lam: the
    coefficients come from the three interpolation conditions (a linear solve), the
    minimiser from q'(t) = 0."""
    M = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [1.0, lam, lam * lam]])
    c0, c1, c2 = np.linalg.solve(M, np.array([f0, g, f_lam]))
    assert c2 > 0  # a rejected trial lies above the tangent line, so q is convex
    return float(np.roots([2.0 * c2, c1])[0])


def _check_trials(f0, g, trials, c=1e-4):
    """Armijo acceptance of the last trial, rejection of the others, clamped quadratic updates."""
    assert trials[0][0] == 1.0
    lam_acc, f_acc = trials[-1]
    assert f_acc <= f0 + c * lam_acc * g
    for (lam, f_lam), (lam_next, _) in zip(trials[:-1], trials[1:]):
        assert f_lam > f0 + c * lam * g
        t = _quadratic_minimiser(f0, g, lam, f_lam)
        expect = min(max(t, 0.1 * lam), 0.5 * lam)
        assert lam_next == pytest.approx(expect, rel=1e-10, abs=1e-300)


def test_backtracking_on_arctan_matches_the_quadratic_model():
    # Newton on Phi(x) = arctan(x) from x0 = 10 overshoots: d = -(1 + x0^2) arctan(x0)
    # and the slope of f = 1/2 Phi^2 along d is -arctan(x0)^2.
    x0 = 10.0
    phi0 = math.atan(x0)
    d = -(1.0 + x0 * x0) * phi0
    f0 = 0.5 * phi0 * phi0
    g = -phi0 * phi0
    lam, ft, _, trials = newton.armijo_backtrack(lambda t: (0.5 * math.atan(x0 + t * d) ** 2, None), f0, g, 1e-4,
                                                 1e-10)
    # by hand: f0 = 1.0821083, d = -148.58390, f(1) = 0.5 atan(-138.58390)^2 = 1.2223922,
    # so the first backtrack is 2.1642166 / (2 (1.2223922 - 1.0821083 + 2.1642166)) = 0.469563
    assert f0 == pytest.approx(1.0821083, rel=1e-7)
    assert trials[0][1] == pytest.approx(1.2223922, rel=1e-7)
    assert trials[1][0] == pytest.approx(0.469563, rel=1e-5)
    assert len(trials) >= 3  # several backtracks before sufficient decrease
    _check_trials(f0, g, trials)
    assert ft < f0 and 0.0 < lam < 0.5


def test_line_search_trials_at_a_sharp_wetting_front():
    # 30 cm column, very dry (-200 cm) under a wet top (-1 cm), dt = 10 s: Newton
    # needs damped steps (quadratic backtracks, and the 0.1 lam clamp)
    grid = synth.Grid(1, 1, 30, 30.0, 30.0, 30.0)
    prob = newton.Problem(grid, SOIL, synth.infiltration_bc(-1.0), synth.KMEAN_ARITH)
    opt = newton.NewtonOptions(krylov="fgmres", coarse_max=10, eta=1e-10)
    p, st = newton.step(prob, np.full(grid.n, -200.0), 10.0, opt)
    assert st.converged
    backtracked = [ls for ls in st.line_searches if len(ls[2]) > 1]
    assert len(backtracked) >= 4
    clamped = 0
    for f0, g, trials in st.line_searches:
        assert g < 0
        _check_trials(f0, g, trials)
        clamped += sum(1 for (a, _), (b, _) in zip(trials[:-1], trials[1:]) if b == 0.1 * a)
    assert clamped >= 1
    assert st.line_search_evals == sum(len(t) for _, _, t in st.line_searches)


def _planted_backtrack(update):
    def bad(merit, f0, slope, c, lambda_min):
        lam, trials = 1.0, []
        while True:
            ft, extra = merit(lam)
            trials.append((lam, ft))
            if ft <= f0 + c * lam * slope:
                return lam, ft, extra, trials
            lam = update(lam, ft, f0, slope)
            if lam < lambda_min:
                raise newton.LineSearchError("line search failed")
    return bad


def test_pins_catch_a_sign_error_in_the_quadratic_backtrack(monkeypatch):
    def update(lam, ft, f0, g):  # + instead of - in front of the slope term
        lq = -g * lam * lam / (2.0 * (ft - f0 + g * lam))
        return min(max(lq, 0.1 * lam), 0.5 * lam)
    monkeypatch.setattr(newton, "armijo_backtrack", _planted_backtrack(update))
    with pytest.raises(AssertionError):
        test_backtracking_on_arctan_matches_the_quadratic_model()


def test_pins_catch_a_wrong_clamp(monkeypatch):
    def update(lam, ft, f0, g):  # clamp to [0.05, 0.5] lam
        lq = -g * lam * lam / (2.0 * (ft - f0 - g * lam))
        return min(max(lq, 0.05 * lam), 0.5 * lam)
    monkeypatch.setattr(newton, "armijo_backtrack", _planted_backtrack(update))
    with pytest.raises(AssertionError):
        test_line_search_trials_at_a_sharp_wetting_front()


# ---------------------------------------------------------------- convergence floor eps ||m||

def _exact_residual(grid, bc, kmean, p, s_old, dt, ks, mp):
    """Phi of eq. (dynamic_of_the_problem) in 40-digit arithmetic on the same FP64 inputs."""
    nx, ny, nz = grid.nx, grid.ny, grid.nz
    h = [mp.mpf(v) for v in grid.h]
    al, be, ts, tr, a, ga = (mp.mpf(v) for v in (SOIL.alpha, SOIL.beta, SOIL.theta_s, SOIL.theta_r, SOIL.a,
                                                  SOIL.gamma))

    def sat(x):
        return ts if x >= 0 else al * (ts - tr) / (al + abs(x) ** be) + tr

    def cond(x, k):
        return k if x >= 0 else k * a / (a + abs(x) ** ga)

    def mean(kl, ku, pl, pu):
        if kmean == synth.KMEAN_ARITH:
            return (kl + ku) / 2
        if kmean == synth.KMEAN_UPSTREAM:
            return ku if pu - pl >= 0 else kl
        if kmean == synth.KMEAN_HARMONIC:
            return 2 * kl * ku / (kl + ku)
        return mp.sqrt(kl * ku)

    P = [mp.mpf(float(v)) for v in p]
    KS = [mp.mpf(float(v)) for v in ks]
    out = np.zeros(grid.n)
    for c in range(grid.n):
        ijk = (c % nx, (c // nx) % ny, c // (nx * ny))
        pc = P[c]
        kc = cond(pc, KS[c])
        phi = (sat(pc) - mp.mpf(float(s_old[c]))) / mp.mpf(dt)
        for f, (axis, side) in enumerate(((0, -1), (0, 1), (1, -1), (1, 1), (2, -1), (2, 1))):
            ext = (nx, ny, nz)[axis]
            if ijk[axis] == (ext - 1 if side > 0 else 0):
                if bc.kind[f] == synth.BC_NOFLUX:
                    continue
                pn, kn = mp.mpf(bc.value[f]), cond(mp.mpf(bc.value[f]), KS[c])
            else:
                q = c + side * (1, nx, nx * ny)[axis]
                pn, kn = P[q], cond(P[q], KS[q])
            kl, ku, pl, pu = (kc, kn, pc, pn) if side > 0 else (kn, kc, pn, pc)
            t = mean(kl, ku, pl, pu) * (pc - pn) / h[axis] ** 2
            if axis == 2:
                t -= side * (kc + kn) / (2 * h[2])
            phi += t
        out[c] = float(phi)
    return out


@pytest.mark.parametrize("kmean", [synth.KMEAN_ARITH, synth.KMEAN_UPSTREAM, synth.KMEAN_HARMONIC,
                                   synth.KMEAN_GEOMETRIC])
def test_floor_bounds_the_fp64_evaluation_error_of_phi(kmean):
    mpmath = pytest.importorskip("mpmath")
    mp = mpmath.mp.clone() if hasattr(mpmath.mp, "clone") else mpmath.mp
    mp.dps = 40
    grid = synth.Grid(5, 4, 6)
    ks = synth.ks_field(grid, 3, 1.0, (2.0, 2.0, 2.0))
    bc = synth.infiltration_bc()
    rng = np.random.default_rng(1)
    eps = np.finfo(np.float64).eps
    # a generic state: the bound holds and is within a factor 20 of the error
    p = rng.uniform(-70.0, -15.0, grid.n)
    s_old = cst.saturation(p + rng.uniform(-1.0, 1.0, grid.n), SOIL)
    F, m = disc.residual(grid, SOIL, bc, kmean, p, s_old, 1.0, ks, with_scale=True)
    err = np.linalg.norm(F - _exact_residual(grid, bc, kmean, p, s_old, 1.0, ks, mp))
    assert 0.05 * eps * m <= err <= eps * m
    # near the steady state Phi is tiny and its evaluation error stays under the floor
    hz = grid.h[2]
    z = (np.arange(grid.nz) + 1) * hz
    p = np.broadcast_to((-20.7 + (grid.nz + 1) * hz - z)[:, None, None], grid.shape).ravel().copy()
    s_old = cst.saturation(p, SOIL)
    F, m = disc.residual(grid, SOIL, bc, kmean, p, s_old, 1.0, ks, with_scale=True)
    err = np.linalg.norm(F - _exact_residual(grid, bc, kmean, p, s_old, 1.0, ks, mp))
    assert err <= eps * m


def test_floor_changes_no_converged_step_and_rescues_the_late_ones(monkeypatch):
    # the 128^3 bench schedule (upstream mean, dt 1 -> 30 s, FGMRES(30), V(2,2)) on 16^3
    w = synth.WORKLOADS["richards128_fp64"]
    grid, soil, bc, ks, p0, dts = synth.workload_inputs(w, 16)
    opt = newton.NewtonOptions(krylov="fgmres", restart=30, nu1=2, nu2=2, amg_seed=2, coarse_max=200,
                               smooth_levels=2)

    def run(floor_on, nsteps):
        monkeypatch.setattr(newton, "FLOOR_EPS", np.finfo(np.float64).eps if floor_on else 0.0)
        prob = newton.Problem(grid, soil, bc, w.kmean, ks)
        p, out = p0.copy(), []
        for dt in dts[:nsteps]:
            try:
                p, st = newton.step(prob, p, dt, opt)
            except newton.LineSearchError:
                out.append(None)
                break
            out.append((p, st))
        return out

    with_floor = run(True, 7)
    without = run(False, 7)
    assert all(r is not None for r in with_floor)
    plain = [r for r in without if r is not None]
    assert len(plain) >= 5 and without[-1] is None  # the plain test fails late in the schedule
    for (pa, sa), (pb, sb) in zip(with_floor, plain):
        assert sa.newton_its == sb.newton_its
        np.testing.assert_array_equal(pa, pb)  # the floor never decided these steps
    # the rescued step stops at the floor, within a few times the relative target
    _, st = with_floor[len(plain)]
    assert st.converged and st.res > 1e-8 * st.res0 and st.res < 1e-6 * st.res0


# ---------------------------------------------------------------- eigenvalue distribution (Sec. 4)

def _symbol_quantiles(values, n):
    """n evenly spaced quantiles of the sorted symbol samples."""
    v = np.sort(values)
    return v[(np.arange(n) * len(v)) // n + len(v) // (2 * n)]


def _discrepancy_1d(kmean, n, offset=0.0, k_scale=1.0):
    grid = synth.Grid(1, 1, n)
    h = grid.h[2]
    z = (np.arange(n) + 1) * h
    p = -30.0 - 20.0 * np.sin(np.pi * z)
    dt = h * h  # C = lim h^2 / dt = 1
    bc = synth.BC(kind=(0, 0, 0, 0, 1, 1), value=(0, 0, 0, 0, -30.0, -30.0))
    ev = np.linalg.eigvals(h * h * disc.jacobian(grid, SOIL, bc, kmean, p, dt).toarray())
    assert np.abs(ev.imag).max() <= 1e-9 * np.abs(ev.real).max()
    ev = np.sort(ev.real)
    x = (np.arange(n) + 0.5) / n
    th = (np.arange(n) + 0.5) * np.pi / n  # the symbol is even in theta
    px = -30.0 - 20.0 * np.sin(np.pi * x)
    kap = (cst.dsaturation(px, SOIL)[:, None]
           + k_scale * cst.conductivity(px, SOIL, SOIL.ks)[:, None] * (offset + 2.0 - 2.0 * np.cos(th))[None, :])
    q = _symbol_quantiles(kap.ravel(), n)
    return np.mean(np.abs(ev - q)) / np.mean(np.abs(q))


@pytest.mark.parametrize("kmean", [synth.KMEAN_ARITH, synth.KMEAN_UPSTREAM])
def test_1d_jacobian_eigenvalues_follow_the_glt_symbol(kmean):
    d = [_discrepancy_1d(kmean, n) for n in (100, 200, 400, 800)]
    for a, b in zip(d[:-1], d[1:]):
        assert b < a / 1.7  # first-order convergence of the distribution
    assert d[-1] < 2e-3
    # a symbol with K doubled does not describe the spectrum
    wrong = [_discrepancy_1d(kmean, n, k_scale=2.0) for n in (100, 400)]
    assert wrong[1] > 0.5 * wrong[0] and wrong[1] > 20.0 * d[2]


def _discrepancy_3d(kmean, n, offset):
    grid = synth.Grid(n, n, n)
    h = grid.h[0]
    c = (np.arange(n) + 1) * h

    def pfun(x, y, zz):
        return -30.0 - 10.0 * np.sin(np.pi * x) * np.sin(np.pi * y) - 10.0 * zz

    Z, Y, X = np.meshgrid(c, c, c, indexing="ij")
    p = pfun(X, Y, Z).ravel()
    J = disc.jacobian(grid, SOIL, synth.all_dirichlet_bc(-30.0), kmean, p, h * h).toarray()
    ev = np.sort(np.linalg.eigvals(h * h * J).real)
    m = 2 * n
    x = (np.arange(m) + 0.5) / m
    th = (np.arange(m) + 0.5) * np.pi / m
    XX = np.meshgrid(x, x, x, indexing="ij")
    px = pfun(XX[2], XX[1], XX[0]).ravel()
    T = np.meshgrid(th, th, th, indexing="ij")
    cs = sum(2.0 - 2.0 * np.cos(t) for t in T).ravel()
    kap = cst.dsaturation(px, SOIL)[:, None] + cst.conductivity(px, SOIL, SOIL.ks)[:, None] * (cs[None, :] + offset)
    q = _symbol_quantiles(kap.ravel(), grid.n)
    return np.mean(np.abs(ev - q)) / np.mean(np.abs(q))


@pytest.mark.parametrize("kmean", [synth.KMEAN_ARITH, synth.KMEAN_UPSTREAM])
def test_3d_jacobian_eigenvalues_follow_the_seven_point_symbol(kmean):
    # sum_d (2 - 2 cos theta_d) = 6 - 2 sum cos theta_d, the 7-point Laplacian's symbol;
    # the theorem prints 8 - 2 sum cos theta_d, which the spectrum does not follow
    ns = (4, 6, 8, 10)
    d6 = [_discrepancy_3d(kmean, n, 0.0) for n in ns]
    for a, b in zip(d6[:-1], d6[1:]):
        assert b < a
    assert d6[-1] < 0.7 * d6[1]
    d8 = _discrepancy_3d(kmean, 10, 2.0)
    assert d8 > 1.5 * d6[-1]


# ---------------------------------------------------------------- time-step control

def test_substep_schedule_halves_on_failure_and_grows_back(monkeypatch):
    calls = []

    def fake_step(prob, p, h, opt):
        calls.append(h)
        st = newton.StepStats(newton_its=1, converged=True, res0=1.0, res=0.0)
        if h > 0.25 and len(calls) < 4:  # the first attempts above a quarter of the step fail
            raise newton.LineSearchError("forced")
        return p + h, st

    monkeypatch.setattr(newton, "step", fake_step)
    p, st = newton.advance(None, np.zeros(3), 1.0, newton.NewtonOptions(max_dt_halvings=4))
    # 1 fails, 1/2 fails, 1/4 passes at t=0, 1/4 at t=1/4 (doubling needs t a multiple of 1/2),
    # then 1/2 at t=1/2 ends exactly at 1
    assert calls == [1.0, 0.5, 0.25, 0.25, 0.5]
    assert st.substeps == 3 and st.dt_failures == 2 and st.dt_min == 0.25
    np.testing.assert_array_equal(p, np.ones(3))


def test_krylov_running_out_of_iterations_is_not_retried(monkeypatch):
    calls = []

    def fake_step(prob, p, h, opt):
        calls.append(h)
        e = newton.LinearSolveError("forced")
        e.stats = newton.StepStats()  # not an indefinite Jacobian: maxit
        raise e

    monkeypatch.setattr(newton, "step", fake_step)
    with pytest.raises(newton.LinearSolveError):
        newton.advance(None, np.zeros(2), 1.0, newton.NewtonOptions(max_dt_halvings=3))
    assert calls == [1.0]


def test_substep_schedule_gives_up_at_the_smallest_step(monkeypatch):
    def fake_step(prob, p, h, opt):
        raise newton.LineSearchError("forced")

    monkeypatch.setattr(newton, "step", fake_step)
    with pytest.raises(newton.LineSearchError):
        newton.advance(None, np.zeros(2), 1.0, newton.NewtonOptions(max_dt_halvings=3))


def test_harmonic_wet_face_fails_with_exact_corrections_and_converges_with_shorter_steps():
    # dry soil (-61.5 cm) under a wet top (-20.7 cm), harmonic mean, sigma 1 field: the
    # Jacobian has negative diagonal entries in the top layer (K'_c (p_c - p_top)/h^2 outweighs
    # K_av/h^2), and even exact Newton corrections make little progress at dt = 1 s
    grid = synth.Grid(12, 12, 12)
    ks = synth.ks_field(grid, 1000, 1.0)
    bc = synth.infiltration_bc(synth.P_TOP)
    p0 = np.full(grid.n, synth.P_INITIAL)
    prob = newton.Problem(grid, SOIL, bc, synth.KMEAN_HARMONIC, ks)
    J = prob.jacobian(p0, 1.0)
    assert np.sum(J.diagonal() < 0) > 0
    ok = True
    try:
        _, st = newton.step(prob, p0, 1.0, newton.NewtonOptions(krylov="direct", max_newton=12))
        ok = st.converged
        assert st.res > 0.05 * st.res0  # little progress after 12 exact Newton corrections
    except newton.LineSearchError:
        ok = False
    assert not ok
    # time-step control covers the same step in shorter backward-Euler steps
    prob = newton.Problem(grid, SOIL, bc, synth.KMEAN_HARMONIC, ks)
    opt = newton.NewtonOptions(krylov="fcg", coarse_max=100, max_dt_halvings=10)
    p1, st = newton.advance(prob, p0, 1.0, opt)
    assert st.converged and st.substeps > 1 and st.dt_min < 0.1
    # the result is a backward-Euler solution at every substep: check the last one's
    # mass balance sign (wetting from the top)
    assert np.all(p1 >= synth.P_INITIAL - 1e-9) and p1.max() > synth.P_INITIAL + 1.0


# ---------------------------------------------------------------- isolated nodes (pass 3 of the aggregation)

def test_isolated_zero_sum_row_joins_its_strongest_neighbour_and_dominant_row_stays_out():
    # path 0-1-2-3-4 with a tail node 5 hanging off 2 by a coupling that is weak by the
    # symmetric measure (|a_25|^2 < theta^2 a_22 a_55 fails only for row 2's large diagonal)
    # and a Dirichlet-like node 6 coupled weakly to 4
    n = 7
    A = np.zeros((n, n))
    for i, j, w in ((0, 1, 100.0), (1, 2, 100.0), (2, 3, 100.0), (3, 4, 100.0), (2, 5, 1.0), (4, 6, 0.1), (5, 6, 0.2)):
        A[i, j] = A[j, i] = -w
    for i in range(n):
        A[i, i] = -A[i].sum()
    A[6, 6] += 50.0  # node 6: diagonal excess far above its couplings (dominant)
    A = sp.csr_matrix(A)
    S = amg.strength(A, 0.08)
    assert S[5].nnz == 0 and S[6].nnz == 0  # both isolated by the symmetric measure
    keys = amg.priority_keys(n, 1)
    state, _ = amg.mis2(S, keys)
    agg0, nc = amg.aggregate(S, state, keys)
    assert agg0[5] == -1 and agg0[6] == -1
    agg, nc = amg.aggregate(S, state, keys, A)
    assert agg[5] == agg[2]  # strongest aggregated neighbour of 5 is 2 (|a_25| = 1 > |a_56| = 0.2)
    assert agg[6] == -1
    np.testing.assert_array_equal(np.delete(agg, 5), np.delete(agg0, 5))


def test_pass_three_restores_the_vcycle_on_a_high_contrast_field():
    # sigma 2 (about 16 decades of K_s), arithmetic mean, dt = 10 s
    w = synth.WORKLOADS["richards512_mixed"]
    grid, soil, bc, ks, p0, dts = synth.workload_inputs(w, 48)
    A = disc.aux_matrix(grid, soil, bc, w.kmean, p0, dts[0], ks)
    F = disc.residual(grid, soil, bc, w.kmean, p0, cst.saturation(p0, soil), dts[0], ks)
    its = {}
    for join in (False, True):
        h = amg.setup(A, 0.08, w.amg_seed, 2000, smooth_levels=2, isolated_join=join)
        _, its[join], ok, _ = krylov.fcg(lambda v: A @ v, lambda v: amg.vcycle(h, v), -F, 1e-7, 300)
        assert ok
        left = h.levels[0].agg < 0
        Ad = A.diagonal()
        offsum = np.asarray(abs(A).sum(axis=1)).ravel() - np.abs(Ad)
        if join:  # only dominant rows (or rows without an aggregated neighbour) stay out
            assert np.all(Ad[left] >= 2.0 * offsum[left] - 1e-12 * Ad[left]) or left.sum() < 10
    assert its[True] < 0.8 * its[False]
