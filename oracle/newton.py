"""Backward-Euler step by inexact Newton with Armijo backtracking, FP64 (oracle; test infrastructure).

Sec. 3: at each time step solve Phi(p) = 0 (eq. (dynamic_of_the_problem)) by
Newton corrections J(p_r) d_r = -Phi(p_r) (eq. (linearsystemtosolve)), each
solved with a right-preconditioned Krylov method (eq. (precsystem)) and
preconditioned by the AMG V-cycle built on the diffusion-only matrix; the
step length lambda comes from an Armijo-type line search.  The paper gives
no constants; the readings used here (shared with the CUDA path) are:

  * convergence: ||Phi(p_r)||_2 <= max(rtol ||Phi(p_0)||_2, atol, eps ||m||_2)
    where m_c sums the magnitudes of the products that make up Phi_c before
    they cancel (discretization.residual, with_scale): late in a run, when a
    step starts close to steady state, rtol ||Phi_0|| falls below the accuracy
    to which Phi can be evaluated and the line search cannot make progress;
    the last term declares convergence at that attainable accuracy instead.
  * a fresh J and A_aux every Newton iteration.  The AMG hierarchy is built
    on the first A_aux of the run; afterwards
      'refresh'      (default) keeps aggregates, P and R and recomputes the
                     Galerkin coarse matrices from each new A_aux;
      'setup_once'   replaces only the finest matrix and its smoother (the
                     paper's reuse scheme, Sec. 6);
      'rebuild_step' rebuilds the whole hierarchy at the first Newton
                     iteration of every step and refreshes it afterwards.
  * linear tolerance eta (||J d + Phi|| <= eta ||Phi||), maximum maxit.
  * line search on f(lambda) = 1/2 ||Phi(p + lambda d)||^2 with slope
    g = Phi^T (J d): accept when f(lambda) <= f(0) + 1e-4 lambda g, else
    lambda <- clamp(-g lambda^2 / (2 (f(lambda) - f(0) - g lambda)),
    0.1 lambda, 0.5 lambda); fail below 1e-10.  A non-negative slope is a
    failure.
  * time-step control (advance, off unless max_dt_halvings > 0): a failed
    step is retried with half its length, down to dt / 2^H, and the length
    doubles back once the time reached allows it.
"""
import dataclasses
import math

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import amg
from . import constitutive as cst
from . import schwarz
from . import discretization as disc
from . import krylov


FLOOR_EPS = np.finfo(np.float64).eps


@dataclasses.dataclass
class NewtonOptions:
    krylov: str = "fcg"           # "fcg" or "fgmres"
    restart: int = 30
    eta: float = 1e-7
    maxit: int = 200
    stall: float = 0.0            # give up after an FGMRES cycle / 30 FCG iterations reducing the residual by less
    nu1: int = 1
    nu2: int = 1
    rtol: float = 1e-8
    atol: float = 1e-30
    max_newton: int = 50
    amg_policy: str = "refresh"   # "setup_once", "rebuild_step"
    theta: float = 0.08
    amg_seed: int = 1
    coarse_max: int = 2000
    max_levels: int = 10
    smooth_levels: int = 10
    aggregation: str = "mis2"     # or "matching" (the paper's SMATCH-style coarsening)
    max_agg_size: int = 8
    armijo_c: float = 1e-4
    lambda_min: float = 1e-10
    isolated_join: bool = True    # pass 3 of the MIS-2 aggregation (amg module docstring)
    smoother: str = "l1jacobi"    # or "hgs": hybrid backward/forward Gauss-Seidel (amg module)
    precond: str = "amg"          # or "as": one-level additive Schwarz with ILU(0) (schwarz module)
    as_block: int = 8
    as_overlap: int = 1
    hgs_seg: int = 16
    hgs_block: int = 16
    max_dt_halvings: int = 0      # time-step control (advance); 0 = off


@dataclasses.dataclass
class StepStats:
    newton_its: int = 0
    linear_its: int = 0
    line_search_evals: int = 0
    fallbacks: int = 0
    converged: bool = False
    res0: float = 0.0
    res: float = 0.0
    lambdas: list = dataclasses.field(default_factory=list)
    lin_its: list = dataclasses.field(default_factory=list)
    res_hist: list = dataclasses.field(default_factory=list)
    line_searches: list = dataclasses.field(default_factory=list)  # (f0, slope, [(lam, f(lam)), ...]) per iteration
    indefinite: bool = False      # the last attempt ended on (p, J p) <= 0 in FCG
    substeps: int = 1             # backward-Euler steps taken to cover dt (advance)
    dt_min: float = 0.0           # smallest of them
    dt_failures: int = 0          # attempts that failed and were retried with half the step


class Problem:
    def __init__(self, grid, soil, bc, kmean, ks=None):
        self.grid, self.soil, self.bc, self.kmean = grid, soil, bc, kmean
        self.ks = soil.ks if ks is None else ks
        self.hierarchy = None

    def residual(self, p, s_old, dt, with_scale=False):
        return disc.residual(self.grid, self.soil, self.bc, self.kmean, p, s_old, dt, self.ks, with_scale)

    def jacobian(self, p, dt):
        return disc.jacobian(self.grid, self.soil, self.bc, self.kmean, p, dt, self.ks)

    def aux(self, p, dt):
        return disc.aux_matrix(self.grid, self.soil, self.bc, self.kmean, p, dt, self.ks)


class LineSearchError(RuntimeError):
    pass


class LinearSolveError(RuntimeError):
    pass


class NewtonError(RuntimeError):
    pass


def armijo_backtrack(merit, f0, slope, c, lambda_min):
    """Armijo backtracking along a descent direction (Sec. 3, the line search of KINSOL's
    inexact Newton method; constants in the module docstring).

    merit(lam) returns (f(lam), extra) with f(lam) = 1/2 ||Phi(p + lam d)||^2; f0 = f(0)
    and slope = f'(0) < 0.  The trial steps start at lam = 1.  A trial is accepted
    when f(lam) <= f0 + c lam slope; otherwise the next trial minimises the quadratic
    that matches f(0), f'(0) and f(lam), clamped to [0.1 lam, 0.5 lam] (quadratic
    backtracking).  Returns (lam, f(lam), extra, trials) with trials the list of
    (lam, f(lam)) evaluated in order; raises LineSearchError once lam < lambda_min.
    """
    lam = 1.0
    trials = []
    while True:
        ft, extra = merit(lam)
        trials.append((lam, ft))
        if ft <= f0 + c * lam * slope:
            return lam, ft, extra, trials
        lq = -slope * lam * lam / (2.0 * (ft - f0 - slope * lam))
        lam = min(max(lq, 0.1 * lam), 0.5 * lam)
        if lam < lambda_min:
            raise LineSearchError("line search failed")


def linear_solve(J, h, rhs, opt, stats):
    if opt.krylov == "direct":  # exact correction (tests: separates Newton from the preconditioner)
        return spla.spsolve(sp.csc_matrix(J), rhs), 0, True
    if isinstance(h, schwarz.AS):
        prec = h.apply
    else:
        prec = lambda v: amg.vcycle(h, v, opt.nu1, opt.nu2)
    mv = lambda v: J @ v
    if opt.krylov == "fcg":
        info = {}
        d, its, ok, _ = krylov.fcg(mv, prec, rhs, opt.eta, opt.maxit, info=info, stall=opt.stall)
        stats.linear_its += its
        if ok:
            return d, its, True
        if opt.max_dt_halvings > 0 and info.get("reason") == "curvature":
            # under time-step control a Jacobian that is not positive definite along
            # a preconditioned direction ends the attempt: the step is retried shorter
            stats.indefinite = True
            return d, its, False
        stats.fallbacks += 1
    d, its, ok, _ = krylov.fgmres(mv, prec, rhs, opt.eta, opt.maxit, opt.restart, opt.stall)
    stats.linear_its += its
    return d, its, ok


def step(prob, p, dt, opt):
    """Advance p by one backward-Euler step of size dt; returns (p_new, stats).

    A failure raises LinearSolveError or LineSearchError carrying the statistics
    gathered until then (attribute stats); Newton non-convergence returns with
    stats.converged False."""
    st = StepStats()
    try:
        return _step(prob, p, dt, opt, st)
    except (LinearSolveError, LineSearchError) as e:
        e.stats = st
        raise


def _step(prob, p, dt, opt, st):
    p = np.array(p, dtype=np.float64)
    s_old = cst.saturation(p, prob.soil)
    F, scale = prob.residual(p, s_old, dt, with_scale=True)
    fn = np.linalg.norm(F)
    st.res0 = fn
    tol = max(opt.rtol * fn, opt.atol)
    st.res_hist.append(fn)
    for r in range(opt.max_newton + 1):
        if fn <= max(tol, FLOOR_EPS * scale):
            st.converged = True
            break
        if r == opt.max_newton:
            break
        J = prob.jacobian(p, dt)
        A = prob.aux(p, dt)
        if opt.precond == "as":  # subdomain factors of the current A_aux
            prob.hierarchy = schwarz.AS(A, (prob.grid.nx, prob.grid.ny, prob.grid.nz), opt.as_block, opt.as_overlap)
        elif prob.hierarchy is None or (opt.amg_policy == "rebuild_step" and r == 0):
            prob.hierarchy = amg.setup(A, opt.theta, opt.amg_seed, opt.coarse_max, opt.max_levels,
                                       smooth_levels=opt.smooth_levels, aggregation=opt.aggregation,
                                       max_agg_size=opt.max_agg_size, isolated_join=opt.isolated_join,
                                       smoother=opt.smoother, grid=(prob.grid.nx, prob.grid.ny, prob.grid.nz),
                                       hgs_seg=opt.hgs_seg, hgs_block=opt.hgs_block)
        elif opt.amg_policy == "setup_once":
            amg.update_fine(prob.hierarchy, A)
        else:
            amg.refresh(prob.hierarchy, A)
        d, its, ok = linear_solve(J, prob.hierarchy, -F, opt, st)
        st.lin_its.append(its)
        if not ok:
            raise LinearSolveError("linear solver did not converge")
        g = float(F @ (J @ d))
        if not g < 0.0:
            raise LineSearchError("non-descent Newton direction")
        f0 = 0.5 * fn * fn

        def merit(lam):
            Ft, scale_t = prob.residual(p + lam * d, s_old, dt, with_scale=True)
            return 0.5 * float(Ft @ Ft), (Ft, scale_t)

        lam, ft, (Ft, scale_t), trials = armijo_backtrack(merit, f0, g, opt.armijo_c, opt.lambda_min)
        st.line_search_evals += len(trials)
        st.line_searches.append((f0, g, trials))
        p = p + lam * d
        F, scale = Ft, scale_t
        fn = np.linalg.norm(F)
        st.res_hist.append(fn)
        st.lambdas.append(lam)
        st.newton_its += 1
    st.res = fn
    return p, st


def advance(prob, p, dt, opt):
    """Cover one time step dt with backward-Euler steps under time-step control.

    The paper fixes dt per step (Sec. 6) and gives no control; this is the usual
    host-side remedy when Newton fails at a steep wetting front.  With
    opt.max_dt_halvings = H > 0 the step is tried whole; an attempt that fails
    in the line search, in Newton, or in FCG on a Jacobian that is not positive
    definite along a preconditioned direction is discarded and retried with half
    its length, down to dt / 2^H (a Krylov solve that merely runs out of
    iterations ends the step: a shorter step does not mend the preconditioner,
    and retrying it would multiply the cost); after each accepted substep the
    length doubles again whenever the time reached is a multiple of the doubled
    length, so the substeps land exactly on dt.  Lengths are dt / 2^k (exact in
    binary floating point).  Returns (p_new, stats) with the Newton and Krylov
    counts summed over accepted and failed attempts; raises the last failure
    when a step of dt / 2^H fails.
    """
    H = int(opt.max_dt_halvings)
    if H <= 0:
        return step(prob, p, dt, opt)
    total = 1 << H          # dt in units of dt / 2^H
    t = 0                   # time reached, in those units
    k = 0                   # current substep length dt / 2^k = 2^(H-k) units
    acc = StepStats(substeps=0, dt_min=dt)
    acc.res0 = None
    p = np.array(p, dtype=np.float64)
    while t < total:
        h = math.ldexp(dt, -k)
        length = 1 << (H - k)
        try:
            p_new, st = step(prob, p, h, opt)
            ok = st.converged
            err = None if ok else NewtonError("Newton did not converge")
        except (LinearSolveError, LineSearchError) as e:
            st, ok, err = getattr(e, "stats", None), False, e
            if isinstance(e, LinearSolveError) and not (st is not None and st.indefinite):
                raise
        if st is not None:
            acc.newton_its += st.newton_its
            acc.linear_its += st.linear_its
            acc.line_search_evals += st.line_search_evals
            acc.fallbacks += st.fallbacks
            acc.lambdas += st.lambdas
            acc.lin_its += st.lin_its
            acc.line_searches += st.line_searches
            if acc.res0 is None:
                acc.res0 = st.res0
            acc.res = st.res
        if not ok:
            acc.dt_failures += 1
            if k == H:
                raise err
            k += 1
            continue
        p = p_new
        t += length
        acc.substeps += 1
        acc.dt_min = min(acc.dt_min, h)
        if k > 0 and t % (2 * length) == 0:
            k -= 1
    acc.converged = True
    if acc.res0 is None:
        acc.res0 = 0.0
    return p, acc
