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
"""
import dataclasses

import numpy as np

from . import amg
from . import constitutive as cst
from . import discretization as disc
from . import krylov


FLOOR_EPS = np.finfo(np.float64).eps


@dataclasses.dataclass
class NewtonOptions:
    krylov: str = "fcg"           # "fcg" or "fgmres"
    restart: int = 30
    eta: float = 1e-7
    maxit: int = 200
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


def linear_solve(J, h, rhs, opt, stats):
    prec = lambda v: amg.vcycle(h, v, opt.nu1, opt.nu2)
    mv = lambda v: J @ v
    if opt.krylov == "fcg":
        d, its, ok, _ = krylov.fcg(mv, prec, rhs, opt.eta, opt.maxit)
        stats.linear_its += its
        if ok:
            return d, its, True
        stats.fallbacks += 1
    d, its, ok, _ = krylov.fgmres(mv, prec, rhs, opt.eta, opt.maxit, opt.restart)
    stats.linear_its += its
    return d, its, ok


def step(prob, p, dt, opt):
    """Advance p by one backward-Euler step of size dt; returns (p_new, stats)."""
    p = np.array(p, dtype=np.float64)
    s_old = cst.saturation(p, prob.soil)
    st = StepStats()
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
        if prob.hierarchy is None or (opt.amg_policy == "rebuild_step" and r == 0):
            prob.hierarchy = amg.setup(A, opt.theta, opt.amg_seed, opt.coarse_max, opt.max_levels,
                                       smooth_levels=opt.smooth_levels, aggregation=opt.aggregation,
                                       max_agg_size=opt.max_agg_size)
        elif opt.amg_policy == "setup_once":
            amg.update_fine(prob.hierarchy, A)
        else:
            amg.refresh(prob.hierarchy, A)
        d, its, ok = linear_solve(J, prob.hierarchy, -F, opt, st)
        st.lin_its.append(its)
        if not ok:
            raise RuntimeError("linear solver did not converge")
        g = float(F @ (J @ d))
        if not g < 0.0:
            raise RuntimeError("non-descent Newton direction")
        f0 = 0.5 * fn * fn
        lam = 1.0
        while True:
            Ft, scale_t = prob.residual(p + lam * d, s_old, dt, with_scale=True)
            st.line_search_evals += 1
            ft = 0.5 * float(Ft @ Ft)
            if ft <= f0 + opt.armijo_c * lam * g:
                break
            lq = -g * lam * lam / (2.0 * (ft - f0 - g * lam))
            lam = min(max(lq, 0.1 * lam), 0.5 * lam)
            if lam < opt.lambda_min:
                raise RuntimeError("line search failed")
        p = p + lam * d
        F, scale = Ft, scale_t
        fn = np.linalg.norm(F)
        st.res_hist.append(fn)
        st.lambdas.append(lam)
        st.newton_its += 1
    st.res = fn
    return p, st
