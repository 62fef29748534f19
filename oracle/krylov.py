"""Flexible Krylov solvers with right preconditioning, FP64 (oracle; test infrastructure).

The Newton correction solves J d = -Phi through the right-preconditioned
system J M^-1 (M d) = -Phi of eq. (precsystem), Sec. 3.  The paper uses
restarted GMRES; because the preconditioner is a V-cycle (a fixed linear
operator only in exact arithmetic and FP64), both solvers here are the
flexible variants, which keep the preconditioned directions:

  fgmres   Saad's flexible GMRES(m): Arnoldi on J Z with Z = B V stored,
           classical Gram-Schmidt with selective re-orthogonalisation (a
           second pass when ||w'||^2 < ||w||^2 / 2, the DGKS criterion),
           Givens rotations, restart every m iterations.
  fcg      Notay's flexible CG with truncation 1:
           z_k = B r_k, p_k = z_k - ((z_k, q_{k-1}) / (p_{k-1}, q_{k-1})) p_{k-1},
           q_k = J p_k, alpha_k = (p_k, r_k) / (p_k, q_k).

Both start from x0 = 0 and stop when ||b - J x||_2 <= eta ||b||_2.  FCG
reports failure (converged=False) when it reaches maxit, when (p, q) <= 0, or
when its residual norm grows above 10x the smallest seen; the Newton driver
then retries the solve with FGMRES(30).  With stall > 0 (an option of this
implementation, not the paper's; off by default) FGMRES also gives up after a
restart cycle that reduced the true residual norm by less than the fraction
stall of its value at the cycle's start, and FCG after a window of 30
iterations that did the same.
"""
import numpy as np


STALL_WINDOW = 30  # FCG iterations per stagnation test


def fcg(matvec, prec, b, eta, maxit, info=None, stall=0.0):
    """Returns (x, iterations, converged, residual history); info, if a dict, receives
    the reason of a failure: "maxit", "curvature" ((p, q) <= 0), "growth", or "stall"
    (stall > 0: after every STALL_WINDOW iterations, the residual norm is above
    (1 - stall) times its value STALL_WINDOW iterations earlier)."""
    if info is None:
        info = {}
    b = np.asarray(b, dtype=np.float64)
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b)
    if bnorm == 0.0:
        return x, 0, True, [0.0]
    r = b.copy()
    target = eta * bnorm
    hist = [bnorm]
    best = bnorm
    p_prev = q_prev = None
    pq_prev = None
    for k in range(1, maxit + 1):
        z = prec(r)
        if p_prev is None:
            p = z
        else:
            p = z - (np.dot(z, q_prev) / pq_prev) * p_prev
        q = matvec(p)
        pq = np.dot(p, q)
        if not pq > 0.0:
            info["reason"] = "curvature"
            return x, k, False, hist
        alpha = np.dot(p, r) / pq
        x = x + alpha * p
        r = r - alpha * q
        rn = np.linalg.norm(r)
        hist.append(rn)
        if rn <= target:
            return x, k, True, hist
        if rn > 10.0 * best:
            info["reason"] = "growth"
            return x, k, False, hist
        if stall > 0.0 and k % STALL_WINDOW == 0 and rn > (1.0 - stall) * hist[k - STALL_WINDOW]:
            info["reason"] = "stall"
            return x, k, False, hist
        best = min(best, rn)
        p_prev, q_prev, pq_prev = p, q, pq
    info["reason"] = "maxit"
    return x, maxit, False, hist


def fgmres(matvec, prec, b, eta, maxit, m, stall=0.0):
    b = np.asarray(b, dtype=np.float64)
    n = b.shape[0]
    bnorm = np.linalg.norm(b)
    x = np.zeros_like(b)
    if bnorm == 0.0:
        return x, 0, True, [0.0]
    target = eta * bnorm
    r = b.copy()
    beta = bnorm
    hist = [beta]
    its = 0
    while True:
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        j_done = 0
        converged = False
        for j in range(m):
            Z[j] = prec(V[j])
            w = matvec(Z[j])
            wn2 = float(w @ w)
            h1 = V[: j + 1] @ w
            w = w - h1 @ V[: j + 1]
            if float(w @ w) < 0.5 * wn2:
                h2 = V[: j + 1] @ w
                w = w - h2 @ V[: j + 1]
                h1 = h1 + h2
            H[: j + 1, j] = h1
            hn = np.linalg.norm(w)
            H[j + 1, j] = hn
            if hn > 0.0:
                V[j + 1] = w / hn
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            its += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]))
            if abs(g[j + 1]) <= target or hn == 0.0:
                converged = True
                break
            if its >= maxit:
                break
        y = np.zeros(j_done)
        for i in range(j_done - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1: j_done] @ y[i + 1: j_done]) / H[i, i]
        x = x + y @ Z[:j_done]
        if converged or its >= maxit:
            return x, its, converged, hist
        r = b - matvec(x)
        beta_cycle, beta = beta, np.linalg.norm(r)
        if beta <= target:
            return x, its, True, hist
        if stall > 0.0 and beta > (1.0 - stall) * beta_cycle:
            # the restart cycle reduced the true residual by less than the fraction stall
            return x, its, False, hist
