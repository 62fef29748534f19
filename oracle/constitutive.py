"""Constitutive laws of the Celia/Haverkamp soil model, FP64 (oracle; test infrastructure).

s(p)  = alpha (S_s - S_r) / (alpha + |p|^beta) + S_r          eq. (s(p)), Sec. 2
K(p)  = K_s a / (a + |p|^gamma)                                eq. (K(p)), Sec. 2
s'(p) = -alpha beta |p|^(beta-1) sgn(p) (S_s-S_r)/(alpha+|p|^beta)^2
K'(p) = -a gamma K_s |p|^(gamma-1) sgn(p) / (a+|p|^gamma)^2     eq. (derivativeofcoefficients), Sec. 3

The laws hold for p < 0 only; for p >= 0 the medium is saturated and the
paper sets K = K_s and s = S_s (Sec. 2, text after Fig. 1 of the model), so
the oracle clamps there with zero derivatives.  Both laws are continuous at
p = 0.  ``ks`` may be a scalar or a per-cell array (heterogeneous field).
"""
import numpy as np


def _abs_neg(p):
    p = np.asarray(p, dtype=np.float64)
    return p, np.abs(p), p < 0.0


def saturation(p, soil):
    p, ap, unsat = _abs_neg(p)
    val = soil.alpha * (soil.theta_s - soil.theta_r) / (soil.alpha + ap ** soil.beta) + soil.theta_r
    return np.where(unsat, val, soil.theta_s)


def dsaturation(p, soil):
    p, ap, unsat = _abs_neg(p)
    sgn = np.sign(p)
    val = -(soil.alpha * soil.beta * ap ** (soil.beta - 1.0) * sgn * (soil.theta_s - soil.theta_r)
            / (soil.alpha + ap ** soil.beta) ** 2)
    return np.where(unsat, val, 0.0)


def conductivity(p, soil, ks):
    p, ap, unsat = _abs_neg(p)
    ks = np.broadcast_to(np.asarray(ks, dtype=np.float64), p.shape)
    val = ks * soil.a / (soil.a + ap ** soil.gamma)
    return np.where(unsat, val, ks)


def dconductivity(p, soil, ks):
    p, ap, unsat = _abs_neg(p)
    ks = np.broadcast_to(np.asarray(ks, dtype=np.float64), p.shape)
    sgn = np.sign(p)
    val = -(soil.a * soil.gamma * ks * ap ** (soil.gamma - 1.0) * sgn / (soil.a + ap ** soil.gamma) ** 2)
    return np.where(unsat, val, 0.0)
