"""GPU parity of time-step control and of the harmonic-mean failure, against the FP64 oracle.

Time-step control (rich_newton_opts.max_dt_halvings) is host logic around the
step: the GPU and the oracle must take the same substeps, discard the same
attempts and reach the same pressure (1e-8 relative).  The 256^3 harmonic
workload (sigma 1.5) fails on both sides at a reduced grid, with and without
control: its exact Jacobian has negative diagonal entries under the wet top face.
"""
import numpy as np
import pytest

from oracle import constitutive as cst
from oracle import discretization as disc
from oracle import newton
from paper_2112_05051_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SOIL = synth.Soil()


def _rb():
    from paper_2112_05051_gb300 import richards as rb
    rb.load()
    return rb


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


@pytest.mark.parametrize("prec", [0, 1])
def test_time_step_control_takes_the_oracles_substeps(prec):
    rb = _rb()
    grid = synth.Grid(12, 12, 12)
    ks = synth.ks_field(grid, 1000, 1.0)
    bc = synth.infiltration_bc(synth.P_TOP)
    p0 = np.full(grid.n, synth.P_INITIAL)
    opts = rb.default_newton_opts(kind=rb.KRYLOV_FCG, seed=1, coarse_max=100, max_dt_halvings=10)
    ctx = rb.Context(grid, SOIL, bc, synth.KMEAN_HARMONIC, ks, precision=prec)
    pd = torch.tensor(p0, device="cuda")
    st = ctx.step(pd, 1.0, opts)
    prob = newton.Problem(grid, SOIL, bc, synth.KMEAN_HARMONIC, ks)
    po, ost = newton.advance(prob, p0, 1.0, newton.NewtonOptions(krylov="fcg", amg_seed=1, coarse_max=100,
                                                                  max_dt_halvings=10))
    assert st.converged and ost.converged
    assert st.substeps == ost.substeps and st.dt_failures == ost.dt_failures and st.dt_min == ost.dt_min
    assert st.substeps > 1
    if prec == 0:
        assert st.newton_its == ost.newton_its
    assert _rel(pd.cpu().numpy(), po) <= 1e-8
    # a second step of the same length needs no cut any more
    st2 = ctx.step(pd, 1.0, opts)
    po2, ost2 = newton.advance(prob, po, 1.0, newton.NewtonOptions(krylov="fcg", amg_seed=1, coarse_max=100,
                                                                    max_dt_halvings=10))
    assert st2.substeps == ost2.substeps
    assert _rel(pd.cpu().numpy(), po2) <= 1e-8
    ctx.close()


def test_harmonic_workload_fails_on_both_sides_at_a_reduced_grid():
    rb = _rb()
    w = synth.WORKLOADS["richards256_mixed"]
    grid, soil, bc, ks, p0, dts = synth.workload_inputs(w, 12)
    dt = dts[0]
    # the exact Jacobian is indefinite: negative diagonal entries under the wet top face
    ctx = rb.Context(grid, soil, bc, w.kmean, ks, precision=rb.PREC_MIXED)
    pd = torch.tensor(p0, device="cuda")
    J7 = torch.empty(7 * grid.n, dtype=torch.float64, device="cuda")
    ctx.jacobian(pd, dt, J7=J7)
    diag = J7[:grid.n].cpu().numpy()
    Jo = disc.jacobian(grid, soil, bc, w.kmean, p0, dt, ks)
    np.testing.assert_array_equal(diag < 0, Jo.diagonal() < 0)
    neg = np.flatnonzero(diag < 0)
    assert len(neg) > 0 and np.all(neg // (grid.nx * grid.ny) == grid.nz - 1)  # all in the top layer
    lam_min = np.linalg.eigvals(Jo.toarray()).real.min()
    assert lam_min < 0  # a dense eigensolve: J is not positive definite
    opt_o = newton.NewtonOptions(krylov="fcg", amg_seed=w.amg_seed, coarse_max=100, smooth_levels=2)
    for halvings in (0, 6):
        opts = rb.default_newton_opts(kind=rb.KRYLOV_FCG, seed=w.amg_seed, coarse_max=100, smooth_levels=2,
                                      max_dt_halvings=halvings)
        pd = torch.tensor(p0, device="cuda")
        st = rb.StepStats()
        s = rb.load().rich_step(ctx.h, rb._ptr(pd), dt, rb.ctypes.byref(opts), rb.ctypes.byref(st))
        assert s == -4  # RICH_ENOTCONV_LIN
        opt_o.max_dt_halvings = halvings
        with pytest.raises(newton.LinearSolveError):
            newton.advance(newton.Problem(grid, soil, bc, w.kmean, ks), p0, dt, opt_o)
        if halvings:
            assert st.dt_failures == halvings + 1
        # the pressure is left at the start of the failed (sub)step
        np.testing.assert_array_equal(pd.cpu().numpy(), p0)
    ctx.close()
