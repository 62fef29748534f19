"""Batched steps (rich_create_batch / rich_step_batch) and the server's packed launches (GPU).

A batch stacks problems of one grid shape along z and steps them with one launch
per operation; Newton and FCG keep their scalars per problem.  Each problem's
result must be its lone result within the pressure tolerance of a converged step
(1e-8 relative; the batch's AMG hierarchy is built on all problems at once, so
its Krylov iterates differ from a lone run's at rounding level), and the FP64
oracle's within the same bar.  A problem that fails does not hold the others back.
"""
import numpy as np
import pytest

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
    return float(np.abs(a - b).max() / np.abs(b).max())


def _opts(rb, **kw):
    return rb.default_newton_opts(kind=rb.KRYLOV_FCG, seed=3, coarse_max=100, smooth_levels=2, **kw)


def _lone(rb, grid, kmean, ks, p0, dt, prec, dt2=None):
    """A lone step (and, with dt2, a second one on the same context): (status, stats, p) per step."""
    ctx = rb.Context(grid, SOIL, synth.infiltration_bc(), kmean, ks, precision=prec)
    pd = torch.tensor(p0, device="cuda")
    s, st = ctx.step(pd, dt, _opts(rb), check_status=False)
    out = [(s, st, pd.cpu().numpy())]
    if dt2 is not None and s == 0:
        s2, st2 = ctx.step(pd, dt2, _opts(rb), check_status=False)
        out.append((s2, st2, pd.cpu().numpy()))
    ctx.close()
    return out if dt2 is not None else out[0]


@pytest.mark.parametrize("kmean,prec", [(synth.KMEAN_ARITH, 0), (synth.KMEAN_UPSTREAM, 1)])
def test_batch_equals_lone_steps_and_the_oracle(kmean, prec):
    # Fields (sigma 0.5) and steps (dt 0.25, twice) on which the oracle's FCG needs
    # no FGMRES fallback for any of the three problems: a batch has no fallback, and
    # its hierarchy (built on all problems at once) differs from a lone one, so on
    # inputs where FCG is near breakdown the two could part ways.
    rb = _rb()
    grid = synth.Grid(14, 13, 12)
    fields = [synth.ks_field(grid, 40 + b, 0.5, (4.0, 4.0, 2.0)) for b in range(3)]
    p0 = np.full(grid.n, synth.P_INITIAL)
    dt = 0.25
    bctx = rb.BatchContext(grid, 3, SOIL, synth.infiltration_bc(), kmean, np.concatenate(fields), precision=prec)
    pb = torch.tensor(np.tile(p0, 3), device="cuda")
    status, stats = bctx.step_batch(pb, dt, _opts(rb))
    assert status == [0, 0, 0]
    step1 = pb.cpu().numpy().reshape(3, grid.n)
    # a second step of the batch reuses its hierarchy (numeric refresh)
    status2, stats2 = bctx.step_batch(pb, dt, _opts(rb))
    assert status2 == [0, 0, 0] and all(s.amg_setups == 0 for s in stats2)
    step2 = pb.cpu().numpy().reshape(3, grid.n)
    bctx.close()
    for b in range(3):
        (s, st, pl), (s2, st2, pl2) = _lone(rb, grid, kmean, fields[b], p0, dt, prec, dt2=dt)
        assert s == 0 and s2 == 0
        assert _rel(step1[b], pl) <= 1e-8 and _rel(step2[b], pl2) <= 1e-8
        assert abs(stats[b].newton_its - st.newton_its) <= 1 and stats[b].converged
        po, ost = newton.step(newton.Problem(grid, SOIL, synth.infiltration_bc(), kmean, fields[b]), p0, dt,
                              newton.NewtonOptions(krylov="fcg", amg_seed=3, coarse_max=100, smooth_levels=2))
        assert ost.fallbacks == 0
        assert _rel(step1[b], po) <= 1e-8


def test_a_failing_problem_does_not_hold_the_batch_back():
    rb = _rb()
    grid = synth.Grid(12, 12, 12)
    good = synth.ks_field(grid, 7, 1.0, (4.0, 4.0, 2.0))
    bad = synth.ks_field(grid, 3, 1.5)  # harmonic mean on this field: indefinite J at the wet top
    p0 = np.full(grid.n, synth.P_INITIAL)
    for kmean in (synth.KMEAN_HARMONIC,):
        bctx = rb.BatchContext(grid, 2, SOIL, synth.infiltration_bc(), kmean, np.concatenate([good, bad]),
                               precision=1)
        pb = torch.tensor(np.tile(p0, 2), device="cuda")
        status, stats = bctx.step_batch(pb, 1.0, _opts(rb))
        s_good, _, p_good = _lone(rb, grid, kmean, good, p0, 1.0, 1)
        s_bad, _, _ = _lone(rb, grid, kmean, bad, p0, 1.0, 1)
        assert s_bad != 0 and status[1] != 0  # fails alone and in the batch
        assert status[0] == s_good
        if s_good == 0:
            assert _rel(pb.cpu().numpy()[:grid.n], p_good) <= 1e-8
        bctx.close()


def test_batch_rejects_options_it_cannot_run():
    rb = _rb()
    grid = synth.Grid(6, 6, 6)
    bctx = rb.BatchContext(grid, 2, SOIL, synth.infiltration_bc(), 0, None)
    pb = torch.tensor(np.full(2 * grid.n, -40.0), device="cuda")
    with pytest.raises(rb.RichError):
        bctx.step_batch(pb, 1.0, rb.default_newton_opts(kind=rb.KRYLOV_FGMRES))
    with pytest.raises(rb.RichError):
        bctx.step_batch(pb, 1.0, rb.default_newton_opts(max_dt_halvings=3))
    bctx.close()
    with pytest.raises(rb.RichError):  # per-cell values on an x face cannot be stacked
        rb.BatchContext(grid, 2, SOIL, synth.BC(kind=(1, 0, 0, 0, 0, 1), value=(-30.0, 0, 0, 0, 0, -20.0),
                                               fields=(np.full(36, -30.0), None, None, None, None, None)), 0, None)


def test_server_packs_same_shape_requests_and_matches_lone_results():
    rb = _rb()
    grid = synth.Grid(12, 12, 12)
    p0 = np.full(grid.n, synth.P_INITIAL)
    opts = _opts(rb)
    qs = [(synth.ks_field(grid, 60 + i, 1.0, (4.0, 4.0, 2.0)), i % 2) for i in range(8)]
    srv = rb.Server(slots=1, batch_max=4)
    ids = [srv.submit(grid, SOIL, synth.infiltration_bc(), km, 1.0, p0=p0, ks=ks, precision=1, opts=opts)
           for ks, km in qs]
    res = [srv.wait(i) for i in ids]
    srv.close()
    assert max(r["batch_size"] for r in res) > 1  # one slot and eight queued requests: packed
    for (ks, km), r in zip(qs, res):
        s, st, pl = _lone(rb, grid, km, ks, p0, 1.0, 1)
        assert r["status"] == s
        if s == 0:
            assert _rel(r["p"], pl) <= 1e-8
