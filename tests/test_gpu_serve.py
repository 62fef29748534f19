"""Request server (rich_server_*) on the GPU.

A served request runs the same kernels as a lone rich_step on its own context,
so its status and pressure must equal the lone ones (pressure within 1e-12
relative, far inside the 1e-8 pressure bar) whatever else is in flight;
sessions continue from their resident state; admission keeps the reserved
device memory within the budget; requests overlap on the device.
"""
import numpy as np
import pytest

from paper_2112_05051_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SOIL = synth.Soil()


def _rb():
    from paper_2112_05051_gb300 import richards as rb
    rb.load()
    return rb


def _requests():
    """Mixed sizes, all four means, both precisions, seeded log-normal K_s fields."""
    dims = [(12, 12, 12), (16, 16, 16), (20, 18, 16), (24, 24, 24), (14, 22, 10), (16, 16, 16), (24, 20, 18),
            (10, 10, 30)]
    out = []
    for k, d in enumerate(dims):
        grid = synth.Grid(*d)
        ks = synth.ks_field(grid, 100 + k, 1.0, (4.0, 4.0, 2.0))
        out.append(dict(grid=grid, ks=ks, kmean=k % 4, prec=k % 2,
                        p0=np.full(grid.n, synth.P_INITIAL), dt=1.0))
    return out


def _opts(rb):
    return rb.default_newton_opts(kind=rb.KRYLOV_FCG, nu1=1, nu2=1, seed=3, smooth_levels=2)


def _alone(rb, q, steps=1, with_status=False):
    """Lone steps on a context of its own; a failed step leaves p at its last accepted iterate."""
    ctx = rb.Context(q["grid"], SOIL, synth.infiltration_bc(), q["kmean"], q["ks"], precision=q["prec"])
    p = torch.tensor(q["p0"], device="cuda")
    status = 0
    for _ in range(steps):
        try:
            ctx.step(p, q["dt"], _opts(rb))
        except rb.RichError as e:
            status = e.status
            break
    out = p.cpu().numpy()
    ctx.close()
    return (status, out) if with_status else out


def _rel(a, b):
    return np.abs(a - b).max() / np.abs(b).max()


def test_mixed_requests_equal_their_lone_results():
    rb = _rb()
    qs = _requests()
    alone = [_alone(rb, q, with_status=True) for q in qs]
    srv = rb.Server(slots=4)
    ids = [srv.submit(q["grid"], SOIL, synth.infiltration_bc(), q["kmean"], q["dt"], p0=q["p0"], ks=q["ks"],
                      precision=q["prec"], opts=_opts(rb)) for q in qs]
    res = [srv.wait(i) for i in ids]
    cnt = srv.counters()
    srv.close()
    # the same status and pressure as alone, for converged and failed steps alike
    for r, (st, a) in zip(res, alone):
        assert r["status"] == st
        assert _rel(r["p"], a) <= 1e-12
    # arithmetic and upstream means converge; the harmonic and geometric ones meet
    # negative Jacobian diagonals at the wet Dirichlet top on these fields, which the
    # AMG of the SPD diffusion matrix cannot precondition (the oracle fails alike)
    assert all(r["status"] == 0 for r, q in zip(res, qs) if q["kmean"] in (0, 1))
    assert cnt["admitted"] == len(qs)
    assert cnt["max_in_flight"] > 1  # several requests were on the device at once


def test_served_request_matches_the_oracle_step():
    from oracle import newton
    rb = _rb()
    w = synth.WORKLOADS["richards16_fp64"]
    grid, soil, bc, ks, p0, dts = synth.workload_inputs(w)
    opts = rb.default_newton_opts(kind=rb.KRYLOV_FCG, nu1=w.nu, nu2=w.nu, seed=w.amg_seed,
                                  smooth_levels=w.smooth_levels)
    srv = rb.Server(slots=2)
    rid = srv.submit(grid, soil, bc, w.kmean, dts[0], p0=p0, ks=ks, precision=rb.PREC_FP64, opts=opts)
    r = srv.wait(rid)
    srv.close()
    prob = newton.Problem(grid, soil, bc, w.kmean, ks)
    po, _ = newton.step(prob, p0.copy(), dts[0], newton.NewtonOptions(krylov="fcg", nu1=w.nu, nu2=w.nu,
                                                                       amg_seed=w.amg_seed,
                                                                       smooth_levels=w.smooth_levels))
    assert r["status"] == 0
    assert _rel(r["p"], po) <= 1e-8


def test_sessions_continue_from_their_resident_state():
    rb = _rb()
    # arithmetic-mean problems whose three steps converge in the oracle (8/8/5, 7/9/5,
    # 8/9/7 Newton iterations)
    qs = []
    for k, d in enumerate([(12, 12, 12), (14, 22, 10), (16, 16, 16)]):
        grid = synth.Grid(*d)
        qs.append(dict(grid=grid, ks=synth.ks_field(grid, 200 + k, 1.0, (4.0, 4.0, 2.0)), kmean=0, prec=k % 2,
                       p0=np.full(grid.n, synth.P_INITIAL), dt=1.0))
    srv = rb.Server(slots=3)
    last = {}
    for step in range(3):
        ids = []
        for k, q in enumerate(qs):
            ids.append(srv.submit(q["grid"], SOIL, synth.infiltration_bc(), q["kmean"], q["dt"],
                                  p0=q["p0"] if step == 0 else None, ks=q["ks"] if step == 0 else None,
                                  precision=q["prec"], opts=_opts(rb), session=50 + k))
        for k, i in enumerate(ids):
            r = srv.wait(i)
            assert r["status"] == 0
            last[k] = r["p"]
    srv.close()
    for k, q in enumerate(qs):
        assert _rel(last[k], _alone(rb, q, steps=3)) <= 1e-12


def test_admission_keeps_reserved_memory_within_the_budget():
    rb = _rb()
    grid = synth.Grid(24, 24, 24)
    ks = synth.ks_field(grid, 7, 1.0, (4.0, 4.0, 2.0))
    p0 = np.full(grid.n, synth.P_INITIAL)
    opts = _opts(rb)
    # the server's estimate of one such request, read back from a first run
    probe = rb.Server(slots=1)
    est = probe.wait(probe.submit(grid, SOIL, synth.infiltration_bc(), 0, 1.0, p0=p0, ks=ks,
                                  opts=opts))["mem_estimate"]
    probe.close()
    budget = 2.5 * est
    srv = rb.Server(slots=6, mem_budget_bytes=budget)
    ids = [srv.submit(grid, SOIL, synth.infiltration_bc(), 0, 1.0, p0=p0, ks=ks, opts=opts) for _ in range(6)]
    res = [srv.wait(i) for i in ids]
    cnt = srv.counters()
    srv.close()
    assert all(r["status"] == 0 for r in res)
    assert all(r["mem_in_flight"] <= budget for r in res)
    assert cnt["max_in_flight"] <= 2
    first = res[0]["p"]
    assert all(_rel(r["p"], first) <= 1e-12 for r in res)
    srv2 = rb.Server(slots=1, mem_budget_bytes=0.5 * est)
    try:  # a request larger than the whole budget is refused at submit
        with pytest.raises(rb.RichError) as e:
            srv2.submit(grid, SOIL, synth.infiltration_bc(), 0, 1.0, p0=p0, ks=ks, opts=opts)
        assert e.value.status == -9
    finally:
        srv2.close()


def test_sessions_beyond_the_limit_are_evicted_least_recently_used_first():
    rb = _rb()
    grid = synth.Grid(12, 12, 12)
    ks = synth.ks_field(grid, 3, 1.0, (4.0, 4.0, 2.0))
    p0 = np.full(grid.n, synth.P_INITIAL)
    bc = synth.infiltration_bc()
    srv = rb.Server(slots=1, max_sessions=1)

    def run(session, first):
        return srv.wait(srv.submit(grid, SOIL, bc, 0, 1.0, p0=p0 if first else None, ks=ks if first else None,
                                   opts=_opts(rb), session=session))

    assert run(1, True)["status"] == 0
    assert run(1, False)["status"] == 0          # session 1 resident: continues
    assert run(2, True)["status"] == 0           # a second session evicts session 1
    assert run(1, False)["status"] == -8         # RICH_ESTATE: nothing left to continue from
    r = run(2, False)                            # the failed request kept nothing: session 2 was evicted
    assert r["status"] == -8
    r1 = run(1, True)                            # starting again from p0 works
    r2 = run(1, False)
    srv.close()
    assert r1["status"] == 0 and r2["status"] == 0
    q = dict(grid=grid, ks=ks, kmean=0, prec=1, p0=p0, dt=1.0)
    assert _rel(r2["p"], _alone(rb, q, steps=2)) <= 1e-12
