"""GPU parity of the residual, Jacobian, diffusion matrix and stencil SpMV against the FP64 oracle.

Tolerance (FP64 path): normwise 1e-10 relative per array, i.e.
max |gpu - oracle| <= 1e-10 max |oracle|.  The GPU evaluates |p|^beta and
|p|^gamma through one shared log|p| (a few ulp from libm's pow), far inside
the bound.
"""
import numpy as np
import pytest

from oracle import constitutive as cst
from oracle import discretization as disc
from paper_2112_05051_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SOIL = synth.Soil()
TOL = 1e-10


def _rb():
    from paper_2112_05051_gb300 import richards as rb
    rb.load()
    return rb


def _nrel(a, b):
    return np.abs(a - b).max() / max(np.abs(b).max(), 1e-300)


BCS = {
    "infiltration": synth.infiltration_bc(-20.7),
    "dirichlet": synth.BC(kind=(1,) * 6, value=(-30.0, -35.0, -25.0, -40.0, -50.0, -20.0)),
    "mixed": synth.BC(kind=(1, 0, 0, 1, 1, 0), value=(-22.0, 0, 0, -44.0, -61.5, 0)),
    "fields": None,
}


def _field_bc(grid):
    rng = np.random.default_rng(23)
    return synth.BC(kind=(1, 1, 0, 0, 0, 1), value=(-30.0, -40.0, 0, 0, 0, -20.0),
                    fields=(rng.uniform(-60, -10, grid.ny * grid.nz), None, None, None, None,
                            rng.uniform(-40, 0, grid.nx * grid.ny)))
GRIDS = [(7, 5, 6), (16, 16, 16), (33, 17, 9), (1, 1, 23), (19, 1, 1), (1, 1, 1)]


def _inputs(grid, seed, het=True):
    rng = np.random.default_rng(seed)
    p = rng.uniform(-70.0, -15.0, grid.n)
    p[:: 7] = p[:: 7] * 0 + 0.5  # a few saturated cells exercise the p >= 0 branch
    ks = synth.ks_field(grid, seed, 1.2, (3.0, 3.0, 2.0)) if het else None
    s_old = cst.saturation(p + rng.uniform(-5, 5, grid.n), SOIL)
    return p, ks, s_old


@pytest.mark.parametrize("kmean", [0, 1, 2, 3, synth.kmean_split(1, 2), synth.kmean_split(3, 0)])
@pytest.mark.parametrize("bcname", list(BCS))
@pytest.mark.parametrize("dims", GRIDS)
def test_residual_jacobian_parity(kmean, bcname, dims):
    rb = _rb()
    grid = synth.Grid(*dims, lx=1.0, ly=0.9, lz=1.3)
    bc = BCS[bcname] if bcname != "fields" else _field_bc(grid)
    p, ks, s_old = _inputs(grid, sum(dims) + kmean)
    dt = 0.8
    ctx = rb.Context(grid, SOIL, bc, kmean, ks)
    pd = torch.tensor(p, device="cuda")
    sd = torch.tensor(s_old, device="cuda")
    F = torch.empty_like(pd)
    norms = ctx.residual(pd, sd, dt, F)
    ref = disc.residual(grid, SOIL, bc, kmean, p, s_old, dt, ks)
    assert _nrel(F.cpu().numpy(), ref) <= TOL
    assert norms[0] == pytest.approx(np.linalg.norm(ref), rel=1e-12)
    assert norms[1] == pytest.approx(np.abs(ref).max(), rel=1e-12)
    J7 = torch.empty(7 * grid.n, dtype=torch.float64, device="cuda")
    A7 = torch.empty_like(J7)
    ctx.jacobian(pd, dt, J7, A7)
    Jref = disc.jacobian_stencil(grid, SOIL, bc, kmean, p, dt, ks)
    Aref = disc.aux_stencil(grid, SOIL, bc, kmean, p, dt, ks)
    Jg = J7.cpu().numpy().reshape(7, grid.n).T
    Ag = A7.cpu().numpy().reshape(7, grid.n).T
    for col in range(7):
        assert _nrel(Jg[:, col], Jref[:, col]) <= TOL or np.abs(Jref[:, col]).max() == 0
        assert _nrel(Ag[:, col], Aref[:, col]) <= TOL or np.abs(Aref[:, col]).max() == 0
    # zero pattern outside the grid is exact
    np.testing.assert_array_equal(Jg == 0, Jref == 0)
    x = np.random.default_rng(1).standard_normal(grid.n)
    y = torch.empty_like(pd)
    ctx.jacobian_apply(torch.tensor(x, device="cuda"), y)
    assert _nrel(y.cpu().numpy(), disc.jacobian(grid, SOIL, bc, kmean, p, dt, ks) @ x) <= TOL
    ctx.close()


def test_saturation_parity_and_invalid_arguments():
    rb = _rb()
    grid = synth.Grid(9, 8, 7)
    p, ks, _ = _inputs(grid, 3)
    ctx = rb.Context(grid, SOIL, synth.infiltration_bc(), 0, ks)
    pd = torch.tensor(p, device="cuda")
    s = torch.empty_like(pd)
    ctx.saturation(pd, s)
    assert _nrel(s.cpu().numpy(), cst.saturation(p, SOIL)) <= 1e-14
    with pytest.raises(rb.RichError) as e:
        ctx.residual(pd, s, 0.0, torch.empty_like(pd))
    assert e.value.status == -1
    with pytest.raises(rb.RichError) as e:
        ctx.jacobian_apply(pd, torch.empty_like(pd))
    assert e.value.status == -8
    ctx.close()


def test_full_size_residual_and_jacobian_128():
    rb = _rb()
    w = synth.WORKLOADS["richards128_fp64"]
    grid, soil, bc, ks, p0, dts = synth.workload_inputs(w)
    rng = np.random.default_rng(9)
    p = p0 + rng.uniform(0, 40, grid.n)
    s_old = cst.saturation(p0, soil)
    ctx = rb.Context(grid, soil, bc, w.kmean, ks)
    pd = torch.tensor(p, device="cuda")
    F = torch.empty_like(pd)
    ctx.residual(pd, torch.tensor(s_old, device="cuda"), dts[5], F)
    ref = disc.residual(grid, soil, bc, w.kmean, p, s_old, dts[5], ks)
    assert _nrel(F.cpu().numpy(), ref) <= TOL
    J7 = torch.empty(7 * grid.n, dtype=torch.float64, device="cuda")
    ctx.jacobian(pd, dts[5], J7, None)
    Jref = disc.jacobian_stencil(grid, soil, bc, w.kmean, p, dts[5], ks)
    Jg = J7.cpu().numpy().reshape(7, grid.n).T
    for col in range(7):
        assert _nrel(Jg[:, col], Jref[:, col]) <= TOL
    ctx.close()
