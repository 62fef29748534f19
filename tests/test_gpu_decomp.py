"""Slab decomposition on the GPU (Sec. 5.1): the blocks of a split grid, each a
context of its own with interface faces, run one after another on one device
(no kernel waits on another block: the host exchanges the halos between the
launches), reproduce the whole grid.

* the face-pack kernel writes the cells next to a face in the face layout;
* after a halo exchange of p, the blocks' residuals put together are the whole
  grid's residual bit for bit (the interface ghost's conductivity is evaluated
  by the same constitutive code as an interior neighbour's), and the oracle's
  within 1e-12; the whole grid's norms follow from the blocks' pieces;
* the blocks' J and A_aux (7 planes each) are the whole grid's rows, the
  couplings across an interface kept in the plane of that face;
* J x of the split grid (each block's stencil SpMV plus its interface couplings
  times the neighbours' x after a halo exchange of x) is the whole grid's J x
  within 1e-14 (the terms are summed in another order);
* the split grid's Newton step and Krylov solves reach the whole grid's, and
  near a steady state stop at the same round-off floor.
"""
import math

import numpy as np
import pytest

from oracle import constitutive as cst, discretization as disc
from paper_2112_05051_gb300 import decomp, synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SOIL = synth.Soil()


def _rb():
    from paper_2112_05051_gb300 import richards as rb
    rb.load()
    return rb


def _state(grid, seed):
    rng = np.random.default_rng(seed)
    z = (np.arange(grid.nz) + 1.0) / (grid.nz + 1)
    front = -61.5 + 40.8 * np.exp(-(1.0 - z) / 0.2)
    p = np.broadcast_to(front[:, None, None], grid.shape).ravel() + rng.uniform(-0.5, 0.5, grid.n)
    return p


def _blocks_of(a, grid, blocks):
    a3 = np.asarray(a).reshape(grid.shape)
    return [np.ascontiguousarray(decomp.cell_block(a3, b)).ravel() for b in blocks]


def _whole(parts, grid, blocks, planes=1):
    out = np.empty((planes,) + grid.shape)
    for b, x in zip(blocks, parts):
        out[:, :, b.j0:b.j1, b.i0:b.i1] = x.reshape((planes, grid.nz, b.j1 - b.j0, b.i1 - b.i0))
    return out.reshape(planes, -1) if planes > 1 else out.ravel()


def test_pack_face_kernel_layout():
    rb = _rb()
    grid = synth.Grid(7, 5, 4)
    ctx = rb.Context(grid, SOIL, synth.infiltration_bc(), 0, None)
    a3 = np.arange(grid.n, dtype=np.float64).reshape(grid.shape)
    x = torch.tensor(a3.ravel(), device="cuda")
    want = [a3[:, :, 0], a3[:, :, -1], a3[:, 0, :], a3[:, -1, :], a3[0], a3[-1]]
    for f in range(6):
        out = torch.empty(decomp.face_cells(grid, f), dtype=torch.float64, device="cuda")
        ctx.pack_face(f, x, out)
        np.testing.assert_array_equal(out.cpu().numpy(), want[f].ravel())
    ctx.close()


@pytest.mark.parametrize("px,py,kmean,paper_bc", [(2, 2, synth.KMEAN_UPSTREAM, False), (3, 1, synth.KMEAN_ARITH, True),
                                                  (2, 3, synth.KMEAN_HARMONIC, False)])
def test_blocks_reproduce_the_whole_grid(px, py, kmean, paper_bc):
    rb = _rb()
    grid = synth.Grid(24, 20, 12)
    bc = synth.paper_infiltration_bc(grid, -30.0) if paper_bc else synth.infiltration_bc()
    ks = synth.ks_field(grid, 8, 1.0, (3.0, 3.0, 2.0))
    p = _state(grid, 5)
    s_old = cst.saturation(p - 1.0, SOIL)
    dt = 0.7
    # the whole grid on the GPU and in the oracle
    whole = rb.Context(grid, SOIL, bc, kmean, ks)
    pd = torch.tensor(p, device="cuda")
    F = torch.empty_like(pd)
    n2, ninf = whole.residual(pd, torch.tensor(s_old, device="cuda"), dt, F)
    Fw = F.cpu().numpy()
    F3 = torch.empty_like(pd)
    n2_3, ninf_3, nm = whole.residual3(pd, torch.tensor(s_old, device="cuda"), dt, F3)
    assert (n2_3, ninf_3) == (n2, ninf)
    np.testing.assert_array_equal(F3.cpu().numpy(), Fw)
    J7 = torch.empty(7 * grid.n, dtype=torch.float64, device="cuda")
    A7 = torch.empty_like(J7)
    whole.jacobian(pd, dt, J7, A7)
    J7w, A7w = J7.cpu().numpy().reshape(7, -1), A7.cpu().numpy().reshape(7, -1)
    x = np.random.default_rng(11).standard_normal(grid.n)
    yw = torch.empty_like(pd)
    whole.jacobian_apply(torch.tensor(x, device="cuda"), yw)
    yw = yw.cpu().numpy()
    whole.close()
    ref, ref_m = disc.residual(grid, SOIL, bc, kmean, p, s_old, dt, ks, with_scale=True)
    assert abs(nm - ref_m) <= 1e-12 * ref_m  # the round-off scale ||m||_2 of the Newton test
    # the blocks, one context each, on this device
    blocks = decomp.partition(grid, px, py)
    probs = [decomp.BlockProblem(grid, SOIL, bc, kmean, ks, blocks, r) for r in range(len(blocks))]
    pb = [torch.tensor(x, device="cuda") for x in _blocks_of(p, grid, blocks)]
    sb = [torch.tensor(x, device="cuda") for x in _blocks_of(s_old, grid, blocks)]
    decomp.exchange_blocks(probs, pb)
    Fb, parts, Jb, Ab = [], [], [], []
    for q, pq, so in zip(probs, pb, sb):
        f = torch.empty_like(pq)
        parts.append(q.residual(pq, so, dt, f))
        Fb.append(f.cpu().numpy())
        jb = torch.empty(7 * pq.numel(), dtype=torch.float64, device="cuda")
        ab = torch.empty_like(jb)
        q.ctx.jacobian(pq, dt, jb, ab)
        Jb.append(jb.cpu().numpy())
        Ab.append(ab.cpu().numpy())
    # J x of the split grid: local stencil SpMV, then the interface couplings times
    # the neighbours' x after a halo exchange of x
    xb = [torch.tensor(v, device="cuda") for v in _blocks_of(x, grid, blocks)]
    yb = [torch.empty_like(v) for v in xb]
    decomp.apply_J_blocks(probs, xb, yb)
    ys = _whole([y.cpu().numpy() for y in yb], grid, blocks)
    assert np.abs(ys - yw).max() <= 1e-14 * np.abs(yw).max()
    # the A_aux coupling of one interface face alone: plane f of A_aux times the ghosts
    q, b = probs[0], blocks[0]
    f = next(f for f in range(4) if b.nbr[f] >= 0)
    ghost = torch.tensor(np.ascontiguousarray(decomp.ghost_plane(x.reshape(grid.shape), b, f)).ravel(), device="cuda")
    y0 = torch.zeros_like(xb[0])
    q.ctx.face_apply(f, 1, ghost, y0)
    sg = q.grid
    a3 = Ab[0].reshape(7, sg.nz, sg.ny, sg.nx)[1 + f]
    face = [a3[:, :, 0], a3[:, :, -1], a3[:, 0, :], a3[:, -1, :]][f].ravel() * ghost.cpu().numpy()
    y03 = y0.cpu().numpy().reshape(sg.nz, sg.ny, sg.nx)
    got = [y03[:, :, 0], y03[:, :, -1], y03[:, 0, :], y03[:, -1, :]][f].ravel()
    np.testing.assert_array_equal(got, face)
    assert np.count_nonzero(y03) == np.count_nonzero(got)  # nothing but the face cells
    for q in probs:
        q.close()
    Fs = _whole(Fb, grid, blocks)
    np.testing.assert_array_equal(Fs, Fw)  # bit for bit
    assert np.abs(Fs - ref).max() <= 1e-12 * np.abs(ref).max()
    n2s, ninfs = decomp.combine_norms(parts)
    assert abs(n2s - n2) <= 1e-13 * n2 and ninfs == ninf
    nms = math.sqrt(sum(pt[2] for pt in parts))  # the blocks' m^2 add up to the whole grid's
    assert abs(nms - nm) <= 1e-13 * nm
    np.testing.assert_array_equal(_whole(Jb, grid, blocks, 7), J7w)
    np.testing.assert_array_equal(_whole(Ab, grid, blocks, 7), A7w)


def test_interface_faces_need_their_ghost_pressures():
    rb = _rb()
    grid = synth.Grid(6, 6, 4)
    bad = synth.BC(kind=(rb.BC_INTERFACE, 0, 0, 0, 0, 1), value=(0.0,) * 5 + (-20.0,))  # no per-cell field
    with pytest.raises(rb.RichError):
        rb.Context(grid, SOIL, bad, 0, None)
    ctx = rb.Context(grid, SOIL, synth.infiltration_bc(), 0, None)
    with pytest.raises(rb.RichError):  # the face was created without per-cell values
        ctx.set_face_values(0, torch.zeros(grid.ny * grid.nz, dtype=torch.float64, device="cuda"))
    ctx.close()


@pytest.mark.parametrize("px,py,kmean,kind", [(2, 2, synth.KMEAN_UPSTREAM, "fcg"), (3, 1, synth.KMEAN_ARITH, "fcg"),
                                              (2, 2, synth.KMEAN_UPSTREAM, "fgmres")])
def test_split_grid_newton_step_matches_the_whole_grid(px, py, kmean, kind):
    """One backward-Euler step of the split grid (halo exchanges, FCG preconditioned
    by each block's own hierarchy, sums over the blocks) converges to the whole
    grid's step: the preconditioners differ (decoupled aggregation), so the Krylov
    iterates do, and the pressures agree within the converged-step tolerance."""
    rb = _rb()
    grid = synth.Grid(24, 20, 12)
    bc = synth.infiltration_bc()
    ks = synth.ks_field(grid, 6, 0.5, (4.0, 4.0, 2.0))
    p0 = np.full(grid.n, synth.P_INITIAL)
    dt = 0.25
    k = rb.KRYLOV_FCG if kind == "fcg" else rb.KRYLOV_FGMRES
    opts = rb.default_newton_opts(kind=k, restart=30, seed=3, coarse_max=100, smooth_levels=2)
    whole = rb.Context(grid, SOIL, bc, kmean, ks)
    pw = torch.tensor(p0, device="cuda")
    st = whole.step(pw, dt, opts)
    whole.close()
    assert st.converged and st.fallbacks == 0
    blocks = decomp.partition(grid, px, py)
    probs = [decomp.BlockProblem(grid, SOIL, bc, kmean, ks, blocks, r) for r in range(len(blocks))]
    pb = [torch.tensor(v, device="cuda") for v in _blocks_of(p0, grid, blocks)]
    ok, its, lin, why = decomp.newton_step(probs, decomp.LocalComm(probs), pb, dt, opts)
    assert ok, why
    assert abs(its - st.newton_its) <= 1
    ps = _whole([v.cpu().numpy() for v in pb], grid, blocks)
    pwh = pw.cpu().numpy()
    assert np.abs(ps - pwh).max() <= 1e-8 * np.abs(pwh).max()
    for q in probs:
        q.close()


@pytest.mark.parametrize("perturb", [0.0, 1e-9])
def test_split_grid_step_stops_at_the_round_off_floor(perturb):
    """Near a steady state the Newton test's round-off floor (eps ||m||_2, from the
    blocks' summed m^2) decides, on the split grid as on the whole grid: the
    hydrostatic column (arithmetic mean: Phi is rounding noise, ~0.02 of the floor)
    needs no iteration, and perturbed by 1e-9 cm it needs one, after which
    ||Phi|| is below the floor but far above rtol ||Phi_0||, which rounding alone
    keeps out of reach."""
    rb = _rb()
    grid = synth.Grid(16, 16, 10)
    hz = grid.h[2]
    z = (np.arange(grid.nz) + 1) * hz
    p0 = np.broadcast_to((-12.0 - z)[:, None, None], grid.shape).ravel().copy()
    p0 = p0 + perturb * np.random.default_rng(4).standard_normal(grid.n)
    bc = synth.BC(kind=(0, 0, 0, 0, 0, 1), value=(0, 0, 0, 0, 0, -12.0 - (grid.nz + 1) * hz))
    ks = synth.ks_field(grid, 2, 0.5, (3.0, 3.0, 2.0))
    kmean, dt = synth.KMEAN_ARITH, 0.25
    opts = rb.default_newton_opts(kind=rb.KRYLOV_FCG, seed=3, coarse_max=100, smooth_levels=2)
    whole = rb.Context(grid, SOIL, bc, kmean, ks)
    pw = torch.tensor(p0, device="cuda")
    st = whole.step(pw, dt, opts)
    whole.close()
    assert st.converged and st.newton_its == (0 if perturb == 0 else 1)
    assert st.res > opts.rtol * st.res0  # the floor, not rtol, ended the step
    blocks = decomp.partition(grid, 2, 2)
    probs = [decomp.BlockProblem(grid, SOIL, bc, kmean, ks, blocks, r) for r in range(len(blocks))]
    pb = [torch.tensor(v, device="cuda") for v in _blocks_of(p0, grid, blocks)]
    ok, its, lin, why = decomp.newton_step(probs, decomp.LocalComm(probs), pb, dt, opts)
    assert ok, why
    assert its == st.newton_its
    ps = _whole([v.cpu().numpy() for v in pb], grid, blocks)
    pwh = pw.cpu().numpy()
    if perturb == 0:
        np.testing.assert_array_equal(ps, p0)
    assert np.abs(ps - pwh).max() <= 1e-12 * np.abs(pwh).max()
    for q in probs:
        q.close()


@pytest.mark.parametrize("kind", ["fcg", "fgmres"])
def test_split_grid_krylov_solves_the_whole_grids_system(kind):
    """FCG and FGMRES(10) on the split grid solve the whole grid's J x = b to their
    tolerance."""
    rb = _rb()
    grid = synth.Grid(20, 18, 10)
    bc = synth.infiltration_bc()
    ks = synth.ks_field(grid, 2, 0.5, (4.0, 4.0, 2.0))
    p = _state(grid, 3)
    dt = 0.5
    blocks = decomp.partition(grid, 2, 2)
    probs = [decomp.BlockProblem(grid, SOIL, bc, synth.KMEAN_UPSTREAM, ks, blocks, r) for r in range(len(blocks))]
    comm = decomp.LocalComm(probs)
    pb = [torch.tensor(v, device="cuda") for v in _blocks_of(p, grid, blocks)]
    comm.exchange(pb)
    for q, x in zip(probs, pb):
        q.ctx.jacobian(x, dt)
        q.ctx.amg_setup(rb.default_amg_opts(seed=3, coarse_max=50))
    b = np.random.default_rng(4).standard_normal(grid.n)
    bb = [torch.tensor(v, device="cuda") for v in _blocks_of(b, grid, blocks)]
    if kind == "fcg":
        x, its, ok, why = decomp.fcg(probs, comm, bb, 1e-10, 400)
    else:
        x, its, ok, why = decomp.fgmres(probs, comm, bb, 1e-10, 400, 10)
    assert ok, why
    J = disc.jacobian(grid, SOIL, bc, synth.KMEAN_UPSTREAM, p, dt, ks)
    xs = _whole([v.cpu().numpy() for v in x], grid, blocks)
    assert np.linalg.norm(J @ xs - b) <= 1e-10 * np.linalg.norm(b) * 1.0001
    for q in probs:
        q.close()
