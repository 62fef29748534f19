"""rich_residual_noalloc against rich_residual (GPU).

rich_residual_noalloc serves callers that cannot allocate device memory when
they need a residual (fixed memory budget, a foreign allocator, no implicit
synchronisation allowed): it takes inputs and outputs only and keeps its
scratch in a fixed device array.  It must give the same Phi and norms as the
context-based rich_residual, call after call (the shared scratch must not carry
state from one call into the next).  This file is collected last on purpose.
"""
import numpy as np
import pytest

from paper_2112_05051_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = 1e-10  # normwise, as for every FP64 residual parity test


def test_noalloc_residual_matches_context_residual_twice():
    from paper_2112_05051_gb300 import richards as rb
    rb.load()
    soil = synth.Soil()
    grid = synth.Grid(37, 29, 23)
    ks = synth.ks_field(grid, 11, 1.3, (4.0, 4.0, 2.0))
    ksd = torch.tensor(ks, device="cuda")
    rng = np.random.default_rng(5)
    # (bc, kmean, dt, heterogeneous K_s, norms wanted): constant and per-cell Dirichlet
    # values (the paper's infiltration faces, read in place), all four means, a device
    # K_s field and the constant K_s (NULL field), with and without the norms
    cases = [(synth.infiltration_bc(), synth.KMEAN_UPSTREAM, 0.7, True, True),
             (synth.BC(kind=(1, 0, 1, 0, 1, 1), value=(-25.0, 0, -33.0, 0, -61.5, -20.7)), synth.KMEAN_HARMONIC, 3.0,
              True, True),
             (synth.paper_infiltration_bc(grid, -61.5), synth.KMEAN_ARITH, 0.2, False, True),
             (synth.paper_infiltration_bc(grid, -40.0), synth.KMEAN_GEOMETRIC, 1.5, True, False),
             (synth.all_dirichlet_bc(-30.0), synth.KMEAN_ARITH, 2.0, False, False)]
    for bc, kmean, dt, het, norms in cases:  # calls in a row, different inputs
        p = torch.tensor(rng.uniform(-70.0, -15.0, grid.n), device="cuda")
        s_old = torch.tensor(rng.uniform(0.08, 0.28, grid.n), device="cuda")
        ctx = rb.Context(grid, soil, bc, kmean, ks if het else None)
        F_ref = torch.empty_like(p)
        n_ref = ctx.residual(p, s_old, dt, F_ref)
        ctx.close()
        F = torch.full_like(p, float("nan"))
        st, nrm = rb.residual_noalloc(grid, soil, bc, kmean, p, s_old, dt, F, ks=ksd if het else None, norms=norms)
        torch.cuda.synchronize()  # without the norms the call does not synchronise
        assert st == 0
        err = (F - F_ref).abs().max().item() / F_ref.abs().max().item()
        assert err <= TOL
        if norms:
            assert nrm[0] == pytest.approx(n_ref[0], rel=1e-12)
            assert nrm[1] == pytest.approx(n_ref[1], rel=1e-12)
        else:
            assert nrm is None


def test_noalloc_rejects_grids_beyond_its_scratch():
    from paper_2112_05051_gb300 import richards as rb
    rb.load()
    big = synth.Grid(513, 512, 512)  # one plane more than the 512^3 the scratch array covers
    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    st, _ = rb.residual_noalloc(big, synth.Soil(), synth.infiltration_bc(), 0, x, x, 1.0, x)
    assert st == -9  # RICH_ELIMIT, checked before any device work
