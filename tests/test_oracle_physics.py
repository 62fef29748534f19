"""Pins of the oracle's constitutive laws, residual and Jacobian against what the paper and mathematics fix.

None of these re-evaluate the oracle's own formulas: they use closed-form
special points, derivative consistency, the paper's printed Jacobian
entries (transcribed from the paper independently of the oracle's
face-by-face form), textbook tridiagonal-Toeplitz spectra, conservation and
the hydrostatic steady state.
"""
import math

import numpy as np
import pytest

from oracle import constitutive as cst
from oracle import discretization as disc
from paper_2112_05051_gb300 import synth

SOIL = synth.Soil()
MEANS = [synth.KMEAN_ARITH, synth.KMEAN_UPSTREAM, synth.KMEAN_HARMONIC, synth.KMEAN_GEOMETRIC]


# ---------------------------------------------------------------- constitutive (eqs. (s(p)), (K(p)))

def test_saturation_special_points():
    # |p|^beta = alpha gives the midpoint between S_r and S_s
    p_half = -(SOIL.alpha ** (1.0 / SOIL.beta))
    mid = 0.5 * (SOIL.theta_s + SOIL.theta_r)
    assert cst.saturation(p_half, SOIL) == pytest.approx(mid, rel=1e-14)
    # limits: saturated at p -> 0-, residual content as p -> -inf
    assert cst.saturation(-1e-12, SOIL) == pytest.approx(SOIL.theta_s, rel=1e-14)
    assert cst.saturation(-1e8, SOIL) == pytest.approx(SOIL.theta_r, rel=1e-12)
    # saturated regime (Sec. 2): s = S_s, K = K_s for p >= 0
    assert cst.saturation(3.0, SOIL) == SOIL.theta_s
    assert cst.dsaturation(3.0, SOIL) == 0.0


def test_conductivity_special_points():
    p_half = -(SOIL.a ** (1.0 / SOIL.gamma))
    assert cst.conductivity(p_half, SOIL, SOIL.ks) == pytest.approx(0.5 * SOIL.ks, rel=1e-14)
    assert cst.conductivity(-1e-12, SOIL, SOIL.ks) == pytest.approx(SOIL.ks, rel=1e-14)
    assert cst.conductivity(0.5, SOIL, 2.0) == 2.0
    assert cst.dconductivity(0.5, SOIL, 2.0) == 0.0
    # K is proportional to K_s (heterogeneous field scales the law)
    assert cst.conductivity(-30.0, SOIL, 3.0) == pytest.approx(3.0 / SOIL.ks * cst.conductivity(-30.0, SOIL, SOIL.ks))


@pytest.mark.parametrize("p", [-61.5, -20.7, -5.0, -1.0, -150.0])
def test_derivatives_match_central_differences(p):
    # eq. (derivativeofcoefficients) against the laws themselves
    h = 1e-5 * abs(p)
    fd_s = (cst.saturation(p + h, SOIL) - cst.saturation(p - h, SOIL)) / (2 * h)
    fd_k = (cst.conductivity(p + h, SOIL, SOIL.ks) - cst.conductivity(p - h, SOIL, SOIL.ks)) / (2 * h)
    assert cst.dsaturation(p, SOIL) == pytest.approx(fd_s, rel=1e-6)
    assert cst.dconductivity(p, SOIL, SOIL.ks) == pytest.approx(fd_k, rel=1e-6)
    # for p < 0 both laws increase with p (sgn(p) = -1 in the printed derivatives)
    assert cst.dsaturation(p, SOIL) > 0 and cst.dconductivity(p, SOIL, SOIL.ks) > 0


# ---------------------------------------------------------------- residual / Jacobian

def _distinct_p(grid, seed):
    rng = np.random.default_rng(seed)
    # pairwise-distinct neighbours keep every upstream choice away from its kink
    return -60.0 + 40.0 * rng.permutation(grid.n) / grid.n + rng.uniform(0, 1e-3, grid.n)


def _field_bc(dims):
    # per-cell Dirichlet values on the top face and on -x (the paper's Sec. 6 problem has a
    # p = 0 square on top); value arrays follow the face index convention
    rng = np.random.default_rng(17)
    nx, ny, nz = dims
    return synth.BC(kind=(1, 0, 0, 1, 0, 1), value=(-30.0, 0, 0, -45.0, 0, -20.0),
                    fields=(rng.uniform(-50, -10, ny * nz), None, None, None, None, rng.uniform(-40, 0, nx * ny)))


BCS = {
    "infiltration": synth.infiltration_bc(-20.7),
    "dirichlet": synth.BC(kind=(1,) * 6, value=(-30.0, -35.0, -25.0, -40.0, -50.0, -20.0)),
    "noflux": synth.all_noflux_bc(),
    "fields": None,
}


SPLITS = [synth.kmean_split(synth.KMEAN_UPSTREAM, synth.KMEAN_HARMONIC),
          synth.kmean_split(synth.KMEAN_GEOMETRIC, synth.KMEAN_ARITH)]


@pytest.mark.parametrize("kmean", MEANS + SPLITS)
@pytest.mark.parametrize("bcname", list(BCS))
@pytest.mark.parametrize("dims", [(4, 4, 4), (3, 4, 5)])
def test_jacobian_matches_finite_differences(kmean, bcname, dims):
    grid = synth.Grid(*dims, lx=1.0, ly=1.3, lz=0.8)
    bc = BCS[bcname] if bcname != "fields" else _field_bc(dims)
    p = _distinct_p(grid, 7)
    ks = synth.ks_field(grid, 3, 1.0, (2.0, 2.0, 1.0))
    s_old = cst.saturation(p + 1.0, SOIL)
    dt = 0.7
    J = disc.jacobian(grid, SOIL, bc, kmean, p, dt, ks).toarray()
    Jfd = np.zeros_like(J)
    for c in range(grid.n):
        e = np.zeros(grid.n)
        h = 1e-6 * abs(p[c])
        e[c] = h
        Jfd[:, c] = (disc.residual(grid, SOIL, bc, kmean, p + e, s_old, dt, ks)
                     - disc.residual(grid, SOIL, bc, kmean, p - e, s_old, dt, ks)) / (2 * h)
    scale = np.abs(J).max()
    assert np.abs(J - Jfd).max() <= 1e-6 * scale
    # structural 7-point pattern: every in-grid neighbour present, nothing else
    Jc = disc.jacobian(grid, SOIL, bc, kmean, p, dt, ks)
    assert Jc.nnz == grid.n + 2 * ((grid.nx - 1) * grid.ny * grid.nz + grid.nx * (grid.ny - 1) * grid.nz
                                   + grid.nx * grid.ny * (grid.nz - 1))


def _column(nz, kmean, seed=3):
    grid = synth.Grid(1, 1, nz, lz=40.0)
    bc = synth.BC(kind=(0, 0, 0, 0, 1, 1), value=(0, 0, 0, 0, -61.5, -20.7))
    p = _distinct_p(grid, seed)
    return grid, bc, p


def test_1d_arithmetic_jacobian_matches_printed_entries():
    # eq. (jacobian_arithmetic_mean), Sec. 4.2: tridiag(eta, zeta, xi), interior rows
    nz = 12
    grid, bc, p = _column(nz, synth.KMEAN_ARITH)
    dt, hz = 0.1, grid.h[2]
    J = disc.jacobian(grid, SOIL, bc, synth.KMEAN_ARITH, p, dt).toarray()
    K = lambda q: cst.conductivity(q, SOIL, SOIL.ks)
    Kp = lambda q: cst.dconductivity(q, SOIL, SOIL.ks)
    Sp = lambda q: cst.dsaturation(q, SOIL)
    for i in range(1, nz - 1):
        pm, pc, pp = p[i - 1], p[i], p[i + 1]
        zeta = ((dt * K(pm) + dt * K(pp) + 2 * dt * K(pc) + 2 * hz ** 2 * Sp(pc)) / (2 * dt * hz ** 2)
                - pm * Kp(pc) / (2 * hz ** 2) + pc * Kp(pc) / hz ** 2 - pp * Kp(pc) / (2 * hz ** 2))
        xi = (-(K(pp) + K(pc) + hz * Kp(pp)) / (2 * hz ** 2) - pp * Kp(pp) / (2 * hz ** 2)
              + pc * Kp(pp) / (2 * hz ** 2))
        eta = (-(K(pm) + K(pc) - hz * Kp(pm)) / (2 * hz ** 2) - pm * Kp(pm) / (2 * hz ** 2)
               + pc * Kp(pm) / (2 * hz ** 2))
        assert J[i, i] == pytest.approx(zeta, rel=1e-13)
        assert J[i, i + 1] == pytest.approx(xi, rel=1e-12)
        assert J[i, i - 1] == pytest.approx(eta, rel=1e-12)


def test_1d_upstream_jacobian_matches_printed_entries():
    # eq. (jacobian_upstream_mean), Supplementary B: tridiag(eta, zeta, xi), interior rows
    nz = 40
    grid, bc, p = _column(nz, synth.KMEAN_UPSTREAM, seed=11)
    dt, hz = 0.1, grid.h[2]
    J = disc.jacobian(grid, SOIL, bc, synth.KMEAN_UPSTREAM, p, dt).toarray()
    K = lambda q: cst.conductivity(q, SOIL, SOIL.ks)
    Kp = lambda q: cst.dconductivity(q, SOIL, SOIL.ks)
    Sp = lambda q: cst.dsaturation(q, SOIL)
    seen = set()
    for i in range(1, nz - 1):
        pm, pc, pp = p[i - 1], p[i], p[i + 1]
        lo_up = pc - pm >= 0       # face i-1/2: upstream is the upper cell i
        hi_up = pp - pc >= 0       # face i+1/2: upstream is the upper cell i+1
        seen.add((lo_up, hi_up))
        zeta = (Sp(pc) / dt
                - pm / hz ** 2 * (Kp(pc) if lo_up else 0.0)
                - pp / hz ** 2 * (0.0 if hi_up else Kp(pc))
                + pc / hz ** 2 * ((Kp(pc) if lo_up else 0.0) + (0.0 if hi_up else Kp(pc)))
                + ((K(pc) if lo_up else K(pm)) + (K(pp) if hi_up else K(pc))) / hz ** 2)
        xi = (-Kp(pp) / (2 * hz) - (K(pp) if hi_up else K(pc)) / hz ** 2
              + pc / hz ** 2 * (Kp(pp) if hi_up else 0.0) - pp / hz ** 2 * (Kp(pp) if hi_up else 0.0))
        eta = (Kp(pm) / (2 * hz) - (K(pc) if lo_up else K(pm)) / hz ** 2
               + pc / hz ** 2 * (0.0 if lo_up else Kp(pm)) - pm / hz ** 2 * (0.0 if lo_up else Kp(pm)))
        assert J[i, i] == pytest.approx(zeta, rel=1e-12)
        assert J[i, i + 1] == pytest.approx(xi, rel=1e-12)
        assert J[i, i - 1] == pytest.approx(eta, rel=1e-12)
    assert len(seen) == 4  # every branch combination was exercised


def test_3d_arithmetic_jacobian_matches_printed_entries():
    # eq. (jacobian_arithmeticaverage), Supplementary A, interior cells
    grid = synth.Grid(5, 4, 6, lx=1.0, ly=0.7, lz=1.4)
    p = _distinct_p(grid, 5)
    dt = 0.3
    hx, hy, hz = grid.h
    J = disc.jacobian(grid, SOIL, synth.infiltration_bc(), synth.KMEAN_ARITH, p, dt).toarray()
    P = p.reshape(grid.shape)
    K = lambda q: cst.conductivity(q, SOIL, SOIL.ks)
    Kp = lambda q: cst.dconductivity(q, SOIL, SOIL.ks)
    Sp = lambda q: cst.dsaturation(q, SOIL)
    idx = lambda i, j, k: i + grid.nx * (j + grid.ny * k)
    for k in range(1, grid.nz - 1):
        for j in range(1, grid.ny - 1):
            for i in range(1, grid.nx - 1):
                c = P[k, j, i]
                xm, xp, ym, yp, zm, zp = P[k, j, i - 1], P[k, j, i + 1], P[k, j - 1, i], P[k, j + 1, i], P[k - 1, j, i], P[k + 1, j, i]
                diag = (SOIL.rho_phi * Sp(c) / dt + (K(xm) + K(xp) + 2 * K(c)) / (2 * hx ** 2)
                        + (K(ym) + K(yp) + 2 * K(c)) / (2 * hy ** 2) + (K(zm) + K(zp) + 2 * K(c)) / (2 * hz ** 2)
                        + c * (Kp(c) / hx ** 2 + Kp(c) / hy ** 2 + Kp(c) / hz ** 2)
                        - ym * Kp(c) / (2 * hy ** 2) - zm * Kp(c) / (2 * hz ** 2) - zp * Kp(c) / (2 * hz ** 2)
                        - xm * Kp(c) / (2 * hx ** 2) - xp * Kp(c) / (2 * hx ** 2) - yp * Kp(c) / (2 * hy ** 2))
                r = idx(i, j, k)
                assert J[r, r] == pytest.approx(diag, rel=1e-12)
                for q, h, col, grav in ((xm, hx, idx(i - 1, j, k), 0), (xp, hx, idx(i + 1, j, k), 0),
                                        (ym, hy, idx(i, j - 1, k), 0), (yp, hy, idx(i, j + 1, k), 0),
                                        (zm, hz, idx(i, j, k - 1), -1), (zp, hz, idx(i, j, k + 1), +1)):
                    off = (-(K(q) + K(c) + grav * h * Kp(q)) / (2 * h ** 2) - q * Kp(q) / (2 * h ** 2)
                           + c * Kp(q) / (2 * h ** 2))
                    assert J[r, col] == pytest.approx(off, rel=1e-12)


@pytest.mark.parametrize("kmean", MEANS)
def test_constant_state_spectrum_is_kronecker_sum_of_toeplitz(kmean):
    # uniform p, homogeneous soil, Dirichlet faces at the same p: only the
    # gravity derivative survives beside the scaled 7-point Laplacian, and the
    # spectrum is the Kronecker sum of tridiagonal Toeplitz spectra.
    n = (6, 5, 7)
    grid = synth.Grid(*n, lx=1.0, ly=0.8, lz=1.2)
    pu = -30.0
    p = np.full(grid.n, pu)
    bc = synth.all_dirichlet_bc(pu)
    dt = 0.5
    Kc = cst.conductivity(pu, SOIL, SOIL.ks)
    Kd = cst.dconductivity(pu, SOIL, SOIL.ks)
    sd = cst.dsaturation(pu, SOIL)
    hx, hy, hz = grid.h

    def lap(m, h):
        th = np.arange(1, m + 1) * math.pi / (m + 1)
        return (Kc / h ** 2) * (2 - 2 * np.cos(th))

    th_z = np.arange(1, n[2] + 1) * math.pi / (n[2] + 1)
    lz = 2 * Kc / hz ** 2 - 2 * math.sqrt((Kc / hz ** 2) ** 2 - (Kd / (2 * hz)) ** 2) * np.cos(th_z)
    expect = (sd / dt + lap(n[0], hx)[None, None, :] + lap(n[1], hy)[None, :, None] + lz[:, None, None]).ravel()
    ev = np.linalg.eigvals(disc.jacobian(grid, SOIL, bc, kmean, p, dt).toarray())
    assert np.abs(ev.imag).max() < 1e-9 * np.abs(ev.real).max()
    np.testing.assert_allclose(np.sort(ev.real), np.sort(expect), rtol=1e-10)
    # A_aux: same with the gravity derivative removed (the scaled 7-point Laplacian)
    lz0 = (Kc / hz ** 2) * (2 - 2 * np.cos(th_z))
    expect0 = (sd / dt + lap(n[0], hx)[None, None, :] + lap(n[1], hy)[None, :, None] + lz0[:, None, None]).ravel()
    ev0 = np.linalg.eigvalsh(disc.aux_matrix(grid, SOIL, bc, kmean, p, dt).toarray())
    np.testing.assert_allclose(np.sort(ev0), np.sort(expect0), rtol=1e-10)


@pytest.mark.parametrize("kmean", MEANS)
@pytest.mark.parametrize("het", [False, True])
def test_mass_balance_all_noflux(kmean, het):
    # With no-flux on every face the interior face fluxes telescope:
    # sum_c Phi_c = rho_phi sum_c (s(p_c) - s_old_c)/dt exactly (up to rounding).
    grid = synth.Grid(5, 6, 4)
    p = _distinct_p(grid, 21)
    ks = synth.ks_field(grid, 8, 1.5, (2.0, 3.0, 1.0)) if het else None
    s_old = cst.saturation(p - 3.0, SOIL)
    dt = 2.0
    phi = disc.residual(grid, SOIL, synth.all_noflux_bc(), kmean, p, s_old, dt, ks)
    storage = SOIL.rho_phi * (cst.saturation(p, SOIL) - s_old) / dt
    scale = np.abs(phi).sum() + np.abs(storage).sum()
    assert abs(phi.sum() - storage.sum()) <= 1e-13 * scale


def test_hydrostatic_state_has_zero_residual_with_arithmetic_mean():
    # p = H0 - z: Darcy flux -K (dp/dz + 1) vanishes; with the arithmetic mean the
    # discrete diffusive and centred gravity fluxes cancel face by face.
    grid = synth.Grid(4, 3, 9, lz=2.0)
    hz = grid.h[2]
    z = (np.arange(grid.nz) + 1) * hz
    p = np.broadcast_to((-15.0 - z)[:, None, None], grid.shape).ravel().copy()
    ks = synth.ks_field(grid, 2, 1.0, (2.0, 2.0, 2.0))
    s_old = cst.saturation(p, SOIL)
    # consistent Dirichlet top (ghost at z = (nz+1) h_z) and no-flux elsewhere
    bc = synth.BC(kind=(0, 0, 0, 0, 0, 1), value=(0, 0, 0, 0, 0, -15.0 - (grid.nz + 1) * hz))
    phi = disc.residual(grid, SOIL, bc, synth.KMEAN_ARITH, p, s_old, 1.0, ks)
    kscale = cst.conductivity(p, SOIL, ks).max() / hz
    assert np.abs(phi).max() <= 1e-12 * kscale
    # the upstream mean takes the lower cell on every vertical face (p decreases upward),
    # so it does NOT vanish: flux (K_L - K_U)/2 per face.
    phi_up = disc.residual(grid, SOIL, bc, synth.KMEAN_UPSTREAM, p, s_old, 1.0, ks)
    assert np.abs(phi_up).max() > 1e-6 * kscale


def test_face_field_equals_constant_value_when_uniform():
    # a per-cell face array holding one value everywhere is the constant Dirichlet face
    grid = synth.Grid(5, 4, 6)
    p = _distinct_p(grid, 4)
    s_old = cst.saturation(p, SOIL)
    const = synth.BC(kind=(1, 0, 0, 0, 0, 1), value=(-33.0, 0, 0, 0, 0, -21.0))
    fld = synth.BC(kind=(1, 0, 0, 0, 0, 1), value=(0.0, 0, 0, 0, 0, 0.0),
                   fields=(np.full(4 * 6, -33.0), None, None, None, None, np.full(5 * 4, -21.0)))
    for kmean in MEANS:
        a = disc.residual(grid, SOIL, const, kmean, p, s_old, 0.5)
        b = disc.residual(grid, SOIL, fld, kmean, p, s_old, 0.5)
        np.testing.assert_array_equal(a, b)
    # the paper's top-face pattern: 0 inside the centred square, h_r outside
    g2 = synth.Grid(12, 8, 4, 64.0, 64.0, 1.0)
    bc = synth.paper_infiltration_bc(g2, -61.5)
    top = bc.field(5).reshape(g2.ny, g2.nx)
    assert top.max() == 0.0 and top.min() == -61.5
    assert top[g2.ny // 2, g2.nx // 2] == 0.0 and top[0, 0] == -61.5


def test_aux_is_spd_and_equals_jacobian_without_conductivity_slope():
    grid = synth.Grid(4, 3, 5)
    p = _distinct_p(grid, 2)
    for kmean in MEANS:
        A = disc.aux_matrix(grid, SOIL, synth.infiltration_bc(), kmean, p, 0.5).toarray()
        assert np.abs(A - A.T).max() == 0.0
        np.linalg.cholesky(A)
    # a soil whose K does not depend on p (a -> infinity): J and A_aux coincide
    flat = synth.Soil(a=1e300)
    for kmean in MEANS:
        J = disc.jacobian(grid, flat, synth.infiltration_bc(), kmean, p, 0.5).toarray()
        A = disc.aux_matrix(grid, flat, synth.infiltration_bc(), kmean, p, 0.5).toarray()
        assert np.abs(J - A).max() <= 1e-14 * np.abs(A).max()


def test_face_means_obey_the_mean_inequality_and_the_upstream_rule():
    # harmonic <= geometric <= arithmetic, all between min and max, all equal to K
    # when both sides agree (the textbook inequality of the three Pythagorean means)
    rng = np.random.default_rng(17)
    kl = 10.0 ** rng.uniform(-8, 0, 2000)
    ku = 10.0 ** rng.uniform(-8, 0, 2000)
    pl = rng.uniform(-70, -10, 2000)
    pu = rng.uniform(-70, -10, 2000)
    a = disc.face_mean(disc.KMEAN_ARITH, kl, ku, pl, pu)
    g = disc.face_mean(disc.KMEAN_GEOMETRIC, kl, ku, pl, pu)
    h = disc.face_mean(disc.KMEAN_HARMONIC, kl, ku, pl, pu)
    lo, hi = np.minimum(kl, ku), np.maximum(kl, ku)
    tol = 1e-14 * hi
    assert np.all(h <= g + tol) and np.all(g <= a + tol)
    assert np.all(lo - tol <= h) and np.all(a <= hi + tol)
    for m in (disc.KMEAN_ARITH, disc.KMEAN_UPSTREAM, disc.KMEAN_HARMONIC, disc.KMEAN_GEOMETRIC):
        np.testing.assert_allclose(disc.face_mean(m, kl, kl, pl, pu), kl, rtol=1e-15)
    # upstream: the conductivity of the cell with the higher head, the upper cell on a tie
    u = disc.face_mean(disc.KMEAN_UPSTREAM, kl, ku, pl, pu)
    assert np.array_equal(u, np.where(pu >= pl, ku, kl))
    assert np.array_equal(disc.face_mean(disc.KMEAN_UPSTREAM, kl, ku, pl, pl), ku)


@pytest.mark.parametrize("kmean", [0, 1, 2, 3])
def test_face_mean_partials_match_central_differences(kmean):
    rng = np.random.default_rng(3 + kmean)
    kl = 10.0 ** rng.uniform(-6, -1, 200)
    ku = 10.0 ** rng.uniform(-6, -1, 200)
    pl = rng.uniform(-70, -10, 200)
    pu = pl + rng.choice([-1.0, 1.0], 200) * rng.uniform(1, 5, 200)  # away from upstream ties
    dl, du = disc.face_mean_partials(kmean, kl, ku, pl, pu)
    for k_var, d in ((0, dl), (1, du)):
        e = 1e-4 * (kl if k_var == 0 else ku)  # central differences: O(e^2) truncation
        if k_var == 0:
            fd = (disc.face_mean(kmean, kl + e, ku, pl, pu) - disc.face_mean(kmean, kl - e, ku, pl, pu)) / (2 * e)
        else:
            fd = (disc.face_mean(kmean, kl, ku + e, pl, pu) - disc.face_mean(kmean, kl, ku - e, pl, pu)) / (2 * e)
        np.testing.assert_allclose(d, fd, rtol=1e-5, atol=1e-9)


def test_all_means_give_the_same_residual_where_neighbour_conductivities_agree():
    # a uniform head on a homogeneous soil makes K equal on both sides of every
    # interior face (Dirichlet ghosts at the same head too): the four means coincide
    grid = synth.Grid(6, 5, 7)
    bc = synth.all_dirichlet_bc(-35.0)
    p = np.full(grid.n, -35.0)
    s_old = cst.saturation(p + 3.0, SOIL)
    ref = disc.residual(grid, SOIL, bc, disc.KMEAN_ARITH, p, s_old, 0.7)
    for m in (disc.KMEAN_UPSTREAM, disc.KMEAN_HARMONIC, disc.KMEAN_GEOMETRIC):
        np.testing.assert_allclose(disc.residual(grid, SOIL, bc, m, p, s_old, 0.7), ref, rtol=1e-13,
                                   atol=1e-13 * np.abs(ref).max())


# ---------------------------------------------------------------- the pins catch planted mistakes
# Each test plants one plausible mistake in the oracle (on the CPU, for the
# duration of the test) and checks that the pin above it fails.

def test_pins_catch_a_geometric_mean_without_its_root(monkeypatch):
    orig = disc.face_mean
    monkeypatch.setattr(disc, "face_mean", lambda m, kl, ku, pl, pu: kl * ku if m == disc.KMEAN_GEOMETRIC
                        else orig(m, kl, ku, pl, pu))
    with pytest.raises(AssertionError):
        test_face_means_obey_the_mean_inequality_and_the_upstream_rule()


def test_pins_catch_a_harmonic_mean_without_its_factor_two(monkeypatch):
    orig = disc.face_mean
    monkeypatch.setattr(disc, "face_mean", lambda m, kl, ku, pl, pu: kl * ku / (kl + ku) if m == disc.KMEAN_HARMONIC
                        else orig(m, kl, ku, pl, pu))
    with pytest.raises(AssertionError):
        test_face_means_obey_the_mean_inequality_and_the_upstream_rule()


def test_pins_catch_a_saturation_derivative_with_the_wrong_exponent(monkeypatch):
    def bad(p, soil):
        ap = np.abs(p)
        pb = ap ** soil.beta
        return soil.alpha * soil.beta * pb * (soil.theta_s - soil.theta_r) / (soil.alpha + pb) ** 2  # |p|^beta
    monkeypatch.setattr(cst, "dsaturation", bad)
    with pytest.raises(AssertionError):
        test_derivatives_match_central_differences(-61.5)


def test_pins_catch_swapped_harmonic_mean_partials(monkeypatch):
    orig = disc.face_mean_partials

    def bad(m, kl, ku, pl, pu):
        dl, du = orig(m, kl, ku, pl, pu)
        return (du, dl) if m == disc.KMEAN_HARMONIC else (dl, du)
    monkeypatch.setattr(disc, "face_mean_partials", bad)
    with pytest.raises(AssertionError):
        test_jacobian_matches_finite_differences(disc.KMEAN_HARMONIC, list(BCS)[0], (4, 4, 4))


# ---------------------------------------------------------------- split horizontal/vertical mean (Sec. 2.1)

@pytest.mark.parametrize("kmean", MEANS)
def test_split_mean_of_one_kind_is_that_mean(kmean):
    grid = synth.Grid(5, 4, 6)
    p = _distinct_p(grid, 2)
    ks = synth.ks_field(grid, 4, 1.0, (2.0, 2.0, 1.0))
    s_old = cst.saturation(p + 0.5, SOIL)
    bc = synth.BC(kind=(1, 0, 1, 0, 1, 1), value=(-30.0, 0, -35.0, 0, -50.0, -20.0))
    sp_ = synth.kmean_split(kmean, kmean)
    np.testing.assert_array_equal(disc.residual(grid, SOIL, bc, sp_, p, s_old, 0.9, ks),
                                  disc.residual(grid, SOIL, bc, kmean, p, s_old, 0.9, ks))
    np.testing.assert_array_equal(disc.jacobian_stencil(grid, SOIL, bc, sp_, p, 0.9, ks),
                                  disc.jacobian_stencil(grid, SOIL, bc, kmean, p, 0.9, ks))
    np.testing.assert_array_equal(disc.aux_stencil(grid, SOIL, bc, sp_, p, 0.9, ks),
                                  disc.aux_stencil(grid, SOIL, bc, kmean, p, 0.9, ks))


@pytest.mark.parametrize("h,v", [(synth.KMEAN_UPSTREAM, synth.KMEAN_HARMONIC), (synth.KMEAN_GEOMETRIC, synth.KMEAN_ARITH)])
def test_split_mean_takes_the_horizontal_mean_across_x_y_faces_and_the_vertical_one_across_z(h, v):
    sp_ = synth.kmean_split(h, v)
    # a single horizontal layer with closed z faces has only x and y faces
    layer = synth.Grid(6, 5, 1)
    p = _distinct_p(layer, 5)
    s_old = cst.saturation(p + 0.5, SOIL)
    bc = synth.BC(kind=(1, 1, 1, 0, 0, 0), value=(-30.0, -20.0, -40.0, 0, 0, 0))
    np.testing.assert_array_equal(disc.residual(layer, SOIL, bc, sp_, p, s_old, 0.9),
                                  disc.residual(layer, SOIL, bc, h, p, s_old, 0.9))
    # a vertical column with closed side faces has only z faces
    col = synth.Grid(1, 1, 9)
    p = _distinct_p(col, 6)
    s_old = cst.saturation(p + 0.5, SOIL)
    bc = synth.infiltration_bc(-20.7)
    np.testing.assert_array_equal(disc.residual(col, SOIL, bc, sp_, p, s_old, 0.9),
                                  disc.residual(col, SOIL, bc, v, p, s_old, 0.9))
    # in 3D the split differs from both of its parts
    g3 = synth.Grid(4, 4, 4)
    p = _distinct_p(g3, 7)
    s_old = cst.saturation(p + 0.5, SOIL)
    r = disc.residual(g3, SOIL, synth.infiltration_bc(), sp_, p, s_old, 0.9)
    assert not np.allclose(r, disc.residual(g3, SOIL, synth.infiltration_bc(), h, p, s_old, 0.9))
    assert not np.allclose(r, disc.residual(g3, SOIL, synth.infiltration_bc(), v, p, s_old, 0.9))
