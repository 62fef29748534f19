"""Cell-centred 7-point discretisation of the mixed-form Richards equation (oracle; test infrastructure).

Follows eq. (dynamic_of_the_problem) of Sec. 2.1.  For cell c and each of its
six faces f (direction d = x, y, z, side +/-1, neighbour nb) the paper's flux
differences q_{+1/2} - q_{-1/2} regroup face by face into

    T_f = K_av,f (p_c - p_nb) / h_d^2                    (both sides of an axis)
    G_f = -side * (K_c + K_nb) / (2 h_z)                 (z faces only)

so that Phi_c = rho_phi (s(p_c) - s(p_c^old)) / dt + sum_f (T_f + G_f).  In the
interior the two G terms add up to the paper's centred gravity difference
-(K_{k+1} - K_{k-1}) / (2 h_z); each face carries one value of K_av, so the
discrete fluxes telescope.

Readings where the paper is silent (all listed in the design notes):
  * face means (Sec. 2.1): arithmetic (K_L+K_U)/2; upstream (eq.
    (upstream_mean)) K_U if p_U - p_L >= 0 else K_L, where U is the cell on
    the +d side of the face, ties taking K_U; harmonic 2 K_L K_U/(K_L+K_U)
    (the abstract names it, no formula is printed); geometric sqrt(K_L K_U)
    (Sec. 2.1); or a split of two of them, one on the horizontal (x, y) and
    one on the vertical (z) faces (Sec. 2.1, axis_kmean).
  * Dirichlet face: the ghost node holds p = p_bc (a constant or a per-cell
    value of the face) and K = K(p_bc) with the Ks of the adjacent interior
    cell; T and G use it as a neighbour.
  * No-flux face: the whole face flux T + G is zero.
  * f = 0, rho_phi from the soil (1 by default).

The Jacobian is the exact derivative of this residual (chain rule through
K_av); in the interior it equals the printed entries of Supplementary A
(eq. (jacobian_arithmeticaverage)) and, for the upstream mean, Supplementary
C (eq. (jacobian_upstreamaverage), with its typos corrected).  At an
upstream tie the derivative takes the ">= 0" branch.

The preconditioner matrix A_aux keeps only the diffusion part with frozen
coefficients: q_prec = -K(p) grad p (Sec. 4, after Theorem
(spectraldescription)).  It is
    A_aux = diag(rho_phi s'(p)/dt) + sum_f (K_av,f/h_d^2) (e_c - e_nb)(e_c - e_nb)^T
with Dirichlet faces adding K_av/h_d^2 to the diagonal only; it is SPD.

Stencil layout returned by the *_stencil functions: column 0 = diagonal,
then -x, +x, -y, +y, -z, +z neighbours (zero where the neighbour is outside).
"""
import numpy as np
import scipy.sparse as sp

from . import constitutive as cst

# (axis, side) per face, axis 0 = x, 1 = y, 2 = z; order -x,+x,-y,+y,-z,+z.
FACES = ((0, -1), (0, 1), (1, -1), (1, 1), (2, -1), (2, 1))
KMEAN_ARITH, KMEAN_UPSTREAM, KMEAN_HARMONIC, KMEAN_GEOMETRIC = 0, 1, 2, 3
BC_NOFLUX, BC_DIRICHLET = 0, 1


def _np_axis(axis):
    return 2 - axis  # arrays are shaped (nz, ny, nx)


def _shift(a3, axis, side):
    """out[c] = a3[c + side*e_axis] where that cell exists; boundary layer left as a copy of a3."""
    ax = _np_axis(axis)
    out = a3.copy()
    dst = [slice(None)] * 3
    src = [slice(None)] * 3
    if side > 0:
        dst[ax], src[ax] = slice(0, -1), slice(1, None)
    else:
        dst[ax], src[ax] = slice(1, None), slice(0, -1)
    out[tuple(dst)] = a3[tuple(src)]
    return out


def _boundary_mask(shape, axis, side):
    ax = _np_axis(axis)
    m = np.zeros(shape, dtype=bool)
    idx = [slice(None)] * 3
    idx[ax] = -1 if side > 0 else 0
    m[tuple(idx)] = True
    return m


def axis_kmean(kmean, axis):
    """The mean used on the faces normal to axis.  Sec. 2.1 allows "two different
    means, one for the horizontal and another for the vertical direction": such a
    split mean is coded 0x100 | (horizontal << 4) | vertical and applies the
    horizontal mean on the x and y faces, the vertical one on the z faces."""
    if kmean & 0x100:
        return kmean & 0xF if axis == 2 else (kmean >> 4) & 0xF
    return kmean


def face_mean(kmean, k_lo, k_up, p_lo, p_up):
    """K_av of a face between the lower (L) and upper (U, +d side) cell."""
    if kmean == KMEAN_ARITH:
        return 0.5 * (k_lo + k_up)
    if kmean == KMEAN_UPSTREAM:
        return np.where(p_up - p_lo >= 0.0, k_up, k_lo)
    if kmean == KMEAN_HARMONIC:
        s = k_lo + k_up
        with np.errstate(divide="ignore", invalid="ignore"):
            return np.where(s > 0.0, 2.0 * k_lo * k_up / s, 0.0)
    if kmean == KMEAN_GEOMETRIC:
        return np.sqrt(k_lo * k_up)
    raise ValueError("unknown K mean")


def face_mean_partials(kmean, k_lo, k_up, p_lo, p_up):
    """(dK_av/dK_L, dK_av/dK_U) at fixed choice of the upstream branch."""
    if kmean == KMEAN_ARITH:
        h = np.full(np.shape(k_lo), 0.5)
        return h, h.copy()
    if kmean == KMEAN_UPSTREAM:
        up = p_up - p_lo >= 0.0
        return np.where(up, 0.0, 1.0), np.where(up, 1.0, 0.0)
    if kmean == KMEAN_HARMONIC:
        s = k_lo + k_up
        with np.errstate(divide="ignore", invalid="ignore"):
            d_lo = np.where(s > 0.0, 2.0 * k_up * k_up / (s * s), 0.0)
            d_up = np.where(s > 0.0, 2.0 * k_lo * k_lo / (s * s), 0.0)
        return d_lo, d_up
    if kmean == KMEAN_GEOMETRIC:
        g = np.sqrt(k_lo * k_up)
        with np.errstate(divide="ignore", invalid="ignore"):
            d_lo = np.where(k_lo > 0.0, 0.5 * g / k_lo, 0.0)
            d_up = np.where(k_up > 0.0, 0.5 * g / k_up, 0.0)
        return d_lo, d_up
    raise ValueError("unknown K mean")


class _Faces:
    """Per-face neighbour data for every cell (ghost values on Dirichlet faces)."""

    def __init__(self, grid, soil, bc, p, ks):
        shape = grid.shape
        self.shape = shape
        self.h = grid.h
        p3 = np.asarray(p, dtype=np.float64).reshape(shape)
        ks3 = np.broadcast_to(np.asarray(ks, dtype=np.float64), (grid.n,)).reshape(shape)
        self.p3 = p3
        self.K3 = cst.conductivity(p3, soil, ks3)
        self.dK3 = cst.dconductivity(p3, soil, ks3)
        self.faces = []
        for f, (axis, side) in enumerate(FACES):
            bnd = _boundary_mask(shape, axis, side)
            kind = bc.kind[f]
            pbc = bc.value[f]
            fld = bc.field(f) if hasattr(bc, "field") else None
            nb_p = _shift(p3, axis, side)
            nb_K = _shift(self.K3, axis, side)
            nb_dK = _shift(self.dK3, axis, side)
            if kind == BC_DIRICHLET:
                ghost_p = np.full(shape, pbc)
                if fld is not None:  # per-cell values of the face, broadcast along its normal
                    ax = _np_axis(axis)
                    fs = list(shape)
                    fs[ax] = 1
                    ghost_p = np.broadcast_to(np.asarray(fld, dtype=np.float64).reshape(fs), shape)
                nb_p = np.where(bnd, ghost_p, nb_p)
                nb_K = np.where(bnd, cst.conductivity(ghost_p, soil, ks3), nb_K)
            nb_dK = np.where(bnd, 0.0, nb_dK)
            interior = ~bnd
            active = interior | (bnd & (kind == BC_DIRICHLET))
            self.faces.append((axis, side, nb_p, nb_K, nb_dK, interior, active))

    def lower_upper(self, side, nb_p, nb_K):
        """(K_L, K_U, p_L, p_U) with U the +d cell of the face."""
        if side > 0:
            return self.K3, nb_K, self.p3, nb_p
        return nb_K, self.K3, nb_p, self.p3


def residual(grid, soil, bc, kmean, p, s_old, dt, ks=None, with_scale=False):
    """Phi(p) of eq. (dynamic_of_the_problem), flat array of n cells.

    with_scale=True also returns ||m||_2 with m_c = rho_phi (|s_c| + |s_old,c|)/dt
    + sum_f [K_av,f (|p_c| + |p_nb|)/h_d^2 + (K_c + K_nb)/(2 h_z) on z faces],
    the magnitudes of the products summed into Phi_c before they cancel:
    machine epsilon times it is the accuracy to which Phi can be evaluated.
    """
    ks = soil.ks if ks is None else ks
    fd = _Faces(grid, soil, bc, p, ks)
    s_new = cst.saturation(fd.p3, soil)
    s_o = np.asarray(s_old).reshape(fd.shape)
    phi = soil.rho_phi * (s_new - s_o) / dt
    mag = soil.rho_phi * (np.abs(s_new) + np.abs(s_o)) / dt
    for axis, side, nb_p, nb_K, nb_dK, interior, active in fd.faces:
        h = fd.h[axis]
        k_lo, k_up, p_lo, p_up = fd.lower_upper(side, nb_p, nb_K)
        kav = face_mean(axis_kmean(kmean, axis), k_lo, k_up, p_lo, p_up)
        t = kav * (fd.p3 - nb_p) / (h * h)
        m = kav * (np.abs(fd.p3) + np.abs(nb_p)) / (h * h)
        if axis == 2:
            t = t - side * (fd.K3 + nb_K) / (2.0 * h)
            m = m + (fd.K3 + nb_K) / (2.0 * h)
        phi = phi + np.where(active, t, 0.0)
        mag = mag + np.where(active, m, 0.0)
    if with_scale:
        return phi.reshape(-1), float(np.sqrt(np.sum(mag * mag)))
    return phi.reshape(-1)


def _stencil_to_csr(grid, st):
    """CSR (sorted columns) from a (n, 7) stencil; structural pattern = neighbours inside the grid."""
    n = grid.n
    nx, ny = grid.nx, grid.ny
    c = np.arange(n, dtype=np.int64)
    i = c % nx
    j = (c // nx) % ny
    k = c // (nx * ny)
    sz, sy = nx * ny, nx
    # ascending column order: -z, -y, -x, diag, +x, +y, +z
    cols = np.stack([c - sz, c - sy, c - 1, c, c + 1, c + sy, c + sz], axis=1)
    vals = np.stack([st[:, 5], st[:, 3], st[:, 1], st[:, 0], st[:, 2], st[:, 4], st[:, 6]], axis=1)
    mask = np.stack([k > 0, j > 0, i > 0, np.ones(n, bool), i < nx - 1, j < ny - 1, k < grid.nz - 1], axis=1)
    indptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(mask.sum(axis=1), out=indptr[1:])
    return sp.csr_matrix((vals[mask], cols[mask], indptr), shape=(n, n))


def jacobian_stencil(grid, soil, bc, kmean, p, dt, ks=None):
    """dPhi/dp as a (n, 7) stencil [diag, -x, +x, -y, +y, -z, +z]."""
    ks = soil.ks if ks is None else ks
    fd = _Faces(grid, soil, bc, p, ks)
    diag = soil.rho_phi * cst.dsaturation(fd.p3, soil) / dt
    st = np.zeros((grid.n, 7))
    for f, (axis, side, nb_p, nb_K, nb_dK, interior, active) in enumerate(fd.faces):
        h = fd.h[axis]
        k_lo, k_up, p_lo, p_up = fd.lower_upper(side, nb_p, nb_K)
        kav = face_mean(axis_kmean(kmean, axis), k_lo, k_up, p_lo, p_up)
        d_lo, d_up = face_mean_partials(axis_kmean(kmean, axis), k_lo, k_up, p_lo, p_up)
        d_self, d_nb = (d_lo, d_up) if side > 0 else (d_up, d_lo)
        dp = (fd.p3 - nb_p) / (h * h)
        dd = d_self * fd.dK3 * dp + kav / (h * h)
        off = d_nb * nb_dK * dp - kav / (h * h)
        if axis == 2:
            dd = dd - side * fd.dK3 / (2.0 * h)
            off = off - side * nb_dK / (2.0 * h)
        diag = diag + np.where(active, dd, 0.0)
        st[:, 1 + f] = np.where(interior, off, 0.0).reshape(-1)
    st[:, 0] = diag.reshape(-1)
    return st


def jacobian(grid, soil, bc, kmean, p, dt, ks=None):
    """J(p) as scipy CSR with the 7-point structural pattern."""
    return _stencil_to_csr(grid, jacobian_stencil(grid, soil, bc, kmean, p, dt, ks))


def aux_stencil(grid, soil, bc, kmean, p, dt, ks=None):
    """Diffusion-only frozen-coefficient preconditioner matrix A_aux as a (n, 7) stencil."""
    ks = soil.ks if ks is None else ks
    fd = _Faces(grid, soil, bc, p, ks)
    diag = soil.rho_phi * cst.dsaturation(fd.p3, soil) / dt
    st = np.zeros((grid.n, 7))
    for f, (axis, side, nb_p, nb_K, nb_dK, interior, active) in enumerate(fd.faces):
        h = fd.h[axis]
        k_lo, k_up, p_lo, p_up = fd.lower_upper(side, nb_p, nb_K)
        w = face_mean(axis_kmean(kmean, axis), k_lo, k_up, p_lo, p_up) / (h * h)
        diag = diag + np.where(active, w, 0.0)
        st[:, 1 + f] = np.where(interior, -w, 0.0).reshape(-1)
    st[:, 0] = diag.reshape(-1)
    return st


def aux_matrix(grid, soil, bc, kmean, p, dt, ks=None):
    return _stencil_to_csr(grid, aux_stencil(grid, soil, bc, kmean, p, dt, ks))


def stencil_matvec(grid, st, x):
    """y = A x for a (n, 7) stencil (plain reference used by tests)."""
    return _stencil_to_csr(grid, st) @ np.asarray(x, dtype=np.float64)
