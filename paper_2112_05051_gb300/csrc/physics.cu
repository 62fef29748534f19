// Constitutive evaluation, residual Phi(p), Jacobian/diffusion-matrix assembly and the
// stencil SpMV of the cell-centred 7-point discretisation (Sec. 2.1, eq.
// (dynamic_of_the_problem)), plus the context lifetime entry points.
//
// Face form of the residual for cell c and each face f (axis d, side s = -1/+1,
// neighbour nb or Dirichlet ghost):
//     Phi_c = rho_phi (S(p_c) - S_old,c)/dt + sum_f [ K_av,f (p_c - p_nb)/h_d^2
//             - s (K_c + K_nb)/(2 h_z) (z faces only) ],
// with no-flux faces contributing nothing; in the interior this is the paper's
// q_{+1/2} - q_{-1/2} with the centred gravity term -(K_{k+1} - K_{k-1})/(2 h_z).
// The Jacobian is its exact derivative (chain rule through K_av; Supplementary A
// and C print the interior entries), and the diffusion-only matrix keeps
// K_av/h_d^2 couplings plus the storage diagonal (Sec. 4, q_prec = -K grad p).
#include "common.cuh"

namespace rich {

static __thread char g_cuda_err[256];

void set_cuda_error(cudaError_t e, const char* where) {
  snprintf(g_cuda_err, sizeof(g_cuda_err), "%s: %s", where, cudaGetErrorString(e));
}

__global__ void k_constit(long long n, SoilP so, const double* __restrict__ p, const double* __restrict__ ks,
                          double* __restrict__ K, double* __restrict__ dK, double* __restrict__ S,
                          double* __restrict__ dS) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    double s_, ds_, k_, dk_;
    constit(p[c], ks ? ks[c] : so.ks, so, s_, ds_, k_, dk_);
    K[c] = k_;
    dK[c] = dk_;
    S[c] = s_;
    dS[c] = ds_;
  }
}

// out[t] = field[cell next to face f whose face index is t] (the layout of the
// per-cell face arrays: i + nx j on z faces, i + nx k on y faces, j + ny k on x faces).
__global__ void k_pack_face(GridP g, int f, long long m, const double* __restrict__ field,
                            double* __restrict__ out) {
  const int axis = f >> 1;
  const bool hi = f & 1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < m; t += (long long)gridDim.x * blockDim.x) {
    long long i, j, k;
    if (axis == 0) {
      j = t % g.ny;
      k = t / g.ny;
      i = hi ? g.nx - 1 : 0;
    } else if (axis == 1) {
      i = t % g.nx;
      k = t / g.nx;
      j = hi ? g.ny - 1 : 0;
    } else {
      i = t % g.nx;
      j = t / g.nx;
      k = hi ? g.nz - 1 : 0;
    }
    out[t] = field[i + (long long)g.nx * (j + (long long)g.ny * k)];
  }
}

// y[c] += M_f[c] ghost[t] for the cells c next to face f (t their face index): the
// coupling of a subdomain's face cells to its neighbour's cells, kept in plane f of
// the 7-plane stencil M.
__global__ void k_face_apply(GridP g, int f, long long m, const double* __restrict__ M,
                             const double* __restrict__ ghost, double* __restrict__ y) {
  const int axis = f >> 1;
  const bool hi = f & 1;
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < m; t += (long long)gridDim.x * blockDim.x) {
    long long i, j, k;
    if (axis == 0) {
      j = t % g.ny;
      k = t / g.ny;
      i = hi ? g.nx - 1 : 0;
    } else if (axis == 1) {
      i = t % g.nx;
      k = t / g.nx;
      j = hi ? g.ny - 1 : 0;
    } else {
      i = t % g.nx;
      j = t / g.nx;
      k = hi ? g.nz - 1 : 0;
    }
    const long long c = i + (long long)g.nx * (j + (long long)g.ny * k);
    y[c] += M[(1 + f) * g.n + c] * ghost[t];
  }
}

__global__ void k_saturation(long long n, SoilP so, const double* __restrict__ p, double* __restrict__ s) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    double s_, ds_, k_, dk_;
    constit(p[c], so.ks, so, s_, ds_, k_, dk_);
    s[c] = s_;
  }
}

// Neighbour data of face f of cell (i,j,k).  Returns false for a no-flux boundary face.
struct FaceNb {
  double p, K, dK;
  long long idx;   // -1 for a Dirichlet ghost, kInterfaceGhost for a neighbouring subdomain's cell
};
constexpr long long kInterfaceGhost = -2;

__device__ __forceinline__ bool face_neighbour(const GridP& g, const BCP& bc, const SoilP& so, int f, int i, int j,
                                               int k, long long c, const double* __restrict__ p,
                                               const double* __restrict__ K, const double* __restrict__ dK,
                                               double ksc, FaceNb& nb) {
  int axis = f >> 1;
  int side = (f & 1) ? 1 : -1;
  // a batch stacks problems along z: their top and bottom layers are boundaries
  int coord = axis == 0 ? i : (axis == 1 ? j : (g.nzs == g.nz ? k : k % g.nzs));
  int extent = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nzs);
  bool bnd = side > 0 ? (coord == extent - 1) : (coord == 0);
  if (bnd) {
    if (bc.kind[f] == RICH_BC_NOFLUX) return false;
    nb.p = bc_value(bc, f, i, j, k, g.nx, g.ny);
    if (bc.kind[f] == RICH_BC_INTERFACE) {  // a cell of the neighbouring subdomain, with its own K_s
      const double* gk = bc.gks[f];
      double s_, ds_;
      constit(nb.p, gk ? gk[face_index(f, i, j, k, g.nx, g.ny)] : so.ks, so, s_, ds_, nb.K, nb.dK);
      if (!dK) nb.dK = 0.0;
      nb.idx = kInterfaceGhost;
      return true;
    }
    nb.K = conductivity_only(nb.p, ksc, so);
    nb.dK = 0.0;
    nb.idx = -1;
    return true;
  }
  long long stride = axis == 0 ? 1LL : (axis == 1 ? (long long)g.nx : (long long)g.nx * g.ny);
  long long q = c + side * stride;
  nb.p = p[q];
  nb.K = K[q];
  nb.dK = dK ? dK[q] : 0.0;
  nb.idx = q;
  return true;
}

__global__ void k_residual(GridP g, SoilP so, BCP bc, int kmean, const double* __restrict__ p,
                           const double* __restrict__ K, const double* __restrict__ S,
                           const double* __restrict__ s_old, const double* __restrict__ ks, double dt,
                           double* __restrict__ F, double* __restrict__ partials) {
  double acc[2] = {0.0, 0.0};
  double amax = 0.0;
  const double rdt = so.rho_phi / dt;  // one division per thread, not per cell
  // gridDim.y problems stacked along z: block row y sums the cells of problem y
  const long long ns = g.n / gridDim.y;
  const long long c0 = (long long)blockIdx.y * ns, c1 = c0 + ns;
  for (long long c = c0 + blockIdx.x * (long long)blockDim.x + threadIdx.x; c < c1;
       c += (long long)gridDim.x * blockDim.x) {
    int i = (int)(c % g.nx);
    long long r = c / g.nx;
    int j = (int)(r % g.ny);
    int k = (int)(r / g.ny);
    double pc = p[c], Kc = K[c];
    double ksc = ks ? ks[c] : so.ks;
    double sc = S[c], so_c = s_old[c];
    double phi = (sc - so_c) * rdt;
    double mag = (fabs(sc) + fabs(so_c)) * rdt;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      FaceNb nb;
      if (!face_neighbour(g, bc, so, f, i, j, k, c, p, K, nullptr, ksc, nb)) continue;
      int axis = f >> 1;
      double side = (f & 1) ? 1.0 : -1.0;
      double dL, dU;
      double ka = (f & 1) ? face_mean(axis_mean(kmean, axis), Kc, nb.K, pc, nb.p, dL, dU)
                          : face_mean(axis_mean(kmean, axis), nb.K, Kc, nb.p, pc, dL, dU);
      double t = ka * (pc - nb.p) * g.inv_h2[axis];
      double m = ka * (fabs(pc) + fabs(nb.p)) * g.inv_h2[axis];
      if (axis == 2) {
        t -= side * (Kc + nb.K) * 0.5 * g.inv_h[2];
        m += (Kc + nb.K) * 0.5 * g.inv_h[2];
      }
      phi += t;
      mag += m;
    }
    F[c] = phi;
    acc[0] += phi * phi;
    acc[1] += mag * mag;
    double a = fabs(phi);
    amax = (a > amax || a != a) ? a : amax;  // NaN propagates into the max
  }
  block_sum<2>(acc);
  double m = block_max(amax);
  if (threadIdx.x == 0) {  // partials[(q * nseg + seg) * gridDim.x + block]
    const long long S = gridDim.y, b = blockIdx.y * (long long)gridDim.x + blockIdx.x;
    partials[b] = acc[0];
    partials[S * gridDim.x + b] = m;
    partials[2 * S * gridDim.x + b] = acc[1];
  }
}

__global__ void k_assemble(GridP g, SoilP so, BCP bc, int kmean, const double* __restrict__ p,
                           const double* __restrict__ K, const double* __restrict__ dK,
                           const double* __restrict__ dS, const double* __restrict__ ks, double dt,
                           double* __restrict__ J7, double* __restrict__ A7) {
  const double rdt = so.rho_phi / dt;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.n;
       c += (long long)gridDim.x * blockDim.x) {
    int i = (int)(c % g.nx);
    long long r = c / g.nx;
    int j = (int)(r % g.ny);
    int k = (int)(r / g.ny);
    double pc = p[c], Kc = K[c], dKc = dK[c];
    double ksc = ks ? ks[c] : so.ks;
    double dj = dS[c] * rdt;
    double da = dj;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      FaceNb nb;
      double offj = 0.0, offa = 0.0;
      if (face_neighbour(g, bc, so, f, i, j, k, c, p, K, dK, ksc, nb)) {
        int axis = f >> 1;
        double side = (f & 1) ? 1.0 : -1.0;
        double dL, dU;
        double ka = (f & 1) ? face_mean(axis_mean(kmean, axis), Kc, nb.K, pc, nb.p, dL, dU)
                            : face_mean(axis_mean(kmean, axis), nb.K, Kc, nb.p, pc, dL, dU);
        double dself = (f & 1) ? dL : dU;
        double dnb = (f & 1) ? dU : dL;
        double w = ka * g.inv_h2[axis];
        double dp = (pc - nb.p) * g.inv_h2[axis];
        double dd = dself * dKc * dp + w;
        double off = dnb * nb.dK * dp - w;
        if (axis == 2) {
          dd -= side * dKc * 0.5 * g.inv_h[2];
          off -= side * nb.dK * 0.5 * g.inv_h[2];
        }
        dj += dd;
        da += w;
        if (nb.idx >= 0 || nb.idx == kInterfaceGhost) {  // a Dirichlet ghost is no unknown
          offj = off;
          offa = -w;
        }
      }
      J7[(1 + f) * g.n + c] = offj;
      A7[(1 + f) * g.n + c] = offa;
    }
    J7[c] = dj;
    A7[c] = da;
  }
}

// y = A x for a 7n stencil.  The neighbour coefficient is zero outside the grid,
// so the index is only guarded, never wrapped.
__global__ void __launch_bounds__(kLineThreads) k_stencil_spmv(GridP g, const double* __restrict__ A7,
                                                               const double* __restrict__ x, double* __restrict__ y) {
  int i = blockIdx.y * kLineThreads + threadIdx.x;
  if (i >= g.nx) return;
  int r = blockIdx.x;
  int j = r % g.ny;
  int k = r / g.ny;
  int nx = g.nx;
  int sxy = g.nx * g.ny;
  long long n = g.n;
  int c = r * nx + i;
  double s = A7[c] * x[c];
  if (i > 0) s += A7[1 * n + c] * x[c - 1];
  if (i < nx - 1) s += A7[2 * n + c] * x[c + 1];
  if (j > 0) s += A7[3 * n + c] * x[c - nx];
  if (j < g.ny - 1) s += A7[4 * n + c] * x[c + nx];
  if (k > 0) s += A7[5 * n + c] * x[c - sxy];
  if (k < g.nz - 1) s += A7[6 * n + c] * x[c + sxy];
  y[c] = s;
}

// Finest-level CSR pattern of the 7-point stencil (sorted columns: -z,-y,-x,c,+x,+y,+z).
__global__ void k_a0_rowcount(GridP g, int* __restrict__ cnt) {
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < g.n;
       c += (long long)gridDim.x * blockDim.x) {
    int i = (int)(c % g.nx);
    long long r = c / g.nx;
    int j = (int)(r % g.ny);
    int k = (int)(r / g.ny);
    cnt[c] = 1 + (i > 0) + (i < g.nx - 1) + (j > 0) + (j < g.ny - 1) + (k > 0) + (k < g.nz - 1);
  }
}

__global__ void k_a0_fill(GridP g, const int* __restrict__ rowptr, int* __restrict__ col,
                          const double* __restrict__ A7, double* __restrict__ val) {
  long long n = g.n;
  long long sxy = (long long)g.nx * g.ny;
  for (long long c = blockIdx.x * (long long)blockDim.x + threadIdx.x; c < n;
       c += (long long)gridDim.x * blockDim.x) {
    int i = (int)(c % g.nx);
    long long r = c / g.nx;
    int j = (int)(r % g.ny);
    int k = (int)(r / g.ny);
    int o = rowptr[c];
    // stencil slot order: 0 diag, 1 -x, 2 +x, 3 -y, 4 +y, 5 -z, 6 +z
    if (k > 0) { if (col) col[o] = (int)(c - sxy); if (val) val[o] = A7[5 * n + c]; ++o; }
    if (j > 0) { if (col) col[o] = (int)(c - g.nx); if (val) val[o] = A7[3 * n + c]; ++o; }
    if (i > 0) { if (col) col[o] = (int)(c - 1); if (val) val[o] = A7[1 * n + c]; ++o; }
    if (col) col[o] = (int)c;
    if (val) val[o] = A7[c];
    ++o;
    if (i < g.nx - 1) { if (col) col[o] = (int)(c + 1); if (val) val[o] = A7[2 * n + c]; ++o; }
    if (j < g.ny - 1) { if (col) col[o] = (int)(c + g.nx); if (val) val[o] = A7[4 * n + c]; ++o; }
    if (k < g.nz - 1) { if (col) col[o] = (int)(c + sxy); if (val) val[o] = A7[6 * n + c]; ++o; }
  }
}

// ---------------------------------------------------------------- host wrappers

int constit_eval(rich_ctx* c, const double* p) {
  k_constit<<<grid_for(c->g.n), kBlock, 0, c->st>>>(c->g.n, c->soil, p, c->ks, c->K, c->dK, c->S, c->dS);
  RICH_LAUNCH_CHECK();
  return RICH_OK;
}

int residual_eval(rich_ctx* c, const double* p, const double* s_old, double dt, double* F, bool want_norms,
                  bool constit_current, int nseg) {
  if (!constit_current) RICH_CHECK(constit_eval(c, p));
  int nb = red_grid(c->g.n / nseg);
  if ((long long)nb * nseg * 3 > (long long)kRedBlocks * 64) return RICH_ELIMIT;  // partials buffer
  {
    ProfScope ps("residual", c->st, (double)c->g.n * (32.0 + (c->ks ? 8.0 : 0.0)));
    k_residual<<<dim3(nb, nseg), kBlock, 0, c->st>>>(c->g, c->soil, c->bc, c->kmean, p, c->K, c->S, s_old, c->ks, dt,
                                                     F, c->partials);
  }
  RICH_LAUNCH_CHECK();
  if (want_norms) {  // dsc[q * nseg + s]: q = 0 ||F||^2, 1 ||F||_inf, 2 ||term magnitudes||^2
    const long long S = nseg;
    RICH_CHECK(finish_sums(c, c->partials, nb, nseg, c->dsc + 0));
    for (int s = 0; s < nseg; ++s) RICH_CHECK(finish_max(c, c->partials + (S + s) * nb, nb, c->dsc + S + s));
    RICH_CHECK(finish_sums(c, c->partials + 2 * S * nb, nb, nseg, c->dsc + 2 * S));
  }
  return RICH_OK;
}

int jacobian_eval(rich_ctx* c, const double* p, double dt, bool constit_current) {
  if (!constit_current) RICH_CHECK(constit_eval(c, p));
  {
    ProfScope ps("assemble", c->st, (double)c->g.n * (8.0 + (c->ks ? 8.0 : 0.0) + 14 * 8.0));
    k_assemble<<<grid_for(c->g.n), kBlock, 0, c->st>>>(c->g, c->soil, c->bc, c->kmean, p, c->K, c->dK, c->dS,
                                                      c->ks, dt, c->J7, c->A7);
  }
  RICH_LAUNCH_CHECK();
  c->have_jac = true;
  c->a0_fresh = false;
  return RICH_OK;
}

int stencil_apply(rich_ctx* c, const double* A7, const double* x, double* y) {
  ProfScope ps("stencil_spmv", c->st, (double)c->g.n * 72.0, (double)c->g.n * 13.0);
  k_stencil_spmv<<<line_grid(c->g), kLineThreads, 0, c->st>>>(c->g, A7, x, y);
  RICH_LAUNCH_CHECK();
  return RICH_OK;
}

int refresh_a0_values(rich_ctx* c) {
  if (c->a0_fresh) return RICH_OK;
  k_a0_fill<<<grid_for(c->g.n), kBlock, 0, c->st>>>(c->g, c->A0.rowptr, nullptr, c->A7, c->A0.val);
  RICH_LAUNCH_CHECK();
  c->a0_fresh = true;
  return RICH_OK;
}

static int build_a0_pattern(rich_ctx* c) {
  long long n = c->g.n;
  int* cnt = nullptr;
  RICH_CHECK(dalloc(&cnt, n));
  RICH_CHECK(dalloc(&c->A0.rowptr, n + 1));
  k_a0_rowcount<<<grid_for(n), kBlock, 0, c->st>>>(c->g, cnt);
  RICH_LAUNCH_CHECK();
  RICH_CHECK(scan_exclusive_int(c, cnt, c->A0.rowptr, n));
  long long nnz = n + 2LL * ((long long)(c->g.nx - 1) * c->g.ny * c->g.nz +
                             (long long)c->g.nx * (c->g.ny - 1) * c->g.nz +
                             (long long)c->g.nx * c->g.ny * (c->g.nz - 1));
  RICH_CHECK(dalloc(&c->A0.col, nnz));
  RICH_CHECK(dalloc(&c->A0.val, nnz));
  k_a0_fill<<<grid_for(n), kBlock, 0, c->st>>>(c->g, c->A0.rowptr, c->A0.col, c->A7, nullptr);
  RICH_LAUNCH_CHECK();
  c->A0.nrows = c->A0.ncols = (int)n;
  c->A0.nnz = nnz;
  RICH_CUDA(cudaStreamSynchronize(c->st));
  dfree(cnt);
  return RICH_OK;
}

}  // namespace rich

using namespace rich;

extern "C" {

const char* rich_last_cuda_error(void) { return g_cuda_err; }

const char* rich_strerror(int s) {
  switch (s) {
    case RICH_OK: return "ok";
    case RICH_EINVAL: return "invalid argument";
    case RICH_ENOMEM: return "device out of memory";
    case RICH_ECUDA: return "CUDA error";
    case RICH_ENOTCONV_LIN: return "Krylov solver did not converge";
    case RICH_ENOTCONV_NEWTON: return "Newton iteration did not converge";
    case RICH_ELINESEARCH: return "line search failed";
    case RICH_ENONFINITE: return "non-finite value";
    case RICH_ESTATE: return "call made before its prerequisite";
    case RICH_ELIMIT: return "implementation size limit exceeded";
    default: return "unknown status";
  }
}

void rich_default_amg_opts(rich_amg_opts* o) {
  o->theta = 0.08;
  o->seed = 1;
  o->coarse_max = 2000;
  o->max_levels = 10;
  o->nu1 = 1;
  o->nu2 = 1;
  o->smooth_levels = 10;
  o->product_lists = 1;
  o->aggregation = RICH_AGG_MIS2;
  o->max_agg_size = 8;
  o->smoother = RICH_SMOOTH_L1JACOBI;
  o->hgs_seg = 16;
  o->hgs_block = 16;
  o->precond = RICH_PRECOND_AMG;
  o->as_block = 8;
  o->as_overlap = 1;
  o->autotune = 1;
  o->isolated_join = 1;
  o->csr_layout = RICH_LAYOUT_AUTO;
  o->graph = 1;
}

void rich_default_newton_opts(rich_newton_opts* o) {
  o->krylov.kind = RICH_KRYLOV_FCG;
  o->krylov.restart = 30;
  o->krylov.eta = 1e-7;
  o->krylov.maxit = 200;
  o->krylov.stall = 0.0;
  rich_default_amg_opts(&o->amg);
  o->amg_policy = RICH_AMG_REFRESH;
  o->rtol = 1e-8;
  o->atol = 1e-30;
  o->max_newton = 50;
  o->armijo_c = 1e-4;
  o->lambda_min = 1e-10;
  o->fcg_fallback_restart = 30;
  o->max_dt_halvings = 0;
}

int rich_num_cells(const rich_ctx* c, long long* n) {
  if (!c || !n) return RICH_EINVAL;
  *n = c->g.n;
  return RICH_OK;
}

int rich_create(const rich_grid* grid, const rich_soil* soil, int kmean, const rich_bc* bc, int precision,
                void* stream, rich_ctx** out) {
  if (!grid || !soil || !bc || !out) return RICH_EINVAL;
  *out = nullptr;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1) return RICH_EINVAL;
  if (!(grid->lx > 0 && grid->ly > 0 && grid->lz > 0)) return RICH_EINVAL;
  for (int d = 0; d < 3; ++d)
    if (!(grid->h[d] >= 0.0) || !std::isfinite(grid->h[d])) return RICH_EINVAL;
  if (!kmean_valid(kmean) || (precision != RICH_PREC_FP64 && precision != RICH_PREC_MIXED)) return RICH_EINVAL;
  long long n = (long long)grid->nx * grid->ny * grid->nz;
  if (n > 2147483647LL / 8) return RICH_ELIMIT;  // 32-bit CSR indices of the 7-point pattern
  for (int f = 0; f < 6; ++f) {
    if (bc->kind[f] != RICH_BC_NOFLUX && bc->kind[f] != RICH_BC_DIRICHLET && bc->kind[f] != RICH_BC_INTERFACE)
      return RICH_EINVAL;
    if (bc->kind[f] == RICH_BC_INTERFACE && !bc->value_field_dev[f]) return RICH_EINVAL;  // ghost pressures
  }
  rich_ctx* c = new rich_ctx();
  c->g.nx = grid->nx;
  c->g.ny = grid->ny;
  c->g.nz = grid->nz;
  c->g.nzs = grid->nz;
  c->g.n = n;
  double h[3];
  grid_spacing(grid, h);
  for (int d = 0; d < 3; ++d) {
    c->g.inv_h[d] = 1.0 / h[d];
    c->g.inv_h2[d] = 1.0 / (h[d] * h[d]);
  }
  c->soil = SoilP{soil->alpha, soil->beta, soil->theta_s, soil->theta_r, soil->a, soil->gamma, soil->ks_const,
                  soil->rho_phi};
  for (int f = 0; f < 6; ++f) {
    c->bc.kind[f] = bc->kind[f];
    c->bc.value[f] = bc->value[f];
    c->bc.field[f] = nullptr;
    c->bc.gks[f] = nullptr;
  }
  c->kmean = kmean;
  c->prec = precision;
  c->st = (cudaStream_t)stream;
  cudaGetDevice(&c->device);
  AllocStream guard(c->st);
  int s = RICH_OK;
  auto fail = [&](int st_) {
    rich_destroy(c);
    return st_;
  };
  if ((s = dalloc(&c->K, n)) || (s = dalloc(&c->dK, n)) || (s = dalloc(&c->S, n)) || (s = dalloc(&c->dS, n)) ||
      (s = dalloc(&c->J7, 7 * n)) || (s = dalloc(&c->A7, 7 * n)) || (s = dalloc(&c->partials, (long long)kRedBlocks * 64)) ||
      (s = dalloc(&c->dsc, 256)) || (s = dalloc(&c->iflag, 16)))
    return fail(s);
  {
    // 128 doubles then 16 ints of pinned host memory from the process-wide pool
    char* blk = static_cast<char*>(pinned_get());
    if (!blk) return fail(RICH_ENOMEM);
    c->hsc = reinterpret_cast<double*>(blk);
    c->hflag = reinterpret_cast<int*>(blk + 128 * sizeof(double));
  }
  if (soil->ks_field_dev) {
    if ((s = dalloc(&c->ks, n))) return fail(s);
    if (cudaMemcpyAsync(c->ks, soil->ks_field_dev, n * sizeof(double), cudaMemcpyDeviceToDevice, c->st) !=
        cudaSuccess)
      return fail(RICH_ECUDA);
  }
  for (int f = 0; f < 6; ++f) {  // owned copies of per-cell Dirichlet values
    if (!bc->value_field_dev[f]) continue;
    int axis = f >> 1;
    long long m = axis == 2 ? (long long)grid->nx * grid->ny
                            : (axis == 1 ? (long long)grid->nx * grid->nz : (long long)grid->ny * grid->nz);
    double* dst = nullptr;
    if ((s = dalloc(&dst, m))) return fail(s);
    c->bc_fields[f] = dst;
    c->bc.field[f] = dst;
    if (cudaMemcpyAsync(dst, bc->value_field_dev[f], m * sizeof(double), cudaMemcpyDeviceToDevice, c->st) !=
        cudaSuccess)
      return fail(RICH_ECUDA);
    if (bc->kind[f] != RICH_BC_INTERFACE || !bc->ghost_ks_dev[f]) continue;
    double* gk = nullptr;
    if ((s = dalloc(&gk, m))) return fail(s);
    c->bc_gks[f] = gk;
    c->bc.gks[f] = gk;
    if (cudaMemcpyAsync(gk, bc->ghost_ks_dev[f], m * sizeof(double), cudaMemcpyDeviceToDevice, c->st) !=
        cudaSuccess)
      return fail(RICH_ECUDA);
  }
  if ((s = build_a0_pattern(c))) return fail(s);
  *out = c;
  return RICH_OK;
}

int rich_destroy(rich_ctx* c) {
  if (!c) return RICH_OK;
  AllocStream guard(c->st);
  cudaStreamSynchronize(c->st);
  amg_free(c);
  dfree(c->ks);
  dfree(c->K);
  dfree(c->dK);
  dfree(c->S);
  dfree(c->dS);
  dfree(c->J7);
  dfree(c->A7);
  dfree(c->A0.rowptr);
  dfree(c->A0.col);
  dfree(c->A0.val);
  dfree(c->partials);
  dfree(c->dsc);
  dfree(c->iflag);
  dfree(c->s_old);
  dfree(c->F);
  dfree(c->Ft);
  dfree(c->d);
  dfree(c->ptrial);
  dfree(c->rhs);
  dfree(c->pbuf);
  dfree(c->psave);
  for (int f = 0; f < 6; ++f) {
    dfree(c->bc_fields[f]);
    dfree(c->bc_gks[f]);
  }
  KrylovWork& k = c->kw;
  dfree(k.V);
  dfree(k.Z);
  dfree(k.x);
  dfree(k.r);
  dfree(k.p);
  dfree(k.q);
  dfree(k.qprev);
  dfree(k.z);
  dfree(k.w);
  dfree(k.hcoef);
  pinned_put(c->hsc);
  delete c;
  return RICH_OK;
}

int rich_pack_face(rich_ctx* c, int face, const double* field, double* out) {
  if (!c || face < 0 || face > 5 || !field || !out) return RICH_EINVAL;
  const int axis = face >> 1;
  const long long m = axis == 2 ? (long long)c->g.nx * c->g.ny
                                : (axis == 1 ? (long long)c->g.nx * c->g.nz : (long long)c->g.ny * c->g.nz);
  k_pack_face<<<grid_for(m), kBlock, 0, c->st>>>(c->g, face, m, field, out);
  RICH_LAUNCH_CHECK();
  return RICH_OK;
}

int rich_face_apply(rich_ctx* c, int face, int which, const double* ghost, double* y) {
  if (!c || face < 0 || face > 5 || (which != 0 && which != 1) || !ghost || !y) return RICH_EINVAL;
  if (c->bc.kind[face] != RICH_BC_INTERFACE) return RICH_EINVAL;
  if (!c->have_jac) return RICH_ESTATE;
  const int axis = face >> 1;
  const long long m = axis == 2 ? (long long)c->g.nx * c->g.ny
                                : (axis == 1 ? (long long)c->g.nx * c->g.nz : (long long)c->g.ny * c->g.nz);
  k_face_apply<<<grid_for(m), kBlock, 0, c->st>>>(c->g, face, m, which ? c->A7 : c->J7, ghost, y);
  RICH_LAUNCH_CHECK();
  return RICH_OK;
}

int rich_set_face_values(rich_ctx* c, int face, const double* values) {
  if (!c || face < 0 || face > 5 || !values) return RICH_EINVAL;
  if (!c->bc_fields[face]) return RICH_ESTATE;
  const int axis = face >> 1;
  const long long m = axis == 2 ? (long long)c->g.nx * c->g.ny
                                : (axis == 1 ? (long long)c->g.nx * c->g.nz : (long long)c->g.ny * c->g.nz);
  RICH_CUDA(cudaMemcpyAsync(c->bc_fields[face], values, m * sizeof(double), cudaMemcpyDeviceToDevice, c->st));
  return RICH_OK;
}

int rich_saturation(rich_ctx* c, const double* p, double* s) {
  if (!c || !p || !s) return RICH_EINVAL;
  AllocStream guard(c->st);
  k_saturation<<<grid_for(c->g.n), kBlock, 0, c->st>>>(c->g.n, c->soil, p, s);
  RICH_LAUNCH_CHECK();
  return RICH_OK;
}

int rich_residual(rich_ctx* c, const double* p, const double* s_old, double dt, double* F, double* norms) {
  if (!c || !p || !s_old || !F || !(dt > 0)) return RICH_EINVAL;
  AllocStream guard(c->st);
  RICH_CHECK(residual_eval(c, p, s_old, dt, F, norms != nullptr));
  if (norms) {
    double h[2];
    RICH_CHECK(fetch_scalars(c, c->dsc, 2, h));
    norms[0] = sqrt(h[0]);
    norms[1] = h[1];
    if (!std::isfinite(norms[0]) || !std::isfinite(norms[1])) return RICH_ENONFINITE;
  }
  return RICH_OK;
}

int rich_residual3(rich_ctx* c, const double* p, const double* s_old, double dt, double* F, double* norms) {
  if (!c || !p || !s_old || !F || !norms || !(dt > 0)) return RICH_EINVAL;
  AllocStream guard(c->st);
  RICH_CHECK(residual_eval(c, p, s_old, dt, F, true));
  double h[3];
  RICH_CHECK(fetch_scalars(c, c->dsc, 3, h));  // ||F||^2, ||F||_inf, ||m||^2
  norms[0] = sqrt(h[0]);
  norms[1] = h[1];
  norms[2] = sqrt(h[2]);
  if (!std::isfinite(norms[0]) || !std::isfinite(norms[1])) return RICH_ENONFINITE;
  return RICH_OK;
}

int rich_jacobian(rich_ctx* c, const double* p, double dt, double* J7, double* A7) {
  if (!c || !p || !(dt > 0)) return RICH_EINVAL;
  AllocStream guard(c->st);
  RICH_CHECK(jacobian_eval(c, p, dt));
  long long bytes = 7 * c->g.n * (long long)sizeof(double);
  if (J7) RICH_CUDA(cudaMemcpyAsync(J7, c->J7, bytes, cudaMemcpyDeviceToDevice, c->st));
  if (A7) RICH_CUDA(cudaMemcpyAsync(A7, c->A7, bytes, cudaMemcpyDeviceToDevice, c->st));
  return RICH_OK;
}

int rich_jacobian_apply(rich_ctx* c, const double* x, double* y) {
  if (!c || !x || !y) return RICH_EINVAL;
  AllocStream guard(c->st);
  if (!c->have_jac) return RICH_ESTATE;
  return stencil_apply(c, c->J7, x, y);
}

}  // extern "C"
