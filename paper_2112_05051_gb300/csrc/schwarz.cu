// One-level additive Schwarz preconditioner with ILU(0) subdomain solves
// (Sec. 5.2, eq. (AS); the setup of Sec. 6: one layer of overlap, ILU with no
// fill-in on each subdomain matrix):
//
//     M_AS^{-1} = sum_t R_t^T M_t^{-1} R_t,   M_t = R_t A_aux R_t^T.
//
// On one GPU a subdomain is a box of the grid instead of a process: the cells are
// tiled by boxes of `as_block` cells per side, and subdomain t is box t grown by
// `as_overlap` layers (clipped to the grid).  One thread block owns a subdomain
// and keeps its vectors in shared memory.
//
// ILU(0) in the subdomain's lexicographic order: for the 7-point matrix the
// elimination never updates an off-diagonal entry (two neighbours of a cell are
// never neighbours of each other), so the factors are L = I + L_A D^-1 and
// U = D + U_A with D_c = m_cc - sum over the lower neighbours k of m_ck^2 / D_k.
// Every recurrence runs over wavefronts li + lj + lk = w of the box: the lower
// neighbours of a cell lie on the previous wavefront.  The contributions of the
// (up to eight) subdomains that cover a cell are summed by a gather in a fixed
// order, so the result does not depend on scheduling.
#include "common.cuh"

namespace rich {

struct Box {
  int a0, b0, c0;  // origin of the extended box in the grid
  int ex, ey, ez;  // extents
};

__device__ __forceinline__ Box as_box(const GridP& g, int bs, int ov, int t) {
  int tx = (g.nx + bs - 1) / bs, ty = (g.ny + bs - 1) / bs;
  int ti = t % tx, tj = (t / tx) % ty, tk = t / (tx * ty);
  int i0 = ti * bs, j0 = tj * bs, k0 = tk * bs;
  Box b;
  b.a0 = max(0, i0 - ov);
  b.b0 = max(0, j0 - ov);
  b.c0 = max(0, k0 - ov);
  b.ex = min(g.nx, i0 + bs + ov) - b.a0;
  b.ey = min(g.ny, j0 + bs + ov) - b.b0;
  b.ez = min(g.nz, k0 + bs + ov) - b.c0;
  return b;
}

// D of the ILU(0) of every subdomain matrix (stride E^3 per subdomain, E = bs + 2 ov).
template <class T>
__global__ void k_as_factor(GridP g, Stencil4<T> A, int bs, int ov, T* __restrict__ Dall) {
  extern __shared__ unsigned char smem_raw[];
  T* D = reinterpret_cast<T*>(smem_raw);
  const int E = bs + 2 * ov;
  const Box b = as_box(g, bs, ov, blockIdx.x);
  const int nloc = b.ex * b.ey * b.ez;
  const int nx = g.nx, sxy = g.nx * g.ny;
  for (int w = 0; w <= b.ex + b.ey + b.ez - 3; ++w) {
    for (int q = threadIdx.x; q < nloc; q += blockDim.x) {
      int li = q % b.ex, lj = (q / b.ex) % b.ey, lk = q / (b.ex * b.ey);
      if (li + lj + lk != w) continue;
      int c = (b.a0 + li) + nx * ((b.b0 + lj) + g.ny * (b.c0 + lk));
      T d = A.diag[c];
      if (li > 0) { T a = A.wx[c - 1]; d -= a * a / D[q - 1]; }
      if (lj > 0) { T a = A.wy[c - nx]; d -= a * a / D[q - b.ex]; }
      if (lk > 0) { T a = A.wz[c - sxy]; d -= a * a / D[q - b.ex * b.ey]; }
      D[q] = d;
    }
    __syncthreads();
  }
  T* out = Dall + (long long)blockIdx.x * E * E * E;
  for (int q = threadIdx.x; q < nloc; q += blockDim.x) out[q] = D[q];
}

// y = (L U)^{-1} r on every subdomain, into zpart (stride E^3 per subdomain).
template <class T>
__global__ void k_as_solve(GridP g, Stencil4<T> A, int bs, int ov, const T* __restrict__ Dall,
                           const T* __restrict__ r, T* __restrict__ zpart) {
  extern __shared__ unsigned char smem_raw[];
  const int E = bs + 2 * ov;
  T* D = reinterpret_cast<T*>(smem_raw);
  T* y = D + E * E * E;
  const Box b = as_box(g, bs, ov, blockIdx.x);
  const int nloc = b.ex * b.ey * b.ez;
  const int nx = g.nx, sxy = g.nx * g.ny;
  const T* Dt = Dall + (long long)blockIdx.x * E * E * E;
  for (int q = threadIdx.x; q < nloc; q += blockDim.x) D[q] = Dt[q];
  __syncthreads();
  const int W = b.ex + b.ey + b.ez - 3;
  // (D + L_A) t = r, couplings -w: t_c = (r_c + sum over lower neighbours of w t_nb) / D_c
  for (int w = 0; w <= W; ++w) {
    for (int q = threadIdx.x; q < nloc; q += blockDim.x) {
      int li = q % b.ex, lj = (q / b.ex) % b.ey, lk = q / (b.ex * b.ey);
      if (li + lj + lk != w) continue;
      int c = (b.a0 + li) + nx * ((b.b0 + lj) + g.ny * (b.c0 + lk));
      T s = r[c];
      if (li > 0) s += A.wx[c - 1] * y[q - 1];
      if (lj > 0) s += A.wy[c - nx] * y[q - b.ex];
      if (lk > 0) s += A.wz[c - sxy] * y[q - b.ex * b.ey];
      y[q] = s / D[q];
    }
    __syncthreads();
  }
  // y_c = t_c + (sum over upper neighbours of w y_nb) / D_c, backward
  for (int w = W; w >= 0; --w) {
    for (int q = threadIdx.x; q < nloc; q += blockDim.x) {
      int li = q % b.ex, lj = (q / b.ex) % b.ey, lk = q / (b.ex * b.ey);
      if (li + lj + lk != w) continue;
      int c = (b.a0 + li) + nx * ((b.b0 + lj) + g.ny * (b.c0 + lk));
      T s = 0;
      if (li < b.ex - 1) s += A.wx[c] * y[q + 1];
      if (lj < b.ey - 1) s += A.wy[c] * y[q + b.ex];
      if (lk < b.ez - 1) s += A.wz[c] * y[q + b.ex * b.ey];
      y[q] = y[q] + s / D[q];
    }
    __syncthreads();
  }
  T* out = zpart + (long long)blockIdx.x * E * E * E;
  for (int q = threadIdx.x; q < nloc; q += blockDim.x) out[q] = y[q];
}

// z_c = sum of the subdomain solutions covering c, subdomains in increasing order.
template <class T>
__global__ void __launch_bounds__(kLineThreads) k_as_gather(GridP g, int bs, int ov, const T* __restrict__ zpart,
                                                            T* __restrict__ z) {
  int i = blockIdx.y * kLineThreads + threadIdx.x;
  if (i >= g.nx) return;
  int r = blockIdx.x;
  int j = r % g.ny, k = r / g.ny;
  const int E = bs + 2 * ov;
  const int tx = (g.nx + bs - 1) / bs, ty = (g.ny + bs - 1) / bs, tz = (g.nz + bs - 1) / bs;
  int ti0 = max(0, (i - ov) / bs), ti1 = min(tx - 1, (i + ov) / bs);
  int tj0 = max(0, (j - ov) / bs), tj1 = min(ty - 1, (j + ov) / bs);
  int tk0 = max(0, (k - ov) / bs), tk1 = min(tz - 1, (k + ov) / bs);
  T s = 0;
  for (int tk = tk0; tk <= tk1; ++tk)
    for (int tj = tj0; tj <= tj1; ++tj)
      for (int ti = ti0; ti <= ti1; ++ti) {
        int t = ti + tx * (tj + ty * tk);
        Box b = as_box(g, bs, ov, t);
        int li = i - b.a0, lj = j - b.b0, lk = k - b.c0;
        if (li < 0 || lj < 0 || lk < 0 || li >= b.ex || lj >= b.ey || lk >= b.ez) continue;
        s += zpart[(long long)t * E * E * E + li + b.ex * (lj + b.ey * lk)];
      }
  z[(long long)r * g.nx + i] = s;
}

static long long as_tiles(const GridP& g, int bs) {
  long long tx = (g.nx + bs - 1) / bs, ty = (g.ny + bs - 1) / bs, tz = (g.nz + bs - 1) / bs;
  return tx * ty * tz;
}

template <class T>
static int as_factor_t(rich_ctx* c, const Stencil4<T>& A) {
  Hierarchy& H = c->H;
  const int bs = H.opts.as_block, ov = H.opts.as_overlap, E = bs + 2 * ov;
  const long long nt = as_tiles(c->g, bs);
  size_t smem = sizeof(T) * (size_t)E * E * E;
  k_as_factor<T><<<(unsigned)nt, 128, smem, c->st>>>(c->g, A, bs, ov, (T*)H.asD);
  RICH_LAUNCH_CHECK();
  return RICH_OK;
}

int as_setup(rich_ctx* c) {
  Hierarchy& H = c->H;
  const int bs = H.opts.as_block, ov = H.opts.as_overlap;
  if (bs < 1 || ov < 0 || bs + 2 * ov > 24) return RICH_EINVAL;  // the subdomain lives in shared memory
  const int E = bs + 2 * ov;
  const long long nt = as_tiles(c->g, bs);
  if (nt > 2147483647LL) return RICH_ELIMIT;
  const bool mp = c->prec == RICH_PREC_MIXED;
  const size_t es = mp ? sizeof(float) : sizeof(double);
  if (!H.asD) {
    char *d = nullptr, *z = nullptr;
    RICH_CHECK(dalloc(&d, nt * E * E * E * (long long)es));
    RICH_CHECK(dalloc(&z, nt * E * E * E * (long long)es));
    H.asD = d;
    H.asZ = z;
    if (mp) {
      RICH_CHECK(dalloc(&H.asR32, c->g.n));
      RICH_CHECK(dalloc(&H.asZ32, c->g.n));
    }
    // dynamic shared memory above 48 KB needs the opt-in (E = 24 in FP64: 108 KB and 216 KB)
    const size_t smem1 = es * (size_t)E * E * E, smem2 = 2 * smem1;
    if (smem1 > 48 * 1024) {
      if (mp) RICH_CUDA(cudaFuncSetAttribute(k_as_factor<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1));
      else RICH_CUDA(cudaFuncSetAttribute(k_as_factor<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem1));
    }
    if (smem2 > 48 * 1024) {
      if (mp) RICH_CUDA(cudaFuncSetAttribute(k_as_solve<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
      else RICH_CUDA(cudaFuncSetAttribute(k_as_solve<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem2));
    }
  }
  return mp ? as_factor_t<float>(c, H.st32) : as_factor_t<double>(c, H.st64);
}

void as_free(rich_ctx* c) {
  Hierarchy& H = c->H;
  char* d = static_cast<char*>(H.asD);
  char* z = static_cast<char*>(H.asZ);
  dfree(d);
  dfree(z);
  H.asD = H.asZ = nullptr;
  dfree(H.asR32);
  dfree(H.asZ32);
}

__global__ void k_as_d2f(long long n, const double* __restrict__ a, float* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void k_as_f2d(long long n, const float* __restrict__ a, double* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

template <class T>
static int as_apply_t(rich_ctx* c, const Stencil4<T>& A, const T* r, T* z) {
  Hierarchy& H = c->H;
  const int bs = H.opts.as_block, ov = H.opts.as_overlap, E = bs + 2 * ov;
  const long long nt = as_tiles(c->g, bs);
  size_t smem = 2 * sizeof(T) * (size_t)E * E * E;
  {
    ProfScope ps("as_solve", c->st, (double)c->g.n * sizeof(T) * 14.0);
    k_as_solve<T><<<(unsigned)nt, 128, smem, c->st>>>(c->g, A, bs, ov, (const T*)H.asD, r, (T*)H.asZ);
  }
  RICH_LAUNCH_CHECK();
  k_as_gather<T><<<line_grid(c->g), kLineThreads, 0, c->st>>>(c->g, bs, ov, (const T*)H.asZ, z);
  RICH_LAUNCH_CHECK();
  return RICH_OK;
}

int as_apply(rich_ctx* c, const double* r, double* z) {
  Hierarchy& H = c->H;
  const long long n = c->g.n;
  if (c->prec == RICH_PREC_MIXED) {
    k_as_d2f<<<grid_for(n), kBlock, 0, c->st>>>(n, r, H.asR32);
    RICH_LAUNCH_CHECK();
    RICH_CHECK(as_apply_t<float>(c, H.st32, H.asR32, H.asZ32));
    k_as_f2d<<<grid_for(n), kBlock, 0, c->st>>>(n, H.asZ32, z);
    RICH_LAUNCH_CHECK();
    return RICH_OK;
  }
  return as_apply_t<double>(c, H.st64, r, z);
}

}  // namespace rich
