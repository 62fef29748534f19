// Residual evaluation that allocates nothing (rich_residual_noalloc).
//
// Some callers cannot call cudaMalloc at the point where they need a residual:
// a serving loop that runs with a fixed, pre-reserved device memory budget, code
// that must not trigger the implicit device synchronisation a fresh allocation
// can cause, or an embedding application whose allocator owns all device memory.
// For them this entry point needs no context and no allocation: the caller
// passes the inputs and the output buffer, the block partial sums of the norms
// live in a fixed file-scope device array, and the constitutive values of each
// cell's neighbours are recomputed in registers instead of being stored.
//
// The scratch array holds 2 partial sums for each of at most kNoAllocMaxBlocks
// blocks of kNoAllocCells cells, so grids up to kNoAllocMaxBlocks * kNoAllocCells
// = 134,217,728 cells (512^3) are accepted; larger ones return RICH_ELIMIT.  The
// array (about 1 MB) stays resident on every device that loads the library until
// the process exits.  All calls share it: every call rewrites all the partials it
// reads, so nothing carries over between calls, but calls that overlap on the GPU
// (different streams, or different host threads) race on it and must be
// serialised by the caller.
#include <mutex>

#include "common.cuh"

namespace rich {

constexpr int kNoAllocThreads = 256;
constexpr int kNoAllocItems = 8;  // cells per thread
constexpr long long kNoAllocCells = (long long)kNoAllocThreads * kNoAllocItems;
constexpr int kNoAllocMaxBlocks = 65536;
constexpr int kNoAllocSlots = 2 * kNoAllocMaxBlocks + 8;  // partials, then the two results
// block_sum / block_max size their shared arrays and final warp pass by kBlock
static_assert(kNoAllocThreads == kBlock, "the norm reductions assume kBlock threads per block");

static __device__ __align__(256) double g_noalloc_scratch[kNoAllocSlots];

// Neighbour of face f of cell c (conductivity recomputed from its pressure).
__device__ __forceinline__ bool noalloc_face(const GridP& g, const BCP& bc, const SoilP& so, int f, int i, int j,
                                             int k, long long c, const double* __restrict__ p,
                                             const double* __restrict__ ks, double ksc, double& pn, double& Kn) {
  int axis = f >> 1;
  int side = (f & 1) ? 1 : -1;
  int coord = axis == 0 ? i : (axis == 1 ? j : k);
  int extent = axis == 0 ? g.nx : (axis == 1 ? g.ny : g.nz);
  bool bnd = side > 0 ? (coord == extent - 1) : (coord == 0);
  if (bnd) {
    if (bc.kind[f] == RICH_BC_NOFLUX) return false;
    pn = bc_value(bc, f, i, j, k, g.nx, g.ny);
    Kn = conductivity_only(pn, ksc, so);
    return true;
  }
  long long stride = axis == 0 ? 1LL : (axis == 1 ? (long long)g.nx : (long long)g.nx * g.ny);
  long long q = c + side * stride;
  pn = p[q];
  Kn = conductivity_only(pn, ks ? ks[q] : so.ks, so);
  return true;
}

__global__ void __launch_bounds__(kNoAllocThreads) k_residual_noalloc(
    GridP g, SoilP so, BCP bc, int kmean, const double* __restrict__ p, const double* __restrict__ s_old,
    const double* __restrict__ ks, double dt, double* __restrict__ F, double* __restrict__ scratch) {
  double acc[1] = {0.0};
  double amax = 0.0;
  long long base = (long long)blockIdx.x * kNoAllocCells;
  for (int t = 0; t < kNoAllocItems; ++t) {
    long long c = base + (long long)t * kNoAllocThreads + threadIdx.x;
    if (c >= g.n) break;
    int i = (int)(c % g.nx);
    long long r = c / g.nx;
    int j = (int)(r % g.ny);
    int k = (int)(r / g.ny);
    double pc = p[c];
    double ksc = ks ? ks[c] : so.ks;
    double Sc, dSc, Kc, dKc;
    constit(pc, ksc, so, Sc, dSc, Kc, dKc);
    double phi = so.rho_phi * (Sc - s_old[c]) / dt;
#pragma unroll
    for (int f = 0; f < 6; ++f) {
      double pn, Kn;
      if (!noalloc_face(g, bc, so, f, i, j, k, c, p, ks, ksc, pn, Kn)) continue;
      int axis = f >> 1;
      double side = (f & 1) ? 1.0 : -1.0;
      double dL, dU;
      const int km = axis_mean(kmean, f >> 1);
      double ka = (f & 1) ? face_mean(km, Kc, Kn, pc, pn, dL, dU) : face_mean(km, Kn, Kc, pn, pc, dL, dU);
      double tt = ka * (pc - pn) * g.inv_h2[axis];
      if (axis == 2) tt -= side * (Kc + Kn) * 0.5 * g.inv_h[2];
      phi += tt;
    }
    F[c] = phi;
    acc[0] += phi * phi;
    double a = fabs(phi);
    amax = (a > amax || a != a) ? a : amax;
  }
  block_sum<1>(acc);
  double m = block_max(amax);
  if (threadIdx.x == 0) {
    scratch[blockIdx.x] = acc[0];
    scratch[kNoAllocMaxBlocks + blockIdx.x] = m;
  }
}

// One block: sum / max of the nb partials in block order; results at slots 2*max, 2*max+1.
__global__ void k_residual_noalloc_finish(int nb, double* __restrict__ scratch) {
  double v[1] = {0.0};
  double m = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    v[0] += scratch[b];
    double a = scratch[kNoAllocMaxBlocks + b];
    m = (a > m || a != a) ? a : m;
  }
  block_sum<1>(v);
  m = block_max(m);
  if (threadIdx.x == 0) {
    scratch[2 * kNoAllocMaxBlocks] = v[0];
    scratch[2 * kNoAllocMaxBlocks + 1] = m;
  }
}

// Device address of the scratch array, looked up once per device with that
// device current (in host code the symbol itself is only a host-side stand-in).
static std::mutex g_noalloc_mu;
static double* g_noalloc_ptr[64] = {nullptr};

static int noalloc_scratch(double** out) {
  int dev = 0;
  RICH_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return RICH_ELIMIT;
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_ptr[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) {
      set_cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
      return RICH_ECUDA;
    }
    g_noalloc_ptr[dev] = (double*)ptr;
  }
  *out = g_noalloc_ptr[dev];
  return RICH_OK;
}

}  // namespace rich

using namespace rich;

extern "C" int rich_residual_noalloc(const rich_grid* grid, const rich_soil* soil, int kmean, const rich_bc* bc,
                                     const double* p_dev, const double* s_old_dev, double dt, double* F_dev,
                                     double* norms_host, void* stream) {
  if (!grid || !soil || !bc || !p_dev || !s_old_dev || !F_dev || !(dt > 0)) return RICH_EINVAL;
  if (grid->nx < 1 || grid->ny < 1 || grid->nz < 1 || !(grid->lx > 0 && grid->ly > 0 && grid->lz > 0) ||
      !(grid->h[0] >= 0.0 && grid->h[1] >= 0.0 && grid->h[2] >= 0.0))
    return RICH_EINVAL;
  if (!kmean_valid(kmean)) return RICH_EINVAL;
  for (int f = 0; f < 6; ++f)
    if (bc->kind[f] != RICH_BC_NOFLUX && bc->kind[f] != RICH_BC_DIRICHLET) return RICH_EINVAL;
  long long n = (long long)grid->nx * grid->ny * grid->nz;
  long long nb = (n + kNoAllocCells - 1) / kNoAllocCells;
  if (nb > kNoAllocMaxBlocks) return RICH_ELIMIT;  // beyond 134,217,728 cells
  double* scratch = nullptr;
  RICH_CHECK(noalloc_scratch(&scratch));
  GridP g;
  g.nx = grid->nx;
  g.ny = grid->ny;
  g.nz = grid->nz;
  g.nzs = grid->nz;
  g.n = n;
  double h[3];
  grid_spacing(grid, h);
  for (int d = 0; d < 3; ++d) {
    g.inv_h[d] = 1.0 / h[d];
    g.inv_h2[d] = 1.0 / (h[d] * h[d]);
  }
  SoilP so{soil->alpha, soil->beta, soil->theta_s, soil->theta_r, soil->a, soil->gamma, soil->ks_const,
           soil->rho_phi};
  BCP b;
  for (int f = 0; f < 6; ++f) {
    b.kind[f] = bc->kind[f];
    b.value[f] = bc->value[f];
    b.field[f] = bc->value_field_dev[f];
    b.gks[f] = nullptr;
  }
  cudaStream_t st = (cudaStream_t)stream;
  k_residual_noalloc<<<(int)nb, kNoAllocThreads, 0, st>>>(g, so, b, kmean, p_dev, s_old_dev, soil->ks_field_dev, dt,
                                                          F_dev, scratch);
  RICH_LAUNCH_CHECK();
  if (norms_host) {
    k_residual_noalloc_finish<<<1, kBlock, 0, st>>>((int)nb, scratch);
    RICH_LAUNCH_CHECK();
    double r[2];
    RICH_CUDA(cudaMemcpyAsync(r, scratch + 2 * kNoAllocMaxBlocks, 2 * sizeof(double), cudaMemcpyDeviceToHost, st));
    RICH_CUDA(cudaStreamSynchronize(st));
    norms_host[0] = sqrt(r[0]);
    norms_host[1] = r[1];
    if (!std::isfinite(norms_host[0]) || !std::isfinite(norms_host[1])) return RICH_ENONFINITE;
  }
  return RICH_OK;
}
