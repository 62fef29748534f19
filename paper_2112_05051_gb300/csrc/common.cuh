// Shared definitions of the GB300 Richards solver: context, sparse/level structs,
// launch helpers, deterministic block reductions and the constitutive law.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/richards.h"

namespace rich {

constexpr int kBlock = 256;          // threads per block of every elementwise kernel
constexpr int kNumSM = 152;          // GB300 SM count (2 dies x 76)
constexpr int kRedBlocks = 8 * kNumSM;  // fixed grid of the reduction kernels (deterministic order)

void set_cuda_error(cudaError_t e, const char* where);

#define RICH_CUDA(call)                                              \
  do {                                                               \
    cudaError_t e_ = (call);                                         \
    if (e_ != cudaSuccess) {                                         \
      ::rich::set_cuda_error(e_, #call);                             \
      return RICH_ECUDA;                                             \
    }                                                                \
  } while (0)

#define RICH_CHECK(...)                  \
  do {                                   \
    int s_ = (__VA_ARGS__);              \
    if (s_ != RICH_OK) return s_;        \
  } while (0)

// Every kernel launch is followed by RICH_LAUNCH_CHECK, which also counts it.
void count_launch();
void count_launches(long long k);  // k may be negative (launches recorded into a graph)
#define RICH_LAUNCH_CHECK()        \
  do {                             \
    ::rich::count_launch();        \
    RICH_CUDA(cudaGetLastError()); \
  } while (0)

// Optional live timing of one named kernel: when its name matches the profiling
// target, CUDA events are recorded around its launches on the launching stream.
// Moves the start of the open timed launch to now (work done on the stream since
// it opened, e.g. a one-time layout, is not charged to the launch).
void prof_restart(cudaStream_t st);
// Corrects the algorithmic bytes and flops of the last timed launch if it was `name`
// (for launches whose work a device-side decision settled after they were queued).
void prof_adjust_last(const char* name, double bytes, double flops);
struct ProfScope {
  bool on;
  cudaStream_t st;
  double bytes, flops;
  ProfScope(const char* name, cudaStream_t s, double algorithmic_bytes, double algorithmic_flops = 0.0);
  ~ProfScope();
};

inline int grid_for(long long n, int block = kBlock) {
  long long g = (n + block - 1) / block;
  if (g < 1) g = 1;
  if (g > 2147483647LL) g = 2147483647LL;
  return (int)g;
}
inline int red_grid(long long n) {
  long long g = (n + kBlock - 1) / kBlock;
  if (g > kRedBlocks) g = kRedBlocks;
  if (g < 1) g = 1;
  return (int)g;
}

struct SoilP {
  double alpha, beta, ts, tr, a, gamma, ks, rho_phi;
};

struct GridP {
  int nx, ny, nz;
  int nzs;           // layers per stacked problem (nz unless a batch stacks several problems along z)
  long long n;
  double inv_h[3];   // 1/h_d
  double inv_h2[3];  // 1/h_d^2
};

struct BCP {
  int kind[6];
  double value[6];
  const double* field[6];  // per-cell Dirichlet values (ghost pressures of an interface face), or nullptr
  const double* gks[6];    // interface faces: per-cell K_s of the ghost cells, or nullptr (soil ks)
};

// Cell spacing of a grid: the explicit h[d] where given, else l / (n + 1).
inline void grid_spacing(const rich_grid* g, double h[3]) {
  h[0] = g->h[0] > 0 ? g->h[0] : g->lx / (g->nx + 1);
  h[1] = g->h[1] > 0 ? g->h[1] : g->ly / (g->ny + 1);
  h[2] = g->h[2] > 0 ? g->h[2] : g->lz / (g->nz + 1);
}

// Index of the boundary cell (i, j, k) in the per-cell arrays of face f.
__device__ __forceinline__ long long face_index(int f, int i, int j, int k, int nx, int ny) {
  int axis = f >> 1;
  return axis == 2 ? (long long)i + (long long)nx * j
                   : (axis == 1 ? (long long)i + (long long)nx * k : (long long)j + (long long)ny * k);
}

// Dirichlet value of face f at the boundary cell (i, j, k).
__device__ __forceinline__ double bc_value(const BCP& bc, int f, int i, int j, int k, int nx, int ny) {
  const double* fv = bc.field[f];
  if (!fv) return bc.value[f];
  return fv[face_index(f, i, j, k, nx, ny)];
}

template <class T>
struct Csr {
  int nrows = 0, ncols = 0;
  long long nnz = 0;
  int* rowptr = nullptr;
  int* col = nullptr;
  T* val = nullptr;
};

// SELL-C-sigma copy of a CSR matrix for the coarse-level row operations: rows are
// sorted by decreasing length within windows of kSellSigma rows and cut into slices
// of kSellC = 32 (one warp, one thread per row); slice s is stored column by column,
// slot sptr[s] + 32 j + t holding the j-th entry of row perm[32 s + t] (value and
// column), or a zero with column 0 past the end of that row.  Loads of a slice are
// coalesced and a row needs no cross-lane reduction.
constexpr int kSellC = 32;
constexpr int kSellSigma = 1024;
constexpr int kSellMinRows = 2048;
struct Sell {
  int nrows = 0, nslice = 0;
  long long slots = 0;
  int* sptr = nullptr;      // nslice + 1 slot offsets
  int* perm = nullptr;      // 32 nslice rows, -1 past nrows
  int* col = nullptr;       // slots
  double* val = nullptr;    // values for an FP64 hierarchy
  float* val32 = nullptr;   // values for an FP32 hierarchy (MIXED)
  bool built() const { return sptr != nullptr; }
};

// One level of the AMG hierarchy.  Level 0 holds the diffusion matrix of the
// finest grid; levels 1.. hold Galerkin products.  FP32 copies exist in MIXED mode.
// Galerkin refresh by product lists: entry q of C = A B is the sum over
// t in [start(q), start(q+1)) of a[pa[t]] * b[pb[t]], the pairs sorted by A
// entry; start(q) = base[q >> kPlShift] + seg[q] (64-bit pair offsets stored as
// one base per 2^kPlShift entries plus a 32-bit remainder).
constexpr int kPlShift = 10;
struct ProdList {
  int* seg = nullptr;        // nnz(C) + 1 offsets within the entry's chunk
  long long* base = nullptr; // (nnz(C) >> kPlShift) + 1 chunk offsets
  int* pa = nullptr;         // A entry of each pair
  int* pb = nullptr;         // B entry of each pair
  long long np = 0;          // pairs (= scalar products of C = A B)
};

struct Level {
  int n = 0;
  Csr<double> A;
  float* A32 = nullptr;            // values of A in FP32 (pattern of A)
  double* dinv = nullptr;          // 1 / sum_j |a_ij|
  float* dinv32 = nullptr;
  int* agg = nullptr;              // aggregate of each node (levels with a coarser level)
  Csr<double> P, R, AP;            // to the next level; AP = A P (pattern kept for refresh)
  int* u_ap = nullptr;             // products per row of A P and of R (A P) (refresh kernels' split)
  int* u_rap = nullptr;
  float* P32 = nullptr;            // values of P/R in FP32
  float* R32 = nullptr;
  float* AP32 = nullptr;           // values of A P in FP32 (MIXED-precision refresh)
  ProdList pl_ap, pl_rap;          // product lists of A P and R (A P), built at the first refresh
  Sell sA, sP, sR;                 // SELL-C-sigma copies (levels with >= kSellMinRows rows)
  bool pl_tried = false;
  int mis_rounds = 0;
  double omega = 0.0;
  // V-cycle work vectors, typed by the hierarchy precision (double or float)
  void* x = nullptr;
  void* b = nullptr;
  void* r = nullptr;
  void* t = nullptr;
};

// Finest level of the V-cycle in stencil form: the diffusion matrix is symmetric
// with non-negative face weights w (coupling -w), so four arrays hold it:
// diagonal, and the +x, +y, +z face weights of each cell (0 on the boundary).
template <class T>
struct Stencil4 {
  T* diag = nullptr;
  T* wx = nullptr;
  T* wy = nullptr;
  T* wz = nullptr;
  T* dinv = nullptr;  // 1 / (diag + sum of the six face weights), the l1-Jacobi scaling
};

// Launch shape of the structured-grid kernels: one block row per (j, k) grid line,
// blockIdx.y tiles the x direction; no 64-bit division per thread.
constexpr int kLineThreads = 128;
inline dim3 line_grid(const GridP& g) {
  return dim3((unsigned)((long long)g.ny * g.nz), (unsigned)((g.nx + kLineThreads - 1) / kLineThreads), 1);
}

struct Hierarchy {
  Stencil4<double> st64;
  Stencil4<float> st32;
  std::vector<Level> lv;
  int nlev = 0;
  int cn = 0;                     // coarsest size
  double* cdense = nullptr;       // coarsest matrix, dense, then its inverse (cn x cn)
  float* cinv32 = nullptr;
  double* cwork = nullptr;        // blocked Gauss-Jordan work: panel rows, old panel columns, panel inverse
  rich_amg_opts opts{};
  bool built = false;
  bool dense = true;              // coarsest level by dense inverse (else kCoarseSweeps l1-Jacobi sweeps)
  cudaGraphExec_t gj_exec = nullptr;  // the coarsest inverse (one launch per pivot) as one graph
  long long gj_nodes = 0;
  // the V-cycle as one graph (opts.graph): captured at its second application,
  // reading the level-0 right-hand side buffer and leaving its result at vc_out
  cudaGraphExec_t vc_exec = nullptr;
  long long vc_nodes = 0;
  void* vc_out = nullptr;
  int vc_calls = 0;
  bool vc_off = false;            // capture failed: direct launches for this hierarchy
  // an FCG iteration (it >= 2, V-cycle to the read-back of its scalars) as one graph
  // per parity of it (q and q_prev alternate), writing the correction fcg_x
  cudaGraphExec_t fcg_exec[2] = {nullptr, nullptr};
  long long fcg_nodes[2] = {0, 0};
  const double* fcg_x = nullptr;
  bool fcg_off = false;
  // one-level additive Schwarz (precond = RICH_PRECOND_AS): ILU(0) diagonals and
  // subdomain solutions (hierarchy precision), FP32 staging of r and z in MIXED
  void* asD = nullptr;
  void* asZ = nullptr;
  float* asR32 = nullptr;
  float* asZ32 = nullptr;
};

constexpr int kStallWindow = 30;        // FCG iterations per stagnation test (krylov.stall)
constexpr int kMaxCoarseDense = 8192;  // largest coarsest level inverted densely
constexpr int kCoarseSweeps = 8;       // l1-Jacobi sweeps on a stalled (larger) coarsest level

struct KrylovWork {
  long long n = 0;
  int m = 0;
  double* V = nullptr;  // (m+1) x n
  double* Z = nullptr;  // m x n
  double* x = nullptr;
  double* r = nullptr;
  double* p = nullptr;
  double* q = nullptr;
  double* qprev = nullptr;
  double* z = nullptr;
  double* w = nullptr;
  double* hcoef = nullptr;  // device coefficients (m+1)
  int fail_reason = 0;      // last failure: 0 none, FCG 1 maxit, 2 (p, J p) <= 0, 3 residual growth;
                            // 4 stagnation (an FCG window or an FGMRES restart cycle, krylov.stall)
};

}  // namespace rich

struct rich_ctx {
  rich::GridP g{};
  rich::SoilP soil{};
  rich::BCP bc{};
  int kmean = 0;
  int prec = 0;
  cudaStream_t st = nullptr;
  int device = 0;
  double* ks = nullptr;        // per-cell K_s or nullptr
  // constitutive values at the last p given to constit()
  double* K = nullptr;
  double* dK = nullptr;
  double* S = nullptr;
  double* dS = nullptr;
  // stencils (7n)
  double* J7 = nullptr;
  double* A7 = nullptr;
  bool have_jac = false;
  bool a0_fresh = false;       // finest CSR values match A7
  // finest-level CSR pattern (built at create)
  rich::Csr<double> A0;
  rich::Hierarchy H;
  rich::KrylovWork kw;
  // reductions: partial sums per block and device scalars
  double* partials = nullptr;  // kRedBlocks * 64
  double* dsc = nullptr;       // device scalars (256)
  double* hsc = nullptr;       // pinned host mirror (128)
  int* iflag = nullptr;        // device int flags (16)
  int* hflag = nullptr;        // pinned host (16)
  // Newton work
  double* s_old = nullptr;
  double* F = nullptr;
  double* Ft = nullptr;
  double* d = nullptr;
  double* ptrial = nullptr;
  double* rhs = nullptr;
  double* pbuf = nullptr;      // device p for rich_step_host
  double* psave = nullptr;     // p at the start of a substep (time-step control)
  int nbatch = 1;              // problems stacked along z (rich_create_batch)
  double* bc_fields[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // owned per-cell BC values
  double* bc_gks[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};     // owned ghost K_s (interfaces)
  bool amg_ever = false;
};

namespace rich {

// ---------------------------------------------------------------- device helpers

// Constitutive law, eqs. (s(p)), (K(p)) and (derivativeofcoefficients) of Sec. 2-3.
// |p|^beta and |p|^gamma share one log|p|; |p|^(x-1) = |p|^x / |p|.
__device__ __forceinline__ void constit(double p, double ks, const SoilP& so, double& S, double& dS,
                                        double& K, double& dK) {
  if (p < 0.0) {
    double ap = -p;
    double lp = log(ap);
    double pb = exp(so.beta * lp);
    double pg = exp(so.gamma * lp);
    // three reciprocals instead of six divisions (FP64 division is a software
    // sequence on GB300's narrow FP64 pipe)
    const double r_ap = 1.0 / ap;
    const double r_s = 1.0 / (so.alpha + pb);
    const double r_k = 1.0 / (so.a + pg);
    S = so.alpha * (so.ts - so.tr) * r_s + so.tr;
    dS = so.alpha * so.beta * (pb * r_ap) * (so.ts - so.tr) * (r_s * r_s);
    K = ks * so.a * r_k;
    dK = so.a * so.gamma * ks * (pg * r_ap) * (r_k * r_k);
  } else {
    S = so.ts;
    dS = 0.0;
    K = ks;
    dK = 0.0;
  }
}

__device__ __forceinline__ double conductivity_only(double p, double ks, const SoilP& so) {
  if (p < 0.0) return ks * so.a / (so.a + exp(so.gamma * log(-p)));
  return ks;
}

// The mean used on the faces normal to axis: a split code (RICH_KMEAN_SPLIT) takes
// its horizontal mean on the x and y faces and its vertical mean on the z faces.
__host__ __device__ __forceinline__ int axis_mean(int kmean, int axis) {
  if (kmean & RICH_KMEAN_SPLIT_FLAG) return axis == 2 ? (kmean & 0xF) : ((kmean >> 4) & 0xF);
  return kmean;
}
inline bool kmean_valid(int kmean) {
  if (kmean >= 0 && kmean <= 3) return true;
  if ((kmean & ~0x1FF) != 0 || !(kmean & RICH_KMEAN_SPLIT_FLAG)) return false;
  return ((kmean >> 4) & 0xF) <= 3 && (kmean & 0xF) <= 3;
}

// Face mean between the lower (L) and upper (+d side, U) cell and its partials.
__device__ __forceinline__ double face_mean(int kmean, double kL, double kU, double pL, double pU,
                                            double& dL, double& dU) {
  if (kmean == RICH_KMEAN_ARITH) {
    dL = 0.5;
    dU = 0.5;
    return 0.5 * (kL + kU);
  }
  if (kmean == RICH_KMEAN_UPSTREAM) {
    bool up = (pU - pL) >= 0.0;
    dL = up ? 0.0 : 1.0;
    dU = up ? 1.0 : 0.0;
    return up ? kU : kL;
  }
  if (kmean == RICH_KMEAN_GEOMETRIC) {
    double g = sqrt(kL * kU);
    dL = kL > 0.0 ? 0.5 * g / kL : 0.0;
    dU = kU > 0.0 ? 0.5 * g / kU : 0.0;
    return g;
  }
  double s = kL + kU;
  if (s > 0.0) {
    double is = 1.0 / s;
    dL = 2.0 * kU * kU * is * is;
    dU = 2.0 * kL * kL * is * is;
    return 2.0 * kL * kU * is;
  }
  dL = dU = 0.0;
  return 0.0;
}

// Warp/block sum of NQ doubles in a fixed order; result valid in thread 0.
template <int NQ>
__device__ __forceinline__ void block_sum(double (&v)[NQ]) {
  __shared__ double sh[NQ][kBlock / 32];
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v[q] += __shfl_down_sync(0xffffffffu, v[q], o);
  }
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) sh[q][wid] = v[q];
  }
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      double t = lane < kBlock / 32 ? sh[q][lane] : 0.0;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
      v[q] = t;
    }
  }
}

__device__ __forceinline__ double block_max(double v) {
  __shared__ double shm[kBlock / 32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) shm[wid] = v;
  __syncthreads();
  if (wid == 0) {
    double t = lane < kBlock / 32 ? shm[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_down_sync(0xffffffffu, t, o));
    v = t;
  }
  return v;
}

// ---------------------------------------------------------------- host helpers (blas.cu)

// Sum nq quantities of per-block partials (partials[q*nb + b]) into dst[q] (device), fixed order.
int finish_sums(rich_ctx* c, const double* partials, int nb, int nq, double* dst);
int finish_max(rich_ctx* c, const double* partials, int nb, double* dst);
int fetch_scalars(rich_ctx* c, const double* dsrc, int count, double* host);
int scan_exclusive_int(rich_ctx* c, const int* in, int* out, long long n);         // out[n] = total
int scan_exclusive_ll(rich_ctx* c, const long long* in, long long* out, long long n);
int scan_exclusive_int_ll(rich_ctx* c, const int* in, long long* out, long long n);
int dot(rich_ctx* c, const double* x, const double* y, long long n, double* dst_dev);
int nrm2sq(rich_ctx* c, const double* x, long long n, double* dst_dev);

// Device memory is stream-ordered: cudaMallocAsync / cudaFreeAsync on the
// stream of the context being worked on, so allocating or freeing never waits
// for the work of other streams (the request server runs several contexts at
// once).  Every entry point that may allocate names its stream with an
// AllocStream guard; outside one the legacy default stream is used, which is
// ordered with every blocking stream.  Freed blocks stay in the device's pool
// for reuse (release threshold raised once per device, see pool_setup).
extern thread_local cudaStream_t t_alloc_stream;
struct AllocStream {
  cudaStream_t prev;
  explicit AllocStream(cudaStream_t s) : prev(t_alloc_stream) { t_alloc_stream = s; }
  ~AllocStream() { t_alloc_stream = prev; }
};
void pool_setup();         // keeps freed device memory in the current device's pool
void pool_trim();          // returns the pool's unused memory (before free-memory queries)
void* pinned_get();        // a 2 KB pinned host block from a process-wide free list
void pinned_put(void* b);  // back to the list (never cudaFreeHost: that synchronises the device)
constexpr size_t kPinnedBlock = 2048;

template <class T>
int dalloc(T** p, long long count) {
  if (count <= 0) count = 1;
  pool_setup();
  cudaError_t e = cudaMallocAsync((void**)p, sizeof(T) * (size_t)count, t_alloc_stream);
  if (e != cudaSuccess) {
    set_cuda_error(e, "cudaMallocAsync");
    *p = nullptr;
    return RICH_ENOMEM;
  }
  return RICH_OK;
}
template <class T>
void dfree(T*& p) {
  if (p) cudaFreeAsync((void*)p, t_alloc_stream);
  p = nullptr;
}

// physics.cu
int constit_eval(rich_ctx* c, const double* p);
// constit_current: the context's K, K', s, s' already hold the values of this p
// (the last constitutive evaluation was at the same pressure), so they are reused.
// nseg > 1: the grid stacks nseg problems along z and the norms are summed per problem
// (dsc[q * nseg + s] for quantity q of problem s).
int residual_eval(rich_ctx* c, const double* p, const double* s_old, double dt, double* F, bool want_norms,
                  bool constit_current = false, int nseg = 1);
int jacobian_eval(rich_ctx* c, const double* p, double dt, bool constit_current = false);
int stencil_apply(rich_ctx* c, const double* A7, const double* x, double* y);
int refresh_a0_values(rich_ctx* c);

// amg_setup.cu
int amg_build(rich_ctx* c, const rich_amg_opts* o);
int amg_refresh(rich_ctx* c);
int amg_update_fine(rich_ctx* c);
void amg_free(rich_ctx* c);

// blas.cu: whether a profiling target is set (the autotuner then stays off)
bool profiling_active();

// schwarz.cu
int as_setup(rich_ctx* c);   // allocate (first call) and factor every subdomain of the current A_aux
int as_apply(rich_ctx* c, const double* r, double* z);
void as_free(rich_ctx* c);

// sell.cu: SELL-C-sigma copies of the coarse-level matrices
int sell_build(rich_ctx* c, const Csr<double>& M, Sell& S);  // pattern; nothing below kSellMinRows rows
int sell_fill(rich_ctx* c, const Csr<double>& M, const double* val, Sell& S);  // values, M's entry order
int sell_fill(rich_ctx* c, const Csr<double>& M, const float* val, Sell& S);
void sell_free(Sell& S);

// solve.cu
int autotune_table(char* buf, int cap);
int autotune_load(const char* text);
int vcycle_apply(rich_ctx* c, const double* r, double* z);
int krylov_run(rich_ctx* c, const double* b, double* x, const rich_krylov_opts* o, rich_krylov_stats* st);

}  // namespace rich
