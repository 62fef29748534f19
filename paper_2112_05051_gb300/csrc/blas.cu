// Deterministic reductions, scans and dot products.  Every reduction writes one
// partial per block of a fixed grid and a second single-block kernel sums the
// partials in block order, so FP64 results reproduce bit for bit run to run.
#include <mutex>

#include <cstring>

#include "common.cuh"

#include <atomic>
#include <string>

namespace rich {

thread_local cudaStream_t t_alloc_stream = 0;

static std::mutex g_pool_mu;
static bool g_pool_done[64] = {false};

void pool_setup() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return;
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (g_pool_done[dev]) return;
  g_pool_done[dev] = true;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
  unsigned long long keep = ~0ULL;  // keep freed blocks for the next allocation
  cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
}

void pool_trim() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return;
  cudaMemPool_t pool;
  if (cudaDeviceGetDefaultMemPool(&pool, dev) != cudaSuccess) return;
  cudaMemPoolTrimTo(pool, 0);
}

static std::mutex g_pinned_mu;
static std::vector<void*> g_pinned_free;

void* pinned_get() {
  {
    std::lock_guard<std::mutex> lock(g_pinned_mu);
    if (!g_pinned_free.empty()) {
      void* b = g_pinned_free.back();
      g_pinned_free.pop_back();
      return b;
    }
  }
  void* b = nullptr;
  if (cudaMallocHost(&b, kPinnedBlock) != cudaSuccess) return nullptr;
  return b;
}

void pinned_put(void* b) {
  if (!b) return;
  std::lock_guard<std::mutex> lock(g_pinned_mu);
  g_pinned_free.push_back(b);
}

static std::atomic<long long> g_launches{0};
void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void count_launches(long long k) { g_launches.fetch_add(k, std::memory_order_relaxed); }

// ---------------------------------------------------------------- live kernel timing

constexpr int kProfEvents = 65536;
static std::string g_prof_target;   // a kernel name, "*" for every named kernel, "" = off
static std::vector<cudaEvent_t> g_prof_ev;
static std::vector<const char*> g_prof_name;
static std::vector<double> g_prof_b;
static std::vector<double> g_prof_f;
static int g_prof_n = 0;          // recorded launch pairs
static long long g_prof_seen = 0; // launches of the target (recorded or not)
static long long g_prof_stride = 1;  // record every stride-th launch of the target
static double g_prof_bytes = 0.0;
static double g_prof_flops = 0.0;
static int g_prof_open = -1;         // the pair whose end is still to be recorded

bool profiling_active() { return !g_prof_target.empty(); }

// Keeps the stream busy for a fixed number of clock cycles (the loop ends by itself):
// queued ahead of a timed launch's start event, it lets the host enqueue the event
// and the launch before the GPU reaches them, so the pair measures the kernel and not
// the host's submission gap (the Krylov loops synchronise every iteration, leaving the
// GPU idle between launches).
__global__ void k_prof_delay(long long cycles) {
  const long long t0 = clock64();
  while (clock64() - t0 < cycles) {
  }
}
constexpr long long kProfDelayCycles = 40000;  // ~20 us at 2 GHz

void prof_adjust_last(const char* name, double bytes, double flops) {
  if (g_prof_n < 1 || g_prof_open >= 0 || strcmp(g_prof_name[g_prof_n - 1], name) != 0) return;
  g_prof_bytes += bytes - g_prof_b[g_prof_n - 1];
  g_prof_flops += flops - g_prof_f[g_prof_n - 1];
  g_prof_b[g_prof_n - 1] = bytes;
  g_prof_f[g_prof_n - 1] = flops;
}

void prof_restart(cudaStream_t st) {
  if (g_prof_open < 0) return;
  k_prof_delay<<<1, 32, 0, st>>>(kProfDelayCycles);
  cudaEventRecord(g_prof_ev[2 * g_prof_open], st);
}

ProfScope::ProfScope(const char* name, cudaStream_t s, double b, double f) : on(false), st(s), bytes(b), flops(f) {
  if (g_prof_target.empty() || (g_prof_target != "*" && g_prof_target != name)) return;
  if (g_prof_seen++ % g_prof_stride != 0) return;  // only every stride-th launch is timed
  if (g_prof_n >= kProfEvents / 2) return;
  if (g_prof_ev.empty()) {
    g_prof_ev.resize(kProfEvents);
    for (auto& e : g_prof_ev) cudaEventCreate(&e);
    g_prof_name.resize(kProfEvents / 2);
    g_prof_b.resize(kProfEvents / 2);
    g_prof_f.resize(kProfEvents / 2);
  }
  on = true;
  g_prof_name[g_prof_n] = name;
  g_prof_open = g_prof_n;
  k_prof_delay<<<1, 32, 0, st>>>(kProfDelayCycles);
  cudaEventRecord(g_prof_ev[2 * g_prof_n], st);
}

ProfScope::~ProfScope() {
  if (!on) return;
  cudaEventRecord(g_prof_ev[2 * g_prof_n + 1], st);
  g_prof_b[g_prof_n] = bytes;
  g_prof_f[g_prof_n] = flops;
  g_prof_bytes += bytes;
  g_prof_flops += flops;
  g_prof_open = -1;
  ++g_prof_n;
}

// one block per quantity: the same fixed reduction tree for each
__global__ void k_finish_sums(const double* __restrict__ partials, int nb, int nq, double* __restrict__ dst) {
  int q = blockIdx.x;
  double v[1] = {0.0};
  for (int b = threadIdx.x; b < nb; b += blockDim.x) v[0] += partials[(long long)q * nb + b];
  block_sum<1>(v);
  if (threadIdx.x == 0) dst[q] = v[0];
}

__global__ void k_finish_max(const double* __restrict__ partials, int nb, double* __restrict__ dst) {
  double m = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) {
    double a = partials[b];
    m = (a > m || a != a) ? a : m;
  }
  m = block_max(m);
  if (threadIdx.x == 0) dst[0] = m;
}

int finish_sums(rich_ctx* c, const double* partials, int nb, int nq, double* dst) {
  k_finish_sums<<<nq, kBlock, 0, c->st>>>(partials, nb, nq, dst);
  RICH_LAUNCH_CHECK();
  return RICH_OK;
}

int finish_max(rich_ctx* c, const double* partials, int nb, double* dst) {
  k_finish_max<<<1, kBlock, 0, c->st>>>(partials, nb, dst);
  RICH_LAUNCH_CHECK();
  return RICH_OK;
}

int fetch_scalars(rich_ctx* c, const double* dsrc, int count, double* host) {
  RICH_CUDA(cudaMemcpyAsync(c->hsc, dsrc, count * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  RICH_CUDA(cudaStreamSynchronize(c->st));
  for (int i = 0; i < count; ++i) host[i] = c->hsc[i];
  return RICH_OK;
}

// ---------------------------------------------------------------- dot products

__global__ void k_dot(const double* __restrict__ x, const double* __restrict__ y, long long n,
                      double* __restrict__ partials) {
  double v[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    v[0] += x[i] * y[i];
  block_sum<1>(v);
  if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}

int dot(rich_ctx* c, const double* x, const double* y, long long n, double* dst) {
  int nb = red_grid(n);
  k_dot<<<nb, kBlock, 0, c->st>>>(x, y, n, c->partials);
  RICH_LAUNCH_CHECK();
  return finish_sums(c, c->partials, nb, 1, dst);
}

int nrm2sq(rich_ctx* c, const double* x, long long n, double* dst) { return dot(c, x, x, n, dst); }

// y = a x + b y (y = a x when b == 0, whatever y held)
__global__ void k_vec_axpby(long long n, double a, const double* __restrict__ x, double b, double* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = b == 0.0 ? a * x[i] : a * x[i] + b * y[i];
}

// ---------------------------------------------------------------- exclusive scan (3 phases)

constexpr int kScanItems = 8;
constexpr int kScanTile = kBlock * kScanItems;

template <class T>
__device__ __forceinline__ T block_exclusive_scan(T v, T* total) {
  __shared__ T sh[kBlock / 32];
  int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  T inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  __syncthreads();
  if (lane == 31) sh[wid] = inc;
  __syncthreads();
  if (wid == 0) {
    T w = lane < kBlock / 32 ? sh[lane] : T(0);
    T wi = w;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T t = __shfl_up_sync(0xffffffffu, wi, o);
      if (lane >= o) wi += t;
    }
    if (lane < kBlock / 32) sh[lane] = wi - w;
    if (lane == kBlock / 32 - 1) *total = wi;
  }
  __syncthreads();
  return sh[wid] + inc - v;
}

template <class TI, class TO>
__global__ void k_scan_tiles(const TI* __restrict__ in, long long n, TO* __restrict__ tile_sums) {
  long long base = (long long)blockIdx.x * kScanTile;
  TO s = 0;
  for (int t = 0; t < kScanItems; ++t) {
    long long i = base + (long long)t * kBlock + threadIdx.x;
    if (i < n) s += (TO)in[i];
  }
  __shared__ TO tot;
  block_exclusive_scan<TO>(s, &tot);
  __syncthreads();
  if (threadIdx.x == 0) tile_sums[blockIdx.x] = tot;
}

template <class TO>
__global__ void k_scan_sums(TO* __restrict__ sums, long long nt, TO* __restrict__ total_out) {
  __shared__ TO carry;
  __shared__ TO tot;
  if (threadIdx.x == 0) carry = 0;
  __syncthreads();
  for (long long base = 0; base < nt; base += blockDim.x) {
    long long i = base + threadIdx.x;
    TO v = i < nt ? sums[i] : TO(0);
    TO ex = block_exclusive_scan<TO>(v, &tot);
    if (i < nt) sums[i] = ex + carry;
    __syncthreads();
    if (threadIdx.x == 0) carry += tot;
    __syncthreads();
  }
  if (threadIdx.x == 0) *total_out = carry;
}

template <class TI, class TO>
__global__ void k_scan_apply(const TI* __restrict__ in, long long n, const TO* __restrict__ tile_off,
                             TO* __restrict__ out) {
  long long base = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanItems;
  TO loc[kScanItems];
  TO s = 0;
  for (int t = 0; t < kScanItems; ++t) {
    long long i = base + t;
    loc[t] = i < n ? (TO)in[i] : TO(0);
    s += loc[t];
  }
  __shared__ TO tot;
  TO ex = block_exclusive_scan<TO>(s, &tot) + tile_off[blockIdx.x];
  for (int t = 0; t < kScanItems; ++t) {
    long long i = base + t;
    if (i < n) out[i] = ex;
    ex += loc[t];
  }
}

// The tile sums of k_scan_tiles are taken over strided items while k_scan_apply
// scans contiguous items; both cover the same tile [base, base + kScanTile), so the
// tile total is the same.
template <class TI, class TO>
static int scan_impl(rich_ctx* c, const TI* in, TO* out, long long n) {
  long long nt = (n + kScanTile - 1) / kScanTile;
  if (nt < 1) nt = 1;
  TO* sums = nullptr;
  RICH_CHECK(dalloc(&sums, nt));
  k_scan_tiles<TI, TO><<<(int)nt, kBlock, 0, c->st>>>(in, n, sums);
  RICH_LAUNCH_CHECK();
  k_scan_sums<TO><<<1, kBlock, 0, c->st>>>(sums, nt, out + n);
  RICH_LAUNCH_CHECK();
  k_scan_apply<TI, TO><<<(int)nt, kBlock, 0, c->st>>>(in, n, sums, out);
  RICH_LAUNCH_CHECK();
  RICH_CUDA(cudaStreamSynchronize(c->st));
  dfree(sums);
  return RICH_OK;
}

int scan_exclusive_int(rich_ctx* c, const int* in, int* out, long long n) { return scan_impl<int, int>(c, in, out, n); }
int scan_exclusive_int_ll(rich_ctx* c, const int* in, long long* out, long long n) {
  return scan_impl<int, long long>(c, in, out, n);
}
int scan_exclusive_ll(rich_ctx* c, const long long* in, long long* out, long long n) {
  return scan_impl<long long, long long>(c, in, out, n);
}

// Arithmetic peak probe: every thread runs kChains independent fused multiply-add
// chains, so the pipe is limited by issue rate, not by the latency of one chain.
constexpr int kChains = 8;
template <class T>
__global__ void k_fma_peak(int iters, T b, T c, T* __restrict__ sink) {
  T a[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) a[q] = T(threadIdx.x + q);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) a[q] = a[q] * b + c;
  }
  T s = 0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s += a[q];
  if (s == T(-12345.0)) sink[threadIdx.x] = s;  // keeps the chains live; never true for these inputs
}

template <class T>
static int fma_peak(cudaStream_t st, double* tflops) {
  T* sink = nullptr;
  RICH_CUDA(cudaMalloc(&sink, kBlock * sizeof(T)));
  const int blocks = 8 * kNumSM;
  const int iters = sizeof(T) == 8 ? 4096 : 65536;
  cudaEvent_t e0, e1;
  RICH_CUDA(cudaEventCreate(&e0));
  RICH_CUDA(cudaEventCreate(&e1));
  float best = 1e30f;
  for (int rep = 0; rep < 4; ++rep) {  // the first launch warms the clocks up
    RICH_CUDA(cudaEventRecord(e0, st));
    k_fma_peak<T><<<blocks, kBlock, 0, st>>>(iters, T(0.999999), T(1e-7), sink);
    RICH_CUDA(cudaEventRecord(e1, st));
    RICH_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    RICH_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    if (rep > 0 && ms < best) best = ms;
  }
  count_launches(4);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(sink);
  *tflops = 2.0 * kChains * (double)iters * blocks * kBlock / (best * 1e-3) / 1e12;
  return RICH_OK;
}

}  // namespace rich

extern "C" {

int rich_vec_dot(rich_ctx* c, const double* x, const double* y, double* out) {
  if (!c || !x || !y || !out) return RICH_EINVAL;
  rich::AllocStream guard(c->st);
  double* d = c->dsc + 200;  // a slot no solver uses
  RICH_CHECK(rich::dot(c, x, y, c->g.n, d));
  return rich::fetch_scalars(c, d, 1, out);
}

int rich_vec_axpby(rich_ctx* c, double a, const double* x, double b, double* y) {
  if (!c || !x || !y) return RICH_EINVAL;
  rich::k_vec_axpby<<<rich::grid_for(c->g.n), rich::kBlock, 0, c->st>>>(c->g.n, a, x, b, y);
  RICH_LAUNCH_CHECK();
  return RICH_OK;
}

int rich_autotune_table(char* buf, int cap) {
  if (!buf || cap < 1) return RICH_EINVAL;
  return rich::autotune_table(buf, cap);
}

int rich_autotune_load(const char* text) {
  if (!text) return RICH_EINVAL;
  return rich::autotune_load(text);
}

int rich_measure_fma_peak(int fp64, double* tflops) {
  if (!tflops) return RICH_EINVAL;
  return fp64 ? rich::fma_peak<double>(nullptr, tflops) : rich::fma_peak<float>(nullptr, tflops);
}

int rich_kernel_launches(long long* out) {
  if (!out) return RICH_EINVAL;
  *out = rich::g_launches.load();
  return RICH_OK;
}

int rich_profile_kernel(const char* name) {
  rich::g_prof_target = name ? name : "";
  rich::g_prof_n = 0;
  rich::g_prof_seen = 0;
  rich::g_prof_open = -1;
  rich::g_prof_bytes = 0.0;
  rich::g_prof_flops = 0.0;
  return RICH_OK;
}

int rich_memory_peak(long long* used_high, long long* reserved_high, int reset) {
  int dev = 0;
  RICH_CUDA(cudaGetDevice(&dev));
  cudaMemPool_t pool;
  RICH_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t u = 0, r = 0;  // the attribute values are 64-bit
  RICH_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &u));
  RICH_CUDA(cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemHigh, &r));
  if (used_high) *used_high = (long long)u;
  if (reserved_high) *reserved_high = (long long)r;
  if (reset) {
    uint64_t zero = 0;
    RICH_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrUsedMemHigh, &zero));
    RICH_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReservedMemHigh, &zero));
  }
  return RICH_OK;
}

int rich_profile_stride(int stride) {
  if (stride < 1) return RICH_EINVAL;
  rich::g_prof_stride = stride;
  return RICH_OK;
}

int rich_profile_result(double* ms_total, long long* launches, double* bytes_total, double* flops_total) {
  if (!ms_total || !launches || !bytes_total) return RICH_EINVAL;
  if (flops_total) *flops_total = rich::g_prof_flops;
  double ms = 0.0;
  for (int i = 0; i < rich::g_prof_n; ++i) {
    cudaEventSynchronize(rich::g_prof_ev[2 * i + 1]);
    float t = 0.f;
    cudaEventElapsedTime(&t, rich::g_prof_ev[2 * i], rich::g_prof_ev[2 * i + 1]);
    ms += t;
  }
  *ms_total = ms;
  *launches = rich::g_prof_n;
  *bytes_total = rich::g_prof_bytes;
  return RICH_OK;
}

// Per-kernel totals of the recorded launches (profiling target "*"): writes up
// to cap lines "name launches total_ms bytes" into buf (NUL-terminated).
int rich_profile_table(char* buf, int cap) {
  if (!buf || cap < 1) return RICH_EINVAL;
  struct Acc { double ms = 0.0; long long n = 0; double bytes = 0.0, flops = 0.0; };
  std::vector<std::pair<std::string, Acc>> tab;
  for (int i = 0; i < rich::g_prof_n; ++i) {
    cudaEventSynchronize(rich::g_prof_ev[2 * i + 1]);
    float t = 0.f;
    cudaEventElapsedTime(&t, rich::g_prof_ev[2 * i], rich::g_prof_ev[2 * i + 1]);
    std::string nm = rich::g_prof_name[i];
    size_t k = 0;
    while (k < tab.size() && tab[k].first != nm) ++k;
    if (k == tab.size()) tab.push_back({nm, Acc()});
    tab[k].second.ms += t;
    tab[k].second.n += 1;
    tab[k].second.bytes += rich::g_prof_b[i];
    tab[k].second.flops += rich::g_prof_f[i];
  }
  int off = 0;
  buf[0] = 0;
  for (auto& e : tab) {
    int w = snprintf(buf + off, cap - off, "%s %lld %.6f %.6e %.6e\n", e.first.c_str(), e.second.n, e.second.ms,
                     e.second.bytes, e.second.flops);
    if (w < 0 || w >= cap - off) break;
    off += w;
  }
  return RICH_OK;
}

}  // extern "C"
