// Smoothed-aggregation AMG setup on the GPU (Sec. 5.2: DSVMB-style decoupled
// smoothed aggregation; on one GPU the whole domain is one block).
//
//   strength   j != i strong iff max(a_ij^2, a_ji^2) >= theta_l^2 |a_ii a_jj|
//              (symmetrised; a_ji found by binary search, the pattern is symmetric),
//              theta_l = theta 2^-l on level l
//              (a constant threshold lets the coarse-operator density explode)
//   MIS-2      synchronous rounds over 64-bit tuples (state << 62 | key),
//              key(i) = top30(splitmix64(seed ^ i)) << 32 | i; two 1-hop max passes
//   aggregates roots numbered by an exclusive scan; pass 1 joins the strong
//              root neighbour of largest key, pass 2 the pass-1 neighbour whose
//              root has the largest key
//   P          (I - omega D^-1 A) P_tent, omega = 4/(3 max_i sum_j|a_ij|/|a_ii|)
//   Galerkin   A_c = R (A P), R = P^T
// Sparse products are row-wise expand-sort-compress: one warp per output row
// sorts 64-bit keys (column << 32 | product index) with a bitonic network and
// sums each column's products in product order, so patterns are structural
// and values deterministic.  The numeric refresh recomputes values on the kept
// patterns with one thread per row in the same product order.
#include <math_constants.h>

#include "common.cuh"

namespace rich {

// ---------------------------------------------------------------- priorities

__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x + 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t prio_key(uint64_t seed, long long i) {
  uint64_t pi = splitmix64(seed ^ (uint64_t)i);
  return ((pi >> 34) << 32) | (uint64_t)i;
}

constexpr uint64_t kStateShift = 62;
constexpr uint64_t kUndecided = 1;
constexpr uint64_t kIn = 2;
constexpr uint64_t kLow32 = 0xFFFFFFFFull;
constexpr uint64_t kKeyMask = (1ull << 62) - 1;

// ---------------------------------------------------------------- small kernels

__global__ void k_diag(int n, const int* __restrict__ rp, const int* __restrict__ col, const double* __restrict__ val,
                       double* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double v = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e)
      if (col[e] == i) v = val[e];
    d[i] = v;
  }
}

__device__ __forceinline__ int find_col(const int* __restrict__ col, int lo, int hi, int key) {
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (col[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ bool strong_sym(int i, int e, const int* __restrict__ rp, const int* __restrict__ col,
                                           const double* __restrict__ val, const double* __restrict__ d,
                                           double theta2) {
  int j = col[e];
  if (j == i) return false;
  double rhs = theta2 * fabs(d[i] * d[j]);
  double a = val[e];
  if (a * a >= rhs) return true;
  int q = find_col(col, rp[j], rp[j + 1], i);
  if (q < rp[j + 1] && col[q] == i) {
    double b = val[q];
    if (b * b >= theta2 * fabs(d[j] * d[i])) return true;
  }
  return false;
}

__global__ void k_strength(int n, const int* __restrict__ rp, const int* __restrict__ col,
                           const double* __restrict__ val, const double* __restrict__ d, double theta2,
                           const int* __restrict__ srp, int* __restrict__ cnt, int* __restrict__ scol) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int o = srp ? srp[i] : 0;
    int c = 0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      if (strong_sym(i, e, rp, col, val, d, theta2)) {
        if (scol) scol[o + c] = col[e];
        ++c;
      }
    }
    if (cnt) cnt[i] = c;
  }
}

// Isolated nodes (no strong neighbour) start OUT: they join no aggregate.
__global__ void k_mis_init(int n, uint64_t seed, const int* __restrict__ srp, uint64_t* __restrict__ t) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    bool isolated = srp[i + 1] == srp[i];
    t[i] = (isolated ? 0ull : (kUndecided << kStateShift)) | prio_key(seed, i);
  }
}

// m[i] = max of v over the closed strength neighbourhood of i
__global__ void k_max_closed(int n, const int* __restrict__ srp, const int* __restrict__ scol,
                             const uint64_t* __restrict__ v, uint64_t* __restrict__ m) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint64_t best = v[i];
    for (int e = srp[i]; e < srp[i + 1]; ++e) {
      uint64_t w = v[scol[e]];
      best = w > best ? w : best;
    }
    m[i] = best;
  }
}

// second 1-hop pass and the state update of one MIS-2 round
__global__ void k_mis_update(int n, const int* __restrict__ srp, const int* __restrict__ scol,
                             const uint64_t* __restrict__ m1, uint64_t* __restrict__ t, int* __restrict__ undecided) {
  int any = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint64_t ti = t[i];
    if ((ti >> kStateShift) != kUndecided) continue;
    uint64_t best = m1[i];
    for (int e = srp[i]; e < srp[i + 1]; ++e) {
      uint64_t w = m1[scol[e]];
      best = w > best ? w : best;
    }
    if (best == ti) {
      t[i] = (kIn << kStateShift) | (ti & kKeyMask);
    } else if ((best >> kStateShift) == kIn) {
      t[i] = ti & kKeyMask;  // OUT = 0
    } else {
      any = 1;
    }
  }
  if (any) atomicOr(undecided, 1);
}

__global__ void k_is_root(int n, const uint64_t* __restrict__ t, int* __restrict__ isroot) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    isroot[i] = (t[i] >> kStateShift) == kIn ? 1 : 0;
}

__global__ void k_rootval(int n, const uint64_t* __restrict__ t, uint64_t* __restrict__ rv) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    uint64_t ti = t[i];
    rv[i] = (ti >> kStateShift) == kIn ? (ti & kKeyMask) + 1 : 0;
  }
}

// pass 1 result: agg (or -1) and the root index of pass-1 nodes (-1 otherwise)
__global__ void k_agg_pass1(int n, const uint64_t* __restrict__ t, const uint64_t* __restrict__ best,
                            const int* __restrict__ aggid, int* __restrict__ agg, int* __restrict__ p1root) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    bool root = (t[i] >> kStateShift) == kIn;
    p1root[i] = -1;
    if (root) {
      agg[i] = aggid[i];
    } else if (best[i] > 0) {
      int r = (int)((best[i] - 1) & kLow32);
      agg[i] = aggid[r];
      p1root[i] = r;
    } else {
      agg[i] = -1;
    }
  }
}

__global__ void k_val2(int n, const uint64_t* __restrict__ t, const int* __restrict__ p1root, uint64_t* __restrict__ v) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int r = p1root[i];
    v[i] = r >= 0 ? (t[r] & kKeyMask) + 1 : 0;
  }
}

__global__ void k_agg_pass2(int n, const int* __restrict__ srp, const uint64_t* __restrict__ best2,
                            const int* __restrict__ aggid, int* __restrict__ agg, int* __restrict__ unassigned) {
  int miss = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (agg[i] >= 0) continue;
    if (best2[i] > 0) agg[i] = aggid[(int)((best2[i] - 1) & kLow32)];
    else if (srp[i + 1] != srp[i]) miss = 1;  // isolated nodes stay unaggregated (agg = -1)
  }
  if (miss) atomicOr(unassigned, 1);
}

// Pass 3: a node left out by passes 1-2 (no strong neighbour) whose row is not
// diagonally dominant (a_ii < 2 sum_{j!=i} |a_ij|) joins the aggregate of its
// aggregated neighbour j with the largest (fp32 |a_ij|, key(j)).  On high-contrast
// fields such a row sums to about zero although every coupling is weak relative to
// the neighbours' diagonals; left out, its error is corrected by the smoother alone.
// Reads the aggregates of passes 1-2 (agg_in) only, so the pass is synchronous.
__global__ void k_agg_pass3(int n, const int* __restrict__ rp, const int* __restrict__ col,
                            const double* __restrict__ val, uint64_t seed, const int* __restrict__ agg_in,
                            int* __restrict__ agg_out) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int a = agg_in[i];
    if (a >= 0) continue;
    double diag = 0.0, off = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      if (col[e] == i) diag = val[e];
      else off += fabs(val[e]);
    }
    if (!(fabs(diag) < 2.0 * off)) continue;
    int bj = -1;
    float bw = 0.0f;
    uint64_t bk = 0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      int j = col[e];
      if (j == i || agg_in[j] < 0) continue;
      float w = (float)fabs(val[e]);
      uint64_t kj = prio_key(seed, j);
      if (bj < 0 || w > bw || (w == bw && kj > bk)) {
        bj = j;
        bw = w;
        bk = kj;
      }
    }
    if (bj >= 0) agg_out[i] = agg_in[bj];
  }
}

// P_tent: one unit entry per aggregated node, empty rows for isolated nodes
__global__ void k_ptent_count(int n, const int* __restrict__ agg, int* __restrict__ cnt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) cnt[i] = agg[i] >= 0;
}
__global__ void k_ptent_fill(int n, const int* __restrict__ agg, const int* __restrict__ rp, int* __restrict__ col) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (agg[i] >= 0) col[rp[i]] = agg[i];
}

__global__ void k_rowratio(int n, const int* __restrict__ rp, const double* __restrict__ val,
                           const double* __restrict__ d, double* __restrict__ partials) {
  double m = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) s += fabs(val[e]);
    double r = s / fabs(d[i]);
    m = (r > m || r != r) ? r : m;
  }
  m = block_max(m);
  if (threadIdx.x == 0) partials[blockIdx.x] = m;
}

// S = I - omega D^-1 A on the pattern of A (same operation order as the oracle)
__global__ void k_smoother_vals(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ d, double omega,
                                double* __restrict__ sval) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int e = rp[i]; e < rp[i + 1]; ++e) sval[e] = -omega * val[e] / d[i] + (col[e] == i ? 1.0 : 0.0);
}

__global__ void k_seq(int n, int* __restrict__ a) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i <= n; i += gridDim.x * blockDim.x) a[i] = i;
}

__global__ void k_fill(long long n, double v, double* __restrict__ a) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    a[i] = v;
}

__global__ void k_l1dinv(int n, const int* __restrict__ rp, const double* __restrict__ val, double* __restrict__ dinv,
                         float* __restrict__ dinv32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) s += fabs(val[e]);
    double r = 1.0 / s;
    dinv[i] = r;
    if (dinv32) dinv32[i] = (float)r;
  }
}

__global__ void k_l1dinv32(int n, const int* __restrict__ rp, const float* __restrict__ val, float* __restrict__ dinv32) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    float s = 0.0f;
    for (int e = rp[i]; e < rp[i + 1]; ++e) s += fabsf(val[e]);
    dinv32[i] = 1.0f / s;
  }
}

__global__ void k_cast(long long n, const double* __restrict__ a, float* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}

// ---------------------------------------------------------------- transpose

__global__ void k_tr_count(int n, const int* __restrict__ rp, const int* __restrict__ col, int* __restrict__ cnt) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int e = rp[i]; e < rp[i + 1]; ++e) atomicAdd(&cnt[col[e]], 1);
}

__global__ void k_tr_fill(int n, const int* __restrict__ rp, const int* __restrict__ col,
                          const double* __restrict__ val, const int* __restrict__ trp, int* __restrict__ fillc,
                          int* __restrict__ tcol, double* __restrict__ tval) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      int J = col[e];
      int pos = trp[J] + atomicAdd(&fillc[J], 1);
      tcol[pos] = i;
      tval[pos] = val[e];
    }
}

// ---------------------------------------------------------------- expand-sort-compress SpGEMM

__global__ void k_spgemm_upper(int n, const int* __restrict__ arp, const int* __restrict__ acol,
                               const int* __restrict__ brp, int* __restrict__ u) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    long long s = 0;
    for (int e = arp[i]; e < arp[i + 1]; ++e) s += brp[acol[e] + 1] - brp[acol[e]];
    u[i] = s > 2147483647LL ? 2147483647 : (int)s;
  }
}

__global__ void k_max_int(int n, const int* __restrict__ a, int* __restrict__ out) {
  int m = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) m = max(m, a[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_down_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__device__ __forceinline__ void warp_bitonic_sort(uint64_t* keys, int M, int lane) {
  for (int k = 2; k <= M; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int t = lane; t < M; t += 32) {
        int ixj = t ^ j;
        if (ixj > t) {
          uint64_t a = keys[t], b = keys[ixj];
          bool asc = (t & k) == 0;
          if ((a > b) == asc) {
            keys[t] = b;
            keys[ixj] = a;
          }
        }
      }
      __syncwarp();
    }
  }
}

constexpr int kEscCap = 1024;    // most products per row the shared-memory ESC kernel takes

// mode 0: cnt[row] = number of distinct columns; mode 1: write the compressed row at crp[row];
// mode 2 (single pass): write it at the row's product offset uoff[row] of a temporary
// and set cnt[row].
// Each warp owns `cap` key/value slots of shared memory (cap = the launch's largest
// product count rounded up to a power of two, at most kEscCap), so short rows
// (the 7-point level: tens of products) run many warps per SM.  Rows whose product
// count exceeds kEscCap are left to k_spgemm_hash.
__global__ void k_spgemm_esc(int nrows, const int* __restrict__ arp, const int* __restrict__ acol,
                             const double* __restrict__ aval, const int* __restrict__ brp,
                             const int* __restrict__ bcol, const double* __restrict__ bval,
                             const int* __restrict__ u, int mode, const int* __restrict__ crp,
                             const long long* __restrict__ uoff, int* __restrict__ ccol, double* __restrict__ cval,
                             int* __restrict__ cnt, int cap) {
  extern __shared__ unsigned char smem[];
  int wpb = blockDim.x >> 5;
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  uint64_t* skeys = reinterpret_cast<uint64_t*>(smem) + (size_t)w * cap;
  double* svals = reinterpret_cast<double*>(smem + (size_t)wpb * cap * sizeof(uint64_t)) + (size_t)w * cap;
  for (int row = blockIdx.x * wpb + w; row < nrows; row += gridDim.x * wpb) {
    int ur = u[row];
    if (ur > cap) continue;
    uint64_t* keys = skeys;
    double* vals = svals;
    int M = 1;
    while (M < ur) M <<= 1;
    // expand in product order: A entries in column order, then B entries in column order
    int t0 = 0;
    for (int e = arp[row]; e < arp[row + 1]; ++e) {
      int j = acol[e];
      double a = aval ? aval[e] : 1.0;
      int b0 = brp[j], len = brp[j + 1] - b0;
      for (int q = lane; q < len; q += 32) {
        int t = t0 + q;
        keys[t] = ((uint64_t)(uint32_t)bcol[b0 + q] << 32) | (uint32_t)t;
        vals[t] = a * (bval ? bval[b0 + q] : 1.0);
      }
      t0 += len;
    }
    for (int t = ur + lane; t < M; t += 32) keys[t] = ~0ull;
    __syncwarp();
    warp_bitonic_sort(keys, M, lane);
    // segment heads
    const long long base = mode == 1 ? (long long)crp[row] : (mode == 2 ? uoff[row] : 0);
    int running = 0;
    for (int t0s = 0; t0s < ur; t0s += 32) {
      int t = t0s + lane;
      bool head = false;
      uint32_t c = 0;
      if (t < ur) {
        c = (uint32_t)(keys[t] >> 32);
        head = (t == 0) || ((uint32_t)(keys[t - 1] >> 32) != c);
      }
      unsigned mask = __ballot_sync(0xffffffffu, head);
      if (mode != 0 && head) {
        const long long pos = base + running + __popc(mask & ((1u << lane) - 1));
        double s = 0.0;
        for (int q = t; q < ur && (uint32_t)(keys[q] >> 32) == c; ++q) s += vals[(uint32_t)(keys[q] & kLow32)];
        ccol[pos] = (int)c;
        cval[pos] = s;
      }
      running += __popc(mask);
    }
    if (mode != 1 && lane == 0) cnt[row] = running;
    __syncwarp();
  }
}

// Rows with more than kEscCap products: one block per row accumulates the products
// into a shared-memory hash table keyed by column (linear probing, atomicCAS), then
// sorts the occupied keys.  The column set is exact; the FP64 sums depend on the
// order of the shared-memory atomics (rounding-level differences only).
constexpr int kHashSlots = 8192;
constexpr int kHashThreads = 256;

__global__ void __launch_bounds__(kHashThreads) k_spgemm_hash(
    int nrows, const int* __restrict__ arp, const int* __restrict__ acol, const double* __restrict__ aval,
    const int* __restrict__ brp, const int* __restrict__ bcol, const double* __restrict__ bval,
    const int* __restrict__ u, int mode, const int* __restrict__ crp, const long long* __restrict__ uoff,
    int* __restrict__ ccol, double* __restrict__ cval, int* __restrict__ cnt, int* __restrict__ overflow) {
  extern __shared__ unsigned char smem[];
  int* hkey = reinterpret_cast<int*>(smem);
  double* hval = reinterpret_cast<double*>(smem + kHashSlots * sizeof(int));
  __shared__ int nfill;
  __shared__ int fail;
  for (int row = blockIdx.x; row < nrows; row += gridDim.x) {
    if (u[row] <= kEscCap) continue;
    for (int t = threadIdx.x; t < kHashSlots; t += blockDim.x) {
      hkey[t] = -1;
      hval[t] = 0.0;
    }
    if (threadIdx.x == 0) {
      nfill = 0;
      fail = 0;
    }
    __syncthreads();
    // products: A entries of the row in turn, B entries strided over the block
    for (int e = arp[row]; e < arp[row + 1]; ++e) {
      int j = acol[e];
      double a = aval ? aval[e] : 1.0;
      for (int f = brp[j] + threadIdx.x; f < brp[j + 1]; f += blockDim.x) {
        int col = bcol[f];
        double v = a * (bval ? bval[f] : 1.0);
        unsigned h = ((unsigned)col * 2654435761u) & (kHashSlots - 1);
        int probes = 0;
        for (;;) {
          int k = ((volatile int*)hkey)[h];
          if (k == col) break;
          if (k == -1) {
            int prev = atomicCAS(&hkey[h], -1, col);
            if (prev == -1 || prev == col) break;
          }
          h = (h + 1) & (kHashSlots - 1);
          if (++probes >= kHashSlots) {
            fail = 1;
            break;
          }
        }
        if (probes < kHashSlots) atomicAdd(&hval[h], v);
      }
    }
    __syncthreads();
    if (fail) {
      if (threadIdx.x == 0) atomicOr(overflow, 1);
      __syncthreads();
      continue;
    }
    // compact occupied slots to the front: (col << 32 | slot) keys reuse hkey/hval storage order
    // via a second pass; collect into a sorted list with a block bitonic sort of 64-bit keys
    // stored in the (now free) upper part of smem.
    uint64_t* keys = reinterpret_cast<uint64_t*>(smem + kHashSlots * (sizeof(int) + sizeof(double)));
    for (int t = threadIdx.x; t < kHashSlots; t += blockDim.x) {
      int k = hkey[t];
      if (k >= 0) {
        int pos = atomicAdd(&nfill, 1);
        keys[pos] = ((uint64_t)(uint32_t)k << 32) | (uint32_t)t;
      }
    }
    __syncthreads();
    int L = nfill;
    int M = 1;
    while (M < L) M <<= 1;
    for (int t = L + threadIdx.x; t < M; t += blockDim.x) keys[t] = ~0ull;
    __syncthreads();
    for (int k = 2; k <= M; k <<= 1) {
      for (int jj = k >> 1; jj > 0; jj >>= 1) {
        for (int t = threadIdx.x; t < M; t += blockDim.x) {
          int ixj = t ^ jj;
          if (ixj > t) {
            uint64_t x = keys[t], y = keys[ixj];
            bool asc = (t & k) == 0;
            if ((x > y) == asc) {
              keys[t] = y;
              keys[ixj] = x;
            }
          }
        }
        __syncthreads();
      }
    }
    if (mode != 1 && threadIdx.x == 0) cnt[row] = L;
    if (mode != 0) {
      const long long base = mode == 1 ? (long long)crp[row] : uoff[row];
      for (int t = threadIdx.x; t < L; t += blockDim.x) {
        ccol[base + t] = (int)(keys[t] >> 32);
        cval[base + t] = hval[(uint32_t)(keys[t] & kLow32)];
      }
    }
    __syncthreads();
  }
}

// Values of C = A B on C's known pattern.  Rows with at most kNumSmall products:
// one thread per row, products in the ESC order (sums identical to the symbolic
// pass).  Larger rows: k_spgemm_numeric_block.
constexpr int kNumSmall = 64;

template <class T>
__global__ void k_spgemm_numeric(int nrows, const int* __restrict__ arp, const int* __restrict__ acol,
                                 const T* __restrict__ aval, const int* __restrict__ brp,
                                 const int* __restrict__ bcol, const T* __restrict__ bval,
                                 const int* __restrict__ crp, const int* __restrict__ ccol,
                                 T* __restrict__ cval, const int* __restrict__ u) {
  constexpr int kReg = 32;  // rows with at most kReg entries accumulate in a per-thread array
  for (int row = blockIdx.x * blockDim.x + threadIdx.x; row < nrows; row += gridDim.x * blockDim.x) {
    if (u[row] > kNumSmall) continue;
    int c0 = crp[row], c1 = crp[row + 1], L = c1 - c0;
    if (L <= kReg) {
      int cc[kReg];
      T acc[kReg];
#pragma unroll
      for (int q = 0; q < kReg; ++q) {
        cc[q] = q < L ? ccol[c0 + q] : -1;
        acc[q] = T(0);
      }
      for (int e = arp[row]; e < arp[row + 1]; ++e) {
        int j = acol[e];
        T a = aval[e];
        for (int f = brp[j]; f < brp[j + 1]; ++f) {
          int key = bcol[f];
          T v = a * bval[f];
          int pos = 0;
#pragma unroll
          for (int q = 0; q < kReg; ++q) pos = cc[q] == key ? q : pos;
          acc[pos] += v;
        }
      }
      for (int q = 0; q < L; ++q) cval[c0 + q] = acc[q];
      continue;
    }
    for (int q = c0; q < c1; ++q) cval[q] = T(0);
    for (int e = arp[row]; e < arp[row + 1]; ++e) {
      int j = acol[e];
      T a = aval[e];
      for (int f = brp[j]; f < brp[j + 1]; ++f) {
        int pos = find_col(ccol, c0, c1, bcol[f]);
        cval[pos] += a * bval[f];
      }
    }
  }
}

// One warp per row with more than kNumSmall products and at most kWarpL output
// entries: the row's columns and accumulators sit in the warp's slice of shared
// memory; A entries are taken 32 at a time, a warp scan of their B-row lengths
// flattens the products over the lanes.
constexpr int kWarpL = 256;
constexpr int kWarpRowsPerBlock = 8;

template <class T>
__global__ void __launch_bounds__(32 * kWarpRowsPerBlock) k_spgemm_numeric_warp(
    int nrows, const int* __restrict__ arp, const int* __restrict__ acol, const T* __restrict__ aval,
    const int* __restrict__ brp, const int* __restrict__ bcol, const T* __restrict__ bval,
    const int* __restrict__ crp, const int* __restrict__ ccol, T* __restrict__ cval,
    const int* __restrict__ u) {
  __shared__ T sacc_all[kWarpRowsPerBlock][kWarpL];
  __shared__ int scol_all[kWarpRowsPerBlock][kWarpL];
  __shared__ int pre_all[kWarpRowsPerBlock][33];
  __shared__ int bst_all[kWarpRowsPerBlock][32];
  __shared__ T av_all[kWarpRowsPerBlock][32];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  T* sacc = sacc_all[w];
  int* scol = scol_all[w];
  int* pre = pre_all[w];
  int nw = gridDim.x * kWarpRowsPerBlock;
  for (int row = blockIdx.x * kWarpRowsPerBlock + w; row < nrows; row += nw) {
    int c0 = crp[row], c1 = crp[row + 1], L = c1 - c0;
    if (u[row] <= kNumSmall || L > kWarpL) continue;
    for (int t = lane; t < L; t += 32) {
      scol[t] = ccol[c0 + t];
      sacc[t] = T(0);
    }
    __syncwarp();
    for (int e0 = arp[row]; e0 < arp[row + 1]; e0 += 32) {
      int e = e0 + lane;
      bool has = e < arp[row + 1];
      int j = has ? acol[e] : 0;
      T a = has ? aval[e] : T(0);
      int b0 = has ? brp[j] : 0;
      int len = has ? brp[j + 1] - b0 : 0;
      int inc = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      pre[lane + 1] = inc;
      if (lane == 0) pre[0] = 0;
      int total = __shfl_sync(0xffffffffu, inc, 31);
      bst_all[w][lane] = b0;
      av_all[w][lane] = a;
      __syncwarp();
      for (int t = lane; t < total; t += 32) {
        int lo = 0, hi = 32;  // owner q of product t: pre[q] <= t < pre[q+1]
        while (hi - lo > 1) {
          int mid = (lo + hi) >> 1;
          if (pre[mid] <= t) lo = mid; else hi = mid;
        }
        int f = bst_all[w][lo] + (t - pre[lo]);
        int key = bcol[f];
        T v = av_all[w][lo] * bval[f];
        int pos = find_col(scol, 0, L, key);
        atomicAdd(&sacc[pos], v);
      }
      __syncwarp();
    }
    for (int t = lane; t < L; t += 32) cval[c0 + t] = sacc[t];
    __syncwarp();
  }
}

// One block per row with more than kNumSmall products.  The row's products are
// flattened: a block scan of the B-row lengths over the row's A entries gives
// each product index t an (A entry, B entry) pair, so every thread has work
// however short the B rows are.  The row's column list and accumulators sit in
// shared memory (rows up to kNumLmax entries; longer rows accumulate in global
// memory); products are added with atomics (rounding-level order dependence).
constexpr int kNumLmax = 4096;
constexpr int kNumAmax = 2048;   // A entries per row staged at once
constexpr int kNumThreads = 256;
constexpr int kDenseCols = 8192; // C with at most this many columns: accumulate by column directly

// DENSE: the shared accumulator is indexed by column (C has <= kDenseCols columns),
// so a product needs no search; otherwise the row's sorted column list is searched.
template <class T, bool DENSE>
__global__ void __launch_bounds__(kNumThreads) k_spgemm_numeric_block(
    int nrows, const int* __restrict__ arp, const int* __restrict__ acol, const T* __restrict__ aval,
    const int* __restrict__ brp, const int* __restrict__ bcol, const T* __restrict__ bval,
    const int* __restrict__ crp, const int* __restrict__ ccol, T* __restrict__ cval,
    const int* __restrict__ u, int ncols) {
  // dynamic shared memory: sacc[kNumLmax] av[kNumAmax] (doubles), then scol[kNumLmax]
  // off[kNumAmax + 1] bstart[kNumAmax] (ints)
  extern __shared__ unsigned char dsm[];
  T* sacc = reinterpret_cast<T*>(dsm);
  T* av = sacc + (DENSE ? kDenseCols : kNumLmax);
  int* scol = reinterpret_cast<int*>(av + kNumAmax);
  int* off = scol + kNumLmax;         // prefix of B-row lengths over the staged A entries
  int* bstart = off + kNumAmax + 1;
  __shared__ int wsum[kNumThreads / 32];
  for (int row = blockIdx.x; row < nrows; row += gridDim.x) {
    if (u[row] <= kNumSmall) continue;
    int c0 = crp[row], c1 = crp[row + 1], L = c1 - c0;
    if (L <= kWarpL) continue;  // k_spgemm_numeric_warp
    bool sh = DENSE || L <= kNumLmax;
    if (DENSE) {
      for (int t = threadIdx.x; t < L; t += blockDim.x) sacc[ccol[c0 + t]] = T(0);
    } else if (sh) {
      for (int t = threadIdx.x; t < L; t += blockDim.x) {
        scol[t] = ccol[c0 + t];
        sacc[t] = T(0);
      }
    } else {
      for (int t = threadIdx.x; t < L; t += blockDim.x) cval[c0 + t] = T(0);
    }
    __syncthreads();
    for (int e0 = arp[row]; e0 < arp[row + 1]; e0 += kNumAmax) {
      int na = min(kNumAmax, arp[row + 1] - e0);
      // stage A entries and the lengths of their B rows; block-wide exclusive scan
      int per = (na + blockDim.x - 1) / blockDim.x;
      int lo = threadIdx.x * per, hi = min(na, lo + per);
      int local = 0;
      for (int q = lo; q < hi; ++q) {
        int j = acol[e0 + q];
        int b0 = brp[j];
        bstart[q] = b0;
        av[q] = aval[e0 + q];
        int len = brp[j + 1] - b0;
        off[q] = local;
        local += len;
      }
      // exclusive scan of the per-thread totals
      int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
      int inc = local;
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      if (lane == 31) wsum[wid] = inc;
      __syncthreads();
      int wbase = 0;
      for (int q = 0; q < wid; ++q) wbase += wsum[q];
      int tbase = wbase + inc - local;
      for (int q = lo; q < hi; ++q) off[q] += tbase;
      __syncthreads();
      int total = 0;
      for (int q = 0; q < (int)(blockDim.x >> 5); ++q) total += wsum[q];
      if (threadIdx.x == 0) off[na] = total;
      __syncthreads();
      for (int t = threadIdx.x; t < total; t += blockDim.x) {
        // A entry q with off[q] <= t < off[q+1]
        int lo2 = 0, hi2 = na;
        while (hi2 - lo2 > 1) {
          int mid = (lo2 + hi2) >> 1;
          if (off[mid] <= t) lo2 = mid; else hi2 = mid;
        }
        int f = bstart[lo2] + (t - off[lo2]);
        int key = bcol[f];
        T v = av[lo2] * bval[f];
        if (DENSE) {
          atomicAdd(&sacc[key], v);
        } else if (sh) {
          int pos = find_col(scol, 0, L, key);
          atomicAdd(&sacc[pos], v);
        } else {
          int pos = find_col(ccol, c0, c1, key);
          atomicAdd(&cval[pos], v);
        }
      }
      __syncthreads();
    }
    if (DENSE)
      for (int t = threadIdx.x; t < L; t += blockDim.x) cval[c0 + t] = sacc[ccol[c0 + t]];
    else if (sh)
      for (int t = threadIdx.x; t < L; t += blockDim.x) cval[c0 + t] = sacc[t];
    __syncthreads();
  }
}

// ---------------------------------------------------------------- Galerkin refresh by product lists
// The patterns of A P and R (A P) do not change between refreshes, so the pair
// (A entry, B entry) behind each scalar product, and the C entry it adds to, are
// the same every time.  k_plist enumerates the products of each row (one warp
// per row, A entries 32 at a time, a warp scan of their B-row lengths spreads
// the products over the lanes) and either counts the products of every C entry
// or files each pair into its C entry's segment; k_plist_sort then orders each
// segment by A entry, which is the order a row-by-row product sums in.
constexpr int kPlWarps = 8;

template <bool FILL>
__global__ void __launch_bounds__(32 * kPlWarps) k_plist(int nrows, const int* __restrict__ arp,
                                                         const int* __restrict__ acol, const int* __restrict__ brp,
                                                         const int* __restrict__ bcol, const int* __restrict__ crp,
                                                         const int* __restrict__ ccol, int* __restrict__ cnt,
                                                         const int* __restrict__ seg,
                                                         const long long* __restrict__ base, int* __restrict__ pa,
                                                         int* __restrict__ pb) {
  __shared__ int pre_all[kPlWarps][33];
  __shared__ int bst_all[kPlWarps][32];
  int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int* pre = pre_all[w];
  int* bst = bst_all[w];
  int nw = gridDim.x * kPlWarps;
  for (int row = blockIdx.x * kPlWarps + w; row < nrows; row += nw) {
    int c0 = crp[row], c1 = crp[row + 1];
    int a1 = arp[row + 1];
    for (int e0 = arp[row]; e0 < a1; e0 += 32) {
      int e = e0 + lane;
      bool has = e < a1;
      int j = has ? acol[e] : 0;
      int b0 = has ? brp[j] : 0;
      int len = has ? brp[j + 1] - b0 : 0;
      int inc = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
      }
      int total = __shfl_sync(0xffffffffu, inc, 31);
      pre[lane + 1] = inc;
      if (lane == 0) pre[0] = 0;
      bst[lane] = b0;
      __syncwarp();
      for (int t = lane; t < total; t += 32) {
        int lo = 0, hi = 32;  // owner q of product t: pre[q] <= t < pre[q+1]
        while (hi - lo > 1) {
          int mid = (lo + hi) >> 1;
          if (pre[mid] <= t) lo = mid; else hi = mid;
        }
        int f = bst[lo] + (t - pre[lo]);
        int q = find_col(ccol, c0, c1, bcol[f]);
        int slot = atomicAdd(&cnt[q], 1);
        if (FILL) {
          long long at = base[q >> kPlShift] + seg[q] + slot;
          pa[at] = e0 + lo;
          pb[at] = f;
        }
      }
      __syncwarp();
    }
  }
}

// 64-bit segment starts -> chunk bases and 32-bit remainders.
__global__ void k_plist_split(int nnz, const long long* __restrict__ segll, int* __restrict__ seg,
                              long long* __restrict__ base) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q <= nnz; q += gridDim.x * blockDim.x) {
    long long b = segll[(q >> kPlShift) << kPlShift];
    seg[q] = (int)(segll[q] - b);
    if ((q & ((1 << kPlShift) - 1)) == 0) base[q >> kPlShift] = b;
  }
}

__device__ __forceinline__ long long plist_start(const int* __restrict__ seg, const long long* __restrict__ base,
                                                 int q) {
  return base[q >> kPlShift] + seg[q];
}

// Insertion sort of each segment by A entry (segments hold tens of pairs).
__global__ void k_plist_sort(int nnz, const int* __restrict__ seg, const long long* __restrict__ base,
                             int* __restrict__ pa, int* __restrict__ pb) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += gridDim.x * blockDim.x) {
    long long s0 = plist_start(seg, base, q), s1 = plist_start(seg, base, q + 1);
    for (long long t = s0 + 1; t < s1; ++t) {
      int ka = pa[t], kb = pb[t];
      long long v = t - 1;
      while (v >= s0 && pa[v] > ka) {
        pa[v + 1] = pa[v];
        pb[v + 1] = pb[v];
        --v;
      }
      pa[v + 1] = ka;
      pb[v + 1] = kb;
    }
  }
}

__global__ void k_sum_rows_ll(int n, const int* __restrict__ u, unsigned long long* __restrict__ out) {
  unsigned long long s = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) s += (unsigned)u[i];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) atomicAdd(out, s);
}

// c[q] = sum over the segment of q of a[pa] * b[pb], in segment order: no
// search, no atomics, the same sum every refresh.  One thread per entry keeps
// the threads of a warp on neighbouring entries of one C row, whose pairs read
// neighbouring B entries (a lane group per entry was measured slower: its
// gathers from B, too large for L2, lose that locality).
template <class T>
__global__ void __launch_bounds__(256) k_galerkin_lists(int nnz, const int* __restrict__ seg,
                                                        const long long* __restrict__ base,
                                                        const int* __restrict__ pa, const int* __restrict__ pb,
                                                        const T* __restrict__ aval, const T* __restrict__ bval,
                                                        T* __restrict__ cval) {
  for (int q = blockIdx.x * blockDim.x + threadIdx.x; q < nnz; q += gridDim.x * blockDim.x) {
    long long s0 = plist_start(seg, base, q), s1 = plist_start(seg, base, q + 1);
    T acc = T(0);
    for (long long t = s0; t < s1; ++t) acc += aval[pa[t]] * bval[pb[t]];
    cval[q] = acc;
  }
}

// ---------------------------------------------------------------- coarsest level: dense inverse

template <class T>
__global__ void k_csr_to_dense(int n, const int* __restrict__ rp, const int* __restrict__ col,
                               const T* __restrict__ val, double* __restrict__ dense) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    for (int j = 0; j < n; ++j) dense[(long long)i * n + j] = 0.0;
    for (int e = rp[i]; e < rp[i + 1]; ++e) dense[(long long)i * n + col[e]] = (double)val[e];
  }
}

// Blocked Gauss-Jordan inversion in place (no pivoting: the matrix is SPD).
// For a panel P of kGjB consecutive pivots and the other indices O, one block
// step turns [[A_PP, A_PO], [A_OP, A_OO]] into
//   [[A_PP^-1, A_PP^-1 A_PO], [-A_OP A_PP^-1, A_OO - A_OP A_PP^-1 A_PO]];
// after every panel the matrix holds A^-1.  Three launches per panel:
// k_gj_panel inverts A_PP in shared memory; k_gj_rows forms the new panel rows
// and saves the old panel columns; k_gj_update applies the rank-kGjB update as
// a shared-memory tiled product.  Work buffer (2 kGjB n + kGjB^2 doubles):
// R[p][j] (new panel rows; for j in P the panel inverse), C[p][i] (old panel
// columns), Pinv (kGjB x kGjB).
constexpr int kGjB = 32;

__global__ void __launch_bounds__(kGjB* kGjB) k_gj_panel(int n, int K, int bs, double* __restrict__ a,
                                                        double* __restrict__ pinv) {
  __shared__ double m[kGjB][kGjB + 1];
  __shared__ double rowk[kGjB], colk[kGjB];  // pivot row, and pivot column scaled by 1/pivot
  __shared__ double inv;
  const int r = threadIdx.y, q = threadIdx.x;  // element (r, q) of the bs x bs panel block
  const bool in = r < bs && q < bs;
  if (in) m[r][q] = a[(long long)(K + r) * n + K + q];
  __syncthreads();
  for (int k = 0; k < bs; ++k) {
    if (r == 0 && q == 0) inv = 1.0 / m[k][k];  // the step's one division
    if (in && r == k) rowk[q] = m[k][q];
    __syncthreads();
    if (in && q == k) colk[r] = m[r][k] * inv;
    __syncthreads();
    if (in) {
      double v;
      if (r == k) v = (q == k) ? inv : rowk[q] * inv;
      else if (q == k) v = -colk[r];
      else v = fma(-colk[r], rowk[q], m[r][q]);
      m[r][q] = v;
    }
    __syncthreads();
  }
  if (in) a[(long long)(K + r) * n + K + q] = m[r][q];
  pinv[r * kGjB + q] = in ? m[r][q] : 0.0;  // zeros outside a partial last panel
}

// Columns j0 .. j0+7 per block, thread (p, jj): R[p][j] = (Pinv A_P,j)_p written
// back to panel row p (j outside P), or the panel inverse's entry (j in P); the
// same thread saves row i = j's old panel entry C[p][i] = a_i,K+p (i outside P).
constexpr int kGjCols = 8;

__global__ void __launch_bounds__(kGjB* kGjCols) k_gj_rows(int n, int K, int bs, double* __restrict__ a,
                                                          const double* __restrict__ pinv, double* __restrict__ R,
                                                          double* __restrict__ C) {
  __shared__ double ps[kGjB][kGjB + 1];
  __shared__ double cs[kGjB][kGjCols];
  const int p = threadIdx.x, jj = threadIdx.y;
  for (int t = jj; t < kGjB; t += kGjCols) ps[t][p] = pinv[t * kGjB + p];
  const int j = blockIdx.x * kGjCols + jj;
  const bool inP = j >= K && j < K + bs;
  cs[p][jj] = (j < n && p < bs && !inP) ? a[(long long)(K + p) * n + j] : 0.0;
  __syncthreads();
  if (j >= n || p >= bs) return;
  if (inP) {
    R[(long long)p * n + j] = ps[p][j - K];
    return;
  }
  double v = 0.0;
#pragma unroll
  for (int q = 0; q < kGjB; ++q) v = fma(ps[p][q], cs[q][jj], v);
  R[(long long)p * n + j] = v;
  a[(long long)(K + p) * n + j] = v;
  C[(long long)p * n + j] = a[(long long)j * n + K + p];
}

// a_ij <- (j in P ? 0 : a_ij) - sum_p C[p][i] R[p][j] for rows i outside P; one
// kGjB x kGjB tile of (i, j) per block.
__global__ void __launch_bounds__(kGjB* kGjB) k_gj_update(int n, int K, int bs, double* __restrict__ a,
                                                         const double* __restrict__ R, const double* __restrict__ C) {
  __shared__ double cs[kGjB][kGjB + 1];  // cs[p][ti]
  __shared__ double rs[kGjB][kGjB + 1];  // rs[p][tj]
  const int ti = threadIdx.y, tj = threadIdx.x;
  const int i0 = blockIdx.y * kGjB, j0 = blockIdx.x * kGjB;
  for (int p = ti; p < kGjB; p += blockDim.y) {
    const int i = i0 + tj, j = j0 + tj;
    cs[p][tj] = (p < bs && i < n) ? C[(long long)p * n + i] : 0.0;
    rs[p][tj] = (p < bs && j < n) ? R[(long long)p * n + j] : 0.0;
  }
  __syncthreads();
  const int i = i0 + ti, j = j0 + tj;
  if (i >= n || j >= n || (i >= K && i < K + bs)) return;
  double acc = (j >= K && j < K + bs) ? 0.0 : a[(long long)i * n + j];
#pragma unroll 8
  for (int p = 0; p < kGjB; ++p) acc = fma(-cs[p][ti], rs[p][tj], acc);
  a[(long long)i * n + j] = acc;
}

// ---------------------------------------------------------------- matching aggregation
// Coupled aggregation by compatible weighted matching (the paper's SMATCH
// coarsening, Sec. 5.2).  Edge {i, j} of a negative coupling has the weight
// w_ij = 1 - (a_ij + a_ji) / (a_ii + a_jj) (smooth vector of ones), rounded to
// FP32 so that rounding-order differences of the FP64 matrices do not reorder
// equal weights; edges are ordered by weight, then by (min, max) index pair.
// The matching is locally dominant: synchronous rounds in which every unmatched
// node proposes to its best unmatched neighbour and mutual proposals match.

__device__ __forceinline__ bool match_better(float w1, int lo1, int hi1, float w2, int lo2, int hi2) {
  if (w1 != w2) return w1 > w2;
  if (lo1 != lo2) return lo1 < lo2;
  return hi1 < hi2;
}

__global__ void k_match_weights(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                const double* __restrict__ val, const double* __restrict__ d,
                                float* __restrict__ w) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    for (int e = rp[i]; e < rp[i + 1]; ++e) {
      int j = col[e];
      float wv = -CUDART_INF_F;
      if (j != i) {
        int q = find_col(col, rp[j], rp[j + 1], i);  // a_ji (the pattern is symmetric)
        if (q < rp[j + 1] && col[q] == i) {
          double sum = val[e] + val[q];
          if (sum < 0.0) wv = (float)(1.0 - sum / (d[i] + d[j]));
        }
      }
      w[e] = wv;
    }
  }
}

// Proposals of one round; *any = 1 if some node proposed.
__global__ void k_match_propose(int n, const int* __restrict__ rp, const int* __restrict__ col,
                                const float* __restrict__ w, const int* __restrict__ mate, int* __restrict__ cand,
                                int* __restrict__ any) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int best = -1;
    float bw = -CUDART_INF_F;
    int blo = 0, bhi = 0;
    if (mate[i] < 0) {
      for (int e = rp[i]; e < rp[i + 1]; ++e) {
        int j = col[e];
        float we = w[e];
        if (we == -CUDART_INF_F || mate[j] >= 0) continue;
        int lo = min(i, j), hi = max(i, j);
        if (best < 0 || match_better(we, lo, hi, bw, blo, bhi)) {
          best = j;
          bw = we;
          blo = lo;
          bhi = hi;
        }
      }
    }
    cand[i] = best;
    if (best >= 0) *any = 1;
  }
}

__global__ void k_match_commit(int n, const int* __restrict__ cand, int* __restrict__ mate) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int j = cand[i];
    if (j >= 0 && cand[j] == i) mate[i] = j;
  }
}

// 1 for the smallest member of each pair and for every unmatched node.
__global__ void k_pair_first(int n, const int* __restrict__ mate, int* __restrict__ first) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    first[i] = mate[i] < 0 || i < mate[i];
}

__global__ void k_pair_ids(int n, const int* __restrict__ mate, const int* __restrict__ pos, int* __restrict__ ids) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    int m = mate[i];
    ids[i] = pos[m < 0 ? i : min(i, m)];
  }
}

// agg[i] = ids[agg[i]] (composition of the pairing passes).
__global__ void k_compose(int n, const int* __restrict__ ids, int* __restrict__ agg) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) agg[i] = ids[agg[i]];
}

__global__ void k_iota(int n, int* __restrict__ a) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) a[i] = i;
}

// Single-pass SpGEMM: row r's cnt[r] compressed entries move from the temporary at
// its product offset uoff[r] to crp[r]; one warp per row.
__global__ void k_compact_rows(int n, const long long* __restrict__ uoff, const int* __restrict__ cnt,
                               const int* __restrict__ crp, const int* __restrict__ tcol,
                               const double* __restrict__ tval, int* __restrict__ ccol, double* __restrict__ cval) {
  const int lane = threadIdx.x & 31;
  for (long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; row < n;
       row += ((long long)gridDim.x * blockDim.x) >> 5) {
    const long long src = uoff[row];
    const int dst = crp[row], m = cnt[row];
    for (int t = lane; t < m; t += 32) {
      ccol[dst + t] = tcol[src + t];
      cval[dst + t] = tval[src + t];
    }
  }
}

// ---------------------------------------------------------------- host side

// One int from the device, on the context's stream only (a plain cudaMemcpy would
// run on the legacy default stream and wait for every blocking stream, e.g. the
// other request-server slots).
static int read_dev_int(rich_ctx* c, const int* src, int* out) {
  RICH_CUDA(cudaMemcpyAsync(c->hflag + 8, src, sizeof(int), cudaMemcpyDeviceToHost, c->st));
  RICH_CUDA(cudaStreamSynchronize(c->st));
  *out = c->hflag[8];
  return RICH_OK;
}

static int spgemm_upper(rich_ctx* c, const Csr<double>& A, const Csr<double>& B, int* u, int* umax) {
  int n = A.nrows;
  k_spgemm_upper<<<grid_for(n), kBlock, 0, c->st>>>(n, A.rowptr, A.col, B.rowptr, u);
  RICH_LAUNCH_CHECK();
  if (umax) {
    RICH_CUDA(cudaMemsetAsync(c->iflag, 0, sizeof(int), c->st));
    k_max_int<<<grid_for(n), kBlock, 0, c->st>>>(n, u, c->iflag);
    RICH_LAUNCH_CHECK();
    RICH_CUDA(cudaMemcpyAsync(c->hflag, c->iflag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    RICH_CUDA(cudaStreamSynchronize(c->st));
    *umax = c->hflag[0];
  }
  return RICH_OK;
}

// C = A B: structural pattern (sorted columns) and values.  *u_keep, if given,
// receives the per-row product counts (kept for the numeric refresh); *hashed, if
// given, whether rows with more than kEscCap products went through the hash kernel,
// whose FP64 sums follow the order of shared-memory atomics.
static int spgemm_symbolic(rich_ctx* c, const Csr<double>& A, const Csr<double>& B, Csr<double>& C,
                           int** u_keep = nullptr, bool* hashed = nullptr) {
  int n = A.nrows;
  C.nrows = n;
  C.ncols = B.ncols;
  int* u = nullptr;
  int* cnt = nullptr;
  RICH_CHECK(dalloc(&u, n));
  RICH_CHECK(dalloc(&cnt, n));
  RICH_CHECK(dalloc(&C.rowptr, (long long)n + 1));
  int umax = 0;
  RICH_CHECK(spgemm_upper(c, A, B, u, &umax));
  if (umax >= (1 << 30)) return RICH_ELIMIT;
  // shared memory per warp sized by the largest row of this product
  int cap = 32;
  while (cap < umax && cap < kEscCap) cap <<= 1;
  const int esc_warps = cap <= 128 ? 8 : (cap <= 512 ? 4 : 2);
  size_t smem = (size_t)esc_warps * cap * (sizeof(uint64_t) + sizeof(double));
  int nblk = (n + esc_warps - 1) / esc_warps;
  if (nblk > 65535 * 4) nblk = 65535 * 4;
  bool big = umax > kEscCap;
  if (hashed) *hashed = big;
  size_t hsmem = (size_t)kHashSlots * (sizeof(int) + sizeof(double) + sizeof(uint64_t));
  if (big) RICH_CUDA(cudaFuncSetAttribute(k_spgemm_hash, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)hsmem));
  int* ovf = c->iflag + 1;
  RICH_CUDA(cudaMemsetAsync(ovf, 0, sizeof(int), c->st));
  // One pass when a temporary of every product's slot fits in a quarter of the free
  // memory: each row is expanded, sorted and compressed once, at its product offset,
  // then compacted.  Otherwise two passes (count, then write at the final offsets).
  long long* uoff = nullptr;
  RICH_CHECK(dalloc(&uoff, (long long)n + 1));
  RICH_CHECK(scan_exclusive_int_ll(c, u, uoff, n));
  long long nprod = 0;
  RICH_CUDA(cudaMemcpyAsync(&nprod, uoff + n, sizeof(long long), cudaMemcpyDeviceToHost, c->st));
  RICH_CUDA(cudaStreamSynchronize(c->st));
  size_t mfree = 0, mtotal = 0;
  RICH_CUDA(cudaMemGetInfo(&mfree, &mtotal));
  const bool one_pass = (double)nprod * (sizeof(int) + sizeof(double)) <= 0.25 * (double)mfree;
  int* tcol = nullptr;
  double* tval = nullptr;
  if (one_pass) {
    RICH_CHECK(dalloc(&tcol, nprod));
    RICH_CHECK(dalloc(&tval, nprod));
  }
  for (int pass = 0; pass < 2; ++pass) {
    const int mode = one_pass ? 2 : pass;
    if (pass == 1) {
      // the row offsets are 32-bit: check the total in 64 bits before the scan
      unsigned long long* dsum = reinterpret_cast<unsigned long long*>(c->iflag + 4);  // slots 4-5
      RICH_CUDA(cudaMemsetAsync(dsum, 0, sizeof(unsigned long long), c->st));
      k_sum_rows_ll<<<red_grid(n), kBlock, 0, c->st>>>(n, cnt, dsum);
      RICH_LAUNCH_CHECK();
      unsigned long long total = 0;
      RICH_CUDA(cudaMemcpyAsync(&total, dsum, sizeof(total), cudaMemcpyDeviceToHost, c->st));
      RICH_CUDA(cudaStreamSynchronize(c->st));
      if (total > 2147483647ull) return RICH_ELIMIT;
      RICH_CHECK(scan_exclusive_int(c, cnt, C.rowptr, n));
      int nnz = 0;
      RICH_CHECK(read_dev_int(c, C.rowptr + n, &nnz));
      if (nnz < 0 || (unsigned long long)nnz != total) return RICH_ELIMIT;
      C.nnz = nnz;
      RICH_CHECK(dalloc(&C.col, nnz));
      RICH_CHECK(dalloc(&C.val, nnz));
      if (one_pass) {
        k_compact_rows<<<grid_for(32LL * n), kBlock, 0, c->st>>>(n, uoff, cnt, C.rowptr, tcol, tval, C.col, C.val);
        RICH_LAUNCH_CHECK();
        break;
      }
    }
    int* ocol = mode == 2 ? tcol : C.col;
    double* oval = mode == 2 ? tval : C.val;
    k_spgemm_esc<<<nblk, 32 * esc_warps, smem, c->st>>>(n, A.rowptr, A.col, A.val, B.rowptr, B.col, B.val, u, mode,
                                                       C.rowptr, uoff, ocol, oval, cnt, cap);
    RICH_LAUNCH_CHECK();
    if (big) {
      int hb = n < 8 * kNumSM ? n : 8 * kNumSM;
      k_spgemm_hash<<<hb, kHashThreads, hsmem, c->st>>>(n, A.rowptr, A.col, A.val, B.rowptr, B.col, B.val, u, mode,
                                                        C.rowptr, uoff, ocol, oval, cnt, ovf);
      RICH_LAUNCH_CHECK();
      RICH_CUDA(cudaMemcpyAsync(c->hflag + 1, ovf, sizeof(int), cudaMemcpyDeviceToHost, c->st));
      RICH_CUDA(cudaStreamSynchronize(c->st));
      if (c->hflag[1]) return RICH_ELIMIT;  // a row has more distinct columns than the hash table holds
    }
  }
  dfree(tcol);
  dfree(tval);
  dfree(uoff);
  RICH_CUDA(cudaStreamSynchronize(c->st));
  if (u_keep) *u_keep = u; else dfree(u);
  dfree(cnt);
  return RICH_OK;
}

static const char* kNumericName[2][16] = {
    {"galerkin_ap_l0", "galerkin_ap_l1", "galerkin_ap_l2", "galerkin_ap_l3", "galerkin_ap_l4", "galerkin_ap_l5",
     "galerkin_ap_l6", "galerkin_ap_l7", "galerkin_ap_l8", "galerkin_ap_l9", "galerkin_ap", "galerkin_ap",
     "galerkin_ap", "galerkin_ap", "galerkin_ap", "galerkin_ap"},
    {"galerkin_rap_l0", "galerkin_rap_l1", "galerkin_rap_l2", "galerkin_rap_l3", "galerkin_rap_l4",
     "galerkin_rap_l5", "galerkin_rap_l6", "galerkin_rap_l7", "galerkin_rap_l8", "galerkin_rap_l9", "galerkin_rap",
     "galerkin_rap", "galerkin_rap", "galerkin_rap", "galerkin_rap", "galerkin_rap"}};

static void plist_free(ProdList& pl) {
  dfree(pl.seg);
  dfree(pl.base);
  dfree(pl.pa);
  dfree(pl.pb);
  pl.np = 0;
}

// Product lists of C = A B (u = products per row).  Leaves pl empty, and
// returns RICH_OK, when the lists would not fit in half the free device
// memory; the refresh then falls back to the searching kernels.
static int plist_build(rich_ctx* c, const Csr<double>& A, const Csr<double>& B, const Csr<double>& C, const int* u,
                       ProdList& pl) {
  plist_free(pl);
  unsigned long long* dsum = reinterpret_cast<unsigned long long*>(c->iflag + 4);  // slots 4-5, 16-byte aligned
  RICH_CUDA(cudaMemsetAsync(dsum, 0, sizeof(unsigned long long), c->st));
  k_sum_rows_ll<<<red_grid(A.nrows), kBlock, 0, c->st>>>(A.nrows, u, dsum);
  RICH_LAUNCH_CHECK();
  unsigned long long np = 0;
  RICH_CUDA(cudaMemcpyAsync(&np, dsum, sizeof(np), cudaMemcpyDeviceToHost, c->st));
  RICH_CUDA(cudaStreamSynchronize(c->st));
  size_t fr = 0, tot = 0;
  RICH_CUDA(cudaStreamSynchronize(c->st));
  pool_trim();  // blocks freed into the pool count as free here
  RICH_CUDA(cudaMemGetInfo(&fr, &tot));
  double need = 8.0 * (double)np + 24.0 * ((double)C.nnz + 1);  // lists, offsets and the build's scratch
  if (need > 0.5 * (double)fr) return RICH_OK;
  int* cnt = nullptr;
  long long* segll = nullptr;
  RICH_CHECK(dalloc(&cnt, (long long)C.nnz + 1));
  RICH_CHECK(dalloc(&segll, (long long)C.nnz + 1));
  RICH_CHECK(dalloc(&pl.seg, (long long)C.nnz + 1));
  RICH_CHECK(dalloc(&pl.base, ((long long)C.nnz >> kPlShift) + 1));
  RICH_CHECK(dalloc(&pl.pa, (long long)np + 1));
  RICH_CHECK(dalloc(&pl.pb, (long long)np + 1));
  pl.np = (long long)np;
  int nwb = (A.nrows + kPlWarps - 1) / kPlWarps;
  if (nwb > 64 * kNumSM) nwb = 64 * kNumSM;
  RICH_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * ((size_t)C.nnz + 1), c->st));
  k_plist<false><<<nwb, 32 * kPlWarps, 0, c->st>>>(A.nrows, A.rowptr, A.col, B.rowptr, B.col, C.rowptr, C.col, cnt,
                                                   nullptr, nullptr, nullptr, nullptr);
  RICH_LAUNCH_CHECK();
  RICH_CHECK(scan_exclusive_int_ll(c, cnt, segll, C.nnz));
  k_plist_split<<<grid_for((long long)C.nnz + 1), kBlock, 0, c->st>>>(C.nnz, segll, pl.seg, pl.base);
  RICH_LAUNCH_CHECK();
  RICH_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * ((size_t)C.nnz + 1), c->st));
  k_plist<true><<<nwb, 32 * kPlWarps, 0, c->st>>>(A.nrows, A.rowptr, A.col, B.rowptr, B.col, C.rowptr, C.col, cnt,
                                                  pl.seg, pl.base, pl.pa, pl.pb);
  RICH_LAUNCH_CHECK();
  k_plist_sort<<<grid_for(C.nnz), kBlock, 0, c->st>>>(C.nnz, pl.seg, pl.base, pl.pa, pl.pb);
  RICH_LAUNCH_CHECK();
  RICH_CUDA(cudaStreamSynchronize(c->st));
  dfree(cnt);
  dfree(segll);
  return RICH_OK;
}

// C = A B on C's pattern with values of type T (aval/bval/cval); which = 0 for
// A P, 1 for R (A P); level for the profile name.  pl, if it holds lists, is used.
template <class T>
static int spgemm_numeric_t(rich_ctx* c, const Csr<double>& A, const T* aval, const Csr<double>& B, const T* bval,
                            const Csr<double>& C, T* cval, const int* u, int which, int level,
                            const ProdList* pl = nullptr) {
  if (pl && pl->seg) {
    ProfScope ps(kNumericName[which][level & 15], c->st,
                 4.0 * ((double)C.nnz + 1) + 8.0 * (double)pl->np +
                     (double)sizeof(T) * ((double)A.nnz + (double)B.nnz + (double)C.nnz),
                 2.0 * (double)pl->np);
    k_galerkin_lists<T><<<grid_for(C.nnz, 256), 256, 0, c->st>>>(C.nnz, pl->seg, pl->base, pl->pa, pl->pb, aval,
                                                                  bval, cval);
    RICH_LAUNCH_CHECK();
    return RICH_OK;
  }
  ProfScope ps(kNumericName[which][level & 15], c->st,
               (double)A.nrows * 4 + A.nnz * (4.0 + sizeof(T)) + (double)C.nrows * 4 + C.nnz * (4.0 + sizeof(T)));
  k_spgemm_numeric<T><<<grid_for(A.nrows, 128), 128, 0, c->st>>>(A.nrows, A.rowptr, A.col, aval, B.rowptr, B.col,
                                                                 bval, C.rowptr, C.col, cval, u);
  RICH_LAUNCH_CHECK();
  {
    int nwb = (A.nrows + kWarpRowsPerBlock - 1) / kWarpRowsPerBlock;
    if (nwb > 32 * kNumSM) nwb = 32 * kNumSM;
    k_spgemm_numeric_warp<T><<<nwb, 32 * kWarpRowsPerBlock, 0, c->st>>>(A.nrows, A.rowptr, A.col, aval, B.rowptr,
                                                                        B.col, bval, C.rowptr, C.col, cval, u);
    RICH_LAUNCH_CHECK();
  }
  int nb = A.nrows < 8 * kNumSM ? A.nrows : 8 * kNumSM;
  if (C.ncols <= kDenseCols) {
    const int dsm = (int)((kDenseCols + kNumAmax) * sizeof(double) + (kNumLmax + 2 * kNumAmax + 1) * sizeof(int));
    RICH_CUDA(cudaFuncSetAttribute(k_spgemm_numeric_block<T, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm));
    k_spgemm_numeric_block<T, true><<<nb, kNumThreads, dsm, c->st>>>(A.nrows, A.rowptr, A.col, aval, B.rowptr, B.col,
                                                                    bval, C.rowptr, C.col, cval, u, C.ncols);
  } else {
    const int dsm = (int)((kNumLmax + kNumAmax) * sizeof(double) + (kNumLmax + 2 * kNumAmax + 1) * sizeof(int));
    RICH_CUDA(cudaFuncSetAttribute(k_spgemm_numeric_block<T, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, dsm));
    k_spgemm_numeric_block<T, false><<<nb, kNumThreads, dsm, c->st>>>(A.nrows, A.rowptr, A.col, aval, B.rowptr,
                                                                     B.col, bval, C.rowptr, C.col, cval, u, C.ncols);
  }
  RICH_LAUNCH_CHECK();
  return RICH_OK;
}

static int spgemm_numeric(rich_ctx* c, const Csr<double>& A, const Csr<double>& B, Csr<double>& C, const int* u,
                          int which = 0, int level = 0, const ProdList* pl = nullptr) {
  return spgemm_numeric_t<double>(c, A, A.val, B, B.val, C, C.val, u, which, level, pl);
}

static void csr_free(Csr<double>& m, bool pattern = true) {
  if (pattern) {
    dfree(m.rowptr);
    dfree(m.col);
  }
  dfree(m.val);
  m.nnz = 0;
}

static int identity_csr(rich_ctx* c, int m, Csr<double>& I) {
  I.nrows = I.ncols = m;
  I.nnz = m;
  RICH_CHECK(dalloc(&I.rowptr, (long long)m + 1));
  RICH_CHECK(dalloc(&I.col, m));
  I.val = nullptr;  // treated as all-ones by the ESC kernel
  k_seq<<<grid_for(m + 1), kBlock, 0, c->st>>>(m, I.rowptr);
  RICH_LAUNCH_CHECK();
  k_seq<<<grid_for(m), kBlock, 0, c->st>>>(m - 1, I.col);
  RICH_LAUNCH_CHECK();
  return RICH_OK;
}

// R = P^T with sorted columns (atomic placement, then a sort through R_unsorted * I)
static int transpose(rich_ctx* c, const Csr<double>& P, Csr<double>& R) {
  int n = P.nrows, m = P.ncols;
  Csr<double> T;
  T.nrows = m;
  T.ncols = n;
  T.nnz = P.nnz;
  int* cnt = nullptr;
  int* fillc = nullptr;
  RICH_CHECK(dalloc(&cnt, m));
  RICH_CHECK(dalloc(&fillc, m));
  RICH_CHECK(dalloc(&T.rowptr, (long long)m + 1));
  RICH_CHECK(dalloc(&T.col, P.nnz));
  RICH_CHECK(dalloc(&T.val, P.nnz));
  RICH_CUDA(cudaMemsetAsync(cnt, 0, sizeof(int) * m, c->st));
  RICH_CUDA(cudaMemsetAsync(fillc, 0, sizeof(int) * m, c->st));
  k_tr_count<<<grid_for(n), kBlock, 0, c->st>>>(n, P.rowptr, P.col, cnt);
  RICH_LAUNCH_CHECK();
  RICH_CHECK(scan_exclusive_int(c, cnt, T.rowptr, m));
  k_tr_fill<<<grid_for(n), kBlock, 0, c->st>>>(n, P.rowptr, P.col, P.val, T.rowptr, fillc, T.col, T.val);
  RICH_LAUNCH_CHECK();
  Csr<double> I;
  RICH_CHECK(identity_csr(c, n, I));
  RICH_CHECK(spgemm_symbolic(c, T, I, R));
  csr_free(T);
  csr_free(I);
  dfree(cnt);
  dfree(fillc);
  return RICH_OK;
}

static int coarse_inverse_launches(rich_ctx* c);

// The coarsest inverse is n_c pivot launches; they are recorded once per hierarchy
// into a CUDA graph (fixed buffers) and replayed on every refresh.
static int coarse_inverse(rich_ctx* c) {
  Hierarchy& H = c->H;
  if (!H.dense) return RICH_OK;
  if (H.gj_exec) {
    ProfScope ps("coarse_inverse", c->st, 8.0 * (double)H.cn * H.cn * 2.0);
    RICH_CUDA(cudaGraphLaunch(H.gj_exec, c->st));
    count_launches(H.gj_nodes);
    return RICH_OK;
  }
  return coarse_inverse_launches(c);
}

static int capture_coarse_graph(rich_ctx* c) {
  Hierarchy& H = c->H;
  if (!H.dense || H.gj_exec) return RICH_OK;
  cudaStream_t cs;
  RICH_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaStream_t saved = c->st;
  RICH_CUDA(cudaStreamSynchronize(saved));
  c->st = cs;
  cudaGraph_t graph = nullptr;
  long long before = 0;
  rich_kernel_launches(&before);
  int rc = RICH_OK;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rc = coarse_inverse_launches(c);
    e = cudaStreamEndCapture(cs, &graph);
  }
  c->st = saved;
  long long after = 0;
  rich_kernel_launches(&after);
  count_launches(before - after);  // recorded, not launched
  if (e == cudaSuccess && rc == RICH_OK) {
    e = cudaGraphInstantiate(&H.gj_exec, graph, 0);
    if (e == cudaSuccess) H.gj_nodes = after - before;
    else H.gj_exec = nullptr;
  }
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) {
    cudaGetLastError();  // fall back to direct launches
    H.gj_exec = nullptr;
  }
  return rc;
}

static int coarse_inverse_launches(rich_ctx* c) {
  Hierarchy& H = c->H;
  Level& L = H.lv[H.nlev - 1];
  int n = L.n;
  // in MIXED precision the refreshed coarse values are the FP32 ones
  if (c->prec == RICH_PREC_MIXED && H.nlev > 1)
    k_csr_to_dense<float><<<grid_for(n), kBlock, 0, c->st>>>(n, L.A.rowptr, L.A.col, L.A32, H.cdense);
  else
    k_csr_to_dense<double><<<grid_for(n), kBlock, 0, c->st>>>(n, L.A.rowptr, L.A.col, L.A.val, H.cdense);
  RICH_LAUNCH_CHECK();
  long long nn = (long long)n * n;
  double* R = H.cwork;
  double* C = R + (long long)kGjB * n;
  double* pinv = C + (long long)kGjB * n;
  const dim3 tile(kGjB, kGjB);
  const dim3 tiles((unsigned)((n + kGjB - 1) / kGjB), (unsigned)((n + kGjB - 1) / kGjB));
  for (int K = 0; K < n; K += kGjB) {
    const int bs = n - K < kGjB ? n - K : kGjB;
    k_gj_panel<<<1, tile, 0, c->st>>>(n, K, bs, H.cdense, pinv);
    RICH_LAUNCH_CHECK();
    k_gj_rows<<<(n + kGjCols - 1) / kGjCols, dim3(kGjB, kGjCols), 0, c->st>>>(n, K, bs, H.cdense, pinv, R, C);
    RICH_LAUNCH_CHECK();
    k_gj_update<<<tiles, tile, 0, c->st>>>(n, K, bs, H.cdense, R, C);
    RICH_LAUNCH_CHECK();
  }
  if (H.cinv32) {
    k_cast<<<grid_for(nn), kBlock, 0, c->st>>>(nn, H.cdense, H.cinv32);
    RICH_LAUNCH_CHECK();
  }
  return RICH_OK;
}

// Finest-level stencil arrays from the 7n diffusion stencil; dinv = 1 / (l1 row norm)
// = 1 / (diag + sum of the six face weights).
__global__ void k_stencil4(long long n, const double* __restrict__ A7, Stencil4<double> s64, Stencil4<float> s32) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double a = A7[i], x = -A7[2 * n + i], y = -A7[4 * n + i], z = -A7[6 * n + i];
    double l1 = a + ((-A7[1 * n + i] + x) + (-A7[3 * n + i] + y) + (-A7[5 * n + i] + z));
    double r = 1.0 / l1;
    if (s64.diag) { s64.diag[i] = a; s64.wx[i] = x; s64.wy[i] = y; s64.wz[i] = z; s64.dinv[i] = r; }
    if (s32.diag) {
      s32.diag[i] = (float)a; s32.wx[i] = (float)x; s32.wy[i] = (float)y; s32.wz[i] = (float)z;
      s32.dinv[i] = (float)r;
    }
  }
}

// Finest-level stencil copy of the diffusion matrix for the V-cycle (FP64 or FP32).
static int fine_stencil(rich_ctx* c) {
  Hierarchy& H = c->H;
  long long n = c->g.n;
  bool mp = c->prec == RICH_PREC_MIXED;
  if (mp && !H.st32.diag) {
    RICH_CHECK(dalloc(&H.st32.diag, n));
    RICH_CHECK(dalloc(&H.st32.wx, n));
    RICH_CHECK(dalloc(&H.st32.wy, n));
    RICH_CHECK(dalloc(&H.st32.wz, n));
    RICH_CHECK(dalloc(&H.st32.dinv, n));
  }
  if (!mp && !H.st64.diag) {
    RICH_CHECK(dalloc(&H.st64.diag, n));
    RICH_CHECK(dalloc(&H.st64.wx, n));
    RICH_CHECK(dalloc(&H.st64.wy, n));
    RICH_CHECK(dalloc(&H.st64.wz, n));
    RICH_CHECK(dalloc(&H.st64.dinv, n));
  }
  k_stencil4<<<grid_for(n), kBlock, 0, c->st>>>(n, c->A7, H.st64, H.st32);
  RICH_LAUNCH_CHECK();
  return RICH_OK;
}

static int level_diag_data(rich_ctx* c, Level& L) {
  bool mp = c->prec == RICH_PREC_MIXED;
  k_l1dinv<<<grid_for(L.n), kBlock, 0, c->st>>>(L.n, L.A.rowptr, L.A.val, L.dinv, mp ? L.dinv32 : nullptr);
  RICH_LAUNCH_CHECK();
  if (mp) {
    k_cast<<<grid_for(L.A.nnz), kBlock, 0, c->st>>>(L.A.nnz, L.A.val, L.A32);
    RICH_LAUNCH_CHECK();
  }
  return RICH_OK;
}

// Values of level L's SELL copy of A (if the V-cycle has laid one out) from the
// values the V-cycle uses (FP32 in MIXED).
static int sell_fill_a(rich_ctx* c, Level& L) {
  if (c->prec == RICH_PREC_MIXED) return sell_fill(c, L.A, L.A32, L.sA);
  return sell_fill(c, L.A, L.A.val, L.sA);
}

static int level_alloc_vectors(rich_ctx* c, Level& L) {
  size_t es = c->prec == RICH_PREC_MIXED ? sizeof(float) : sizeof(double);
  long long n = L.n > 0 ? L.n : 1;
  void** vecs[4] = {&L.x, &L.b, &L.r, &L.t};
  for (void** v : vecs) {
    char* m = nullptr;
    RICH_CHECK(dalloc(&m, (long long)es * n));
    *v = m;
  }
  RICH_CHECK(dalloc(&L.dinv, n));
  if (c->prec == RICH_PREC_MIXED) {
    RICH_CHECK(dalloc(&L.dinv32, n));
    RICH_CHECK(dalloc(&L.A32, L.A.nnz));
  }
  return RICH_OK;
}

void amg_free(rich_ctx* c) {
  Hierarchy& H = c->H;
  for (int l = 0; l < (int)H.lv.size(); ++l) {
    Level& L = H.lv[l];
    if (l > 0) csr_free(L.A);
    csr_free(L.P);
    csr_free(L.R);
    csr_free(L.AP);
    dfree(L.A32);
    dfree(L.dinv);
    dfree(L.dinv32);
    dfree(L.agg);
    dfree(L.P32);
    dfree(L.R32);
    dfree(L.AP32);
    plist_free(L.pl_ap);
    plist_free(L.pl_rap);
    sell_free(L.sA);
    sell_free(L.sP);
    sell_free(L.sR);
    L.pl_tried = false;
    dfree(L.u_ap);
    dfree(L.u_rap);
    void** vecs[4] = {&L.x, &L.b, &L.r, &L.t};
    for (void** v : vecs) {
      char* m = static_cast<char*>(*v);
      dfree(m);
      *v = nullptr;
    }
  }
  H.lv.clear();
  H.nlev = 0;
  dfree(H.st64.diag); dfree(H.st64.wx); dfree(H.st64.wy); dfree(H.st64.wz); dfree(H.st64.dinv);
  dfree(H.st32.diag); dfree(H.st32.wx); dfree(H.st32.wy); dfree(H.st32.wz); dfree(H.st32.dinv);
  dfree(H.cdense);
  dfree(H.cinv32);
  dfree(H.cwork);
  if (H.gj_exec) cudaGraphExecDestroy(H.gj_exec);
  H.gj_exec = nullptr;
  H.gj_nodes = 0;
  if (H.vc_exec) cudaGraphExecDestroy(H.vc_exec);
  H.vc_exec = nullptr;
  H.vc_nodes = 0;
  H.vc_out = nullptr;
  H.vc_calls = 0;
  H.vc_off = false;
  for (int q = 0; q < 2; ++q) {
    if (H.fcg_exec[q]) cudaGraphExecDestroy(H.fcg_exec[q]);
    H.fcg_exec[q] = nullptr;
    H.fcg_nodes[q] = 0;
  }
  H.fcg_x = nullptr;
  H.fcg_off = false;
  as_free(c);
  H.built = false;
}


// Coarsen level L into a new level; returns RICH_OK with *stop = true when coarsening stops.
// Aggregates of at most max_size nodes by log2(max_size) matching passes on A
// (the first pass) and on the successive pair graphs P_p^T A P_p.  agg (n ints)
// receives the aggregate of every node, *nc their number, *rounds the matching
// rounds summed over the passes.
static int matching_aggregate(rich_ctx* c, const Csr<double>& A, int max_size, int* agg, int* nc, int* rounds) {
  int n = A.nrows;
  int passes = 0;
  while ((2 << passes) <= max_size) ++passes;
  k_iota<<<grid_for(n), kBlock, 0, c->st>>>(n, agg);
  RICH_LAUNCH_CHECK();
  *nc = n;
  *rounds = 0;
  Csr<double> Ak = A;  // the first pass reads A itself
  bool own = false;
  for (int pass = 0; pass < passes; ++pass) {
    int m = Ak.nrows;
    double* d = nullptr;
    float* w = nullptr;
    int *mate = nullptr, *cand = nullptr, *first = nullptr, *pos = nullptr, *ids = nullptr;
    RICH_CHECK(dalloc(&d, m));
    RICH_CHECK(dalloc(&w, Ak.nnz));
    RICH_CHECK(dalloc(&mate, m));
    RICH_CHECK(dalloc(&cand, m));
    RICH_CHECK(dalloc(&first, m));
    RICH_CHECK(dalloc(&pos, (long long)m + 1));
    RICH_CHECK(dalloc(&ids, m));
    k_diag<<<grid_for(m), kBlock, 0, c->st>>>(m, Ak.rowptr, Ak.col, Ak.val, d);
    RICH_LAUNCH_CHECK();
    k_match_weights<<<grid_for(m), kBlock, 0, c->st>>>(m, Ak.rowptr, Ak.col, Ak.val, d, w);
    RICH_LAUNCH_CHECK();
    RICH_CUDA(cudaMemsetAsync(mate, 0xff, sizeof(int) * (size_t)m, c->st));  // -1: unmatched
    for (;;) {
      RICH_CUDA(cudaMemsetAsync(c->iflag, 0, sizeof(int), c->st));
      k_match_propose<<<grid_for(m), kBlock, 0, c->st>>>(m, Ak.rowptr, Ak.col, w, mate, cand, c->iflag);
      RICH_LAUNCH_CHECK();
      int any = 0;
      RICH_CHECK(read_dev_int(c, c->iflag, &any));
      if (!any) break;
      k_match_commit<<<grid_for(m), kBlock, 0, c->st>>>(m, cand, mate);
      RICH_LAUNCH_CHECK();
      ++*rounds;
      if (*rounds > 1000000) return RICH_ELIMIT;  // every round matches the globally best free edge
    }
    k_pair_first<<<grid_for(m), kBlock, 0, c->st>>>(m, mate, first);
    RICH_LAUNCH_CHECK();
    RICH_CHECK(scan_exclusive_int(c, first, pos, m));
    int mc = 0;
    RICH_CHECK(read_dev_int(c, pos + m, &mc));
    k_pair_ids<<<grid_for(m), kBlock, 0, c->st>>>(m, mate, pos, ids);
    RICH_LAUNCH_CHECK();
    k_compose<<<grid_for(n), kBlock, 0, c->st>>>(n, ids, agg);
    RICH_LAUNCH_CHECK();
    *nc = mc;
    if (pass + 1 < passes) {  // the pair graph's matrix for the next pass
      Csr<double> Pp, Rp, AP, Ac;
      Pp.nrows = m;
      Pp.ncols = mc;
      Pp.nnz = m;
      RICH_CHECK(dalloc(&Pp.rowptr, (long long)m + 1));
      RICH_CHECK(dalloc(&Pp.col, m));
      RICH_CHECK(dalloc(&Pp.val, m));
      k_iota<<<grid_for((long long)m + 1), kBlock, 0, c->st>>>(m + 1, Pp.rowptr);
      RICH_LAUNCH_CHECK();
      RICH_CUDA(cudaMemcpyAsync(Pp.col, ids, sizeof(int) * (size_t)m, cudaMemcpyDeviceToDevice, c->st));
      k_fill<<<grid_for(m), kBlock, 0, c->st>>>(m, 1.0, Pp.val);
      RICH_LAUNCH_CHECK();
      RICH_CHECK(transpose(c, Pp, Rp));
      RICH_CHECK(spgemm_symbolic(c, Ak, Pp, AP));
      RICH_CHECK(spgemm_symbolic(c, Rp, AP, Ac));
      csr_free(Pp);
      csr_free(Rp);
      csr_free(AP);
      if (own) csr_free(Ak);
      Ak = Ac;
      own = true;
    }
    dfree(d);
    dfree(w);
    dfree(mate);
    dfree(cand);
    dfree(first);
    dfree(pos);
    dfree(ids);
  }
  if (own) csr_free(Ak);
  return RICH_OK;
}

static int coarsen(rich_ctx* c, int l, bool* stop) {
  Hierarchy& H = c->H;
  const rich_amg_opts& o = H.opts;
  Level& L = H.lv[l];
  int n = L.n;
  *stop = false;
  double* d = nullptr;
  int* cnt = nullptr;
  Csr<double> S;
  RICH_CHECK(dalloc(&d, n));
  RICH_CHECK(dalloc(&cnt, n));
  k_diag<<<grid_for(n), kBlock, 0, c->st>>>(n, L.A.rowptr, L.A.col, L.A.val, d);
  RICH_LAUNCH_CHECK();
  int rounds = 0;
  int nc = 0;
  int* aggid = nullptr;
  bool unassigned = false;
  if (o.aggregation == RICH_AGG_MATCHING) {
    RICH_CHECK(dalloc(&L.agg, n));
    RICH_CHECK(dalloc(&aggid, 1));
    RICH_CHECK(matching_aggregate(c, L.A, o.max_agg_size, L.agg, &nc, &rounds));
  } else {
    double theta_l = o.theta * std::ldexp(1.0, -l);
    double theta2 = theta_l * theta_l;
    k_strength<<<grid_for(n), kBlock, 0, c->st>>>(n, L.A.rowptr, L.A.col, L.A.val, d, theta2, nullptr, cnt, nullptr);
    RICH_LAUNCH_CHECK();
    RICH_CHECK(dalloc(&S.rowptr, (long long)n + 1));
    RICH_CHECK(scan_exclusive_int(c, cnt, S.rowptr, n));
    int snnz = 0;
    RICH_CHECK(read_dev_int(c, S.rowptr + n, &snnz));
    RICH_CHECK(dalloc(&S.col, snnz));
    k_strength<<<grid_for(n), kBlock, 0, c->st>>>(n, L.A.rowptr, L.A.col, L.A.val, d, theta2, S.rowptr, nullptr, S.col);
    RICH_LAUNCH_CHECK();
    // MIS-2
    uint64_t *t = nullptr, *m1 = nullptr;
    RICH_CHECK(dalloc(&t, n));
    RICH_CHECK(dalloc(&m1, n));
    k_mis_init<<<grid_for(n), kBlock, 0, c->st>>>(n, o.seed, S.rowptr, t);
    RICH_LAUNCH_CHECK();
    for (;;) {
      RICH_CUDA(cudaMemsetAsync(c->iflag, 0, sizeof(int), c->st));
      k_max_closed<<<grid_for(n), kBlock, 0, c->st>>>(n, S.rowptr, S.col, t, m1);
      RICH_LAUNCH_CHECK();
      k_mis_update<<<grid_for(n), kBlock, 0, c->st>>>(n, S.rowptr, S.col, m1, t, c->iflag);
      RICH_LAUNCH_CHECK();
      ++rounds;
      RICH_CUDA(cudaMemcpyAsync(c->hflag, c->iflag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
      RICH_CUDA(cudaStreamSynchronize(c->st));
      if (!c->hflag[0]) break;
      if (rounds > 100000) return RICH_ELIMIT;  // a round always decides the largest undecided key
    }
    // aggregates
    int* isroot = cnt;
    int* p1root = nullptr;
    uint64_t* rv = m1;
    uint64_t* best = nullptr;
    RICH_CHECK(dalloc(&aggid, (long long)n + 1));
    RICH_CHECK(dalloc(&p1root, n));
    RICH_CHECK(dalloc(&best, n));
    RICH_CHECK(dalloc(&L.agg, n));
    k_is_root<<<grid_for(n), kBlock, 0, c->st>>>(n, t, isroot);
    RICH_LAUNCH_CHECK();
    RICH_CHECK(scan_exclusive_int(c, isroot, aggid, n));
    RICH_CHECK(read_dev_int(c, aggid + n, &nc));
    k_rootval<<<grid_for(n), kBlock, 0, c->st>>>(n, t, rv);
    RICH_LAUNCH_CHECK();
    k_max_closed<<<grid_for(n), kBlock, 0, c->st>>>(n, S.rowptr, S.col, rv, best);
    RICH_LAUNCH_CHECK();
    k_agg_pass1<<<grid_for(n), kBlock, 0, c->st>>>(n, t, best, aggid, L.agg, p1root);
    RICH_LAUNCH_CHECK();
    k_val2<<<grid_for(n), kBlock, 0, c->st>>>(n, t, p1root, rv);
    RICH_LAUNCH_CHECK();
    k_max_closed<<<grid_for(n), kBlock, 0, c->st>>>(n, S.rowptr, S.col, rv, best);
    RICH_LAUNCH_CHECK();
    RICH_CUDA(cudaMemsetAsync(c->iflag, 0, sizeof(int), c->st));
    k_agg_pass2<<<grid_for(n), kBlock, 0, c->st>>>(n, S.rowptr, best, aggid, L.agg, c->iflag);
    RICH_LAUNCH_CHECK();
    RICH_CUDA(cudaMemcpyAsync(c->hflag, c->iflag, sizeof(int), cudaMemcpyDeviceToHost, c->st));
    RICH_CUDA(cudaStreamSynchronize(c->st));
    unassigned = c->hflag[0] != 0;
    if (!unassigned && o.isolated_join) {
      int* agg_in = p1root;  // pass-1 scratch, free now
      RICH_CUDA(cudaMemcpyAsync(agg_in, L.agg, sizeof(int) * (size_t)n, cudaMemcpyDeviceToDevice, c->st));
      k_agg_pass3<<<grid_for(n), kBlock, 0, c->st>>>(n, L.A.rowptr, L.A.col, L.A.val, o.seed, agg_in, L.agg);
      RICH_LAUNCH_CHECK();
    }
    dfree(t);
    dfree(m1);
    dfree(p1root);
    dfree(best);
    csr_free(S);
  }
  if (unassigned) {
    dfree(d);
    dfree(cnt);
    dfree(aggid);
    return RICH_ELIMIT;
  }
  L.mis_rounds = rounds;
  if (nc > 0.8 * n || nc < 1) {  // coarsening stalled: this level becomes the coarsest
    dfree(L.agg);
    dfree(d);
    dfree(cnt);
    dfree(aggid);
    *stop = true;
    return RICH_OK;
  }
  // prolongator: smoothed on the first smooth_levels levels, P_tent below
  Csr<double> Pt;
  Pt.nrows = n;
  Pt.ncols = nc;
  RICH_CHECK(dalloc(&Pt.rowptr, (long long)n + 1));
  k_ptent_count<<<grid_for(n), kBlock, 0, c->st>>>(n, L.agg, cnt);
  RICH_LAUNCH_CHECK();
  RICH_CHECK(scan_exclusive_int(c, cnt, Pt.rowptr, n));
  int ptnnz = 0;
  RICH_CHECK(read_dev_int(c, Pt.rowptr + n, &ptnnz));
  Pt.nnz = ptnnz;
  RICH_CHECK(dalloc(&Pt.col, ptnnz));
  k_ptent_fill<<<grid_for(n), kBlock, 0, c->st>>>(n, L.agg, Pt.rowptr, Pt.col);
  RICH_LAUNCH_CHECK();
  Pt.val = nullptr;
  if (l < o.smooth_levels) {
    int nb = red_grid(n);
    k_rowratio<<<nb, kBlock, 0, c->st>>>(n, L.A.rowptr, L.A.val, d, c->partials);
    RICH_LAUNCH_CHECK();
    RICH_CHECK(finish_max(c, c->partials, nb, c->dsc));
    double rho = 0.0;
    RICH_CHECK(fetch_scalars(c, c->dsc, 1, &rho));
    double omega = 4.0 / (3.0 * rho);
    L.omega = omega;
    Csr<double> Sm;
    Sm.nrows = Sm.ncols = n;
    Sm.nnz = L.A.nnz;
    Sm.rowptr = L.A.rowptr;
    Sm.col = L.A.col;
    RICH_CHECK(dalloc(&Sm.val, L.A.nnz));
    k_smoother_vals<<<grid_for(n), kBlock, 0, c->st>>>(n, L.A.rowptr, L.A.col, L.A.val, d, omega, Sm.val);
    RICH_LAUNCH_CHECK();
    RICH_CHECK(spgemm_symbolic(c, Sm, Pt, L.P));
    dfree(Sm.val);
  } else {
    // P = P_tent (pattern and unit values copied)
    L.omega = 0.0;
    L.P.nrows = n;
    L.P.ncols = nc;
    L.P.nnz = ptnnz;
    RICH_CHECK(dalloc(&L.P.rowptr, (long long)n + 1));
    RICH_CHECK(dalloc(&L.P.col, ptnnz));
    RICH_CHECK(dalloc(&L.P.val, ptnnz));
    RICH_CUDA(cudaMemcpyAsync(L.P.rowptr, Pt.rowptr, sizeof(int) * ((size_t)n + 1), cudaMemcpyDeviceToDevice, c->st));
    RICH_CUDA(cudaMemcpyAsync(L.P.col, Pt.col, sizeof(int) * (size_t)ptnnz, cudaMemcpyDeviceToDevice, c->st));
    k_fill<<<grid_for(ptnnz), kBlock, 0, c->st>>>(ptnnz, 1.0, L.P.val);
    RICH_LAUNCH_CHECK();
  }
  dfree(Pt.rowptr);
  dfree(Pt.col);
  RICH_CHECK(transpose(c, L.P, L.R));
  bool hashed_ap = false, hashed_rap = false;
  RICH_CHECK(spgemm_symbolic(c, L.A, L.P, L.AP, &L.u_ap, &hashed_ap));
  Level nxt;
  nxt.n = nc;
  RICH_CHECK(spgemm_symbolic(c, L.R, L.AP, nxt.A, &L.u_rap, &hashed_rap));
  if ((hashed_ap || hashed_rap) && o.product_lists) {
    // The next level's P is smoothed from these values and kept through every
    // refresh: sum them in the product lists' fixed order now (the lists the first
    // refresh would build), so that a setup does not depend on the order of atomics.
    L.pl_tried = true;
    RICH_CHECK(plist_build(c, L.A, L.P, L.AP, L.u_ap, L.pl_ap));
    if (L.pl_ap.seg) RICH_CHECK(plist_build(c, L.R, L.AP, nxt.A, L.u_rap, L.pl_rap));
    if (L.pl_ap.seg && L.pl_rap.seg) {
      RICH_CHECK(spgemm_numeric(c, L.A, L.P, L.AP, L.u_ap, 0, l, &L.pl_ap));
      RICH_CHECK(spgemm_numeric(c, L.R, L.AP, nxt.A, L.u_rap, 1, l, &L.pl_rap));
    }
  }
  if (c->prec == RICH_PREC_MIXED) {
    RICH_CHECK(dalloc(&L.P32, L.P.nnz));
    RICH_CHECK(dalloc(&L.R32, L.R.nnz));
    RICH_CHECK(dalloc(&L.AP32, L.AP.nnz));
    k_cast<<<grid_for(L.P.nnz), kBlock, 0, c->st>>>(L.P.nnz, L.P.val, L.P32);
    RICH_LAUNCH_CHECK();
    k_cast<<<grid_for(L.R.nnz), kBlock, 0, c->st>>>(L.R.nnz, L.R.val, L.R32);
    RICH_LAUNCH_CHECK();
  }
  dfree(d);
  dfree(cnt);
  dfree(aggid);
  H.lv.push_back(nxt);
  return RICH_OK;
}

int amg_build(rich_ctx* c, const rich_amg_opts* o) {
  if (!c->have_jac) return RICH_ESTATE;
  amg_free(c);
  Hierarchy& H = c->H;
  if (o) H.opts = *o; else rich_default_amg_opts(&H.opts);
  if (H.opts.max_levels < 1 || H.opts.max_levels > 16 || H.opts.nu1 < 0 || H.opts.nu2 < 0 || H.opts.coarse_max < 1)
    return RICH_EINVAL;
  if (H.opts.aggregation != RICH_AGG_MIS2 && H.opts.aggregation != RICH_AGG_MATCHING) return RICH_EINVAL;
  if (H.opts.smoother != RICH_SMOOTH_L1JACOBI && H.opts.smoother != RICH_SMOOTH_HYBRID_GS) return RICH_EINVAL;
  if (H.opts.smoother == RICH_SMOOTH_HYBRID_GS && (H.opts.hgs_seg < 1 || H.opts.hgs_block < 1 ||
                                                  H.opts.hgs_block > 4096))
    return RICH_EINVAL;
  if (H.opts.aggregation == RICH_AGG_MATCHING && (H.opts.max_agg_size < 2 || H.opts.max_agg_size > 1024))
    return RICH_EINVAL;
  if (H.opts.precond != RICH_PRECOND_AMG && H.opts.precond != RICH_PRECOND_AS) return RICH_EINVAL;
  if (H.opts.csr_layout < RICH_LAYOUT_AUTO || H.opts.csr_layout > RICH_LAYOUT_SELLP) return RICH_EINVAL;
  if (H.opts.graph != 0 && H.opts.graph != 1) return RICH_EINVAL;
  if (H.opts.precond == RICH_PRECOND_AS) {  // one level: the subdomain factors of A_aux
    RICH_CHECK(fine_stencil(c));
    RICH_CHECK(as_setup(c));
    H.built = true;
    return RICH_OK;
  }
  RICH_CHECK(refresh_a0_values(c));
  Level L0;
  L0.n = (int)c->g.n;
  L0.A = c->A0;  // aliases the context's finest CSR
  H.lv.push_back(L0);
  for (;;) {
    int l = (int)H.lv.size() - 1;
    if (H.lv[l].n < H.opts.coarse_max || (int)H.lv.size() >= H.opts.max_levels) break;
    bool stop = false;
    RICH_CHECK(coarsen(c, l, &stop));
    if (stop) break;
  }
  H.nlev = (int)H.lv.size();
  H.cn = H.lv[H.nlev - 1].n;
  // coarsening stalled above the dense limit: the coarsest level is smoothed
  H.dense = H.cn <= kMaxCoarseDense;
  for (int l = 0; l < H.nlev; ++l) {
    RICH_CHECK(level_alloc_vectors(c, H.lv[l]));
    RICH_CHECK(level_diag_data(c, H.lv[l]));
  }
  RICH_CHECK(fine_stencil(c));
  if (H.dense) {
    RICH_CHECK(dalloc(&H.cdense, (long long)H.cn * H.cn));
    RICH_CHECK(dalloc(&H.cwork, 2LL * kGjB * H.cn + kGjB * kGjB));
    if (c->prec == RICH_PREC_MIXED) RICH_CHECK(dalloc(&H.cinv32, (long long)H.cn * H.cn));
    RICH_CHECK(coarse_inverse(c));
    RICH_CHECK(capture_coarse_graph(c));
  }
  RICH_CUDA(cudaStreamSynchronize(c->st));
  H.built = true;
  return RICH_OK;
}

// New finest matrix: recompute every Galerkin product on the kept patterns.
int amg_refresh(rich_ctx* c) {
  Hierarchy& H = c->H;
  if (!H.built) return RICH_ESTATE;
  if (H.opts.precond == RICH_PRECOND_AS) {
    RICH_CHECK(fine_stencil(c));
    return as_setup(c);
  }
  RICH_CHECK(refresh_a0_values(c));
  H.lv[0].A = c->A0;
  for (int l = 0; l + 1 < H.nlev; ++l) {
    Level& L = H.lv[l];
    if (L.pl_tried || !H.opts.product_lists) continue;
    L.pl_tried = true;
    RICH_CHECK(plist_build(c, L.A, L.P, L.AP, L.u_ap, L.pl_ap));
    if (L.pl_ap.seg) RICH_CHECK(plist_build(c, L.R, L.AP, H.lv[l + 1].A, L.u_rap, L.pl_rap));
  }
  if (c->prec == RICH_PREC_MIXED) {
    // The V-cycle runs in FP32, so the Galerkin products do too: A32_{l+1} =
    // R32 (A32_l P32), on the patterns kept from the setup.  The FP64 values of
    // the coarse levels keep their setup-time content and are not read again.
    RICH_CHECK(level_diag_data(c, H.lv[0]));
    for (int l = 0; l + 1 < H.nlev; ++l) {
      Level& L = H.lv[l];
      Level& N = H.lv[l + 1];
      RICH_CHECK(spgemm_numeric_t<float>(c, L.A, L.A32, L.P, L.P32, L.AP, L.AP32, L.u_ap, 0, l, &L.pl_ap));
      RICH_CHECK(spgemm_numeric_t<float>(c, L.R, L.R32, L.AP, L.AP32, N.A, N.A32, L.u_rap, 1, l, &L.pl_rap));
      k_l1dinv32<<<grid_for(N.n), kBlock, 0, c->st>>>(N.n, N.A.rowptr, N.A32, N.dinv32);
      RICH_LAUNCH_CHECK();
    }
  } else {
    for (int l = 0; l + 1 < H.nlev; ++l) {
      Level& L = H.lv[l];
      RICH_CHECK(spgemm_numeric(c, L.A, L.P, L.AP, L.u_ap, 0, l, &L.pl_ap));
      RICH_CHECK(spgemm_numeric(c, L.R, L.AP, H.lv[l + 1].A, L.u_rap, 1, l, &L.pl_rap));
    }
    for (int l = 0; l < H.nlev; ++l) RICH_CHECK(level_diag_data(c, H.lv[l]));
  }
  for (int l = 1; l < H.nlev; ++l) RICH_CHECK(sell_fill_a(c, H.lv[l]));
  RICH_CHECK(fine_stencil(c));
  return coarse_inverse(c);
}

// The paper's reuse: only the finest matrix and its smoother change.
int amg_update_fine(rich_ctx* c) {
  Hierarchy& H = c->H;
  if (!H.built) return RICH_ESTATE;
  if (H.opts.precond == RICH_PRECOND_AS) {
    RICH_CHECK(fine_stencil(c));
    return as_setup(c);
  }
  RICH_CHECK(refresh_a0_values(c));
  H.lv[0].A = c->A0;
  RICH_CHECK(level_diag_data(c, H.lv[0]));
  RICH_CHECK(fine_stencil(c));
  if (H.nlev == 1) return coarse_inverse(c);
  return RICH_OK;
}

}  // namespace rich

using namespace rich;

extern "C" {

int amg_setup(rich_ctx* c, const rich_amg_opts* o, rich_amg_info* info) {
  if (!c) return RICH_EINVAL;
  AllocStream guard(c->st);
  RICH_CHECK(amg_build(c, o));
  if (info) {
    Hierarchy& H = c->H;
    memset(info, 0, sizeof(*info));
    if (H.opts.precond == RICH_PRECOND_AS || H.nlev == 0) return RICH_OK;  // no hierarchy: all zero
    info->levels = H.nlev;
    long long tot = 0;
    for (int l = 0; l < H.nlev && l < 16; ++l) {
      info->n[l] = H.lv[l].n;
      info->nnz[l] = H.lv[l].A.nnz;
      info->mis_rounds[l] = H.lv[l].mis_rounds;
      info->omega[l] = H.lv[l].omega;
      tot += H.lv[l].A.nnz;
    }
    info->operator_complexity = (double)tot / (double)H.lv[0].A.nnz;
  }
  return RICH_OK;
}

int amg_update(rich_ctx* c, int policy) {
  if (!c) return RICH_EINVAL;
  AllocStream guard(c->st);
  if (policy == RICH_AMG_SETUP_ONCE) return amg_update_fine(c);
  if (policy == RICH_AMG_REFRESH) return amg_refresh(c);
  return RICH_EINVAL;
}

int amg_export_level(rich_ctx* c, int level, int* agg, int* rp, int* col, double* val) {
  if (!c) return RICH_EINVAL;
  AllocStream guard(c->st);
  Hierarchy& H = c->H;
  if (!H.built) return RICH_ESTATE;
  if (level < 0 || level >= H.nlev) return RICH_EINVAL;
  Level& L = H.lv[level];
  RICH_CUDA(cudaStreamSynchronize(c->st));
  if (agg) {
    if (!L.agg) return RICH_EINVAL;
    RICH_CUDA(cudaMemcpy(agg, L.agg, sizeof(int) * L.n, cudaMemcpyDeviceToHost));
  }
  if (rp) RICH_CUDA(cudaMemcpy(rp, L.A.rowptr, sizeof(int) * (L.n + 1), cudaMemcpyDeviceToHost));
  if (col) RICH_CUDA(cudaMemcpy(col, L.A.col, sizeof(int) * L.A.nnz, cudaMemcpyDeviceToHost));
  if (val) {
    if (c->prec == RICH_PREC_MIXED && level > 0) {
      // the FP32 values the V-cycle uses (refreshed in FP32), widened
      std::vector<float> v32((size_t)L.A.nnz);
      RICH_CUDA(cudaMemcpy(v32.data(), L.A32, sizeof(float) * L.A.nnz, cudaMemcpyDeviceToHost));
      for (long long e = 0; e < L.A.nnz; ++e) val[e] = (double)v32[(size_t)e];
    } else {
      RICH_CUDA(cudaMemcpy(val, L.A.val, sizeof(double) * L.A.nnz, cudaMemcpyDeviceToHost));
    }
  }
  return RICH_OK;
}

int amg_export_prolongator(rich_ctx* c, int level, long long* nnz, int* rp, int* col, double* val) {
  if (!c) return RICH_EINVAL;
  AllocStream guard(c->st);
  Hierarchy& H = c->H;
  if (!H.built) return RICH_ESTATE;
  if (level < 0 || level + 1 >= H.nlev) return RICH_EINVAL;
  Level& L = H.lv[level];
  RICH_CUDA(cudaStreamSynchronize(c->st));
  if (nnz) *nnz = L.P.nnz;
  if (rp) RICH_CUDA(cudaMemcpy(rp, L.P.rowptr, sizeof(int) * (L.n + 1), cudaMemcpyDeviceToHost));
  if (col) RICH_CUDA(cudaMemcpy(col, L.P.col, sizeof(int) * L.P.nnz, cudaMemcpyDeviceToHost));
  if (val) RICH_CUDA(cudaMemcpy(val, L.P.val, sizeof(double) * L.P.nnz, cudaMemcpyDeviceToHost));
  return RICH_OK;
}

}  // extern "C"
