// V-cycle (eq. (Vcycle), Sec. 5.2), flexible Krylov solvers for the right-
// preconditioned Newton system (eq. (precsystem), Sec. 3) and the inexact
// Newton-Armijo backward-Euler step (Sec. 3).
//
// V-cycle on level l with zero initial guess: nu1 l1-Jacobi sweeps
// x <- x + D_l1^-1 (b - A x), residual r = b - A x, b_{l+1} = R r, recursion
// (the coarsest level multiplies by its dense inverse), x <- x + P x_{l+1},
// nu2 sweeps.  In MIXED precision every level works in FP32 with FP32
// accumulation; the Krylov vectors and dot products stay FP64.
//
// Krylov scalars live in device memory; each iteration reads one small block
// of them back for the convergence test.
#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <vector>

#include "common.cuh"

namespace rich {

// ---------------------------------------------------------------- V-cycle kernels (T = double | float)

template <class T>
__global__ void k_jacobi0(int n, const T* __restrict__ dinv, const T* __restrict__ b, T* __restrict__ x) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) x[i] = dinv[i] * b[i];
}

template <class T>
__global__ void k_jacobi(int n, const int* __restrict__ rp, const int* __restrict__ col, const T* __restrict__ val,
                         const T* __restrict__ dinv, const T* __restrict__ b, const T* __restrict__ x,
                         T* __restrict__ xo) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    T s = b[i];
    for (int e = rp[i]; e < rp[i + 1]; ++e) s -= val[e] * x[col[e]];
    xo[i] = x[i] + dinv[i] * s;
  }
}

template <class T>
__global__ void k_resid(int n, const int* __restrict__ rp, const int* __restrict__ col, const T* __restrict__ val,
                        const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ r) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    T s = b[i];
    for (int e = rp[i]; e < rp[i + 1]; ++e) s -= val[e] * x[col[e]];
    r[i] = s;
  }
}

template <class T>
__global__ void k_spmv(int n, const int* __restrict__ rp, const int* __restrict__ col, const T* __restrict__ val,
                       const T* __restrict__ x, T* __restrict__ y, int add) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    T s = add ? y[i] : T(0);
    for (int e = rp[i]; e < rp[i + 1]; ++e) s += val[e] * x[col[e]];
    y[i] = s;
  }
}

// CSR row operation with G lanes per row (G = 4..32), for levels whose rows are
// long (coarse Galerkin operators carry tens to hundreds of entries per row).
// MODE 0: y = A x; 1: y += A x; 2: y = x + dinv (b - A x); 3: y = b - A x.
// U = 4: each lane keeps four partial sums over entries e, e+G, e+2G, e+3G, so four
// independent gathers of x are in flight (the coarse levels are gather-latency bound).
template <class T, int MODE, int G, int U = 1>
__global__ void k_csr_grp(int n, const int* __restrict__ rp, const int* __restrict__ col, const T* __restrict__ val,
                          const T* __restrict__ dinv, const T* __restrict__ b, const T* __restrict__ x,
                          T* __restrict__ y) {
  int lane = threadIdx.x & (G - 1);
  unsigned mask = G == 32 ? 0xffffffffu : (((1u << G) - 1) << ((threadIdx.x & 31) & ~(G - 1)));
  int rows_per_grid = (gridDim.x * blockDim.x) / G;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) / G; row < n; row += rows_per_grid) {
    T s = 0;
    int e = rp[row] + lane;
    const int end = rp[row + 1];
    if (U == 4) {
      T s1 = 0, s2 = 0, s3 = 0;
      for (; e + 3 * G < end; e += 4 * G) {
        const int c0 = col[e], c1 = col[e + G], c2 = col[e + 2 * G], c3 = col[e + 3 * G];
        const T v0 = val[e], v1 = val[e + G], v2 = val[e + 2 * G], v3 = val[e + 3 * G];
        s += v0 * x[c0];
        s1 += v1 * x[c1];
        s2 += v2 * x[c2];
        s3 += v3 * x[c3];
      }
      s = (s + s1) + (s2 + s3);
    }
    for (; e < end; e += G) s += val[e] * x[col[e]];
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) s += __shfl_down_sync(mask, s, o, G);
    if (lane == 0) {
      if (MODE == 0) y[row] = s;
      else if (MODE == 1) y[row] += s;
      else if (MODE == 2) y[row] = x[row] + dinv[row] * (b[row] - s);
      else y[row] = b[row] - s;
    }
  }
}

// The same row operations on the SELL-C-sigma copy: one warp per slice of 32 rows,
// one thread per row, slot loads coalesced across the warp, U gathers of x in flight
// per thread (U = 4 or 8), no cross-lane reduction (on GB300's narrow FP64 pipe the
// shuffle-add reductions and the idle lanes of ragged rows cost as much as the
// products themselves).  Past a row's end the slots hold zeros.
template <class T, int MODE, int U>
__global__ void __launch_bounds__(kBlock) k_sell(int nslice, const int* __restrict__ sptr,
                                                 const int* __restrict__ perm, const int* __restrict__ col,
                                                 const T* __restrict__ val, const T* __restrict__ dinv,
                                                 const T* __restrict__ b, const T* __restrict__ x,
                                                 T* __restrict__ y) {
  const int lane = threadIdx.x & (kSellC - 1);
  const int warps = (gridDim.x * blockDim.x) / kSellC;
  for (int s = (blockIdx.x * blockDim.x + threadIdx.x) / kSellC; s < nslice; s += warps) {
    const int row = perm[s * kSellC + lane];
    const int end = sptr[s + 1];
    int e = sptr[s] + lane;
    T s0 = 0, s1 = 0;
    for (; e + (U - 1) * kSellC < end; e += U * kSellC) {  // warp-uniform: the slice's columns are full
      int cc[U];
      T vv[U], xx[U];
#pragma unroll
      for (int u = 0; u < U; ++u) cc[u] = col[e + u * kSellC];
#pragma unroll
      for (int u = 0; u < U; ++u) vv[u] = val[e + u * kSellC];
#pragma unroll
      for (int u = 0; u < U; ++u) xx[u] = x[cc[u]];
#pragma unroll
      for (int u = 0; u < U; u += 2) {
        s0 += vv[u] * xx[u];
        s1 += vv[u + 1] * xx[u + 1];
      }
    }
    for (; e < end; e += kSellC) s0 += val[e] * x[col[e]];
    const T a = s0 + s1;
    if (row >= 0) {
      if (MODE == 0) y[row] = a;
      else if (MODE == 1) y[row] += a;
      else if (MODE == 2) y[row] = x[row] + dinv[row] * (b[row] - a);
      else y[row] = b[row] - a;
    }
  }
}

// SELL, software-pipelined: while the gathers of x for four columns and their
// products run, the slot loads (column and value) of the next four are already in
// flight, so the DRAM latency of the copy overlaps the L2 latency of the gathers
// instead of adding to it.
template <class T, int MODE>
__global__ void __launch_bounds__(kBlock) k_sellp(int nslice, const int* __restrict__ sptr,
                                                  const int* __restrict__ perm, const int* __restrict__ col,
                                                  const T* __restrict__ val, const T* __restrict__ dinv,
                                                  const T* __restrict__ b, const T* __restrict__ x,
                                                  T* __restrict__ y) {
  const int lane = threadIdx.x & (kSellC - 1);
  const int warps = (gridDim.x * blockDim.x) / kSellC;
  for (int s = (blockIdx.x * blockDim.x + threadIdx.x) / kSellC; s < nslice; s += warps) {
    const int row = perm[s * kSellC + lane];
    const int end = sptr[s + 1];
    int e = sptr[s] + lane;
    T s0 = 0, s1 = 0;
    bool have = e + 3 * kSellC < end;  // warp-uniform, as every test below
    int c0 = 0, c1 = 0, c2 = 0, c3 = 0;
    T v0 = 0, v1 = 0, v2 = 0, v3 = 0;
    if (have) {
      c0 = col[e];
      c1 = col[e + kSellC];
      c2 = col[e + 2 * kSellC];
      c3 = col[e + 3 * kSellC];
      v0 = val[e];
      v1 = val[e + kSellC];
      v2 = val[e + 2 * kSellC];
      v3 = val[e + 3 * kSellC];
    }
    while (have) {
      const int en = e + 4 * kSellC;
      const bool next = en + 3 * kSellC < end;
      int d0 = 0, d1 = 0, d2 = 0, d3 = 0;
      T w0 = 0, w1 = 0, w2 = 0, w3 = 0;
      if (next) {
        d0 = col[en];
        d1 = col[en + kSellC];
        d2 = col[en + 2 * kSellC];
        d3 = col[en + 3 * kSellC];
        w0 = val[en];
        w1 = val[en + kSellC];
        w2 = val[en + 2 * kSellC];
        w3 = val[en + 3 * kSellC];
      }
      const T x0 = x[c0], x1 = x[c1], x2 = x[c2], x3 = x[c3];
      s0 += v0 * x0;
      s1 += v1 * x1;
      s0 += v2 * x2;
      s1 += v3 * x3;
      c0 = d0;
      c1 = d1;
      c2 = d2;
      c3 = d3;
      v0 = w0;
      v1 = w1;
      v2 = w2;
      v3 = w3;
      e = en;
      have = next;
    }
    for (; e < end; e += kSellC) s0 += val[e] * x[col[e]];
    const T a = s0 + s1;
    if (row >= 0) {
      if (MODE == 0) y[row] = a;
      else if (MODE == 1) y[row] += a;
      else if (MODE == 2) y[row] = x[row] + dinv[row] * (b[row] - a);
      else y[row] = b[row] - a;
    }
  }
}

// SELL with two lanes per row: one warp per half-slice (16 rows); lane t + 16 ph
// takes the row's columns j = ph, ph + 2, ... (each load instruction reads two
// contiguous 128-byte runs), and one shuffle-add joins the two partial sums.  Twice
// the warps of k_sell for the same slices: more loads in flight on levels whose
// slices alone fill only part of the GPU.
template <class T, int MODE>
__global__ void __launch_bounds__(kBlock) k_sell2(int nslice, const int* __restrict__ sptr,
                                                  const int* __restrict__ perm, const int* __restrict__ col,
                                                  const T* __restrict__ val, const T* __restrict__ dinv,
                                                  const T* __restrict__ b, const T* __restrict__ x,
                                                  T* __restrict__ y) {
  const int lane = threadIdx.x & 31, ph = lane >> 4;
  const int warps = (gridDim.x * blockDim.x) / 32;
  for (int hs = (blockIdx.x * blockDim.x + threadIdx.x) / 32; hs < 2 * nslice; hs += warps) {
    const int s = hs >> 1, r = (hs & 1) * 16 + (lane & 15);
    const int row = perm[s * kSellC + r];
    const int base = sptr[s] + r, w = (sptr[s + 1] - sptr[s]) / kSellC;
    T s0 = 0, s1 = 0;
    int j = ph;
    for (; j + 6 < w; j += 8) {  // columns j, j + 2, j + 4, j + 6 of this lane
      const int c0 = col[base + j * kSellC], c1 = col[base + (j + 2) * kSellC];
      const int c2 = col[base + (j + 4) * kSellC], c3 = col[base + (j + 6) * kSellC];
      const T v0 = val[base + j * kSellC], v1 = val[base + (j + 2) * kSellC];
      const T v2 = val[base + (j + 4) * kSellC], v3 = val[base + (j + 6) * kSellC];
      const T x0 = x[c0], x1 = x[c1], x2 = x[c2], x3 = x[c3];
      s0 += v0 * x0;
      s1 += v1 * x1;
      s0 += v2 * x2;
      s1 += v3 * x3;
    }
    for (; j < w; j += 2) s0 += val[base + j * kSellC] * x[col[base + j * kSellC]];
    T a = s0 + s1;
    a += __shfl_xor_sync(0xffffffffu, a, 16);
    if (ph == 0 && row >= 0) {
      if (MODE == 0) y[row] = a;
      else if (MODE == 1) y[row] += a;
      else if (MODE == 2) y[row] = x[row] + dinv[row] * (b[row] - a);
      else y[row] = b[row] - a;
    }
  }
}

// Variant v of the CSR row kernel: lanes per row G = v & 0xff, four-way unrolled
// rows when v & kUnroll; v == kSellVariant (4 gathers in flight per thread),
// kSellVariant8 (8), kSellVariant2 (two lanes per row) or kSellVariantP
// (software-pipelined) runs the SELL copy (sl, sval) instead.
constexpr int kUnroll = 0x100;
constexpr int kSellVariant = 0x200;
constexpr int kSellVariant8 = 0x201;
constexpr int kSellVariant2 = 0x202;
constexpr int kSellVariantP = 0x203;
inline bool is_sell(int v) { return (v & kSellVariant) != 0; }
template <class T, int MODE>
static void csr_launch(cudaStream_t st, int v, int n, const int* rp, const int* col, const T* val, const T* dinv,
                       const T* b, const T* x, T* y, const Sell* sl = nullptr, const T* sval = nullptr) {
  if (is_sell(v)) {
    const int g = grid_for((long long)sl->nslice * kSellC);
    if (v == kSellVariant8)
      k_sell<T, MODE, 8><<<g, kBlock, 0, st>>>(sl->nslice, sl->sptr, sl->perm, sl->col, sval, dinv, b, x, y);
    else if (v == kSellVariant2)
      k_sell2<T, MODE><<<grid_for(2LL * sl->nslice * kSellC), kBlock, 0, st>>>(sl->nslice, sl->sptr, sl->perm,
                                                                               sl->col, sval, dinv, b, x, y);
    else if (v == kSellVariantP)
      k_sellp<T, MODE><<<g, kBlock, 0, st>>>(sl->nslice, sl->sptr, sl->perm, sl->col, sval, dinv, b, x, y);
    else
      k_sell<T, MODE, 4><<<g, kBlock, 0, st>>>(sl->nslice, sl->sptr, sl->perm, sl->col, sval, dinv, b, x, y);
    return;
  }
  const int G = v & 0xff;
  long long thr = (long long)n * G;
  const dim3 gr(grid_for(thr));
  if (v & kUnroll) {
    switch (G) {
      case 1: k_csr_grp<T, MODE, 1, 4><<<gr, kBlock, 0, st>>>(n, rp, col, val, dinv, b, x, y); break;
      case 2: k_csr_grp<T, MODE, 2, 4><<<gr, kBlock, 0, st>>>(n, rp, col, val, dinv, b, x, y); break;
      case 4: k_csr_grp<T, MODE, 4, 4><<<gr, kBlock, 0, st>>>(n, rp, col, val, dinv, b, x, y); break;
      default: k_csr_grp<T, MODE, 8, 4><<<gr, kBlock, 0, st>>>(n, rp, col, val, dinv, b, x, y); break;
    }
    return;
  }
  switch (G) {
    case 1: k_csr_grp<T, MODE, 1><<<gr, kBlock, 0, st>>>(n, rp, col, val, dinv, b, x, y); break;
    case 2: k_csr_grp<T, MODE, 2><<<gr, kBlock, 0, st>>>(n, rp, col, val, dinv, b, x, y); break;
    case 4: k_csr_grp<T, MODE, 4><<<gr, kBlock, 0, st>>>(n, rp, col, val, dinv, b, x, y); break;
    case 8: k_csr_grp<T, MODE, 8><<<gr, kBlock, 0, st>>>(n, rp, col, val, dinv, b, x, y); break;
    case 16: k_csr_grp<T, MODE, 16><<<gr, kBlock, 0, st>>>(n, rp, col, val, dinv, b, x, y); break;
    default: k_csr_grp<T, MODE, 32><<<gr, kBlock, 0, st>>>(n, rp, col, val, dinv, b, x, y); break;
  }
}

// Lanes per row when nothing has been measured: one thread per short row, wider
// groups as rows grow.
static int default_lanes(double avg) {
  if (avg <= 6) return 1;
  if (avg > 96) return 32;
  if (avg > 64) return 16;
  if (avg > 40) return 8;
  return 4;
}

// Autotuner of the CSR row operations: the first time an operation meets a shape
// class (mode, value type, rows in quarter-octave bins, mean row length rounded to
// an integer), every candidate is timed on the actual operands (output to a scratch
// vector, one warm-up and three timed launches each, CUDA events) and the fastest
// is kept for the rest of the process.  Classes, not exact shapes, so that
// a stream of requests of similar size (whose coarse levels differ by a few rows)
// tunes once.  The table is shared by all contexts (under a mutex, held while
// tuning, so concurrent requests of one class agree); a class therefore always runs
// the same kernel, and results do not depend on what else is in flight.
struct TuneKey {
  int mode, tsize, n;   // n: quarter-octave bin of the row count
  long long nnz;        // rounded mean row length
  int sell;             // 1: a SELL copy is among the candidates
  bool operator<(const TuneKey& o) const {
    if (mode != o.mode) return mode < o.mode;
    if (tsize != o.tsize) return tsize < o.tsize;
    if (n != o.n) return n < o.n;
    if (nnz != o.nnz) return nnz < o.nnz;
    return sell < o.sell;
  }
};
struct TuneVal {
  int variant;   // fastest candidate
  float us;      // its time per launch
  int best_csr;  // fastest CSR candidate (used where a matrix of the class has no SELL copy)
};
static std::mutex g_tune_mu;
static std::map<TuneKey, TuneVal> g_tune;

// Where a row operation's matrix can get a SELL copy: the copy, the CSR it is laid
// out from and the values in the hierarchy precision.
template <class T>
struct SellSrc {
  Sell* s;
  const Csr<double>* M;
  const T* vals;
};

// Lays out the SELL copy on first use (the row operations of a class that chose it,
// or a class being tuned): matrices whose class keeps CSR never get one.
template <class T>
static int sell_ensure(rich_ctx* c, const SellSrc<T>& src, bool* ok) {
  if (!src.s->built()) {
    RICH_CHECK(sell_build(c, *src.M, *src.s));
    if (src.s->built()) RICH_CHECK(sell_fill(c, *src.M, src.vals, *src.s));
    prof_restart(c->st);
  }
  *ok = src.s->built();
  return RICH_OK;
}

// src: the matrix's SELL source (nullptr: CSR only).
template <class T, int MODE>
static int csr_op(rich_ctx* c, int n, long long nnz, const int* rp, const int* col, const T* val, const T* dinv,
                  const T* b, const T* x, T* y, const SellSrc<T>* src = nullptr) {
  if (n <= 0) return RICH_OK;
  const int layout = c->H.opts.csr_layout;
  const bool offer = src && src->s && n >= kSellMinRows && layout != RICH_LAYOUT_CSR;
  int v = default_lanes((double)nnz / n);
  bool sell_ok = false;
  if (offer && layout >= RICH_LAYOUT_SELL) {  // a SELL kernel named by the option
    RICH_CHECK(sell_ensure(c, *src, &sell_ok));
    if (sell_ok)
      v = layout == RICH_LAYOUT_SELL8   ? kSellVariant8
          : layout == RICH_LAYOUT_SELL2 ? kSellVariant2
          : layout == RICH_LAYOUT_SELLP ? kSellVariantP
                                        : kSellVariant;
  } else if (c->H.opts.autotune) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    TuneKey key{MODE, (int)sizeof(T), (int)std::floor(4.0 * std::log2((double)n)),
                (long long)std::llround((double)nnz / n), offer ? 1 : 0};
    auto it = g_tune.find(key);
    if (it != g_tune.end()) {
      v = it->second.variant;
      if (is_sell(v)) {
        RICH_CHECK(sell_ensure(c, *src, &sell_ok));
        if (!sell_ok) v = it->second.best_csr;
      }
    } else if (!profiling_active()) {  // a profiled pass runs what is tuned, and tunes nothing
      const bool had_copy = offer && src->s->built();
      if (offer) RICH_CHECK(sell_ensure(c, *src, &sell_ok));
      T* scratch = nullptr;
      RICH_CHECK(dalloc(&scratch, n));
      RICH_CUDA(cudaMemsetAsync(scratch, 0, sizeof(T) * (size_t)n, c->st));
      // Back-to-back launches on warm operands.  Timing each launch from a cold L2
      // (a 256 MB write before it) was measured and chose worse variants: the same
      // headline, 3 % less in the mixed mode, whose FP32 levels stay in L2 between
      // the sweeps of a V-cycle.
      cudaEvent_t e0, e1;
      RICH_CUDA(cudaEventCreate(&e0));
      RICH_CUDA(cudaEventCreate(&e1));
      float best = 1e30f, best_csr_us = 1e30f;
      int best_csr = v;
      const Sell* sl = sell_ok ? src->s : nullptr;
      const T* sval = sell_ok ? (sizeof(T) == 8 ? (const T*)sl->val : (const T*)sl->val32) : nullptr;
      for (int g : {1, 2, 4, 8, 16, 32, 1 | kUnroll, 2 | kUnroll, 4 | kUnroll, 8 | kUnroll, kSellVariant,
                    kSellVariant8, kSellVariant2, kSellVariantP}) {
        if (is_sell(g) && !sell_ok) continue;
        csr_launch<T, MODE>(c->st, g, n, rp, col, val, dinv, b, x, scratch, sl, sval);
        RICH_CUDA(cudaEventRecord(e0, c->st));
        for (int rep = 0; rep < 3; ++rep) csr_launch<T, MODE>(c->st, g, n, rp, col, val, dinv, b, x, scratch, sl, sval);
        RICH_CUDA(cudaEventRecord(e1, c->st));
        RICH_CUDA(cudaEventSynchronize(e1));
        float ms = 0.f;
        RICH_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        count_launches(4);
        if (ms < best) {
          best = ms;
          v = g;
        }
        if (!is_sell(g) && ms < best_csr_us) {
          best_csr_us = ms;
          best_csr = g;
        }
      }
      RICH_CUDA(cudaGetLastError());
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      dfree(scratch);
      g_tune[key] = {v, best * 1000.f / 3.f, best_csr};
      if (sell_ok && !is_sell(v) && !had_copy) {  // the copy lost: not kept, not refreshed
        sell_free(*src->s);
        sell_ok = false;
      }
    }
  }
  const Sell* sl = nullptr;
  const T* sval = nullptr;
  if (is_sell(v)) {
    sl = src->s;
    sval = sizeof(T) == 8 ? (const T*)sl->val : (const T*)sl->val32;
  }
  csr_launch<T, MODE>(c->st, v, n, rp, col, val, dinv, b, x, y, sl, sval);
  return RICH_OK;
}

int autotune_table(char* buf, int cap) {
  std::lock_guard<std::mutex> lk(g_tune_mu);
  int off = 0;
  buf[0] = 0;
  for (auto& e : g_tune) {
    int w = snprintf(buf + off, cap - off, "%d %d %d %lld %d %d %.3f %d\n", e.first.mode, e.first.tsize,
                     e.first.n, e.first.nnz, e.first.sell, e.second.variant, e.second.us, e.second.best_csr);
    if (w < 0 || w >= cap - off) break;
    off += w;
  }
  return RICH_OK;
}

// Entries in autotune_table's format (a saved table): classes already present keep
// their choice.  A variant that is not one of the candidates is rejected.
int autotune_load(const char* text) {
  auto valid = [](int v) {
    if (v == kSellVariant || v == kSellVariant8 || v == kSellVariant2 || v == kSellVariantP) return true;
    const int g = v & 0xff, u = v & ~0xff;
    if (u != 0 && u != kUnroll) return false;
    if (g != 1 && g != 2 && g != 4 && g != 8 && g != 16 && g != 32) return false;
    return u == 0 || g <= 8;
  };
  std::vector<std::pair<TuneKey, TuneVal>> rows;
  const char* p = text;
  while (*p) {
    int mode, tsize, n, sell, variant, best_csr, used = 0;
    long long nnz;
    float us;
    if (sscanf(p, "%d %d %d %lld %d %d %f %d%n", &mode, &tsize, &n, &nnz, &sell, &variant, &us, &best_csr, &used) !=
        8)
      return RICH_EINVAL;
    if (mode < 0 || mode > 3 || (tsize != 4 && tsize != 8) || (sell != 0 && sell != 1) || !valid(variant) ||
        !valid(best_csr) || best_csr >= kSellVariant || (!sell && variant >= kSellVariant))
      return RICH_EINVAL;
    rows.push_back({TuneKey{mode, tsize, n, nnz, sell}, TuneVal{variant, us, best_csr}});
    p += used;
    while (*p == '\n' || *p == ' ' || *p == '\r') ++p;
  }
  std::lock_guard<std::mutex> lk(g_tune_mu);
  for (auto& r : rows) g_tune.insert(r);
  return RICH_OK;
}

// x = M b for a dense row-major n x n matrix; one warp per row.
template <class T>
__global__ void k_gemv(int n, const T* __restrict__ M, const T* __restrict__ b, T* __restrict__ x) {
  int lane = threadIdx.x & 31;
  for (int row = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; row < n; row += (gridDim.x * blockDim.x) >> 5) {
    T s = 0;
    for (int j = lane; j < n; j += 32) s += M[(long long)row * n + j] * b[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (lane == 0) x[row] = s;
  }
}

__global__ void k_d2f(long long n, const double* __restrict__ a, float* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (float)a[i];
}
__global__ void k_f2d(long long n, const float* __restrict__ a, double* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = (double)a[i];
}

// Finest-level l1-Jacobi sweep and residual on the stencil form.  The l1 row norm
// is diag + sum of the six face weights (all couplings are -w with w >= 0).
// mode 1: xo = x + D_l1^-1 (b - A x); 2: xo = b - A x (residual).  The first
// sweep from x = 0 (x = D_l1^-1 b) is the elementwise k_jacobi0.
template <class T, int MODE>
__global__ void __launch_bounds__(kLineThreads) k_st_smooth(GridP g, Stencil4<T> A, const T* __restrict__ b,
                                                            const T* __restrict__ x, T* __restrict__ xo) {
  int i = blockIdx.y * kLineThreads + threadIdx.x;
  if (i >= g.nx) return;
  int r = blockIdx.x;
  int j = r % g.ny;
  int k = r / g.ny;
  int nx = g.nx;
  int sxy = g.nx * g.ny;
  int c = r * nx + i;
  T wxp = A.wx[c], wyp = A.wy[c], wzp = A.wz[c];
  T xc = x[c];
  T ax = A.diag[c] * xc;
  if (i > 0) ax -= A.wx[c - 1] * x[c - 1];
  if (i < nx - 1) ax -= wxp * x[c + 1];
  if (j > 0) ax -= A.wy[c - nx] * x[c - nx];
  if (j < g.ny - 1) ax -= wyp * x[c + nx];
  if (k > 0) ax -= A.wz[c - sxy] * x[c - sxy];
  if (k < g.nz - 1) ax -= wzp * x[c + sxy];
  if (MODE == 2) xo[c] = b[c] - ax;
  else xo[c] = xc + A.dinv[c] * (b[c] - ax);
}

// The first l1-Jacobi sweep from zero, y = D_l1^-1 b, folded into the next stencil
// pass on the finest level: y is recomputed from b and the l1 scaling wherever the
// next pass reads it (own cell and the six neighbours, all cache hits), so it is
// never written and read back.  MODE 1: out = y + D_l1^-1 (b - A y), the second
// sweep; MODE 2: x1 = y and out = b - A y, the residual after a single sweep.
template <class T, int MODE>
__global__ void __launch_bounds__(kLineThreads) k_st_first(GridP g, Stencil4<T> A, const T* __restrict__ b,
                                                           T* __restrict__ x1, T* __restrict__ out) {
  int i = blockIdx.y * kLineThreads + threadIdx.x;
  if (i >= g.nx) return;
  int r = blockIdx.x;
  int j = r % g.ny;
  int k = r / g.ny;
  int nx = g.nx;
  int sxy = g.nx * g.ny;
  int c = r * nx + i;
  T bc = b[c];
  T yc = A.dinv[c] * bc;
  T ay = A.diag[c] * yc;
  if (i > 0) ay -= A.wx[c - 1] * (A.dinv[c - 1] * b[c - 1]);
  if (i < nx - 1) ay -= A.wx[c] * (A.dinv[c + 1] * b[c + 1]);
  if (j > 0) ay -= A.wy[c - nx] * (A.dinv[c - nx] * b[c - nx]);
  if (j < g.ny - 1) ay -= A.wy[c] * (A.dinv[c + nx] * b[c + nx]);
  if (k > 0) ay -= A.wz[c - sxy] * (A.dinv[c - sxy] * b[c - sxy]);
  if (k < g.nz - 1) ay -= A.wz[c] * (A.dinv[c + sxy] * b[c + sxy]);
  if (MODE == 2) {
    x1[c] = yc;
    out[c] = bc - ay;
  } else {
    out[c] = yc + A.dinv[c] * (bc - ay);
  }
}

// Hybrid Gauss-Seidel (the paper's smoother, Sec. 5.2 / Sec. 6): Gauss-Seidel inside
// the block one thread (or lane group) owns, Jacobi between blocks, scaled by
// a_ii + sum over couplings to other blocks of |a_ij| (the l1 form).  x == nullptr
// sweeps from zero; xo receives the new values (blocks read only x for each other).
//
// Finest level: a block is a segment of `seg` cells of one vertical column; the
// thread walks it upward (FWD) or downward carrying the new value of the cell just
// updated, so the in-block coupling costs no extra load.  Launch: blockIdx.x over
// (j, segment), blockIdx.y over x tiles, threadIdx.x = i (coalesced in x).
template <class T, bool FWD>
__global__ void __launch_bounds__(kLineThreads) k_hgs_st(GridP g, Stencil4<T> A, int seg, const T* __restrict__ b,
                                                         const T* __restrict__ x, T* __restrict__ xo) {
  int i = blockIdx.y * kLineThreads + threadIdx.x;
  if (i >= g.nx) return;
  int r = blockIdx.x;
  int j = r % g.ny;
  int k0 = (r / g.ny) * seg;
  int k1 = min(g.nz, k0 + seg);
  int nx = g.nx;
  int sxy = g.nx * g.ny;
  T carry = T(0);
  for (int q = 0; q < k1 - k0; ++q) {
    int k = FWD ? k0 + q : k1 - 1 - q;
    int c = (k * g.ny + j) * nx + i;
    T xc = x ? x[c] : T(0);
    T ax = A.diag[c] * xc;
    T d = A.diag[c];
    T w;
    if (i > 0) { w = A.wx[c - 1]; ax -= w * (x ? x[c - 1] : T(0)); d += w; }
    if (i < nx - 1) { w = A.wx[c]; ax -= w * (x ? x[c + 1] : T(0)); d += w; }
    if (j > 0) { w = A.wy[c - nx]; ax -= w * (x ? x[c - nx] : T(0)); d += w; }
    if (j < g.ny - 1) { w = A.wy[c]; ax -= w * (x ? x[c + nx] : T(0)); d += w; }
    if (k > 0) {
      w = A.wz[c - sxy];
      if (k - 1 >= k0) ax -= w * (FWD ? carry : (x ? x[c - sxy] : T(0)));  // in block: new below (FWD)
      else { ax -= w * (x ? x[c - sxy] : T(0)); d += w; }
    }
    if (k < g.nz - 1) {
      w = A.wz[c];
      if (k + 1 < k1) ax -= w * (FWD ? (x ? x[c + sxy] : T(0)) : carry);  // in block: new above (backward)
      else { ax -= w * (x ? x[c + sxy] : T(0)); d += w; }
    }
    T xn = xc + (b[c] - ax) / d;
    xo[c] = xn;
    carry = xn;
  }
}

// Coarser levels: a block is `bs` consecutive rows, walked by one group of G lanes
// (rows of tens to hundreds of entries); lane 0 writes each new value and the group
// synchronises before the next row reads it.
template <class T, bool FWD, int G>
__global__ void k_hgs_csr(int n, const int* __restrict__ rp, const int* __restrict__ col, const T* __restrict__ val,
                          int bs, const T* __restrict__ b, const T* __restrict__ x, T* __restrict__ xo) {
  int lane = threadIdx.x & (G - 1);
  unsigned mask = G == 32 ? 0xffffffffu : (((1u << G) - 1) << ((threadIdx.x & 31) & ~(G - 1)));
  int nblk = (n + bs - 1) / bs;
  int groups = (gridDim.x * blockDim.x) / G;
  for (int blk = (blockIdx.x * blockDim.x + threadIdx.x) / G; blk < nblk; blk += groups) {
    int r0 = blk * bs;
    int r1 = min(n, r0 + bs);
    for (int q = 0; q < r1 - r0; ++q) {
      int i = FWD ? r0 + q : r1 - 1 - q;
      T s = 0, d = 0;
      for (int e = rp[i] + lane; e < rp[i + 1]; e += G) {
        int jj = col[e];
        T a = val[e];
        T xv;
        if (jj >= r0 && jj < r1) {
          bool updated = FWD ? jj < i : jj > i;
          xv = updated ? xo[jj] : (x ? x[jj] : T(0));
          if (jj == i) d += a;
        } else {
          xv = x ? x[jj] : T(0);
          d += a < T(0) ? -a : a;
        }
        s += a * xv;
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        s += __shfl_down_sync(mask, s, o, G);
        d += __shfl_down_sync(mask, d, o, G);
      }
      if (lane == 0) xo[i] = (x ? x[i] : T(0)) + (b[i] - s) / d;
      __syncwarp(mask);
    }
  }
}

template <class T, bool FWD>
static void hgs_csr(cudaStream_t st, int n, long long nnz, const int* rp, const int* col, const T* val, int bs,
                    const T* b, const T* x, T* y) {
  double avg = n > 0 ? (double)nnz / n : 0.0;
  long long nblk = (n + bs - 1) / bs;
  if (avg > 64) k_hgs_csr<T, FWD, 32><<<grid_for(nblk * 32), kBlock, 0, st>>>(n, rp, col, val, bs, b, x, y);
  else if (avg > 24) k_hgs_csr<T, FWD, 16><<<grid_for(nblk * 16), kBlock, 0, st>>>(n, rp, col, val, bs, b, x, y);
  else if (avg > 10) k_hgs_csr<T, FWD, 8><<<grid_for(nblk * 8), kBlock, 0, st>>>(n, rp, col, val, bs, b, x, y);
  else k_hgs_csr<T, FWD, 4><<<grid_for(nblk * 4), kBlock, 0, st>>>(n, rp, col, val, bs, b, x, y);
}

template <class T>
static const Stencil4<T>& fine(rich_ctx* c);
template <>
const Stencil4<double>& fine<double>(rich_ctx* c) { return c->H.st64; }
template <>
const Stencil4<float>& fine<float>(rich_ctx* c) { return c->H.st32; }

template <class T>
struct LevelView {
  int n;
  const int *rp, *col;
  const T* val;
  const T* dinv;
  const int *prp, *pcol, *rrp, *rcol;
  const T *pval, *rval;
  SellSrc<T> sa, sp, sr;  // SELL sources of A, P, R
};

template <class T>
static LevelView<T> view(rich_ctx* c, int l);

template <>
LevelView<double> view<double>(rich_ctx* c, int l) {
  Level& L = c->H.lv[l];
  return LevelView<double>{L.n,     L.A.rowptr, L.A.col, L.A.val,
                           L.dinv,  L.P.rowptr, L.P.col, L.R.rowptr,
                           L.R.col, L.P.val,    L.R.val, {&L.sA, &L.A, L.A.val},
                           {&L.sP, &L.P, L.P.val}, {&L.sR, &L.R, L.R.val}};
}
template <>
LevelView<float> view<float>(rich_ctx* c, int l) {
  Level& L = c->H.lv[l];
  return LevelView<float>{L.n,       L.A.rowptr, L.A.col, L.A32,
                          L.dinv32,  L.P.rowptr, L.P.col, L.R.rowptr,
                          L.R.col,   L.P32,      L.R32,   {&L.sA, &L.A, L.A32},
                          {&L.sP, &L.P, L.P32},  {&L.sR, &L.R, L.R32}};
}

template <class T>
static const T* coarse_inv(rich_ctx* c);
template <>
const double* coarse_inv<double>(rich_ctx* c) { return c->H.cdense; }
template <>
const float* coarse_inv<float>(rich_ctx* c) { return c->H.cinv32; }

template <class T>
static int vcycle_level(rich_ctx* c, int l, const T* b, T** xres);

// One hybrid Gauss-Seidel sweep on level l (x == nullptr: from zero) into xo.
template <class T>
static int hgs_sweep(rich_ctx* c, int l, bool forward, const T* b, const T* x, T* xo) {
  Hierarchy& H = c->H;
  Level& L = H.lv[l];
  const double es = sizeof(T);
  if (l == 0) {
    const GridP& g = c->g;
    int nseg = (g.nz + H.opts.hgs_seg - 1) / H.opts.hgs_seg;
    dim3 grid((unsigned)((long long)g.ny * nseg), (unsigned)((g.nx + kLineThreads - 1) / kLineThreads), 1);
    ProfScope ps("hgs_l0", c->st, (double)g.n * (x ? 8.0 : 7.0) * es, 20.0 * (double)g.n);
    if (forward) k_hgs_st<T, true><<<grid, kLineThreads, 0, c->st>>>(g, fine<T>(c), H.opts.hgs_seg, b, x, xo);
    else k_hgs_st<T, false><<<grid, kLineThreads, 0, c->st>>>(g, fine<T>(c), H.opts.hgs_seg, b, x, xo);
  } else {
    LevelView<T> v = view<T>(c, l);
    ProfScope ps("hgs", c->st, (double)L.n * (4.0 + 3.0 * es) + (double)L.A.nnz * (4.0 + es), 4.0 * L.A.nnz);
    if (forward) hgs_csr<T, true>(c->st, L.n, L.A.nnz, v.rp, v.col, v.val, H.opts.hgs_block, b, x, xo);
    else hgs_csr<T, false>(c->st, L.n, L.A.nnz, v.rp, v.col, v.val, H.opts.hgs_block, b, x, xo);
  }
  RICH_LAUNCH_CHECK();
  return RICH_OK;
}

// V-cycle level with hybrid Gauss-Seidel: nu1 backward sweeps (the first from zero),
// residual, restriction, coarse correction, nu2 forward sweeps.
template <class T>
static int vcycle_level_hgs(rich_ctx* c, int l, const T* b, T** xres) {
  Hierarchy& H = c->H;
  Level& L = H.lv[l];
  LevelView<T> v = view<T>(c, l);
  int n = v.n;
  int g = grid_for(n);
  T* x = (T*)L.x;
  T* t = (T*)L.t;
  const double es = sizeof(T);
  const bool st0 = (l == 0);
  for (int s = 0; s < H.opts.nu1; ++s) {
    RICH_CHECK(hgs_sweep<T>(c, l, false, b, s == 0 ? (const T*)nullptr : (const T*)x, t));
    std::swap(x, t);
  }
  if (H.opts.nu1 == 0) RICH_CUDA(cudaMemsetAsync(x, 0, sizeof(T) * n, c->st));
  {
    ProfScope ps(st0 ? "resid_l0" : "csr_resid", c->st,
                 st0 ? (double)n * 7.0 * es : (double)n * (4.0 + 3.0 * es) + (double)L.A.nnz * (4.0 + es));
    if (st0) k_st_smooth<T, 2><<<line_grid(c->g), kLineThreads, 0, c->st>>>(c->g, fine<T>(c), b, x, (T*)L.r);
    else RICH_CHECK(csr_op<T, 3>(c, n, L.A.nnz, v.rp, v.col, v.val, (const T*)nullptr, b, x, (T*)L.r, &v.sa));
  }
  RICH_LAUNCH_CHECK();
  Level& C = H.lv[l + 1];
  {
    ProfScope ps("restrict", c->st, (double)C.n * (4.0 + es) + (double)L.R.nnz * (4.0 + es) + (double)n * es);
    RICH_CHECK(csr_op<T, 0>(c, C.n, L.R.nnz, v.rrp, v.rcol, v.rval, (const T*)nullptr, (const T*)nullptr,
                            (const T*)L.r, (T*)C.b, &v.sr));
  }
  RICH_LAUNCH_CHECK();
  T* xc = nullptr;
  RICH_CHECK(vcycle_level<T>(c, l + 1, (const T*)C.b, &xc));
  {
    ProfScope ps("prolong", c->st, (double)n * (4.0 + 2.0 * es) + (double)L.P.nnz * (4.0 + es) + (double)C.n * es);
    RICH_CHECK(csr_op<T, 1>(c, n, L.P.nnz, v.prp, v.pcol, v.pval, (const T*)nullptr, (const T*)nullptr, xc, x,
                            &v.sp));
  }
  RICH_LAUNCH_CHECK();
  for (int s = 0; s < H.opts.nu2; ++s) {
    RICH_CHECK(hgs_sweep<T>(c, l, true, b, x, t));
    std::swap(x, t);
  }
  if (x != (T*)L.x) {
    L.t = L.x;
    L.x = x;
  }
  *xres = x;
  return RICH_OK;
}

// b is the level's right-hand side, the result is left in *xres (one of the level's buffers).
template <class T>
static int vcycle_level(rich_ctx* c, int l, const T* b, T** xres) {
  Hierarchy& H = c->H;
  Level& L = H.lv[l];
  LevelView<T> v = view<T>(c, l);
  int n = v.n;
  int g = grid_for(n);
  T* x = (T*)L.x;
  T* t = (T*)L.t;
  const double es = sizeof(T);
  // algorithmic bytes of one sweep over this level's CSR matrix (pattern + values + 4 vectors)
  const double sweep_bytes = (double)n * (4.0 + 4.0 * es) + (double)L.A.nnz * (4.0 + es);
  if (l == H.nlev - 1) {
    if (H.dense) {
      ProfScope ps("coarse_gemv", c->st, (double)n * n * es + 2.0 * n * es);
      k_gemv<T><<<grid_for((long long)n * 32), kBlock, 0, c->st>>>(n, coarse_inv<T>(c), b, x);
      RICH_LAUNCH_CHECK();
    } else {  // stalled coarsening: l1-Jacobi sweeps from zero on the (large) coarsest level
      k_jacobi0<T><<<g, kBlock, 0, c->st>>>(n, v.dinv, b, x);
      RICH_LAUNCH_CHECK();
      for (int s = 1; s < kCoarseSweeps; ++s) {
        RICH_CHECK(csr_op<T, 2>(c, n, L.A.nnz, v.rp, v.col, v.val, v.dinv, b, x, t, &v.sa));
        RICH_LAUNCH_CHECK();
        std::swap(x, t);
      }
    }
    *xres = x;
    return RICH_OK;
  }
  int nu1 = H.opts.nu1, nu2 = H.opts.nu2;
  // finest level: stencil form (4 coefficient arrays + b + x in, x out)
  const bool st0 = (l == 0);
  if (H.opts.smoother == RICH_SMOOTH_HYBRID_GS) return vcycle_level_hgs<T>(c, l, b, xres);
  // warp-per-row CSR kernels where rows are long
  const double st_bytes = (double)n * 8.0 * es;  // diag, 3 face weights, dinv, b, x in; x out
  // In FP32 the first sweep from zero is folded into the next stencil pass (one pass
  // over the finest level less); in FP64 the fold's extra products (D^-1 b at the six
  // neighbours) cost more on GB300's narrow FP64 pipe than the pass it saves (ncu:
  // 88-91 % FP64-pipe utilisation in these sweeps), so FP64 keeps separate passes.
  constexpr bool kFold = sizeof(T) == 4;
  if (kFold && st0 && nu1 == 1) {
    // finest level, one pre-sweep: the sweep from zero and the residual in one pass
    ProfScope ps("resid_l0", c->st, (double)n * 8.0 * es, 17.0 * n);
    k_st_first<T, 2><<<line_grid(c->g), kLineThreads, 0, c->st>>>(c->g, fine<T>(c), b, x, (T*)L.r);
    RICH_LAUNCH_CHECK();
  } else if (nu1 > 0) {
    int s0 = 1;
    if (kFold && st0) {
      // finest level: the first two sweeps from zero in one pass
      ProfScope ps("l1jacobi_l0", c->st, (double)n * 7.0 * es, 20.0 * n);
      k_st_first<T, 1><<<line_grid(c->g), kLineThreads, 0, c->st>>>(c->g, fine<T>(c), b, nullptr, x);
      RICH_LAUNCH_CHECK();
      s0 = 2;
    } else {
      // first sweep from x = 0: x = D_l1^-1 b, elementwise (on the finest level the
      // stencil copy's 1/l1 array)
      k_jacobi0<T><<<g, kBlock, 0, c->st>>>(n, st0 ? fine<T>(c).dinv : v.dinv, b, x);
      RICH_LAUNCH_CHECK();
    }
    for (int s = s0; s < nu1; ++s) {
      {
        ProfScope ps(l == 0 ? "l1jacobi_l0" : "l1jacobi", c->st, st0 ? st_bytes : sweep_bytes,
                     st0 ? 16.0 * n : 2.0 * L.A.nnz + 3.0 * n);
        if (st0) k_st_smooth<T, 1><<<line_grid(c->g), kLineThreads, 0, c->st>>>(c->g, fine<T>(c), b, x, t);
        else RICH_CHECK(csr_op<T, 2>(c, n, L.A.nnz, v.rp, v.col, v.val, v.dinv, b, x, t, &v.sa));
      }
      RICH_LAUNCH_CHECK();
      std::swap(x, t);
    }
    {
      ProfScope ps(st0 ? "resid_l0" : "csr_resid", c->st, st0 ? st_bytes : sweep_bytes - (double)n * es);
      if (st0) k_st_smooth<T, 2><<<line_grid(c->g), kLineThreads, 0, c->st>>>(c->g, fine<T>(c), b, x, (T*)L.r);
      else RICH_CHECK(csr_op<T, 3>(c, n, L.A.nnz, v.rp, v.col, v.val, (const T*)nullptr, b, x, (T*)L.r, &v.sa));
    }
    RICH_LAUNCH_CHECK();
  } else {
    RICH_CUDA(cudaMemsetAsync(x, 0, sizeof(T) * n, c->st));
    RICH_CUDA(cudaMemcpyAsync(L.r, b, sizeof(T) * n, cudaMemcpyDeviceToDevice, c->st));
  }
  Level& C = H.lv[l + 1];
  {
    ProfScope ps("restrict", c->st, (double)C.n * (4.0 + es) + (double)L.R.nnz * (4.0 + es) + (double)n * es);
    RICH_CHECK(csr_op<T, 0>(c, C.n, L.R.nnz, v.rrp, v.rcol, v.rval, (const T*)nullptr, (const T*)nullptr,
                            (const T*)L.r, (T*)C.b, &v.sr));
  }
  RICH_LAUNCH_CHECK();
  T* xc = nullptr;
  RICH_CHECK(vcycle_level<T>(c, l + 1, (const T*)C.b, &xc));
  {
    ProfScope ps("prolong", c->st, (double)n * (4.0 + 2.0 * es) + (double)L.P.nnz * (4.0 + es) + (double)C.n * es);
    RICH_CHECK(csr_op<T, 1>(c, n, L.P.nnz, v.prp, v.pcol, v.pval, (const T*)nullptr, (const T*)nullptr, xc, x,
                            &v.sp));
  }
  RICH_LAUNCH_CHECK();
  for (int s = 0; s < nu2; ++s) {
    {
      ProfScope ps(l == 0 ? "l1jacobi_l0" : "l1jacobi", c->st, st0 ? st_bytes : sweep_bytes,
                   st0 ? 16.0 * n : 2.0 * L.A.nnz + 3.0 * n);
      if (st0) k_st_smooth<T, 1><<<line_grid(c->g), kLineThreads, 0, c->st>>>(c->g, fine<T>(c), b, x, t);
      else RICH_CHECK(csr_op<T, 2>(c, n, L.A.nnz, v.rp, v.col, v.val, v.dinv, b, x, t, &v.sa));
    }
    RICH_LAUNCH_CHECK();
    std::swap(x, t);
  }
  // keep the level's buffer pointers consistent with where the result lives
  if (x != (T*)L.x) {
    L.t = L.x;
    L.x = x;
  }
  *xres = x;
  return RICH_OK;
}

// Captures the V-cycle from the level-0 right-hand side buffer L0.b as one graph
// (H.vc_exec, its result at H.vc_out).  It runs after a direct application, so the
// tuner's choices and the SELL copies exist and nothing in the cycle allocates or
// synchronises.  The capture stream is a private non-blocking one (the context's
// stream may be the legacy default stream, which cannot be captured).  A failed
// capture leaves direct launches for the rest of this hierarchy.
static int vcycle_capture(rich_ctx* c) {
  Hierarchy& H = c->H;
  Level& L0 = H.lv[0];
  cudaStream_t cs;
  RICH_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaStream_t saved = c->st;
  RICH_CUDA(cudaStreamSynchronize(saved));
  c->st = cs;
  long long before = 0, after = 0;
  rich_kernel_launches(&before);
  cudaGraph_t graph = nullptr;
  void* out = nullptr;
  int rc = RICH_OK;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    if (c->prec == RICH_PREC_MIXED) {
      float* x = nullptr;
      rc = vcycle_level<float>(c, 0, (const float*)L0.b, &x);
      out = x;
    } else {
      double* x = nullptr;
      rc = vcycle_level<double>(c, 0, (const double*)L0.b, &x);
      out = x;
    }
    e = cudaStreamEndCapture(cs, &graph);
  }
  c->st = saved;
  rich_kernel_launches(&after);
  count_launches(before - after);  // recorded, not launched
  if (e == cudaSuccess && rc == RICH_OK) {
    e = cudaGraphInstantiate(&H.vc_exec, graph, 0);
    if (e == cudaSuccess) {
      H.vc_nodes = after - before;
      H.vc_out = out;
    } else {
      H.vc_exec = nullptr;
    }
  }
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess || rc != RICH_OK || !H.vc_exec) {
    cudaGetLastError();
    if (H.vc_exec) cudaGraphExecDestroy(H.vc_exec);
    H.vc_exec = nullptr;
    H.vc_off = true;
  }
  return RICH_OK;
}

// The V-cycle's kernels from r into z, launched (or captured) as they come.
static int vcycle_direct(rich_ctx* c, const double* r, double* z) {
  Hierarchy& H = c->H;
  const long long n = c->g.n;
  if (c->prec == RICH_PREC_MIXED) {
    Level& L0 = H.lv[0];
    k_d2f<<<grid_for(n), kBlock, 0, c->st>>>(n, r, (float*)L0.b);
    RICH_LAUNCH_CHECK();
    float* x = nullptr;
    RICH_CHECK(vcycle_level<float>(c, 0, (const float*)L0.b, &x));
    k_f2d<<<grid_for(n), kBlock, 0, c->st>>>(n, x, z);
    RICH_LAUNCH_CHECK();
  } else {
    double* x = nullptr;
    RICH_CHECK(vcycle_level<double>(c, 0, r, &x));
    RICH_CUDA(cudaMemcpyAsync(z, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st));
  }
  return RICH_OK;
}

// Whether the V-cycle of this hierarchy may run from a captured graph now.
static bool vcycle_graphable(rich_ctx* c) {
  const Hierarchy& H = c->H;
  return H.opts.graph && H.opts.precond == RICH_PRECOND_AMG && H.opts.smoother == RICH_SMOOTH_L1JACOBI && !H.vc_off &&
         !profiling_active();
}

int vcycle_apply(rich_ctx* c, const double* r, double* z) {
  Hierarchy& H = c->H;
  if (!H.built) return RICH_ESTATE;
  if (H.opts.precond == RICH_PRECOND_AS) return as_apply(c, r, z);
  long long n = c->g.n;
  if (vcycle_graphable(c) && H.vc_calls > 0) {  // the first application launched directly
    if (!H.vc_exec) RICH_CHECK(vcycle_capture(c));
    if (H.vc_exec) {
      Level& L0 = H.lv[0];
      if (c->prec == RICH_PREC_MIXED) {
        k_d2f<<<grid_for(n), kBlock, 0, c->st>>>(n, r, (float*)L0.b);
        RICH_LAUNCH_CHECK();
      } else {
        RICH_CUDA(cudaMemcpyAsync(L0.b, r, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st));
      }
      RICH_CUDA(cudaGraphLaunch(H.vc_exec, c->st));
      count_launches(H.vc_nodes);
      if (c->prec == RICH_PREC_MIXED) {
        k_f2d<<<grid_for(n), kBlock, 0, c->st>>>(n, (const float*)H.vc_out, z);
        RICH_LAUNCH_CHECK();
      } else {
        RICH_CUDA(cudaMemcpyAsync(z, H.vc_out, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st));
      }
      return RICH_OK;
    }
  }
  ++H.vc_calls;
  return vcycle_direct(c, r, z);
}

// ---------------------------------------------------------------- Krylov kernels (FP64)

__global__ void k_dot2(long long n, const double* __restrict__ a, const double* __restrict__ b,
                       const double* __restrict__ cc, const double* __restrict__ d, double* __restrict__ partials) {
  double v[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    v[0] += a[i] * b[i];
    v[1] += cc[i] * d[i];
  }
  block_sum<2>(v);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = v[0];
    partials[gridDim.x + blockIdx.x] = v[1];
  }
}

// p = z - (s[num] / s[den]) p
__global__ void k_fcg_dir(long long n, const double* __restrict__ z, double* __restrict__ p,
                          const double* __restrict__ s, int num, int den) {
  double beta = s[num] / s[den];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    p[i] = z[i] - beta * p[i];
}

// alpha = s[num]/s[den]; x += alpha p; r -= alpha q; partial sums of r.r
__global__ void k_fcg_update(long long n, double* __restrict__ x, double* __restrict__ r, const double* __restrict__ p,
                             const double* __restrict__ q, const double* __restrict__ s, int num, int den,
                             double* __restrict__ partials) {
  double alpha = s[num] / s[den];
  double v[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    double ri = r[i] - alpha * q[i];
    r[i] = ri;
    v[0] += ri * ri;
  }
  block_sum<1>(v);
  if (threadIdx.x == 0) partials[blockIdx.x] = v[0];
}

// Batched dot products h[q] = V[q] . w: block (bx, q) reduces its share of one
// vector; w is re-read per q from L2, V streams from HBM once.
__global__ void k_bdot(long long n, const double* __restrict__ V, const double* __restrict__ w,
                       double* __restrict__ partials, const int* __restrict__ run) {
  int q = blockIdx.y;
  if (run && !*run) {  // skipped pass: zero partials
    if (threadIdx.x == 0) partials[(long long)q * gridDim.x + blockIdx.x] = 0.0;
    return;
  }
  const double* v = V + (long long)q * n;
  double acc[1] = {0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    acc[0] += v[i] * w[i];
  block_sum<1>(acc);
  if (threadIdx.x == 0) partials[(long long)q * gridDim.x + blockIdx.x] = acc[0];
}

constexpr int kBdotBlocks = 2 * kNumSM;  // x-blocks per vector (fixed: deterministic summation order)

static void launch_multidot(int nb, cudaStream_t st, long long n, int nv, const double* V, const double* w,
                            double* partials, const int* run = nullptr) {
  (void)nb;
  k_bdot<<<dim3(kBdotBlocks, nv), kBlock, 0, st>>>(n, V, w, partials, run);
}

// w -= sum_q h[q] V[q], in place
__global__ void k_orth_axpy(long long n, int nv, const double* __restrict__ V, const double* __restrict__ h,
                            double* w) {
  __shared__ double hs[64];
  for (int q = threadIdx.x; q < nv; q += blockDim.x) hs[q] = h[q];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double t = w[i];
    for (int q = 0; q < nv; ++q) t -= hs[q] * V[(long long)q * n + i];
    w[i] = t;
  }
}

// Device scalars of an FGMRES iteration (restart <= 63, so j <= 62): h1 in [0, j],
// h2 in [64, 64 + j]; ||w'||^2 and the DGKS decision in the slots neither reaches
// (both come back with the one 128-double read-back); ||w||^2, read on the device
// only, past the read-back.
constexpr int kSlotW1 = 63, kSlotRun = 127, kSlotW = 130;

// DGKS decision on the device: run the second pass when ||w'||^2 < ||w||^2 / 2
// (also left in s[i_out] as 1.0 / 0.0 for the host's read-back of the scalars)
__global__ void k_dgks(double* __restrict__ s, int i_w, int i_wp, int i_out, int* __restrict__ run) {
  const int r = s[i_wp] < 0.5 * s[i_w] ? 1 : 0;
  *run = r;
  s[i_out] = r;
}

// out = f * (w - sum_q h2[q] V[q]); without a second pass (run == 0) out = f * w
__global__ void k_orth_final(long long n, int nv, const double* __restrict__ V, const double* __restrict__ h2,
                             const double* __restrict__ w, double f, double* __restrict__ out,
                             const int* __restrict__ run) {
  __shared__ double hs[64];
  if (run && !*run) nv = 0;
  for (int q = threadIdx.x; q < nv; q += blockDim.x) hs[q] = h2[q];
  __syncthreads();
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double t = w[i];
    for (int q = 0; q < nv; ++q) t -= hs[q] * V[(long long)q * n + i];
    out[i] = f * t;
  }
}

// y += sign * sum_q coef[q] V[q]
__global__ void k_multiaxpy(long long n, int nv, const double* __restrict__ V, const double* __restrict__ coef,
                            double sign, double* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < nv; ++q) s += coef[q] * V[(long long)q * n + i];
    y[i] += sign * s;
  }
}

__global__ void k_scale(long long n, const double* __restrict__ a, double f, double* __restrict__ b) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    b[i] = f * a[i];
}

// y = a - b
__global__ void k_sub(long long n, const double* __restrict__ a, const double* __restrict__ b, double* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a[i] - b[i];
}

// y = a + lam * d
__global__ void k_axpby(long long n, const double* __restrict__ a, double lam, const double* __restrict__ d,
                        double* __restrict__ y) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    y[i] = a[i] + lam * d[i];
}

__global__ void k_copy_scalar(double* s, int from, int to) { s[to] = s[from]; }

static int ensure_krylov(rich_ctx* c, int m) {
  KrylovWork& k = c->kw;
  long long n = c->g.n;
  if (k.n != n) {
    dfree(k.x); dfree(k.r); dfree(k.p); dfree(k.q); dfree(k.qprev); dfree(k.z); dfree(k.w);
    RICH_CHECK(dalloc(&k.x, n));
    RICH_CHECK(dalloc(&k.r, n));
    RICH_CHECK(dalloc(&k.p, n));
    RICH_CHECK(dalloc(&k.q, n));
    RICH_CHECK(dalloc(&k.qprev, n));
    RICH_CHECK(dalloc(&k.z, n));
    RICH_CHECK(dalloc(&k.w, n));
    RICH_CHECK(dalloc(&k.hcoef, 128));
    k.n = n;
  }
  if (m > 0 && k.m < m) {
    dfree(k.V);
    dfree(k.Z);
    RICH_CHECK(dalloc(&k.V, (long long)(m + 1) * n));
    RICH_CHECK(dalloc(&k.Z, (long long)m * n));
    k.m = m;
  }
  return RICH_OK;
}

// Flexible CG (Notay, truncation 1).  Returns RICH_ENOTCONV_LIN on maxit, on
// (p, q) <= 0, or when ||r|| exceeds 10x the smallest seen.
// One FCG iteration from the preconditioner application to the copy of its scalars
// (rr, zq, pq) into the pinned host mirror; `first`: the first iteration (p = z).
// Under capture the V-cycle's kernels are recorded directly.
static int fcg_iteration(rich_ctx* c, double* x, double* q, const double* qprev, bool first, bool capturing) {
  KrylovWork& k = c->kw;
  const long long n = c->g.n;
  const int g = grid_for(n), nb = red_grid(n);
  double* s = c->dsc;  // 0 rr, 1 zq, 2 pq, 3 pr, 4 pq_prev
  RICH_CHECK(capturing ? vcycle_direct(c, k.r, k.z) : vcycle_apply(c, k.r, k.z));
  if (first) {
    RICH_CUDA(cudaMemcpyAsync(k.p, k.z, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st));
  } else {
    RICH_CHECK(dot(c, k.z, qprev, n, s + 1));
    k_fcg_dir<<<g, kBlock, 0, c->st>>>(n, k.z, k.p, s, 1, 4);
    RICH_LAUNCH_CHECK();
  }
  RICH_CHECK(stencil_apply(c, c->J7, k.p, q));
  k_dot2<<<nb, kBlock, 0, c->st>>>(n, k.p, q, k.p, k.r, c->partials);
  RICH_LAUNCH_CHECK();
  RICH_CHECK(finish_sums(c, c->partials, nb, 2, s + 2));
  {
    ProfScope ps("fcg_update", c->st, (double)n * 48.0);
    k_fcg_update<<<nb, kBlock, 0, c->st>>>(n, x, k.r, k.p, q, s, 3, 2, c->partials);
  }
  RICH_LAUNCH_CHECK();
  RICH_CHECK(finish_sums(c, c->partials, nb, 1, s + 0));
  k_copy_scalar<<<1, 1, 0, c->st>>>(s, 2, 4);
  RICH_LAUNCH_CHECK();
  RICH_CUDA(cudaMemcpyAsync(c->hsc, s, 3 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
  return RICH_OK;
}

// Captures fcg_iteration (not the first) with these q, q_prev and x as graph `par`,
// as vcycle_capture does; a failed capture leaves direct launches.
static void fcg_capture(rich_ctx* c, int par, double* x, double* q, const double* qprev) {
  Hierarchy& H = c->H;
  cudaStream_t cs;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    H.fcg_off = true;
    return;
  }
  cudaStream_t saved = c->st;
  cudaError_t e = cudaStreamSynchronize(saved);
  c->st = cs;
  long long before = 0, after = 0;
  rich_kernel_launches(&before);
  cudaGraph_t graph = nullptr;
  int rc = RICH_OK;
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    rc = fcg_iteration(c, x, q, qprev, false, true);
    e = cudaStreamEndCapture(cs, &graph);
  }
  c->st = saved;
  rich_kernel_launches(&after);
  count_launches(before - after);  // recorded, not launched
  if (e == cudaSuccess && rc == RICH_OK) {
    e = cudaGraphInstantiate(&H.fcg_exec[par], graph, 0);
    if (e == cudaSuccess) H.fcg_nodes[par] = after - before;
    else H.fcg_exec[par] = nullptr;
  }
  if (graph) cudaGraphDestroy(graph);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess || rc != RICH_OK || !H.fcg_exec[par]) {
    cudaGetLastError();
    H.fcg_off = true;
  }
}

// Notay's flexible CG (truncation 1).  With o->stall > 0 it gives up when a window
// of kStallWindow iterations reduced the residual by less than that fraction.
// From the second iteration on, an iteration is a graph replay where the V-cycle
// may be (rich_amg_opts.graph): the same kernels on the same buffers.
static int fcg(rich_ctx* c, const double* b, double* x, const rich_krylov_opts* o, rich_krylov_stats* st) {
  KrylovWork& k = c->kw;
  Hierarchy& H = c->H;
  long long n = c->g.n;
  double* s = c->dsc;
  RICH_CHECK(nrm2sq(c, b, n, s + 0));
  double h[4];
  RICH_CHECK(fetch_scalars(c, s, 1, h));
  double bn = sqrt(h[0]);
  st->res0 = bn;
  st->res = bn;
  st->iterations = 0;
  st->converged = 0;
  k.fail_reason = 0;
  RICH_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, c->st));
  if (!(bn > 0)) {
    st->converged = std::isfinite(bn) ? 1 : 0;
    return std::isfinite(bn) ? RICH_OK : RICH_ENONFINITE;
  }
  if (!std::isfinite(bn)) return RICH_ENONFINITE;
  RICH_CUDA(cudaMemcpyAsync(k.r, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st));
  double target = o->eta * bn, best = bn, window_start = bn;
  double* q = k.q;
  double* qprev = k.qprev;
  const bool graphs = vcycle_graphable(c) && !H.fcg_off && (!H.fcg_x || H.fcg_x == x);
  for (int it = 1; it <= o->maxit; ++it) {
    bool replayed = false;
    if (graphs && it >= 2 && H.vc_calls > 0 && !H.fcg_off) {
      const int par = it & 1;  // it even: q = k.qprev, q_prev = k.q; odd: the other way round
      if (!H.fcg_exec[par]) {
        H.fcg_x = x;
        fcg_capture(c, par, x, q, qprev);
      }
      if (H.fcg_exec[par]) {
        RICH_CUDA(cudaGraphLaunch(H.fcg_exec[par], c->st));
        count_launches(H.fcg_nodes[par]);
        replayed = true;
      }
    }
    if (!replayed) RICH_CHECK(fcg_iteration(c, x, q, qprev, it == 1, false));
    RICH_CUDA(cudaStreamSynchronize(c->st));
    for (int i = 0; i < 3; ++i) h[i] = c->hsc[i];
    double rn = sqrt(h[0]);
    st->iterations = it;
    st->res = rn;
    if (!std::isfinite(rn) || !std::isfinite(h[2])) return RICH_ENONFINITE;
    if (!(h[2] > 0)) {
      k.fail_reason = 2;
      return RICH_ENOTCONV_LIN;
    }
    if (rn <= target) {
      st->converged = 1;
      return RICH_OK;
    }
    if (rn > 10.0 * best) {
      k.fail_reason = 3;
      return RICH_ENOTCONV_LIN;
    }
    if (it % kStallWindow == 0) {  // stagnation over the last window
      if (o->stall > 0 && rn > (1.0 - o->stall) * window_start) {
        k.fail_reason = 4;
        return RICH_ENOTCONV_LIN;
      }
      window_start = rn;
    }
    best = std::min(best, rn);
    std::swap(q, qprev);
  }
  k.fail_reason = 1;
  return RICH_ENOTCONV_LIN;
}

// Flexible GMRES(m) (Saad) with classical Gram-Schmidt and one re-orthogonalisation.
static int fgmres(rich_ctx* c, const double* b, double* x, const rich_krylov_opts* o, rich_krylov_stats* st) {
  KrylovWork& k = c->kw;
  long long n = c->g.n;
  int m = o->restart;
  int g = grid_for(n);
  int nb = red_grid(n);
  double* s = c->dsc;
  RICH_CHECK(nrm2sq(c, b, n, s));
  double h0[1];
  RICH_CHECK(fetch_scalars(c, s, 1, h0));
  double bn = sqrt(h0[0]);
  st->res0 = bn;
  st->res = bn;
  st->iterations = 0;
  st->converged = 0;
  RICH_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * n, c->st));
  if (!std::isfinite(bn)) return RICH_ENONFINITE;
  if (!(bn > 0)) {
    st->converged = 1;
    return RICH_OK;
  }
  double target = o->eta * bn;
  std::vector<double> H((m + 1) * m), cs(m), sn(m), gv(m + 1), y(m);
  auto Hij = [&](int i, int j) -> double& { return H[(size_t)i * m + j]; };
  double beta = bn;
  const double* r0 = b;
  int its = 0;
  for (;;) {
    k_scale<<<g, kBlock, 0, c->st>>>(n, r0, 1.0 / beta, k.V);
    RICH_LAUNCH_CHECK();
    std::fill(gv.begin(), gv.end(), 0.0);
    gv[0] = beta;
    int jdone = 0;
    bool conv = false;
    for (int j = 0; j < m; ++j) {
      double* Vj = k.V + (long long)j * n;
      double* Zj = k.Z + (long long)j * n;
      RICH_CHECK(vcycle_apply(c, Vj, Zj));
      RICH_CHECK(stencil_apply(c, c->J7, Zj, k.w));
      // Classical Gram-Schmidt with selective re-orthogonalisation (DGKS):
      //   h1 = V^T w; w' = w - V h1; if ||w'||^2 < ||w||^2/2: h2 = V^T w' (else 0);
      //   V[j+1] = (w' - V h2) / hn, hn^2 = ||w'||^2 - ||h2||^2 (V orthonormal).
      // The decision stays on the device; one read-back per iteration.
      int* run = c->iflag + 2;
      RICH_CHECK(nrm2sq(c, k.w, n, s + kSlotW));
      {
        ProfScope ps("multidot", c->st, (double)n * 8.0 * (j + 2), 2.0 * n * (j + 1));
        launch_multidot(nb, c->st, n, j + 1, k.V, k.w, c->partials);
      }
      RICH_LAUNCH_CHECK();
      RICH_CHECK(finish_sums(c, c->partials, kBdotBlocks, j + 1, s));
      {
        // w -= V h1 (w read and written; j + 1 FMAs per cell)
        ProfScope ps("orth_axpy", c->st, (double)n * 8.0 * (j + 3), 2.0 * n * (j + 1));
        k_orth_axpy<<<g, kBlock, 0, c->st>>>(n, j + 1, k.V, s, k.w);
      }
      RICH_LAUNCH_CHECK();
      RICH_CHECK(nrm2sq(c, k.w, n, s + kSlotW1));
      k_dgks<<<1, 1, 0, c->st>>>(s, kSlotW, kSlotW1, kSlotRun, run);
      RICH_LAUNCH_CHECK();
      {
        ProfScope ps("multidot", c->st, (double)n * 8.0 * (j + 2), 2.0 * n * (j + 1));
        launch_multidot(nb, c->st, n, j + 1, k.V, k.w, c->partials, run);
      }
      RICH_LAUNCH_CHECK();
      RICH_CHECK(finish_sums(c, c->partials, kBdotBlocks, j + 1, s + 64));
      RICH_CUDA(cudaMemcpyAsync(c->hsc, s, 128 * sizeof(double), cudaMemcpyDeviceToHost, c->st));
      RICH_CUDA(cudaStreamSynchronize(c->st));
      const bool second = c->hsc[kSlotRun] != 0.0;
      if (!second) prof_adjust_last("multidot", 0.0, 0.0);  // the skipped pass only zeroed its partials
      double h2sq = 0.0;
      for (int i = 0; i <= j; ++i) {
        Hij(i, j) = c->hsc[i] + c->hsc[64 + i];
        h2sq += c->hsc[64 + i] * c->hsc[64 + i];
      }
      double wsq = c->hsc[kSlotW1] - h2sq;
      double hn = wsq > 0 ? sqrt(wsq) : 0.0;
      if (!std::isfinite(hn)) return RICH_ENONFINITE;
      Hij(j + 1, j) = hn;
      {
        // with the second pass: w' - V h2, scaled (j + 3 vectors); without: w' scaled (2 vectors)
        ProfScope ps("orth_final", c->st, second ? (double)n * 8.0 * (j + 3) : 16.0 * n,
                     second ? 2.0 * n * (j + 1) + n : (double)n);
        k_orth_final<<<g, kBlock, 0, c->st>>>(n, j + 1, k.V, s + 64, k.w, hn > 0 ? 1.0 / hn : 0.0,
                                             k.V + (long long)(j + 1) * n, run);
      }
      RICH_LAUNCH_CHECK();
      for (int i = 0; i < j; ++i) {
        double t = cs[i] * Hij(i, j) + sn[i] * Hij(i + 1, j);
        Hij(i + 1, j) = -sn[i] * Hij(i, j) + cs[i] * Hij(i + 1, j);
        Hij(i, j) = t;
      }
      double den = std::hypot(Hij(j, j), Hij(j + 1, j));
      cs[j] = Hij(j, j) / den;
      sn[j] = Hij(j + 1, j) / den;
      Hij(j, j) = den;
      Hij(j + 1, j) = 0.0;
      gv[j + 1] = -sn[j] * gv[j];
      gv[j] = cs[j] * gv[j];
      ++its;
      jdone = j + 1;
      st->res = fabs(gv[j + 1]);
      if (fabs(gv[j + 1]) <= target || hn == 0.0) {
        conv = true;
        break;
      }
      if (its >= o->maxit) break;
    }
    for (int i = jdone - 1; i >= 0; --i) {
      double acc = gv[i];
      for (int q = i + 1; q < jdone; ++q) acc -= Hij(i, q) * y[q];
      y[i] = acc / Hij(i, i);
    }
    for (int i = 0; i < jdone; ++i) c->hsc[i] = y[i];
    RICH_CUDA(cudaMemcpyAsync(k.hcoef, c->hsc, sizeof(double) * jdone, cudaMemcpyHostToDevice, c->st));
    k_multiaxpy<<<g, kBlock, 0, c->st>>>(n, jdone, k.Z, k.hcoef, 1.0, x);
    RICH_LAUNCH_CHECK();
    st->iterations = its;
    if (conv) {
      st->converged = 1;
      return RICH_OK;
    }
    if (its >= o->maxit) return RICH_ENOTCONV_LIN;
    // restart: r = b - J x
    RICH_CHECK(stencil_apply(c, c->J7, x, k.w));
    k_sub<<<g, kBlock, 0, c->st>>>(n, b, k.w, k.r);
    RICH_LAUNCH_CHECK();
    RICH_CHECK(nrm2sq(c, k.r, n, s));
    RICH_CHECK(fetch_scalars(c, s, 1, h0));
    const double beta_cycle = beta;
    beta = sqrt(h0[0]);
    st->res = beta;
    if (beta <= target) {
      st->converged = 1;
      return RICH_OK;
    }
    if (o->stall > 0 && beta > (1.0 - o->stall) * beta_cycle) {  // the cycle stagnated
      c->kw.fail_reason = 4;
      return RICH_ENOTCONV_LIN;
    }
    r0 = k.r;
  }
}

int krylov_run(rich_ctx* c, const double* b, double* x, const rich_krylov_opts* o, rich_krylov_stats* st) {
  if (o->maxit < 1 || !(o->eta > 0) || !(o->stall >= 0.0 && o->stall < 1.0)) return RICH_EINVAL;
  c->kw.fail_reason = 0;
  if (o->kind == RICH_KRYLOV_FGMRES) {
    if (o->restart < 1 || o->restart > 63) return RICH_EINVAL;
    RICH_CHECK(ensure_krylov(c, o->restart));
    return fgmres(c, b, x, o, st);
  }
  if (o->kind != RICH_KRYLOV_FCG) return RICH_EINVAL;
  RICH_CHECK(ensure_krylov(c, 0));
  return fcg(c, b, x, o, st);
}

// ---------------------------------------------------------------- Newton-Armijo step

static int ensure_newton(rich_ctx* c) {
  if (c->F) return RICH_OK;
  long long n = c->g.n;
  RICH_CHECK(dalloc(&c->s_old, n));
  RICH_CHECK(dalloc(&c->F, n));
  RICH_CHECK(dalloc(&c->Ft, n));
  RICH_CHECK(dalloc(&c->d, n));
  RICH_CHECK(dalloc(&c->ptrial, n));
  RICH_CHECK(dalloc(&c->rhs, n));
  return RICH_OK;
}

// CUDA-event timers of the step's phases; ms accumulate into the target at resolve().
struct PhaseTimers {
  std::vector<cudaEvent_t> ev;
  std::vector<double*> acc;
  std::vector<char> closed;
  cudaStream_t st;
  explicit PhaseTimers(cudaStream_t s) : st(s) {}
  ~PhaseTimers() {
    for (auto e : ev) cudaEventDestroy(e);
  }
  int begin(double* target) {
    int i = (int)acc.size();
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    ev.push_back(a);
    ev.push_back(b);
    acc.push_back(target);
    closed.push_back(0);
    cudaEventRecord(a, st);
    return i;
  }
  void end(int i) {
    cudaEventRecord(ev[2 * i + 1], st);
    closed[i] = 1;
  }
  void resolve() {
    for (size_t i = 0; i < acc.size(); ++i) {
      if (!closed[i]) continue;
      cudaEventSynchronize(ev[2 * i + 1]);
      float t = 0.f;
      cudaEventElapsedTime(&t, ev[2 * i], ev[2 * i + 1]);
      *acc[i] += t;
    }
  }
};

// RAII phase: ends on scope exit, including early error returns.
struct Phase {
  PhaseTimers& pt;
  int i;
  Phase(PhaseTimers& p, double* target) : pt(p), i(p.begin(target)) {}
  ~Phase() { pt.end(i); }
};

static int step_body(rich_ctx* c, double* p, double dt, const rich_newton_opts* o, rich_step_stats* st,
                     PhaseTimers& pt);

static int step_impl(rich_ctx* c, double* p, double dt, const rich_newton_opts* o, rich_step_stats* st) {
  RICH_CHECK(ensure_newton(c));
  long long n = c->g.n;
  int g = grid_for(n);
  memset(st, 0, sizeof(*st));
  st->min_lambda = 1.0;
  PhaseTimers pt(c->st);
  int rc;
  {
    Phase whole(pt, &st->ms_total);
    rc = step_body(c, p, dt, o, st, pt);
  }
  pt.resolve();
  return rc;
}

static int step_body(rich_ctx* c, double* p, double dt, const rich_newton_opts* o, rich_step_stats* st,
                     PhaseTimers& pt) {
  long long n = c->g.n;
  int g = grid_for(n);
  // Converged when ||Phi|| <= max(rtol ||Phi_0||, atol, floor): the floor is
  // eps times the norm of the per-cell magnitudes of the products summed into
  // Phi, the accuracy to which Phi can be evaluated (a step that starts near
  // steady state cannot be driven to rtol ||Phi_0|| below it).
  const double kFloor = 2.220446049250313e-16;
  double h[3];
  {
    Phase ph(pt, &st->ms_feval);
    // s_old = s(p^{l-1}) is the saturation the constitutive pass computes at p
    RICH_CHECK(constit_eval(c, p));
    RICH_CUDA(cudaMemcpyAsync(c->s_old, c->S, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st));
    RICH_CHECK(residual_eval(c, p, c->s_old, dt, c->F, true, true));
  }
  RICH_CHECK(fetch_scalars(c, c->dsc, 3, h));
  double fn = sqrt(h[0]);
  double floor_ = kFloor * sqrt(h[2]);
  if (!std::isfinite(fn)) return RICH_ENONFINITE;
  st->res0 = st->res = fn;
  double tol = std::max(o->rtol * fn, o->atol);
  for (int r = 0;; ++r) {
    if (fn <= std::max(tol, floor_)) {
      st->converged = 1;
      break;
    }
    if (r == o->max_newton) return RICH_ENOTCONV_NEWTON;
    {
      Phase ph(pt, &st->ms_jacobian);
      // the last residual evaluation was at this p (the start or the accepted trial point)
      RICH_CHECK(jacobian_eval(c, p, dt, true));
    }
    bool rebuild = !c->H.built || (o->amg_policy == RICH_AMG_REBUILD_STEP && r == 0);
    {
      Phase ph(pt, &st->ms_setup);
      if (rebuild) {
        RICH_CHECK(amg_build(c, &o->amg));
        st->amg_setups++;
      } else {
        RICH_CHECK(o->amg_policy == RICH_AMG_SETUP_ONCE ? amg_update_fine(c) : amg_refresh(c));
        st->amg_refreshes++;
      }
    }
    k_scale<<<g, kBlock, 0, c->st>>>(n, c->F, -1.0, c->rhs);
    RICH_LAUNCH_CHECK();
    rich_krylov_stats ks;
    int lin_phase = pt.begin(&st->ms_linsol);
    int s = krylov_run(c, c->rhs, c->d, &o->krylov, &ks);
    st->linear_its += ks.iterations;
    // under time-step control, (p, J p) <= 0 in FCG ends the attempt: the step is retried shorter
    const bool indefinite = o->max_dt_halvings > 0 && c->kw.fail_reason == 2;
    if (s == RICH_ENOTCONV_LIN && o->krylov.kind == RICH_KRYLOV_FCG && !indefinite) {
      rich_krylov_opts fb = o->krylov;
      fb.kind = RICH_KRYLOV_FGMRES;
      fb.restart = o->fcg_fallback_restart;
      st->fallbacks++;
      s = krylov_run(c, c->rhs, c->d, &fb, &ks);
      st->linear_its += ks.iterations;
    }
    pt.end(lin_phase);
    if (s != RICH_OK) return s;
    // slope of f = 1/2 ||Phi||^2 along d: g = Phi . (J d)
    RICH_CHECK(stencil_apply(c, c->J7, c->d, c->Ft));
    RICH_CHECK(dot(c, c->F, c->Ft, n, c->dsc + 2));
    RICH_CHECK(fetch_scalars(c, c->dsc + 2, 1, h));
    double slope = h[0];
    if (!(slope < 0.0)) return RICH_ELINESEARCH;
    double f0 = 0.5 * fn * fn;
    double lam = 1.0, ft = 0.0, floor_t = 0.0;
    for (;;) {
      {
        Phase ph(pt, &st->ms_feval);
        k_axpby<<<g, kBlock, 0, c->st>>>(n, p, lam, c->d, c->ptrial);
        RICH_LAUNCH_CHECK();
        RICH_CHECK(residual_eval(c, c->ptrial, c->s_old, dt, c->Ft, true));
      }
      RICH_CHECK(fetch_scalars(c, c->dsc, 3, h));
      st->line_search_evals++;
      ft = 0.5 * h[0];
      floor_t = kFloor * sqrt(h[2]);
      if (!std::isfinite(ft)) return RICH_ENONFINITE;
      if (ft <= f0 + o->armijo_c * lam * slope) break;
      double lq = -slope * lam * lam / (2.0 * (ft - f0 - slope * lam));
      lam = std::min(std::max(lq, 0.1 * lam), 0.5 * lam);
      if (lam < o->lambda_min) return RICH_ELINESEARCH;
    }
    RICH_CUDA(cudaMemcpyAsync(p, c->ptrial, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st));
    std::swap(c->F, c->Ft);
    fn = sqrt(2.0 * ft);
    floor_ = floor_t;
    st->res = fn;
    st->newton_its++;
    st->min_lambda = std::min(st->min_lambda, lam);
  }
  return RICH_OK;
}

// Time-step control: cover dt with backward-Euler substeps of length dt / 2^k.  A
// substep that fails to converge is discarded (p restored) and retried with half
// its length, down to dt / 2^H; after an accepted substep the length doubles back
// whenever the time reached (counted in units of dt / 2^H) is a multiple of the
// doubled length, so the substeps end exactly at dt.
// A Krylov solve that merely ran out of iterations ends the step: a shorter step
// does not mend the preconditioner, and retrying would multiply the cost.  FCG's
// (p, J p) <= 0 on an indefinite Jacobian is retried.
static bool retryable(rich_ctx* c, int s) {
  if (s == RICH_ENOTCONV_NEWTON || s == RICH_ELINESEARCH) return true;
  return s == RICH_ENOTCONV_LIN && c->kw.fail_reason == 2;
}

static int advance_impl(rich_ctx* c, double* p, double dt, const rich_newton_opts* o, rich_step_stats* st) {
  const int H = o->max_dt_halvings;
  if (H > 40) return RICH_EINVAL;
  long long n = c->g.n;
  if (!c->psave) RICH_CHECK(dalloc(&c->psave, n));
  memset(st, 0, sizeof(*st));
  st->min_lambda = 1.0;
  st->dt_min = dt;
  const long long total = 1LL << H;
  long long t = 0;
  int k = 0;
  bool first = true;
  while (t < total) {
    const double h = std::ldexp(dt, -k);
    const long long len = 1LL << (H - k);
    RICH_CUDA(cudaMemcpyAsync(c->psave, p, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st));
    rich_step_stats sub;
    int s = step_impl(c, p, h, o, &sub);
    st->newton_its += sub.newton_its;
    st->linear_its += sub.linear_its;
    st->line_search_evals += sub.line_search_evals;
    st->fallbacks += sub.fallbacks;
    st->amg_setups += sub.amg_setups;
    st->amg_refreshes += sub.amg_refreshes;
    st->ms_feval += sub.ms_feval;
    st->ms_jacobian += sub.ms_jacobian;
    st->ms_setup += sub.ms_setup;
    st->ms_linsol += sub.ms_linsol;
    st->ms_total += sub.ms_total;
    if (first) st->res0 = sub.res0;
    first = false;
    st->res = sub.res;
    if (s != RICH_OK) {
      if (s != RICH_ECUDA)  // the substep's start is the last accepted state
        RICH_CUDA(cudaMemcpyAsync(p, c->psave, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st));
      if (!retryable(c, s)) return s;
      st->dt_failures++;
      if (k == H) return s;
      ++k;
      continue;
    }
    st->min_lambda = std::min(st->min_lambda, sub.min_lambda);
    t += len;
    st->substeps++;
    st->dt_min = std::min(st->dt_min, h);
    if (k > 0 && t % (2 * len) == 0) --k;
  }
  st->converged = 1;
  return RICH_OK;
}

}  // namespace rich

using namespace rich;

extern "C" {

int amg_vcycle(rich_ctx* c, const double* r, double* z) {
  if (!c || !r || !z) return RICH_EINVAL;
  AllocStream guard(c->st);
  return vcycle_apply(c, r, z);
}

int krylov_solve(rich_ctx* c, const double* b, double* x, const rich_krylov_opts* o, rich_krylov_stats* st) {
  if (!c || !b || !x || !o) return RICH_EINVAL;
  AllocStream guard(c->st);
  if (!c->have_jac || !c->H.built) return RICH_ESTATE;
  rich_krylov_stats tmp;
  return krylov_run(c, b, x, o, st ? st : &tmp);
}

int rich_step(rich_ctx* c, double* p, double dt, const rich_newton_opts* o, rich_step_stats* st) {
  if (!c || !p || !(dt > 0)) return RICH_EINVAL;
  AllocStream guard(c->st);
  rich_newton_opts def;
  if (!o) {
    rich_default_newton_opts(&def);
    o = &def;
  }
  rich_step_stats tmp;
  if (!st) st = &tmp;
  if (o->max_dt_halvings < 0) return RICH_EINVAL;
  if (o->max_dt_halvings > 0) return advance_impl(c, p, dt, o, st);
  int s = step_impl(c, p, dt, o, st);
  st->substeps = s == RICH_OK ? 1 : 0;
  st->dt_min = dt;
  return s;
}

int rich_step_host(rich_ctx* c, double* p_host, double dt, const rich_newton_opts* o, rich_step_stats* st) {
  if (!c || !p_host || !(dt > 0)) return RICH_EINVAL;
  AllocStream guard(c->st);
  long long n = c->g.n;
  if (!c->pbuf) RICH_CHECK(dalloc(&c->pbuf, n));
  RICH_CUDA(cudaMemcpyAsync(c->pbuf, p_host, sizeof(double) * n, cudaMemcpyHostToDevice, c->st));
  int s = rich_step(c, c->pbuf, dt, o, st);
  RICH_CUDA(cudaMemcpyAsync(p_host, c->pbuf, sizeof(double) * n, cudaMemcpyDeviceToHost, c->st));
  RICH_CUDA(cudaStreamSynchronize(c->st));
  return s;
}

}  // extern "C"
