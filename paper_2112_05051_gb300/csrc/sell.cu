// SELL-C-sigma copies of the coarse-level CSR matrices (the layout is described
// with struct Sell).  The pattern is laid out once per hierarchy: the row pointer
// comes to the host, rows are counting-sorted by decreasing length within each
// window of kSellSigma rows (ties keep their order, so the layout is a function of
// the pattern alone), and one kernel scatters the column indices into the slots.
// Values are gathered into the slots by a second kernel, again after every
// Galerkin refresh of the matrix.
#include <vector>

#include "common.cuh"

namespace rich {

// One thread per (slice, lane): columns of the lane's row into its slots, 0 past the row.
__global__ void k_sell_cols(int nslice, const int* __restrict__ sptr, const int* __restrict__ perm,
                            const int* __restrict__ rp, const int* __restrict__ col, int* __restrict__ scol) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)nslice * kSellC;
       t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t / kSellC), lane = (int)(t % kSellC);
    const int row = perm[t];
    const int base = sptr[s], w = (sptr[s + 1] - base) / kSellC;
    const int e0 = row >= 0 ? rp[row] : 0, len = row >= 0 ? rp[row + 1] - e0 : 0;
    for (int j = 0; j < w; ++j) scol[base + j * kSellC + lane] = j < len ? col[e0 + j] : 0;
  }
}

template <class T>
__global__ void k_sell_vals(int nslice, const int* __restrict__ sptr, const int* __restrict__ perm,
                            const int* __restrict__ rp, const T* __restrict__ val, T* __restrict__ sval) {
  for (long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x; t < (long long)nslice * kSellC;
       t += (long long)gridDim.x * blockDim.x) {
    const int s = (int)(t / kSellC), lane = (int)(t % kSellC);
    const int row = perm[t];
    const int base = sptr[s], w = (sptr[s + 1] - base) / kSellC;
    const int e0 = row >= 0 ? rp[row] : 0, len = row >= 0 ? rp[row + 1] - e0 : 0;
    for (int j = 0; j < w; ++j) sval[base + j * kSellC + lane] = j < len ? val[e0 + j] : T(0);
  }
}

// The layout of a SELL copy from the row pointer alone (host): perm (32 ns entries,
// -1 past n) and sptr (ns + 1 slot offsets).  Returns the slot count, or -1 when it
// exceeds 32-bit offsets.
long long sell_layout(const int* rp, int n, int* perm, int* sptr) {
  const int ns = (n + kSellC - 1) / kSellC;
  for (long long t = 0; t < (long long)ns * kSellC; ++t) perm[t] = -1;
  std::vector<int> cnt;
  for (int w0 = 0; w0 < n; w0 += kSellSigma) {
    const int w1 = std::min(n, w0 + kSellSigma);
    int lmax = 0;
    for (int i = w0; i < w1; ++i) lmax = std::max(lmax, rp[i + 1] - rp[i]);
    cnt.assign(lmax + 2, 0);  // counting sort, longest first: cnt[lmax - len + 1] counts len
    for (int i = w0; i < w1; ++i) cnt[lmax - (rp[i + 1] - rp[i]) + 1]++;
    for (int k = 1; k <= lmax + 1; ++k) cnt[k] += cnt[k - 1];
    for (int i = w0; i < w1; ++i) perm[w0 + cnt[lmax - (rp[i + 1] - rp[i])]++] = i;
  }
  long long slots = 0;
  for (int s = 0; s < ns; ++s) {  // a slice lies in one window, so its first row is its longest
    sptr[s] = (int)slots;
    const int r0 = perm[(size_t)s * kSellC];
    slots += (long long)kSellC * (rp[r0 + 1] - rp[r0]);
    if (slots > 2147483647LL) return -1;
  }
  sptr[ns] = (int)slots;
  return slots;
}

int sell_build(rich_ctx* c, const Csr<double>& M, Sell& S) {
  sell_free(S);
  const int n = M.nrows;
  if (n < kSellMinRows) return RICH_OK;
  std::vector<int> rp(n + 1);
  RICH_CUDA(cudaMemcpyAsync(rp.data(), M.rowptr, sizeof(int) * (n + 1), cudaMemcpyDeviceToHost, c->st));
  RICH_CUDA(cudaStreamSynchronize(c->st));
  const int ns = (n + kSellC - 1) / kSellC;
  std::vector<int> perm((size_t)ns * kSellC), sptr(ns + 1);
  const long long slots = sell_layout(rp.data(), n, perm.data(), sptr.data());
  if (slots < 0) return RICH_OK;  // too large for 32-bit slot offsets: CSR only
  RICH_CHECK(dalloc(&S.sptr, ns + 1));
  RICH_CHECK(dalloc(&S.perm, (long long)ns * kSellC));
  RICH_CHECK(dalloc(&S.col, slots));
  if (c->prec == RICH_PREC_MIXED) RICH_CHECK(dalloc(&S.val32, slots));
  else RICH_CHECK(dalloc(&S.val, slots));
  S.nrows = n;
  S.nslice = ns;
  S.slots = slots;
  RICH_CUDA(cudaMemcpyAsync(S.sptr, sptr.data(), sizeof(int) * (ns + 1), cudaMemcpyHostToDevice, c->st));
  RICH_CUDA(cudaMemcpyAsync(S.perm, perm.data(), sizeof(int) * perm.size(), cudaMemcpyHostToDevice, c->st));
  k_sell_cols<<<grid_for((long long)ns * kSellC), kBlock, 0, c->st>>>(ns, S.sptr, S.perm, M.rowptr, M.col, S.col);
  RICH_LAUNCH_CHECK();
  // the host vectors are read by the copies above before they go out of scope
  RICH_CUDA(cudaStreamSynchronize(c->st));
  return RICH_OK;
}

int sell_fill(rich_ctx* c, const Csr<double>& M, const double* val, Sell& S) {
  if (!S.built() || !S.val) return RICH_OK;
  k_sell_vals<double><<<grid_for((long long)S.nslice * kSellC), kBlock, 0, c->st>>>(S.nslice, S.sptr, S.perm,
                                                                                   M.rowptr, val, S.val);
  RICH_LAUNCH_CHECK();
  return RICH_OK;
}

int sell_fill(rich_ctx* c, const Csr<double>& M, const float* val, Sell& S) {
  if (!S.built() || !S.val32) return RICH_OK;
  k_sell_vals<float><<<grid_for((long long)S.nslice * kSellC), kBlock, 0, c->st>>>(S.nslice, S.sptr, S.perm,
                                                                                  M.rowptr, val, S.val32);
  RICH_LAUNCH_CHECK();
  return RICH_OK;
}

void sell_free(Sell& S) {
  dfree(S.sptr);
  dfree(S.perm);
  dfree(S.col);
  dfree(S.val);
  dfree(S.val32);
  S.nrows = S.nslice = 0;
  S.slots = 0;
}

}  // namespace rich

extern "C" int rich_sell_layout(const int* rowptr_host, int n, int* perm_host, int* sptr_host,
                                long long* slots) {
  if (!rowptr_host || n < 1 || !perm_host || !sptr_host || !slots) return RICH_EINVAL;
  for (int i = 0; i < n; ++i)
    if (rowptr_host[i + 1] < rowptr_host[i]) return RICH_EINVAL;
  const long long s = rich::sell_layout(rowptr_host, n, perm_host, sptr_host);
  if (s < 0) return RICH_ELIMIT;
  *slots = s;
  return RICH_OK;
}
