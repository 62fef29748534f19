// Batched backward-Euler steps: several independent problems of one grid shape,
// stacked along z in one context, stepped with one launch per operation.
//
// The request server packs small queued requests this way.  The stacked grid has
// nb * nz layers; the faces between two stacked problems are the problems' own top
// and bottom faces (the residual and assembly kernels test z boundaries per
// problem), so every matrix is block diagonal and every problem sees exactly its
// own equations.  One kernel launch then evaluates the constitutive law, the
// residual, the Jacobian, the diffusion matrix, the stencil SpMV and each level
// operation of the V-cycle for all problems at once; the AMG hierarchy is built
// on the block-diagonal diffusion matrix (aggregates never cross problems: the
// couplings between them are zero, never strong).
//
// What stays per problem is everything with a scalar in it: the Newton iteration
// (norms, convergence test, line search with its own step length, statistics) and
// FCG (its own alpha, beta and stopping test).  Dot products are segmented: grid
// row y of a reduction kernel sums problem y, in the same fixed order for every
// problem.  A problem that has converged, or failed, is frozen: its Newton
// correction is zero and its Krylov scalars are not applied.  A batch has no
// FGMRES fallback: a problem whose FCG fails is reported RICH_ENOTCONV_LIN and the
// server reruns it alone on the ordinary path.
#include <algorithm>
#include <vector>

#include "common.cuh"

namespace rich {

constexpr int kMaxBatch = 32;

// partials[(q * S + s) * gridDim.x + block] of q = 0: a.b, q = 1: c.d (if c)
__global__ void k_seg_dot2(long long ns, const double* __restrict__ a, const double* __restrict__ b,
                           const double* __restrict__ cc, const double* __restrict__ d, double* __restrict__ part) {
  const int S = gridDim.y, s = blockIdx.y;
  const long long base = (long long)s * ns;
  double v[2] = {0.0, 0.0};
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ns; i += (long long)gridDim.x * blockDim.x) {
    v[0] += a[base + i] * b[base + i];
    if (cc) v[1] += cc[base + i] * d[base + i];
  }
  block_sum<2>(v);
  if (threadIdx.x == 0) {
    part[(long long)s * gridDim.x + blockIdx.x] = v[0];
    part[((long long)S + s) * gridDim.x + blockIdx.x] = v[1];
  }
}

// p_s = z_s - (sc[num + s] / sc[den + s]) p_s for active problems
__global__ void k_seg_fcg_dir(long long ns, const double* __restrict__ z, double* __restrict__ p,
                              const double* __restrict__ sc, int num, int den, const int* __restrict__ act) {
  const int s = blockIdx.y;
  if (!act[s]) return;
  const long long base = (long long)s * ns;
  const double beta = sc[num + s] / sc[den + s];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ns; i += (long long)gridDim.x * blockDim.x)
    p[base + i] = z[base + i] - beta * p[base + i];
}

// b_s = a_s for active problems
__global__ void k_seg_copy(long long ns, const double* __restrict__ a, double* __restrict__ b,
                           const int* __restrict__ act) {
  const int s = blockIdx.y;
  if (!act[s]) return;
  const long long base = (long long)s * ns;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ns; i += (long long)gridDim.x * blockDim.x)
    b[base + i] = a[base + i];
}

// active problems: alpha = sc[num + s] / sc[den + s]; x += alpha p; r -= alpha q;
// partials of ||r_s||^2 (zero for frozen problems)
__global__ void k_seg_fcg_update(long long ns, double* __restrict__ x, double* __restrict__ r,
                                 const double* __restrict__ p, const double* __restrict__ q,
                                 const double* __restrict__ sc, int num, int den, const int* __restrict__ act,
                                 double* __restrict__ part) {
  const int s = blockIdx.y;
  const long long base = (long long)s * ns;
  double v[1] = {0.0};
  if (act[s]) {
    const double alpha = sc[num + s] / sc[den + s];
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ns;
         i += (long long)gridDim.x * blockDim.x) {
      x[base + i] += alpha * p[base + i];
      double ri = r[base + i] - alpha * q[base + i];
      r[base + i] = ri;
      v[0] += ri * ri;
    }
  }
  block_sum<1>(v);
  if (threadIdx.x == 0) part[(long long)s * gridDim.x + blockIdx.x] = v[0];
}

// y_s = a_s + lam[s] d_s
__global__ void k_seg_axpby(long long ns, const double* __restrict__ a, const double* __restrict__ lam,
                            const double* __restrict__ d, double* __restrict__ y) {
  const int s = blockIdx.y;
  const long long base = (long long)s * ns;
  const double l = lam[s];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ns; i += (long long)gridDim.x * blockDim.x)
    y[base + i] = a[base + i] + l * d[base + i];
}

// y_s = -x_s for active problems, 0 for the others
__global__ void k_seg_neg(long long ns, const double* __restrict__ x, const int* __restrict__ act,
                          double* __restrict__ y) {
  const int s = blockIdx.y;
  const long long base = (long long)s * ns;
  const bool a = act[s] != 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < ns; i += (long long)gridDim.x * blockDim.x)
    y[base + i] = a ? -x[base + i] : 0.0;
}

struct BatchWork {
  double* dsc = nullptr;   // device scalars, 8 per problem
  int* dact = nullptr;     // device activity flags
  double* dlam = nullptr;  // device step lengths
  double* hsc = nullptr;   // pinned host mirror (256 doubles)
  int* hact = nullptr;     // pinned host flags (kMaxBatch)
};

static int batch_work(rich_ctx* c, BatchWork& w, int S) {
  RICH_CHECK(dalloc(&w.dsc, 8LL * S));
  RICH_CHECK(dalloc(&w.dact, S));
  RICH_CHECK(dalloc(&w.dlam, S));
  char* blk = static_cast<char*>(pinned_get());
  if (!blk) return RICH_ENOMEM;
  w.hsc = reinterpret_cast<double*>(blk);
  char* blk2 = static_cast<char*>(pinned_get());
  if (!blk2) return RICH_ENOMEM;
  w.hact = reinterpret_cast<int*>(blk2);
  (void)c;
  return RICH_OK;
}

static void batch_free(BatchWork& w) {
  dfree(w.dsc);
  dfree(w.dact);
  dfree(w.dlam);
  if (w.hsc) pinned_put(w.hsc);
  if (w.hact) pinned_put(w.hact);
  w.hsc = nullptr;
  w.hact = nullptr;
}

// q quantities per problem, summed from block partials into dsc[q * S + s], copied to host
static int seg_finish(rich_ctx* c, const double* part, int nb, int q, int S, double* dst_dev, double* host) {
  RICH_CHECK(finish_sums(c, part, nb, q * S, dst_dev));
  RICH_CUDA(cudaMemcpyAsync(host, dst_dev, sizeof(double) * q * S, cudaMemcpyDeviceToHost, c->st));
  RICH_CUDA(cudaStreamSynchronize(c->st));
  return RICH_OK;
}

static int upload_flags(rich_ctx* c, BatchWork& w, const std::vector<int>& a) {
  for (size_t s = 0; s < a.size(); ++s) w.hact[s] = a[s];
  RICH_CUDA(cudaMemcpyAsync(w.dact, w.hact, sizeof(int) * a.size(), cudaMemcpyHostToDevice, c->st));
  return RICH_OK;
}

// Segmented FCG (Notay, truncation 1) for J x = b with x0 = 0.  Problems with
// active[s] == 0 on entry keep x_s = 0.  On return fail[s] = 1 where FCG stopped
// on (p, q) <= 0, on residual growth, on stagnation (krylov.stall) or at maxit;
// its[s] counts the iterations.
static int batch_fcg(rich_ctx* c, BatchWork& w, int S, const double* b, double* x, const rich_krylov_opts* o,
                     std::vector<int> active, std::vector<int>& fail, std::vector<int>& its) {
  KrylovWork& k = c->kw;
  const long long ns = c->g.n / S;
  const int nb = red_grid(ns);
  const dim3 grid(nb, S), vgrid(grid_for(ns), S);
  double* sc = w.dsc;  // [0] rr, [1] zq, [2] pq, [3] pr, [4] pq_prev (each S wide)
  fail.assign(S, 0);
  its.assign(S, 0);
  RICH_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * c->g.n, c->st));
  RICH_CUDA(cudaMemcpyAsync(k.r, b, sizeof(double) * c->g.n, cudaMemcpyDeviceToDevice, c->st));
  k_seg_dot2<<<grid, kBlock, 0, c->st>>>(ns, b, b, nullptr, nullptr, c->partials);
  RICH_LAUNCH_CHECK();
  RICH_CHECK(seg_finish(c, c->partials, nb, 1, S, sc, w.hsc));
  std::vector<double> target(S), best(S), window_start(S);
  for (int s = 0; s < S; ++s) {
    double bn = sqrt(w.hsc[s]);
    if (!std::isfinite(bn)) return RICH_ENONFINITE;
    if (!(bn > 0)) active[s] = 0;
    target[s] = o->eta * bn;
    best[s] = bn;
    window_start[s] = bn;
  }
  double* q = k.q;
  double* qprev = k.qprev;
  for (int it = 1; it <= o->maxit; ++it) {
    if (std::none_of(active.begin(), active.end(), [](int a) { return a != 0; })) break;
    RICH_CHECK(upload_flags(c, w, active));
    RICH_CHECK(vcycle_apply(c, k.r, k.z));
    if (it == 1) {
      k_seg_copy<<<vgrid, kBlock, 0, c->st>>>(ns, k.z, k.p, w.dact);
    } else {
      k_seg_dot2<<<grid, kBlock, 0, c->st>>>(ns, k.z, qprev, nullptr, nullptr, c->partials);
      RICH_LAUNCH_CHECK();
      RICH_CHECK(finish_sums(c, c->partials, nb, S, sc + 1 * S));
      k_seg_fcg_dir<<<vgrid, kBlock, 0, c->st>>>(ns, k.z, k.p, sc, 1 * S, 4 * S, w.dact);
    }
    RICH_LAUNCH_CHECK();
    RICH_CHECK(stencil_apply(c, c->J7, k.p, q));
    k_seg_dot2<<<grid, kBlock, 0, c->st>>>(ns, k.p, q, k.p, k.r, c->partials);
    RICH_LAUNCH_CHECK();
    RICH_CHECK(finish_sums(c, c->partials, nb, 2 * S, sc + 2 * S));  // pq at 2S, pr at 3S
    k_seg_fcg_update<<<grid, kBlock, 0, c->st>>>(ns, x, k.r, k.p, q, sc, 3 * S, 2 * S, w.dact, c->partials);
    RICH_LAUNCH_CHECK();
    RICH_CHECK(finish_sums(c, c->partials, nb, S, sc + 0));
    RICH_CUDA(cudaMemcpyAsync(sc + 4 * S, sc + 2 * S, sizeof(double) * S, cudaMemcpyDeviceToDevice, c->st));
    RICH_CUDA(cudaMemcpyAsync(w.hsc, sc, sizeof(double) * 4 * S, cudaMemcpyDeviceToHost, c->st));
    RICH_CUDA(cudaStreamSynchronize(c->st));
    for (int s = 0; s < S; ++s) {
      if (!active[s]) continue;
      double rn = sqrt(w.hsc[s]), pq = w.hsc[2 * S + s];
      its[s] = it;
      if (!std::isfinite(rn) || !std::isfinite(pq)) return RICH_ENONFINITE;
      if (!(pq > 0) || rn > 10.0 * best[s]) {  // the update applied: x is no better than before; stop here
        fail[s] = 1;
        active[s] = 0;
        continue;
      }
      if (rn <= target[s]) {
        active[s] = 0;
        continue;
      }
      if (it % kStallWindow == 0) {  // stagnation over the last window (krylov.stall)
        if (o->stall > 0 && rn > (1.0 - o->stall) * window_start[s]) {
          fail[s] = 1;
          active[s] = 0;
          continue;
        }
        window_start[s] = rn;
      }
      best[s] = std::min(best[s], rn);
    }
    std::swap(q, qprev);
  }
  for (int s = 0; s < S; ++s)
    if (active[s]) fail[s] = 1;  // maxit
  return RICH_OK;
}

static int ensure_newton_batch(rich_ctx* c) {
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

static int ensure_krylov_batch(rich_ctx* c) {
  KrylovWork& k = c->kw;
  long long n = c->g.n;
  if (k.n == n) return RICH_OK;
  RICH_CHECK(dalloc(&k.x, n));
  RICH_CHECK(dalloc(&k.r, n));
  RICH_CHECK(dalloc(&k.p, n));
  RICH_CHECK(dalloc(&k.q, n));
  RICH_CHECK(dalloc(&k.qprev, n));
  RICH_CHECK(dalloc(&k.z, n));
  RICH_CHECK(dalloc(&k.w, n));
  RICH_CHECK(dalloc(&k.hcoef, 128));
  k.n = n;
  return RICH_OK;
}

// The Newton-Armijo step of every problem (Sec. 3), with the constants and the
// convergence test of the lone step, per problem.
static int batch_step(rich_ctx* c, BatchWork& w, int S, double* p, double dt, const rich_newton_opts* o,
                      rich_step_stats* st, int* status) {
  const long long n = c->g.n, ns = n / S;
  const int nb = red_grid(ns);
  const dim3 grid(nb, S), vgrid(grid_for(ns), S);
  const double kFloor = 2.220446049250313e-16;
  RICH_CHECK(ensure_newton_batch(c));
  RICH_CHECK(ensure_krylov_batch(c));
  cudaEvent_t e0, e1;
  RICH_CUDA(cudaEventCreate(&e0));
  RICH_CUDA(cudaEventCreate(&e1));
  RICH_CUDA(cudaEventRecord(e0, c->st));
  for (int s = 0; s < S; ++s) {
    memset(&st[s], 0, sizeof(rich_step_stats));
    st[s].min_lambda = 1.0;
    st[s].dt_min = dt;
    status[s] = RICH_OK;
  }
  std::vector<double> fn(S), tol(S), flo(S), f0(S), slope(S), lam(S), ft(S), flo_t(S);
  std::vector<int> conv(S, 0), done(S, 0), newton_act(S, 0), search(S, 0), lin_fail, lin_its;
  RICH_CHECK(constit_eval(c, p));
  RICH_CUDA(cudaMemcpyAsync(c->s_old, c->S, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st));
  RICH_CHECK(residual_eval(c, p, c->s_old, dt, c->F, true, true, S));
  RICH_CUDA(cudaMemcpyAsync(w.hsc, c->dsc, sizeof(double) * 3 * S, cudaMemcpyDeviceToHost, c->st));
  RICH_CUDA(cudaStreamSynchronize(c->st));
  for (int s = 0; s < S; ++s) {
    fn[s] = sqrt(w.hsc[s]);
    flo[s] = kFloor * sqrt(w.hsc[2 * S + s]);
    if (!std::isfinite(fn[s])) return RICH_ENONFINITE;
    st[s].res0 = st[s].res = fn[s];
    tol[s] = std::max(o->rtol * fn[s], o->atol);
  }
  for (int r = 0;; ++r) {
    bool any = false;
    for (int s = 0; s < S; ++s) {
      newton_act[s] = 0;
      if (done[s]) continue;
      if (fn[s] <= std::max(tol[s], flo[s])) {
        conv[s] = done[s] = 1;
        st[s].converged = 1;
        continue;
      }
      if (r == o->max_newton) {
        done[s] = 1;
        status[s] = RICH_ENOTCONV_NEWTON;
        continue;
      }
      newton_act[s] = 1;
      any = true;
    }
    if (!any) break;
    RICH_CHECK(jacobian_eval(c, p, dt, true));
    if (!c->H.built) {
      RICH_CHECK(amg_build(c, &o->amg));
      for (int s = 0; s < S; ++s) st[s].amg_setups++;
    } else {
      RICH_CHECK(amg_refresh(c));
      for (int s = 0; s < S; ++s) st[s].amg_refreshes += newton_act[s];
    }
    // correction J d = -Phi for the active problems (0 for the others)
    RICH_CHECK(upload_flags(c, w, newton_act));
    k_seg_neg<<<vgrid, kBlock, 0, c->st>>>(ns, c->F, w.dact, c->rhs);
    RICH_LAUNCH_CHECK();
    RICH_CHECK(batch_fcg(c, w, S, c->rhs, c->d, &o->krylov, newton_act, lin_fail, lin_its));
    for (int s = 0; s < S; ++s) {
      st[s].linear_its += lin_its[s];
      if (newton_act[s] && lin_fail[s]) {
        newton_act[s] = 0;
        done[s] = 1;
        status[s] = RICH_ENOTCONV_LIN;
      }
    }
    // slopes g_s = Phi_s . (J d)_s; problems that failed keep d_s out of the step
    RICH_CHECK(stencil_apply(c, c->J7, c->d, c->Ft));
    k_seg_dot2<<<grid, kBlock, 0, c->st>>>(ns, c->F, c->Ft, nullptr, nullptr, c->partials);
    RICH_LAUNCH_CHECK();
    RICH_CHECK(seg_finish(c, c->partials, nb, 1, S, w.dsc, w.hsc));
    for (int s = 0; s < S; ++s) {
      slope[s] = w.hsc[s];
      search[s] = 0;
      lam[s] = 0.0;
      if (!newton_act[s]) continue;
      if (!(slope[s] < 0.0)) {
        done[s] = 1;
        status[s] = RICH_ELINESEARCH;
        continue;
      }
      f0[s] = 0.5 * fn[s] * fn[s];
      lam[s] = 1.0;
      search[s] = 1;
    }
    // line search: every problem still searching tries its own step length
    for (;;) {
      for (int s = 0; s < S; ++s) w.hsc[s] = lam[s];
      RICH_CUDA(cudaMemcpyAsync(w.dlam, w.hsc, sizeof(double) * S, cudaMemcpyHostToDevice, c->st));
      k_seg_axpby<<<vgrid, kBlock, 0, c->st>>>(ns, p, w.dlam, c->d, c->ptrial);
      RICH_LAUNCH_CHECK();
      RICH_CHECK(residual_eval(c, c->ptrial, c->s_old, dt, c->Ft, true, false, S));
      RICH_CUDA(cudaMemcpyAsync(w.hsc, c->dsc, sizeof(double) * 3 * S, cudaMemcpyDeviceToHost, c->st));
      RICH_CUDA(cudaStreamSynchronize(c->st));
      bool more = false;
      for (int s = 0; s < S; ++s) {
        ft[s] = 0.5 * w.hsc[s];
        flo_t[s] = kFloor * sqrt(w.hsc[2 * S + s]);
        if (!search[s]) continue;
        st[s].line_search_evals++;
        if (!std::isfinite(ft[s])) return RICH_ENONFINITE;
        if (ft[s] <= f0[s] + o->armijo_c * lam[s] * slope[s]) {
          search[s] = 0;
          continue;
        }
        double lq = -slope[s] * lam[s] * lam[s] / (2.0 * (ft[s] - f0[s] - slope[s] * lam[s]));
        lam[s] = std::min(std::max(lq, 0.1 * lam[s]), 0.5 * lam[s]);
        if (lam[s] < o->lambda_min) {
          search[s] = 0;
          lam[s] = 0.0;  // the trial of the next evaluation is p itself
          done[s] = 1;
          status[s] = RICH_ELINESEARCH;
          newton_act[s] = 0;
          more = true;  // re-evaluate so that the accepted state of every problem is consistent
          continue;
        }
        more = true;
      }
      if (!more) break;
    }
    // accept: p <- p + lam d (lam = 0 for problems that did not step); F <- Phi(p)
    RICH_CUDA(cudaMemcpyAsync(p, c->ptrial, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->st));
    std::swap(c->F, c->Ft);
    for (int s = 0; s < S; ++s) {
      fn[s] = sqrt(2.0 * ft[s]);
      flo[s] = flo_t[s];
      if (!newton_act[s]) continue;
      st[s].res = fn[s];
      st[s].newton_its++;
      st[s].min_lambda = std::min(st[s].min_lambda, lam[s]);
    }
  }
  RICH_CUDA(cudaEventRecord(e1, c->st));
  RICH_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  for (int s = 0; s < S; ++s) {
    st[s].ms_total = ms;  // the batch's device time, shared by its problems
    st[s].substeps = status[s] == RICH_OK ? 1 : 0;
  }
  return RICH_OK;
}

}  // namespace rich

using namespace rich;

extern "C" {

int rich_create_batch(const rich_grid* grid, int nbatch, const rich_soil* soil, int kmean, const rich_bc* bc,
                      int precision, void* stream, rich_ctx** out) {
  if (!grid || !soil || !bc || !out || nbatch < 1 || nbatch > kMaxBatch) return RICH_EINVAL;
  if (grid->nz < 1) return RICH_EINVAL;
  for (int f = 0; f < 4; ++f)  // per-cell values on x and y faces are indexed by layer: one problem only
    if (bc->value_field_dev[f]) return RICH_EINVAL;
  for (int f = 0; f < 6; ++f)  // stacked problems are whole grids, not subdomains
    if (bc->kind[f] == RICH_BC_INTERFACE) return RICH_EINVAL;
  rich_grid g = *grid;
  double hs[3];
  grid_spacing(grid, hs);
  const double hz = hs[2];
  g.nz = grid->nz * nbatch;
  g.lz = hz * (g.nz + 1);  // the stacked grid keeps the problems' spacing
  int s = rich_create(&g, soil, kmean, bc, precision, stream, out);
  if (s != RICH_OK) return s;
  (*out)->g.nzs = grid->nz;
  (*out)->g.inv_h[2] = 1.0 / hz;
  (*out)->g.inv_h2[2] = 1.0 / (hz * hz);
  (*out)->nbatch = nbatch;
  return RICH_OK;
}

int rich_step_batch(rich_ctx* c, double* p, double dt, const rich_newton_opts* o, rich_step_stats* stats,
                    int* status) {
  if (!c || !p || !(dt > 0) || !stats || !status) return RICH_EINVAL;
  AllocStream guard(c->st);
  rich_newton_opts def;
  if (!o) {
    rich_default_newton_opts(&def);
    o = &def;
  }
  if (o->krylov.kind != RICH_KRYLOV_FCG || o->max_dt_halvings != 0) return RICH_EINVAL;
  const int S = c->nbatch;
  if (S < 1 || c->g.n % S) return RICH_EINVAL;
  // every segmented reduction writes at most 3 quantities x S problems x its blocks of partials
  if (3LL * S * red_grid(c->g.n / S) > (long long)kRedBlocks * 64) return RICH_ELIMIT;
  BatchWork w;
  int rc = batch_work(c, w, S);
  if (rc == RICH_OK) rc = batch_step(c, w, S, p, dt, o, stats, status);
  batch_free(w);
  return rc;
}

}  // extern "C"
