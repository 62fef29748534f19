#include "common.cuh"
namespace rich {
int vcycle_apply(rich_ctx* c, const double* r, double* z) { return RICH_ESTATE; }
int krylov_run(rich_ctx* c, const double* b, double* x, const rich_krylov_opts* o, rich_krylov_stats* st) { return RICH_ESTATE; }
}
extern "C" {
int amg_setup(rich_ctx* c, const rich_amg_opts* o, rich_amg_info* info) { return RICH_ESTATE; }
int amg_update(rich_ctx* c, int policy) { return RICH_ESTATE; }
int amg_vcycle(rich_ctx* c, const double* r, double* z) { return RICH_ESTATE; }
int amg_export_level(rich_ctx* c, int level, int* agg, int* rp, int* col, double* val) { return RICH_ESTATE; }
int amg_export_prolongator(rich_ctx* c, int level, long long* nnz, int* rp, int* col, double* val) { return RICH_ESTATE; }
int krylov_solve(rich_ctx* c, const double* b, double* x, const rich_krylov_opts* o, rich_krylov_stats* st) { return RICH_ESTATE; }
int rich_step(rich_ctx* c, double* p, double dt, const rich_newton_opts* o, rich_step_stats* st) { return RICH_ESTATE; }
int rich_step_host(rich_ctx* c, double* p, double dt, const rich_newton_opts* o, rich_step_stats* st) { return RICH_ESTATE; }
}
