// Batched multi-vector solves (filled in by the batched engine).
#include "solver.cuh"

namespace fem {
fem_status pcg_multi(System& S, Hierarchy& H, const double* f, double* u, int nrhs,
                     const double* rho_k, const pcg_opts& o, cudaStream_t user, pcg_result* res) {
  (void)S; (void)H; (void)f; (void)u; (void)nrhs; (void)rho_k; (void)o; (void)user; (void)res;
  fail(FEM_EUNSUPPORTED, "pcg_solve: batched solves are not built yet");
}
}  // namespace fem

extern "C" {
fem_status pcg_batch_create(fem_system, amg_hier, int32_t, const pcg_opts*, void*, pcg_batch* out) {
  if (out) *out = nullptr;
  fem::set_last_error("pcg_batch_create: not built yet");
  return FEM_EUNSUPPORTED;
}
fem_status pcg_batch_admit(pcg_batch, const double*, double, int32_t*, void*) { return FEM_EUNSUPPORTED; }
fem_status pcg_batch_step(pcg_batch, int32_t, void*) { return FEM_EUNSUPPORTED; }
fem_status pcg_batch_poll(pcg_batch, int32_t*, int32_t*, double*, void*) { return FEM_EUNSUPPORTED; }
fem_status pcg_batch_retire(pcg_batch, int32_t, double*, void*) { return FEM_EUNSUPPORTED; }
int64_t pcg_batch_footprint(fem_system, amg_hier, int32_t) { return -1; }
void pcg_batch_destroy(pcg_batch) {}
const char* fem_autotune_report(void) { return "{}"; }
}
