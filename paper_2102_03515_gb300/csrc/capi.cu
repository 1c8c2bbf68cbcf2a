// extern "C" entry points of include/femamg.h: argument checks, handles, and the
// translation of internal failures into fem_status codes with a per-thread message.
#include <atomic>
#include <cmath>
#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include "solver.cuh"

namespace fem {

static thread_local std::string g_last_error;
static std::atomic<long long> g_launches{0};

Tracer::Tracer(cudaStream_t s) : st(s) {
  const char* e = std::getenv("FEM_TRACE");
  on = e && e[0] == '1';
  if (on) {
    cudaStreamSynchronize(st);
    t = std::chrono::duration<double, std::milli>(
            std::chrono::steady_clock::now().time_since_epoch()).count();
  }
}

void Tracer::mark(const char* what) {
  if (!on) return;
  cudaStreamSynchronize(st);
  double now = std::chrono::duration<double, std::milli>(
                   std::chrono::steady_clock::now().time_since_epoch()).count();
  std::fprintf(stderr, "[fem] %-40s %9.3f ms\n", what, now - t);
  t = now;
}

void init_memory_pool() {
  static bool done = false;
  if (done) return;
  int dev = 0;
  FEM_CUDA(cudaGetDevice(&dev));
  cudaMemPool_t pool;
  FEM_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t thr = UINT64_MAX;
  FEM_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
  done = true;
}

cudaStream_t& current_alloc_stream() {
  static thread_local cudaStream_t s = nullptr;
  return s;
}

void count_launches(long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }
long long launches_now() { return g_launches.load(std::memory_order_relaxed); }

void set_last_error(const std::string& msg) { g_last_error = msg; }

[[noreturn]] void fail(fem_status s, const std::string& msg) { throw Error{s, msg}; }

void alloc_level_vectors(Hierarchy& H);
void pcg_single(System& S, Hierarchy* H, const double* f, double* u, const pcg_opts& o,
                cudaStream_t user, pcg_result& res);
fem_status pcg_multi(System& S, Hierarchy& H, const double* f, double* u, int nrhs,
                     const double* rho_k, const pcg_opts& o, cudaStream_t user, pcg_result* res);

template <typename F>
static fem_status guarded(F&& f) {
  try {
    g_last_error.clear();
    return f();
  } catch (const Error& e) {
    g_last_error = e.msg;
    return e.status;
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return FEM_ENOMEM;
  } catch (const std::exception& e) {
    g_last_error = e.what();
    return FEM_EINVAL;
  }
}

}  // namespace fem

struct fem_system_s {
  fem::System S;
};
struct amg_hier_s {
  fem::Hierarchy H;
  fem_system_s* sys = nullptr;
};
struct fem_mesh_s {
  fem::Mesh M;
};
struct pcg_batch_s {
  fem::BatchSession* W = nullptr;
  fem_system_s* sys = nullptr;
};

using namespace fem;

static cudaStream_t as_stream(void* s) { return reinterpret_cast<cudaStream_t>(s); }

extern "C" {

const char* fem_last_error(void) { return g_last_error.c_str(); }

const char* fem_version(void) { return "femamg 0.1 (sm_103a)"; }

fem_status fem_measure_fp64_rate(int32_t reps, void* stream, double* tflops_out) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(tflops_out && reps >= 1, FEM_EINVAL, "fem_measure_fp64_rate: bad argument");
    StreamScope scope(as_stream(stream));
    *tflops_out = fp64_fma_rate(reps, as_stream(stream));
    return FEM_OK;
  });
}

int64_t fem_kernel_launches(void) { return (int64_t)launches_now(); }

fem_status fem_assemble(const fem_kuhn_desc* mesh, double rho, const fem_target* target,
                        const fem_assemble_opts* opts, void* stream, fem_system* out) {
  return guarded([&]() -> fem_status {
    StreamScope scope(as_stream(stream));
    FEM_REQUIRE(mesh && target && out, FEM_EINVAL, "fem_assemble: null argument");
    *out = nullptr;
    fem_assemble_opts o{FEM_FMT_AUTO, 0};
    if (opts) o = *opts;
    init_memory_pool();
    auto* h = new fem_system_s();
    try {
      assemble_system(h->S, *mesh, rho, *target, o, as_stream(stream));
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
    return FEM_OK;
  });
}

fem_status fem_assemble_mesh(const fem_mesh_desc* mesh, double rho, const fem_target* target,
                             const fem_assemble_opts* opts, void* stream, fem_system* out) {
  return guarded([&]() -> fem_status {
    StreamScope scope(as_stream(stream));
    FEM_REQUIRE(mesh && target && out, FEM_EINVAL, "fem_assemble_mesh: null argument");
    *out = nullptr;
    fem_assemble_opts o{FEM_FMT_AUTO, 0};
    if (opts) o = *opts;
    init_memory_pool();
    auto* h = new fem_system_s();
    try {
      assemble_mesh(h->S, *mesh, rho, *target, o, as_stream(stream));
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
    return FEM_OK;
  });
}

fem_status fem_system_get_info(fem_system sys, fem_system_info* info) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(sys && info, FEM_EINVAL, "fem_system_get_info: null argument");
    const System& S = sys->S;
    info->n = S.n;
    info->N = S.N;
    info->nnz = S.A.nnz;
    info->h = S.h;
    info->rho = S.rho;
    info->is_stencil = S.stencil;
    info->has_pencil = S.pencil;
    return FEM_OK;
  });
}

fem_status fem_assemble_rhs(fem_system sys, const fem_target* target, double* f_dev,
                            void* stream) {
  return guarded([&]() -> fem_status {
    StreamScope scope(as_stream(stream));
    FEM_REQUIRE(sys && target && f_dev, FEM_EINVAL, "fem_assemble_rhs: null argument");
    assemble_rhs(sys->S, *target, f_dev, as_stream(stream));
    return FEM_OK;
  });
}

fem_status fem_assemble_rhs_noalloc(fem_system sys, const fem_target* target, double* f_dev,
                                    void* stream) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(sys && target && f_dev, FEM_EINVAL, "fem_assemble_rhs_noalloc: null argument");
    assemble_rhs_noalloc(sys->S, *target, f_dev, as_stream(stream));
    return FEM_OK;
  });
}

fem_status fem_errors(fem_system sys, const double* u_dev, const fem_target* target,
                      double scale, int32_t qlevel, void* stream, fem_errors_result* out) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(sys && u_dev && target && out, FEM_EINVAL, "fem_errors: null argument");
    StreamScope scope(as_stream(stream));
    double r[2] = {0.0, 0.0};
    fem_error_norms(sys->S, u_dev, *target, scale, qlevel, r, as_stream(stream));
    out->l2sq = r[0];
    out->h1sq = r[1];
    return FEM_OK;
  });
}

fem_status fem_recover(fem_system sys, const double* u_dev, const fem_target* target,
                       double* z_dev, double* p_dev, void* stream) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(sys && u_dev && target, FEM_EINVAL, "fem_recover: null argument");
    StreamScope scope(as_stream(stream));
    fem_recovery(sys->S, u_dev, *target, z_dev, p_dev, as_stream(stream));
    return FEM_OK;
  });
}

fem_status fem_error_indicator(fem_system sys, const double* u_dev, const fem_target* target,
                               int32_t qlevel, double* eta2_dev, void* stream, double* total) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(sys && u_dev && target && eta2_dev, FEM_EINVAL,
                "fem_error_indicator: null argument");
    StreamScope scope(as_stream(stream));
    const double s = error_indicator(sys->S, u_dev, *target, qlevel, eta2_dev, as_stream(stream));
    if (total) *total = s;
    return FEM_OK;
  });
}

fem_status fem_mark_bulk(const double* eta2_dev, int64_t n, double theta, uint8_t* mark_dev,
                         void* stream, double* threshold, int64_t* nmarked) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(eta2_dev && mark_dev, FEM_EINVAL, "fem_mark_bulk: null argument");
    StreamScope scope(as_stream(stream));
    mark_bulk(eta2_dev, n, theta, mark_dev, as_stream(stream), threshold, nmarked);
    return FEM_OK;
  });
}

fem_status fem_mesh_create(const fem_mesh_desc* mesh, void* stream, fem_mesh* out) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(mesh && out, FEM_EINVAL, "fem_mesh_create: null argument");
    *out = nullptr;
    StreamScope scope(as_stream(stream));
    init_memory_pool();
    auto* h = new fem_mesh_s();
    try {
      mesh_create(h->M, *mesh, as_stream(stream));
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
    return FEM_OK;
  });
}

fem_status fem_mesh_get_info(fem_mesh m, fem_mesh_info* info) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(m && info, FEM_EINVAL, "fem_mesh_get_info: null argument");
    info->nv = m->M.nv;
    info->nt = m->M.nt;
    return FEM_OK;
  });
}

fem_status fem_mesh_download(fem_mesh m, double* xyz, int32_t* tet, uint8_t* dirichlet,
                             void* stream) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(m, FEM_EINVAL, "fem_mesh_download: null mesh");
    cudaStream_t st = as_stream(stream);
    const Mesh& M = m->M;
    if (xyz) FEM_CUDA(cudaMemcpyAsync(xyz, M.xyz, 24 * M.nv, cudaMemcpyDeviceToHost, st));
    if (tet) FEM_CUDA(cudaMemcpyAsync(tet, M.tet, 16 * M.nt, cudaMemcpyDeviceToHost, st));
    if (dirichlet) FEM_CUDA(cudaMemcpyAsync(dirichlet, M.dir, M.nv, cudaMemcpyDeviceToHost, st));
    FEM_CUDA(cudaStreamSynchronize(st));
    return FEM_OK;
  });
}

fem_status fem_mesh_refine(fem_mesh m, const uint8_t* mark_dev, void* stream,
                           fem_refine_stats* stats) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(m && mark_dev, FEM_EINVAL, "fem_mesh_refine: null argument");
    StreamScope scope(as_stream(stream));
    fem_refine_stats r{0, 0, 0};
    mesh_refine(m->M, mark_dev, as_stream(stream), r);
    if (stats) *stats = r;
    return FEM_OK;
  });
}

fem_status fem_assemble_on_mesh(fem_mesh m, double rho, const fem_target* target,
                                const fem_assemble_opts* opts, void* stream, fem_system* out) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(m && target && out, FEM_EINVAL, "fem_assemble_on_mesh: null argument");
    *out = nullptr;
    StreamScope scope(as_stream(stream));
    fem_assemble_opts o{FEM_FMT_AUTO, 0};
    if (opts) o = *opts;
    init_memory_pool();
    auto* h = new fem_system_s();
    try {
      assemble_mesh_dev(h->S, m->M.nv, m->M.nt, m->M.xyz, m->M.tet, m->M.dir, rho, *target, o,
                        as_stream(stream));
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
    return FEM_OK;
  });
}

void fem_mesh_destroy(fem_mesh m) { delete m; }

fem_status fem_system_dof_vertices(fem_system sys, int64_t* vert_dev, void* stream) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(sys && vert_dev, FEM_EINVAL, "fem_system_dof_vertices: null argument");
    StreamScope scope(as_stream(stream));
    dof_vertices(sys->S, vert_dev, as_stream(stream));
    return FEM_OK;
  });
}

fem_status fem_system_get_rhs(fem_system sys, double* f_dev, void* stream) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(sys && f_dev, FEM_EINVAL, "fem_system_get_rhs: null argument");
    FEM_CUDA(cudaMemcpyAsync(f_dev, sys->S.f, 8 * sys->S.N, cudaMemcpyDeviceToDevice,
                             as_stream(stream)));
    FEM_CUDA(cudaStreamSynchronize(as_stream(stream)));
    return FEM_OK;
  });
}

fem_status fem_system_export(fem_system sys, int32_t which, int32_t* rowptr_dev, int32_t* col_dev,
                             double* val_dev, void* stream) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(sys && rowptr_dev && col_dev && val_dev, FEM_EINVAL,
                "fem_system_export: null argument");
    const System& S = sys->S;
    const double* v = nullptr;
    if (which == 0) v = S.A.val;
    else if (which == 1) v = S.Kv.p;
    else if (which == 2) v = S.Mv.p;
    FEM_REQUIRE(which >= 0 && which <= 2, FEM_EINVAL, "fem_system_export: which must be 0, 1, 2");
    FEM_REQUIRE(v, FEM_EINVAL, "fem_system_export: K and M need keep_pencil at assembly");
    cudaStream_t st = as_stream(stream);
    FEM_CUDA(cudaMemcpyAsync(rowptr_dev, S.A.rowptr, 4 * (S.N + 1), cudaMemcpyDeviceToDevice, st));
    FEM_CUDA(cudaMemcpyAsync(col_dev, S.A.col, 4 * S.A.nnz, cudaMemcpyDeviceToDevice, st));
    FEM_CUDA(cudaMemcpyAsync(val_dev, v, 8 * S.A.nnz, cudaMemcpyDeviceToDevice, st));
    FEM_CUDA(cudaStreamSynchronize(st));
    return FEM_OK;
  });
}

fem_status fem_spmv(fem_system sys, const double* x_dev, double* y_dev, void* stream) {
  return guarded([&]() -> fem_status {
    StreamScope scope(as_stream(stream));
    FEM_REQUIRE(sys && x_dev && y_dev, FEM_EINVAL, "fem_spmv: null argument");
    Level L;
    system_level(sys->S, L);
    cudaStream_t st = as_stream(stream);
    op_apply_d(L, x_dev, y_dev, nullptr, nullptr, st);
    FEM_CUDA(cudaStreamSynchronize(as_stream(stream)));
    return FEM_OK;
  });
}

fem_status fem_spmv_timed(fem_system sys, const double* x_dev, double* y_dev, int32_t reps,
                          void* stream, double* ms_out) {
  return guarded([&]() -> fem_status {
    StreamScope scope(as_stream(stream));
    FEM_REQUIRE(sys && x_dev && y_dev && reps >= 1, FEM_EINVAL, "fem_spmv_timed: bad argument");
    Level L;
    system_level(sys->S, L);
    cudaStream_t st = as_stream(stream);
    const int64_t N = sys->S.N;
    DevBuf<float2> x2;
    DevBuf<int> rflag;
    DfOperator D;
    if (L.stencil) {
      x2.alloc_async(N > 0 ? N : 1, st);
      rflag.alloc_async(1, st);
      FEM_CUDA(cudaMemsetAsync(rflag, 0, sizeof(int), st));
      df_split_vec(N, x_dev, nullptr, x2, rflag, st);
      D = df_operator(L.st);
    }
    auto once = [&]() {
      if (L.stencil)
        op_apply_df(L, D, x2, x_dev, y_dev, nullptr, st, nullptr, rflag);
      else
        op_apply_d(L, x_dev, y_dev, nullptr, nullptr, st);
    };
    once();
    cudaEvent_t e0, e1;
    FEM_CUDA(cudaEventCreate(&e0));
    FEM_CUDA(cudaEventCreate(&e1));
    FEM_CUDA(cudaEventRecord(e0, st));
    for (int i = 0; i < reps; i++) once();
    FEM_CUDA(cudaEventRecord(e1, st));
    FEM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (ms_out) *ms_out = (double)ms / reps;
    return FEM_OK;
  });
}

void fem_system_destroy(fem_system sys) {
  if (!sys) return;
  cudaDeviceSynchronize();
  delete sys;
}

void amg_default_opts(amg_opts* o) {
  if (!o) return;
  o->theta = 0.05;
  o->smoother = AMG_SMOOTHER_CHEBYSHEV;
  o->degree = 2;
  o->cheb_ratio = 6.0;
  o->coarse_max = 256;
  o->max_levels = 16;
  o->precision = AMG_PREC_FP64;
  o->seed = 0;
  o->rho_setup = 0.0;
  o->coarsening = AMG_COARSEN_SA;
  o->max_row = 8192;
  o->order = AMG_ORDER_HASH;
}

fem_status amg_setup(fem_system sys, const amg_opts* opts, void* stream, amg_hier* out) {
  return guarded([&]() -> fem_status {
    StreamScope scope(as_stream(stream));
    FEM_REQUIRE(sys && out, FEM_EINVAL, "amg_setup: null argument");
    *out = nullptr;
    amg_opts o;
    amg_default_opts(&o);
    if (opts) o = *opts;
    FEM_REQUIRE(o.theta >= 0.0 && o.theta < 1.0, FEM_EINVAL, "amg_setup: theta in [0, 1)");
    FEM_REQUIRE(o.max_row >= 0 && o.max_row <= 8192, FEM_EINVAL, "amg_setup: max_row in [0, 8192]");
    FEM_REQUIRE(o.order == AMG_ORDER_HASH || o.order == AMG_ORDER_NATURAL, FEM_EINVAL,
                "amg_setup: order is AMG_ORDER_HASH or AMG_ORDER_NATURAL");
    FEM_REQUIRE(o.degree >= 1 && o.degree <= 15, FEM_EINVAL, "amg_setup: degree in [1, 15]");
    FEM_REQUIRE(o.cheb_ratio > 1.0, FEM_EINVAL, "amg_setup: cheb_ratio > 1");
    FEM_REQUIRE(o.coarse_max >= 1 && o.coarse_max <= 4096, FEM_EINVAL,
                "amg_setup: coarse_max in [1, 4096]");
    FEM_REQUIRE(o.max_levels >= 1 && o.max_levels <= 32, FEM_EINVAL,
                "amg_setup: max_levels in [1, 32]");
    FEM_REQUIRE(o.precision >= 0 && o.precision <= 2, FEM_EINVAL, "amg_setup: bad precision");
    FEM_REQUIRE(o.smoother >= 0 && o.smoother <= 2, FEM_EINVAL, "amg_setup: bad smoother");
    FEM_REQUIRE(o.coarsening == AMG_COARSEN_SA || o.coarsening == AMG_COARSEN_RED_BLACK,
                FEM_EINVAL, "amg_setup: bad coarsening");
    FEM_REQUIRE(o.rho_setup >= 0.0 && std::isfinite(o.rho_setup), FEM_EINVAL,
                "amg_setup: rho_setup >= 0");
    FEM_REQUIRE(o.rho_setup == 0.0 || sys->S.pencil, FEM_EINVAL,
                "amg_setup: rho_setup needs a system that keeps its pencil");
    cudaStream_t st = as_stream(stream);
    auto* h = new amg_hier_s();
    h->sys = sys;
    try {
      cudaEvent_t e0, e1;
      FEM_CUDA(cudaEventCreate(&e0));
      FEM_CUDA(cudaEventCreate(&e1));
      FEM_CUDA(cudaEventRecord(e0, st));
      build_hierarchy(h->H, sys->S, o, st);
      alloc_level_vectors(h->H);
      tune_hierarchy(h->H, sys->S, st);
      reset_ghost_vectors(h->H, st);
      FEM_CUDA(cudaEventRecord(e1, st));
      FEM_CUDA(cudaEventSynchronize(e1));
      float ms = 0;
      cudaEventElapsedTime(&ms, e0, e1);
      h->H.setup_ms = ms;
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    } catch (...) {
      delete h;
      throw;
    }
    *out = h;
    return FEM_OK;
  });
}

fem_status amg_hier_get_info(amg_hier h, amg_hier_info* info) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(h && info, FEM_EINVAL, "amg_hier_get_info: null argument");
    std::memset(info, 0, sizeof(*info));
    info->levels = (int32_t)h->H.L.size();
    for (size_t l = 0; l < h->H.L.size() && l < 32; l++) {
      info->rows[l] = h->H.L[l]->N;
      info->nnz[l] = h->H.L[l]->A->nnz;
      info->lmax[l] = h->H.L[l]->lmax;
      info->pnnz[l] = h->H.L[l]->coarsest ? 0 : h->H.L[l]->P.nnz;
      info->rnnz[l] = h->H.L[l]->coarsest ? 0 : h->H.L[l]->R.nnz;
      info->colours[l] = h->H.L[l]->coff.empty() ? 0 : (int32_t)h->H.L[l]->coff.size() - 1;
    }
    info->finest_stencil = h->H.L.empty() ? 0 : (h->H.L[0]->stencil ? 1 : 0);
    info->setup_ms = h->H.setup_ms;
    return FEM_OK;
  });
}

fem_status amg_hier_export(amg_hier h, int32_t level, int32_t which, int32_t* rowptr_dev,
                           int32_t* col_dev, double* val_dev, int64_t* nnz_out, void* stream) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(h, FEM_EINVAL, "amg_hier_export: null handle");
    FEM_REQUIRE(level >= 0 && level < (int)h->H.L.size(), FEM_EINVAL, "amg_hier_export: bad level");
    Level& L = *h->H.L[level];
    cudaStream_t st = as_stream(stream);
    if (which == 4) {
      FEM_REQUIRE(L.colour.p, FEM_EINVAL, "amg_hier_export: no colouring (SGS smoother only)");
      if (nnz_out) *nnz_out = L.N;
      if (col_dev)
        FEM_CUDA(cudaMemcpyAsync(col_dev, L.colour, 4 * L.N, cudaMemcpyDeviceToDevice, st));
      FEM_CUDA(cudaStreamSynchronize(st));
      return FEM_OK;
    }
    if (which == 3) {
      FEM_REQUIRE(!L.coarsest, FEM_EINVAL, "amg_hier_export: the coarsest level has no aggregates");
      if (nnz_out) *nnz_out = L.N;
      if (col_dev) FEM_CUDA(cudaMemcpyAsync(col_dev, L.agg, 4 * L.N, cudaMemcpyDeviceToDevice, st));
      FEM_CUDA(cudaStreamSynchronize(st));
      return FEM_OK;
    }
    const Csr4* M = nullptr;
    if (which == 0) M = L.A;
    else if (which == 1 || which == 2) {
      FEM_REQUIRE(!L.coarsest, FEM_EINVAL, "amg_hier_export: the coarsest level has no P/R");
      M = which == 1 ? &L.P : &L.R;
    }
    FEM_REQUIRE(M, FEM_EINVAL, "amg_hier_export: which must be 0..4");
    if (nnz_out) *nnz_out = M->nnz;
    if (rowptr_dev)
      FEM_CUDA(cudaMemcpyAsync(rowptr_dev, M->rowptr, 4 * ((int64_t)M->nrows + 1),
                               cudaMemcpyDeviceToDevice, st));
    if (col_dev) FEM_CUDA(cudaMemcpyAsync(col_dev, M->col, 4 * M->nnz, cudaMemcpyDeviceToDevice, st));
    if (val_dev) FEM_CUDA(cudaMemcpyAsync(val_dev, M->val, 8 * M->nnz, cudaMemcpyDeviceToDevice, st));
    FEM_CUDA(cudaStreamSynchronize(st));
    return FEM_OK;
  });
}

fem_status amg_vcycle(amg_hier h, const double* r_dev, double* z_dev, void* stream) {
  return guarded([&]() -> fem_status {
    StreamScope scope(as_stream(stream));
    FEM_REQUIRE(h && r_dev && z_dev, FEM_EINVAL, "amg_vcycle: null argument");
    vcycle(h->H, r_dev, z_dev, as_stream(stream), nullptr);
    FEM_CUDA(cudaStreamSynchronize(as_stream(stream)));
    return FEM_OK;
  });
}

struct bddc_s {
  fem::Bddc* B = nullptr;
  fem_system_s* sys = nullptr;
  ~bddc_s() { fem::bddc_free(B); }
};

fem_status fem_bddc_partition(int32_t n, int32_t slabs, int32_t* layer_begin,
                              int64_t* interface_unknowns) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(n >= 4 && slabs >= 2 && slabs <= n / 2, FEM_EINVAL,
                "fem_bddc_partition: n >= 4 and 2 <= slabs <= n/2");
    if (layer_begin)
      for (int s = 0; s <= slabs; s++) layer_begin[s] = slab_layer(n, slabs, s);
    if (interface_unknowns) *interface_unknowns = (int64_t)(slabs - 1) * (n - 1) * (n - 1);
    return FEM_OK;
  });
}

fem_status bddc_setup(fem_system sys, const bddc_opts* opts, fem_allreduce_fn reduce, void* ctx,
                      void* stream, bddc_solver* out) {
  return guarded([&]() -> fem_status {
    StreamScope scope(as_stream(stream));
    FEM_REQUIRE(sys && opts && out, FEM_EINVAL, "bddc_setup: null argument");
    *out = nullptr;
    const int p = opts->slabs;
    const int s0 = opts->slab_begin, s1 = opts->slab_end > 0 ? opts->slab_end : p;
    FEM_REQUIRE(opts->inner_tol > 0.0 && opts->inner_tol < 1e-6, FEM_EINVAL,
                "bddc_setup: inner_tol in (0, 1e-6)");
    amg_opts ao;
    amg_default_opts(&ao);
    auto* b = new bddc_s();
    try {
      b->B = bddc_create(sys->S, p, s0, s1, ao, opts->inner_tol, reduce, ctx, as_stream(stream));
    } catch (...) {
      delete b;
      throw;
    }
    b->sys = sys;
    *out = b;
    return FEM_OK;
  });
}

fem_status bddc_solve(bddc_solver b, const double* f_dev, double* u_dev, const pcg_opts* opts,
                      fem_allreduce_fn reduce, void* ctx, void* stream, pcg_result* res) {
  return guarded([&]() -> fem_status {
    StreamScope scope(as_stream(stream));
    FEM_REQUIRE(b && u_dev && res, FEM_EINVAL, "bddc_solve: null argument");
    pcg_opts o;
    pcg_default_opts(&o);
    if (opts) o = *opts;
    FEM_REQUIRE(o.tol > 0.0 && o.max_iter >= 0, FEM_EINVAL, "bddc_solve: tol > 0, max_iter >= 0");
    *res = pcg_result{};
    bddc_run(*b->B, f_dev, u_dev, o, reduce, ctx, as_stream(stream), *res);
    res->solve_ms += 0.0;
    return (fem_status)res->status;
  });
}

double bddc_get_setup_ms(bddc_solver b) { return b ? bddc_setup_ms(*b->B) : 0.0; }

void bddc_destroy(bddc_solver b) {
  if (!b) return;
  cudaDeviceSynchronize();
  delete b;
}

fem_status amg_galerkin_timed(amg_hier h, int32_t level, int32_t reps, void* stream,
                              double* ms_out, int64_t* ap_entries_out) {
  return guarded([&]() -> fem_status {
    StreamScope scope(as_stream(stream));
    FEM_REQUIRE(h && reps >= 1, FEM_EINVAL, "amg_galerkin_timed: bad argument");
    int64_t ape = 0;
    const double ms = galerkin_timed(h->H, level, reps, as_stream(stream), &ape);
    if (ms_out) *ms_out = ms;
    if (ap_entries_out) *ap_entries_out = ape;
    return FEM_OK;
  });
}

fem_status amg_vcycle_graph(amg_hier h, const double* r_dev, double* z_dev, int32_t reps,
                            void* stream, double* ms_out) {
  return guarded([&]() -> fem_status {
    StreamScope scope(as_stream(stream));
    FEM_REQUIRE(h && r_dev && z_dev && reps >= 1, FEM_EINVAL, "amg_vcycle_graph: bad argument");
    cudaStream_t st = as_stream(stream);
    // one application on the caller's stream first: it settles every launch shape and
    // allocation, so the captured graph holds kernels only
    vcycle(h->H, r_dev, z_dev, st, nullptr);
    cudaStream_t cs;
    FEM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
    cudaEvent_t e0, e1;
    FEM_CUDA(cudaEventCreate(&e0));
    FEM_CUDA(cudaEventCreate(&e1));
    FEM_CUDA(cudaEventRecord(e0, st));
    FEM_CUDA(cudaStreamWaitEvent(cs, e0, 0));
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    const long long c0 = launches_now();
    FEM_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
    try {
      vcycle(h->H, r_dev, z_dev, cs, nullptr);
    } catch (...) {
      cudaStreamEndCapture(cs, &graph);
      if (graph) cudaGraphDestroy(graph);
      cudaStreamDestroy(cs);
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      throw;
    }
    FEM_CUDA(cudaStreamEndCapture(cs, &graph));
    const long long per = launches_now() - c0;
    count_launches(-per);
    FEM_CUDA(cudaGraphInstantiate(&exec, graph, 0));
    FEM_CUDA(cudaEventRecord(e0, st));
    for (int i = 0; i < reps; i++) {
      FEM_CUDA(cudaGraphLaunch(exec, st));
      count_launches(per);
    }
    FEM_CUDA(cudaEventRecord(e1, st));
    FEM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms_out) *ms_out = (double)ms / reps;
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    cudaStreamDestroy(cs);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return FEM_OK;
  });
}

void amg_hier_destroy(amg_hier h) {
  if (!h) return;
  cudaDeviceSynchronize();
  delete h;
}

void pcg_default_opts(pcg_opts* o) {
  if (!o) return;
  o->tol = 1e-8;
  o->max_iter = 1000;
  o->stop = PCG_STOP_RESIDUAL;
  o->flexible = -1;
  o->use_x0 = 0;
  o->use_graph = 1;
  o->cancel_host = nullptr;
}

fem_status pcg_solve(fem_system sys, amg_hier hier, const double* f_dev, double* u_dev,
                     int32_t nrhs, const double* rho_k_host, const pcg_opts* opts, void* stream,
                     pcg_result* res) {
  return guarded([&]() -> fem_status {
    StreamScope scope(as_stream(stream));
    FEM_REQUIRE(sys && u_dev && res, FEM_EINVAL, "pcg_solve: null argument");
    FEM_REQUIRE(nrhs >= 1, FEM_EINVAL, "pcg_solve: nrhs >= 1");
    FEM_REQUIRE(!hier || hier->sys == sys, FEM_EINVAL, "pcg_solve: hierarchy of another system");
    pcg_opts o;
    pcg_default_opts(&o);
    if (opts) o = *opts;
    FEM_REQUIRE(o.tol > 0.0 && o.max_iter >= 0, FEM_EINVAL, "pcg_solve: tol > 0, max_iter >= 0");
    if (nrhs == 1 && !rho_k_host) {
      pcg_single(sys->S, hier ? &hier->H : nullptr, f_dev, u_dev, o, as_stream(stream), res[0]);
      return (fem_status)res[0].status;
    }
    FEM_REQUIRE(hier && rho_k_host && f_dev, FEM_EINVAL,
                "pcg_solve: several right-hand sides need a hierarchy, rho_k and f");
    return pcg_multi(sys->S, hier->H, f_dev, u_dev, nrhs, rho_k_host, o, as_stream(stream), res);
  });
}

fem_status fem_error_hm1(fem_system sys, const double* u_dev, const fem_target* target,
                         double scale, double tol, void* stream, double* hm1sq_out,
                         pcg_result* res) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(sys && u_dev && target && hm1sq_out, FEM_EINVAL, "fem_error_hm1: null argument");
    StreamScope scope(as_stream(stream));
    pcg_result r{};
    *hm1sq_out = error_hm1(sys->S, u_dev, *target, scale, tol, as_stream(stream), r);
    if (res) *res = r;
    return (fem_status)r.status;
  });
}

fem_status pcg_batch_create(fem_system sys, amg_hier hier, int32_t slots, const pcg_opts* opts,
                            void* stream, pcg_batch* out) {
  return guarded([&]() -> fem_status {
    StreamScope scope(as_stream(stream));
    FEM_REQUIRE(sys && hier && out, FEM_EINVAL, "pcg_batch_create: null argument");
    FEM_REQUIRE(hier->sys == sys, FEM_EINVAL, "pcg_batch_create: hierarchy of another system");
    *out = nullptr;
    pcg_opts o;
    pcg_default_opts(&o);
    if (opts) o = *opts;
    auto* b = new pcg_batch_s();
    try {
      b->W = batch_create(sys->S, hier->H, slots, o, as_stream(stream));
      b->sys = sys;
    } catch (...) {
      delete b;
      throw;
    }
    *out = b;
    return FEM_OK;
  });
}

fem_status pcg_batch_admit(pcg_batch b, const double* f_dev, double rho, int32_t* slot_out,
                           void* stream) {
  return guarded([&]() -> fem_status {
    StreamScope scope(as_stream(stream));
    FEM_REQUIRE(b && f_dev && slot_out, FEM_EINVAL, "pcg_batch_admit: null argument");
    *slot_out = batch_admit(*b->W, f_dev, 1, 0, rho, as_stream(stream));
    return FEM_OK;
  });
}

fem_status pcg_batch_step(pcg_batch b, int32_t iters, void* stream) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(b && iters >= 0, FEM_EINVAL, "pcg_batch_step: bad argument");
    batch_step(*b->W, iters, as_stream(stream));
    return FEM_OK;
  });
}

fem_status pcg_batch_poll(pcg_batch b, int32_t* state_host, int32_t* iters_host,
                          double* relres_host, void* stream) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(b, FEM_EINVAL, "pcg_batch_poll: null handle");
    batch_poll(*b->W, state_host, iters_host, relres_host, as_stream(stream));
    return FEM_OK;
  });
}

fem_status pcg_batch_retire(pcg_batch b, int32_t slot, double* u_dev, void* stream) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(b && u_dev, FEM_EINVAL, "pcg_batch_retire: null argument");
    batch_retire(*b->W, slot, u_dev, 1, 0, as_stream(stream));
    return FEM_OK;
  });
}

int64_t pcg_batch_footprint(fem_system sys, amg_hier hier, int32_t slots) {
  if (!sys || !hier || slots < 1 || slots > 64) return -1;
  try {
    return batch_footprint(sys->S, hier->H, slots);
  } catch (...) {
    return -1;
  }
}

void pcg_batch_destroy(pcg_batch b) {
  if (!b) return;
  cudaDeviceSynchronize();
  batch_destroy(b->W);
  delete b;
}

const char* fem_autotune_report(void) {
  static thread_local std::string rep;
  try {
    rep = autotune_report();
  } catch (...) {
    rep = "{}";
  }
  return rep.c_str();
}

fem_status fem_autotune_pin(const char* kernel, int32_t variant) {
  return guarded([&]() -> fem_status {
    FEM_REQUIRE(kernel, FEM_EINVAL, "fem_autotune_pin: null kernel name");
    autotune_pin(kernel, variant);
    return FEM_OK;
  });
}

void fem_autotune_clear(void) {
  try {
    autotune_clear();
  } catch (...) {
  }
}

}  // extern "C"
