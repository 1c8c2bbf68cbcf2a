// Internal data structures of the solver library and the launchers shared between
// translation units.  Nothing here is part of the C ABI.
#pragma once

#include <functional>
#include <map>
#include <memory>
#include <vector>

#include "common.cuh"

namespace fem {

// 15-point stencil of a matrix on the uniform Kuhn grid of interior points (m per axis):
// c0 at the centre, ca on the 6 axis neighbours +-e_d, cf on the 6 face diagonals
// +-(e_a + e_b), cb on the 2 body diagonals +-(1,1,1); neighbours outside the interior
// grid are Dirichlet zeros.
struct Stencil {
  int m = 0;
  double c0 = 0, ca = 0, cf = 0, cb = 0;
};

struct System {
  int n = 0;
  int64_t N = 0;
  double h = 0, rho = 0;
  bool uniform = false;   // vertex coordinates are the uniform grid
  bool stencil = false;   // finest operator applied matrix-free
  bool pencil = false;    // K and M values kept
  Stencil stA, stK, stM;  // uniform grid only
  Csr4 A;                 // A = rho K + M (CSR4, FP64), pattern shared by Kv/Mv
  DevBuf<double> Kv, Mv;  // pencil values on A's pattern
  DevBuf<double> f;       // load vector
  DevBuf<double> dinv;    // 1 / a_ii
  DevBuf<double> xyz;     // vertex coordinates of a non-uniform grid or a general mesh
  // general tetrahedral mesh (fem_assemble_mesh): tets, unknown of each vertex (-1:
  // Dirichlet), vertex of each unknown, vertex -> incident tets in increasing order
  bool general = false;
  int64_t nv = 0, nt = 0;
  DevBuf<int32_t> tet, vdof, vtet;
  DevBuf<int64_t> rvert, vptr;
};

// A general tetrahedral mesh kept on the device for adaptive refinement: boundary-face mask
// per tet (bit k: the face opposite local vertex k lies on the boundary); dir is padded to a
// multiple of 4 bytes.
struct Mesh {
  int64_t nv = 0, nt = 0;
  DevBuf<double> xyz;
  DevBuf<int32_t> tet;
  DevBuf<uint8_t> dir, bmask;
};

struct Level {
  int64_t N = 0;
  bool stencil = false;
  Stencil st;
  Csr4 Aown;                 // coarse levels own their matrix
  const Csr4* A = nullptr;   // level matrix (the system's for level 0)
  Csr4 P, R;                 // N x Nc and Nc x N
  DevBuf<int32_t> agg;       // aggregate of each node (-1 isolated); red-black: coarse id
                             // of coarse nodes, -1 for fine ones
  DevBuf<int32_t> colour;    // Gauss-Seidel colour of each node (SGS smoother)
  DevBuf<int32_t> cnodes;    // nodes grouped by colour
  std::vector<int64_t> coff; // colour c owns cnodes[coff[c] .. coff[c+1])
  DevBuf<double> dinv;       // 1 / a_ii
  DevBuf<float> dinv32;
  double lmax = 0;           // Gershgorin bound of D^-1 A
  bool scalar_sinv = false;  // smoother diagonal is the constant 1/c0 (stencil, Chebyshev)
  const int* done = nullptr; // early-exit flag of the running solve (null: none)
  bool coarsest = false;
  DevBuf<double> Ainv;       // coarsest: dense inverse, N x N
  // pencil (batched solves): values of P^T K P and P^T M P on A's pattern
  DevBuf<double> Kv, Mv;
  DevBuf<float> Kv32, Mv32;
  double stK_c[4] = {0, 0, 0, 0}, stM_c[4] = {0, 0, 0, 0};
  // single-vector work space (FP64 or FP32 according to the hierarchy precision)
  DevBuf<double> x, b, r, d0, d1;
  DevBuf<float> xf, bf, rf, d0f, d1f;
  // ghost: the FP32 vectors xf, bf, rf, d0f, d1f of a matrix-free finest level use the
  // layout with zero ghost faces ((m+2)^3 entries); rdf is its dense residual (restriction)
  bool ghost = false;
  DevBuf<float> rdf;
  // uniform finest level with the stencil's smoothed prolongator: P = (I - w D^-1 A_F) P_t
  // applied as x += [agg >= 0] (pc[13] t + sum over the strong directions d of pc[d] t(. + d)),
  // t = P_t x_c (tf, ghost layout); pst set by the set-up, tf by the level vectors
  bool pst = false;
  uint32_t pst_strong = 0;
  float pst_c[27];
  DevBuf<float> tf;
};

struct Hierarchy {
  System* sys = nullptr;
  amg_opts o;
  std::vector<std::unique_ptr<Level>> L;
  double setup_ms = 0;
  DevBuf<double> partials;   // per-block partial sums of fused reductions
  DevBuf<double> scal;       // small device scalars
};

// Partial-sum buffer size (doubles) any fused kernel may need: 4 dot products per block.
constexpr int kMaxPartialBlocks = 1 << 16;

// ------------------------------------------------------------------ assembly (assemble.cu)
void assemble_system(System& S, const fem_kuhn_desc& mesh, double rho, const fem_target& t,
                     const fem_assemble_opts& o, cudaStream_t st);
void assemble_rhs(System& S, const fem_target& t, double* f, cudaStream_t st);
void assemble_rhs_noalloc(System& S, const fem_target& t, double* f, cudaStream_t st);
// general tetrahedral mesh: nv vertices (xyz host), nt tets (host), Dirichlet flags (host)
void assemble_mesh(System& S, const fem_mesh_desc& mesh, double rho, const fem_target& t,
                   const fem_assemble_opts& o, cudaStream_t st);
// the same from device arrays (copied: the caller keeps them)
void assemble_mesh_dev(System& S, int64_t nv, int64_t nt, const double* xyz_dev,
                       const int32_t* tet_dev, const uint8_t* dir_dev, double rho,
                       const fem_target& t, const fem_assemble_opts& o, cudaStream_t st);
// vertex -> incident tets (vptr[nv + 1], vtet sorted per vertex); FEM_EINVAL on an index
// out of range
void build_incidence(int64_t nv, int64_t nt, const int32_t* tet, DevBuf<int64_t>& vptr,
                     DevBuf<int32_t>& vtet, cudaStream_t st);
// ||scale*t - u_h||^2 and ||grad(scale*t - u_h)||^2 (NaN without a gradient) by quadrature
void fem_error_norms(System& S, const double* u, const fem_target& t, double scale, int qlevel,
                     double out[2], cudaStream_t st);
// y = M x with the system's mass matrix (from the pencil, or the uniform grid's stencil)
void mass_apply(const System& S, const double* x, double* y, cudaStream_t st);
// SK = the system's stiffness matrix K as a system of its own (rho = 1, no mass term)
void stiffness_system(const System& S, System& SK, cudaStream_t st);
// discrete H^-1 error r^T K^-1 r, r = scale * f(t) - M u, K^-1 r by AMG-PCG to tol
double error_hm1(System& S, const double* u, const fem_target& t, double scale, double tol,
                 cudaStream_t st, pcg_result& res);
// vertex of every unknown (device int64[N])
void dof_vertices(System& S, int64_t* vert, cudaStream_t st);
// residual error indicator eta_T^2 of every tet of a general mesh (eta2[nt]); returns the sum
double error_indicator(System& S, const double* u, const fem_target& t, int qlevel,
                       double* eta2, cudaStream_t st);
// z = (ubar - u) / rho and p = -rho u at the unknowns (either output may be null)
void fem_recovery(System& S, const double* u, const fem_target& t, double* z, double* p,
                  cudaStream_t st);

// ------------------------------------------------------------------ adaptivity (adapt.cu)
void mesh_create(Mesh& M, const fem_mesh_desc& d, cudaStream_t st);
void mesh_refine(Mesh& M, const uint8_t* mark, cudaStream_t st, fem_refine_stats& out);
void mark_bulk(const double* eta, int64_t n, double theta, uint8_t* mark, cudaStream_t st,
               double* threshold, int64_t* nmarked);

// ------------------------------------------------------------------ operators (ops.cu)
// Chebyshev coefficients of one smoothing application of degree k on [lmax/ratio, lmax].
struct ChebCoef {
  int degree = 0;
  double inv_theta = 0;          // 1/theta for the first step
  double c1[16] = {0}, c2[16] = {0};   // d_i = c1[i] d_{i-1} + c2[i] r_i, i >= 1
};
ChebCoef cheb_coefficients(double lmax, double ratio, int degree);

// y = A x (FP64) for a level / system operator; optional <x, y> partials.
void op_apply_d(const Level& Lv, const double* x, double* y, double* partials, int* nblocks,
                cudaStream_t st);
void op_apply_d_done(const Level& Lv, const double* x, double* y, double* partials,
                     int* nblocks, cudaStream_t st, const int* done);
// Non-owning finest-level view of a system's operator.
void system_level(System& S, Level& Lv);
// CG's operator on the uniform grid in double-float arithmetic (ops.cu): coefficients
// prepared once per system; p split into FP32 pairs by df_split_vec (or by CG's p update)
struct DfOperator {
  float C[4][3];
  int s = 0;
  double c64[4];
};
DfOperator df_operator(const Stencil& st);
int op_apply_df(const Level& Lv, const DfOperator& D, const float2* p2, const double* p64,
                double* y, double* partials, cudaStream_t st, const int* done, const int* rflag);
void df_split_vec(int64_t N, const double* x, double* x_out, float2* p2, int* rflag,
                  cudaStream_t st);
// r = b - A x (r dense when the level is in the ghost layout)
template <typename T>
void op_residual(const Level& Lv, int prec, const T* b, const T* x, T* r, cudaStream_t st);
// zero the ghost-layout vectors of a hierarchy (after anything wrote them densely)
void reset_ghost_vectors(Hierarchy& H, cudaStream_t st);
// y (+)= M x for a CSR4 matrix M (restriction / prolongation).
template <typename T>
void csr_spmv(const Csr4& M, int prec, const T* x, T* y, bool accumulate, cudaStream_t st,
              const int* done = nullptr, int ghost_m = 0);
// x += P x_c on a level with the stencil prolongator (pst, ghost layout; FP32 vectors)
void prolong_stencil(const Level& L, const float* xc, float* x, cudaStream_t st);

// One Gauss-Seidel sweep over the colour classes (increasing order when forward):
// x_i = (b_i - sum_{j != i} a_ij x_j) / a_ii.
template <typename T>
void gs_sweep(const Level& Lv, int prec, const T* b, T* x, bool forward, cudaStream_t st);

// Smoother pieces used by the V-cycle.
template <typename T>
void smooth_pre_zero(const Level& Lv, int prec, const amg_opts& o, const ChebCoef& cc,
                     const T* b, T* x, T* r, T* d0, T* d1, cudaStream_t st,
                     const double* b64 = nullptr);
struct DotOut {   // fused dot products of the final smoothing kernel
  double* z64 = nullptr;        // output z (FP64)
  const double* r1 = nullptr;   // <z, r1>
  const double* r2 = nullptr;   // <z, r2>
  double* partials = nullptr;
  int* nblocks = nullptr;
  const int* done = nullptr;
};
template <typename T>
void smooth_post(const Level& Lv, int prec, const amg_opts& o, const ChebCoef& cc, const T* b,
                 T* x, T* r, T* d0, T* d1, cudaStream_t st, const DotOut* dot = nullptr);

// ------------------------------------------------------------------ setup (amg_setup.cu)
void build_hierarchy(Hierarchy& H, System& S, const amg_opts& o, cudaStream_t st);
void spgemm(const Csr4& A, const double* Aval, const Csr4& B, const double* Bval, Csr4& C,
            cudaStream_t st, bool values = true, bool* too_long = nullptr,
            int64_t limit = 8192);
// T = A^T.  A product row beyond the products' limits (8192 distinct columns, 8 GB of
// long-row hash tables) or a transposed row beyond 8192 entries throws FEM_EUNSUPPORTED, or,
// when too_long is given, sets *too_long and returns with the output unset; with too_long
// given, a row longer than limit (<= 8192) counts as too long as well.
void transpose(const Csr4& A, Csr4& T, int64_t ncols, cudaStream_t st, bool* too_long = nullptr,
               int64_t limit = 8192);
double gershgorin(const Csr4& A, const double* val, cudaStream_t st);
// level lev's Galerkin product R (A P) repeated reps times (after one untimed product), mean
// ms by CUDA events on st; the stored entries of A P in *ap_entries
double galerkin_timed(const Hierarchy& H, int lev, int reps, cudaStream_t st, int64_t* ap_entries);
void dense_inverse(const Csr4& A, const double* val, DevBuf<double>& Ainv, cudaStream_t st);

// ------------------------------------------------------------------ V-cycle (vcycle.cu)
void vcycle(Hierarchy& H, const double* r, double* z, cudaStream_t st, const DotOut* dot);

// ------------------------------------------------------------------ batched (batched.cu)
struct BatchSession;
BatchSession* batch_create(System& S, Hierarchy& H, int slots, const pcg_opts& o, cudaStream_t st);
int batch_admit(BatchSession& W, const double* f, int64_t ld, int fcol, double rho, cudaStream_t st);
void batch_step(BatchSession& W, int iters, cudaStream_t st);
void batch_poll(BatchSession& W, int32_t* state, int32_t* iters, double* relres, cudaStream_t st);
void batch_retire(BatchSession& W, int slot, double* u, int64_t ld, int ucol, cudaStream_t st);
void batch_destroy(BatchSession* W);
int64_t batch_footprint(const System& S, const Hierarchy& H, int slots);

// ------------------------------------------------------------------ autotuning (autotune.cu)
// Variant cached for (kernel, a, b, c), else def (also when the cached index is not below
// nvariants).
int tuned_variant(const char* kernel, int64_t a, int64_t b, int c, int def, int nvariants);
// Times every variant (run(v) launches variant v on st) and caches the fastest; returns
// the cached or default choice without timing when tuning is off or st is capturing.
int autotune(const char* kernel, int64_t a, int64_t b, int c, int nvariants,
             const char* const* names, int def, cudaStream_t st,
             const std::function<void(int)>& run);
std::string autotune_report();
void autotune_clear();
void autotune_pin(const char* kernel, int variant);
// Tunes the launch shapes of a hierarchy's operators (ops.cu); runs on scratch vectors
// after the set-up, before any solve uses the hierarchy.
void tune_hierarchy(Hierarchy& H, System& S, cudaStream_t st);

// ------------------------------------------------------------------ scans (amg_setup.cu)
// out[i] = sum_{j < i} in[j] (out has n + 1 entries); returns the total
int64_t exclusive_scan(const int64_t* in, int64_t n, int64_t* out, cudaStream_t st);
// C.rowptr from per-row counts padded to multiples of 4; sets C.nnz and allocates C.col
void rowptr_from_counts(const int64_t* cnt, int64_t n, Csr4& C, cudaStream_t st);

// measured FP64 FMA throughput (TFLOP/s) over reps timed launches of a probe kernel (ops.cu)
double fp64_fma_rate(int reps, cudaStream_t st);

// ------------------------------------------------------------------ BDDC (bddc.cu)
// sums over the slabs of other ranks: buf (count doubles, device memory when on_device) is
// replaced by its sum over all ranks
typedef void (*bddc_reduce_t)(double* buf, int64_t count, int on_device, void* ctx);
struct Bddc;
int slab_layer(int n, int p, int s);
Bddc* bddc_create(System& S, int p, int s0, int s1, const amg_opts& ao, double inner_tol,
                  bddc_reduce_t reduce, void* ctx, cudaStream_t st);
void bddc_free(Bddc* B);
double bddc_setup_ms(const Bddc& B);
void bddc_run(Bddc& B, const double* f, double* u, const pcg_opts& o, bddc_reduce_t reduce,
              void* ctx, cudaStream_t st, pcg_result& res);

// ------------------------------------------------------------------ utilities
void finalize_sums(const double* partials, int nblocks, int nv, double* out, cudaStream_t st,
                   const int* done = nullptr);

}  // namespace fem
