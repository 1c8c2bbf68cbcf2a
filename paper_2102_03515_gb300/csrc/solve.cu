// V-cycle and (flexible) preconditioned conjugate gradients.
//
// V-cycle (arXiv 2102.03515, Sec. 3.1, eq. (amgpre) applied recursively with zero initial
// guess): pre-smooth, residual, restrict with R = P^T, recurse, prolong, post-smooth; the
// coarsest level is solved with its dense FP64 inverse.  In FP32/BF16 hierarchies the
// levels compute in FP32 and only the coarsest solve and the interface to CG are FP64.
//
// PCG (Sec. 4: CG preconditioned by one V-cycle, stopped on a relative residual) keeps
// every scalar on the device.  One iteration is
//   K1  q = A p, <p,q>          -> alpha = <r,z>/<p,q>
//   K2  x += alpha p, r -= alpha q, <r,r>   (r_prev kept for flexible CG)
//   K3  z = V(r) with <z,r> (and <z,r_prev>) fused into the last smoothing kernel
//                               -> beta = <z,r>/<z,r>_old  (flexible: Polak-Ribiere form)
//   K4  p = z + beta p
// Reductions are per-block partial sums added in a fixed order by a one-block kernel, so
// results are bitwise reproducible.  Every kernel returns at once when the device flag
// `done` is set, which lets the host queue iterations ahead (or replay a CUDA graph of
// one iteration) and check convergence only every few iterations.
#include <chrono>
#include <cmath>
#include <cstring>
#include <type_traits>

#include "dfloat.cuh"
#include "solver.cuh"

namespace fem {
long long launches_now();
namespace {

// x = Ainv b on the coarsest level, FP64 arithmetic; warp per row.
template <typename T>
__global__ void k_dense_solve(int64_t N, const double* __restrict__ Ainv, const T* __restrict__ b,
                              const double* __restrict__ b64, T* x, const int* done) {
  if (done && *done) return;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= N) return;
  double s = 0.0;
  for (int64_t c = lane; c < N; c += 32) s += Ainv[row * N + c] * (b64 ? b64[c] : (double)b[c]);
  s = warp_sum(s);
  if (lane == 0) x[row] = (T)s;
}

// z64 = x (FP64) with <z, r1>, <z, r2>.
template <typename T>
__global__ void k_out_dots(int64_t N, const T* x, double* z64, const double* r1, const double* r2,
                           double* partials, int nblocks, const int* done) {
  if (done && *done) return;
  double acc[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double z = (double)x[i];
    z64[i] = z;
    acc[0] += z * r1[i];
    if (r2) acc[1] += z * r2[i];
  }
  block_sum<2>(acc);
  if (threadIdx.x == 0 && partials) {
    partials[blockIdx.x] = acc[0];
    partials[nblocks + blockIdx.x] = acc[1];
  }
}

// Start of the Gauss-Seidel pre-smoothing: x = 0 (and b from its FP64 form at the finest
// level of a low-precision hierarchy).
template <typename T>
__global__ void k_sgs_start(int64_t N, const double* __restrict__ b64, T* b, T* x, const int* done) {
  if (done && *done) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    if (b64) b[i] = (T)b64[i];
    x[i] = (T)0;
  }
}

template <typename T>
struct Bufs;
template <>
struct Bufs<double> {
  static double* x(Level& L) { return L.x.p; }
  static double* b(Level& L) { return L.b.p; }
  static double* r(Level& L) { return L.r.p; }
  static double* d0(Level& L) { return L.d0.p; }
  static double* d1(Level& L) { return L.d1.p; }
};
template <>
struct Bufs<float> {
  static float* x(Level& L) { return L.xf.p; }
  static float* b(Level& L) { return L.bf.p; }
  static float* r(Level& L) { return L.rf.p; }
  static float* d0(Level& L) { return L.d0f.p; }
  static float* d1(Level& L) { return L.d1f.p; }
};

ChebCoef level_cheb(const Level& L, const amg_opts& o) {
  if (o.smoother == AMG_SMOOTHER_L1_JACOBI) {
    ChebCoef c;
    c.degree = 1;
    c.inv_theta = 1.0;
    return c;
  }
  return cheb_coefficients(L.lmax, o.cheb_ratio, o.degree);
}

template <typename T>
void vc(Hierarchy& H, int lev, const T* b, T* x, const double* b64, const DotOut* dot,
        cudaStream_t st);

// V-cycle with symmetric Gauss-Seidel (Sec. 3.1): one forward sweep from x = 0 on the way
// down, one backward sweep on the way up (both at a coarsest level without a dense
// inverse), so that the preconditioner is symmetric.
template <typename T>
void vc_sgs(Hierarchy& H, int lev, const T* b, T* x, const double* b64, const DotOut* dot,
            cudaStream_t st) {
  Level& L = *H.L[lev];
  const int prec = H.o.precision;
  const int64_t N = L.N;
  T* bb = const_cast<T*>(b);
  k_sgs_start<T><<<persistent_grid(N, 256, 8), 256, 0, st>>>(N, b64, bb, x, L.done);
  FEM_CHECK_LAUNCH();
  gs_sweep<T>(L, prec, b, x, true, st);
  if (!L.coarsest) {
    T* r = Bufs<T>::r(L);
    op_residual<T>(L, prec, b, x, r, st);
    Level& C = *H.L[lev + 1];
    csr_spmv<T>(L.R, prec, r, Bufs<T>::b(C), false, st, L.done);
    vc<T>(H, lev + 1, Bufs<T>::b(C), Bufs<T>::x(C), nullptr, nullptr, st);
    csr_spmv<T>(L.P, prec, Bufs<T>::x(C), x, true, st, L.done);
  }
  gs_sweep<T>(L, prec, b, x, false, st);
  if (dot) {
    unsigned g = persistent_grid(N, 256, 8);
    k_out_dots<T><<<g, 256, 0, st>>>(N, x, dot->z64, dot->r1, dot->r2, dot->partials, g, L.done);
    FEM_CHECK_LAUNCH();
    if (dot->nblocks) *dot->nblocks = (int)g;
  }
}

// One V-cycle on levels lev.. with right-hand side b (or b64 at the finest FP32 level) and
// output x.  dot (finest level only) makes the last kernel emit z in FP64 with dot products.
template <typename T>
void vc(Hierarchy& H, int lev, const T* b, T* x, const double* b64, const DotOut* dot,
        cudaStream_t st) {
  Level& L = *H.L[lev];
  const int prec = H.o.precision;
  const amg_opts& o = H.o;
  const int64_t N = L.N;
  if (o.smoother == AMG_SMOOTHER_SGS && !(L.coarsest && L.Ainv.p)) {
    vc_sgs<T>(H, lev, b, x, b64, dot, st);
    return;
  }
  if (L.coarsest) {
    if (L.Ainv.p) {
      unsigned g = grid_for(N * 32, 256);
      k_dense_solve<T><<<g, 256, 0, st>>>(N, L.Ainv, b, b64, x, L.done);
      FEM_CHECK_LAUNCH();
    } else {
      ChebCoef cc = level_cheb(L, o);
      smooth_pre_zero<T>(L, prec, o, cc, b, x, Bufs<T>::r(L), Bufs<T>::d0(L), Bufs<T>::d1(L), st,
                         b64);
    }
    if (dot) {
      unsigned g = persistent_grid(N, 256, 8);
      k_out_dots<T><<<g, 256, 0, st>>>(N, x, dot->z64, dot->r1, dot->r2, dot->partials, g, L.done);
      FEM_CHECK_LAUNCH();
      if (dot->nblocks) *dot->nblocks = (int)g;
    }
    return;
  }
  ChebCoef cc = level_cheb(L, o);
  T* r = Bufs<T>::r(L);
  T* d0 = Bufs<T>::d0(L);
  T* d1 = Bufs<T>::d1(L);
  smooth_pre_zero<T>(L, prec, o, cc, b, x, r, d0, d1, st, b64);
  // the residual for the restriction is dense (on a ghost-layout level in a buffer of its own)
  T* rres = L.ghost ? reinterpret_cast<T*>(L.rdf.p) : r;
  op_residual<T>(L, prec, b, x, rres, st);
  Level& C = *H.L[lev + 1];
  csr_spmv<T>(L.R, prec, rres, Bufs<T>::b(C), false, st, L.done);
  vc<T>(H, lev + 1, Bufs<T>::b(C), Bufs<T>::x(C), nullptr, nullptr, st);
  if constexpr (std::is_same<T, float>::value) {
    if (L.ghost && L.pst && L.tf.p)   // the stencil prolongator (uniform finest level)
      prolong_stencil(L, Bufs<T>::x(C), x, st);
    else
      csr_spmv<T>(L.P, prec, Bufs<T>::x(C), x, true, st, L.done, L.ghost ? L.st.m : 0);
  } else {
    csr_spmv<T>(L.P, prec, Bufs<T>::x(C), x, true, st, L.done, L.ghost ? L.st.m : 0);
  }
  smooth_post<T>(L, prec, o, cc, b, x, r, d0, d1, st, dot);
}

}  // namespace

void alloc_level_vectors(Hierarchy& H) {
  const bool lowp = H.o.precision != AMG_PREC_FP64;
  for (size_t lev = 0; lev < H.L.size(); lev++) {
    Level& L = *H.L[lev];
    const int64_t N = L.N;
    // the matrix-free finest level of a Chebyshev V-cycle keeps its FP32 vectors with zero
    // ghost faces, so that its stencil kernels need no bounds checks
    L.ghost = lowp && lev == 0 && L.stencil && L.scalar_sinv && !L.coarsest &&
              H.o.smoother == AMG_SMOOTHER_CHEBYSHEV && H.o.degree >= 2;
    if (lowp) {
      const int64_t NV = L.ghost ? (int64_t)(L.st.m + 2) * (L.st.m + 2) * (L.st.m + 2) : N;
      L.xf.alloc(NV);
      L.bf.alloc(NV);
      L.rf.alloc(NV);
      L.d0f.alloc(NV);
      L.d1f.alloc(NV);
      if (L.ghost) {
        L.rdf.alloc(N);
        if (L.pst) L.tf.alloc(NV);
        for (DevBuf<float>* v : {&L.xf, &L.bf, &L.rf, &L.d0f, &L.d1f, &L.tf})
          if (v->p) FEM_CUDA(cudaMemset(v->p, 0, sizeof(float) * NV));
      }
    } else {
      L.x.alloc(N);
      L.b.alloc(N);
      L.r.alloc(N);
      L.d0.alloc(N);
      L.d1.alloc(N);
    }
  }
  H.partials.alloc(4 * (size_t)kMaxPartialBlocks);
  H.scal.alloc(64);
}

// z = V(r).  In FP64 the finest level reads r and writes z directly; in FP32/BF16 r is
// converted by the first kernel and z written by the last.
void vcycle(Hierarchy& H, const double* r, double* z, cudaStream_t st, const DotOut* dot) {
  DotOut local;
  if (!dot) {
    local.z64 = z;
    local.r1 = r;
    local.partials = H.partials;
    dot = &local;
  }
  if (H.o.precision == AMG_PREC_FP64) {
    vc<double>(H, 0, r, z, nullptr, dot, st);
  } else {
    Level& L0 = *H.L[0];
    vc<float>(H, 0, L0.bf.p, L0.xf.p, r, dot, st);
  }
}

// ------------------------------------------------------------------ PCG

namespace {

struct PcgState {
  double bb, rr, rz, rz0, pq, alpha, beta, zrp;
  double tol2_res, tol2_prec;
  int iter, done, status, maxit, stop, flexible, pad0, pad1;
};

__global__ void k_pcg_start(PcgState* S, const double* sums_bb, const double* sums_rz,
                            double tol, int maxit, int stop, int flexible) {
  S->bb = sums_bb[0];
  S->rz = sums_rz[0];
  S->zrp = 0.0;
  S->rz0 = S->rz;
  S->rr = sums_bb[1];
  S->tol2_res = tol * tol * S->bb;
  S->tol2_prec = tol * tol * S->rz0;
  S->iter = 0;
  S->status = FEM_OK;
  S->maxit = maxit;
  S->stop = stop;
  S->flexible = flexible;
  S->alpha = S->beta = S->pq = 0.0;
  int done = 0;
  if (!isfinite(S->bb) || !isfinite(S->rr)) {   // a non-finite right-hand side or start
    done = 1;
    S->status = FEM_EBREAKDOWN;
  } else if (!(S->bb > 0.0)) done = 1;  // f = 0: u = 0 is exact
  else if (stop == PCG_STOP_RESIDUAL && S->rr <= S->tol2_res) done = 1;
  else if (!(S->rz > 0.0) || !isfinite(S->rz)) {
    done = 1;
    S->status = FEM_EBREAKDOWN;
  }
  if (maxit <= 0 && !done) {
    done = 1;
    S->status = FEM_ENOCONV;
  }
  S->done = done;
}

__global__ void k_fin_pq(const double* partials, int nb, PcgState* S) {
  if (S->done) return;
  double v[1] = {0.0};
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v[0] += partials[i];
  block_sum<1>(v);
  if (threadIdx.x == 0) {
    S->pq = v[0];
    if (!(v[0] > 0.0) || !isfinite(v[0])) {
      S->status = FEM_EBREAKDOWN;
      S->done = 1;
    } else {
      S->alpha = S->rz / v[0];
    }
  }
}

__global__ void k_update_xr(int64_t N, double* x, const double* p, double* r, const double* q,
                            double* rprev, const PcgState* S, double* partials) {
  if (S->done) return;
  const double alpha = S->alpha;
  double acc[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    double ri = r[i];
    if (rprev) rprev[i] = ri;
    ri -= alpha * q[i];
    r[i] = ri;
    acc[0] += ri * ri;
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc[0];
}

__global__ void k_fin_rr(const double* partials, int nb, PcgState* S) {
  if (S->done) return;
  double v[1] = {0.0};
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v[0] += partials[i];
  block_sum<1>(v);
  if (threadIdx.x == 0) {
    S->rr = v[0];
    S->iter += 1;
    if (!isfinite(v[0])) {
      S->status = FEM_EBREAKDOWN;
      S->done = 1;
    } else if (S->stop == PCG_STOP_RESIDUAL && v[0] <= S->tol2_res) {
      S->done = 1;
    } else if (S->iter >= S->maxit) {
      S->status = FEM_ENOCONV;
      S->done = 1;
    }
  }
}

__global__ void k_fin_rz(const double* partials, int nb, PcgState* S, int* rflag) {
  if (S->done) return;
  if (rflag && threadIdx.x == 0) *rflag = 0;   // the p update that follows raises it again
  double v[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    v[0] += partials[i];
    v[1] += partials[nb + i];
  }
  block_sum<2>(v);
  if (threadIdx.x == 0) {
    const double rz_new = v[0];
    const double beta = S->flexible ? (rz_new - v[1]) / S->rz : rz_new / S->rz;
    S->zrp = v[1];
    S->beta = beta;
    S->rz = rz_new;
    if (!isfinite(beta) || !(rz_new > 0.0)) {
      S->status = FEM_EBREAKDOWN;
      S->done = 1;
    } else if (S->stop == PCG_STOP_PRECONDITIONED && rz_new <= S->tol2_prec) {
      S->done = 1;
    }
  }
}

// p = z + beta p; with p2 given, p is rounded to 48 bits and kept as FP32 pairs as well (the
// input of the double-float operator), rflag raised for entries outside the pairs' range
__global__ void k_update_p(int64_t N, const double* z, double* p, const PcgState* S, float2* p2,
                           int* rflag) {
  if (S->done) return;
  const double beta = S->beta;
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double v = z[i] + beta * p[i];
    if (p2) {
      float hi, lo;
      double vs;
      if (df_split(v, hi, lo, vs)) {
        p2[i] = make_float2(hi, lo);
        p[i] = vs;
      } else {
        p[i] = v;
        bad = true;
      }
    } else {
      p[i] = v;
    }
  }
  if (p2 && __any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(rflag, 1);
}

__global__ void k_jacobi_prec(int64_t N, const double* dinv, const double* r, const double* rprev,
                              double* z, double* partials, const int* done) {
  if (done && *done) return;
  double acc[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double zi = dinv[i] * r[i];
    z[i] = zi;
    acc[0] += zi * r[i];
    if (rprev) acc[1] += zi * rprev[i];
  }
  block_sum<2>(acc);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = acc[0];
    partials[gridDim.x + blockIdx.x] = acc[1];
  }
}

// partials of <a,a> and <b,b> (b may be null)
__global__ void k_dot_self(int64_t N, const double* a, const double* b, double* partials) {
  double acc[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    acc[0] += a[i] * a[i];
    if (b) acc[1] += b[i] * b[i];
  }
  block_sum<2>(acc);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = acc[0];
    partials[gridDim.x + blockIdx.x] = acc[1];
  }
}

__global__ void k_sub(int64_t N, const double* f, double* r) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    r[i] = f[i] - r[i];
}

__global__ void k_copy(int64_t N, const double* a, double* b) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    b[i] = a[i];
}

}  // namespace

struct PcgWork {
  int64_t N = 0;
  DevBuf<double> r, rprev, p, q, z, partials, sums;
  DevBuf<float2> p2;     // p as FP32 pairs (double-float operator on the uniform grid)
  DevBuf<int> rflag;     // p has entries outside the pairs' range: FP64 operator
  DevBuf<PcgState> state;
  PcgState* hstate = nullptr;  // pinned, 2 slots
  cudaStream_t s = nullptr;
  cudaEvent_t ev[2] = {nullptr, nullptr}, t0 = nullptr, t1 = nullptr;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  ~PcgWork() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    for (auto& e : ev)
      if (e) cudaEventDestroy(e);
    if (t0) cudaEventDestroy(t0);
    if (t1) cudaEventDestroy(t1);
    if (hstate) cudaFreeHost(hstate);
    if (s) cudaStreamDestroy(s);
  }
};

void pcg_single(System& S, Hierarchy* H, const double* f, double* u, const pcg_opts& o,
                cudaStream_t user, pcg_result& res) {
  const int64_t N = S.N;
  PcgWork W;
  W.N = N;
  W.r.alloc(N);
  W.p.alloc(N);
  W.q.alloc(N);
  W.z.alloc(N);
  const bool flexible =
      o.flexible == 1 || (o.flexible < 0 && H && H->o.precision != AMG_PREC_FP64);
  if (flexible) W.rprev.alloc(N);
  W.partials.alloc(4 * (size_t)kMaxPartialBlocks);
  W.sums.alloc(8);
  W.state.alloc(1);
  FEM_CUDA(cudaMallocHost(&W.hstate, 2 * sizeof(PcgState)));
  FEM_CUDA(cudaStreamCreateWithFlags(&W.s, cudaStreamNonBlocking));
  for (auto& e : W.ev) FEM_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  FEM_CUDA(cudaEventCreate(&W.t0));
  FEM_CUDA(cudaEventCreate(&W.t1));
  cudaStream_t st = W.s;
  // order after the caller's stream
  FEM_CUDA(cudaEventRecord(W.ev[0], user));
  FEM_CUDA(cudaStreamWaitEvent(st, W.ev[0], 0));

  Level sysL;
  system_level(S, sysL);
  struct DoneReset {  // levels never keep a pointer to this solve's flag
    Hierarchy* H;
    ~DoneReset() {
      if (H)
        for (auto& Lp : H->L) Lp->done = nullptr;
    }
  } done_reset{H};
  // CG's operator is always the system's (a hierarchy may be set up from another rho); on
  // the uniform grid it runs in double-float arithmetic on p split into FP32 pairs
  Level& L0 = sysL;
  const bool dfop = L0.stencil;
  DfOperator dfo;
  if (dfop) {
    W.p2.alloc(N);
    W.rflag.alloc(1);
    dfo = df_operator(L0.st);
  }
  const int* done = &W.state.p->done;
  const unsigned gv = persistent_grid(N, 256, 8);
  if (!f) f = S.f.p;

  // z = V(r) with <z, r>
  int nb_rz = 0;
  DotOut dot;
  dot.z64 = W.z;
  dot.r1 = W.r;
  dot.r2 = flexible ? W.rprev.p : nullptr;
  dot.partials = W.partials;
  dot.nblocks = &nb_rz;
  auto precondition = [&](const int* dflag) {
    if (H) {
      for (auto& Lp : H->L) Lp->done = dflag;
      dot.done = dflag;
      vcycle(*H, W.r, W.z, st, &dot);
    } else {
      k_jacobi_prec<<<gv, 256, 0, st>>>(N, S.dinv, W.r, dot.r2, W.z, W.partials, dflag);
      FEM_CHECK_LAUNCH();
      nb_rz = (int)gv;
    }
  };
  // one iteration, all kernels gated by the device flag
  auto iteration = [&]() {
    int nb_pq = 0;
    if (dfop)
      nb_pq = op_apply_df(L0, dfo, W.p2, W.p, W.q, W.partials, st, done, W.rflag);
    else
      op_apply_d_done(L0, W.p, W.q, W.partials, &nb_pq, st, done);
    k_fin_pq<<<1, 1024, 0, st>>>(W.partials, nb_pq, W.state);
    FEM_CHECK_LAUNCH();
    k_update_xr<<<gv, 256, 0, st>>>(N, u, W.p, W.r, W.q, flexible ? W.rprev.p : nullptr, W.state,
                                    W.partials);
    FEM_CHECK_LAUNCH();
    k_fin_rr<<<1, 1024, 0, st>>>(W.partials, gv, W.state);
    FEM_CHECK_LAUNCH();
    precondition(done);
    k_fin_rz<<<1, 1024, 0, st>>>(W.partials, nb_rz, W.state, dfop ? W.rflag.p : nullptr);
    FEM_CHECK_LAUNCH();
    k_update_p<<<gv, 256, 0, st>>>(N, W.z, W.p, W.state, dfop ? W.p2.p : nullptr,
                                   dfop ? W.rflag.p : nullptr);
    FEM_CHECK_LAUNCH();
  };

  bool use_graph = o.use_graph != 0;
  long long per_iter = 0;
  if (use_graph) {
    const long long c0 = launches_now();
    FEM_CUDA(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
    try {
      iteration();
    } catch (...) {
      cudaGraph_t g;
      cudaStreamEndCapture(st, &g);
      if (g) cudaGraphDestroy(g);
      throw;
    }
    FEM_CUDA(cudaStreamEndCapture(st, &W.graph));
    FEM_CUDA(cudaGraphInstantiate(&W.exec, W.graph, 0));
    per_iter = launches_now() - c0;   // captured, not run: counted again per replay
    count_launches(-per_iter);
  }
  FEM_CUDA(cudaEventRecord(W.t0, st));
  // With the double-float operator CG's recursive residual can run ahead of the FP64 one by
  // about 2^-44 cond(A): when the FP64 residual recomputed at the end is above the
  // tolerance, CG starts again from its iterate (at most twice).
  bool from_u = o.use_x0 != 0;
  int status = FEM_OK, iters = 0;
  PcgState hs{};
  double hs2[2] = {0.0, 0.0};
  for (int pass = 0;; pass++) {
    // r = f - A x0  (or f)
    if (from_u) {
      op_apply_d(L0, u, W.r, nullptr, nullptr, st);
      k_sub<<<gv, 256, 0, st>>>(N, f, W.r);
      FEM_CHECK_LAUNCH();
    } else {
      FEM_CUDA(cudaMemsetAsync(u, 0, 8 * N, st));
      k_copy<<<gv, 256, 0, st>>>(N, f, W.r);
      FEM_CHECK_LAUNCH();
    }
    if (flexible) FEM_CUDA(cudaMemsetAsync(W.rprev, 0, 8 * N, st));
    // bb = <f,f>, rr = <r,r>
    k_dot_self<<<gv, 256, 0, st>>>(N, f, W.r, W.partials);
    FEM_CHECK_LAUNCH();
    finalize_sums(W.partials, gv, 2, W.sums, st);
    precondition(nullptr);
    finalize_sums(W.partials, nb_rz, 1, W.sums.p + 4, st);
    k_pcg_start<<<1, 1, 0, st>>>(W.state, W.sums, W.sums.p + 4, o.tol, o.max_iter - iters, o.stop,
                                 flexible);
    FEM_CHECK_LAUNCH();
    if (dfop) {
      FEM_CUDA(cudaMemsetAsync(W.rflag, 0, sizeof(int), st));
      df_split_vec(N, W.z, W.p, W.p2, W.rflag, st);
    } else {
      k_copy<<<gv, 256, 0, st>>>(N, W.z, W.p);
      FEM_CHECK_LAUNCH();
    }

    const int chunk = 2;
    int k = 0;
    int launched = 0;
    bool finished = false;
    while (!finished) {
      for (int c = 0; c < chunk; c++) {
        if (use_graph) {
          FEM_CUDA(cudaGraphLaunch(W.exec, st));
          count_launches(per_iter);
        } else
          iteration();
        launched++;
      }
      FEM_CUDA(cudaMemcpyAsync(&W.hstate[k & 1], W.state, sizeof(PcgState), cudaMemcpyDeviceToHost, st));
      FEM_CUDA(cudaEventRecord(W.ev[k & 1], st));
      if (k > 0) {
        FEM_CUDA(cudaEventSynchronize(W.ev[(k - 1) & 1]));
        const PcgState& h1 = W.hstate[(k - 1) & 1];
        if (h1.done) finished = true;
        if (!finished && o.cancel_host && *o.cancel_host) {   // a finished solve stands
          status = FEM_ECANCELLED;
          finished = true;
        }
      }
      if (launched > o.max_iter + 4 * chunk) finished = true;  // safety: flag never set
      k++;
    }
    FEM_CUDA(cudaMemcpyAsync(&W.hstate[0], W.state, sizeof(PcgState), cudaMemcpyDeviceToHost, st));
    FEM_CUDA(cudaStreamSynchronize(st));
    hs = W.hstate[0];
    // the flag was read while the last chunk was still queued: a solve that finished in
    // that chunk stands
    if (status == FEM_ECANCELLED && hs.done) status = FEM_OK;
    iters += hs.iter;
    // true residual: with the double-float operator when the tolerance leaves room for its
    // 2^-44 bound (u split into pairs; an entry out of their range takes the FP64 rows), in
    // FP64 otherwise
    if (dfop && o.tol >= 1e-10) {
      FEM_CUDA(cudaMemsetAsync(W.rflag, 0, sizeof(int), st));
      df_split_vec(N, u, nullptr, W.p2, W.rflag, st);
      op_apply_df(L0, dfo, W.p2, u, W.q, nullptr, st, nullptr, W.rflag);
    } else {
      op_apply_d(L0, u, W.q, nullptr, nullptr, st);
    }
    k_sub<<<gv, 256, 0, st>>>(N, f, W.q);
    FEM_CHECK_LAUNCH();
    k_dot_self<<<gv, 256, 0, st>>>(N, W.q, f, W.partials);
    FEM_CHECK_LAUNCH();
    finalize_sums(W.partials, gv, 2, W.sums, st);
    FEM_CUDA(cudaMemcpyAsync(hs2, W.sums, 16, cudaMemcpyDeviceToHost, st));
    FEM_CUDA(cudaStreamSynchronize(st));
    const bool again = dfop && status == FEM_OK && hs.done && hs.status == FEM_OK &&
                       o.stop == PCG_STOP_RESIDUAL && hs2[1] > 0 &&
                       hs2[0] > o.tol * o.tol * hs2[1] && pass < 2 && iters < o.max_iter;
    if (!again) break;
    from_u = true;
  }
  FEM_CUDA(cudaEventRecord(W.t1, st));
  FEM_CUDA(cudaEventSynchronize(W.t1));
  float ms = 0.f;
  FEM_CUDA(cudaEventElapsedTime(&ms, W.t0, W.t1));
  // the caller's stream continues after the solve
  FEM_CUDA(cudaEventRecord(W.ev[0], st));
  FEM_CUDA(cudaStreamWaitEvent(user, W.ev[0], 0));
  res.iterations = iters;
  res.status = status != FEM_OK ? status : (hs.done ? hs.status : FEM_ENOCONV);
  res.relres = hs2[1] > 0 ? std::sqrt(hs2[0] / hs2[1]) : 0.0;
  res.prec_relres = hs.rz0 > 0 ? std::sqrt(std::fabs(hs.rz / hs.rz0)) : 0.0;
  res.solve_ms = ms;
}

// ------------------------------------------------------------------ discrete H^-1 error

namespace {
__global__ void k_hm1_residual(int64_t N, double scale, const double* fw, const double* mu,
                               double* r) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) r[i] = scale * fw[i] - mu[i];
}

// per-block partial sums of <a, b> (fixed order: deterministic)
__global__ void k_dot_partials(int64_t N, const double* a, const double* b, double* part) {
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x)
    v[0] = fma(a[i], b[i], v[0]);
  block_sum<1>(v);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}

double device_dot(int64_t N, const double* a, const double* b, cudaStream_t st) {
  const unsigned g = persistent_grid(N, 256, 4);
  DevBuf<double> part(g, st), sum(1, st);
  k_dot_partials<<<g, 256, 0, st>>>(N, a, b, part);
  FEM_CHECK_LAUNCH();
  finalize_sums(part, (int)g, 1, sum, st);
  double out = 0.0;
  FEM_CUDA(cudaMemcpyAsync(&out, sum, 8, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  return out;
}
}  // namespace

// ||w - u_h||^2 in the dual norm of the P1 space with zero boundary values, w = scale * t:
// r_i = (w - u_h, phi_i) = scale * f_i(t) - (M u)_i, value r^T K^-1 r.  The stiffness solve
// is CG with an FP64 smoothed-aggregation V-cycle built on K, started from zero; CG's
// iterate y_k satisfies r^T y_k = y_k^T K y_k, so r^T K^-1 r - r^T y_k is the squared energy
// norm of its error and the value is accurate to about tol^2 cond(K) relative.
double error_hm1(System& S, const double* u, const fem_target& t, double scale, double tol,
                 cudaStream_t st, pcg_result& res) {
  FEM_REQUIRE(tol > 0.0 && tol < 1.0, FEM_EINVAL, "fem_error_hm1: tol in (0, 1)");
  std::memset(&res, 0, sizeof(res));
  res.status = FEM_OK;
  const int64_t N = S.N;
  if (N == 0) return 0.0;
  System SK;
  stiffness_system(S, SK, st);   // checks that K and M are available first
  DevBuf<double> r(N, st), mu(N, st), y(N, st);
  assemble_rhs(S, t, r, st);     // load vector of t: the rule of the system's f
  mass_apply(S, u, mu, st);
  k_hm1_residual<<<grid_for(N, 256), 256, 0, st>>>(N, scale, r, mu, r);
  FEM_CHECK_LAUNCH();
  if (device_dot(N, r, r, st) == 0.0) return 0.0;
  Hierarchy HK;
  amg_opts ao;
  amg_default_opts(&ao);
  build_hierarchy(HK, SK, ao, st);
  alloc_level_vectors(HK);
  pcg_opts po;
  pcg_default_opts(&po);
  po.tol = tol;
  FEM_CUDA(cudaMemsetAsync(y, 0, 8 * N, st));
  pcg_single(SK, &HK, r, y, po, st, res);
  return device_dot(N, r, y, st);
}

}  // namespace fem
