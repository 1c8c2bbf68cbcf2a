// Batched multi-vector PCG: up to 64 independent solves (rho_b K + M) u_b = f_b on one mesh
// and one smoothed-aggregation hierarchy, advanced together (no counterpart in the paper;
// each column is the paper's PCG of Sec. 4 with the V-cycle of Sec. 3.1).
//
// Vectors are multivectors X[N][B] (row-major, B a power of two): element (i, b) is slot b
// of unknown i, so a warp reads 32 slots of one row with one coalesced access.  The
// prolongators are built once; with P fixed every level's operator is the pencil
// A_l(rho_b) = rho_b K_l + M_l, K_l = P^T K P and M_l = P^T M P, so one pass over the
// level's K and M values serves every slot.  Per slot: rho, the Gershgorin bound and the
// Chebyshev coefficients of each level, and the dense inverse of the coarsest operator.
//
// Each iteration runs, for every active slot,
//     z = V(r);  rz = <r,z>;  beta = first ? 0 : (rz - <z,r_prev>) / rz_old  (flexible CG)
//     p = z + beta p;  q = A p;  alpha = rz / <p,q>;  x += alpha p;  r_prev = r;  r -= alpha q
// which is PCG with the V-cycle moved to the top, so a slot admitted between iterations
// starts with x = 0, r = f and joins at the next V-cycle.  Per-slot reductions add
// per-block partial sums in a fixed order that does not involve other slots: a slot's
// iterates do not depend on what else is in the batch.  One iteration is captured once as
// a CUDA graph and replayed.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "solver.cuh"

namespace fem {

long long launches_now();

namespace {

constexpr int MAXB = 64;

struct SlotState {
  double rho, bb, rr, rz, rz_old, pq, alpha, beta, zrp, tol2;
  int iter, first, active, done, status, maxit, pad0, pad1;
};

// per (level, slot) smoother coefficients: inv_theta, c1, c2 (degree 2) and, for the
// stencil level, the four stencil coefficients of A(rho_b) and 1/c0
struct LevCoef {
  float inv_theta, c1, c2, pad;
  float c0, ca, cf, cb;
  float sinv;
  float pad2[3];
};

// ------------------------------------------------------------------ multivector stencil

// y[i][b] op (A(rho_b) v)[i][b] on the uniform grid; one thread per (point, slot).
// Modes as in the single-vector epilogue: 0 store (+dot <v,Av>), 1 residual y = b - Av,
// 2 Chebyshev step, 3 Chebyshev init.  Dots are per slot: partials[b * nblocks + block].
template <typename T>
struct MvEpi {
  int mode;
  T* y;
  const T* b;
  T* r;
  const T* dold;
  T* dnew;
  T* x;
  int add_prev;
  int level;
  const LevCoef* lc;      // [L][B]
  int B;
  const float* kd;        // CSR levels: diag of K and M for the smoother diagonal
  const float* md;
  const double* rho;      // [B]
  int want_dot;
  const SlotState* slots; // masking of done slots (FP64 CG kernels)
  double* z64;            // final output (finest level)
  const double* r1;
  const double* r2;
};

template <typename T>
__device__ __forceinline__ float smoother_sinv(const MvEpi<T>& e, int64_t i, int b) {
  const LevCoef& c = e.lc[e.level * e.B + b];
  if (e.kd) return 1.0f / ((float)e.rho[b] * e.kd[i] + e.md[i]);
  return c.sinv;
}

template <typename T>
__device__ __forceinline__ void mv_epi(const MvEpi<T>& e, int64_t i, int b, typename Arith<T>::type av,
                                       double acc[2]) {
  using AT = typename Arith<T>::type;
  const int64_t idx = i * e.B + b;
  switch (e.mode) {
    case 0:
      e.y[idx] = (T)av;
      if (e.want_dot) acc[0] += (double)e.x[idx] * (double)av;
      break;
    case 1:
      e.y[idx] = (T)((AT)e.b[idx] - av);
      break;
    case 3: {
      const LevCoef& c = e.lc[e.level * e.B + b];
      AT s = (AT)smoother_sinv(e, i, b);
      AT rr = s * ((AT)e.b[idx] - av);
      e.r[idx] = (T)rr;
      e.dnew[idx] = (T)((AT)c.inv_theta * rr);
    } break;
    case 2: {
      const LevCoef& c = e.lc[e.level * e.B + b];
      AT s = (AT)smoother_sinv(e, i, b);
      AT rr = (AT)e.r[idx] - s * av;
      AT dl = (AT)e.dold[idx];
      AT dn = (AT)c.c1 * dl + (AT)c.c2 * rr;
      e.r[idx] = (T)rr;
      e.dnew[idx] = (T)dn;
      AT xv = (AT)e.x[idx] + (e.add_prev ? dl : (AT)0) + dn;
      e.x[idx] = (T)xv;
      if (e.z64) {
        double z = (double)xv;
        e.z64[idx] = z;
        acc[0] += z * e.r1[idx];
        acc[1] += z * e.r2[idx];
      }
    } break;
  }
}

// per-slot block reduction: threads of a block cover (points x slots) with slot = tid % B
template <int NV>
__device__ __forceinline__ void slot_partials(double (&acc)[NV], int B, double* partials,
                                              int nblocks, int bid) {
  __shared__ double sh[NV][256];
  for (int k = 0; k < NV; k++) sh[k][threadIdx.x] = acc[k];
  __syncthreads();
  if ((int)threadIdx.x < B) {
    for (int k = 0; k < NV; k++) {
      double s = 0.0;
      for (int t = threadIdx.x; t < (int)blockDim.x; t += B) s += sh[k][t];
      partials[((int64_t)k * B + threadIdx.x) * nblocks + bid] = s;
    }
  }
}

// grid: x over blocks of points along i, y strides over the (j, k) planes
template <typename T, int NV>
__global__ void __launch_bounds__(256) k_mv_stencil(const T* __restrict__ v, int m, MvEpi<T> e,
                                                    double* partials, int nblocks) {
  using AT = typename Arith<T>::type;
  const int B = e.B;
  const int b = threadIdx.x & (B - 1);
  const int ppb = blockDim.x / B;
  const int i = blockIdx.x * ppb + threadIdx.x / B;
  double acc[2] = {0.0, 0.0};
  const LevCoef& c = e.lc[e.level * B + b];
  const AT c0 = (AT)c.c0, ca = (AT)c.ca, cf = (AT)c.cf, cb = (AT)c.cb;
  const int64_t sj = (int64_t)m * B, sk = (int64_t)m * m * B;
  for (int jk = blockIdx.y; jk < m * m; jk += gridDim.y) {
    const int k = jk / m, j = jk - k * m;
    if (i < m) {
      const int64_t o = ((int64_t)i + (int64_t)m * j + (int64_t)m * m * k) * B + b;
      const bool im = i > 0, ip = i < m - 1, jm = j > 0, jp = j < m - 1, km = k > 0, kp = k < m - 1;
      auto X = [&](bool ok, int64_t off) -> AT { return ok ? (AT)v[o + off] : (AT)0; };
      AT axis = X(im, -B) + X(ip, B) + X(jm, -sj) + X(jp, sj) + X(km, -sk) + X(kp, sk);
      AT face = X(ip && jp, B + sj) + X(im && jm, -B - sj) + X(ip && kp, B + sk) +
                X(im && km, -B - sk) + X(jp && kp, sj + sk) + X(jm && km, -sj - sk);
      AT body = X(ip && jp && kp, B + sj + sk) + X(im && jm && km, -B - sj - sk);
      AT av = c0 * (AT)v[o] + ca * axis + cf * face + cb * body;
      mv_epi<T>(e, (int64_t)i + (int64_t)m * j + (int64_t)m * m * k, b, av, acc);
    }
  }
  if (NV > 0 && partials)
    slot_partials<2>(acc, B, partials, nblocks, blockIdx.x + gridDim.x * blockIdx.y);
}

// FP64 stencil for q = A(rho_b) p with per-slot coefficients in FP64 and <p, q> per slot
// (slots null: every slot, no dots).
__global__ void __launch_bounds__(256) k_mv_stencil64(const double* __restrict__ v, int m,
                                                      const double* coef /* [B][4] */, int B,
                                                      double* y, const SlotState* slots,
                                                      double* partials, int nblocks) {
  const int b = threadIdx.x & (B - 1);
  const int ppb = blockDim.x / B;
  const int i = blockIdx.x * ppb + threadIdx.x / B;
  double acc[1] = {0.0};
  const bool live = !slots || (slots[b].active && !slots[b].done);
  const double c0 = coef[4 * b], ca = coef[4 * b + 1], cf = coef[4 * b + 2], cb = coef[4 * b + 3];
  const int64_t sj = (int64_t)m * B, sk = (int64_t)m * m * B;
  for (int jk = blockIdx.y; jk < m * m; jk += gridDim.y) {
    const int k = jk / m, j = jk - k * m;
    if (i < m && live) {
      const int64_t o = ((int64_t)i + (int64_t)m * j + (int64_t)m * m * k) * B + b;
      const bool im = i > 0, ip = i < m - 1, jm = j > 0, jp = j < m - 1, km = k > 0, kp = k < m - 1;
      auto X = [&](bool ok, int64_t off) -> double { return ok ? v[o + off] : 0.0; };
      double av = c0 * v[o];
      av = fma(ca, X(im, -B), av);
      av = fma(ca, X(ip, B), av);
      av = fma(ca, X(jm, -sj), av);
      av = fma(ca, X(jp, sj), av);
      av = fma(ca, X(km, -sk), av);
      av = fma(ca, X(kp, sk), av);
      av = fma(cf, X(ip && jp, B + sj), av);
      av = fma(cf, X(im && jm, -B - sj), av);
      av = fma(cf, X(ip && kp, B + sk), av);
      av = fma(cf, X(im && km, -B - sk), av);
      av = fma(cf, X(jp && kp, sj + sk), av);
      av = fma(cf, X(jm && km, -sj - sk), av);
      av = fma(cb, X(ip && jp && kp, B + sj + sk), av);
      av = fma(cb, X(im && jm && km, -B - sj - sk), av);
      y[o] = av;
      acc[0] += v[o] * av;
    }
  }
  if (slots) slot_partials<1>(acc, B, partials, nblocks, blockIdx.x + gridDim.x * blockIdx.y);
}

// ------------------------------------------------------------------ multivector CSR

// y[i][b] op ((rho_b K + M) v)[i][b] (pencil) or (Mat v)[i][b] (kv null: single values mv).
// One thread per (row, slot): the row's entries are broadcast, the slot reads coalesce.
template <typename T, typename VT, int NV>
__global__ void __launch_bounds__(256) k_mv_csr(int64_t nrows, const int32_t* __restrict__ rowptr,
                                                const int32_t* __restrict__ col,
                                                const VT* __restrict__ kv, const VT* __restrict__ mv,
                                                const T* __restrict__ v, MvEpi<T> e, int accumulate,
                                                double* partials, int nblocks) {
  using AT = typename Arith<T>::type;
  const int B = e.B;
  const int b = threadIdx.x % B;
  const int rpb = blockDim.x / B;
  const AT rb = kv ? (AT)e.rho[b] : (AT)0;
  double acc[2] = {0.0, 0.0};
  for (int64_t base = (int64_t)blockIdx.x * rpb; base < nrows; base += (int64_t)gridDim.x * rpb) {
    const int64_t i = base + threadIdx.x / B;
    if (i < nrows) {
      AT s = 0;
      for (int q = rowptr[i]; q < rowptr[i + 1]; q++) {
        const int c = col[q];
        if (c < 0) continue;
        const AT w = kv ? rb * (AT)kv[q] + (AT)mv[q] : (AT)mv[q];
        s += w * (AT)v[(int64_t)c * B + b];
      }
      if (accumulate) {
        const int64_t idx = i * B + b;
        e.y[idx] = (T)((AT)e.y[idx] + s);
      } else {
        mv_epi<T>(e, i, b, s, acc);
      }
    }
  }
  if (NV > 0 && partials) slot_partials<2>(acc, B, partials, nblocks, blockIdx.x);
}

// ------------------------------------------------------------------ elementwise

template <typename T>
__global__ void k_mv_cheb_zero(int64_t N, int B, const double* __restrict__ b64, T* bT,
                               const LevCoef* lc, int level, const float* kd, const float* md,
                               const double* rho, T* r, T* d, T* x) {
  using AT = typename Arith<T>::type;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N * B;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(idx & (B - 1));
    const int64_t i = idx >> (31 - __clz(B));
    const LevCoef& c = lc[level * B + b];
    AT bv;
    if (b64) {
      bv = (AT)b64[idx];
      bT[idx] = (T)bv;
    } else {
      bv = (AT)bT[idx];
    }
    AT s = kd ? (AT)(1.0f / ((float)rho[b] * kd[i] + md[i])) : (AT)c.sinv;
    AT rr = s * bv;
    AT dd = (AT)c.inv_theta * rr;
    r[idx] = (T)rr;
    d[idx] = (T)dd;
    x[idx] = (T)dd;
  }
}

// dense coarsest solve per slot: x[i][b] = sum_j Ainv_b[i][j] rhs[j][b]
template <typename T>
__global__ void k_mv_dense(int64_t Nc, int B, const double* Ainv, const T* rhs, T* x) {
  const int64_t w = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w >= Nc * B) return;
  const int64_t i = w / B;
  const int b = (int)(w % B);
  const double* M = Ainv + (int64_t)b * Nc * Nc + i * Nc;
  double s = 0.0;
  for (int64_t j = lane; j < Nc; j += 32) s += M[j] * (double)rhs[j * B + b];
  s = warp_sum(s);
  if (lane == 0) x[i * B + b] = (T)s;
}

// dense per-slot coarse matrices from the pencil: D_b = rho_b K + M
__global__ void k_mv_dense_build(int64_t Nc, const int32_t* rowptr, const int32_t* col,
                                 const double* kv, const double* mv, const double* rho, int slot,
                                 double* D) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= Nc) return;
  double* Dr = D + r * Nc;
  for (int64_t c = 0; c < Nc; c++) Dr[c] = 0.0;
  for (int e = rowptr[r]; e < rowptr[r + 1]; e++)
    if (col[e] >= 0) Dr[col[e]] += rho[slot] * kv[e] + mv[e];
}

__global__ void k_gj_step_b(int64_t N, int64_t k, const double* __restrict__ D, double* __restrict__ E) {
  __shared__ double inv_p;
  if (threadIdx.x == 0) inv_p = 1.0 / D[k * N + k];
  __syncthreads();
  const double ip = inv_p;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N * N;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / N, j = t % N;
    double v;
    if (i == k && j == k) v = ip;
    else if (i == k) v = D[t] * ip;
    else if (j == k) v = -D[t] * ip;
    else v = D[t] - D[i * N + k] * (D[k * N + j] * ip);
    E[t] = v;
  }
}

// Gershgorin bound of D^{-1} A(rho) for one slot: block maxima of sum_j |a_ij| / a_ii
__global__ void k_mv_gersh(int64_t N, const int32_t* rowptr, const int32_t* col, const double* kv,
                           const double* mv, double rho, double* bmax) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double q = -1.0;
  if (r < N) {
    double s = 0.0, d = 0.0;
    for (int e = rowptr[r]; e < rowptr[r + 1]; e++) {
      if (col[e] < 0) continue;
      double a = rho * kv[e] + mv[e];
      s += fabs(a);
      if (col[e] == r) d = a;
    }
    q = s / d;
  }
  q = block_max(q);
  if (threadIdx.x == 0) bmax[blockIdx.x] = q;
}

__global__ void k_max_red(const double* in, int n, double* out) {
  double q = -1.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) q = fmax(q, in[i]);
  q = block_max(q);
  if (threadIdx.x == 0) *out = q;
}

__global__ void k_diag_f(int64_t N, const int32_t* rowptr, const int32_t* col, const double* v,
                         float* d) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  double x = 0.0;
  for (int e = rowptr[r]; e < rowptr[r + 1]; e++)
    if (col[e] == r) x = v[e];
  d[r] = (float)x;
}

__global__ void k_to_f32(int64_t n, const double* a, float* b) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}

// column copies between a [N][ld] user array and slot b of a [N][B] multivector
__global__ void k_col_in(int64_t N, int B, int slot, const double* src, int64_t ld, int scol,
                         double* dst) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) dst[i * B + slot] = src[i * ld + scol];
}
__global__ void k_col_out(int64_t N, int B, int slot, const double* src, double* dst, int64_t ld,
                          int dcol) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) dst[i * ld + dcol] = src[i * B + slot];
}
__global__ void k_col_set(int64_t N, int B, int slot, double v, double* dst) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < N) dst[i * B + slot] = v;
}

// per-slot dot products <a_b, a_b> (for ||f||) of one column
__global__ void k_col_norm2(int64_t N, int B, int slot, const double* a, double* partials) {
  double acc[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    double v = a[i * B + slot];
    acc[0] += v * v;
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc[0];
}

// partial sums of ||f_b - q_b||^2 and ||f_b||^2 for one slot
__global__ void k_col_resid2(int64_t N, int B, int slot, const double* f, const double* q,
                             double* partials) {
  double acc[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double fv = f[i * B + slot], d = fv - q[i * B + slot];
    acc[0] += d * d;
    acc[1] += fv * fv;
  }
  block_sum<2>(acc);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = acc[0];
    partials[gridDim.x + blockIdx.x] = acc[1];
  }
}

__global__ void k_slot_admit(SlotState* S, int slot, const double* sums, int nb, double rho,
                             double tol, int maxit) {
  double v[1] = {0.0};
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v[0] += sums[i];
  block_sum<1>(v);
  if (threadIdx.x == 0) {
    SlotState& s = S[slot];
    std::memset(&s, 0, sizeof(SlotState));
    s.rho = rho;
    s.bb = v[0];
    s.rr = v[0];
    s.tol2 = tol * tol * v[0];
    s.first = 1;
    s.active = 1;
    s.maxit = maxit;
    s.status = FEM_OK;
    s.done = (v[0] > 0.0) ? 0 : 1;
  }
}

// per-slot finalisations (one block per slot, fixed order over the block partials)
__global__ void k_slot_fin_rz(SlotState* S, const double* partials, int nb, int B) {
  const int b = blockIdx.x;
  double v[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    v[0] += partials[(int64_t)(0 * B + b) * nb + i];
    v[1] += partials[(int64_t)(1 * B + b) * nb + i];
  }
  block_sum<2>(v);
  if (threadIdx.x == 0) {
    SlotState& s = S[b];
    if (!s.active || s.done) return;
    const double rz = v[0];
    double beta = 0.0;
    if (!s.first) beta = (rz - v[1]) / s.rz;
    if (!(rz > 0.0) || !isfinite(beta)) {
      s.status = FEM_EBREAKDOWN;
      s.done = 1;
    }
    s.beta = beta;
    s.rz = rz;
    s.zrp = v[1];
  }
}

__global__ void k_slot_fin_pq(SlotState* S, const double* partials, int nb, int B) {
  const int b = blockIdx.x;
  double v[1] = {0.0};
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v[0] += partials[(int64_t)b * nb + i];
  block_sum<1>(v);
  if (threadIdx.x == 0) {
    SlotState& s = S[b];
    if (!s.active || s.done) return;
    s.pq = v[0];
    if (!(v[0] > 0.0) || !isfinite(v[0])) {
      s.status = FEM_EBREAKDOWN;
      s.done = 1;
    } else {
      s.alpha = s.rz / v[0];
    }
  }
}

__global__ void k_slot_fin_rr(SlotState* S, const double* partials, int nb, int B) {
  const int b = blockIdx.x;
  double v[1] = {0.0};
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v[0] += partials[(int64_t)b * nb + i];
  block_sum<1>(v);
  if (threadIdx.x == 0) {
    SlotState& s = S[b];
    if (!s.active || s.done) return;
    s.rr = v[0];
    s.iter += 1;
    s.first = 0;
    if (!isfinite(v[0])) {
      s.status = FEM_EBREAKDOWN;
      s.done = 1;
    } else if (v[0] <= s.tol2) {
      s.done = 1;
    } else if (s.iter >= s.maxit) {
      s.status = FEM_ENOCONV;
      s.done = 1;
    }
  }
}

// p = z + beta p for live slots
__global__ void k_mv_update_p(int64_t N, int B, const double* z, double* p, const SlotState* S) {
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N * B;
       idx += (int64_t)gridDim.x * blockDim.x) {
    const int b = (int)(idx & (B - 1));
    const SlotState& s = S[b];
    if (!s.active || s.done) continue;
    p[idx] = z[idx] + s.beta * p[idx];
  }
}

// x += alpha p; r_prev = r; r -= alpha q; per-slot <r, r>
__global__ void k_mv_update_xr(int64_t N, int B, double* x, const double* p, double* r,
                               const double* q, double* rprev, const SlotState* S,
                               double* partials, int nblocks) {
  double acc[1] = {0.0};
  const int b = threadIdx.x % B;
  const bool live = S[b].active && !S[b].done;
  const double alpha = S[b].alpha;
  const int rpb = blockDim.x / B;
  for (int64_t base = (int64_t)blockIdx.x * rpb; base < N; base += (int64_t)gridDim.x * rpb) {
    const int64_t i = base + threadIdx.x / B;
    if (i < N && live) {
      const int64_t idx = i * B + b;
      x[idx] += alpha * p[idx];
      double ri = r[idx];
      rprev[idx] = ri;
      ri -= alpha * q[idx];
      r[idx] = ri;
      acc[0] += ri * ri;
    }
  }
  slot_partials<1>(acc, B, partials, nblocks, blockIdx.x);
}

// multivector dense-inverse output to FP64 z with per-slot dots (coarsest = finest case)
template <typename T>
__global__ void k_mv_out_dots(int64_t N, int B, const T* x, double* z64, const double* r1,
                              const double* r2, double* partials, int nblocks) {
  double acc[2] = {0.0, 0.0};
  const int b = threadIdx.x % B;
  const int rpb = blockDim.x / B;
  for (int64_t base = (int64_t)blockIdx.x * rpb; base < N; base += (int64_t)gridDim.x * rpb) {
    const int64_t i = base + threadIdx.x / B;
    if (i < N) {
      const int64_t idx = i * B + b;
      double z = (double)x[idx];
      z64[idx] = z;
      acc[0] += z * r1[idx];
      acc[1] += z * r2[idx];
    }
  }
  slot_partials<2>(acc, B, partials, nblocks, blockIdx.x);
}

template <typename T>
__global__ void k_mv_add_out(int64_t N, int B, const T* d, T* x, double* z64, const double* r1,
                             const double* r2, double* partials, int nblocks) {
  using AT = typename Arith<T>::type;
  double acc[2] = {0.0, 0.0};
  const int b = threadIdx.x % B;
  const int rpb = blockDim.x / B;
  for (int64_t base = (int64_t)blockIdx.x * rpb; base < N; base += (int64_t)gridDim.x * rpb) {
    const int64_t i = base + threadIdx.x / B;
    if (i < N) {
      const int64_t idx = i * B + b;
      AT xv = (AT)x[idx] + (AT)d[idx];
      x[idx] = (T)xv;
      if (z64) {
        double z = (double)xv;
        z64[idx] = z;
        acc[0] += z * r1[idx];
        acc[1] += z * r2[idx];
      }
    }
  }
  if (z64) slot_partials<2>(acc, B, partials, nblocks, blockIdx.x);
}

}  // namespace

// ------------------------------------------------------------------ session

struct BatchLevel {
  int64_t N = 0;
  bool stencil = false;
  const Csr4* A = nullptr;          // pattern (K and M values on it)
  const double* Kv64 = nullptr;     // FP64 pencil values
  const double* Mv64 = nullptr;
  DevBuf<float> Kv, Mv;             // FP32 pencil values
  DevBuf<float> kd, md;             // FP32 diagonals of K and M
  const Csr4* P = nullptr;
  const Csr4* R = nullptr;
  DevBuf<float> Pv, Rv;             // FP32 prolongation / restriction values
  bool coarsest = false;
  bool dense = false;
  DevBuf<double> Ainv;              // [B][N][N]
  DevBuf<float> x, b, r, d0, d1;    // [N][B]
};

struct BatchSession {
  System* S = nullptr;
  Hierarchy* H = nullptr;
  int B = 0;          // multivector width (power of two)
  int slots = 0;      // usable slots
  int64_t N = 0;
  pcg_opts o;
  std::vector<std::unique_ptr<BatchLevel>> L;
  DevBuf<double> x, r, rprev, p, q, z, f;   // [N][B] FP64
  DevBuf<double> rho;                       // [B]
  DevBuf<double> coef64;                    // [B][4] FP64 stencil coefficients of A(rho_b)
  DevBuf<LevCoef> lc;                       // [L][B]
  std::vector<LevCoef> hlc;
  DevBuf<SlotState> state;                  // [B]
  DevBuf<double> partials;
  DevBuf<double> scratch;
  SlotState* hstate = nullptr;              // pinned
  std::vector<int> in_use;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  long long per_iter = 0;
  int nb_fine = 0;
  ~BatchSession() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    if (hstate) cudaFreeHost(hstate);
  }
};

namespace {

unsigned mv_grid(int64_t N, int B) {
  const int ppb = 256 / B;
  return persistent_grid((N + ppb - 1) / ppb * 256, 256, 8);
}

// stencil grid: x covers the i-line in blocks of 256/B points, y strides over planes
dim3 mv_sgrid(int m, int B) {
  const int ppb = 256 / B;
  const int gx = (m + ppb - 1) / ppb;
  int gy = (8 * num_sms() + gx - 1) / gx;
  if (gy > m * m) gy = m * m;
  return dim3(gx, gy, 1);
}

// One V-cycle on all slots (FP32), levels lev.., with the finest-level right-hand side
// given in FP64 (b64) and the output written to z64 with per-slot dots.
void mv_vcycle(BatchSession& W, int lev, const double* b64, cudaStream_t st) {
  BatchLevel& L = *W.L[lev];
  const int B = W.B;
  const int64_t N = L.N;
  const int deg = W.H->o.degree;
  const bool l1 = W.H->o.smoother == AMG_SMOOTHER_L1_JACOBI;
  (void)l1;
  MvEpi<float> base;
  std::memset(&base, 0, sizeof(base));
  base.level = lev;
  base.lc = W.lc;
  base.B = B;
  base.rho = W.rho;
  if (!L.stencil) {
    base.kd = L.kd;
    base.md = L.md;
  }
  const unsigned g = mv_grid(N, B);
  const bool finest = lev == 0;
  double* part = W.partials;
  const int m = W.S->n - 1;
  const dim3 sg = mv_sgrid(m, B);
  auto op = [&](const float* v, MvEpi<float> e, bool dots) {
    if (L.stencil) {
      if (dots) {
        k_mv_stencil<float, 2><<<sg, 256, 0, st>>>(v, m, e, part, sg.x * sg.y);
        W.nb_fine = sg.x * sg.y;
      } else {
        k_mv_stencil<float, 0><<<sg, 256, 0, st>>>(v, m, e, nullptr, sg.x * sg.y);
      }
    } else {
      if (dots)
        k_mv_csr<float, float, 2><<<g, 256, 0, st>>>(N, L.A->rowptr, L.A->col, L.Kv, L.Mv, v, e, 0,
                                                     part, g);
      else
        k_mv_csr<float, float, 0><<<g, 256, 0, st>>>(N, L.A->rowptr, L.A->col, L.Kv, L.Mv, v, e, 0,
                                                     nullptr, g);
    }
    FEM_CHECK_LAUNCH();
  };
  if (L.coarsest && L.dense) {
    if (finest) {
      // single-level hierarchy: convert, solve, emit
      k_mv_cheb_zero<float><<<g, 256, 0, st>>>(N, B, b64, L.b, W.lc, lev, nullptr, nullptr, W.rho,
                                               L.r, L.d0, L.x);
      FEM_CHECK_LAUNCH();
    }
    unsigned gd = grid_for(N * B * 32, 256);
    k_mv_dense<float><<<gd, 256, 0, st>>>(N, B, L.Ainv, L.b, L.x);
    FEM_CHECK_LAUNCH();
    if (finest) {
      k_mv_out_dots<float><<<g, 256, 0, st>>>(N, B, L.x, W.z, W.r, W.rprev, part, g);
      FEM_CHECK_LAUNCH();
      W.nb_fine = (int)g;
    }
    return;
  }
  // pre-smoothing from zero
  k_mv_cheb_zero<float><<<g, 256, 0, st>>>(N, B, b64, L.b, W.lc, lev, base.kd, base.md, W.rho, L.r,
                                           L.d0, L.x);
  FEM_CHECK_LAUNCH();
  float* dold = L.d0;
  float* dnew = L.d1;
  for (int i = 1; i < deg; i++) {
    MvEpi<float> e = base;
    e.mode = 2;
    e.r = L.r;
    e.dold = dold;
    e.dnew = dnew;
    e.x = L.x;
    e.add_prev = 0;
    op(dold, e, false);
    std::swap(dold, dnew);
  }
  if (L.coarsest) {
    if (finest) {
      k_mv_out_dots<float><<<g, 256, 0, st>>>(N, B, L.x, W.z, W.r, W.rprev, part, g);
      FEM_CHECK_LAUNCH();
      W.nb_fine = (int)g;
    }
    return;
  }
  // residual, restriction, coarse correction, prolongation
  {
    MvEpi<float> e = base;
    e.mode = 1;
    e.y = L.r;
    e.b = L.b;
    op(L.x, e, false);
  }
  BatchLevel& C = *W.L[lev + 1];
  {
    MvEpi<float> e = base;
    e.y = C.b;
    e.mode = 0;
    k_mv_csr<float, float, 0><<<mv_grid(C.N, B), 256, 0, st>>>(C.N, L.R->rowptr, L.R->col, nullptr,
                                                               L.Rv, L.r, e, 0, nullptr, 0);
    FEM_CHECK_LAUNCH();
  }
  mv_vcycle(W, lev + 1, nullptr, st);
  {
    MvEpi<float> e = base;
    e.y = L.x;
    k_mv_csr<float, float, 0><<<g, 256, 0, st>>>(N, L.P->rowptr, L.P->col, nullptr, L.Pv, C.x, e, 1,
                                                 nullptr, 0);
    FEM_CHECK_LAUNCH();
  }
  // post-smoothing
  {
    MvEpi<float> e = base;
    e.mode = 3;
    e.b = L.b;
    e.r = L.r;
    e.dnew = L.d0;
    op(L.x, e, false);
  }
  if (deg == 1) {
    k_mv_add_out<float><<<g, 256, 0, st>>>(N, B, L.d0, L.x, finest ? W.z.p : nullptr, W.r, W.rprev,
                                           part, g);
    FEM_CHECK_LAUNCH();
    if (finest) W.nb_fine = (int)g;
    return;
  }
  dold = L.d0;
  dnew = L.d1;
  for (int i = 1; i < deg; i++) {
    const bool last = i == deg - 1;
    MvEpi<float> e = base;
    e.mode = 2;
    e.r = L.r;
    e.dold = dold;
    e.dnew = dnew;
    e.x = L.x;
    e.add_prev = i == 1;
    if (last && finest) {
      e.z64 = W.z;
      e.r1 = W.r;
      e.r2 = W.rprev;
    }
    op(dold, e, last && finest);
    if (last && finest && !L.stencil) W.nb_fine = (int)g;
    std::swap(dold, dnew);
  }
}

// q = A(rho_b) p in FP64 with per-slot <p, q>
int mv_apply64(BatchSession& W, cudaStream_t st) {
  BatchLevel& L = *W.L[0];
  const int B = W.B;
  const unsigned g = mv_grid(W.N, B);
  if (L.stencil) {
    const dim3 sg = mv_sgrid(W.S->n - 1, B);
    k_mv_stencil64<<<sg, 256, 0, st>>>(W.p, W.S->n - 1, W.coef64, B, W.q, W.state, W.partials,
                                       sg.x * sg.y);
    FEM_CHECK_LAUNCH();
    return (int)(sg.x * sg.y);
  } else {
    MvEpi<double> e;
    std::memset(&e, 0, sizeof(e));
    e.mode = 0;
    e.y = W.q;
    e.x = W.p;
    e.want_dot = 1;
    e.B = B;
    e.rho = W.rho;
    k_mv_csr<double, double, 1><<<g, 256, 0, st>>>(W.N, L.A->rowptr, L.A->col, L.Kv64, L.Mv64, W.p,
                                                   e, 0, W.partials, g);
  }
  FEM_CHECK_LAUNCH();
  return (int)g;
}

void batch_iteration(BatchSession& W, cudaStream_t st) {
  const int B = W.B;
  const int64_t N = W.N;
  mv_vcycle(W, 0, W.r, st);
  k_slot_fin_rz<<<B, 256, 0, st>>>(W.state, W.partials, W.nb_fine, B);
  FEM_CHECK_LAUNCH();
  const unsigned ge = persistent_grid(N * B, 256, 8);
  k_mv_update_p<<<ge, 256, 0, st>>>(N, B, W.z, W.p, W.state);
  FEM_CHECK_LAUNCH();
  int nb = mv_apply64(W, st);
  k_slot_fin_pq<<<B, 256, 0, st>>>(W.state, W.partials, nb, B);
  FEM_CHECK_LAUNCH();
  const unsigned gx = mv_grid(N, B);
  k_mv_update_xr<<<gx, 256, 0, st>>>(N, B, W.x, W.p, W.r, W.q, W.rprev, W.state, W.partials, gx);
  FEM_CHECK_LAUNCH();
  k_slot_fin_rr<<<B, 256, 0, st>>>(W.state, W.partials, gx, B);
  FEM_CHECK_LAUNCH();
}

double slot_gershgorin(const Csr4& A, const double* kv, const double* mv, double rho,
                       DevBuf<double>& scratch, cudaStream_t st) {
  const int64_t N = A.nrows;
  unsigned g = grid_for(N, 256);
  if (scratch.n < g + 1) scratch.alloc(g + 1);
  k_mv_gersh<<<g, 256, 0, st>>>(N, A.rowptr, A.col, kv, mv, rho, scratch);
  FEM_CHECK_LAUNCH();
  k_max_red<<<1, 1024, 0, st>>>(scratch, (int)g, scratch.p + g);
  FEM_CHECK_LAUNCH();
  double h = 0;
  FEM_CUDA(cudaMemcpyAsync(&h, scratch.p + g, 8, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  return h;
}

}  // namespace

int64_t batch_footprint(const System& S, const Hierarchy& H, int slots) {
  int B = 1;
  while (B < slots) B <<= 1;
  int64_t bytes = 7 * S.N * B * 8;  // x r rprev p q z f
  for (auto& Lp : H.L) {
    bytes += 5 * Lp->N * B * 4;
    bytes += (Lp->A->nnz) * 8 + Lp->N * 8;
    if (!Lp->coarsest) bytes += (Lp->P.nnz + Lp->R.nnz) * 4;
    if (Lp->coarsest && Lp->N <= H.o.coarse_max) bytes += (int64_t)B * Lp->N * Lp->N * 8;
  }
  return bytes;
}

BatchSession* batch_create(System& S, Hierarchy& H, int slots, const pcg_opts& o, cudaStream_t st) {
  FEM_REQUIRE(slots >= 1 && slots <= MAXB, FEM_EINVAL, "pcg_batch_create: slots in [1, 64]");
  FEM_REQUIRE(S.pencil, FEM_EINVAL,
              "pcg_batch_create: the system must keep its pencil (keep_pencil at assembly)");
  FEM_REQUIRE(H.o.degree <= 2 || H.o.smoother == AMG_SMOOTHER_L1_JACOBI, FEM_EUNSUPPORTED,
              "pcg_batch_create: Chebyshev degree <= 2 in batched solves");
  auto W = std::make_unique<BatchSession>();
  W->S = &S;
  W->H = &H;
  int B = 1;
  while (B < slots) B <<= 1;
  if (B < 1) B = 1;
  W->B = B;
  W->slots = slots;
  W->N = S.N;
  W->o = o;
  const int64_t N = S.N;
  for (size_t l = 0; l < H.L.size(); l++) {
    Level& Lv = *H.L[l];
    auto BL = std::make_unique<BatchLevel>();
    BL->N = Lv.N;
    BL->stencil = Lv.stencil;
    BL->A = Lv.A;
    BL->Kv64 = l == 0 ? S.Kv.p : Lv.Kv.p;
    BL->Mv64 = l == 0 ? S.Mv.p : Lv.Mv.p;
    FEM_REQUIRE(BL->Kv64 && BL->Mv64, FEM_EINVAL, "pcg_batch_create: hierarchy without pencil values");
    const int64_t nnz = Lv.A->nnz;
    if (!BL->stencil) {
      BL->Kv.alloc(nnz);
      BL->Mv.alloc(nnz);
      k_to_f32<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, BL->Kv64, BL->Kv);
      k_to_f32<<<grid_for(nnz, 256), 256, 0, st>>>(nnz, BL->Mv64, BL->Mv);
      BL->kd.alloc(Lv.N);
      BL->md.alloc(Lv.N);
      k_diag_f<<<grid_for(Lv.N, 256), 256, 0, st>>>(Lv.N, Lv.A->rowptr, Lv.A->col, BL->Kv64, BL->kd);
      k_diag_f<<<grid_for(Lv.N, 256), 256, 0, st>>>(Lv.N, Lv.A->rowptr, Lv.A->col, BL->Mv64, BL->md);
      FEM_CHECK_LAUNCH();
    }
    BL->coarsest = Lv.coarsest;
    if (!Lv.coarsest) {
      BL->P = &Lv.P;
      BL->R = &Lv.R;
      BL->Pv.alloc(Lv.P.nnz);
      BL->Rv.alloc(Lv.R.nnz);
      k_to_f32<<<grid_for(Lv.P.nnz, 256), 256, 0, st>>>(Lv.P.nnz, Lv.P.val, BL->Pv);
      k_to_f32<<<grid_for(Lv.R.nnz, 256), 256, 0, st>>>(Lv.R.nnz, Lv.R.val, BL->Rv);
      FEM_CHECK_LAUNCH();
    } else {
      BL->dense = Lv.N <= H.o.coarse_max;
      if (BL->dense) BL->Ainv.alloc((size_t)B * Lv.N * Lv.N);
    }
    BL->x.alloc(Lv.N * B);
    BL->b.alloc(Lv.N * B);
    BL->r.alloc(Lv.N * B);
    BL->d0.alloc(Lv.N * B);
    BL->d1.alloc(Lv.N * B);
    W->L.push_back(std::move(BL));
  }
  for (auto* v : {&W->x, &W->r, &W->rprev, &W->p, &W->q, &W->z, &W->f}) {
    v->alloc(N * B);
    FEM_CUDA(cudaMemsetAsync(v->p, 0, 8 * N * B, st));
  }
  W->rho.alloc(B);
  W->coef64.alloc(4 * B);
  W->lc.alloc(H.L.size() * B);
  W->hlc.assign(H.L.size() * B, LevCoef{});
  W->state.alloc(B);
  FEM_CUDA(cudaMemsetAsync(W->state, 0, sizeof(SlotState) * B, st));
  FEM_CUDA(cudaMemsetAsync(W->rho, 0, 8 * B, st));
  FEM_CUDA(cudaMemsetAsync(W->coef64, 0, 32 * B, st));
  FEM_CUDA(cudaMemsetAsync(W->lc, 0, sizeof(LevCoef) * H.L.size() * B, st));
  W->partials.alloc((size_t)2 * B * (8 * num_sms() + 1) + 4 * (size_t)kMaxPartialBlocks);
  W->scratch.alloc(4 * 8 * (size_t)num_sms() + 64);
  FEM_CUDA(cudaMallocHost(&W->hstate, sizeof(SlotState) * B));
  W->in_use.assign(B, 0);
  // one iteration as a CUDA graph
  cudaStream_t cs;
  FEM_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaEvent_t ev;
  FEM_CUDA(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
  FEM_CUDA(cudaEventRecord(ev, st));
  FEM_CUDA(cudaStreamWaitEvent(cs, ev, 0));
  const long long c0 = launches_now();
  FEM_CUDA(cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal));
  try {
    batch_iteration(*W, cs);
  } catch (...) {
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(cs, &g);
    if (g) cudaGraphDestroy(g);
    cudaStreamDestroy(cs);
    cudaEventDestroy(ev);
    throw;
  }
  FEM_CUDA(cudaStreamEndCapture(cs, &W->graph));
  FEM_CUDA(cudaGraphInstantiate(&W->exec, W->graph, 0));
  W->per_iter = launches_now() - c0;
  count_launches(-W->per_iter);
  FEM_CUDA(cudaStreamSynchronize(st));
  cudaStreamDestroy(cs);
  cudaEventDestroy(ev);
  return W.release();
}

// Load f (length N, column fcol of an [N][ld] array) and rho into a free slot.
int batch_admit(BatchSession& W, const double* f, int64_t ld, int fcol, double rho, cudaStream_t st) {
  FEM_REQUIRE(rho > 0.0 && std::isfinite(rho), FEM_EINVAL, "pcg_batch_admit: rho > 0");
  int slot = -1;
  for (int b = 0; b < W.slots; b++)
    if (!W.in_use[b]) {
      slot = b;
      break;
    }
  FEM_REQUIRE(slot >= 0, FEM_ENOMEM, "pcg_batch_admit: no free slot");
  const int B = W.B;
  const int64_t N = W.N;
  System& S = *W.S;
  Hierarchy& H = *W.H;
  const unsigned g1 = grid_for(N, 256);
  k_col_in<<<g1, 256, 0, st>>>(N, B, slot, f, ld, fcol, W.f);
  k_col_in<<<g1, 256, 0, st>>>(N, B, slot, f, ld, fcol, W.r);
  k_col_set<<<g1, 256, 0, st>>>(N, B, slot, 0.0, W.x);
  k_col_set<<<g1, 256, 0, st>>>(N, B, slot, 0.0, W.p);
  k_col_set<<<g1, 256, 0, st>>>(N, B, slot, 0.0, W.rprev);
  FEM_CHECK_LAUNCH();
  FEM_CUDA(cudaMemcpyAsync(W.rho.p + slot, &rho, 8, cudaMemcpyHostToDevice, st));
  // per-level smoother coefficients for this rho
  for (size_t l = 0; l < H.L.size(); l++) {
    Level& Lv = *H.L[l];
    BatchLevel& BL = *W.L[l];
    LevCoef c{};
    double lmax;
    const double* kv = BL.Kv64;
    const double* mv = BL.Mv64;
    if (Lv.stencil) {
      const double a[4] = {rho * S.stK.c0 + S.stM.c0, rho * S.stK.ca + S.stM.ca,
                           rho * S.stK.cf + S.stM.cf, rho * S.stK.cb + S.stM.cb};
      c.c0 = (float)a[0];
      c.ca = (float)a[1];
      c.cf = (float)a[2];
      c.cb = (float)a[3];
      c.sinv = (float)(1.0 / a[0]);
      double coef[4] = {a[0], a[1], a[2], a[3]};
      FEM_CUDA(cudaMemcpyAsync(W.coef64.p + 4 * slot, coef, 32, cudaMemcpyHostToDevice, st));
      // every row has the diagonal a[0] and a subset of the interior row's neighbours, so
      // the Gershgorin bound is the interior row's sum
      lmax = (std::fabs(a[0]) + 6 * std::fabs(a[1]) + 6 * std::fabs(a[2]) + 2 * std::fabs(a[3])) /
             a[0];
    } else {
      lmax = slot_gershgorin(*Lv.A, kv, mv, rho, W.scratch, st);
    }
    if (H.o.smoother == AMG_SMOOTHER_L1_JACOBI) {
      c.inv_theta = 1.0f;
    } else {
      ChebCoef cc = cheb_coefficients(lmax, H.o.cheb_ratio, H.o.degree);
      c.inv_theta = (float)cc.inv_theta;
      c.c1 = (float)cc.c1[1];
      c.c2 = (float)cc.c2[1];
    }
    W.hlc[l * B + slot] = c;
    FEM_CUDA(cudaMemcpyAsync(W.lc.p + l * B + slot, &W.hlc[l * B + slot], sizeof(LevCoef),
                             cudaMemcpyHostToDevice, st));
    if (BL.coarsest && BL.dense) {
      const int64_t Nc = Lv.N;
      double* A0 = BL.Ainv.p + (int64_t)slot * Nc * Nc;
      DevBuf<double> tmp(Nc * Nc, st);
      k_mv_dense_build<<<grid_for(Nc, 128), 128, 0, st>>>(Nc, Lv.A->rowptr, Lv.A->col, kv, mv,
                                                          W.rho, slot, A0);
      FEM_CHECK_LAUNCH();
      double* src = A0;
      double* dst = tmp.p;
      const unsigned gg = persistent_grid(Nc * Nc, 256, 4);
      for (int64_t k = 0; k < Nc; k++) {
        k_gj_step_b<<<gg, 256, 0, st>>>(Nc, k, src, dst);
        FEM_CHECK_LAUNCH();
        std::swap(src, dst);
      }
      if (src != A0) FEM_CUDA(cudaMemcpyAsync(A0, src, 8 * Nc * Nc, cudaMemcpyDeviceToDevice, st));
    }
  }
  // ||f|| and the slot's CG state
  const unsigned gn = persistent_grid(N, 256, 4);
  k_col_norm2<<<gn, 256, 0, st>>>(N, B, slot, W.f, W.scratch);
  FEM_CHECK_LAUNCH();
  k_slot_admit<<<1, 256, 0, st>>>(W.state, slot, W.scratch, gn, rho, W.o.tol, W.o.max_iter);
  FEM_CHECK_LAUNCH();
  FEM_CUDA(cudaStreamSynchronize(st));
  W.in_use[slot] = 1;
  return slot;
}

void batch_step(BatchSession& W, int iters, cudaStream_t st) {
  for (int i = 0; i < iters; i++) {
    FEM_CUDA(cudaGraphLaunch(W.exec, st));
    count_launches(W.per_iter);
  }
}

void batch_poll(BatchSession& W, int32_t* state, int32_t* iters, double* relres, cudaStream_t st) {
  FEM_CUDA(cudaMemcpyAsync(W.hstate, W.state, sizeof(SlotState) * W.B, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  for (int b = 0; b < W.slots; b++) {
    const SlotState& s = W.hstate[b];
    int code = -1;
    if (W.in_use[b]) code = !s.done ? 0 : (s.status == FEM_OK ? 1 : 2);
    if (state) state[b] = code;
    if (iters) iters[b] = W.in_use[b] ? s.iter : 0;
    if (relres) relres[b] = (W.in_use[b] && s.bb > 0) ? std::sqrt(s.rr / s.bb) : 0.0;
  }
}

void batch_retire(BatchSession& W, int slot, double* u, int64_t ld, int ucol, cudaStream_t st) {
  FEM_REQUIRE(slot >= 0 && slot < W.slots && W.in_use[slot], FEM_EINVAL,
              "pcg_batch_retire: slot not in use");
  k_col_out<<<grid_for(W.N, 256), 256, 0, st>>>(W.N, W.B, slot, W.x, u, ld, ucol);
  FEM_CHECK_LAUNCH();
  // deactivate
  SlotState off{};
  FEM_CUDA(cudaMemcpyAsync(W.state.p + slot, &off, sizeof(SlotState), cudaMemcpyHostToDevice, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  W.in_use[slot] = 0;
}

void batch_destroy(BatchSession* W) { delete W; }

// ||f_b - A(rho_b) x_b|| / ||f_b|| for every slot in use (FP64, recomputed).
static void batch_true_residual(BatchSession& W, double* out, cudaStream_t st) {
  const int B = W.B;
  const int64_t N = W.N;
  BatchLevel& L = *W.L[0];
  const unsigned g = mv_grid(N, B);
  if (L.stencil) {
    const dim3 sg = mv_sgrid(W.S->n - 1, B);
    k_mv_stencil64<<<sg, 256, 0, st>>>(W.x, W.S->n - 1, W.coef64, B, W.q, nullptr, W.partials,
                                       sg.x * sg.y);
  } else {
    MvEpi<double> e;
    std::memset(&e, 0, sizeof(e));
    e.mode = 0;
    e.y = W.q;
    e.x = W.x;
    e.B = B;
    e.rho = W.rho;
    k_mv_csr<double, double, 0><<<g, 256, 0, st>>>(N, L.A->rowptr, L.A->col, L.Kv64, L.Mv64, W.x, e,
                                                   0, nullptr, 0);
  }
  FEM_CHECK_LAUNCH();
  const unsigned gn = persistent_grid(N, 256, 4);
  std::vector<double> h(2 * gn);
  for (int b = 0; b < W.slots; b++) {
    if (!W.in_use[b]) continue;
    k_col_resid2<<<gn, 256, 0, st>>>(N, B, b, W.f, W.q, W.scratch);
    FEM_CHECK_LAUNCH();
    FEM_CUDA(cudaMemcpyAsync(h.data(), W.scratch, 16 * gn, cudaMemcpyDeviceToHost, st));
    FEM_CUDA(cudaStreamSynchronize(st));
    double rr = 0, ff = 0;
    for (unsigned i = 0; i < gn; i++) {
      rr += h[i];
      ff += h[gn + i];
    }
    out[b] = ff > 0 ? std::sqrt(rr / ff) : 0.0;
  }
}

fem_status pcg_multi(System& S, Hierarchy& H, const double* f, double* u, int nrhs,
                     const double* rho_k, const pcg_opts& o, cudaStream_t user, pcg_result* res) {
  FEM_REQUIRE(nrhs >= 1 && nrhs <= MAXB, FEM_EINVAL, "pcg_solve: nrhs in [1, 64]");
  std::unique_ptr<BatchSession> W(batch_create(S, H, nrhs, o, user));
  for (int k = 0; k < nrhs; k++) batch_admit(*W, f, nrhs, k, rho_k[k], user);
  cudaEvent_t e0, e1;
  FEM_CUDA(cudaEventCreate(&e0));
  FEM_CUDA(cudaEventCreate(&e1));
  FEM_CUDA(cudaEventRecord(e0, user));
  std::vector<int32_t> st(nrhs), it(nrhs);
  std::vector<double> rr(nrhs);
  int done_all = 0;
  for (int guard = 0; guard < o.max_iter + 8 && !done_all; guard += 4) {
    batch_step(*W, 4, user);
    batch_poll(*W, st.data(), it.data(), rr.data(), user);
    done_all = 1;
    for (int k = 0; k < nrhs; k++)
      if (st[k] == 0) done_all = 0;
    if (o.cancel_host && *o.cancel_host) break;
  }
  FEM_CUDA(cudaEventRecord(e1, user));
  FEM_CUDA(cudaEventSynchronize(e1));
  float ms = 0;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  fem_status all = FEM_OK;
  std::vector<double> trr(W->B, 0.0);
  batch_true_residual(*W, trr.data(), user);
  for (int k = 0; k < nrhs; k++) {
    batch_retire(*W, k, u, nrhs, k, user);
    res[k].iterations = it[k];
    res[k].status = st[k] == 1 ? FEM_OK : (st[k] == 0 ? FEM_ENOCONV : W->hstate[k].status);
    res[k].relres = trr[k];
    res[k].prec_relres = 0.0;
    res[k].solve_ms = ms;
    if (res[k].status != FEM_OK && all == FEM_OK) all = (fem_status)res[k].status;
  }
  if (o.cancel_host && *o.cancel_host) all = FEM_ECANCELLED;
  FEM_CUDA(cudaStreamSynchronize(user));
  return all;
}

}  // namespace fem

