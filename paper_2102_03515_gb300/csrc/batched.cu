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

#include "dfloat.cuh"
#include "solver.cuh"

namespace fem {

long long launches_now();

namespace {

constexpr int MAXB = 64;

struct SlotState {
  double rho, bb, rr, rz, rz_old, pq, alpha, beta, zrp, tol2;
  int iter, first, active, done, status, maxit;
  int dfop;   // q = A p in double-float (the uniform grid, tolerance >= 1e-12)
  int pad1;
};

// per-slot coefficients of the double-float operator: c0, ca, cf, cb times 2^s, each as
// three FP32 numbers (exact)
struct MvDf {
  float C[4][3];
  int s;
  int pad[3];
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

// The epilogue in two parts, like the single-vector one: mv_load() fetches the operands of
// (i, b) so that kernels can issue those loads early, mv_apply() finishes the entry;
// "centre" is v[i][b] (dold in mode 2), which the stencil kernels hold in a register.
template <typename T>
struct MvOps {
  typename Arith<T>::type a, x, s;
  double r1, r2;
};

// MODE >= 0 fixes the mode at compile time (5: mode 2 with the FP64 output, 2: without);
// -1 reads it at run time.
template <typename T, int MODE = -1>
__device__ __forceinline__ MvOps<T> mv_load(const MvEpi<T>& e, int64_t i, int b) {
  using AT = typename Arith<T>::type;
  MvOps<T> o;
  o.a = (AT)0;
  o.x = (AT)0;
  o.s = (AT)0;
  o.r1 = 0.0;
  o.r2 = 0.0;
  const int64_t idx = i * e.B + b;
  const bool zo = MODE == 5 || (MODE < 0 && e.z64 != nullptr);
  switch (MODE >= 0 ? (MODE == 5 ? 2 : MODE) : e.mode) {
    case 0:
      if (e.want_dot) o.a = (AT)e.x[idx];
      break;
    case 1:
      o.a = (AT)e.b[idx];
      break;
    case 3:
      o.a = (AT)e.b[idx];
      o.s = (AT)smoother_sinv(e, i, b);
      break;
    case 2:
      o.a = (AT)e.r[idx];
      o.s = (AT)smoother_sinv(e, i, b);
      o.x = (AT)e.x[idx];
      if (zo) {
        o.r1 = e.r1[idx];
        o.r2 = e.r2[idx];
      }
      break;
  }
  return o;
}

template <typename T, int MODE = -1>
__device__ __forceinline__ void mv_apply(const MvEpi<T>& e, int64_t i, int b,
                                         typename Arith<T>::type av,
                                         typename Arith<T>::type centre, const MvOps<T>& o,
                                         double acc[2]) {
  using AT = typename Arith<T>::type;
  const int64_t idx = i * e.B + b;
  const bool zo = MODE == 5 || (MODE < 0 && e.z64 != nullptr);
  switch (MODE >= 0 ? (MODE == 5 ? 2 : MODE) : e.mode) {
    case 0:
      e.y[idx] = (T)av;
      if (e.want_dot) acc[0] += (double)o.a * (double)av;
      break;
    case 1:
      e.y[idx] = (T)(o.a - av);
      break;
    case 3: {
      const LevCoef& c = e.lc[e.level * e.B + b];
      AT rr = o.s * (o.a - av);
      e.r[idx] = (T)rr;
      e.dnew[idx] = (T)((AT)c.inv_theta * rr);
    } break;
    case 2: {
      const LevCoef& c = e.lc[e.level * e.B + b];
      AT rr = o.a - o.s * av;
      AT dl = centre;
      AT dn = (AT)c.c1 * dl + (AT)c.c2 * rr;
      e.r[idx] = (T)rr;
      e.dnew[idx] = (T)dn;
      AT xv = o.x + (e.add_prev ? dl : (AT)0) + dn;
      e.x[idx] = (T)xv;
      if (zo) {
        double z = (double)xv;
        e.z64[idx] = z;
        acc[0] += z * o.r1;
        acc[1] += z * o.r2;
      }
    } break;
  }
}

__device__ __forceinline__ void l2_prefetch(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

// hint the L2 to fetch the epilogue operands of (i, b) (no registers, no wait)
template <typename T, int MODE = -1>
__device__ __forceinline__ void mv_prefetch(const MvEpi<T>& e, int64_t i, int b) {
  const int64_t idx = i * e.B + b;
  switch (MODE >= 0 ? (MODE == 5 ? 2 : MODE) : e.mode) {
    case 1:
    case 3:
      l2_prefetch(e.b + idx);
      break;
    case 2:
      l2_prefetch(e.r + idx);
      l2_prefetch(e.x + idx);
      if (MODE == 5) {
        if (e.r1) l2_prefetch(e.r1 + idx);
        if (e.r2) l2_prefetch(e.r2 + idx);
      }
      break;
    default:
      break;
  }
}

template <typename T>
__device__ __forceinline__ void mv_epi(const MvEpi<T>& e, int64_t i, int b, typename Arith<T>::type av,
                                       double acc[2]) {
  using AT = typename Arith<T>::type;
  const AT centre = e.mode == 2 ? (AT)e.dold[i * e.B + b] : (AT)0;
  mv_apply<T>(e, i, b, av, centre, mv_load<T>(e, i, b), acc);
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

// The same reduction for kernels whose threads each hold VS consecutive slots of one row:
// thread t covers row t / (B / VS) of the block and slots (t % (B / VS)) * VS + q.  The
// partial sum of a slot adds the block's rows in ascending order, as above.
template <int VS>
__device__ __forceinline__ void slot_partials_vs(double (&acc)[VS][2], int nv, int B,
                                                 double* partials, int nblocks, int bid) {
  __shared__ double sh[2][256 * VS];
  const int tpr = B / VS;
  const int r = threadIdx.x / tpr, g = threadIdx.x % tpr;
  const int rpb = blockDim.x / tpr;
  for (int k = 0; k < nv; k++)
    for (int q = 0; q < VS; q++) sh[k][r * B + g * VS + q] = acc[q][k];
  __syncthreads();
  if ((int)threadIdx.x < B) {
    for (int k = 0; k < nv; k++) {
      double s = 0.0;
      for (int rr = 0; rr < rpb; rr++) s += sh[k][rr * B + threadIdx.x];
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

// Column marching (as in the single-vector stencil): thread (point i, slot b) of a block
// walks k over KZV planes of each of its rows j, keeping in registers the values it needs
// again one plane later (7 loads per point instead of 15) and issuing the loads of point
// k + 1 before finishing point k.  grid: x over groups of 256 / B points along i, y strides
// over j, z over plane ranges.
template <typename T, int NV, int KZV, int MODE, int PF = 0>
__global__ void __launch_bounds__(256) k_mv_stencil_col(const T* __restrict__ v, int m, MvEpi<T> e,
                                                        double* partials, int nblocks) {
  using AT = typename Arith<T>::type;
  using Ops = MvOps<T>;
  const int B = e.B;
  const int b = threadIdx.x & (B - 1);
  const int ppb = blockDim.x / B;
  const int i = blockIdx.x * ppb + threadIdx.x / B;
  const int k0 = blockIdx.z * KZV;
  const int kend = min(k0 + KZV, m);
  double acc[2] = {0.0, 0.0};
  const LevCoef& c = e.lc[e.level * B + b];
  const AT a0 = (AT)c.c0, aa = (AT)c.ca, af = (AT)c.cf, ab = (AT)c.cb;
  const int64_t sB = B, sj = (int64_t)m * B, sk = (int64_t)m * m * B, pk = (int64_t)m * m;
  if (i < m) {
    for (int j = blockIdx.y; j < m; j += gridDim.y) {
      const bool im = i > 0, ip = i < m - 1, jm = j > 0, jp = j < m - 1;
      const int64_t row0 = (int64_t)i + (int64_t)m * j;
      const T* col = v + row0 * B + b;
      auto ld = [&](bool ok, int k, int64_t off) -> AT {
        return (ok && k >= 0 && k < m) ? (AT)__ldg(col + sk * k + off) : (AT)0;
      };
      AT cm = ld(true, k0 - 1, 0);
      AT m_im = ld(im, k0 - 1, -sB), m_jm = ld(jm, k0 - 1, -sj), m_ijm = ld(im && jm, k0 - 1, -sB - sj);
      AT c0v = ld(true, k0, 0);
      AT p_ip = ld(ip, k0, sB), p_jp = ld(jp, k0, sj), p_ijp = ld(ip && jp, k0, sB + sj);
      AT z_im = ld(im, k0, -sB), z_jm = ld(jm, k0, -sj), z_ijm = ld(im && jm, k0, -sB - sj);
      AT cp = ld(true, k0 + 1, 0);
      AT n_ip = ld(ip, k0 + 1, sB), n_jp = ld(jp, k0 + 1, sj), n_ijp = ld(ip && jp, k0 + 1, sB + sj);
      Ops op = mv_load<T, MODE>(e, row0 + pk * k0, b);
      for (int k = k0; k < kend; k++) {
        if (PF > 0 && k + PF < kend) {  // L2 prefetch of the streams PF planes ahead (in bounds)
          if (k + PF + 1 < m) l2_prefetch(col + sk * (k + PF + 1));
          mv_prefetch<T, MODE>(e, row0 + pk * (k + PF), b);
        }
        const bool more = k + 1 < kend;
        const AT z2_im = ld(im && more, k + 1, -sB), z2_jm = ld(jm && more, k + 1, -sj),
                 z2_ijm = ld(im && jm && more, k + 1, -sB - sj);
        const AT cp2 = ld(more, k + 2, 0);
        const AT n2_ip = ld(ip && more, k + 2, sB), n2_jp = ld(jp && more, k + 2, sj),
                 n2_ijp = ld(ip && jp && more, k + 2, sB + sj);
        Ops op2;
        if (more) op2 = mv_load<T, MODE>(e, row0 + pk * (k + 1), b);
        const AT axis = z_im + p_ip + z_jm + p_jp + cm + cp;
        const AT face = p_ijp + z_ijm + n_ip + m_im + n_jp + m_jm;
        const AT body = n_ijp + m_ijm;
        const AT av = a0 * c0v + aa * axis + af * face + ab * body;
        mv_apply<T, MODE>(e, row0 + pk * k, b, av, c0v, op, acc);
        cm = c0v;
        m_im = z_im;
        m_jm = z_jm;
        m_ijm = z_ijm;
        c0v = cp;
        p_ip = n_ip;
        p_jp = n_jp;
        p_ijp = n_ijp;
        z_im = z2_im;
        z_jm = z2_jm;
        z_ijm = z2_ijm;
        cp = cp2;
        n_ip = n2_ip;
        n_jp = n2_jp;
        n_ijp = n2_ijp;
        if (more) op = op2;
      }
    }
  }
  if (NV > 0 && partials)
    slot_partials<2>(acc, B, partials, nblocks,
                     blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z));
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

// q = A(rho_b) p for CG's FP64 search directions in double-float arithmetic (the FP32 pipe):
// p arrives also as FP32 pairs (hi, lo) with p = hi + lo exactly (the update rounds p to 48
// bits), and the class sums, products and their sum follow the single-vector operator
// k_stencil_df term for term, in the same order; the result is hi + lo rounded to FP64 and
// <p, q> is summed in FP64.  Thread (i, j, slot) marches its column in k like
// k_mv_stencil_col (7 pair loads per point).  Slots without the double-float operator, and a
// slot one of whose entries of p left the pairs' range (its rflag), take the FP64 operator.
__global__ void __launch_bounds__(256) k_mv_stencil_df(const float2* __restrict__ v2,
                                                       const double* __restrict__ v, int m,
                                                       const MvDf* __restrict__ dfc,
                                                       const double* coef /* [B][4] */, int B,
                                                       double* y, const SlotState* slots,
                                                       const int* rflag, double* partials,
                                                       int nblocks) {
  const int b = threadIdx.x & (B - 1);
  const int ppb = blockDim.x / B;
  const int i = blockIdx.x * ppb + threadIdx.x / B;
  constexpr int KZV = 16;
  const int k0 = blockIdx.z * KZV;
  const int kend = min(k0 + KZV, m);
  double acc[1] = {0.0};
  const bool live = slots[b].active && !slots[b].done;
  const bool df = slots[b].dfop && !rflag[b];
  const int64_t sB = B, sj = (int64_t)m * B, sk = (int64_t)m * m * B;
  if (i < m && live && df) {
    float C[4][3];
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
      for (int w = 0; w < 3; w++) C[u][w] = dfc[b].C[u][w];
    const int sc = dfc[b].s;
    for (int j = blockIdx.y; j < m; j += gridDim.y) {
      const bool im = i > 0, ip = i < m - 1, jm = j > 0, jp = j < m - 1;
      const int64_t row0 = ((int64_t)i + (int64_t)m * j) * B + b;
      const float2* col = v2 + row0;
      const float2 Z = make_float2(0.0f, 0.0f);
      auto ld = [&](bool ok, int k, int64_t off) -> float2 {
        return (ok && k >= 0 && k < m) ? __ldg(col + sk * k + off) : Z;
      };
      float2 cm = ld(true, k0 - 1, 0);
      float2 m_im = ld(im, k0 - 1, -sB), m_jm = ld(jm, k0 - 1, -sj), m_ijm = ld(im && jm, k0 - 1, -sB - sj);
      float2 c0v = ld(true, k0, 0);
      float2 p_ip = ld(ip, k0, sB), p_jp = ld(jp, k0, sj), p_ijp = ld(ip && jp, k0, sB + sj);
      float2 z_im = ld(im, k0, -sB), z_jm = ld(jm, k0, -sj), z_ijm = ld(im && jm, k0, -sB - sj);
      float2 cp = ld(true, k0 + 1, 0);
      float2 n_ip = ld(ip, k0 + 1, sB), n_jp = ld(jp, k0 + 1, sj), n_ijp = ld(ip && jp, k0 + 1, sB + sj);
      for (int k = k0; k < kend; k++) {
        const bool more = k + 1 < kend;
        const float2 z2_im = ld(im && more, k + 1, -sB), z2_jm = ld(jm && more, k + 1, -sj),
                     z2_ijm = ld(im && jm && more, k + 1, -sB - sj);
        const float2 cp2 = ld(more, k + 2, 0);
        const float2 n2_ip = ld(ip && more, k + 2, sB), n2_jp = ld(jp && more, k + 2, sj),
                     n2_ijp = ld(ip && jp && more, k + 2, sB + sj);
        const int64_t o = row0 + sk * k;
        const double pc = v[o];
        // class sums (the order of k_stencil_df)
        float as = z_im.x, ac = z_im.y;
        df_acc(as, ac, p_ip.x, p_ip.y);
        df_acc(as, ac, z_jm.x, z_jm.y);
        df_acc(as, ac, p_jp.x, p_jp.y);
        df_acc(as, ac, cm.x, cm.y);
        df_acc(as, ac, cp.x, cp.y);
        float fs = p_ijp.x, fc = p_ijp.y;
        df_acc(fs, fc, z_ijm.x, z_ijm.y);
        df_acc(fs, fc, n_ip.x, n_ip.y);
        df_acc(fs, fc, m_im.x, m_im.y);
        df_acc(fs, fc, n_jp.x, n_jp.y);
        df_acc(fs, fc, m_jm.x, m_jm.y);
        float bs = n_ijp.x, bc = n_ijp.y;
        df_acc(bs, bc, m_ijm.x, m_ijm.y);
        float p0, l0, p1, l1, p2, l2, p3, l3;
        df_mul(C[0][0], C[0][1], C[0][2], c0v.x, c0v.y, p0, l0);
        df_mul(C[1][0], C[1][1], C[1][2], as, ac, p1, l1);
        df_mul(C[2][0], C[2][1], C[2][2], fs, fc, p2, l2);
        df_mul(C[3][0], C[3][1], C[3][2], bs, bc, p3, l3);
        float ys = p0, yc = l0;
        df_acc(ys, yc, p1, l1);
        df_acc(ys, yc, p2, l2);
        df_acc(ys, yc, p3, l3);
        const float yh = ys + yc;   // FastTwoSum: |yc| small against ys
        const float yl = yc - (yh - ys);
        const double av = df_to_double(yh, sc) + df_to_double(yl, sc);
        y[o] = av;
        acc[0] += pc * av;
        cm = c0v;
        m_im = z_im;
        m_jm = z_jm;
        m_ijm = z_ijm;
        c0v = cp;
        p_ip = n_ip;
        p_jp = n_jp;
        p_ijp = n_ijp;
        z_im = z2_im;
        z_jm = z2_jm;
        z_ijm = z2_ijm;
        cp = cp2;
        n_ip = n2_ip;
        n_jp = n2_jp;
        n_ijp = n2_ijp;
      }
    }
  } else if (i < m && live) {   // FP64
    const double c0 = coef[4 * b], ca = coef[4 * b + 1], cf = coef[4 * b + 2], cb = coef[4 * b + 3];
    for (int j = blockIdx.y; j < m; j += gridDim.y) {
      for (int k = k0; k < kend; k++) {
        const int64_t o = ((int64_t)i + (int64_t)m * j + (int64_t)m * m * k) * B + b;
        const bool im = i > 0, ip = i < m - 1, jm = j > 0, jp = j < m - 1, km = k > 0, kp = k < m - 1;
        auto X = [&](bool ok, int64_t off) -> double { return ok ? v[o + off] : 0.0; };
        double av = c0 * v[o];
        av = fma(ca, X(im, -sB), av);
        av = fma(ca, X(ip, sB), av);
        av = fma(ca, X(jm, -sj), av);
        av = fma(ca, X(jp, sj), av);
        av = fma(ca, X(km, -sk), av);
        av = fma(ca, X(kp, sk), av);
        av = fma(cf, X(ip && jp, sB + sj), av);
        av = fma(cf, X(im && jm, -sB - sj), av);
        av = fma(cf, X(ip && kp, sB + sk), av);
        av = fma(cf, X(im && km, -sB - sk), av);
        av = fma(cf, X(jp && kp, sj + sk), av);
        av = fma(cf, X(jm && km, -sj - sk), av);
        av = fma(cb, X(ip && jp && kp, sB + sj + sk), av);
        av = fma(cb, X(im && jm && km, -sB - sj - sk), av);
        y[o] = av;
        acc[0] += v[o] * av;
      }
    }
  }
  slot_partials<1>(acc, B, partials, nblocks,
                   blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z));
}

// ------------------------------------------------------------------ multivector CSR

template <typename T, int VS>
struct VecLd;
template <typename T>
struct VecLd<T, 1> {
  __device__ static void load(const T* p, T o[1]) { o[0] = __ldg(p); }
};
template <>
struct VecLd<float, 2> {
  __device__ static void load(const float* p, float o[2]) {
    float2 a = __ldg(reinterpret_cast<const float2*>(p));
    o[0] = a.x; o[1] = a.y;
  }
};
template <>
struct VecLd<float, 4> {
  __device__ static void load(const float* p, float o[4]) {
    float4 a = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
  }
};
template <>
struct VecLd<double, 2> {
  __device__ static void load(const double* p, double o[2]) {
    double2 a = __ldg(reinterpret_cast<const double2*>(p));
    o[0] = a.x; o[1] = a.y;
  }
};
template <>
struct VecLd<double, 4> {
  __device__ static void load(const double* p, double o[4]) {
    double2 a = __ldg(reinterpret_cast<const double2*>(p));
    double2 c = __ldg(reinterpret_cast<const double2*>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = c.x; o[3] = c.y;
  }
};

// y[i][b] op ((rho_b K + M) v)[i][b] (pencil) or (Mat v)[i][b] (kv null: single values mv).
// B / VS threads per row, each holding VS consecutive slots (vector loads of v); the row's
// entries are read once per thread and shared by its VS slots.  Per (row, slot) the sum
// runs over the row's entries in stored order whatever VS is.
template <typename T, typename VT, int NV, int VS>
__global__ void __launch_bounds__(256) k_mv_csr(int64_t nrows, const int32_t* __restrict__ rowptr,
                                                const int32_t* __restrict__ col,
                                                const VT* __restrict__ kv, const VT* __restrict__ mv,
                                                const T* __restrict__ v, MvEpi<T> e, int accumulate,
                                                double* partials, int nblocks) {
  using AT = typename Arith<T>::type;
  const int B = e.B;
  const int tpr = B / VS;
  const int b0 = (threadIdx.x % tpr) * VS;
  const int rpb = blockDim.x / tpr;
  AT rb[VS];
#pragma unroll
  for (int q = 0; q < VS; q++) rb[q] = kv ? (AT)e.rho[b0 + q] : (AT)0;
  double acc[VS][2];
#pragma unroll
  for (int q = 0; q < VS; q++) acc[q][0] = acc[q][1] = 0.0;
  for (int64_t base = (int64_t)blockIdx.x * rpb; base < nrows; base += (int64_t)gridDim.x * rpb) {
    const int64_t i = base + threadIdx.x / tpr;
    if (i < nrows) {
      AT s[VS];
#pragma unroll
      for (int q = 0; q < VS; q++) s[q] = (AT)0;
      const int e1 = rowptr[i + 1];
      for (int p = rowptr[i]; p < e1; p++) {
        const int c = col[p];
        if (c < 0) continue;
        const AT kq = kv ? (AT)kv[p] : (AT)0;
        const AT mq = (AT)mv[p];
        T vv[VS];
        VecLd<T, VS>::load(v + (int64_t)c * B + b0, vv);
#pragma unroll
        for (int q = 0; q < VS; q++) {
          const AT w = kv ? rb[q] * kq + mq : mq;
          s[q] += w * (AT)vv[q];
        }
      }
#pragma unroll
      for (int q = 0; q < VS; q++) {
        if (accumulate) {
          const int64_t idx = i * B + b0 + q;
          e.y[idx] = (T)((AT)e.y[idx] + s[q]);
        } else {
          mv_epi<T>(e, i, b0 + q, s[q], acc[q]);
        }
      }
    }
  }
  if (NV > 0 && partials) slot_partials_vs<VS>(acc, NV, B, partials, nblocks, blockIdx.x);
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

// dense coarse matrices from the pencil, D = rho K + M, for the admitted slots (grid.y)
__global__ void k_mv_dense_build(int64_t Nc, const int32_t* rowptr, const int32_t* col,
                                 const double* kv, const double* mv, const double* rho,
                                 const int32_t* slots, double* Ainv) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= Nc) return;
  const double rh = rho[blockIdx.y];
  double* Dr = Ainv + (int64_t)slots[blockIdx.y] * Nc * Nc + r * Nc;
  for (int64_t c = 0; c < Nc; c++) Dr[c] = 0.0;
  for (int e = rowptr[r]; e < rowptr[r + 1]; e++)
    if (col[e] >= 0) Dr[col[e]] += rh * kv[e] + mv[e];
}

// One Gauss-Jordan step (pivot k) for the admitted slots (grid.y): between the slot's
// matrix in Ainv and its ping-pong buffer in tmp, direction given by from_tmp.
__global__ void k_gj_step_b(int64_t N, int64_t k, double* Ainv, double* tmp, const int32_t* slots,
                            int from_tmp) {
  const double* D = from_tmp ? tmp + (int64_t)blockIdx.y * N * N
                             : Ainv + (int64_t)slots[blockIdx.y] * N * N;
  double* E = from_tmp ? Ainv + (int64_t)slots[blockIdx.y] * N * N
                       : tmp + (int64_t)blockIdx.y * N * N;
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

__global__ void k_gj_copy_back(int64_t N, const double* tmp, double* Ainv, const int32_t* slots) {
  const double* src = tmp + (int64_t)blockIdx.y * N * N;
  double* dst = Ainv + (int64_t)slots[blockIdx.y] * N * N;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N * N;
       t += (int64_t)gridDim.x * blockDim.x)
    dst[t] = src[t];
}

// Gershgorin bounds of D^{-1} A(rho) for the admitted rho values (grid.y): block maxima of
// sum_j |a_ij| / a_ii in bmax[y * nb + block]
__global__ void k_mv_gersh(int64_t N, const int32_t* rowptr, const int32_t* col, const double* kv,
                           const double* mv, const double* rhos, double* bmax, int nb) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const double rho = rhos[blockIdx.y];
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
  if (threadIdx.x == 0) bmax[(int64_t)blockIdx.y * nb + blockIdx.x] = q;
}

// per-block maxima of row y (one block per row) -> out[y]
__global__ void k_max_red(const double* in, int n, double* out) {
  double q = -1.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) q = fmax(q, in[(int64_t)blockIdx.x * n + i]);
  q = block_max(q);
  if (threadIdx.x == 0) out[blockIdx.x] = q;
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

// admission of `count` columns: f and r of slot slots[k] from column c0 + k of the caller's
// [N][ld] array, x = p = r_prev = 0, and the slot's rho.  Block (kx, ty): threadIdx.x = k,
// so a warp reads consecutive columns of one row of the caller's array.
__global__ void k_cols_admit(int64_t N, int B, int count, const int32_t* slots,
                             const double* rhos, const double* src, int64_t ld, int c0, double* f,
                             double* r, double* x, double* p, double* rprev, double* rho) {
  const int k = threadIdx.x;
  if (k >= count) return;
  const int slot = slots[k];
  if (blockIdx.x == 0 && threadIdx.y == 0) rho[slot] = rhos[k];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i < N;
       i += (int64_t)gridDim.x * blockDim.y) {
    const double v = src[i * ld + c0 + k];
    const int64_t idx = i * B + slot;
    f[idx] = v;
    r[idx] = v;
    x[idx] = 0.0;
    p[idx] = 0.0;
    rprev[idx] = 0.0;
  }
}

// retirement of `count` slots: column c0 + k of the caller's [N][ld] array = x of slots[k]
__global__ void k_cols_out(int64_t N, int B, int count, const int32_t* slots, const double* src,
                           double* dst, int64_t ld, int c0) {
  const int k = threadIdx.x;
  if (k >= count) return;
  const int slot = slots[k];
  for (int64_t i = (int64_t)blockIdx.x * blockDim.y + threadIdx.y; i < N;
       i += (int64_t)gridDim.x * blockDim.y)
    dst[i * ld + c0 + k] = src[i * B + slot];
}

// per-slot partial sums of <a_b, a_b> (for ||f||), every slot at once (the order of a
// slot's sum does not depend on which slots are being admitted)
__global__ void k_mv_norm2(int64_t N, int B, const double* a, double* partials, int nblocks) {
  double acc[1] = {0.0};
  const int b = threadIdx.x % B;
  const int rpb = blockDim.x / B;
  for (int64_t base = (int64_t)blockIdx.x * rpb; base < N; base += (int64_t)gridDim.x * rpb) {
    const int64_t i = base + threadIdx.x / B;
    if (i < N) {
      const double v = a[i * B + b];
      acc[0] += v * v;
    }
  }
  slot_partials<1>(acc, B, partials, nblocks, blockIdx.x);
}

// per-slot partial sums of ||f_b - q_b||^2 and ||f_b||^2, every slot at once
__global__ void k_mv_resid2(int64_t N, int B, const double* f, const double* q, double* partials,
                            int nblocks) {
  double acc[2] = {0.0, 0.0};
  const int b = threadIdx.x % B;
  const int rpb = blockDim.x / B;
  for (int64_t base = (int64_t)blockIdx.x * rpb; base < N; base += (int64_t)gridDim.x * rpb) {
    const int64_t i = base + threadIdx.x / B;
    if (i < N) {
      const int64_t idx = i * B + b;
      const double fv = f[idx], d = fv - q[idx];
      acc[0] += d * d;
      acc[1] += fv * fv;
    }
  }
  slot_partials<2>(acc, B, partials, nblocks, blockIdx.x);
}

// out[2 b + k] = sum over blocks of partial k of slot b (fixed order)
__global__ void k_slot_sums2(const double* partials, int nb, int B, double* out) {
  const int b = blockIdx.x;
  double v[2] = {0.0, 0.0};
  for (int i = threadIdx.x; i < nb; i += blockDim.x) {
    v[0] += partials[(int64_t)(0 * B + b) * nb + i];
    v[1] += partials[(int64_t)(1 * B + b) * nb + i];
  }
  block_sum<2>(v);
  if (threadIdx.x == 0) {
    out[2 * b] = v[0];
    out[2 * b + 1] = v[1];
  }
}

__global__ void k_slot_admit(SlotState* S, const int32_t* slots, const double* sums, int nb,
                             const double* rhos, double tol, int maxit, int df_ok) {
  const int slot = slots[blockIdx.x];
  const double rho = rhos[blockIdx.x];
  double v[1] = {0.0};
  for (int i = threadIdx.x; i < nb; i += blockDim.x) v[0] += sums[(int64_t)slot * nb + i];
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
    s.dfop = df_ok && tol >= 1e-12;
    s.status = FEM_OK;
    s.done = (v[0] > 0.0) ? 0 : 1;
    if (!isfinite(v[0])) s.status = FEM_EBREAKDOWN;   // a non-finite right-hand side
  }
}

// per-slot finalisations (one block per slot, fixed order over the block partials)
__global__ void k_slot_fin_rz(SlotState* S, const double* partials, int nb, int B, int* rflag) {
  const int b = blockIdx.x;
  if (rflag && threadIdx.x == 0) rflag[b] = 0;   // raised again by this iteration's p
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

// p = z + beta p for live slots; slots with the double-float operator round p to 48 bits and
// write its FP32 pairs (p2), raising the slot's rflag for an entry outside the pairs' range.
// (The grid stride is a multiple of B: a thread stays on one slot.)
__global__ void k_mv_update_p(int64_t N, int B, const double* z, double* p, const SlotState* S,
                              float2* p2, int* rflag) {
  bool bad = false;
  const int b = (int)(((int64_t)blockIdx.x * blockDim.x + threadIdx.x) & (B - 1));
  const SlotState& s = S[b];
  if (!s.active || s.done) return;
  for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < N * B;
       idx += (int64_t)gridDim.x * blockDim.x) {
    double pv = z[idx] + s.beta * p[idx];
    if (p2 && s.dfop) {
      float hi, lo;
      double xs;
      if (df_split(pv, hi, lo, xs)) {
        p2[idx] = make_float2(hi, lo);
        pv = xs;
      } else {
        bad = true;
      }
    }
    p[idx] = pv;
  }
  if (bad) atomicOr(&rflag[b], 1);
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
  DevBuf<MvDf> dfc;                         // [B] their double-float split (uniform grid)
  DevBuf<float2> p2;                        // [N][B] p as FP32 pairs (uniform grid)
  DevBuf<int> rflag;                        // [B] an entry of p outside the pairs' range
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

// ------------------------------------------------------------------ tuned launches

// FP32 multivector stencil variants: 0 one thread per (point, slot) striding over planes,
// 1..3 column marching over 16, 32, 64 planes per block, 4..5 column marching over 16, 32
// planes with an L2 prefetch of the streams 4 planes ahead.
constexpr int kMvStencilVariants = 6;
const char* const kMvStencilNames[kMvStencilVariants] = {"point", "col_kz16", "col_kz32",
                                                         "col_kz64", "col_kz16_pf4",
                                                         "col_kz32_pf4"};
// multivector CSR variants: 1, 2, 4 slots per thread
constexpr int kMvCsrVariants = 3;
const char* const kMvCsrNames[kMvCsrVariants] = {"vs1", "vs2", "vs4"};

dim3 mv_colgrid(int m, int B, int kz) {
  const int ppb = 256 / B;
  const int gx = (m + ppb - 1) / ppb, gz = (m + kz - 1) / kz;
  int gy = (8 * num_sms() + gx * gz - 1) / (gx * gz);
  if (gy > m) gy = m;
  if (gy < 1) gy = 1;
  return dim3(gx, gy, gz);
}

dim3 mv_stencil_grid(int var, int m, int B) {
  switch (var) {
    case 1: return mv_colgrid(m, B, 16);
    case 2: return mv_colgrid(m, B, 32);
    case 3: return mv_colgrid(m, B, 64);
    case 4: return mv_colgrid(m, B, 16);
    case 5: return mv_colgrid(m, B, 32);
    default: return mv_sgrid(m, B);
  }
}

template <int NV, int KZV, int PF = 0>
void launch_mv_col(dim3 g, int nb, const float* v, int m, const MvEpi<float>& e, double* part,
                   cudaStream_t st) {
  switch (e.mode) {
    case 0: k_mv_stencil_col<float, NV, KZV, 0, PF><<<g, 256, 0, st>>>(v, m, e, part, nb); break;
    case 1: k_mv_stencil_col<float, NV, KZV, 1, PF><<<g, 256, 0, st>>>(v, m, e, part, nb); break;
    case 3: k_mv_stencil_col<float, NV, KZV, 3, PF><<<g, 256, 0, st>>>(v, m, e, part, nb); break;
    default:
      if (e.z64)
        k_mv_stencil_col<float, NV, KZV, 5, PF><<<g, 256, 0, st>>>(v, m, e, part, nb);
      else
        k_mv_stencil_col<float, NV, KZV, 2, PF><<<g, 256, 0, st>>>(v, m, e, part, nb);
  }
}

template <int NV>
int launch_mv_stencil32(int var, const float* v, int m, const MvEpi<float>& e, double* part,
                        cudaStream_t st) {
  const dim3 g = mv_stencil_grid(var, m, e.B);
  const int nb = (int)(g.x * g.y * g.z);
  switch (var) {
    case 1: launch_mv_col<NV, 16>(g, nb, v, m, e, part, st); break;
    case 2: launch_mv_col<NV, 32>(g, nb, v, m, e, part, st); break;
    case 3: launch_mv_col<NV, 64>(g, nb, v, m, e, part, st); break;
    case 4: launch_mv_col<NV, 16, 4>(g, nb, v, m, e, part, st); break;
    case 5: launch_mv_col<NV, 32, 4>(g, nb, v, m, e, part, st); break;
    default: k_mv_stencil<float, NV><<<g, 256, 0, st>>>(v, m, e, part, nb); break;
  }
  FEM_CHECK_LAUNCH();
  return nb;
}

int mv_stencil32(int m, const float* v, const MvEpi<float>& e, double* part, cudaStream_t st) {
  const int var = tuned_variant("mv_stencil_f32", m, 0, e.B, 1, kMvStencilVariants);
  return part ? launch_mv_stencil32<2>(var, v, m, e, part, st)
              : launch_mv_stencil32<0>(var, v, m, e, nullptr, st);
}

template <typename T>
const char* mv_csr_key() { return sizeof(T) == 8 ? "mv_csr_f64" : "mv_csr_f32"; }

template <typename T, typename VT, int NV>
int launch_mv_csr(int var, const Csr4& A, const VT* kv, const VT* mv, const T* v,
                  const MvEpi<T>& e, int accumulate, double* part, cudaStream_t st) {
  const int64_t N = A.nrows;
  int vs = 1 << var;
  if (vs > e.B) vs = e.B;
  const int tpr = e.B / vs, rpb = 256 / tpr;
  const unsigned g = persistent_grid((N + rpb - 1) / rpb * 256, 256, 8);
  switch (vs) {
    case 2:
      k_mv_csr<T, VT, NV, 2><<<g, 256, 0, st>>>(N, A.rowptr, A.col, kv, mv, v, e, accumulate, part, g);
      break;
    case 4:
      k_mv_csr<T, VT, NV, 4><<<g, 256, 0, st>>>(N, A.rowptr, A.col, kv, mv, v, e, accumulate, part, g);
      break;
    default:
      k_mv_csr<T, VT, NV, 1><<<g, 256, 0, st>>>(N, A.rowptr, A.col, kv, mv, v, e, accumulate, part, g);
  }
  FEM_CHECK_LAUNCH();
  return (int)g;
}

template <typename T, typename VT, int NV>
int mv_csr(const Csr4& A, const VT* kv, const VT* mv, const T* v, const MvEpi<T>& e,
           int accumulate, double* part, cudaStream_t st) {
  const int var = tuned_variant(mv_csr_key<T>(), A.nrows, A.nnz, e.B, 0, kMvCsrVariants);
  return launch_mv_csr<T, VT, NV>(var, A, kv, mv, v, e, accumulate, part, st);
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
  auto op = [&](const float* v, MvEpi<float> e, bool dots) {
    int nb;
    if (L.stencil)
      nb = mv_stencil32(m, v, e, dots ? part : nullptr, st);
    else if (dots)
      nb = mv_csr<float, float, 2>(*L.A, L.Kv.p, L.Mv.p, v, e, 0, part, st);
    else
      nb = mv_csr<float, float, 0>(*L.A, L.Kv.p, L.Mv.p, v, e, 0, nullptr, st);
    if (dots) W.nb_fine = nb;
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
    mv_csr<float, float, 0>(*L.R, (const float*)nullptr, L.Rv.p, L.r, e, 0, nullptr, st);
  }
  mv_vcycle(W, lev + 1, nullptr, st);
  {
    MvEpi<float> e = base;
    e.y = L.x;
    mv_csr<float, float, 0>(*L.P, (const float*)nullptr, L.Pv.p, C.x, e, 1, nullptr, st);
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
    std::swap(dold, dnew);
  }
}

// q = A(rho_b) p with per-slot <p, q> (double-float on the uniform grid, else FP64)
int mv_apply64(BatchSession& W, cudaStream_t st) {
  BatchLevel& L = *W.L[0];
  const int B = W.B;
  if (L.stencil) {
    const dim3 sg = mv_colgrid(W.S->n - 1, B, 16);
    const int nb = (int)(sg.x * sg.y * sg.z);
    k_mv_stencil_df<<<sg, 256, 0, st>>>(W.p2, W.p, W.S->n - 1, W.dfc, W.coef64, B, W.q, W.state,
                                        W.rflag, W.partials, nb);
    FEM_CHECK_LAUNCH();
    return nb;
  } else {
    MvEpi<double> e;
    std::memset(&e, 0, sizeof(e));
    e.mode = 0;
    e.y = W.q;
    e.x = W.p;
    e.want_dot = 1;
    e.B = B;
    e.rho = W.rho;
    return mv_csr<double, double, 1>(*L.A, L.Kv64, L.Mv64, W.p, e, 0, W.partials, st);
  }
}

void batch_iteration(BatchSession& W, cudaStream_t st) {
  const int B = W.B;
  const int64_t N = W.N;
  mv_vcycle(W, 0, W.r, st);
  k_slot_fin_rz<<<B, 256, 0, st>>>(W.state, W.partials, W.nb_fine, B, W.rflag.p);
  FEM_CHECK_LAUNCH();
  const unsigned ge = persistent_grid(N * B, 256, 8);
  k_mv_update_p<<<ge, 256, 0, st>>>(N, B, W.z, W.p, W.state, W.p2.p, W.rflag.p);
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


// Launch shapes of the session's multivector kernels, timed on its scratch vectors
// before the iteration is captured (a graph keeps the shapes it was captured with).
void tune_session(BatchSession& W, cudaStream_t st) {
  const int B = W.B;
  const int m = W.S->n - 1;
  for (size_t l = 0; l < W.L.size(); l++) {
    BatchLevel& L = *W.L[l];
    MvEpi<float> e;
    std::memset(&e, 0, sizeof(e));
    e.level = (int)l;
    e.lc = W.lc;
    e.B = B;
    e.rho = W.rho;
    if (L.stencil) {
      e.mode = 2;
      e.r = L.r;
      e.dold = L.d0;
      e.dnew = L.d1;
      e.x = L.x;
      autotune("mv_stencil_f32", m, 0, B, kMvStencilVariants, kMvStencilNames, 1, st,
               [&](int v) { launch_mv_stencil32<0>(v, L.d0.p, m, e, nullptr, st); });
    } else if (!(L.coarsest && L.dense) && L.A->nnz >= (1 << 16)) {
      e.kd = L.kd;
      e.md = L.md;
      e.mode = 1;
      e.y = L.r;
      e.b = L.b;
      autotune("mv_csr_f32", L.A->nrows, L.A->nnz, B, kMvCsrVariants, kMvCsrNames, 0, st,
               [&](int v) {
                 launch_mv_csr<float, float, 0>(v, *L.A, L.Kv.p, L.Mv.p, L.x.p, e, 0, nullptr, st);
               });
    }
    if (!L.coarsest && l + 1 < W.L.size()) {
      BatchLevel& C = *W.L[l + 1];
      MvEpi<float> er;
      std::memset(&er, 0, sizeof(er));
      er.B = B;
      er.y = C.b;
      if (L.R->nnz >= (1 << 16))
        autotune("mv_csr_f32", L.R->nrows, L.R->nnz, B, kMvCsrVariants, kMvCsrNames, 0, st,
                 [&](int v) {
                   launch_mv_csr<float, float, 0>(v, *L.R, (const float*)nullptr, L.Rv.p, L.r.p,
                                                  er, 0, nullptr, st);
                 });
      MvEpi<float> ep = er;
      ep.y = L.x;
      if (L.P->nnz >= (1 << 16))
        autotune("mv_csr_f32", L.P->nrows, L.P->nnz, B, kMvCsrVariants, kMvCsrNames, 0, st,
                 [&](int v) {
                   launch_mv_csr<float, float, 0>(v, *L.P, (const float*)nullptr, L.Pv.p, C.x.p,
                                                  ep, 1, nullptr, st);
                 });
    }
  }
  BatchLevel& L0 = *W.L[0];
  if (!L0.stencil && L0.A->nnz >= (1 << 16)) {
    MvEpi<double> e;
    std::memset(&e, 0, sizeof(e));
    e.mode = 0;
    e.y = W.q;
    e.x = W.p;
    e.want_dot = 1;
    e.B = B;
    e.rho = W.rho;
    autotune("mv_csr_f64", L0.A->nrows, L0.A->nnz, B, kMvCsrVariants, kMvCsrNames, 0, st,
             [&](int v) {
               launch_mv_csr<double, double, 1>(v, *L0.A, L0.Kv64, L0.Mv64, W.p.p, e, 0,
                                                W.partials.p, st);
             });
  }
}

}  // namespace

int64_t batch_footprint(const System& S, const Hierarchy& H, int slots) {
  int B = 1;
  while (B < slots) B <<= 1;
  int64_t bytes = 7 * S.N * B * 8;  // x r rprev p q z f
  if (S.stencil) bytes += S.N * B * 8;   // p as FP32 pairs
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
  FEM_REQUIRE(H.o.smoother != AMG_SMOOTHER_SGS, FEM_EUNSUPPORTED,
              "pcg_batch_create: batched solves smooth with Chebyshev or l1-Jacobi");
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
    for (auto* v : {&BL->x, &BL->b, &BL->r, &BL->d0, &BL->d1}) {
      v->alloc(Lv.N * B);
      FEM_CUDA(cudaMemsetAsync(v->p, 0, 4 * Lv.N * B, st));
    }
    W->L.push_back(std::move(BL));
  }
  for (auto* v : {&W->x, &W->r, &W->rprev, &W->p, &W->q, &W->z, &W->f}) {
    v->alloc(N * B);
    FEM_CUDA(cudaMemsetAsync(v->p, 0, 8 * N * B, st));
  }
  W->rho.alloc(B);
  W->coef64.alloc(4 * B);
  W->rflag.alloc(B);
  FEM_CUDA(cudaMemsetAsync(W->rflag, 0, 4 * B, st));
  if (S.stencil) {
    W->dfc.alloc(B);
    FEM_CUDA(cudaMemsetAsync(W->dfc, 0, sizeof(MvDf) * B, st));
    W->p2.alloc(N * B);
    FEM_CUDA(cudaMemsetAsync(W->p2, 0, 8 * N * B, st));
  }
  W->lc.alloc(H.L.size() * B);
  W->hlc.assign(H.L.size() * B, LevCoef{});
  W->state.alloc(B);
  FEM_CUDA(cudaMemsetAsync(W->state, 0, sizeof(SlotState) * B, st));
  FEM_CUDA(cudaMemsetAsync(W->rho, 0, 8 * B, st));
  FEM_CUDA(cudaMemsetAsync(W->coef64, 0, 32 * B, st));
  FEM_CUDA(cudaMemsetAsync(W->lc, 0, sizeof(LevCoef) * H.L.size() * B, st));
  // per-slot partial sums: the largest block count of any kernel that emits them
  int64_t maxnb = 8 * (int64_t)num_sms() + 1;
  if (S.stencil) {
    for (int v = 0; v < kMvStencilVariants; v++) {
      const dim3 gv = mv_stencil_grid(v, S.n - 1, B);
      maxnb = std::max<int64_t>(maxnb, (int64_t)gv.x * gv.y * gv.z);
    }
    const dim3 g64 = mv_sgrid(S.n - 1, B);
    maxnb = std::max<int64_t>(maxnb, (int64_t)g64.x * g64.y);
  }
  W->partials.alloc((size_t)2 * B * maxnb + 4 * (size_t)kMaxPartialBlocks);
  W->scratch.alloc(4 * 8 * (size_t)num_sms() + 64);
  FEM_CUDA(cudaMallocHost(&W->hstate, sizeof(SlotState) * B));
  W->in_use.assign(B, 0);
  tune_session(*W, st);
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

// Admit `count` solves at once: column fcol0 + k of f ([N][ld]) with rho[k] goes into the
// k-th free slot.  Every kernel covers all admitted slots (grid.y = admitted slot), and
// each slot's arithmetic and reduction order is the same as when it is admitted alone.
void batch_admit_many(BatchSession& W, const double* f, int64_t ld, int fcol0, const double* rho,
                      int count, int* slots_out, cudaStream_t st) {
  FEM_REQUIRE(count >= 1, FEM_EINVAL, "pcg_batch_admit: nothing to admit");
  std::vector<int> slot;
  for (int b = 0; b < W.slots && (int)slot.size() < count; b++)
    if (!W.in_use[b]) slot.push_back(b);
  FEM_REQUIRE((int)slot.size() == count, FEM_ENOMEM, "pcg_batch_admit: no free slot");
  for (int k = 0; k < count; k++)
    FEM_REQUIRE(rho[k] > 0.0 && std::isfinite(rho[k]), FEM_EINVAL, "pcg_batch_admit: rho > 0");
  const int B = W.B;
  const int64_t N = W.N;
  System& S = *W.S;
  Hierarchy& H = *W.H;
  // admitted slots and their rho on the device
  std::vector<double> hr(rho, rho + count);
  DevBuf<int32_t> dslot(count, st);
  DevBuf<double> drho(count, st);
  FEM_CUDA(cudaMemcpyAsync(dslot, slot.data(), 4 * count, cudaMemcpyHostToDevice, st));
  FEM_CUDA(cudaMemcpyAsync(drho, hr.data(), 8 * count, cudaMemcpyHostToDevice, st));
  {
    int kx = 1;
    while (kx < count) kx <<= 1;
    const dim3 blk(kx, 256 / kx);
    k_cols_admit<<<persistent_grid(N * kx, 256, 8), blk, 0, st>>>(
        N, B, count, dslot, drho, f, ld, fcol0, W.f, W.r, W.x, W.p, W.rprev, W.rho);
    FEM_CHECK_LAUNCH();
  }
  // per-level smoother coefficients of every admitted rho
  for (size_t l = 0; l < H.L.size(); l++) {
    Level& Lv = *H.L[l];
    BatchLevel& BL = *W.L[l];
    const double* kv = BL.Kv64;
    const double* mv = BL.Mv64;
    std::vector<double> lmax(count);
    if (Lv.stencil) {
      // every row has the diagonal a[0] and a subset of the interior row's neighbours, so
      // the Gershgorin bound is the interior row's sum
      for (int k = 0; k < count; k++) {
        const double r = rho[k];
        const double a[4] = {r * S.stK.c0 + S.stM.c0, r * S.stK.ca + S.stM.ca,
                             r * S.stK.cf + S.stM.cf, r * S.stK.cb + S.stM.cb};
        FEM_CUDA(cudaMemcpyAsync(W.coef64.p + 4 * slot[k], a, 32, cudaMemcpyHostToDevice, st));
        if (l == 0 && W.dfc.p) {
          Stencil sa;
          sa.c0 = a[0];
          sa.ca = a[1];
          sa.cf = a[2];
          sa.cb = a[3];
          const DfOperator D = df_operator(sa);
          MvDf md{};
          std::memcpy(md.C, D.C, sizeof(md.C));
          md.s = D.s;
          FEM_CUDA(cudaMemcpyAsync(W.dfc.p + slot[k], &md, sizeof(MvDf), cudaMemcpyHostToDevice, st));
        }
        lmax[k] = (std::fabs(a[0]) + 6 * std::fabs(a[1]) + 6 * std::fabs(a[2]) +
                   2 * std::fabs(a[3])) / a[0];
        LevCoef& c = W.hlc[l * B + slot[k]];
        c = LevCoef{};
        c.c0 = (float)a[0];
        c.ca = (float)a[1];
        c.cf = (float)a[2];
        c.cb = (float)a[3];
        c.sinv = (float)(1.0 / a[0]);
      }
      FEM_CUDA(cudaStreamSynchronize(st));   // the host arrays above go out of scope
    } else {
      const int64_t NL = Lv.N;
      const unsigned g = grid_for(NL, 256);
      DevBuf<double> bm((size_t)count * (g + 1), st);
      k_mv_gersh<<<dim3(g, count), 256, 0, st>>>(NL, Lv.A->rowptr, Lv.A->col, kv, mv, drho, bm, g);
      FEM_CHECK_LAUNCH();
      k_max_red<<<count, 1024, 0, st>>>(bm, (int)g, bm.p + (size_t)count * g);
      FEM_CHECK_LAUNCH();
      FEM_CUDA(cudaMemcpyAsync(lmax.data(), bm.p + (size_t)count * g, 8 * count,
                               cudaMemcpyDeviceToHost, st));
      FEM_CUDA(cudaStreamSynchronize(st));
      for (int k = 0; k < count; k++) W.hlc[l * B + slot[k]] = LevCoef{};
    }
    for (int k = 0; k < count; k++) {
      LevCoef& c = W.hlc[l * B + slot[k]];
      if (H.o.smoother == AMG_SMOOTHER_L1_JACOBI) {
        c.inv_theta = 1.0f;
      } else {
        ChebCoef cc = cheb_coefficients(lmax[k], H.o.cheb_ratio, H.o.degree);
        c.inv_theta = (float)cc.inv_theta;
        c.c1 = (float)cc.c1[1];
        c.c2 = (float)cc.c2[1];
      }
      FEM_CUDA(cudaMemcpyAsync(W.lc.p + l * B + slot[k], &c, sizeof(LevCoef),
                               cudaMemcpyHostToDevice, st));
    }
    if (BL.coarsest && BL.dense) {
      // dense coarse matrix of each rho, inverted by Gauss-Jordan (ping-pong buffers)
      const int64_t Nc = Lv.N;
      DevBuf<double> tmp((size_t)count * Nc * Nc, st);
      k_mv_dense_build<<<dim3(grid_for(Nc, 128), count), 128, 0, st>>>(
          Nc, Lv.A->rowptr, Lv.A->col, kv, mv, drho, dslot, BL.Ainv);
      FEM_CHECK_LAUNCH();
      const unsigned gg = persistent_grid(Nc * Nc, 256, 4);
      bool in_tmp = false;
      for (int64_t k = 0; k < Nc; k++) {
        k_gj_step_b<<<dim3(gg, count), 256, 0, st>>>(Nc, k, BL.Ainv, tmp, dslot, in_tmp);
        FEM_CHECK_LAUNCH();
        in_tmp = !in_tmp;
      }
      if (in_tmp) {
        k_gj_copy_back<<<dim3(gg, count), 256, 0, st>>>(Nc, tmp, BL.Ainv, dslot);
        FEM_CHECK_LAUNCH();
      }
    }
  }
  FEM_CUDA(cudaStreamSynchronize(st));
  // ||f|| and the slots' CG state
  const unsigned gn = mv_grid(N, B);
  k_mv_norm2<<<gn, 256, 0, st>>>(N, B, W.f, W.partials, gn);
  FEM_CHECK_LAUNCH();
  k_slot_admit<<<count, 256, 0, st>>>(W.state, dslot, W.partials, gn, drho, W.o.tol, W.o.max_iter,
                                      W.dfc.p != nullptr ? 1 : 0);
  FEM_CHECK_LAUNCH();
  FEM_CUDA(cudaStreamSynchronize(st));
  for (int k = 0; k < count; k++) {
    W.in_use[slot[k]] = 1;
    if (slots_out) slots_out[k] = slot[k];
  }
}

int batch_admit(BatchSession& W, const double* f, int64_t ld, int fcol, double rho, cudaStream_t st) {
  int slot = -1;
  batch_admit_many(W, f, ld, fcol, &rho, 1, &slot, st);
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

// Copy x of slots[k] to column c0 + k of u ([N][ld]) and free the slots.
void batch_retire_many(BatchSession& W, const int* slots, int count, double* u, int64_t ld, int c0,
                       cudaStream_t st) {
  for (int k = 0; k < count; k++)
    FEM_REQUIRE(slots[k] >= 0 && slots[k] < W.slots && W.in_use[slots[k]], FEM_EINVAL,
                "pcg_batch_retire: slot not in use");
  DevBuf<int32_t> dslot(count, st);
  std::vector<int32_t> hs(slots, slots + count);
  FEM_CUDA(cudaMemcpyAsync(dslot, hs.data(), 4 * count, cudaMemcpyHostToDevice, st));
  int kx = 1;
  while (kx < count) kx <<= 1;
  k_cols_out<<<persistent_grid(W.N * kx, 256, 8), dim3(kx, 256 / kx), 0, st>>>(
      W.N, W.B, count, dslot, W.x, u, ld, c0);
  FEM_CHECK_LAUNCH();
  // deactivate
  std::vector<SlotState> off(count);
  std::memset(off.data(), 0, sizeof(SlotState) * count);
  for (int k = 0; k < count; k++)
    FEM_CUDA(cudaMemcpyAsync(W.state.p + slots[k], &off[k], sizeof(SlotState),
                             cudaMemcpyHostToDevice, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  for (int k = 0; k < count; k++) W.in_use[slots[k]] = 0;
}

void batch_retire(BatchSession& W, int slot, double* u, int64_t ld, int ucol, cudaStream_t st) {
  batch_retire_many(W, &slot, 1, u, ld, ucol, st);
}

void batch_destroy(BatchSession* W) { delete W; }

// ||f_b - A(rho_b) x_b|| / ||f_b|| for every slot in use (FP64, recomputed).
static void batch_true_residual(BatchSession& W, double* out, cudaStream_t st) {
  const int B = W.B;
  const int64_t N = W.N;
  BatchLevel& L = *W.L[0];
  if (L.stencil) {
    const dim3 sg = mv_sgrid(W.S->n - 1, B);
    k_mv_stencil64<<<sg, 256, 0, st>>>(W.x, W.S->n - 1, W.coef64, B, W.q, nullptr, W.partials,
                                       sg.x * sg.y);
    FEM_CHECK_LAUNCH();
  } else {
    MvEpi<double> e;
    std::memset(&e, 0, sizeof(e));
    e.mode = 0;
    e.y = W.q;
    e.x = W.x;
    e.B = B;
    e.rho = W.rho;
    mv_csr<double, double, 0>(*L.A, L.Kv64, L.Mv64, W.x, e, 0, nullptr, st);
  }
  const unsigned g = mv_grid(N, B);
  k_mv_resid2<<<g, 256, 0, st>>>(N, B, W.f, W.q, W.partials, g);
  FEM_CHECK_LAUNCH();
  DevBuf<double> sums(2 * B, st);
  k_slot_sums2<<<B, 256, 0, st>>>(W.partials, g, B, sums);
  FEM_CHECK_LAUNCH();
  std::vector<double> h(2 * B);
  FEM_CUDA(cudaMemcpyAsync(h.data(), sums, 16 * B, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  for (int b = 0; b < W.slots; b++) {
    if (!W.in_use[b]) continue;
    out[b] = h[2 * b + 1] > 0 ? std::sqrt(h[2 * b] / h[2 * b + 1]) : 0.0;
  }
}

fem_status pcg_multi(System& S, Hierarchy& H, const double* f, double* u, int nrhs,
                     const double* rho_k, const pcg_opts& o, cudaStream_t user, pcg_result* res) {
  FEM_REQUIRE(nrhs >= 1 && nrhs <= MAXB, FEM_EINVAL, "pcg_solve: nrhs in [1, 64]");
  std::unique_ptr<BatchSession> W(batch_create(S, H, nrhs, o, user));
  batch_admit_many(*W, f, nrhs, 0, rho_k, nrhs, nullptr, user);
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
  {
    std::vector<int> all_slots(nrhs);
    for (int k = 0; k < nrhs; k++) all_slots[k] = k;
    batch_retire_many(*W, all_slots.data(), nrhs, u, nrhs, 0, user);
  }
  for (int k = 0; k < nrhs; k++) {
    res[k].iterations = it[k];
    res[k].status = st[k] == 1 ? FEM_OK : (st[k] == 0 ? FEM_ENOCONV : W->hstate[k].status);
    res[k].relres = trr[k];
    res[k].prec_relres = 0.0;
    res[k].solve_ms = ms;
    if (res[k].status != FEM_OK && all == FEM_OK) all = (fem_status)res[k].status;
  }
  bool unfinished = false;
  for (int k = 0; k < nrhs; k++)
    if (st[k] == 0) unfinished = true;
  // a cancel raised after every slot had finished leaves the results standing
  if (o.cancel_host && *o.cancel_host && unfinished) all = FEM_ECANCELLED;
  FEM_CUDA(cudaStreamSynchronize(user));
  return all;
}

}  // namespace fem

