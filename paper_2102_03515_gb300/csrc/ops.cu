// Operator applications of the V-cycle and of CG: the matrix-free 15-point stencil of
// A = rho K + M on the uniform Kuhn grid and CSR4 SpMV, each with a fused epilogue
// (plain product, residual, Chebyshev / l1-Jacobi smoothing step, dot products).
//
// Smoothing (one "step" of the paper's V-cycle, Sec. 3.1 and Sec. 4) is a Chebyshev
// polynomial of degree k in D^{-1}A over [lambda/ratio, lambda], lambda the Gershgorin
// bound, run by the three-term recurrence
//     r_0 = D^{-1}(b - A x_0),  d_0 = r_0 / theta,  x_1 = x_0 + d_0,
//     r_i = r_{i-1} - D^{-1} A d_{i-1},  d_i = c1_i d_{i-1} + c2_i r_i,  x_{i+1} = x_i + d_i,
// (theta, delta the centre and half-width of the interval, sigma = theta/delta,
// rho_0 = 1/sigma, rho_i = 1/(2 sigma - rho_{i-1}), c1_i = rho_i rho_{i-1}, c2_i = 2 rho_i/delta).
// One l1-Jacobi step is the degree-1 case with D replaced by the l1 row norms, theta = 1.
#include <algorithm>
#include <cmath>

#include "dfloat.cuh"
#include "solver.cuh"

namespace fem {

ChebCoef cheb_coefficients(double lmax, double ratio, int degree) {
  ChebCoef c;
  c.degree = degree;
  double a = lmax / ratio, b = lmax;
  double theta = 0.5 * (b + a), delta = 0.5 * (b - a);
  double sigma = theta / delta;
  c.inv_theta = 1.0 / theta;
  double rho_old = 1.0 / sigma;
  for (int i = 1; i < degree && i < 16; i++) {
    double rho_new = 1.0 / (2.0 * sigma - rho_old);
    c.c1[i] = rho_new * rho_old;
    c.c2[i] = 2.0 * rho_new / delta;
    rho_old = rho_new;
  }
  return c;
}

namespace {

enum EpiMode {
  E_STORE = 0, E_RESIDUAL = 1, E_CHEB_STEP = 2, E_CHEB_INIT = 3, E_ADD = 4, E_CHEB_PRE1 = 6
};
// compile-time variants of E_CHEB_STEP for kernels specialised on the mode: without the
// FP64 output (z64 null) and with it
constexpr int E_CHEB_STEP_NOZ = 2, E_CHEB_STEP_Z = 5;

// Fused epilogue applied to (row, (A v)_row).  Modes:
//   E_STORE     y = Av              (dot: <v, Av> with v = vin)
//   E_ADD       y += Av
//   E_RESIDUAL  y = b - Av
//   E_CHEB_INIT r = s (b - Av); d_new = c2 r                       (v = x, x not written)
//   E_CHEB_STEP r -= s Av; d_new = c1 d_old + c2 r; x += [d_old] + d_new   (v = d_old;
//               with xonly, the last step of a smoothing, r and d_new are not written)
//   E_CHEB_PRE1 the step above right after the start from x = 0, when it is the last of
//               the pre-smoothing (degree 2): r = s b and x = d_old are implied by that
//               start, and only the new x is used afterwards: x = d_old + c1 d_old
//               + c2 (s b - s Av)                                         (v = d_old)
// s is the smoother's diagonal inverse (scalar sinv_c when sinv is null).  When z64 is
// set, the final x is written in FP64 only (the step is the V-cycle's last: its FP32 r,
// d_new and x are not used again) and <z, r1>, <z, r2> are accumulated.
//
// The epilogue is split into load() (the row's operands, so that a kernel can issue these
// loads early, together with its stencil loads) and apply(); "centre" is v[row], which
// the stencil kernels already hold in a register (it is vin[row] in E_STORE and d_old[row]
// in E_CHEB_STEP).
__device__ __forceinline__ void l2_prefetch(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

template <typename T>
struct Epi {
  using AT = typename Arith<T>::type;
  struct Ops {
    AT a, x, s;
    double r1, r2;
  };
  int mode;
  T* y;
  const T* b;
  T* r;
  const T* dold;
  T* dnew;
  T* x;
  const T* sinv;
  T sinv_c;
  T c1, c2;
  int add_prev;
  int xonly;   // E_CHEB_STEP: the last smoothing step, only x is used afterwards
  const T* vin;
  int want_dot;
  double* z64;
  const double* r1;
  const double* r2;
  // gm > 0: the level vectors (y, b, r, d_old, d_new, x, vin) live in the ghost layout of the
  // gm^3 grid: (gm + 2)^3 entries, interior (i, j, k) at (i+1) + G ((j+1) + G (k+1)),
  // G = gm + 2, zero faces.  z64, r1, r2 are always dense; ydense: y too (the residual
  // handed to the restriction).
  int gm;
  int ydense;

  // MODE >= 0: the mode fixed at compile time (the switch folds away); -1: run time.
  template <int MODE = -1>
  __device__ __forceinline__ Ops load(int64_t row, int64_t drow) const {
    Ops o;
    o.a = (AT)0;
    o.x = (AT)0;
    o.s = (AT)0;
    o.r1 = 0.0;
    o.r2 = 0.0;
    const bool zo = MODE == E_CHEB_STEP_Z || (MODE < 0 && z64 != nullptr);
    switch (MODE >= 0 ? (MODE == E_CHEB_STEP_Z ? E_CHEB_STEP : MODE) : mode) {
      case E_ADD:
        o.a = (AT)y[row];
        break;
      case E_RESIDUAL:
        o.a = (AT)b[row];
        break;
      case E_CHEB_INIT:
      case E_CHEB_PRE1:
        o.a = (AT)b[row];
        o.s = sinv ? (AT)sinv[row] : (AT)sinv_c;
        break;
      case E_CHEB_STEP:
        o.a = (AT)r[row];
        o.s = sinv ? (AT)sinv[row] : (AT)sinv_c;
        o.x = (AT)x[row];
        if (zo) {
          o.r1 = r1[drow];
          if (r2) o.r2 = r2[drow];
        }
        break;
      default:
        break;
    }
    return o;
  }

  template <int MODE = -1>
  __device__ __forceinline__ void apply(int64_t row, int64_t drow, AT av, AT centre,
                                        const Ops& o, double acc[2]) const {
    const bool zo = MODE == E_CHEB_STEP_Z || (MODE < 0 && z64 != nullptr);
    switch (MODE >= 0 ? (MODE == E_CHEB_STEP_Z ? E_CHEB_STEP : MODE) : mode) {
      case E_STORE:
        y[row] = (T)av;
        if (want_dot) acc[0] += (double)centre * (double)av;
        break;
      case E_ADD:
        y[row] = (T)(o.a + av);
        break;
      case E_RESIDUAL:
        y[ydense ? drow : row] = (T)(o.a - av);
        break;
      case E_CHEB_INIT: {
        AT rr = o.s * (o.a - av);
        r[row] = (T)rr;
        dnew[row] = (T)((AT)c2 * rr);
      } break;
      case E_CHEB_STEP: {
        AT rr = o.a - o.s * av;
        AT dl = centre;
        AT dn = (AT)c1 * dl + (AT)c2 * rr;
        AT xv = o.x + (add_prev ? dl : (AT)0) + dn;
        if (zo) {
          double z = (double)xv;
          z64[drow] = z;
          acc[0] += z * o.r1;
          if (r2) acc[1] += z * o.r2;
        } else {
          if (!xonly) {
            r[row] = (T)rr;
            dnew[row] = (T)dn;
          }
          x[row] = (T)xv;
        }
      } break;
      case E_CHEB_PRE1: {
        AT r0 = o.s * o.a;
        AT rr = r0 - o.s * av;
        AT dl = centre;
        AT dn = (AT)c1 * dl + (AT)c2 * rr;
        x[row] = (T)(dl + dn);
      } break;
    }
  }

  // hint the L2 to fetch the operands of a later row (no registers, no wait)
  template <int MODE = -1>
  __device__ __forceinline__ void prefetch(int64_t row) const {
    const int md = MODE >= 0 ? (MODE == E_CHEB_STEP_Z ? E_CHEB_STEP : MODE) : mode;
    if (md == E_CHEB_STEP) {
      l2_prefetch(r + row);
      l2_prefetch(x + row);
    } else if (md == E_RESIDUAL || md == E_CHEB_INIT || md == E_CHEB_PRE1) {
      l2_prefetch(b + row);
    } else if (md == E_ADD) {
      l2_prefetch(y + row);
    }
  }

  // centre value of a kernel that does not hold v[row]
  __device__ __forceinline__ AT centre_of(int64_t row) const {
    if (mode == E_STORE && want_dot) return (AT)vin[row];
    if (mode == E_CHEB_STEP || mode == E_CHEB_PRE1) return (AT)dold[row];
    return (AT)0;
  }

  // row: the dense row (CSR and shared-memory stencil kernels)
  __device__ __forceinline__ void operator()(int64_t row, AT av, double acc[2]) const {
    int64_t g = row;
    if (gm) {
      const uint32_t r32 = (uint32_t)row, um = (uint32_t)gm, q1 = r32 / um;
      const int64_t G = gm + 2;
      g = (int64_t)(r32 - q1 * um) + 1 + G * ((int64_t)(q1 % um) + 1 + G * ((int64_t)(q1 / um) + 1));
    }
    apply(g, row, av, centre_of(g), load(g, row), acc);
  }
};

template <typename T>
__device__ __forceinline__ void write_partials(double (&acc)[2], double* partials, int want,
                                               int nblocks) {
  if (!want) return;
  block_sum<2>(acc);
  if (threadIdx.x == 0) {
    int bid = blockIdx.x + gridDim.x * (blockIdx.y + gridDim.y * blockIdx.z);
    partials[bid] = acc[0];
    partials[nblocks + bid] = acc[1];
  }
}

// ------------------------------------------------------------------ stencil

constexpr int TX = 32, TY = 8, KZ = 16;

template <typename T>
struct SC {
  T c0, ca, cf, cb;
};

// 2.5D tiling: a block owns a 32 x 8 column of the (i, j) plane and marches KZ planes in
// k, keeping planes k-1, k, k+1 (with a one-point halo) in shared memory.
template <typename T>
__global__ void __launch_bounds__(TX* TY) k_stencil(const T* __restrict__ v, int m, SC<T> c,
                                                    Epi<T> epi, double* partials, int nblocks,
                                                    const int* done) {
  using AT = typename Arith<T>::type;
  if (done && *done) return;
  __shared__ T pl[3][TY + 2][TX + 2];
  const int tx = threadIdx.x & (TX - 1), ty = threadIdx.x / TX;
  const int i0 = blockIdx.x * TX, j0 = blockIdx.y * TY, k0 = blockIdx.z * KZ;
  const int i = i0 + tx, j = j0 + ty;
  const int64_t mm = (int64_t)m * m;
  auto load = [&](int k) {
    const int slot = (k - k0 + 1 + 3) % 3;
    for (int t = threadIdx.x; t < (TY + 2) * (TX + 2); t += TX * TY) {
      const int a = t % (TX + 2), b = t / (TX + 2);
      const int ii = i0 + a - 1, jj = j0 + b - 1;
      T val = (T)0;
      if (k >= 0 && k < m && ii >= 0 && ii < m && jj >= 0 && jj < m)
        val = v[ii + (int64_t)m * jj + mm * k];
      pl[slot][b][a] = val;
    }
  };
  double acc[2] = {0.0, 0.0};
  const int kend = min(k0 + KZ, m);
  load(k0 - 1);
  load(k0);
  const AT c0 = (AT)c.c0, ca = (AT)c.ca, cf = (AT)c.cf, cb = (AT)c.cb;
  for (int k = k0; k < kend; k++) {
    load(k + 1);
    __syncthreads();
    const int sm = (k - k0 + 3) % 3, s0 = (k - k0 + 1) % 3, sp = (k - k0 + 2) % 3;
    if (i < m && j < m) {
      const int a = tx + 1, b = ty + 1;
      AT axis = (AT)pl[s0][b][a - 1] + (AT)pl[s0][b][a + 1] + (AT)pl[s0][b - 1][a] +
                (AT)pl[s0][b + 1][a] + (AT)pl[sm][b][a] + (AT)pl[sp][b][a];
      AT face = (AT)pl[s0][b + 1][a + 1] + (AT)pl[s0][b - 1][a - 1] + (AT)pl[sp][b][a + 1] +
                (AT)pl[sm][b][a - 1] + (AT)pl[sp][b + 1][a] + (AT)pl[sm][b - 1][a];
      AT body = (AT)pl[sp][b + 1][a + 1] + (AT)pl[sm][b - 1][a - 1];
      AT av = c0 * (AT)pl[s0][b][a] + ca * axis + cf * face + cb * body;
      epi((int64_t)i + (int64_t)m * j + mm * k, av, acc);
    }
    __syncthreads();
  }
  write_partials<T>(acc, partials, partials != nullptr, nblocks);
}

// Column marching without shared memory: thread (i, j) walks k, carrying in registers the
// values it needs again one plane later, and loads 7 values per point (plane k: the three
// "minus" neighbours (i-1,j), (i,j-1), (i-1,j-1); plane k+1: (i,j), (i+1,j), (i,j+1),
// (i+1,j+1)).  Warps run along i, so every load is coalesced; there are no barriers.
// The loads of point k+1 (stencil values and the epilogue's operands) are issued before
// point k is finished, so each thread keeps two points' loads in flight.
template <typename T, int TYV, int KZV, int MODE, int MINB, int PF = 0>
__global__ void __launch_bounds__(TX* TYV, MINB) k_stencil_col(const T* __restrict__ v, int m, SC<T> c,
                                                         Epi<T> epi, double* partials,
                                                         int nblocks, const int* done) {
  using AT = typename Arith<T>::type;
  using Ops = typename Epi<T>::Ops;
  if (done && *done) return;
  const int i = blockIdx.x * TX + (threadIdx.x & (TX - 1));
  const int j = blockIdx.y * TYV + threadIdx.x / TX;
  const int k0 = blockIdx.z * KZV;
  const int kend = min(k0 + KZV, m);
  double acc[2] = {0.0, 0.0};
  if (i < m && j < m) {
    const int64_t sj = m, sk = (int64_t)m * m;
    const bool im = i > 0, ip = i < m - 1, jm = j > 0, jp = j < m - 1;
    const T* col = v + (int64_t)i + sj * j;
    const int64_t row0 = (int64_t)i + sj * j;
    auto ld = [&](bool ok, int k, int64_t off) -> AT {
      return (ok && k >= 0 && k < m) ? (AT)__ldg(col + sk * k + off) : (AT)0;
    };
    // plane k0 - 1: centre and minus set; plane k0: centre and plus set
    AT cm = ld(true, k0 - 1, 0);
    AT m_im = ld(im, k0 - 1, -1), m_jm = ld(jm, k0 - 1, -sj), m_ijm = ld(im && jm, k0 - 1, -1 - sj);
    AT c0v = ld(true, k0, 0);
    AT p_ip = ld(ip, k0, 1), p_jp = ld(jp, k0, sj), p_ijp = ld(ip && jp, k0, 1 + sj);
    // loads of the first point: plane k0 minus set, plane k0 + 1 centre and plus set
    AT z_im = ld(im, k0, -1), z_jm = ld(jm, k0, -sj), z_ijm = ld(im && jm, k0, -1 - sj);
    AT cp = ld(true, k0 + 1, 0);
    AT n_ip = ld(ip, k0 + 1, 1), n_jp = ld(jp, k0 + 1, sj), n_ijp = ld(ip && jp, k0 + 1, 1 + sj);
    Ops op = epi.template load<MODE>(row0 + sk * k0, row0 + sk * k0);
    const AT a0 = (AT)c.c0, aa = (AT)c.ca, af = (AT)c.cf, ab = (AT)c.cb;
    for (int k = k0; k < kend; k++) {
      if (PF > 0 && k + PF < kend) {  // L2 prefetch of the streams PF planes ahead (in bounds)
        if (k + PF + 1 < m) l2_prefetch(col + sk * (k + PF + 1));
        epi.template prefetch<MODE>(row0 + sk * (k + PF));
      }
      // issue the next point's loads (beyond kend they are not used)
      const bool more = k + 1 < kend;
      const AT z2_im = ld(im && more, k + 1, -1), z2_jm = ld(jm && more, k + 1, -sj),
               z2_ijm = ld(im && jm && more, k + 1, -1 - sj);
      const AT cp2 = ld(more, k + 2, 0);
      const AT n2_ip = ld(ip && more, k + 2, 1), n2_jp = ld(jp && more, k + 2, sj),
               n2_ijp = ld(ip && jp && more, k + 2, 1 + sj);
      Ops op2;
      if (more) op2 = epi.template load<MODE>(row0 + sk * (k + 1), row0 + sk * (k + 1));
      const AT axis = z_im + p_ip + z_jm + p_jp + cm + cp;
      const AT face = p_ijp + z_ijm + n_ip + m_im + n_jp + m_jm;
      const AT body = n_ijp + m_ijm;
      const AT av = a0 * c0v + aa * axis + af * face + ab * body;
      epi.template apply<MODE>(row0 + sk * k, row0 + sk * k, av, c0v, op, acc);
      // shift: plane k becomes k-1, plane k+1 becomes k
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
  write_partials<T>(acc, partials, partials != nullptr, nblocks);
}

// The column march on the ghost layout (Epi::gm): every neighbour load hits either the grid
// or a zero face, so no load needs a bounds check; only the plane two ahead of the last point
// would leave the array and is not loaded.  Same loads, sums and epilogue as k_stencil_col.
template <typename T, int TYV, int KZV, int MODE, int PF>
__global__ void __launch_bounds__(TX* TYV) k_stencil_gh(const T* __restrict__ v, int m, SC<T> c,
                                                        Epi<T> epi, double* partials,
                                                        int nblocks, const int* done) {
  using AT = typename Arith<T>::type;
  using Ops = typename Epi<T>::Ops;
  if (done && *done) return;
  const int i = blockIdx.x * TX + (threadIdx.x & (TX - 1));
  const int j = blockIdx.y * TYV + threadIdx.x / TX;
  const int k0 = blockIdx.z * KZV;
  const int kend = min(k0 + KZV, m);
  double acc[2] = {0.0, 0.0};
  if (i < m && j < m) {
    const int64_t G = m + 2, sj = G, sk = G * G;
    const int64_t g0 = (int64_t)(i + 1) + sj * (j + 1) + sk * (k0 + 1);   // (i, j, k0)
    const int64_t dsk = (int64_t)m * m;
    const int64_t d0 = (int64_t)i + (int64_t)m * j + dsk * k0;
    const T* pc = v + g0;
    AT cm = (AT)__ldg(pc - sk), m_im = (AT)__ldg(pc - sk - 1), m_jm = (AT)__ldg(pc - sk - sj),
       m_ijm = (AT)__ldg(pc - sk - 1 - sj);
    AT c0v = (AT)__ldg(pc), p_ip = (AT)__ldg(pc + 1), p_jp = (AT)__ldg(pc + sj),
       p_ijp = (AT)__ldg(pc + 1 + sj);
    AT z_im = (AT)__ldg(pc - 1), z_jm = (AT)__ldg(pc - sj), z_ijm = (AT)__ldg(pc - 1 - sj);
    AT cp = (AT)__ldg(pc + sk), n_ip = (AT)__ldg(pc + sk + 1), n_jp = (AT)__ldg(pc + sk + sj),
       n_ijp = (AT)__ldg(pc + sk + 1 + sj);
    Ops op = epi.template load<MODE>(g0, d0);
    const AT a0 = (AT)c.c0, aa = (AT)c.ca, af = (AT)c.cf, ab = (AT)c.cb;
    int64_t g = g0, d = d0;
#pragma unroll 2
    for (int k = k0; k < kend; k++) {
      if (PF > 0 && k + PF < kend) {
        l2_prefetch(pc + (PF + 1) * sk);
        epi.template prefetch<MODE>(g + PF * sk);
      }
      const bool more = k + 1 < kend;
      // next point: plane k + 1 minus set (in the array), plane k + 2 centre and plus set
      // (plane m, the zero face, at the last interior plane; beyond it not loaded)
      const bool two = k + 1 < m;
      const AT z2_im = (AT)__ldg(pc + sk - 1), z2_jm = (AT)__ldg(pc + sk - sj),
               z2_ijm = (AT)__ldg(pc + sk - 1 - sj);
      const AT cp2 = two ? (AT)__ldg(pc + 2 * sk) : (AT)0;
      const AT n2_ip = two ? (AT)__ldg(pc + 2 * sk + 1) : (AT)0,
               n2_jp = two ? (AT)__ldg(pc + 2 * sk + sj) : (AT)0,
               n2_ijp = two ? (AT)__ldg(pc + 2 * sk + 1 + sj) : (AT)0;
      Ops op2;
      if (more) op2 = epi.template load<MODE>(g + sk, d + dsk);
      const AT axis = z_im + p_ip + z_jm + p_jp + cm + cp;
      const AT face = p_ijp + z_ijm + n_ip + m_im + n_jp + m_jm;
      const AT body = n_ijp + m_ijm;
      const AT av = a0 * c0v + aa * axis + af * face + ab * body;
      epi.template apply<MODE>(g, d, av, c0v, op, acc);
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
      pc += sk;
      g += sk;
      d += dsk;
    }
  }
  write_partials<T>(acc, partials, partials != nullptr, nblocks);
}

template <typename T>
int launch_stencil_ghost(const Stencil& s, const T* v, const Epi<T>& epi, double* partials,
                         cudaStream_t st, const int* done) {
  constexpr int TYV = 8, KZV = 16, PF = 4;
  SC<T> c{(T)s.c0, (T)s.ca, (T)s.cf, (T)s.cb};
  const int m = s.m;
  dim3 grid((m + TX - 1) / TX, (m + TYV - 1) / TYV, (m + KZV - 1) / KZV);
  int nb = grid.x * grid.y * grid.z;
  FEM_REQUIRE(!partials || nb <= kMaxPartialBlocks, FEM_EUNSUPPORTED, "stencil grid too large");
  switch (epi.mode) {
    case E_RESIDUAL:
      k_stencil_gh<T, TYV, KZV, E_RESIDUAL, PF><<<grid, TX * TYV, 0, st>>>(v, m, c, epi, partials, nb, done);
      break;
    case E_CHEB_STEP:
      if (epi.z64)
        k_stencil_gh<T, TYV, KZV, E_CHEB_STEP_Z, PF><<<grid, TX * TYV, 0, st>>>(v, m, c, epi, partials, nb, done);
      else
        k_stencil_gh<T, TYV, KZV, E_CHEB_STEP_NOZ, PF><<<grid, TX * TYV, 0, st>>>(v, m, c, epi, partials, nb, done);
      break;
    case E_CHEB_INIT:
      k_stencil_gh<T, TYV, KZV, E_CHEB_INIT, PF><<<grid, TX * TYV, 0, st>>>(v, m, c, epi, partials, nb, done);
      break;
    case E_CHEB_PRE1:
      k_stencil_gh<T, TYV, KZV, E_CHEB_PRE1, PF><<<grid, TX * TYV, 0, st>>>(v, m, c, epi, partials, nb, done);
      break;
    default:
      FEM_REQUIRE(false, FEM_EUNSUPPORTED, "ghost-layout stencil: unsupported epilogue");
  }
  FEM_CHECK_LAUNCH();
  return nb;
}

// Variants of the stencil launch (chosen per (precision, m) by the autotuner):
//   0: shared-memory planes (32 x 8 tile, 16 planes); 1..5: column marching with
//   (rows of the tile, planes per block) = (8,16), (8,32), (4,32), (16,16), (8,64).
//   6, 7: (8,16) and (8,32) with an L2 prefetch of the streamed vectors 4 planes ahead
//   (13% faster than without at 255^3; 8 planes ahead gains less).  Forcing 6 or 8 resident
//   blocks per SM spills registers and runs 1.5-3x slower; an L2 prefetch of the next CSR
//   rows slows the CSR kernels down (extra row-pointer loads on the issue path).
constexpr int kStencilVariants = 8;
const char* const kStencilNames[kStencilVariants] = {
    "smem32x8x16", "col32x8x16", "col32x8x32", "col32x4x32", "col32x16x16", "col32x8x64",
    "col32x8x16_pf4", "col32x8x32_pf4"};

template <typename T, int TYV, int KZV, int MINB = 1, int PF = 0>
int launch_col(const Stencil& s, SC<T> c, const T* v, const Epi<T>& epi, double* partials,
               cudaStream_t st, const int* done) {
  const int m = s.m;
  dim3 grid((m + TX - 1) / TX, (m + TYV - 1) / TYV, (m + KZV - 1) / KZV);
  int nb = grid.x * grid.y * grid.z;
  FEM_REQUIRE(!partials || nb <= kMaxPartialBlocks, FEM_EUNSUPPORTED, "stencil grid too large");
  if (sizeof(T) == 8) {  // ALU-bound: one kernel for every epilogue
    k_stencil_col<T, TYV, KZV, -1, MINB, PF><<<grid, TX * TYV, 0, st>>>(v, m, c, epi, partials, nb, done);
  } else {
    switch (epi.mode) {
      case E_STORE:
        k_stencil_col<T, TYV, KZV, E_STORE, MINB, PF><<<grid, TX * TYV, 0, st>>>(v, m, c, epi, partials, nb, done);
        break;
      case E_RESIDUAL:
        k_stencil_col<T, TYV, KZV, E_RESIDUAL, MINB, PF><<<grid, TX * TYV, 0, st>>>(v, m, c, epi, partials, nb, done);
        break;
      case E_CHEB_STEP:
        if (epi.z64)
          k_stencil_col<T, TYV, KZV, E_CHEB_STEP_Z, MINB, PF><<<grid, TX * TYV, 0, st>>>(v, m, c, epi, partials, nb, done);
        else
          k_stencil_col<T, TYV, KZV, E_CHEB_STEP_NOZ, MINB, PF><<<grid, TX * TYV, 0, st>>>(v, m, c, epi, partials, nb, done);
        break;
      case E_CHEB_INIT:
        k_stencil_col<T, TYV, KZV, E_CHEB_INIT, MINB, PF><<<grid, TX * TYV, 0, st>>>(v, m, c, epi, partials, nb, done);
        break;
      case E_CHEB_PRE1:
        k_stencil_col<T, TYV, KZV, E_CHEB_PRE1, MINB, PF><<<grid, TX * TYV, 0, st>>>(v, m, c, epi, partials, nb, done);
        break;
      default:
        k_stencil_col<T, TYV, KZV, E_ADD, MINB, PF><<<grid, TX * TYV, 0, st>>>(v, m, c, epi, partials, nb, done);
    }
  }
  FEM_CHECK_LAUNCH();
  return nb;
}

template <typename T>
int launch_stencil_variant(int var, const Stencil& s, const T* v, const Epi<T>& epi,
                           double* partials, cudaStream_t st, const int* done) {
  SC<T> c{(T)s.c0, (T)s.ca, (T)s.cf, (T)s.cb};
  switch (var) {
    case 1: return launch_col<T, 8, 16>(s, c, v, epi, partials, st, done);
    case 2: return launch_col<T, 8, 32>(s, c, v, epi, partials, st, done);
    case 3: return launch_col<T, 4, 32>(s, c, v, epi, partials, st, done);
    case 4: return launch_col<T, 16, 16>(s, c, v, epi, partials, st, done);
    case 5: return launch_col<T, 8, 64>(s, c, v, epi, partials, st, done);
    case 6: return launch_col<T, 8, 16, 1, 4>(s, c, v, epi, partials, st, done);
    case 7: return launch_col<T, 8, 32, 1, 4>(s, c, v, epi, partials, st, done);
    default: break;
  }
  const int m = s.m;
  dim3 grid((m + TX - 1) / TX, (m + TY - 1) / TY, (m + KZ - 1) / KZ);
  int nb = grid.x * grid.y * grid.z;
  FEM_REQUIRE(!partials || nb <= kMaxPartialBlocks, FEM_EUNSUPPORTED, "stencil grid too large");
  k_stencil<T><<<grid, TX * TY, 0, st>>>(v, m, c, epi, partials, nb, done);
  FEM_CHECK_LAUNCH();
  return nb;
}

template <typename T>
const char* stencil_key() { return sizeof(T) == 8 ? "stencil_f64" : "stencil_f32"; }

template <typename T>
int launch_stencil(const Stencil& s, const T* v, const Epi<T>& epi, double* partials,
                   cudaStream_t st, const int* done = nullptr) {
  if (epi.gm) return launch_stencil_ghost<T>(s, v, epi, partials, st, done);
  // untuned default: FP64 is ALU-bound (shared-memory planes), FP32 bandwidth-bound
  const int def = sizeof(T) == 8 ? 0 : 6;
  const int var = tuned_variant(stencil_key<T>(), s.m, 0, 0, def, kStencilVariants);
  return launch_stencil_variant<T>(var, s, v, epi, partials, st, done);
}

// ------------------------------------------------------------------ double-float stencil

// q = A p for CG's FP64 vectors without the FP64 pipe: p arrives split into FP32 pairs
// (hi, lo) with p = hi + lo exactly (the split rounds p to 48 bits when CG forms it), the
// four stencil coefficients, scaled by 2^s to about 1, as three FP32 numbers each (exact),
// and the sums of each coefficient class (axis, face, body neighbours) are carried in
// double-float arithmetic: TwoSum on the high parts, the low parts and the rounding errors
// collected in FP32.  The four products and their sum follow the same way; only the final
// hi + lo (one FP64 addition) and <p, q> (one FP64 fused multiply-add) touch the FP64 pipe,
// against 15 FP64 operations per row in FP64.  When any entry of p lies outside the split's
// range (rflag set by the split), the kernel computes the rows in FP64 instead.
// Thread (i, j) marches its column in k like k_stencil_col: 7 pair loads per point, the
// next point's loads issued before the current point is finished.
struct DfCoef {
  float C[4][3];     // c0, ca, cf, cb times 2^s, each as C1 + C2 + C3
  int s;
  double c64[4];     // the FP64 coefficients (fallback)
};

template <int TYV, int KZV>
__global__ void __launch_bounds__(TX* TYV) k_stencil_df(const float2* __restrict__ v,
                                                       const double* __restrict__ v64, int m,
                                                       DfCoef cf, double* __restrict__ y,
                                                       double* partials, int nblocks,
                                                       const int* done, const int* rflag) {
  if (done && *done) return;
  const int i = blockIdx.x * TX + (threadIdx.x & (TX - 1));
  const int j = blockIdx.y * TYV + threadIdx.x / TX;
  const int k0 = blockIdx.z * KZV;
  const int kend = min(k0 + KZV, m);
  double acc[2] = {0.0, 0.0};
  const bool fp64 = *rflag != 0;
  if (i < m && j < m) {
    const int64_t sj = m, sk = (int64_t)m * m;
    const bool im = i > 0, ip = i < m - 1, jm = j > 0, jp = j < m - 1;
    const int64_t row0 = (int64_t)i + sj * j;
    if (fp64) {
      const double* col = v64 + row0;
      auto ld = [&](bool ok, int k, int64_t off) -> double {
        return (ok && k >= 0 && k < m) ? __ldg(col + sk * k + off) : 0.0;
      };
      for (int k = k0; k < kend; k++) {
        const double axis = ld(im, k, -1) + ld(ip, k, 1) + ld(jm, k, -sj) + ld(jp, k, sj) +
                            ld(true, k - 1, 0) + ld(true, k + 1, 0);
        const double face = ld(ip && jp, k, 1 + sj) + ld(im && jm, k, -1 - sj) +
                            ld(ip, k + 1, 1) + ld(im, k - 1, -1) + ld(jp, k + 1, sj) +
                            ld(jm, k - 1, -sj);
        const double body = ld(ip && jp, k + 1, 1 + sj) + ld(im && jm, k - 1, -1 - sj);
        const double c0v = ld(true, k, 0);
        const double av = cf.c64[0] * c0v + cf.c64[1] * axis + cf.c64[2] * face + cf.c64[3] * body;
        y[row0 + sk * k] = av;
        acc[0] = fma(c0v, av, acc[0]);
      }
    } else {
      const float2* col = v + row0;
      const float2 Z = make_float2(0.0f, 0.0f);
      auto ld = [&](bool ok, int k, int64_t off) -> float2 {
        return (ok && k >= 0 && k < m) ? __ldg(col + sk * k + off) : Z;
      };
      float2 cm = ld(true, k0 - 1, 0);
      float2 m_im = ld(im, k0 - 1, -1), m_jm = ld(jm, k0 - 1, -sj), m_ijm = ld(im && jm, k0 - 1, -1 - sj);
      float2 c0v = ld(true, k0, 0);
      float2 p_ip = ld(ip, k0, 1), p_jp = ld(jp, k0, sj), p_ijp = ld(ip && jp, k0, 1 + sj);
      float2 z_im = ld(im, k0, -1), z_jm = ld(jm, k0, -sj), z_ijm = ld(im && jm, k0, -1 - sj);
      float2 cp = ld(true, k0 + 1, 0);
      float2 n_ip = ld(ip, k0 + 1, 1), n_jp = ld(jp, k0 + 1, sj), n_ijp = ld(ip && jp, k0 + 1, 1 + sj);
      double pc = v64 ? __ldg(v64 + row0 + sk * k0) : 0.0;
      for (int k = k0; k < kend; k++) {
        const bool more = k + 1 < kend;
        const float2 z2_im = ld(im && more, k + 1, -1), z2_jm = ld(jm && more, k + 1, -sj),
                     z2_ijm = ld(im && jm && more, k + 1, -1 - sj);
        const float2 cp2 = ld(more, k + 2, 0);
        const float2 n2_ip = ld(ip && more, k + 2, 1), n2_jp = ld(jp && more, k + 2, sj),
                     n2_ijp = ld(ip && jp && more, k + 2, 1 + sj);
        const double pc2 = (v64 && more) ? __ldg(v64 + row0 + sk * (k + 1)) : 0.0;
        // class sums: s exact part, c collected low parts and errors
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
        df_mul(cf.C[0][0], cf.C[0][1], cf.C[0][2], c0v.x, c0v.y, p0, l0);
        df_mul(cf.C[1][0], cf.C[1][1], cf.C[1][2], as, ac, p1, l1);
        df_mul(cf.C[2][0], cf.C[2][1], cf.C[2][2], fs, fc, p2, l2);
        df_mul(cf.C[3][0], cf.C[3][1], cf.C[3][2], bs, bc, p3, l3);
        float ys = p0, yc = l0;
        df_acc(ys, yc, p1, l1);
        df_acc(ys, yc, p2, l2);
        df_acc(ys, yc, p3, l3);
        const float yh = ys + yc;                 // FastTwoSum: |yc| small against ys
        const float yl = yc - (yh - ys);
        const double av = df_to_double(yh, cf.s) + df_to_double(yl, cf.s);
        y[row0 + sk * k] = av;
        acc[0] = fma(pc, av, acc[0]);
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
        pc = pc2;
      }
    }
  }
  write_partials<double>(acc, partials, partials != nullptr, nblocks);
}

// split of an FP64 vector into FP32 pairs (x_out = hi + lo, the 48-bit value; x_out may be
// x), rflag raised when an entry lies outside the split's range
__global__ void k_df_split_vec(int64_t N, const double* x, double* x_out, float2* p2, int* rflag) {
  bool bad = false;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    float hi, lo;
    double xs;
    if (df_split(x[i], hi, lo, xs)) {
      p2[i] = make_float2(hi, lo);
      if (x_out) x_out[i] = xs;
    } else {
      bad = true;
      if (x_out) x_out[i] = x[i];
    }
  }
  if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(rflag, 1);
}

// ------------------------------------------------------------------ CSR4

template <typename VT>
struct Vals4;
template <>
struct Vals4<double> {
  __device__ static void load(const double* p, double o[4]) {
    double2 a = __ldg(reinterpret_cast<const double2*>(p));
    double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
  }
};
template <>
struct Vals4<float> {
  __device__ static void load(const float* p, float o[4]) {
    float4 a = __ldg(reinterpret_cast<const float4*>(p));
    o[0] = a.x; o[1] = a.y; o[2] = a.z; o[3] = a.w;
  }
};
template <>
struct Vals4<__nv_bfloat16> {
  __device__ static void load(const __nv_bfloat16* p, float o[4]) {
    uint2 u = __ldg(reinterpret_cast<const uint2*>(p));
    __nv_bfloat162 a = *reinterpret_cast<__nv_bfloat162*>(&u.x);
    __nv_bfloat162 b = *reinterpret_cast<__nv_bfloat162*>(&u.y);
    float2 fa = __bfloat1622float2(a), fb = __bfloat1622float2(b);
    o[0] = fa.x; o[1] = fa.y; o[2] = fb.x; o[3] = fb.y;
  }
};

// TPR lanes per row; every lane loads 4 consecutive entries (int4 of columns and
// 16/32 bytes of values) per iteration: coalesced 128-bit loads along the rows.
template <int TPR, typename VT, typename T>
__global__ void __launch_bounds__(256) k_csr(int nrows, const int32_t* __restrict__ rowptr,
                                             const int32_t* __restrict__ col,
                                             const VT* __restrict__ val, const T* __restrict__ v,
                                             Epi<T> epi, double* partials, int nblocks,
                                             const int* done) {
  using AT = typename Arith<T>::type;
  if (done && *done) return;
  const int lane = threadIdx.x % TPR;
  const int rows_per_block = blockDim.x / TPR;
  double acc[2] = {0.0, 0.0};
  for (int64_t base = (int64_t)blockIdx.x * rows_per_block; base < nrows;
       base += (int64_t)gridDim.x * rows_per_block) {
    const int64_t row = base + threadIdx.x / TPR;
    AT sum = 0;
    if (row < nrows) {
      const int e0 = rowptr[row], e1 = rowptr[row + 1];
      int e = e0 + 4 * lane;
      // two groups of 4 per step: 8 independent gathers in flight per lane
      for (; e + 4 * TPR < e1; e += 8 * TPR) {
        const int4 ca = __ldg(reinterpret_cast<const int4*>(col + e));
        const int4 cb = __ldg(reinterpret_cast<const int4*>(col + e + 4 * TPR));
        AT wa[4], wb[4];
        Vals4<VT>::load(val + e, wa);
        Vals4<VT>::load(val + e + 4 * TPR, wb);
        const int cs[8] = {ca.x, ca.y, ca.z, ca.w, cb.x, cb.y, cb.z, cb.w};
        AT xv[8];
#pragma unroll
        for (int q = 0; q < 8; q++) xv[q] = cs[q] >= 0 ? (AT)__ldg(v + cs[q]) : (AT)0;
#pragma unroll
        for (int q = 0; q < 4; q++) sum += wa[q] * xv[q];
#pragma unroll
        for (int q = 0; q < 4; q++) sum += wb[q] * xv[4 + q];
      }
      if (e < e1) {
        const int4 c4 = __ldg(reinterpret_cast<const int4*>(col + e));
        AT w[4];
        Vals4<VT>::load(val + e, w);
        const int cs[4] = {c4.x, c4.y, c4.z, c4.w};
#pragma unroll
        for (int q = 0; q < 4; q++)
          if (cs[q] >= 0) sum += w[q] * (AT)__ldg(v + cs[q]);
      }
    }
#pragma unroll
    for (int o = TPR / 2; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o, TPR);
    if (row < nrows && lane == 0) epi(row, sum, acc);
  }
  write_partials<T>(acc, partials, partials != nullptr, nblocks);
}

template <typename VT>
const char* csr_key();
template <>
const char* csr_key<double>() { return "csr_f64"; }
template <>
const char* csr_key<float>() { return "csr_f32"; }
template <>
const char* csr_key<__nv_bfloat16>() { return "csr_bf16"; }

// Variants of the CSR launch: lanes per row (TPR) 1, 2, 4, 8, 16, 32, 256-thread blocks.
constexpr int kCsrVariants = 6;
const char* const kCsrNames[kCsrVariants] = {"tpr1", "tpr2", "tpr4", "tpr8", "tpr16", "tpr32"};

// untuned default from the average stored entries per row
inline int csr_default_variant(double avg) {
  return avg <= 8 ? 1 : (avg <= 16 ? 2 : (avg <= 32 ? 3 : (avg <= 96 ? 4 : 5)));
}

template <typename VT, typename T>
int launch_csr_variant(int var, const Csr4& M, const VT* val, const T* v, const Epi<T>& epi,
                       double* partials, cudaStream_t st, const int* done) {
  const int64_t nr = M.nrows;
  if (nr == 0) return 0;
  const int block = 256;
  const int tpr = 1 << var;
  const int rpb = block / tpr;
  unsigned grid = persistent_grid((nr + rpb - 1) / rpb * block, block, 16);
  FEM_REQUIRE(!partials || (int)grid <= kMaxPartialBlocks, FEM_EUNSUPPORTED, "grid too large");
  switch (tpr) {
    case 1:
      k_csr<1, VT, T><<<grid, block, 0, st>>>(M.nrows, M.rowptr, M.col, val, v, epi, partials, grid, done);
      break;
    case 2:
      k_csr<2, VT, T><<<grid, block, 0, st>>>(M.nrows, M.rowptr, M.col, val, v, epi, partials, grid, done);
      break;
    case 4:
      k_csr<4, VT, T><<<grid, block, 0, st>>>(M.nrows, M.rowptr, M.col, val, v, epi, partials, grid, done);
      break;
    case 8:
      k_csr<8, VT, T><<<grid, block, 0, st>>>(M.nrows, M.rowptr, M.col, val, v, epi, partials, grid, done);
      break;
    case 16:
      k_csr<16, VT, T><<<grid, block, 0, st>>>(M.nrows, M.rowptr, M.col, val, v, epi, partials, grid, done);
      break;
    default:
      k_csr<32, VT, T><<<grid, block, 0, st>>>(M.nrows, M.rowptr, M.col, val, v, epi, partials, grid, done);
  }
  FEM_CHECK_LAUNCH();
  return (int)grid;
}

template <typename VT, typename T>
int launch_csr(const Csr4& M, const VT* val, const T* v, const Epi<T>& epi, double* partials,
               cudaStream_t st, const int* done = nullptr) {
  if (M.nrows == 0) return 0;
  const int def = csr_default_variant((double)M.nnz / (double)M.nrows);
  const int var = tuned_variant(csr_key<VT>(), M.nrows, M.nnz, 0, def, kCsrVariants);
  return launch_csr_variant<VT, T>(var, M, val, v, epi, partials, st, done);
}

// Level operator with the precision's value array.
template <typename T>
int launch_op(const Level& Lv, int prec, const T* v, const Epi<T>& epi, double* partials,
              cudaStream_t st, const int* done = nullptr);

template <>
int launch_op<double>(const Level& Lv, int prec, const double* v, const Epi<double>& epi,
                      double* partials, cudaStream_t st, const int* done) {
  (void)prec;
  if (Lv.stencil) return launch_stencil<double>(Lv.st, v, epi, partials, st, done);
  return launch_csr<double, double>(*Lv.A, Lv.A->val.p, v, epi, partials, st, done);
}
template <>
int launch_op<float>(const Level& Lv, int prec, const float* v, const Epi<float>& epi,
                     double* partials, cudaStream_t st, const int* done) {
  if (Lv.stencil) return launch_stencil<float>(Lv.st, v, epi, partials, st, done);
  if (prec == AMG_PREC_BF16 && Lv.A->val16.p)
    return launch_csr<__nv_bfloat16, float>(*Lv.A, Lv.A->val16.p, v, epi, partials, st, done);
  return launch_csr<float, float>(*Lv.A, Lv.A->val32.p, v, epi, partials, st, done);
}

template <typename T>
Epi<T> epi_base(int mode) {
  Epi<T> e;
  e.mode = mode;
  e.y = nullptr;
  e.b = nullptr;
  e.r = nullptr;
  e.dold = nullptr;
  e.dnew = nullptr;
  e.x = nullptr;
  e.sinv = nullptr;
  e.sinv_c = (T)0;
  e.c1 = e.c2 = (T)0;
  e.add_prev = 0;
  e.xonly = 0;
  e.vin = nullptr;
  e.gm = 0;
  e.ydense = 0;
  e.want_dot = 0;
  e.z64 = nullptr;
  e.r1 = e.r2 = nullptr;
  return e;
}

template <typename T>
const T* level_sinv(const Level& Lv);
template <>
const double* level_sinv<double>(const Level& Lv) { return Lv.scalar_sinv ? nullptr : Lv.dinv.p; }
template <>
const float* level_sinv<float>(const Level& Lv) { return Lv.scalar_sinv ? nullptr : Lv.dinv32.p; }

// ------------------------------------------------------------------ elementwise

// Chebyshev start from x = 0: r = s b, d = r / theta, x = d.  With b64 given the FP64
// right-hand side is converted into b as well (mixed precision, finest level).
// r and x null: only d (and bout) are written (the next kernel is E_CHEB_PRE1).  gm > 0:
// b, bout, r, d, x in the ghost layout of the gm^3 grid (b64 stays dense).
template <typename T>
__global__ void k_cheb_zero(int64_t N, const T* __restrict__ b, const double* __restrict__ b64,
                            T* bout, const T* __restrict__ sinv, T sinv_c, T inv_theta, T* r,
                            T* d, T* x, const int* done, int gm) {
  using AT = typename Arith<T>::type;
  if (done && *done) return;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    int64_t g = i;
    if (gm) {
      const uint32_t r32 = (uint32_t)i, um = (uint32_t)gm, q1 = r32 / um;
      const int64_t G = gm + 2;
      g = (int64_t)(r32 - q1 * um) + 1 + G * ((int64_t)(q1 % um) + 1 + G * ((int64_t)(q1 / um) + 1));
    }
    AT bv;
    if (b64) {
      bv = (AT)b64[i];
      bout[g] = (T)bv;
    } else {
      bv = (AT)b[g];
    }
    AT s = sinv ? (AT)sinv[i] : (AT)sinv_c;
    AT rr = s * bv;
    AT dd = (AT)inv_theta * rr;
    if (r) r[g] = (T)rr;
    d[g] = (T)dd;
    if (x) x[g] = (T)dd;
  }
}

// x += d; optional FP64 output of x with <z, r1>, <z, r2>.
template <typename T>
__global__ void k_add_out(int64_t N, const T* __restrict__ d, T* x, double* z64,
                          const double* r1, const double* r2, double* partials, int nblocks,
                          const int* done) {
  using AT = typename Arith<T>::type;
  if (done && *done) return;
  double acc[2] = {0.0, 0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < N;
       i += (int64_t)gridDim.x * blockDim.x) {
    AT xv = (AT)x[i] + (AT)d[i];
    x[i] = (T)xv;
    if (z64) {
      double z = (double)xv;
      z64[i] = z;
      acc[0] += z * r1[i];
      if (r2) acc[1] += z * r2[i];
    }
  }
  write_partials<T>(acc, partials, partials != nullptr, nblocks);
}

}  // namespace

// ------------------------------------------------------------------ public launchers

void system_level(System& S, Level& Lv) {
  Lv.N = S.N;
  Lv.A = &S.A;
  Lv.stencil = S.stencil;
  Lv.st = S.stA;
}

void op_apply_d(const Level& Lv, const double* x, double* y, double* partials, int* nblocks,
                cudaStream_t st) {
  Epi<double> e = epi_base<double>(E_STORE);
  e.y = y;
  e.vin = x;
  e.want_dot = partials != nullptr;
  int nb = launch_op<double>(Lv, AMG_PREC_FP64, x, e, partials, st);
  if (nblocks) *nblocks = nb;
}

void op_apply_d_done(const Level& Lv, const double* x, double* y, double* partials, int* nblocks,
                     cudaStream_t st, const int* done) {
  Epi<double> e = epi_base<double>(E_STORE);
  e.y = y;
  e.vin = x;
  e.want_dot = partials != nullptr;
  int nb = launch_op<double>(Lv, AMG_PREC_FP64, x, e, partials, st, done);
  if (nblocks) *nblocks = nb;
}

DfOperator df_operator(const Stencil& st) {
  DfOperator D;
  const double c[4] = {st.c0, st.ca, st.cf, st.cb};
  double mx = 0.0;
  for (double v : c) mx = std::max(mx, std::fabs(v));
  D.s = mx > 0.0 ? -std::ilogb(mx) : 0;
  for (int k = 0; k < 4; k++) {
    const double cs = std::ldexp(c[k], D.s);
    const float c1 = (float)cs;
    const float c2 = (float)(cs - (double)c1);
    const float c3 = (float)(cs - (double)c1 - (double)c2);
    D.C[k][0] = c1;
    D.C[k][1] = c2;
    D.C[k][2] = c3;
    D.c64[k] = c[k];
  }
  return D;
}

int op_apply_df(const Level& Lv, const DfOperator& D, const float2* p2, const double* p64,
                double* y, double* partials, cudaStream_t st, const int* done, const int* rflag) {
  constexpr int TYV = 8, KZV = 32;
  DfCoef c;
  for (int k = 0; k < 4; k++) {
    for (int t = 0; t < 3; t++) c.C[k][t] = D.C[k][t];
    c.c64[k] = D.c64[k];
  }
  c.s = D.s;
  const int m = Lv.st.m;
  dim3 grid((m + TX - 1) / TX, (m + TYV - 1) / TYV, (m + KZV - 1) / KZV);
  const int nb = grid.x * grid.y * grid.z;
  FEM_REQUIRE(!partials || nb <= kMaxPartialBlocks, FEM_EUNSUPPORTED, "stencil grid too large");
  k_stencil_df<TYV, KZV><<<grid, TX * TYV, 0, st>>>(p2, p64, m, c, y, partials, nb, done, rflag);
  FEM_CHECK_LAUNCH();
  return nb;
}

void df_split_vec(int64_t N, const double* x, double* x_out, float2* p2, int* rflag,
                  cudaStream_t st) {
  k_df_split_vec<<<persistent_grid(N, 256, 8), 256, 0, st>>>(N, x, x_out, p2, rflag);
  FEM_CHECK_LAUNCH();
}

template <typename T>
void op_residual(const Level& Lv, int prec, const T* b, const T* x, T* r, cudaStream_t st) {
  Epi<T> e = epi_base<T>(E_RESIDUAL);
  e.y = r;
  e.b = b;
  if (Lv.ghost) {
    e.gm = Lv.st.m;
    e.ydense = 1;
  }
  launch_op<T>(Lv, prec, x, e, nullptr, st, Lv.done);
}

template <>
void csr_spmv<double>(const Csr4& M, int prec, const double* x, double* y, bool accumulate,
                      cudaStream_t st, const int* done, int ghost_m) {
  (void)prec;
  Epi<double> e = epi_base<double>(accumulate ? E_ADD : E_STORE);
  e.y = y;
  e.gm = ghost_m;
  launch_csr<double, double>(M, M.val.p, x, e, nullptr, st, done);
}
template <>
void csr_spmv<float>(const Csr4& M, int prec, const float* x, float* y, bool accumulate,
                     cudaStream_t st, const int* done, int ghost_m) {
  Epi<float> e = epi_base<float>(accumulate ? E_ADD : E_STORE);
  e.y = y;
  e.gm = ghost_m;
  if (prec == AMG_PREC_BF16 && M.val16.p)
    launch_csr<__nv_bfloat16, float>(M, M.val16.p, x, e, nullptr, st, done);
  else
    launch_csr<float, float>(M, M.val32.p, x, e, nullptr, st, done);
}

// ------------------------------------------------------------------ stencil prolongation

namespace {

// t = P_t x_c on the uniform finest level in the ghost layout: each node takes its
// aggregate's value (isolated nodes 0); the ghost faces of t stay zero.  Four nodes per
// thread and round, their loads in flight together.
constexpr int PST_U = 4;
__global__ void k_inject_ghost(int m, const int32_t* __restrict__ agg, const float* __restrict__ xc,
                               float* __restrict__ t, const int* done) {
  if (done && *done) return;
  const int64_t N = (int64_t)m * m * m;
  const int64_t G = m + 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r0 < N; r0 += PST_U * stride) {
    int a[PST_U];
#pragma unroll
    for (int u = 0; u < PST_U; u++) {
      const int64_t r = r0 + u * stride;
      a[u] = r < N ? __ldg(agg + r) : -1;
    }
    float v[PST_U];
#pragma unroll
    for (int u = 0; u < PST_U; u++) v[u] = a[u] >= 0 ? __ldg(xc + a[u]) : 0.0f;
#pragma unroll
    for (int u = 0; u < PST_U; u++) {
      const int64_t r = r0 + u * stride;
      if (r >= N) break;
      const uint32_t r32 = (uint32_t)r, um = (uint32_t)m, q1 = r32 / um;
      const int i = (int)(r32 - q1 * um), j = (int)(q1 % um), k = (int)(q1 / um);
      t[(i + 1) + G * ((j + 1) + G * (k + 1))] = v[u];
    }
  }
}

struct PstCoef {
  float c[27];
};

// x += [agg >= 0] (c[13] t + sum over the strong directions d of c[d] t(. + d)): the smoothed
// prolongator's row of every node, from its own and its neighbours' aggregates (a direction
// leaving the grid reads a zero ghost face).  Four nodes per thread and round.
template <uint32_t MASK>   // the strong directions (0: the run-time mask `strong`)
__global__ void k_prolong_st(int m, uint32_t strong, PstCoef pc, const int32_t* __restrict__ agg,
                             const float* __restrict__ t, float* __restrict__ x, const int* done) {
  if (done && *done) return;
  const int64_t N = (int64_t)m * m * m;
  const int64_t G = m + 2;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r0 < N; r0 += PST_U * stride) {
    int64_t g[PST_U];
    bool live[PST_U];
    float s[PST_U], xo[PST_U];
#pragma unroll
    for (int u = 0; u < PST_U; u++) {
      const int64_t r = r0 + u * stride;
      live[u] = r < N && __ldg(agg + r) >= 0;
      const int64_t rr = r < N ? r : 0;
      const uint32_t r32 = (uint32_t)rr, um = (uint32_t)m, q1 = r32 / um;
      const int i = (int)(r32 - q1 * um), j = (int)(q1 % um), k = (int)(q1 / um);
      g[u] = (i + 1) + G * ((j + 1) + G * (k + 1));
    }
#pragma unroll
    for (int u = 0; u < PST_U; u++) {
      s[u] = 0.0f;
      xo[u] = 0.0f;
      if (!live[u]) continue;
      xo[u] = x[g[u]];
      s[u] = pc.c[13] * __ldg(t + g[u]);
#pragma unroll
      for (int d = 0; d < 27; d++) {
        if (d == 13 || !(((MASK ? MASK : strong) >> d) & 1u)) continue;
        const int64_t off = (int64_t)(d % 3 - 1) + G * ((d / 3 % 3 - 1) + G * (d / 9 - 1));
        s[u] += pc.c[d] * __ldg(t + g[u] + off);
      }
    }
#pragma unroll
    for (int u = 0; u < PST_U; u++)
      if (live[u]) x[g[u]] = xo[u] + s[u];
  }
}

}  // namespace

void prolong_stencil(const Level& L, const float* xc, float* x, cudaStream_t st) {
  const int m = L.st.m;
  const unsigned g = persistent_grid((int64_t)m * m * m, 256, 8);
  const int bt = 256;
  k_inject_ghost<<<g, bt, 0, st>>>(m, L.agg, xc, L.tf, L.done);
  FEM_CHECK_LAUNCH();
  PstCoef pc;
  for (int d = 0; d < 27; d++) pc.c[d] = L.pst_c[d];
  // the axis directions (strong on the Kuhn stencil's mass-dominated regime) compiled in
  constexpr uint32_t kAxis = (1u << 4) | (1u << 10) | (1u << 12) | (1u << 14) | (1u << 16) | (1u << 22);
  if (L.pst_strong == kAxis)
    k_prolong_st<kAxis><<<g, bt, 0, st>>>(m, L.pst_strong, pc, L.agg, L.tf, x, L.done);
  else
    k_prolong_st<0u><<<g, bt, 0, st>>>(m, L.pst_strong, pc, L.agg, L.tf, x, L.done);
  FEM_CHECK_LAUNCH();
}

// Pre-smoothing from the zero initial guess.
template <typename T>
void smooth_pre_zero(const Level& Lv, int prec, const amg_opts& o, const ChebCoef& cc,
                     const T* b, T* x, T* r, T* d0, T* d1, cudaStream_t st, const double* b64) {
  const int64_t N = Lv.N;
  const T* sinv = level_sinv<T>(Lv);
  T sinv_c = Lv.scalar_sinv ? (T)(1.0 / Lv.st.c0) : (T)0;
  unsigned g = persistent_grid(N, 256, 8);
  if (cc.degree == 2) {
    // start from x = 0 and the one step after it, which needs only d, b and writes x
    k_cheb_zero<T><<<g, 256, 0, st>>>(N, b, b64, const_cast<T*>(b), sinv, sinv_c,
                                      (T)cc.inv_theta, nullptr, d0, nullptr, Lv.done,
                                      Lv.ghost ? Lv.st.m : 0);
    FEM_CHECK_LAUNCH();
    Epi<T> e = epi_base<T>(E_CHEB_PRE1);
    e.gm = Lv.ghost ? Lv.st.m : 0;
    e.b = b;
    e.dold = d0;
    e.x = x;
    e.sinv = sinv;
    e.sinv_c = sinv_c;
    e.c1 = (T)cc.c1[1];
    e.c2 = (T)cc.c2[1];
    launch_op<T>(Lv, prec, d0, e, nullptr, st, Lv.done);
    (void)r;
    (void)d1;
    (void)o;
    return;
  }
  k_cheb_zero<T><<<g, 256, 0, st>>>(N, b, b64, const_cast<T*>(b), sinv, sinv_c,
                                    (T)cc.inv_theta, r, d0, x, Lv.done, Lv.ghost ? Lv.st.m : 0);
  FEM_CHECK_LAUNCH();
  T* dold = d0;
  T* dnew = d1;
  for (int i = 1; i < cc.degree; i++) {
    Epi<T> e = epi_base<T>(E_CHEB_STEP);
    e.gm = Lv.ghost ? Lv.st.m : 0;
    e.r = r;
    e.dold = dold;
    e.dnew = dnew;
    e.x = x;
    e.sinv = sinv;
    e.sinv_c = sinv_c;
    e.c1 = (T)cc.c1[i];
    e.c2 = (T)cc.c2[i];
    e.add_prev = 0;
    launch_op<T>(Lv, prec, dold, e, nullptr, st, Lv.done);
    std::swap(dold, dnew);
  }
  (void)o;
}

// Post-smoothing from the current x; the last kernel may emit z (FP64) and dots.
template <typename T>
void smooth_post(const Level& Lv, int prec, const amg_opts& o, const ChebCoef& cc, const T* b,
                 T* x, T* r, T* d0, T* d1, cudaStream_t st, const DotOut* dot) {
  const int64_t N = Lv.N;
  const T* sinv = level_sinv<T>(Lv);
  T sinv_c = Lv.scalar_sinv ? (T)(1.0 / Lv.st.c0) : (T)0;
  const int* done = Lv.done;
  {
    Epi<T> e = epi_base<T>(E_CHEB_INIT);
    e.gm = Lv.ghost ? Lv.st.m : 0;
    e.b = b;
    e.r = r;
    e.dnew = d0;
    e.sinv = sinv;
    e.sinv_c = sinv_c;
    e.c2 = (T)cc.inv_theta;
    launch_op<T>(Lv, prec, x, e, nullptr, st, done);
  }
  if (cc.degree == 1) {
    unsigned g = persistent_grid(N, 256, 8);
    k_add_out<T><<<g, 256, 0, st>>>(N, d0, x, dot ? dot->z64 : nullptr, dot ? dot->r1 : nullptr,
                                    dot ? dot->r2 : nullptr, dot ? dot->partials : nullptr, g,
                                    done);
    FEM_CHECK_LAUNCH();
    if (dot && dot->nblocks) *dot->nblocks = (int)g;
    return;
  }
  T* dold = d0;
  T* dnew = d1;
  for (int i = 1; i < cc.degree; i++) {
    const bool last = (i == cc.degree - 1);
    Epi<T> e = epi_base<T>(E_CHEB_STEP);
    e.gm = Lv.ghost ? Lv.st.m : 0;
    e.r = r;
    e.dold = dold;
    e.dnew = dnew;
    e.x = x;
    e.sinv = sinv;
    e.sinv_c = sinv_c;
    e.c1 = (T)cc.c1[i];
    e.c2 = (T)cc.c2[i];
    e.add_prev = (i == 1);
    e.xonly = last ? 1 : 0;
    double* partials = nullptr;
    if (last && dot) {
      e.z64 = dot->z64;
      e.r1 = dot->r1;
      e.r2 = dot->r2;
      partials = dot->partials;
    }
    int nb = launch_op<T>(Lv, prec, dold, e, partials, st, done);
    if (last && dot && dot->nblocks) *dot->nblocks = nb;
    std::swap(dold, dnew);
  }
  (void)o;
}

template void op_residual<double>(const Level&, int, const double*, const double*, double*,
                                  cudaStream_t);
template void op_residual<float>(const Level&, int, const float*, const float*, float*,
                                 cudaStream_t);
template void smooth_pre_zero<double>(const Level&, int, const amg_opts&, const ChebCoef&,
                                      const double*, double*, double*, double*, double*,
                                      cudaStream_t, const double*);
template void smooth_pre_zero<float>(const Level&, int, const amg_opts&, const ChebCoef&,
                                     const float*, float*, float*, float*, float*, cudaStream_t,
                                     const double*);
template void smooth_post<double>(const Level&, int, const amg_opts&, const ChebCoef&,
                                  const double*, double*, double*, double*, double*,
                                  cudaStream_t, const DotOut*);
template void smooth_post<float>(const Level&, int, const amg_opts&, const ChebCoef&,
                                 const float*, float*, float*, float*, float*, cudaStream_t,
                                 const DotOut*);

// ------------------------------------------------------------------ Gauss-Seidel

namespace {

__device__ __forceinline__ double val_of(double v) { return v; }
__device__ __forceinline__ float val_of(float v) { return v; }
__device__ __forceinline__ float val_of(__nv_bfloat16 v) { return __bfloat162float(v); }

// x_i = (b_i - sum_{j != i} a_ij x_j) / a_ii for the nodes of one colour class (thread per
// node, the row's entries in column order; FP64 without contraction, as in the oracle).
template <typename VT, typename T>
__global__ void k_gs(int64_t cnt, const int32_t* __restrict__ nodes,
                     const int32_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                     const VT* __restrict__ val, const T* __restrict__ b, T* x, const int* done) {
  using AT = typename Arith<T>::type;
  if (done && *done) return;
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= cnt) return;
  const int i = nodes[t];
  AT sum = (AT)0, dg = (AT)0;
  for (int e = rowptr[i]; e < rowptr[i + 1]; e++) {
    const int j = col[e];
    if (j < 0) continue;
    const AT a = (AT)val_of(val[e]);
    if (j == i) {
      dg = a;
    } else if (sizeof(AT) == 8) {
      sum = (AT)__dadd_rn((double)sum, __dmul_rn((double)a, (double)x[j]));
    } else {
      sum += a * (AT)x[j];
    }
  }
  x[i] = (T)(((AT)b[i] - sum) / dg);
}

template <typename VT, typename T>
void gs_launch(const Level& Lv, const VT* val, const T* b, T* x, bool forward, cudaStream_t st) {
  const int ncol = (int)Lv.coff.size() - 1;
  for (int q = 0; q < ncol; q++) {
    const int c = forward ? q : ncol - 1 - q;
    const int64_t c0 = Lv.coff[c], cnt = Lv.coff[c + 1] - c0;
    if (cnt == 0) continue;
    k_gs<VT, T><<<grid_for(cnt, 256), 256, 0, st>>>(cnt, Lv.cnodes.p + c0, Lv.A->rowptr,
                                                    Lv.A->col, val, b, x, Lv.done);
    FEM_CHECK_LAUNCH();
  }
}

}  // namespace

template <>
void gs_sweep<double>(const Level& Lv, int prec, const double* b, double* x, bool forward,
                      cudaStream_t st) {
  (void)prec;
  gs_launch<double, double>(Lv, Lv.A->val.p, b, x, forward, st);
}
template <>
void gs_sweep<float>(const Level& Lv, int prec, const float* b, float* x, bool forward,
                     cudaStream_t st) {
  if (prec == AMG_PREC_BF16 && Lv.A->val16.p)
    gs_launch<__nv_bfloat16, float>(Lv, Lv.A->val16.p, b, x, forward, st);
  else
    gs_launch<float, float>(Lv, Lv.A->val32.p, b, x, forward, st);
}

// ------------------------------------------------------------------ launch-shape tuning

namespace {
constexpr int64_t kTuneMinEntries = 1 << 18;   // smaller operators: launch-bound, default

template <typename VT, typename T>
void tune_csr(const Csr4& M, const VT* val, const T* x, T* y, int mode, cudaStream_t st) {
  if (M.nrows == 0 || M.nnz < kTuneMinEntries || !val) return;
  const int def = csr_default_variant((double)M.nnz / (double)M.nrows);
  Epi<T> e = epi_base<T>(mode);
  e.y = y;
  autotune(csr_key<VT>(), M.nrows, M.nnz, 0, kCsrVariants, kCsrNames, def, st,
           [&](int v) { launch_csr_variant<VT, T>(v, M, val, x, e, nullptr, st, nullptr); });
}

template <typename T>
void tune_csr_prec(const Csr4& M, int prec, const T* x, T* y, int mode, cudaStream_t st);
template <>
void tune_csr_prec<double>(const Csr4& M, int prec, const double* x, double* y, int mode,
                           cudaStream_t st) {
  (void)prec;
  tune_csr<double, double>(M, M.val.p, x, y, mode, st);
}
template <>
void tune_csr_prec<float>(const Csr4& M, int prec, const float* x, float* y, int mode,
                          cudaStream_t st) {
  if (prec == AMG_PREC_BF16 && M.val16.p)
    tune_csr<__nv_bfloat16, float>(M, M.val16.p, x, y, mode, st);
  else
    tune_csr<float, float>(M, M.val32.p, x, y, mode, st);
}

// Stencil: the FP32 shape is tuned on the Chebyshev step (the V-cycle's most frequent
// launch), the FP64 shape on y = A x with <x, y> (the CG operator).
void tune_stencil_f32(const Stencil& s, float* v, float* r, float* dn, float* x, cudaStream_t st) {
  Epi<float> e = epi_base<float>(E_CHEB_STEP);
  e.r = r;
  e.dold = v;
  e.dnew = dn;
  e.x = x;
  e.sinv_c = (float)(1.0 / s.c0);
  e.c1 = 0.5f;
  e.c2 = 0.5f;
  autotune("stencil_f32", s.m, 0, 0, kStencilVariants, kStencilNames, 6, st,
           [&](int var) { launch_stencil_variant<float>(var, s, v, e, nullptr, st, nullptr); });
}

void tune_stencil_f64(const Stencil& s, double* v, double* y, double* partials, cudaStream_t st) {
  Epi<double> e = epi_base<double>(E_STORE);
  e.y = y;
  e.vin = v;
  e.want_dot = 1;
  autotune("stencil_f64", s.m, 0, 0, kStencilVariants, kStencilNames, 0, st,
           [&](int var) { launch_stencil_variant<double>(var, s, v, e, partials, st, nullptr); });
}

template <typename T>
void tune_levels(Hierarchy& H, cudaStream_t st, T* (*vec)(Level&, int)) {
  const int prec = H.o.precision;
  for (size_t l = 0; l < H.L.size(); l++) {
    Level& L = *H.L[l];
    T* x = vec(L, 0);
    T* b = vec(L, 1);
    T* r = vec(L, 2);
    T* d0 = vec(L, 3);
    T* d1 = vec(L, 4);
    FEM_CUDA(cudaMemsetAsync(x, 0, L.N * sizeof(T), st));
    FEM_CUDA(cudaMemsetAsync(r, 0, L.N * sizeof(T), st));
    FEM_CUDA(cudaMemsetAsync(d0, 0, L.N * sizeof(T), st));
    if (L.stencil) {
      if (sizeof(T) == 4)
        tune_stencil_f32(L.st, (float*)(void*)d0, (float*)(void*)r, (float*)(void*)d1,
                         (float*)(void*)x, st);
    } else if (!L.coarsest || !L.Ainv.p) {
      tune_csr_prec<T>(*L.A, prec, x, b, E_STORE, st);
    }
    if (!L.coarsest && l + 1 < H.L.size()) {
      Level& C = *H.L[l + 1];
      T* cx = vec(C, 0);
      T* cb = vec(C, 1);
      FEM_CUDA(cudaMemsetAsync(cx, 0, C.N * sizeof(T), st));
      tune_csr_prec<T>(L.R, prec, r, cb, E_STORE, st);
      tune_csr_prec<T>(L.P, prec, cx, x, E_ADD, st);
    }
  }
}

float* vec_f(Level& L, int k) {
  DevBuf<float>* v[5] = {&L.xf, &L.bf, &L.rf, &L.d0f, &L.d1f};
  return v[k]->p;
}
double* vec_d(Level& L, int k) {
  DevBuf<double>* v[5] = {&L.x, &L.b, &L.r, &L.d0, &L.d1};
  return v[k]->p;
}
}  // namespace

void reset_ghost_vectors(Hierarchy& H, cudaStream_t st) {
  for (auto& Lp : H.L) {
    Level& L = *Lp;
    if (!L.ghost) continue;
    for (DevBuf<float>* v : {&L.xf, &L.bf, &L.rf, &L.d0f, &L.d1f})
      FEM_CUDA(cudaMemsetAsync(v->p, 0, sizeof(float) * v->n, st));
  }
}

void tune_hierarchy(Hierarchy& H, System& S, cudaStream_t st) {
  if (H.o.precision == AMG_PREC_FP64)
    tune_levels<double>(H, st, vec_d);
  else
    tune_levels<float>(H, st, vec_f);
  // the CG operator (FP64) on the finest level
  const int64_t N = S.N;
  if (N == 0) return;
  DevBuf<double> tmp(2 * (size_t)N, st);
  FEM_CUDA(cudaMemsetAsync(tmp.p, 0, 2 * (size_t)N * sizeof(double), st));
  if (S.stencil)
    tune_stencil_f64(S.stA, tmp.p, tmp.p + N, H.partials.p, st);
  else
    tune_csr<double, double>(S.A, S.A.val.p, tmp.p, tmp.p + N, E_STORE, st);
}

// ------------------------------------------------------------------ reductions

namespace {
__global__ void k_finalize(const double* partials, int nblocks, int nv, double* out,
                           const int* done) {
  if (done && *done) return;
  for (int k = 0; k < nv; k++) {
    double v[1] = {0.0};
    for (int i = threadIdx.x; i < nblocks; i += blockDim.x) v[0] += partials[(int64_t)k * nblocks + i];
    block_sum<1>(v);
    if (threadIdx.x == 0) out[k] = v[0];
    __syncthreads();
  }
}
}  // namespace

void finalize_sums(const double* partials, int nblocks, int nv, double* out, cudaStream_t st,
                   const int* done) {
  k_finalize<<<1, 1024, 0, st>>>(partials, nblocks, nv, out, done);
  FEM_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ FP64 throughput probe

namespace {
// 8 independent chains of fused multiply-adds per thread, so that the FP64 pipe's throughput
// and not its latency bounds the kernel; the chains converge to c / (1 - m) (no overflow or
// subnormal values), and the final test keeps them live
__global__ void __launch_bounds__(256) k_fp64_fma_probe(int iters, double m, double c,
                                                        double* out) {
  double a[8];
  const double s = 1.0 + 1e-9 * (double)(blockIdx.x * blockDim.x + threadIdx.x);
#pragma unroll
  for (int k = 0; k < 8; k++) a[k] = s + k;
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int k = 0; k < 8; k++) a[k] = fma(a[k], m, c);
  }
  const double t = ((a[0] + a[1]) + (a[2] + a[3])) + ((a[4] + a[5]) + (a[6] + a[7]));
  if (t == -1.0) out[0] = t;
}
}  // namespace

double fp64_fma_rate(int reps, cudaStream_t st) {
  int dev = 0, sms = 0;
  FEM_CUDA(cudaGetDevice(&dev));
  FEM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const unsigned blocks = 8u * (unsigned)sms;
  const int iters = 4096;
  DevBuf<double> out(1, st);
  k_fp64_fma_probe<<<blocks, 256, 0, st>>>(iters, 0.9999999, 1e-7, out);
  FEM_CHECK_LAUNCH();
  cudaEvent_t e0, e1;
  FEM_CUDA(cudaEventCreate(&e0));
  FEM_CUDA(cudaEventCreate(&e1));
  FEM_CUDA(cudaEventRecord(e0, st));
  for (int r = 0; r < reps; r++) {
    k_fp64_fma_probe<<<blocks, 256, 0, st>>>(iters, 0.9999999, 1e-7, out);
    FEM_CHECK_LAUNCH();
  }
  FEM_CUDA(cudaEventRecord(e1, st));
  FEM_CUDA(cudaEventSynchronize(e1));
  float ms = 0.0f;
  FEM_CUDA(cudaEventElapsedTime(&ms, e0, e1));
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  const double flops = 2.0 * 8.0 * iters * (double)blocks * 256.0 * reps;
  return flops / (ms * 1e-3) / 1e12;
}

}  // namespace fem
