// Device assembly of K, M, f for P1 elements on the Kuhn mesh of the unit cube
// (arXiv 2102.03515, Sec. 2: K_ij = int grad phi_j . grad phi_i, M_ij = int phi_j phi_i,
// f_i = int ubar phi_i; A = rho K + M, eq. (linsys)).
//
// Layout.  Unknowns are the interior vertices (i,j,k), 1..n-1 per axis, numbered
// (i-1) + m((j-1) + m(k-1)), m = n-1.  In the Kuhn mesh vertex v is joined to
// v +- e_d, v +- (e_a + e_b) and v +- (1,1,1): 14 neighbours, so every CSR4 row has at
// most 15 entries and is stored with 16 slots (rowptr[r] = 16 r), real entries first in
// increasing column order, then (col -1, value 0) padding.
//
// Element arithmetic is done without FMA contraction (this file is compiled with
// -fmad=false) so that sums of element contributions follow plain IEEE rounding.
#include <cmath>
#include <mutex>
#include <vector>

#include "solver.cuh"

namespace fem {
namespace {

// The 15 stencil slots in increasing linear-offset order (di + m dj + m^2 dk).
__constant__ int kSlotOff[15][3] = {
    {-1, -1, -1}, {0, -1, -1}, {-1, 0, -1}, {0, 0, -1}, {-1, -1, 0}, {0, -1, 0}, {-1, 0, 0},
    {0, 0, 0},    {1, 0, 0},   {0, 1, 0},   {1, 1, 0},  {0, 0, 1},   {1, 0, 1},  {0, 1, 1},
    {1, 1, 1}};
// Slot type: 0 centre, 1 axis, 2 face diagonal, 3 body diagonal.
__constant__ int kSlotType[15] = {3, 2, 2, 1, 2, 1, 1, 0, 1, 1, 2, 1, 2, 2, 3};
// Tet paths: permutation p steps along kPerm[p][0], then [1], then [2].
__constant__ int kPerm[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};

__device__ __forceinline__ int slot_of(int di, int dj, int dk) {
  // inverse of kSlotOff for Kuhn neighbours; -1 if not a neighbour
  int code = (di + 1) + 3 * (dj + 1) + 9 * (dk + 1);
  switch (code) {
    case 0: return 0;   // (-1,-1,-1)
    case 1: return 1;   // (0,-1,-1)
    case 3: return 2;   // (-1,0,-1)
    case 4: return 3;   // (0,0,-1)
    case 9: return 4;   // (-1,-1,0)
    case 10: return 5;  // (0,-1,0)
    case 12: return 6;  // (-1,0,0)
    case 13: return 7;  // (0,0,0)
    case 14: return 8;  // (1,0,0)
    case 16: return 9;  // (0,1,0)
    case 17: return 10; // (1,1,0)
    case 22: return 11; // (0,0,1)
    case 23: return 12; // (1,0,1)
    case 25: return 13; // (0,1,1)
    case 26: return 14; // (1,1,1)
  }
  return -1;
}

// det J and barycentric gradients of a tet (rows of J^{-1}; grad lambda_0 = -sum).
__device__ double tet_grads(const double X[4][3], double g[4][3]) {
  double J[3][3];
  for (int r = 0; r < 3; r++)
    for (int c = 0; c < 3; c++) J[r][c] = X[c + 1][r] - X[0][r];
  double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
               J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
               J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  double inv[3][3];
  inv[0][0] = (J[1][1] * J[2][2] - J[1][2] * J[2][1]) / det;
  inv[0][1] = (J[0][2] * J[2][1] - J[0][1] * J[2][2]) / det;
  inv[0][2] = (J[0][1] * J[1][2] - J[0][2] * J[1][1]) / det;
  inv[1][0] = (J[1][2] * J[2][0] - J[1][0] * J[2][2]) / det;
  inv[1][1] = (J[0][0] * J[2][2] - J[0][2] * J[2][0]) / det;
  inv[1][2] = (J[0][2] * J[1][0] - J[0][0] * J[1][2]) / det;
  inv[2][0] = (J[1][0] * J[2][1] - J[1][1] * J[2][0]) / det;
  inv[2][1] = (J[0][1] * J[2][0] - J[0][0] * J[2][1]) / det;
  inv[2][2] = (J[0][0] * J[1][1] - J[0][1] * J[1][0]) / det;
  for (int d = 0; d < 3; d++) {
    g[1][d] = inv[0][d];
    g[2][d] = inv[1][d];
    g[3][d] = inv[2][d];
    g[0][d] = -(inv[0][d] + inv[1][d] + inv[2][d]);
  }
  return det;
}

struct Coords {
  const double* xyz;  // null: uniform grid
  int n;
  double h;
  __device__ void get(int i, int j, int k, double out[3]) const {
    if (xyz) {
      int64_t v = (int64_t)i + (int64_t)(n + 1) * ((int64_t)j + (int64_t)(n + 1) * k);
      out[0] = xyz[3 * v];
      out[1] = xyz[3 * v + 1];
      out[2] = xyz[3 * v + 2];
    } else {
      out[0] = i * h;
      out[1] = j * h;
      out[2] = k * h;
    }
  }
};

// Row r of K and M (15 slots each) for the interior vertex (i,j,k): element
// contributions of its 24 tets, visited in increasing tet index (cube id, then path).
__device__ void vertex_row(const Coords& C, int i, int j, int k, double kv[15], double mv[15]) {
  for (int s = 0; s < 15; s++) kv[s] = mv[s] = 0.0;
  for (int dd = 7; dd >= 0; dd--) {
    const int ci = i - (dd & 1), cj = j - ((dd >> 1) & 1), ck = k - ((dd >> 2) & 1);
    if (ci < 0 || cj < 0 || ck < 0 || ci >= C.n || cj >= C.n || ck >= C.n) continue;
    for (int p = 0; p < 6; p++) {
      int v[4][3];
      v[0][0] = ci; v[0][1] = cj; v[0][2] = ck;
      for (int s = 0; s < 3; s++) {
        for (int d = 0; d < 3; d++) v[s + 1][d] = v[s][d];
        v[s + 1][kPerm[p][s]] += 1;
      }
      int loc = -1;
      for (int a = 0; a < 4; a++)
        if (v[a][0] == i && v[a][1] == j && v[a][2] == k) loc = a;
      if (loc < 0) continue;
      double X[4][3], g[4][3];
      for (int a = 0; a < 4; a++) C.get(v[a][0], v[a][1], v[a][2], X[a]);
      double det = tet_grads(X, g);
      double vol = fabs(det) / 6.0;
      for (int b = 0; b < 4; b++) {
        int s = slot_of(v[b][0] - i, v[b][1] - j, v[b][2] - k);
        double ke = vol * (g[loc][0] * g[b][0] + g[loc][1] * g[b][1] + g[loc][2] * g[b][2]);
        double me = vol * (loc == b ? 2.0 : 1.0) / 20.0;
        kv[s] += ke;
        mv[s] += me;
      }
    }
  }
}

// One interior vertex's row on the uniform grid gives the stencils of K and M.
__global__ void k_uniform_row(int n, double rho, double* out /* 45: K, M, A slots */) {
  Coords C{nullptr, n, 1.0 / n};
  double kv[15], mv[15];
  vertex_row(C, 1, 1, 1, kv, mv);
  for (int s = 0; s < 15; s++) {
    out[s] = kv[s];
    out[15 + s] = mv[s];
    out[30 + s] = rho * kv[s] + mv[s];
  }
}

// CSR4 rows (16 slots) with values from per-type stencil coefficients, one thread per row
// with 16-byte stores: slot p of row r holds the p-th existing neighbour.  Interior rows
// (all 15 neighbours on the grid) take their columns from fixed offsets, rows next to the
// boundary list their existing neighbours in slot order and pad.
__global__ void k_csr_uniform_rows(int m, Stencil sa, Stencil sk, Stencil sm, int32_t* rowptr,
                                   int32_t* col, double* aval, double* kval, double* mval) {
  const int64_t N = (int64_t)m * m * m;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r > N) return;
  rowptr[r] = (int32_t)(16 * r);
  if (r == N) return;
  const uint32_t r32 = (uint32_t)r, um = (uint32_t)m, q1 = r32 / um;
  const int i = (int)(r32 - q1 * um), j = (int)(q1 % um), k = (int)(q1 / um);
  const int64_t o = 16 * r;
  if (i > 0 && j > 0 && k > 0 && i < m - 1 && j < m - 1 && k < m - 1) {
    // the slot tables above, as compile-time constants
    constexpr int off[15][3] = {{-1, -1, -1}, {0, -1, -1}, {-1, 0, -1}, {0, 0, -1}, {-1, -1, 0},
                                {0, -1, 0},   {-1, 0, 0},  {0, 0, 0},   {1, 0, 0},  {0, 1, 0},
                                {1, 1, 0},    {0, 0, 1},   {1, 0, 1},   {0, 1, 1},  {1, 1, 1}};
    constexpr int type[15] = {3, 2, 2, 1, 2, 1, 1, 0, 1, 1, 2, 1, 2, 2, 3};
    int32_t cl[16];
    double av[16], kv[16], mv[16];
#pragma unroll
    for (int s = 0; s < 15; s++) {
      cl[s] = (int32_t)(r + off[s][0] + (int64_t)m * (off[s][1] + (int64_t)m * off[s][2]));
      av[s] = type[s] == 0 ? sa.c0 : type[s] == 1 ? sa.ca : type[s] == 2 ? sa.cf : sa.cb;
      kv[s] = type[s] == 0 ? sk.c0 : type[s] == 1 ? sk.ca : type[s] == 2 ? sk.cf : sk.cb;
      mv[s] = type[s] == 0 ? sm.c0 : type[s] == 1 ? sm.ca : type[s] == 2 ? sm.cf : sm.cb;
    }
    cl[15] = -1;
    av[15] = kv[15] = mv[15] = 0.0;
    int4* c4 = reinterpret_cast<int4*>(col + o);
#pragma unroll
    for (int q = 0; q < 4; q++) c4[q] = make_int4(cl[4 * q], cl[4 * q + 1], cl[4 * q + 2], cl[4 * q + 3]);
    double2* a2 = reinterpret_cast<double2*>(aval + o);
#pragma unroll
    for (int q = 0; q < 8; q++) a2[q] = make_double2(av[2 * q], av[2 * q + 1]);
    if (kval) {
      double2* k2 = reinterpret_cast<double2*>(kval + o);
      double2* m2 = reinterpret_cast<double2*>(mval + o);
#pragma unroll
      for (int q = 0; q < 8; q++) {
        k2[q] = make_double2(kv[2 * q], kv[2 * q + 1]);
        m2[q] = make_double2(mv[2 * q], mv[2 * q + 1]);
      }
    }
    return;
  }
  const double at[4] = {sa.c0, sa.ca, sa.cf, sa.cb}, kt[4] = {sk.c0, sk.ca, sk.cf, sk.cb},
               mt[4] = {sm.c0, sm.ca, sm.cf, sm.cb};
  int cnt = 0;
  for (int s = 0; s < 15; s++) {
    const int ii = i + kSlotOff[s][0], jj = j + kSlotOff[s][1], kk = k + kSlotOff[s][2];
    if (ii < 0 || jj < 0 || kk < 0 || ii >= m || jj >= m || kk >= m) continue;
    const int t = kSlotType[s];
    col[o + cnt] = (int32_t)(ii + (int64_t)m * (jj + (int64_t)m * kk));
    aval[o + cnt] = at[t];
    if (kval) {
      kval[o + cnt] = kt[t];
      mval[o + cnt] = mt[t];
    }
    cnt++;
  }
  for (int p = cnt; p < 16; p++) {
    col[o + p] = -1;
    aval[o + p] = 0.0;
    if (kval) {
      kval[o + p] = 0.0;
      mval[o + p] = 0.0;
    }
  }
}

// CSR4 rows on a general (jittered) vertex grid with Kuhn connectivity.
__global__ void k_csr_general(int n, const double* xyz, double rho, int32_t* rowptr,
                              int32_t* col, double* aval, double* kval, double* mval) {
  const int m = n - 1;
  int64_t N = (int64_t)m * m * m;
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r > N) return;
  rowptr[r] = (int32_t)(16 * r);
  if (r == N) return;
  int i = (int)(r % m), j = (int)((r / m) % m), k = (int)(r / ((int64_t)m * m));
  Coords C{xyz, n, 1.0 / n};
  double kv[15], mv[15];
  vertex_row(C, i + 1, j + 1, k + 1, kv, mv);
  int64_t e = 16 * r;
  int cnt = 0;
  for (int s = 0; s < 15; s++) {
    int ii = i + kSlotOff[s][0], jj = j + kSlotOff[s][1], kk = k + kSlotOff[s][2];
    if (ii < 0 || jj < 0 || kk < 0 || ii >= m || jj >= m || kk >= m) continue;
    col[e + cnt] = (int32_t)(ii + (int64_t)m * (jj + (int64_t)m * kk));
    aval[e + cnt] = rho * kv[s] + mv[s];
    if (kval) kval[e + cnt] = kv[s];
    if (mval) mval[e + cnt] = mv[s];
    cnt++;
  }
  for (; cnt < 16; cnt++) {
    col[e + cnt] = -1;
    aval[e + cnt] = 0.0;
    if (kval) kval[e + cnt] = 0.0;
    if (mval) mval[e + cnt] = 0.0;
  }
}

// ------------------------------------------------------------------ load vector

struct TargetDev {
  int kind;
  int nb;
  const double* c;  // nb*3
  const double* w;
  const double* a;
  double lo, hi;
  const double* qv = nullptr;  // FEM_TARGET_QUADVALS: [tet][4] values at the load's points
};

__device__ double target_eval(const TargetDev& T, double x, double y, double z) {
  switch (T.kind) {
    case FEM_TARGET_SINE:
      return sinpi(x) * sinpi(y) * sinpi(z);
    case FEM_TARGET_SINE_PLUS_ONE:
      return 1.0 + sinpi(x) * sinpi(y) * sinpi(z);
    case FEM_TARGET_BOX:
      return (x > T.lo && x < T.hi && y > T.lo && y < T.hi && z > T.lo && z < T.hi) ? 1.0 : 0.0;
    case FEM_TARGET_BUMPS: {
      double s = 0.0;
      for (int b = 0; b < T.nb; b++) {
        double dx = x - T.c[3 * b], dy = y - T.c[3 * b + 1], dz = z - T.c[3 * b + 2];
        double r2 = dx * dx + dy * dy + dz * dz;
        s += T.a[b] * exp(-r2 / (2.0 * T.w[b] * T.w[b]));
      }
      return s;
    }
  }
  return 0.0;
}

// On the uniform grid every target here is a sum of separable terms
//   ubar(x) = sum_t alpha_t g_t0(x) g_t1(y) g_t2(z),
// and a quadrature point of the 4-point rule in a Kuhn tet sits at h*(c_d + o) along each
// axis with o one of 6 offsets; tab[(t*3 + d)*n*6 + c*6 + o] = g_td(h*(c + o)).
__device__ __forceinline__ double qoff(int o) {
  const double A = (5.0 + 3.0 * sqrt(5.0)) / 20.0, B = (5.0 - sqrt(5.0)) / 20.0;
  switch (o) {
    case 0: return B;
    case 1: return A;
    case 2: return 2.0 * B;
    case 3: return A + B;
    case 4: return 3.0 * B;
    default: return A + 2.0 * B;
  }
}

__global__ void k_target_tables(TargetDev T, int n, int nterms, double* tab, double* alpha) {
  int idx = blockIdx.x * blockDim.x + threadIdx.x;
  int total = nterms * 3 * n * 6;
  if (idx < nterms) {
    if (T.kind == FEM_TARGET_BUMPS) alpha[idx] = T.a[idx];
    else alpha[idx] = 1.0;
  }
  if (idx >= total) return;
  int o = idx % 6, c = (idx / 6) % n, d = (idx / (6 * n)) % 3, t = idx / (18 * n);
  double x = (c + qoff(o)) / n;
  double v = 1.0;
  switch (T.kind) {
    case FEM_TARGET_SINE: v = sinpi(x); break;
    case FEM_TARGET_SINE_PLUS_ONE: v = (t == 0) ? 1.0 : sinpi(x); break;
    case FEM_TARGET_BOX: v = (x > T.lo && x < T.hi) ? 1.0 : 0.0; break;
    case FEM_TARGET_BUMPS: {
      double dx = x - T.c[3 * t + d], w = T.w[t];
      v = exp(-dx * dx / (2.0 * w * w));
    } break;
  }
  tab[idx] = v;
}

// Per-cube load contributions: cube c gets cf[c*8 + local vertex] with local vertex
// dx + 2 dy + 4 dz, summing w_q |tau| ubar(x_q) lambda_a(x_q) over its 6 tets and the
// 4 points of each (Hammer-Stroud, barycentric (A,B,B,B) permutations, weight 1/4).
// Loops over tets and points are unrolled so that every local index is static.  Used for
// jittered meshes and for targets given at the quadrature points (xyz null: the uniform
// grid).
__global__ void k_cube_load(int n, const double* xyz, TargetDev T, double* cf) {
  constexpr int PP[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  int64_t nc = (int64_t)n * n * n;
  int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= nc) return;
  const int ci = (int)(c % n), cj = (int)((c / n) % n), ck = (int)(c / ((int64_t)n * n));
  const double A = (5.0 + 3.0 * sqrt(5.0)) / 20.0, B = (5.0 - sqrt(5.0)) / 20.0;
  double acc[8];
#pragma unroll
  for (int a = 0; a < 8; a++) acc[a] = 0.0;
  double Xc[8][3];
  Coords C{xyz, n, 1.0 / n};
#pragma unroll
  for (int a = 0; a < 8; a++) C.get(ci + (a & 1), cj + ((a >> 1) & 1), ck + ((a >> 2) & 1), Xc[a]);
#pragma unroll
  for (int p = 0; p < 6; p++) {
    int lv[4];
    lv[0] = 0;
#pragma unroll
    for (int s = 0; s < 3; s++) lv[s + 1] = lv[s] | (1 << PP[p][s]);
    double X[4][3], g[4][3];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
      for (int d = 0; d < 3; d++) X[a][d] = Xc[lv[a]][d];
    const double vol = fabs(tet_grads(X, g)) / 6.0;
    double uq[4];
#pragma unroll
    for (int q = 0; q < 4; q++) {
      double mu[4] = {B, B, B, B};
      mu[q] = A;
      double x[3] = {0, 0, 0};
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int d = 0; d < 3; d++) x[d] += mu[a] * Xc[lv[a]][d];
      uq[q] = T.kind == FEM_TARGET_QUADVALS ? T.qv[4 * (6 * c + p) + q]
                                            : target_eval(T, x[0], x[1], x[2]);
    }
    // sum_q (|tau|/4) u_q lambda_a(x_q) with lambda_a(x_q) = B + (A - B) [q == a]
    const double S = (uq[0] + uq[1]) + (uq[2] + uq[3]);
    const double w = 0.25 * vol;
#pragma unroll
    for (int a = 0; a < 4; a++) acc[lv[a]] += w * (B * S + (A - B) * uq[a]);
  }
#pragma unroll
  for (int a = 0; a < 8; a++) cf[8 * c + a] = acc[a];
}

// Uniform grid, separable target: the load of node (I, J, K) collects, over the 6 tets of
// each of its 8 cubes that contain it and the 4 points of each, 96 terms
//   (|tau| / 4) lambda_a(x_q) ubar(x_q),   lambda_a(x_q) = B + (A - B) [q == a],
// and every point sits, along axis d, at table row i_d - dd_d (dd the node's corner of the
// cube) and one of the 6 offsets: its class along d is e_d = 6 dd_d + o_d, 12 classes per
// axis.  With ubar = sum_t alpha_t g_t0 g_t1 g_t2 the load is
//   f = scale sum_t sum_e0 g_t0(I, e0) T_t(e0),  T_t(e0) = alpha_t sum_{terms with e0} coef g_t1 g_t2,
// and T depends on the row (J, K) only: one block per row of nodes computes it (in the
// terms' fixed order: deterministic), then each node costs 12 products per target term.
// Term k = 16 p + 4 a + q: tet p of the cube whose corner dd = lv_p(a) is the node, point q.
__device__ __forceinline__ void load_term(int k, int e[3], bool& at_a) {
  const int p = k >> 4, a = (k >> 2) & 3, q = k & 3;
  // tet p walks from the cube's corner 0 to corner 7 along axes f0, f1, f2: the six
  // orders (0,1,2) (0,2,1) (1,0,2) (1,2,0) (2,0,1) (2,1,0)
  const int f0 = p >> 1, lo = f0 == 0 ? 1 : 0, hi = f0 == 2 ? 1 : 2;
  const int f1 = (p & 1) ? hi : lo, f2 = (p & 1) ? lo : hi;
  const int dd = (a >= 1 ? 1 << f0 : 0) | (a >= 2 ? 1 << f1 : 0) | (a >= 3 ? 1 << f2 : 0);
  const int o0 = q == 0 ? 4 : 5, o1 = q >= 2 ? 3 : 2, o2 = q == 3 ? 1 : 0;
#pragma unroll
  for (int d = 0; d < 3; d++) e[d] = 6 * ((dd >> d) & 1) + (d == f0 ? o0 : d == f1 ? o1 : o2);
  at_a = (q == a);
}

// table value of term t along axis d for node coordinate i (1..n-1) and class e
__device__ __forceinline__ double tab_at(const double* tab, int n, int t, int d, int i, int e) {
  return __ldg(tab + ((t * 3 + d) * n + (i - e / 6)) * 6 + e % 6);
}

__global__ void __launch_bounds__(128) k_load_sep(int n, const double* __restrict__ tab,
                                                  const double* __restrict__ alpha, int nterms,
                                                  double* __restrict__ f) {
  extern __shared__ double Tt[];   // [nterms][12]
  const int m = n - 1;
  const int J = blockIdx.x + 1, K = blockIdx.y + 1;
  const double A = (5.0 + 3.0 * sqrt(5.0)) / 20.0, B = (5.0 - sqrt(5.0)) / 20.0;
  for (int te = threadIdx.x; te < nterms * 12; te += blockDim.x) {
    const int t = te / 12, e0 = te % 12;
    double s = 0.0;
    for (int k = 0; k < 96; k++) {
      int e[3];
      bool at_a;
      load_term(k, e, at_a);
      if (e[0] != e0) continue;
      s += (at_a ? A : B) * (tab_at(tab, n, t, 1, J, e[1]) * tab_at(tab, n, t, 2, K, e[2]));
    }
    Tt[te] = alpha[t] * s;
  }
  __syncthreads();
  const double h = 1.0 / n;
  const double scale = 0.25 * (h * h * h / 6.0);
  double* frow = f + (int64_t)m * ((J - 1) + (int64_t)m * (K - 1));
  for (int I = threadIdx.x + 1; I <= m; I += blockDim.x) {
    double s = 0.0;
    for (int t = 0; t < nterms; t++) {
      const double* x = tab + ((t * 3) * n + (I - 1)) * 6;   // classes 6..11 (cube I-1), 0..5 (cube I)
#pragma unroll
      for (int e0 = 0; e0 < 12; e0++) s = fma(__ldg(x + (e0 < 6 ? 6 + e0 : e0 - 6)), Tt[t * 12 + e0], s);
    }
    frow[I - 1] = scale * s;
  }
}

__global__ void k_gather_load(int n, const double* cf, double* f) {
  const int m = n - 1;
  int64_t N = (int64_t)m * m * m;
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  const uint32_t r32 = (uint32_t)r, um = (uint32_t)m, q1 = r32 / um;
  const int i = (int)(r32 - q1 * um) + 1, j = (int)(q1 % um) + 1, k = (int)(q1 / um) + 1;
  double s = 0.0;
  for (int dd = 7; dd >= 0; dd--) {
    int ci = i - (dd & 1), cj = j - ((dd >> 1) & 1), ck = k - ((dd >> 2) & 1);
    int64_t c = ci + (int64_t)n * (cj + (int64_t)n * ck);
    s += cf[8 * c + dd];
  }
  f[r] = s;
}

__global__ void k_fill_value(int64_t N, double value, double* out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < N) out[r] = value;
}

__global__ void k_diag_inv(int64_t N, const int32_t* rowptr, const int32_t* col, const double* v,
                           double* dinv) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  double d = 0.0;
  for (int e = rowptr[r]; e < rowptr[r + 1]; e++)
    if (col[e] == r) d = v[e];
  dinv[r] = 1.0 / d;
}

// f_i = sum over tets of the 4-point rule applied to ubar phi_i (per-cube partial sums,
// then a gather over the 8 cubes around each vertex in a fixed order).
void load_vector(System& S, const TargetDev& T, const fem_target& t, double* f, cudaStream_t st) {
  const int n = S.n;
  const int64_t N = S.N;
  if (N == 0) return;
  if (S.uniform && t.kind != FEM_TARGET_QUADVALS) {
    int nterms = (t.kind == FEM_TARGET_BUMPS) ? t.nb : (t.kind == FEM_TARGET_SINE_PLUS_ONE ? 2 : 1);
    DevBuf<double> tab((size_t)nterms * 3 * n * 6, st), alpha(nterms, st);
    int total = nterms * 3 * n * 6;
    k_target_tables<<<grid_for(total, 256), 256, 0, st>>>(T, n, nterms, tab, alpha);
    FEM_CHECK_LAUNCH();
    k_load_sep<<<dim3(n - 1, n - 1), 128, (size_t)nterms * 12 * 8, st>>>(n, tab, alpha, nterms, f);
    FEM_CHECK_LAUNCH();
    return;
  }
  int64_t ncube = (int64_t)n * n * n;
  DevBuf<double> cf(8 * ncube, st);
  k_cube_load<<<grid_for(ncube, 128), 128, 0, st>>>(n, S.uniform ? nullptr : S.xyz.p, T, cf);
  FEM_CHECK_LAUNCH();
  k_gather_load<<<grid_for(N, 256), 256, 0, st>>>(n, cf, f);
  FEM_CHECK_LAUNCH();
}

struct TargetHolder {
  DevBuf<double> tc, tw, ta;
  TargetDev T;
};

void target_to_device(const fem_target& t, TargetHolder& h, cudaStream_t st) {
  FEM_REQUIRE(t.kind >= 0 && t.kind <= 4, FEM_EINVAL, "unknown target kind");
  FEM_REQUIRE(t.kind != FEM_TARGET_QUADVALS || t.quadvals_dev, FEM_EINVAL,
              "point-value target without values");
  FEM_REQUIRE(t.kind != FEM_TARGET_BUMPS || (t.nb >= 1 && t.nb <= 64 && t.centers_host &&
                                             t.widths_host && t.amps_host),
              FEM_EINVAL, "bumps need 1..64 centres/widths/amplitudes");
  h.T = TargetDev{t.kind, 0, nullptr, nullptr, nullptr, t.lo, t.hi, t.quadvals_dev};
  if (t.kind == FEM_TARGET_BUMPS) {
    h.tc.alloc_async(3 * t.nb, st);
    h.tw.alloc_async(t.nb, st);
    h.ta.alloc_async(t.nb, st);
    FEM_CUDA(cudaMemcpyAsync(h.tc, t.centers_host, 24 * t.nb, cudaMemcpyHostToDevice, st));
    FEM_CUDA(cudaMemcpyAsync(h.tw, t.widths_host, 8 * t.nb, cudaMemcpyHostToDevice, st));
    FEM_CUDA(cudaMemcpyAsync(h.ta, t.amps_host, 8 * t.nb, cudaMemcpyHostToDevice, st));
    h.T.nb = t.nb;
    h.T.c = h.tc;
    h.T.w = h.tw;
    h.T.a = h.ta;
  }
}

// ------------------------------------------------------------------ post-processing

// Quadrature for the error norms: the 4-point Hammer-Stroud rule applied on each of the
// 8^level children of `level` rounds of Bey's red refinement of the tet, as barycentric
// points of the parent with weights summing to 1.
void bey_rule(const double P[4][4], int level, double w, std::vector<double>& bary,
              std::vector<double>& wt) {
  if (level == 0) {
    const double A = (5.0 + 3.0 * std::sqrt(5.0)) / 20.0, B = (5.0 - std::sqrt(5.0)) / 20.0;
    for (int q = 0; q < 4; q++)
      for (int d = 0; d < 4; d++) {
        double s = 0.0;
        for (int v = 0; v < 4; v++) s += (v == q ? A : B) * P[v][d];
        bary.push_back(s);
        if (d == 3) wt.push_back(0.25 * w);
      }
    return;
  }
  // edge midpoints mid(a, b); the 4 corner children and the 4 children of the inner
  // octahedron split along the diagonal between the midpoints of edges 02 and 13
  static const int kid[8][4][2] = {{{0, 0}, {0, 1}, {0, 2}, {0, 3}}, {{0, 1}, {1, 1}, {1, 2}, {1, 3}},
                                   {{0, 2}, {1, 2}, {2, 2}, {2, 3}}, {{0, 3}, {1, 3}, {2, 3}, {3, 3}},
                                   {{0, 1}, {0, 2}, {0, 3}, {1, 3}}, {{0, 1}, {0, 2}, {1, 2}, {1, 3}},
                                   {{0, 2}, {0, 3}, {1, 3}, {2, 3}}, {{0, 2}, {1, 2}, {1, 3}, {2, 3}}};
  for (int c = 0; c < 8; c++) {
    double Q[4][4];
    for (int v = 0; v < 4; v++)
      for (int d = 0; d < 4; d++) Q[v][d] = 0.5 * (P[kid[c][v][0]][d] + P[kid[c][v][1]][d]);
    bey_rule(Q, level - 1, w / 8.0, bary, wt);
  }
}

// w = scale * target and its gradient (sine targets only)
__device__ __forceinline__ void target_grad(const TargetDev& T, double scale, double x, double y,
                                            double z, double g[3]) {
  double s0, c0, s1, c1, s2, c2;
  sincospi(x, &s0, &c0);
  sincospi(y, &s1, &c1);
  sincospi(z, &s2, &c2);
  const double f = scale * 3.14159265358979323846;
  g[0] = f * c0 * s1 * s2;
  g[1] = f * s0 * c1 * s2;
  g[2] = f * s0 * s1 * c2;
}

// ||w - u_h||^2 and ||grad(w - u_h)||^2 over the tets of one cube per thread (grid-stride,
// fixed grid): u_h is the P1 function with nodal values u on interior vertices and 0 on the
// boundary.  Per-block partial sums in partials[block], partials[nb + block].
__global__ void k_errors(int n, const double* xyz, const double* __restrict__ u, TargetDev T,
                         double scale, int grad, const double* __restrict__ qb,
                         const double* __restrict__ qw, int np, double* partials) {
  constexpr int PP[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  const int64_t nc = (int64_t)n * n * n;
  const int m = n - 1;
  Coords C{xyz, n, 1.0 / n};
  double acc[2] = {0.0, 0.0};
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int ci = (int)(c % n), cj = (int)((c / n) % n), ck = (int)(c / ((int64_t)n * n));
    double Xc[8][3], Uc[8];
#pragma unroll
    for (int a = 0; a < 8; a++) {
      const int vi = ci + (a & 1), vj = cj + ((a >> 1) & 1), vk = ck + ((a >> 2) & 1);
      C.get(vi, vj, vk, Xc[a]);
      const bool in = vi >= 1 && vj >= 1 && vk >= 1 && vi <= m && vj <= m && vk <= m;
      Uc[a] = in ? u[(int64_t)(vi - 1) + (int64_t)m * ((vj - 1) + (int64_t)m * (vk - 1))] : 0.0;
    }
#pragma unroll
    for (int p = 0; p < 6; p++) {
      int lv[4];
      lv[0] = 0;
#pragma unroll
      for (int s2 = 0; s2 < 3; s2++) lv[s2 + 1] = lv[s2] | (1 << PP[p][s2]);
      double X[4][3], g[4][3], U[4];
#pragma unroll
      for (int a = 0; a < 4; a++) {
        U[a] = Uc[lv[a]];
#pragma unroll
        for (int d = 0; d < 3; d++) X[a][d] = Xc[lv[a]][d];
      }
      const double vol = fabs(tet_grads(X, g)) / 6.0;
      double guh[3] = {0.0, 0.0, 0.0};
#pragma unroll
      for (int a = 0; a < 4; a++)
#pragma unroll
        for (int d = 0; d < 3; d++) guh[d] += U[a] * g[a][d];
      double e2 = 0.0, g2 = 0.0;
      for (int q = 0; q < np; q++) {
        double x[3] = {0.0, 0.0, 0.0}, uh = 0.0;
#pragma unroll
        for (int a = 0; a < 4; a++) {
          const double b = qb[4 * q + a];
#pragma unroll
          for (int d = 0; d < 3; d++) x[d] += b * X[a][d];
          uh += b * U[a];
        }
        const double diff = scale * target_eval(T, x[0], x[1], x[2]) - uh;
        e2 += qw[q] * diff * diff;
        if (grad) {
          double ge[3];
          target_grad(T, scale, x[0], x[1], x[2], ge);
          const double d0 = ge[0] - guh[0], d1 = ge[1] - guh[1], d2 = ge[2] - guh[2];
          g2 += qw[q] * (d0 * d0 + d1 * d1 + d2 * d2);
        }
      }
      acc[0] += vol * e2;
      acc[1] += vol * g2;
    }
  }
  block_sum<2>(acc);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = acc[0];
    partials[gridDim.x + blockIdx.x] = acc[1];
  }
}

// The same norms on the uniform grid for the sine targets (ubar = sin sin sin, or 1 + it),
// whose values factor by axis: a quadrature point (p, q) of Kuhn tet p in cube (i, j, k)
// sits at h (i + xi_pq, j + eta_pq, k + zeta_pq), so sin(pi x) = Sx[pq][i] with
// Sx[pq][i] = sin(pi h (i + xi_pq)) from a table (and cos for the gradient), instead of
// three FP64 sine evaluations per point.  Each Kuhn tet has volume h^3 / 6 and fixed
// barycentric gradients gref[p] / h.
__global__ void k_err_tables(int n, int npq, const double* __restrict__ xi, double* tabs,
                             double* tabc) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t per = (int64_t)npq * n;
  if (t >= 3 * per) return;
  const int d = (int)(t / per), pq = (int)((t % per) / n), i = (int)(t % n);
  double sv, cv;
  sincospi((i + xi[3 * pq + d]) / n, &sv, &cv);
  tabs[t] = sv;
  if (tabc) tabc[t] = cv;
}

__global__ void k_errors_sep(int n, const double* __restrict__ u, double scale, double add,
                             int grad, int np, const double* __restrict__ tabs,
                             const double* __restrict__ tabc, const double* __restrict__ bary,
                             const double* __restrict__ qw, const double* __restrict__ gref,
                             double* partials) {
  constexpr int PP[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  const int64_t nc = (int64_t)n * n * n;
  const int m = n - 1;
  const int npq = 6 * np;
  const int64_t per = (int64_t)npq * n;
  const double vol = 1.0 / (6.0 * (double)n * n * n), hinv = (double)n;
  const double spi = scale * 3.14159265358979323846;
  double acc[2] = {0.0, 0.0};
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nc;
       c += (int64_t)gridDim.x * blockDim.x) {
    const int ci = (int)(c % n), cj = (int)((c / n) % n), ck = (int)(c / ((int64_t)n * n));
    double Uc[8];
#pragma unroll
    for (int a = 0; a < 8; a++) {
      const int vi = ci + (a & 1), vj = cj + ((a >> 1) & 1), vk = ck + ((a >> 2) & 1);
      const bool in = vi >= 1 && vj >= 1 && vk >= 1 && vi <= m && vj <= m && vk <= m;
      Uc[a] = in ? u[(int64_t)(vi - 1) + (int64_t)m * ((vj - 1) + (int64_t)m * (vk - 1))] : 0.0;
    }
    const double* sx = tabs + ci;
    const double* sy = tabs + per + cj;
    const double* sz = tabs + 2 * per + ck;
    const double* cx = tabc + ci;
    const double* cy = tabc + per + cj;
    const double* cz = tabc + 2 * per + ck;
#pragma unroll
    for (int p = 0; p < 6; p++) {
      int lv[4];
      lv[0] = 0;
#pragma unroll
      for (int s2 = 0; s2 < 3; s2++) lv[s2 + 1] = lv[s2] | (1 << PP[p][s2]);
      double U[4];
#pragma unroll
      for (int a = 0; a < 4; a++) U[a] = Uc[lv[a]];
      double guh[3] = {0.0, 0.0, 0.0};
      if (grad) {
#pragma unroll
        for (int a = 0; a < 4; a++)
#pragma unroll
          for (int d = 0; d < 3; d++) guh[d] += U[a] * (gref[(p * 4 + a) * 3 + d] * hinv);
      }
      double e2 = 0.0, g2 = 0.0;
      for (int q = 0; q < np; q++) {
        const int64_t o = (int64_t)(p * np + q) * n;
        const double* b = bary + 4 * (p * np + q);
        const double uh = b[0] * U[0] + b[1] * U[1] + b[2] * U[2] + b[3] * U[3];
        const double vx = sx[o], vy = sy[o], vz = sz[o];
        const double diff = scale * (add + vx * vy * vz) - uh;
        e2 += qw[q] * diff * diff;
        if (grad) {
          const double d0 = spi * cx[o] * vy * vz - guh[0];
          const double d1 = spi * vx * cy[o] * vz - guh[1];
          const double d2 = spi * vx * vy * cz[o] - guh[2];
          g2 += qw[q] * (d0 * d0 + d1 * d1 + d2 * d2);
        }
      }
      acc[0] += vol * e2;
      acc[1] += vol * g2;
    }
  }
  block_sum<2>(acc);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = acc[0];
    partials[gridDim.x + blockIdx.x] = acc[1];
  }
}

// Control and adjoint at the unknowns' vertices: z = (ubar - u) / rho, p = -rho u.
__global__ void k_recover(int n, const double* xyz, TargetDev T, double rho,
                          const double* __restrict__ u, double* z, double* p) {
  const int m = n - 1;
  const int64_t N = (int64_t)m * m * m;
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  const int i = (int)(r % m) + 1, j = (int)((r / m) % m) + 1, k = (int)(r / ((int64_t)m * m)) + 1;
  Coords C{xyz, n, 1.0 / n};
  double x[3];
  C.get(i, j, k, x);
  const double ur = u[r];
  if (z) z[r] = (target_eval(T, x[0], x[1], x[2]) - ur) / rho;
  if (p) p[r] = -rho * ur;
}

// ------------------------------------------------------------------ general meshes

// Rows are built vertex by vertex from the vertex's incident tets, visited in increasing
// tet order: the unknowns of those tets (sorted, unique) are the row's columns, and the
// element contributions are added in that order.
constexpr int kGmMaxInc = 64;    // tets per vertex
constexpr int kGmMaxRow = 128;   // distinct unknowns per row

__global__ void k_gm_dof(int64_t nv, const uint8_t* dir, const int64_t* scan, int32_t* vdof,
                         int64_t* rvert) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  if (dir[v]) {
    vdof[v] = -1;
  } else {
    vdof[v] = (int32_t)scan[v];
    rvert[scan[v]] = v;
  }
}

__global__ void k_gm_free_flags(int64_t nv, const uint8_t* dir, int64_t* flag) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v < nv) flag[v] = dir[v] ? 0 : 1;
}

__global__ void k_gm_inc_count(int64_t nt, const int32_t* tet, int64_t nv, int64_t* cnt,
                               unsigned long long* bad) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  for (int a = 0; a < 4; a++) {
    const int32_t v = tet[4 * t + a];
    if (v < 0 || v >= nv) {
      atomicAdd(bad, 1ull);
      continue;
    }
    atomicAdd(reinterpret_cast<unsigned long long*>(cnt) + v, 1ull);
  }
}

__global__ void k_gm_inc_fill(int64_t nt, const int32_t* tet, const int64_t* vptr,
                              unsigned long long* cursor, int32_t* vtet) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  for (int a = 0; a < 4; a++) {
    const int32_t v = tet[4 * t + a];
    vtet[vptr[v] + (int64_t)atomicAdd(cursor + v, 1ull)] = (int32_t)t;
  }
}

// every tet must have a nonzero volume
__global__ void k_gm_tet_check(int64_t nt, const int32_t* tet, const double* xyz,
                               unsigned long long* bad) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double X[4][3], g[4][3];
  for (int a = 0; a < 4; a++)
    for (int d = 0; d < 3; d++) X[a][d] = xyz[3 * (int64_t)tet[4 * t + a] + d];
  const double det = tet_grads(X, g);
  if (!(det != 0.0) || !isfinite(det)) atomicAdd(bad, 1ull);
}

// incident tets of each vertex in increasing order (lists are short: insertion sort)
__global__ void k_gm_inc_sort(int64_t nv, const int64_t* vptr, int32_t* vtet,
                              unsigned long long* over) {
  const int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (v >= nv) return;
  const int64_t a = vptr[v], b = vptr[v + 1];
  if (b - a > kGmMaxInc) atomicAdd(over, 1ull);
  for (int64_t i = a + 1; i < b; i++) {
    const int32_t x = vtet[i];
    int64_t j = i - 1;
    while (j >= a && vtet[j] > x) {
      vtet[j + 1] = vtet[j];
      j--;
    }
    vtet[j + 1] = x;
  }
}

// sorted unique unknowns of the tets around vertex v; -1 when the row is too long
__device__ int gm_row_cols(int64_t v, const int64_t* vptr, const int32_t* vtet,
                           const int32_t* tet, const int32_t* vdof, int32_t* buf) {
  int cnt = 0;
  for (int64_t e = vptr[v]; e < vptr[v + 1]; e++) {
    const int64_t t = vtet[e];
    for (int a = 0; a < 4; a++) {
      const int32_t w = vdof[tet[4 * t + a]];
      if (w < 0) continue;
      int q = 0;
      while (q < cnt && buf[q] < w) q++;
      if (q < cnt && buf[q] == w) continue;
      if (cnt == kGmMaxRow) return -1;
      for (int z = cnt; z > q; z--) buf[z] = buf[z - 1];
      buf[q] = w;
      cnt++;
    }
  }
  return cnt;
}

__global__ void k_gm_row_count(int64_t N, const int64_t* rvert, const int64_t* vptr,
                               const int32_t* vtet, const int32_t* tet, const int32_t* vdof,
                               int64_t* cnt, unsigned long long* over) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  int32_t buf[kGmMaxRow];
  const int c = gm_row_cols(rvert[r], vptr, vtet, tet, vdof, buf);
  if (c < 0) {
    atomicAdd(over, 1ull);
    cnt[r] = 0;
    return;
  }
  cnt[r] = c;
}

// Element quantities, once per tet: |tau| (in vol), the stiffness entries
// |tau| grad(lambda_a).grad(lambda_b) for a <= b (ke, 10 per tet, index kGmPair[a][b]) and
// the load integrals sum_q w_q ubar(x_q) lambda_a(x_q) (fe, 4 per tet, without |tau|),
// with ubar evaluated once per point.  ke null: only vol and fe.
__constant__ int8_t kGmPair[4][4] = {{0, 1, 2, 3}, {1, 4, 5, 6}, {2, 5, 7, 8}, {3, 6, 8, 9}};

__global__ void k_gm_elements(int64_t nt, const int32_t* __restrict__ tet,
                              const double* __restrict__ xyz, TargetDev T,
                              const double* __restrict__ qb, const double* __restrict__ qw,
                              int np, double* vol, double* ke, double* fe,
                              unsigned long long* bad) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  double X[4][3], g[4][3];
  for (int a = 0; a < 4; a++) {
    const int32_t v = tet[4 * t + a];
    for (int d = 0; d < 3; d++) X[a][d] = xyz[3 * (int64_t)v + d];
  }
  const double det = tet_grads(X, g);
  if (!(det != 0.0)) atomicAdd(bad, 1ull);
  const double V = fabs(det) / 6.0;
  vol[t] = V;
  if (ke)
    for (int a = 0; a < 4; a++)
      for (int b = a; b < 4; b++)
        ke[10 * t + kGmPair[a][b]] = V * (g[a][0] * g[b][0] + g[a][1] * g[b][1] + g[a][2] * g[b][2]);
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int q = 0; q < np; q++) {
    double x[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 4; a++)
      for (int d = 0; d < 3; d++) x[d] += qb[4 * q + a] * X[a][d];
    const double u = T.kind == FEM_TARGET_QUADVALS ? T.qv[4 * t + q]
                                                   : target_eval(T, x[0], x[1], x[2]);
    for (int a = 0; a < 4; a++) acc[a] += qw[q] * u * qb[4 * q + a];
  }
  for (int a = 0; a < 4; a++) fe[4 * t + a] = acc[a];
}

// One row: columns, K, M, A = rho K + M and f from the element quantities, summed over the
// row's tets in increasing tet order.  With Aval null only f is written.
__global__ void k_gm_row_fill(int64_t N, const int64_t* rvert, const int64_t* vptr,
                              const int32_t* vtet, const int32_t* tet, const int32_t* vdof,
                              double rho, const double* __restrict__ vol,
                              const double* __restrict__ ke, const double* __restrict__ fe,
                              const int32_t* rowptr, int32_t* col, double* Aval, double* Kv,
                              double* Mv, double* f) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  const int64_t v = rvert[r];
  int32_t cols[kGmMaxRow];
  double kacc[kGmMaxRow], macc[kGmMaxRow];
  int nc = 0;
  if (Aval) {
    nc = gm_row_cols(v, vptr, vtet, tet, vdof, cols);
    if (nc < 0) return;
    for (int q = 0; q < nc; q++) kacc[q] = macc[q] = 0.0;
  }
  double fr = 0.0;
  for (int64_t e = vptr[v]; e < vptr[v + 1]; e++) {
    const int64_t t = vtet[e];
    const int4 tv4 = reinterpret_cast<const int4*>(tet)[t];
    const int32_t tv[4] = {tv4.x, tv4.y, tv4.z, tv4.w};
    int loc = 0;
    for (int a = 0; a < 4; a++)
      if (tv[a] == v) loc = a;
    const double V = vol[t];
    if (Aval) {
      for (int b = 0; b < 4; b++) {
        const int32_t w = vdof[tv[b]];
        if (w < 0) continue;
        int lo = 0, hi = nc - 1;
        while (lo < hi) {
          const int mid = (lo + hi) / 2;
          if (cols[mid] < w) lo = mid + 1; else hi = mid;
        }
        kacc[lo] += ke[10 * t + kGmPair[loc][b]];
        macc[lo] += V * (loc == b ? 2.0 : 1.0) / 20.0;
      }
    }
    fr += V * fe[4 * t + loc];
  }
  f[r] = fr;
  if (!Aval) return;
  const int64_t o0 = rowptr[r], o1 = rowptr[r + 1];
  for (int q = 0; q < nc; q++) {
    col[o0 + q] = cols[q];
    Aval[o0 + q] = rho * kacc[q] + macc[q];
    if (Kv) {
      Kv[o0 + q] = kacc[q];
      Mv[o0 + q] = macc[q];
    }
  }
  for (int64_t o = o0 + nc; o < o1; o++) {
    col[o] = -1;
    Aval[o] = 0.0;
    if (Kv) {
      Kv[o] = 0.0;
      Mv[o] = 0.0;
    }
  }
}

// errors over the tets of a general mesh (thread per tet, grid-stride, fixed grid)
__global__ void k_gm_errors(int64_t nt, const int32_t* tet, const int32_t* vdof, const double* xyz,
                            const double* __restrict__ u, TargetDev T, double scale, int grad,
                            const double* __restrict__ qb, const double* __restrict__ qw, int np,
                            double* partials) {
  double acc[2] = {0.0, 0.0};
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt;
       t += (int64_t)gridDim.x * blockDim.x) {
    double X[4][3], g[4][3], U[4];
    for (int a = 0; a < 4; a++) {
      const int32_t v = tet[4 * t + a];
      const int32_t w = vdof[v];
      U[a] = w >= 0 ? u[w] : 0.0;
      for (int d = 0; d < 3; d++) X[a][d] = xyz[3 * (int64_t)v + d];
    }
    const double vol = fabs(tet_grads(X, g)) / 6.0;
    double guh[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 4; a++)
      for (int d = 0; d < 3; d++) guh[d] += U[a] * g[a][d];
    double e2 = 0.0, g2 = 0.0;
    for (int q = 0; q < np; q++) {
      double x[3] = {0.0, 0.0, 0.0}, uh = 0.0;
      for (int a = 0; a < 4; a++) {
        const double b = qb[4 * q + a];
        for (int d = 0; d < 3; d++) x[d] += b * X[a][d];
        uh += b * U[a];
      }
      const double diff = scale * target_eval(T, x[0], x[1], x[2]) - uh;
      e2 += qw[q] * diff * diff;
      if (grad) {
        double ge[3];
        target_grad(T, scale, x[0], x[1], x[2], ge);
        const double d0 = ge[0] - guh[0], d1 = ge[1] - guh[1], d2 = ge[2] - guh[2];
        g2 += qw[q] * (d0 * d0 + d1 * d1 + d2 * d2);
      }
    }
    acc[0] += vol * e2;
    acc[1] += vol * g2;
  }
  block_sum<2>(acc);
  if (threadIdx.x == 0) {
    partials[blockIdx.x] = acc[0];
    partials[gridDim.x + blockIdx.x] = acc[1];
  }
}

// The other tet of the face (b, c, d) of tet t: walks the tets around b (sorted, short) and
// keeps those holding c and d.  -1 on the boundary, -2 when more than one tet has the face.
__device__ __forceinline__ int64_t face_neighbour(int64_t t, int32_t b, int32_t c, int32_t d,
                                                  const int64_t* vptr, const int32_t* vtet,
                                                  const int32_t* tet) {
  int64_t found = -1;
  for (int64_t e = vptr[b]; e < vptr[b + 1]; e++) {
    const int32_t s = vtet[e];
    if (s == t) continue;
    const int4 v = reinterpret_cast<const int4*>(tet)[s];
    const bool hc = v.x == c || v.y == c || v.z == c || v.w == c;
    const bool hd = v.x == d || v.y == d || v.z == d || v.w == d;
    if (hc && hd) {
      if (found >= 0) return -2;
      found = s;
    }
  }
  return found;
}

__device__ __forceinline__ double len2_rn(const double* a, const double* b) {
  const double dx = b[0] - a[0], dy = b[1] - a[1], dz = b[2] - a[2];
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Residual error indicator of -rho Lap u + u = ubar on P1 elements (robust residual
// estimator after Verfurth), one thread per tet, grid-stride over a fixed grid:
//   eta_T^2 = a_T^2 ||ubar - u_h||^2_T
//           + 1/2 sum_{interior faces F} rho^{-1/2} a_F |F| (rho [grad u_h . n_F])^2,
// a_S = min(h_S / sqrt(rho), 1), h_S the longest edge of S; the volume integral by the
// quadrature (qb, qw).  Writes eta2[t] and per-block partial sums of eta2.
// grad u_h on every tet (gu[3 t .. 3 t + 2]) and |tau| (vol[t])
__global__ void k_gm_grad_uh(int64_t nt, const int32_t* __restrict__ tet,
                             const int32_t* __restrict__ vdof, const double* __restrict__ xyz,
                             const double* __restrict__ u, double* gu, double* vol) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const int4 tv = reinterpret_cast<const int4*>(tet)[t];
  const int32_t v[4] = {tv.x, tv.y, tv.z, tv.w};
  double X[4][3], g[4][3], U[4];
  for (int a = 0; a < 4; a++) {
    const int32_t w = vdof[v[a]];
    U[a] = w >= 0 ? u[w] : 0.0;
    for (int d = 0; d < 3; d++) X[a][d] = xyz[3 * (int64_t)v[a] + d];
  }
  vol[t] = fabs(tet_grads(X, g)) / 6.0;
  double s[3] = {0.0, 0.0, 0.0};
  for (int a = 0; a < 4; a++)
    for (int d = 0; d < 3; d++) s[d] += U[a] * g[a][d];
  for (int d = 0; d < 3; d++) gu[3 * t + d] = s[d];
}

__global__ void k_gm_indicator(int64_t nt, const int32_t* __restrict__ tet,
                               const int32_t* __restrict__ vdof, const double* __restrict__ xyz,
                               const double* __restrict__ u, const double* __restrict__ guh,
                               const double* __restrict__ tvol, const int64_t* __restrict__ vptr,
                               const int32_t* __restrict__ vtet, TargetDev T, double rho,
                               const double* __restrict__ qb, const double* __restrict__ qw,
                               int np, double* __restrict__ eta2, double* partials,
                               unsigned long long* bad) {
  const double srho = sqrt(rho), rho_m12 = 1.0 / srho;
  double acc[1] = {0.0};
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nt;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int4 tv = reinterpret_cast<const int4*>(tet)[t];
    const int32_t v[4] = {tv.x, tv.y, tv.z, tv.w};
    double X[4][3], U[4];
    for (int a = 0; a < 4; a++) {
      const int32_t w = vdof[v[a]];
      U[a] = w >= 0 ? u[w] : 0.0;
      for (int d = 0; d < 3; d++) X[a][d] = xyz[3 * (int64_t)v[a] + d];
    }
    const double vol = tvol[t];
    const double gu[3] = {guh[3 * t], guh[3 * t + 1], guh[3 * t + 2]};
    double h2 = 0.0;
    for (int a = 0; a < 4; a++)
      for (int b = a + 1; b < 4; b++) h2 = fmax(h2, len2_rn(X[a], X[b]));
    const double aT = fmin(sqrt(h2) / srho, 1.0);
    double e2 = 0.0;
    for (int q = 0; q < np; q++) {
      double x[3] = {0.0, 0.0, 0.0}, uh = 0.0;
      for (int a = 0; a < 4; a++) {
        const double bq = qb[4 * q + a];
        for (int d = 0; d < 3; d++) x[d] += bq * X[a][d];
        uh += bq * U[a];
      }
      const double diff = target_eval(T, x[0], x[1], x[2]) - uh;
      e2 += qw[q] * diff * diff;
    }
    double eta = aT * aT * vol * e2;
    for (int a = 0; a < 4; a++) {
      const int i0 = (a + 1) & 3, i1 = (a + 2) & 3, i2 = (a + 3) & 3;
      const int64_t s = face_neighbour(t, v[i0], v[i1], v[i2], vptr, vtet, tet);
      if (s == -2) atomicAdd(bad, 1ull);
      if (s < 0) continue;
      const double jg[3] = {gu[0] - guh[3 * s], gu[1] - guh[3 * s + 1], gu[2] - guh[3 * s + 2]};
      const double* P0 = X[i0];
      const double* P1 = X[i1];
      const double* P2 = X[i2];
      const double e1[3] = {P1[0] - P0[0], P1[1] - P0[1], P1[2] - P0[2]};
      const double e2v[3] = {P2[0] - P0[0], P2[1] - P0[1], P2[2] - P0[2]};
      const double cr[3] = {e1[1] * e2v[2] - e1[2] * e2v[1], e1[2] * e2v[0] - e1[0] * e2v[2],
                            e1[0] * e2v[1] - e1[1] * e2v[0]};
      const double cn = sqrt(cr[0] * cr[0] + cr[1] * cr[1] + cr[2] * cr[2]);
      const double jump = (jg[0] * cr[0] + jg[1] * cr[1] + jg[2] * cr[2]) / cn;
      const double hF2 = fmax(fmax(len2_rn(P0, P1), len2_rn(P0, P2)), len2_rn(P1, P2));
      const double aF = fmin(sqrt(hF2) / srho, 1.0);
      const double rj = rho * jump;
      eta += 0.5 * (rho_m12 * aF * (0.5 * cn) * (rj * rj));
    }
    eta2[t] = eta;
    acc[0] += eta;
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc[0];
}

__global__ void k_gm_recover(int64_t N, const int64_t* rvert, const double* xyz, TargetDev T,
                             double rho, const double* __restrict__ u, double* z, double* p) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  const int64_t v = rvert[r];
  const double ur = u[r];
  if (z) z[r] = (target_eval(T, xyz[3 * v], xyz[3 * v + 1], xyz[3 * v + 2]) - ur) / rho;
  if (p) p[r] = -rho * ur;
}

// 4-point Hammer-Stroud rule (level 0) for assembly
void hs_rule(DevBuf<double>& qb, DevBuf<double>& qw, int level, cudaStream_t st) {
  std::vector<double> bary, wt;
  const double P[4][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
  bey_rule(P, level, 1.0, bary, wt);
  qb.alloc_async(bary.size(), st);
  qw.alloc_async(wt.size(), st);
  FEM_CUDA(cudaMemcpyAsync(qb, bary.data(), 8 * bary.size(), cudaMemcpyHostToDevice, st));
  FEM_CUDA(cudaMemcpyAsync(qw, wt.data(), 8 * wt.size(), cudaMemcpyHostToDevice, st));
  FEM_CUDA(cudaStreamSynchronize(st));
}

void gm_load_vector(System& S, const TargetDev& T, double* f, cudaStream_t st) {
  DevBuf<double> qb, qw;
  hs_rule(qb, qw, 0, st);
  DevBuf<unsigned long long> bad(1, st);
  FEM_CUDA(cudaMemsetAsync(bad, 0, 8, st));
  DevBuf<double> vol(S.nt, st), fe(4 * S.nt, st);
  k_gm_elements<<<grid_for(S.nt, 128), 128, 0, st>>>(S.nt, S.tet, S.xyz, T, qb, qw, 4, vol,
                                                     nullptr, fe, bad);
  FEM_CHECK_LAUNCH();
  k_gm_row_fill<<<grid_for(S.N, 128), 128, 0, st>>>(
      S.N, S.rvert, S.vptr, S.vtet, S.tet, S.vdof, S.rho, vol, nullptr, fe, nullptr, nullptr,
      nullptr, nullptr, nullptr, f);
  FEM_CHECK_LAUNCH();
  FEM_CUDA(cudaStreamSynchronize(st));
}

}  // namespace

void assemble_rhs(System& S, const fem_target& t, double* f, cudaStream_t st) {
  TargetHolder th;
  target_to_device(t, th, st);
  if (S.general)
    gm_load_vector(S, th.T, f, st);
  else
    load_vector(S, th.T, t, f, st);
  FEM_CUDA(cudaStreamSynchronize(st));
}

void assemble_system(System& S, const fem_kuhn_desc& mesh, double rho, const fem_target& t,
                     const fem_assemble_opts& o, cudaStream_t st) {
  const int n = mesh.n;
  FEM_REQUIRE(n >= 2 && n <= 1290, FEM_EINVAL, "fem_assemble: n must be in [2, 1290]");
  FEM_REQUIRE(rho > 0.0 && std::isfinite(rho), FEM_EINVAL, "fem_assemble: rho must be > 0");
  FEM_REQUIRE(t.kind >= 0 && t.kind <= 4, FEM_EINVAL, "fem_assemble: unknown target kind");
  FEM_REQUIRE(t.kind != FEM_TARGET_BUMPS || (t.nb >= 1 && t.nb <= 64 && t.centers_host &&
                                             t.widths_host && t.amps_host),
              FEM_EINVAL, "fem_assemble: bumps need 1..64 centres/widths/amplitudes");
  FEM_REQUIRE(o.format >= 0 && o.format <= 2, FEM_EINVAL, "fem_assemble: bad format");
  const int m = n - 1;
  const int64_t N = (int64_t)m * m * m;
  FEM_REQUIRE(16 * N < ((int64_t)1 << 31), FEM_EUNSUPPORTED,
              "fem_assemble: more than 2^31 stored entries");
  S.n = n;
  S.N = N;
  S.h = 1.0 / n;
  S.rho = rho;
  S.uniform = (mesh.xyz_host == nullptr);
  FEM_REQUIRE(!(o.format == FEM_FMT_STENCIL && !S.uniform), FEM_EINVAL,
              "fem_assemble: the stencil format needs the uniform grid");
  S.stencil = S.uniform && o.format != FEM_FMT_CSR;
  S.pencil = o.keep_pencil != 0;

  Tracer tr(st);
  // target on the device
  TargetHolder th;
  target_to_device(t, th, st);
  const TargetDev& T = th.T;

  // operator
  S.A.nrows = S.A.ncols = (int32_t)N;
  S.A.nnz = 16 * N;
  S.A.rowptr.alloc(N + 1);
  S.A.col.alloc(16 * N);
  S.A.val.alloc(16 * N);
  if (S.pencil) {
    S.Kv.alloc(16 * N);
    S.Mv.alloc(16 * N);
  }
  DevBuf<double>& xyz = S.xyz;
  if (S.uniform) {
    DevBuf<double> row(45, st);
    k_uniform_row<<<1, 1, 0, st>>>(n, rho, row);
    FEM_CHECK_LAUNCH();
    double hrow[45];
    FEM_CUDA(cudaMemcpyAsync(hrow, row, sizeof(hrow), cudaMemcpyDeviceToHost, st));
    FEM_CUDA(cudaStreamSynchronize(st));
    // per-type coefficients: centre slot 7, axis +x slot 8, face (1,1,0) slot 10,
    // body (1,1,1) slot 14; all slots of one type agree (checked)
    const int rep[4] = {7, 8, 10, 14};
    const int type_of[15] = {3, 2, 2, 1, 2, 1, 1, 0, 1, 1, 2, 1, 2, 2, 3};
    for (int s = 0; s < 15; s++) {
      for (int w = 0; w < 3; w++) {
        double a = hrow[15 * w + s], b = hrow[15 * w + rep[type_of[s]]];
        double scale = fabs(hrow[15 * w + 7]);
        FEM_REQUIRE(fabs(a - b) <= 1e-12 * scale, FEM_EDEVCHECK,
                    "fem_assemble: uniform stencil slots of one type disagree");
      }
    }
    auto mk = [&](int w) {
      Stencil s;
      s.m = m;
      s.c0 = hrow[15 * w + 7];
      s.ca = hrow[15 * w + 8];
      s.cf = hrow[15 * w + 10];
      s.cb = hrow[15 * w + 14];
      return s;
    };
    S.stK = mk(0);
    S.stM = mk(1);
    S.stA = mk(2);
    k_csr_uniform_rows<<<grid_for(N + 1, 128), 128, 0, st>>>(m, S.stA, S.stK, S.stM, S.A.rowptr,
                                                              S.A.col, S.A.val, S.Kv.p, S.Mv.p);
    FEM_CHECK_LAUNCH();
  } else {
    int64_t nv = (int64_t)(n + 1) * (n + 1) * (n + 1);
    xyz.alloc_async(3 * nv, st);
    FEM_CUDA(cudaMemcpyAsync(xyz, mesh.xyz_host, 24 * nv, cudaMemcpyHostToDevice, st));
    k_csr_general<<<grid_for(N + 1, 128), 128, 0, st>>>(n, xyz, rho, S.A.rowptr, S.A.col,
                                                         S.A.val, S.Kv.p, S.Mv.p);
    FEM_CHECK_LAUNCH();
  }

  tr.mark("assemble: operator (CSR4)");
  S.f.alloc(N);
  load_vector(S, T, t, S.f, st);
  tr.mark("assemble: load vector");
  S.dinv.alloc(N);
  if (S.uniform)   // every row of the uniform grid has the centre coefficient on its diagonal
    k_fill_value<<<grid_for(N, 256), 256, 0, st>>>(N, 1.0 / S.stA.c0, S.dinv);
  else
    k_diag_inv<<<grid_for(N, 256), 256, 0, st>>>(N, S.A.rowptr, S.A.col, S.A.val, S.dinv);
  FEM_CHECK_LAUNCH();
  // temporaries are freed stream-ordered; make sure the caller's data is complete
  FEM_CUDA(cudaStreamSynchronize(st));
}

// ------------------------------------------------------------------ allocation-free load vector
//
// Some callers cannot allocate device memory: code that runs while another allocator owns
// (nearly) all of the GPU's memory, callers with a fixed, pre-reserved memory budget, and
// latency-critical loops that must not pay for an allocation and its implicit
// synchronisation.  assemble_rhs_noalloc computes the same load vector as assemble_rhs with
// every scratch buffer (the per-cube partial sums, the separable target tables and the
// copies of the target's parameters) placed in the file-scope array below instead of being
// allocated.  The array is a fixed 17 MB that every GPU loading the library holds until the
// process exits, which limits this path to meshes with n <= 64 cells per side.  All calls
// share it and it keeps the last call's contents; each call overwrites every entry it
// reads, so nothing needs clearing, but calls whose work overlaps on the GPU (different
// streams, no ordering between them) race on it.

namespace {
constexpr int kNoAllocMaxN = 64;
constexpr int kNoAllocMaxTerms = 64;
constexpr size_t kNoAllocCube = 8ull * kNoAllocMaxN * kNoAllocMaxN * kNoAllocMaxN;
constexpr size_t kNoAllocTab = (size_t)kNoAllocMaxTerms * 3 * kNoAllocMaxN * 6;
constexpr size_t kNoAllocDoubles = kNoAllocCube + kNoAllocTab + kNoAllocMaxTerms + 5 * kNoAllocMaxTerms;
}  // namespace

static __device__ __align__(256) double g_rhs_scratch[kNoAllocDoubles];

// Device address of g_rhs_scratch on the current device.  The first call on a device looks
// it up with cudaGetSymbolAddress (with that device current) and caches it; that first call
// must not happen during a stream capture.
static double* noalloc_scratch() {
  static std::mutex mu;
  static double* addr[128] = {nullptr};
  int dev = 0;
  FEM_CUDA(cudaGetDevice(&dev));
  FEM_REQUIRE(dev >= 0 && dev < 128, FEM_EUNSUPPORTED, "fem_assemble_rhs_noalloc: device index");
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    FEM_CUDA(cudaGetSymbolAddress(&p, g_rhs_scratch));
    addr[dev] = static_cast<double*>(p);
  }
  return addr[dev];
}

void assemble_mesh(System& S, const fem_mesh_desc& mesh, double rho, const fem_target& t,
                   const fem_assemble_opts& o, cudaStream_t st) {
  const int64_t nv = mesh.nv, nt = mesh.nt;
  FEM_REQUIRE(nv >= 4 && nt >= 1 && nt < ((int64_t)1 << 31) && nv < ((int64_t)1 << 31),
              FEM_EINVAL, "fem_assemble_mesh: bad sizes");
  FEM_REQUIRE(mesh.xyz && mesh.tet && mesh.dirichlet, FEM_EINVAL,
              "fem_assemble_mesh: null array");
  DevBuf<double> xyz(3 * nv, st);
  DevBuf<int32_t> tet(4 * nt, st);
  DevBuf<uint8_t> dir(nv, st);
  FEM_CUDA(cudaMemcpyAsync(xyz, mesh.xyz, 24 * nv, cudaMemcpyHostToDevice, st));
  FEM_CUDA(cudaMemcpyAsync(tet, mesh.tet, 16 * nt, cudaMemcpyHostToDevice, st));
  FEM_CUDA(cudaMemcpyAsync(dir, mesh.dirichlet, nv, cudaMemcpyHostToDevice, st));
  assemble_mesh_dev(S, nv, nt, xyz, tet, dir, rho, t, o, st);
}

void build_incidence(int64_t nv, int64_t nt, const int32_t* tet, DevBuf<int64_t>& vptr,
                     DevBuf<int32_t>& vtet, cudaStream_t st) {
  DevBuf<int64_t> cnt(nv, st);
  DevBuf<unsigned long long> flags(2, st);
  FEM_CUDA(cudaMemsetAsync(cnt, 0, 8 * nv, st));
  FEM_CUDA(cudaMemsetAsync(flags, 0, 16, st));
  const unsigned gt = grid_for(nt, 256);
  k_gm_inc_count<<<gt, 256, 0, st>>>(nt, tet, nv, cnt, flags);
  FEM_CHECK_LAUNCH();
  unsigned long long hf = 0;
  FEM_CUDA(cudaMemcpyAsync(&hf, flags, 8, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  FEM_REQUIRE(hf == 0, FEM_EINVAL, "mesh: a tet vertex index is out of range");
  vptr.alloc(nv + 1);
  const int64_t ninc = exclusive_scan(cnt, nv, vptr, st);
  vtet.alloc(ninc);
  FEM_CUDA(cudaMemsetAsync(cnt, 0, 8 * nv, st));
  k_gm_inc_fill<<<gt, 256, 0, st>>>(nt, tet, vptr, reinterpret_cast<unsigned long long*>(cnt.p),
                                    vtet);
  FEM_CHECK_LAUNCH();
  k_gm_inc_sort<<<grid_for(nv, 256), 256, 0, st>>>(nv, vptr, vtet, flags.p + 1);
  FEM_CHECK_LAUNCH();
  FEM_CUDA(cudaStreamSynchronize(st));
}

void assemble_mesh_dev(System& S, int64_t nv, int64_t nt, const double* xyz_dev,
                       const int32_t* tet_dev, const uint8_t* dir, double rho,
                       const fem_target& t, const fem_assemble_opts& o, cudaStream_t st) {
  FEM_REQUIRE(nv >= 4 && nt >= 1 && nt < ((int64_t)1 << 31) && nv < ((int64_t)1 << 31),
              FEM_EINVAL, "fem_assemble_mesh: bad sizes");
  FEM_REQUIRE(rho > 0.0 && std::isfinite(rho), FEM_EINVAL, "fem_assemble_mesh: rho must be > 0");
  FEM_REQUIRE(o.format == FEM_FMT_AUTO || o.format == FEM_FMT_CSR, FEM_EINVAL,
              "fem_assemble_mesh: a general mesh has no stencil format");
  TargetHolder th;
  target_to_device(t, th, st);
  S.general = true;
  S.uniform = false;
  S.stencil = false;
  S.pencil = o.keep_pencil != 0;
  S.rho = rho;
  S.n = 0;
  S.nv = nv;
  S.nt = nt;
  Tracer tr(st);
  S.xyz.alloc_async(3 * nv, st);
  S.tet.alloc_async(4 * nt, st);
  FEM_CUDA(cudaMemcpyAsync(S.xyz, xyz_dev, 24 * nv, cudaMemcpyDeviceToDevice, st));
  FEM_CUDA(cudaMemcpyAsync(S.tet, tet_dev, 16 * nt, cudaMemcpyDeviceToDevice, st));
  const unsigned gv = grid_for(nv, 256), gt = grid_for(nt, 256);
  // unknowns
  DevBuf<int64_t> flag(nv, st), scan(nv + 1, st);
  k_gm_free_flags<<<gv, 256, 0, st>>>(nv, dir, flag);
  FEM_CHECK_LAUNCH();
  const int64_t N = exclusive_scan(flag, nv, scan, st);
  FEM_REQUIRE(N >= 1, FEM_EINVAL, "fem_assemble_mesh: every vertex is a Dirichlet vertex");
  S.N = N;
  S.vdof.alloc(nv);
  S.rvert.alloc(N);
  k_gm_dof<<<gv, 256, 0, st>>>(nv, dir, scan, S.vdof, S.rvert);
  FEM_CHECK_LAUNCH();
  // vertex -> incident tets
  DevBuf<int64_t> cnt(nv, st);
  DevBuf<unsigned long long> flags(3, st);
  FEM_CUDA(cudaMemsetAsync(cnt, 0, 8 * nv, st));
  FEM_CUDA(cudaMemsetAsync(flags, 0, 24, st));
  k_gm_inc_count<<<gt, 256, 0, st>>>(nt, S.tet, nv, cnt, flags);
  FEM_CHECK_LAUNCH();
  unsigned long long hf[3];
  FEM_CUDA(cudaMemcpyAsync(hf, flags, 24, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  FEM_REQUIRE(hf[0] == 0, FEM_EINVAL, "fem_assemble_mesh: a tet vertex index is out of range");
  k_gm_tet_check<<<gt, 256, 0, st>>>(nt, S.tet, S.xyz, flags.p + 2);
  FEM_CHECK_LAUNCH();
  S.vptr.alloc(nv + 1);
  const int64_t ninc = exclusive_scan(cnt, nv, S.vptr, st);
  S.vtet.alloc(ninc);
  FEM_CUDA(cudaMemsetAsync(cnt, 0, 8 * nv, st));
  k_gm_inc_fill<<<gt, 256, 0, st>>>(nt, S.tet, S.vptr,
                                    reinterpret_cast<unsigned long long*>(cnt.p), S.vtet);
  FEM_CHECK_LAUNCH();
  k_gm_inc_sort<<<gv, 256, 0, st>>>(nv, S.vptr, S.vtet, flags.p + 1);
  FEM_CHECK_LAUNCH();
  // pattern
  DevBuf<int64_t> rc(N, st);
  k_gm_row_count<<<grid_for(N, 128), 128, 0, st>>>(N, S.rvert, S.vptr, S.vtet, S.tet, S.vdof, rc,
                                                   flags.p + 1);
  FEM_CHECK_LAUNCH();
  FEM_CUDA(cudaMemcpyAsync(hf, flags, 24, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  FEM_REQUIRE(hf[1] == 0, FEM_EUNSUPPORTED,
              "fem_assemble_mesh: more than 64 tets at a vertex or 128 neighbours in a row");
  S.A.nrows = S.A.ncols = (int32_t)N;
  rowptr_from_counts(rc, N, S.A, st);
  S.A.val.alloc(S.A.nnz);
  if (S.pencil) {
    S.Kv.alloc(S.A.nnz);
    S.Mv.alloc(S.A.nnz);
  }
  S.f.alloc(N);
  DevBuf<double> qb, qw;
  hs_rule(qb, qw, 0, st);
  {
    DevBuf<double> vol(nt, st), ke(10 * nt, st), fe(4 * nt, st);
    k_gm_elements<<<grid_for(nt, 128), 128, 0, st>>>(nt, S.tet, S.xyz, th.T, qb, qw, 4, vol, ke,
                                                     fe, flags.p + 2);
    FEM_CHECK_LAUNCH();
    k_gm_row_fill<<<grid_for(N, 128), 128, 0, st>>>(
        N, S.rvert, S.vptr, S.vtet, S.tet, S.vdof, rho, vol, ke, fe, S.A.rowptr, S.A.col, S.A.val,
        S.pencil ? S.Kv.p : nullptr, S.pencil ? S.Mv.p : nullptr, S.f);
    FEM_CHECK_LAUNCH();
  }
  tr.mark("assemble: general mesh");
  S.dinv.alloc(N);
  k_diag_inv<<<grid_for(N, 256), 256, 0, st>>>(N, S.A.rowptr, S.A.col, S.A.val, S.dinv);
  FEM_CHECK_LAUNCH();
  FEM_CUDA(cudaMemcpyAsync(hf, flags, 24, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  FEM_REQUIRE(hf[2] == 0, FEM_EINVAL, "fem_assemble_mesh: a tet has zero volume");
}

void fem_error_norms(System& S, const double* u, const fem_target& t, double scale, int qlevel,
                     double out[2], cudaStream_t st) {
  FEM_REQUIRE(t.kind != FEM_TARGET_QUADVALS, FEM_EINVAL,
              "fem_errors: needs a target it can evaluate anywhere (not point values)");
  FEM_REQUIRE(qlevel >= 0 && qlevel <= 2, FEM_EINVAL, "fem_errors: qlevel in [0, 2]");
  TargetHolder th;
  target_to_device(t, th, st);
  std::vector<double> bary, wt;
  const double P[4][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
  bey_rule(P, qlevel, 1.0, bary, wt);
  const int np = (int)wt.size();
  DevBuf<double> qb(bary.size(), st), qw(wt.size(), st);
  FEM_CUDA(cudaMemcpyAsync(qb, bary.data(), 8 * bary.size(), cudaMemcpyHostToDevice, st));
  FEM_CUDA(cudaMemcpyAsync(qw, wt.data(), 8 * wt.size(), cudaMemcpyHostToDevice, st));
  const int grad = (t.kind == FEM_TARGET_SINE || t.kind == FEM_TARGET_SINE_PLUS_ONE) ? 1 : 0;
  const int64_t ncube = S.general ? S.nt : (int64_t)S.n * S.n * S.n;
  const unsigned g = persistent_grid(ncube, 128, 8);
  DevBuf<double> part(2 * (size_t)g, st), sums(2, st);
  if (!S.general && S.uniform && grad) {
    // separable sine targets on the uniform grid: per-axis tables of the point coordinates'
    // sines and cosines
    static const int PP[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    const int n = S.n;
    const int npq = 6 * np;
    std::vector<double> xi(3 * (size_t)npq), bq(4 * (size_t)npq), gref(6 * 4 * 3);
    for (int p = 0; p < 6; p++) {
      int lv[4] = {0, 0, 0, 0};
      for (int s2 = 0; s2 < 3; s2++) lv[s2 + 1] = lv[s2] | (1 << PP[p][s2]);
      double X[4][3];
      for (int a = 0; a < 4; a++)
        for (int d = 0; d < 3; d++) X[a][d] = (double)((lv[a] >> d) & 1);
      for (int q = 0; q < np; q++) {
        const int pq = p * np + q;
        for (int d = 0; d < 3; d++) {
          double v = 0.0;
          for (int a = 0; a < 4; a++) v += bary[4 * q + a] * X[a][d];
          xi[3 * pq + d] = v;
        }
        for (int a = 0; a < 4; a++) bq[4 * pq + a] = bary[4 * q + a];
      }
      // barycentric gradients of the unit-cube tet: rows of the inverse of [x_a - x_0]
      double J[3][3], Ji[3][3];
      for (int r = 0; r < 3; r++)
        for (int d = 0; d < 3; d++) J[r][d] = X[r + 1][d] - X[0][d];
      const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                         J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                         J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
      for (int r = 0; r < 3; r++)
        for (int d = 0; d < 3; d++) {
          const int r1 = (d + 1) % 3, r2 = (d + 2) % 3, c1 = (r + 1) % 3, c2 = (r + 2) % 3;
          Ji[r][d] = (J[r1][c1] * J[r2][c2] - J[r1][c2] * J[r2][c1]) / det;   // (J^-1)_{r d}
        }
      // grad lambda_a = column a-1 of J^-T for a >= 1, lambda_0 = -(sum of the others)
      for (int d = 0; d < 3; d++) {
        double s0 = 0.0;
        for (int a = 1; a < 4; a++) {
          gref[(p * 4 + a) * 3 + d] = Ji[d][a - 1];
          s0 += Ji[d][a - 1];
        }
        gref[(p * 4 + 0) * 3 + d] = -s0;
      }
    }
    DevBuf<double> dxi(xi.size(), st), dbq(bq.size(), st), dg(gref.size(), st);
    DevBuf<double> tabs(3 * (size_t)npq * n, st), tabc(3 * (size_t)npq * n, st);
    FEM_CUDA(cudaMemcpyAsync(dxi, xi.data(), 8 * xi.size(), cudaMemcpyHostToDevice, st));
    FEM_CUDA(cudaMemcpyAsync(dbq, bq.data(), 8 * bq.size(), cudaMemcpyHostToDevice, st));
    FEM_CUDA(cudaMemcpyAsync(dg, gref.data(), 8 * gref.size(), cudaMemcpyHostToDevice, st));
    k_err_tables<<<grid_for(3 * (int64_t)npq * n, 256), 256, 0, st>>>(n, npq, dxi, tabs, tabc);
    FEM_CHECK_LAUNCH();
    k_errors_sep<<<g, 128, 0, st>>>(n, u, scale, t.kind == FEM_TARGET_SINE_PLUS_ONE ? 1.0 : 0.0,
                                    grad, np, tabs, tabc, dbq, qw, dg, part);
    FEM_CHECK_LAUNCH();
    finalize_sums(part, (int)g, 2, sums, st);
    FEM_CUDA(cudaMemcpyAsync(out, sums, 16, cudaMemcpyDeviceToHost, st));
    FEM_CUDA(cudaStreamSynchronize(st));
    return;
  }
  if (S.general)
    k_gm_errors<<<g, 128, 0, st>>>(S.nt, S.tet, S.vdof, S.xyz, u, th.T, scale, grad, qb, qw, np,
                                   part);
  else
    k_errors<<<g, 128, 0, st>>>(S.n, S.uniform ? nullptr : S.xyz.p, u, th.T, scale, grad, qb, qw,
                                np, part);
  FEM_CHECK_LAUNCH();
  finalize_sums(part, (int)g, 2, sums, st);
  FEM_CUDA(cudaMemcpyAsync(out, sums, 16, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  if (!grad) out[1] = std::nan("");
}

// ------------------------------------------------------------------ mass and stiffness alone

namespace {
// y = V x for values V on a CSR4 pattern (padding columns are -1), FP64
__global__ void k_csr_values_apply(int64_t N, const int32_t* __restrict__ rowptr,
                                   const int32_t* __restrict__ col, const double* __restrict__ v,
                                   const double* __restrict__ x, double* __restrict__ y) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  double s = 0.0;
  for (int e = rowptr[r]; e < rowptr[r + 1]; e++) {
    const int j = col[e];
    if (j >= 0) s = fma(v[e], x[j], s);
  }
  y[r] = s;
}
}  // namespace

void mass_apply(const System& S, const double* x, double* y, cudaStream_t st) {
  const int64_t N = S.N;
  if (N == 0) return;
  FEM_REQUIRE(S.pencil || (S.uniform && !S.general), FEM_EINVAL,
              "mass matrix: a system on a non-uniform mesh needs keep_pencil");
  if (S.pencil) {
    k_csr_values_apply<<<grid_for(N, 256), 256, 0, st>>>(N, S.A.rowptr, S.A.col, S.Mv, x, y);
    FEM_CHECK_LAUNCH();
    return;
  }
  // the uniform grid's mass rows from its stencil
  DevBuf<int32_t> rp(N + 1, st), cl(16 * N, st);
  DevBuf<double> mv(16 * N, st);
  k_csr_uniform_rows<<<grid_for(N + 1, 128), 128, 0, st>>>(S.n - 1, S.stM, S.stK, S.stM, rp, cl,
                                                            mv, nullptr, nullptr);
  FEM_CHECK_LAUNCH();
  k_csr_values_apply<<<grid_for(N, 256), 256, 0, st>>>(N, rp, cl, mv, x, y);
  FEM_CHECK_LAUNCH();
}

void stiffness_system(const System& S, System& SK, cudaStream_t st) {
  FEM_REQUIRE(S.pencil || (S.uniform && !S.general), FEM_EINVAL,
              "stiffness matrix: a system on a non-uniform mesh needs keep_pencil");
  const int64_t N = S.N;
  SK.n = S.n;
  SK.N = N;
  SK.h = S.h;
  SK.rho = 1.0;
  SK.uniform = S.uniform;
  SK.stencil = S.stencil;
  SK.pencil = false;
  SK.general = false;
  SK.stA = S.stK;
  SK.stK = S.stK;
  SK.A.nrows = SK.A.ncols = S.A.nrows;
  SK.A.nnz = S.A.nnz;
  SK.A.rowptr.alloc(N + 1);
  SK.A.col.alloc(S.A.nnz);
  SK.A.val.alloc(S.A.nnz);
  if (S.pencil) {
    FEM_CUDA(cudaMemcpyAsync(SK.A.rowptr, S.A.rowptr, 4 * (N + 1), cudaMemcpyDeviceToDevice, st));
    FEM_CUDA(cudaMemcpyAsync(SK.A.col, S.A.col, 4 * S.A.nnz, cudaMemcpyDeviceToDevice, st));
    FEM_CUDA(cudaMemcpyAsync(SK.A.val, S.Kv, 8 * S.A.nnz, cudaMemcpyDeviceToDevice, st));
  } else {
    k_csr_uniform_rows<<<grid_for(N + 1, 128), 128, 0, st>>>(S.n - 1, S.stK, S.stK, S.stM,
                                                              SK.A.rowptr, SK.A.col, SK.A.val,
                                                              nullptr, nullptr);
    FEM_CHECK_LAUNCH();
  }
  SK.dinv.alloc(N);
  if (N > 0) {
    k_diag_inv<<<grid_for(N, 256), 256, 0, st>>>(N, SK.A.rowptr, SK.A.col, SK.A.val, SK.dinv);
    FEM_CHECK_LAUNCH();
  }
}

double error_indicator(System& S, const double* u, const fem_target& t, int qlevel,
                       double* eta2, cudaStream_t st) {
  FEM_REQUIRE(t.kind != FEM_TARGET_QUADVALS, FEM_EINVAL,
              "fem_error_indicator: needs a target it can evaluate anywhere (not point values)");
  FEM_REQUIRE(S.general, FEM_EINVAL,
              "fem_error_indicator: general meshes only (assemble Kuhn meshes with "
              "fem_assemble_mesh to use it)");
  FEM_REQUIRE(qlevel >= 0 && qlevel <= 2, FEM_EINVAL, "fem_error_indicator: qlevel in [0, 2]");
  TargetHolder th;
  target_to_device(t, th, st);
  std::vector<double> bary, wt;
  const double P[4][4] = {{1, 0, 0, 0}, {0, 1, 0, 0}, {0, 0, 1, 0}, {0, 0, 0, 1}};
  bey_rule(P, qlevel, 1.0, bary, wt);
  DevBuf<double> qb(bary.size(), st), qw(wt.size(), st);
  FEM_CUDA(cudaMemcpyAsync(qb, bary.data(), 8 * bary.size(), cudaMemcpyHostToDevice, st));
  FEM_CUDA(cudaMemcpyAsync(qw, wt.data(), 8 * wt.size(), cudaMemcpyHostToDevice, st));
  const unsigned g = persistent_grid(S.nt, 128, 8);
  DevBuf<double> part(g, st), sum(1, st), gu(3 * S.nt, st), vol(S.nt, st);
  DevBuf<unsigned long long> bad(1, st);
  FEM_CUDA(cudaMemsetAsync(bad, 0, 8, st));
  k_gm_grad_uh<<<grid_for(S.nt, 128), 128, 0, st>>>(S.nt, S.tet, S.vdof, S.xyz, u, gu, vol);
  FEM_CHECK_LAUNCH();
  k_gm_indicator<<<g, 128, 0, st>>>(S.nt, S.tet, S.vdof, S.xyz, u, gu, vol, S.vptr, S.vtet, th.T,
                                    S.rho, qb, qw, (int)wt.size(), eta2, part, bad);
  FEM_CHECK_LAUNCH();
  finalize_sums(part, (int)g, 1, sum, st);
  double out = 0.0;
  unsigned long long hb = 0;
  FEM_CUDA(cudaMemcpyAsync(&out, sum, 8, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaMemcpyAsync(&hb, bad, 8, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  FEM_REQUIRE(hb == 0, FEM_EINVAL, "fem_error_indicator: a face belongs to more than two tets");
  return out;
}

namespace {
__global__ void k_kuhn_dof_vertices(int n, int64_t N, int64_t* vert) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  const int64_t m = n - 1;
  const int64_t i = r % m + 1, j = (r / m) % m + 1, k = r / (m * m) + 1;
  vert[r] = i + (int64_t)(n + 1) * (j + (int64_t)(n + 1) * k);
}
}  // namespace

void dof_vertices(System& S, int64_t* vert, cudaStream_t st) {
  if (S.general) {
    FEM_CUDA(cudaMemcpyAsync(vert, S.rvert, 8 * S.N, cudaMemcpyDeviceToDevice, st));
  } else {
    k_kuhn_dof_vertices<<<grid_for(S.N, 256), 256, 0, st>>>(S.n, S.N, vert);
    FEM_CHECK_LAUNCH();
  }
  FEM_CUDA(cudaStreamSynchronize(st));
}

void fem_recovery(System& S, const double* u, const fem_target& t, double* z, double* p,
                  cudaStream_t st) {
  FEM_REQUIRE(t.kind != FEM_TARGET_QUADVALS, FEM_EINVAL,
              "fem_recover: needs a target it can evaluate at the vertices (not point values)");
  TargetHolder th;
  target_to_device(t, th, st);
  if (S.general)
    k_gm_recover<<<grid_for(S.N, 256), 256, 0, st>>>(S.N, S.rvert, S.xyz, th.T, S.rho, u, z, p);
  else
    k_recover<<<grid_for(S.N, 256), 256, 0, st>>>(S.n, S.uniform ? nullptr : S.xyz.p, th.T,
                                                   S.rho, u, z, p);
  FEM_CHECK_LAUNCH();
  FEM_CUDA(cudaStreamSynchronize(st));
}

void assemble_rhs_noalloc(System& S, const fem_target& t, double* f, cudaStream_t st) {
  FEM_REQUIRE(!S.general, FEM_EINVAL,
              "fem_assemble_rhs_noalloc: Kuhn meshes only (no general meshes)");
  FEM_REQUIRE(S.n <= kNoAllocMaxN, FEM_EINVAL,
              "fem_assemble_rhs_noalloc: n = " + std::to_string(S.n) +
                  " exceeds the allocation-free limit of 64 cells per side");
  FEM_REQUIRE(t.kind != FEM_TARGET_QUADVALS, FEM_EINVAL,
              "fem_assemble_rhs_noalloc: targets given at quadrature points are not taken "
              "(formula targets only: sine, box, bumps, 1 + sine)");
  FEM_REQUIRE(t.kind >= 0 && t.kind <= 3, FEM_EINVAL, "fem_assemble_rhs_noalloc: unknown target");
  FEM_REQUIRE(t.kind != FEM_TARGET_BUMPS || (t.nb >= 1 && t.nb <= kNoAllocMaxTerms &&
                                             t.centers_host && t.widths_host && t.amps_host),
              FEM_EINVAL, "fem_assemble_rhs_noalloc: bumps need 1..64 centres/widths/amplitudes");
  double* base = noalloc_scratch();
  double* cf = base;
  double* tab = cf + kNoAllocCube;
  double* alpha = tab + kNoAllocTab;
  double* par = alpha + kNoAllocMaxTerms;
  const int n = S.n;
  TargetDev T{t.kind, 0, nullptr, nullptr, nullptr, t.lo, t.hi};
  if (t.kind == FEM_TARGET_BUMPS) {
    FEM_CUDA(cudaMemcpyAsync(par, t.centers_host, 24 * t.nb, cudaMemcpyHostToDevice, st));
    FEM_CUDA(cudaMemcpyAsync(par + 3 * kNoAllocMaxTerms, t.widths_host, 8 * t.nb,
                             cudaMemcpyHostToDevice, st));
    FEM_CUDA(cudaMemcpyAsync(par + 4 * kNoAllocMaxTerms, t.amps_host, 8 * t.nb,
                             cudaMemcpyHostToDevice, st));
    T.nb = t.nb;
    T.c = par;
    T.w = par + 3 * kNoAllocMaxTerms;
    T.a = par + 4 * kNoAllocMaxTerms;
  }
  const int64_t ncube = (int64_t)n * n * n;
  if (S.uniform) {
    const int nterms = (t.kind == FEM_TARGET_BUMPS) ? t.nb : (t.kind == FEM_TARGET_SINE_PLUS_ONE ? 2 : 1);
    const int total = nterms * 3 * n * 6;
    k_target_tables<<<grid_for(total, 256), 256, 0, st>>>(T, n, nterms, tab, alpha);
    FEM_CHECK_LAUNCH();
    if (S.N > 0) {
      k_load_sep<<<dim3(n - 1, n - 1), 128, (size_t)nterms * 12 * 8, st>>>(n, tab, alpha, nterms, f);
      FEM_CHECK_LAUNCH();
    }
  } else {
    k_cube_load<<<grid_for(ncube, 128), 128, 0, st>>>(n, S.xyz, T, cf);
    FEM_CHECK_LAUNCH();
    k_gather_load<<<grid_for(S.N, 256), 256, 0, st>>>(n, cf, f);
    FEM_CHECK_LAUNCH();
  }
  // the host parameter arrays are read by the copies above: finish before returning
  FEM_CUDA(cudaStreamSynchronize(st));
}

}  // namespace fem
