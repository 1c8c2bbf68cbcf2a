// BDDC-preconditioned CG on the interface Schur complement (arXiv 2102.03515, Sec. 3.2).
//
// The unit cube's Kuhn mesh is split into p slabs of whole cube layers along z (the paper's
// subdomains come from a graph partitioner; slabs are this library's non-overlapping
// decomposition).  Unknowns are internal to one slab (I) or lie on one of the p - 1 vertex
// planes between slabs (the interface, C).  Every slab keeps two systems of its own, both
// assembled from its tets with the P1 element matrices of the global system (so that they sum
// to it): the Neumann matrix A^i on all its unknowns (Dirichlet only on the cube's boundary)
// and the Dirichlet matrix A^i_II on its internal unknowns; each has a smoothed-aggregation
// hierarchy, and every local solve is AMG-PCG in FP64 to a tight tolerance.
//   * Schur complement S_C = sum_i R_i^T (A^i_CC - A^i_CI (A^i_II)^-1 A^i_IC) R_i, applied as
//     S^i v = (A^i [x_I; v])_C with x_I = -(A^i_II)^-1 (A^i [0; v])_I;
//   * right-hand side g = f_C - sum_i A^i_CI (A^i_II)^-1 f_I^i;
//   * primal constraints: the average over each interface plane (one coarse unknown per
//     plane: a slab has the planes below and above it, C^i its averages);
//   * P_BDDC^-1 = R_D^T (T_sub + T_0) R_D with the multiplicity scaling D = 1/2 (every
//     interface unknown lies in two slabs, the coefficients are uniform);
//     T_sub: the Neumann problem of each slab with zero primal values, by Lagrange
//     multipliers: w = A^-1 r - Q G^-1 Q^T r, Q = A^-1 C^T, G = C Q;
//     T_0 = Phi (Phi^T S_C Phi)^-1 Phi^T with Phi^i = Q G^-1 (the constrained energy-minimal
//     extensions of the primal unit values); Phi^iT S^i Phi^i = G^-1, so the coarse matrix is
//     the assembled sum of the slabs' G^-1, inverted densely;
//   * CG on S_C u_C = g with that preconditioner, then u_I^i = (A^i_II)^-1 (f_I - A^i_IC u_C).
// A process may own a subset of the slabs: every sum over slabs then goes through the
// caller's all-reduce (interface vectors and the coarse vector are replicated on all ranks).
#include <chrono>
#include <cmath>
#include <cstring>
#include <memory>
#include <vector>

#include "solver.cuh"

namespace fem {

void pcg_single(System& S, Hierarchy* H, const double* f, double* u, const pcg_opts& o,
                cudaStream_t user, pcg_result& res);
void alloc_level_vectors(Hierarchy& H);

namespace {

// xN = scale * v on the slab's interface unknowns, 0 elsewhere
__global__ void k_bd_from_iface(int64_t nN, const int32_t* __restrict__ n2G,
                                const double* __restrict__ v, double scale, double* xN) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nN) return;
  const int32_t g = n2G[l];
  xN[l] = g >= 0 ? scale * v[g] : 0.0;
}

// out[n2G[l]] += scale * yN[l] on the slab's interface unknowns (each appears once per slab)
__global__ void k_bd_to_iface(int64_t nN, const int32_t* __restrict__ n2G,
                              const double* __restrict__ yN, double scale, double* out) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nN) return;
  const int32_t g = n2G[l];
  if (g >= 0) out[g] += scale * yN[l];
}

// bI[n2i[l]] = scale * xN[l] on the internal unknowns
__global__ void k_bd_to_internal(int64_t nN, const int32_t* __restrict__ n2i,
                                 const double* __restrict__ xN, double scale, double* bI) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nN) return;
  const int32_t q = n2i[l];
  if (q >= 0) bI[q] = scale * xN[l];
}

// xN[l] = xI[n2i[l]] on the internal unknowns (interface entries unchanged)
__global__ void k_bd_from_internal(int64_t nN, const int32_t* __restrict__ n2i,
                                   const double* __restrict__ xI, double* xN) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nN) return;
  const int32_t q = n2i[l];
  if (q >= 0) xN[l] = xI[q];
}

// f_I of the slab from the global load vector: bI[n2i[l]] = f[n2g[l]]
__global__ void k_bd_load_internal(int64_t nN, const int32_t* __restrict__ n2i,
                                   const int64_t* __restrict__ n2g, const double* __restrict__ f,
                                   double* bI) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nN) return;
  const int32_t q = n2i[l];
  if (q >= 0) bI[q] = f[n2g[l]];
}

// u[n2g[l]] = xN[l] on the internal unknowns and on the interface plane [Glo, Ghi) (the
// plane below the slab: every plane is written by one slab only)
__global__ void k_bd_store(int64_t nN, const int32_t* __restrict__ n2i,
                           const int32_t* __restrict__ n2G, const int64_t* __restrict__ n2g,
                           const double* __restrict__ xN, int64_t Glo, int64_t Ghi, double* u) {
  const int64_t l = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (l >= nN) return;
  const int64_t G = n2G[l];
  if (n2i[l] >= 0 || (G >= Glo && G < Ghi)) u[n2g[l]] = xN[l];
}

// r = f - r
__global__ void k_bd_rsub(int64_t n, const double* f, double* r) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) r[i] = f[i] - r[i];
}

// g = f on the interface unknowns: g[G] = f[global of interface G]
__global__ void k_bd_iface_load(int64_t NG, const int64_t* __restrict__ G2g,
                                const double* __restrict__ f, double* g) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < NG) g[q] = f[G2g[q]];
}

// per-block partial sums of <a, b> (fixed grid: deterministic order)
__global__ void k_bd_dot(int64_t n, const double* a, const double* b, double* part) {
  double v[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    v[0] = fma(a[i], b[i], v[0]);
  block_sum<1>(v);
  if (threadIdx.x == 0) part[blockIdx.x] = v[0];
}

__global__ void k_bd_axpy(int64_t n, double a, const double* x, double* y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] += a * x[i];
}

// p = z + beta p
__global__ void k_bd_xpby(int64_t n, const double* z, double beta, double* p) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) p[i] = z[i] + beta * p[i];
}

}  // namespace

// slab s covers cube layers [K_s, K_{s+1}), K_s = floor(s n / p)
int slab_layer(int n, int p, int s) { return (int)(((int64_t)s * n) / p); }

struct BddcSlab {
  int s = 0, k0 = 0, k1 = 0;          // cube layers [k0, k1)
  System SN, SI;                        // Neumann (all unknowns) and internal systems
  Hierarchy HN, HI;
  int64_t nN = 0, nI = 0;
  DevBuf<int32_t> n2G, n2i;             // Neumann unknown -> interface / internal index (-1)
  DevBuf<int64_t> n2g;                  // Neumann unknown -> global unknown
  int nc = 0;                           // primal constraints (planes below / above)
  int face[2] = {-1, -1};               // their coarse indices
  DevBuf<double> Q;                     // [nc][nN]: A^-1 C^T
  double Ginv[2][2] = {{0, 0}, {0, 0}};
  DevBuf<double> xN, yN, bI, xI;        // work vectors
};

struct Bddc {
  System* sys = nullptr;
  int n = 0, p = 0, s0 = 0, s1 = 0;
  int64_t NG = 0;                       // interface unknowns (p - 1 planes of (n-1)^2)
  std::vector<std::unique_ptr<BddcSlab>> slabs;
  DevBuf<int64_t> G2g;                  // interface index -> global unknown
  std::vector<double> Spi_inv;          // (p-1)^2 coarse inverse
  DevBuf<double> part;
  pcg_opts inner;
  double setup_ms = 0.0;
};


static double bd_dot(Bddc& B, int64_t n, const double* a, const double* b, cudaStream_t st) {
  const unsigned g = persistent_grid(n, 256, 4);
  k_bd_dot<<<g, 256, 0, st>>>(n, a, b, B.part);
  FEM_CHECK_LAUNCH();
  DevBuf<double> s(1, st);
  finalize_sums(B.part, (int)g, 1, s, st);
  double h = 0.0;
  FEM_CUDA(cudaMemcpyAsync(&h, s, 8, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  return h;
}

static void bd_solve(System& S, Hierarchy& H, const double* b, double* x, const pcg_opts& o,
                     cudaStream_t st) {
  pcg_result r{};
  pcg_single(S, &H, b, x, o, st, r);
  FEM_REQUIRE(r.status == FEM_OK, (fem_status)r.status,
              "bddc: a subdomain solve did not converge");
}

// Dense inverse of a small SPD matrix (Gauss-Jordan, no pivoting needed), in place.
static void small_inverse(std::vector<double>& A, int n) {
  std::vector<double> I(n * (size_t)n, 0.0);
  for (int i = 0; i < n; i++) I[i * (size_t)n + i] = 1.0;
  for (int k = 0; k < n; k++) {
    const double piv = A[k * (size_t)n + k];
    FEM_REQUIRE(piv > 0.0, FEM_EDEVCHECK, "bddc: coarse matrix not positive definite");
    for (int j = 0; j < n; j++) {
      A[k * (size_t)n + j] /= piv;
      I[k * (size_t)n + j] /= piv;
    }
    for (int i = 0; i < n; i++) {
      if (i == k) continue;
      const double f = A[i * (size_t)n + k];
      if (f == 0.0) continue;
      for (int j = 0; j < n; j++) {
        A[i * (size_t)n + j] -= f * A[k * (size_t)n + j];
        I[i * (size_t)n + j] -= f * I[k * (size_t)n + j];
      }
    }
  }
  A = I;
}

// Slab s's mesh: vertices (i, j, k) of its layers, tets of its cubes (the Kuhn split of
// every cube along the 6 paths from its first to its last corner), Dirichlet flags on the
// cube's boundary and, for the internal system, on its interface planes too.
static void slab_mesh(int n, int k0, int k1, bool internal, int p, std::vector<double>& xyz,
                      std::vector<int32_t>& tet, std::vector<uint8_t>& dir) {
  static const int PP[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
  const int nl = k1 - k0;
  const int64_t nv = (int64_t)(n + 1) * (n + 1) * (nl + 1);
  xyz.resize(3 * nv);
  dir.resize(nv);
  const double h = 1.0 / n;
  for (int k = 0; k <= nl; k++)
    for (int j = 0; j <= n; j++)
      for (int i = 0; i <= n; i++) {
        const int64_t v = i + (int64_t)(n + 1) * (j + (int64_t)(n + 1) * k);
        const int kg = k0 + k;
        xyz[3 * v] = i * h;
        xyz[3 * v + 1] = j * h;
        xyz[3 * v + 2] = kg * h;
        bool d = i == 0 || i == n || j == 0 || j == n || kg == 0 || kg == n;
        if (internal && ((k == 0 && k0 > 0) || (k == nl && k1 < n))) d = true;
        dir[v] = d ? 1 : 0;
      }
  (void)p;
  tet.resize(4 * 6 * (size_t)n * n * nl);
  size_t t = 0;
  for (int k = 0; k < nl; k++)
    for (int j = 0; j < n; j++)
      for (int i = 0; i < n; i++)
        for (int q = 0; q < 6; q++) {
          int bits = 0;
          for (int a = 0; a < 4; a++) {
            if (a > 0) bits |= 1 << PP[q][a - 1];
            const int vi = i + (bits & 1), vj = j + ((bits >> 1) & 1), vk = k + ((bits >> 2) & 1);
            tet[t++] = (int32_t)(vi + (int64_t)(n + 1) * (vj + (int64_t)(n + 1) * vk));
          }
        }
}

void bddc_build(Bddc& B, System& S, int p, int s0, int s1, const amg_opts& ao,
                       double inner_tol, bddc_reduce_t reduce, void* ctx, cudaStream_t st) {
  FEM_REQUIRE(!S.general && S.n >= 4, FEM_EINVAL, "bddc_setup: a Kuhn-mesh system is needed");
  const int n = S.n, m = n - 1;
  FEM_REQUIRE(p >= 2 && p <= n / 2, FEM_EINVAL, "bddc_setup: 2 <= slabs <= n/2");
  FEM_REQUIRE(0 <= s0 && s0 < s1 && s1 <= p, FEM_EINVAL, "bddc_setup: bad slab range");
  FEM_REQUIRE(S.uniform, FEM_EINVAL, "bddc_setup: the uniform Kuhn mesh is needed");
  B.sys = &S;
  B.n = n;
  B.p = p;
  B.s0 = s0;
  B.s1 = s1;
  B.NG = (int64_t)(p - 1) * m * m;
  B.part.alloc(1024);
  pcg_default_opts(&B.inner);
  B.inner.tol = inner_tol;
  B.inner.max_iter = 500;
  B.inner.use_graph = 0;
  {  // interface index -> global unknown: plane q (vertex layer K_{q+1}), then (i, j)
    std::vector<int64_t> h(B.NG);
    for (int q = 0; q < p - 1; q++) {
      const int kz = slab_layer(n, p, q + 1);
      for (int j = 1; j <= m; j++)
        for (int i = 1; i <= m; i++)
          h[(int64_t)q * m * m + (i - 1) + (int64_t)m * (j - 1)] =
              (i - 1) + (int64_t)m * ((j - 1) + (int64_t)m * (kz - 1));
    }
    B.G2g.alloc(B.NG);
    FEM_CUDA(cudaMemcpyAsync(B.G2g, h.data(), 8 * B.NG, cudaMemcpyHostToDevice, st));
    FEM_CUDA(cudaStreamSynchronize(st));
  }
  fem_target tg{};
  tg.kind = FEM_TARGET_SINE;
  fem_assemble_opts fo{FEM_FMT_CSR, 0};
  std::vector<double> Spi((size_t)(p - 1) * (p - 1), 0.0);
  for (int s = s0; s < s1; s++) {
    auto sl = std::make_unique<BddcSlab>();
    BddcSlab& L = *sl;
    L.s = s;
    L.k0 = slab_layer(n, p, s);
    L.k1 = slab_layer(n, p, s + 1);
    std::vector<double> xyz;
    std::vector<int32_t> tet;
    std::vector<uint8_t> dirN, dirI;
    slab_mesh(n, L.k0, L.k1, false, p, xyz, tet, dirN);
    {
      std::vector<double> x2;
      std::vector<int32_t> t2;
      slab_mesh(n, L.k0, L.k1, true, p, x2, t2, dirI);
    }
    const int64_t nv = (int64_t)dirN.size(), nt = (int64_t)tet.size() / 4;
    fem_mesh_desc dN{nv, nt, xyz.data(), tet.data(), dirN.data()};
    fem_mesh_desc dI{nv, nt, xyz.data(), tet.data(), dirI.data()};
    assemble_mesh(L.SN, dN, S.rho, tg, fo, st);
    assemble_mesh(L.SI, dI, S.rho, tg, fo, st);
    L.nN = L.SN.N;
    L.nI = L.SI.N;
    // unknown maps: Neumann unknowns in increasing vertex order, internal ones likewise
    std::vector<int32_t> n2G(L.nN), n2i(L.nN);
    std::vector<int64_t> n2g(L.nN);
    int64_t a = 0, b = 0;
    const int nl = L.k1 - L.k0;
    for (int k = 0; k <= nl; k++)
      for (int j = 0; j <= n; j++)
        for (int i = 0; i <= n; i++) {
          const int64_t v = i + (int64_t)(n + 1) * (j + (int64_t)(n + 1) * k);
          if (dirN[v]) continue;
          const int kg = L.k0 + k;
          n2g[a] = (i - 1) + (int64_t)m * ((j - 1) + (int64_t)m * (kg - 1));
          int32_t G = -1;
          if (k == 0 && L.k0 > 0) G = (int32_t)((int64_t)(s - 1) * m * m + (i - 1) + (int64_t)m * (j - 1));
          if (k == nl && L.k1 < n) G = (int32_t)((int64_t)s * m * m + (i - 1) + (int64_t)m * (j - 1));
          n2G[a] = G;
          n2i[a] = dirI[v] ? -1 : (int32_t)b++;
          a++;
        }
    FEM_REQUIRE(a == L.nN && b == L.nI, FEM_EDEVCHECK, "bddc: subdomain numbering mismatch");
    L.n2G.alloc(L.nN);
    L.n2i.alloc(L.nN);
    L.n2g.alloc(L.nN);
    FEM_CUDA(cudaMemcpyAsync(L.n2G, n2G.data(), 4 * L.nN, cudaMemcpyHostToDevice, st));
    FEM_CUDA(cudaMemcpyAsync(L.n2i, n2i.data(), 4 * L.nN, cudaMemcpyHostToDevice, st));
    FEM_CUDA(cudaMemcpyAsync(L.n2g, n2g.data(), 8 * L.nN, cudaMemcpyHostToDevice, st));
    build_hierarchy(L.HN, L.SN, ao, st);
    alloc_level_vectors(L.HN);
    build_hierarchy(L.HI, L.SI, ao, st);
    alloc_level_vectors(L.HI);
    L.xN.alloc(L.nN);
    L.yN.alloc(L.nN);
    L.bI.alloc(L.nI > 0 ? L.nI : 1);
    L.xI.alloc(L.nI > 0 ? L.nI : 1);
    // primal constraints: the averages over the planes below (s > 0) and above (s < p-1)
    if (s > 0) L.face[L.nc++] = s - 1;
    if (s < p - 1) L.face[L.nc++] = s;
    L.Q.alloc((size_t)L.nc * L.nN);
    const double avg = 1.0 / ((double)m * m);
    DevBuf<double> cvec(L.nN, st);
    std::vector<double> hc(L.nN);
    for (int c = 0; c < L.nc; c++) {
      const int q = L.face[c];
      for (int64_t l = 0; l < L.nN; l++)
        hc[l] = (n2G[l] >= (int64_t)q * m * m && n2G[l] < (int64_t)(q + 1) * m * m) ? avg : 0.0;
      FEM_CUDA(cudaMemcpyAsync(cvec, hc.data(), 8 * L.nN, cudaMemcpyHostToDevice, st));
      FEM_CUDA(cudaMemsetAsync(L.Q.p + (size_t)c * L.nN, 0, 8 * L.nN, st));
      bd_solve(L.SN, L.HN, cvec, L.Q.p + (size_t)c * L.nN, B.inner, st);
    }
    // G = C Q (nc x nc, symmetric up to the solves' tolerance: symmetrised)
    double G[2][2] = {{0, 0}, {0, 0}};
    for (int c = 0; c < L.nc; c++) {
      const int q = L.face[c];
      for (int64_t l = 0; l < L.nN; l++)
        hc[l] = (n2G[l] >= (int64_t)q * m * m && n2G[l] < (int64_t)(q + 1) * m * m) ? avg : 0.0;
      FEM_CUDA(cudaMemcpyAsync(cvec, hc.data(), 8 * L.nN, cudaMemcpyHostToDevice, st));
      for (int d = 0; d < L.nc; d++) G[c][d] = bd_dot(B, L.nN, cvec, L.Q.p + (size_t)d * L.nN, st);
    }
    if (L.nc == 2) G[0][1] = G[1][0] = 0.5 * (G[0][1] + G[1][0]);
    if (L.nc == 1) {
      L.Ginv[0][0] = 1.0 / G[0][0];
    } else {
      const double det = G[0][0] * G[1][1] - G[0][1] * G[1][0];
      FEM_REQUIRE(det > 0.0, FEM_EDEVCHECK, "bddc: constraint matrix not positive definite");
      L.Ginv[0][0] = G[1][1] / det;
      L.Ginv[1][1] = G[0][0] / det;
      L.Ginv[0][1] = L.Ginv[1][0] = -G[0][1] / det;
    }
    // coarse matrix: the assembled G^-1 of every slab (Phi^T S Phi = G^-1)
    for (int c = 0; c < L.nc; c++)
      for (int d = 0; d < L.nc; d++)
        Spi[(size_t)L.face[c] * (p - 1) + L.face[d]] += L.Ginv[c][d];
    B.slabs.push_back(std::move(sl));
  }
  if (reduce) reduce(Spi.data(), (int64_t)Spi.size(), 0, ctx);
  small_inverse(Spi, p - 1);
  B.Spi_inv = Spi;
}

// out = S_C v (sums of the owned slabs, then the caller's all-reduce)
static void bddc_schur(Bddc& B, const double* v, double* out, bddc_reduce_t reduce, void* ctx,
                       cudaStream_t st) {
  FEM_CUDA(cudaMemsetAsync(out, 0, 8 * B.NG, st));
  for (auto& sp : B.slabs) {
    BddcSlab& L = *sp;
    const unsigned g = grid_for(L.nN, 256);
    Level LN;
    system_level(L.SN, LN);
    k_bd_from_iface<<<g, 256, 0, st>>>(L.nN, L.n2G, v, 1.0, L.xN);
    FEM_CHECK_LAUNCH();
    op_apply_d(LN, L.xN, L.yN, nullptr, nullptr, st);
    if (L.nI > 0) {
      k_bd_to_internal<<<g, 256, 0, st>>>(L.nN, L.n2i, L.yN, -1.0, L.bI);
      FEM_CHECK_LAUNCH();
      FEM_CUDA(cudaMemsetAsync(L.xI, 0, 8 * L.nI, st));
      bd_solve(L.SI, L.HI, L.bI, L.xI, B.inner, st);
      k_bd_from_internal<<<g, 256, 0, st>>>(L.nN, L.n2i, L.xI, L.xN);
      FEM_CHECK_LAUNCH();
      op_apply_d(LN, L.xN, L.yN, nullptr, nullptr, st);
    }
    k_bd_to_iface<<<g, 256, 0, st>>>(L.nN, L.n2G, L.yN, 1.0, out);
    FEM_CHECK_LAUNCH();
  }
  if (reduce) {
    FEM_CUDA(cudaStreamSynchronize(st));
    reduce(out, B.NG, 1, ctx);
  }
}

// z = P_BDDC^-1 r = R_D^T (T_sub + T_0) R_D r
static void bddc_precond(Bddc& B, const double* r, double* z, bddc_reduce_t reduce, void* ctx,
                         cudaStream_t st) {
  const int nc = B.p - 1;
  std::vector<double> c(nc, 0.0);
  std::vector<std::vector<double>> t(B.slabs.size());
  // local Neumann solves of the scaled residual, and the coarse right-hand side
  // Phi^T R_D r = sum_i G_i^-1 Q_i^T (D r)_i
  size_t si = 0;
  for (auto& sp : B.slabs) {
    BddcSlab& L = *sp;
    const unsigned g = grid_for(L.nN, 256);
    k_bd_from_iface<<<g, 256, 0, st>>>(L.nN, L.n2G, r, 0.5, L.yN);
    FEM_CHECK_LAUNCH();
    t[si].assign(2, 0.0);
    for (int a = 0; a < L.nc; a++) t[si][a] = bd_dot(B, L.nN, L.Q.p + (size_t)a * L.nN, L.yN, st);
    for (int a = 0; a < L.nc; a++) {
      double v = 0.0;
      for (int b = 0; b < L.nc; b++) v += L.Ginv[a][b] * t[si][b];
      c[L.face[a]] += v;
    }
    si++;
  }
  if (reduce) reduce(c.data(), nc, 0, ctx);
  std::vector<double> y0(nc, 0.0);
  for (int a = 0; a < nc; a++)
    for (int b = 0; b < nc; b++) y0[a] += B.Spi_inv[(size_t)a * nc + b] * c[b];
  FEM_CUDA(cudaMemsetAsync(z, 0, 8 * B.NG, st));
  si = 0;
  for (auto& sp : B.slabs) {
    BddcSlab& L = *sp;
    const unsigned g = grid_for(L.nN, 256);
    k_bd_from_iface<<<g, 256, 0, st>>>(L.nN, L.n2G, r, 0.5, L.yN);
    FEM_CHECK_LAUNCH();
    FEM_CUDA(cudaMemsetAsync(L.xN, 0, 8 * L.nN, st));
    bd_solve(L.SN, L.HN, L.yN, L.xN, B.inner, st);
    // w = A^-1 r_i - Q G^-1 Q^T r_i  (zero primal values)  +  Phi_i y0_i = Q G^-1 y0_i
    for (int a = 0; a < L.nc; a++) {
      double coef = 0.0;
      for (int b = 0; b < L.nc; b++) coef += L.Ginv[a][b] * (y0[L.face[b]] - t[si][b]);
      k_bd_axpy<<<grid_for(L.nN, 256), 256, 0, st>>>(L.nN, coef, L.Q.p + (size_t)a * L.nN, L.xN);
      FEM_CHECK_LAUNCH();
    }
    k_bd_to_iface<<<g, 256, 0, st>>>(L.nN, L.n2G, L.xN, 0.5, z);
    FEM_CHECK_LAUNCH();
    si++;
  }
  if (reduce) {
    FEM_CUDA(cudaStreamSynchronize(st));
    reduce(z, B.NG, 1, ctx);
  }
}

void bddc_solve_run(Bddc& B, const double* f, double* u, const pcg_opts& o,
                           bddc_reduce_t reduce, void* ctx, cudaStream_t st, pcg_result& res) {
  System& S = *B.sys;
  const int64_t NG = B.NG, N = S.N;
  if (!f) f = S.f.p;
  DevBuf<double> g(NG, st), x(NG, st), rr(NG, st), zz(NG, st), pp(NG, st), qq(NG, st);
  cudaEvent_t e0, e1;
  FEM_CUDA(cudaEventCreate(&e0));
  FEM_CUDA(cudaEventCreate(&e1));
  FEM_CUDA(cudaEventRecord(e0, st));
  // g = f_C - sum_i A_CI (A_II)^-1 f_I
  FEM_CUDA(cudaMemsetAsync(g, 0, 8 * NG, st));
  for (auto& sp : B.slabs) {
    BddcSlab& L = *sp;
    if (L.nI == 0) continue;
    const unsigned gl = grid_for(L.nN, 256);
    Level LN;
    system_level(L.SN, LN);
    k_bd_load_internal<<<gl, 256, 0, st>>>(L.nN, L.n2i, L.n2g, f, L.bI);
    FEM_CHECK_LAUNCH();
    FEM_CUDA(cudaMemsetAsync(L.xI, 0, 8 * L.nI, st));
    bd_solve(L.SI, L.HI, L.bI, L.xI, B.inner, st);
    FEM_CUDA(cudaMemsetAsync(L.xN, 0, 8 * L.nN, st));
    k_bd_from_internal<<<gl, 256, 0, st>>>(L.nN, L.n2i, L.xI, L.xN);
    FEM_CHECK_LAUNCH();
    op_apply_d(LN, L.xN, L.yN, nullptr, nullptr, st);
    k_bd_to_iface<<<gl, 256, 0, st>>>(L.nN, L.n2G, L.yN, -1.0, g);
    FEM_CHECK_LAUNCH();
  }
  if (reduce) {
    FEM_CUDA(cudaStreamSynchronize(st));
    reduce(g, NG, 1, ctx);
  }
  {
    DevBuf<double> fc(NG, st);
    k_bd_iface_load<<<grid_for(NG, 256), 256, 0, st>>>(NG, B.G2g, f, fc);
    FEM_CHECK_LAUNCH();
    k_bd_axpy<<<grid_for(NG, 256), 256, 0, st>>>(NG, 1.0, fc, g);
    FEM_CHECK_LAUNCH();
  }
  // CG on S_C x = g from x = 0, preconditioned by P_BDDC; stop on ||r|| / ||g||
  FEM_CUDA(cudaMemsetAsync(x, 0, 8 * NG, st));
  FEM_CUDA(cudaMemcpyAsync(rr, g, 8 * NG, cudaMemcpyDeviceToDevice, st));
  const double gg = bd_dot(B, NG, g, g, st);
  int it = 0;
  int status = FEM_OK;
  double rnorm2 = gg, rz0 = 0.0, rz = 0.0;
  if (gg > 0.0) {
    bddc_precond(B, rr, zz, reduce, ctx, st);
    rz = rz0 = bd_dot(B, NG, rr, zz, st);
    FEM_CUDA(cudaMemcpyAsync(pp, zz, 8 * NG, cudaMemcpyDeviceToDevice, st));
    const unsigned gN = grid_for(NG, 256);
    while (rnorm2 > o.tol * o.tol * gg) {
      if (it >= o.max_iter) {
        status = FEM_ENOCONV;
        break;
      }
      if (o.cancel_host && *o.cancel_host) {
        status = FEM_ECANCELLED;
        break;
      }
      bddc_schur(B, pp, qq, reduce, ctx, st);
      const double pq = bd_dot(B, NG, pp, qq, st);
      if (!(pq > 0.0) || !std::isfinite(pq)) {
        status = FEM_EBREAKDOWN;
        break;
      }
      const double alpha = rz / pq;
      k_bd_axpy<<<gN, 256, 0, st>>>(NG, alpha, pp, x);
      FEM_CHECK_LAUNCH();
      k_bd_axpy<<<gN, 256, 0, st>>>(NG, -alpha, qq, rr);
      FEM_CHECK_LAUNCH();
      rnorm2 = bd_dot(B, NG, rr, rr, st);
      bddc_precond(B, rr, zz, reduce, ctx, st);
      const double rz_new = bd_dot(B, NG, rr, zz, st);
      if (!(rz_new > 0.0) || !std::isfinite(rz_new)) {
        status = FEM_EBREAKDOWN;
        it++;
        break;
      }
      k_bd_xpby<<<gN, 256, 0, st>>>(NG, zz, rz_new / rz, pp);
      FEM_CHECK_LAUNCH();
      rz = rz_new;
      it++;
    }
  }
  // the solution: interface values, then every slab's internal unknowns
  FEM_CUDA(cudaMemsetAsync(u, 0, 8 * N, st));
  for (auto& sp : B.slabs) {
    BddcSlab& L = *sp;
    const unsigned gl = grid_for(L.nN, 256);
    Level LN;
    system_level(L.SN, LN);
    k_bd_from_iface<<<gl, 256, 0, st>>>(L.nN, L.n2G, x, 1.0, L.xN);
    FEM_CHECK_LAUNCH();
    if (L.nI > 0) {
      op_apply_d(LN, L.xN, L.yN, nullptr, nullptr, st);
      k_bd_to_internal<<<gl, 256, 0, st>>>(L.nN, L.n2i, L.yN, -1.0, L.xI);
      FEM_CHECK_LAUNCH();
      k_bd_load_internal<<<gl, 256, 0, st>>>(L.nN, L.n2i, L.n2g, f, L.bI);
      FEM_CHECK_LAUNCH();
      k_bd_axpy<<<grid_for(L.nI, 256), 256, 0, st>>>(L.nI, 1.0, L.xI, L.bI);
      FEM_CHECK_LAUNCH();
      FEM_CUDA(cudaMemsetAsync(L.xI, 0, 8 * L.nI, st));
      bd_solve(L.SI, L.HI, L.bI, L.xI, B.inner, st);
      k_bd_from_internal<<<gl, 256, 0, st>>>(L.nN, L.n2i, L.xI, L.xN);
      FEM_CHECK_LAUNCH();
    }
    // internal unknowns, and the interface plane below the slab (plane s - 1)
    const int64_t mm = (int64_t)(B.n - 1) * (B.n - 1);
    k_bd_store<<<gl, 256, 0, st>>>(L.nN, L.n2i, L.n2G, L.n2g, L.xN,
                                   L.s > 0 ? (int64_t)(L.s - 1) * mm : 0,
                                   L.s > 0 ? (int64_t)L.s * mm : 0, u);
    FEM_CHECK_LAUNCH();
  }
  // every unknown was written by exactly one slab: the sum over ranks completes u
  if (reduce) {
    FEM_CUDA(cudaStreamSynchronize(st));
    reduce(u, N, 1, ctx);
  }
  FEM_CUDA(cudaEventRecord(e1, st));
  FEM_CUDA(cudaEventSynchronize(e1));
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  // true residual of the global system
  DevBuf<double> Au(N, st);
  Level L0;
  system_level(S, L0);
  op_apply_d(L0, u, Au, nullptr, nullptr, st);
  k_bd_rsub<<<grid_for(N, 256), 256, 0, st>>>(N, f, Au);
  FEM_CHECK_LAUNCH();
  const double r2 = bd_dot(B, N, Au, Au, st), f2 = bd_dot(B, N, f, f, st);
  res.iterations = it;
  res.status = status;
  res.relres = f2 > 0 ? std::sqrt(r2 / f2) : 0.0;
  res.prec_relres = rz0 > 0 ? std::sqrt(std::fabs(rz / rz0)) : 0.0;
  res.solve_ms = ms;
}

Bddc* bddc_create(System& S, int p, int s0, int s1, const amg_opts& ao, double inner_tol,
                  bddc_reduce_t reduce, void* ctx, cudaStream_t st) {
  auto B = std::make_unique<Bddc>();
  auto t0 = std::chrono::steady_clock::now();
  bddc_build(*B, S, p, s0, s1, ao, inner_tol, reduce, ctx, st);
  FEM_CUDA(cudaStreamSynchronize(st));
  B->setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  return B.release();
}

void bddc_free(Bddc* B) { delete B; }

double bddc_setup_ms(const Bddc& B) { return B.setup_ms; }

void bddc_run(Bddc& B, const double* f, double* u, const pcg_opts& o, bddc_reduce_t reduce,
              void* ctx, cudaStream_t st, pcg_result& res) {
  bddc_solve_run(B, f, u, o, reduce, ctx, st, res);
}

}  // namespace fem
