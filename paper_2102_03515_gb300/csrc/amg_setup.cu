// Smoothed-aggregation AMG set-up on the device.
//
// The paper (Sec. 3.1) coarsens by red-black colouring with averaging interpolation and
// forms A_c = P^T A P by Galerkin's method.  This library keeps the Galerkin product and
// replaces the coarsening by smoothed aggregation with these rules:
//  * strength: i != j strong iff a_ij != 0 and |a_ij| >= theta sqrt(a_ii) sqrt(a_jj);
//    nodes without strong neighbours are isolated and not aggregated;
//  * MIS-2: node keys (state, priority), IN > UNDECIDED > OUT, priority
//    (fmix32(i xor s) >> 1) * 2^31 + i with fmix32 the MurmurHash3 finaliser and
//    s = 0x9E3779B9 (seed + level + 1); per round each node takes the largest key within
//    distance 2; an UNDECIDED node whose own key wins enters, one whose winner is IN leaves;
//  * aggregates: roots numbered in index order; phase 1: strong neighbours of a root join
//    it; phase 2: every other non-isolated node joins the phase-1 aggregate it has the
//    most strong edges to (ties: smaller aggregate id);
//  * P = P_t - omega D^{-1} A_F P_t, A_F = diagonal + strong entries, omega = 4/(3 lambda_F),
//    lambda_F = max_i sum_j |A_F(i,j)| / a_ii;
//  * coarsest level: dense FP64 inverse (Gauss-Jordan, SPD so no pivoting) when it has at
//    most coarse_max unknowns, else (coarsening stopped early) the smoother alone.
// Everything is deterministic: integer atomics only, fixed summation orders.
#include <algorithm>
#include <cmath>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "solver.cuh"

namespace fem {
namespace {

// ------------------------------------------------------------------ scan

// Exclusive prefix sums over tiles of SCAN_TILE elements in three passes: the tiles' sums,
// one block's scan of those sums, then every tile's scan from its offset.  Warp w of a
// tile owns SCAN_V consecutive runs of 32 elements (coalesced loads, one value per lane
// and run kept in registers between the tile's sum and its scan).  Integer sums: the
// result does not depend on the order.  A loader maps an index to the summed value.
constexpr int SCAN_T = 256, SCAN_V = 16, SCAN_TILE = SCAN_T * SCAN_V;

struct LoadI64 {
  const int64_t* p;
  __device__ int64_t operator()(int64_t i) const { return p[i]; }
};
struct LoadPad4 {  // counts rounded up to multiples of 4 (CSR4 rows)
  const int64_t* p;
  __device__ int64_t operator()(int64_t i) const { return (p[i] + 3) & ~(int64_t)3; }
};
struct LoadEqU8 {  // 1 where a byte equals v
  const uint8_t* p;
  uint8_t v;
  __device__ int64_t operator()(int64_t i) const { return p[i] == v ? 1 : 0; }
};

__device__ __forceinline__ int64_t warp_sum_i64(int64_t x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}
__device__ __forceinline__ int64_t warp_incl_scan_i64(int64_t x) {
  const int lane = threadIdx.x & 31;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int64_t y = __shfl_up_sync(0xffffffffu, x, o);
    if (lane >= o) x += y;
  }
  return x;
}

template <class L>
__global__ void __launch_bounds__(SCAN_T) k_scan_tiles(L ld, int64_t n, int64_t* tsum) {
  __shared__ int64_t sh[SCAN_T / 32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)w * (32 * SCAN_V) + lane;
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_V; k++) {
    const int64_t i = base + 32 * k;
    if (i < n) s += ld(i);
  }
  s = warp_sum_i64(s);
  if (lane == 0) sh[w] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
#pragma unroll
    for (int q = 0; q < SCAN_T / 32; q++) t += sh[q];
    tsum[blockIdx.x] = t;
  }
}

// One block of 1024 threads: exclusive scan of the nb tile sums in place, total in t[nb].
__global__ void __launch_bounds__(1024) k_scan_tsums(int64_t* t, int64_t nb) {
  __shared__ int64_t ws[32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  int64_t carry = 0;
  for (int64_t b0 = 0; b0 < nb; b0 += 1024) {
    const int64_t i = b0 + threadIdx.x;
    const int64_t v = i < nb ? t[i] : 0;
    const int64_t x = warp_incl_scan_i64(v);
    if (lane == 31) ws[w] = x;
    __syncthreads();
    if (w == 0) ws[lane] = warp_incl_scan_i64(ws[lane]);
    __syncthreads();
    if (i < nb) t[i] = carry + (w ? ws[w - 1] : 0) + x - v;
    carry += ws[31];
    __syncthreads();
  }
  if (threadIdx.x == 0) t[nb] = carry;
}

template <class L, class O>
__global__ void __launch_bounds__(SCAN_T) k_scan_out(L ld, int64_t n, const int64_t* tsum, O* out) {
  __shared__ int64_t sh[SCAN_T / 32];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)w * (32 * SCAN_V) + lane;
  int64_t v[SCAN_V];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < SCAN_V; k++) {
    const int64_t i = base + 32 * k;
    v[k] = i < n ? ld(i) : 0;
    s += v[k];
  }
  s = warp_sum_i64(s);
  if (lane == 0) sh[w] = s;
  __syncthreads();
  int64_t carry = tsum[blockIdx.x];
  for (int q = 0; q < w; q++) carry += sh[q];
#pragma unroll
  for (int k = 0; k < SCAN_V; k++) {
    const int64_t x = warp_incl_scan_i64(v[k]);
    const int64_t i = base + 32 * k;
    if (i < n) out[i] = (O)(carry + x - v[k]);
    carry += __shfl_sync(0xffffffffu, x, 31);
  }
  if (blockIdx.x == gridDim.x - 1 && threadIdx.x == 0) out[n] = (O)tsum[gridDim.x];
}

// out[0..n]: exclusive scan of ld(0..n-1), the total in out[n]; returns the total (n > 0)
template <class L, class O>
int64_t scan_impl(L ld, int64_t n, O* out, cudaStream_t st) {
  const int64_t nb = (n + SCAN_TILE - 1) / SCAN_TILE;
  DevBuf<int64_t> tsum(nb + 1, st);
  k_scan_tiles<L><<<(unsigned)nb, SCAN_T, 0, st>>>(ld, n, tsum);
  FEM_CHECK_LAUNCH();
  k_scan_tsums<<<1, 1024, 0, st>>>(tsum, nb);
  FEM_CHECK_LAUNCH();
  k_scan_out<L, O><<<(unsigned)nb, SCAN_T, 0, st>>>(ld, n, tsum, out);
  FEM_CHECK_LAUNCH();
  int64_t total = 0;
  FEM_CUDA(cudaMemcpyAsync(&total, tsum.p + nb, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  return total;
}

}  // namespace

// out[0..n]: exclusive scan of in[0..n-1] and the total in out[n].  Returns the total.
int64_t exclusive_scan(const int64_t* in, int64_t n, int64_t* out, cudaStream_t st) {
  if (n == 0) {
    FEM_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
    return 0;
  }
  return scan_impl(LoadI64{in}, n, out, st);
}

// out[0..n]: exclusive scan of [s[i] == v]; returns the number of such i.
static int64_t count_scan_eq(const uint8_t* s, uint8_t v, int64_t n, int64_t* out, cudaStream_t st) {
  if (n == 0) {
    FEM_CUDA(cudaMemsetAsync(out, 0, sizeof(int64_t), st));
    return 0;
  }
  return scan_impl(LoadEqU8{s, v}, n, out, st);
}

void rowptr_from_counts(const int64_t* cnt, int64_t n, Csr4& C, cudaStream_t st) {
  C.rowptr.alloc(n + 1);
  int64_t total = 0;
  if (n == 0)
    FEM_CUDA(cudaMemsetAsync(C.rowptr, 0, sizeof(int32_t), st));
  else
    total = scan_impl(LoadPad4{cnt}, n, C.rowptr.p, st);
  // (row pointers past 2^31 were truncated on the device; the matrix is refused here)
  FEM_REQUIRE(total < ((int64_t)1 << 31), FEM_EUNSUPPORTED, "matrix with more than 2^31 entries");
  C.nnz = total;
  C.col.alloc(total);
}

namespace {

// ------------------------------------------------------------------ small kernels

// the diagonal of each row (0 if none), 8 lanes per row; a row holds its diagonal once
// a_ii (0 if the row has no diagonal entry): four lanes per row, one int4 of columns each
// per step; at most one lane finds the column.
constexpr int DG_G = 4;
__global__ void k_diag(int64_t N, const int32_t* rowptr, const int32_t* col, const double* v,
                       double* d) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / DG_G;
  const int sub = threadIdx.x % DG_G;
  const int sh = threadIdx.x & 31 & ~(DG_G - 1);
  if (r >= N) return;
  int pos = -1;
  const int e1 = rowptr[r + 1];
  for (int e = rowptr[r] + 4 * sub; e < e1; e += 4 * DG_G) {
    const int4 c = *reinterpret_cast<const int4*>(col + e);
    if (c.x == r) pos = e;
    if (c.y == r) pos = e + 1;
    if (c.z == r) pos = e + 2;
    if (c.w == r) pos = e + 3;
  }
  const unsigned any = (__ballot_sync(0xFu << sh, pos >= 0) >> sh) & 0xFu;
  if (pos >= 0) d[r] = v[pos];
  if (!any && sub == 0) d[r] = 0.0;
}

__global__ void k_recip(int64_t N, const double* d, double* o, float* o32) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  double v = 1.0 / d[r];
  o[r] = v;
  if (o32) o32[r] = (float)v;
}

// Row sums of |a_ij| over entries selected by mask (null: all), divided by a_ii; block
// maxima into bmax.  Optionally the l1 norms themselves.
__global__ void k_rowabs(int64_t N, const int32_t* rowptr, const int32_t* col, const double* v,
                         const uint8_t* mask, const double* d, double* bmax, double* l1) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double q = -1.0;
  if (r < N) {
    double s = 0.0;
    for (int e = rowptr[r]; e < rowptr[r + 1]; e++) {
      if (col[e] < 0) continue;
      if (mask && !mask[e] && col[e] != r) continue;
      s += fabs(v[e]);
    }
    if (l1) l1[r] = s;
    q = s / d[r];
  }
  q = block_max(q);
  if (threadIdx.x == 0) bmax[blockIdx.x] = q;
}

__global__ void k_max_reduce(const double* in, int n, double* out) {
  double q = -1.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) q = fmax(q, in[i]);
  q = block_max(q);
  if (threadIdx.x == 0) *out = q;
}

template <typename S, typename D>
__global__ void k_convert(int64_t n, const S* in, D* out);
template <>
__global__ void k_convert<double, float>(int64_t n, const double* in, float* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}
template <>
__global__ void k_convert<double, __nv_bfloat16>(int64_t n, const double* in, __nv_bfloat16* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = __float2bfloat16_rn((float)in[i]);
}
// four values per thread (CSR4 value arrays: n a multiple of 4, 32-byte aligned)
__global__ void k_convert4_f32(int64_t n4, const double* in, float* out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n4) return;
  const double2 a = reinterpret_cast<const double2*>(in)[2 * i];
  const double2 b = reinterpret_cast<const double2*>(in)[2 * i + 1];
  reinterpret_cast<float4*>(out)[i] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
}

// ------------------------------------------------------------------ strength + MIS-2

__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85EBCA6Bu;
  h ^= h >> 13;
  h *= 0xC2B2AE35u;
  h ^= h >> 16;
  return h;
}

__device__ __forceinline__ uint64_t prio_of(int64_t i, uint32_t s) {
  uint32_t h = fmix32((uint32_t)i ^ s);
  return ((uint64_t)(h >> 1) << 31) | (uint64_t)i;
}

enum : uint8_t { ST_OUT = 0, ST_UND = 1, ST_IN = 2 };

__global__ void k_sqrt(int64_t N, const double* d, double* sq) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < N) sq[r] = sqrt(d[r]);
}

// strong pair: a_ij != 0 and |a_ij| >= (theta sqrt(a_ii)) sqrt(a_jj)
// Strength of connection, 8 lanes per row (coalesced loads; rows in their stored order):
// smask[e] for every entry, the row's strong count; then the strong columns in entry order
constexpr int ST_G = 8;
__global__ void k_strength(int64_t N, const int32_t* rowptr, const int32_t* col, const double* v,
                           const double* sq, double theta, uint8_t* smask, int64_t* scount) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / ST_G;
  const int lane = threadIdx.x % ST_G;
  const unsigned gm = 0xFFu << (threadIdx.x & 31 & ~(ST_G - 1));
  if (r >= N) return;
  int c = 0;
  const double tr = theta * sq[r];
  for (int e = rowptr[r] + lane; e < rowptr[r + 1]; e += ST_G) {
    const int j = col[e];
    uint8_t s = 0;
    if (j >= 0 && j != r) {
      const double a = v[e];
      s = (a != 0.0) && (fabs(a) >= tr * sq[j]);
    }
    smask[e] = s;
    c += s;
  }
#pragma unroll
  for (int o = ST_G / 2; o > 0; o >>= 1) c += __shfl_xor_sync(gm, c, o, ST_G);
  if (lane == 0) scount[r] = c;
}
__global__ void k_strength_fill(int64_t N, const int32_t* rowptr, const int32_t* col,
                                const uint8_t* smask, const int64_t* sptr, int32_t* scol) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) / ST_G;
  const int lane = threadIdx.x % ST_G;
  const int sh = threadIdx.x & 31 & ~(ST_G - 1);
  const unsigned gm = 0xFFu << sh;
  if (r >= N) return;
  int64_t p = sptr[r];
  const int e0 = rowptr[r], e1 = rowptr[r + 1];
  for (int b = e0; b < e1; b += ST_G) {   // the group's rounds run together (same row)
    const int e = b + lane;
    const bool s = e < e1 && smask[e];
    const unsigned bal = (__ballot_sync(gm, s) >> sh) & 0xFFu;
    if (s) scol[p + __popc(bal & ((1u << lane) - 1u))] = col[e];
    p += __popc(bal);
  }
}

__global__ void k_mis_init(int64_t N, const int64_t* sptr, uint8_t* state) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  state[r] = (sptr[r + 1] == sptr[r]) ? ST_OUT : ST_UND;
}

__global__ void k_mis_m1(int64_t N, const int64_t* sptr, const int32_t* scol,
                         const uint8_t* state, uint32_t s, uint64_t* m1) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  uint64_t best = ((uint64_t)state[r] << 62) | prio_of(r, s);
  for (int64_t e = sptr[r]; e < sptr[r + 1]; e++) {
    int j = scol[e];
    uint64_t kj = ((uint64_t)state[j] << 62) | prio_of(j, s);
    best = kj > best ? kj : best;
  }
  m1[r] = best;
}

__global__ void k_mis_m2(int64_t N, const int64_t* sptr, const int32_t* scol, const uint64_t* m1,
                         uint32_t s, uint8_t* state_in, uint8_t* state_out,
                         unsigned long long* undecided) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  uint8_t st = state_in[r];
  uint64_t best = m1[r];
  for (int64_t e = sptr[r]; e < sptr[r + 1]; e++) {
    uint64_t kj = m1[scol[e]];
    best = kj > best ? kj : best;
  }
  uint8_t ns = st;
  if (st == ST_UND) {
    uint64_t key = ((uint64_t)ST_UND << 62) | prio_of(r, s);
    if (best == key)
      ns = ST_IN;
    else if ((best >> 62) == ST_IN)
      ns = ST_OUT;
    else
      *undecided = 1ull;  // any undecided node (a plain store: only "nonzero" is read)
  }
  state_out[r] = ns;
}

__global__ void k_agg_phase1(int64_t N, const int64_t* sptr, const int32_t* scol,
                             const uint8_t* state, const int64_t* rootid, int32_t* agg,
                             uint8_t* p1, unsigned long long* err) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  int32_t a = -1;
  if (state[r] == ST_IN) {
    a = (int32_t)rootid[r];
  } else {
    int found = 0;
    for (int64_t e = sptr[r]; e < sptr[r + 1]; e++) {
      int j = scol[e];
      if (state[j] == ST_IN) {
        if (found) atomicAdd(err, 1ull);  // two roots within distance 1: MIS-2 violated
        a = (int32_t)rootid[j];
        found = 1;
      }
    }
  }
  agg[r] = a;
  p1[r] = a >= 0;
}

__global__ void k_agg_phase2(int64_t N, const int64_t* sptr, const int32_t* scol, const uint8_t* p1,
                             int32_t* agg, unsigned long long* err) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  if (p1[r]) return;
  const int64_t e0 = sptr[r], e1 = sptr[r + 1];
  if (e0 == e1) return;  // isolated
  int32_t best = -1;
  int bestc = 0;
  for (int64_t e = e0; e < e1; e++) {
    int j = scol[e];
    if (!p1[j]) continue;
    int32_t a = agg[j];
    int c = 0;
    for (int64_t f = e0; f < e1; f++) {
      int q = scol[f];
      if (p1[q] && agg[q] == a) c++;
    }
    if (c > bestc || (c == bestc && a < best)) {
      best = a;
      bestc = c;
    }
  }
  if (best < 0) atomicAdd(err, 1ull);
  agg[r] = best;
}

// tentative prolongator, 4 slots per row
__global__ void k_axpby(int64_t n, double a, const double* x, const double* y, double* z) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) z[i] = a * x[i] + y[i];
}

__global__ void k_tentative(int64_t N, const int32_t* agg, int32_t* rowptr, int32_t* col,
                            double* val) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r > N) return;
  rowptr[r] = (int32_t)(4 * r);
  if (r == N) return;
  int32_t a = agg[r];
  col[4 * r] = a;
  val[4 * r] = a >= 0 ? 1.0 : 0.0;
  for (int q = 1; q < 4; q++) {
    col[4 * r + q] = -1;
    val[4 * r + q] = 0.0;
  }
}

// D^{-1} A_F on A's pattern (weak entries become padding).
__global__ void k_scaled_filtered(int64_t N, const int32_t* rowptr, const int32_t* col,
                                  const double* v, const uint8_t* smask, const double* dinv,
                                  int32_t* ocol, double* oval) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  for (int e = rowptr[r]; e < rowptr[r + 1]; e++) {
    int j = col[e];
    bool keep = (j == r) || smask[e];
    ocol[e] = keep ? j : -1;
    oval[e] = keep ? __dmul_rn(v[e], dinv[r]) : 0.0;
  }
}

// P = P_t - omega B on B's pattern.
__global__ void k_smooth_p(int64_t N, const int32_t* rowptr, const int32_t* col, double* val,
                           const int32_t* agg, double omega) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  for (int e = rowptr[r]; e < rowptr[r + 1]; e++) {
    if (col[e] < 0) continue;
    double t = __dmul_rn(-omega, val[e]);
    val[e] = (col[e] == agg[r]) ? __dadd_rn(1.0, t) : t;
  }
}

// ------------------------------------------------------------------ SpGEMM

// G lanes per output row (a "group"), 256 / G groups per block.  Each group owns a hash
// table of HT slots in shared memory.  The count pass inserts every product column and
// counts distinct keys; the fill pass inserts again, sorts the keys (rank sort), and sums
// the products of each output entry in the order of A's row: lanes split one row of B,
// whose columns are distinct, so each step adds at most once to an output entry.
constexpr int SG_BLOCK = 256;
constexpr int kHTMax = 1024;

__device__ __forceinline__ uint32_t hslot(int key, int mask) {
  return ((uint32_t)key * 2654435761u) & (uint32_t)mask;
}

template <int G>
__device__ __forceinline__ unsigned group_mask() {
  if constexpr (G == 32) {
    return 0xffffffffu;
  } else {
    const int lw = threadIdx.x & 31;
    return ((1u << G) - 1u) << (lw & ~(G - 1));
  }
}

template <int G>
__device__ __forceinline__ int group_sum(int v, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, G);
  return v;
}

template <int G>
__device__ int group_insert(const int32_t* Arp, const int32_t* Acol, const int32_t* Brp,
                            const int32_t* Bcol, int64_t r, int* keys, int ht, int lane,
                            unsigned mask) {
  for (int q = lane; q < ht; q += G) keys[q] = -1;
  __syncwarp(mask);
  int count = 0;
  const int ea = Arp[r], e1 = Arp[r + 1];
  // each round the G lanes load G entries of A's row and their B row ranges at once
  for (int e0 = ea; e0 < e1; e0 += G) {
    const int e = e0 + lane;
    const int k = e < e1 ? Acol[e] : -1;
    const int fb = k >= 0 ? Brp[k] : 0, fe = k >= 0 ? Brp[k + 1] : 0;
    const int nt = min(G, e1 - e0);
    for (int t = 0; t < nt; t++) {
      const int b0 = __shfl_sync(mask, fb, t, G), b1 = __shfl_sync(mask, fe, t, G);
      for (int f = b0 + lane; f < b1; f += G) {
        const int j = Bcol[f];
        if (j < 0) continue;
        uint32_t h = hslot(j, ht - 1);
        for (int probe = 0; probe < ht; probe++) {
          const int old = atomicCAS(&keys[h], -1, j);
          if (old == -1) {
            count++;
            break;
          }
          if (old == j) break;
          h = (h + 1) & (ht - 1);
        }
      }
    }
  }
  count = group_sum<G>(count, mask);
  __syncwarp(mask);
  return count;
}

template <int G, int HT>
__global__ void __launch_bounds__(SG_BLOCK)
    k_sg_count(int64_t nrows, const int32_t* Arp, const int32_t* Acol, const int32_t* Brp,
               const int32_t* Bcol, const int64_t* rows, int64_t* cnt) {
  extern __shared__ __align__(16) char smem[];
  const int grp = threadIdx.x / G, lane = threadIdx.x % G;
  const int64_t q = (int64_t)blockIdx.x * (SG_BLOCK / G) + grp;
  if (q >= nrows) return;
  const int64_t r = rows ? rows[q] : q;   // a listed subset of the rows, or all of them
  int* keys = reinterpret_cast<int*>(smem) + grp * HT;
  const int c = group_insert<G>(Arp, Acol, Brp, Bcol, r, keys, HT, lane, group_mask<G>());
  if (lane == 0) cnt[r] = c;
}

template <int G, int HT>
__global__ void __launch_bounds__(SG_BLOCK)
    k_sg_fill(int64_t nrows, const int32_t* Arp, const int32_t* Acol, const double* Aval,
              const int32_t* Brp, const int32_t* Bcol, const double* Bval, const int32_t* Crp,
              int32_t* Ccol, double* Cval) {
  extern __shared__ __align__(16) char smem[];
  const int grp = threadIdx.x / G, lane = threadIdx.x % G;
  const int64_t r = (int64_t)blockIdx.x * (SG_BLOCK / G) + grp;
  if (r >= nrows) return;
  if (Crp[r + 1] - Crp[r] > HT / 2) return;   // a long row: k_long_fill writes it
  const unsigned mask = group_mask<G>();
  char* base = smem + (size_t)grp * (14 * HT);
  int* keys = reinterpret_cast<int*>(base);
  int* rank = keys + HT;
  double* acc = reinterpret_cast<double*>(base + 8 * HT);
  int* list = reinterpret_cast<int*>(base + 12 * HT);
  const int c = group_insert<G>(Arp, Acol, Brp, Bcol, r, keys, HT, lane, mask);
  // compact the keys (order of table slots)
  const int shift = (threadIdx.x & 31) & ~(G - 1);
  int nb = 0;
  for (int q0 = 0; q0 < HT; q0 += G) {
    const int k = keys[q0 + lane];
    const unsigned bal = (__ballot_sync(mask, k >= 0) >> shift) & (G == 32 ? 0xffffffffu : ((1u << G) - 1u));
    if (k >= 0) list[nb + __popc(bal & ((1u << lane) - 1u))] = k;
    nb += __popc(bal);
  }
  __syncwarp(mask);
  // rank sort: position = number of smaller keys
  const int64_t out0 = Crp[r];
  for (int a = lane; a < c; a += G) {
    const int key = list[a];
    int rk = 0;
    for (int b = 0; b < c; b++) rk += list[b] < key;
    Ccol[out0 + rk] = key;
    uint32_t h = hslot(key, HT - 1);
    while (keys[h] != key) h = (h + 1) & (HT - 1);
    rank[h] = rk;
    if (Cval) acc[rk] = 0.0;
  }
  const int64_t out1 = Crp[r + 1];
  for (int64_t q = out0 + c + lane; q < out1; q += G) {
    Ccol[q] = -1;
    if (Cval) Cval[q] = 0.0;
  }
  __syncwarp(mask);
  if (!Cval) return;
  const int ea = Arp[r], e1 = Arp[r + 1];
  for (int e0 = ea; e0 < e1; e0 += G) {
    const int e = e0 + lane;
    const int k = e < e1 ? Acol[e] : -1;
    const int fb = k >= 0 ? Brp[k] : 0, fe = k >= 0 ? Brp[k + 1] : 0;
    const double av = k >= 0 ? Aval[e] : 0.0;
    const int nt = min(G, e1 - e0);
    for (int t = 0; t < nt; t++) {
      const int b0 = __shfl_sync(mask, fb, t, G), b1 = __shfl_sync(mask, fe, t, G);
      const double a = __shfl_sync(mask, av, t, G);
      for (int f = b0 + lane; f < b1; f += G) {
        const int j = Bcol[f];
        if (j < 0) continue;
        uint32_t h = hslot(j, HT - 1);
        while (keys[h] != j) h = (h + 1) & (HT - 1);
        const int rk = rank[h];
        acc[rk] = __dadd_rn(acc[rk], __dmul_rn(a, Bval[f]));
      }
      __syncwarp(mask);
    }
  }
  __syncwarp(mask);
  for (int a = lane; a < c; a += G) Cval[out0 + a] = acc[a];
}

// Upper bound of the products of each row of A*B (stored entries of B's rows).
__global__ void k_row_ub(int64_t nrows, const int32_t* Arp, const int32_t* Acol,
                         const int32_t* Brp, int64_t* ub) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  int64_t s = 0;
  for (int e = Arp[r]; e < Arp[r + 1]; e++) {
    int k = Acol[e];
    if (k >= 0) s += Brp[k + 1] - Brp[k];
  }
  ub[r] = s;
}

__global__ void k_row_len(int64_t nrows, const int32_t* rp, int64_t* len) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < nrows) len[r] = rp[r + 1] - rp[r];
}

__global__ void k_max_i64(const int64_t* v, int64_t n, unsigned long long* out) {
  unsigned long long m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, (unsigned long long)v[i]);
  for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

// ---- long rows (more distinct product columns than a shared-memory table holds): one block
// per row, the hash table in global memory, the sorted column list and the accumulators in
// shared memory.  The sums run in the order of A's row like the short path.
constexpr int kLongRowMax = 8192;
constexpr int kLongBlock = 256;

constexpr int64_t kSgSample = 4096;

// kSgSample evenly spaced rows of n (n > kSgSample)
__global__ void k_sample_rows(int64_t n, int64_t ns, int64_t* rows) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < ns) rows[q] = q * (n / ns);
}

__global__ void k_gather_i64(int64_t n, const int64_t* idx, const int64_t* src, int64_t* dst) {
  const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (q < n) dst[q] = src[idx[q]];
}

__global__ void k_flag_list(int64_t n, const int64_t* flag, const int64_t* scan, int64_t* list) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n && flag[r]) list[scan[r]] = r;
}

__global__ void k_long_flag(int64_t n, const int64_t* cnt, int64_t limit, int64_t* flag) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < n) flag[r] = cnt[r] > limit ? 1 : 0;
}

// list of the long rows and the size of each one's table (power of two >= 2 * bound)
__global__ void k_long_list(int64_t n, const int64_t* flag, const int64_t* scan,
                            const int64_t* ub, int64_t* list, int64_t* tsz) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= n || !flag[r]) return;
  const int64_t i = scan[r];
  list[i] = r;
  int64_t t = 1024;
  while (t < 2 * ub[r]) t <<= 1;
  tsz[i] = t;
}

__global__ void __launch_bounds__(kLongBlock)
    k_long_count(const int64_t* list, const int64_t* off, const int64_t* tsz, const int32_t* Arp,
                 const int32_t* Acol, const int32_t* Brp, const int32_t* Bcol, int32_t* gkeys,
                 int64_t* cnt) {
  __shared__ int count;
  const int64_t r = list[blockIdx.x];
  int32_t* keys = gkeys + off[blockIdx.x];
  const int64_t T = tsz[blockIdx.x];
  for (int64_t q = threadIdx.x; q < T; q += blockDim.x) keys[q] = -1;
  if (threadIdx.x == 0) count = 0;
  __syncthreads();
  int mine = 0;
  for (int e = Arp[r] + threadIdx.x; e < Arp[r + 1]; e += blockDim.x) {
    const int k = Acol[e];
    if (k < 0) continue;
    for (int f = Brp[k]; f < Brp[k + 1]; f++) {
      const int j = Bcol[f];
      if (j < 0) continue;
      uint32_t h = hslot(j, (int)(T - 1));
      for (int64_t probe = 0; probe < T; probe++) {
        const int old = atomicCAS(keys + h, -1, j);
        if (old == -1) {
          mine++;
          break;
        }
        if (old == j) break;
        h = (h + 1) & (uint32_t)(T - 1);
      }
    }
  }
  atomicAdd(&count, mine);
  __syncthreads();
  if (threadIdx.x == 0) cnt[r] = count;
}

// Ascending bitonic sort of n2 (a power of two) keys in shared memory, values alongside.
__device__ void block_bitonic(int* key, double* val, int n2) {
  for (int k = 2; k <= n2; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < n2; i += blockDim.x) {
        const int l = i ^ j;
        if (l > i) {
          const bool up = (i & k) == 0;
          const int a = key[i], b = key[l];
          if ((a > b) == up) {
            key[i] = b;
            key[l] = a;
            if (val) {
              const double t = val[i];
              val[i] = val[l];
              val[l] = t;
            }
          }
        }
      }
      __syncthreads();
    }
  }
}

__global__ void __launch_bounds__(kLongBlock)
    k_long_fill(const int64_t* list, const int64_t* off, const int64_t* tsz, const int64_t* cnt,
                const int32_t* Arp, const int32_t* Acol, const double* Aval, const int32_t* Brp,
                const int32_t* Bcol, const double* Bval, const int32_t* Crp, int32_t* Ccol,
                double* Cval, const int32_t* gkeys) {
  extern __shared__ __align__(16) char smem[];
  __shared__ int n;
  const int64_t r = list[blockIdx.x];
  const int32_t* keys = gkeys + off[blockIdx.x];
  const int64_t T = tsz[blockIdx.x];
  const int c = (int)cnt[r];
  int n2 = 1;
  while (n2 < c) n2 <<= 1;
  double* acc = reinterpret_cast<double*>(smem);
  int* skey = reinterpret_cast<int*>(smem + 8 * (size_t)kLongRowMax);
  if (threadIdx.x == 0) n = 0;
  __syncthreads();
  for (int64_t q = threadIdx.x; q < T; q += blockDim.x) {
    const int k = keys[q];
    if (k >= 0) skey[atomicAdd(&n, 1)] = k;
  }
  __syncthreads();
  for (int i = c + threadIdx.x; i < n2; i += blockDim.x) skey[i] = 0x7fffffff;
  __syncthreads();
  block_bitonic(skey, nullptr, n2);
  const int64_t o0 = Crp[r], o1 = Crp[r + 1];
  for (int i = threadIdx.x; i < c; i += blockDim.x) {
    Ccol[o0 + i] = skey[i];
    acc[i] = 0.0;
  }
  for (int64_t q = o0 + c + threadIdx.x; q < o1; q += blockDim.x) {
    Ccol[q] = -1;
    if (Cval) Cval[q] = 0.0;
  }
  __syncthreads();
  if (!Cval) return;
  for (int e = Arp[r]; e < Arp[r + 1]; e++) {
    const int k = Acol[e];
    if (k < 0) continue;
    const double a = Aval[e];
    for (int f = Brp[k] + threadIdx.x; f < Brp[k + 1]; f += blockDim.x) {
      const int j = Bcol[f];
      if (j < 0) continue;
      int lo = 0, hi = c - 1;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (skey[mid] < j) lo = mid + 1; else hi = mid;
      }
      acc[lo] = __dadd_rn(acc[lo], __dmul_rn(a, Bval[f]));
    }
    __syncthreads();
  }
  for (int i = threadIdx.x; i < c; i += blockDim.x) Cval[o0 + i] = acc[i];
}

// rows of a transpose longer than the warp sort holds: block bitonic sort by column
__global__ void __launch_bounds__(kLongBlock)
    k_sort_long(int64_t nrows, const int32_t* rp, const int64_t* cnt, int limit, int32_t* col,
                double* val, unsigned long long* err) {
  extern __shared__ __align__(16) char smem[];
  const int64_t r = blockIdx.x;
  if (r >= nrows) return;
  const int c = (int)cnt[r];
  if (c <= limit) return;
  if (c > kLongRowMax) {
    if (threadIdx.x == 0) atomicAdd(err, 1ull);
    return;
  }
  int n2 = 1;
  while (n2 < c) n2 <<= 1;
  double* sv = reinterpret_cast<double*>(smem);
  int* sc = reinterpret_cast<int*>(smem + 8 * (size_t)kLongRowMax);
  const int o = rp[r];
  for (int i = threadIdx.x; i < n2; i += blockDim.x) {
    sc[i] = i < c ? col[o + i] : 0x7fffffff;
    sv[i] = i < c ? val[o + i] : 0.0;
  }
  __syncthreads();
  block_bitonic(sc, sv, n2);
  for (int i = threadIdx.x; i < c; i += blockDim.x) {
    col[o + i] = sc[i];
    val[o + i] = sv[i];
  }
  for (int q = o + c + threadIdx.x; q < rp[r + 1]; q += blockDim.x) {
    col[q] = -1;
    val[q] = 0.0;
  }
}

// Numeric product on a known output pattern (sorted real columns per row).
constexpr int SG_WARPS = 4;
__global__ void __launch_bounds__(32 * SG_WARPS)
    k_spgemm_numeric(int64_t nrows, const int32_t* Arp, const int32_t* Acol, const double* Aval,
                     const int32_t* Brp, const int32_t* Bcol, const double* Bval,
                     const int32_t* Crp, const int32_t* Ccol, double* Cval) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * SG_WARPS + w;
  if (r >= nrows) return;
  const int c0 = Crp[r], c1 = Crp[r + 1];
  int cl = c1;
  while (cl > c0 && Ccol[cl - 1] < 0) cl--;
  for (int q = c0 + lane; q < c1; q += 32) Cval[q] = 0.0;
  __syncwarp();
  for (int e = Arp[r]; e < Arp[r + 1]; e++) {
    int k = Acol[e];
    if (k < 0) continue;
    double a = Aval[e];
    for (int f = Brp[k] + lane; f < Brp[k + 1]; f += 32) {
      int j = Bcol[f];
      if (j < 0) continue;
      int lo = c0, hi = cl - 1;
      while (lo < hi) {
        int mid = (lo + hi) >> 1;
        if (Ccol[mid] < j) lo = mid + 1; else hi = mid;
      }
      Cval[lo] = __dadd_rn(Cval[lo], __dmul_rn(a, Bval[f]));
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------ smoothed prolongator

// P = P_t - omega D^{-1} A_F P_t row by row: the row's diagonal and strong entries give
// (agg(j), a_ij / a_ii); they are stably sorted by aggregate, each run is summed in A's
// order, and the entry of the row's own aggregate gets 1 - omega * sum, the others
// -omega * sum.  Count pass (Pcol == null) writes the number of distinct aggregates.
constexpr int PS_MAX = 32;
__global__ void k_psmooth(int64_t N, const int32_t* rowptr, const int32_t* col, const double* val,
                          const uint8_t* smask, const int32_t* agg, const double* dinv,
                          double omega, int64_t* cnt, const int32_t* Prp, int32_t* Pcol,
                          double* Pval, unsigned long long* overflow) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  const int32_t ar = agg[r];
  int keys[PS_MAX];
  double vals[PS_MAX];
  int m = 0;
  if (ar >= 0) {
    const double di = dinv[r];
    for (int e = rowptr[r]; e < rowptr[r + 1]; e++) {
      const int j = col[e];
      if (j < 0 || (j != r && !smask[e])) continue;
      const int a = agg[j];
      if (a < 0) continue;
      if (m == PS_MAX) {
        atomicAdd(overflow, 1ull);
        return;
      }
      const double v = __dmul_rn(val[e], di);
      int q = m++;
      while (q > 0 && keys[q - 1] > a) {
        keys[q] = keys[q - 1];
        vals[q] = vals[q - 1];
        q--;
      }
      keys[q] = a;
      vals[q] = v;
    }
  }
  if (!Pcol) {
    int d = 0;
    for (int q = 0; q < m; q++) d += (q == 0 || keys[q] != keys[q - 1]);
    cnt[r] = d;
    return;
  }
  int64_t o = Prp[r];
  const int64_t o1 = Prp[r + 1];
  int q = 0;
  while (q < m) {
    const int key = keys[q];
    double sum = vals[q++];
    while (q < m && keys[q] == key) sum = __dadd_rn(sum, vals[q++]);
    const double t = __dmul_rn(-omega, sum);
    Pcol[o] = key;
    Pval[o] = key == ar ? __dadd_rn(1.0, t) : t;
    o++;
  }
  for (; o < o1; o++) {
    Pcol[o] = -1;
    Pval[o] = 0.0;
  }
}

// ------------------------------------------------------------------ transpose

__global__ void k_col_count(int64_t nnz, const int32_t* col, unsigned long long* cnt) {
  int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e < nnz && col[e] >= 0) atomicAdd(&cnt[col[e]], 1ull);
}
__global__ void k_u64_to_i64(int64_t n, const unsigned long long* a, int64_t* b) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (int64_t)a[i];
}
__global__ void k_scatter_t(int64_t nrows, const int32_t* rowptr, const int32_t* col,
                            const double* val, const int32_t* Trp, unsigned long long* fill,
                            int32_t* Tcol, double* Tval) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= nrows) return;
  for (int e = rowptr[r]; e < rowptr[r + 1]; e++) {
    int c = col[e];
    if (c < 0) continue;
    unsigned long long p = atomicAdd(&fill[c], 1ull);
    Tcol[Trp[c] + p] = (int32_t)r;
    Tval[Trp[c] + p] = val[e];
  }
}
// sort each row's first cnt entries by column (rank sort in a warp), pad the rest of the row:
// rows of at most TM entries (rows of at most lo entries were sorted by an earlier pass;
// longer rows are counted in err for the next one)
constexpr int TMAX = 1024;
template <int TM>
__global__ void k_sort_rows(int64_t nrows, const int32_t* rp, const int64_t* cnt, int lo,
                            int32_t* col, double* val, unsigned long long* err) {
  __shared__ int sc[4][TM];
  __shared__ double sv[4][TM];
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * 4 + w;
  if (r >= nrows) return;
  const int c = (int)cnt[r];
  if (c <= lo) return;
  const int o = rp[r];
  if (c > TM) {
    if (lane == 0) atomicAdd(err, 1ull);   // counted: the next pass sorts these rows
    return;
  }
  for (int a = lane; a < c; a += 32) {
    sc[w][a] = col[o + a];
    sv[w][a] = val[o + a];
  }
  __syncwarp();
  for (int a = lane; a < c; a += 32) {
    int key = sc[w][a];
    int rk = 0;
    for (int b = 0; b < c; b++) rk += sc[w][b] < key;
    col[o + rk] = key;
    val[o + rk] = sv[w][a];
  }
  for (int q = o + c + lane; q < rp[r + 1]; q += 32) {
    col[q] = -1;
    val[q] = 0.0;
  }
}

// ------------------------------------------------------------------ dense coarsest

__global__ void k_dense_from_csr(int64_t N, const int32_t* rowptr, const int32_t* col,
                                 const double* v, double* D) {
  int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  for (int64_t c = 0; c < N; c++) D[r * N + c] = 0.0;
  for (int e = rowptr[r]; e < rowptr[r + 1]; e++)
    if (col[e] >= 0) D[r * N + col[e]] += v[e];
}

// Gauss-Jordan step k (no pivoting: A is SPD), from D into E:
//   E_kk = 1/p, E_kj = D_kj / p, E_ik = -D_ik / p, E_ij = D_ij - D_ik D_kj / p,  p = D_kk.
__global__ void k_gj_step(int64_t N, int64_t k, const double* __restrict__ D, double* __restrict__ E) {
  __shared__ double inv_p;
  if (threadIdx.x == 0) inv_p = 1.0 / D[k * N + k];
  __syncthreads();
  const double ip = inv_p;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < N * N;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t i = t / N, j = t % N;
    double v;
    if (i == k && j == k)
      v = ip;
    else if (i == k)
      v = D[t] * ip;
    else if (j == k)
      v = -D[t] * ip;
    else
      v = D[t] - D[i * N + k] * (D[k * N + j] * ip);
    E[t] = v;
  }
}

// On the finest level of a uniform Kuhn grid every row of A holds the same values at the
// same offsets (a subset of them at the boundary), so the strength graph, the Gershgorin
// bounds and the smoothed prolongator follow from one interior row.  The kernels below
// walk the stencil's offsets instead of A's columns; they take the same decisions and do
// the same arithmetic, in the same order, as the CSR kernels above.
struct StencilRow {
  int m = 0;
  uint32_t present = 0;      // bit d: the interior row has an entry at direction d
  uint32_t strong = 0;       // bit d: that entry is a strong pair (never the diagonal)
  double a[27];              // value at direction d
};
// direction d = (dx + 1) + 3 (dy + 1) + 9 (dz + 1): increasing d is increasing column
// offset dx + m dy + m^2 dz (m >= 3), i.e. A's column order; d = 13 is the diagonal.
constexpr int ST_DIAG = 13;

__device__ __forceinline__ bool st_inb(int i, int j, int k, int d, int m) {
  const int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
  return (unsigned)(i + dx) < (unsigned)m && (unsigned)(j + dy) < (unsigned)m &&
         (unsigned)(k + dz) < (unsigned)m;
}

__device__ __forceinline__ int64_t st_off(int d, int m) {
  return (int64_t)(d % 3 - 1) + (int64_t)m * (d / 3 % 3 - 1) + (int64_t)m * m * (d / 9 - 1);
}

// strong-direction test: compile-time mask when MASK != 0, else the runtime one
template <uint32_t MASK>
__device__ __forceinline__ bool st_sel(uint32_t strong, int d) {
  return MASK ? ((MASK >> d) & 1u) != 0 : ((strong >> d) & 1u) != 0;
}

__device__ __forceinline__ void st_ijk(int64_t r, int m, int& i, int& j, int& k) {
  const uint32_t rr = (uint32_t)r, mm = (uint32_t)m;
  const uint32_t q = rr / mm;
  i = (int)(rr - q * mm);
  k = (int)(q / mm);
  j = (int)(q - (uint32_t)k * mm);
}


// ------------------------------------------------------------------ merge SpGEMM

// C = A B when every row of B holds sorted, distinct columns: CSR4 rows, whose (-1, 0)
// padding ends a row, or rows at a fixed stride with their lengths (an earlier product).
// G lanes per row of C; lane l holds the B rows named by the entries t = l + G s (s < K) of
// the A row, each as a cursor and its current column (the head).
//  * keys: each step the group takes the smallest head over all its lists (a lane's own
//    minimum, then a shuffle reduction), writes it as the next column of the row and
//    advances every list whose head it is, noting in shared memory the output position of
//    the B entry it passed: the distinct columns come out in increasing order, with no hash
//    table and no sort;
//  * values: the A row is walked in its stored order; for each entry the lanes split the B
//    row and add each product at the noted position.  A B row's columns are distinct, so
//    one step adds at most once to an output entry, and every entry is summed in the order
//    of A's row whatever G.
// C is written at a fixed stride W with its row lengths.  A row with more than W columns
// writes only its length and raises the overflow flag (the caller repeats the product
// with a wider stride).
constexpr int MG_BLOCK = 256;
constexpr int MG_INF = 0x7fffffff;

struct MgRows {
  const int32_t* rp;    // CSR4 row pointer, or null: rows at a fixed stride
  const int64_t* len;   // row lengths at the fixed stride
  int32_t stride;
  __device__ __forceinline__ int beg(int k) const { return rp ? rp[k] : k * stride; }
  __device__ __forceinline__ int end(int k) const {
    return rp ? rp[k + 1] : k * stride + (int)len[k];
  }
};

template <int G>
__device__ __forceinline__ int group_min(int v, unsigned mask) {
#pragma unroll
  for (int o = G / 2; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(mask, v, o, G));
  return v;
}

template <int G, int K>
__global__ void __launch_bounds__(MG_BLOCK)
    k_mg(int64_t nrows, const int64_t* __restrict__ rlist, const int32_t* __restrict__ Arp,
         const int32_t* __restrict__ Acol, const double* __restrict__ Aval, MgRows B,
         const int32_t* __restrict__ Bcol, const double* __restrict__ Bval, int W, int lmax,
         int32_t* __restrict__ Ccol, double* __restrict__ Cval, int64_t* __restrict__ Clen,
         unsigned int* overflow, int upper) {
  extern __shared__ __align__(16) char smem[];
  const int grp = threadIdx.x / G, lane = threadIdx.x % G;
  const int64_t rr = (int64_t)blockIdx.x * (MG_BLOCK / G) + grp;
  if (rr >= nrows) return;
  const int64_t r = rlist ? rlist[rr] : rr;   // the rows of C wanted (null: all)
  const unsigned mask = group_mask<G>();
  // per group: W + 1 sums, then the output position of every entry of every list (G K lists
  // of at most lmax entries) and 4 bytes (the odd strides start the groups in different
  // shared-memory banks)
  constexpr int NG = MG_BLOCK / G;
  double* acc = reinterpret_cast<double*>(smem) + (size_t)grp * (W + 1);
  uint8_t* pos = reinterpret_cast<uint8_t*>(reinterpret_cast<double*>(smem) + (size_t)NG * (W + 1)) +
                 (size_t)grp * (G * K * lmax + 4);
  // upper part: each list's first entry at or above the row (B's rows are then unpadded)
  int* skp = reinterpret_cast<int*>(reinterpret_cast<uint8_t*>(reinterpret_cast<double*>(smem) +
                                                               (size_t)NG * (W + 1)) +
                                    (size_t)NG * (G * K * lmax + 4)) +
             grp * G * K;
  const int ea = Arp[r], e1 = Arp[r + 1];
  const int lo = upper ? (int)r : 0;   // the smallest column wanted
  int cur[K], end[K], head[K], base[K];   // base + cursor: the entry's position slot
#pragma unroll
  for (int s = 0; s < K; s++) {
    const int e = ea + lane + G * s;
    const int k = e < e1 ? Acol[e] : -1;
    cur[s] = k >= 0 ? B.beg(k) : 0;
    end[s] = k >= 0 ? B.end(k) : 0;
    base[s] = (lane + G * s) * lmax - cur[s];
    if (upper) {   // lower bound of the row in the sorted list
      int n = end[s] - cur[s];
      while (n > 0) {
        const int half = n >> 1;
        if (Bcol[cur[s] + half] < lo) {
          cur[s] += half + 1;
          n -= half + 1;
        } else {
          n = half;
        }
      }
      skp[lane + G * s] = cur[s];
    }
    const int h = cur[s] < end[s] ? Bcol[cur[s]] : MG_INF;
    head[s] = h < 0 ? MG_INF : h;
  }
  int32_t* crow = Ccol + r * W;
  int c = 0;
  for (;;) {
    int lm = head[0];
#pragma unroll
    for (int s = 1; s < K; s++) lm = min(lm, head[s]);
    const int m = group_min<G>(lm, mask);
    if (m == MG_INF) break;
    const bool keep = c < W;
    if (keep && lane == (c & (G - 1))) crow[c] = m;
#pragma unroll
    for (int s = 0; s < K; s++) {
      if (head[s] == m) {
        if (keep) pos[base[s] + cur[s]] = (uint8_t)c;
        const int q = ++cur[s];
        const int h = q < end[s] ? Bcol[q] : MG_INF;
        head[s] = h < 0 ? MG_INF : h;
      }
    }
    c++;
  }
  if (c > W) {   // the row does not fit: its length only
    if (lane == 0) {
      Clen[r] = c;
      atomicOr(overflow, 1u);
    }
    return;
  }
  for (int q = lane; q < c; q += G) acc[q] = 0.0;
  __syncwarp(mask);
  for (int e0 = ea; e0 < e1; e0 += G) {
    const int e = e0 + lane;
    const int k = e < e1 ? Acol[e] : -1;
    const int fb = k >= 0 ? B.beg(k) : 0, fe = k >= 0 ? B.end(k) : 0;
    const int fs = (upper && k >= 0) ? skp[e - ea] : fb;   // first entry taken
    const double av = k >= 0 ? Aval[e] : 0.0;
    const int nt = min(G, e1 - e0);
    for (int t = 0; t < nt; t++) {
      const int b0 = __shfl_sync(mask, fb, t, G), b1 = __shfl_sync(mask, fe, t, G);
      const int bs = __shfl_sync(mask, fs, t, G);
      const double a = __shfl_sync(mask, av, t, G);
      const uint8_t* pt = pos + (e0 - ea + t) * lmax - b0;
      for (int f = bs + lane; f < b1; f += G) {
        if (Bcol[f] < 0) continue;   // padding
        const int q = pt[f];
        acc[q] = fma(a, Bval[f], acc[q]);
      }
      __syncwarp(mask);
    }
  }
  double* vrow = Cval + r * W;
  for (int q = lane; q < c; q += G) vrow[q] = acc[q];
  if (lane == 0) Clen[r] = c;
}

// A symmetric product from its upper part U (columns >= row, at a fixed stride): row I of
// the product is the lower part {(J, U[J][I]) : J < I} followed by U's row I.  A warp per row
// of U: the count and the scatter of the lower entries (unordered until the rows are
// sorted), then U's row after the sorted lower part.
__global__ void k_u_count(int64_t nrows, int W, const int32_t* __restrict__ Ucol,
                          const int64_t* __restrict__ Ulen, unsigned long long* cnt) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= nrows) return;
  const int c = (int)Ulen[r];
  for (int q = lane; q < c; q += 32) {
    const int j = Ucol[r * W + q];
    if (j > r) atomicAdd(&cnt[j], 1ull);
  }
}

__global__ void k_u_len(int64_t n, const unsigned long long* lcnt, const int64_t* Ulen,
                        int64_t* lower, int64_t* total) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  lower[i] = (int64_t)lcnt[i];
  total[i] = (int64_t)lcnt[i] + Ulen[i];
}

__global__ void k_u_scatter(int64_t nrows, int W, const int32_t* __restrict__ Ucol,
                            const double* __restrict__ Uval, const int64_t* __restrict__ Ulen,
                            const int32_t* __restrict__ Crp, unsigned long long* fill,
                            int32_t* __restrict__ Ccol, double* __restrict__ Cval) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= nrows) return;
  const int c = (int)Ulen[r];
  for (int q = lane; q < c; q += 32) {
    const int j = Ucol[r * W + q];
    if (j <= r) continue;
    const unsigned long long p = atomicAdd(&fill[j], 1ull);
    Ccol[Crp[j] + p] = (int32_t)r;
    Cval[Crp[j] + p] = Uval[r * W + q];
  }
}

__global__ void k_u_upper(int64_t nrows, int W, const int32_t* __restrict__ Ucol,
                          const double* __restrict__ Uval, const int64_t* __restrict__ Ulen,
                          const int32_t* __restrict__ Crp, const int64_t* __restrict__ lower,
                          int32_t* __restrict__ Ccol, double* __restrict__ Cval) {
  const int64_t r = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (r >= nrows) return;
  const int c = (int)Ulen[r];
  const int64_t o = Crp[r] + lower[r];
  for (int q = lane; q < c; q += 32) {
    Ccol[o + q] = Ucol[r * W + q];
    Cval[o + q] = Uval[r * W + q];
  }
}

// A P on the uniform finest level.  A's rows are the stencil (directions in column order,
// the same values in every row), so only P is read.  A block takes a brick of 8 x 4 x 4
// rows, four lanes per row, and stages the P rows of the brick and its one-node halo
// (every P row an A row of the brick names):
//  1. the staged columns go into a hash set, and each distinct column gets as local id its
//     rank among them, so local ids follow the column order; each staged row keeps its
//     entries' local ids and values (in column order) and a 256-bit mask of its ids;
//  2. a row's columns are the bits of the OR of its neighbours' masks (each lane ORs a
//     quarter of the directions, shuffles join them), written out in increasing order;
//  3. the directions are walked in column order, the four lanes splitting the neighbour's
//     P row, and each product is added at its output position (the row mask's bits below
//     its id): the merge kernel's products in the merge kernel's order, rounding for
//     rounding (a P row's ids are distinct, so one direction adds once per position).
// A row longer than the stride W writes its length only (flag bit 0); a brick beyond the
// staging limits (256 distinct columns, AB_E staged entries, P rows of more than 8 stored
// entries) gives up (bit 1: the caller takes the merge kernel).
constexpr int AB_X = 8, AB_Y = 4, AB_Z = 4, AB_R = AB_X * AB_Y * AB_Z;   // 128 rows
constexpr int AB_G = 4, AB_T = AB_G * AB_R;                              // 512 threads
constexpr int AB_HX = AB_X + 2, AB_HY = AB_Y + 2, AB_HZ = AB_Z + 2;
constexpr int AB_H = AB_HX * AB_HY * AB_HZ;   // 360 staged rows
constexpr int AB_L = 8;                        // stored entries per staged P row
constexpr int AB_E = 2048;                     // staged entries per brick
constexpr int AB_IDS = 256;                    // local ids per brick
constexpr int AB_W = AB_IDS / 32;              // mask words per row
constexpr int AB_HASH = 512;                   // hash slots
constexpr int AB_NIT = (AB_H * AB_L + AB_T - 1) / AB_T;   // staged entries per thread
constexpr uint16_t AB_NONE = 0xFFFF;

// shared-memory layout (bytes).  The first region holds the hash set and the staged
// entries' slots while the brick is staged, then the rows' sums (row stride W | 1).
struct AbSmem {
  static constexpr size_t hkey = 0;                                   // int32 [AB_HASH]
  static constexpr size_t slot = hkey + 4 * AB_HASH;                  // uint16 [AB_L][AB_H]
  static constexpr size_t hlid = slot + 2 * AB_L * AB_H;              // uint8 [AB_HASH]
  static constexpr size_t stage_end = (hlid + AB_HASH + 15) & ~size_t(15);
  // after the first region
  static constexpr size_t vals = 0;                                   // double [AB_E]
  static constexpr size_t pa = vals + 8 * AB_E;                       // double [27]
  static constexpr size_t nmask = pa + 8 * 28;                        // uint32 [AB_H][AB_W]
  static constexpr size_t rmask = nmask + 4 * AB_H * AB_W;            // uint32 [AB_W][AB_R]
  static constexpr size_t keys = rmask + 4 * AB_W * AB_R;             // int32 [AB_IDS]
  static constexpr size_t lcol = keys + 4 * AB_IDS;                   // int32 [AB_IDS]
  static constexpr size_t hrow = lcol + 4 * AB_IDS;                   // int32 [AB_H]
  static constexpr size_t poff = hrow + 4 * AB_H;                     // int32 [28]
  static constexpr size_t pdir = poff + 4 * 28;                       // int32 [28]
  static constexpr size_t wsum = pdir + 4 * 28;                       // int32 [AB_T / 32]
  static constexpr size_t ctl = wsum + 4 * (AB_T / 32);               // int32 [4]
  static constexpr size_t kslot = ctl + 16;                           // uint16 [AB_IDS]
  static constexpr size_t hoff = kslot + 2 * AB_IDS;                  // uint16 [AB_H]
  static constexpr size_t elid = hoff + 2 * AB_H;                     // uint8 [AB_E]
  static constexpr size_t rpre = elid + AB_E;                         // uint8 [AB_W][AB_R]
  static constexpr size_t hlen = rpre + AB_W * AB_R;                  // uint8 [AB_H]
  static constexpr size_t hcnt = hlen + AB_H;                         // uint8 [AB_H]
  static constexpr size_t size = hcnt + AB_H;
};
static_assert(AbSmem::hcnt % 4 == 0 && AbSmem::nmask % 16 == 0, "shared-memory alignment");
__host__ __device__ inline size_t ab_region(int W) {
  const size_t acc = (((size_t)(W | 1) * AB_R * 8) + 15) & ~size_t(15);
  return acc > AbSmem::stage_end ? acc : AbSmem::stage_end;
}
static size_t ab_smem(int W) { return ab_region(W) + AbSmem::size; }

__global__ void __launch_bounds__(AB_T, 3) k_ap_brick(StencilRow S, const int32_t* __restrict__ Prp,
                                                      const int32_t* __restrict__ Pcol,
                                                      const double* __restrict__ Pval, int W,
                                                      int32_t* __restrict__ Ccol,
                                                      double* __restrict__ Cval,
                                                      int64_t* __restrict__ Clen,
                                                      unsigned int* flags) {
  extern __shared__ __align__(16) char smem[];
  int32_t* hkey = reinterpret_cast<int32_t*>(smem + AbSmem::hkey);
  uint16_t* slot = reinterpret_cast<uint16_t*>(smem + AbSmem::slot);
  uint8_t* hlid = reinterpret_cast<uint8_t*>(smem + AbSmem::hlid);
  double* acc = reinterpret_cast<double*>(smem);
  char* fx = smem + ab_region(W);
  double* vals = reinterpret_cast<double*>(fx + AbSmem::vals);
  double* pa = reinterpret_cast<double*>(fx + AbSmem::pa);
  uint32_t* nmask = reinterpret_cast<uint32_t*>(fx + AbSmem::nmask);
  uint32_t* rmask = reinterpret_cast<uint32_t*>(fx + AbSmem::rmask);
  int32_t* keys = reinterpret_cast<int32_t*>(fx + AbSmem::keys);
  int32_t* lcol = reinterpret_cast<int32_t*>(fx + AbSmem::lcol);
  int32_t* hrow = reinterpret_cast<int32_t*>(fx + AbSmem::hrow);
  int32_t* poff = reinterpret_cast<int32_t*>(fx + AbSmem::poff);
  int32_t* pdir = reinterpret_cast<int32_t*>(fx + AbSmem::pdir);
  int* wsum = reinterpret_cast<int*>(fx + AbSmem::wsum);
  int* ctl = reinterpret_cast<int*>(fx + AbSmem::ctl);   // [0] distinct columns, [1] give up
  uint16_t* kslot = reinterpret_cast<uint16_t*>(fx + AbSmem::kslot);
  uint16_t* hoff = reinterpret_cast<uint16_t*>(fx + AbSmem::hoff);
  uint8_t* elid = reinterpret_cast<uint8_t*>(fx + AbSmem::elid);
  uint8_t* rpre = reinterpret_cast<uint8_t*>(fx + AbSmem::rpre);
  uint8_t* hlen = reinterpret_cast<uint8_t*>(fx + AbSmem::hlen);
  uint8_t* hcnt = reinterpret_cast<uint8_t*>(fx + AbSmem::hcnt);
  const int m = S.m, tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
  const int x0 = blockIdx.x * AB_X, y0 = blockIdx.y * AB_Y, z0 = blockIdx.z * AB_Z;
  const int np = __popc(S.present);
  if (tid < 27 && ((S.present >> tid) & 1u)) {   // the present directions in column order
    const int j = __popc(S.present & ((1u << tid) - 1u));
    pdir[j] = tid;
    poff[j] = tid % 3 + AB_HX * (tid / 3 % 3 + AB_HY * (tid / 9));
    pa[j] = S.a[tid];
  }
  for (int q = tid; q < AB_HASH; q += AB_T) hkey[q] = -1;
  for (int q = tid; q < AB_H * AB_W; q += AB_T) nmask[q] = 0u;
  if (tid == 0) {
    ctl[0] = 0;
    ctl[1] = 0;
  }
  // 1. the halo's P rows (staged entry t of halo row h at t AB_H + h)
  for (int h = tid; h < AB_H; h += AB_T) {
    const int gx = x0 + h % AB_HX - 1, gy = y0 + (h / AB_HX) % AB_HY - 1, gz = z0 + h / (AB_HX * AB_HY) - 1;
    int b = 0, len = 0;
    if ((unsigned)gx < (unsigned)m && (unsigned)gy < (unsigned)m && (unsigned)gz < (unsigned)m) {
      const int64_t g = gx + (int64_t)m * (gy + (int64_t)m * gz);
      b = Prp[g];
      len = Prp[g + 1] - b;
    }
    hrow[h] = b;
    hlen[h] = (uint8_t)min(len, AB_L);
    hcnt[h] = 0;
    if (len > AB_L) ctl[1] = 1;
  }
  __syncthreads();
  // every staged entry's column and value loaded at once; columns into the hash set
  int cst[AB_NIT];
  double vst[AB_NIT];
#pragma unroll
  for (int u = 0; u < AB_NIT; u++) {
    const int it = tid + AB_T * u;
    const int h = it % AB_H, t = it / AB_H;
    const bool ok = it < AB_H * AB_L && t < hlen[h];
    cst[u] = ok ? Pcol[hrow[h] + t] : -1;
    vst[u] = ok ? Pval[hrow[h] + t] : 0.0;
  }
#pragma unroll
  for (int u = 0; u < AB_NIT; u++) {
    const int it = tid + AB_T * u;
    if (it < AB_H * AB_L) {
      uint16_t sl = AB_NONE;
      if (cst[u] >= 0) {
        uint32_t hs = ((uint32_t)cst[u] * 0x9E3779B1u) >> 23;
        for (int probe = 0; probe < AB_HASH; probe++) {
          const int prev = atomicCAS(&hkey[hs], -1, cst[u]);
          if (prev == -1 || prev == cst[u]) {
            sl = (uint16_t)hs;
            break;
          }
          hs = (hs + 1) & (AB_HASH - 1);
        }
        if (sl == AB_NONE) ctl[1] = 1;   // the set is full
        else {
          const int h = it % AB_H;
          atomicAdd(reinterpret_cast<unsigned int*>(hcnt + (h & ~3)), 1u << (8 * (h & 3)));
        }
      }
      slot[it] = sl;
    }
  }
  __syncthreads();
  // 2. local ids (the rank of each distinct column) and the staged rows' offsets
  for (int q = tid; q < AB_HASH; q += AB_T) {
    const int c = hkey[q];
    if (c >= 0) {
      const int u = atomicAdd(&ctl[0], 1);
      if (u < AB_IDS) {
        keys[u] = c;
        kslot[u] = (uint16_t)q;
      }
    }
  }
  {  // exclusive scan of the true entry counts over the staged rows, one per thread
    const int v = tid < AB_H ? hcnt[tid] : 0;
    int incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wsum[wid] = incl;
    __syncthreads();
    int base = 0;
    for (int w = 0; w < wid; w++) base += wsum[w];
    const int ex = base + incl - v;
    if (tid < AB_H) hoff[tid] = (uint16_t)min(ex, 0xFFFF);
    if (tid == AB_T - 1 && ex + v > AB_E) ctl[1] = 1;
  }
  __syncthreads();
  const int nd = ctl[0];
  if (nd > AB_IDS || ctl[1]) {
    if (tid == 0) atomicOr(flags, 2u);
    return;
  }
  if (tid < nd) {
    const int c = keys[tid];
    int rk = 0;
    for (int u = 0; u < nd; u++) rk += keys[u] < c;
    hlid[kslot[tid]] = (uint8_t)rk;
    lcol[rk] = c;
  }
  __syncthreads();
  // each staged row's ids, values and mask (true entries lead a CSR4 row, in column order)
#pragma unroll
  for (int u = 0; u < AB_NIT; u++) {
    const int it = tid + AB_T * u;
    if (it < AB_H * AB_L) {
      const uint16_t sl = slot[it];
      if (sl != AB_NONE) {
        const int h = it % AB_H, t = it / AB_H;
        const int L = hlid[sl];
        atomicOr(&nmask[h * AB_W + (L >> 5)], 1u << (L & 31));
        elid[hoff[h] + t] = (uint8_t)L;
        vals[hoff[h] + t] = vst[u];
      }
    }
  }
  __syncthreads();   // the hash set and the slots are dead from here: the sums' space
  // 3. row tid / 4, lane k of its group
  const int row = tid >> 2, k = tid & 3;
  const unsigned gm = 0xFu << (lane & ~3);
  const int tx = row % AB_X, ty = (row / AB_X) % AB_Y, tz = row / (AB_X * AB_Y);
  const int gx = x0 + tx, gy = y0 + ty, gz = z0 + tz;
  if (gx >= m || gy >= m || gz >= m) return;   // the whole group
  const int64_t r = gx + (int64_t)m * (gy + (int64_t)m * gz);
  const int h0 = tx + AB_HX * (ty + AB_HY * tz);   // halo index of direction d = 0
  uint32_t inb = (1u << np) - 1u;                  // the row's present directions
  if (!(gx >= 1 && gy >= 1 && gz >= 1 && gx <= m - 2 && gy <= m - 2 && gz <= m - 2)) {
    inb = 0u;
    for (int j = 0; j < np; j++)
      if (st_inb(gx, gy, gz, pdir[j], m)) inb |= 1u << j;
  }
  uint32_t rm[AB_W];
#pragma unroll
  for (int w = 0; w < AB_W; w++) rm[w] = 0u;
  for (int j = k; j < np; j += AB_G) {
    if (!((inb >> j) & 1u)) continue;
    const uint4* nm = reinterpret_cast<const uint4*>(nmask + (h0 + poff[j]) * AB_W);
    const uint4 a = nm[0], b = nm[1];
    rm[0] |= a.x; rm[1] |= a.y; rm[2] |= a.z; rm[3] |= a.w;
    rm[4] |= b.x; rm[5] |= b.y; rm[6] |= b.z; rm[7] |= b.w;
  }
  int c = 0;
#pragma unroll
  for (int w = 0; w < AB_W; w++) {
    rm[w] |= __shfl_xor_sync(gm, rm[w], 1, AB_G);
    rm[w] |= __shfl_xor_sync(gm, rm[w], 2, AB_G);
    if ((w & 3) == k) {
      rmask[w * AB_R + row] = rm[w];
      rpre[w * AB_R + row] = (uint8_t)c;
    }
    c += __popc(rm[w]);
  }
  if (c > W) {
    if (k == 0) {
      Clen[r] = c;
      atomicOr(flags, 1u);
    }
    return;
  }
  double* ac = acc + (size_t)row * (W | 1);
  for (int q = k; q < c; q += AB_G) ac[q] = 0.0;
  __syncwarp(gm);
  const uint32_t* rmk = rmask + row;
  const uint8_t* rpr = rpre + row;
  for (int j = 0; j < np; j++) {
    if (!((inb >> j) & 1u)) continue;
    const int h = h0 + poff[j];
    const int n = hcnt[h], o = hoff[h];
    const double a = pa[j];
    for (int e = k; e < n; e += AB_G) {
      const int L = elid[o + e];
      const int w = L >> 5;
      const int p = rpr[w * AB_R] + __popc(rmk[w * AB_R] & ((1u << (L & 31)) - 1u));
      ac[p] = fma(a, vals[o + e], ac[p]);
    }
    __syncwarp(gm);
  }
  int32_t* crow = Ccol + r * W;
  int q = 0;
#pragma unroll
  for (int w = 0; w < AB_W; w++) {
    uint32_t word = rm[w];
    while (word) {
      const int bt = __ffs(word) - 1;
      word &= word - 1;
      if ((q & 3) == k) crow[q] = lcol[w * 32 + bt];
      q++;
    }
  }
  double* vrow = Cval + r * W;
  for (int u = k; u < c; u += AB_G) vrow[u] = ac[u];
  if (k == 0) Clen[r] = c;
}

}  // namespace

// ------------------------------------------------------------------ host wrappers

static int64_t max_of(const int64_t* v, int64_t n, cudaStream_t st) {
  DevBuf<unsigned long long> m(1, st);
  FEM_CUDA(cudaMemsetAsync(m, 0, 8, st));
  if (n > 0) {
    k_max_i64<<<persistent_grid(n, 256, 4), 256, 0, st>>>(v, n, m);
    FEM_CHECK_LAUNCH();
  }
  unsigned long long h = 0;
  FEM_CUDA(cudaMemcpyAsync(&h, m, 8, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  return (int64_t)h;
}

// Widest needed group first; wider groups (fewer per block) when the tables of a
// 256-thread block would not fit in 200 KB of shared memory.
static int group_for_smem(int G, int ht, int bytes_per_slot) {
  while (G < 32 && (size_t)(SG_BLOCK / G) * ht * bytes_per_slot > 200 * 1024) G <<= 1;
  return G;
}

static int pow2_at_least(int64_t v, int lo) {
  int64_t t = lo;
  while (t < v) t <<= 1;
  return (int)t;
}

template <int G, int HT>
static void sg_count_launch(int64_t nr, const Csr4& A, const Csr4& B, const int64_t* rows,
                            int64_t* cnt, cudaStream_t st) {
  const size_t smem = (size_t)(SG_BLOCK / G) * HT * 4;
  static bool attr = false;
  if (!attr) {
    FEM_CUDA(cudaFuncSetAttribute(k_sg_count<G, HT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    attr = true;
  }
  unsigned g = (unsigned)((nr + SG_BLOCK / G - 1) / (SG_BLOCK / G));
  k_sg_count<G, HT><<<g, SG_BLOCK, smem, st>>>(nr, A.rowptr, A.col, B.rowptr, B.col, rows, cnt);
  FEM_CHECK_LAUNCH();
}

template <int G, int HT>
static void sg_fill_launch(int64_t nr, const Csr4& A, const double* Aval, const Csr4& B,
                           const double* Bval, Csr4& C, double* Cval, cudaStream_t st) {
  const size_t smem = (size_t)(SG_BLOCK / G) * HT * 14;
  static bool attr = false;
  if (!attr) {
    FEM_CUDA(cudaFuncSetAttribute(k_sg_fill<G, HT>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    attr = true;
  }
  unsigned g = (unsigned)((nr + SG_BLOCK / G - 1) / (SG_BLOCK / G));
  k_sg_fill<G, HT><<<g, SG_BLOCK, smem, st>>>(nr, A.rowptr, A.col, Aval, B.rowptr, B.col, Bval,
                                              C.rowptr, C.col, Cval);
  FEM_CHECK_LAUNCH();
}

template <int G>
static void sg_count_ht(int ht, int64_t nr, const Csr4& A, const Csr4& B, const int64_t* rows,
                        int64_t* cnt, cudaStream_t st) {
  switch (ht) {
    case 64: sg_count_launch<G, 64>(nr, A, B, rows, cnt, st); break;
    case 128: sg_count_launch<G, 128>(nr, A, B, rows, cnt, st); break;
    case 256: sg_count_launch<G, 256>(nr, A, B, rows, cnt, st); break;
    case 512: sg_count_launch<G, 512>(nr, A, B, rows, cnt, st); break;
    default: sg_count_launch<G, 1024>(nr, A, B, rows, cnt, st); break;
  }
}

// count pass over nr rows (or the listed ones) with hash tables of ht slots
static void sg_count(int G, int ht, int64_t nr, const Csr4& A, const Csr4& B,
                     const int64_t* rows, int64_t* cnt, cudaStream_t st) {
  switch (group_for_smem(G, ht, 4)) {
    case 4: sg_count_ht<4>(ht, nr, A, B, rows, cnt, st); break;
    case 8: sg_count_ht<8>(ht, nr, A, B, rows, cnt, st); break;
    case 16: sg_count_ht<16>(ht, nr, A, B, rows, cnt, st); break;
    default: sg_count_ht<32>(ht, nr, A, B, rows, cnt, st); break;
  }
}

template <int G>
static void sg_fill_ht(int ht, int64_t nr, const Csr4& A, const double* Aval, const Csr4& B,
                       const double* Bval, Csr4& C, double* Cval, cudaStream_t st) {
  switch (ht) {
    case 64: sg_fill_launch<G, 64>(nr, A, Aval, B, Bval, C, Cval, st); break;
    case 128: sg_fill_launch<G, 128>(nr, A, Aval, B, Bval, C, Cval, st); break;
    case 256: sg_fill_launch<G, 256>(nr, A, Aval, B, Bval, C, Cval, st); break;
    case 512: sg_fill_launch<G, 512>(nr, A, Aval, B, Bval, C, Cval, st); break;
    default: sg_fill_launch<G, 1024>(nr, A, Aval, B, Bval, C, Cval, st); break;
  }
}

void spgemm(const Csr4& A, const double* Aval, const Csr4& B, const double* Bval, Csr4& C,
            cudaStream_t st, bool values, bool* too_long, int64_t limit) {
  const int64_t nr = A.nrows;
  C.nrows = A.nrows;
  C.ncols = B.ncols;
  DevBuf<int64_t> cnt(nr > 0 ? nr : 1, st);
  int G = 32, htc = 64;
  int64_t nlong = 0;
  DevBuf<int64_t> llist, loff, ltsz;
  DevBuf<int32_t> lkeys;
  DevBuf<int64_t> tmp(std::max<int64_t>(nr, B.nrows) + 1, st);
  if (nr > 0) {
    // group width from B's longest row, count-table size from the product bound
    k_row_len<<<grid_for(B.nrows, 256), 256, 0, st>>>(B.nrows, B.rowptr, tmp);
    FEM_CHECK_LAUNCH();
    const int64_t maxb = max_of(tmp, B.nrows, st);
    k_row_ub<<<grid_for(nr, 256), 256, 0, st>>>(nr, A.rowptr, A.col, B.rowptr, tmp);
    FEM_CHECK_LAUNCH();
    const int64_t maxub = max_of(tmp, nr, st);
    G = maxb <= 4 ? 4 : (maxb <= 8 ? 8 : (maxb <= 16 ? 16 : 32));
    htc = pow2_at_least(std::min<int64_t>(2 * maxub, kHTMax), 64);
    if (htc > 64 && nr > 4 * kSgSample) {
      // the bound overestimates the distinct columns several times over, and clearing and
      // holding the tables is most of the count's work: size the tables from an exact count
      // of evenly spaced sample rows, then count again (with full tables) the rows whose
      // table filled up
      DevBuf<int64_t> srow(kSgSample, st), sval(kSgSample, st);
      k_sample_rows<<<grid_for(kSgSample, 256), 256, 0, st>>>(nr, kSgSample, srow);
      FEM_CHECK_LAUNCH();
      sg_count(G, htc, kSgSample, A, B, srow, cnt, st);   // counts land in cnt[sampled row]
      k_gather_i64<<<grid_for(kSgSample, 256), 256, 0, st>>>(kSgSample, srow, cnt, sval);
      FEM_CHECK_LAUNCH();
      const int64_t smax = max_of(sval, kSgSample, st);
      const int hts = pow2_at_least(std::min<int64_t>(4 * smax, htc), 64);
      if (hts < htc) {
        sg_count(G, hts, nr, A, B, nullptr, cnt, st);
        DevBuf<int64_t> flag(nr, st), scan(nr + 1, st);
        k_long_flag<<<grid_for(nr, 256), 256, 0, st>>>(nr, cnt, hts - 1, flag);
        FEM_CHECK_LAUNCH();
        const int64_t nfull = exclusive_scan(flag, nr, scan, st);
        if (nfull > 0) {
          DevBuf<int64_t> list(nfull, st);
          k_flag_list<<<grid_for(nr, 256), 256, 0, st>>>(nr, flag, scan, list);
          FEM_CHECK_LAUNCH();
          sg_count(G, htc, nfull, A, B, list, cnt, st);
        }
      } else {
        sg_count(G, htc, nr, A, B, nullptr, cnt, st);
      }
    } else {
      sg_count(G, htc, nr, A, B, nullptr, cnt, st);
    }
    if (maxub > kHTMax / 2) {
      // rows whose count reached half a table (exact up to kHTMax, saturated beyond): count
      // them again with a global table each
      DevBuf<int64_t> flag(nr, st), scan(nr + 1, st);
      k_long_flag<<<grid_for(nr, 256), 256, 0, st>>>(nr, cnt, kHTMax / 2, flag);
      FEM_CHECK_LAUNCH();
      nlong = exclusive_scan(flag, nr, scan, st);
      if (nlong > 0) {
        llist.alloc_async(nlong, st);
        ltsz.alloc_async(nlong, st);
        loff.alloc_async(nlong + 1, st);
        k_long_list<<<grid_for(nr, 256), 256, 0, st>>>(nr, flag, scan, tmp, llist, ltsz);
        FEM_CHECK_LAUNCH();
        const int64_t total = exclusive_scan(ltsz, nlong, loff, st);
        if (total > ((int64_t)1 << 31) && too_long) {
          *too_long = true;
          return;
        }
        FEM_REQUIRE(total <= ((int64_t)1 << 31), FEM_EUNSUPPORTED,
                    "spgemm: long product rows need more than 8 GB of hash tables");
        lkeys.alloc_async(total, st);
        k_long_count<<<(unsigned)nlong, kLongBlock, 0, st>>>(llist, loff, ltsz, A.rowptr, A.col,
                                                             B.rowptr, B.col, lkeys, cnt);
        FEM_CHECK_LAUNCH();
      }
    }
  }
  const int64_t maxc = nr > 0 ? max_of(cnt, nr, st) : 0;
  if (too_long && maxc > std::min<int64_t>(limit, kLongRowMax)) {
    *too_long = true;
    return;
  }
  FEM_REQUIRE(maxc <= kLongRowMax, FEM_EUNSUPPORTED,
              "spgemm: a product row has more than 8192 distinct columns");
  rowptr_from_counts(cnt, nr, C, st);
  if (values) C.val.alloc(C.nnz);
  if (nlong > 0) {
    const size_t smem = 12 * (size_t)kLongRowMax;
    static bool attr = false;
    if (!attr) {
      FEM_CUDA(cudaFuncSetAttribute(k_long_fill, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)smem));
      attr = true;
    }
    k_long_fill<<<(unsigned)nlong, kLongBlock, smem, st>>>(
        llist, loff, ltsz, cnt, A.rowptr, A.col, Aval, B.rowptr, B.col, Bval, C.rowptr, C.col,
        values ? C.val.p : nullptr, lkeys);
    FEM_CHECK_LAUNCH();
  }
  if (nr > 0) {
    const int htf = pow2_at_least(2 * std::min<int64_t>(maxc, kHTMax / 2), 64);
    double* cv = values ? C.val.p : nullptr;
    switch (group_for_smem(G, htf, 14)) {
      case 4: sg_fill_ht<4>(htf, nr, A, Aval, B, Bval, C, cv, st); break;
      case 8: sg_fill_ht<8>(htf, nr, A, Aval, B, Bval, C, cv, st); break;
      case 16: sg_fill_ht<16>(htf, nr, A, Aval, B, Bval, C, cv, st); break;
      default: sg_fill_ht<32>(htf, nr, A, Aval, B, Bval, C, cv, st); break;
    }
  }
}

// C's pattern must be that of A*B.
void spgemm_numeric(const Csr4& A, const double* Aval, const Csr4& B, const double* Bval,
                    const Csr4& C, double* Cval, cudaStream_t st) {
  const int64_t nr = A.nrows;
  if (nr == 0) return;
  unsigned g = (unsigned)((nr + SG_WARPS - 1) / SG_WARPS);
  k_spgemm_numeric<<<g, 32 * SG_WARPS, 0, st>>>(nr, A.rowptr, A.col, Aval, B.rowptr, B.col,
                                                Bval, C.rowptr, C.col, Cval);
  FEM_CHECK_LAUNCH();
}

static int64_t row_sum(const int64_t* len, int64_t n, cudaStream_t st) {
  DevBuf<int64_t> scan(n + 1, st);
  return exclusive_scan(len, n, scan, st);
}

// A product at a fixed stride: column indices, values and row lengths.
struct Strided {
  int64_t nrows = 0;
  int32_t ncols = 0, W = 0;
  int64_t maxlen = 0;
  DevBuf<int32_t> col;
  DevBuf<double> val;
  DevBuf<int64_t> len;
};

static size_t mg_smem(int G, int K, int W, int lmax) {
  return (size_t)(MG_BLOCK / G) * ((size_t)(W + 1) * 8 + (size_t)G * K * lmax + 4 + (size_t)G * K * 4);
}

template <int G, int K>
static void mg_launch(int64_t nr, const int64_t* rlist, const Csr4& A, const double* Aval,
                      MgRows Brows, const int32_t* Bcol, const double* Bval, int lmax,
                      Strided& C, unsigned int* ovf, int upper, cudaStream_t st) {
  const unsigned g = (unsigned)((nr + MG_BLOCK / G - 1) / (MG_BLOCK / G));
  const size_t smem = mg_smem(G, K, C.W, lmax);
  static size_t attr = 48 * 1024;
  if (smem > attr) {
    FEM_CUDA(cudaFuncSetAttribute(k_mg<G, K>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    attr = smem;
  }
  k_mg<G, K><<<g, MG_BLOCK, smem, st>>>(nr, rlist, A.rowptr, A.col, Aval, Brows, Bcol, Bval, C.W,
                                        lmax, C.col, C.val, C.len, ovf, upper);
  FEM_CHECK_LAUNCH();
}

template <int G>
static void mg_launch_k(int K, int64_t nr, const int64_t* rlist, const Csr4& A, const double* Aval,
                        MgRows Brows, const int32_t* Bcol, const double* Bval, int lmax,
                        Strided& C, unsigned int* ovf, int upper, cudaStream_t st) {
  switch (K) {
    case 2: mg_launch<G, 2>(nr, rlist, A, Aval, Brows, Bcol, Bval, lmax, C, ovf, upper, st); break;
    case 4: mg_launch<G, 4>(nr, rlist, A, Aval, Brows, Bcol, Bval, lmax, C, ovf, upper, st); break;
    case 8: mg_launch<G, 8>(nr, rlist, A, Aval, Brows, Bcol, Bval, lmax, C, ovf, upper, st); break;
    default: mg_launch<G, 16>(nr, rlist, A, Aval, Brows, Bcol, Bval, lmax, C, ovf, upper, st); break;
  }
}

// stride last used for a product of this shape (the next set-up of the same system starts
// from it); dflt for a new shape
static int mg_stride_guess(uint64_t key, int set, int dflt = 32) {
  static std::mutex mu;
  static std::unordered_map<uint64_t, int> seen;
  std::lock_guard<std::mutex> lk(mu);
  if (set > 0) {
    seen[key] = set;
    return set;
  }
  auto it = seen.find(key);
  return it == seen.end() ? dflt : it->second;
}

// C = A B by the merge kernel, C at a fixed stride.  B's rows: CSR4 (Bs null) or the
// strided product Bs.  Returns false when the kernel cannot take the product (an A row
// beyond 16 x 32 entries, B rows beyond 255 entries, or tables beyond the shared memory):
// the caller takes the hash path.
static bool spgemm_merge(const Csr4& A, const double* Aval, const Csr4* Bc, const double* Bval,
                         const Strided* Bs, Strided& C, cudaStream_t st,
                         const int64_t* rlist = nullptr, int64_t nlist = 0, int upper = 0) {
  const int64_t nr = A.nrows;
  const int64_t nb = Bc ? Bc->nrows : Bs->nrows;
  if (nr == 0 || nb == 0 || (upper && Bc)) return false;   // (upper part: unpadded B rows)
  DevBuf<int64_t> len(nr, st);
  k_row_len<<<grid_for(nr, 256), 256, 0, st>>>(nr, A.rowptr, len);
  FEM_CHECK_LAUNCH();
  const int64_t maxa = max_of(len, nr, st);
  int64_t lmax;
  MgRows R{};
  if (Bc) {
    DevBuf<int64_t> blen(nb, st);
    k_row_len<<<grid_for(nb, 256), 256, 0, st>>>(nb, Bc->rowptr, blen);
    FEM_CHECK_LAUNCH();
    lmax = max_of(blen, nb, st);
    R.rp = Bc->rowptr;
  } else {
    lmax = Bs->maxlen;
    R.len = Bs->len;
    R.stride = Bs->W;
  }
  if (lmax > 255 || lmax < 1) return false;
  lmax = (lmax + 3) & ~(int64_t)3;
  // lanes per row from B's mean row (the lanes split B rows; CSR4 padding adds 1.5 stored
  // entries per row on average), wide enough that K <= 16 lists per lane cover the longest
  // A row
  const double meanb = Bc ? (double)Bc->nnz / (double)nb - 1.5 : 0.6 * (double)Bs->maxlen;
  int G = 4;
  while (G < 32 && (G < meanb || (int64_t)G * 16 < maxa)) G <<= 1;
  if ((int64_t)G * 16 < maxa) return false;
  int K = 2;
  while ((int64_t)G * K < maxa) K <<= 1;
  const int64_t bcols = Bc ? Bc->ncols : Bs->ncols;
  const uint64_t key = (uint64_t)nr * 0x9E3779B97F4A7C15ull ^ (uint64_t)A.nnz * 0xC2B2AE3D27D4EB4Full ^
                       (uint64_t)nb * 0x165667B19E3779F9ull ^ (uint64_t)bcols ^ (uint64_t)upper << 63;
  int W = mg_stride_guess(key, 0);
  DevBuf<unsigned int> ovf(1, st);
  for (int attempt = 0; attempt < 2; attempt++) {
    if (mg_smem(G, K, W, (int)lmax) > 200 * 1024 || nr * (int64_t)W >= ((int64_t)1 << 31) ||
        W > 255)
      return false;
    C.nrows = nr;
    C.ncols = (int32_t)bcols;
    C.W = W;
    C.col.alloc_async((size_t)nr * W, st);
    C.val.alloc_async((size_t)nr * W, st);
    C.len.alloc_async(nr, st);
    FEM_CUDA(cudaMemsetAsync(ovf, 0, 4, st));
    // only the listed rows (when a list is given): the others stay empty
    if (rlist) FEM_CUDA(cudaMemsetAsync(C.len, 0, 8 * nr, st));
    const int64_t nrun = rlist ? nlist : nr;
    const int32_t* bcol = Bc ? Bc->col.p : Bs->col.p;
    if (nrun > 0) {
      switch (G) {
        case 4: mg_launch_k<4>(K, nrun, rlist, A, Aval, R, bcol, Bval, (int)lmax, C, ovf, upper, st); break;
        case 8: mg_launch_k<8>(K, nrun, rlist, A, Aval, R, bcol, Bval, (int)lmax, C, ovf, upper, st); break;
        case 16: mg_launch_k<16>(K, nrun, rlist, A, Aval, R, bcol, Bval, (int)lmax, C, ovf, upper, st); break;
        default: mg_launch_k<32>(K, nrun, rlist, A, Aval, R, bcol, Bval, (int)lmax, C, ovf, upper, st); break;
      }
    }
    C.maxlen = max_of(C.len, nr, st);
    unsigned int hov = 0;
    FEM_CUDA(cudaMemcpyAsync(&hov, ovf, 4, cudaMemcpyDeviceToHost, st));
    FEM_CUDA(cudaStreamSynchronize(st));
    if (!hov) {
      mg_stride_guess(key, W);
      return true;
    }
    W = 4;
    while (W < C.maxlen) W <<= 1;
  }
  return false;
}

// A P on the uniform finest level by the brick kernel, at a fixed stride.  Returns false
// when the kernel cannot take it (P rows beyond its staging, a brick beyond its limits):
// the caller takes the merge kernel.
static bool ap_brick(const StencilRow& S, const Csr4& P, Strided& C, cudaStream_t st) {
  const int m = S.m;
  const int64_t nr = P.nrows;
  if (m < 3 || (int64_t)m * m * m != nr || nr == 0) return false;
  {
    DevBuf<int64_t> plen(nr, st);
    k_row_len<<<grid_for(nr, 256), 256, 0, st>>>(nr, P.rowptr, plen);
    FEM_CHECK_LAUNCH();
    if (max_of(plen, nr, st) > AB_L) return false;
  }
  const uint64_t key = (uint64_t)nr * 0xD6E8FEB86659FD93ull ^ (uint64_t)P.nnz * 0x9E3779B97F4A7C15ull ^
                       (uint64_t)P.ncols ^ 0xABull;
  // rows of the uniform level's A P hold about 13 entries, 21 at most at 255^3
  int W = mg_stride_guess(key, 0, 24);
  static size_t attr = 48 * 1024;
  DevBuf<unsigned int> flags(1, st);
  const dim3 grid((unsigned)((m + AB_X - 1) / AB_X), (unsigned)((m + AB_Y - 1) / AB_Y),
                  (unsigned)((m + AB_Z - 1) / AB_Z));
  for (int attempt = 0; attempt < 2; attempt++) {
    const size_t smem = ab_smem(W);
    if (smem > 200 * 1024 || nr * (int64_t)W >= ((int64_t)1 << 31) || W > 255) return false;
    if (smem > attr) {
      FEM_CUDA(cudaFuncSetAttribute(k_ap_brick, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      attr = smem;
    }
    C.nrows = nr;
    C.ncols = P.ncols;
    C.W = W;
    C.col.alloc_async((size_t)nr * W, st);
    C.val.alloc_async((size_t)nr * W, st);
    C.len.alloc_async(nr, st);
    FEM_CUDA(cudaMemsetAsync(flags, 0, 4, st));
    k_ap_brick<<<grid, AB_T, smem, st>>>(S, P.rowptr, P.col, P.val, W, C.col, C.val, C.len, flags);
    FEM_CHECK_LAUNCH();
    unsigned int hf = 0;
    FEM_CUDA(cudaMemcpyAsync(&hf, flags, 4, cudaMemcpyDeviceToHost, st));
    FEM_CUDA(cudaStreamSynchronize(st));
    if (hf & 2u) return false;
    C.maxlen = max_of(C.len, nr, st);
    if (!hf) {
      // the next product of this shape starts from the stride its rows need
      mg_stride_guess(key, std::max(4, (int)((C.maxlen + 3) & ~3)));
      return true;
    }
    W = (int)((C.maxlen + 3) & ~3);
  }
  return false;
}

static bool sort_rows(int64_t nrows, const int32_t* rp, const int64_t* cnt, int32_t* col,
                      double* val, cudaStream_t st);

// Galerkin product A_c = R (A P) by the merge kernels (A P at a fixed stride: the brick kernel
// on the uniform finest level; the upper part of A_c merged, its lower part mirrored, CSR4).
// Returns false when the kernels cannot take it (the hash path then runs); sets *too_long
// when A P or A_c has a row longer than limit; *ap_entries (if given) receives the entries of
// A P.
bool galerkin_merge(const Csr4& A, const Csr4& P, const Csr4& R, Csr4& Ac, cudaStream_t st,
                    bool* too_long, int64_t limit, int64_t* ap_entries, const StencilRow* sr) {
  Strided AP, RAP;
  // R (A P) reads the rows of A P that R's columns name, those of the nonempty rows of P:
  // where many rows of P are empty (isolated nodes on the coarser levels), A P is formed on
  // those rows only
  DevBuf<int64_t> rlist;
  int64_t nlist = 0;
  if (!sr) {   // (the uniform finest level: every node has an aggregate)
    const int64_t nr = P.nrows;
    DevBuf<int64_t> plen(nr, st), flag(nr, st), scan(nr + 1, st);
    k_row_len<<<grid_for(nr, 256), 256, 0, st>>>(nr, P.rowptr, plen);
    FEM_CHECK_LAUNCH();
    k_long_flag<<<grid_for(nr, 256), 256, 0, st>>>(nr, plen, 0, flag);
    FEM_CHECK_LAUNCH();
    nlist = exclusive_scan(flag, nr, scan, st);
    if (4 * nlist < 3 * nr) {
      rlist.alloc_async(std::max<int64_t>(nlist, 1), st);
      k_flag_list<<<grid_for(nr, 256), 256, 0, st>>>(nr, flag, scan, rlist);
      FEM_CHECK_LAUNCH();
    }
  }
  if (!(sr && ap_brick(*sr, P, AP, st)) &&
      !spgemm_merge(A, A.val, &P, P.val, nullptr, AP, st, rlist.p, nlist))
    return false;
  if (ap_entries) *ap_entries = row_sum(AP.len, AP.nrows, st);
  if (AP.maxlen > limit) {
    *too_long = true;
    return true;
  }
  // A_c is symmetric (A is, and R = P^T): the merge forms its upper part (columns >= row),
  // the lower part is that part's transpose
  if (!spgemm_merge(R, R.val, nullptr, AP.val, &AP, RAP, st, nullptr, 0, 1)) return false;
  AP = Strided();
  const int64_t nc = RAP.nrows;
  DevBuf<unsigned long long> lcnt(nc, st), fill(nc, st);
  FEM_CUDA(cudaMemsetAsync(lcnt, 0, 8 * nc, st));
  FEM_CUDA(cudaMemsetAsync(fill, 0, 8 * nc, st));
  const unsigned gw = grid_for(nc * 32, 256);
  k_u_count<<<gw, 256, 0, st>>>(nc, RAP.W, RAP.col, RAP.len, lcnt);
  FEM_CHECK_LAUNCH();
  DevBuf<int64_t> lower(nc, st), total(nc, st);
  k_u_len<<<grid_for(nc, 256), 256, 0, st>>>(nc, lcnt, RAP.len, lower, total);
  FEM_CHECK_LAUNCH();
  if (max_of(total, nc, st) > limit) {
    *too_long = true;
    return true;
  }
  Ac.nrows = (int32_t)nc;
  Ac.ncols = P.ncols;
  rowptr_from_counts(total, nc, Ac, st);
  Ac.val.alloc(Ac.nnz);
  k_u_scatter<<<gw, 256, 0, st>>>(nc, RAP.W, RAP.col, RAP.val, RAP.len, Ac.rowptr, fill, Ac.col,
                                  Ac.val);
  FEM_CHECK_LAUNCH();
  FEM_REQUIRE(sort_rows(nc, Ac.rowptr, lower, Ac.col, Ac.val, st), FEM_EUNSUPPORTED,
              "Galerkin product: a coarse row has more than 8192 entries");
  k_u_upper<<<gw, 256, 0, st>>>(nc, RAP.W, RAP.col, RAP.val, RAP.len, Ac.rowptr, lower, Ac.col,
                                Ac.val);
  FEM_CHECK_LAUNCH();
  return true;
}

namespace {
bool stencil_row(const Csr4& A, int m, double theta, StencilRow& R, cudaStream_t st);
}  // namespace

double galerkin_timed(const Hierarchy& H, int lev, int reps, cudaStream_t st,
                      int64_t* ap_entries) {
  FEM_REQUIRE(lev >= 0 && lev < (int)H.L.size() && !H.L[lev]->coarsest, FEM_EINVAL,
              "amg_galerkin_timed: level without a coarse operator");
  const Level& L = *H.L[lev];
  FEM_REQUIRE(L.A && L.A->val.p && L.A->nnz > 0, FEM_EINVAL,
              "amg_galerkin_timed: the level keeps no FP64 matrix");
  // the uniform finest level's A P from the stencil, as the set-up takes it
  StencilRow SR;
  const bool sr = lev == 0 && L.stencil && stencil_row(*L.A, L.st.m, H.o.theta, SR, st);
  cudaEvent_t e0, e1;
  FEM_CUDA(cudaEventCreate(&e0));
  FEM_CUDA(cudaEventCreate(&e1));
  double ms_sum = 0.0;
  for (int rep = -1; rep < reps; rep++) {   // one untimed product first
    Csr4 Ac;
    bool too_long = false;
    FEM_CUDA(cudaEventRecord(e0, st));
    int64_t ape = 0;
    const bool merged = galerkin_merge(*L.A, L.P, L.R, Ac, st, &too_long, kLongRowMax, &ape,
                                       sr ? &SR : nullptr);
    if (!merged && !too_long) {
      Csr4 AP;
      spgemm(*L.A, L.A->val, L.P, L.P.val, AP, st, true);
      spgemm(L.R, L.R.val, AP, AP.val, Ac, st, true);
      ape = AP.nnz;
    }
    FEM_CUDA(cudaEventRecord(e1, st));
    FEM_CUDA(cudaEventSynchronize(e1));
    float ms = 0.f;
    cudaEventElapsedTime(&ms, e0, e1);
    if (rep >= 0) ms_sum += ms;
    if (ap_entries) *ap_entries = ape;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ms_sum / reps;
}

// Sort the first cnt[r] entries of every row r by column and pad the rest of the row: warp
// rank sorts for rows of up to 128 and up to TMAX entries, a block bitonic sort beyond.
// Returns false when a row holds more than kLongRowMax entries (left unsorted).
static bool sort_rows(int64_t nrows, const int32_t* rp, const int64_t* cnt, int32_t* col,
                      double* val, cudaStream_t st) {
  if (nrows <= 0) return true;
  DevBuf<unsigned long long> err(1, st);
  FEM_CUDA(cudaMemsetAsync(err, 0, 8, st));
  const unsigned g = (unsigned)((nrows + 3) / 4);
  k_sort_rows<128><<<g, 128, 0, st>>>(nrows, rp, cnt, -1, col, val, err);
  FEM_CHECK_LAUNCH();
  unsigned long long he = 0;
  FEM_CUDA(cudaMemcpyAsync(&he, err, 8, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  if (!he) return true;
  FEM_CUDA(cudaMemsetAsync(err, 0, 8, st));
  k_sort_rows<TMAX><<<g, 128, 0, st>>>(nrows, rp, cnt, 128, col, val, err);
  FEM_CHECK_LAUNCH();
  FEM_CUDA(cudaMemcpyAsync(&he, err, 8, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  if (!he) return true;
  FEM_CUDA(cudaMemsetAsync(err, 0, 8, st));
  const size_t smem = 12 * (size_t)kLongRowMax;
  static bool attr = false;
  if (!attr) {
    FEM_CUDA(cudaFuncSetAttribute(k_sort_long, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)smem));
    attr = true;
  }
  k_sort_long<<<(unsigned)nrows, kLongBlock, smem, st>>>(nrows, rp, cnt, TMAX, col, val, err);
  FEM_CHECK_LAUNCH();
  FEM_CUDA(cudaMemcpyAsync(&he, err, 8, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  return he == 0;
}

void transpose(const Csr4& A, Csr4& T, int64_t ncols, cudaStream_t st, bool* too_long,
               int64_t limit) {
  T.nrows = (int32_t)ncols;
  T.ncols = A.nrows;
  DevBuf<unsigned long long> cnt(ncols, st), fill(ncols, st);
  FEM_CUDA(cudaMemsetAsync(cnt, 0, 8 * ncols, st));
  FEM_CUDA(cudaMemsetAsync(fill, 0, 8 * ncols, st));
  if (A.nnz > 0) {
    k_col_count<<<grid_for(A.nnz, 256), 256, 0, st>>>(A.nnz, A.col, cnt);
    FEM_CHECK_LAUNCH();
  }
  DevBuf<int64_t> c64(ncols, st);
  if (ncols > 0) {
    k_u64_to_i64<<<grid_for(ncols, 256), 256, 0, st>>>(ncols, cnt, c64);
    FEM_CHECK_LAUNCH();
  }
  if (too_long && ncols > 0 && max_of(c64, ncols, st) > std::min<int64_t>(limit, kLongRowMax)) {
    *too_long = true;
    return;
  }
  rowptr_from_counts(c64, ncols, T, st);
  T.val.alloc(T.nnz);
  if (A.nrows > 0) {
    k_scatter_t<<<grid_for(A.nrows, 256), 256, 0, st>>>(A.nrows, A.rowptr, A.col, A.val, T.rowptr,
                                                        fill, T.col, T.val);
    FEM_CHECK_LAUNCH();
  }
  if (!sort_rows(ncols, T.rowptr, c64, T.col, T.val, st)) {
    if (too_long) {
      *too_long = true;
      return;
    }
    FEM_REQUIRE(false, FEM_EUNSUPPORTED, "transpose: a row has more than 8192 entries");
  }
}

static double rowabs_max(const Csr4& A, const double* val, const uint8_t* mask, const double* d,
                         double* l1, cudaStream_t st) {
  const int64_t N = A.nrows;
  unsigned g = grid_for(N, 256);
  DevBuf<double> bmax(g, st), out(1, st);
  k_rowabs<<<g, 256, 0, st>>>(N, A.rowptr, A.col, val, mask, d, bmax, l1);
  FEM_CHECK_LAUNCH();
  k_max_reduce<<<1, 1024, 0, st>>>(bmax, (int)g, out);
  FEM_CHECK_LAUNCH();
  double h = 0;
  FEM_CUDA(cudaMemcpyAsync(&h, out, 8, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  return h;
}

double gershgorin(const Csr4& A, const double* val, cudaStream_t st) {
  DevBuf<double> d(A.nrows, st);
  k_diag<<<grid_for((int64_t)A.nrows * DG_G, 256), 256, 0, st>>>(A.nrows, A.rowptr, A.col, val, d);
  FEM_CHECK_LAUNCH();
  return rowabs_max(A, val, nullptr, d, nullptr, st);
}

void dense_inverse(const Csr4& A, const double* val, DevBuf<double>& Ainv, cudaStream_t st) {
  const int64_t N = A.nrows;
  Ainv.alloc(N * N);
  if (N == 0) return;
  DevBuf<double> other(N * N, st);
  k_dense_from_csr<<<grid_for(N, 128), 128, 0, st>>>(N, A.rowptr, A.col, val, Ainv);
  FEM_CHECK_LAUNCH();
  double* src = Ainv.p;
  double* dst = other.p;
  const unsigned g = persistent_grid(N * N, 256, 4);
  for (int64_t k = 0; k < N; k++) {
    k_gj_step<<<g, 256, 0, st>>>(N, k, src, dst);
    FEM_CHECK_LAUNCH();
    std::swap(src, dst);
  }
  if (src != Ainv.p)
    FEM_CUDA(cudaMemcpyAsync(Ainv.p, src, 8 * N * N, cudaMemcpyDeviceToDevice, st));
}

namespace {

struct Aggregation {
  DevBuf<int32_t> agg;
  DevBuf<uint8_t> smask;
  int64_t nagg = 0;
};

Aggregation aggregate(const Csr4& A, const double* d, double theta, uint32_t seed_s,
                      cudaStream_t st) {
  const int64_t N = A.nrows;
  Aggregation R;
  R.smask.alloc(A.nnz);
  DevBuf<int64_t> scount(N, st), sptr(N + 1, st);
  unsigned g = grid_for(N, 256);
  DevBuf<double> sq(N, st);
  k_sqrt<<<g, 256, 0, st>>>(N, d, sq);
  FEM_CHECK_LAUNCH();
  const unsigned gs = grid_for(N * ST_G, 256);
  k_strength<<<gs, 256, 0, st>>>(N, A.rowptr, A.col, A.val, sq, theta, R.smask, scount);
  FEM_CHECK_LAUNCH();
  int64_t snnz = exclusive_scan(scount, N, sptr, st);
  DevBuf<int32_t> scol(snnz > 0 ? snnz : 1, st);
  k_strength_fill<<<gs, 256, 0, st>>>(N, A.rowptr, A.col, R.smask, sptr, scol);
  FEM_CHECK_LAUNCH();
  DevBuf<uint8_t> s0(N, st), s1(N, st);
  DevBuf<uint64_t> m1(N, st);
  DevBuf<unsigned long long> und(1, st);
  k_mis_init<<<g, 256, 0, st>>>(N, sptr, s0);
  FEM_CHECK_LAUNCH();
  uint8_t* cur = s0;
  uint8_t* nxt = s1;
  bool finished = false;
  for (int round = 0; round < 10000; round++) {
    FEM_CUDA(cudaMemsetAsync(und, 0, 8, st));
    k_mis_m1<<<g, 256, 0, st>>>(N, sptr, scol, cur, seed_s, m1);
    FEM_CHECK_LAUNCH();
    k_mis_m2<<<g, 256, 0, st>>>(N, sptr, scol, m1, seed_s, cur, nxt, und);
    FEM_CHECK_LAUNCH();
    std::swap(cur, nxt);
    unsigned long long hu = 0;
    FEM_CUDA(cudaMemcpyAsync(&hu, und, 8, cudaMemcpyDeviceToHost, st));
    FEM_CUDA(cudaStreamSynchronize(st));
    if (hu == 0) {
      finished = true;
      break;
    }
  }
  FEM_REQUIRE(finished, FEM_EDEVCHECK, "aggregation: MIS-2 did not terminate");
  DevBuf<int64_t> rootid(N + 1, st);
  R.nagg = count_scan_eq(cur, ST_IN, N, rootid, st);
  R.agg.alloc(N);
  DevBuf<uint8_t> p1(N, st);
  DevBuf<unsigned long long> err(1, st);
  FEM_CUDA(cudaMemsetAsync(err, 0, 8, st));
  k_agg_phase1<<<g, 256, 0, st>>>(N, sptr, scol, cur, rootid, R.agg, p1, err);
  FEM_CHECK_LAUNCH();
  k_agg_phase2<<<g, 256, 0, st>>>(N, sptr, scol, p1, R.agg, err);
  FEM_CHECK_LAUNCH();
  unsigned long long he = 0;
  FEM_CUDA(cudaMemcpyAsync(&he, err, 8, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  FEM_REQUIRE(he == 0, FEM_EDEVCHECK, "aggregation: inconsistent MIS-2 / aggregate assignment");
  return R;
}

// ------------------------------------------------------------------ red-black coarsening

// The paper's coarsening (Sec. 3.1, after KF1998): visit the unknowns in a fixed order
// (decreasing hash priority); an unmarked one becomes coarse and its unmarked matrix-graph
// neighbours fine.  The greedy result is computed in rounds: an undecided node becomes
// coarse when it has the largest key among itself and its neighbours (IN > UNDECIDED >
// OUT, then priority) and fine when a neighbour is already coarse -- the same set as the
// sequential visit.  Neighbours: columns j != i of stored nonzero a_ij.
// visiting priority of the red-black split: hashed, or decreasing with the index (the
// index order)
__device__ __forceinline__ uint64_t rb_prio(int64_t i, uint32_t s, int natural) {
  return natural ? (((uint64_t)1 << 62) - 1 - (uint64_t)i) : prio_of(i, s);
}

__global__ void k_rb_round(int64_t N, const int32_t* rowptr, const int32_t* col, const double* val,
                           uint32_t s, int natural, const uint8_t* state_in, uint8_t* state_out,
                           unsigned long long* undecided) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  const uint8_t st = state_in[r];
  if (st != ST_UND) {
    state_out[r] = st;
    return;
  }
  const uint64_t key = ((uint64_t)ST_UND << 62) | rb_prio(r, s, natural);
  uint64_t best = key;
  for (int e = rowptr[r]; e < rowptr[r + 1]; e++) {
    const int j = col[e];
    if (j < 0 || j == r || val[e] == 0.0) continue;
    const uint64_t kj = ((uint64_t)state_in[j] << 62) | rb_prio(j, s, natural);
    best = kj > best ? kj : best;
  }
  uint8_t ns = ST_UND;
  if (best == key)
    ns = ST_IN;
  else if ((best >> 62) == ST_IN)
    ns = ST_OUT;
  else
    *undecided = 1ull;
  state_out[r] = ns;
}

// Averaging interpolation: coarse i -> (cid(i), 1); fine i -> (cid(j), 1 / #C_i) for its
// coarse neighbours j in column order (cid increases with j).  Count pass when Pcol is null.
__global__ void k_rb_prolong(int64_t N, const int32_t* rowptr, const int32_t* col,
                             const double* val, const uint8_t* state, const int64_t* cid,
                             int64_t* cnt, const int32_t* Prp, int32_t* Pcol, double* Pval,
                             unsigned long long* err) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  if (state[r] == ST_IN) {
    if (!Pcol) {
      cnt[r] = 1;
      return;
    }
    int64_t o = Prp[r];
    Pcol[o] = (int32_t)cid[r];
    Pval[o++] = 1.0;
    for (; o < Prp[r + 1]; o++) {
      Pcol[o] = -1;
      Pval[o] = 0.0;
    }
    return;
  }
  int c = 0;
  for (int e = rowptr[r]; e < rowptr[r + 1]; e++) {
    const int j = col[e];
    if (j >= 0 && j != r && val[e] != 0.0 && state[j] == ST_IN) c++;
  }
  if (!Pcol) {
    if (c == 0) atomicAdd(err, 1ull);
    cnt[r] = c;
    return;
  }
  const double w = 1.0 / (double)c;
  int64_t o = Prp[r];
  for (int e = rowptr[r]; e < rowptr[r + 1]; e++) {
    const int j = col[e];
    if (j >= 0 && j != r && val[e] != 0.0 && state[j] == ST_IN) {
      Pcol[o] = (int32_t)cid[j];
      Pval[o++] = w;
    }
  }
  for (; o < Prp[r + 1]; o++) {
    Pcol[o] = -1;
    Pval[o] = 0.0;
  }
}

__global__ void k_rb_cid(int64_t N, const uint8_t* state, const int64_t* cid, int32_t* out) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < N) out[r] = state[r] == ST_IN ? (int32_t)cid[r] : -1;
}

// ------------------------------------------------------------------ greedy colouring

// Colour of each node: the smallest colour not used by its higher-priority neighbours,
// assigned once all of them are coloured (the same colouring as a sequential visit by
// decreasing priority).  In place: a colour never changes once written.
constexpr int kMaxColours = 256;
__global__ void k_colour_round(int64_t N, const int32_t* rowptr, const int32_t* col,
                               const double* val, uint32_t s, int32_t* colour,
                               unsigned long long* pending, unsigned long long* overflow) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N || colour[r] >= 0) return;
  const uint64_t pr = prio_of(r, s);
  uint64_t used[kMaxColours / 64] = {0, 0, 0, 0};
  for (int e = rowptr[r]; e < rowptr[r + 1]; e++) {
    const int j = col[e];
    if (j < 0 || j == r || val[e] == 0.0) continue;
    if (prio_of(j, s) < pr) continue;
    const int cj = ((volatile int32_t*)colour)[j];
    if (cj < 0) {
      *pending = 1ull;
      return;
    }
    used[cj >> 6] |= 1ull << (cj & 63);
  }
  int c = 0;
  while (c < kMaxColours && ((used[c >> 6] >> (c & 63)) & 1ull)) c++;
  if (c == kMaxColours) {
    atomicAdd(overflow, 1ull);
    c = kMaxColours - 1;
  }
  colour[r] = c;
}

// per-colour counts (block histograms in shared memory, one atomic per colour per block)
__global__ void k_colour_count(int64_t N, const int32_t* colour, unsigned long long* cnt) {
  __shared__ unsigned int h[kMaxColours];
  for (int c = threadIdx.x; c < kMaxColours; c += blockDim.x) h[c] = 0;
  __syncthreads();
  for (int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; r < N;
       r += (int64_t)gridDim.x * blockDim.x)
    atomicAdd(&h[colour[r]], 1u);
  __syncthreads();
  for (int c = threadIdx.x; c < kMaxColours; c += blockDim.x)
    if (h[c]) atomicAdd(&cnt[c], (unsigned long long)h[c]);
}

// node lists per colour: each block reserves a range per colour, then fills it (the order
// inside a colour is irrelevant: its nodes do not couple)
__global__ void k_colour_scatter(int64_t N, const int32_t* colour, unsigned long long* cursor,
                                 int32_t* nodes) {
  __shared__ unsigned int h[kMaxColours];
  __shared__ unsigned long long base[kMaxColours];
  for (int64_t r0 = (int64_t)blockIdx.x * blockDim.x; r0 < N; r0 += (int64_t)gridDim.x * blockDim.x) {
    for (int c = threadIdx.x; c < kMaxColours; c += blockDim.x) h[c] = 0;
    __syncthreads();
    const int64_t r = r0 + threadIdx.x;
    unsigned int slot = 0;
    int c = -1;
    if (r < N) {
      c = colour[r];
      slot = atomicAdd(&h[c], 1u);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < kMaxColours; q += blockDim.x)
      if (h[q]) base[q] = atomicAdd(&cursor[q], (unsigned long long)h[q]);
    __syncthreads();
    if (r < N) nodes[base[c] + slot] = (int32_t)r;
    __syncthreads();
  }
}

// ------------------------------------------------------------------ uniform-grid level

template <uint32_t MASK>
__global__ void k_st_mis_init(int64_t N, int m, uint32_t strong, uint8_t* state, uint32_t s,
                              uint64_t* key) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  int i, j, k;
  st_ijk(r, m, i, j, k);
  bool any = false;
#pragma unroll
  for (int d = 0; d < 27; d++)
    if (st_sel<MASK>(strong, d)) any |= st_inb(i, j, k, d, m);
  const uint8_t st = any ? ST_UND : ST_OUT;
  state[r] = st;
  key[r] = ((uint64_t)st << 62) | prio_of(r, s);
}

template <uint32_t MASK>
// (key: each node's state above its priority, written by the previous round)
__global__ void k_st_mis_m1(int64_t N, int m, uint32_t strong, const uint64_t* __restrict__ key,
                            uint64_t* m1) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  int i, j, k;
  st_ijk(r, m, i, j, k);
  uint64_t best = key[r];
#pragma unroll
  for (int d = 0; d < 27; d++) {
    if (!st_sel<MASK>(strong, d) || !st_inb(i, j, k, d, m)) continue;
    const uint64_t kq = key[r + st_off(d, m)];
    best = kq > best ? kq : best;
  }
  m1[r] = best;
}

template <uint32_t MASK>
// (in place: a node reads and writes only its own state and key; a decided node keeps both)
// With a counter, the nodes still undecided are added to it, one atomic per block (one
// address for the whole grid: per-warp atomics were most of the round's time).
__global__ void k_st_mis_m2(int64_t N, int m, uint32_t strong, const uint64_t* m1, uint32_t s,
                            uint8_t* state, uint64_t* key, unsigned long long* undecided) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  bool und = false;
  if (r < N && state[r] == ST_UND) {
    int i, j, k;
    st_ijk(r, m, i, j, k);
    uint64_t best = m1[r];
#pragma unroll
    for (int d = 0; d < 27; d++) {
      if (!st_sel<MASK>(strong, d) || !st_inb(i, j, k, d, m)) continue;
      const uint64_t kq = m1[r + st_off(d, m)];
      best = kq > best ? kq : best;
    }
    uint8_t ns = ST_UND;
    const uint64_t pr = prio_of(r, s);
    if (best == (((uint64_t)ST_UND << 62) | pr))
      ns = ST_IN;
    else if ((best >> 62) == ST_IN)
      ns = ST_OUT;
    if (ns != ST_UND) {
      state[r] = ns;
      key[r] = ((uint64_t)ns << 62) | pr;
    }
    und = ns == ST_UND;
  }
  if (!undecided) return;  // (the same for the whole grid)
  const int c = __syncthreads_count(und);
  if (threadIdx.x == 0 && c) atomicAdd(undecided, (unsigned long long)c);
}

// List rounds (once few nodes are undecided): m1 over the nodes within distance 1 of an
// undecided node, then the decision for the undecided ones, written after the round.
template <uint32_t MASK>
__global__ void k_st_list_m1(int64_t nv, const int64_t* __restrict__ vlist, int m, uint32_t strong,
                             const uint8_t* state, uint32_t s, uint64_t* m1) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nv) return;
  const int64_t r = vlist[t];
  int i, j, k;
  st_ijk(r, m, i, j, k);
  uint64_t best = ((uint64_t)state[r] << 62) | prio_of(r, s);
#pragma unroll
  for (int d = 0; d < 27; d++) {
    if (!st_sel<MASK>(strong, d) || !st_inb(i, j, k, d, m)) continue;
    const int64_t q = r + st_off(d, m);
    const uint64_t kq = ((uint64_t)state[q] << 62) | prio_of(q, s);
    best = kq > best ? kq : best;
  }
  m1[r] = best;
}

template <uint32_t MASK>
__global__ void k_st_list_m2(int64_t nu, const int64_t* __restrict__ ulist, int m, uint32_t strong,
                             const uint64_t* m1, uint32_t s, const uint8_t* state,
                             uint8_t* newst, unsigned long long* undecided) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nu) return;
  const int64_t r = ulist[t];
  const uint8_t st = state[r];
  uint8_t ns = st;
  if (st == ST_UND) {
    int i, j, k;
    st_ijk(r, m, i, j, k);
    uint64_t best = m1[r];
#pragma unroll
    for (int d = 0; d < 27; d++) {
      if (!st_sel<MASK>(strong, d) || !st_inb(i, j, k, d, m)) continue;
      const uint64_t kq = m1[r + st_off(d, m)];
      best = kq > best ? kq : best;
    }
    const uint64_t key = ((uint64_t)ST_UND << 62) | prio_of(r, s);
    if (best == key)
      ns = ST_IN;
    else if ((best >> 62) == ST_IN)
      ns = ST_OUT;
    if (ns == ST_UND) atomicAdd(undecided, 1ull);
  }
  newst[t] = ns;
}

__global__ void k_st_list_apply(int64_t nu, const int64_t* __restrict__ ulist,
                                const uint8_t* __restrict__ newst, uint8_t* state) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < nu) state[ulist[t]] = newst[t];
}

// the indices flagged in an exclusive scan of 0/1 flags, in order
__global__ void k_list_from_scan(int64_t N, const int64_t* scan, int64_t* list) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r < N && scan[r + 1] != scan[r]) list[scan[r]] = r;
}

// flag every node within distance 1 (strong directions) of a listed node
template <uint32_t MASK>
__global__ void k_st_mark_ring(int64_t nu, const int64_t* __restrict__ ulist, int m,
                               uint32_t strong, uint8_t* flag) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nu) return;
  const int64_t r = ulist[t];
  int i, j, k;
  st_ijk(r, m, i, j, k);
  flag[r] = 1;
#pragma unroll
  for (int d = 0; d < 27; d++) {
    if (!st_sel<MASK>(strong, d) || !st_inb(i, j, k, d, m)) continue;
    flag[r + st_off(d, m)] = 1;
  }
}

template <uint32_t MASK>
__global__ void k_st_agg_phase1(int64_t N, int m, uint32_t strong, const uint8_t* state,
                                const int64_t* rootid, int32_t* agg, uint8_t* p1,
                                unsigned long long* err) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  int i, j, k;
  st_ijk(r, m, i, j, k);
  int32_t a = -1;
  if (state[r] == ST_IN) {
    a = (int32_t)rootid[r];
  } else {
    int found = 0;
#pragma unroll
    for (int d = 0; d < 27; d++) {
      if (!st_sel<MASK>(strong, d) || !st_inb(i, j, k, d, m)) continue;
      const int64_t q = r + st_off(d, m);
      if (state[q] == ST_IN) {
        if (found) atomicAdd(err, 1ull);
        a = (int32_t)rootid[q];
        found = 1;
      }
    }
  }
  agg[r] = a;
  p1[r] = a >= 0;
}

template <uint32_t MASK>
__global__ void k_st_agg_phase2(int64_t N, int m, uint32_t strong, const uint8_t* p1, int32_t* agg,
                                unsigned long long* err) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= N) return;
  if (p1[r]) return;
  int i, j, k;
  st_ijk(r, m, i, j, k);
  // aggregate of each strong in-bounds neighbour that is in a phase-1 aggregate (-1 else)
  int32_t na[27];
  bool any = false;
#pragma unroll
  for (int d = 0; d < 27; d++) {
    na[d] = -1;
    if (!st_sel<MASK>(strong, d) || !st_inb(i, j, k, d, m)) continue;
    any = true;
    const int64_t q = r + st_off(d, m);
    if (p1[q]) na[d] = agg[q];
  }
  if (!any) return;  // isolated
  int32_t best = -1;
  int bestc = 0;
#pragma unroll
  for (int d = 0; d < 27; d++) {
    if (na[d] < 0) continue;
    int c = 0;
#pragma unroll
    for (int f = 0; f < 27; f++) c += na[f] == na[d];
    if (c > bestc || (c == bestc && na[d] < best)) {
      best = na[d];
      bestc = c;
    }
  }
  if (best < 0) atomicAdd(err, 1ull);
  agg[r] = best;
}

// k_psmooth on the stencil: the row's in-bounds diagonal and strong entries in column order.
// With the strong set known at compile time the candidates (diagonal and strong directions,
// in d order) stay in registers: a key's entry is its first candidate, its position the
// number of smaller distinct keys, its sum taken over the candidates with that key in d
// order -- the order of the insertion sort of the run-time path, so both give the same
// bits.  V.a[d] = a_d / a_ii as the host rounds the product a_d * (1 / a_ii), the same
// product the run-time path forms per row (GB300's FP64 pipe is the scarce one).
__host__ __device__ constexpr int sel_count(uint32_t s) {
  int c = 0;
  for (int d = 0; d < 27; d++) c += (int)((s >> d) & 1u);
  return c;
}
// the direction of the q-th set bit of s
__host__ __device__ constexpr int sel_nth(uint32_t s, int q) {
  for (int d = 0; d < 27; d++)
    if ((s >> d) & 1u) {
      if (q == 0) return d;
      q--;
    }
  return 0;
}
template <uint32_t MASK>
__global__ void k_st_psmooth(int64_t N, StencilRow S, StencilRow V, const int32_t* agg,
                             double dinv, double omega, int64_t* cnt, const int32_t* Prp,
                             int32_t* Pcol, double* Pval) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (MASK != 0u) {
    constexpr uint32_t SEL = MASK | (1u << ST_DIAG);
    constexpr int K = sel_count(SEL);
    if (r >= N) return;
    int i, j, k;
    st_ijk(r, S.m, i, j, k);
    const int32_t ar = agg[r];
    int key[K];
    double val[K];
#pragma unroll
    for (int q = 0; q < K; q++) {
      const int d = sel_nth(SEL, q);
      key[q] = -1;
      val[q] = 0.0;
      if (ar >= 0 && st_inb(i, j, k, d, S.m)) {
        key[q] = agg[r + st_off(d, S.m)];  // (-1: the neighbour is not aggregated)
        val[q] = V.a[d];
      }
    }
    bool first[K];
    int nd = 0;
#pragma unroll
    for (int q = 0; q < K; q++) {
      bool f = key[q] >= 0;
#pragma unroll
      for (int e = 0; e < q; e++)
        if (key[e] == key[q]) f = false;
      first[q] = f;
      nd += f;
    }
    if (!Pcol) {
      cnt[r] = nd;
      return;
    }
    const int64_t o = Prp[r], o1 = Prp[r + 1];
#pragma unroll
    for (int q = 0; q < K; q++) {
      if (!first[q]) continue;
      int rank = 0;
#pragma unroll
      for (int e = 0; e < K; e++)
        if (first[e] && key[e] < key[q]) rank++;
      double sum = val[q];
#pragma unroll
      for (int e = q + 1; e < K; e++)
        if (key[e] == key[q]) sum = __dadd_rn(sum, val[e]);
      const double t = __dmul_rn(-omega, sum);
      Pcol[o + rank] = key[q];
      Pval[o + rank] = key[q] == ar ? __dadd_rn(1.0, t) : t;
    }
    for (int64_t p = o + nd; p < o1; p++) {
      Pcol[p] = -1;
      Pval[p] = 0.0;
    }
  } else {
    if (r >= N) return;
    int i, j, k;
    st_ijk(r, S.m, i, j, k);
    const int32_t ar = agg[r];
    int keys[27];
    double vals[27];
    int m = 0;
    if (ar >= 0) {
      for (int d = 0; d < 27; d++) {
        if ((d != ST_DIAG && !st_sel<MASK>(S.strong, d)) || !st_inb(i, j, k, d, S.m)) continue;
        const int a = agg[r + st_off(d, S.m)];
        if (a < 0) continue;
        const double v = __dmul_rn(S.a[d], dinv);
        int q = m++;
        while (q > 0 && keys[q - 1] > a) {
          keys[q] = keys[q - 1];
          vals[q] = vals[q - 1];
          q--;
        }
        keys[q] = a;
        vals[q] = v;
      }
    }
    if (!Pcol) {
      int dd = 0;
      for (int q = 0; q < m; q++) dd += (q == 0 || keys[q] != keys[q - 1]);
      cnt[r] = dd;
      return;
    }
    int64_t o = Prp[r];
    const int64_t o1 = Prp[r + 1];
    int q = 0;
    while (q < m) {
      const int key = keys[q];
      double sum = vals[q++];
      while (q < m && keys[q] == key) sum = __dadd_rn(sum, vals[q++]);
      const double t = __dmul_rn(-omega, sum);
      Pcol[o] = key;
      Pval[o] = key == ar ? __dadd_rn(1.0, t) : t;
      o++;
    }
    for (; o < o1; o++) {
      Pcol[o] = -1;
      Pval[o] = 0.0;
    }
  }
}

__global__ void k_fill(int64_t n, double v, double* out, float* out32 = nullptr) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  out[i] = v;
  if (out32) out32[i] = (float)v;
}

// The interior row of A (centre of the grid) with its strong pairs, by the same test as
// k_strength.  Returns false when the level does not have the uniform-stencil structure
// this path relies on (then the CSR path runs).
bool stencil_row(const Csr4& A, int m, double theta, StencilRow& R, cudaStream_t st) {
  if (m < 3 || (int64_t)m * m * m != A.nrows) return false;
  const int64_t c = (int64_t)(m / 2) * (1 + m + (int64_t)m * m);
  int32_t rp[2];
  FEM_CUDA(cudaMemcpyAsync(rp, A.rowptr.p + c, 8, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  const int len = rp[1] - rp[0];
  if (len <= 0 || len > 32) return false;
  int32_t col[32];
  double val[32];
  FEM_CUDA(cudaMemcpyAsync(col, A.col.p + rp[0], 4 * len, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaMemcpyAsync(val, A.val.p + rp[0], 8 * len, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  R = StencilRow{};
  R.m = m;
  for (int d = 0; d < 27; d++) R.a[d] = 0.0;
  double dg = 0.0;
  for (int e = 0; e < len; e++)
    if (col[e] == c) dg = val[e];
  if (!(dg > 0.0)) return false;
  const double sq = std::sqrt(dg), tr = theta * sq;
  int64_t prev = -1;
  for (int e = 0; e < len; e++) {
    if (col[e] < 0) continue;
    const int64_t t = (int64_t)col[e] - c + (1 + m + (int64_t)m * m);
    if (t < 0 || col[e] <= prev) return false;
    prev = col[e];
    const int64_t ex = t % m, ey = (t / m) % m, ez = t / ((int64_t)m * m);
    if (ex > 2 || ey > 2 || ez > 2) return false;
    const int d = (int)(ex + 3 * ey + 9 * ez);
    R.present |= 1u << d;
    R.a[d] = val[e];
    if (d != ST_DIAG && val[e] != 0.0 && std::fabs(val[e]) >= tr * sq) R.strong |= 1u << d;
  }
  return (R.present >> ST_DIAG) & 1u;
}

// Row-sum bound max_i sum_j |a_ij| / a_ii over the selected entries (all, or diagonal and
// strong) in column order: attained on interior rows (boundary rows hold a subset of the
// same terms).
double stencil_rowabs(const StencilRow& R, bool strong_only) {
  const uint32_t sel = strong_only ? (R.strong | (1u << ST_DIAG)) : R.present;
  double s = 0.0;
  for (int d = 0; d < 27; d++)
    if ((sel >> d) & 1u) s += std::fabs(R.a[d]);
  return s / R.a[ST_DIAG];
}

// Strong-direction sets of the Kuhn stencil by class (the kernels are compiled for each
// combination; any other set runs with the mask read at run time).
constexpr uint32_t kStAxis = (1u << 4) | (1u << 10) | (1u << 12) | (1u << 14) | (1u << 16) | (1u << 22);
constexpr uint32_t kStFace = (1u << 1) | (1u << 3) | (1u << 9) | (1u << 17) | (1u << 23) | (1u << 25);
constexpr uint32_t kStBody = (1u << 0) | (1u << 26);

template <uint32_t M>
Aggregation aggregate_stencil_t(int64_t N, const StencilRow& S, uint32_t seed_s, cudaStream_t st) {
  Aggregation R;
  const unsigned g = grid_for(N, 256), g2 = grid_for(N, 512);
  DevBuf<uint8_t> s0(N, st);
  DevBuf<uint64_t> m1(N, st), k0(N, st);
  DevBuf<unsigned long long> und(1, st);
  k_st_mis_init<M><<<g, 256, 0, st>>>(N, S.m, S.strong, s0, seed_s, k0);
  FEM_CHECK_LAUNCH();
  uint8_t* cur = s0;
  uint64_t* kcur = k0;
  bool finished = false;
  unsigned long long hu = (unsigned long long)N;
  int round = 0;
  for (; round < 10000; round += 2) {
    // two rounds per check of the undecided count (a round after the last is a no-op)
    for (int t = 0; t < 2; t++) {
      k_st_mis_m1<M><<<g, 256, 0, st>>>(N, S.m, S.strong, kcur, m1);
      FEM_CHECK_LAUNCH();
      if (t == 1) FEM_CUDA(cudaMemsetAsync(und, 0, 8, st));
      k_st_mis_m2<M><<<g2, 512, 0, st>>>(N, S.m, S.strong, m1, seed_s, cur, kcur,
                                          t == 1 ? und.p : nullptr);
      FEM_CHECK_LAUNCH();
    }
    FEM_CUDA(cudaMemcpyAsync(&hu, und, 8, cudaMemcpyDeviceToHost, st));
    FEM_CUDA(cudaStreamSynchronize(st));
    if (hu == 0) {
      finished = true;
      break;
    }
    if ((int64_t)hu * 64 < N) break;   // few left: continue on lists
  }
  if (!finished && round < 10000) {
    // the same rounds on the undecided nodes only (m1 on the nodes around them)
    DevBuf<uint8_t> flag(N, st);
    DevBuf<int64_t> scan(N + 1, st);
    const int64_t nu = count_scan_eq(cur, ST_UND, N, scan, st);
    DevBuf<int64_t> ul(nu, st);
    k_list_from_scan<<<g, 256, 0, st>>>(N, scan, ul);
    FEM_CHECK_LAUNCH();
    FEM_CUDA(cudaMemsetAsync(flag, 0, N, st));
    k_st_mark_ring<M><<<grid_for(nu, 256), 256, 0, st>>>(nu, ul, S.m, S.strong, flag);
    FEM_CHECK_LAUNCH();
    const int64_t nvr = count_scan_eq(flag, 1, N, scan, st);
    DevBuf<int64_t> vl(nvr, st);
    k_list_from_scan<<<g, 256, 0, st>>>(N, scan, vl);
    FEM_CHECK_LAUNCH();
    DevBuf<uint8_t> newst(nu, st);
    const unsigned gu = grid_for(nu, 256), gv = grid_for(nvr, 256);
    for (; round < 10000; round += 2) {
      for (int t = 0; t < 2; t++) {
        k_st_list_m1<M><<<gv, 256, 0, st>>>(nvr, vl, S.m, S.strong, cur, seed_s, m1);
        FEM_CHECK_LAUNCH();
        if (t == 1) FEM_CUDA(cudaMemsetAsync(und, 0, 8, st));
        k_st_list_m2<M><<<gu, 256, 0, st>>>(nu, ul, S.m, S.strong, m1, seed_s, cur, newst, und);
        FEM_CHECK_LAUNCH();
        k_st_list_apply<<<gu, 256, 0, st>>>(nu, ul, newst, cur);
        FEM_CHECK_LAUNCH();
      }
      FEM_CUDA(cudaMemcpyAsync(&hu, und, 8, cudaMemcpyDeviceToHost, st));
      FEM_CUDA(cudaStreamSynchronize(st));
      if (hu == 0) {
        finished = true;
        break;
      }
    }
  }
  FEM_REQUIRE(finished, FEM_EDEVCHECK, "aggregation: MIS-2 did not terminate");
  DevBuf<int64_t> rootid(N + 1, st);
  R.nagg = count_scan_eq(cur, ST_IN, N, rootid, st);
  R.agg.alloc(N);
  DevBuf<uint8_t> p1(N, st);
  DevBuf<unsigned long long> err(1, st);
  FEM_CUDA(cudaMemsetAsync(err, 0, 8, st));
  k_st_agg_phase1<M><<<g, 256, 0, st>>>(N, S.m, S.strong, cur, rootid, R.agg, p1, err);
  FEM_CHECK_LAUNCH();
  k_st_agg_phase2<M><<<g, 256, 0, st>>>(N, S.m, S.strong, p1, R.agg, err);
  FEM_CHECK_LAUNCH();
  unsigned long long he = 0;
  FEM_CUDA(cudaMemcpyAsync(&he, err, 8, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  FEM_REQUIRE(he == 0, FEM_EDEVCHECK, "aggregation: inconsistent MIS-2 / aggregate assignment");
  return R;
}

template <uint32_t M>
void psmooth_stencil_t(int64_t N, const StencilRow& S, const int32_t* agg, double dinv,
                       double omega, Csr4& P, int64_t nagg, cudaStream_t st) {
  const unsigned g = grid_for(N, 256);
  StencilRow V = S;
  for (int d = 0; d < 27; d++) V.a[d] = S.a[d] * dinv;
  DevBuf<int64_t> pc(N, st);
  k_st_psmooth<M><<<g, 256, 0, st>>>(N, S, V, agg, dinv, omega, pc, nullptr, nullptr, nullptr);
  FEM_CHECK_LAUNCH();
  P.nrows = (int32_t)N;
  P.ncols = (int32_t)nagg;
  rowptr_from_counts(pc, N, P, st);
  P.val.alloc(P.nnz);
  k_st_psmooth<M><<<g, 256, 0, st>>>(N, S, V, agg, dinv, omega, nullptr, P.rowptr, P.col,
                                     P.val);
  FEM_CHECK_LAUNCH();
}

#define FEM_ST_DISPATCH(strong, F, ...)                                        \
  switch (strong) {                                                           \
    case kStAxis: F<kStAxis>(__VA_ARGS__); break;                               \
    case kStFace: F<kStFace>(__VA_ARGS__); break;                               \
    case kStBody: F<kStBody>(__VA_ARGS__); break;                               \
    case kStAxis | kStFace: F<kStAxis | kStFace>(__VA_ARGS__); break;           \
    case kStAxis | kStBody: F<kStAxis | kStBody>(__VA_ARGS__); break;           \
    case kStFace | kStBody: F<kStFace | kStBody>(__VA_ARGS__); break;           \
    case kStAxis | kStFace | kStBody: F<kStAxis | kStFace | kStBody>(__VA_ARGS__); break; \
    default: F<0u>(__VA_ARGS__); break;                                         \
  }

Aggregation aggregate_stencil(int64_t N, const StencilRow& S, uint32_t seed_s, cudaStream_t st) {
  Aggregation R;
  FEM_ST_DISPATCH(S.strong, R = aggregate_stencil_t, N, S, seed_s, st);
  return R;
}

void psmooth_stencil(int64_t N, const StencilRow& S, const int32_t* agg, double dinv, double omega,
                     Csr4& P, int64_t nagg, cudaStream_t st) {
  FEM_ST_DISPATCH(S.strong, psmooth_stencil_t, N, S, agg, dinv, omega, P, nagg, st);
}

// Red-black split of a level: state (IN = coarse), coarse ids cid (exclusive scan of the
// coarse flags); returns the number of coarse nodes.
int64_t red_black_split(const Csr4& A, uint32_t s, int natural, DevBuf<uint8_t>& state,
                        DevBuf<int64_t>& cid, cudaStream_t st) {
  const int64_t N = A.nrows;
  const unsigned g = grid_for(N, 256);
  DevBuf<uint8_t> s0(N, st), s1(N, st);
  DevBuf<unsigned long long> und(1, st);
  FEM_CUDA(cudaMemsetAsync(s0, ST_UND, N, st));
  uint8_t* cur = s0;
  uint8_t* nxt = s1;
  bool finished = false;
  // several rounds per check (extra rounds are no-ops): the index order decides a front of
  // the grid per round, so it takes more rounds per check
  const int per = natural ? 16 : 4;
  for (int round = 0; round < 100000; round++) {
    FEM_CUDA(cudaMemsetAsync(und, 0, 8, st));
    for (int t = 0; t < per; t++) {
      if (t == per - 1) FEM_CUDA(cudaMemsetAsync(und, 0, 8, st));
      k_rb_round<<<g, 256, 0, st>>>(N, A.rowptr, A.col, A.val, s, natural, cur, nxt, und);
      FEM_CHECK_LAUNCH();
      std::swap(cur, nxt);
    }
    unsigned long long hu = 0;
    FEM_CUDA(cudaMemcpyAsync(&hu, und, 8, cudaMemcpyDeviceToHost, st));
    FEM_CUDA(cudaStreamSynchronize(st));
    if (hu == 0) {
      finished = true;
      break;
    }
  }
  FEM_REQUIRE(finished, FEM_EDEVCHECK, "red-black coarsening did not terminate");
  state.alloc(N);
  FEM_CUDA(cudaMemcpyAsync(state, cur, N, cudaMemcpyDeviceToDevice, st));
  cid.alloc(N + 1);
  return count_scan_eq(state, ST_IN, N, cid, st);
}

// Greedy colouring of a level's matrix graph and the node lists per colour.
void colour_level(Level& Lv, const Csr4& A, uint32_t s, cudaStream_t st) {
  const int64_t N = A.nrows;
  const unsigned g = grid_for(N, 256);
  Lv.colour.alloc(N);
  FEM_CUDA(cudaMemsetAsync(Lv.colour, 0xff, 4 * N, st));
  DevBuf<unsigned long long> flags(2, st);
  FEM_CUDA(cudaMemsetAsync(flags.p + 1, 0, 8, st));
  bool finished = false;
  for (int round = 0; round < 100000; round++) {
    FEM_CUDA(cudaMemsetAsync(flags, 0, 8, st));
    for (int t = 0; t < 4; t++) {
      if (t == 3) FEM_CUDA(cudaMemsetAsync(flags, 0, 8, st));
      k_colour_round<<<g, 256, 0, st>>>(N, A.rowptr, A.col, A.val, s, Lv.colour, flags,
                                        flags.p + 1);
      FEM_CHECK_LAUNCH();
    }
    unsigned long long hf[2] = {0, 0};
    FEM_CUDA(cudaMemcpyAsync(hf, flags, 16, cudaMemcpyDeviceToHost, st));
    FEM_CUDA(cudaStreamSynchronize(st));
    FEM_REQUIRE(hf[1] == 0, FEM_EUNSUPPORTED, "colouring: more than 256 colours");
    if (hf[0] == 0) {
      finished = true;
      break;
    }
  }
  FEM_REQUIRE(finished, FEM_EDEVCHECK, "colouring did not terminate");
  DevBuf<unsigned long long> cnt(kMaxColours, st), cursor(kMaxColours, st);
  FEM_CUDA(cudaMemsetAsync(cnt, 0, 8 * kMaxColours, st));
  const unsigned gp = persistent_grid(N, 256, 4);
  k_colour_count<<<gp, 256, 0, st>>>(N, Lv.colour, cnt);
  FEM_CHECK_LAUNCH();
  std::vector<unsigned long long> hc(kMaxColours);
  FEM_CUDA(cudaMemcpyAsync(hc.data(), cnt, 8 * kMaxColours, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  int ncol = 0;
  for (int c = 0; c < kMaxColours; c++)
    if (hc[c]) ncol = c + 1;
  Lv.coff.assign(ncol + 1, 0);
  for (int c = 0; c < ncol; c++) Lv.coff[c + 1] = Lv.coff[c] + (int64_t)hc[c];
  std::vector<unsigned long long> hcur(kMaxColours, 0);
  for (int c = 0; c < ncol; c++) hcur[c] = (unsigned long long)Lv.coff[c];
  FEM_CUDA(cudaMemcpyAsync(cursor, hcur.data(), 8 * kMaxColours, cudaMemcpyHostToDevice, st));
  Lv.cnodes.alloc(N > 0 ? N : 1);
  k_colour_scatter<<<gp, 256, 0, st>>>(N, Lv.colour, cursor, Lv.cnodes);
  FEM_CHECK_LAUNCH();
  FEM_CUDA(cudaStreamSynchronize(st));
}

void make_lowp(Csr4& A, int prec, cudaStream_t st) {
  if (prec == AMG_PREC_FP32 || prec == AMG_PREC_BF16) {
    A.val32.alloc(A.nnz);
    if (A.nnz % 4 == 0)
      k_convert4_f32<<<grid_for(A.nnz / 4, 256), 256, 0, st>>>(A.nnz / 4, A.val, A.val32);
    else
      k_convert<double, float><<<grid_for(A.nnz, 256), 256, 0, st>>>(A.nnz, A.val, A.val32);
    FEM_CHECK_LAUNCH();
  }
  if (prec == AMG_PREC_BF16) {
    A.val16.alloc(A.nnz);
    if (A.nnz)
      k_convert<double, __nv_bfloat16><<<grid_for(A.nnz, 256), 256, 0, st>>>(A.nnz, A.val, A.val16);
    FEM_CHECK_LAUNCH();
  }
}

}  // namespace

void build_hierarchy(Hierarchy& H, System& S, const amg_opts& o, cudaStream_t st) {
  H.sys = &S;
  H.o = o;
  H.L.clear();
  const int prec = o.precision;
  const bool lowp = prec != AMG_PREC_FP64;
  Tracer tr(st);
  auto cur = std::make_unique<Level>();
  cur->A = &S.A;
  cur->stencil = S.stencil;
  cur->st = S.stA;
  if (o.rho_setup > 0.0 && o.rho_setup != S.rho) {
    // finest level of the set-up from rho_setup K + M on the system's pattern
    Csr4& A0 = cur->Aown;
    A0.nrows = S.A.nrows;
    A0.ncols = S.A.ncols;
    A0.nnz = S.A.nnz;
    A0.rowptr.alloc(A0.nrows + 1);
    A0.col.alloc(A0.nnz);
    A0.val.alloc(A0.nnz);
    FEM_CUDA(cudaMemcpyAsync(A0.rowptr, S.A.rowptr, 4 * ((int64_t)A0.nrows + 1),
                             cudaMemcpyDeviceToDevice, st));
    FEM_CUDA(cudaMemcpyAsync(A0.col, S.A.col, 4 * A0.nnz, cudaMemcpyDeviceToDevice, st));
    k_axpby<<<grid_for(A0.nnz, 256), 256, 0, st>>>(A0.nnz, o.rho_setup, S.Kv, S.Mv, A0.val);
    FEM_CHECK_LAUNCH();
    cur->A = &A0;
    cur->st.c0 = o.rho_setup * S.stK.c0 + S.stM.c0;
    cur->st.ca = o.rho_setup * S.stK.ca + S.stM.ca;
    cur->st.cf = o.rho_setup * S.stK.cf + S.stM.cf;
    cur->st.cb = o.rho_setup * S.stK.cb + S.stM.cb;
  }
  for (int lev = 0;; lev++) {
    Level& Lv = *cur;
    const Csr4* Acur = Lv.A;
    Lv.N = Acur->nrows;
    const int64_t N = Lv.N;
    unsigned g = grid_for(N, 256);
    // uniform finest level: graph, bounds and prolongator from the stencil
    StencilRow SR;
    const bool rb = o.coarsening == AMG_COARSEN_RED_BLACK;
    const uint32_t seed_s = (uint32_t)(0x9E3779B9u * (uint32_t)(o.seed + lev + 1));
    const bool st0 = lev == 0 && Lv.stencil && o.smoother == AMG_SMOOTHER_CHEBYSHEV && !rb &&
                     N > o.coarse_max && stencil_row(*Acur, Lv.st.m, o.theta, SR, st);
    // (the stencil level's diagonal is one number: its reciprocal is formed on the host,
    // correctly rounded like the device's division)
    DevBuf<double> d;
    if (!st0) {
      d.alloc_async(N, st);
      k_diag<<<grid_for(N * DG_G, 256), 256, 0, st>>>(N, Acur->rowptr, Acur->col, Acur->val, d);
      FEM_CHECK_LAUNCH();
    }
    Lv.dinv.alloc(N);
    if (lowp) Lv.dinv32.alloc(N);
    Lv.scalar_sinv = Lv.stencil && o.smoother == AMG_SMOOTHER_CHEBYSHEV;
    if (o.smoother == AMG_SMOOTHER_L1_JACOBI) {
      DevBuf<double> l1(N, st);
      rowabs_max(*Acur, Acur->val, nullptr, d, l1, st);
      k_recip<<<g, 256, 0, st>>>(N, l1, Lv.dinv, lowp ? Lv.dinv32.p : nullptr);
      Lv.lmax = 1.0;
    } else if (st0) {
      k_fill<<<g, 256, 0, st>>>(N, 1.0 / SR.a[ST_DIAG], Lv.dinv, lowp ? Lv.dinv32.p : nullptr);
      Lv.lmax = stencil_rowabs(SR, false);
    } else {
      k_recip<<<g, 256, 0, st>>>(N, d, Lv.dinv, lowp ? Lv.dinv32.p : nullptr);
      Lv.lmax = rowabs_max(*Acur, Acur->val, nullptr, d, nullptr, st);
    }
    FEM_CHECK_LAUNCH();
    if (lowp) {
      Csr4& Am = (lev == 0 && Lv.A == &S.A) ? S.A : Lv.Aown;
      if (!(lev == 0 && Lv.stencil) || o.smoother == AMG_SMOOTHER_SGS) {
        if (!Am.val32.p) make_lowp(Am, AMG_PREC_FP32, st);
        if (prec == AMG_PREC_BF16 && !Am.val16.p) make_lowp(Am, AMG_PREC_BF16, st);
      }
    }

    tr.mark("level: diagonal, lambda, low precision");
    if (o.smoother == AMG_SMOOTHER_SGS) {
      colour_level(Lv, *Acur, seed_s, st);
      tr.mark("level: colouring");
    }
    bool last = (N <= o.coarse_max) || (lev == o.max_levels - 1);
    Aggregation ag;
    DevBuf<uint8_t> rbstate;
    DevBuf<int64_t> rbcid;
    if (!last) {
      if (rb)
        ag.nagg = red_black_split(*Acur, seed_s, o.order == AMG_ORDER_NATURAL ? 1 : 0, rbstate,
                                  rbcid, st);
      else
        ag = st0 ? aggregate_stencil(N, SR, seed_s, st) : aggregate(*Acur, d, o.theta, seed_s, st);
      tr.mark("level: aggregation");
      if (ag.nagg == 0 || (double)ag.nagg >= 0.9 * (double)N) last = true;
    }
    if (last) {
      Lv.coarsest = true;
      if (N <= o.coarse_max) dense_inverse(*Acur, Acur->val, Lv.Ainv, st);
      tr.mark("coarsest: dense inverse");
      H.L.push_back(std::move(cur));
      break;
    }
    bool done_p = false;
    if (rb) {
      // averaging interpolation of the red-black split (Sec. 3.1)
      DevBuf<int64_t> pc(N, st);
      DevBuf<unsigned long long> err(1, st);
      FEM_CUDA(cudaMemsetAsync(err, 0, 8, st));
      k_rb_prolong<<<g, 256, 0, st>>>(N, Acur->rowptr, Acur->col, Acur->val, rbstate, rbcid, pc,
                                      nullptr, nullptr, nullptr, err);
      FEM_CHECK_LAUNCH();
      Lv.P.nrows = (int32_t)N;
      Lv.P.ncols = (int32_t)ag.nagg;
      rowptr_from_counts(pc, N, Lv.P, st);
      Lv.P.val.alloc(Lv.P.nnz);
      k_rb_prolong<<<g, 256, 0, st>>>(N, Acur->rowptr, Acur->col, Acur->val, rbstate, rbcid,
                                      nullptr, Lv.P.rowptr, Lv.P.col, Lv.P.val, err);
      FEM_CHECK_LAUNCH();
      Lv.agg.alloc(N);
      k_rb_cid<<<g, 256, 0, st>>>(N, rbstate, rbcid, Lv.agg);
      FEM_CHECK_LAUNCH();
      unsigned long long he = 0;
      FEM_CUDA(cudaMemcpyAsync(&he, err, 8, cudaMemcpyDeviceToHost, st));
      FEM_CUDA(cudaStreamSynchronize(st));
      FEM_REQUIRE(he == 0, FEM_EDEVCHECK, "red-black: a fine node without a coarse neighbour");
      done_p = true;
    }
    // smoothed prolongator P = P_t - omega D^{-1} A_F P_t
    if (!rb) Lv.agg = std::move(ag.agg);
    const double lamF = rb ? 0.0
                           : (st0 ? stencil_rowabs(SR, true)
                                  : rowabs_max(*Acur, Acur->val, ag.smask, d, nullptr, st));
    const double omega = rb ? 0.0 : 4.0 / (3.0 * lamF);
    if (st0) {
      psmooth_stencil(N, SR, Lv.agg, 1.0 / SR.a[ST_DIAG], omega, Lv.P, ag.nagg, st);
      // the same prolongator as a stencil on the aggregates' values, for the V-cycle: centre
      // 1 - w a_ii / a_ii (the identity and the diagonal term), strong direction d -w a_d / a_ii
      const double dinv = 1.0 / SR.a[ST_DIAG];
      Lv.pst = true;
      Lv.pst_strong = SR.strong & ~(1u << ST_DIAG);
      for (int d = 0; d < 27; d++) Lv.pst_c[d] = 0.0f;
      Lv.pst_c[ST_DIAG] = (float)(1.0 - omega * (SR.a[ST_DIAG] * dinv));
      for (int d = 0; d < 27; d++)
        if ((Lv.pst_strong >> d) & 1u) Lv.pst_c[d] = (float)(-omega * (SR.a[d] * dinv));
      done_p = true;
    }
    DevBuf<double> dinvA;
    if (!done_p) {
      dinvA.alloc(N);
      k_recip<<<g, 256, 0, st>>>(N, d, dinvA, nullptr);
      FEM_CHECK_LAUNCH();
    }
    if (!done_p) {
      DevBuf<int64_t> pc(N, st);
      DevBuf<unsigned long long> ovf(1, st);
      FEM_CUDA(cudaMemsetAsync(ovf, 0, 8, st));
      k_psmooth<<<g, 256, 0, st>>>(N, Acur->rowptr, Acur->col, Acur->val, ag.smask, Lv.agg, dinvA,
                                   omega, pc, nullptr, nullptr, nullptr, ovf);
      FEM_CHECK_LAUNCH();
      unsigned long long hov = 0;
      FEM_CUDA(cudaMemcpyAsync(&hov, ovf, 8, cudaMemcpyDeviceToHost, st));
      FEM_CUDA(cudaStreamSynchronize(st));
      if (hov == 0) {
        Lv.P.nrows = (int32_t)N;
        Lv.P.ncols = (int32_t)ag.nagg;
        rowptr_from_counts(pc, N, Lv.P, st);
        Lv.P.val.alloc(Lv.P.nnz);
        k_psmooth<<<g, 256, 0, st>>>(N, Acur->rowptr, Acur->col, Acur->val, ag.smask, Lv.agg,
                                     dinvA, omega, nullptr, Lv.P.rowptr, Lv.P.col, Lv.P.val, ovf);
        FEM_CHECK_LAUNCH();
        done_p = true;
      }
    }
    if (!done_p) {
      // long rows: D^{-1} A_F as a CSR4 matrix times the tentative prolongator
      Csr4 Pt;
      Pt.nrows = (int32_t)N;
      Pt.ncols = (int32_t)ag.nagg;
      Pt.nnz = 4 * N;
      Pt.rowptr.alloc(N + 1);
      Pt.col.alloc(4 * N);
      Pt.val.alloc(4 * N);
      k_tentative<<<grid_for(N + 1, 256), 256, 0, st>>>(N, Lv.agg, Pt.rowptr, Pt.col, Pt.val);
      FEM_CHECK_LAUNCH();
      Csr4 DF;
      DF.nrows = DF.ncols = (int32_t)N;
      DF.nnz = Acur->nnz;
      DF.rowptr.alloc(N + 1);
      DF.col.alloc(DF.nnz);
      DF.val.alloc(DF.nnz);
      FEM_CUDA(cudaMemcpyAsync(DF.rowptr, Acur->rowptr, 4 * (N + 1), cudaMemcpyDeviceToDevice, st));
      k_scaled_filtered<<<g, 256, 0, st>>>(N, Acur->rowptr, Acur->col, Acur->val, ag.smask,
                                           dinvA, DF.col, DF.val);
      FEM_CHECK_LAUNCH();
      spgemm(DF, DF.val, Pt, Pt.val, Lv.P, st, true);
      Lv.P.ncols = (int32_t)ag.nagg;
      k_smooth_p<<<g, 256, 0, st>>>(N, Lv.P.rowptr, Lv.P.col, Lv.P.val, Lv.agg, omega);
      FEM_CHECK_LAUNCH();
    }
    tr.mark("level: P = (I - w D^-1 A_F) P_t");
    // a level whose restriction or Galerkin products would have a row longer than max_row
    // (at most the products' limit; graded meshes make the coarse levels of the Laplacian
    // that dense) becomes the coarsest level instead
    bool too_long = false;
    const int64_t row_limit = o.max_row > 0 ? o.max_row : kLongRowMax;
    transpose(Lv.P, Lv.R, ag.nagg, st, &too_long, row_limit);
    tr.mark("level: R = P^T");
    if (lowp) {
      make_lowp(Lv.P, AMG_PREC_FP32, st);
      make_lowp(Lv.R, AMG_PREC_FP32, st);
      if (prec == AMG_PREC_BF16) {
        make_lowp(Lv.P, AMG_PREC_BF16, st);
        make_lowp(Lv.R, AMG_PREC_BF16, st);
      }
    }
    // Galerkin coarse operator A_c = R (A P)  (Sec. 3.1)
    // (the merge kernels when they take the product; the pencil keeps A P for its parts)
    Csr4 AP;
    auto nxt = std::make_unique<Level>();
    bool merged = false;
    // (the uniform finest level's A P from the stencil: A is not read)
    StencilRow SRa;
    const StencilRow* ap_sr = nullptr;
    if (lev == 0 && Lv.stencil && !too_long && !S.pencil) {
      if (st0) ap_sr = &SR;
      else if (stencil_row(*Acur, Lv.st.m, o.theta, SRa, st)) ap_sr = &SRa;
    }
    if (!too_long && !S.pencil)
      merged = galerkin_merge(*Acur, Lv.P, Lv.R, nxt->Aown, st, &too_long, row_limit, nullptr,
                              ap_sr);
    if (!merged && !too_long)
      spgemm(*Acur, Acur->val, Lv.P, Lv.P.val, AP, st, true, &too_long, row_limit);
    tr.mark("level: A P (spgemm)");
    if (!merged && !too_long)
      spgemm(Lv.R, Lv.R.val, AP, AP.val, nxt->Aown, st, true, &too_long, row_limit);
    tr.mark("level: R (A P) (spgemm)");
    if (too_long) {
      Lv.P = Csr4();
      Lv.R = Csr4();
      Lv.coarsest = true;
      if (N <= o.coarse_max) dense_inverse(*Acur, Acur->val, Lv.Ainv, st);
      tr.mark("coarsest (dense coarse rows): dense inverse");
      H.L.push_back(std::move(cur));
      break;
    }
    nxt->Aown.ncols = (int32_t)ag.nagg;
    nxt->A = &nxt->Aown;
    if (S.pencil) {
      // with P fixed, R (rho K + M) P = rho R K P + R M P: keep both pencil parts
      const double* Kv = lev == 0 ? S.Kv.p : Lv.Kv.p;
      const double* Mv = lev == 0 ? S.Mv.p : Lv.Mv.p;
      DevBuf<double> KP(AP.nnz, st), MP(AP.nnz, st);
      spgemm_numeric(*Acur, Kv, Lv.P, Lv.P.val, AP, KP, st);
      spgemm_numeric(*Acur, Mv, Lv.P, Lv.P.val, AP, MP, st);
      nxt->Kv.alloc(nxt->Aown.nnz);
      nxt->Mv.alloc(nxt->Aown.nnz);
      spgemm_numeric(Lv.R, Lv.R.val, AP, KP, nxt->Aown, nxt->Kv, st);
      spgemm_numeric(Lv.R, Lv.R.val, AP, MP, nxt->Aown, nxt->Mv, st);
    }
    tr.mark("level: pencil / low precision copies");
    H.L.push_back(std::move(cur));
    cur = std::move(nxt);
  }
  FEM_CUDA(cudaStreamSynchronize(st));
}

}  // namespace fem
