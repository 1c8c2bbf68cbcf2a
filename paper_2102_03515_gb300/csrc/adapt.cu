// Adaptive loop pieces (Sec. 4.2-4.3: meshes refined where a residual indicator is large):
// bulk marking of the tets with the largest indicators and local refinement of a device mesh
// by longest-edge bisection with conforming closure.  The residual indicator itself sits with
// the quadrature in assemble.cu.
//
// Refinement rules (fixed so that every run gives the same mesh):
//  * the edges of a tet are ordered by squared length (dx*dx + dy*dy) + dz*dz, computed
//    without contraction, ties broken by the smaller vertex pair (min, max); the longest edge
//    of a tet is the largest, at local positions i < j;
//  * bisecting a tet with midpoint m = 0.5 * (x_a + x_b): child 0 = the tet with vertex j
//    replaced by m stays at the tet's index, child 1 = the tet with vertex i replaced by m is
//    appended (in the order of the parents); both keep the orientation;
//  * a call bisects the longest edge of every marked tet, then whatever conformity needs, in
//    passes: close the set of edges to bisect (add the longest edge of every tet that holds
//    one, until nothing changes), then bisect every tet whose longest edge is in the set; stop
//    when no tet holds an edge of the set;
//  * the new vertices of a pass are numbered in the order of the first tet (lowest index)
//    that bisects their edge;
//  * a new vertex on the boundary of the mesh is a Dirichlet vertex (u = 0 on all of the
//    boundary, Sec. 2).  Each tet carries a 4-bit mask of its faces on the boundary (bit k:
//    the face opposite local vertex k); a child keeps the parent's bits except the one of the
//    new interior face, and a midpoint is on the boundary when one of the two parent faces
//    holding the bisected edge is.
//
// Edges to bisect live in an open-addressing hash table keyed by the vertex pair, holding the
// midpoint (-1 until it exists) and the first tet that bisects the edge.
#include <cstring>

#include "solver.cuh"

namespace fem {

namespace {

constexpr unsigned long long kEmpty = ~0ull;
constexpr int kMaxPasses = 4096;
constexpr int kMaxCloseRounds = 1 << 16;

__constant__ int8_t kEdgeI[6] = {0, 0, 0, 1, 1, 2};
__constant__ int8_t kEdgeJ[6] = {1, 2, 3, 2, 3, 3};

__device__ __forceinline__ unsigned long long fmix64(unsigned long long k) {
  k ^= k >> 33;
  k *= 0xff51afd7ed558ccdull;
  k ^= k >> 33;
  k *= 0xc4ceb9fe1a85ec53ull;
  k ^= k >> 33;
  return k;
}

__device__ __forceinline__ unsigned long long edge_key(int32_t a, int32_t b) {
  const unsigned long long lo = (unsigned)min(a, b), hi = (unsigned)max(a, b);
  return (lo << 32) | hi;
}

struct Table {
  unsigned long long* key;
  int32_t* mid;
  int32_t* own;
  long long cap;   // power of two
};

// slot of key, -1 when absent (probing ends at an empty slot or after cap probes)
__device__ long long ht_find(const Table& T, unsigned long long k) {
  long long s = (long long)(fmix64(k) & (unsigned long long)(T.cap - 1));
  for (long long p = 0; p < T.cap; p++) {
    const unsigned long long c = *((volatile unsigned long long*)T.key + s);
    if (c == k) return s;
    if (c == kEmpty) return -1;
    s = (s + 1) & (T.cap - 1);
  }
  return -1;
}

// inserts key (idempotent); returns 1 when this call inserted it, 0 when it was there, -1
// when the table is full
__device__ int ht_insert(const Table& T, unsigned long long k) {
  long long s = (long long)(fmix64(k) & (unsigned long long)(T.cap - 1));
  for (long long p = 0; p < T.cap; p++) {
    const unsigned long long c = atomicCAS(T.key + s, kEmpty, k);
    if (c == kEmpty) return 1;
    if (c == k) return 0;
    s = (s + 1) & (T.cap - 1);
  }
  return -1;
}

__device__ __forceinline__ double len2_rn(const double* xyz, int32_t a, int32_t b) {
  const double dx = xyz[3 * (int64_t)b] - xyz[3 * (int64_t)a];
  const double dy = xyz[3 * (int64_t)b + 1] - xyz[3 * (int64_t)a + 1];
  const double dz = xyz[3 * (int64_t)b + 2] - xyz[3 * (int64_t)a + 2];
  return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// longest edge of every tet: its key and local index 0..5
__global__ void k_leb_longest(int64_t nt, const int32_t* __restrict__ tet,
                              const double* __restrict__ xyz, unsigned long long* lkey,
                              uint8_t* li) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const int4 tv = reinterpret_cast<const int4*>(tet)[t];
  const int32_t v[4] = {tv.x, tv.y, tv.z, tv.w};
  double bl = len2_rn(xyz, v[0], v[1]);
  unsigned long long bk = edge_key(v[0], v[1]);
  int best = 0;
  for (int e = 1; e < 6; e++) {
    const int32_t a = v[kEdgeI[e]], b = v[kEdgeJ[e]];
    const double l2 = len2_rn(xyz, a, b);
    const unsigned long long k = edge_key(a, b);
    if (l2 > bl || (l2 == bl && k < bk)) {
      bl = l2;
      bk = k;
      best = e;
    }
  }
  lkey[t] = bk;
  li[t] = (uint8_t)best;
}

__global__ void k_leb_seed(int64_t nt, const uint8_t* mark, const unsigned long long* lkey,
                           Table T, unsigned long long* count, int* full) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt || !mark[t]) return;
  const int r = ht_insert(T, lkey[t]);
  if (r == 1) atomicAdd(count, 1ull);
  if (r < 0) atomicExch(full, 1);
}

// closure round: a tet holding an edge of the table puts its longest edge in the table
__global__ void k_leb_close(int64_t nt, const int32_t* __restrict__ tet,
                            const unsigned long long* __restrict__ lkey, Table T,
                            unsigned long long* count, int* changed, int* full) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const unsigned long long lk = lkey[t];
  if (ht_find(T, lk) >= 0) return;
  const int4 tv = reinterpret_cast<const int4*>(tet)[t];
  const int32_t v[4] = {tv.x, tv.y, tv.z, tv.w};
  bool any = false;
  for (int e = 0; e < 6 && !any; e++) any = ht_find(T, edge_key(v[kEdgeI[e]], v[kEdgeJ[e]])) >= 0;
  if (!any) return;
  const int r = ht_insert(T, lk);
  if (r == 1) {
    atomicAdd(count, 1ull);
    atomicExch(changed, 1);
  }
  if (r < 0) atomicExch(full, 1);
}

// tets to bisect (longest edge in the table) and the first of them for each edge still
// without a midpoint
__global__ void k_leb_own(int64_t nt, const unsigned long long* __restrict__ lkey, Table T,
                          int64_t* bis, long long* slot) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const long long s = ht_find(T, lkey[t]);
  bis[t] = s >= 0 ? 1 : 0;
  slot[t] = s;
  if (s >= 0 && T.mid[s] < 0) atomicMin(T.own + s, (int32_t)t);
}

__global__ void k_leb_newflag(int64_t nt, const long long* __restrict__ slot, Table T,
                              int64_t* nm) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const long long s = slot[t];
  nm[t] = (s >= 0 && T.mid[s] < 0 && T.own[s] == (int32_t)t) ? 1 : 0;
}

// midpoints of the new edges, numbered nv + (rank of the owning tet)
__global__ void k_leb_mid(int64_t nt, int64_t nv, const int64_t* __restrict__ nm,
                          const int64_t* __restrict__ nm_scan, const long long* __restrict__ slot,
                          Table T, double* xyz, uint8_t* dir) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt || !nm[t]) return;
  const long long s = slot[t];
  const int64_t id = nv + nm_scan[t];
  const unsigned long long k = T.key[s];
  const int64_t a = (int64_t)(k >> 32), b = (int64_t)(k & 0xffffffffull);
  for (int d = 0; d < 3; d++)
    xyz[3 * id + d] = __dmul_rn(0.5, __dadd_rn(xyz[3 * a + d], xyz[3 * b + d]));
  dir[id] = 0;
  T.mid[s] = (int32_t)id;
}

__device__ __forceinline__ void set_flag_byte(uint8_t* dir, int64_t i) {
  unsigned* w = reinterpret_cast<unsigned*>(dir + (i & ~(int64_t)3));
  atomicOr(w, 1u << (8 * (unsigned)(i & 3)));
}

// every tet whose longest edge is in the table splits on it
__global__ void k_leb_bisect(int64_t nt, const int64_t* __restrict__ bis,
                             const int64_t* __restrict__ bis_scan,
                             const long long* __restrict__ slot, const uint8_t* __restrict__ li,
                             Table T, int32_t* tet, uint8_t* bmask, uint8_t* dir,
                             int* bad) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt || !bis[t]) return;
  const int32_t m = T.mid[slot[t]];
  if (m < 0) {   // every bisected edge has its midpoint by now; keep the mesh intact if not
    atomicExch(bad, 1);
    return;
  }
  const int e = li[t];
  const int i = kEdgeI[e], j = kEdgeJ[e];
  int4 tv = reinterpret_cast<int4*>(tet)[t];
  int32_t v[4] = {tv.x, tv.y, tv.z, tv.w};
  const unsigned bm = bmask[t];
  // the two faces holding edge (i, j) are those opposite the other two vertices
  const unsigned other = 0xFu & ~((1u << i) | (1u << j));
  if (bm & other) set_flag_byte(dir, m);
  int32_t c0[4] = {v[0], v[1], v[2], v[3]}, c1[4] = {v[0], v[1], v[2], v[3]};
  c0[j] = m;
  c1[i] = m;
  const int64_t u = nt + bis_scan[t];
  reinterpret_cast<int4*>(tet)[t] = make_int4(c0[0], c0[1], c0[2], c0[3]);
  reinterpret_cast<int4*>(tet)[u] = make_int4(c1[0], c1[1], c1[2], c1[3]);
  bmask[t] = (uint8_t)(bm & ~(1u << i));
  bmask[u] = (uint8_t)(bm & ~(1u << j));
}

__global__ void k_ht_clear(Table T) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= T.cap) return;
  T.key[s] = kEmpty;
  T.mid[s] = -1;
  T.own[s] = 0x7fffffff;
}

__global__ void k_ht_rehash(Table from, Table to, int* full) {
  const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= from.cap) return;
  const unsigned long long k = from.key[s];
  if (k == kEmpty) return;
  long long d = (long long)(fmix64(k) & (unsigned long long)(to.cap - 1));
  for (long long p = 0; p < to.cap; p++) {
    if (atomicCAS(to.key + d, kEmpty, k) == kEmpty) {
      to.mid[d] = from.mid[s];
      to.own[d] = from.own[s];
      return;
    }
    d = (d + 1) & (to.cap - 1);
  }
  atomicExch(full, 1);
}

// boundary faces of every tet: bit k when the face opposite local vertex k has no other tet
__global__ void k_mesh_bmask(int64_t nt, const int32_t* __restrict__ tet,
                             const int64_t* __restrict__ vptr, const int32_t* __restrict__ vtet,
                             uint8_t* bmask, unsigned long long* bad) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const int4 tv = reinterpret_cast<const int4*>(tet)[t];
  const int32_t v[4] = {tv.x, tv.y, tv.z, tv.w};
  unsigned m = 0;
  for (int a = 0; a < 4; a++) {
    const int32_t b = v[(a + 1) & 3], c = v[(a + 2) & 3], d = v[(a + 3) & 3];
    int found = 0;
    for (int64_t e = vptr[b]; e < vptr[b + 1]; e++) {
      const int32_t s = vtet[e];
      if (s == t) continue;
      const int4 w = reinterpret_cast<const int4*>(tet)[s];
      const bool hc = w.x == c || w.y == c || w.z == c || w.w == c;
      const bool hd = w.x == d || w.y == d || w.z == d || w.w == d;
      found += (hc && hd) ? 1 : 0;
    }
    if (found == 0) m |= 1u << a;
    if (found > 1) atomicAdd(bad, 1ull);
  }
  bmask[t] = (uint8_t)m;
}

// every tet must have a nonzero volume; repeated vertices are errors too
__global__ void k_mesh_check(int64_t nt, const int32_t* __restrict__ tet,
                             const double* __restrict__ xyz, unsigned long long* bad) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nt) return;
  const int4 tv = reinterpret_cast<const int4*>(tet)[t];
  const int32_t v[4] = {tv.x, tv.y, tv.z, tv.w};
  double J[3][3];
  for (int r = 0; r < 3; r++)
    for (int c = 0; c < 3; c++) J[r][c] = xyz[3 * (int64_t)v[c + 1] + r] - xyz[3 * (int64_t)v[0] + r];
  const double det = J[0][0] * (J[1][1] * J[2][2] - J[1][2] * J[2][1]) -
                     J[0][1] * (J[1][0] * J[2][2] - J[1][2] * J[2][0]) +
                     J[0][2] * (J[1][0] * J[2][1] - J[1][1] * J[2][0]);
  if (!(det != 0.0) || !isfinite(det)) atomicAdd(bad, 1ull);
}

// ------------------------------------------------------------------ bulk marking

// sum of the eta >= t (t = the double with the bit pattern (lo + hi) / 2; all when
// state == null), per-block partials over a fixed grid; flags negative or non-finite values
__global__ void k_mark_sum(int64_t n, const double* __restrict__ eta,
                           const unsigned long long* state, double* partials, int* bad) {
  double t = 0.0;
  if (state) t = __longlong_as_double((long long)((state[0] + state[1]) >> 1));
  double acc[1] = {0.0};
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double e = eta[i];
    if (!state && !(e >= 0.0 && e <= 1.7976931348623157e308)) atomicExch(bad, 1);
    if (e >= t) acc[0] += e;
  }
  block_sum<1>(acc);
  if (threadIdx.x == 0) partials[blockIdx.x] = acc[0];
}

// fixed-order sum of the partials (one block) and one bisection step on the threshold's bits:
// state = {lo, hi, goal bits}; lo keeps S(lo) >= goal, hi keeps S(hi) < goal
__global__ void k_mark_step(const double* partials, int nb, unsigned long long* state,
                            double theta, int init) {
  double acc[1] = {0.0};
  for (int i = threadIdx.x; i < nb; i += blockDim.x) acc[0] += partials[i];
  block_sum<1>(acc);
  if (threadIdx.x != 0) return;
  const double S = acc[0];
  if (init) {
    state[0] = 0ull;
    state[1] = 0x7ff0000000000000ull;   // +inf: no finite value reaches it
    state[2] = (unsigned long long)__double_as_longlong(theta * S);
    return;
  }
  const double goal = __longlong_as_double((long long)state[2]);
  const unsigned long long mid = (state[0] + state[1]) >> 1;
  if (S >= goal)
    state[0] = mid;
  else
    state[1] = mid;
}

__global__ void k_mark_apply(int64_t n, const double* __restrict__ eta,
                             const unsigned long long* state, uint8_t* mark,
                             unsigned long long* count) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double t = __longlong_as_double((long long)state[0]);
  const bool m = eta[i] >= t;
  mark[i] = m ? 1 : 0;
  if (m) atomicAdd(count, 1ull);
}

void table_alloc(long long cap, DevBuf<unsigned long long>& k, DevBuf<int32_t>& mid,
                 DevBuf<int32_t>& own, Table& T, cudaStream_t st) {
  k.alloc_async(cap, st);
  mid.alloc_async(cap, st);
  own.alloc_async(cap, st);
  T = Table{k.p, mid.p, own.p, cap};
  k_ht_clear<<<grid_for(cap, 256), 256, 0, st>>>(T);
  FEM_CHECK_LAUNCH();
}

template <typename U>
void grow(DevBuf<U>& b, size_t keep, size_t count, cudaStream_t st) {
  DevBuf<U> nb(count, st);
  if (keep) FEM_CUDA(cudaMemcpyAsync(nb.p, b.p, keep * sizeof(U), cudaMemcpyDeviceToDevice, st));
  b = std::move(nb);
}

}  // namespace

void mesh_create(Mesh& M, const fem_mesh_desc& d, cudaStream_t st) {
  FEM_REQUIRE(d.nv >= 4 && d.nt >= 1 && d.nv < ((int64_t)1 << 31) && d.nt < ((int64_t)1 << 31),
              FEM_EINVAL, "fem_mesh_create: bad sizes");
  FEM_REQUIRE(d.xyz && d.tet && d.dirichlet, FEM_EINVAL, "fem_mesh_create: null array");
  M.nv = d.nv;
  M.nt = d.nt;
  M.xyz.alloc(3 * M.nv);
  M.tet.alloc(4 * M.nt);
  M.dir.alloc((M.nv + 3) & ~(int64_t)3);
  M.bmask.alloc(M.nt);
  FEM_CUDA(cudaMemcpyAsync(M.xyz, d.xyz, 24 * M.nv, cudaMemcpyHostToDevice, st));
  FEM_CUDA(cudaMemcpyAsync(M.tet, d.tet, 16 * M.nt, cudaMemcpyHostToDevice, st));
  FEM_CUDA(cudaMemcpyAsync(M.dir, d.dirichlet, M.nv, cudaMemcpyHostToDevice, st));
  DevBuf<int64_t> vptr;
  DevBuf<int32_t> vtet;
  build_incidence(M.nv, M.nt, M.tet, vptr, vtet, st);
  DevBuf<unsigned long long> bad(2, st);
  FEM_CUDA(cudaMemsetAsync(bad, 0, 16, st));
  const unsigned gt = grid_for(M.nt, 256);
  k_mesh_check<<<gt, 256, 0, st>>>(M.nt, M.tet, M.xyz, bad.p);
  FEM_CHECK_LAUNCH();
  k_mesh_bmask<<<gt, 256, 0, st>>>(M.nt, M.tet, vptr, vtet, M.bmask, bad.p + 1);
  FEM_CHECK_LAUNCH();
  unsigned long long hb[2];
  FEM_CUDA(cudaMemcpyAsync(hb, bad, 16, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  FEM_REQUIRE(hb[0] == 0, FEM_EINVAL, "fem_mesh_create: a tet has zero volume");
  FEM_REQUIRE(hb[1] == 0, FEM_EINVAL, "fem_mesh_create: a face belongs to more than two tets");
}

void mesh_refine(Mesh& M, const uint8_t* mark, cudaStream_t st, fem_refine_stats& out) {
  out = fem_refine_stats{0, 0, 0};
  const int64_t nv0 = M.nv, nt0 = M.nt;
  // flags: [0] inserted count, [1] changed, [2] full (as ints inside 8-byte slots)
  DevBuf<unsigned long long> cnt(1, st);
  DevBuf<int> fl(2, st);
  FEM_CUDA(cudaMemsetAsync(cnt, 0, 8, st));
  FEM_CUDA(cudaMemsetAsync(fl, 0, 8, st));
  long long cap = 1 << 12;
  while (cap < 8 * M.nt && cap < ((long long)1 << 40)) cap <<= 1;
  DevBuf<unsigned long long> tk;
  DevBuf<int32_t> tm, to;
  Table T;
  table_alloc(cap, tk, tm, to, T, st);
  DevBuf<int> rfull(1, st);
  auto rehash = [&](long long ncap) {
    DevBuf<unsigned long long> nk;
    DevBuf<int32_t> nmid, nown;
    Table N;
    table_alloc(ncap, nk, nmid, nown, N, st);
    FEM_CUDA(cudaMemsetAsync(rfull, 0, 4, st));
    k_ht_rehash<<<grid_for(T.cap, 256), 256, 0, st>>>(T, N, rfull);
    FEM_CHECK_LAUNCH();
    int hr = 0;
    FEM_CUDA(cudaMemcpyAsync(&hr, rfull, 4, cudaMemcpyDeviceToHost, st));
    FEM_CUDA(cudaStreamSynchronize(st));
    FEM_REQUIRE(hr == 0, FEM_EDEVCHECK, "fem_mesh_refine: edge table full");
    tk = std::move(nk);
    tm = std::move(nmid);
    to = std::move(nown);
    T = N;
  };
  DevBuf<unsigned long long> lkey;
  DevBuf<uint8_t> li;
  bool seeded = false;
  for (int pass = 0;; pass++) {
    FEM_REQUIRE(pass < kMaxPasses, FEM_EDEVCHECK, "fem_mesh_refine: no end of the bisection");
    const int64_t nt = M.nt;
    const unsigned gt = grid_for(nt, 256);
    lkey.alloc_async(nt, st);
    li.alloc_async(nt, st);
    k_leb_longest<<<gt, 256, 0, st>>>(nt, M.tet, M.xyz, lkey, li);
    FEM_CHECK_LAUNCH();
    for (int round = 0;; round++) {
      FEM_REQUIRE(round < kMaxCloseRounds, FEM_EDEVCHECK, "fem_mesh_refine: no end of the closure");
      FEM_CUDA(cudaMemsetAsync(fl, 0, 8, st));
      if (!seeded)
        k_leb_seed<<<gt, 256, 0, st>>>(nt, mark, lkey, T, cnt, fl.p + 1);
      else
        k_leb_close<<<gt, 256, 0, st>>>(nt, M.tet, lkey, T, cnt, fl.p, fl.p + 1);
      FEM_CHECK_LAUNCH();
      int hf[2];
      unsigned long long hc;
      FEM_CUDA(cudaMemcpyAsync(hf, fl, 8, cudaMemcpyDeviceToHost, st));
      FEM_CUDA(cudaMemcpyAsync(&hc, cnt, 8, cudaMemcpyDeviceToHost, st));
      FEM_CUDA(cudaStreamSynchronize(st));
      if (hf[1] || (long long)hc * 2 > T.cap) {
        // grow and repeat the round (rounds only add edges, so repeating is harmless)
        FEM_REQUIRE(T.cap < ((long long)1 << 40), FEM_ENOMEM, "fem_mesh_refine: edge table");
        rehash(T.cap * 2);
        if (hf[1]) continue;
      }
      if (!seeded) {
        seeded = true;
        continue;
      }
      if (!hf[0]) break;
    }
    DevBuf<int64_t> bis(nt, st), bscan(nt + 1, st), nm(nt, st), nscan(nt + 1, st);
    DevBuf<long long> slot(nt, st);
    k_leb_own<<<gt, 256, 0, st>>>(nt, lkey, T, bis, slot);
    FEM_CHECK_LAUNCH();
    k_leb_newflag<<<gt, 256, 0, st>>>(nt, slot, T, nm);
    FEM_CHECK_LAUNCH();
    const int64_t nb = exclusive_scan(bis, nt, bscan, st);
    const int64_t nn = exclusive_scan(nm, nt, nscan, st);
    if (nb == 0) break;
    FEM_REQUIRE(M.nt + nb < ((int64_t)1 << 31) && M.nv + nn < ((int64_t)1 << 31),
                FEM_EUNSUPPORTED, "fem_mesh_refine: more than 2^31 tets or vertices");
    out.passes++;
    if (nn) {
      grow(M.xyz, 3 * M.nv, 3 * (M.nv + nn), st);
      grow(M.dir, M.nv, (M.nv + nn + 3) & ~(int64_t)3, st);
    }
    grow(M.tet, 4 * M.nt, 4 * (M.nt + nb), st);
    grow(M.bmask, M.nt, M.nt + nb, st);
    k_leb_mid<<<gt, 256, 0, st>>>(nt, M.nv, nm, nscan, slot, T, M.xyz, M.dir);
    FEM_CHECK_LAUNCH();
    FEM_CUDA(cudaMemsetAsync(fl, 0, 8, st));
    k_leb_bisect<<<gt, 256, 0, st>>>(nt, bis, bscan, slot, li, T, M.tet, M.bmask, M.dir, fl.p);
    FEM_CHECK_LAUNCH();
    M.nv += nn;
    M.nt += nb;
    int hb = 0;
    FEM_CUDA(cudaMemcpyAsync(&hb, fl, 4, cudaMemcpyDeviceToHost, st));
    FEM_CUDA(cudaStreamSynchronize(st));
    FEM_REQUIRE(hb == 0, FEM_EDEVCHECK, "fem_mesh_refine: a bisected edge has no midpoint");
  }
  FEM_CUDA(cudaStreamSynchronize(st));
  out.new_vertices = M.nv - nv0;
  out.new_tets = M.nt - nt0;
}

void mark_bulk(const double* eta, int64_t n, double theta, uint8_t* mark, cudaStream_t st,
               double* threshold, int64_t* nmarked) {
  FEM_REQUIRE(n >= 1, FEM_EINVAL, "fem_mark_bulk: n must be >= 1");
  FEM_REQUIRE(theta > 0.0 && theta <= 1.0, FEM_EINVAL, "fem_mark_bulk: theta in (0, 1]");
  const unsigned g = persistent_grid(n, 256, 4);
  DevBuf<double> part(g, st);
  DevBuf<unsigned long long> state(3, st), count(1, st);
  DevBuf<int> bad(1, st);
  FEM_CUDA(cudaMemsetAsync(bad, 0, 4, st));
  FEM_CUDA(cudaMemsetAsync(count, 0, 8, st));
  k_mark_sum<<<g, 256, 0, st>>>(n, eta, nullptr, part, bad);
  FEM_CHECK_LAUNCH();
  k_mark_step<<<1, 256, 0, st>>>(part, (int)g, state, theta, 1);
  FEM_CHECK_LAUNCH();
  // 63 steps close the gap between 0 and the bits of +inf (below 2^63)
  for (int it = 0; it < 63; it++) {
    k_mark_sum<<<g, 256, 0, st>>>(n, eta, state, part, bad);
    FEM_CHECK_LAUNCH();
    k_mark_step<<<1, 256, 0, st>>>(part, (int)g, state, theta, 0);
    FEM_CHECK_LAUNCH();
  }
  k_mark_apply<<<grid_for(n, 256), 256, 0, st>>>(n, eta, state, mark, count);
  FEM_CHECK_LAUNCH();
  unsigned long long hs[3], hc;
  int hb;
  FEM_CUDA(cudaMemcpyAsync(hs, state, 24, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaMemcpyAsync(&hc, count, 8, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaMemcpyAsync(&hb, bad, 4, cudaMemcpyDeviceToHost, st));
  FEM_CUDA(cudaStreamSynchronize(st));
  FEM_REQUIRE(hb == 0, FEM_EINVAL, "fem_mark_bulk: indicators must be finite and >= 0");
  double t;
  std::memcpy(&t, &hs[0], 8);
  if (threshold) *threshold = t;
  if (nmarked) *nmarked = (int64_t)hc;
}

}  // namespace fem
