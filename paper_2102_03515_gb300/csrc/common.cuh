// Shared device/host infrastructure of the solver library: error handling, device
// buffers, the CSR4 layout, deterministic reductions and launch helpers.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <utility>
#include <vector>

#include "../../include/femamg.h"

namespace fem {

// ------------------------------------------------------------------ errors

struct Error {
  fem_status status;
  std::string msg;
};

[[noreturn]] void fail(fem_status s, const std::string& msg);
void set_last_error(const std::string& msg);

#define FEM_CUDA(call)                                                                   \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      ::fem::fail(e_ == cudaErrorMemoryAllocation ? FEM_ENOMEM : FEM_ECUDA,              \
                  std::string(#call) + ": " + cudaGetErrorString(e_) + " (" __FILE__ ":" + \
                      std::to_string(__LINE__) + ")");                                   \
  } while (0)

// Every kernel launch site ends with FEM_CHECK_LAUNCH(), which also counts the launch
// (the count is reported by fem_kernel_launches()).
void count_launches(long long n);
#define FEM_CHECK_LAUNCH()            \
  do {                                \
    FEM_CUDA(cudaGetLastError());     \
    ::fem::count_launches(1);         \
  } while (0)

#define FEM_REQUIRE(cond, status, msg)           \
  do {                                           \
    if (!(cond)) ::fem::fail((status), (msg));   \
  } while (0)

// ------------------------------------------------------------------ buffers

// Stream on which DevBuf::alloc places its stream-ordered allocations (thread-local; the
// entry points set it to the caller's stream for the duration of a call).
cudaStream_t& current_alloc_stream();
struct StreamScope {
  cudaStream_t prev;
  explicit StreamScope(cudaStream_t s) : prev(current_alloc_stream()) { current_alloc_stream() = s; }
  ~StreamScope() { current_alloc_stream() = prev; }
};

// Owning device buffer.  Allocations are stream-ordered when a stream is given.
template <typename T>
struct DevBuf {
  T* p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  bool async = false;
  DevBuf() = default;
  explicit DevBuf(size_t count) { alloc(count); }
  DevBuf(size_t count, cudaStream_t st) { alloc_async(count, st); }
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept { swap(o); }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) {
      release();
      swap(o);
    }
    return *this;
  }
  ~DevBuf() { release(); }
  void swap(DevBuf& o) noexcept {
    std::swap(p, o.p);
    std::swap(n, o.n);
    std::swap(s, o.s);
    std::swap(async, o.async);
  }
  void alloc(size_t count) { alloc_async(count, current_alloc_stream()); }
  void alloc_async(size_t count, cudaStream_t st) {
    release();
    n = count;
    s = st;
    async = true;
    if (count) FEM_CUDA(cudaMallocAsync(&p, count * sizeof(T), st));
  }
  void release() noexcept {
    if (p) {
      if (async)
        cudaFreeAsync(p, s);
      else
        cudaFree(p);
    }
    p = nullptr;
    n = 0;
  }
  size_t bytes() const { return n * sizeof(T); }
  T* get() const { return p; }
  operator T*() const { return p; }
};

// ------------------------------------------------------------------ CSR4

// CSR whose rows are padded to a multiple of 4 stored entries with (col -1, value 0):
// every row then starts on a 16-byte boundary for int4 / double2 / float4 loads.
struct Csr4 {
  int32_t nrows = 0, ncols = 0;
  int64_t nnz = 0;             // stored entries including padding
  DevBuf<int32_t> rowptr;      // nrows + 1
  DevBuf<int32_t> col;         // nnz
  DevBuf<double> val;          // nnz, FP64
  DevBuf<float> val32;         // optional FP32 copy
  DevBuf<__nv_bfloat16> val16; // optional BF16 copy
  size_t bytes() const {
    return rowptr.bytes() + col.bytes() + val.bytes() + val32.bytes() + val16.bytes();
  }
};

// ------------------------------------------------------------------ tracing

// Phase timer enabled by the environment variable FEM_TRACE=1: each mark synchronises
// the stream and prints the wall time since the previous mark to stderr.
struct Tracer {
  bool on = false;
  cudaStream_t st = nullptr;
  double t = 0;
  explicit Tracer(cudaStream_t s);
  void mark(const char* what);
};

// Keep freed stream-ordered allocations in the device's default pool (no unmapping at
// every synchronisation): repeated set-ups reuse the same memory.
void init_memory_pool();

// ------------------------------------------------------------------ launch helpers

inline int num_sms() {
  static int sms = -1;
  if (sms < 0) {
    int dev = 0;
    FEM_CUDA(cudaGetDevice(&dev));
    FEM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return sms;
}

inline unsigned grid_for(int64_t work, int block) {
  int64_t g = (work + block - 1) / block;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// Grid-stride launches use a fixed grid of (SMs x per_sm) blocks, so that the number of
// per-block partial sums (and hence the reduction order) depends only on the device.
inline unsigned persistent_grid(int64_t work, int block, int per_sm = 8) {
  int64_t cap = (int64_t)num_sms() * per_sm;
  int64_t g = (work + block - 1) / block;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (unsigned)g;
}

// ------------------------------------------------------------------ reductions

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ double warp_max(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Sum of NV values per thread over the block (fixed tree order: deterministic).  The
// result is valid in thread 0.  blockDim.x must be a multiple of 32, <= 1024.
template <int NV>
__device__ __forceinline__ void block_sum(double (&v)[NV]) {
  __shared__ double sh[NV][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int k = 0; k < NV; k++) v[k] = warp_sum(v[k]);
  __syncthreads();
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < NV; k++) sh[k][wid] = v[k];
  __syncthreads();
  if (wid == 0) {
#pragma unroll
    for (int k = 0; k < NV; k++) {
      double t = lane < nw ? sh[k][lane] : 0.0;
      v[k] = warp_sum(t);
    }
  }
}

__device__ __forceinline__ double block_max(double v) {
  __shared__ double sh[32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) sh[wid] = v;
  __syncthreads();
  if (wid == 0) v = warp_max(lane < nw ? sh[lane] : -1.0e308);
  return v;
}

// Converters between storage and arithmetic types.
__device__ __forceinline__ double to_d(double v) { return v; }
__device__ __forceinline__ double to_d(float v) { return (double)v; }
__device__ __forceinline__ float to_f(double v) { return (float)v; }
__device__ __forceinline__ float to_f(float v) { return v; }
__device__ __forceinline__ float to_f(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T>
struct Arith;  // arithmetic type used for a storage type
template <>
struct Arith<double> {
  using type = double;
};
template <>
struct Arith<float> {
  using type = float;
};

}  // namespace fem
