// Shared device-side definitions of the SCR-FGMRES + AMG library.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>
#include <cstdio>
#include <vector>

#include "../../include/scr_gb300.h"

namespace scr {

// --------------------------------------------------------------- errors
struct CudaError {
  cudaError_t err;
  const char* where;
};

#define SCR_CUDA(call)                                         \
  do {                                                         \
    cudaError_t e_ = (call);                                   \
    if (e_ != cudaSuccess) throw ::scr::CudaError{e_, #call};  \
  } while (0)

#define SCR_LAUNCH() SCR_CUDA(cudaGetLastError())

void set_last_error(const char* fmt, ...);

// --------------------------------------------------------------- matrices
// Block-sparse matrix on the device in "slab" layout: the blocks of one
// block row keep the order of col[], and the values of the block row are
// stored scalar row by scalar row.  For block row i with k = rp[i+1]-rp[i]
// blocks starting at s = rp[i], entry (r, c) of its t-th block sits at
//   val[s*BR*BC + r*(k*BC) + t*BC + c].
// One scalar row of a block row is thus contiguous, so a group of lanes
// streams it with coalesced loads and one multiply-add per value.
template <typename T>
struct DBsr {
  int nbr = 0, nbc = 0, br = 1, bc = 1;
  long long nnzb = 0;
  int* rp = nullptr;
  int* col = nullptr;
  T* val = nullptr;
  int g = 0;                  // product kernel code (0: heuristic; see spmv.cu)
  const void* sell = nullptr; // host pointer to a DSell<T> copy used for products (optional)
  // padded ("vector") copy for 16-byte loads (optional, built by build_vec):
  // 3x3 blocks: vdesc holds one int4 per block row {column start, k, value
  //   start, scalar-row length}; the row's k column indices sit at
  //   vcol[column start ...], padded to a multiple of V = 16 / sizeof(T)
  //   entries; its three scalar rows follow one another from value start,
  //   each rl values long (k * 3 values, zero-padded to a multiple of V);
  // 1x1 blocks: vdesc holds one int2 per row {start, k}; values and column
  //   indices share the start, each row padded to a multiple of V entries.
  // Every start is a multiple of V, so each lane's chunk of V blocks (3x3)
  // or V entries (1x1) loads with 16-byte vector loads.
  const void* vdesc = nullptr;
  const int* vcol = nullptr;
  const T* vval = nullptr;
  // BF16 copy of val (same slab layout): when set, FP32 products read these
  // values instead (coarse AMG levels of the mixed-precision form)
  const void* hval = nullptr;
};

// Sliced block-ELL copy of a block matrix (see sell.cu): chunks of 32 block
// rows, rows ordered by length inside windows of 512.
constexpr int kChunk = 32;
constexpr int kWindow = 512;
template <typename T>
struct DSell {
  int nbr = 0, nbc = 0, br = 1, bc = 1, nchunk = 0;
  long long slots = 0;   // padded block slots per lane, summed over chunks
  int* perm = nullptr;   // lane slot -> block row
  int* cptr = nullptr;   // chunk -> first slot (units of 32 block slots)
  int* col = nullptr;
  T* val = nullptr;
};

__host__ __device__ inline long long slab_index(int s, int k, int t, int r, int c, int BR, int BC) {
  return (long long)s * BR * BC + (long long)r * k * BC + (long long)t * BC + c;
}

// --------------------------------------------------------------- memory
// Stream-ordered device allocations from a pool that keeps its memory, so
// repeated set-ups reuse the same blocks without returning them to the CUDA driver.
class DeviceArena {
 public:
  static constexpr size_t kSlack = 64;
  explicit DeviceArena(cudaStream_t s = 0) : stream_(s) {}
  ~DeviceArena() { release(); }
  template <typename T>
  T* alloc(size_t n) {
    void* p = nullptr;
    if (n == 0) n = 1;
    // kSlack bytes past the last element (vector loads of the last 16-byte
    // group of an array never leave the allocation)
    SCR_CUDA(cudaMallocAsync(&p, n * sizeof(T) + kSlack, stream_));
    ptrs_.push_back(p);
    bytes_ += n * sizeof(T);
    return static_cast<T*>(p);
  }
  void release() {
    for (void* p : ptrs_) cudaFreeAsync(p, stream_);
    ptrs_.clear();
    bytes_ = 0;
  }
  size_t bytes() const { return bytes_; }
  void set_stream(cudaStream_t s) { stream_ = s; }
  cudaStream_t stream() const { return stream_; }

 private:
  cudaStream_t stream_;
  std::vector<void*> ptrs_;
  size_t bytes_ = 0;
};

void configure_pool(int device);

// --------------------------------------------------------------- helpers
inline int ceil_div(long long a, long long b) { return (int)((a + b - 1) / b); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v, int width = 32) {
  for (int o = width / 2; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o, width);
  return v;
}

__device__ __forceinline__ float to_f(double v) { return (float)v; }

// SM count of the current device (cached).
int sm_count();

}  // namespace scr
