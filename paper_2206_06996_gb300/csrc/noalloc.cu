// Block sparse product without any device allocation.
//
// scr_bsr_spmv converts the caller's values into the solver's row layout in
// a temporary buffer it allocates on every call.  Some callers cannot allow
// that: hosts whose device memory belongs to another allocator (a
// framework's caching allocator, or a memory budget fixed at start-up, where
// a library's own cudaMalloc can fail or push the owner out of memory), and
// code that must not call cudaFree, which waits for the whole device.  This
// entry point keeps its scratch in one static device array instead: every
// GPU that loads the library holds that array until the process exits, and
// the size of the matrices it accepts is capped by it.  Each call still
// validates the caller's indices on the device, reads the result flag back
// to the host and synchronises the stream twice.
#include <cstring>
#include <mutex>
#include <stdexcept>

#include "kernels.h"

namespace scr {

// Scratch: the first 32 doubles (256 bytes) hold the validation flag, the
// rest the matrix values in the row layout of the product kernel.
constexpr long long kNoAllocHead = 32;
constexpr long long kNoAllocMaxScalars = 1LL << 21;  // 2,097,152 stored scalars (16 MiB)
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocHead + kNoAllocMaxScalars];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the name of a __device__ variable is only a host-side handle)
// and kept for the life of the process: a cudaDeviceReset would move the
// array, so this entry point must not be used on a device after a reset.
double* scratch_on_current_device() {
  int dev = 0;
  SCR_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) throw std::invalid_argument("device ordinal out of range");
  std::lock_guard<std::mutex> lock(g_noalloc_mutex);
  if (!g_noalloc_ptr[dev]) {
    void* p = nullptr;
    const cudaError_t rc = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (rc != cudaSuccess || !p) throw CudaError{rc != cudaSuccess ? rc : cudaErrorUnknown, "cudaGetSymbolAddress"};
    g_noalloc_ptr[dev] = p;
  }
  return static_cast<double*>(g_noalloc_ptr[dev]);
}

}  // namespace
}  // namespace scr

using namespace scr;

extern "C" int scr_bsr_spmv_noalloc(const scr_bsr* M, const double* x, double* y, void* stream) {
  if (!M || !x || !y) {
    set_last_error("scr_bsr_spmv_noalloc: NULL argument");
    return SCR_INVALID_ARG;
  }
  if (!((M->br == 1 || M->br == 3) && (M->bc == 1 || M->bc == 3)) || M->nb_rows < 0 || M->nb_cols < 0 ||
      M->nnzb < 0) {
    set_last_error("scr_bsr_spmv_noalloc: block sizes must be 1 or 3 and sizes non-negative");
    return SCR_INVALID_ARG;
  }
  const long long scalars = (long long)M->nnzb * M->br * M->bc;
  if (scalars > kNoAllocMaxScalars) {
    set_last_error(
        "scr_bsr_spmv_noalloc: the matrix stores %lld scalars, more than the %lld its static scratch holds; "
        "use scr_bsr_spmv",
        scalars, kNoAllocMaxScalars);
    return SCR_INVALID_ARG;
  }
  try {
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    double* scratch = scratch_on_current_device();
    int* bad = reinterpret_cast<int*>(scratch);
    double* vals = scratch + kNoAllocHead;
    // the flag keeps the previous call's value: clear it first
    SCR_CUDA(cudaMemsetAsync(bad, 0, sizeof(int), s));
    check_bsr_indices(M->nb_rows, M->nb_cols, M->row_ptr, M->col_idx, M->nnzb, bad, s);
    int hb = 0;
    SCR_CUDA(cudaMemcpyAsync(&hb, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    SCR_CUDA(cudaStreamSynchronize(s));
    if (hb) {
      set_last_error("scr_bsr_spmv_noalloc: row_ptr/col_idx invalid");
      return SCR_INVALID_ARG;
    }
    DBsr<double> D;
    D.nbr = M->nb_rows;
    D.nbc = M->nb_cols;
    D.br = M->br;
    D.bc = M->bc;
    D.nnzb = M->nnzb;
    D.rp = const_cast<int*>(M->row_ptr);
    D.col = const_cast<int*>(M->col_idx);
    D.val = vals;
    if (scalars > 0) to_slab<double>(D.rp, M->val, D.val, D.nbr, D.br, D.bc, D.nnzb, s);
    spmv<double, double>(D, x, y, 1, EpiArgs(), s);
    SCR_CUDA(cudaStreamSynchronize(s));
    return SCR_OK;
  } catch (const CudaError& e) {
    set_last_error("CUDA error %s in %s", cudaGetErrorString(e.err), e.where ? e.where : "?");
    cudaGetLastError();
    return SCR_CUDA_ERROR;
  } catch (const std::exception& e) {
    set_last_error("%s", e.what());
    return SCR_INVALID_ARG;
  }
}
