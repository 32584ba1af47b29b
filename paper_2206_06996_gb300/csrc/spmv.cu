// Block-sparse matrix-vector products (slab layout), layout conversions and
// the fused 2x2 block operator calA = [[A, B], [C, D]] of Sec. 5.2.1.
//
// Work decomposition: one group of G lanes per SCALAR row.  A scalar row of
// a block row is contiguous in the slab layout (k*BC values), so the G lanes
// stream it with one multiply-add per stored value and combine their partial
// sums with log2(G) shuffles.  G is small (2-8): on GB300 the FP64 pipe
// (about two FP64 FMAs per SM clock) is the binding resource of an FP64
// SpMV, and a wider group would spend more FP64 adds on the cross-lane
// reduction than on the product itself.
#include <cuda_bf16.h>

#include <cstdarg>
#include <cstring>
#include <map>
#include <mutex>
#include <stdexcept>
#include <tuple>
#include <vector>
#include <type_traits>

#include "epilogue.cuh"
#include "kernels.h"

#ifndef SCR_SPMV_BATCH
#define SCR_SPMV_BATCH 4
#endif
#ifndef SCR_SPMV_MINBLOCKS
#define SCR_SPMV_MINBLOCKS 1
#endif

namespace scr {

LaunchCounter& counters() {
  static LaunchCounter c;
  return c;
}

KernelProfiler& profiler() {
  static KernelProfiler p;
  return p;
}

int prof_start(int kclass, const void* key, cudaStream_t s) {
  KernelProfiler& p = profiler();
  if (!p.active || p.kclass != kclass || (key && key != p.target)) return -1;
  p.launches++;
  if (p.used >= p.cap) return -1;
  const int i = p.used++;
  SCR_CUDA(cudaEventRecord(p.ev[2 * i], s));
  return i;
}

void prof_stop(int idx, double bytes, double flops, cudaStream_t s) {
  if (idx < 0) return;
  KernelProfiler& p = profiler();
  SCR_CUDA(cudaEventRecord(p.ev[2 * idx + 1], s));
  p.bytes += bytes;
  p.flops += flops;
}

int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 1;
  }
  return n;
}

// ------------------------------------------------------------ layouts
template <typename TO>
__global__ void k_to_slab(const int* __restrict__ rp, const double* __restrict__ in, TO* __restrict__ out,
                          int nbr, int br, int bc) {
  int i = blockIdx.x * blockDim.y + threadIdx.y;
  if (i >= nbr) return;
  int s = rp[i], k = rp[i + 1] - s;
  int bs = br * bc;
  for (int q = threadIdx.x; q < k * bs; q += blockDim.x) {
    int t = q / bs, rem = q - t * bs, r = rem / bc, c = rem - r * bc;
    out[slab_index(s, k, t, r, c, br, bc)] = (TO)in[(long long)(s + t) * bs + rem];
  }
}

template <typename TI>
__global__ void k_from_slab(const int* __restrict__ rp, const TI* __restrict__ in, double* __restrict__ out,
                            int nbr, int br, int bc) {
  int i = blockIdx.x * blockDim.y + threadIdx.y;
  if (i >= nbr) return;
  int s = rp[i], k = rp[i + 1] - s;
  int bs = br * bc;
  for (int q = threadIdx.x; q < k * bs; q += blockDim.x) {
    int t = q / bs, rem = q - t * bs, r = rem / bc, c = rem - r * bc;
    out[(long long)(s + t) * bs + rem] = (double)in[slab_index(s, k, t, r, c, br, bc)];
  }
}

template <typename TO>
void to_slab(const int* rp, const double* std_val, TO* slab_val, int nbr, int br, int bc, long long nnzb,
             cudaStream_t s) {
  if (nbr == 0) return;
  dim3 blk(32, 8);
  k_to_slab<TO><<<ceil_div(nbr, 8), blk, 0, s>>>(rp, std_val, slab_val, nbr, br, bc);
  SCR_LAUNCH();
  counters().launches++;
  (void)nnzb;
}
template void to_slab<double>(const int*, const double*, double*, int, int, int, long long, cudaStream_t);
template void to_slab<float>(const int*, const double*, float*, int, int, int, long long, cudaStream_t);

void from_slab(const int* rp, const double* slab_val, double* std_val, int nbr, int br, int bc, long long,
               cudaStream_t s) {
  if (nbr == 0) return;
  dim3 blk(32, 8);
  k_from_slab<double><<<ceil_div(nbr, 8), blk, 0, s>>>(rp, slab_val, std_val, nbr, br, bc);
  SCR_LAUNCH();
}
void from_slab_f(const int* rp, const float* slab_val, double* std_val, int nbr, int br, int bc, long long,
                 cudaStream_t s) {
  if (nbr == 0) return;
  dim3 blk(32, 8);
  k_from_slab<float><<<ceil_div(nbr, 8), blk, 0, s>>>(rp, slab_val, std_val, nbr, br, bc);
  SCR_LAUNCH();
}

__global__ void k_d2f(const double* __restrict__ x, float* __restrict__ y, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long st = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += st) y[i] = (float)x[i];
}
// FP32 -> BF16, round to nearest even (__float2bfloat16_rn)
__global__ void k_f2bf(const float* __restrict__ x, __nv_bfloat16* __restrict__ y, long long n) {
  long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  long long st = (long long)gridDim.x * blockDim.x;
  for (; i < n; i += st) y[i] = __float2bfloat16_rn(x[i]);
}
void slab_to_bf16(const float* in, void* out, long long n, cudaStream_t s) {
  if (n == 0) return;
  k_f2bf<<<std::min<long long>(ceil_div(n, 256), 4 * 1024), 256, 0, s>>>(in, static_cast<__nv_bfloat16*>(out), n);
  SCR_LAUNCH();
  counters().launches++;
}

void slab_to_float(const double* in, float* out, long long n, cudaStream_t s) {
  if (n == 0) return;
  k_d2f<<<std::min<long long>(ceil_div(n, 256), 4 * 1024), 256, 0, s>>>(in, out, n);
  SCR_LAUNCH();
  counters().launches++;
}

// ------------------------------------------------------------ SpMV
// accumulate one scalar row r of block row i of M into acc[h]; the lanes of
// a G-group take the row's blocks in turn (BC values each, contiguous in the
// slab layout) so every stored value costs one multiply-add
template <int BC, int NRHS, int G, typename VT, typename XT, typename AT>
__device__ __forceinline__ void scalar_row_accum(const int* __restrict__ rp, const int* __restrict__ col,
                                                 const VT* __restrict__ val, const XT* __restrict__ x, int BR,
                                                 int i, int r, int lane, AT (&acc)[NRHS]) {
  // U blocks per lane in flight: the column indices are loaded first, then
  // every gather and value of the batch, then the multiply-adds, so a lane
  // keeps U independent load chains outstanding instead of one
  // measured on the 616k-node tube: FP64 rows gain from the lower register
  // count of two blocks in flight, FP32 rows from four
  constexpr int U = sizeof(VT) == 8 ? SCR_SPMV_BATCH / 2 : SCR_SPMV_BATCH;
  const int s = __ldg(rp + i), k = __ldg(rp + i + 1) - s;
  const VT* vr = val + (long long)s * BR * BC + (long long)r * k * BC;
  const int* cr = col + s;
  for (int t0 = lane; t0 < k; t0 += G * U) {
    int cidx[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = t0 + u * G;
      cidx[u] = t < k ? __ldg(cr + t) : -1;
    }
    AT a[U][BC], xv[U][BC][NRHS];
#pragma unroll
    for (int u = 0; u < U; ++u) {
      const int t = t0 + u * G;
      const bool ok = cidx[u] >= 0;
      const long long xb = (long long)(ok ? cidx[u] : 0) * BC * NRHS;
#pragma unroll
      for (int c = 0; c < BC; ++c) {
        a[u][c] = ok ? (AT)__ldg(vr + t * BC + c) : (AT)0;
#pragma unroll
        for (int h = 0; h < NRHS; ++h) xv[u][c][h] = ok ? (AT)__ldg(x + xb + c * NRHS + h) : (AT)0;
      }
    }
#pragma unroll
    for (int u = 0; u < U; ++u)
#pragma unroll
      for (int c = 0; c < BC; ++c)
#pragma unroll
        for (int h = 0; h < NRHS; ++h)
          if (cidx[u] >= 0) acc[h] = fma(a[u][c], xv[u][c][h], acc[h]);
  }
}

// L2 prefetch (cp.async.bulk.prefetch.L2) of the stored values and column
// indices that the CTA with index cta (256 threads, 256 / G scalar rows)
// will read.  The range is cut to whole 16-byte lines inside it: the first
// line may start up to 15 bytes before the range (the same line as a valid
// byte), the last partial line is left out, so no line outside the arrays
// is named.
template <int BR, int BC, int G, typename VT>
__device__ __forceinline__ void l2_prefetch_rows(const int* __restrict__ rp, const int* __restrict__ col,
                                                 const VT* __restrict__ val, int nbr, long long cta) {
  const long long nrows = (long long)nbr * BR;
  const long long o0 = cta * (256 / G);
  if (o0 >= nrows) return;
  const long long o1 = o0 + 256 / G < nrows ? o0 + 256 / G : nrows;
  const long long b0 = __ldg(rp + o0 / BR), b1 = __ldg(rp + (o1 - 1) / BR + 1);
  const unsigned long long v0 = __cvta_generic_to_global(val + b0 * BR * BC) & ~15ULL;
  const unsigned long long v1 = __cvta_generic_to_global(val + b1 * BR * BC) & ~15ULL;
  const unsigned long long c0 = __cvta_generic_to_global(col + b0) & ~15ULL;
  const unsigned long long c1 = __cvta_generic_to_global(col + b1) & ~15ULL;
  if (v1 > v0)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(v0), "r"((unsigned)(v1 - v0)) : "memory");
  if (c1 > c0)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(c0), "r"((unsigned)(c1 - c0)) : "memory");
}

template <int BR, int BC, int NRHS, int G, typename VT, typename XT, typename AT, Epi E>
__global__ void __launch_bounds__(256, SCR_SPMV_MINBLOCKS) k_spmv(int nbr, const int* __restrict__ rp,
                                                                 const int* __restrict__ col,
                                              const VT* __restrict__ val, const XT* __restrict__ x,
                                              Epilogue<XT, E> epi, int pf) {
  const long long o = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / G;  // scalar row
  const int lane = threadIdx.x % G;
  const long long nrows = (long long)nbr * BR;
  if (pf > 0 && threadIdx.x == 0) l2_prefetch_rows<BR, BC, G, VT>(rp, col, val, nbr, blockIdx.x + (long long)pf);
  const bool active = o < nrows;  // inactive lanes still join the shuffles
  AT acc[NRHS];
#pragma unroll
  for (int h = 0; h < NRHS; ++h) acc[h] = (AT)0;
  if (active) {
    const int i = (int)(o / BR), r = (int)(o - (long long)i * BR);
    scalar_row_accum<BC, NRHS, G>(rp, col, val, x, BR, i, r, lane, acc);
  }
  if constexpr (G > 1) {
#pragma unroll
    for (int h = 0; h < NRHS; ++h) {
#pragma unroll
      for (int off = G / 2; off > 0; off >>= 1) acc[h] += __shfl_xor_sync(0xffffffffu, acc[h], off, G);
    }
  }
  if (active && lane == 0) {
#pragma unroll
    for (int h = 0; h < NRHS; ++h) epi(o * NRHS + h, o, acc[h]);
  }
}

// G lanes per BLOCK row: each lane takes blocks t = lane, lane+G, ... and
// accumulates all BR scalar rows, so the column index and the BC source
// values of a block are loaded once for its BR x BC multiply-adds; the
// BR*NRHS sums are combined over the G lanes and written by distinct lanes.
template <int BR, int BC, int NRHS, int G, typename VT, typename XT, typename AT, Epi E>
__global__ void __launch_bounds__(256) k_spmv_brow(int nbr, const int* __restrict__ rp, const int* __restrict__ col,
                                                   const VT* __restrict__ val, const XT* __restrict__ x,
                                                   Epilogue<XT, E> epi) {
  const long long i = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / G;  // block row
  const int lane = threadIdx.x % G;
  const bool active = i < nbr;
  AT acc[BR][NRHS];
#pragma unroll
  for (int r = 0; r < BR; ++r)
#pragma unroll
    for (int h = 0; h < NRHS; ++h) acc[r][h] = (AT)0;
  if (active) {
    const int s = __ldg(rp + i), k = __ldg(rp + i + 1) - s;
    const VT* v0 = val + (long long)s * BR * BC;
    const int* cr = col + s;
#pragma unroll 2
    for (int t = lane; t < k; t += G) {
      const long long xb = (long long)__ldg(cr + t) * BC * NRHS;
      AT xv[BC][NRHS];
#pragma unroll
      for (int c = 0; c < BC; ++c)
#pragma unroll
        for (int h = 0; h < NRHS; ++h) xv[c][h] = (AT)__ldg(x + xb + c * NRHS + h);
#pragma unroll
      for (int r = 0; r < BR; ++r) {
        const VT* vt = v0 + (long long)r * k * BC + t * BC;
#pragma unroll
        for (int c = 0; c < BC; ++c) {
          const AT a = (AT)__ldg(vt + c);
#pragma unroll
          for (int h = 0; h < NRHS; ++h) acc[r][h] = fma(a, xv[c][h], acc[r][h]);
        }
      }
    }
  }
  if constexpr (G > 1) {
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int h = 0; h < NRHS; ++h)
#pragma unroll
        for (int off = G / 2; off > 0; off >>= 1) acc[r][h] += __shfl_xor_sync(0xffffffffu, acc[r][h], off, G);
  }
  if (active) {
#pragma unroll
    for (int q = 0; q < BR * NRHS; ++q) {
      if (q % G != lane) continue;
      const int r = q / NRHS, h = q - r * NRHS;
      const long long o = i * BR + r;
      epi(o * NRHS + h, o, acc[r][h]);
    }
  }
}

// sliced block-ELL product: one lane per block row, no cross-lane sums
template <int BR, int BC, int NRHS, typename VT, typename XT, Epi E>
__global__ void __launch_bounds__(256) k_sell_spmv(DSell<VT> S, const XT* __restrict__ x, Epilogue<XT, E> epi) {
  const long long g = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  const int c = (int)(g / kChunk), lane = (int)(g % kChunk);
  if (c >= S.nchunk) return;
  const int q = c * kChunk + lane;
  if (q >= S.nbr) return;
  const int i = __ldg(S.perm + q);
  const int c0 = __ldg(S.cptr + c), L = __ldg(S.cptr + c + 1) - c0;
  const long long base = (long long)c0 * kChunk;
  const int* __restrict__ cl = S.col + base + lane;
  const VT* __restrict__ vl = S.val + base * (BR * BC) + lane;
  using AT = XT;
  AT acc[BR][NRHS];
#pragma unroll
  for (int r = 0; r < BR; ++r)
#pragma unroll
    for (int h = 0; h < NRHS; ++h) acc[r][h] = (AT)0;
#pragma unroll 2
  for (int t = 0; t < L; ++t) {
    const long long xb = (long long)__ldg(cl + (long long)t * kChunk) * BC * NRHS;
    AT xv[BC][NRHS];
#pragma unroll
    for (int cc = 0; cc < BC; ++cc)
#pragma unroll
      for (int h = 0; h < NRHS; ++h) xv[cc][h] = (AT)__ldg(x + xb + cc * NRHS + h);
    const VT* vt = vl + (long long)t * kChunk * (BR * BC);
#pragma unroll
    for (int r = 0; r < BR; ++r)
#pragma unroll
      for (int cc = 0; cc < BC; ++cc) {
        const AT a = (AT)__ldg(vt + (r * BC + cc) * kChunk);
#pragma unroll
        for (int h = 0; h < NRHS; ++h) acc[r][h] = fma(a, xv[cc][h], acc[r][h]);
      }
  }
#pragma unroll
  for (int r = 0; r < BR; ++r) {
    const long long o = (long long)i * BR + r;
#pragma unroll
    for (int h = 0; h < NRHS; ++h) epi(o * NRHS + h, o, acc[r][h]);
  }
}

// CTAs ahead for the L2 prefetch of the scalar-row kernel (0: off); set
// from the options at scr_create.  Measured on the 616k-node tube: 128 to
// 384 CTAs ahead gave the same level-0 product times (FP32 122 -> 110 us,
// FP64 241 -> 229 us); 1536 and more were slower than none.
static int g_l2_prefetch = 192;
void set_l2_prefetch(int ctas) { g_l2_prefetch = ctas; }
// print every autotune decision with the candidates' times (options.verbose)
static int g_tune_verbose = 0;
void set_tune_verbose(int v) { g_tune_verbose = v; }

template <int BR, int BC, int NRHS, int G, typename VT, typename XT, typename AT, Epi E>
static void launch_spmv_g(const DBsr<VT>& M, const XT* x, XT* y, const EpiArgs& e, cudaStream_t s) {
  const Epilogue<XT, E> epi = make_epilogue<XT, E>(x, y, e);
  const int blk = 256;
  bool done = false;
  if constexpr (sizeof(VT) >= 4) {  // BF16 values: scalar-row kernel only
    if (M.sell) {
      const DSell<VT>& S = *static_cast<const DSell<VT>*>(M.sell);
      const long long threads = (long long)S.nchunk * kChunk;
      k_sell_spmv<BR, BC, NRHS, VT, XT, E><<<ceil_div(threads, blk), blk, 0, s>>>(S, x, epi);
      done = true;
    } else if (BR > 1 && code_of(M) > 0 && code_of(M) < 100) {
      const long long threads = (long long)M.nbr * G;
      k_spmv_brow<BR, BC, NRHS, G, VT, XT, AT, E><<<ceil_div(threads, blk), blk, 0, s>>>(M.nbr, M.rp, M.col,
                                                                                       M.val, x, epi);
      done = true;
    }
  }
  if (!done) {
    const long long threads = (long long)M.nbr * BR * G;
    k_spmv<BR, BC, NRHS, G, VT, XT, AT, E><<<ceil_div(threads, blk), blk, 0, s>>>(M.nbr, M.rp, M.col, M.val, x, epi,
                                                                                  g_l2_prefetch);
  }
  SCR_LAUNCH();
}

template <int BR, int BC, int NRHS, int G, typename VT, typename XT>
static void launch_spmv_e(const DBsr<VT>& M, const XT* x, XT* y, const EpiArgs& e, cudaStream_t s) {
  using AT = XT;  // accumulate in the vector precision
  switch (e.kind) {
    case Epi::Set: launch_spmv_g<BR, BC, NRHS, G, VT, XT, AT, Epi::Set>(M, x, y, e, s); break;
    case Epi::Axpby: launch_spmv_g<BR, BC, NRHS, G, VT, XT, AT, Epi::Axpby>(M, x, y, e, s); break;
    case Epi::Resid: launch_spmv_g<BR, BC, NRHS, G, VT, XT, AT, Epi::Resid>(M, x, y, e, s); break;
    case Epi::Jacobi: launch_spmv_g<BR, BC, NRHS, G, VT, XT, AT, Epi::Jacobi>(M, x, y, e, s); break;
    case Epi::ScaledSub: launch_spmv_g<BR, BC, NRHS, G, VT, XT, AT, Epi::ScaledSub>(M, x, y, e, s); break;
    case Epi::ChebFirst:
    case Epi::ChebStep:
      if constexpr (BR == BC) {
        if (e.kind == Epi::ChebFirst) launch_spmv_g<BR, BC, NRHS, G, VT, XT, AT, Epi::ChebFirst>(M, x, y, e, s);
        else launch_spmv_g<BR, BC, NRHS, G, VT, XT, AT, Epi::ChebStep>(M, x, y, e, s);
      } else {
        throw CudaError{cudaErrorInvalidValue, "Chebyshev epilogue on a non-square block shape"};
      }
      break;
  }
}

// lanes per scalar row: FP64 keeps groups narrow (FP64 adds of the
// reduction compete with the products), FP32 widens them for coalescing
// M.g: lanes per block row (1..16, block-row kernel for BR > 1), 100 +
// lanes per scalar row (scalar-row kernel) or 200 + lanes per scalar row
// (staged kernel, spmv_staged.cu, when M has a tile plan); 0 selects by row
// length
static int g_forced = 0;
void set_forced_group(int code) { g_forced = code; }

template <typename VT>
static int code_of(const DBsr<VT>& M) {
  return g_forced > 0 ? g_forced : M.g;
}

template <typename VT>
static int pick_group(const DBsr<VT>& M) {
  const int g = code_of(M);
  if (g >= 200) return g - 200;
  if (g > 0) return g >= 100 ? g - 100 : g;
  // measured on the 616k-node tube: FP64 3x3 rows are fastest with 2 lanes
  // per scalar row (the FP64 pipe binds), FP32 with 4 (coalescing binds)
  const double per_row = M.nbr ? (double)M.nnzb * M.bc / M.nbr : 0.0;
  int G = sizeof(VT) == 8 ? (per_row >= 24 ? 2 : 1) : (per_row >= 24 ? 4 : 2);
  // small operators (the coarse AMG levels) fill less than a wave of the GPU
  // with one group per row, and their rows are long, so each lane would walk
  // dozens of blocks one dependent L2 round trip at a time: widen the group
  // (up to 16 lanes, at least 4 values per lane) while the grid stays below
  // two waves.  Measured on the coarse tube levels: about 23 us per product
  // with 2 lanes whatever the level's size.
  const long long nrows = (long long)M.nbr * M.br;
  const long long wave = (long long)sm_count() * 2048;
  while (G < 16 && per_row >= 8.0 * G && nrows * G < wave) G *= 2;
  return G;
}

template <int BR, int BC, int NR, typename VT, typename XT>
static void dispatch_g(int G, const DBsr<VT>& M, const XT* x, XT* y, const EpiArgs& e, cudaStream_t s) {
  switch (G) {
    case 1: launch_spmv_e<BR, BC, NR, 1, VT, XT>(M, x, y, e, s); break;
    case 2: launch_spmv_e<BR, BC, NR, 2, VT, XT>(M, x, y, e, s); break;
    case 4: launch_spmv_e<BR, BC, NR, 4, VT, XT>(M, x, y, e, s); break;
    case 8: launch_spmv_e<BR, BC, NR, 8, VT, XT>(M, x, y, e, s); break;
    default: launch_spmv_e<BR, BC, NR, 16, VT, XT>(M, x, y, e, s); break;
  }
}

template <typename VT, typename XT>
static void spmv_launch(int G, const DBsr<VT>& M, const XT* x, XT* y, int nrhs, const EpiArgs& e, cudaStream_t s) {
  const int br = M.br, bc = M.bc;
  if (br == 3 && bc == 3 && nrhs == 1) dispatch_g<3, 3, 1, VT, XT>(G, M, x, y, e, s);
  else if (br == 3 && bc == 1 && nrhs == 1) dispatch_g<3, 1, 1, VT, XT>(G, M, x, y, e, s);
  else if (br == 1 && bc == 3 && nrhs == 1) dispatch_g<1, 3, 1, VT, XT>(G, M, x, y, e, s);
  else if (br == 1 && bc == 1 && nrhs == 1) dispatch_g<1, 1, 1, VT, XT>(G, M, x, y, e, s);
  else if (br == 1 && bc == 1 && nrhs == 3) dispatch_g<1, 1, 3, VT, XT>(G, M, x, y, e, s);
  else throw CudaError{cudaErrorInvalidValue, "spmv: unsupported block shape"};
}

// the product with the values M holds: its BF16 copy when it has one (FP32
// vectors, FP32 sums), else val
template <typename VT, typename XT>
static void product(int G, const DBsr<VT>& M, const XT* x, XT* y, int nrhs, const EpiArgs& e, cudaStream_t s) {
  if constexpr (std::is_same<VT, float>::value) {
    if (M.hval) {
      DBsr<__nv_bfloat16> H;
      H.nbr = M.nbr;
      H.nbc = M.nbc;
      H.br = M.br;
      H.bc = M.bc;
      H.nnzb = M.nnzb;
      H.rp = M.rp;
      H.col = M.col;
      H.val = static_cast<__nv_bfloat16*>(const_cast<void*>(M.hval));
      H.g = M.g;
      spmv_launch<__nv_bfloat16, XT>(G, H, x, y, nrhs, e, s);
      return;
    }
  }
  if (!(code_of(M) >= 200 && !M.sell && spmv_staged<VT, XT>(G, M, x, y, nrhs, e, s)))
    spmv_launch<VT, XT>(G, M, x, y, nrhs, e, s);
}

template <typename VT, typename XT>
void spmv(const DBsr<VT>& M, const XT* x, XT* y, int nrhs, const EpiArgs& e, cudaStream_t s) {
  if (M.nbr == 0) return;
  const int G = M.sell ? 1 : pick_group(M);
  const int pidx = prof_start(0, M.val, s);
  product<VT, XT>(G, M, x, y, nrhs, e, s);
  counters().launches++;
  {
    // algorithmic bytes: stored values + column indices + row pointers once,
    // the source vector once, the result written once, plus what the
    // epilogue reads (z, the current iterate, the inverse diagonal)
    const double nrow = (double)M.nbr * M.br;
    const double vsz = M.hval ? 2.0 : (double)sizeof(VT);
    double b = (double)M.nnzb * (M.br * M.bc * vsz + sizeof(int)) + (M.nbr + 1.0) * sizeof(int) +
               (double)M.nbc * M.bc * nrhs * sizeof(XT) + nrow * nrhs * sizeof(XT);
    if (e.kind == Epi::Resid || (e.kind == Epi::Axpby && e.z)) b += nrow * nrhs * sizeof(XT);
    if (e.kind == Epi::Jacobi) b += 2.0 * nrow * nrhs * sizeof(XT) + nrow * sizeof(XT);
    if (e.kind == Epi::ScaledSub) b += nrow * nrhs * sizeof(XT) + nrow * sizeof(XT);
    if (e.kind == Epi::ChebFirst) b += 4.0 * nrow * nrhs * sizeof(XT) + nrow * sizeof(XT);
    if (e.kind == Epi::ChebStep) b += 5.0 * nrow * nrhs * sizeof(XT) + nrow * sizeof(XT);
    counters().spmv_bytes += (long long)b;
    prof_stop(pidx, b, 2.0 * (double)M.nnzb * M.br * M.bc * nrhs, s);
  }
}

// Decisions are cached by (shape, size, precision, right-hand sides): a
// Newton step's new Jacobian has the pattern of the previous one, so the
// timing runs once per pattern.
struct TuneKey {
  long long nnzb;
  int nbr, nbc, br, bc, vt, nrhs, dev;
  bool operator<(const TuneKey& o) const {
    return std::tie(nnzb, nbr, nbc, br, bc, vt, nrhs, dev) <
           std::tie(o.nnzb, o.nbr, o.nbc, o.br, o.bc, o.vt, o.nrhs, o.dev);
  }
};
static std::map<TuneKey, int>& tune_cache() {
  static std::map<TuneKey, int> m;
  return m;
}
static std::mutex g_tune_mutex;

template <typename VT>
int autotune_spmv(DBsr<VT>& M, int nrhs, cudaStream_t s) {
  if (M.nbr == 0 || M.sell) return M.g;
  int dev = 0;
  cudaGetDevice(&dev);
  const TuneKey key{M.nnzb, M.nbr, M.nbc, M.br, M.bc, (int)sizeof(VT), nrhs, dev};
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    auto it = tune_cache().find(key);
    if (it != tune_cache().end()) {
      M.g = it->second;
      return M.g;
    }
  }
  using XT = VT;
  const long long nx = (long long)M.nbc * M.bc * nrhs + 1, ny = (long long)M.nbr * M.br * nrhs + 1;
  XT *x = nullptr, *y = nullptr;
  SCR_CUDA(cudaMallocAsync(&x, nx * sizeof(XT), s));
  SCR_CUDA(cudaMallocAsync(&y, ny * sizeof(XT), s));
  SCR_CUDA(cudaMemsetAsync(x, 0, nx * sizeof(XT), s));
  cudaEvent_t e0, e1;
  SCR_CUDA(cudaEventCreate(&e0));
  SCR_CUDA(cudaEventCreate(&e1));
  // the scalar-row kernel with 1, 2, 4 or 8 lanes and, when M has a tile
  // plan, the staged kernel with 2, 4 or 8 (the block-row and sliced-ELL
  // variants measured slower on the tube operators)
  int cands[9] = {101, 102, 104, 108};
  int ncand = 4;
  if (M.nbr && (double)M.nnzb * M.bc / M.nbr >= 64) cands[ncand++] = 116;  // long rows
  if (M.tiles && staged_shape_supported(M.br, M.bc, nrhs)) {
    cands[ncand++] = 202;
    cands[ncand++] = 204;
    cands[ncand++] = 208;
  }
  float best = 1e30f;
  int bestg = M.g;
  const int saved = M.g;
  float times[9] = {};
  for (int q = 0; q < ncand; ++q) {
    const int code = cands[q];
    M.g = code;
    const int G = pick_group(M);
    auto run = [&] { product<VT, XT>(G, M, x, y, nrhs, EpiArgs(), s); };
    run();  // warm-up
    SCR_CUDA(cudaEventRecord(e0, s));
    for (int r = 0; r < 5; ++r) run();
    SCR_CUDA(cudaEventRecord(e1, s));
    SCR_CUDA(cudaEventSynchronize(e1));
    float ms = 0;
    SCR_CUDA(cudaEventElapsedTime(&ms, e0, e1));
    times[q] = ms;
    if (ms < best) {
      best = ms;
      bestg = code;
    }
  }
  (void)saved;
  counters().launches += 6 * ncand;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  SCR_CUDA(cudaFreeAsync(x, s));
  SCR_CUDA(cudaFreeAsync(y, s));
  M.g = bestg;
  {
    std::lock_guard<std::mutex> lock(g_tune_mutex);
    tune_cache()[key] = bestg;
  }
  if (g_tune_verbose) {
    fprintf(stderr, "[autotune] %dx%d blocks, %d x %d block rows/cols, %lld blocks, %s, nrhs %d -> code %d |",
            M.br, M.bc, M.nbr, M.nbc, M.nnzb, sizeof(VT) == 8 ? "fp64" : "fp32", nrhs, bestg);
    for (int q = 0; q < ncand; ++q) fprintf(stderr, " %d: %.1f us", cands[q], 200.0f * times[q]);
    fprintf(stderr, "\n");
  }
  return bestg;
}
// text form of the cache: "nnzb nbr nbc br bc value_bytes nrhs code" per line
static bool valid_code(int c) {
  return (c >= 1 && c <= 16) || (c >= 101 && c <= 116) || c == 201 || c == 202 || c == 204 || c == 208;
}

void tune_save(const char* path) {
  FILE* f = fopen(path, "w");
  if (!f) throw std::invalid_argument("scr_tune_save: cannot open the file for writing");
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  fprintf(f, "# scr_gb300 autotune decisions: nnzb nbr nbc br bc value_bytes nrhs code\n");
  for (const auto& kv : tune_cache()) {
    const TuneKey& k = kv.first;
    fprintf(f, "%lld %d %d %d %d %d %d %d\n", k.nnzb, k.nbr, k.nbc, k.br, k.bc, k.vt, k.nrhs, kv.second);
  }
  fclose(f);
}

void tune_load(const char* path) {
  FILE* f = fopen(path, "r");
  if (!f) throw std::invalid_argument("scr_tune_load: cannot open the file");
  int dev = 0;
  cudaGetDevice(&dev);
  std::vector<std::pair<TuneKey, int>> got;
  char line[512];
  bool bad = false;
  while (fgets(line, sizeof line, f)) {
    if (line[0] == '#' || line[0] == '\n') continue;
    TuneKey k{};
    int code = 0;
    if (sscanf(line, "%lld %d %d %d %d %d %d %d", &k.nnzb, &k.nbr, &k.nbc, &k.br, &k.bc, &k.vt, &k.nrhs, &code) != 8 ||
        !valid_code(code) || k.nnzb < 0 || k.nbr < 0 || k.nbc < 0) {
      bad = true;
      break;
    }
    k.dev = dev;
    got.emplace_back(k, code);
  }
  fclose(f);
  if (bad) throw std::invalid_argument("scr_tune_load: malformed line");
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  for (const auto& kv : got) tune_cache()[kv.first] = kv.second;
}

template int autotune_spmv<double>(DBsr<double>&, int, cudaStream_t);
template int autotune_spmv<float>(DBsr<float>&, int, cudaStream_t);

template void spmv<double, double>(const DBsr<double>&, const double*, double*, int, const EpiArgs&, cudaStream_t);
template void spmv<float, float>(const DBsr<float>&, const float*, float*, int, const EpiArgs&, cudaStream_t);

// ------------------------------------------------------------ calA
// Scalar rows 0..3n_v-1: (A x_v + B x_p); rows 3n_v..3n_v+n_p-1:
// (C x_v + D x_p).  One G-group per scalar row.
template <int G, bool RESID>
__global__ void __launch_bounds__(256) k_block_op(int nv, int np, DBsr<double> A, DBsr<double> B, DBsr<double> C,
                                                  DBsr<double> D, const double* __restrict__ x,
                                                  double* __restrict__ y, const double* __restrict__ z) {
  const long long o = (blockIdx.x * (long long)blockDim.x + threadIdx.x) / G;
  const int lane = threadIdx.x % G;
  const long long nrow_v = 3LL * nv;
  const bool active = o < nrow_v + np;  // inactive lanes still join the shuffles
  const double* xv = x;
  const double* xp = x + nrow_v;
  double acc[1] = {0.0};
  if (!active) {
  } else if (o < nrow_v) {
    const int i = (int)(o / 3), r = (int)(o - 3LL * i);
    scalar_row_accum<3, 1, G>(A.rp, A.col, A.val, xv, 3, i, r, lane, acc);
    scalar_row_accum<1, 1, G>(B.rp, B.col, B.val, xp, 3, i, r, lane, acc);
  } else {
    const int i = (int)(o - nrow_v);
    scalar_row_accum<3, 1, G>(C.rp, C.col, C.val, xv, 1, i, 0, lane, acc);
    scalar_row_accum<1, 1, G>(D.rp, D.col, D.val, xp, 1, i, 0, lane, acc);
  }
#pragma unroll
  for (int off = G / 2; off > 0; off >>= 1) acc[0] += __shfl_xor_sync(0xffffffffu, acc[0], off, G);
  if (active && lane == 0) y[o] = RESID ? z[o] - acc[0] : acc[0];
}

void block_op(const DBsr<double>& A, const DBsr<double>& B, const DBsr<double>& C, const DBsr<double>& D,
              const double* x, double* y, const double* z, bool resid, cudaStream_t s) {
  const int nv = A.nbr, np = D.nbr;
  const long long rows = 3LL * nv + np;
  if (rows == 0) return;
  constexpr int G = 4;
  const long long threads = rows * G;
  const int pidx = prof_start(1, nullptr, s);
  if (resid)
    k_block_op<G, true><<<ceil_div(threads, 256), 256, 0, s>>>(nv, np, A, B, C, D, x, y, z);
  else
    k_block_op<G, false><<<ceil_div(threads, 256), 256, 0, s>>>(nv, np, A, B, C, D, x, y, z);
  SCR_LAUNCH();
  counters().launches++;
  const double b = A.nnzb * 76.0 + B.nnzb * 28.0 + C.nnzb * 28.0 + D.nnzb * 12.0 +
                   (A.nbr + D.nbr + 2.0) * 8.0 + rows * 8.0 * (resid ? 3 : 2);
  counters().spmv_bytes += (long long)b;
  prof_stop(pidx, b, 2.0 * (9.0 * A.nnzb + 3.0 * B.nnzb + 3.0 * C.nnzb + D.nnzb), s);
}

}  // namespace scr
