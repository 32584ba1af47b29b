// Product kernels with G lanes per scalar row and their launch dispatch,
// shared by the translation units that instantiate them: spmv.cu (one and
// three right-hand sides) and spmm.cu (eight right-hand sides, the block
// product of the multi-right-hand-side solve).
#pragma once
#include <cuda_bf16.h>

#include "epilogue.cuh"
#include "kernels.h"

#ifndef SCR_SPMV_MINBLOCKS
#define SCR_SPMV_MINBLOCKS 1
#endif
// blocks each lane of a product keeps in flight (FP64 rows use half)
#ifndef SCR_SPMV_BATCH
#define SCR_SPMV_BATCH 4
#endif

namespace scr {

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
  // (with 4 or more right-hand sides a block already brings NRHS gathers per
  // value: one block per lane pass keeps the registers in bounds)
  constexpr int U = NRHS > 3 ? 1 : (sizeof(VT) == 8 ? SCR_SPMV_BATCH / 2 : SCR_SPMV_BATCH);
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

// CTAs ahead for the L2 prefetch of the scalar-row kernel (0: off) and the
// forced kernel code of every product (0: per matrix); defined in spmv.cu
extern int g_l2_prefetch;

template <int BR, int BC, int NRHS, int G, typename VT, typename XT, typename AT, Epi E>
inline void launch_spmv_g(const DBsr<VT>& M, const XT* x, XT* y, const EpiArgs& e, cudaStream_t s) {
  const Epilogue<XT, E> epi = make_epilogue<XT, E>(x, y, e);
  const int blk = 256;
  bool done = false;
  if constexpr (sizeof(VT) >= 4 && NRHS <= 3) {  // BF16 values, multi-column products: scalar-row kernel only
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
inline void launch_spmv_e(const DBsr<VT>& M, const XT* x, XT* y, const EpiArgs& e, cudaStream_t s) {
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
// M.g: lanes per block row (1..16, block-row kernel for BR > 1) or 100 +
// lanes per scalar row (scalar-row kernel); 0 selects by row length
extern int g_forced;

template <typename VT>
inline int code_of(const DBsr<VT>& M) {
  return g_forced > 0 ? g_forced : M.g;
}

template <typename VT>
inline int pick_group(const DBsr<VT>& M) {
  const int g = code_of(M);
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
inline void dispatch_g(int G, const DBsr<VT>& M, const XT* x, XT* y, const EpiArgs& e, cudaStream_t s) {
  switch (G) {
    case 1: launch_spmv_e<BR, BC, NR, 1, VT, XT>(M, x, y, e, s); break;
    case 2: launch_spmv_e<BR, BC, NR, 2, VT, XT>(M, x, y, e, s); break;
    case 4: launch_spmv_e<BR, BC, NR, 4, VT, XT>(M, x, y, e, s); break;
    case 8: launch_spmv_e<BR, BC, NR, 8, VT, XT>(M, x, y, e, s); break;
    default: launch_spmv_e<BR, BC, NR, 16, VT, XT>(M, x, y, e, s); break;
  }
}

}  // namespace scr
